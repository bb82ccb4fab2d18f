// From-scratch FP64 inverse with the trailing updates on the tensor cores.
//
// The refresh (Sec. 2.3 init_det_carrier; Sec. 1 advises double precision) is
// a blocked Gauss-Jordan inversion of M = A^T, n^3 FMAs per walker, and
// GB300's FP64 pipe runs at about 1/64 of its FP32 rate.  Panels of OZ_B = 64
// columns are eliminated in four 16-column sub-panels (eight 8-column ones for
// n > 1024): each in FP64 (refresh.cu: n * 16^2 FMAs), its update of the
// panel's other columns as the split product below with one K-step of 16;
// then the update of every other column by the panel,
//     M[i, j] += sum_c (Pan - E)[i, c] * S[c, j],   S = rows k0 .. k0+63 of M,
// (n^2 * 64 FMAs per panel: 94% of the work at n = 1024) also runs as an
// error-free split product on the BF16 tensor cores, the scheme of Ozaki,
// Ogita, Oishi and Rump (Numer. Algorithms 59, 2012):
//   - every 64-vector (a row of Pan - E, a column of S) is scaled by a power
//     of two 2^E with |x| < 2^E and rounded to a multiple of 2^(E-56), then
//     written exactly as 7 signed base-256 digits, x = 2^E sum_t d_t 2^(-8(t+1))
//     (|d_0| <= 256, |d_t| <= 128), each digit times its power a BF16 value;
//     this uses integer operations only;
//   - the product of digit t of S and digit u of Pan has level l = t + u + 2:
//     an integer times 2^(-8l).  Summed over the 64-wide inner dimension, all
//     products of one level stay below 2^23 in magnitude, so the FP32
//     accumulation of tcgen05.mma is exact for each of the levels 2 .. 6,
//     each in its own TMEM accumulator; levels 7..10 (below 2^(-40) of level
//     2, summed with FP32 rounding) share a sixth; levels above 10 (below
//     2^(-66) of the scale) are dropped.  Levels 7..10 are kept because the
//     row scaling measures errors against the row maxima: a level dropped at
//     2^-56 of the maxima of two rows whose large entries do not meet costs
//     far more than 2^-53 of the products actually summed;
//   - the epilogue recovers the five exact levels as integers, rounds the
//     tail to a multiple of 2^-56, adds all six exactly in int64, converts
//     once to double with the scale 2^(E_i + E_j) folded into the exponent
//     (integer operations), and adds it to M: one FP64 add per element, and
//     the rounding of an FP64 update, at tensor-core speed.
// The output tile is 128 columns j (TMEM lanes, so the FP64 read-modify-write
// of row-major M is coalesced) x 64 rows i; TMA stages the 7 S slices of a
// column block once (112 KiB) and the 7 Pan slices of each row tile (56 KiB)
// behind the previous tile's epilogue (SWIZZLE_128B, no multicast); one
// thread issues the 39 MMAs x 4 K-steps.  Every wait is bounded as in the
// delayed flush.  (Two accumulator sets for an MMA / epilogue overlap do not
// fit the 512 TMEM columns at 64 rows; at 32 rows the MMAs, whose operands
// are re-read from shared memory per instruction, become the bound.)
#include <algorithm>
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace lru {

constexpr int OZ_TJ = 128;                        // output columns j per tile (MMA M)
constexpr int OZ_TI = 64;                         // output rows i per tile (MMA N)
constexpr int OZ_SLICE_A = OZ_TJ * 128;           // bytes of one S slice tile (128 rows x 128 B)
constexpr int OZ_SLICE_B = OZ_TI * 128;           // bytes of one Pan slice tile (64 rows x 128 B)
constexpr int OZ_GROUPS = 6;                      // accumulators: levels 2, 3, 4, 5, 6 (exact), 7..10
constexpr int OZ_MAXLV = 8;                       // products t + u <= 8 (levels up to 10) are kept
constexpr uint32_t OZ_TMEM_COLS = 512;            // 6 x 64 columns, rounded to a power of two
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_TI >> 3) << 17) |
                              ((uint32_t)(OZ_TJ >> 4) << 24);   // BF16 x BF16 -> F32, K-major, 128 x 64

struct OzMaps {
    CUtensorMap S, P;
};

// ---- exact splitting (integer operations only) --------------------------------

__device__ __forceinline__ int oz_bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// X = round(x * 2^(56 - E)) for |x| < 2^E: |X| < 2^56.  Zero and subnormal x give 0.
__device__ __forceinline__ long long oz_fixed(double x, int E) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int eb = (int)((b >> 52) & 0x7FF);
    if (eb == 0) return 0;
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    const int sh = eb - 1075 + 56 - E;   // <= 3 because |x| < 2^E
    long long X;
    if (sh >= 0) X = m << sh;
    else if (sh > -60) X = (m + (1ll << (-sh - 1))) >> (-sh);
    else X = 0;
    return (b >> 63) ? -X : X;
}

// digit t of X (signed, rounded): X = sum_t d_t 2^(48 - 8t); BF16 bits of d_t * 2^(-8(t+1))
__device__ __forceinline__ void oz_digits(long long X, uint16_t (&h)[OZ_S]) {
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) {
        const int sh = 48 - 8 * t;
        const long long q = sh > 0 ? ((X + (1ll << (sh - 1))) >> sh) : X;
        X -= q << sh;
        // |q| <= 256: exact in FP32 via the 1.5 * 2^23 offset, exact in BF16 (8 significant bits)
        const float f = (__int_as_float(0x4B400000 + (int)q) - 12582912.0f) * __int_as_float((127 - 8 * (t + 1)) << 23);
        h[t] = (uint16_t)(__float_as_uint(f) >> 16);
    }
}

// Rows of (Pan - E): row i of walker w, the width (<= 64) columns c0 .. of M,
// minus 1 at (c0 + c, c); columns past the width are zero.  One warp per row;
// lane covers c = lane and lane + 32.  A width of at most 16 (a sub-panel)
// feeds a single K-step of 16, which reads only the first 16 columns of each
// slice row, so only those are written.
__global__ void __launch_bounds__(256) k_oz_slice_P(int n, int c0, int width, int w0, OzWork Z,
                                                    const uint8_t* mask) {
    const int w = w0 + blockIdx.y;
    if (mask && !mask[w]) return;
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= n) return;
    const double* row = Z.M + (long long)w * n * n + (long long)i * n + c0;
    double a = lane < width ? row[lane] : 0.0, b = lane + 32 < width ? row[lane + 32] : 0.0;
    if (lane < width && i == c0 + lane) a -= 1.0;
    if (lane + 32 < width && i == c0 + lane + 32) b -= 1.0;
    const int mx = __reduce_max_sync(0xffffffffu, max(oz_bexp(a), oz_bexp(b)));
    const int E = mx > 0 ? mx - 1022 : 0;
    uint16_t ha[OZ_S], hb[OZ_S];
    oz_digits(oz_fixed(a, E), ha);
    oz_digits(oz_fixed(b, E), hb);
    const bool full = width > 16;
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) {
        uint16_t* dst = Z.Pb + (((long long)w * OZ_S + t) * n + i) * OZ_B;
        if (full || lane < 16) dst[lane] = ha[t];
        if (full) dst[lane + 32] = hb[t];
    }
    if (lane == 0) Z.eP[(long long)w * n + i] = E;
}

// The same rows for a sub-panel (width <= 16): half a warp per row, lane c of
// the half covering column c, so no lane splits a zero.  Writes the first 16
// entries of each slice row and the row's exponent, exactly as k_oz_slice_P.
// n is a multiple of 16, so both halves of a warp always have a row.
__global__ void __launch_bounds__(256) k_oz_slice_P16(int n, int c0, int width, int w0, OzWork Z,
                                                      const uint8_t* mask) {
    const int w = w0 + blockIdx.y;
    if (mask && !mask[w]) return;
    const int c = threadIdx.x & 15;
    const int i = blockIdx.x * 16 + (threadIdx.x >> 4);
    const unsigned hmask = 0xFFFFu << (threadIdx.x & 16);   // this half of the warp
    const bool ok = i < n;
    const double* row = Z.M + (long long)w * n * n + (long long)i * n + c0;
    double a = (ok && c < width) ? row[c] : 0.0;
    if (c < width && i == c0 + c) a -= 1.0;
    int mx = oz_bexp(a);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(hmask, mx, o));
    const int E = mx > 0 ? mx - 1022 : 0;
    uint16_t ha[OZ_S];
    oz_digits(oz_fixed(a, E), ha);
    if (!ok) return;
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) Z.Pb[(((long long)w * OZ_S + t) * n + i) * OZ_B + c] = ha[t];
    if (c == 0) Z.eP[(long long)w * n + i] = E;
}

// Columns of S = the nr (<= 64) rows r0 .. of M, zero past nr: a 64 x 64
// block per CTA (column blocks jb0, jb0 + 1, ..) through shared memory
// (stored transposed), then one warp per column j.  As for the panel rows,
// nr <= 16 writes only the first 16 entries of each slice row.
__global__ void __launch_bounds__(256) k_oz_slice_S(int n, int r0, int nr, int jb0, int w0, OzWork Z,
                                                    const uint8_t* mask) {
    __shared__ double sT[64][65];   // sT[j][c] = S[c][j0 + j]
    const int w = w0 + blockIdx.y;
    if (mask && !mask[w]) return;
    const int j0 = (jb0 + blockIdx.x) * 64;
    const double* M = Z.M + (long long)w * n * n;
    for (int e = threadIdx.x; e < 64 * 64; e += 256) {
        const int c = e >> 6, j = e & 63;
        sT[j][c] = c < nr ? M[(long long)(r0 + c) * n + j0 + j] : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int j = threadIdx.x >> 5; j < 64; j += 8) {
        const double a = sT[j][lane], b = sT[j][lane + 32];
        const int mx = __reduce_max_sync(0xffffffffu, max(oz_bexp(a), oz_bexp(b)));
        const int E = mx > 0 ? mx - 1022 : 0;
        uint16_t ha[OZ_S], hb[OZ_S];
        oz_digits(oz_fixed(a, E), ha);
        oz_digits(oz_fixed(b, E), hb);
#pragma unroll
        for (int t = 0; t < OZ_S; ++t) {
            uint16_t* dst = Z.Sb + (((long long)w * OZ_S + t) * n + j0 + j) * OZ_B;
            if (nr > 16 || lane < 16) dst[lane] = ha[t];
            if (nr > 16) dst[lane + 32] = hb[t];
        }
        if (lane == 0) Z.eS[(long long)w * n + j0 + j] = E;
    }
}

__device__ __forceinline__ void oz_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(dtmem), "l"(a), "l"(b), "r"(OZ_IDESC), "r"(acc)
        : "memory");
}

// F * 2^(e - 56) as a double, rounded to nearest even, by integer operations
// (normal results only: the refresh's scales stay far from the exponent limits)
__device__ __forceinline__ double oz_i64_to_double(long long F, int e) {
    if (F == 0) return 0.0;
    const unsigned long long sgn = (unsigned long long)F & 0x8000000000000000ull;
    unsigned long long a = sgn ? (unsigned long long)(-F) : (unsigned long long)F;
    const int lz = __clzll((long long)a);
    a <<= lz;                                   // leading one at bit 63
    unsigned long long mant = a >> 11;          // 53 bits
    const unsigned r = (unsigned)(a & 0x7FFull);
    mant += (r > 0x400u || (r == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
    int ex = 1023 + 63 - lz + e - 56;
    if (mant >> 53) { mant >>= 1; ++ex; }
    return __longlong_as_double((long long)(sgn | ((unsigned long long)ex << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// M[i][j] += 2^(E_i + E_j) sum_c Pan[i][c] S[c][j] as a split product, with
// NKS K-steps of 16 (4 for a 64-column panel, 1 for a sub-panel or the K = 16
// flush), written only for the columns cols selects.  Persistent CTAs take
// (walker, 128-column block) units: the 7 S slices of the block are loaded
// once, then the 64-row tiles i stream through; the Pan slices of tile i+1
// are loaded (TMA) while the epilogue of tile i runs.
constexpr int OZ_THREADS = 512;   // 16 warps: 4 per TMEM lane quarter, each 16 of the 64 rows i

template <int NKS>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_gemm(const __grid_constant__ OzMaps maps, int W, int w0, int n, OzCols cols, OzWork Z,
              const uint8_t* mask, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = sm;                               // OZ_S slices of S, 128 rows each
    unsigned char* sB = sA + OZ_S * OZ_SLICE_A;           // OZ_S slices of Pan, 64 rows each
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(OZ_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t mb_tma = smem_u32(&mbar[0]), mb_mma = smem_u32(&mbar[1]);
    const uint32_t bytes_a = (uint32_t)OZ_S * OZ_SLICE_A, bytes_b = (uint32_t)OZ_S * OZ_SLICE_B;
    const int ntj = cols.jt_hi - cols.jt_lo, nti = n / OZ_TI;
    const long long units = (long long)W * ntj;
    uint32_t ph_tma = 0, ph_mma = 0;
    for (long long un = blockIdx.x; un < units && !s_abort; un += gridDim.x) {
        const int w = w0 + (int)(un / ntj);
        if (mask && !mask[w]) continue;
        const int j0 = (cols.jt_lo + (int)(un % ntj)) * OZ_TJ;
        const int ys = (int)((long long)w * OZ_S * n);
        if (tid == 0) {
            mbar_expect_tx(mb_tma, bytes_a + bytes_b);
            for (int t = 0; t < OZ_S; ++t) {
                tma_load_2d(smem_u32(sA + t * OZ_SLICE_A), &maps.S, 0, ys + t * n + j0, mb_tma);
                tma_load_2d(smem_u32(sB + t * OZ_SLICE_B), &maps.P, 0, ys + t * n, mb_tma);
            }
        }
        // per thread of the epilogue: column j (TMEM lane) and its scale
        const int quad = warp & 3, part = warp >> 2;
        const int j = j0 + 32 * quad + lane;
        const bool keep = j >= cols.c_lo && j < cols.c_hi && !(j >= cols.s_lo && j < cols.s_hi);
        const bool wact = __any_sync(0xffffffffu, keep);   // a warp with no column to write skips its epilogue
        const int eSj = Z.eS[(long long)w * n + j];
        double* Mw = Z.M + (long long)w * n * n;
        const int* eP = Z.eP + (long long)w * n;
        for (int it = 0; it < nti; ++it) {
            const int i0 = it * OZ_TI;
            if (tid == 0) {
                if (!mbar_wait(mb_tma, ph_tma)) {
                    set_dev_error(err, DEV_ERR_TIMEOUT);
                    s_abort = 1;
                    mbar_wait(mb_tma, ph_tma);   // let copies in flight land before leaving
                } else {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // fully unrolled: descriptors and accumulate flags are compile-time, so
                    // the issuing thread streams back-to-back MMAs
                    const uint64_t a0 = desc_sw128(smem_u32(sA)), b0 = desc_sw128(smem_u32(sB));
                    uint32_t started = 0;   // bit g: accumulator g holds a partial sum
#pragma unroll
                    for (int t = 0; t < OZ_S; ++t)
#pragma unroll
                        for (int u = 0; u < OZ_S; ++u) {
                            if (u + t > OZ_MAXLV) continue;
                            const int g = min(t + u, OZ_GROUPS - 1);   // level t+u+2: 2 .. 6, then 7..10
                            const uint64_t a = a0 + (uint64_t)((t * OZ_SLICE_A) >> 4);
                            const uint64_t b = b0 + (uint64_t)((u * OZ_SLICE_B) >> 4);
#pragma unroll
                            for (int ks = 0; ks < NKS; ++ks) {
                                const uint64_t adv = (uint64_t)(ks * 32) >> 4;   // 16 BF16 along K per MMA
                                oz_mma(tmem + 64u * g, a + adv, b + adv, (started >> g) & 1u);
                                started |= 1u << g;
                            }
                        }
                    mma_commit(mb_mma);
                }
                ph_tma ^= 1u;
            }
            // this thread's 16 values of M (rows i0 + 16 (q / 4) ..): the loads
            // overlap the MMAs
            double m[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) m[c] = keep ? Mw[(long long)(i0 + 16 * part + c) * n + j] : 0.0;
            __syncthreads();
            if (s_abort) break;
            if (!mbar_wait(mb_mma, ph_mma)) {
                set_dev_error(err, DEV_ERR_TIMEOUT);
                s_abort = 1;
            }
            ph_mma ^= 1u;
            __syncthreads();
            if (s_abort) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // the MMAs have read the Pan slices: load the next tile's during the epilogue
            if (tid == 0 && it + 1 < nti) {
                mbar_expect_tx(mb_tma, bytes_b);
                for (int t = 0; t < OZ_S; ++t)
                    tma_load_2d(smem_u32(sB + t * OZ_SLICE_B), &maps.P, 0, ys + t * n + i0 + OZ_TI, mb_tma);
            }
            // ---- epilogue: warp q reads TMEM lanes 32 (q % 4) .. +31 (columns j),
            //      and rows i0 + 16 (q / 4) .. +15 in two chunks of 8 ----
#pragma unroll
            for (int ch = 0; ch < 2 && wact; ++ch) {
                const int c0 = 16 * part + 8 * ch;
                float acc[OZ_GROUPS][8];
#pragma unroll
                for (int g = 0; g < OZ_GROUPS; ++g)
                    tmem_ld8(tmem + ((uint32_t)(32 * quad) << 16) + 64u * g + (uint32_t)c0, acc[g]);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    // levels 2..6 are integers N_l 2^(-8l), |N_l| < 2^23, recovered exactly;
                    // levels 7..10 rounded to a multiple of 2^-56.  F = sum in units of 2^-56
                    // (|F| < 2^62): exact; one rounding to double, one in the add.
                    const int n2 = __float2int_rn(acc[0][c] * 65536.0f);
                    const int n3 = __float2int_rn(acc[1][c] * 16777216.0f);
                    const int n4 = __float2int_rn(acc[2][c] * 4294967296.0f);
                    const int n5 = __float2int_rn(acc[3][c] * 1099511627776.0f);
                    const int n6 = __float2int_rn(acc[4][c] * 281474976710656.0f);
                    const int tl = __float2int_rn(acc[5][c] * 72057594037927936.0f);
                    const long long F = ((long long)(n2 * 256 + n3) << 32) + ((long long)(n4 * 256 + n5) << 16) +
                                        ((long long)n6 << 8) + tl;
                    const double d = oz_i64_to_double(F, eP[i0 + c0 + c] + eSj);
                    if (keep) Mw[(long long)(i0 + c0 + c) * n + j] = m[8 * ch + c] + d;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS)
                     : "memory");
    }
}

// ---- the delayed flush as a split product ------------------------------------

__global__ void k_oz_flush_go(int W, int K, const int* tau, const uint8_t* force, uint8_t* go) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const int t = tau[w];
    go[w] = (force ? (force[w] && t > 0) : (t >= K)) ? 1 : 0;
}

// Column balance of the slot matrices before they are sliced.  Every row is
// written as digits of one power-of-two scale (its largest entry), so a slot
// column much larger than the others (the step of a near-node update) would
// cost the other entries of the row their low bits.  Column c of P is scaled
// by 2^s_c and column c of Q by 2^-s_c, with s_c half the exponent gap of the
// two columns' maxima: P Q^T is unchanged exactly (powers of two), and the
// entries of a row span a far smaller range.  Persistent over walkers.
__global__ void __launch_bounds__(256) k_oz_col_balance(int W, int n, int ldx, int kk, const double* P,
                                                        const double* Q, const int* tau, const uint8_t* go,
                                                        int* cs) {
    __shared__ int sp[4][OZ_B], sq[4][OZ_B];
    const int c = threadIdx.x % OZ_B, g = threadIdx.x / OZ_B;   // 64 columns x 4 row groups
    for (int w = blockIdx.x; w < W; w += gridDim.x) {
        if (!go[w]) continue;
        const int cu = tau[w] * kk;
        int ep = 0, eq = 0;
        if (c < cu)
            for (int r = g; r < n; r += 4) {
                ep = max(ep, oz_bexp(P[((long long)w * n + r) * ldx + c]));
                eq = max(eq, oz_bexp(Q[((long long)w * n + r) * ldx + c]));
            }
        sp[g][c] = ep;
        sq[g][c] = eq;
        __syncthreads();
        if (g == 0) {
            ep = max(max(sp[0][c], sp[1][c]), max(sp[2][c], sp[3][c]));
            eq = max(max(sq[0][c], sq[1][c]), max(sq[2][c], sq[3][c]));
            cs[(long long)w * OZ_B + c] = (ep > 0 && eq > 0) ? (eq - ep) / 2 : 0;
        }
        __syncthreads();
    }
}

// Rows of the walkers' slot matrices X (rows of ldx doubles): the cu =
// tau * kk filled slot columns times sgn * 2^(cdir * cs[c]) (the column
// balance, exact), zeros after; slices and exponent as for the panel rows.
// Persistent over walkers: on steps where no walker flushes every block
// leaves after reading the go flags.
__device__ __forceinline__ double oz_pow2(int k) { return __hiloint2double((1023 + k) << 20, 0); }
__global__ void __launch_bounds__(256) k_oz_slice_rows(int W, int n, int ldx, int kk, const double* X, double sgn,
                                                       const int* cs, int cdir, const int* tau, const uint8_t* go,
                                                       uint16_t* dst, int* ex) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int w = blockIdx.x; w < W; w += gridDim.x) {
        if (!go[w]) continue;
        const int cu = tau[w] * kk;
        const double fa = lane < cu ? sgn * oz_pow2(cdir * cs[(long long)w * OZ_B + lane]) : 0.0;
        const double fb = lane + 32 < cu ? sgn * oz_pow2(cdir * cs[(long long)w * OZ_B + lane + 32]) : 0.0;
        for (int r = wid; r < n; r += 8) {
            const double* row = X + ((long long)w * n + r) * ldx;
            const double a = lane < cu ? fa * row[lane] : 0.0;
            const double b = lane + 32 < cu ? fb * row[lane + 32] : 0.0;
            const int mx = __reduce_max_sync(0xffffffffu, max(oz_bexp(a), oz_bexp(b)));
            const int E = mx > 0 ? mx - 1022 : 0;
            uint16_t ha[OZ_S], hb[OZ_S];
            oz_digits(oz_fixed(a, E), ha);
            oz_digits(oz_fixed(b, E), hb);
#pragma unroll
            for (int t = 0; t < OZ_S; ++t) {
                uint16_t* d = dst + (((long long)w * OZ_S + t) * n + r) * OZ_B;
                d[lane] = ha[t];
                d[lane + 32] = hb[t];
            }
            if (lane == 0) ex[(long long)w * n + r] = E;
        }
    }
}

// ---- host side ----------------------------------------------------------------

size_t oz_work_bytes(int W, int n) {
    const size_t Wn = (size_t)W * n;
    size_t b = 0;
    auto take = [&](size_t x) { b += (x + 255) / 256 * 256; };
    take(Wn * sizeof(int));                        // perm
    take((size_t)W * sizeof(double));              // logacc
    take((size_t)W * sizeof(double));              // sgnacc
    take((size_t)W * sizeof(int));                 // sing
    take(Wn * OZ_S * OZ_B * sizeof(uint16_t));     // Sb
    take(Wn * OZ_S * OZ_B * sizeof(uint16_t));     // Pb
    take(Wn * sizeof(int));                        // eS
    take(Wn * sizeof(int));                        // eP
    take((size_t)W);                               // go
    take(Wn * sizeof(double));                     // piv
    take((size_t)W * OZ_B * sizeof(int));          // cs
    return b;
}

void oz_work_carve(OzWork& Z, void* base, int W, int n) {
    const size_t Wn = (size_t)W * n;
    unsigned char* p = (unsigned char*)base;
    auto take = [&](size_t x) { unsigned char* q = p; p += (x + 255) / 256 * 256; return q; };
    Z.perm = (int*)take(Wn * sizeof(int));
    Z.logacc = (double*)take((size_t)W * sizeof(double));
    Z.sgnacc = (double*)take((size_t)W * sizeof(double));
    Z.sing = (int*)take((size_t)W * sizeof(int));
    Z.Sb = (uint16_t*)take(Wn * OZ_S * OZ_B * sizeof(uint16_t));
    Z.Pb = (uint16_t*)take(Wn * OZ_S * OZ_B * sizeof(uint16_t));
    Z.eS = (int*)take(Wn * sizeof(int));
    Z.eP = (int*)take(Wn * sizeof(int));
    Z.go = (uint8_t*)take((size_t)W);
    Z.piv = (double*)take(Wn * sizeof(double));
    Z.cs = (int*)take((size_t)W * OZ_B * sizeof(int));
}

// rows x 64 BF16 matrix, box 64 x box_rows, SWIZZLE_128B
static bool oz_map(CUtensorMap* m, const void* base, long long rows, int box_rows) {
    EncodeTiled enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)OZ_B, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)OZ_B * 2};
    cuuint32_t box[2] = {(cuuint32_t)OZ_B, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The whole refresh of the selected walkers: M = A^T (Z.M is the state's
// A^{-1} storage), n / 64 panels, then the column permutation and log|det|.
// Needs n % 128 == 0, 128 <= n <= 2048 and W <= 65535 (checked by the caller).
bool launch_refresh_oz(int W, int n, const double* A, const OzWork& Z, const DevState<double>& S,
                       const uint8_t* mask, bool delayed, bool reset_tau, int* err, cudaStream_t st,
                       void (*hook)(void*, int, int), void* hctx) {
    const long long rows = (long long)W * OZ_S * n;
    if (rows >= (1ll << 31)) return false;
    OzMaps maps;
    if (!oz_map(&maps.S, Z.Sb, rows, OZ_TJ) || !oz_map(&maps.P, Z.Pb, rows, OZ_TI)) return false;
    const size_t dyn = 1024 + (size_t)OZ_S * (OZ_SLICE_A + OZ_SLICE_B);
    if (cudaFuncSetAttribute(k_oz_gemm<OZ_B / 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_oz_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    launch_oz_load(W, n, A, Z.M, mask, st);
    const int SW = oz_subpanel_width(n);   // sub-panel width
    for (int k0 = 0; k0 < n; k0 += OZ_B) {
        if (hook) hook(hctx, 4, 1);
        if (n <= OZ_SUBPANEL_MAX_N) {
            // sub-panels: FP64 elimination, then the update of the other panel
            // columns as a one-K-step split product on the panel's 128-column tile
            const int jt = k0 / OZ_TJ;
            for (int sp = 0; sp < OZ_B / SW; ++sp) {
                const int ks = k0 + SW * sp;
                launch_oz_subpanel(W, n, k0, sp, Z, mask, st);
                k_oz_slice_P16<<<dim3(n / 16, W), 256, 0, st>>>(n, ks, SW, 0, Z, mask);
                k_oz_slice_S<<<dim3(OZ_TJ / 64, W), 256, 0, st>>>(n, ks, SW, jt * (OZ_TJ / 64), 0, Z, mask);
                const OzCols inner{k0, k0 + OZ_B, ks, ks + SW, jt, jt + 1};
                k_oz_gemm<1><<<nsm, OZ_THREADS, dyn, st>>>(maps, W, 0, n, inner, Z, mask, err);
            }
        } else {
            launch_oz_panel(W, 0, n, k0, Z, mask, st);
        }
        if (hook) { hook(hctx, 4, 0); hook(hctx, 5, 1); }
        k_oz_slice_P<<<dim3(n / 8, W), 256, 0, st>>>(n, k0, OZ_B, 0, Z, mask);
        k_oz_slice_S<<<dim3(n / 64, W), 256, 0, st>>>(n, k0, OZ_B, 0, 0, Z, mask);
        const OzCols outer{0, n, k0, k0 + OZ_B, 0, n / OZ_TJ};
        k_oz_gemm<OZ_B / 16><<<nsm, OZ_THREADS, dyn, st>>>(maps, W, 0, n, outer, Z, mask, err);
        if (hook) hook(hctx, 5, 0);
    }
    launch_oz_finish(W, n, Z, S, mask, delayed, reset_tau, st);
    return true;
}

// A_0^{-1} -= P Q^T (Sec. 2.3, Eq. delayed_Ainv) for the walkers that flush:
// with M = the stored A_0^{-1} (row l of storage = column l of A_0^{-1}),
// M[l][j] += sum_c (-Q)[l][c] P[j][c]: the P rows take the place of the S
// columns, the -Q rows that of the panel rows, no column is skipped.
bool launch_flush_split(int W, int n, int K, int Kc, int kk, const double* P, const double* Q, double sgnQ,
                        const int* tau, const uint8_t* force, const OzWork& Z, int* err, cudaStream_t st) {
    if (Kc < 1 || Kc > OZ_B) return false;
    const long long rows = (long long)W * OZ_S * n;
    if (rows >= (1ll << 31)) return false;
    static thread_local OzMaps maps;
    static thread_local const void* cached[2] = {nullptr, nullptr};
    static thread_local long long cached_rows = -1;
    if (cached[0] != Z.Sb || cached[1] != Z.Pb || cached_rows != rows) {
        if (!oz_map(&maps.S, Z.Sb, rows, OZ_TJ) || !oz_map(&maps.P, Z.Pb, rows, OZ_TI)) return false;
        cached[0] = Z.Sb;
        cached[1] = Z.Pb;
        cached_rows = rows;
    }
    const size_t dyn = 1024 + (size_t)OZ_S * (OZ_SLICE_A + OZ_SLICE_B);
    static thread_local bool attr = false;
    if (!attr) {
        bool ok = true;
        for (auto kern : {k_oz_gemm<1>, k_oz_gemm<2>, k_oz_gemm<3>, k_oz_gemm<4>})
            ok = ok && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return false;
        }
        attr = true;
    }
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    k_oz_flush_go<<<(W + 255) / 256, 256, 0, st>>>(W, K, tau, force, Z.go);
    const int sgrid = std::min(W, 8 * nsm);
    k_oz_col_balance<<<sgrid, 256, 0, st>>>(W, n, Kc, kk, P, Q, tau, Z.go, Z.cs);
    k_oz_slice_rows<<<sgrid, 256, 0, st>>>(W, n, Kc, kk, P, 1.0, Z.cs, 1, tau, Z.go, Z.Sb, Z.eS);
    k_oz_slice_rows<<<sgrid, 256, 0, st>>>(W, n, Kc, kk, Q, sgnQ, Z.cs, -1, tau, Z.go, Z.Pb, Z.eP);
    auto kern = k_oz_gemm<1>;
    switch ((Kc + 15) / 16) {
        case 2: kern = k_oz_gemm<2>; break;
        case 3: kern = k_oz_gemm<3>; break;
        case 4: kern = k_oz_gemm<4>; break;
        default: break;
    }
    const OzCols all{0, n, -1, -1, 0, n / OZ_TJ};
    kern<<<nsm, OZ_THREADS, dyn, st>>>(maps, W, 0, n, all, Z, Z.go, err);
    return true;
}

// Exact skew symmetry of the flushed walkers' A_0^{-1}, after the Pfaffian
// split-product flush A_0^{-1} += P Q^T: the product of the rounded slots
// (P = a M^{-1}, Q = a) is skew only up to that rounding, so the upper
// triangle (each entry one rounding of an exact product) is kept and the
// lower triangle is written as its exact negative (a sign flip, no FP64
// arithmetic), the diagonal as zero -- the same rule as the FP64 skew flush.
// Reads the upper half, writes the lower half.  One CTA per (walker, 32 x 32
// upper tile).
__global__ void __launch_bounds__(256) k_skew_project(int n, double* G, const uint8_t* go) {
    __shared__ double sU[32][33];
    const int w = blockIdx.y;
    if (!go[w]) return;
    const int nt = n / 32;
    int r = 0, rem = (int)blockIdx.x;
    while (rem >= nt - r) { rem -= nt - r; ++r; }
    const int j0 = 32 * r, l0 = 32 * (r + rem);
    double* Gw = G + (long long)w * n * n;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    // sU[l][j] = G(j0 + j, l0 + l), stored at Gw[(l0 + l) * n + j0 + j]
    for (int q = 0; q < 4; ++q) {
        const int a = ty + 8 * q;
        sU[a][tx] = Gw[(long long)(l0 + a) * n + j0 + tx];
    }
    __syncthreads();
    const auto neg = [](double v) {
        return __hiloint2double(__double2hiint(v) ^ (int)0x80000000, __double2loint(v));
    };
    if (rem != 0) {
        // lower block: G(l0 + l, j0 + j) = -G(j0 + j, l0 + l), stored at Gw[(j0 + j) * n + l0 + l]
        for (int q = 0; q < 4; ++q) {
            const int a = ty + 8 * q;   // j within the tile, tx = l
            Gw[(long long)(j0 + a) * n + l0 + tx] = neg(sU[tx][a]);
        }
    } else {
        // diagonal tile: entries below the diagonal from the ones above it
        for (int q = 0; q < 4; ++q) {
            const int a = ty + 8 * q;   // column l = j0 + a, row j = j0 + tx
            if (tx > a) Gw[(long long)(j0 + a) * n + j0 + tx] = neg(sU[tx][a]);
            else if (tx == a) Gw[(long long)(j0 + a) * n + j0 + tx] = 0.0;
        }
    }
}

void launch_skew_project(int W, int n, double* G, const uint8_t* go, cudaStream_t st) {
    const int nt = n / 32;
    k_skew_project<<<dim3(nt * (nt + 1) / 2, W), 256, 0, st>>>(n, G, go);
}

}  // namespace lru
