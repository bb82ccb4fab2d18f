// Delayed flush on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The delayed forms keep A_0^{-1} and K correction slots and fold them every K
// accepted steps (Sec. 2.3 Eq. delayed_Ainv: A^{-1} = A_0^{-1} - P Q^T; Sec.
// 3.3 Eq. pf_delayed_Ainv: A^{-1} = A_0^{-1} + P Q^T).  The contraction P Q^T
// has inner dimension K*k (16..64): it is tiny for the tensor cores, and the
// cost is the FP64 read-modify-write of A_0^{-1}.  The kernel therefore
// streams 128 x 128 output tiles through one persistent CTA per SM slot:
//   TMA (SWIZZLE_128B, no multicast) brings the TF32 hi/lo splits of the P and
//   Q rows of the tile into shared memory; one thread issues the MMAs
//   (3 terms hi*hi + hi*lo + lo*hi for FP32-class accuracy, or 1 term) into a
//   128 x 128 FP32 accumulator in tensor memory; all eight warps read it back
//   with tcgen05.ld and update the FP64 tile in global memory (coalesced
//   256-byte rows, float->double by integer ops so only the final add uses the
//   slow FP64 pipe).  For the Pfaffian only tiles with J <= L are computed and
//   the mirror tile is written as the exact negative transpose, keeping
//   A_0^{-1} exactly skew.
// Every wait on an mbarrier is bounded; on time-out the kernel records
// DEV_ERR_TIMEOUT, waits (bounded) for its copies in flight, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace lru {

constexpr int TC_THREADS = 256;
constexpr int TILE = 128;         // M = N = 128
constexpr int ROW_BYTES = 128;    // one 128-byte swizzle row per tile row and K chunk
constexpr int CHUNK_BYTES = TILE * ROW_BYTES;    // 16 KiB per operand per K chunk
constexpr uint32_t TMEM_COLS = 128;

struct TcMaps {
    CUtensorMap ph, pl, qh, ql;
};

// instruction descriptors: D f32, A and B K-major, M = N = 128;
// kind::tf32 (A/B format 2 = TF32) and kind::f16 (A/B format 1 = BF16)
constexpr uint32_t IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TILE >> 3) << 17) |
                                ((uint32_t)(TILE >> 4) << 24);
constexpr uint32_t IDESC_BF16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TILE >> 3) << 17) |
                                ((uint32_t)(TILE >> 4) << 24);

// one MMA step of K = 32 bytes of each row (8 TF32 or 16 BF16 elements)
template <bool BF16>
__device__ __forceinline__ void mma_step(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
    if constexpr (BF16) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(dtmem), "l"(a), "l"(b), "r"(IDESC_BF16), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(dtmem), "l"(a), "l"(b), "r"(IDESC_TF32), "r"(acc)
            : "memory");
    }
}

// exact float -> double with integer operations (FP32 zeros and subnormals
// become signed zero; the flush values are far from that range)
__device__ __forceinline__ double f2d_int(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t mag = u & 0x7FFFFFFFu;
    uint32_t hi = ((mag >> 3) + 0x38000000u) | (u & 0x80000000u);
    uint32_t lo = u << 29;
    if (mag < 0x00800000u) { hi = u & 0x80000000u; lo = 0u; }
    return __hiloint2double((int)hi, (int)lo);
}

// One CTA per SM slot, persistent over the (walker, tile) list of the walkers
// that flush now.  Walker w flushes when tau_w >= K (or force[w] and tau_w > 0).
template <bool PF, bool BF16>
__global__ void __launch_bounds__(TC_THREADS, 2)
    k_flush_tc(const __grid_constant__ TcMaps maps, DevLayout L, double* G, const int* tau, const uint8_t* force,
               int nkc, int three, int* err) {
    constexpr int KCHUNK = BF16 ? 64 : 32;   // elements per 128-byte row
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // 1024-byte aligned operand area: [Ph | Pl | Qh | Ql] x nkc chunks
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sPh = sm;
    unsigned char* sPl = sPh + nkc * CHUNK_BYTES;
    unsigned char* sQh = sPl + nkc * CHUNK_BYTES;
    unsigned char* sQl = sQh + nkc * CHUNK_BYTES;
    // mirror staging (pf): one 32 x 33 block per warp (warps q and q+4 share TMEM lanes)
    double* sT = reinterpret_cast<double*>(sQl + nkc * CHUNK_BYTES) + (size_t)warp * 32 * 33;
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TMEM_COLS)
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
    const uint32_t tx_bytes = 4u * nkc * CHUNK_BYTES;

    uint32_t phase = 0;
    // this CTA's first tile of the current walker: (blockIdx.x - tiles of the
    // earlier due walkers) mod gridDim.x, advanced in 32 bits per due walker
    int first = (int)blockIdx.x;
    for (int w = 0; w < L.W && !s_abort; ++w) {
        const int t = tau[w];
        const bool go = force ? (force[w] && t > 0) : (t >= L.K);
        if (!go) continue;
        const int n = L.nw(w);
        const int nt = (n + TILE - 1) / TILE;
        const int ntiles = PF ? nt * (nt + 1) / 2 : nt * nt;
        const long long vo = L.vo(w);
        double* Gw = G + L.mo(w);
        // tiles of this walker owned by this CTA
        for (int ti = first; ti < ntiles; ti += gridDim.x) {
            int tJ, tL;
            if (PF) {
                // row-major enumeration of the upper triangle J <= L
                int r = 0, rem = (int)ti;
                while (rem >= nt - r) { rem -= nt - r; ++r; }
                tJ = r;
                tL = r + rem;
            } else {
                tJ = (int)(ti % nt);
                tL = (int)(ti / nt);
            }
            const int j0 = tJ * TILE, l0 = tL * TILE;
            // ---- TMA: P rows j0.. and Q rows l0.. of this walker ----
            if (tid == 0) {
                mbar_expect_tx(mb_tma, tx_bytes);
                for (int kc = 0; kc < nkc; ++kc) {
                    tma_load_2d(smem_u32(sPh + kc * CHUNK_BYTES), &maps.ph, kc * KCHUNK, (int)(vo + j0), mb_tma);
                    tma_load_2d(smem_u32(sPl + kc * CHUNK_BYTES), &maps.pl, kc * KCHUNK, (int)(vo + j0), mb_tma);
                    tma_load_2d(smem_u32(sQh + kc * CHUNK_BYTES), &maps.qh, kc * KCHUNK, (int)(vo + l0), mb_tma);
                    tma_load_2d(smem_u32(sQl + kc * CHUNK_BYTES), &maps.ql, kc * KCHUNK, (int)(vo + l0), mb_tma);
                }
                if (!mbar_wait(mb_tma, phase)) {
                    set_dev_error(err, DEV_ERR_TIMEOUT);
                    s_abort = 1;
                    mbar_wait(mb_tma, phase);   // let copies in flight land before leaving
                } else {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // ---- MMA: D = sum_k P_k Q_k^T (hi*hi [+ hi*lo + lo*hi]) ----
                    uint32_t acc = 0;
                    for (int kc = 0; kc < nkc; ++kc) {
                        const uint64_t ah = desc_sw128(smem_u32(sPh + kc * CHUNK_BYTES));
                        const uint64_t al = desc_sw128(smem_u32(sPl + kc * CHUNK_BYTES));
                        const uint64_t bh = desc_sw128(smem_u32(sQh + kc * CHUNK_BYTES));
                        const uint64_t bl = desc_sw128(smem_u32(sQl + kc * CHUNK_BYTES));
#pragma unroll
                        for (int ks = 0; ks < ROW_BYTES / 32; ++ks) {
                            const uint64_t adv = (uint64_t)(ks * 32) >> 4;   // 32 bytes along K per MMA
                            if (three) {
                                mma_step<BF16>(tmem, al + adv, bh + adv, acc);
                                acc = 1;
                                mma_step<BF16>(tmem, ah + adv, bl + adv, 1);
                            }
                            mma_step<BF16>(tmem, ah + adv, bh + adv, acc);
                            acc = 1;
                        }
                    }
                    mma_commit(mb_mma);
                }
            }
            __syncthreads();
            if (s_abort) break;
            // ---- wait for the accumulator ----
            bool ok = mbar_wait(mb_mma, phase);
            if (!ok) {
                set_dev_error(err, DEV_ERR_TIMEOUT);
                s_abort = 1;
            }
            __syncthreads();
            if (s_abort) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            phase ^= 1u;
            // ---- epilogue: warp q reads TMEM lanes 32 (q % 4) .. +31 (rows j),
            //      warpgroup q / 4 takes columns 64 (q / 4) .. +63 ----
            const int quad = warp & 3, half = warp >> 2;
            const int jl = 32 * quad + lane;
            const int j = j0 + jl;
            for (int ch = 0; ch < 4; ++ch) {
                const int c0 = 64 * half + 16 * ch;
                float acc[16];
                tmem_ld16(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)c0, acc);
                double g[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int l = l0 + c0 + c;
                    const bool keep = j < n && l < n && (!PF || tJ != tL || j < l);
                    g[c] = keep ? Gw[(long long)l * n + j] : 0.0;
                }
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int l = l0 + c0 + c;
                    const double d = f2d_int(acc[c]);
                    const double nv = PF ? g[c] + d : g[c] - d;
                    if (j < n && l < n) {
                        if (!PF || tJ != tL || j < l) Gw[(long long)l * n + j] = nv;
                        else if (j == l) Gw[(long long)l * n + j] = 0.0;
                    }
                    if (PF) sT[lane * 33 + c] = nv;
                }
                if (PF) {
                    __syncwarp();
                    // mirror: (l, j) = -(j, l) at G[j*n + l], 16 consecutive l per row j,
                    // two rows per warp instruction
#pragma unroll 4
                    for (int r2 = 0; r2 < 16; ++r2) {
                        const int r = 2 * r2 + (lane >> 4);
                        const int jr = j0 + 32 * quad + r;
                        const int l = l0 + c0 + (lane & 15);
                        if (jr < n && l < n && (tJ != tL || jr < l))
                            Gw[(long long)jr * n + l] = -sT[r * 33 + (lane & 15)];
                    }
                    __syncwarp();
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
        first -= ntiles % (int)gridDim.x;
        if (first < 0) first += gridDim.x;
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
}

// ---- host side ----------------------------------------------------------------

// rows x cols matrix (row-major, cols = Kc_pad) of fp32 or bf16, box
// (128 bytes) x 128 rows, SWIZZLE_128B
static bool make_map(CUtensorMap* m, const void* base, long long rows, int cols, bool bf16) {
    EncodeTiled enc = get_encode();
    if (!enc) return false;
    const size_t es_bytes = bf16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * es_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / es_bytes), (cuuint32_t)TILE};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base,
                     dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool launch_flush_tc(int mode, bool pf, const DevLayout& L, double* G, const void* Ph, const void* Pl,
                     const void* Qh, const void* Ql, const int* tau, const uint8_t* force_mask, int* err,
                     cudaStream_t st) {
    // mode: 1 = TF32x3, 2 = TF32, 3 = BF16, 4 = BF16x3
    if (mode < 1 || mode > 4) return false;
    const bool bf16 = mode >= 3;
    const int kchunk = bf16 ? 64 : 32;
    if (L.Kc32 <= 0 || L.Kc32 % kchunk) return false;
    static thread_local const void* cached[4] = {nullptr, nullptr, nullptr, nullptr};
    static thread_local long long cached_rows = -1;
    static thread_local int cached_cols = -1, cached_bf16 = -1;
    static thread_local TcMaps maps;
    if (cached[0] != Ph || cached[1] != Pl || cached[2] != Qh || cached[3] != Ql || cached_rows != L.rows ||
        cached_cols != L.Kc32 || cached_bf16 != (int)bf16) {
        if (!make_map(&maps.ph, Ph, L.rows, L.Kc32, bf16) || !make_map(&maps.pl, Pl, L.rows, L.Kc32, bf16) ||
            !make_map(&maps.qh, Qh, L.rows, L.Kc32, bf16) || !make_map(&maps.ql, Ql, L.rows, L.Kc32, bf16))
            return false;
        cached[0] = Ph; cached[1] = Pl; cached[2] = Qh; cached[3] = Ql;
        cached_rows = L.rows;
        cached_cols = L.Kc32;
        cached_bf16 = (int)bf16;
    }
    const int nkc = L.Kc32 / kchunk;
    const size_t dyn = 1024 + (size_t)4 * nkc * CHUNK_BYTES + (pf ? (size_t)8 * 32 * 33 * sizeof(double) : 0);
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    auto kern = pf ? (bf16 ? k_flush_tc<true, true> : k_flush_tc<true, false>)
                   : (bf16 ? k_flush_tc<false, true> : k_flush_tc<false, false>);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // two CTAs per SM (2 x 128 TMEM columns): one streams its epilogue while
    // the other waits on TMA and the MMAs
    const int three = (mode == 1 || mode == 4) ? 1 : 0;
    kern<<<2 * nsm, TC_THREADS, dyn, st>>>(maps, L, G, tau, force_mask, nkc, three, err);
    return true;
}

}  // namespace lru
