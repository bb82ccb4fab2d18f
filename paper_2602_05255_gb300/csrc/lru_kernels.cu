// Propose / accept / flush kernels of the low-rank update path.
//
// Storage: walker w keeps A^{-1} column-major, G[l*n + j] = (A^{-1})_{jl}, so
// column i of A^{-1} (what a one-hot row update reads, Sec. 2.2) is one
// contiguous "chunk" and the row-update GEMV V A^{-1} is one dot product per
// chunk.  The plain accept therefore reads and writes every chunk exactly
// once: chunk_l -= X R^{-1} (V . chunk_l), the Woodbury step of Eq. det_inv.
#include "common.cuh"
#include "internal.h"
#include "small_core.cuh"
#include "df.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

namespace lru {

constexpr int PT = 256;    // threads of the per-walker kernels
constexpr int JPT = 8;     // vector elements per thread: n <= PT * JPT = 2048
constexpr int MAXKK = 16;  // vector slots per update (det k <= 16, pf 2k <= 16)

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// hi + lo split of a double for the tensor-core flush: hi is x rounded to TF32,
// lo the TF32-rounded remainder (3-term products reach about FP32 accuracy).
__device__ __forceinline__ void split_tf32(double x, float& hi, float& lo) {
    float xf = (float)x;
    hi = tf32_round(xf);
    lo = tf32_round((float)(x - (double)hi));
}

// store the hi / lo split of x at element o of the split copies (TF32 in fp32
// words, or bf16); PQ selects the P (0) or Q (1) arrays
template <typename T>
__device__ __forceinline__ void store_split(const DevState<T>& S, int PQ, long long o, double x) {
    float* h = PQ ? S.Q32h : S.P32h;
    float* l = PQ ? S.Q32l : S.P32l;
    if (S.split_bf16) {
        const float xf = (float)x;
        const __nv_bfloat16 bh = __float2bfloat16_rn(xf);
        const __nv_bfloat16 bl = __float2bfloat16_rn((float)(x - (double)__bfloat162float(bh)));
        reinterpret_cast<__nv_bfloat16*>(h)[o] = bh;
        reinterpret_cast<__nv_bfloat16*>(l)[o] = bl;
    } else {
        float hi, lo;
        split_tf32(x, hi, lo);
        h[o] = hi;
        l[o] = lo;
    }
}

template <typename T>
__device__ __forceinline__ const T* vec_ptr(const DevOperand& O, const DevLayout& L, int w, int a, int n) {
    return reinterpret_cast<const T*>(O.dense) + (L.vo(w) * O.slots + (long long)a * n);
}

// Thread-block reduction of NV values per thread into out[0..NV) (smem red has
// >= 8*NV entries).  All threads must call it.
template <typename T, int NV>
__device__ void block_reduce_vec(T (&v)[NV], T* red, T* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[wid * NV + q] = v[q];
    __syncthreads();
    if (threadIdx.x < NV) {
        T s = s_zero(T());
        for (int q = 0; q < PT / 32; ++q) s = s + red[q * NV + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// The (walker, tile) work of a flush, enumerated without atomics: every CTA
// scans the walkers, keeps a running tile offset over those that flush now
// and takes the tiles whose global index is congruent to its block index.
// Pfaffian tiles cover J <= L only.
struct TileIter {
    int first_ = -1;             // (blockIdx.x - tiles of the earlier due walkers) mod gridDim.x
    int last_nt = -1, last_d = 0;
    __device__ static int tiles(int nt, bool pf) { return pf ? nt * (nt + 1) / 2 : nt * nt; }
    __device__ static void coords(int ti, int nt, bool pf, int& tJ, int& tL) {
        if (pf) {
            int r = 0, rem = ti;
            while (rem >= nt - r) { rem -= nt - r; ++r; }
            tJ = r;
            tL = r + rem;
        } else {
            tL = ti / nt;
            tJ = ti - tL * nt;
        }
    }
    // kept in 32 bits and advanced by one subtraction per due walker: a 64-bit
    // modulo here, run by every thread of every CTA for every due walker,
    // cost more instructions than the flush arithmetic itself
    __device__ int first(int ntiles) {
        const int G = (int)gridDim.x;
        if (first_ < 0) first_ = (int)blockIdx.x;
        const int f = first_;
        if (ntiles != last_nt) {
            last_nt = ntiles;
            last_d = ntiles % G;
        }
        first_ -= last_d;
        if (first_ < 0) first_ += G;
        return f;
    }
};

// Walkers due for a flush, read a chunk at a time into shared memory (one
// coalesced read of tau per chunk) rather than by one dependent load per
// walker in every CTA, so that a step with no walker due costs a short scan.
// s_tau[i] = tau of walker w0 + i if it is due, else -1; returns the chunk
// length.  Called by every thread of a FLUSH_SCAN-thread CTA.
constexpr int FLUSH_SCAN = 256;

template <typename T>
__device__ __forceinline__ int flush_scan(const DevLayout& L, const DevState<T>& S, const uint8_t* force, int w0,
                                          int* s_tau) {
    __syncthreads();   // the previous chunk's readers are done
    const int w = w0 + (int)threadIdx.x;
    if (threadIdx.x < FLUSH_SCAN) {
        int t = -1;
        if (w < L.W) {
            const int tau = S.tau[w];
            if (force ? (force[w] && tau > 0) : (tau >= L.K)) t = tau;
        }
        s_tau[threadIdx.x] = t;
    }
    __syncthreads();
    return min(FLUSH_SCAN, L.W - w0);
}

// ---------------------------------------------------------------------------
// propose: X = A^{-1} U (delayed: A_0^{-1} U -/+ P (Q^T U)), core, small solve
// det: Sec. 2.1 Eq. det_R, delayed Sec. 2.3 (R_tau, a_tau equations)
// pf : App. A.2 Eq. pf_low_rank, delayed Sec. 3.3 (R_tau, a_tau equations)
// One CTA per walker.
// ---------------------------------------------------------------------------
// SKEWM (Pfaffian): M is projected onto its skew part before it is inverted
// and M^{-1} after, as the skew-form updates (the delayed slots, the exactly
// skew plain accept) need; the persistent step's generic Woodbury accept
// needs the inverse of M as computed (SKEWM = false there).
template <typename T, bool PF, bool DELAYED, bool SKEWM = DELAYED>
__device__ void propose_walker(const int w, const DevLayout L, const DevState<T> S, const DevOperand U,
                               const DevOperand V, const T* C, T* ratio_out, int* st_out) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    T* s_qtu = reinterpret_cast<T*>(dyn_smem);  // Kc x MAXKK (delayed only)
    __shared__ T s_core[MAXKK * MAXKK];
    __shared__ T s_inv[MAXKK * MAXKK];
    __shared__ T s_cinv[MAXKK * MAXKK];
    __shared__ T s_red[8 * 16];
    __shared__ int s_iu[MAXKK], s_iv[MAXKK];
    __shared__ int s_bad;
    __shared__ T s_pfc;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int n = L.nw(w), kk = L.kv(w);
    const long long vo = L.vo(w);
    const T* G = S.G + L.mo(w);
    T* X = S.X + vo * L.kk;
    const int Kc = L.Kc;
    const int cu = DELAYED ? S.tau[w] * kk : 0;
    const DevOperand& Vop = PF ? U : V;

    if (tid == 0) s_bad = 0;
    __syncthreads();
    if (tid < kk) {
        int iu = -1, iv = -1;
        if ((U.mask >> tid) & 1u) {
            iu = U.idx[(long long)w * U.slots + tid];
            if (iu < 0 || iu >= n) atomicExch(&s_bad, 1);
        }
        if ((Vop.mask >> tid) & 1u) {
            iv = Vop.idx[(long long)w * Vop.slots + tid];
            if (iv < 0 || iv >= n) atomicExch(&s_bad, 1);
        }
        s_iu[tid] = iu;
        s_iv[tid] = iv;
    }
    if (PF && tid == 0) {
        // C^{-1} and pf(C^{-1}); C = NULL means C = -J, so C^{-1} = J (Sec. 3.1)
        const int k2 = kk;
        if (C == nullptr) {
            for (int i = 0; i < k2; ++i)
                for (int j = 0; j < k2; ++j) {
                    double v = (j == i + k2 / 2) ? 1.0 : ((i == j + k2 / 2) ? -1.0 : 0.0);
                    s_cinv[i * MAXKK + j] = make_real<T>(v);
                }
        } else {
            const T* Cw = C + (long long)w * L.kk * L.kk;   // slot of (2 kmax)^2 per walker
            for (int i = 0; i < k2; ++i)
                for (int j = 0; j < k2; ++j) s_cinv[i * MAXKK + j] = Cw[i * k2 + j];
            T dC;
            int stc = small_gj_inverse(s_cinv, k2, MAXKK, &dC);
            if (stc != CORE_OK) atomicExch(&s_bad, 2);
            for (int i = 0; i < k2; ++i)      // exactly skew
                for (int j = i; j < k2; ++j) {
                    T a = s_cinv[i * MAXKK + j], b = s_cinv[j * MAXKK + i];
                    T h = s_half(a - b);
                    s_cinv[i * MAXKK + j] = h;
                    s_cinv[j * MAXKK + i] = s_neg(h);
                }
        }
        for (int i = 0; i < k2; ++i)
            for (int j = 0; j < k2; ++j) s_core[i * MAXKK + j] = s_cinv[i * MAXKK + j];
        s_pfc = small_pf(s_core, k2, MAXKK);
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            int code = s_bad == 1 ? 3 /*LRU_WALKER_BAD_INDEX*/ : 1;
            S.pst[w] = code;
            if (st_out) st_out[w] = code;
            ratio_out[w] = s_zero(T());
            S.ratio[w] = s_zero(T());
        }
        return;
    }

    // ---- delayed: Q^T U (cu x kk), the (b_t^T U) / (a_t^T B) factors ----
    // one-hot columns read row i of Q; dense columns were reduced by k_qtu_dense
    if constexpr (DELAYED) {
        for (int a = 0; a < kk; ++a) {
            if (s_iu[a] >= 0) {
                for (int c = tid; c < cu; c += PT) s_qtu[c * MAXKK + a] = S.Q[(vo + s_iu[a]) * Kc + c];
            } else {
                for (int c = tid; c < cu; c += PT) s_qtu[c * MAXKK + a] = S.QtU[((long long)w * Kc + c) * MAXKK + a];
            }
        }
        __syncthreads();
    }

    // ---- X = A^{-1} U ----
    // one-hot columns: a contiguous chunk copy; dense columns: axpy over chunks
    for (int a = 0; a < kk; ++a) {
        T* Xa = X + (long long)a * n;
        if (s_iu[a] >= 0) {
            const T* col = G + (long long)s_iu[a] * n;
            for (int j = tid; j < n; j += PT) Xa[j] = col[j];
        }
    }
    {
        // dense columns, four at a time
        int dl[MAXKK], nd = 0;
        for (int a = 0; a < kk; ++a)
            if (s_iu[a] < 0 && a != U.pre) dl[nd++] = a;
        if (nd == 1) {
            // one dense column (the Pfaffian row-and-column move, a rank-1
            // dense update): each thread walks the columns for its rows with
            // the loads of eight columns in flight, one accumulator per row
            // (the same FMA order as the grouped loop below)
            const T* u0 = vec_ptr<T>(U, L, w, dl[0], n);
            T* Xa = X + (long long)dl[0] * n;
            for (int j = tid; j < n; j += PT) {
                T acc = s_zero(T());
#pragma unroll 8
                for (int l = 0; l < n; ++l) acc = s_fma(G[(long long)l * n + j], u0[l], acc);
                Xa[j] = acc;
            }
            nd = 0;
        }
        for (int g0 = 0; g0 < nd; g0 += 4) {
            const int ng = min(4, nd - g0);
            T acc[4][JPT];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int m = 0; m < JPT; ++m) acc[q][m] = s_zero(T());
            const T* up[4];
            for (int q = 0; q < 4; ++q) up[q] = vec_ptr<T>(U, L, w, dl[g0 + min(q, ng - 1)], n);
            for (int l = 0; l < n; ++l) {
                const T* col = G + (long long)l * n;
                T ul[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) ul[q] = up[q][l];
#pragma unroll
                for (int m = 0; m < JPT; ++m) {
                    const int j = tid + m * PT;
                    if (j < n) {
                        T g = col[j];
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[q][m] = s_fma(g, ul[q], acc[q][m]);
                    }
                }
            }
            for (int q = 0; q < ng; ++q) {
                T* Xa = X + (long long)dl[g0 + q] * n;
#pragma unroll
                for (int m = 0; m < JPT; ++m) {
                    const int j = tid + m * PT;
                    if (j < n) Xa[j] = acc[q][m];
                }
            }
        }
    }
    __syncthreads();

    if constexpr (DELAYED) {
        // X -= P (Q^T U) (det)   or   X += P (Q^T B) (pf)
        for (int j = tid; j < n; j += PT) {
            const T* prow = S.P + (vo + j) * Kc;
            for (int a = 0; a < kk; ++a) {
                T s = s_zero(T());
                for (int c = 0; c < cu; ++c) s = s_fma(prow[c], s_qtu[c * MAXKK + a], s);
                T* Xa = X + (long long)a * n;
                Xa[j] = PF ? (Xa[j] + s) : (Xa[j] - s);
            }
        }
        __syncthreads();
        if constexpr (!PF) {
            // a_tau = X goes to slot tau of P now (harmless if the proposal is rejected)
            for (int j = tid; j < n; j += PT) {
                for (int a = 0; a < kk; ++a) {
                    const long long off = (vo + j) * Kc + cu + a;
                    T x = X[(long long)a * n + j];
                    S.P[off] = x;
                    if constexpr (!traits<T>::is_complex && sizeof(T) == 8) {
                        if (S.P32h) store_split(S, 0, (vo + j) * L.Kc32 + cu + a, (double)x);
                    }
                }
            }
        }
    }

    // ---- core: R = I + V X (det) or M = C^{-1} + B^T X (pf) ----
    for (int p = wid; p < kk * kk; p += PT / 32) {
        const int b = p / kk, a = p % kk;
        const T* Xa = X + (long long)a * n;
        T s;
        if (s_iv[b] >= 0) {
            s = Xa[s_iv[b]];
        } else {
            const T* vb = vec_ptr<T>(Vop, L, w, b, n);
            T part = s_zero(T());
            for (int j = lane; j < n; j += 32) part = s_fma(vb[j], Xa[j], part);
            s = warp_sum(part);
        }
        if (lane == 0) {
            T base = PF ? s_cinv[b * MAXKK + a] : make_real<T>(b == a ? 1.0 : 0.0);
            s_core[b * MAXKK + a] = base + s;
        }
    }
    // ---- det delayed: V P (kk x cu) for the accept's correction ----
    if constexpr (DELAYED && !PF) {
        T* VP = S.VP + (long long)w * MAXKK * Kc;
        for (int p = wid; p < kk * cu; p += PT / 32) {
            const int b = p / cu, c = p % cu;
            T s;
            if (s_iv[b] >= 0) {
                s = S.P[(vo + s_iv[b]) * Kc + c];
            } else {
                const T* vb = vec_ptr<T>(Vop, L, w, b, n);
                T part = s_zero(T());
                for (int j = lane; j < n; j += 32) part = s_fma(vb[j], S.P[(vo + j) * Kc + c], part);
                s = warp_sum(part);
            }
            if (lane == 0) VP[b * Kc + c] = s;
        }
    }
    __syncthreads();

    // ---- small core ----
    if (tid == 0) {
        int st;
        T ratio;
        if constexpr (!PF) {
            for (int i = 0; i < kk; ++i)
                for (int j = 0; j < kk; ++j) s_inv[i * MAXKK + j] = s_core[i * MAXKK + j];
            st = small_gj_inverse(s_inv, kk, MAXKK, &ratio);
        } else {
            // The skew-form updates (Eq. pf_delayed_Ainv, and the exactly skew
            // plain accept) need M and M^{-1} exactly skew; a generic Woodbury
            // accept needs the inverse of M as computed (projecting M there
            // makes the chain unstable).
            if (SKEWM)
                for (int i = 0; i < kk; ++i)
                    for (int j = i; j < kk; ++j) {
                        T h = s_half(s_core[i * MAXKK + j] - s_core[j * MAXKK + i]);
                        s_core[i * MAXKK + j] = h;
                        s_core[j * MAXKK + i] = s_neg(h);
                    }
            for (int i = 0; i < kk; ++i)
                for (int j = 0; j < kk; ++j) s_inv[i * MAXKK + j] = s_core[i * MAXKK + j];
            T dM;
            st = small_gj_inverse(s_inv, kk, MAXKK, &dM);
            if (SKEWM)
                for (int i = 0; i < kk; ++i)
                    for (int j = i; j < kk; ++j) {
                        T h = s_half(s_inv[i * MAXKK + j] - s_inv[j * MAXKK + i]);
                        s_inv[i * MAXKK + j] = h;
                        s_inv[j * MAXKK + i] = s_neg(h);
                    }
            // pf of the skew part of M (the ratio, Eq. pf_low_rank)
            for (int i = 0; i < kk; ++i)
                for (int j = i; j < kk; ++j) {
                    T h = s_half(s_core[i * MAXKK + j] - s_core[j * MAXKK + i]);
                    s_core[i * MAXKK + j] = h;
                    s_core[j * MAXKK + i] = s_neg(h);
                }
            T pfM = small_pf(s_core, kk, MAXKK);
            ratio = pfM * s_recip(s_pfc);
            if (st == CORE_OK && !s_isfinite(ratio)) st = CORE_NONFINITE;
        }
        T* Ri = S.Rinv + (long long)w * MAXKK * MAXKK;
        for (int i = 0; i < kk; ++i)
            for (int j = 0; j < kk; ++j) Ri[i * MAXKK + j] = s_inv[i * MAXKK + j];
        int code = st == CORE_OK ? 0 : (st == CORE_SINGULAR ? 1 : 2);
        S.pst[w] = code;
        S.ratio[w] = ratio;
        ratio_out[w] = ratio;
        if (st_out) st_out[w] = code;
    }
    if constexpr (DELAYED && PF) {
        __syncthreads();
        // slots: Q[:, tau] = a_tau = X, P[:, tau] = a_tau M^{-1} (Sec. 3.3)
        for (int j = tid; j < n; j += PT) {
            for (int b = 0; b < kk; ++b) {
                T q = X[(long long)b * n + j];
                T p = s_zero(T());
                for (int a = 0; a < kk; ++a) p = s_fma(X[(long long)a * n + j], s_inv[a * MAXKK + b], p);
                const long long off = (vo + j) * Kc + cu + b;
                S.Q[off] = q;
                S.P[off] = p;
                if constexpr (!traits<T>::is_complex && sizeof(T) == 8) {
                    if (S.P32h) {
                        const long long o32 = (vo + j) * L.Kc32 + cu + b;
                        store_split(S, 0, o32, (double)p);
                        store_split(S, 1, o32, (double)q);
                    }
                }
            }
        }
    }
}

// X_a = A^{-1} u_a for the one dense column a of a proposal (the Pfaffian
// row-and-column move B = [x, e_i], a rank-1 dense update), before the
// propose kernel, which then skips that column.  One CTA per walker; thread t
// owns rows t + PT r (r < NR) and walks the columns of A^{-1} (contiguous in
// the rows, so every load is coalesced) with two independent accumulators per
// row (the column range split in halves) and few registers, so that many
// CTAs per SM hide the load latency.  DF (real FP64 only): the products in
// double-float arithmetic on the FP32 pipe (integer-split elements against
// the split u), so the pass is bound by HBM instead of the FP64 pipe.
template <typename T, int NR, bool DF>
__global__ void __launch_bounds__(PT, 4) k_dense_column(DevLayout L, DevState<T> S, DevOperand U, int a) {
    __shared__ T su[2048];
    __shared__ float2 suf[DF ? 2048 : 1];
    const int w = blockIdx.x;
    const int n = L.nw(w);
    const T* u = vec_ptr<T>(U, L, w, a, n);
    for (int l = threadIdx.x; l < n; l += PT) {
        su[l] = u[l];
        if constexpr (DF) {
            float h, lo;
            split_d((double)u[l], h, lo);
            suf[l] = make_float2(h, lo);
        }
    }
    __syncthreads();
    const T* G = S.G + L.mo(w);
    T* Xa = S.X + L.vo(w) * L.kk + (long long)a * n;
    const int h = n / 2;
    if constexpr (DF) {
        float ah0[NR], al0[NR], ah1[NR], al1[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) ah0[r] = al0[r] = ah1[r] = al1[r] = 0.f;
#pragma unroll 4
        for (int l = 0; l < h; ++l) {
            const double* c0 = reinterpret_cast<const double*>(G) + (long long)l * n;
            const double* c1 = reinterpret_cast<const double*>(G) + (long long)(l + h) * n;
            const float2 u0 = suf[l], u1 = suf[l + h];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int j = threadIdx.x + PT * r;
                if (j < n) {
                    float gh, gl;
                    split_d(c0[j], gh, gl);
                    df_fma(ah0[r], al0[r], u0.x, u0.y, gh, gl);
                    split_d(c1[j], gh, gl);
                    df_fma(ah1[r], al1[r], u1.x, u1.y, gh, gl);
                }
            }
        }
        if (n & 1) {
            const double* c = reinterpret_cast<const double*>(G) + (long long)(n - 1) * n;
            const float2 ul = suf[n - 1];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int j = threadIdx.x + PT * r;
                if (j < n) {
                    float gh, gl;
                    split_d(c[j], gh, gl);
                    df_fma(ah0[r], al0[r], ul.x, ul.y, gh, gl);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int j = threadIdx.x + PT * r;
            df_add(ah0[r], al0[r], ah1[r], al1[r]);
            if (j < n) reinterpret_cast<double*>(Xa)[j] = df_to_double(ah0[r], al0[r]);
        }
        return;
    } else {
        T acc0[NR], acc1[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            acc0[r] = s_zero(T());
            acc1[r] = s_zero(T());
        }
#pragma unroll 4
        for (int l = 0; l < h; ++l) {
            const T* c0 = G + (long long)l * n;
            const T* c1 = G + (long long)(l + h) * n;
            const T u0 = su[l], u1 = su[l + h];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int j = threadIdx.x + PT * r;
                if (j < n) {
                    acc0[r] = s_fma(c0[j], u0, acc0[r]);
                    acc1[r] = s_fma(c1[j], u1, acc1[r]);
                }
            }
        }
        if (n & 1) {
            const T* c = G + (long long)(n - 1) * n;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int j = threadIdx.x + PT * r;
                if (j < n) acc0[r] = s_fma(c[j], su[n - 1], acc0[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int j = threadIdx.x + PT * r;
            if (j < n) Xa[j] = acc0[r] + acc1[r];
        }
    }
}

// columns (rows) per CTA of the warp-per-column (row) double-float passes
constexpr int DF_CPB = 64;

// The same pass for an exactly skew A^{-1} (every Pfaffian state: the skew
// accept, the skew flushes and the refresh keep it so), in double-float
// arithmetic: X_j = sum_l (A^{-1})_{jl} u_l = -sum_l (A^{-1})_{lj} u_l, and
// (A^{-1})_{lj} lies at G[j n + l], so row j of the sum is contiguous in
// memory.  One WARP per row j reads it in 16-byte loads (512 contiguous bytes
// per load instruction), with a batch of loads in flight while the previous
// one is multiplied, as in k_accept_delayed_warp_df; the products run on the
// FP32 and integer pipes, so the pass is bound by HBM rather than by the FP64
// pipe.  One CTA (8 warps) per walker and DF_CPB rows.  n even.
template <int NP2>
__global__ void __launch_bounds__(PT, 2) k_dense_column_skew_df(DevLayout L, DevState<double> S, DevOperand U,
                                                                 int a) {
    constexpr int BS = NP2 == 16 ? 4 : (NP2 > 16 ? 8 : NP2 / 2);   // 16-byte loads per lane per batch
    constexpr int NBT = NP2 / BS;                 // batches per row (even)
    __shared__ __align__(16) float4 sU4[32 * NP2];   // (hi u_2p, hi u_2p+1, lo u_2p, lo u_2p+1)
    const int w = blockIdx.x;
    const int n = L.nw(w);
    const int np = n >> 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int j0 = blockIdx.y * DF_CPB;
    if (j0 >= n) return;
    if (!LRU_DEBUG_OK((n & 1) == 0 && np <= 32 * NP2, S.err)) return;
    const int nrow = min(n - j0, DF_CPB);
    const double* ub = vec_ptr<double>(U, L, w, a, n);
    for (int p = threadIdx.x; p < 32 * NP2; p += PT) {
        const double u0 = p < np ? ub[2 * p] : 0.0, u1 = p < np ? ub[2 * p + 1] : 0.0;
        float h0, lo0, h1, lo1;
        split_d(u0, h0, lo0);
        split_d(u1, h1, lo1);
        sU4[p] = make_float4(h0, h1, lo0, lo1);
    }
    __syncthreads();
    const double* Gw = S.G + L.mo(w);
    double* Xa = S.X + L.vo(w) * L.kk + (long long)a * n;
    // this warp's rows j0 + wid + 8 i, as a flat sequence of (row, batch) items
    const int nmine = nrow > wid ? (nrow - wid + 7) / 8 : 0;
    const int T = nmine * NBT;
    auto load = [&](double2 (&buf)[BS], int t) {
        const int c = t / NBT, b = t % NBT;
        const double2* r2 = reinterpret_cast<const double2*>(Gw + (long long)(j0 + wid + 8 * c) * n);
#pragma unroll
        for (int m = 0; m < BS; ++m) {
            const int p = lane + 32 * (b * BS + m);
            buf[m] = p < np ? r2[p] : make_double2(0.0, 0.0);
        }
    };
    float ah0 = 0.f, al0 = 0.f, ah1 = 0.f, al1 = 0.f;
    auto compute = [&](const double2 (&buf)[BS], int t) {
        const int b = t % NBT;
#pragma unroll
        for (int m = 0; m < BS; ++m) {
            const int p = lane + 32 * (b * BS + m);
            float gh, gl;
            const float4 v = sU4[p];
            split_d(buf[m].x, gh, gl);
            df_fma(ah0, al0, v.x, v.z, gh, gl);
            split_d(buf[m].y, gh, gl);
            df_fma(ah1, al1, v.y, v.w, gh, gl);
        }
        if (b == NBT - 1) {
            df_add(ah0, al0, ah1, al1);
            df_warp_sum(ah0, al0);
            if (lane == 0) Xa[j0 + wid + 8 * (t / NBT)] = -df_to_double(ah0, al0);
            ah0 = al0 = ah1 = al1 = 0.f;
        }
    };
    double2 buf0[BS], buf1[BS];
    if (T > 0) load(buf0, 0);
    for (int t = 0; t < T; t += 2) {   // T is even
        load(buf1, t + 1);
        compute(buf0, t);
        if (t + 2 < T) load(buf0, t + 2);
        compute(buf1, t + 1);
    }
}

// the standalone propose: the Pfaffian accept that follows is in skew form
// (plain: k_accept_pf_skew; delayed: the slots), so M is projected
template <typename T, bool PF, bool DELAYED>
__global__ void __launch_bounds__(PT) k_propose(DevLayout L, DevState<T> S, DevOperand U, DevOperand V,
                                                 const T* C, T* ratio_out, int* st_out) {
    propose_walker<T, PF, DELAYED, PF>(blockIdx.x, L, S, U, V, C, ratio_out, st_out);
}

// Q^T U for the dense U columns of the delayed propose, one CTA per walker
// and column: QtU[w][c][a] = sum_j Q[j][c] u_a[j].  Runs before k_propose.
template <typename T>
__global__ void __launch_bounds__(PT) k_qtu_dense(DevLayout L, DevState<T> S, DevOperand U) {
    __shared__ T s_red[8 * 16];
    __shared__ T s_out[16];
    const int w = blockIdx.x, a = blockIdx.y;
    const int n = L.nw(w), kk = L.kv(w);
    if (a >= kk || ((U.mask >> a) & 1u)) return;
    const int Kc = L.Kc, cu = S.tau[w] * kk;
    const long long vo = L.vo(w);
    const T* u = vec_ptr<T>(U, L, w, a, n);
    for (int c0 = 0; c0 < cu; c0 += 16) {
        T part[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) part[q] = s_zero(T());
        for (int j = threadIdx.x; j < n; j += PT) {
            const T* qrow = S.Q + (vo + j) * Kc + c0;
            T uj = u[j];
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (c0 + q < cu) part[q] = s_fma(qrow[q], uj, part[q]);
        }
        block_reduce_vec<T, 16>(part, s_red, s_out);
        if (threadIdx.x < 16 && c0 + threadIdx.x < cu)
            S.QtU[((long long)w * Kc + c0 + threadIdx.x) * MAXKK + a] = s_out[threadIdx.x];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// accept pass: one warp per chunk l (column l of A^{-1})
//   y_b = V_b . chunk_l (dense) or chunk_l[i_b] (one-hot)      [= (V A^{-1})_{bl}]
//   plain  : chunk_l -= X (R^{-1} y)                            (Eq. det_inv; pf:
//            generic Woodbury A^{-1} - X M^{-1} (B^T A^{-1}))
//   delayed: y -= (V P) Q[l,:]^T ; Q[l, tau] = (R^{-1} y)^T     (b_tau equation)
// ---------------------------------------------------------------------------
template <typename T, bool DELAYED, int NPL, int KKS>
__device__ void accept_item(const int4 it, const DevLayout L, const DevState<T> S, const DevOperand V,
                            const uint8_t* mask) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const int w = it.x;
    if (!LRU_DEBUG_OK(w >= 0 && w < L.W, S.err)) return;
    if (mask && !mask[w]) return;
    if (S.pst[w] != 0) return;
    // KKS > 0: the rank is a compile-time constant (register arrays), else runtime
    const int n = L.nw(w), kk = KKS > 0 ? KKS : L.kv(w);
    if (!LRU_DEBUG_OK(it.y >= 0 && it.y <= it.z && it.z <= n, S.err)) return;
    const long long vo = L.vo(w);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // X and the dense V vectors are staged in shared memory when they fit
    // (use_smem), else read from global memory (L2) with the same layout
    T* sXs = reinterpret_cast<T*>(dyn_smem);       // kk x n
    T* sVs = sXs + (size_t)kk * n;                 // kk x n (dense slots)
    const bool use_smem = it.w != 0;
    __shared__ T sR[MAXKK * MAXKK];
    __shared__ int siv[MAXKK];
    __shared__ T sVP[MAXKK * 64];
    const int Kc = L.Kc;
    const int cu = DELAYED ? S.tau[w] * kk : 0;

    const T* Xg = S.X + vo * L.kk;
    const T* sX = Xg;
    const T* sV = (V.dense != nullptr) ? vec_ptr<T>(V, L, w, 0, n) : nullptr;
    if (use_smem) {
        for (int e = threadIdx.x; e < kk * n; e += PT) sXs[e] = Xg[e];
        for (int b = 0; b < kk; ++b) {
            if ((V.mask >> b) & 1u) continue;
            const T* vb = vec_ptr<T>(V, L, w, b, n);
            for (int j = threadIdx.x; j < n; j += PT) sVs[(size_t)b * n + j] = vb[j];
        }
        sX = sXs;
        sV = sVs;
    }
    if (threadIdx.x < kk) siv[threadIdx.x] = ((V.mask >> threadIdx.x) & 1u) ? V.idx[(long long)w * V.slots + threadIdx.x] : -1;
    for (int e = threadIdx.x; e < MAXKK * MAXKK; e += PT) sR[e] = S.Rinv[(long long)w * MAXKK * MAXKK + e];
    if constexpr (DELAYED)
        for (int e = threadIdx.x; e < kk * cu; e += PT) {
            const int b = e / cu, c = e % cu;
            sVP[b * 64 + c] = S.VP[(long long)w * MAXKK * Kc + b * Kc + c];
        }
    __syncthreads();

    T* Gw = S.G + L.mo(w);
    for (int l = it.y + wid; l < it.z; l += PT / 32) {
        T* col = Gw + (long long)l * n;
        T v[NPL];
#pragma unroll
        for (int m = 0; m < NPL; ++m) {
            const int j = lane + 32 * m;
            v[m] = (j < n) ? col[j] : s_zero(T());
        }
        T y[KKS > 0 ? KKS : MAXKK];
#pragma unroll
        for (int b = 0; b < (KKS > 0 ? KKS : kk); ++b) {
            if (siv[b] >= 0) {
                y[b] = col[siv[b]];
            } else {
                const T* vb = sV + (size_t)b * n;
                T part = s_zero(T());
#pragma unroll
                for (int m = 0; m < NPL; ++m) {
                    const int j = lane + 32 * m;
                    if (j < n) part = s_fma(vb[j], v[m], part);
                }
                y[b] = warp_sum(part);
            }
            if constexpr (DELAYED) {
                // lanes split the slot sum (c = lane, lane + 32) and reduce
                const T* qrow = S.Q + (vo + l) * Kc;
                T corr = s_zero(T());
                for (int c = lane; c < cu; c += 32) corr = s_fma(sVP[b * 64 + c], qrow[c], corr);
                y[b] = y[b] - warp_sum(corr);
            }
        }
        T z[KKS > 0 ? KKS : MAXKK];
#pragma unroll
        for (int a = 0; a < (KKS > 0 ? KKS : kk); ++a) {
            T s = s_zero(T());
#pragma unroll
            for (int b = 0; b < (KKS > 0 ? KKS : kk); ++b) s = s_fma(sR[a * MAXKK + b], y[b], s);
            z[a] = s;
        }
        if constexpr (!DELAYED) {
#pragma unroll
            for (int m = 0; m < NPL; ++m) {
                const int j = lane + 32 * m;
                if (j < n) {
                    T d = v[m];
#pragma unroll
                    for (int a = 0; a < (KKS > 0 ? KKS : kk); ++a) d = s_fms(sX[(size_t)a * n + j], z[a], d);
                    col[j] = d;
                }
            }
        } else {
            if (lane < kk) {
                T zz = z[0];
#pragma unroll
                for (int a = 1; a < (KKS > 0 ? KKS : kk); ++a)
                    if (a == lane) zz = z[a];
                const long long off = (vo + l) * Kc + cu + lane;
                S.Q[off] = zz;
                if constexpr (!traits<T>::is_complex && sizeof(T) == 8) {
                    if (S.P32h) store_split(S, 1, (vo + l) * L.Kc32 + cu + lane, (double)zz);
                }
            }
        }
    }
}

template <typename T, bool DELAYED, int NPL, int KKS>
__global__ void __launch_bounds__(PT, 2) k_accept(DevLayout L, DevState<T> S, DevOperand V, const uint8_t* mask,
                                                   const int4* items) {
    accept_item<T, DELAYED, NPL, KKS>(items[blockIdx.x], L, S, V, mask);
}

// Plain Pfaffian accept in skew form (Eq. pf_inv with (A^{-1})^T = -A^{-1}):
//   A'^{-1} = A^{-1} + X M^{-1} X^T,   X = A^{-1} B (from the propose),
// with M^{-1} projected onto its skew part, Z_l = M^{-1} X_l^T per row l.
// The new inverse is exactly skew in exact arithmetic; in floating point the
// two triangles of the update round differently.  One CTA per (walker,
// 32 x 32 upper tile) computes the upper entries j < l and writes the lower
// triangle as their exact negatives and the diagonal as zero, so A^{-1}
// stays exactly skew along the chain, and only the upper half is read.
//   * B with 2 columns (one row-and-column move): U_jl = A^{-1}_jl +
//     sum_a X_ja Z_la, one FMA per element and column.  On the paper's
//     pairing matrices this keeps the accuracy of the skew-part projection
//     (A' + A'^T)/2 of the update (checked against exact ratios).
//   * B with 4 or more columns (two particles at once): a kept triangle
//     carries the rounding of its own FMA chain, which on those chains cost
//     up to 25x the ratio error of the projection.  The kernel therefore also
//     forms U_lj = -A^{-1}_jl + sum_a X_la Z_ja and stores (U_jl - U_lj) / 2,
//     the skew part of the computed update, at twice the FMAs.
template <typename T>
__global__ void __launch_bounds__(256) k_accept_pf_skew(DevLayout L, DevState<T> S, const uint8_t* mask) {
    constexpr int LDX = MAXKK + 1;
    // phase 1: X and Z rows of the tile's j and l ranges; phase 2 (after a
    // barrier): the 32 x 33 result tile, in the same storage
    __shared__ T sbuf[4 * 32 * LDX];
    __shared__ T sMi[MAXKK * MAXKK];
    T* sXj = sbuf;                 // [32][LDX] X rows j0..j0+31
    T* sZl = sbuf + 32 * LDX;      // [32][LDX] Z rows l0..l0+31
    T* sXl = sbuf + 64 * LDX;      // (averaged form) X rows of the l range
    T* sZj = sbuf + 96 * LDX;      // (averaged form) Z rows of the j range
    T* sT = sbuf;                  // [32][33]
    static_assert(32 * 33 <= 4 * 32 * LDX, "result tile fits the operand storage");
    const int w = blockIdx.y;
    if (mask && !mask[w]) return;
    if (S.pst[w] != 0) return;
    const int n = L.nw(w), kk = L.kv(w);
    const int nt = (n + 31) / 32;
    if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
    const bool avg = kk > 2;
    int tJ, tL;
    TileIter::coords((int)blockIdx.x, nt, true, tJ, tL);
    const int j0 = tJ * 32, l0 = tL * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    const T* X = S.X + L.vo(w) * L.kk;                        // kk vectors of n
    const T* Ri = S.Rinv + (long long)w * MAXKK * MAXKK;
    for (int e = threadIdx.x; e < kk * kk; e += 256) {
        const int a = e / kk, b = e % kk;
        sMi[a * MAXKK + b] = s_half(Ri[a * MAXKK + b] - Ri[b * MAXKK + a]);   // skew part
    }
    for (int e = threadIdx.x; e < 32 * kk; e += 256) {
        const int a = e / 32, r = e % 32;
        sXj[r * LDX + a] = (j0 + r < n) ? X[(long long)a * n + j0 + r] : s_zero(T());
        if (avg) sXl[r * LDX + a] = (l0 + r < n) ? X[(long long)a * n + l0 + r] : s_zero(T());
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * kk; e += 256) {
        const int a = e / 32, r = e % 32;
        T z = s_zero(T());
        if (l0 + r < n)
            for (int b = 0; b < kk; ++b) z = s_fma(sMi[a * MAXKK + b], X[(long long)b * n + l0 + r], z);
        sZl[r * LDX + a] = z;
        if (avg) {
            T zj = s_zero(T());
            if (j0 + r < n)
                for (int b = 0; b < kk; ++b) zj = s_fma(sMi[a * MAXKK + b], X[(long long)b * n + j0 + r], zj);
            sZj[r * LDX + a] = zj;
        }
    }
    __syncthreads();
    T* Gw = S.G + L.mo(w);
    const int j = j0 + tx;
    T vals[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int rl = ty + 8 * q, l = l0 + rl;
        T v = s_zero(T());
        if (j < n && l < n && (tJ != tL || tx < rl)) {
            const T g = Gw[(long long)l * n + j];   // (A^{-1})_{jl}, j < l
            v = g;
            for (int a = 0; a < kk; ++a) v = s_fma(sXj[tx * LDX + a], sZl[rl * LDX + a], v);
            if (avg) {
                T u = s_neg(g);                      // (A^{-1})_{lj}, exactly
                for (int a = 0; a < kk; ++a) u = s_fma(sXl[rl * LDX + a], sZj[tx * LDX + a], u);
                v = s_half(v - u);
            }
        }
        vals[q] = v;
    }
    __syncthreads();   // operand rows dead: the storage becomes the result tile
#pragma unroll
    for (int q = 0; q < 4; ++q) sT[(ty + 8 * q) * 33 + tx] = vals[q];
    __syncthreads();
    // (j, l), j < l: the computed value; (l, j): its exact negative; diagonal 0
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int rl = ty + 8 * q, l = l0 + rl;
        if (j >= n || l >= n) continue;
        if (tJ != tL || tx < rl) Gw[(long long)l * n + j] = sT[rl * 33 + tx];
        else if (tx == rl) Gw[(long long)l * n + j] = s_zero(T());
        else Gw[(long long)l * n + j] = s_neg(sT[tx * 33 + rl]);   // diagonal tile, j > l
    }
    if (tJ != tL) {
        // mirror tile: (l, j) for l in the L range, stored at G[j * n + l]
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int rj = ty + 8 * q, jj = j0 + rj, ll = l0 + tx;
            if (jj < n && ll < n) Gw[(long long)jj * n + ll] = s_neg(sT[tx * 33 + rj]);
        }
    }
}

// Delayed accept of a rank-1 update, GEMV in the handle dtype with one THREAD
// per column l of A_0^{-1}: the thread streams its contiguous column in
// 16-byte loads against V (shared memory, broadcast), so the dot product
// needs no cross-lane reduction and costs one FMA per element; it then
// subtracts its own (V P) Q[l,:]^T correction and writes Q[l, tau] = y / r
// (b_tau equation of Sec. 2.3).  One CTA per (walker, PT columns).
template <typename T>
__global__ void __launch_bounds__(PT, 2) k_accept_delayed_lane(DevLayout L, DevState<T> S, DevOperand V,
                                                                const uint8_t* mask) {
    __shared__ __align__(16) T sV[2048];
    __shared__ T sVP[64];
    const int w = blockIdx.x;
    if (mask && !mask[w]) return;
    if (S.pst[w] != 0) return;
    const int n = L.nw(w);
    const long long vo = L.vo(w);
    const int Kc = L.Kc, cu = S.tau[w];
    const T* vb = vec_ptr<T>(V, L, w, 0, n);
    for (int j = threadIdx.x; j < n; j += PT) sV[j] = vb[j];
    for (int c = threadIdx.x; c < cu; c += PT) sVP[c] = S.VP[(long long)w * MAXKK * Kc + c];
    const T rinv = S.Rinv[(long long)w * MAXKK * MAXKK];
    __syncthreads();
    const int l = blockIdx.y * PT + threadIdx.x;
    if (l >= n) return;
    const T* __restrict__ col = S.G + L.mo(w) + (long long)l * n;
    T acc0 = s_zero(T()), acc1 = s_zero(T());
    if constexpr (std::is_same<T, double>::value) {
        const double2* __restrict__ c2 = reinterpret_cast<const double2*>(col);
        const double2* v2 = reinterpret_cast<const double2*>(sV);
        const int np = n >> 1;
        int p = 0;
        for (; p + 4 <= np; p += 4) {
            const double2 g0 = c2[p], g1 = c2[p + 1], g2 = c2[p + 2], g3 = c2[p + 3];
            const double2 v0 = v2[p], v1 = v2[p + 1], vv2 = v2[p + 2], v3 = v2[p + 3];
            acc0 = fma(v0.x, g0.x, acc0); acc1 = fma(v0.y, g0.y, acc1);
            acc0 = fma(v1.x, g1.x, acc0); acc1 = fma(v1.y, g1.y, acc1);
            acc0 = fma(vv2.x, g2.x, acc0); acc1 = fma(vv2.y, g2.y, acc1);
            acc0 = fma(v3.x, g3.x, acc0); acc1 = fma(v3.y, g3.y, acc1);
        }
        for (; p < np; ++p) {
            const double2 g = c2[p], v = v2[p];
            acc0 = fma(v.x, g.x, acc0);
            acc1 = fma(v.y, g.y, acc1);
        }
        if (n & 1) acc0 = fma(sV[n - 1], col[n - 1], acc0);
    } else {
        int j = 0;
        for (; j + 4 <= n; j += 4) {
            const T g0 = col[j], g1 = col[j + 1], g2 = col[j + 2], g3 = col[j + 3];
            acc0 = s_fma(sV[j], g0, acc0);
            acc1 = s_fma(sV[j + 1], g1, acc1);
            acc0 = s_fma(sV[j + 2], g2, acc0);
            acc1 = s_fma(sV[j + 3], g3, acc1);
        }
        for (; j < n; ++j) acc0 = s_fma(sV[j], col[j], acc0);
    }
    T y = acc0 + acc1;
    const T* qrow = S.Q + (vo + l) * Kc;
    for (int c = 0; c < cu; ++c) y = s_fms(sVP[c], qrow[c], y);
    const T z = s_fma(rinv, y, s_zero(T()));
    S.Q[(vo + l) * Kc + cu] = z;
    if constexpr (!traits<T>::is_complex && sizeof(T) == 8) {
        if (S.P32h) store_split(S, 1, (vo + l) * L.Kc32 + cu, (double)z);
    }
}

// Delayed accept of a real rank-1 update (b_tau equation of Sec. 2.3) with
// the GEMV products taken off the FP64 pipe: one WARP per column l of
// A_0^{-1}, so every load instruction reads 512 contiguous bytes (a thread
// per column touches 32 cache lines per load, and the L1 lookups then bind
// near 1.7 ms per pass at 1024 walkers, n = 1024).  Lane t holds the element
// pairs p = t + 32 m of the column, in batches of BS 16-byte loads; the loads
// of the next batch (of this column or the next) are issued before the
// current batch is multiplied, so each warp keeps a batch in flight while it
// computes.  Each element is split into hi + lo floats with integer
// operations and multiplied into a double-float accumulator against the
// split of V (shared memory), so a product costs FP32-pipe and integer
// instructions only.  FP64 work per column (the slot correction
// (V P) Q[l,:]^T, the conversion of the double-float sum, z = y / r) is done
// once per CTA by one thread per column: a warp-wide FP64 instruction
// occupies the FP64 pipe for many cycles even with one lane active.  One CTA
// (8 warps) per walker and DF_CPB columns.

template <int NP2>
__global__ void __launch_bounds__(PT, 2) k_accept_delayed_warp_df(DevLayout L, DevState<double> S, DevOperand V,
                                                                   const uint8_t* mask) {
    constexpr int BS = NP2 >= 16 ? 8 : NP2 / 2;   // 16-byte loads per lane per batch
    constexpr int NBT = NP2 / BS;                 // batches per column (even)
    __shared__ __align__(16) float4 sV4[32 * NP2];   // (hi v_2p, hi v_2p+1, lo v_2p, lo v_2p+1)
    __shared__ double sVP[64];
    __shared__ double sCorr[DF_CPB];
    __shared__ float2 sY[DF_CPB];
    const int w = blockIdx.x;
    if (mask && !mask[w]) return;
    if (S.pst[w] != 0) return;
    const int n = L.nw(w);
    const long long vo = L.vo(w);
    const int Kc = L.Kc, cu = S.tau[w];
    const int np = n >> 1;   // n is even
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int l0 = blockIdx.y * DF_CPB;
    if (!LRU_DEBUG_OK((n & 1) == 0 && np <= 32 * NP2 && l0 < n && cu < Kc, S.err)) return;
    const int ncol = min(n - l0, DF_CPB);
    const double* vb = vec_ptr<double>(V, L, w, 0, n);
    for (int p = threadIdx.x; p < 32 * NP2; p += PT) {
        const double v0 = p < np ? vb[2 * p] : 0.0, v1 = p < np ? vb[2 * p + 1] : 0.0;
        float h0, lo0, h1, lo1;
        split_d(v0, h0, lo0);
        split_d(v1, h1, lo1);
        sV4[p] = make_float4(h0, h1, lo0, lo1);
    }
    for (int c = threadIdx.x; c < cu; c += PT) sVP[c] = S.VP[(long long)w * MAXKK * Kc + c];
    __syncthreads();
    if (threadIdx.x < ncol) {
        // slot correction of column l0 + t: (V P) Q[l,:]^T, in FP64
        const double* qrow = S.Q + (vo + l0 + threadIdx.x) * Kc;
        double c = 0.0;
        for (int t = 0; t < cu; ++t) c = fma(sVP[t], qrow[t], c);
        sCorr[threadIdx.x] = c;
    }
    const double* Gw = S.G + L.mo(w);
    // this warp's columns l0 + wid + 8 i, as a flat sequence of (column, batch) items
    const int nmine = ncol > wid ? (ncol - wid + 7) / 8 : 0;
    const int T = nmine * NBT;
    auto load = [&](double2 (&buf)[BS], int t) {
        const int c = t / NBT, b = t % NBT;
        const double2* c2 = reinterpret_cast<const double2*>(Gw + (long long)(l0 + wid + 8 * c) * n);
#pragma unroll
        for (int m = 0; m < BS; ++m) {
            const int p = lane + 32 * (b * BS + m);
            buf[m] = p < np ? c2[p] : make_double2(0.0, 0.0);
        }
    };
    float ah0 = 0.f, al0 = 0.f, ah1 = 0.f, al1 = 0.f;
    auto compute = [&](const double2 (&buf)[BS], int t) {
        const int b = t % NBT;
#pragma unroll
        for (int m = 0; m < BS; ++m) {
            const int p = lane + 32 * (b * BS + m);
            float gh, gl;
            const float4 v = sV4[p];
            split_d(buf[m].x, gh, gl);
            df_fma(ah0, al0, v.x, v.z, gh, gl);
            split_d(buf[m].y, gh, gl);
            df_fma(ah1, al1, v.y, v.w, gh, gl);
        }
        if (b == NBT - 1) {
            // column done: warp sum, kept as a float pair until the epilogue
            df_add(ah0, al0, ah1, al1);
            df_warp_sum(ah0, al0);
            if (lane == 0) sY[wid + 8 * (t / NBT)] = make_float2(ah0, al0);
            ah0 = al0 = ah1 = al1 = 0.f;
        }
    };
    double2 buf0[BS], buf1[BS];
    if (T > 0) load(buf0, 0);
    for (int t = 0; t < T; t += 2) {   // T is even
        load(buf1, t + 1);
        compute(buf0, t);
        if (t + 2 < T) load(buf0, t + 2);
        compute(buf1, t + 1);
    }
    __syncthreads();
    if (threadIdx.x < ncol) {
        const int l = l0 + threadIdx.x;
        const float2 y2 = sY[threadIdx.x];
        const double z = S.Rinv[(long long)w * MAXKK * MAXKK] * (df_to_double(y2.x, y2.y) - sCorr[threadIdx.x]);
        S.Q[(vo + l) * Kc + cu] = z;
        if (S.P32h) store_split(S, 1, (vo + l) * L.Kc32 + cu, z);
    }
}

// Delayed accept of a real rank-1 update with the GEMV in double-float
// arithmetic (FP32 pipe): per chunk l, y = V . chunk_l accumulated as hi+lo
// floats from integer-split doubles, then in FP64 y -= (V P) Q[l,:]^T and
// Q[l, tau] = y / r (b_tau equation of Sec. 2.3).  Reads A_0^{-1} once, in
// 16-byte loads, eight at a time per lane with two independent accumulators;
// the per-chunk FP64 corrections (V P) Q[l,:]^T are formed by 64 threads in
// the prologue.  NP2 = double2 loads per lane per chunk (n <= 64 NP2).
template <int NP2>
__global__ void __launch_bounds__(PT, 3) k_accept_delayed_df(DevLayout L, DevState<double> S, DevOperand V,
                                                              const uint8_t* mask, const int4* items) {
    __shared__ float2 sVh[1024], sVl[1024];   // V split, as pairs matching the double2 loads
    __shared__ double sCorr[256];
    const int4 it = items[blockIdx.x];
    const int w = it.x;
    if (mask && !mask[w]) return;
    if (S.pst[w] != 0) return;
    const int n = L.nw(w);
    const long long vo = L.vo(w);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int Kc = L.Kc, cu = S.tau[w];
    const double* vb = vec_ptr<double>(V, L, w, 0, n);
    for (int p = threadIdx.x; p < (n + 1) / 2; p += PT) {
        const double v0 = vb[2 * p], v1 = (2 * p + 1 < n) ? vb[2 * p + 1] : 0.0;
        float h0, l0, h1, l1;
        split_d(v0, h0, l0);
        split_d(v1, h1, l1);
        sVh[p] = make_float2(h0, h1);
        sVl[p] = make_float2(l0, l1);
    }
    // corrections of the chunks of this item: corr_l = sum_c (V P)_c Q[l][c]
    const double* VP = S.VP + (long long)w * MAXKK * Kc;
    for (int l = it.y + threadIdx.x; l < it.z; l += PT) {
        const double* qrow = S.Q + (vo + l) * Kc;
        double c = 0.0;
        for (int t = 0; t < cu; ++t) c = fma(VP[t], qrow[t], c);
        sCorr[l - it.y] = c;
    }
    const double rinv = S.Rinv[(long long)w * MAXKK * MAXKK];
    __syncthreads();
    const double* Gw = S.G + L.mo(w);
    const bool even = ((n & 1) == 0) && ((L.mo(w) & 1) == 0);   // 16-byte aligned chunks
    for (int l = it.y + wid; l < it.z; l += PT / 32) {
        const double* col = Gw + (long long)l * n;
        float ah0 = 0.f, al0 = 0.f, ah1 = 0.f, al1 = 0.f;
        if (even) {
            const double2* col2 = reinterpret_cast<const double2*>(col);
#pragma unroll
            for (int m0 = 0; m0 < NP2; m0 += 8) {
                double2 g[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int p = lane + 32 * (m0 + m);
                    g[m] = (m0 + m < NP2 && 2 * p < n) ? col2[p] : make_double2(0.0, 0.0);
                }
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int p = lane + 32 * (m0 + m);
                    if (m0 + m < NP2 && 2 * p < n) {
                        const float2 vh = sVh[p], vl = sVl[p];
                        float gh, gl;
                        split_d(g[m].x, gh, gl);
                        df_fma(ah0, al0, vh.x, vl.x, gh, gl);
                        split_d(g[m].y, gh, gl);
                        df_fma(ah1, al1, vh.y, vl.y, gh, gl);
                    }
                }
            }
        } else {
            for (int j = lane; j < n; j += 32) {
                float gh, gl;
                split_d(col[j], gh, gl);
                const float2 vh = sVh[j >> 1], vl = sVl[j >> 1];
                df_fma(ah0, al0, (j & 1) ? vh.y : vh.x, (j & 1) ? vl.y : vl.x, gh, gl);
            }
        }
        df_add(ah0, al0, ah1, al1);
        df_warp_sum(ah0, al0);
        if (lane == 0) {
            const double y = df_to_double(ah0, al0) - sCorr[l - it.y];
            const double z = rinv * y;
            S.Q[(vo + l) * Kc + cu] = z;
            if (S.P32h) store_split(S, 1, (vo + l) * L.Kc32 + cu, z);
        }
    }
}

#if !defined(LRU_INST_DTYPE) || defined(LRU_INST_PRIMARY)
// Double-float flush: A_0^{-1} -/+= P Q^T with the Kc-term dot products in
// hi+lo float arithmetic (relative error ~1e-14, FP32 pipe) and one FP64
// subtraction per element.  Same tiling and skew mirror as k_flush_native.
struct DfFlushSmem {
    float sPh[32][65], sPl[32][65], sQh[32][65], sQl[32][65];
    double sT[32][33];
};

template <bool PF>
__device__ void flush_df_tile(const DevLayout& L, const DevState<double>& S, int w, int tau, int tJ, int tL,
                              DfFlushSmem& sm) {
    auto& sPh = sm.sPh;
    auto& sPl = sm.sPl;
    auto& sQh = sm.sQh;
    auto& sQl = sm.sQl;
    auto& sT = sm.sT;
    const int n = L.nw(w), kk = L.kv(w);
    const int cu = tau * kk, Kc = L.Kc;
    const long long vo = L.vo(w);
    double* Gw = S.G + L.mo(w);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int j0 = tJ * 32, l0 = tL * 32;
    for (int e = threadIdx.x; e < 32 * cu; e += 256) {
        const int r = e / cu, c = e % cu;
        double p = (j0 + r < n) ? S.P[(vo + j0 + r) * Kc + c] : 0.0;
        double q = (l0 + r < n) ? S.Q[(vo + l0 + r) * Kc + c] : 0.0;
        split_d(p, sPh[r][c], sPl[r][c]);
        split_d(q, sQh[r][c], sQl[r][c]);
    }
    __syncthreads();
    float ah[4], al[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { ah[q] = 0.f; al[q] = 0.f; }
    for (int c = 0; c < cu; ++c) {
        const float ph = sPh[tx][c], pl = sPl[tx][c];
#pragma unroll
        for (int q = 0; q < 4; ++q) df_fma(ah[q], al[q], ph, pl, sQh[ty + 8 * q][c], sQl[ty + 8 * q][c]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + tx, l = l0 + ty + 8 * q;
        double nv = 0.0;
        if (j < n && l < n) {
            const double g = Gw[(long long)l * n + j];
            const double dh = f2d_int(ah[q]), dl = f2d_int(al[q]);
            nv = PF ? (g + dh) + dl : (g - dh) - dl;
        }
        sT[ty + 8 * q][tx] = nv;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + tx, l = l0 + ty + 8 * q;
        if (j >= n || l >= n) continue;
        if (!PF) {
            Gw[(long long)l * n + j] = sT[ty + 8 * q][tx];
        } else {
            double v;
            if (j < l) v = sT[ty + 8 * q][tx];
            else if (j == l) v = 0.0;
            else v = -sT[tx][ty + 8 * q];
            Gw[(long long)l * n + j] = v;
        }
    }
    if (PF && tJ != tL) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = l0 + tx, j = j0 + ty + 8 * q;
            if (j < n && l < n) Gw[(long long)j * n + l] = -sT[tx][ty + 8 * q];
        }
    }
    __syncthreads();
}

template <bool PF>
__global__ void __launch_bounds__(256) k_flush_df(DevLayout L, DevState<double> S, const uint8_t* force) {
    __shared__ DfFlushSmem sm;
    __shared__ int s_tau[FLUSH_SCAN];
    TileIter ti;
    for (int w0 = 0; w0 < L.W; w0 += FLUSH_SCAN) {
        const int wn = flush_scan(L, S, force, w0, s_tau);
        for (int i = 0; i < wn; ++i) {
            const int tau = s_tau[i];
            if (tau < 0) continue;
            const int w = w0 + i;
            const int nt = (L.nw(w) + 31) / 32;
            const int ntl = TileIter::tiles(nt, PF);
            for (int t = ti.first(ntl); t < ntl; t += gridDim.x) {
                int tJ, tL;
                TileIter::coords(t, nt, PF, tJ, tL);
                flush_df_tile<PF>(L, S, w, tau, tJ, tL, sm);
            }
        }
    }
}

#endif

// After the accept pass: log|value| += log|r|, sign *= r/|r|, tau += 1 (delayed)
template <typename T>
__global__ void k_commit(DevLayout L, DevState<T> S, const uint8_t* mask, bool delayed) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= L.W) return;
    if (mask && !mask[w]) return;
    if (S.pst[w] != 0) return;
    T r = S.ratio[w];
    S.logabs[w] += log(s_absd(r));
    S.sgn[w] = s_renorm(S.sgn[w] * s_unit(r));
    if (delayed) S.tau[w] += 1;
    S.pst[w] = 4;  // proposal consumed: a second accept of it is a no-op
}

// ---------------------------------------------------------------------------
// native flush: A_0^{-1} -= P Q^T (det, Eq. delayed_Ainv) or += (pf, Eq.
// pf_delayed_Ainv) over the filled slots.  32 x 32 tiles; for the Pfaffian only
// tiles with J <= L are computed and the mirror is written as the exact
// negative transpose, so A_0^{-1} stays exactly skew (for B of 4 or more
// columns the kept value is the skew part of the update, see below).
// ---------------------------------------------------------------------------
template <typename T, bool PF, int CH = 64>
__device__ void flush_native_tile(const DevLayout& L, const DevState<T>& S, int w, int tau, int tJ, int tL,
                                  T* sP, T* sQ, T* sT) {
    // sP, sQ: 32 x (CH + 1) slot chunks; sT: 32 x 33 result tile
    constexpr int LD = CH + 1;
    const int n = L.nw(w), kk = L.kv(w);
    const int cu = tau * kk, Kc = L.Kc;
    if (!LRU_DEBUG_OK(tJ >= 0 && tL >= 0 && 32 * tJ < n && 32 * tL < n && cu <= Kc, S.err)) return;
    const long long vo = L.vo(w);
    T* Gw = S.G + L.mo(w);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int j0 = tJ * 32, l0 = tL * 32;
    // Pfaffian with B of 4 or more columns (two-particle moves): the update
    // P Q^T is skew in exact arithmetic, and a kept triangle would carry the
    // rounding of its own FMA chain; the tile then also forms (P Q^T)_lj in a
    // second pass over the slots and adds the skew part (D_jl - D_lj) / 2, as
    // the plain skew accept does (one-particle moves measure the same either way).
    const bool avg = PF && kk > 2;
    T acc[4], acc2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = acc2[q] = s_zero(T());
    for (int pass = 0; pass < (avg ? 2 : 1); ++pass) {
        // pass 0: P rows of the j range against Q rows of the l range; pass 1: swapped
        const T* Pa = pass ? S.Q : S.P;
        const T* Qa = pass ? S.P : S.Q;
        for (int c0 = 0; c0 < cu; c0 += CH) {
            for (int e = threadIdx.x; e < 32 * CH; e += 256) {
                const int r = e / CH, c = e % CH;
                const bool okc = c0 + c < cu;
                sP[r * LD + c] = (okc && j0 + r < n) ? Pa[(vo + j0 + r) * Kc + c0 + c] : s_zero(T());
                sQ[r * LD + c] = (okc && l0 + r < n) ? Qa[(vo + l0 + r) * Kc + c0 + c] : s_zero(T());
            }
            __syncthreads();
            const int cm = min(CH, cu - c0);
            for (int c = 0; c < cm; ++c) {
                T pj = sP[tx * LD + c];
                if (pass == 0) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] = s_fma(pj, sQ[(ty + 8 * q) * LD + c], acc[q]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc2[q] = s_fma(pj, sQ[(ty + 8 * q) * LD + c], acc2[q]);
                }
            }
            __syncthreads();
        }
    }
    // element (j0+tx, l0+ty+8q) lives at G[(l0+ty+8q)*n + j0+tx]
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + tx, l = l0 + ty + 8 * q;
        T nv = s_zero(T());
        if (j < n && l < n) {
            T g = Gw[(long long)l * n + j];
            // acc2[q] = (Q P^T)_jl = (P Q^T)_lj
            const T d = avg ? s_half(acc[q] - acc2[q]) : acc[q];
            nv = PF ? (g + d) : (g - d);
        }
        sT[(ty + 8 * q) * 33 + tx] = nv;
    }
    __syncthreads();
    if (!PF) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + tx, l = l0 + ty + 8 * q;
            if (j < n && l < n) Gw[(long long)l * n + j] = sT[(ty + 8 * q) * 33 + tx];
        }
    } else {
        // upper entries (j < l) are kept, lower ones written as their negatives
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + tx, l = l0 + ty + 8 * q;
            if (j < n && l < n) {
                T v;
                if (j < l) v = sT[(ty + 8 * q) * 33 + tx];
                else if (j == l) v = s_zero(T());
                else v = s_neg(sT[tx * 33 + ty + 8 * q]);  // same tile (diagonal tiles only)
                Gw[(long long)l * n + j] = v;
            }
        }
        if (tJ != tL) {
            // mirror tile: (l, j) = -(j, l), stored at G[j*n + l]
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int l = l0 + tx, j = j0 + ty + 8 * q;
                if (j < n && l < n) Gw[(long long)j * n + l] = s_neg(sT[tx * 33 + ty + 8 * q]);
            }
        }
    }
    __syncthreads();
}

template <typename T, bool PF>
__global__ void __launch_bounds__(256) k_flush_native(DevLayout L, DevState<T> S, const uint8_t* force) {
    __shared__ T sP[32][65];
    __shared__ T sQ[32][65];
    __shared__ T sT[32][33];
    __shared__ int s_tau[FLUSH_SCAN];
    TileIter ti;
    for (int w0 = 0; w0 < L.W; w0 += FLUSH_SCAN) {
        const int wn = flush_scan(L, S, force, w0, s_tau);
        for (int i = 0; i < wn; ++i) {
            const int tau = s_tau[i];
            if (tau < 0) continue;
            const int w = w0 + i;
            const int nt = (L.nw(w) + 31) / 32;
            const int ntl = TileIter::tiles(nt, PF);
            for (int t = ti.first(ntl); t < ntl; t += gridDim.x) {
                int tJ, tL;
                TileIter::coords(t, nt, PF, tJ, tL);
                flush_native_tile<T, PF>(L, S, w, tau, tJ, tL, &sP[0][0], &sQ[0][0], &sT[0][0]);
            }
        }
    }
}

// Bounded waits of the persistent step (and of its self-test).
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Spins (acquire loads, 64 ns naps) until *flag == want or `iters` polls have
// failed; on giving up it records DEV_ERR_TIMEOUT in the sticky device error
// and returns false, so the caller skips the dependent work and returns.
__device__ __forceinline__ bool bounded_acquire_wait(const int* flag, int want, long long iters, int* err) {
    for (long long i = 0; i < iters; ++i) {
        if (ld_acquire_gpu(flag) == want) return true;
        __nanosleep(64);
    }
    set_dev_error(err, DEV_ERR_TIMEOUT);
    return false;
}
constexpr long long STEP_WAIT_POLLS = 1ll << 24;   // >= 1 s of polling

#if !defined(LRU_NO_STEP)
// ---------------------------------------------------------------------------
// Persistent fused step for walkers of uneven n and k: one launch of a fixed
// grid that pulls work from a device queue,
//   items [0, W)                  : propose walker order[i] (largest n^2 k
//                                   first), then the accept decision (mask,
//                                   or Metropolis |r|^2 >= u)
//   items [W, W + nacc)           : accept items (walker, chunk range),
//                                   largest first; the last one of a walker
//                                   commits log|value|, the sign (and, in the
//                                   delayed form, tau += 1)
//   items [W + nacc, + nflush)    : delayed form only: flush strips (walker,
//                                   32 columns of A_0^{-1}); a strip waits for
//                                   its walker's commit and, if tau reached K,
//                                   folds the slots in (Eq. delayed_Ainv /
//                                   pf_delayed_Ainv, FP64 tiles); the last
//                                   strip of a walker resets tau.
// Every wait (bounded, acquire) is on an item dequeued earlier, so its
// producer is already running.  The delayed Pfaffian propose writes both
// slots itself, so it has no accept items and commits in the propose item.
// Counters and flags are cleared by a memset in the same stream before the
// launch, so the pair can be captured in a CUDA graph and replayed.
// ---------------------------------------------------------------------------

// log|value| += log|r|, sign *= r / |r|, tau += 1 (delayed); proposal consumed
template <typename T>
__device__ __forceinline__ void commit_walker(const DevState<T>& S, int w, bool delayed) {
    const T r = S.ratio[w];
    S.logabs[w] += log(s_absd(r));
    S.sgn[w] = s_renorm(S.sgn[w] * s_unit(r));
    if (delayed) S.tau[w] += 1;
    S.pst[w] = 4;
}

// Q^T u_a of the dense columns a of U (the (b_t^T U) / (B^T a_t) factors of
// the delayed propose) for walker w, by the whole CTA (k_qtu_dense in one block)
template <typename T>
__device__ void qtu_block(int w, const DevLayout& L, const DevState<T>& S, const DevOperand& U) {
    __shared__ T s_red[8 * 16];
    __shared__ T s_out[16];
    const int n = L.nw(w), kk = L.kv(w);
    const int Kc = L.Kc, cu = S.tau[w] * kk;
    const long long vo = L.vo(w);
    for (int a = 0; a < kk; ++a) {
        if ((U.mask >> a) & 1u) continue;
        const T* u = vec_ptr<T>(U, L, w, a, n);
        for (int c0 = 0; c0 < cu; c0 += 16) {
            T part[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) part[q] = s_zero(T());
            for (int j = threadIdx.x; j < n; j += PT) {
                const T* qrow = S.Q + (vo + j) * Kc + c0;
                const T uj = u[j];
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (c0 + q < cu) part[q] = s_fma(qrow[q], uj, part[q]);
            }
            block_reduce_vec<T, 16>(part, s_red, s_out);
            if (threadIdx.x < 16 && c0 + threadIdx.x < cu)
                S.QtU[((long long)w * Kc + c0 + threadIdx.x) * MAXKK + a] = s_out[threadIdx.x];
            __syncthreads();
        }
    }
    __syncthreads();
}

constexpr int STEP_FLUSH_CH = 16;   // slot columns per chunk of a flush tile inside the step
template <typename T>
constexpr size_t step_flush_smem() {
    return (size_t)(2 * 32 * (STEP_FLUSH_CH + 1) + 32 * 33) * sizeof(T);
}

template <typename T, bool PF, bool DEL, int NPL, int KKS>
__global__ void __launch_bounds__(PT) k_step(DevLayout L, DevState<T> S, DevOperand U, DevOperand V, const T* C,
                                              T* ratio_out, int* st_out, StepCtl ctl) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    __shared__ int s_item, s_ok, s_tau;
    const int nacc = (ctl.do_accept && !(PF && DEL)) ? ctl.nacc : 0;
    const int nfl = (ctl.do_accept && DEL) ? ctl.nflush : 0;
    const int total = L.W + nacc + nfl;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(ctl.counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= total) break;
        if (item < L.W) {
            const int w = ctl.order[item];
            if (!LRU_DEBUG_OK(w >= 0 && w < L.W, S.err)) continue;
            if constexpr (DEL) qtu_block<T>(w, L, S, U);
            propose_walker<T, PF, DEL, DEL>(w, L, S, U, V, C, ratio_out, st_out);
            __syncthreads();
            if (threadIdx.x == 0) {
                bool acc = ctl.do_accept && S.pst[w] == 0;
                if (acc && ctl.mask) acc = ctl.mask[w] != 0;
                if (acc && ctl.u) acc = (double)s_abs2(S.ratio[w]) >= ctl.u[w];
                ctl.acc[w] = acc ? 1 : 0;
                if (PF && DEL) {
                    // the slots are already written: commit here
                    if (acc) commit_walker(S, w, true);
                    __threadfence();
                    st_release_gpu(&ctl.fin[w], 1);
                }
                __threadfence();
                st_release_gpu(&ctl.prop_done[w], 1);
            }
        } else if (item < L.W + nacc) {
            const int4 it = ctl.acc_items[item - L.W];
            const int w = it.x;
            if (threadIdx.x == 0) s_ok = bounded_acquire_wait(&ctl.prop_done[w], 1, STEP_WAIT_POLLS, S.err) ? 1 : 0;
            __syncthreads();
            if (s_ok && ctl.acc[w]) accept_item<T, DEL, NPL, KKS>(it, L, S, V, nullptr);
            __syncthreads();
            if (threadIdx.x == 0 && s_ok) {
                __threadfence();
                const int done = atomicAdd(&ctl.items_done[w], 1) + 1;
                if (done == ctl.nacc_w[w]) {
                    if (ctl.acc[w]) commit_walker(S, w, DEL);
                    __threadfence();
                    st_release_gpu(&ctl.fin[w], 1);
                }
            }
        } else {
            const int2 fi = ctl.flush_items[item - L.W - nacc];
            const int w = fi.x, tL = fi.y;
            if (!LRU_DEBUG_OK(w >= 0 && w < L.W && tL >= 0 && 32 * tL < L.nw(w), S.err)) continue;
            if (threadIdx.x == 0) {
                s_ok = bounded_acquire_wait(&ctl.fin[w], 1, STEP_WAIT_POLLS, S.err) ? 1 : 0;
                s_tau = s_ok ? *(volatile const int*)&S.tau[w] : 0;
            }
            __syncthreads();
            const int tau = s_tau;
            if (s_ok && tau >= L.K) {
                T* sP = reinterpret_cast<T*>(dyn_smem);
                T* sQ = sP + 32 * (STEP_FLUSH_CH + 1);
                T* sT = sQ + 32 * (STEP_FLUSH_CH + 1);
                const int nt = (L.nw(w) + 31) / 32;
                const int tJ_end = PF ? tL + 1 : nt;
                for (int tJ = 0; tJ < tJ_end; ++tJ)
                    flush_native_tile<T, PF, STEP_FLUSH_CH>(L, S, w, tau, tJ, tL, sP, sQ, sT);
            }
            __syncthreads();
            if (threadIdx.x == 0 && s_ok) {
                __threadfence();
                const int done = atomicAdd(&ctl.flush_done[w], 1) + 1;
                if (done == ctl.nflush_w[w] && tau >= L.K) S.tau[w] = 0;
            }
        }
    }
}

template <typename T>
void launch_step(bool pf, bool delayed, const DevLayout& L, const DevState<T>& S, const DevOperand& U,
                 const DevOperand& V, const T* C, T* ratio_out, int* st_out, const StepCtl& ctl, int grid,
                 cudaStream_t st) {
    const int nmax = L.n_max;
    int npl = 1;
    while (32 * npl < nmax) npl *= 2;
    size_t dyn = (size_t)2 * L.kk * nmax * sizeof(T);
    if (dyn > 160 * 1024) dyn = 0;   // accept items then carry use_smem = 0
    if (delayed) {
        dyn = std::max(dyn, (size_t)L.Kc * MAXKK * sizeof(T));   // Q^T U in the propose
        dyn = std::max(dyn, step_flush_smem<T>());
    }
    const bool rank1 = L.kk == 1 && L.kvec == nullptr;
#define LRU_STEP_K(PFV, DELV, N)                                                                          \
    {                                                                                                     \
        auto k = rank1 ? k_step<T, PFV, DELV, N, 1> : k_step<T, PFV, DELV, N, 0>;                         \
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);                 \
        k<<<grid, PT, dyn, st>>>(L, S, U, V, C, ratio_out, st_out, ctl);                                  \
    }
#define LRU_STEP(N)                                                                                       \
    case N:                                                                                               \
        if (pf) {                                                                                         \
            if (delayed) LRU_STEP_K(true, true, N) else LRU_STEP_K(true, false, N)                        \
        } else {                                                                                          \
            if (delayed) LRU_STEP_K(false, true, N) else LRU_STEP_K(false, false, N)                      \
        }                                                                                                 \
        break;
    switch (npl) { LRU_STEP(1) LRU_STEP(2) LRU_STEP(4) LRU_STEP(8) LRU_STEP(16) LRU_STEP(32) LRU_STEP(64) default: break; }
#undef LRU_STEP
#undef LRU_STEP_K
}
#endif  // !LRU_NO_STEP

template <typename T>
__global__ void k_flush_finish(DevLayout L, DevState<T> S, const uint8_t* force) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= L.W) return;
    const int tau = S.tau[w];
    const bool go = force ? (force[w] && tau > 0) : (tau >= L.K);
    if (go) S.tau[w] = 0;
}

// forced partial flush with the tensor cores: the MMA runs over all Kc slot
// columns, so the unfilled ones (>= tau * k) must hold zeros in the P split
template <typename T>
__global__ void k_zero_split_tail(DevLayout L, DevState<T> S, const uint8_t* force) {
    const int w = blockIdx.y;
    if (!force || !force[w]) return;
    const int cu = S.tau[w] * L.kv(w);
    if (cu <= 0 || cu >= L.Kc) return;
    const int n = L.nw(w);
    const long long vo = L.vo(w);
    const int width = L.Kc - cu;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * width;
         e += (long long)gridDim.x * blockDim.x) {
        const long long off = (vo + e / width) * L.Kc32 + cu + e % width;
        if (S.split_bf16) {
            reinterpret_cast<__nv_bfloat16*>(S.P32h)[off] = __float2bfloat16_rn(0.f);
            reinterpret_cast<__nv_bfloat16*>(S.P32l)[off] = __float2bfloat16_rn(0.f);
        } else {
            S.P32h[off] = 0.f;
            S.P32l[off] = 0.f;
        }
    }
}

template <typename T>
void launch_zero_split_tail(const DevLayout& L, const DevState<T>& S, const uint8_t* force, cudaStream_t st) {
    k_zero_split_tail<T><<<dim3(16, L.W), 256, 0, st>>>(L, S, force);
}

template <typename T>
__global__ void k_set_delay_zero(DevLayout L, DevState<T> S) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < L.W) S.tau[w] = 0;
}

// current A^{-1} (row-major out) = A_0^{-1} -/+ P Q^T, 32 x 32 tiles
template <typename T, bool PF, bool DELAYED>
__global__ void __launch_bounds__(256) k_get_inverse(DevLayout L, DevState<T> S, T* out) {
    __shared__ T sT[32][33];
    const int w = blockIdx.z;
    const int n = L.nw(w), kk = L.kv(w);
    const int nt = (n + 31) / 32;
    if ((int)blockIdx.x >= nt || (int)blockIdx.y >= nt) return;
    const int j0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const T* Gw = S.G + L.mo(w);
    const long long vo = L.vo(w);
    const int cu = DELAYED ? S.tau[w] * kk : 0;
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + tx, l = l0 + ty + 8 * q;
        T v = s_zero(T());
        if (j < n && l < n) {
            v = Gw[(long long)l * n + j];
            if (DELAYED) {
                const T* pr = S.P + (vo + j) * L.Kc;
                const T* qr = S.Q + (vo + l) * L.Kc;
                T s = s_zero(T());
                for (int c = 0; c < cu; ++c) s = s_fma(pr[c], qr[c], s);
                v = PF ? v + s : v - s;
            }
        }
        sT[ty + 8 * q][tx] = v;   // (j, l)
    }
    __syncthreads();
    T* ow = out + L.mo(w);
    for (int q = 0; q < 4; ++q) {
        const int i = j0 + ty + 8 * q, jj = l0 + tx;   // out[i][jj] = A^{-1}_{i, jj}
        if (i < n && jj < n) ow[(long long)i * n + jj] = sT[tx][ty + 8 * q];
    }
}

// ---- operand formation -----------------------------------------------------
template <typename T>
__global__ void k_form_row_moves(DevLayout L, const T* Phi, int m, const int* occ, const int* slot,
                                 const int* newrow, T* Vout, int* idx) {
    // k simultaneous moves per walker: slot[w*k + a] -> new_row[w*k + a]
    const int w = blockIdx.x, n = L.n_uni, k = L.kk;
    for (int a = 0; a < k; ++a) {
        const int i = slot[(long long)w * k + a];
        const bool ok_i = i >= 0 && i < n;
        const int nr = newrow[(long long)w * k + a];
        const int old = ok_i ? occ[(long long)w * n + i] : 0;
        const bool ok = ok_i && nr >= 0 && nr < m && old >= 0 && old < m;
        T* vo = Vout + ((long long)w * k + a) * n;
        for (int j = threadIdx.x; j < n; j += blockDim.x)
            vo[j] = ok ? (Phi[(long long)nr * n + j] - Phi[(long long)old * n + j]) : s_zero(T());
        if (threadIdx.x == 0) idx[(long long)w * k + a] = ok ? i : -1;   // -1 is rejected by propose
    }
}

template <typename T>
__global__ void k_form_pf_moves(DevLayout L, const T* F, int m, const int* pos, const int* slot,
                                const int* newsite, T* Bout, int* idx) {
    const int w = blockIdx.x, n = L.n_uni;
    const int i = slot[w];
    const bool ok_i = i >= 0 && i < n;
    const int rn = newsite[w];
    const int ri = ok_i ? pos[(long long)w * n + i] : 0;
    const bool ok = ok_i && rn >= 0 && rn < m && ri >= 0 && ri < m;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int rj = pos[(long long)w * n + j];
        const bool okj = ok && rj >= 0 && rj < m;
        Bout[(long long)w * 2 * n + j] = okj ? (F[(long long)rn * m + rj] - F[(long long)ri * m + rj]) : s_zero(T());
    }
    if (threadIdx.x == 0) {
        idx[2 * w] = -1;
        idx[2 * w + 1] = ok ? i : -1;
    }
}

// Two particles p, q of every walker move to new sites at once (Sec. 3.2,
// the update of 2 rows and 2 columns): B = [x, y, e_p, e_q] (C = -J),
// x_j = F(r'_p, r'_j) - F(r_p, r_j) with both new sites, y_j = F(r'_q, r_j) -
// F(r_q, r_j), y_p = 0, so that entry (p, q) of the change is x_q - y_p.
// slot, newsite: W x 2; Bout: W x 4 vectors of n (slots 0, 1 dense); idx: W x 4.
template <typename T>
__global__ void k_form_pf_moves2(DevLayout L, const T* F, int m, const int* pos, const int* slot,
                                 const int* newsite, T* Bout, int* idx) {
    const int w = blockIdx.x, n = L.n_uni;
    const int p = slot[2 * w], q = slot[2 * w + 1];
    const int sp = newsite[2 * w], sq = newsite[2 * w + 1];
    const bool okpq = p >= 0 && p < n && q >= 0 && q < n && p != q;
    const int rp = okpq ? pos[(long long)w * n + p] : 0, rq = okpq ? pos[(long long)w * n + q] : 0;
    const bool ok = okpq && sp >= 0 && sp < m && sq >= 0 && sq < m && rp >= 0 && rp < m && rq >= 0 && rq < m;
    T* x = Bout + (long long)w * 4 * n;
    T* y = x + n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int rj = pos[(long long)w * n + j];
        const bool okj = ok && rj >= 0 && rj < m;
        const int rj_new = j == p ? sp : (j == q ? sq : rj);
        x[j] = okj ? (F[(long long)sp * m + rj_new] - F[(long long)rp * m + rj]) : s_zero(T());
        y[j] = (okj && j != p) ? (F[(long long)sq * m + rj] - F[(long long)rq * m + rj]) : s_zero(T());
    }
    if (threadIdx.x == 0) {
        idx[4 * w] = -1;
        idx[4 * w + 1] = -1;
        idx[4 * w + 2] = ok ? p : -1;
        idx[4 * w + 3] = ok ? q : -1;
    }
}

// A_w[i][j] = Phi[occ_w[i]][j] (rows) or F[pos_w[i]][pos_w[j]] (pairs)
template <typename T, bool PAIRS>
__global__ void k_gather(DevLayout L, const T* src, int m, const int* occ, T* A, int* err) {
    const int w = blockIdx.y, n = L.n_uni;
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const int ri = occ[(long long)w * n + i];
        T v = s_zero(T());
        if (PAIRS) {
            const int rj = occ[(long long)w * n + j];
            if (ri >= 0 && ri < m && rj >= 0 && rj < m) v = src[(long long)ri * m + rj];
            else set_dev_error(err, DEV_ERR_INDEX);
        } else {
            if (ri >= 0 && ri < m) v = src[(long long)ri * n + j];
            else set_dev_error(err, DEV_ERR_INDEX);
        }
        A[(long long)w * total + e] = v;
    }
}

template <typename T>
void launch_gather(bool pairs, const DevLayout& L, const T* src, int m, const int* occ, T* A, int* err,
                   cudaStream_t st) {
    const long long total = (long long)L.n_uni * L.n_uni;
    dim3 grid((unsigned)std::min<long long>((total + 255) / 256, 64), L.W);
    if (pairs) k_gather<T, true><<<grid, 256, 0, st>>>(L, src, m, occ, A, err);
    else k_gather<T, false><<<grid, 256, 0, st>>>(L, src, m, occ, A, err);
}

#if !defined(LRU_INST_DTYPE) || defined(LRU_INST_PRIMARY)
__global__ void k_commit_moves(int W, int n, int k, int* occ, const int* slot, const int* newrow,
                               const uint8_t* mask, const int* pst) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    if (mask && !mask[w]) return;
    if (pst && pst[w] != 4) return;   // 4: consumed by an accept
    for (int a = 0; a < k; ++a) {
        const int i = slot[(long long)w * k + a];
        if (i >= 0 && i < n) occ[(long long)w * n + i] = newrow[(long long)w * k + a];
    }
}
#endif

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
void launch_propose(bool pf, bool delayed, bool df, const DevLayout& L, const DevState<T>& S,
                    const DevOperand& U_in, const DevOperand& V, const T* C, T* ratio_out, int* st_out,
                    cudaStream_t st) {
    const size_t dyn = delayed ? (size_t)L.Kc * MAXKK * sizeof(T) : 0;
    const unsigned all = (L.kk >= 32) ? 0xffffffffu : ((1u << L.kk) - 1u);
    DevOperand U = U_in;
    if (delayed && (U.mask & all) != all)
        k_qtu_dense<T><<<dim3(L.W, L.kk), PT, 0, st>>>(L, S, U);
    // exactly one dense column: its pass over A^{-1} runs as its own kernel
    const unsigned dense = ~U.mask & all;
    if (dense != 0 && (dense & (dense - 1)) == 0) {
        int a = 0;
        while (!((dense >> a) & 1u)) ++a;
        const int nr = (L.n_max + PT - 1) / PT;
        bool launched = false;
        if constexpr (std::is_same<T, double>::value) {
            if (df && pf && L.n_uni > 0 && (L.n_uni % 2) == 0 && L.n_uni <= 2048) {
                // Pfaffian: A^{-1} is exactly skew, so X = -(u^T A^{-1})^T streams
                // contiguous rows, one warp each
                dim3 grid(L.W, (L.n_max + DF_CPB - 1) / DF_CPB);
                const int np2 = (L.n_max / 2 + 31) / 32;
#define LRU_PF_WDF(N) \
    case N: k_dense_column_skew_df<N><<<grid, PT, 0, st>>>(L, S, U, a); break;
                switch (np2 <= 4 ? 4 : (np2 <= 8 ? 8 : (np2 <= 16 ? 16 : 32))) {
                    LRU_PF_WDF(4) LRU_PF_WDF(8) LRU_PF_WDF(16) LRU_PF_WDF(32) default: break;
                }
#undef LRU_PF_WDF
                launched = true;
            } else if (df) {
                if (nr <= 1) k_dense_column<T, 1, true><<<L.W, PT, 0, st>>>(L, S, U, a);
                else if (nr <= 2) k_dense_column<T, 2, true><<<L.W, PT, 0, st>>>(L, S, U, a);
                else if (nr <= 4) k_dense_column<T, 4, true><<<L.W, PT, 0, st>>>(L, S, U, a);
                else k_dense_column<T, 8, true><<<L.W, PT, 0, st>>>(L, S, U, a);
                launched = true;
            }
        }
        if (!launched) {
            if (nr <= 1) k_dense_column<T, 1, false><<<L.W, PT, 0, st>>>(L, S, U, a);
            else if (nr <= 2) k_dense_column<T, 2, false><<<L.W, PT, 0, st>>>(L, S, U, a);
            else if (nr <= 4) k_dense_column<T, 4, false><<<L.W, PT, 0, st>>>(L, S, U, a);
            else k_dense_column<T, 8, false><<<L.W, PT, 0, st>>>(L, S, U, a);
        }
        U.pre = a;
    }
    if (!pf && !delayed) k_propose<T, false, false><<<L.W, PT, dyn, st>>>(L, S, U, V, C, ratio_out, st_out);
    if (!pf && delayed) {
        cudaFuncSetAttribute(k_propose<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        k_propose<T, false, true><<<L.W, PT, dyn, st>>>(L, S, U, V, C, ratio_out, st_out);
    }
    if (pf && !delayed) k_propose<T, true, false><<<L.W, PT, dyn, st>>>(L, S, U, V, C, ratio_out, st_out);
    if (pf && delayed) {
        cudaFuncSetAttribute(k_propose<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        k_propose<T, true, true><<<L.W, PT, dyn, st>>>(L, S, U, V, C, ratio_out, st_out);
    }
}

template <typename T, bool DELAYED>
static void accept_npl(int npl, const DevLayout& L, const DevState<T>& S, const DevOperand& V,
                       const uint8_t* mask, const int* items, int nitems, size_t dyn, cudaStream_t st) {
    const int4* it = reinterpret_cast<const int4*>(items);
    const bool rank1 = L.kk == 1 && L.kvec == nullptr;
#define LRU_ACC(N)                                                                                          \
    case N:                                                                                                 \
        if (rank1) {                                                                                        \
            cudaFuncSetAttribute(k_accept<T, DELAYED, N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn); \
            k_accept<T, DELAYED, N, 1><<<nitems, PT, dyn, st>>>(L, S, V, mask, it);                          \
        } else {                                                                                            \
            cudaFuncSetAttribute(k_accept<T, DELAYED, N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn); \
            k_accept<T, DELAYED, N, 0><<<nitems, PT, dyn, st>>>(L, S, V, mask, it);                          \
        }                                                                                                   \
        break;
    switch (npl) {
        LRU_ACC(1) LRU_ACC(2) LRU_ACC(4) LRU_ACC(8) LRU_ACC(16) LRU_ACC(32) LRU_ACC(64)
        default: break;
    }
#undef LRU_ACC
}

template <typename T>
void launch_accept(bool pf, bool delayed, bool df, const DevLayout& L, const DevState<T>& S, const DevOperand& V,
                   const uint8_t* mask, const int* items, int nitems, cudaStream_t st) {
    const int nmax = L.n_max;
    int npl = 1;
    while (32 * npl < nmax) npl *= 2;
    size_t dyn = (size_t)2 * L.kk * nmax * sizeof(T);
    if (dyn > 160 * 1024) dyn = 0;   // items carry use_smem = 0 in that case (set by the API)
    if (nitems > 0) {
        bool done = false;
        if constexpr (std::is_same<T, double>::value) {
            if (df && delayed && !pf && L.kk == 1 && L.kvec == nullptr && L.n_uni > 0 && !(V.mask & 1u) &&
                L.n_uni <= 2048 && (L.n_uni % 2) == 0) {
                // rank-1, uniform even n: one warp per column of A_0^{-1}
                dim3 grid(L.W, (L.n_uni + DF_CPB - 1) / DF_CPB);
                const int np2 = (L.n_uni / 2 + 31) / 32;
#define LRU_ACC_WDF(N) \
    case N: k_accept_delayed_warp_df<N><<<grid, PT, 0, st>>>(L, S, V, mask); break;
                switch (np2 <= 4 ? 4 : (np2 <= 8 ? 8 : (np2 <= 16 ? 16 : 32))) {
                    LRU_ACC_WDF(4) LRU_ACC_WDF(8) LRU_ACC_WDF(16) LRU_ACC_WDF(32) default: break;
                }
#undef LRU_ACC_WDF
                done = true;
            }
            if (!done && df && delayed && !pf && L.kk == 1 && !(V.mask & 1u) && L.n_max <= 2048) {
                const int4* it = reinterpret_cast<const int4*>(items);
#define LRU_ACC_DF(N) \
    case N: k_accept_delayed_df<N><<<nitems, PT, 0, st>>>(L, S, V, mask, it); break;
                const int np2 = npl <= 2 ? 1 : npl / 2;   // double2 loads per lane
                switch (np2) { LRU_ACC_DF(1) LRU_ACC_DF(2) LRU_ACC_DF(4) LRU_ACC_DF(8) LRU_ACC_DF(16) LRU_ACC_DF(32) default: break; }
#undef LRU_ACC_DF
                done = true;
            }
        }
        if (!done && delayed && !pf && L.kk == 1 && L.kvec == nullptr && L.n_uni > 0 && !(V.mask & 1u) &&
            L.n_uni <= 2048 && (L.n_uni % 2) == 0) {
            // rank-1 delayed accept: one thread per column of A_0^{-1}
            dim3 grid(L.W, (L.n_uni + PT - 1) / PT);
            k_accept_delayed_lane<T><<<grid, PT, 0, st>>>(L, S, V, mask);
            done = true;
        }
        if (!done && pf && !delayed) {
            // Pfaffian: the exactly skew rank-2k update over the upper triangle
            const int nt = (nmax + 31) / 32;
            k_accept_pf_skew<T><<<dim3(nt * (nt + 1) / 2, L.W), 256, 0, st>>>(L, S, mask);
            done = true;
        }
        if (!done) {
            if (delayed) accept_npl<T, true>(npl, L, S, V, mask, items, nitems, dyn, st);
            else accept_npl<T, false>(npl, L, S, V, mask, items, nitems, dyn, st);
        }
    }
    k_commit<T><<<(L.W + 255) / 256, 256, 0, st>>>(L, S, mask, delayed);
}

template <typename T>
void launch_flush_native(bool pf, const DevLayout& L, const DevState<T>& S, const uint8_t* force_mask,
                         int nmax, cudaStream_t st) {
    (void)nmax;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (pf) k_flush_native<T, true><<<4 * nsm, 256, 0, st>>>(L, S, force_mask);
    else k_flush_native<T, false><<<4 * nsm, 256, 0, st>>>(L, S, force_mask);
}

#if !defined(LRU_INST_DTYPE) || defined(LRU_INST_PRIMARY)
void launch_flush_df(bool pf, const DevLayout& L, const DevState<double>& S, const uint8_t* force_mask,
                     cudaStream_t st) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (pf) k_flush_df<true><<<4 * nsm, 256, 0, st>>>(L, S, force_mask);
    else k_flush_df<false><<<4 * nsm, 256, 0, st>>>(L, S, force_mask);
}

#endif

template <typename T>
void launch_flush_finish(const DevLayout& L, const DevState<T>& S, const uint8_t* force_mask, cudaStream_t st) {
    k_flush_finish<T><<<(L.W + 255) / 256, 256, 0, st>>>(L, S, force_mask);
}

template <typename T>
void launch_set_delay_zero(const DevLayout& L, const DevState<T>& S, cudaStream_t st) {
    k_set_delay_zero<T><<<(L.W + 255) / 256, 256, 0, st>>>(L, S);
}

template <typename T>
void launch_get_inverse(bool pf, bool delayed, const DevLayout& L, const DevState<T>& S, T* out,
                        cudaStream_t st) {
    const int nt = (L.n_max + 31) / 32;
    dim3 grid(nt, nt, L.W);
    if (!pf && !delayed) k_get_inverse<T, false, false><<<grid, 256, 0, st>>>(L, S, out);
    if (!pf && delayed) k_get_inverse<T, false, true><<<grid, 256, 0, st>>>(L, S, out);
    if (pf && !delayed) k_get_inverse<T, true, false><<<grid, 256, 0, st>>>(L, S, out);
    if (pf && delayed) k_get_inverse<T, true, true><<<grid, 256, 0, st>>>(L, S, out);
}

template <typename T>
void launch_form_row_moves(const DevLayout& L, const T* Phi, int m, const int* occ, const int* slot,
                           const int* newrow, T* Vout, int* idx, cudaStream_t st) {
    k_form_row_moves<T><<<L.W, 256, 0, st>>>(L, Phi, m, occ, slot, newrow, Vout, idx);
}

template <typename T>
void launch_form_pf_moves(const DevLayout& L, const T* F, int m, const int* pos, const int* slot,
                          const int* newsite, T* Bout, int* idx, cudaStream_t st) {
    if (L.kk == 4) k_form_pf_moves2<T><<<L.W, 256, 0, st>>>(L, F, m, pos, slot, newsite, Bout, idx);
    else k_form_pf_moves<T><<<L.W, 256, 0, st>>>(L, F, m, pos, slot, newsite, Bout, idx);
}

#if !defined(LRU_INST_DTYPE) || defined(LRU_INST_PRIMARY)
void launch_commit_moves(int W, int n, int k, int* occ, const int* slot, const int* newrow, const uint8_t* mask,
                         const int* pst, cudaStream_t st) {
    k_commit_moves<<<(W + 255) / 256, 256, 0, st>>>(W, n, k, occ, slot, newrow, mask, pst);
}
#endif

#define LRU_INST(T)                                                                                          \
    template void launch_propose<T>(bool, bool, bool, const DevLayout&, const DevState<T>&, const DevOperand&, \
                                    const DevOperand&, const T*, T*, int*, cudaStream_t);                   \
    template void launch_accept<T>(bool, bool, bool, const DevLayout&, const DevState<T>&, const DevOperand&, \
                                   const uint8_t*, const int*, int, cudaStream_t);                          \
    template void launch_flush_native<T>(bool, const DevLayout&, const DevState<T>&, const uint8_t*, int,   \
                                         cudaStream_t);                                                     \
    template void launch_flush_finish<T>(const DevLayout&, const DevState<T>&, const uint8_t*, cudaStream_t); \
    template void launch_set_delay_zero<T>(const DevLayout&, const DevState<T>&, cudaStream_t);             \
    template void launch_zero_split_tail<T>(const DevLayout&, const DevState<T>&, const uint8_t*, cudaStream_t); \
    template void launch_get_inverse<T>(bool, bool, const DevLayout&, const DevState<T>&, T*, cudaStream_t); \
    template void launch_form_row_moves<T>(const DevLayout&, const T*, int, const int*, const int*,         \
                                           const int*, T*, int*, cudaStream_t);                             \
    template void launch_form_pf_moves<T>(const DevLayout&, const T*, int, const int*, const int*,          \
                                          const int*, T*, int*, cudaStream_t);                              \
    template void launch_gather<T>(bool, const DevLayout&, const T*, int, const int*, T*, int*, cudaStream_t);

#define LRU_INST_STEP(T)                                                                                   \
    template void launch_step<T>(bool, bool, const DevLayout&, const DevState<T>&, const DevOperand&,        \
                                 const DevOperand&, const T*, T*, int*, const StepCtl&, int, cudaStream_t);

// The build compiles this file in parallel: once per dtype (LRU_INST_DTYPE)
// without the persistent step (LRU_NO_STEP), and once per dtype with the step
// alone (LRU_STEP_ONLY).
#if defined(LRU_INST_DTYPE)
#if !defined(LRU_STEP_ONLY)
LRU_INST(LRU_INST_DTYPE)
#endif
#if !defined(LRU_NO_STEP)
LRU_INST_STEP(LRU_INST_DTYPE)
#endif
#else
LRU_INST(double)
LRU_INST(float)
LRU_INST(c128)
LRU_INST(c64)
LRU_INST_STEP(double)
LRU_INST_STEP(float)
LRU_INST_STEP(c128)
LRU_INST_STEP(c64)
#endif

#if !defined(LRU_INST_DTYPE) || defined(LRU_INST_PRIMARY)
// One warp waits, with the persistent step's bounded wait, on a flag that no
// kernel ever sets: the wait must give up after `iters` polls and leave
// DEV_ERR_TIMEOUT for the host, with the context still usable.
__global__ void k_wait_selftest(const int* flag, long long iters, int* err) {
    if (threadIdx.x == 0) bounded_acquire_wait(flag, 1, iters, err);
}
void launch_wait_selftest(const int* flag, long long iters, int* err, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(flag, iters, err);
}
#endif

}  // namespace lru
