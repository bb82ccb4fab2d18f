// Adjoint (vector-Jacobian product) of the log ratio of the pending proposal
// and of log|value|, for reverse-mode differentiation.
//
// Determinant (Sec. 2.1, Eqs. det_R, det_ratio): log r = log det R,
// R = I + V A^{-1} U.  With X = A^{-1} U and Y = V A^{-1},
//   d log r = tr(R^{-1} dR) = tr(R^{-1} (dV X + Y dU - Y dA X)),
// so dlogr/dU = (R^{-1} Y)^T, dlogr/dV = (X R^{-1})^T, dlogr/dA = -(X R^{-1} Y)^T.
// Pfaffian (App. A.2 Eq. pf_low_rank, App. A.3 Eq. pf_grad): log r =
// log pf M - log pf C^{-1}, M = C^{-1} + B^T A^{-1} B, d log pf M = tr(M^{-1} dM)/2
// for skew dM; with X = A^{-1} B and A^{-1}, M^{-1} skew:
//   dlogr/dB = X M^{-1},  dlogr/dA_ij = (X M^{-1} X^T)_ji / 2,
//   dlogr/dC = skew part of -[C^{-1} (M^{-1} - C) C^{-1}]^T / 2,
// where A and C enter through their skew parts (A - A^T)/2 as in App. A.3.
// log|value|: dlog det A / dA = A^{-T}; dlog pf A / dA_ij = (A^{-1})_ji / 2.
// For complex dtypes every output is the conjugate-Wirtinger vector-Jacobian
// product  g * conj(J)  that PyTorch's autograd expects for holomorphic maps.
// The delayed state never materialises A^{-1}: Y is recomputed from A_0^{-1}
// and the stored slots, Y = V A_0^{-1} - (V P) Q^T.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace lru {

constexpr int AT = 256;
constexpr int AMAXKK = 16;

template <typename T> __device__ __forceinline__ T s_conj(T a) { return a; }
template <> __device__ __forceinline__ c128 s_conj<c128>(c128 a) { return {a.re, -a.im}; }
template <> __device__ __forceinline__ c64 s_conj<c64>(c64 a) { return {a.re, -a.im}; }

template <typename T>
__device__ __forceinline__ const T* opvec(const DevOperand& O, const DevLayout& L, int w, int a, int n) {
    return reinterpret_cast<const T*>(O.dense) + (L.vo(w) * O.slots + (long long)a * n);
}

// One CTA per walker.  ws: 2 * kk * n_w scalars per walker (Y, then Z).
template <typename T, bool PF, bool DELAYED>
__global__ void __launch_bounds__(AT) k_backward(DevLayout L, DevState<T> S, DevOperand Vop, const T* C, const T* g,
                                                  T* ws, T* gU, T* gV, T* gA, T* gC) {
    __shared__ T sR[AMAXKK * AMAXKK];
    __shared__ int siv[AMAXKK];
    __shared__ T sVP[AMAXKK * 64];
    const int w = blockIdx.x;
    const int n = L.nw(w), kk = L.kv(w);
    const long long vo = L.vo(w);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int slots = L.kk;
    T* gUw = gU ? gU + vo * slots : nullptr;
    T* gVw = gV ? gV + vo * slots : nullptr;
    T* gAw = gA ? gA + L.mo(w) : nullptr;
    if (S.pst[w] != 0) {
        // no pending proposal with a valid core: zero gradient
        for (long long e = threadIdx.x; e < (long long)kk * n; e += AT) {
            if (gUw) gUw[e] = s_zero(T());
            if (gVw) gVw[e] = s_zero(T());
        }
        if (gAw)
            for (long long e = threadIdx.x; e < (long long)n * n; e += AT) gAw[e] = s_zero(T());
        if (gC && threadIdx.x < kk * kk) gC[(long long)w * L.kk * L.kk + threadIdx.x] = s_zero(T());
        return;
    }
    const T gw = g[w];
    const T* X = S.X + vo * L.kk;             // kk vectors of n: X[a*n + j] = (A^{-1} U)_{j a}
    T* Y = ws + vo * 2 * slots;               // kk x n
    T* Z = Y + (long long)slots * n;          // n x kk, Z[j*kk + b]
    for (int e = threadIdx.x; e < AMAXKK * AMAXKK; e += AT) sR[e] = S.Rinv[(long long)w * AMAXKK * AMAXKK + e];
    if (threadIdx.x < kk)
        siv[threadIdx.x] = ((Vop.mask >> threadIdx.x) & 1u) ? Vop.idx[(long long)w * Vop.slots + threadIdx.x] : -1;
    const int cu = DELAYED ? S.tau[w] * kk : 0;
    if constexpr (DELAYED && !PF)
        for (int e = threadIdx.x; e < kk * cu; e += AT) {
            const int b = e / cu, c = e % cu;
            sVP[b * 64 + c] = S.VP[(long long)w * AMAXKK * L.Kc + b * L.Kc + c];
        }
    __syncthreads();

    // Z = X R^{-1} (n x kk)
    for (int j = threadIdx.x; j < n; j += AT)
        for (int b = 0; b < kk; ++b) {
            T z = s_zero(T());
            for (int a = 0; a < kk; ++a) z = s_fma(X[(long long)a * n + j], sR[a * AMAXKK + b], z);
            Z[(long long)j * kk + b] = z;
        }

    if constexpr (!PF) {
        // Y = V A^{-1}: one warp per column l of A^{-1} (a contiguous chunk)
        const T* Gw = S.G + L.mo(w);
        for (int l = wid; l < n; l += AT / 32) {
            const T* col = Gw + (long long)l * n;
            for (int b = 0; b < kk; ++b) {
                T y;
                if (siv[b] >= 0) {
                    y = col[siv[b]];
                } else {
                    const T* vb = opvec<T>(Vop, L, w, b, n);
                    T part = s_zero(T());
                    for (int j = lane; j < n; j += 32) part = s_fma(vb[j], col[j], part);
                    y = warp_sum(part);
                }
                if constexpr (DELAYED) {
                    const T* qrow = S.Q + (vo + l) * L.Kc;
                    for (int c = 0; c < cu; ++c) y = s_fms(sVP[b * 64 + c], qrow[c], y);
                }
                if (lane == 0) Y[(long long)b * n + l] = y;
            }
        }
    }
    __syncthreads();

    if constexpr (!PF) {
        // gU[a][j] = g conj((R^{-1} Y)_{a j}),  gV[b][j] = g conj(Z[j][b])
        for (int j = threadIdx.x; j < n; j += AT)
            for (int a = 0; a < kk; ++a) {
                if (gUw) {
                    T s = s_zero(T());
                    for (int b = 0; b < kk; ++b) s = s_fma(sR[a * AMAXKK + b], Y[(long long)b * n + j], s);
                    gUw[(long long)a * n + j] = gw * s_conj(s);
                }
                if (gVw) gVw[(long long)a * n + j] = gw * s_conj(Z[(long long)j * kk + a]);
            }
        // gA[i][j] = -g conj(sum_b Z[j][b] Y[b][i])  (row-major)
        if (gAw)
            for (long long e = threadIdx.x; e < (long long)n * n; e += AT) {
                const int i = (int)(e / n), j = (int)(e % n);
                T s = s_zero(T());
                for (int b = 0; b < kk; ++b) s = s_fma(Z[(long long)j * kk + b], Y[(long long)b * n + i], s);
                gAw[e] = s_neg(gw * s_conj(s));
            }
    } else {
        // gB[b][j] = g conj(Z[j][b]) with Z = X M^{-1}
        if (gUw)
            for (int j = threadIdx.x; j < n; j += AT)
                for (int b = 0; b < kk; ++b) gUw[(long long)b * n + j] = gw * s_conj(Z[(long long)j * kk + b]);
        // gA[i][j] = g conj((X M^{-1} X^T)_{j i} / 2) = -g conj(sum_b Z[i][b] X_b[j]) / 2
        if (gAw)
            for (long long e = threadIdx.x; e < (long long)n * n; e += AT) {
                const int i = (int)(e / n), j = (int)(e % n);
                T s = s_zero(T());
                for (int b = 0; b < kk; ++b) s = s_fma(Z[(long long)i * kk + b], X[(long long)b * n + j], s);
                gAw[e] = s_neg(s_half(gw * s_conj(s)));
            }
        // gC = skew part of -[C^{-1} (M^{-1} - C) C^{-1}]^T / 2 (C = -J when C is null)
        if (gC && threadIdx.x == 0) {
            T Cm[AMAXKK * AMAXKK], Ci[AMAXKK * AMAXKK], T1[AMAXKK * AMAXKK];
            const int m = kk;
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) {
                    double v = (b == a + m / 2) ? -1.0 : ((a == b + m / 2) ? 1.0 : 0.0);   // -J
                    Cm[a * AMAXKK + b] = C ? C[(long long)w * L.kk * L.kk + a * m + b] : make_real<T>(v);
                }
            // C^{-1} by Gauss-Jordan on a copy (small, m <= 16)
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) Ci[a * AMAXKK + b] = Cm[a * AMAXKK + b];
            {
                int swp[AMAXKK];
                for (int k = 0; k < m; ++k) {
                    int p = k;
                    double best = (double)s_abs2(Ci[k * AMAXKK + k]);
                    for (int i = k + 1; i < m; ++i)
                        if ((double)s_abs2(Ci[i * AMAXKK + k]) > best) { best = (double)s_abs2(Ci[i * AMAXKK + k]); p = i; }
                    swp[k] = p;
                    if (p != k)
                        for (int j = 0; j < m; ++j) {
                            T t = Ci[k * AMAXKK + j]; Ci[k * AMAXKK + j] = Ci[p * AMAXKK + j]; Ci[p * AMAXKK + j] = t;
                        }
                    T ip = s_recip(Ci[k * AMAXKK + k]);
                    Ci[k * AMAXKK + k] = make_real<T>(1.0);
                    for (int j = 0; j < m; ++j) Ci[k * AMAXKK + j] = Ci[k * AMAXKK + j] * ip;
                    for (int i = 0; i < m; ++i) {
                        if (i == k) continue;
                        T f = Ci[i * AMAXKK + k];
                        Ci[i * AMAXKK + k] = s_zero(T());
                        for (int j = 0; j < m; ++j) Ci[i * AMAXKK + j] = s_fms(f, Ci[k * AMAXKK + j], Ci[i * AMAXKK + j]);
                    }
                }
                for (int k = m - 1; k >= 0; --k)
                    if (swp[k] != k)
                        for (int i = 0; i < m; ++i) {
                            T t = Ci[i * AMAXKK + k]; Ci[i * AMAXKK + k] = Ci[i * AMAXKK + swp[k]]; Ci[i * AMAXKK + swp[k]] = t;
                        }
            }
            // T1 = (M^{-1} - C) C^{-1}; then G = C^{-1} T1
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) {
                    T s = s_zero(T());
                    for (int c = 0; c < m; ++c) s = s_fma(sR[a * AMAXKK + c] - Cm[a * AMAXKK + c], Ci[c * AMAXKK + b], s);
                    T1[a * AMAXKK + b] = s;
                }
            T* gCw = gC + (long long)w * L.kk * L.kk;
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) {
                    // unconstrained gradient entry (a, b) = -[C^{-1} T1]_{b a} / 2
                    T sba = s_zero(T()), sab = s_zero(T());
                    for (int c = 0; c < m; ++c) {
                        sba = s_fma(Ci[b * AMAXKK + c], T1[c * AMAXKK + a], sba);
                        sab = s_fma(Ci[a * AMAXKK + c], T1[c * AMAXKK + b], sab);
                    }
                    // skew part: (G_ab - G_ba) / 2 with G_ab = -sba / 2, G_ba = -sab / 2
                    T v = s_half(s_half(sab - sba));
                    gCw[a * m + b] = gw * s_conj(v);
                }
        }
    }
}

// gA = g A^{-T} (det) or g A^{-T}/2 = -g A^{-1}/2 (pf), conjugated for complex;
// A^{-1} = A_0^{-1} -/+ P Q^T for the delayed state.  Row-major output.
template <typename T, bool PF, bool DELAYED>
__global__ void k_backward_logvalue(DevLayout L, DevState<T> S, const T* g, T* gA) {
    const int w = blockIdx.y;
    const int n = L.nw(w), kk = L.kv(w);
    const long long vo = L.vo(w);
    const T* Gw = S.G + L.mo(w);
    T* out = gA + L.mo(w);
    const T gw = g[w];
    const int cu = DELAYED ? S.tau[w] * kk : 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        // (A^{-T})_{ij} = (A^{-1})_{ji}, stored at column-major position [i*n + j] = e
        T v = Gw[e];
        if (DELAYED && cu) {
            const T* pr = S.P + (vo + j) * L.Kc;
            const T* qr = S.Q + (vo + i) * L.Kc;
            T s = s_zero(T());
            for (int c = 0; c < cu; ++c) s = s_fma(pr[c], qr[c], s);
            v = PF ? v + s : v - s;
        }
        v = gw * s_conj(v);
        out[e] = PF ? s_half(v) : v;
    }
}

// log of the stored ratios: real dtypes log|r|, complex the principal log r
template <typename T>
__global__ void k_log_ratio(int W, const T* ratio, T* out) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const T r = ratio[w];
    if constexpr (traits<T>::is_complex) {
        using R = typename traits<T>::real;
        out[w] = T{(R)log(s_absd(r)), (R)atan2((double)r.im, (double)r.re)};
    } else {
        out[w] = (T)log(s_absd(r));
    }
}

// gPhi[rows[w][i]][:] += gA[w][i][:] (atomic; rows shared between walkers)
template <typename T>
__global__ void k_scatter_rows(DevLayout L, const T* gA, const int* rows, int m, T* gPhi, int* err) {
    const int w = blockIdx.y;
    const int n = L.n_uni;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const int r = rows[(long long)w * n + i];
        if (r < 0 || r >= m) { set_dev_error(err, DEV_ERR_INDEX); continue; }
        const T v = gA[(long long)w * n * n + e];
        if constexpr (traits<T>::is_complex) {
            atomicAdd(&gPhi[(long long)r * n + j].re, v.re);
            atomicAdd(&gPhi[(long long)r * n + j].im, v.im);
        } else {
            atomicAdd(&gPhi[(long long)r * n + j], v);
        }
    }
}

template <typename T>
void launch_backward(bool pf, bool delayed, const DevLayout& L, const DevState<T>& S, const DevOperand& V,
                     const T* C, const T* g, T* ws, T* gU, T* gV, T* gA, T* gC, cudaStream_t st) {
    if (!pf && !delayed) k_backward<T, false, false><<<L.W, AT, 0, st>>>(L, S, V, C, g, ws, gU, gV, gA, gC);
    if (!pf && delayed) k_backward<T, false, true><<<L.W, AT, 0, st>>>(L, S, V, C, g, ws, gU, gV, gA, gC);
    if (pf && !delayed) k_backward<T, true, false><<<L.W, AT, 0, st>>>(L, S, V, C, g, ws, gU, gV, gA, gC);
    if (pf && delayed) k_backward<T, true, true><<<L.W, AT, 0, st>>>(L, S, V, C, g, ws, gU, gV, gA, gC);
}

template <typename T>
void launch_backward_logvalue(bool pf, bool delayed, const DevLayout& L, const DevState<T>& S, const T* g, T* gA,
                              cudaStream_t st) {
    dim3 grid(64, L.W);
    if (!pf && !delayed) k_backward_logvalue<T, false, false><<<grid, 256, 0, st>>>(L, S, g, gA);
    if (!pf && delayed) k_backward_logvalue<T, false, true><<<grid, 256, 0, st>>>(L, S, g, gA);
    if (pf && !delayed) k_backward_logvalue<T, true, false><<<grid, 256, 0, st>>>(L, S, g, gA);
    if (pf && delayed) k_backward_logvalue<T, true, true><<<grid, 256, 0, st>>>(L, S, g, gA);
}

template <typename T>
void launch_log_ratio(int W, const T* ratio, T* out, cudaStream_t st) {
    k_log_ratio<T><<<(W + 255) / 256, 256, 0, st>>>(W, ratio, out);
}

template <typename T>
void launch_scatter_rows(const DevLayout& L, const T* gA, const int* rows, int m, T* gPhi, int* err, cudaStream_t st) {
    dim3 grid(64, L.W);
    k_scatter_rows<T><<<grid, 256, 0, st>>>(L, gA, rows, m, gPhi, err);
}

// Gradient of the outputs (sign or phase s, log|value|) of the batched
// slogdet / slogpf: with t = tr(A^{-1} dA), d log|det A| = Re t and
// d s = i s Im t, so for a loss L with dL/dlog|.| = g_l and dL/ds = g_s (torch's
// convention for complex) dL = Re(conj(c) t), c = g_l + i beta,
// beta = -Im(conj(g_s) s), and grad_A = c A^{-H} (real: g_l A^{-T}).  The
// Pfaffian has log pf = (1/2) log det of the skew part (App. A.3, Eq.
// pf_grad): grad_A = (c / 2) (skew part of A^{-1})^H.  Ginv: the column-major
// inverses, Ginv[w][l n + j] = (A_w^{-1})_{jl}, so (A^{-H})_{ij} is
// conj(Ginv[w][i n + j]).
template <typename T>
__global__ void k_slog_grad(int W, int n, bool pf, const T* Ginv, const double* g_l, const T* g_s, const T* sign,
                            T* gA) {
    const long long nn = (long long)n * n, total = nn * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(e / nn);
        const long long r = e - (long long)w * nn;
        const int i = (int)(r / n), j = (int)(r - (long long)i * n);
        const T* G = Ginv + (long long)w * nn;
        T c = make_real<T>(g_l ? g_l[w] : 0.0);
        if constexpr (traits<T>::is_complex) {
            if (g_s) {
                const T q = s_conj(g_s[w]) * sign[w];
                c.im = -q.im;
            }
        }
        T v = G[(long long)i * n + j];
        if (pf) v = s_half(s_half(v - G[(long long)j * n + i]));   // (1/2) of the skew part
        gA[e] = c * s_conj(v);
    }
}

template <typename T>
void launch_slog_grad(int W, int n, bool pf, const T* Ginv, const double* g_l, const T* g_s, const T* sign, T* gA,
                      cudaStream_t st) {
    const long long total = (long long)n * n * W;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152 * 16);
    k_slog_grad<T><<<grid, 256, 0, st>>>(W, n, pf, Ginv, g_l, g_s, sign, gA);
}

#define LRU_INST_A(T)                                                                                        \
    template void launch_slog_grad<T>(int, int, bool, const T*, const double*, const T*, const T*, T*,        \
                                      cudaStream_t);                                                          \
    template void launch_backward<T>(bool, bool, const DevLayout&, const DevState<T>&, const DevOperand&,     \
                                     const T*, const T*, T*, T*, T*, T*, T*, cudaStream_t);                   \
    template void launch_backward_logvalue<T>(bool, bool, const DevLayout&, const DevState<T>&, const T*, T*, \
                                              cudaStream_t);                                                  \
    template void launch_log_ratio<T>(int, const T*, T*, cudaStream_t);                                       \
    template void launch_scatter_rows<T>(const DevLayout&, const T*, const int*, int, T*, int*, cudaStream_t);

LRU_INST_A(double)
LRU_INST_A(float)
LRU_INST_A(c128)
LRU_INST_A(c64)

}  // namespace lru
