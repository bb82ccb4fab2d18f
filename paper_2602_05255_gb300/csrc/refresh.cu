// From-scratch inverse, log|det| and Pfaffian of the walker matrices: the
// initial carrier (Sec. 2.3 init_det_carrier, Sec. 3.3 init_pf_carrier) and
// the periodic refresh that bounds the drift of the update chain (Sec. 2.1
// advises double precision against accumulated error).  Always run in the
// handle dtype (FP64 / complex128 for the double types).
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace lru {

constexpr int RT = 256;   // threads per matrix
constexpr int GB = 16;    // Gauss-Jordan panel width

__device__ void block_argmax(double v, int i, double* sv, int* si, double& bv, int& bi) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi >= 0 && (i < 0 || oi < i))) { v = ov; i = oi; }
    }
    if (lane == 0) { sv[wid] = v; si[wid] = i; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = sv[0];
        int ib = si[0];
        for (int q = 1; q < RT / 32; ++q)
            if (sv[q] > b || (sv[q] == b && si[q] >= 0 && (ib < 0 || si[q] < ib))) { b = sv[q]; ib = si[q]; }
        sv[0] = b;
        si[0] = ib;
    }
    __syncthreads();
    bv = sv[0];
    bi = si[0];
    __syncthreads();
}

// Loads M = A^T (A row-major n x n) through 32 x 32 shared-memory tiles.
template <typename T>
__device__ void load_transposed(T* M, const T* A, int n, T (*tile)[33]) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int b0 = 0; b0 < n; b0 += 32)
        for (int b1 = 0; b1 < n; b1 += 32) {
            for (int q = ty; q < 32; q += RT / 32) {
                const int r = b0 + q, c = b1 + tx;
                if (r < n && c < n) tile[q][tx] = A[(long long)r * n + c];
            }
            __syncthreads();
            for (int q = ty; q < 32; q += RT / 32) {
                const int r = b1 + q, c = b0 + tx;   // M[r][c] = A[c][r]
                if (r < n && c < n) M[(long long)r * n + c] = tile[tx][q];
            }
            __syncthreads();
        }
}

// In-place Gauss-Jordan inversion with partial pivoting of the row-major n x n
// matrix M, blocked in panels of GB columns: each panel is eliminated with the
// row exchanges restricted to it, then the exchanges and the panel's
// accumulated transform T = I + sum_c (panel_c - e_c) e_c^T are applied to the
// other columns as one rank-GB update (a GEMM).  Row exchanges turn into
// column exchanges of the inverse, undone at the end.  Returns log|det M| and
// its sign/phase; *singular is set when a pivot is exactly zero.
template <typename T>
struct GJSmem {
    T sS[GB][64];
    T sPan[64][GB + 1];
    T tile[32][33];
};

// Eliminates columns [c_lo, c_hi) of M (all rows) in panels of GB columns,
// applying each panel's row exchanges and rank-GB transform to the other
// columns of [j_lo, j_hi) only.  Pivot rows go to perm[k]; log|pivot| and the
// sign/phase accumulate into the shared s_log / s_sgn, a zero pivot sets
// s_sing.  The full inverse is c = j = [0, n); the tensor-core refresh runs it
// on one 64-column panel at a time and updates the other columns itself.
template <typename T>
__device__ void gj_columns(T* M, int n, int c_lo, int c_hi, int j_lo, int j_hi, int* perm, double& s_log, T& s_sgn,
                           int& s_sing, GJSmem<T>& sm) {
    __shared__ double s_v[32];
    __shared__ int s_i[32];
    __shared__ T s_rowk[GB];
    auto& sS = sm.sS;
    auto& sPan = sm.sPan;
    const int tid = threadIdx.x;

    for (int k0 = c_lo; k0 < c_hi; k0 += GB) {
        const int bw = min(GB, c_hi - k0);
        // ---- panel ----
        for (int kc = 0; kc < bw; ++kc) {
            const int k = k0 + kc;
            double best = -1.0;
            int bi = -1;
            for (int i = k + tid; i < n; i += RT) {
                double v = (double)s_abs2(M[(long long)i * n + k]);
                if (v > best) { best = v; bi = i; }
            }
            double bv;
            int p;
            block_argmax(best, bi, s_v, s_i, bv, p);
            if (!(bv > 0.0) || p < 0) {
                if (tid == 0) { perm[k] = k; s_sing = 1; }
                __syncthreads();
                continue;
            }
            if (tid == 0) perm[k] = p;
            if (p != k && tid < bw) {
                T a = M[(long long)k * n + k0 + tid];
                M[(long long)k * n + k0 + tid] = M[(long long)p * n + k0 + tid];
                M[(long long)p * n + k0 + tid] = a;
            }
            __syncthreads();
            const T piv = M[(long long)k * n + k];
            const T ipiv = s_recip(piv);
            if (tid < bw) {
                T v = (tid == kc) ? make_real<T>(1.0) : M[(long long)k * n + k0 + tid];
                v = v * ipiv;
                s_rowk[tid] = v;
                M[(long long)k * n + k0 + tid] = v;
            }
            if (tid == 0) {
                s_log += log(s_absd(piv));
                T sg = s_sgn * s_unit(piv);
                s_sgn = (p != k) ? s_neg(sg) : sg;
            }
            __syncthreads();
            for (int i = tid; i < n; i += RT) {
                if (i == k) continue;
                T* row = M + (long long)i * n + k0;
                const T f = row[kc];
                for (int c = 0; c < bw; ++c) {
                    T v = (c == kc) ? s_zero(T()) : row[c];
                    row[c] = s_fms(f, s_rowk[c], v);
                }
            }
            __syncthreads();
        }
        // ---- the panel's row exchanges on the other columns ----
        for (int kc = 0; kc < bw; ++kc) {
            const int k = k0 + kc, p = perm[k];
            if (p != k)
                for (int j = j_lo + tid; j < j_hi; j += RT) {
                    if (j >= k0 && j < k0 + bw) continue;
                    T a = M[(long long)k * n + j];
                    M[(long long)k * n + j] = M[(long long)p * n + j];
                    M[(long long)p * n + j] = a;
                }
            __syncthreads();
        }
        // ---- rank-bw update of the other columns: M += (panel - E) S ----
        const int tx = tid & 15, ty = tid >> 4;   // 16 x 16 threads, 4 x 4 outputs each
        for (int j0 = j_lo; j0 < j_hi; j0 += 64) {
            for (int e = tid; e < GB * 64; e += RT) {
                const int c = e / 64, jj = e % 64;
                sS[c][jj] = (c < bw && j0 + jj < j_hi) ? M[(long long)(k0 + c) * n + j0 + jj] : s_zero(T());
            }
            __syncthreads();
            for (int i0 = 0; i0 < n; i0 += 64) {
                for (int e = tid; e < 64 * GB; e += RT) {
                    const int ii = e / GB, c = e % GB;
                    const int i = i0 + ii;
                    T v = s_zero(T());
                    if (c < bw && i < n) {
                        v = M[(long long)i * n + k0 + c];
                        if (i == k0 + c) v = v - make_real<T>(1.0);
                    }
                    sPan[ii][c] = v;
                }
                __syncthreads();
                T acc[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = s_zero(T());
                for (int cc = 0; cc < bw; ++cc) {
                    T a[4], b[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) a[r] = sPan[ty * 4 + r][cc];
#pragma unroll
                    for (int c = 0; c < 4; ++c) b[c] = sS[cc][tx * 4 + c];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[r][c] = s_fma(a[r], b[c], acc[r][c]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int i = i0 + ty * 4 + r;
                    if (i >= n) continue;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int j = j0 + tx * 4 + c;
                        if (j >= j_hi || (j >= k0 && j < k0 + bw)) continue;
                        M[(long long)i * n + j] = M[(long long)i * n + j] + acc[r][c];
                    }
                }
                __syncthreads();
            }
        }
    }
}

// In-place Gauss-Jordan inverse of M (see gj_columns), exchanges undone.
template <typename T>
__device__ void gj_invert(T* M, int n, int* perm, double* logabs_out, T* sgn_out, int* singular, GJSmem<T>& sm) {
    __shared__ double s_log;
    __shared__ T s_sgn;
    __shared__ int s_sing;
    const int tid = threadIdx.x;
    if (tid == 0) { s_log = 0.0; s_sgn = make_real<T>(1.0); s_sing = 0; }
    __syncthreads();
    gj_columns(M, n, 0, n, 0, n, perm, s_log, s_sgn, s_sing, sm);
    // ---- undo the exchanges as column exchanges, last first ----
    for (int k = n - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p != k)
            for (int i = tid; i < n; i += RT) {
                T a = M[(long long)i * n + k];
                M[(long long)i * n + k] = M[(long long)i * n + p];
                M[(long long)i * n + p] = a;
            }
        __syncthreads();
    }
    if (tid == 0) {
        *logabs_out = s_sing ? -INFINITY : s_log;
        *sgn_out = s_sing ? s_zero(T()) : s_renorm(s_sgn);
        *singular = s_sing;
    }
    __syncthreads();
}

// One CTA per (selected) walker.  target: ws slot of the CTA when ws != null
// (refresh with drift), else the state G itself.
template <typename T>
__global__ void __launch_bounds__(RT) k_refresh(DevLayout L, DevState<T> S, const T* A, const uint8_t* mask,
                                                 T* ws, int nws, double* drift, bool pf, bool delayed,
                                                 bool write_logdet) {
    extern __shared__ __align__(16) unsigned char dsm[];
    GJSmem<T>& sm = *reinterpret_cast<GJSmem<T>*>(dsm);
    __shared__ int perm[2048];
    __shared__ double s_l;
    __shared__ T s_s;
    __shared__ int s_sing;
    __shared__ double s_red[2][32];
    for (int w = blockIdx.x; w < L.W; w += gridDim.x) {
        if (mask && !mask[w]) continue;
        const int n = L.nw(w);
        T* G = S.G + L.mo(w);
        T* M = ws ? ws + (long long)blockIdx.x * (long long)L.n_max * L.n_max : G;
        load_transposed(M, A + L.mo(w), n, sm.tile);
        __syncthreads();
        gj_invert(M, n, perm, &s_l, &s_s, &s_sing, sm);
        if (pf) {
            // the inverse of a skew matrix is skew: keep it exactly so
            for (long long e = threadIdx.x; e < (long long)n * n; e += RT) {
                const int i = (int)(e / n), j = (int)(e % n);
                if (i < j) {
                    T h = s_half(M[(long long)i * n + j] - M[(long long)j * n + i]);
                    M[(long long)i * n + j] = h;
                    M[(long long)j * n + i] = s_neg(h);
                } else if (i == j) {
                    M[e] = s_zero(T());
                }
            }
            __syncthreads();
        }
        if (ws) {
            // drift of the tracked inverse, then replace it
            double num = 0.0, den = 0.0;
            const int kk = L.kv(w);
            const int cu = delayed ? S.tau[w] * kk : 0;
            const long long vo = L.vo(w);
            for (long long e = threadIdx.x; e < (long long)n * n; e += RT) {
                const int l = (int)(e / n), j = (int)(e % n);   // memory [l*n + j] = (A^{-1})_{jl}
                T tr = G[e];
                if (cu) {
                    const T* pr = S.P + (vo + j) * L.Kc;
                    const T* qr = S.Q + (vo + l) * L.Kc;
                    T s = s_zero(T());
                    for (int c = 0; c < cu; ++c) s = s_fma(pr[c], qr[c], s);
                    tr = pf ? tr + s : tr - s;
                }
                T f = M[e];
                num += (double)s_abs2(tr - f);
                den += (double)s_abs2(f);
                G[e] = f;
            }
            num = warp_sum(num);
            den = warp_sum(den);
            if ((threadIdx.x & 31) == 0) { s_red[0][threadIdx.x >> 5] = num; s_red[1][threadIdx.x >> 5] = den; }
            __syncthreads();
            if (threadIdx.x == 0) {
                double a = 0, b = 0;
                for (int q = 0; q < RT / 32; ++q) { a += s_red[0][q]; b += s_red[1][q]; }
                if (drift) drift[w] = b > 0 ? sqrt(a / b) : 0.0;
            }
        }
        if (threadIdx.x == 0) {
            if (write_logdet) {
                S.logabs[w] = s_l;
                S.sgn[w] = s_s;
            }
            if (delayed) S.tau[w] = 0;
            S.pst[w] = s_sing ? 1 : 5;   // 5: fresh, no pending proposal
        }
        __syncthreads();
    }
}

// Pfaffian of a skew n x n matrix (row-major copy in M) by Parlett-Reid
// elimination with pivoting (see small_pf for the step), one CTA per matrix.
template <typename T>
__device__ void pr_pfaffian(T* M, int n, double* logabs, T* sgn, T* s_tau, T* s_row) {
    __shared__ double s_v[32];
    __shared__ int s_i[32];
    __shared__ double s_log;
    __shared__ T s_sg;
    __shared__ int s_zero_pf;
    const int tid = threadIdx.x;
    if (tid == 0) { s_log = 0.0; s_sg = make_real<T>(1.0); s_zero_pf = (n & 1); }
    __syncthreads();
    for (int k = 0; k + 1 < n && !s_zero_pf; k += 2) {
        double best = -1.0;
        int bi = -1;
        for (int i = k + 1 + tid; i < n; i += RT) {
            double v = (double)s_abs2(M[(long long)i * n + k]);
            if (v > best) { best = v; bi = i; }
        }
        double bv;
        int p;
        block_argmax(best, bi, s_v, s_i, bv, p);
        if (!(bv > 0.0) || p < 0) {
            if (tid == 0) s_zero_pf = 1;
            __syncthreads();
            break;
        }
        if (p != k + 1) {
            // swap rows k+1, p, then columns k+1, p
            for (int j = tid; j < n; j += RT) {
                T a = M[(long long)(k + 1) * n + j];
                M[(long long)(k + 1) * n + j] = M[(long long)p * n + j];
                M[(long long)p * n + j] = a;
            }
            __syncthreads();
            for (int i = tid; i < n; i += RT) {
                T a = M[(long long)i * n + k + 1];
                M[(long long)i * n + k + 1] = M[(long long)i * n + p];
                M[(long long)i * n + p] = a;
            }
        }
        __syncthreads();
        const T akk1 = M[(long long)k * n + k + 1];
        if (tid == 0) {
            s_log += log(s_absd(akk1));
            T sg = s_sg * s_unit(akk1);
            s_sg = (p != k + 1) ? s_neg(sg) : sg;
        }
        const T ipiv = s_recip(M[(long long)(k + 1) * n + k]);
        for (int i = k + 2 + tid; i < n; i += RT) {
            s_tau[i] = M[(long long)i * n + k] * ipiv;
            s_row[i] = M[(long long)(k + 1) * n + i];
        }
        __syncthreads();
        const int m = n - k - 2;
        for (long long e = tid; e < (long long)m * m; e += RT) {
            const int i = k + 2 + (int)(e / m), j = k + 2 + (int)(e % m);
            T v = s_fms(s_tau[i], s_row[j], M[(long long)i * n + j]);
            M[(long long)i * n + j] = s_fma(s_tau[j], s_row[i], v);
        }
        __syncthreads();
    }
    if (tid == 0) {
        *logabs = s_zero_pf ? -INFINITY : s_log;
        *sgn = s_zero_pf ? s_zero(T()) : s_renorm(s_sg);
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(RT) k_slogpf(DevLayout L, const T* A, const uint8_t* mask, T* ws,
                                                double* logabs, T* sgn) {
    extern __shared__ __align__(16) unsigned char dsm[];
    T* s_tau = reinterpret_cast<T*>(dsm);
    T* s_row = s_tau + 2048;
    __shared__ double s_l;
    __shared__ T s_s;
    for (int w = blockIdx.x; w < L.W; w += gridDim.x) {
        if (mask && !mask[w]) continue;
        const int n = L.nw(w);
        T* M = ws + (long long)blockIdx.x * (long long)L.n_max * L.n_max;
        const T* Aw = A + L.mo(w);
        for (long long e = threadIdx.x; e < (long long)n * n; e += RT) M[e] = Aw[e];
        __syncthreads();
        pr_pfaffian(M, n, &s_l, &s_s, s_tau, s_row);
        if (threadIdx.x == 0) {
            logabs[w] = s_l;
            sgn[w] = s_s;
        }
        __syncthreads();
    }
}

// standalone slogdet (GJ on a workspace copy)
template <typename T>
__global__ void __launch_bounds__(RT) k_slogdet(int W, int n, const T* A, T* ws, double* logabs, T* sgn) {
    extern __shared__ __align__(16) unsigned char dsm[];
    GJSmem<T>& sm = *reinterpret_cast<GJSmem<T>*>(dsm);
    __shared__ int perm[2048];
    __shared__ double s_l;
    __shared__ T s_s;
    __shared__ int s_sing;
    for (int w = blockIdx.x; w < W; w += gridDim.x) {
        T* M = ws + (long long)blockIdx.x * n * n;
        const T* Aw = A + (long long)w * n * n;
        for (long long e = threadIdx.x; e < (long long)n * n; e += RT) M[e] = Aw[e];
        __syncthreads();
        gj_invert(M, n, perm, &s_l, &s_s, &s_sing, sm);
        if (threadIdx.x == 0) {
            logabs[w] = s_l;
            sgn[w] = s_s;
        }
        __syncthreads();
    }
}

template <typename T>
void launch_refresh(bool pf, bool delayed, const DevLayout& L, const DevState<T>& S, const T* A,
                    const uint8_t* mask, T* ws, int nws, double* drift, bool write_logdet, cudaStream_t st) {
    const int grid = ws ? nws : L.W;
    const int dyn = (int)sizeof(GJSmem<T>);
    cudaFuncSetAttribute(k_refresh<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    k_refresh<T><<<grid, RT, dyn, st>>>(L, S, A, mask, ws, nws, drift, pf, delayed, write_logdet);
}

template <typename T>
void launch_slogpf(const DevLayout& L, const T* A, const uint8_t* mask, T* ws, int nws, double* logabs, T* sgn,
                   cudaStream_t st) {
    const int dyn = (int)(2 * 2048 * sizeof(T));
    cudaFuncSetAttribute(k_slogpf<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    k_slogpf<T><<<nws, RT, dyn, st>>>(L, A, mask, ws, logabs, sgn);
}

template <typename T>
void launch_slogdet(int W, int n, const T* A, T* ws, int nws, double* logabs, T* sgn, cudaStream_t st) {
    const int dyn = (int)sizeof(GJSmem<T>);
    cudaFuncSetAttribute(k_slogdet<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    k_slogdet<T><<<nws, RT, dyn, st>>>(W, n, A, ws, logabs, sgn);
}

// ---------------------------------------------------------------------------
// FP64 parts of the tensor-core refresh (the GEMM is in refresh_oz.cu)
// ---------------------------------------------------------------------------

// M[w] = A[w]^T through 32 x 32 tiles; grid (n/32, n/32, W), block 32 x 8
__global__ void k_oz_load(int n, const double* A, double* M, const uint8_t* mask) {
    __shared__ double tile[32][33];
    const int w = blockIdx.z;
    if (mask && !mask[w]) return;
    const long long off = (long long)w * n * n;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32, tx = threadIdx.x;
    for (int q = threadIdx.y; q < 32; q += 8) tile[q][tx] = A[off + (long long)(r0 + q) * n + c0 + tx];
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += 8) M[off + (long long)(c0 + q) * n + r0 + tx] = tile[tx][q];
}

// Panel [k0, k0 + OZ_B) of walker w: Gauss-Jordan elimination of its columns
// over all rows (updates confined to the panel), then its row exchanges
// applied, in pivot order, to every column outside the panel.  log|pivot|
// and the sign carry over between panels in Z.logacc / Z.sgnacc / Z.sing.
__global__ void __launch_bounds__(RT) k_oz_panel(int n, int k0, int w0, OzWork Z, const uint8_t* mask) {
    extern __shared__ __align__(16) unsigned char dsm[];
    GJSmem<double>& sm = *reinterpret_cast<GJSmem<double>*>(dsm);
    __shared__ double s_log, s_sgn;
    __shared__ int s_sing;
    const int w = w0 + blockIdx.x;
    if (mask && !mask[w]) return;
    double* M = Z.M + (long long)w * n * n;
    int* perm = Z.perm + (long long)w * n;
    if (threadIdx.x == 0) {
        s_log = k0 ? Z.logacc[w] : 0.0;
        s_sgn = k0 ? Z.sgnacc[w] : 1.0;
        s_sing = k0 ? Z.sing[w] : 0;
    }
    __syncthreads();
    gj_columns<double>(M, n, k0, k0 + OZ_B, k0, k0 + OZ_B, perm, s_log, s_sgn, s_sing, sm);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += RT) {
        if (j >= k0 && j < k0 + OZ_B) continue;
        for (int kc = 0; kc < OZ_B; ++kc) {
            const int k = k0 + kc, p = perm[k];
            if (p != k) {
                const double a = M[(long long)k * n + j];
                M[(long long)k * n + j] = M[(long long)p * n + j];
                M[(long long)p * n + j] = a;
            }
        }
    }
    if (threadIdx.x == 0) {
        Z.logacc[w] = s_log;
        Z.sgnacc[w] = s_sgn;
        Z.sing[w] = s_sing;
    }
}

// One SW-column sub-panel of panel [k0, k0 + OZ_B) with the rows in registers
// (SW = 16 for n <= 1024, 8 up to n = 2048): thread t owns rows t + q * blockDim
// (q < RPT, blockDim = n / RPT).  The sub-panel is eliminated in registers (pivot by a block reduction,
// row swaps through shared memory) and its transform columns written back;
// its row exchanges are then applied to the other panel columns, whose update
// by the transform is a split product on the tensor cores (refresh_oz.cu).
// The last sub-panel of a panel also applies the panel's exchanges, in pivot
// order, to the columns outside it.  Pivots go to Z.piv (log|det| and the
// sign are summed at the end).
template <int RPT, int SW>
__global__ void __launch_bounds__(512, 1) k_oz_subpanel_rows(int n, int k0, int sp, OzWork Z, const uint8_t* mask) {
    static_assert(SW % 2 == 0 && OZ_B % SW == 0, "sub-panel width");
    __shared__ double s_rowk[SW], s_bufA[SW], s_bufB[SW];
    __shared__ unsigned long long s_wk[16];
    __shared__ int s_wi[16];
    __shared__ int s_sing;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    const int w = blockIdx.x;
    if (mask && !mask[w]) return;
    double* M = Z.M + (long long)w * n * n;
    int* perm = Z.perm + (long long)w * n;
    if (tid == 0) s_sing = (k0 || sp) ? Z.sing[w] : 0;
    __syncthreads();
    {
        const int ks = k0 + SW * sp;
        double v[RPT][SW];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const double2* src = reinterpret_cast<const double2*>(M + (long long)(tid + q * nt) * n + ks);
#pragma unroll
            for (int c = 0; c < SW / 2; ++c) {
                const double2 x = src[c];
                v[q][2 * c] = x.x;
                v[q][2 * c + 1] = x.y;
            }
        }
#pragma unroll
        for (int kc = 0; kc < SW; ++kc) {
            const int k = ks + kc;
            // ---- pivot: largest |v| over rows >= k (ties: smallest row) ----
            // |v| is compared through its bit pattern (a non-negative double
            // orders like its bits as an unsigned integer), so the search runs on
            // the integer pipe and leaves the FP64 pipe to the elimination; NaN
            // counts as 0.  Every warp then reduces the per-warp winners itself,
            // so the pivot costs one barrier.
            unsigned long long bk = 0ull;
            int bi = -1;
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int r = tid + q * nt;
                unsigned long long a = (unsigned long long)__double_as_longlong(v[q][kc]) & 0x7FFFFFFFFFFFFFFFull;
                if (a > 0x7FF0000000000000ull) a = 0ull;
                if (r >= k && (bi < 0 || a > bk)) { bk = a; bi = r; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (oi >= 0 && (bi < 0 || ok > bk || (ok == bk && oi < bi))) { bk = ok; bi = oi; }
            }
            if (lane == 0) { s_wk[wid] = bk; s_wi[wid] = bi; }
            __syncthreads();
            bk = 0ull;
            bi = -1;
            for (int q = 0; q < nt / 32; ++q) {
                const unsigned long long ok = s_wk[q];
                const int oi = s_wi[q];
                if (oi >= 0 && (bi < 0 || ok > bk || (ok == bk && oi < bi))) { bk = ok; bi = oi; }
            }
            const int p = bi;
            if (bk == 0ull || p < 0) {
                if (tid == 0) { perm[k] = k; s_sing = 1; Z.piv[(long long)w * n + k] = 0.0; }
                __syncthreads();   // every thread has read s_wk before the next pivot writes it
                continue;
            }
            if (tid == 0) perm[k] = p;
            const int tk = k % nt, qk = k / nt, tp = p % nt, qp = p / nt;
            // ---- rows p (the pivot row) and k to shared memory ----
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                if (tid == tp && q == qp)
#pragma unroll
                    for (int c = 0; c < SW; ++c) s_bufA[c] = v[q][c];
                if (p != k && tid == tk && q == qk)
#pragma unroll
                    for (int c = 0; c < SW; ++c) s_bufB[c] = v[q][c];
            }
            __syncthreads();
            // ---- scale the pivot row: 16 threads, one element each; the pivot
            //      is recorded (log|det| and the sign are summed at the end) ----
            if (tid < SW) {
                const double piv = s_bufA[kc];
                s_rowk[tid] = (tid == kc ? 1.0 : s_bufA[tid]) / piv;
                if (tid == 0) Z.piv[(long long)w * n + k] = piv;
            }
            __syncthreads();
            // ---- exchange: row k becomes the scaled pivot row, row p the old row k ----
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                if (tid == tk && q == qk)
#pragma unroll
                    for (int c = 0; c < SW; ++c) v[q][c] = s_rowk[c];
                else if (p != k && tid == tp && q == qp)
#pragma unroll
                    for (int c = 0; c < SW; ++c) v[q][c] = s_bufB[c];
            }
            // ---- eliminate column k from every other row ----
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int r = tid + q * nt;
                if (r != k) {
                    const double f = v[q][kc];
#pragma unroll
                    for (int c = 0; c < SW; ++c) v[q][c] = fma(-f, s_rowk[c], c == kc ? 0.0 : v[q][c]);
                }
            }
        }
        // ---- the sub-panel's transform columns back to M ----
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            double2* dst = reinterpret_cast<double2*>(M + (long long)(tid + q * nt) * n + ks);
#pragma unroll
            for (int c = 0; c < SW / 2; ++c) dst[c] = make_double2(v[q][2 * c], v[q][2 * c + 1]);
        }
        __syncthreads();
        // ---- this sub-panel's exchanges on the other panel columns ----
        for (int t = tid; t < OZ_B - SW; t += nt) {
            const int col = k0 + t + (t >= SW * sp ? SW : 0);
            for (int kc = 0; kc < SW; ++kc) {
                const int kk = ks + kc, p = perm[kk];
                if (p != kk) {
                    const double a = M[(long long)kk * n + col];
                    M[(long long)kk * n + col] = M[(long long)p * n + col];
                    M[(long long)p * n + col] = a;
                }
            }
        }
    }
    // ---- last sub-panel: the panel's exchanges on the columns outside it ----
    // The 64 exchanges (k, perm[k]), applied in pivot order, compose into one
    // permutation of at most 128 rows: row r receives the old row src[r].  It
    // is built once in shared memory; then every 32-column tile of those rows
    // is gathered into shared memory (independent, coalesced loads) and
    // written back permuted, instead of 64 dependent swaps per column.
    if (sp == OZ_B / SW - 1) {
        __shared__ int s_src[2048];            // n <= 2048 for this kernel
        __shared__ int s_from[2 * OZ_B], s_to[2 * OZ_B];
        __shared__ int s_cnt;
        __shared__ double s_xb[2 * OZ_B][33];
        for (int r = tid; r < n; r += nt) s_src[r] = r;
        if (tid == 0) s_cnt = 0;
        __syncthreads();
        if (tid == 0)
            for (int kc = 0; kc < OZ_B; ++kc) {
                const int k = k0 + kc, p = perm[k];
                const int a = s_src[k];
                s_src[k] = s_src[p];
                s_src[p] = a;
            }
        __syncthreads();
        for (int r = tid; r < n; r += nt)
            if (s_src[r] != r) {
                const int e = atomicAdd(&s_cnt, 1);   // at most 2 * OZ_B rows move
                s_to[e] = r;
                s_from[e] = s_src[r];
            }
        __syncthreads();
        const int cnt = s_cnt;
        for (int j0 = 0; j0 < n && cnt > 0; j0 += 32) {
            if (j0 >= k0 && j0 < k0 + OZ_B) continue;   // the panel's own columns (64-aligned)
            // eight independent loads per thread in flight before any store
            for (int e0 = tid; e0 < cnt * 32; e0 += 8 * nt) {
                double x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + u * nt;
                    x[u] = e < cnt * 32 ? M[(long long)s_from[e >> 5] * n + j0 + (e & 31)] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + u * nt;
                    if (e < cnt * 32) s_xb[e >> 5][e & 31] = x[u];
                }
            }
            __syncthreads();
            for (int e = tid; e < cnt * 32; e += nt) {
                const int q = e >> 5, jj = e & 31;
                M[(long long)s_to[q] * n + j0 + jj] = s_xb[q][jj];
            }
            __syncthreads();
        }
    }
    if (tid == 0) Z.sing[w] = s_sing;
}

// Undo the row exchanges of the elimination as one column permutation of
// the inverse (idx composes the swaps, last first: M'[i][c] = M[i][idx[c]]),
// four rows at a time through shared memory; then log|det|, sign and the
// fresh-state flags.
__global__ void __launch_bounds__(RT) k_oz_finish(int n, OzWork Z, DevState<double> S, const uint8_t* mask,
                                                  bool delayed, bool reset_tau) {
    extern __shared__ __align__(16) unsigned char dsm[];
    double* buf = reinterpret_cast<double*>(dsm);
    int* idx = reinterpret_cast<int*>(buf + 4 * n);
    const int w = blockIdx.x;
    if (mask && !mask[w]) return;
    const int* perm = Z.perm + (long long)w * n;
    for (int c = threadIdx.x; c < n; c += RT) idx[c] = c;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = n - 1; k >= 0; --k) {
            const int p = perm[k];
            if (p != k) { const int t = idx[k]; idx[k] = idx[p]; idx[p] = t; }
        }
    __syncthreads();
    double* M = Z.M + (long long)w * n * n;
    for (int i0 = 0; i0 < n; i0 += 4) {
        const int rows = min(4, n - i0);
        for (int e = threadIdx.x; e < rows * n; e += RT) buf[e] = M[(long long)i0 * n + e];
        __syncthreads();
        for (int e = threadIdx.x; e < rows * n; e += RT) {
            const int r = e / n, c = e % n;
            M[(long long)(i0 + r) * n + c] = buf[r * n + idx[c]];
        }
        __syncthreads();
    }
    double la = 0.0;
    int neg = 0;
    const bool piv_rec = n <= OZ_SUBPANEL_MAX_N;   // the sub-panel path records the pivots
    if (piv_rec) {
        // log|det| = sum log|pivot|, sign = prod sign(pivot) * (-1)^(row exchanges)
        const double* pv = Z.piv + (long long)w * n;
        for (int k = threadIdx.x; k < n; k += RT) {
            const double x = pv[k];
            la += log(fabs(x));
            neg += (x < 0.0) + (perm[k] != k);
        }
        la = block_sum(la, buf);
    }
    __shared__ int s_neg;
    if (threadIdx.x == 0) s_neg = 0;
    __syncthreads();
    if (neg & 1) atomicXor(&s_neg, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int sing = Z.sing[w];
        const double lg = piv_rec ? la : Z.logacc[w];
        const double sg = piv_rec ? (s_neg ? -1.0 : 1.0) : Z.sgnacc[w];
        S.logabs[w] = sing ? -INFINITY : lg;
        S.sgn[w] = sing ? 0.0 : s_renorm(sg);
        if (delayed && reset_tau) S.tau[w] = 0;
        S.pst[w] = sing ? 1 : 5;
    }
}

// Drift of the tracked inverse against the fresh one in M (relative
// Frobenius norm; the delayed form's pending slots are applied on the fly,
// A^{-1} = A_0^{-1} - P Q^T), then M replaces the state and tau is reset.
__global__ void __launch_bounds__(RT) k_oz_drift_store(int n, DevLayout L, DevState<double> S, const double* M,
                                                       const uint8_t* mask, double* drift, bool delayed) {
    __shared__ double s_red[32];
    const int w = blockIdx.x;
    if (mask && !mask[w]) return;
    const long long off = (long long)w * n * n;
    const long long vo = (long long)w * n;
    const int cu = delayed ? S.tau[w] * L.kk : 0;
    double num = 0.0, den = 0.0;
    for (long long e = threadIdx.x; e < (long long)n * n; e += RT) {
        const int l = (int)(e / n), j = (int)(e % n);   // storage [l * n + j] = (A^{-1})_{jl}
        double tr = S.G[off + e];
        if (cu) {
            const double* pr = S.P + (vo + j) * L.Kc;
            const double* qr = S.Q + (vo + l) * L.Kc;
            double sm = 0.0;
            for (int c = 0; c < cu; ++c) sm = fma(pr[c], qr[c], sm);
            tr -= sm;
        }
        const double f = M[off + e];
        num += (tr - f) * (tr - f);
        den += f * f;
        S.G[off + e] = f;
    }
    num = block_sum(num, s_red);
    den = block_sum(den, s_red);
    if (threadIdx.x == 0) {
        if (drift) drift[w] = den > 0 ? sqrt(num / den) : 0.0;
        if (delayed) S.tau[w] = 0;
    }
}

void launch_oz_drift_store(int W, int n, const DevLayout& L, const DevState<double>& S, const double* M,
                           const uint8_t* mask, double* drift, bool delayed, cudaStream_t st) {
    k_oz_drift_store<<<W, RT, 0, st>>>(n, L, S, M, mask, drift, delayed);
}

void launch_oz_load(int W, int n, const double* A, double* M, const uint8_t* mask, cudaStream_t st) {
    k_oz_load<<<dim3(n / 32, n / 32, W), dim3(32, 8), 0, st>>>(n, A, M, mask);
}

int oz_subpanel_width(int n) { return n <= 1024 ? 16 : 8; }

bool launch_oz_subpanel(int W, int n, int k0, int sp, const OzWork& Z, const uint8_t* mask, cudaStream_t st) {
    if (n <= 512) {
        k_oz_subpanel_rows<1, 16><<<W, n, 0, st>>>(n, k0, sp, Z, mask);
        return true;
    }
    if (n <= 1024) {
        k_oz_subpanel_rows<2, 16><<<W, n / 2, 0, st>>>(n, k0, sp, Z, mask);
        return true;
    }
    if (n <= OZ_SUBPANEL_MAX_N && n % 4 == 0) {
        // four rows of eight sub-panel columns per thread keep the registers
        // of the 16-column form
        k_oz_subpanel_rows<4, 8><<<W, n / 4, 0, st>>>(n, k0, sp, Z, mask);
        return true;
    }
    return false;
}

void launch_oz_panel(int W, int w0, int n, int k0, const OzWork& Z, const uint8_t* mask, cudaStream_t st) {
    const int dyn = (int)sizeof(GJSmem<double>);
    cudaFuncSetAttribute(k_oz_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    k_oz_panel<<<W, RT, dyn, st>>>(n, k0, w0, Z, mask);
}

void launch_oz_finish(int W, int n, const OzWork& Z, const DevState<double>& S, const uint8_t* mask, bool delayed,
                      bool reset_tau, cudaStream_t st) {
    const int dyn = (int)(4 * n * sizeof(double) + n * sizeof(int));
    cudaFuncSetAttribute(k_oz_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    k_oz_finish<<<W, RT, dyn, st>>>(n, Z, S, mask, delayed, reset_tau);
}

#define LRU_INST_R(T)                                                                                       \
    template void launch_refresh<T>(bool, bool, const DevLayout&, const DevState<T>&, const T*,            \
                                    const uint8_t*, T*, int, double*, bool, cudaStream_t);                 \
    template void launch_slogpf<T>(const DevLayout&, const T*, const uint8_t*, T*, int, double*, T*,       \
                                   cudaStream_t);                                                          \
    template void launch_slogdet<T>(int, int, const T*, T*, int, double*, T*, cudaStream_t);

LRU_INST_R(double)
LRU_INST_R(float)
LRU_INST_R(c128)
LRU_INST_R(c64)

}  // namespace lru

// ---------------------------------------------------------------------------
// slogdet without any allocation (lru_slogdet_batched_noalloc)
//
// Some callers cannot let a library allocate device memory: runtimes that
// preallocate most of the GPU for their own pool (so a cudaMalloc can fail),
// code that must not hit the device-wide synchronisation of cudaFree, and
// callers that record work for later replay.  This entry point runs the same
// Gauss-Jordan kernel as lru_slogdet_batched, with its per-CTA matrix
// workspace taken from the fixed array below instead of cudaMallocAsync.
// ---------------------------------------------------------------------------

#include <mutex>
#include <stdint.h>

#include "../../include/lrugb.h"

namespace lru {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(64) << 20;   // 64 MiB, held by every GPU that loads the library

// The workspace.  Host code may not use this name as a device address: the
// address comes from cudaGetSymbolAddress, per device, in noalloc_scratch().
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the workspace on the current device; looked up once per
// device, with that device current.  Returns nullptr if the lookup failed.
static void* noalloc_scratch(int dev) {
    constexpr int MAXDEV = 64;
    static std::mutex mu;
    static void* addr[MAXDEV] = {};
    static bool done[MAXDEV] = {};
    if (dev < 0 || dev >= MAXDEV) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;   // not cached: the next call tries again
        }
        addr[dev] = p;
        done[dev] = true;
    }
    return addr[dev];
}

}  // namespace lru

extern "C" lru_status lru_slogdet_batched_noalloc(int32_t dtype, int64_t W, int32_t n, const void* A,
                                                  double* logabs, void* sign, void* stream) {
    using namespace lru;
    size_t sz = 0;
    switch (dtype) {
        case LRU_F64: sz = 8; break;
        case LRU_C128: sz = 16; break;
        case LRU_F32: sz = 4; break;
        case LRU_C64: sz = 8; break;
        default: return LRU_ERR_ARG;
    }
    if (W < 1 || W > (int64_t)INT32_MAX || n < 1 || n > 2048 || !A || !logabs || !sign) return LRU_ERR_ARG;
    const size_t per = (size_t)n * n * sz;
    if (per > NOALLOC_SCRATCH_BYTES) return LRU_ERR_ARG;   // one matrix must fit the workspace
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return LRU_ERR_CUDA; }
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        nsm = 148;
    }
    void* ws = noalloc_scratch(dev);
    if (!ws) return LRU_ERR_CUDA;
    long long slots = (long long)(NOALLOC_SCRATCH_BYTES / per);
    slots = std::min<long long>(slots, std::min<long long>(W, 2LL * nsm));
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case LRU_F64: launch_slogdet<double>((int)W, n, (const double*)A, (double*)ws, (int)slots, logabs, (double*)sign, st); break;
        case LRU_C128: launch_slogdet<c128>((int)W, n, (const c128*)A, (c128*)ws, (int)slots, logabs, (c128*)sign, st); break;
        case LRU_F32: launch_slogdet<float>((int)W, n, (const float*)A, (float*)ws, (int)slots, logabs, (float*)sign, st); break;
        case LRU_C64: launch_slogdet<c64>((int)W, n, (const c64*)A, (c64*)ws, (int)slots, logabs, (c64*)sign, st); break;
    }
    return cudaGetLastError() == cudaSuccess ? LRU_OK : LRU_ERR_CUDA;
}
