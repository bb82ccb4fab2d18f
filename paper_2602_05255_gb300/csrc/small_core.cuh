// Small dense cores of a low-rank update, run by one thread per walker:
// the k x k determinant core R (Sec. 2.1, Eqs. det_R, det_ratio) and the
// 2k x 2k skew Pfaffian core M (Sec. 3.1 Eqs. pf_ratio, pf_R; App. A.2 Eq.
// pf_low_rank).  k <= 8, so every routine works on a row-major matrix in
// shared or local memory.  Always run in the handle's dtype (FP64 / complex128
// for the double types).
#pragma once
#include "common.cuh"

namespace lru {

enum : int { CORE_OK = 0, CORE_SINGULAR = 1, CORE_NONFINITE = 2 };

// In-place Gauss-Jordan inverse with partial pivoting of the m x m row-major
// matrix a (stride lda).  det receives det(a).  On a zero pivot the routine
// stops with CORE_SINGULAR and det = 0 (the ratio of a node).
template <typename T>
LRU_D int small_gj_inverse(T* a, int m, int lda, T* det) {
    int swp[16];
    T d = make_real<T>(1.0);
    for (int k = 0; k < m; ++k) {
        int p = k;
        double best = (double)s_abs2(a[k * lda + k]);
        for (int i = k + 1; i < m; ++i) {
            double v = (double)s_abs2(a[i * lda + k]);
            if (v > best) { best = v; p = i; }
        }
        swp[k] = p;
        if (!(best > 0.0)) { *det = s_zero(T()); return CORE_SINGULAR; }
        if (p != k) {
            for (int j = 0; j < m; ++j) {
                T t = a[k * lda + j]; a[k * lda + j] = a[p * lda + j]; a[p * lda + j] = t;
            }
            d = s_neg(d);
        }
        T piv = a[k * lda + k];
        d = d * piv;
        T ip = s_recip(piv);
        a[k * lda + k] = make_real<T>(1.0);
        for (int j = 0; j < m; ++j) a[k * lda + j] = a[k * lda + j] * ip;
        for (int i = 0; i < m; ++i) {
            if (i == k) continue;
            T f = a[i * lda + k];
            a[i * lda + k] = s_zero(T());
            for (int j = 0; j < m; ++j) a[i * lda + j] = s_fms(f, a[k * lda + j], a[i * lda + j]);
        }
    }
    // the row exchanges become column exchanges of the inverse, undone last-first
    for (int k = m - 1; k >= 0; --k) {
        int p = swp[k];
        if (p != k)
            for (int i = 0; i < m; ++i) {
                T t = a[i * lda + k]; a[i * lda + k] = a[i * lda + p]; a[i * lda + p] = t;
            }
    }
    *det = d;
    return s_isfinite(d) ? CORE_OK : CORE_NONFINITE;
}

// Pfaffian of an m x m skew matrix by Parlett-Reid elimination with pivoting
// (Parlett & Reid, 1970).  Step k (k = 0, 2, 4, ...) moves the entry of
// largest modulus of column k below the diagonal to row k+1 (a congruence by a
// transposition, which flips the sign of pf by App. A.2 Eq. pf->det_pf), then
// clears rows k+2.. of column k with the unit-triangular congruence
// row_i -= t_i row_{k+1}, col_i -= t_i col_{k+1}, t_i = a_ik / a_{k+1,k}
// (determinant 1, pf unchanged).  Expanding along row k then gives
// pf(a) = a_{k,k+1} pf(trailing block).  a is destroyed.
template <typename T>
LRU_D T small_pf(T* a, int m, int lda) {
    if (m & 1) return s_zero(T());
    T pf = make_real<T>(1.0);
    for (int k = 0; k + 1 < m; k += 2) {
        int p = k + 1;
        double best = (double)s_abs2(a[(k + 1) * lda + k]);
        for (int i = k + 2; i < m; ++i) {
            double v = (double)s_abs2(a[i * lda + k]);
            if (v > best) { best = v; p = i; }
        }
        if (!(best > 0.0)) return s_zero(T());
        if (p != k + 1) {
            for (int j = 0; j < m; ++j) {
                T t = a[(k + 1) * lda + j]; a[(k + 1) * lda + j] = a[p * lda + j]; a[p * lda + j] = t;
            }
            for (int i = 0; i < m; ++i) {
                T t = a[i * lda + k + 1]; a[i * lda + k + 1] = a[i * lda + p]; a[i * lda + p] = t;
            }
            pf = s_neg(pf);
        }
        pf = pf * a[k * lda + k + 1];
        T ipiv = s_recip(a[(k + 1) * lda + k]);
        T tau[16];
        for (int i = k + 2; i < m; ++i) tau[i] = a[i * lda + k] * ipiv;
        for (int i = k + 2; i < m; ++i)
            for (int j = k + 2; j < m; ++j) {
                T v = s_fms(tau[i], a[(k + 1) * lda + j], a[i * lda + j]);
                a[i * lda + j] = s_fma(tau[j], a[(k + 1) * lda + i], v);
            }
    }
    return pf;
}

}  // namespace lru
