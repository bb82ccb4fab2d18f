// Shared device helpers of the CUDA path: scalar types, warp reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define LRU_HD __host__ __device__ __forceinline__
#define LRU_D __device__ __forceinline__

namespace lru {

// ---------------------------------------------------------------------------
// complex scalar with plain (non-conjugating) arithmetic; 2*sizeof(R) aligned
// ---------------------------------------------------------------------------
template <typename R>
struct alignas(2 * sizeof(R)) cplx {
    R re, im;
};
using c128 = cplx<double>;
using c64 = cplx<float>;

template <typename T> struct traits;
template <> struct traits<double> {
    using real = double;
    static constexpr bool is_complex = false;
};
template <> struct traits<float> {
    using real = float;
    static constexpr bool is_complex = false;
};
template <> struct traits<c128> {
    using real = double;
    static constexpr bool is_complex = true;
};
template <> struct traits<c64> {
    using real = float;
    static constexpr bool is_complex = true;
};

// real ops
LRU_HD double s_zero(double) { return 0.0; }
LRU_HD float s_zero(float) { return 0.f; }
template <typename R> LRU_HD cplx<R> s_zero(cplx<R>) { return {R(0), R(0)}; }

template <typename T> LRU_HD T make_real(double x);
template <> LRU_HD double make_real<double>(double x) { return x; }
template <> LRU_HD float make_real<float>(double x) { return (float)x; }
template <> LRU_HD c128 make_real<c128>(double x) { return {x, 0.0}; }
template <> LRU_HD c64 make_real<c64>(double x) { return {(float)x, 0.f}; }

template <typename R> LRU_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> LRU_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> LRU_HD cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <typename R> LRU_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> LRU_HD cplx<R> operator*(R s, cplx<R> a) { return {s * a.re, s * a.im}; }

// fused multiply-add d + a*b
LRU_D double s_fma(double a, double b, double d) { return fma(a, b, d); }
LRU_D float s_fma(float a, float b, float d) { return fmaf(a, b, d); }
template <typename R> LRU_D cplx<R> s_fma(cplx<R> a, cplx<R> b, cplx<R> d) {
    cplx<R> r;
    r.re = fma(a.re, b.re, fma(-a.im, b.im, d.re));
    r.im = fma(a.re, b.im, fma(a.im, b.re, d.im));
    return r;
}
// d - a*b
LRU_D double s_fms(double a, double b, double d) { return fma(-a, b, d); }
LRU_D float s_fms(float a, float b, float d) { return fmaf(-a, b, d); }
template <typename R> LRU_D cplx<R> s_fms(cplx<R> a, cplx<R> b, cplx<R> d) {
    cplx<R> r;
    r.re = fma(-a.re, b.re, fma(a.im, b.im, d.re));
    r.im = fma(-a.re, b.im, fma(-a.im, b.re, d.im));
    return r;
}

LRU_HD double s_abs2(double a) { return a * a; }
LRU_HD float s_abs2(float a) { return a * a; }
template <typename R> LRU_HD R s_abs2(cplx<R> a) { return a.re * a.re + a.im * a.im; }
LRU_D double s_absd(double a) { return fabs(a); }
LRU_D double s_absd(float a) { return fabs((double)a); }
template <typename R> LRU_D double s_absd(cplx<R> a) { return hypot((double)a.re, (double)a.im); }

LRU_D bool s_isfinite(double a) { return isfinite(a); }
LRU_D bool s_isfinite(float a) { return isfinite(a); }
template <typename R> LRU_D bool s_isfinite(cplx<R> a) { return isfinite(a.re) && isfinite(a.im); }

LRU_D double s_recip(double a) { return 1.0 / a; }
LRU_D float s_recip(float a) { return 1.0f / a; }
template <typename R> LRU_D cplx<R> s_recip(cplx<R> a) {
    // 1/a = conj(a)/|a|^2 with a scaling step against overflow
    R s = fmax(fabs(a.re), fabs(a.im));
    R ar = a.re / s, ai = a.im / s;
    R d = ar * ar + ai * ai;
    return {ar / (d * s), -ai / (d * s)};
}
// negation as a flip of the sign bit with an integer instruction: a
// materialised FP64 negation would take a slot of the (narrow) FP64 pipe
LRU_D double s_neg(double a) {
    return __hiloint2double(__double2hiint(a) ^ (int)0x80000000, __double2loint(a));
}
LRU_D float s_neg(float a) { return __int_as_float(__float_as_int(a) ^ (int)0x80000000); }
template <typename R> LRU_D cplx<R> s_neg(cplx<R> a) { return {s_neg(a.re), s_neg(a.im)}; }
LRU_D double s_half(double a) { return 0.5 * a; }
LRU_D float s_half(float a) { return 0.5f * a; }
template <typename R> LRU_D cplx<R> s_half(cplx<R> a) { return {R(0.5) * a.re, R(0.5) * a.im}; }

// unit "sign" of a nonzero scalar: +-1 for real, a/|a| for complex
LRU_D double s_unit(double a) { return a < 0 ? -1.0 : 1.0; }
LRU_D float s_unit(float a) { return a < 0 ? -1.f : 1.f; }
template <typename R> LRU_D cplx<R> s_unit(cplx<R> a) {
    double h = hypot((double)a.re, (double)a.im);
    return {(R)(a.re / h), (R)(a.im / h)};
}
// renormalise a unit phase (real: snap to +-1)
LRU_D double s_renorm(double a) { return a < 0 ? -1.0 : (a > 0 ? 1.0 : 0.0); }
LRU_D float s_renorm(float a) { return a < 0 ? -1.f : (a > 0 ? 1.f : 0.f); }
template <typename R> LRU_D cplx<R> s_renorm(cplx<R> a) {
    double h = hypot((double)a.re, (double)a.im);
    if (h == 0) return a;
    return {(R)(a.re / h), (R)(a.im / h)};
}

// warp reductions (xor butterfly: every lane ends with the total)
LRU_D double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
LRU_D float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename R> LRU_D cplx<R> warp_sum(cplx<R> v) {
    v.re = warp_sum(v.re);
    v.im = warp_sum(v.im);
    return v;
}
template <typename T> LRU_D T shfl(T v, int src) {
    if constexpr (traits<T>::is_complex) {
        v.re = __shfl_sync(0xffffffffu, v.re, src);
        v.im = __shfl_sync(0xffffffffu, v.im, src);
        return v;
    } else {
        return __shfl_sync(0xffffffffu, v, src);
    }
}

// block-wide sum with a caller-provided shared buffer of >= 32 T
template <typename T> __device__ T block_sum(T v, T* sbuf) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sbuf[wid] = v;
    __syncthreads();
    T t = (threadIdx.x < nw) ? sbuf[threadIdx.x] : s_zero(T());
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sbuf[0] = t;
    __syncthreads();
    T r = sbuf[0];
    __syncthreads();
    return r;
}

// sticky error codes written to the handle's device error word
enum : int { DEV_ERR_NONE = 0, DEV_ERR_TIMEOUT = 1, DEV_ERR_INDEX = 2, DEV_ERR_TMEM = 3, DEV_ERR_CANARY = 4 };
LRU_D void set_dev_error(int* flag, int code) {
    if (flag) atomicCAS(flag, 0, code);
}

// Debug build (-DLRU_DEBUG): checks of work-item indices against the sizes
// they address.  A failed check records DEV_ERR_INDEX in the sticky error word
// and the caller skips the work (no trap, no out-of-range access); `cond` must
// be the same for every thread of the CTA.  Release builds compile nothing.
#ifdef LRU_DEBUG
#define LRU_DEBUG_OK(cond, err) ((cond) ? true : (set_dev_error((err), DEV_ERR_INDEX), false))
#else
#define LRU_DEBUG_OK(cond, err) true
#endif

}  // namespace lru
