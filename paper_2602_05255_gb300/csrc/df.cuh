// Double-float arithmetic on the FP32 pipe for the FP64 data path.
//
// GB300 runs FP64 FMAs at about 1/70 of the FP32 rate, so the streaming
// passes over A^{-1} (the GEMV of the delayed accept, the double-float flush)
// keep their data in FP64 but compute with pairs of floats:
//   - split_d turns a double into hi + lo floats with integer operations only
//     (no FP64 instruction): hi is the double truncated to 24 significant bits,
//     lo the remaining 29 bits rounded to 24, so |x - hi - lo| <= 2^-47 |x|
//     for 2^-74 <= |x| < 2^127 (smaller magnitudes become 0);
//   - products and sums use the error-free transformations of Dekker (1971)
//     and Knuth (TwoSum), written with _rn intrinsics so the compiler cannot
//     contract them into FMAs;
//   - f2d_int converts a float to double exactly with integer operations, so a
//     double-float result costs one FP64 add.
#pragma once
#include <stdint.h>

namespace lru {

__device__ __forceinline__ void split_d(double x, float& hi, float& lo) {
    const uint32_t h = (uint32_t)__double2hiint(x), l = (uint32_t)__double2loint(x);
    const uint32_t sgn = h & 0x80000000u, mag = h & 0x7FFFFFFFu;
    // exponent rebias 1023 -> 127 and keep the top 23 fraction bits
    const uint32_t hb = (__funnelshift_l(l, mag - 0x38000000u, 3) & 0x7FFFFFFFu) | sgn;
    // the low 29 fraction bits are worth 2^(E - 52): a float scale with exponent e8 - 52
    const uint32_t sb = ((hb & 0x7F800000u) - (52u << 23)) | sgn;
    const float lf = __fmul_rn(__uint2float_rn(l & 0x1FFFFFFFu), __uint_as_float(sb));
    const bool ok = mag >= (949u << 20);
    hi = ok ? __uint_as_float(hb) : 0.f;
    lo = ok ? lf : 0.f;
}

__device__ __forceinline__ double f2d_int(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t mag = u & 0x7FFFFFFFu;
    uint32_t hi = ((mag >> 3) + 0x38000000u) | (u & 0x80000000u);
    uint32_t lo = u << 29;
    if (mag < 0x00800000u) { hi = u & 0x80000000u; lo = 0u; }
    return __hiloint2double((int)hi, (int)lo);
}

// (s, e) with s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += (ah + al)(bh + bl), the lo * lo term dropped (below 2^-46 relative)
__device__ __forceinline__ void df_fma(float& acc_h, float& acc_l, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);           // exact low part of ah*bh (Dekker)
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    float s, t;
    two_sum(acc_h, p, s, t);
    acc_h = s;
    acc_l = __fadd_rn(acc_l, __fadd_rn(t, e));
}

__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
    float s, t;
    two_sum(ah, bh, s, t);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(t, bl));
}

__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        df_add(h, l, oh, ol);
    }
}

__device__ __forceinline__ double df_to_double(float h, float l) { return f2d_int(h) + f2d_int(l); }

}  // namespace lru
