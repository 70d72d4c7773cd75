// ff.cuh - float-float ("double-FP32") arithmetic for the FP64-class Dirac kernels.
//
// A real number a is held as an unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi)/2 (8 bytes, the size of an FP64 number).  Products and
// sums use the error-free transformations of Dekker (1971) and Knuth (TAOCP
// vol. 2, 4.2.2): TwoProduct via a fused multiply-add, TwoSum with six
// additions.  An accumulator keeps the FP32 running sum of the leading
// products (s, updated with TwoSum) and one FP32 sum of every lower-order
// term (e); the accumulated value is s + e, with a relative rounding of about
// 2^-48 per term.  Every step uses the _rn intrinsics so that the compiler
// cannot contract a product into a neighbouring addition (which would break
// the error-free transformations).
//
// Range: both words are FP32, so magnitudes must stay within about
// [1e-30, 1e30]; lower words of numbers below ~1e-31 lose bits to
// subnormals.
#pragma once

#include <cuda_runtime.h>

namespace stag {

// complex float-float in one 16-byte word: (re_hi, re_lo, im_hi, im_lo)
__device__ __forceinline__ float2 ff_from_double(double a) {
    const float hi = __double2float_rn(a);
    const float lo = __double2float_rn(a - (double)hi);
    return make_float2(hi, lo);
}

__device__ __forceinline__ float4 ff_from_complex(double2 a) {
    const float2 re = ff_from_double(a.x);
    const float2 im = ff_from_double(a.y);
    return make_float4(re.x, re.y, im.x, im.y);
}

__device__ __forceinline__ double2 ff_to_complex(float4 a) {
    return make_double2((double)a.x + (double)a.y, (double)a.z + (double)a.w);
}

struct FFAcc {
    float s;  // running sum of the leading products
    float e;  // running sum of all lower-order terms
};

__device__ __forceinline__ FFAcc ff_zero() { return FFAcc{0.0f, 0.0f}; }

// acc += p exactly in (s, e): TwoSum(s, p) -> (s', err), e += err.
__device__ __forceinline__ void ff_add_exact(FFAcc& a, float p) {
    const float t = __fadd_rn(a.s, p);
    const float z = __fsub_rn(t, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, z)), __fsub_rn(p, z));
    a.s = t;
    a.e = __fadd_rn(a.e, err);
}

// acc += (xh + xl) * (yh + yl), dropping xl*yl (relative 2^-48).
__device__ __forceinline__ void ff_mac(FFAcc& a, float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);
    const float q = __fmaf_rn(xh, yh, -p);  // exact: xh*yh - p
    float e = __fadd_rn(a.e, q);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    a.e = e;
    ff_add_exact(a, p);
}

// Normalised (hi, lo) of the accumulated value s + e.
__device__ __forceinline__ float2 ff_result(const FFAcc& a) {
    const float t = __fadd_rn(a.s, a.e);
    const float z = __fsub_rn(t, a.s);
    const float lo = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, z)), __fsub_rn(a.e, z));
    return make_float2(t, lo);
}

__device__ __forceinline__ double ff_acc_to_double(const FFAcc& a) {
    return (double)a.s + (double)a.e;
}

// Complex accumulator ops.  x = (re_hi, re_lo, im_hi, im_lo).
// acc += x * y
__device__ __forceinline__ void ff_cmac(FFAcc& re, FFAcc& im, float4 x, float4 y) {
    ff_mac(re, x.x, x.y, y.x, y.y);
    ff_mac(re, -x.z, -x.w, y.z, y.w);
    ff_mac(im, x.x, x.y, y.z, y.w);
    ff_mac(im, x.z, x.w, y.x, y.y);
}
// acc -= conj(x) * y
__device__ __forceinline__ void ff_cmsc_conj(FFAcc& re, FFAcc& im, float4 x, float4 y) {
    ff_mac(re, -x.x, -x.y, y.x, y.y);
    ff_mac(re, -x.z, -x.w, y.z, y.w);
    ff_mac(im, -x.x, -x.y, y.z, y.w);
    ff_mac(im, x.z, x.w, y.x, y.y);
}

}  // namespace stag
