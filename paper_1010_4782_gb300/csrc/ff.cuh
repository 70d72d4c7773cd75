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

// TwoSum (Knuth): t + err == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
    const float t = __fadd_rn(a, b);
    const float z = __fsub_rn(t, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(t, z)), __fsub_rn(b, z));
    return t;
}

// (xh + xl) * (yh + yl) as (p, lo): p = fl(xh*yh), lo = the rest (xl*yl dropped, ~2^-48).
__device__ __forceinline__ FFAcc ff_prod(float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);
    float lo = __fmaf_rn(xh, yh, -p);  // exact: xh*yh - p (TwoProduct)
    lo = __fmaf_rn(xh, yl, lo);
    lo = __fmaf_rn(xl, yh, lo);
    return FFAcc{p, lo};
}

// acc += (xh + xl) * (yh + yl): the leading product enters s through TwoSum, the
// product's lower part and TwoSum's error enter e with one addition.
__device__ __forceinline__ void ff_mac(FFAcc& a, float xh, float xl, float yh, float yl) {
    const FFAcc p = ff_prod(xh, xl, yh, yl);
    float err;
    a.s = two_sum(a.s, p.s, err);
    a.e = __fadd_rn(a.e, __fadd_rn(p.e, err));
}

// acc += h, where h is a small local sum (one hop): one TwoSum and one addition to e.
__device__ __forceinline__ void ff_merge(FFAcc& a, const FFAcc& h) {
    float err;
    a.s = two_sum(a.s, h.s, err);
    a.e = __fadd_rn(a.e, __fadd_rn(h.e, err));
}

// Normalised (hi, lo) of the accumulated value s + e.
__device__ __forceinline__ float2 ff_result(const FFAcc& a) {
    float lo;
    const float hi = two_sum(a.s, a.e, lo);
    return make_float2(hi, lo);
}

__device__ __forceinline__ double ff_acc_to_double(const FFAcc& a) {
    return (double)a.s + (double)a.e;
}

// One row of a 3x3 complex product for one hop, accumulated locally and
// merged once into the site sums (re, im):
//   fwd:  (re, im) += sum_c u_c * v_c            (u_c = U_{r c})
//   bwd:  (re, im) -= sum_c conj(u_c) * v_c      (u_c = U_{c r})
// complex float-float words are (re_hi, re_lo, im_hi, im_lo).
__device__ __forceinline__ void ff_row_fwd(FFAcc& re, FFAcc& im, float4 u0, float4 u1, float4 u2,
                                           float4 v0, float4 v1, float4 v2) {
    FFAcc hr = ff_prod(u0.x, u0.y, v0.x, v0.y);
    ff_mac(hr, -u0.z, -u0.w, v0.z, v0.w);
    ff_mac(hr, u1.x, u1.y, v1.x, v1.y);
    ff_mac(hr, -u1.z, -u1.w, v1.z, v1.w);
    ff_mac(hr, u2.x, u2.y, v2.x, v2.y);
    ff_mac(hr, -u2.z, -u2.w, v2.z, v2.w);
    FFAcc hi = ff_prod(u0.x, u0.y, v0.z, v0.w);
    ff_mac(hi, u0.z, u0.w, v0.x, v0.y);
    ff_mac(hi, u1.x, u1.y, v1.z, v1.w);
    ff_mac(hi, u1.z, u1.w, v1.x, v1.y);
    ff_mac(hi, u2.x, u2.y, v2.z, v2.w);
    ff_mac(hi, u2.z, u2.w, v2.x, v2.y);
    ff_merge(re, hr);
    ff_merge(im, hi);
}

__device__ __forceinline__ void ff_row_bwd(FFAcc& re, FFAcc& im, float4 u0, float4 u1, float4 u2,
                                           float4 v0, float4 v1, float4 v2) {
    // -conj(u) v = (-ur vr - ui vi) + i (-ur vi + ui vr)
    FFAcc hr = ff_prod(-u0.x, -u0.y, v0.x, v0.y);
    ff_mac(hr, -u0.z, -u0.w, v0.z, v0.w);
    ff_mac(hr, -u1.x, -u1.y, v1.x, v1.y);
    ff_mac(hr, -u1.z, -u1.w, v1.z, v1.w);
    ff_mac(hr, -u2.x, -u2.y, v2.x, v2.y);
    ff_mac(hr, -u2.z, -u2.w, v2.z, v2.w);
    FFAcc hi = ff_prod(-u0.x, -u0.y, v0.z, v0.w);
    ff_mac(hi, u0.z, u0.w, v0.x, v0.y);
    ff_mac(hi, -u1.x, -u1.y, v1.z, v1.w);
    ff_mac(hi, u1.z, u1.w, v1.x, v1.y);
    ff_mac(hi, -u2.x, -u2.y, v2.z, v2.w);
    ff_mac(hi, u2.z, u2.w, v2.x, v2.y);
    ff_merge(re, hr);
    ff_merge(im, hi);
}

// s * conj(a1 b2 - a2 b1) for complex float-float words (re_hi, re_lo, im_hi,
// im_lo) and a real float-float s: one entry of the third row of a scaled
// SU(3) matrix from its first two rows (Sec. 3.3's reconstruction, with s =
// eta / scale).
__device__ __forceinline__ float4 ff_cross_conj_scaled(float4 a1, float4 b2, float4 a2, float4 b1, float2 s) {
    FFAcc re = ff_prod(a1.x, a1.y, b2.x, b2.y);  // a1r b2r - a1i b2i - a2r b1r + a2i b1i
    ff_mac(re, -a1.z, -a1.w, b2.z, b2.w);
    ff_mac(re, -a2.x, -a2.y, b1.x, b1.y);
    ff_mac(re, a2.z, a2.w, b1.z, b1.w);
    FFAcc im = ff_prod(a1.x, a1.y, b2.z, b2.w);  // a1r b2i + a1i b2r - a2r b1i - a2i b1r
    ff_mac(im, a1.z, a1.w, b2.x, b2.y);
    ff_mac(im, -a2.x, -a2.y, b1.z, b1.w);
    ff_mac(im, -a2.z, -a2.w, b1.x, b1.y);
    const float2 r = ff_result(re), i = ff_result(im);
    const float2 pr = ff_result(ff_prod(s.x, s.y, r.x, r.y));
    const float2 pi = ff_result(ff_prod(-s.x, -s.y, i.x, i.y));
    return make_float4(pr.x, pr.y, pi.x, pi.y);
}

// ---------------------------------------------- float-float scalar algebra
// Values are float2 (hi, lo).  Error about 2^-48 relative per operation.
__device__ __forceinline__ float2 ff_renorm(float s, float e) {
    float lo;
    const float hi = two_sum(s, e, lo);
    return make_float2(hi, lo);
}

__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    float err;
    const float s = two_sum(a.x, b.x, err);
    return ff_renorm(s, __fadd_rn(err, __fadd_rn(a.y, b.y)));
}

// a * b + c
__device__ __forceinline__ float2 ff_fma(float2 a, float2 b, float2 c) {
    const FFAcc p = ff_prod(a.x, a.y, b.x, b.y);
    float err;
    const float s = two_sum(c.x, p.s, err);
    return ff_renorm(s, __fadd_rn(__fadd_rn(p.e, err), c.y));
}

__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ double ff_to_double(float2 a) { return (double)a.x + (double)a.y; }

// complex helpers on (re_hi, re_lo, im_hi, im_lo)
__device__ __forceinline__ float2 ff_re(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 ff_im(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 ff_cplx(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }

// s * a + b for a real float-float scalar s and complex float-float a, b
__device__ __forceinline__ float4 ff_caxpy(float2 s, float4 a, float4 b) {
    return ff_cplx(ff_fma(s, ff_re(a), ff_re(b)), ff_fma(s, ff_im(a), ff_im(b)));
}

// acc += |a|^2 (complex float-float), exact products via TwoProduct
__device__ __forceinline__ void ff_norm2_acc(FFAcc& acc, float4 a) {
    ff_mac(acc, a.x, a.y, a.x, a.y);
    ff_mac(acc, a.z, a.w, a.z, a.w);
}

// acc += Re(conj(a) * b)
__device__ __forceinline__ void ff_redot_acc(FFAcc& acc, float4 a, float4 b) {
    ff_mac(acc, a.x, a.y, b.x, b.y);
    ff_mac(acc, a.z, a.w, b.z, b.w);
}

}  // namespace stag
