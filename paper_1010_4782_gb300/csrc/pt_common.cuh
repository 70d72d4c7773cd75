// pt_common.cuh - definitions shared by the parallel-transport network kernels
// (pt.cu: CUDA-core layers, gradients, training; pt_tc.cu: tensor-core channel
// mixing).  Paths p = 0..8: the identity and the one-hop transports
// T_{+mu} psi(x) = U_mu(x) psi(x + mu), T_{-mu} psi(x) = U_mu(x - mu)^dag psi(x - mu)
// with the eta-folded fat links, p = 1 + 2 mu + s (s = 0: from x + mu, 1: from x - mu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "stag_kernels.h"

namespace stag {

constexpr int kPaths = 9;
constexpr int kHidden = 8;
constexpr int kLayers = 3;
constexpr int kChan[kLayers + 1] = {1, kHidden, kHidden, 1};
constexpr int kWgradBlocks = 608;  // x-blocks of the weight-gradient grid (4 per SM)

__device__ __forceinline__ float2 ldc(const float2* p) { return *p; }
__device__ __forceinline__ float2 ldc(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
// a float-float complex (re_hi, re_lo, im_hi, im_lo) or an FP64 complex, rounded to FP32
__device__ __forceinline__ float2 ldc(const float4* p) {
    const float4 v = *p;
    return make_float2(v.x + v.y, v.z + v.w);
}
__device__ __forceinline__ float2 ldc(const double2* p) {
    const double2 v = *p;
    return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ void stc(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void stc(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }

// whole-lattice field of C channels, channel innermost: [parity][colour][site][C],
// so that the channels of one site and colour are contiguous (vector accesses)
__device__ __forceinline__ size_t fidx(int ch, int c, int P, int i, size_t vs, int C) {
    return ((size_t)(P * 3 + c) * vs + i) * C + ch;
}

// channels ch0 .. ch0 + 3 of one (parity, colour, site); p = the field at fidx(ch0, ...)
// with ch0 a multiple of 4 and C a multiple of 4 (16-byte aligned for BF16, 32 for FP32)
__device__ __forceinline__ float2 bf16x2_word(uint32_t w) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
}
__device__ __forceinline__ void ld4c(const __nv_bfloat162* p, float2 (&v)[4]) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
    v[0] = bf16x2_word(q.x);
    v[1] = bf16x2_word(q.y);
    v[2] = bf16x2_word(q.z);
    v[3] = bf16x2_word(q.w);
}
__device__ __forceinline__ void ld4c(const float2* p, float2 (&v)[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y);
    v[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ uint32_t bf16x2_bits(float2 v) {
    const __nv_bfloat162 b = __float22bfloat162_rn(v);
    return *reinterpret_cast<const uint32_t*>(&b);
}
__device__ __forceinline__ void st4c(__nv_bfloat162* p, float2 v0, float2 v1, float2 v2, float2 v3) {
    *reinterpret_cast<uint4*>(p) = make_uint4(bf16x2_bits(v0), bf16x2_bits(v1), bf16x2_bits(v2), bf16x2_bits(v3));
}
__device__ __forceinline__ void st4c(float2* p, float2 v0, float2 v1, float2 v2, float2 v3) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v0.x, v0.y, v1.x, v1.y);
    reinterpret_cast<float4*>(p)[1] = make_float4(v2.x, v2.y, v3.x, v3.y);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ float2 cmulf_conj(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ int pt_neighbour(const Geom& g, int x, int y, int z, int t, int mu, bool up) {
    switch (mu) {
        case 0: x = up ? wrap_up(x, 1, g.lx) : wrap_dn(x, 1, g.lx); break;
        case 1: y = up ? wrap_up(y, 1, g.ly) : wrap_dn(y, 1, g.ly); break;
        case 2: z = up ? wrap_up(z, 1, g.lz) : wrap_dn(z, 1, g.lz); break;
        default: t = up ? wrap_up(t, 1, g.lt) : wrap_dn(t, 1, g.lt); break;
    }
    return site_index(x, y, z, t, g);
}

// Source site (parity Pn, index nb) and link of transport direction d
// (0: from x + mu with U_mu(x); 1: from x - mu with U_mu(x - mu)^dag); links
// stored as L (float2, or __half2 for the two-hop inference kernels).
template <class L>
struct HopT {
    int Pn, nb;
    const L* u;
};
using Hop = HopT<float2>;

template <class L>
__device__ __forceinline__ HopT<L> pt_hop(const Geom& g, const L* links, int P, int i, int x, int y, int z, int t,
                                          int mu, int d) {
    HopT<L> h;
    h.Pn = 1 - P;
    const size_t vs = (size_t)g.vs;
    if (d == 0) {
        h.nb = pt_neighbour(g, x, y, z, t, mu, true);
        h.u = links + ((size_t)(P * 4 + mu) * 9) * vs + i;
    } else {
        h.nb = pt_neighbour(g, x, y, z, t, mu, false);
        h.u = links + ((size_t)((1 - P) * 4 + mu) * 9) * vs + h.nb;
    }
    return h;
}

// one link entry in FP32
__device__ __forceinline__ float2 ldu(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldu(const __half2* p) { return __half22float2(__ldg(p)); }

// t = U v (d = 0) or U^dag v (d = 1), on packed FP32 pairs: per row the real
// and the imaginary parts of the link each multiply the whole complex v[c],
//   A = sum_c (Re u, Re u) * (Re v, Im v),  B = sum_c (Im u, Im u) * (Re v, Im v),
// and U v = (A.x - B.y, A.y + B.x), U^dag v = (A.x + B.y, A.y - B.x): six packed
// multiply-adds and two adds a row instead of twelve scalar multiply-adds.
__device__ __forceinline__ void pt_apply(const float2 (&U)[9], int d, const float2 (&v)[3], float2 (&t)[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 u = d == 0 ? U[3 * r + c] : U[3 * c + r];
            a = __ffma2_rn(make_float2(u.x, u.x), v[c], a);
            b = __ffma2_rn(make_float2(u.y, u.y), v[c], b);
        }
        t[r] = d == 0 ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, a.y - b.x);
    }
}

// ------------------------------------------------ collapsed inference form
// With the input on even sites and the output read on even sites, the linear
// network is M r = k0 r + sum_{p,q = 1..8} H[p][q] T_p T_q r (coefficients from
// pt_collapse_kernel, coef[0] = k0, coef[1 + 8 (p - 1) + (q - 1)] = H[p][q]).
// chi: [8][3][vs] on odd sites, chi_p = sum_q H[p][q] T_q r, in channel p - 1.
// Links as FP32, or (BF16 storage of chi) as FP16 divided by a power of two s
// near their largest entry: every two-hop term then carries 1/s^2, which the
// coefficients H take back (k0, with no hop, is unscaled).
constexpr int kCollapsedCoefs = 1 + 8 * 8;

// chi of odd site i (P = 1) from r on even sites (float-float, FP64 or FP32),
// with H in shared memory; returns the 8 x 3 values in acc.
template <class V, class L>
__device__ __forceinline__ void pt_chi_site(const Geom& g, const L* __restrict__ links, const float2* sH,
                                            const V* __restrict__ r, int i, float2 (&acc)[8][3]) {
    const size_t vs = (size_t)g.vs;
    int x, y, z, t;
    site_coords(i, 1, g, x, y, z, t);
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[p][c] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int q = 1; q < kPaths; ++q) {
        const int mu = (q - 1) >> 1, d = (q - 1) & 1;
        const HopT<L> hp = pt_hop(g, links, 1, i, x, y, z, t, mu, d);
        float2 U[9], v[3], tv[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) U[k] = ldu(hp.u + k * vs);
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = ldc(r + c * vs + hp.nb);
        pt_apply(U, d, v, tv);
        // acc_p += H[p][q] tv on packed pairs: (Re h)(Re, Im) + (Im h)(-Im, Re)
        float2 sw[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) sw[c] = make_float2(-tv[c].y, tv[c].x);
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const float2 h = sH[8 * p + (q - 1)];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[p][c] = __ffma2_rn(make_float2(h.x, h.x), tv[c], acc[p][c]);
                acc[p][c] = __ffma2_rn(make_float2(h.y, h.y), sw[c], acc[p][c]);
            }
        }
    }
}

// z(x) = k0 r(x) + sum_p (T_p chi_p)(x) at even site i (P = 0); r0: r(x) in FP32.
template <class TS, class L>
__device__ __forceinline__ void pt_out_site(const Geom& g, const L* __restrict__ links, float2 k0,
                                            const TS* __restrict__ chi, int i, const float2 (&r0)[3],
                                            float2 (&out)[3]) {
    const size_t vs = (size_t)g.vs;
    int x, y, z, t;
    site_coords(i, 0, g, x, y, z, t);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = cmulf(k0, r0[c]);
#pragma unroll 1
    for (int p = 1; p < kPaths; ++p) {
        const int mu = (p - 1) >> 1, d = (p - 1) & 1;
        const HopT<L> hp = pt_hop(g, links, 0, i, x, y, z, t, mu, d);
        float2 U[9], v[3], tv[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) U[k] = ldu(hp.u + k * vs);
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = ldc(chi + ((size_t)(p - 1) * 3 + c) * vs + hp.nb);
        pt_apply(U, d, v, tv);
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c] = __fadd2_rn(out[c], tv[c]);
    }
}

// The 8 -> 8 layer (forward, BF16 activations) with the channel mixing on the
// tensor cores (pt_tc.cu).  w: the layer's complex weights [9][8][8]; err: set
// to 1 if a bounded wait ran out.  w3 (nullable): the 8 -> 1 layer's weights;
// given, the kernel stores phi_p = sum_i W3[p][0][i] psi_i (odd sites: paths
// 1..8 in channels 0..7; even sites: path 0 in channel 0) instead of psi, and
// launch_pt_transport_sum finishes the 8 -> 1 layer on even sites.  skip
// (nullable): a device flag; where it is nonzero when a kernel starts, the
// kernel returns at once (a captured solver iteration after convergence).
void launch_pt_mix8_tc(const Geom& g, const float2* links, const float2* w, const __nv_bfloat162* in,
                       __nv_bfloat162* out, const float2* w3, int* err, cudaStream_t s, const int* skip = nullptr);
void launch_pt_transport_sum(const Geom& g, const float2* links, const __nv_bfloat162* phi, __nv_bfloat162* out,
                             cudaStream_t s, const int* skip = nullptr);

}  // namespace stag
