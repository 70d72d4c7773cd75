// dslash.cu - half of the staggered Dirac operator on one parity
// (Sec. 2, Eqs. (4)-(5), plus the optional Naik three-hop term):
//
//   out(y) = sum_mu  U_mu(y) in(y+mu) - U_mu(y-mu)^dag in(y-mu)
//          [+ sum_mu L_mu(y) in(y+3mu) - L_mu(y-3mu)^dag in(y-3mu)]
//
// for every site y of the output parity P, with eta folded into the links.
// Forward links are read at y (parity P), backward links at the neighbour
// (parity 1-P), so each half-Dslash streams every link of the field exactly
// once.  One thread per output site; links and vectors are structure-of-
// arrays with the site index fastest (Sec. 3.1: consecutive threads read
// consecutive 16-byte words).  Each 3x3 product is accumulated straight into
// the output registers (Sec. 3.4, Eq. (smallreg)).  The neighbour vectors
// (8 or 16 reads of each input site) are served by L1/L2: a 28^3 x 96
// half-lattice FP64 vector is 50.6 MB, well inside the 126 MB L2.
//
// Two arithmetics share the kernel body: native FP64 FMA (F64) and
// float-float on the FP32 pipelines (FF, see ff.cuh).
//
// Epilogues (used by A = m^2 - D_eo D_oe, Eq. (3)):
//   EPI_PLAIN  out = D in
//   EPI_AXPY   out = m2 * src - D in
//   EPI_CG     as EPI_AXPY with m2 from the CG state, plus the grid-wide
//              Re(src^dag out) = d^dag A d; the last block forms
//              alpha = delta_new / d^dag A d (Fig. 1) on the device.
#include <cuda_fp16.h>

#include <type_traits>

#include "ff.cuh"
#include "stag_kernels.h"

namespace stag {

// ------------------------------------------------------------ arithmetics
struct ArithF64 {
    using T = double2;  // storage
    using C = double2;  // compute
    static __device__ __forceinline__ C ld(const T* p) { return __ldg(p); }
    using TL = T;  // link storage
    static constexpr int kEntries = 9;  // stored entries per link
    static constexpr bool kRecon = false;
    static __device__ __forceinline__ C ldl(const TL* p) { return ld(p); }
    struct Acc {
        double2 c[3];
    };
    static __device__ __forceinline__ void zero(Acc& a) {
#pragma unroll
        for (int r = 0; r < 3; ++r) a.c[r] = make_double2(0.0, 0.0);
    }
    // a_r += sum_c u_c v_c
    static __device__ __forceinline__ void row_fwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        cmac(a.c[r], u0, v0);
        cmac(a.c[r], u1, v1);
        cmac(a.c[r], u2, v2);
    }
    // a_r -= sum_c conj(u_c) v_c
    static __device__ __forceinline__ void row_bwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        cmsc_conj(a.c[r], u0, v0);
        cmsc_conj(a.c[r], u1, v1);
        cmsc_conj(a.c[r], u2, v2);
    }
    static __device__ __forceinline__ T store_val(const Acc& a, int r) { return a.c[r]; }
    // o = m2 * s - acc_r; dot += Re(conj(s) o)
    static __device__ __forceinline__ T epilogue(Acc& a, int r, C s, double m2, float2, double& dot) {
        const double2 d = a.c[r];
        const double2 o = make_double2(fma(m2, s.x, -d.x), fma(m2, s.y, -d.y));
        dot = fma(s.x, o.x, dot);
        dot = fma(s.y, o.y, dot);
        return o;
    }
};

struct ArithFF {
    using T = float4;
    using C = float4;
    static __device__ __forceinline__ C ld(const T* p) { return __ldg(p); }
    using TL = T;  // link storage
    static constexpr int kEntries = 9;  // stored entries per link
    static constexpr bool kRecon = false;
    static __device__ __forceinline__ C ldl(const TL* p) { return ld(p); }
    struct Acc {
        FFAcc re[3], im[3];
        FFAcc dot;
    };
    static __device__ __forceinline__ void zero(Acc& a) {
#pragma unroll
        for (int r = 0; r < 3; ++r) a.re[r] = a.im[r] = ff_zero();
        a.dot = ff_zero();
    }
    static __device__ __forceinline__ void row_fwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        ff_row_fwd(a.re[r], a.im[r], u0, u1, u2, v0, v1, v2);
    }
    static __device__ __forceinline__ void row_bwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        ff_row_bwd(a.re[r], a.im[r], u0, u1, u2, v0, v1, v2);
    }
    static __device__ __forceinline__ T store_val(const Acc& a, int r) {
        return ff_cplx(ff_result(a.re[r]), ff_result(a.im[r]));
    }
    // o = m2 * s - acc_r in float-float; Re(conj(s) o) accumulated in float-float,
    // converted to FP64 once per thread (dot is only valid after the last row).
    static __device__ __forceinline__ T epilogue(Acc& a, int r, C s, double, float2 m2, double& dot) {
        const float2 re = ff_fma(m2, ff_re(s), ff_neg(ff_result(a.re[r])));
        const float2 im = ff_fma(m2, ff_im(s), ff_neg(ff_result(a.im[r])));
        const float4 o = ff_cplx(re, im);
        ff_redot_acc(a.dot, s, o);
        if (r == 2) dot = ff_acc_to_double(a.dot);
        return o;
    }
};

// FP32 storage and arithmetic (inner solver of the mixed-precision CG).
struct ArithF32 {
    using T = float2;
    using C = float2;
    static __device__ __forceinline__ C ld(const T* p) { return __ldg(p); }
    using TL = T;  // link storage
    static constexpr int kEntries = 9;  // stored entries per link
    static constexpr bool kRecon = false;
    static __device__ __forceinline__ C ldl(const TL* p) { return ld(p); }
    struct Acc {
        float2 c[3];
        float dot;
    };
    static __device__ __forceinline__ void zero(Acc& a) {
#pragma unroll
        for (int r = 0; r < 3; ++r) a.c[r] = make_float2(0.f, 0.f);
        a.dot = 0.f;
    }
    static __device__ __forceinline__ void row_fwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        cmacf(a.c[r], u0, v0);
        cmacf(a.c[r], u1, v1);
        cmacf(a.c[r], u2, v2);
    }
    static __device__ __forceinline__ void row_bwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        cmscf_conj(a.c[r], u0, v0);
        cmscf_conj(a.c[r], u1, v1);
        cmscf_conj(a.c[r], u2, v2);
    }
    static __device__ __forceinline__ T store_val(const Acc& a, int r) { return a.c[r]; }
    static __device__ __forceinline__ T epilogue(Acc& a, int r, C s, double, float2 m2, double& dot) {
        const float2 d = a.c[r];
        const float2 o = make_float2(fmaf(m2.x, s.x, -d.x), fmaf(m2.x, s.y, -d.y));
        a.dot = fmaf(s.x, o.x, a.dot);
        a.dot = fmaf(s.y, o.y, a.dot);
        if (r == 2) dot = (double)a.dot;
        return o;
    }
};

// FP16 storage (links and vectors as half2 = (re, im)), FP32 arithmetic.
struct ArithH16 {
    using T = __half2;
    using C = float2;
    static __device__ __forceinline__ C ld(const T* p) { return __half22float2(__ldg(p)); }
    using TL = T;  // link storage
    static constexpr int kEntries = 9;  // stored entries per link
    static constexpr bool kRecon = false;
    static __device__ __forceinline__ C ldl(const TL* p) { return ld(p); }
    using Acc = ArithF32::Acc;
    static __device__ __forceinline__ void zero(Acc& a) { ArithF32::zero(a); }
    static __device__ __forceinline__ void row_fwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        ArithF32::row_fwd(a, r, u0, u1, u2, v0, v1, v2);
    }
    static __device__ __forceinline__ void row_bwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        ArithF32::row_bwd(a, r, u0, u1, u2, v0, v1, v2);
    }
    static __device__ __forceinline__ T store_val(const Acc& a, int r) { return __float22half2_rn(a.c[r]); }
    static __device__ __forceinline__ T epilogue(Acc& a, int r, C s, double m2, float2 m2f, double& dot) {
        return __float22half2_rn(ArithF32::epilogue(a, r, s, m2, m2f, dot));
    }
};

// BF16 storage (links and vectors as bfloat162 = (re, im)), FP32 arithmetic:
// FP32's exponent range with an 8-bit significand.
struct ArithB16 {
    using T = __nv_bfloat162;
    using C = float2;
    static __device__ __forceinline__ C ld(const T* p) { return __bfloat1622float2(__ldg(p)); }
    using TL = T;  // link storage
    static constexpr int kEntries = 9;  // stored entries per link
    static constexpr bool kRecon = false;
    static __device__ __forceinline__ C ldl(const TL* p) { return ld(p); }
    using Acc = ArithF32::Acc;
    static __device__ __forceinline__ void zero(Acc& a) { ArithF32::zero(a); }
    static __device__ __forceinline__ void row_fwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        ArithF32::row_fwd(a, r, u0, u1, u2, v0, v1, v2);
    }
    static __device__ __forceinline__ void row_bwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        ArithF32::row_bwd(a, r, u0, u1, u2, v0, v1, v2);
    }
    static __device__ __forceinline__ T store_val(const Acc& a, int r) { return __float22bfloat162_rn(a.c[r]); }
    static __device__ __forceinline__ T epilogue(Acc& a, int r, C s, double m2, float2 m2f, double& dot) {
        return __float22bfloat162_rn(ArithF32::epilogue(a, r, s, m2, m2f, dot));
    }
};

// FP32 with 12-parameter links (Sec. 3.3): two stored rows a, b of each
// eta-folded SU(3) link; the third is eta (a x b)^* (for U in SU(3) the third
// row is the conjugate cross product of the first two, and eta^2 = 1).  Link
// bytes drop by a third for 6 complex multiply-adds per row.
struct ArithF32R {
    using T = float2;
    using TL = float2;
    using C = float2;
    static constexpr int kEntries = 6;
    static constexpr bool kRecon = true;
    static __device__ __forceinline__ C ld(const T* p) { return __ldg(p); }
    static __device__ __forceinline__ C ldl(const TL* p) { return __ldg(p); }
    using Acc = ArithF32::Acc;
    static __device__ __forceinline__ void zero(Acc& a) { ArithF32::zero(a); }
    static __device__ __forceinline__ void row_fwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        ArithF32::row_fwd(a, r, u0, u1, u2, v0, v1, v2);
    }
    static __device__ __forceinline__ void row_bwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        ArithF32::row_bwd(a, r, u0, u1, u2, v0, v1, v2);
    }
    static __device__ __forceinline__ T store_val(const Acc& a, int r) { return ArithF32::store_val(a, r); }
    static __device__ __forceinline__ T epilogue(Acc& a, int r, C s, double m2, float2 m2f, double& dot) {
        return ArithF32::epilogue(a, r, s, m2, m2f, dot);
    }
};

// FP16-stored links, FP32 vectors and arithmetic: the links carry most of the
// bytes, the vectors keep FP32's significand (the CG direction and residual).
struct ArithL16 {
    using T = float2;
    using TL = __half2;
    static constexpr int kEntries = 9;
    static constexpr bool kRecon = false;
    using C = float2;
    static __device__ __forceinline__ C ld(const T* p) { return __ldg(p); }
    static __device__ __forceinline__ C ldl(const TL* p) { return __half22float2(__ldg(p)); }
    using Acc = ArithF32::Acc;
    static __device__ __forceinline__ void zero(Acc& a) { ArithF32::zero(a); }
    static __device__ __forceinline__ void row_fwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        ArithF32::row_fwd(a, r, u0, u1, u2, v0, v1, v2);
    }
    static __device__ __forceinline__ void row_bwd(Acc& a, int r, C u0, C u1, C u2, C v0, C v1, C v2) {
        ArithF32::row_bwd(a, r, u0, u1, u2, v0, v1, v2);
    }
    static __device__ __forceinline__ T store_val(const Acc& a, int r) { return ArithF32::store_val(a, r); }
    static __device__ __forceinline__ T epilogue(Acc& a, int r, C s, double m2, float2 m2f, double& dot) {
        return ArithF32::epilogue(a, r, s, m2, m2f, dot);
    }
};

template <class A>
struct DslashParams {
    Geom g;
    int P;                     // output parity
    const typename A::TL* fat;  // [2][4][9][vs]
    const typename A::TL* lng;  // [2][4][9][vs] or nullptr
    const typename A::T* in;   // [3][vs], parity 1-P
    typename A::T* out;        // [3][vs], parity P
    const typename A::T* src;  // [3][vs], parity P (EPI_AXPY / EPI_CG)
    double m2;                 // m^2 (EPI_AXPY)
    float2 m2_ff;              // m^2 as float-float (EPI_AXPY, FF)
    CgScalars* scal;
    double* partials;
    int i0, i1;                // output sites [i0, i1) of parity P
    float2 lng_s = make_float2(0.f, 0.f);  // NAIK == 2: 1 / scale of the two-row Naik links (float-float)
};

// Link entries 6..8 (the third row) from the first two: eta * conj(row0 x row1).
__device__ __forceinline__ float2 cross_conj(float2 a1, float2 b2, float2 a2, float2 b1, float eta) {
    // conj(a1 b2 - a2 b1) * eta
    const float re = a1.x * b2.x - a1.y * b2.y - (a2.x * b1.x - a2.y * b1.y);
    const float im = a1.x * b2.y + a1.y * b2.x - (a2.x * b1.y + a2.y * b1.x);
    return make_float2(eta * re, -eta * im);
}
template <class A>
__device__ __forceinline__ void load_recon(typename A::C (&U)[9], const typename A::TL* __restrict__ u, size_t vs,
                                           float eta) {
#pragma unroll
    for (int k = 0; k < 6; ++k) U[k] = A::ldl(u + k * vs);
    U[6] = cross_conj(U[1], U[5], U[2], U[4], eta);
    U[7] = cross_conj(U[2], U[3], U[0], U[5], eta);
    U[8] = cross_conj(U[0], U[4], U[1], U[3], eta);
}

// Float-float Naik link stored as its first two rows ([6][vs], eta folded); the
// third row is (eta / scale) conj(row0 x row1), s = eta / scale (Sec. 3.3's
// 12-parameter form applied to scale x SU(3)).
__device__ __forceinline__ void load_recon_ff(float4 (&U)[9], const float4* __restrict__ u, size_t vs, float2 s) {
#pragma unroll
    for (int k = 0; k < 6; ++k) U[k] = __ldg(u + k * vs);
    U[6] = ff_cross_conj_scaled(U[1], U[5], U[2], U[4], s);
    U[7] = ff_cross_conj_scaled(U[2], U[3], U[0], U[5], s);
    U[8] = ff_cross_conj_scaled(U[0], U[4], U[1], U[3], s);
}
__device__ __forceinline__ void hop_fwd_ffr(ArithFF::Acc& acc, const float4* __restrict__ u,
                                            const float4* __restrict__ in, int nb, size_t vs, float2 s) {
    const float4 v0 = __ldg(in + nb), v1 = __ldg(in + vs + nb), v2 = __ldg(in + 2 * vs + nb);
    float4 U[9];
    load_recon_ff(U, u, vs, s);
#pragma unroll
    for (int r = 0; r < 3; ++r) ArithFF::row_fwd(acc, r, U[3 * r], U[3 * r + 1], U[3 * r + 2], v0, v1, v2);
}
__device__ __forceinline__ void hop_bwd_ffr(ArithFF::Acc& acc, const float4* __restrict__ u,
                                            const float4* __restrict__ in, int nb, size_t vs, float2 s) {
    const float4 v0 = __ldg(in + nb), v1 = __ldg(in + vs + nb), v2 = __ldg(in + 2 * vs + nb);
    float4 U[9];
    load_recon_ff(U, u, vs, s);
#pragma unroll
    for (int r = 0; r < 3; ++r) ArithFF::row_bwd(acc, r, U[r], U[3 + r], U[6 + r], v0, v1, v2);
}

template <class A>
__device__ __forceinline__ void hop_fwd(typename A::Acc& acc, const typename A::TL* __restrict__ u,
                                        const typename A::T* __restrict__ in, int nb, size_t vs, float eta = 1.f) {
    const typename A::C v0 = A::ld(in + nb), v1 = A::ld(in + vs + nb), v2 = A::ld(in + 2 * vs + nb);
    if constexpr (A::kRecon) {
        typename A::C U[9];
        load_recon<A>(U, u, vs, eta);
#pragma unroll
        for (int r = 0; r < 3; ++r) A::row_fwd(acc, r, U[3 * r], U[3 * r + 1], U[3 * r + 2], v0, v1, v2);
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r)
            A::row_fwd(acc, r, A::ldl(u + (3 * r) * vs), A::ldl(u + (3 * r + 1) * vs), A::ldl(u + (3 * r + 2) * vs),
                       v0, v1, v2);
    }
}

template <class A>
__device__ __forceinline__ void hop_bwd(typename A::Acc& acc, const typename A::TL* __restrict__ u,
                                        const typename A::T* __restrict__ in, int nb, size_t vs, float eta = 1.f) {
    const typename A::C v0 = A::ld(in + nb), v1 = A::ld(in + vs + nb), v2 = A::ld(in + 2 * vs + nb);
    // (U^dag v)_r = sum_c conj(U_cr) v_c
    if constexpr (A::kRecon) {
        typename A::C U[9];
        load_recon<A>(U, u, vs, eta);
#pragma unroll
        for (int r = 0; r < 3; ++r) A::row_bwd(acc, r, U[r], U[3 + r], U[6 + r], v0, v1, v2);
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r)
            A::row_bwd(acc, r, A::ldl(u + r * vs), A::ldl(u + (3 + r) * vs), A::ldl(u + (6 + r) * vs), v0, v1, v2);
    }
}

// Half-lattice index of the neighbour of (x,y,z,t) at +-h along mu.
__device__ __forceinline__ int neighbour(const Geom& g, int x, int y, int z, int t, int mu, int h,
                                         bool up) {
    switch (mu) {
        case 0: x = up ? wrap_up(x, h, g.lx) : wrap_dn(x, h, g.lx); break;
        case 1: y = up ? wrap_up(y, h, g.ly) : wrap_dn(y, h, g.ly); break;
        case 2: z = up ? wrap_up(z, h, g.lz) : wrap_dn(z, h, g.lz); break;
        default: t = up ? wrap_up(t, h, g.lt) : wrap_dn(t, h, g.lt); break;
    }
    return site_index(x, y, z, t, g);
}

// acc += (D_{P,1-P} in)(i) for output site i of parity p.P (all hops).
// NAIK: 0 one-hop only; 1 Naik links with nine entries; 2 float-float Naik
// links with two rows (A = ArithFF only).
template <class A, int NAIK>
__device__ __forceinline__ void dslash_site(const DslashParams<A>& p, int i, typename A::Acc& acc) {
    const Geom& g = p.g;
    const size_t vs = (size_t)g.vs;
    {
        int x, y, z, t;
        site_coords(i, p.P, g, x, y, z, t);
        const int P = p.P, Q = 1 - p.P;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const int f1 = neighbour(g, x, y, z, t, mu, 1, true);
            const int b1 = neighbour(g, x, y, z, t, mu, 1, false);
            // eta_mu(x) = eta_mu(x - mu): the phase of both links of this direction
            const int ps = (mu >= 1 ? x : 0) + (mu >= 2 ? y : 0) + (mu >= 3 ? z : 0);
            const float eta = (ps & 1) ? -1.f : 1.f;
            hop_fwd<A>(acc, p.fat + ((size_t)(P * 4 + mu) * A::kEntries) * vs + i, p.in, f1, vs, eta);
            hop_bwd<A>(acc, p.fat + ((size_t)(Q * 4 + mu) * A::kEntries) * vs + b1, p.in, b1, vs, eta);
            if constexpr (NAIK == 1) {
                const int h = g.hop3[mu];
                const int f3 = neighbour(g, x, y, z, t, mu, h, true);
                const int b3 = neighbour(g, x, y, z, t, mu, h, false);
                hop_fwd<A>(acc, p.lng + ((size_t)(P * 4 + mu) * 9) * vs + i, p.in, f3, vs);
                hop_bwd<A>(acc, p.lng + ((size_t)(Q * 4 + mu) * 9) * vs + b3, p.in, b3, vs);
            }
        }
        if constexpr (NAIK == 2) {
            // A rolled loop: unrolled, the four copies of the float-float
            // reconstruction overflow the instruction cache.
#pragma unroll 1
            for (int mu = 0; mu < 4; ++mu) {
                const int h = mu == 0 ? g.hop3[0] : mu == 1 ? g.hop3[1] : mu == 2 ? g.hop3[2] : g.hop3[3];
                const int f3 = neighbour(g, x, y, z, t, mu, h, true);
                const int b3 = neighbour(g, x, y, z, t, mu, h, false);
                // the Naik link of x and the one arriving from x - 3 mu share eta_mu(x)
                const int ps = (mu >= 1 ? x : 0) + (mu >= 2 ? y : 0) + (mu >= 3 ? z : 0);
                if constexpr (std::is_same<A, ArithFF>::value) {
                    const float2 s = (ps & 1) ? make_float2(-p.lng_s.x, -p.lng_s.y) : p.lng_s;
                    hop_fwd_ffr(acc, p.lng + ((size_t)(P * 4 + mu) * 6) * vs + i, p.in, f3, vs, s);
                    hop_bwd_ffr(acc, p.lng + ((size_t)(Q * 4 + mu) * 6) * vs + b3, p.in, b3, vs, s);
                } else {
                    // FP32 (the mixed-precision iteration): the same rows, the third
                    // rebuilt in FP32 with the factor eta / scale
                    const float s = (ps & 1) ? -p.lng_s.x : p.lng_s.x;
                    hop_fwd<ArithF32R>(acc, p.lng + ((size_t)(P * 4 + mu) * 6) * vs + i, p.in, f3, vs, s);
                    hop_bwd<ArithF32R>(acc, p.lng + ((size_t)(Q * 4 + mu) * 6) * vs + b3, p.in, b3, vs, s);
                }
            }
        }
    }
}

// Resident 256-thread blocks per SM the register allocation is held to.  The
// float-float kernels are bound by memory latency: with up to 128 registers
// (2 blocks) the compiler keeps more of a site's loads in flight, and the
// float-float CG solve at 28^3 x 96 measured 1304 ms against 1320 ms with 3
// blocks (80 registers), 1339 ms with 4 (64) and 1734 ms with 1.  The others
// keep 4 blocks (64 registers; 3 and 80 with two-row Naik links): FP64 is
// bound by its pipe and FP32 by HBM, where more registers measured no gain.
template <class A, int NAIK>
constexpr int dslash_min_blocks() {
    return std::is_same<A, ArithFF>::value ? 2 : (NAIK == 2 ? 3 : 4);
}

template <class A, int NAIK, int EPI>
__global__ void __launch_bounds__(kBlock, dslash_min_blocks<A, NAIK>()) dslash_kernel(const DslashParams<A> p) {
    // Inside a solver iteration (CG state given): return once the loop has
    // stopped, so that the rest of a captured block of iterations costs nothing.
    if (p.scal && p.scal->done) return;
    const Geom& g = p.g;
    const int i = p.i0 + blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    typename A::Acc acc;
    A::zero(acc);
    const bool active = i < p.i1;
    // the epilogue's operands are loaded before the stencil, so that their
    // latency overlaps it instead of following it
    using SrcT = decltype(A::ld(p.src));
    SrcT srcv[3];
    double m2 = 0.0;
    float2 m2_ff = make_float2(0.f, 0.f);
    if (EPI != EPI_PLAIN) {
        m2 = (EPI == EPI_CG) ? p.scal->m2 : p.m2;
        m2_ff = (EPI == EPI_CG) ? p.scal->m2_ff : p.m2_ff;
        if (active) {
#pragma unroll
            for (int r = 0; r < 3; ++r) srcv[r] = A::ld(p.src + r * vs + i);
        }
    }
    if (active) dslash_site<A, NAIK>(p, i, acc);
    if (EPI == EPI_PLAIN) {
        if (active) {
#pragma unroll
            for (int r = 0; r < 3; ++r) p.out[r * vs + i] = A::store_val(acc, r);
        }
        return;
    }
    // out = m2 * src - D in
    double dot = 0.0;
    if (active) {
#pragma unroll
        for (int r = 0; r < 3; ++r) p.out[r * vs + i] = A::epilogue(acc, r, srcv[r], m2, m2_ff, dot);
    }
    if (EPI == EPI_CG) {
        double total;
        if (grid_sum_last_block<kBlock>(dot, p.partials, &p.scal->counter, &total)) {
            if (threadIdx.x == 0) {
                CgScalars* sc = p.scal;
                sc->pAp = total;
                const double alpha = sc->delta_new / total;
                if (!(total > 0.0) || !isfinite(alpha)) {
                    sc->status = 4;  // STAG_ERR_BREAKDOWN
                    sc->done = 1;
                    sc->alpha = 0.0;
                    sc->alpha_ff = make_float2(0.f, 0.f);
                } else {
                    sc->alpha = alpha;
                    sc->alpha_ff = ff_from_double(alpha);
                }
            }
        }
    }
}

// Half-Dslash of several systems in one launch (EPI_PLAIN or EPI_AXPY): the
// systems list[0 .. *count) take consecutive runs of kBlock-site tiles,
// prefix[j] .. prefix[j + 1] for entry j, and the grid's blocks stride over
// all of them.  The list lives on the device, so a captured graph runs
// whichever systems the kernels before it selected.
template <class A, int EPI>
__global__ void __launch_bounds__(kBlock, 3) dslash_list_kernel(const SysDirac* __restrict__ sys,
                                                               const int* __restrict__ list,
                                                               const int* __restrict__ prefix,
                                                               const int* __restrict__ count) {
    using T = typename A::T;
    using TL = typename A::TL;
    const int n = *count;
    const int total = prefix[n];
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        int j = 0;
        while (prefix[j + 1] <= tile) ++j;
        const SysDirac& sd = sys[list[j]];
        const int i = (tile - prefix[j]) * kBlock + threadIdx.x;
        if (i >= sd.g.vh) continue;
        const DslashParams<A> p{sd.g,
                                sd.P,
                                static_cast<const TL*>(sd.fat),
                                static_cast<const TL*>(sd.lng),
                                static_cast<const T*>(sd.in),
                                static_cast<T*>(sd.out),
                                static_cast<const T*>(sd.src),
                                sd.m2,
                                sd.m2_ff,
                                nullptr,
                                nullptr,
                                0,
                                sd.g.vh};
        typename A::Acc acc;
        A::zero(acc);
        if (p.lng)
            dslash_site<A, 1>(p, i, acc);
        else
            dslash_site<A, 0>(p, i, acc);
        const size_t vs = (size_t)sd.g.vs;
        double dot = 0.0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            if (EPI == EPI_PLAIN)
                p.out[r * vs + i] = A::store_val(acc, r);
            else
                p.out[r * vs + i] = A::epilogue(acc, r, A::ld(p.src + r * vs + i), p.m2, p.m2_ff, dot);
        }
    }
}

void launch_dslash_list(bool ff, Epilogue epi, const SysDirac* sys, const int* list, const int* prefix,
                        const int* count, int grid, cudaStream_t s) {
    if (ff) {
        if (epi == EPI_PLAIN)
            dslash_list_kernel<ArithFF, EPI_PLAIN><<<grid, kBlock, 0, s>>>(sys, list, prefix, count);
        else
            dslash_list_kernel<ArithFF, EPI_AXPY><<<grid, kBlock, 0, s>>>(sys, list, prefix, count);
    } else {
        if (epi == EPI_PLAIN)
            dslash_list_kernel<ArithF64, EPI_PLAIN><<<grid, kBlock, 0, s>>>(sys, list, prefix, count);
        else
            dslash_list_kernel<ArithF64, EPI_AXPY><<<grid, kBlock, 0, s>>>(sys, list, prefix, count);
    }
}

template <class A, int EPI>
static void launch_one(const DslashParams<A>& p, int naik, cudaStream_t s) {
    const int blocks = blocks_for(p.i1 - p.i0);
    if constexpr (std::is_same<A, ArithFF>::value || std::is_same<A, ArithF32>::value) {
        if (naik == 2) {
            dslash_kernel<A, 2, EPI><<<blocks, kBlock, 0, s>>>(p);
            return;
        }
    }
    if (naik)
        dslash_kernel<A, 1, EPI><<<blocks, kBlock, 0, s>>>(p);
    else
        dslash_kernel<A, 0, EPI><<<blocks, kBlock, 0, s>>>(p);
}

template <class A>
static void launch_any(const DslashParams<A>& p, int naik, Epilogue epi, cudaStream_t s) {
    switch (epi) {
        case EPI_PLAIN: launch_one<A, EPI_PLAIN>(p, naik, s); break;
        case EPI_AXPY: launch_one<A, EPI_AXPY>(p, naik, s); break;
        default: launch_one<A, EPI_CG>(p, naik, s); break;
    }
}

void launch_dslash_f64(const Geom& g, int out_parity, const LinkSet& L, const double2* in,
                       double2* out, Epilogue epi, const double2* src, double m2,
                       CgScalars* scal, double* partials, cudaStream_t s) {
    DslashParams<ArithF64> p{g, out_parity, L.fat64, L.lng64, in, out, src, m2,
                             make_float2(0.f, 0.f), scal, partials, 0, g.vh};
    launch_any(p, L.lng64 != nullptr, epi, s);
}

void launch_dslash_f64_range(const Geom& g, int out_parity, const LinkSet& L, const double2* in, double2* out,
                             Epilogue epi, const double2* src, double m2, int i0, int i1, cudaStream_t s) {
    if (i1 <= i0) return;
    DslashParams<ArithF64> p{g, out_parity, L.fat64, L.lng64, in, out, src, m2,
                             make_float2(0.f, 0.f), nullptr, nullptr, i0, i1};
    launch_any(p, L.lng64 != nullptr, epi, s);
}

void launch_dslash_ff(const Geom& g, int out_parity, const LinkSet& L, const float4* in,
                      float4* out, Epilogue epi, const float4* src, double m2, CgScalars* scal,
                      double* partials, cudaStream_t s) {
    DslashParams<ArithFF> p{g, out_parity, L.fatff, L.lngff, in, out, src, m2,
                            host_ff_from_double(m2), scal, partials, 0, g.vh, L.lng_inv_scale_ff};
    const bool two_row = L.lng_inv_scale_ff.x != 0.f;
    launch_any(p, L.lngff == nullptr ? 0 : two_row ? 2 : 1, epi, s);
}

void launch_dslash_f32(const Geom& g, int out_parity, const float2* fat, const float2* lng,
                       const float2* in, float2* out, Epilogue epi, const float2* src, double m2,
                       CgScalars* scal, double* partials, cudaStream_t s, float lng_inv_scale) {
    DslashParams<ArithF32> p{g, out_parity, fat, lng, in, out, src, m2, host_ff_from_double(m2), scal, partials, 0,
                             g.vh, make_float2(lng_inv_scale, 0.f)};
    launch_any(p, lng == nullptr ? 0 : lng_inv_scale != 0.f ? 2 : 1, epi, s);
}

void launch_dslash_h16(const Geom& g, int out_parity, const __half2* fat, const __half2* lng,
                       const __half2* in, __half2* out, Epilogue epi, const __half2* src, double m2,
                       CgScalars* scal, double* partials, cudaStream_t s) {
    DslashParams<ArithH16> p{g, out_parity, fat, lng, in, out, src, m2, host_ff_from_double(m2), scal, partials, 0,
                             g.vh};
    launch_any(p, lng != nullptr, epi, s);
}

void launch_dslash_b16(const Geom& g, int out_parity, const __nv_bfloat162* fat, const __nv_bfloat162* lng,
                       const __nv_bfloat162* in, __nv_bfloat162* out, Epilogue epi, const __nv_bfloat162* src,
                       double m2, CgScalars* scal, double* partials, cudaStream_t s) {
    DslashParams<ArithB16> p{g, out_parity, fat, lng, in, out, src, m2, host_ff_from_double(m2), scal, partials, 0,
                             g.vh};
    launch_any(p, lng != nullptr, epi, s);
}

void launch_dslash_f32l16(const Geom& g, int out_parity, const __half2* fat, const __half2* lng, const float2* in,
                          float2* out, Epilogue epi, const float2* src, double m2, CgScalars* scal, double* partials,
                          cudaStream_t s) {
    DslashParams<ArithL16> p{g, out_parity, fat, lng, in, out, src, m2, host_ff_from_double(m2), scal, partials, 0,
                             g.vh};
    launch_any(p, lng != nullptr, epi, s);
}

void launch_dslash_f32r12(const Geom& g, int out_parity, const float2* fat_rows2, const float2* in, float2* out,
                          Epilogue epi, const float2* src, double m2, CgScalars* scal, double* partials,
                          cudaStream_t s) {
    DslashParams<ArithF32R> p{g, out_parity, fat_rows2, nullptr, in, out, src, m2, host_ff_from_double(m2), scal,
                              partials, 0, g.vh};
    launch_any(p, false, epi, s);
}

}  // namespace stag
