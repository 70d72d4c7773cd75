// blas_lo.cu - vector steps of the mixed-precision CG with reliable updates.
//
// The paper names mixed precision as the next step for its CG (Sec. 5).  The
// inner iteration is Fig. 1 run on low-precision vectors (FP32, or FP16 or
// BF16 storage with FP32 arithmetic) with the low-precision Dirac kernels; FP64
// holds the solution x, the source b and the replaced residual.  Following the
// reliable-update scheme (Sleijpen & van der Vorst 1996), the iterated
// residual is replaced by the true residual b - A x, computed in FP64-class
// arithmetic, whenever |r| has fallen below delta * max|r| since the last
// replacement, after reliable_interval iterations, or when the iterated
// residual meets the tolerance.  The search direction is kept across a
// replacement.  The low-precision solution increment y is folded into x at
// each replacement.  For FP16 storage the replaced residual is scaled by 1/sigma
// (sigma = rms entry) so that the inner vectors stay within FP16 range.
//
// Scalars (alpha, beta, delta) are reduced in FP64 on the device.
#include <cuda_fp16.h>

#include <type_traits>

#include <algorithm>

#include "ff.cuh"
#include "stag_kernels.h"

namespace stag {

__device__ __forceinline__ float2 ldv(const float2* p) { return *p; }
__device__ __forceinline__ float2 ldv(const __half2* p) { return __half22float2(*p); }
__device__ __forceinline__ void stv(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void stv(__half2* p, float2 v) { *p = __float22half2_rn(v); }
__device__ __forceinline__ float2 ldv(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ void stv(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }
// the value stv stores, as ldv would read it back (rounded in registers)
__device__ __forceinline__ float2 as_stored(const float2*, float2 v) { return v; }
__device__ __forceinline__ float2 as_stored(const __half2*, float2 v) { return __half22float2(__float22half2_rn(v)); }
__device__ __forceinline__ float2 as_stored(const __nv_bfloat162*, float2 v) {
    return __bfloat1622float2(__float22bfloat162_rn(v));
}

// r64 = b - Ax (Ax in FP64 or float-float); scal->red_out = |r64|^2
template <class AXT>
__global__ void __launch_bounds__(kBlock) residual_kernel(Geom g, const double2* __restrict__ b,
                                                          const AXT* __restrict__ ax,
                                                          double2* __restrict__ r, CgScalars* scal,
                                                          double* partials) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    double acc = 0.0;
    if (i < g.vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            const double2 bb = b[k];
            double2 aa;
            if constexpr (std::is_same<AXT, float4>::value)
                aa = ff_to_complex(ax[k]);
            else
                aa = ax[k];
            const double2 rr = make_double2(bb.x - aa.x, bb.y - aa.y);
            r[k] = rr;
            acc = fma(rr.x, rr.x, acc);
            acc = fma(rr.y, rr.y, acc);
        }
    }
    double total;
    if (grid_sum_last_block<kBlock>(acc, partials, &scal->counter, &total)) {
        if (threadIdx.x == 0) scal->red_out = total;
    }
}

// r_lo = inv_sigma * r64; d_lo = r_lo (first) or r_lo + beta * d_lo; y = 0
template <class V>
__global__ void __launch_bounds__(kBlock) lo_set_residual_kernel(Geom g, const double2* __restrict__ r64,
                                                                 V* __restrict__ r, V* __restrict__ d,
                                                                 float2* __restrict__ y, double inv_sigma,
                                                                 float beta, int first) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = c * vs + i;
        const double2 rr = r64[k];
        const float2 rl = make_float2((float)(rr.x * inv_sigma), (float)(rr.y * inv_sigma));
        stv(r + k, rl);
        const float2 rq = as_stored(r, rl);  // the stored (rounded) residual
        if (first) {
            stv(d + k, rq);
        } else {
            const float2 dd = ldv(d + k);
            stv(d + k, make_float2(fmaf(beta, dd.x, rq.x), fmaf(beta, dd.y, rq.y)));
        }
        y[k] = make_float2(0.f, 0.f);
    }
}

__global__ void lo_reset_kernel(CgScalars* scal, double delta, double threshold, double m2,
                                long long max_iter, long long rel_interval, double rel_delta) {
    scal->delta_new = delta;
    scal->delta_old = delta;
    scal->threshold = threshold;
    scal->m2 = m2;
    scal->m2_ff = ff_from_double(m2);
    scal->iter = 0;
    scal->max_iter = max_iter;
    scal->iter_since = 0;
    scal->rel_interval = rel_interval;
    scal->rel_delta = rel_delta;
    scal->maxr = sqrt(delta);
    scal->done = 0;
    scal->status = 0;
}

// y += alpha d; r -= alpha Ad; delta = |r|^2; decide whether a reliable update is due.
template <class V>
__global__ void __launch_bounds__(kBlock) lo_update_xr_kernel(Geom g, float2* __restrict__ y,
                                                              V* __restrict__ r, const V* __restrict__ d,
                                                              const V* __restrict__ ad, CgScalars* scal,
                                                              double* partials) {
    if (scal->done) return;
    const float alpha = scal->alpha_ff.x;
    const size_t vs = (size_t)g.vs;
    float acc = 0.f;
    // grid-stride over sites: one resident wave of blocks, so that the grid
    // reduction's ticket and partial sums come from a few hundred blocks
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < g.vh; i += gridDim.x * kBlock) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            const float2 dd = ldv(d + k);
            float2 yy = y[k];
            yy.x = fmaf(alpha, dd.x, yy.x);
            yy.y = fmaf(alpha, dd.y, yy.y);
            y[k] = yy;
            const float2 aa = ldv(ad + k);
            float2 rr = ldv(r + k);
            rr.x = fmaf(-alpha, aa.x, rr.x);
            rr.y = fmaf(-alpha, aa.y, rr.y);
            stv(r + k, rr);
            const float2 rq = as_stored(r, rr);  // the stored residual, without reading it back
            acc = fmaf(rq.x, rq.x, acc);
            acc = fmaf(rq.y, rq.y, acc);
        }
    }
    double total;
    if (grid_sum_last_block<kBlock>((double)acc, partials, &scal->counter, &total)) {
        if (threadIdx.x == 0) {
            CgScalars* sc = scal;
            sc->delta_old = sc->delta_new;
            sc->delta_new = total;
            sc->beta = total / sc->delta_old;
            sc->beta_ff = ff_from_double(sc->beta);
            sc->iter += 1;
            sc->iter_since += 1;
            const double rn = sqrt(total);
            if (!isfinite(total)) {
                sc->status = 4;
                sc->done = 1;
            } else if (total <= sc->threshold || rn < sc->rel_delta * sc->maxr ||
                       sc->iter_since >= sc->rel_interval || sc->iter >= sc->max_iter) {
                sc->done = 2;  // reliable update due
            } else {
                sc->maxr = fmax(sc->maxr, rn);
            }
        }
    }
}

template <class V>
__global__ void __launch_bounds__(kBlock) lo_update_d_kernel(Geom g, const V* __restrict__ r, V* __restrict__ d,
                                                             CgScalars* scal) {
    if (scal->done) return;
    const float beta = scal->beta_ff.x;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = c * vs + i;
        const float2 rr = ldv(r + k);
        const float2 dd = ldv(d + k);
        stv(d + k, make_float2(fmaf(beta, dd.x, rr.x), fmaf(beta, dd.y, rr.y)));
    }
}

// x += sigma * y (FP64); y = 0
__global__ void __launch_bounds__(kBlock) lo_fold_y_kernel(Geom g, double2* __restrict__ x,
                                                           float2* __restrict__ y, double sigma) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = c * vs + i;
        const float2 yy = y[k];
        double2 xx = x[k];
        xx.x = fma(sigma, (double)yy.x, xx.x);
        xx.y = fma(sigma, (double)yy.y, xx.y);
        x[k] = xx;
        y[k] = make_float2(0.f, 0.f);
    }
}

// out = scale * in (F64 SoA -> low precision) and back
template <class V>
__global__ void __launch_bounds__(kBlock) to_lo_kernel(Geom g, const double2* __restrict__ in, V* __restrict__ out,
                                                       double scale) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vs) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 v = in[c * vs + i];
        stv(out + c * vs + i, make_float2((float)(v.x * scale), (float)(v.y * scale)));
    }
}

template <class V>
__global__ void __launch_bounds__(kBlock) from_lo_kernel(Geom g, const V* __restrict__ in, double2* __restrict__ out,
                                                         double scale) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vs) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 v = ldv(in + c * vs + i);
        out[c * vs + i] = make_double2(scale * (double)v.x, scale * (double)v.y);
    }
}

// ------------------------------------------------------------ launchers
template <class V>
void launch_to_lo(const Geom& g, const double2* in, V* out, double scale, cudaStream_t s) {
    to_lo_kernel<V><<<blocks_for(g.vs), kBlock, 0, s>>>(g, in, out, scale);
}
template <class V>
void launch_from_lo(const Geom& g, const V* in, double2* out, double scale, cudaStream_t s) {
    from_lo_kernel<V><<<blocks_for(g.vs), kBlock, 0, s>>>(g, in, out, scale);
}
template void launch_to_lo<float2>(const Geom&, const double2*, float2*, double, cudaStream_t);
template void launch_to_lo<__half2>(const Geom&, const double2*, __half2*, double, cudaStream_t);
template void launch_from_lo<float2>(const Geom&, const float2*, double2*, double, cudaStream_t);
template void launch_from_lo<__half2>(const Geom&, const __half2*, double2*, double, cudaStream_t);

void launch_residual(const Geom& g, const double2* b, const void* ax, bool ax_ff, double2* r,
                     CgScalars* scal, double* partials, cudaStream_t s) {
    if (ax_ff)
        residual_kernel<float4><<<blocks_for(g.vh), kBlock, 0, s>>>(g, b, static_cast<const float4*>(ax), r,
                                                                     scal, partials);
    else
        residual_kernel<double2><<<blocks_for(g.vh), kBlock, 0, s>>>(g, b, static_cast<const double2*>(ax), r,
                                                                      scal, partials);
}

void launch_lo_reset(CgScalars* scal, double delta, double threshold, double m2, long long max_iter,
                     long long rel_interval, double rel_delta, cudaStream_t s) {
    lo_reset_kernel<<<1, 1, 0, s>>>(scal, delta, threshold, m2, max_iter, rel_interval, rel_delta);
}

template <class V>
void launch_lo_set_residual(const Geom& g, const double2* r64, V* r, V* d, float2* y, double inv_sigma,
                            double beta, bool first, cudaStream_t s) {
    lo_set_residual_kernel<V><<<blocks_for(g.vh), kBlock, 0, s>>>(g, r64, r, d, y, inv_sigma, (float)beta,
                                                                   first ? 1 : 0);
}

template <class V>
void launch_lo_update_xr(const Geom& g, float2* y, V* r, const V* d, const V* ad, CgScalars* scal,
                         double* partials, cudaStream_t s) {
    const int grid = std::min(blocks_for(g.vh), resident_wave_blocks());
    lo_update_xr_kernel<V><<<grid, kBlock, 0, s>>>(g, y, r, d, ad, scal, partials);
}

template <class V>
void launch_lo_update_d(const Geom& g, const V* r, V* d, CgScalars* scal, cudaStream_t s) {
    lo_update_d_kernel<V><<<blocks_for(g.vh), kBlock, 0, s>>>(g, r, d, scal);
}

void launch_lo_fold_y(const Geom& g, double2* x, float2* y, double sigma, cudaStream_t s) {
    lo_fold_y_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, x, y, sigma);
}

template void launch_lo_set_residual<float2>(const Geom&, const double2*, float2*, float2*, float2*, double,
                                             double, bool, cudaStream_t);
template void launch_lo_set_residual<__half2>(const Geom&, const double2*, __half2*, __half2*, float2*, double,
                                              double, bool, cudaStream_t);
template void launch_lo_update_xr<float2>(const Geom&, float2*, float2*, const float2*, const float2*,
                                          CgScalars*, double*, cudaStream_t);
template void launch_lo_update_xr<__half2>(const Geom&, float2*, __half2*, const __half2*, const __half2*,
                                           CgScalars*, double*, cudaStream_t);
template void launch_lo_update_d<float2>(const Geom&, const float2*, float2*, CgScalars*, cudaStream_t);
template void launch_lo_update_d<__half2>(const Geom&, const __half2*, __half2*, CgScalars*, cudaStream_t);

template void launch_to_lo<__nv_bfloat162>(const Geom&, const double2*, __nv_bfloat162*, double, cudaStream_t);
template void launch_from_lo<__nv_bfloat162>(const Geom&, const __nv_bfloat162*, double2*, double, cudaStream_t);
template void launch_lo_set_residual<__nv_bfloat162>(const Geom&, const double2*, __nv_bfloat162*, __nv_bfloat162*, float2*, double,
                                              double, bool, cudaStream_t);
template void launch_lo_update_xr<__nv_bfloat162>(const Geom&, float2*, __nv_bfloat162*, const __nv_bfloat162*, const __nv_bfloat162*,
                                           CgScalars*, double*, cudaStream_t);
template void launch_lo_update_d<__nv_bfloat162>(const Geom&, const __nv_bfloat162*, __nv_bfloat162*, CgScalars*, cudaStream_t);

}  // namespace stag
