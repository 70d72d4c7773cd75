// blas.cu - the vector steps of CG (Sec. 2, Fig. 1), fused so that each
// vector is streamed once per step and every scalar stays on the device:
//
//   cg_init      r = b - A x, d = r, delta_new = delta_0 = r^dag r
//   cg_update_xr x += alpha d, r -= alpha A d, delta_old = delta_new,
//                delta_new = r^dag r, beta = delta_new / delta_old
//   cg_update_d  d = r + beta d
//
// alpha comes from the Dirac epilogue (dslash.cu).  Reductions are
// deterministic: a fixed shuffle tree per block, then the last block to
// finish sums the per-block partials in block order.  The loop condition of
// Fig. 1 (i < N_dim and delta_new > eps^2 delta_0) is evaluated by that last
// block and stored in scal->done; every kernel of the iteration returns at
// once when it is set, so a captured block of iterations stops exactly
// where Fig. 1 stops.
//
// Two sets of kernels: FP64 vectors with native FP64 arithmetic, and
// float-float vectors (ff.cuh) whose arithmetic runs on the FP32 pipelines.
// GB300 issues FP64 operations - and FP64<->FP32 conversions - at about 1/58
// of the FP32 rate, so the float-float set keeps the iteration free of them:
// x is accumulated in float-float since the last fold and added into the FP64
// solution by fold_x once per block of iterations.
#include <algorithm>
#include <atomic>

#include "ff.cuh"
#include "stag_kernels.h"

namespace stag {

__device__ __forceinline__ void set_done(CgScalars* sc) {
    sc->done = (sc->delta_new <= sc->threshold || sc->iter >= sc->max_iter) ? 1 : 0;
}

__device__ __forceinline__ void finish_delta(CgScalars* sc, double total) {
    sc->delta_old = sc->delta_new;
    sc->delta_new = total;
    sc->beta = total / sc->delta_old;
    sc->beta_ff = ff_from_double(sc->beta);
    sc->iter += 1;
    if (!isfinite(total)) {
        sc->status = 4;  // STAG_ERR_BREAKDOWN
        sc->done = 1;
    } else {
        set_done(sc);
    }
}

// Start of one run of Fig. 1: clear the counters and set the loop bounds.
__global__ void cg_reset_kernel(CgScalars* scal, double threshold, double m2, float2 m2_ff,
                                long long max_iter) {
    scal->threshold = threshold;
    scal->m2 = m2;
    scal->m2_ff = m2_ff;
    scal->iter = 0;
    scal->max_iter = max_iter;
    scal->done = 0;
    scal->status = 0;
    scal->alpha = 0.0;
    scal->beta = 0.0;
    scal->alpha_ff = make_float2(0.f, 0.f);
    scal->beta_ff = make_float2(0.f, 0.f);
}

// ------------------------------------------------------------ FP64 set
__global__ void __launch_bounds__(kBlock) cg_init_kernel(Geom g, const double2* __restrict__ b,
                                                         const double2* __restrict__ ad,
                                                         double2* __restrict__ r, double2* __restrict__ d,
                                                         CgScalars* scal, double* partials) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    double acc = 0.0;
    if (i < g.vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            const double2 bb = b[k], aa = ad[k];
            const double2 rr = make_double2(bb.x - aa.x, bb.y - aa.y);
            r[k] = rr;
            d[k] = rr;
            acc = fma(rr.x, rr.x, acc);
            acc = fma(rr.y, rr.y, acc);
        }
    }
    double total;
    if (grid_sum_last_block<kBlock>(acc, partials, &scal->counter, &total)) {
        if (threadIdx.x == 0) {
            scal->delta_new = total;
            scal->delta_old = total;
            set_done(scal);
        }
    }
}

__global__ void __launch_bounds__(kBlock) cg_update_xr_kernel(Geom g, double2* __restrict__ x,
                                                              double2* __restrict__ r,
                                                              const double2* __restrict__ d,
                                                              const double2* __restrict__ ad,
                                                              CgScalars* scal, double* partials) {
    if (scal->done) return;
    const double alpha = scal->alpha;
    const size_t vs = (size_t)g.vs;
    double acc = 0.0;
    // grid-stride over sites (one resident wave of blocks: a short grid reduction)
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < g.vh; i += gridDim.x * kBlock) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            const double2 dd = __ldg(d + k);
            double2 xx = x[k];
            xx.x = fma(alpha, dd.x, xx.x);
            xx.y = fma(alpha, dd.y, xx.y);
            x[k] = xx;
            const double2 aa = __ldg(ad + k);
            double2 rr = r[k];
            rr.x = fma(-alpha, aa.x, rr.x);
            rr.y = fma(-alpha, aa.y, rr.y);
            r[k] = rr;
            acc = fma(rr.x, rr.x, acc);
            acc = fma(rr.y, rr.y, acc);
        }
    }
    double total;
    if (grid_sum_last_block<kBlock>(acc, partials, &scal->counter, &total)) {
        if (threadIdx.x == 0) finish_delta(scal, total);
    }
}

__global__ void __launch_bounds__(kBlock) cg_update_d_kernel(Geom g, const double2* __restrict__ r,
                                                             double2* __restrict__ d, CgScalars* scal) {
    if (scal->done) return;
    const double beta = scal->beta;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = c * vs + i;
        const double2 rr = __ldg(r + k);
        const double2 dd = d[k];
        d[k] = make_double2(fma(beta, dd.x, rr.x), fma(beta, dd.y, rr.y));
    }
}

// ------------------------------------------------------ float-float set
__global__ void __launch_bounds__(kBlock) cg_init_ff_kernel(Geom g, const double2* __restrict__ b,
                                                            const double2* __restrict__ ad,
                                                            float4* __restrict__ r, float4* __restrict__ d,
                                                            float4* __restrict__ xff, CgScalars* scal,
                                                            double* partials) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    double acc = 0.0;
    if (i < g.vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            const double2 bb = b[k], aa = ad[k];
            const double2 rr = make_double2(bb.x - aa.x, bb.y - aa.y);
            const float4 rf = ff_from_complex(rr);
            r[k] = rf;
            d[k] = rf;
            xff[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            acc = fma(rr.x, rr.x, acc);
            acc = fma(rr.y, rr.y, acc);
        }
    }
    double total;
    if (grid_sum_last_block<kBlock>(acc, partials, &scal->counter, &total)) {
        if (threadIdx.x == 0) {
            scal->delta_new = total;
            scal->delta_old = total;
            set_done(scal);
        }
    }
}

__global__ void __launch_bounds__(kBlock) cg_update_xr_ff_kernel(Geom g, float4* __restrict__ xff,
                                                                 float4* __restrict__ r,
                                                                 const float4* __restrict__ d,
                                                                 const float4* __restrict__ ad,
                                                                 CgScalars* scal, double* partials) {
    if (scal->done) return;
    const float2 alpha = scal->alpha_ff;
    const size_t vs = (size_t)g.vs;
    FFAcc n2 = ff_zero();
    // grid-stride over sites (one resident wave of blocks: a short grid reduction)
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < g.vh; i += gridDim.x * kBlock) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            xff[k] = ff_caxpy(alpha, __ldg(d + k), xff[k]);
            const float4 rr = ff_caxpy(ff_neg(alpha), __ldg(ad + k), r[k]);
            r[k] = rr;
            ff_norm2_acc(n2, rr);
        }
    }
    double total;
    if (grid_sum_last_block<kBlock>(ff_acc_to_double(n2), partials, &scal->counter, &total)) {
        if (threadIdx.x == 0) finish_delta(scal, total);
    }
}

__global__ void __launch_bounds__(kBlock) cg_update_d_ff_kernel(Geom g, const float4* __restrict__ r,
                                                                float4* __restrict__ d, CgScalars* scal) {
    if (scal->done) return;
    const float2 beta = scal->beta_ff;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = c * vs + i;
        d[k] = ff_caxpy(beta, d[k], __ldg(r + k));
    }
}

// x += x_ff (into FP64), x_ff = 0
__global__ void __launch_bounds__(kBlock) fold_x_kernel(Geom g, double2* __restrict__ x,
                                                        float4* __restrict__ xff) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = c * vs + i;
        const double2 a = ff_to_complex(xff[k]);
        double2 xx = x[k];
        xx.x += a.x;
        xx.y += a.y;
        x[k] = xx;
        xff[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ----------------------------------------------------------- utilities
__global__ void __launch_bounds__(kBlock) norm2_diff_kernel(Geom g, const double2* __restrict__ a,
                                                            const double2* __restrict__ b,
                                                            CgScalars* scal, double* partials) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    double acc = 0.0;
    if (i < g.vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            double2 v = a[k];
            if (b) {
                const double2 w = b[k];
                v.x -= w.x;
                v.y -= w.y;
            }
            acc = fma(v.x, v.x, acc);
            acc = fma(v.y, v.y, acc);
        }
    }
    double total;
    if (grid_sum_last_block<kBlock>(acc, partials, &scal->counter, &total)) {
        if (threadIdx.x == 0) scal->red_out = total;
    }
}

__global__ void __launch_bounds__(kBlock) to_ff_kernel(Geom g, const double2* __restrict__ in,
                                                       float4* __restrict__ out) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vs) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c * vs + i] = ff_from_complex(in[c * vs + i]);
}

__global__ void __launch_bounds__(kBlock) from_ff_kernel(Geom g, const float4* __restrict__ in,
                                                         double2* __restrict__ out) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vs) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c * vs + i] = ff_to_complex(in[c * vs + i]);
}

// ------------------------------------------------------------ launchers
int resident_wave_blocks() {
    static std::atomic<int> cached[64];  // per device ordinal; 0 = not yet queried
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1024;
    int n = cached[dev].load(std::memory_order_relaxed);
    if (!n) {
        int sms = 0, threads = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
        n = sms > 0 && threads > 0 ? sms * std::max(1, threads / kBlock) : 1024;
        cached[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

void launch_cg_reset(CgScalars* scal, double threshold, double m2, long long max_iter, cudaStream_t s) {
    cg_reset_kernel<<<1, 1, 0, s>>>(scal, threshold, m2, host_ff_from_double(m2), max_iter);
}

void launch_cg_init(const Geom& g, const double2* b, const double2* ad, double2* r, double2* d,
                    CgScalars* scal, double* partials, cudaStream_t s) {
    cg_init_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, b, ad, r, d, scal, partials);
}

void launch_cg_update_xr(const Geom& g, double2* x, double2* r, const double2* d, const double2* ad,
                         CgScalars* scal, double* partials, cudaStream_t s) {
    cg_update_xr_kernel<<<std::min(blocks_for(g.vh), resident_wave_blocks()), kBlock, 0, s>>>(g, x, r, d, ad, scal,
                                                                                             partials);
}

void launch_cg_update_d(const Geom& g, const double2* r, double2* d, CgScalars* scal, cudaStream_t s) {
    cg_update_d_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, r, d, scal);
}

void launch_cg_init_ff(const Geom& g, const double2* b, const double2* ad, float4* r, float4* d,
                       float4* xff, CgScalars* scal, double* partials, cudaStream_t s) {
    cg_init_ff_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, b, ad, r, d, xff, scal, partials);
}

void launch_cg_update_xr_ff(const Geom& g, float4* xff, float4* r, const float4* d, const float4* ad,
                            CgScalars* scal, double* partials, cudaStream_t s) {
    cg_update_xr_ff_kernel<<<std::min(blocks_for(g.vh), resident_wave_blocks()), kBlock, 0, s>>>(g, xff, r, d, ad,
                                                                                                scal, partials);
}

void launch_cg_update_d_ff(const Geom& g, const float4* r, float4* d, CgScalars* scal, cudaStream_t s) {
    cg_update_d_ff_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, r, d, scal);
}

void launch_fold_x(const Geom& g, double2* x, float4* xff, cudaStream_t s) {
    fold_x_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, x, xff);
}

void launch_norm2_diff(const Geom& g, const double2* a, const double2* b, CgScalars* scal,
                       double* partials, cudaStream_t s) {
    norm2_diff_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, a, b, scal, partials);
}

void launch_to_ff(const Geom& g, const double2* in, float4* out, cudaStream_t s) {
    to_ff_kernel<<<blocks_for(g.vs), kBlock, 0, s>>>(g, in, out);
}

void launch_from_ff(const Geom& g, const float4* in, double2* out, cudaStream_t s) {
    from_ff_kernel<<<blocks_for(g.vs), kBlock, 0, s>>>(g, in, out);
}

}  // namespace stag
