// fcg.cu - flexible CG with the learned preconditioner M (pt.cu), driven on
// the device (stag_fcg_solve).
//
// Flexible CG (Notay 2000) with the Polak-Ribiere beta, from r = b - A x,
// z = M r, p = z:
//   q = A p;  alpha = (r, z) / (p, q);  x += alpha p;  r_new = r - alpha q;
//   z_new = M r_new;  beta = (z_new, r_new - r) / (r, z);  p = z_new + beta p.
// Since r_new - r = -alpha q, beta is computed as -alpha (z_new, q) / (r, z),
// so the old residual is never stored.  The paper's CG (Sec. 2, Fig. 1) has no
// preconditioner; the vectors, the operator A = m^2 - D_eo D_oe and its
// kernels are the plain solver's, in the handle's arithmetic (float-float or
// FP64).
//
// Every scalar stays on the device, in the CG state the Dirac kernels'
// reduction epilogue already fills ((p, A p) and alpha) plus a small
// flexible-CG record: per iteration
//   D_oe p, D_eo with (p, q) and alpha  (dslash.cu),
//   x, r update with |r|^2 and the stopping rules  (fcg_update_kernel),
//   the network on r  (pt.cu, pt_tc.cu),
//   (z, r) and (z, q) with beta  (fcg_zdots_kernel),
//   p = z + beta p  (fcg_dir_kernel).
// Blocks of check_interval iterations are captured once as a CUDA graph; the
// host reads the state between blocks only.  Once a rule stops the cycle,
// every later kernel of the block returns at once (the network's too).
//
// Stopping rules of a cycle (evaluated after each update): |r| <= tol |b|;
// the iteration budget; (p, A p) <= 0 or a non-finite |r|^2 (breakdown);
// (r, z) <= 0; the best |r| not 10 % lower than it was 100 iterations ago
// (stall).  Then the true residual is recomputed in native FP64; a cycle that
// stalled after cutting the residual 100-fold restarts flexible CG from the
// current x, any other early stop hands over to plain CG (the solver's
// fallback), and the FP64 true residual decides the result.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <type_traits>

#include "../../include/stag.h"
#include "ff.cuh"
#include "handle.h"
#include "pt_net.h"
#include "stag_kernels.h"

namespace stag {
namespace {

// Vector arithmetic of the two forms: float-float (float4, sums of exact
// products on the FP32 pipes) and FP64 (double2).
template <class V>
struct Arith;

template <>
struct Arith<float4> {
    using Acc = FFAcc;
    static __device__ __forceinline__ Acc zero() { return ff_zero(); }
    static __device__ __forceinline__ void norm(Acc& a, float4 v) { ff_norm2_acc(a, v); }
    // a += Re(conj(z) v), z an FP32 complex
    static __device__ __forceinline__ void zdot(Acc& a, float2 z, float4 v) {
        ff_mac(a, z.x, 0.f, v.x, v.y);
        ff_mac(a, z.y, 0.f, v.z, v.w);
    }
    static __device__ __forceinline__ double total(const Acc& a) { return ff_acc_to_double(a); }
    // s a + b, the scalar given in FP64 and as a float-float pair
    static __device__ __forceinline__ float4 axpy(double, float2 s, float4 a, float4 b) { return ff_caxpy(s, a, b); }
    static __device__ __forceinline__ float4 from_z(float2 z) { return make_float4(z.x, 0.f, z.y, 0.f); }
    static __device__ __forceinline__ float4 from_c64(double2 v) { return ff_from_complex(v); }
    static __device__ __forceinline__ float4 zero_v() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    static __device__ __forceinline__ float2 f2(float4 v) { return make_float2(v.x + v.y, v.z + v.w); }
};

template <>
struct Arith<double2> {
    using Acc = double;
    static __device__ __forceinline__ Acc zero() { return 0.0; }
    static __device__ __forceinline__ void norm(Acc& a, double2 v) { a = fma(v.x, v.x, fma(v.y, v.y, a)); }
    static __device__ __forceinline__ void zdot(Acc& a, float2 z, double2 v) {
        a = fma((double)z.x, v.x, fma((double)z.y, v.y, a));
    }
    static __device__ __forceinline__ double total(const Acc& a) { return a; }
    static __device__ __forceinline__ double2 axpy(double s, float2, double2 a, double2 b) {
        return make_double2(fma(s, a.x, b.x), fma(s, a.y, b.y));
    }
    static __device__ __forceinline__ double2 from_z(float2 z) { return make_double2(z.x, z.y); }
    static __device__ __forceinline__ double2 from_c64(double2 v) { return v; }
    static __device__ __forceinline__ double2 zero_v() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ float2 f2(double2 v) { return make_float2((float)v.x, (float)v.y); }
};

// Two grid sums at once: per-block partials of a and b, then the last block to
// finish adds them in block order (deterministic).  True in every thread of
// that block, with the sums in out[0..1].
__device__ __forceinline__ bool grid_sum2_last_block(double a, double b, double* partials, unsigned int* counter,
                                                     double* out) {
    __shared__ double sm[kBlock / 32];
    __shared__ bool is_last;
    __shared__ double res[2];
    a = block_sum<kBlock>(a, sm);
    __syncthreads();
    b = block_sum<kBlock>(b, sm);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
        __threadfence();
        is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double sa = 0.0, sb = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += kBlock) {
        sa += __ldcg(partials + 2 * k);
        sb += __ldcg(partials + 2 * k + 1);
    }
    __syncthreads();
    sa = block_sum<kBlock>(sa, sm);
    __syncthreads();
    sb = block_sum<kBlock>(sb, sm);
    if (threadIdx.x == 0) {
        res[0] = sa;
        res[1] = sb;
        *counter = 0u;
    }
    __syncthreads();
    out[0] = res[0];
    out[1] = res[1];
    return true;
}

// Start of a cycle: r = b - A x (A x from the native FP64 kernels), x_acc = 0
// (float-float accumulator; nullptr for FP64, where x is updated in place),
// |r|^2 and the stall record.
template <class V>
__global__ void __launch_bounds__(kBlock) fcg_start_kernel(Geom g, const double2* __restrict__ b,
                                                           const double2* __restrict__ ax, V* __restrict__ r,
                                                           V* __restrict__ xacc, FcgDev* d, double* partials) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    double acc = 0.0;
    if (i < g.vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            const double2 bb = b[k], aa = ax[k];
            const double2 rr = make_double2(bb.x - aa.x, bb.y - aa.y);
            r[k] = Arith<V>::from_c64(rr);
            if (xacc) xacc[k] = Arith<V>::zero_v();
            acc = fma(rr.x, rr.x, fma(rr.y, rr.y, acc));
        }
    }
    double total;
    if (grid_sum_last_block<kBlock>(acc, partials, &d->sc.counter, &total)) {
        if (threadIdx.x == 0) {
            d->st.rr = total;
            d->st.best = total;
            d->st.mark = total;
            d->st.mark_it = 0;
            d->st.why = FCG_WHY_NONE;
        }
    }
}

// The stopping rules after an update with |r|^2 = rr (one thread).
__device__ __forceinline__ void after_update(FcgDev* d, double rr) {
    CgScalars& sc = d->sc;
    FcgState& st = d->st;
    st.rr = rr;
    sc.iter += 1;
    if (!isfinite(rr)) {
        sc.status = STAG_ERR_BREAKDOWN;
        sc.done = 1;
        return;
    }
    if (rr <= sc.threshold || sc.iter >= sc.max_iter) {
        sc.done = 1;
        return;
    }
    st.best = fmin(st.best, rr);
    if (st.best < 0.81 * st.mark) {  // |r| 10 % below the last mark
        st.mark = st.best;
        st.mark_it = sc.iter;
    } else if (sc.iter - st.mark_it > 100) {
        st.why = FCG_WHY_STALL;
        sc.done = 1;
    }
}

// x_acc += alpha p; r -= alpha q; |r|^2; the stopping rules.
template <class V>
__global__ void __launch_bounds__(kBlock) fcg_update_kernel(Geom g, V* __restrict__ xacc, V* __restrict__ r,
                                                            const V* __restrict__ p, const V* __restrict__ q,
                                                            FcgDev* d, double* partials) {
    if (d->sc.done) return;
    const double alpha = d->sc.alpha;
    const float2 alpha_ff = d->sc.alpha_ff;
    const size_t vs = (size_t)g.vs;
    typename Arith<V>::Acc n2 = Arith<V>::zero();
    // grid-stride over sites (one resident wave of blocks: a short grid reduction)
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < g.vh; i += gridDim.x * kBlock) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            xacc[k] = Arith<V>::axpy(alpha, alpha_ff, __ldg(p + k), xacc[k]);
            const V rr = Arith<V>::axpy(-alpha, ff_neg(alpha_ff), __ldg(q + k), r[k]);
            r[k] = rr;
            Arith<V>::norm(n2, rr);
        }
    }
    double total;
    if (grid_sum_last_block<kBlock>(Arith<V>::total(n2), partials, &d->sc.counter, &total)) {
        if (threadIdx.x == 0) after_update(d, total);
    }
}

// rz = (z, r) = tot[0]; beta = -alpha (z, q) / rz_old with (z, q) = tot[1]
// (start: beta = 0); the cycle stops if (z, r) <= 0 (one thread).
__device__ __forceinline__ void finish_zdots(FcgDev* d, const double (&tot)[2], int start) {
    CgScalars& sc = d->sc;
    const double beta = start ? 0.0 : -sc.alpha * tot[1] / sc.delta_new;
    sc.delta_new = tot[0];
    sc.beta = beta;
    sc.beta_ff = ff_from_double(beta);
    if (!(tot[0] > 0.0) || !isfinite(beta)) {
        d->st.why = FCG_WHY_RZ;
        sc.done = 1;
    }
}

// (z, r) and (z, q) over even sites, z = the network's output (act3, even
// sites [3][vs]); the last block sets rz = (z, r) and beta = -alpha (z, q) / rz_old
// (start: beta = 0, no q) and stops the cycle if (z, r) <= 0.
template <class V, class T>
__global__ void __launch_bounds__(kBlock) fcg_zdots_kernel(Geom g, const T* __restrict__ z, const V* __restrict__ r,
                                                           const V* __restrict__ q, FcgDev* d, double* partials,
                                                           int start) {
    if (d->sc.done) return;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    typename Arith<V>::Acc zr = Arith<V>::zero(), zq = Arith<V>::zero();
    if (i < g.vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            const float2 zz = ldc(z + k);
            Arith<V>::zdot(zr, zz, r[k]);
            if (!start) Arith<V>::zdot(zq, zz, q[k]);
        }
    }
    double tot[2];
    if (grid_sum2_last_block(Arith<V>::total(zr), Arith<V>::total(zq), partials, &d->sc.counter, tot)) {
        if (threadIdx.x == 0) finish_zdots(d, tot, start);
    }
}

// Collapsed form of the network, fused: z = k0 r + sum_p T_p chi_p on even
// sites (pt_out_site; chi from pt_chi_kernel), stored in FP32, with (z, r),
// (z, q) and beta as in fcg_zdots_kernel.
template <class V, class TS, class L>
__global__ void __launch_bounds__(kBlock) fcg_out_kernel(Geom g, const L* __restrict__ links,
                                                         const float2* __restrict__ coef, const TS* __restrict__ chi,
                                                         const V* __restrict__ r, const V* __restrict__ q,
                                                         float2* __restrict__ z, FcgDev* d, double* partials,
                                                         int start) {
    if (d->sc.done) return;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    typename Arith<V>::Acc zr = Arith<V>::zero(), zq = Arith<V>::zero();
    if (i < g.vh) {
        V rv[3];
        float2 r0[3], zz[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rv[c] = r[c * vs + i];
            r0[c] = Arith<V>::f2(rv[c]);
        }
        pt_out_site(g, links, coef[0], chi, i, r0, zz);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = c * vs + i;
            z[k] = zz[c];
            Arith<V>::zdot(zr, zz[c], rv[c]);
            if (!start) Arith<V>::zdot(zq, zz[c], q[k]);
        }
    }
    double tot[2];
    if (grid_sum2_last_block(Arith<V>::total(zr), Arith<V>::total(zq), partials, &d->sc.counter, tot)) {
        if (threadIdx.x == 0) finish_zdots(d, tot, start);
    }
}

// p = z + beta p (start: p = z)
template <class V, class T>
__global__ void __launch_bounds__(kBlock) fcg_dir_kernel(Geom g, const T* __restrict__ z, V* __restrict__ p,
                                                         const FcgDev* d, int start) {
    if (d->sc.done) return;
    const double beta = d->sc.beta;
    const float2 beta_ff = d->sc.beta_ff;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = c * vs + i;
        const V zz = Arith<V>::from_z(ldc(z + k));
        p[k] = start ? zz : Arith<V>::axpy(beta, beta_ff, p[k], zz);
    }
}

// ------------------------------------------------------------------ host
struct Vecs {
    void *r, *p, *q, *t, *xacc;
};

Vecs vecs(stag_ptnet* n, bool ff) {
    return Vecs{n->fcg_r, n->fcg_p, n->fcg_q, n->fcg_t, ff ? n->fcg_x : static_cast<void*>(n->h->x)};
}

LinkSet handle_links(const stag_handle* h) { return LinkSet{h->fat64, h->lng64, h->fatff, h->lngff, h->lng_s}; }

// q = A p with (p, q) and alpha in the CG state (t: odd-parity scratch)
void enqueue_A(stag_handle* h, FcgDev* d, const float4* p, float4* t, float4* q) {
    const LinkSet L = handle_links(h);
    launch_dslash_ff(h->g, 1, L, p, t, EPI_PLAIN, nullptr, 0.0, &d->sc, h->partials, h->s);
    launch_dslash_ff(h->g, 0, L, t, q, EPI_CG, p, 0.0, &d->sc, h->partials, h->s);
}
void enqueue_A(stag_handle* h, FcgDev* d, const double2* p, double2* t, double2* q) {
    const LinkSet L = handle_links(h);
    launch_dslash_f64(h->g, 1, L, p, t, EPI_PLAIN, nullptr, 0.0, &d->sc, h->partials, h->s);
    launch_dslash_f64(h->g, 0, L, t, q, EPI_CG, p, 0.0, &d->sc, h->partials, h->s);
}

// z = M r, rz = (z, r), beta (start: 0) and p = z + beta p (start: p = z).
// Collapsed form: chi, then z fused with the dots; layered: the network's
// three layers (or two and the final transports), then the dots.
template <class V, class T>
void enqueue_precond(stag_ptnet* n, const V* r, const V* q, int start) {
    stag_handle* h = n->h;
    const Geom& g = h->g;
    FcgDev* d = n->fcg_dev;
    V* p = static_cast<V*>(n->fcg_p);
    if (n->inf_form == STAG_PTNET_COLLAPSED) {
        float2* z = static_cast<float2*>(n->act[kLayers]);
        launch_pt_chi(n, r, &d->sc.done);
        if constexpr (std::is_same<T, __nv_bfloat162>::value)  // FP16 links with BF16 storage
            fcg_out_kernel<V, T, __half2><<<blocks_for(g.vh), kBlock, 0, h->s>>>(
                g, n->links16, n->coef, static_cast<const T*>(n->act[2]), r, q, z, d, h->partials, start);
        else
            fcg_out_kernel<V, T, float2><<<blocks_for(g.vh), kBlock, 0, h->s>>>(
                g, n->links, n->coef, static_cast<const T*>(n->act[2]), r, q, z, d, h->partials, start);
        fcg_dir_kernel<V, float2><<<blocks_for(g.vh), kBlock, 0, h->s>>>(g, z, p, d, start);
    } else {
        const T* z = static_cast<const T*>(n->act[kLayers]);
        pt_network_from_vec(n, r, &d->sc.done);
        fcg_zdots_kernel<V, T><<<blocks_for(g.vh), kBlock, 0, h->s>>>(g, z, r, q, d, h->partials, start);
        fcg_dir_kernel<V, T><<<blocks_for(g.vh), kBlock, 0, h->s>>>(g, z, p, d, start);
    }
}

// One flexible-CG iteration: six kernels with the collapsed network, eight or
// nine with the layered one.
template <class V, class T>
void enqueue_iteration(stag_ptnet* n, const Vecs& v) {
    stag_handle* h = n->h;
    const Geom& g = h->g;
    FcgDev* d = n->fcg_dev;
    V* r = static_cast<V*>(v.r);
    V* p = static_cast<V*>(v.p);
    V* q = static_cast<V*>(v.q);
    enqueue_A(h, d, p, static_cast<V*>(v.t), q);
    fcg_update_kernel<V><<<std::min(blocks_for(g.vh), resident_wave_blocks()), kBlock, 0, h->s>>>(
        g, static_cast<V*>(v.xacc), r, p, q, d, h->partials);
    enqueue_precond<V, T>(n, r, q, 0);
}

// check_interval iterations, then (float-float) the fold of x_acc into x
template <class V, class T>
void enqueue_block(stag_ptnet* n, const Vecs& v, int K) {
    for (int k = 0; k < K; ++k) enqueue_iteration<V, T>(n, v);
    if constexpr (std::is_same<V, float4>::value) launch_fold_x(n->g, n->h->x, static_cast<float4*>(v.xacc), n->h->s);
}

void read_state(stag_ptnet* n) {
    pcheck(n, cudaMemcpyAsync(n->fcg_host, n->fcg_dev, sizeof(FcgDev), cudaMemcpyDeviceToHost, S(n)), "read FCG state");
    pcheck(n, cudaStreamSynchronize(S(n)), "sync");
}

template <class V, class T>
void ensure_graph(stag_ptnet* n, const Vecs& v, int K, int key) {
    if (n->fcg_graph && n->fcg_graph_key == key) return;
    if (n->fcg_graph) {
        cudaGraphExecDestroy(n->fcg_graph);
        n->fcg_graph = nullptr;
    }
    cudaGraph_t graph = nullptr;
    pcheck(n, cudaStreamBeginCapture(S(n), cudaStreamCaptureModeThreadLocal), "begin capture");
    enqueue_block<V, T>(n, v, K);
    pcheck(n, cudaStreamEndCapture(S(n), &graph), "end capture");
    const cudaError_t e = cudaGraphInstantiate(&n->fcg_graph, graph, 0);
    cudaGraphDestroy(graph);
    pcheck(n, e, "graph instantiate");
    n->fcg_graph_key = key;
}

struct Outcome {
    long long iters = 0;
    int restarts = 0, fallbacks = 0, status = STAG_OK;
    double rel = 0.0;
};

template <class V, class T>
Outcome solve(stag_ptnet* n, double bnorm2, double tol, long long max_it) {
    stag_handle* h = n->h;
    const Geom& g = h->g;
    constexpr bool ff = std::is_same<V, float4>::value;
    const Vecs v = vecs(n, ff);
    FcgDev* d = n->fcg_dev;
    const FcgDev& hs = *n->fcg_host;
    const int K = std::max(1, h->opt.check_interval);
    const bool graphs = h->opt.use_graphs != 0;
    const bool collapsed = n->inf_form == STAG_PTNET_COLLAPSED;
    if (collapsed) pt_collapse(n);  // the weights do not change during a solve
    if (graphs)
        ensure_graph<V, T>(n, v, K,
                           (((K * 2 + (ff ? 1 : 0)) * 2 + (infer_bf16(n) ? 1 : 0)) * 2 + (n->use_tc ? 1 : 0)) * 2 +
                               (collapsed ? 1 : 0));
    Outcome o;
    bool use_plain = false;
    while (true) {
        // r = b - A x with native FP64 arithmetic
        handle_apply_A_f64(h, h->x, n->fq);
        fcg_start_kernel<V><<<blocks_for(g.vh), kBlock, 0, h->s>>>(g, h->b, n->fq, static_cast<V*>(v.r),
                                                                    ff ? static_cast<V*>(v.xacc) : nullptr, d,
                                                                    h->partials);
        read_state(n);
        o.rel = std::sqrt(hs.st.rr / bnorm2);
        const double cycle_start_rel = o.rel;
        if (o.rel <= tol) break;
        if (o.iters >= max_it) {
            o.status = STAG_ERR_NOT_CONVERGED;
            break;
        }
        if (use_plain) {
            // plain FP64-class CG from the current x, stopped by its own FP64 residual
            stag_solve_info pi{};
            o.status = handle_solve_packed(h, bnorm2, tol, max_it - o.iters, pi);
            o.iters += pi.iters;
            o.rel = pi.true_rel_residual;
            break;
        }
        // z = M r, p = z, (r, z)
        launch_cg_reset(&d->sc, tol * tol * bnorm2, h->mass * h->mass, max_it - o.iters, h->s);
        enqueue_precond<V, T>(n, static_cast<const V*>(v.r), nullptr, 1);
        pcheck(n, cudaGetLastError(), "flexible CG start");
        read_state(n);
        while (!hs.sc.done) {
            if (graphs) {
                pcheck(n, cudaGraphLaunch(n->fcg_graph, S(n)), "cudaGraphLaunch");
            } else {
                enqueue_block<V, T>(n, v, K);
                pcheck(n, cudaGetLastError(), "flexible CG iteration");
            }
            read_state(n);
        }
        o.iters += hs.sc.iter;
        if (hs.sc.status == STAG_OK && hs.st.why == FCG_WHY_NONE) continue;  // converged or out of budget
        // an early stop: restart after a 100-fold cut by a stalled cycle, else plain CG
        const double rel_now = std::sqrt(hs.st.rr / bnorm2);
        const bool progress = hs.sc.status == STAG_OK && hs.st.why == FCG_WHY_STALL && rel_now < 0.01 * cycle_start_rel;
        if (std::getenv("STAG_DEBUG")) {
            const char* why = hs.sc.status != STAG_OK ? "(p, A p) <= 0 or a non-finite residual"
                              : hs.st.why == FCG_WHY_RZ ? "(r, z) <= 0"
                                                        : "no 10 % drop of the best residual in 100 iterations";
            std::fprintf(stderr, "stag_fcg_solve: %s after %lld iterations: %s (|r|/|b| = %.3e)\n",
                         progress ? "restart" : "fallback to plain CG", o.iters, why, rel_now);
        }
        if (progress) {
            ++o.restarts;
        } else {
            use_plain = true;
            ++o.fallbacks;
        }
    }
    return o;
}

}  // namespace
}  // namespace stag

using namespace stag;

extern "C" int stag_fcg_solve(stag_handle* h, stag_ptnet* n, const double* b_even, double* x_even, double tol,
                              int32_t max_iter, stag_solve_info* info) {
    if (!h || !n || n->h != h || !b_even || !x_even || b_even == x_even) return STAG_ERR_INVALID_ARG;
    NvtxRange range("stag_fcg_solve");
    if (!(tol > 0.0) || !std::isfinite(tol)) return STAG_ERR_INVALID_ARG;
    stag_solve_info inf{};
    int status = STAG_OK;
    const auto t0 = std::chrono::steady_clock::now();
    try {
        handle_begin(h);
        const Geom& g = h->g;
        const size_t ab = (size_t)3 * g.vh * sizeof(double2);
        const bool x_dev = handle_is_device_ptr(h, x_even);
        const double* bs = b_even;
        if (!handle_is_device_ptr(h, bs)) {
            pcheck(n, cudaMemcpyAsync(h->io_a, bs, ab, cudaMemcpyHostToDevice, S(n)), "copy b");
            bs = h->io_a;
        }
        launch_pack_vec(g, bs, h->b, S(n));
        const double* xs = x_even;
        if (!x_dev) {
            pcheck(n, cudaMemcpyAsync(h->io_b, xs, ab, cudaMemcpyHostToDevice, S(n)), "copy x");
            xs = h->io_b;
        }
        launch_pack_vec(g, xs, h->x, S(n));
        launch_norm2_diff(g, h->b, nullptr, &n->fcg_dev->sc, h->partials, S(n));
        read_state(n);
        const double bnorm2 = n->fcg_host->sc.red_out;
        if (!std::isfinite(bnorm2)) pfail(n, STAG_ERR_INVALID_ARG, "source has non-finite entries");
        const long long max_it = max_iter > 0 ? max_iter : 3LL * g.vh;
        if (bnorm2 == 0.0) {
            pcheck(n, cudaMemsetAsync(h->x, 0, (size_t)3 * g.vs * sizeof(double2), S(n)), "zero x");
        } else {
            const bool ff = h->opt.arith == STAG_ARITH_FF && h->fatff;
            Outcome o;
            if (ff)
                o = infer_bf16(n) ? solve<float4, __nv_bfloat162>(n, bnorm2, tol, max_it)
                                  : solve<float4, float2>(n, bnorm2, tol, max_it);
            else
                o = infer_bf16(n) ? solve<double2, __nv_bfloat162>(n, bnorm2, tol, max_it)
                                  : solve<double2, float2>(n, bnorm2, tol, max_it);
            status = o.status;
            inf.iters = (int32_t)o.iters;
            inf.restarts = o.restarts;
            inf.fallbacks = o.fallbacks;
            inf.true_rel_residual = o.rel;
            inf.iter_rel_residual = o.rel;
        }
        if (status == STAG_ERR_NOT_CONVERGED) h->err = "flexible CG: not converged";
        launch_unpack_vec(g, h->x, x_dev ? x_even : h->io_b, S(n));
        if (!x_dev) pcheck(n, cudaMemcpyAsync(x_even, h->io_b, ab, cudaMemcpyDeviceToHost, S(n)), "copy x");
        pcheck(n, cudaGetLastError(), "flexible CG");
        check_tc(n);
        handle_end(h);
    } catch (const PFail& f) {
        status = f.code;
        h->err = n->err;
    } catch (const HandleError& f) {
        status = f.code;
    }
    inf.status = status;
    inf.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return status;
}
