// batch_dev.cu - the batched solver's reliable updates, decided and applied on
// the device.
//
// Each system of a batch runs the mixed-precision CG of blas_lo.cu (FP32
// iteration, FP64-class true residuals): when its iterated residual has dropped
// by reliable_delta, after reliable_interval iterations, or once it meets the
// tolerance, the inner iteration marks it (CgScalars::done = 2) and idles.  The
// pass below, enqueued after every iteration inside the captured graph, then
//   1. selects the marked systems (one thread; builds device-side lists),
//   2. folds their FP32 solution increments into x (FP64),
//   3. computes b - A x in float-float arithmetic (the list Dirac kernels of
//      dslash.cu) and its norm, writing the FP32 residual into the system's slot,
//   4. decides per system: converged candidates are confirmed with native FP64
//      Dirac kernels; the others (or candidates that fail the confirmation)
//      replace the iterated residual - d = r + beta d with beta from the true
//      residual, the inner CG state reset - and resume at the next iteration;
//      non-finite residuals and exhausted iteration budgets finish the system;
//   5. counts the systems still running into a host-mapped word.
// No step returns to the host, so a system whose replacement falls due waits
// at most one iteration, and the host only reads that word between graph
// launches.  The per-system sums are taken over fixed tiles in tile order, so
// the pass is deterministic.
#include <cuda_runtime.h>

#include "ff.cuh"
#include "multi.cuh"

namespace stag {

namespace {

constexpr int kTile = kBlock;  // sites per tile of the list kernels

// Entry j of a list of n entries whose tile range [prefix[j], prefix[j + 1])
// holds `tile` (0 <= tile < prefix[n]; prefix ascending): binary search.
__device__ __forceinline__ int list_entry(const int* prefix, int n, int tile) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void list_reset(PassList L) { *L.count = 0, L.prefix[0] = 0; }

__device__ __forceinline__ void list_add(PassList L, int k, int vh) {
    const int n = *L.count;
    L.sys[n] = k;
    L.prefix[n + 1] = L.prefix[n] + (vh + kTile - 1) / kTile;
    *L.count = n + 1;
}

// Sum of a block's values (kTile threads), valid in thread 0; fixed order.
__device__ __forceinline__ double tile_sum(double v) {
    __shared__ double ws[kTile / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kTile / 32; ++k) s += ws[k];
    __syncthreads();
    return s;
}

// Sum of the tile partials of list entry j, by one warp, in a fixed order.
__device__ __forceinline__ double entry_sum(const double* partials, const int* prefix, int j) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int t = prefix[j] + lane; t < prefix[j + 1]; t += 32) s += partials[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// The replacement of system k's iterated residual by its true residual
// (squared norm st.dtrue), or the end of the system when its iteration budget
// is spent.  Sets the inner CG state for the next run (blas_lo.cu's reset);
// the vectors follow in pass_set_residual_kernel.
__device__ void replace_or_stop(const PassArgs& a, int k) {
    SysState& st = a.state[k];
    CgScalars& sc = a.scal[k];
    if (st.iters >= st.max_iter) {
        st.status = STAG_STATUS_NOT_CONVERGED;
        st.phase = SYS_FINISHED;
        sc.done = 1;
        return;
    }
    st.beta = st.first ? 0.0 : st.dtrue / sc.delta_old;
    if (!st.first) st.updates += 1;
    st.phase = SYS_REPLACE;
    sc.delta_new = st.dtrue;
    sc.delta_old = st.dtrue;
    sc.threshold = st.tol2;
    sc.m2 = a.sys[k].m2;
    sc.m2_ff = ff_from_double(a.sys[k].m2);
    sc.iter = 0;
    sc.max_iter = st.max_iter - st.iters;
    sc.iter_since = 0;
    sc.rel_interval = st.rel_interval;
    sc.rel_delta = st.rel_delta;
    sc.maxr = sqrt(st.dtrue);
    sc.status = 0;
    sc.done = 0;  // the next iteration kernels run after the vectors are set
}

// 1. systems marked by the inner iteration (or not started) -> fold and FF lists
__global__ void pass_select_kernel(PassArgs a) {
    if (threadIdx.x != 0) return;
    list_reset(a.fold);
    list_reset(a.ff);
    for (int k = 0; k < a.n_sys; ++k) {
        SysState& st = a.state[k];
        const CgScalars& sc = a.scal[k];
        if (st.phase == SYS_RUNNING && sc.done != 0) {
            st.iters += sc.iter;
            if (sc.status != 0) {
                st.status = STAG_STATUS_BREAKDOWN;
                st.phase = SYS_FINISHED;  // keep the iterate: fold, no replacement
                list_add(a.fold, k, a.sys[k].g.vh);
                continue;
            }
            st.phase = SYS_DUE;
        } else if (st.phase == SYS_START) {
            st.phase = SYS_DUE;
        }
        if (st.phase == SYS_DUE) {
            list_add(a.fold, k, a.sys[k].g.vh);
            list_add(a.ff, k, a.sys[k].g.vh);
        }
    }
}

// 2. x += y[slot]; y[slot] = 0
__global__ void __launch_bounds__(kTile) pass_fold_kernel(PassArgs a) {
    const int n = *a.fold.count, total = a.fold.prefix[n];
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int j = list_entry(a.fold.prefix, n, tile);
        const SysDev& s = a.sys[a.fold.sys[j]];
        const int i = (tile - a.fold.prefix[j]) * kTile + threadIdx.x;
        if (i >= s.g.vh) continue;
        const size_t vs = (size_t)s.g.vs;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2* yp = s.y + ((size_t)c * vs + i) * s.rpad + s.slot;
            const float2 yy = *yp;
            double2 xx = s.x64[(size_t)c * vs + i];
            xx.x += (double)yy.x;
            xx.y += (double)yy.y;
            s.x64[(size_t)c * vs + i] = xx;
            *yp = make_float2(0.f, 0.f);
        }
    }
}

// 3a. u = x as float-float
__global__ void __launch_bounds__(kTile) pass_to_ff_kernel(PassArgs a) {
    const int n = *a.ff.count, total = a.ff.prefix[n];
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int j = list_entry(a.ff.prefix, n, tile);
        const SysDev& s = a.sys[a.ff.sys[j]];
        const int i = (tile - a.ff.prefix[j]) * kTile + threadIdx.x;
        if (i >= s.g.vh) continue;
        const size_t vs = (size_t)s.g.vs;
#pragma unroll
        for (int c = 0; c < 3; ++c) s.u_ff[(size_t)c * vs + i] = ff_from_complex(s.x64[(size_t)c * vs + i]);
    }
}

// 3c. r = b - A x (A x float-float in ax, or FP64 when f64): the FP32 residual
// into the system's slot (FF case), |r|^2 per tile into partials
template <bool F64>
__global__ void __launch_bounds__(kTile) pass_residual_kernel(PassArgs a, PassList L) {
    const int n = *L.count, total = L.prefix[n];
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int j = list_entry(L.prefix, n, tile);
        const SysDev& s = a.sys[L.sys[j]];
        const int i = (tile - L.prefix[j]) * kTile + threadIdx.x;
        double acc = 0.0;
        if (i < s.g.vh) {
            const size_t vs = (size_t)s.g.vs;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t k = (size_t)c * vs + i;
                const double2 ax = F64 ? reinterpret_cast<const double2*>(s.ax)[k] : ff_to_complex(s.ax[k]);
                const double2 bb = s.b64[k];
                const double2 r = make_double2(bb.x - ax.x, bb.y - ax.y);
                acc = fma(r.x, r.x, acc);
                acc = fma(r.y, r.y, acc);
                if (!F64) s.r[k * s.rpad + s.slot] = make_float2((float)r.x, (float)r.y);
            }
        }
        const double tot = tile_sum(acc);
        if (threadIdx.x == 0) a.partials[tile] = tot;
    }
}

// 4a. true residuals of the FF list: finished, to be confirmed, or replaced;
// then the list of systems to confirm
__global__ void pass_decide_kernel(PassArgs a) {
    const int n = *a.ff.count;
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = w; j < n; j += nw) {
        const double dtrue = entry_sum(a.partials, a.ff.prefix, j);
        if ((threadIdx.x & 31) != 0) continue;
        const int k = a.ff.sys[j];
        SysState& st = a.state[k];
        st.dtrue = dtrue;
        st.rel = sqrt(dtrue / st.bnorm2);
        if (!isfinite(dtrue)) {
            st.status = STAG_STATUS_BREAKDOWN;
            st.phase = SYS_FINISHED;
            a.scal[k].done = 1;
        } else if (st.rel <= st.tol) {
            st.phase = SYS_CONFIRM;
        } else {
            replace_or_stop(a, k);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        list_reset(a.confirm);
        for (int j = 0; j < n; ++j) {
            const int k = a.ff.sys[j];
            if (a.state[k].phase == SYS_CONFIRM) list_add(a.confirm, k, a.sys[k].g.vh);
        }
    }
}

// 4c. confirmations: finished with the native-FP64 residual, or replaced; then
// the list of systems whose vectors are to be replaced, and the running count
__global__ void pass_confirm_kernel(PassArgs a) {
    const int n = *a.confirm.count;
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = w; j < n; j += nw) {
        const double d64 = entry_sum(a.partials, a.confirm.prefix, j);
        if ((threadIdx.x & 31) != 0) continue;
        const int k = a.confirm.sys[j];
        SysState& st = a.state[k];
        const double rel = sqrt(d64 / st.bnorm2);
        st.rel = rel;
        if (rel <= st.tol) {
            st.status = STAG_STATUS_OK;
            st.phase = SYS_FINISHED;
            a.scal[k].done = 1;
        } else {
            replace_or_stop(a, k);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        list_reset(a.replace);
        int running = 0;
        for (int k = 0; k < a.n_sys; ++k) {
            const int ph = a.state[k].phase;
            if (ph == SYS_REPLACE) list_add(a.replace, k, a.sys[k].g.vh);
            if (ph != SYS_FINISHED) ++running;
        }
        *a.running = running;
    }
}

// 4d. d[slot] = r[slot] (first) or r[slot] + beta d[slot]; y[slot] = 0; the
// system runs again from the next iteration
__global__ void __launch_bounds__(kTile) pass_set_residual_kernel(PassArgs a) {
    const int n = *a.replace.count, total = a.replace.prefix[n];
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int j = list_entry(a.replace.prefix, n, tile);
        const int k = a.replace.sys[j];
        const SysDev& s = a.sys[k];
        const SysState& st = a.state[k];
        const int i = (tile - a.replace.prefix[j]) * kTile + threadIdx.x;
        if (i >= s.g.vh) continue;
        const size_t vs = (size_t)s.g.vs;
        const float beta = (float)st.beta;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t q = ((size_t)c * vs + i) * s.rpad + s.slot;
            const float2 rr = s.r[q];
            if (st.first) {
                s.d[q] = rr;
            } else {
                const float2 dd = s.d[q];
                s.d[q] = make_float2(fmaf(beta, dd.x, rr.x), fmaf(beta, dd.y, rr.y));
            }
            s.y[q] = make_float2(0.f, 0.f);
        }
    }
}

// 5. replaced systems resume: phase running, first replacement done
__global__ void pass_resume_kernel(PassArgs a) {
    if (threadIdx.x != 0) return;
    const int n = *a.replace.count;
    for (int j = 0; j < n; ++j) {
        SysState& st = a.state[a.replace.sys[j]];
        st.phase = SYS_RUNNING;
        st.first = 0;
    }
}

}  // namespace

void enqueue_reliable_pass(const PassArgs& a, const SysDirac* oe_ff, const SysDirac* eo_ff, const SysDirac* oe_64,
                           const SysDirac* eo_64, int grid_dirac, int grid_vec, cudaStream_t s) {
    pass_select_kernel<<<1, 32, 0, s>>>(a);
    pass_fold_kernel<<<grid_vec, kTile, 0, s>>>(a);
    pass_to_ff_kernel<<<grid_vec, kTile, 0, s>>>(a);
    launch_dslash_list(true, EPI_PLAIN, oe_ff, a.ff.sys, a.ff.prefix, a.ff.count, grid_dirac, s);
    launch_dslash_list(true, EPI_AXPY, eo_ff, a.ff.sys, a.ff.prefix, a.ff.count, grid_dirac, s);
    pass_residual_kernel<false><<<grid_vec, kTile, 0, s>>>(a, a.ff);
    pass_decide_kernel<<<1, 256, 0, s>>>(a);
    launch_dslash_list(false, EPI_PLAIN, oe_64, a.confirm.sys, a.confirm.prefix, a.confirm.count, grid_dirac, s);
    launch_dslash_list(false, EPI_AXPY, eo_64, a.confirm.sys, a.confirm.prefix, a.confirm.count, grid_dirac, s);
    pass_residual_kernel<true><<<grid_vec, kTile, 0, s>>>(a, a.confirm);
    pass_confirm_kernel<<<1, 256, 0, s>>>(a);
    pass_set_residual_kernel<<<grid_vec, kTile, 0, s>>>(a);
    pass_resume_kernel<<<1, 32, 0, s>>>(a);
}

}  // namespace stag
