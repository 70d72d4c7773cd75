// capi.cu - the C ABI (include/stag.h): handle, argument checks, host/device
// staging, and the CG driver of Sec. 2, Fig. 1.
//
// The driver keeps alpha, beta and delta on the device (the paper's CUBLAS
// dot returned a scalar to the host every step).  It enqueues blocks of
// check_interval iterations - captured once as a CUDA graph - and reads the
// CG state back only between blocks.  After Fig. 1 stops, the true residual
// b - A x is recomputed with native FP64 arithmetic and Fig. 1 restarts from
// the current x while it exceeds tol.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/stag.h"
#include "handle.h"
#include "stag_kernels.h"

using namespace stag;

namespace stag {
NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }
}  // namespace stag

namespace {

thread_local std::string g_create_error = "no error";

struct Fail {
    int code;
};

}  // namespace

namespace {

void fail(stag_handle* h, int code, const std::string& msg) {
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    throw Fail{code};
}

void cuda_check(stag_handle* h, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    const int code = (e == cudaErrorMemoryAllocation) ? STAG_ERR_OOM : STAG_ERR_CUDA;
    fail(h, code, std::string(what) + ": " + cudaGetErrorString(e));
}

void launch_check(stag_handle* h, const char* what) { cuda_check(h, cudaGetLastError(), what); }

// A zeroed device buffer owned by the handle (freed by destroy_handle).  With
// opt.guard_bands it lies between two guard bands of kGuardBytes filled with
// kGuardByte, which stag_check_guards reads back: a kernel that writes past
// either end of the buffer changes them.
template <class T>
T* dev_alloc(stag_handle* h, size_t bytes, const char* what) {
    const size_t guard = h->opt.guard_bands ? kGuardBytes : 0;
    void* base = nullptr;
    cuda_check(h, cudaMalloc(&base, bytes + 2 * guard), what);
    char* p = static_cast<char*>(base) + guard;
    try {
        h->allocs.push_back(stag_handle::Alloc{p, base, bytes});
    } catch (...) {
        cudaFree(base);
        throw;
    }
    h->device_bytes += (long long)bytes;
    cudaError_t e = cudaMemsetAsync(p, 0, bytes, h->s);
    if (e == cudaSuccess && guard) e = cudaMemsetAsync(base, kGuardByte, guard, h->s);
    if (e == cudaSuccess && guard) e = cudaMemsetAsync(p + bytes, kGuardByte, guard, h->s);
    cuda_check(h, e, what);
    return reinterpret_cast<T*>(p);
}

// Bytes of the guard bands of [base, base + n) that differ from kGuardByte.
__global__ void count_guard_kernel(const unsigned char* __restrict__ base, size_t n, unsigned long long* bad) {
    unsigned int local = 0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        local += base[k] != kGuardByte;
    if (local) atomicAdd(bad, (unsigned long long)local);
}

size_t vec_bytes(const Geom& g) { return (size_t)3 * g.vs * sizeof(double2); }
size_t abi_vec_bytes(const Geom& g) { return (size_t)3 * g.vh * sizeof(double2); }
size_t link_bytes(const Geom& g) { return (size_t)2 * 4 * 9 * g.vs * sizeof(double2); }

// Is p device-accessible memory of the handle's device?
bool is_device_ptr(stag_handle* h, const void* p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        if (a.type == cudaMemoryTypeDevice && a.device != h->device)
            fail(h, STAG_ERR_INVALID_ARG, "device pointer belongs to another device");
        return true;
    }
    return false;
}

// Device view of an ABI input vector (staged into `stage` when on the host).
const double* input_vec(stag_handle* h, const double* p, double* stage) {
    if (is_device_ptr(h, p)) return p;
    cuda_check(h, cudaMemcpyAsync(stage, p, abi_vec_bytes(h->g), cudaMemcpyHostToDevice, h->s),
               "copy vector to device");
    return stage;
}

void begin_call(stag_handle* h) {
    cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice");
    cuda_check(h, cudaEventRecord(h->ev_in, h->user_stream), "cudaEventRecord");
    cuda_check(h, cudaStreamWaitEvent(h->s, h->ev_in, 0), "cudaStreamWaitEvent");
}

void end_call(stag_handle* h) { cuda_check(h, cudaStreamSynchronize(h->s), "cudaStreamSynchronize"); }

// long_recon = 12 accepts Naik links whose L / long_scale deviates from SU(3)
// by at most this (entries of L^dag L / c^2 - 1, and det L / c^3 - 1): the third
// row rebuilt from the first two then agrees with the stored one to about this
// relative size, far below the solver's tolerances.
constexpr float kLongReconMaxDeviation = 1e-12f;
// Range of |long_scale| accepted with long_recon = 12 (see stag_create_ex).
constexpr double kLongScaleMin = 1e-10;
constexpr double kLongScaleMax = 1e18;

bool use_ff(const stag_handle* h) { return h->opt.arith == STAG_ARITH_FF; }

LinkSet links(const stag_handle* h) {
    return LinkSet{h->fat64, h->lng64, h->fatff, h->lngff, h->lng_s};
}

// out = m2 * in - D_eo D_oe in on internal F64 vectors, native FP64; uses h->t.
void apply_A_f64(stag_handle* h, const double2* in, double2* out) {
    const LinkSet L = links(h);
    launch_dslash_f64(h->g, 1, L, in, reinterpret_cast<double2*>(h->t), EPI_PLAIN, nullptr, 0.0,
                      nullptr, nullptr, h->s);
    launch_dslash_f64(h->g, 0, L, reinterpret_cast<const double2*>(h->t), out, EPI_AXPY, in,
                      h->mass * h->mass, nullptr, nullptr, h->s);
    h->launches += 2;
    launch_check(h, "apply_A (F64)");
}

double read_red_out(stag_handle* h) {
    cuda_check(h, cudaMemcpyAsync(h->scal_host, h->scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, h->s),
               "read CG state");
    end_call(h);
    return h->scal_host->red_out;
}

void read_state(stag_handle* h) {
    cuda_check(h, cudaMemcpyAsync(h->scal_host, h->scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, h->s),
               "read CG state");
    end_call(h);
}

// Low-precision Dirac kernels and links by storage type.
void dslash_lo(const Geom& g, int P, const float2* fat, const float2* lng, const float2* in, float2* out, Epilogue e,
               const float2* src, double m2, CgScalars* sc, double* pa, cudaStream_t s, bool r12 = false,
               float lng_inv_scale = 0.f) {
    if (r12)
        launch_dslash_f32r12(g, P, fat, in, out, e, src, m2, sc, pa, s);  // fat: two rows per link
    else
        launch_dslash_f32(g, P, fat, lng, in, out, e, src, m2, sc, pa, s, lng_inv_scale);
}
void dslash_lo(const Geom& g, int P, const __half2* fat, const __half2* lng, const float2* in, float2* out, Epilogue e,
               const float2* src, double m2, CgScalars* sc, double* pa, cudaStream_t s, bool = false, float = 0.f) {
    launch_dslash_f32l16(g, P, fat, lng, in, out, e, src, m2, sc, pa, s);
}
void dslash_lo(const Geom& g, int P, const __half2* fat, const __half2* lng, const __half2* in, __half2* out,
               Epilogue e, const __half2* src, double m2, CgScalars* sc, double* pa, cudaStream_t s, bool = false,
               float = 0.f) {
    launch_dslash_h16(g, P, fat, lng, in, out, e, src, m2, sc, pa, s);
}
void dslash_lo(const Geom& g, int P, const __nv_bfloat162* fat, const __nv_bfloat162* lng, const __nv_bfloat162* in,
               __nv_bfloat162* out, Epilogue e, const __nv_bfloat162* src, double m2, CgScalars* sc, double* pa,
               cudaStream_t s, bool = false, float = 0.f) {
    launch_dslash_b16(g, P, fat, lng, in, out, e, src, m2, sc, pa, s);
}
// 1 / scale of the FP32 Naik links when they are stored as two rows (long_recon
// = 12 with the FP32 inner iteration), else 0 (nine entries).
float lo_long_inv_scale(const stag_handle* h) {
    return (h->naik && h->opt.long_recon == 12 && h->opt.inner == STAG_INNER_F32) ? h->lng_s.x : 0.f;
}
const float2* lo_fat(const stag_handle* h, const float2*) { return h->fat32; }
const float2* lo_lng(const stag_handle* h, const float2*) { return h->lng32; }
const __half2* lo_fat(const stag_handle* h, const __half2*) { return h->fat16; }
const __half2* lo_lng(const stag_handle* h, const __half2*) { return h->lng16; }
const __nv_bfloat162* lo_fat(const stag_handle* h, const __nv_bfloat162*) { return h->fatb16; }
const __nv_bfloat162* lo_lng(const stag_handle* h, const __nv_bfloat162*) { return h->lngb16; }

// One inner iteration of the mixed-precision CG on vectors stored as V and
// links stored as L.
template <class V, class L = V, class Mark>
void enqueue_lo_iteration(stag_handle* h, Mark mark) {
    const Geom& g = h->g;
    V* d = static_cast<V*>(h->lo_d);
    V* t = static_cast<V*>(h->lo_t);
    V* ad = static_cast<V*>(h->lo_ad);
    V* r = static_cast<V*>(h->lo_r);
    const L* fat = lo_fat(h, static_cast<const L*>(nullptr));
    const L* lng = lo_lng(h, static_cast<const L*>(nullptr));
    const bool r12 = h->opt.link_recon == 12;
    const float ls = lo_long_inv_scale(h);
    mark(0);
    dslash_lo(g, 1, fat, lng, d, t, EPI_PLAIN, nullptr, 0.0, h->scal, h->partials, h->s, r12, ls);
    mark(1);
    dslash_lo(g, 0, fat, lng, t, ad, EPI_CG, d, 0.0, h->scal, h->partials, h->s, r12, ls);
    mark(2);
    launch_lo_update_xr<V>(g, h->lo_y, r, d, ad, h->scal, h->partials, h->s);
    mark(3);
    launch_lo_update_d<V>(g, r, d, h->scal, h->s);
    mark(4);
}

// h->ad = A h->x with links and vectors stored as V (FP32 arithmetic); the
// input is divided by scale before the conversion and the result multiplied by it.
template <class V>
void apply_A_lo(stag_handle* h, double m2, double scale) {
    const Geom& g = h->g;
    V* in = static_cast<V*>(h->lo_d);
    V* t = static_cast<V*>(h->lo_t);
    V* o = static_cast<V*>(h->lo_ad);
    const V* fat = lo_fat(h, in);
    const V* lng = lo_lng(h, in);
    const bool r12 = h->opt.link_recon == 12;
    const float ls = lo_long_inv_scale(h);
    launch_to_lo<V>(g, h->x, in, 1.0 / scale, h->s);
    dslash_lo(g, 1, fat, lng, in, t, EPI_PLAIN, nullptr, 0.0, nullptr, nullptr, h->s, r12, ls);
    dslash_lo(g, 0, fat, lng, t, o, EPI_AXPY, in, m2, nullptr, nullptr, h->s, r12, ls);
    launch_from_lo<V>(g, o, h->ad, scale, h->s);
}

// One CG iteration (Fig. 1 loop body): four kernels.
void enqueue_iteration(stag_handle* h, cudaEvent_t* ev, bool count) {
    const Geom& g = h->g;
    const LinkSet L = links(h);
    auto mark = [&](int k) {
        if (ev) cudaEventRecord(ev[k], h->s);
    };
    if (h->opt.inner == STAG_INNER_F32) {
        enqueue_lo_iteration<float2>(h, mark);
    } else if (h->opt.inner == STAG_INNER_F16) {
        enqueue_lo_iteration<__half2>(h, mark);
    } else if (h->opt.inner == STAG_INNER_BF16) {
        enqueue_lo_iteration<__nv_bfloat162>(h, mark);
    } else if (h->opt.inner == STAG_INNER_F32_L16) {
        enqueue_lo_iteration<float2, __half2>(h, mark);
    } else if (use_ff(h)) {
        float4* d = static_cast<float4*>(h->d);
        float4* t = static_cast<float4*>(h->t);
        float4* r = reinterpret_cast<float4*>(h->r);
        float4* ad = reinterpret_cast<float4*>(h->ad);
        mark(0);
        launch_dslash_ff(g, 1, L, d, t, EPI_PLAIN, nullptr, 0.0, h->scal, h->partials, h->s);
        mark(1);
        launch_dslash_ff(g, 0, L, t, ad, EPI_CG, d, 0.0, h->scal, h->partials, h->s);
        mark(2);
        launch_cg_update_xr_ff(g, h->xff, r, d, ad, h->scal, h->partials, h->s);
        mark(3);
        launch_cg_update_d_ff(g, r, d, h->scal, h->s);
        mark(4);
    } else {
        double2* d = static_cast<double2*>(h->d);
        double2* t = static_cast<double2*>(h->t);
        mark(0);
        launch_dslash_f64(g, 1, L, d, t, EPI_PLAIN, nullptr, 0.0, h->scal, h->partials, h->s);
        mark(1);
        launch_dslash_f64(g, 0, L, t, h->ad, EPI_CG, d, 0.0, h->scal, h->partials, h->s);
        mark(2);
        launch_cg_update_xr(g, h->x, h->r, d, h->ad, h->scal, h->partials, h->s);
        mark(3);
        launch_cg_update_d(g, h->r, d, h->scal, h->s);
        mark(4);
    }
    if (count) h->launches += 4;
}

// check_interval iterations, then (float-float) the fold of x_ff into x.
void enqueue_block(stag_handle* h, bool timing, bool count) {
    const int K = h->opt.check_interval;
    for (int k = 0; k < K; ++k) enqueue_iteration(h, timing ? &h->events[5 * k] : nullptr, count);
    if (use_ff(h) && h->opt.inner == STAG_INNER_NONE) {
        launch_fold_x(h->g, h->x, h->xff, h->s);
        if (count) h->launches += 1;
    }
}

void ensure_graph(stag_handle* h) {
    if (h->graph) return;
    cudaGraph_t graph = nullptr;
    cuda_check(h, cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal), "begin capture");
    enqueue_block(h, false, false);
    cudaError_t e = cudaStreamEndCapture(h->s, &graph);
    cuda_check(h, e, "end capture");
    e = cudaGraphInstantiate(&h->graph, graph, 0);
    cudaGraphDestroy(graph);
    cuda_check(h, e, "graph instantiate");
}

// Runs Fig. 1 from the state prepared by cg_init until scal->done.
void run_fig1(stag_handle* h) {
    const int K = h->opt.check_interval;
    const bool timing = h->opt.timing != 0;
    const bool graphs = h->opt.use_graphs != 0 && !timing;
    if (timing && h->events.size() < (size_t)(5 * K)) {
        for (cudaEvent_t e : h->events) cudaEventDestroy(e);
        h->events.assign(5 * K, nullptr);
        for (auto& e : h->events) cuda_check(h, cudaEventCreate(&e), "cudaEventCreate");
    }
    if (graphs) ensure_graph(h);
    read_state(h);
    while (!h->scal_host->done) {
        const long long iter_before = h->scal_host->iter;
        if (graphs) {
            cuda_check(h, cudaGraphLaunch(h->graph, h->s), "cudaGraphLaunch");
            h->launches += 4LL * K + ((use_ff(h) && h->opt.inner == STAG_INNER_NONE) ? 1 : 0);
        } else {
            enqueue_block(h, timing, true);
            launch_check(h, "CG iteration");
        }
        read_state(h);
        if (h->block_hook) h->block_hook();
        if (timing) {
            const long long active = h->scal_host->iter - iter_before;
            for (long long k = 0; k < active && k < K; ++k) {
                const bool last_done = (k == active - 1) && h->scal_host->done;
                for (int j = 0; j < 4; ++j) {
                    if (j == 3 && last_done) continue;  // d update skipped after the last step
                    float ms = 0.f;
                    cuda_check(h, cudaEventElapsedTime(&ms, h->events[5 * k + j], h->events[5 * k + j + 1]),
                               "cudaEventElapsedTime");
                    h->stats[j].ms += ms;
                    h->stats[j].launches += 1;
                }
            }
        }
    }
}

void destroy_handle(stag_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->s) cudaStreamSynchronize(h->s);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    for (const stag_handle::Alloc& a : h->allocs) cudaFree(a.base);
    h->allocs.clear();
    if (h->scal_host) cudaFreeHost(h->scal_host);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->s) cudaStreamDestroy(h->s);
    delete h;
}

// check_scale != 0: also the scaled-SU(3) check of the links (largest deviation
// into *maxdev) and the float-float two-row copy soaff instead of nine entries.
void pack_field(stag_handle* h, const double* links_in, double2* soa64, float4* soaff, float2* soa32,
                __half2* soa16, __nv_bfloat162* soab16, float2* soa32r = nullptr, double check_scale = 0.0,
                unsigned int* maxdev = nullptr) {
    const size_t aos_bytes = (size_t)2 * h->g.vh * 4 * 9 * sizeof(double2);
    const double* src = links_in;
    void* stage = nullptr;
    cudaPointerAttributes pa{};
    bool pinned = false;
    if (cudaPointerGetAttributes(&pa, links_in) == cudaSuccess)
        pinned = pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr;
    else
        cudaGetLastError();  // an unregistered host pointer
    if (pinned) {
        // pinned host memory: the pack kernel reads it in place over the host link
        src = static_cast<const double*>(pa.devicePointer);
    } else if (!is_device_ptr(h, links_in)) {
        cuda_check(h, cudaMalloc(&stage, aos_bytes), "allocate link staging buffer");
        cudaError_t e = cudaMemcpyAsync(stage, links_in, aos_bytes, cudaMemcpyHostToDevice, h->s);
        if (e != cudaSuccess) {
            cudaFree(stage);
            cuda_check(h, e, "copy links to device");
        }
        src = static_cast<const double*>(stage);
    }
    if (check_scale != 0.0) {
        launch_check_scaled_su3(h->g, src, check_scale, maxdev, h->s);
        launch_pack_links_ff_rows2(h->g, src, soaff, h->s);
        h->launches += 2;
        soaff = nullptr;
    }
    launch_pack_links(h->g, src, soa64, soaff, soa32, soa16, soab16, h->s);
    h->launches += 1;
    if (soa32r) {
        launch_pack_links_rows2(h->g, src, soa32r, h->s);
        h->launches += 1;
    }
    cudaError_t e = cudaGetLastError();
    if (stage) {
        cudaError_t e2 = cudaStreamSynchronize(h->s);
        cudaFree(stage);
        if (e == cudaSuccess) e = e2;
    }
    cuda_check(h, e, "pack links");
}

}  // namespace

namespace {

// A x in the handle's FP64-class arithmetic into h->ad (float-float or FP64);
// returns true when h->ad holds float-float.  Uses h->u and h->t.
bool apply_A_fp64class(stag_handle* h, const double2* x) {
    if (!use_ff(h)) {
        apply_A_f64(h, x, h->ad);
        return false;
    }
    const Geom& g = h->g;
    float4* u = static_cast<float4*>(h->u);
    float4* t = static_cast<float4*>(h->t);
    float4* ad = reinterpret_cast<float4*>(h->ad);
    launch_to_ff(g, x, u, h->s);
    launch_dslash_ff(g, 1, links(h), u, t, EPI_PLAIN, nullptr, 0.0, nullptr, nullptr, h->s);
    launch_dslash_ff(g, 0, links(h), t, ad, EPI_AXPY, u, h->mass * h->mass, nullptr, nullptr, h->s);
    h->launches += 3;
    launch_check(h, "apply_A (float-float)");
    return true;
}

void solve_plain(stag_handle* h, double bnorm2, double tol, long long max_it, stag_solve_info& inf, int& status,
                 double& rel);

void drop_graph(stag_handle* h) {
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
}

// Mixed-precision CG with reliable updates (header: STAG_INNER_*).  Each pass
// of the loop folds the inner solution increment into x, recomputes the true
// residual b - A x in FP64-class arithmetic, stops if it meets tol (confirmed
// with native FP64), and otherwise replaces the inner residual by it - scaled
// to unit rms entries for FP16 storage - keeps the search direction (with beta
// from the replaced residual), and runs the inner iteration until the next
// replacement is due.  BF16 shares FP32's exponent range and needs no scaling.
// Safeguard: the iterate with the smallest true residual is kept; when a true
// residual exceeds 10 times that smallest one, or 5 replacements in a row bring
// no improvement (the low-precision operator is too far from A for this system:
// its rounding moves the low modes more than m^2), the best iterate is restored
// and the solve finishes with plain CG in the FP64-class arithmetic (counted in
// info.fallbacks).
void solve_mixed(stag_handle* h, double bnorm2, double tol, long long max_it, stag_solve_info& inf,
                 int& status, double& rel) {
    const Geom& g = h->g;
    const bool f16 = h->opt.inner == STAG_INNER_F16;
    const double m2 = h->mass * h->mass;
    const double thr_true = tol * tol * bnorm2;
    double sigma_old = 1.0;
    bool first = true;
    long long iters = 0;
    int updates = 0;
    double best = INFINITY;
    int since_best = 0;
    bool fallback = false;
    const size_t vb = (size_t)3 * g.vs * sizeof(double2);
    while (true) {
        if (!first) {
            launch_lo_fold_y(g, h->x, h->lo_y, sigma_old, h->s);
            h->launches += 1;
        }
        const bool ax_ff = apply_A_fp64class(h, h->x);
        launch_residual(g, h->b, h->ad, ax_ff, h->r, h->scal, h->partials, h->s);
        h->launches += 1;
        launch_check(h, "true residual");
        const double dtrue = read_red_out(h);
        rel = std::sqrt(dtrue / bnorm2);
        if (std::isfinite(dtrue) && rel < best) {
            best = rel;
            since_best = 0;
            cuda_check(h, cudaMemcpyAsync(h->x_best, h->x, vb, cudaMemcpyDeviceToDevice, h->s), "keep best iterate");
        } else if (!first && (!std::isfinite(dtrue) || rel > 10.0 * best || ++since_best >= 5)) {
            cuda_check(h, cudaMemcpyAsync(h->x, h->x_best, vb, cudaMemcpyDeviceToDevice, h->s), "restore best iterate");
            fallback = true;
            break;
        }
        if (!std::isfinite(dtrue)) {
            status = STAG_ERR_BREAKDOWN;
            h->err = "mixed-precision CG: non-finite residual";
            break;
        }
        if (rel <= tol) {
            if (!use_ff(h)) break;
            apply_A_f64(h, h->x, h->ad);  // confirm with native FP64 arithmetic
            launch_norm2_diff(g, h->b, h->ad, h->scal, h->partials, h->s);
            h->launches += 1;
            launch_check(h, "true residual (FP64)");
            rel = std::sqrt(read_red_out(h) / bnorm2);
            if (rel <= tol) break;
        }
        if (iters >= max_it) {
            status = STAG_ERR_NOT_CONVERGED;
            h->err = "not converged: true residual " + std::to_string(rel) + " after " + std::to_string(iters) +
                     " iterations";
            break;
        }
        const double sigma = f16 ? std::sqrt(dtrue / (6.0 * g.vh)) : 1.0;
        double beta = 0.0;
        if (!first) {
            const double delta_old_true = h->scal_host->delta_old * sigma_old * sigma_old;
            beta = (dtrue / delta_old_true) * (sigma_old / sigma);
            ++updates;
        }
        if (f16)
            launch_lo_set_residual<__half2>(g, h->r, static_cast<__half2*>(h->lo_r), static_cast<__half2*>(h->lo_d),
                                            h->lo_y, 1.0 / sigma, beta, first, h->s);
        else if (h->opt.inner == STAG_INNER_BF16)
            launch_lo_set_residual<__nv_bfloat162>(g, h->r, static_cast<__nv_bfloat162*>(h->lo_r),
                                                   static_cast<__nv_bfloat162*>(h->lo_d), h->lo_y, 1.0 / sigma, beta,
                                                   first, h->s);
        else
            launch_lo_set_residual<float2>(g, h->r, static_cast<float2*>(h->lo_r), static_cast<float2*>(h->lo_d),
                                           h->lo_y, 1.0 / sigma, beta, first, h->s);
        launch_lo_reset(h->scal, dtrue / (sigma * sigma), thr_true / (sigma * sigma), m2, max_it - iters,
                        h->opt.reliable_interval, h->opt.reliable_delta, h->s);
        h->launches += 2;
        launch_check(h, "residual replacement");
        first = false;
        sigma_old = sigma;
        run_fig1(h);
        iters += h->scal_host->iter;
        if (h->scal_host->status != 0) {
            launch_lo_fold_y(g, h->x, h->lo_y, sigma_old, h->s);
            h->launches += 1;
            apply_A_f64(h, h->x, h->ad);
            launch_norm2_diff(g, h->b, h->ad, h->scal, h->partials, h->s);
            h->launches += 1;
            rel = std::sqrt(read_red_out(h) / bnorm2);
            status = STAG_ERR_BREAKDOWN;
            h->err = "CG breakdown: d^dag A d <= 0 or non-finite";
            break;
        }
    }
    if (fallback) {
        const int inner = h->opt.inner;
        drop_graph(h);
        h->opt.inner = STAG_INNER_NONE;
        try {
            solve_plain(h, bnorm2, tol, max_it - iters, inf, status, rel);
        } catch (...) {
            h->opt.inner = inner;
            drop_graph(h);
            throw;
        }
        h->opt.inner = inner;
        drop_graph(h);
        inf.fallbacks += 1;
        inf.iters += (int32_t)iters;
        inf.reliable_updates = updates;
        return;
    }
    inf.iters = (int32_t)iters;
    inf.reliable_updates = updates;
    inf.iter_rel_residual = rel;
}

// Plain CG (Fig. 1) with the true-residual check and restarts, on vectors
// already packed into h->b and h->x.
void solve_plain(stag_handle* h, double bnorm2, double tol, long long max_it, stag_solve_info& inf, int& status,
                 double& rel) {
    const Geom& g = h->g;
    const double threshold = tol * tol * bnorm2;
    const double m2 = h->mass * h->mass;
    const bool ff = use_ff(h);
    apply_A_f64(h, h->x, h->ad);  // A x for r = b - A x
    long long iters = 0;
    int restarts = 0;
    while (true) {
        launch_cg_reset(h->scal, threshold, m2, max_it - iters, h->s);
        if (ff)
            launch_cg_init_ff(g, h->b, h->ad, reinterpret_cast<float4*>(h->r), static_cast<float4*>(h->d), h->xff,
                              h->scal, h->partials, h->s);
        else
            launch_cg_init(g, h->b, h->ad, h->r, static_cast<double2*>(h->d), h->scal, h->partials, h->s);
        h->launches += 2;
        launch_check(h, "CG init");
        run_fig1(h);
        iters += h->scal_host->iter;
        inf.iter_rel_residual = std::sqrt(h->scal_host->delta_new / bnorm2);
        const bool breakdown = h->scal_host->status != 0;
        // true residual with native FP64 arithmetic
        apply_A_f64(h, h->x, h->ad);
        launch_norm2_diff(g, h->b, h->ad, h->scal, h->partials, h->s);
        h->launches += 1;
        launch_check(h, "true residual");
        rel = std::sqrt(read_red_out(h) / bnorm2);
        if (breakdown) {
            status = STAG_ERR_BREAKDOWN;
            h->err = "CG breakdown: d^dag A d <= 0 or non-finite";
            break;
        }
        if (rel <= tol) break;
        if (iters >= max_it || restarts >= h->opt.max_restarts) {
            status = STAG_ERR_NOT_CONVERGED;
            h->err = "not converged: true residual " + std::to_string(rel) + " after " + std::to_string(iters) +
                     " iterations";
            break;
        }
        ++restarts;
    }
    inf.iters = (int32_t)iters;
    inf.restarts = restarts;
}

}  // namespace

namespace stag {
// Error message of a handle-free call, read with stag_last_error(NULL).
void set_noalloc_error(const std::string& msg) { g_create_error = msg; }

void handle_apply_A_f64(stag_handle* h, const double2* in, double2* out) {
    try {
        apply_A_f64(h, in, out);
    } catch (const Fail& f) {
        throw HandleError{f.code};
    }
}

int handle_solve_packed(stag_handle* h, double bnorm2, double tol, long long max_it, stag_solve_info& info) {
    int status = STAG_OK;
    if (max_it <= 0) max_it = 3LL * h->g.vh;
    double rel = 0.0;
    try {
        if (h->opt.inner != STAG_INNER_NONE)
            solve_mixed(h, bnorm2, tol, max_it, info, status, rel);
        else
            solve_plain(h, bnorm2, tol, max_it, info, status, rel);
    } catch (const Fail& f) {
        throw HandleError{f.code};
    }
    info.true_rel_residual = rel;
    info.status = status;
    return status;
}

void handle_begin(stag_handle* h) {
    try {
        begin_call(h);
    } catch (const Fail& f) {
        throw HandleError{f.code};
    }
}

void handle_end(stag_handle* h) {
    try {
        end_call(h);
    } catch (const Fail& f) {
        throw HandleError{f.code};
    }
}

bool handle_is_device_ptr(stag_handle* h, const void* p) {
    try {
        return is_device_ptr(h, p);
    } catch (const Fail& f) {
        throw HandleError{f.code};
    }
}
}  // namespace stag

// ====================================================================== ABI
extern "C" {

int stag_default_options(stag_options* opt) {
    if (!opt) return STAG_ERR_INVALID_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->arith = STAG_ARITH_F64;
    opt->check_interval = 32;
    opt->max_restarts = 5;
    opt->use_graphs = 1;
    opt->timing = 0;
    opt->inner = STAG_INNER_NONE;
    opt->reliable_interval = 100;
    opt->reliable_delta = 0.1;
    opt->autotune = 1;
    return STAG_OK;
}

int stag_create_ex(stag_handle** out, const double* fat, const double* naik_long,
                   const int32_t dims[4], double mass, const stag_options* opt) {
    NvtxRange range("stag_create_ex");
    if (out) *out = nullptr;
    stag_handle* h = nullptr;
    try {
        if (!out) fail(nullptr, STAG_ERR_INVALID_ARG, "out is NULL");
        if (!fat) fail(nullptr, STAG_ERR_INVALID_ARG, "links pointer is NULL");
        if (!dims) fail(nullptr, STAG_ERR_INVALID_ARG, "dims is NULL");
        long long V = 1;
        for (int k = 0; k < 4; ++k) {
            if (dims[k] < 2 || dims[k] % 2)
                fail(nullptr, STAG_ERR_INVALID_ARG,
                     "every lattice extent must be even and >= 2 (got " + std::to_string(dims[k]) + ")");
            V *= dims[k];
        }
        if (V / 2 >= (1LL << 31) - 64)
            fail(nullptr, STAG_ERR_INVALID_ARG, "lattice too large (V/2 must be < 2^31)");
        if (!std::isfinite(mass)) fail(nullptr, STAG_ERR_INVALID_ARG, "mass must be finite");
        stag_options o;
        stag_default_options(&o);
        if (opt) o = *opt;
        if (o.arith != STAG_ARITH_F64 && o.arith != STAG_ARITH_FF)
            fail(nullptr, STAG_ERR_INVALID_ARG, "unknown arith option");
        if (o.guard_bands != 0 && o.guard_bands != 1) fail(nullptr, STAG_ERR_INVALID_ARG, "guard_bands must be 0 or 1");
        if (o.check_interval < 1 || o.check_interval > 4096)
            fail(nullptr, STAG_ERR_INVALID_ARG, "check_interval must be in [1, 4096]");
        if (o.max_restarts < 0) fail(nullptr, STAG_ERR_INVALID_ARG, "max_restarts must be >= 0");
        if (o.inner != STAG_INNER_NONE && o.inner != STAG_INNER_F32 && o.inner != STAG_INNER_F16 &&
            o.inner != STAG_INNER_BF16 && o.inner != STAG_INNER_F32_L16)
            fail(nullptr, STAG_ERR_INVALID_ARG, "unknown inner precision");
        if (o.link_recon != 0 && o.link_recon != 12)
            fail(nullptr, STAG_ERR_INVALID_ARG, "link_recon must be 0 or 12");
        if (o.link_recon == 12 && (naik_long != nullptr || o.inner != STAG_INNER_F32))
            fail(nullptr, STAG_ERR_INVALID_ARG, "12-parameter links need the one-hop operator and inner = F32");
        if (o.long_recon != 0 && o.long_recon != 12)
            fail(nullptr, STAG_ERR_INVALID_ARG, "long_recon must be 0 or 12");
        // The rebuilt third row is formed from products of two stored entries, of
        // size long_scale^2, in float-float: above about 1.8e19 that overflows
        // FP32, and below about 1e-12 the low words of the products go
        // subnormal and lose the float-float precision.  The accepted range
        // keeps a margin on both sides.
        if (o.long_recon == 12 &&
            (naik_long == nullptr || o.arith != STAG_ARITH_FF || !std::isfinite(o.long_scale) ||
             !(std::fabs(o.long_scale) >= kLongScaleMin && std::fabs(o.long_scale) <= kLongScaleMax)))
            fail(nullptr, STAG_ERR_INVALID_ARG,
                 "long_recon = 12 needs Naik links, arith = FF and a finite long_scale with 1e-10 <= |long_scale| <= 1e18");
        if (o.inner != STAG_INNER_NONE &&
            (o.reliable_interval < 1 || !(o.reliable_delta > 0.0 && o.reliable_delta < 1.0)))
            fail(nullptr, STAG_ERR_INVALID_ARG, "reliable_interval must be >= 1 and reliable_delta in (0, 1)");

        h = new stag_handle();
        h->opt = o;
        h->mass = mass;
        h->naik = naik_long != nullptr;
        Geom& g = h->g;
        g.lx = dims[0];
        g.ly = dims[1];
        g.lz = dims[2];
        g.lt = dims[3];
        g.lxh = g.lx / 2;
        g.vh = (int)(V / 2);
        g.vs = (int)(((V / 2) + 63) / 64 * 64);
        for (int k = 0; k < 4; ++k) g.hop3[k] = 3 % dims[k];
        if (blocks_for(g.vs, 64) > kMaxPartials) fail(h, STAG_ERR_INVALID_ARG, "lattice too large");

        cuda_check(h, cudaGetDevice(&h->device), "cudaGetDevice");
        cuda_check(h, cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking), "cudaStreamCreate");
        cuda_check(h, cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming), "cudaEventCreate");
        begin_call(h);

        const bool ff = use_ff(h);
        h->fat64 = dev_alloc<double2>(h, link_bytes(g), "allocate links");
        if (ff) h->fatff = dev_alloc<float4>(h, link_bytes(g), "allocate FF links");
        if (h->naik) {
            h->lng64 = dev_alloc<double2>(h, link_bytes(g), "allocate Naik links");
            if (ff) h->lngff = dev_alloc<float4>(h, link_bytes(g), "allocate FF Naik links");
        }
        const size_t vb = vec_bytes(g);
        h->x = dev_alloc<double2>(h, vb, "allocate x");
        h->r = dev_alloc<double2>(h, vb, "allocate r");
        h->ad = dev_alloc<double2>(h, vb, "allocate Ad");
        h->b = dev_alloc<double2>(h, vb, "allocate b");
        h->d = dev_alloc<void>(h, vb, "allocate d");
        h->t = dev_alloc<void>(h, vb, "allocate t");
        h->u = dev_alloc<void>(h, vb, "allocate u");
        if (ff) h->xff = dev_alloc<float4>(h, vb, "allocate x_ff");
        const size_t lo_links = (size_t)2 * 4 * 9 * g.vs;  // complex entries per field
        if (h->opt.inner == STAG_INNER_F32 && h->opt.link_recon == 12) {
            h->fat32 = dev_alloc<float2>(h, lo_links / 9 * 6 * sizeof(float2), "allocate FP32 two-row links");
        } else if (h->opt.inner == STAG_INNER_F32) {
            h->fat32 = dev_alloc<float2>(h, lo_links * sizeof(float2), "allocate FP32 links");
            const size_t lng_entries = h->opt.long_recon == 12 ? lo_links / 9 * 6 : lo_links;  // two rows or nine
            if (h->naik) h->lng32 = dev_alloc<float2>(h, lng_entries * sizeof(float2), "allocate FP32 Naik links");
        } else if (h->opt.inner == STAG_INNER_F16 || h->opt.inner == STAG_INNER_F32_L16) {
            h->fat16 = dev_alloc<__half2>(h, lo_links * sizeof(__half2), "allocate FP16 links");
            if (h->naik) h->lng16 = dev_alloc<__half2>(h, lo_links * sizeof(__half2), "allocate FP16 Naik links");
        } else if (h->opt.inner == STAG_INNER_BF16) {
            h->fatb16 = dev_alloc<__nv_bfloat162>(h, lo_links * sizeof(__nv_bfloat162), "allocate BF16 links");
            if (h->naik)
                h->lngb16 = dev_alloc<__nv_bfloat162>(h, lo_links * sizeof(__nv_bfloat162), "allocate BF16 Naik links");
        }
        if (h->opt.inner != STAG_INNER_NONE) {
            const bool vec32 = h->opt.inner == STAG_INNER_F32 || h->opt.inner == STAG_INNER_F32_L16;
            const size_t lo_vb = (size_t)3 * g.vs * (vec32 ? sizeof(float2) : sizeof(__half2));
            h->lo_d = dev_alloc<void>(h, lo_vb, "allocate inner d");
            h->lo_t = dev_alloc<void>(h, lo_vb, "allocate inner t");
            h->lo_ad = dev_alloc<void>(h, lo_vb, "allocate inner Ad");
            h->lo_r = dev_alloc<void>(h, lo_vb, "allocate inner r");
            h->lo_y = dev_alloc<float2>(h, (size_t)3 * g.vs * sizeof(float2), "allocate inner y");
            h->x_best = dev_alloc<double2>(h, vb, "allocate best iterate");
        }
        h->io_a = dev_alloc<double>(h, abi_vec_bytes(g), "allocate staging");
        h->io_b = dev_alloc<double>(h, abi_vec_bytes(g), "allocate staging");
        // one partial sum per block of any reducing kernel (blocks of 64 threads or more)
        h->partials = dev_alloc<double>(h, sizeof(double) * (size_t)blocks_for(g.vs, 64), "allocate partials");
        h->scal = dev_alloc<CgScalars>(h, sizeof(CgScalars), "allocate CG state");
        cuda_check(h, cudaMallocHost(reinterpret_cast<void**>(&h->scal_host), sizeof(CgScalars)),
                   "allocate pinned CG state");
        std::memset(h->scal_host, 0, sizeof(CgScalars));

        const bool r12 = h->opt.link_recon == 12;
        pack_field(h, fat, h->fat64, h->fatff, r12 ? nullptr : h->fat32, h->fat16, h->fatb16, r12 ? h->fat32 : nullptr);
        if (h->naik && h->opt.long_recon == 12) {
            unsigned int* maxdev = reinterpret_cast<unsigned int*>(h->partials);
            cuda_check(h, cudaMemsetAsync(maxdev, 0, sizeof(unsigned int), h->s), "clear link check");
            // the FP32 Naik links of the inner iteration are two rows as well
            const bool f32_rows = h->opt.inner == STAG_INNER_F32;
            pack_field(h, naik_long, h->lng64, h->lngff, f32_rows ? nullptr : h->lng32, h->lng16, h->lngb16,
                       f32_rows ? h->lng32 : nullptr, h->opt.long_scale, maxdev);
            unsigned int bits = 0;
            cuda_check(h, cudaMemcpyAsync(&bits, maxdev, sizeof(bits), cudaMemcpyDeviceToHost, h->s),
                       "read link check");
            cuda_check(h, cudaStreamSynchronize(h->s), "cudaStreamSynchronize");
            float dev;
            std::memcpy(&dev, &bits, sizeof(dev));
            if (!(dev <= kLongReconMaxDeviation))
                fail(h, STAG_ERR_INVALID_ARG,
                     "long_recon = 12: a Naik link / long_scale is not in SU(3) (deviation " + std::to_string(dev) +
                         ")");
            h->lng_s = host_ff_from_double(1.0 / h->opt.long_scale);
        } else if (h->naik) {
            pack_field(h, naik_long, h->lng64, h->lngff, h->lng32, h->lng16, h->lngb16);
        }
        end_call(h);
        *out = h;
        return STAG_OK;
    } catch (const Fail& f) {
        if (h) {
            g_create_error = h->err;
            destroy_handle(h);
        }
        return f.code;
    } catch (const std::bad_alloc&) {
        g_create_error = "host allocation failed";
        destroy_handle(h);
        return STAG_ERR_OOM;
    } catch (...) {
        g_create_error = "unexpected exception";
        destroy_handle(h);
        return STAG_ERR_CUDA;
    }
}

int stag_create(stag_handle** out, const double* links, const int32_t dims[4], double mass) {
    return stag_create_ex(out, links, nullptr, dims, mass, nullptr);
}

int stag_set_stream(stag_handle* h, void* cuda_stream) {
    if (!h) return STAG_ERR_INVALID_ARG;
    h->user_stream = static_cast<cudaStream_t>(cuda_stream);
    return STAG_OK;
}

int stag_set_mass(stag_handle* h, double mass) {
    if (!h) return STAG_ERR_INVALID_ARG;
    if (!std::isfinite(mass)) {
        h->err = "mass must be finite";
        return STAG_ERR_INVALID_ARG;
    }
    h->mass = mass;
    return STAG_OK;
}

int stag_dslash(stag_handle* h, int32_t out_parity, const double* in, double* out) {
    if (!h) return STAG_ERR_INVALID_ARG;
    NvtxRange range("stag_dslash");
    try {
        if (!in || !out) fail(h, STAG_ERR_INVALID_ARG, "NULL vector");
        if (out_parity != 0 && out_parity != 1) fail(h, STAG_ERR_INVALID_ARG, "out_parity must be 0 or 1");
        if (in == out) fail(h, STAG_ERR_INVALID_ARG, "in and out must not overlap");
        begin_call(h);
        const Geom& g = h->g;
        const bool out_dev = is_device_ptr(h, out);
        const double* src = input_vec(h, in, h->io_a);
        launch_pack_vec(g, src, h->x, h->s);
        if (use_ff(h)) {
            float4* in_ff = reinterpret_cast<float4*>(h->u);
            launch_to_ff(g, h->x, in_ff, h->s);
            launch_dslash_ff(g, out_parity, links(h), in_ff, static_cast<float4*>(h->t), EPI_PLAIN,
                             nullptr, 0.0, nullptr, nullptr, h->s);
            launch_from_ff(g, static_cast<const float4*>(h->t), h->ad, h->s);
            h->launches += 3;
        } else {
            launch_dslash_f64(g, out_parity, links(h), h->x, h->ad, EPI_PLAIN, nullptr, 0.0, nullptr,
                              nullptr, h->s);
            h->launches += 1;
        }
        double* dst = out_dev ? out : h->io_b;
        launch_unpack_vec(g, h->ad, dst, h->s);
        h->launches += 2;
        launch_check(h, "dslash");
        if (!out_dev)
            cuda_check(h, cudaMemcpyAsync(out, h->io_b, abi_vec_bytes(g), cudaMemcpyDeviceToHost, h->s),
                       "copy result to host");
        end_call(h);
        return STAG_OK;
    } catch (const Fail& f) {
        return f.code;
    } catch (...) {
        h->err = "unexpected exception";
        return STAG_ERR_CUDA;
    }
}

int stag_apply_A(stag_handle* h, const double* in_even, double* out_even) {
    if (!h) return STAG_ERR_INVALID_ARG;
    NvtxRange range("stag_apply_A");
    try {
        if (!in_even || !out_even) fail(h, STAG_ERR_INVALID_ARG, "NULL vector");
        if (in_even == out_even) fail(h, STAG_ERR_INVALID_ARG, "in and out must not overlap");
        begin_call(h);
        const Geom& g = h->g;
        const bool out_dev = is_device_ptr(h, out_even);
        const double* src = input_vec(h, in_even, h->io_a);
        launch_pack_vec(g, src, h->x, h->s);
        const double m2 = h->mass * h->mass;
        if (use_ff(h)) {
            float4* in_ff = reinterpret_cast<float4*>(h->u);
            launch_to_ff(g, h->x, in_ff, h->s);
            float4* t = static_cast<float4*>(h->t);
            float4* out_ff = reinterpret_cast<float4*>(h->r);
            launch_dslash_ff(g, 1, links(h), in_ff, t, EPI_PLAIN, nullptr, 0.0, nullptr, nullptr, h->s);
            launch_dslash_ff(g, 0, links(h), t, out_ff, EPI_AXPY, in_ff, m2, nullptr, nullptr, h->s);
            launch_from_ff(g, out_ff, h->ad, h->s);
            h->launches += 4;
        } else {
            apply_A_f64(h, h->x, h->ad);
        }
        double* dst = out_dev ? out_even : h->io_b;
        launch_unpack_vec(g, h->ad, dst, h->s);
        h->launches += 2;
        launch_check(h, "apply_A");
        if (!out_dev)
            cuda_check(h, cudaMemcpyAsync(out_even, h->io_b, abi_vec_bytes(g), cudaMemcpyDeviceToHost, h->s),
                       "copy result to host");
        end_call(h);
        return STAG_OK;
    } catch (const Fail& f) {
        return f.code;
    } catch (...) {
        h->err = "unexpected exception";
        return STAG_ERR_CUDA;
    }
}

int stag_apply_A_prec(stag_handle* h, int32_t arith, const double* in_even, double* out_even) {
    if (!h) return STAG_ERR_INVALID_ARG;
    try {
        if (!in_even || !out_even) fail(h, STAG_ERR_INVALID_ARG, "NULL vector");
        if (in_even == out_even) fail(h, STAG_ERR_INVALID_ARG, "in and out must not overlap");
        const bool ok = arith == STAG_ARITH_F64 || (arith == STAG_ARITH_FF && h->fatff) ||
                        (arith == STAG_ARITH_F32 && h->fat32) || (arith == STAG_ARITH_F16 && h->fat16) ||
                        (arith == STAG_ARITH_BF16 && h->fatb16);
        if (!ok) fail(h, STAG_ERR_INVALID_ARG, "the handle holds no links in the requested arithmetic");
        if (arith == STAG_ARITH_F64 || arith == STAG_ARITH_FF) {
            const int saved = h->opt.arith;
            h->opt.arith = arith;
            const int code = stag_apply_A(h, in_even, out_even);
            h->opt.arith = saved;
            return code;
        }
        begin_call(h);
        const Geom& g = h->g;
        const bool out_dev = is_device_ptr(h, out_even);
        const double* src = input_vec(h, in_even, h->io_a);
        launch_pack_vec(g, src, h->x, h->s);
        double scale = 1.0;
        if (arith == STAG_ARITH_F16) {  // unit rms entries in FP16
            launch_norm2_diff(g, h->x, nullptr, h->scal, h->partials, h->s);
            const double n2 = read_red_out(h);
            scale = n2 > 0.0 ? std::sqrt(n2 / (6.0 * g.vh)) : 1.0;
        }
        const double m2 = h->mass * h->mass;
        if (arith == STAG_ARITH_F32)
            apply_A_lo<float2>(h, m2, 1.0);
        else if (arith == STAG_ARITH_F16)
            apply_A_lo<__half2>(h, m2, scale);
        else
            apply_A_lo<__nv_bfloat162>(h, m2, 1.0);
        double* dst = out_dev ? out_even : h->io_b;
        launch_unpack_vec(g, h->ad, dst, h->s);
        h->launches += 6;
        launch_check(h, "apply_A (low precision)");
        if (!out_dev)
            cuda_check(h, cudaMemcpyAsync(out_even, h->io_b, abi_vec_bytes(g), cudaMemcpyDeviceToHost, h->s),
                       "copy result to host");
        end_call(h);
        return STAG_OK;
    } catch (const Fail& f) {
        return f.code;
    } catch (...) {
        h->err = "unexpected exception";
        return STAG_ERR_CUDA;
    }
}

int stag_cg_solve(stag_handle* h, const double* b_even, double* x_even, double tol, int32_t max_iter,
                  stag_solve_info* info) {
    if (!h) return STAG_ERR_INVALID_ARG;
    NvtxRange range("stag_cg_solve");
    stag_solve_info inf{};
    int status = STAG_OK;
    auto t0 = std::chrono::steady_clock::now();
    try {
        if (!b_even || !x_even) fail(h, STAG_ERR_INVALID_ARG, "NULL vector");
        if (b_even == x_even) fail(h, STAG_ERR_INVALID_ARG, "b and x must not overlap");
        if (!(tol > 0.0) || !std::isfinite(tol)) fail(h, STAG_ERR_INVALID_ARG, "tol must be positive and finite");
        begin_call(h);
        const Geom& g = h->g;
        const bool x_dev = is_device_ptr(h, x_even);
        const double* bsrc = input_vec(h, b_even, h->io_a);
        launch_pack_vec(g, bsrc, h->b, h->s);
        const double* xsrc = input_vec(h, x_even, h->io_b);
        launch_pack_vec(g, xsrc, h->x, h->s);
        launch_norm2_diff(g, h->b, nullptr, h->scal, h->partials, h->s);
        h->launches += 3;
        launch_check(h, "norm of b");
        const double bnorm2 = read_red_out(h);
        if (!std::isfinite(bnorm2)) fail(h, STAG_ERR_INVALID_ARG, "source has non-finite entries");
        const long long n_dim = 3LL * g.vh;
        const long long max_it = max_iter > 0 ? (long long)max_iter : n_dim;
        double rel = 0.0;
        if (bnorm2 == 0.0) {
            cuda_check(h, cudaMemsetAsync(h->x, 0, vec_bytes(g), h->s), "zero x");
        } else {
            if (h->opt.inner != STAG_INNER_NONE)
                solve_mixed(h, bnorm2, tol, max_it, inf, status, rel);
            else
                solve_plain(h, bnorm2, tol, max_it, inf, status, rel);
        }
        inf.true_rel_residual = rel;
        double* dst = x_dev ? x_even : h->io_b;
        launch_unpack_vec(g, h->x, dst, h->s);
        h->launches += 1;
        launch_check(h, "unpack x");
        if (!x_dev)
            cuda_check(h, cudaMemcpyAsync(x_even, h->io_b, abi_vec_bytes(g), cudaMemcpyDeviceToHost, h->s),
                       "copy x to host");
        end_call(h);
    } catch (const Fail& f) {
        status = f.code;
    } catch (...) {
        h->err = "unexpected exception";
        status = STAG_ERR_CUDA;
    }
    inf.status = status;
    inf.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return status;
}

int stag_destroy(stag_handle* h) {
    destroy_handle(h);
    return STAG_OK;
}

const char* stag_last_error(const stag_handle* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

int stag_kernel_stats(const stag_handle* h, int32_t kernel, double* total_ms, int64_t* launches) {
    if (!h || kernel < 0 || kernel >= STAG_KERNEL_COUNT) return STAG_ERR_INVALID_ARG;
    if (total_ms) *total_ms = h->stats[kernel].ms;
    if (launches) *launches = h->stats[kernel].launches;
    return STAG_OK;
}

int stag_reset_stats(stag_handle* h) {
    if (!h) return STAG_ERR_INVALID_ARG;
    for (auto& s : h->stats) s = KernelStat{};
    return STAG_OK;
}

int stag_check_guards(stag_handle* h, int64_t* checked_bytes, int64_t* bad_bytes) {
    if (!h || !checked_bytes || !bad_bytes || !h->opt.guard_bands) return STAG_ERR_INVALID_ARG;
    unsigned long long* bad = nullptr;
    try {
        cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice");
        cuda_check(h, cudaMalloc(&bad, sizeof(*bad)), "allocate guard count");
        cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(*bad), h->s);
        long long checked = 0;
        for (const stag_handle::Alloc& a : h->allocs) {
            if (e != cudaSuccess) break;
            const unsigned char* lo = static_cast<const unsigned char*>(a.base);
            const unsigned char* hi = static_cast<const unsigned char*>(a.user) + a.bytes;
            count_guard_kernel<<<8, 256, 0, h->s>>>(lo, kGuardBytes, bad);
            count_guard_kernel<<<8, 256, 0, h->s>>>(hi, kGuardBytes, bad);
            checked += 2 * (long long)kGuardBytes;
            e = cudaGetLastError();
        }
        unsigned long long host_bad = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&host_bad, bad, sizeof(host_bad), cudaMemcpyDeviceToHost, h->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
        cudaFree(bad);
        bad = nullptr;
        cuda_check(h, e, "check guard bands");
        *checked_bytes = checked;
        *bad_bytes = (int64_t)host_bad;
        return STAG_OK;
    } catch (const Fail& f) {
        if (bad) cudaFree(bad);
        return f.code;
    }
}

int64_t stag_device_bytes(const stag_handle* h) { return h ? h->device_bytes : 0; }

int64_t stag_launch_count(const stag_handle* h) { return h ? h->launches : 0; }

}  // extern "C"
