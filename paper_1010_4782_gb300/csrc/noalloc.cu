// noalloc.cu - stag_apply_A_noalloc: A = m^2 - D_eo D_oe on even sites for
// callers that must not have the library allocate device memory.
//
// Everything else in the library works through a handle whose create call
// allocates the packed links and the work vectors.  Some callers cannot allow
// that: applications that give all device memory out of their own pool, or
// that must not pay the device-wide synchronisation cudaMalloc/cudaFree can
// cause in the middle of their own work.  This entry point needs no handle:
// it reads the caller's links in the ABI layout (eta applied on the fly), and
// keeps its one work array - the odd-site vector D_oe in - in a fixed
// file-scope device array instead of allocated memory.
//
// The work array holds at most kNoallocMaxHalfSites sites (3 MiB); every GPU
// that loads the library keeps it until the process exits.  All calls share
// it, so calls that overlap on the GPU race; each call overwrites the part it
// uses before reading it.  Its device address is looked up on the first call
// made in each CUDA context (with that context's device current) and cached
// for that context only: after a device reset the next call looks it up again.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/stag.h"
#include "stag_internal.cuh"

namespace stag {

constexpr int kNoallocMaxHalfSites = STAG_NOALLOC_MAX_HALF_SITES;
constexpr int kNoallocMaxDevices = 64;

// D_oe in for the current call: [site][colour] complex128, odd sites.
static __device__ __align__(256) double2 g_noalloc_scratch[3 * kNoallocMaxHalfSites];

namespace {

std::mutex g_mu;
// Per device: the context the cached address belongs to (cuCtxGetId, unique
// for the process lifetime) and the array's device address in it.
unsigned long long g_scratch_ctx[kNoallocMaxDevices] = {};
double2* g_scratch_addr[kNoallocMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Identifier of the current CUDA context, or 0 when it cannot be had (the
// caller then looks the address up on every call).  The driver functions are
// fetched through the runtime, so the library needs no link to libcuda.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Do the byte ranges [a, a + na) and [b, b + nb) overlap?
bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    return pa < pb + nb && pb < pa + na;
}

// out(y) = D_{P,1-P} in (y), or m2 * src(y) - D in (y) when EPI; links and
// vectors in the ABI layouts, eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) applied
// to each link as it is read.  Native FP64 arithmetic.
template <bool NAIK, bool EPI>
__global__ void __launch_bounds__(kBlock) apply_aos_kernel(Geom g, int P, const double2* __restrict__ fat,
                                                           const double2* __restrict__ lng,
                                                           const double2* __restrict__ in,
                                                           double2* __restrict__ out,
                                                           const double2* __restrict__ src, double m2) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    int x, y, z, t;
    site_coords(i, P, g, x, y, z, t);
    const int c[4] = {x, y, z, t};
    const int L[4] = {g.lx, g.ly, g.lz, g.lt};
    double2 acc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) acc[r] = make_double2(0.0, 0.0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int phase = 0;
        for (int nu = 0; nu < mu; ++nu) phase += c[nu];
        const double eta = (phase & 1) ? -1.0 : 1.0;  // eta_mu is the same at x and x -/+ k mu
#pragma unroll
        for (int hop = 0; hop < (NAIK ? 2 : 1); ++hop) {
            const double2* links = hop ? lng : fat;
            const int k = hop ? g.hop3[mu] : 1;
            int cf[4] = {x, y, z, t}, cb[4] = {x, y, z, t};
            cf[mu] = wrap_up(c[mu], k, L[mu]);
            cb[mu] = wrap_dn(c[mu], k, L[mu]);
            const int lex_here = ((t * g.lz + z) * g.ly + y) * g.lx + x;
            const int lex_f = ((cf[3] * g.lz + cf[2]) * g.ly + cf[1]) * g.lx + cf[0];
            const int lex_b = ((cb[3] * g.lz + cb[2]) * g.ly + cb[1]) * g.lx + cb[0];
            const double2* uf = links + ((size_t)lex_here * 4 + mu) * 9;
            const double2* ub = links + ((size_t)lex_b * 4 + mu) * 9;
            const double2* vf = in + (size_t)(lex_f >> 1) * 3;
            const double2* vb = in + (size_t)(lex_b >> 1) * 3;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int col = 0; col < 3; ++col) {
                    double2 u = uf[3 * r + col];
                    u.x *= eta;
                    u.y *= eta;
                    cmac(acc[r], u, vf[col]);
                    double2 w = ub[3 * col + r];
                    w.x *= eta;
                    w.y *= eta;
                    cmsc_conj(acc[r], w, vb[col]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        if (EPI) {
            const double2 s = src[(size_t)i * 3 + r];
            out[(size_t)i * 3 + r] = make_double2(fma(m2, s.x, -acc[r].x), fma(m2, s.y, -acc[r].y));
        } else {
            out[(size_t)i * 3 + r] = acc[r];
        }
    }
}

template <bool EPI>
void launch_aos(const Geom& g, int P, const double2* fat, const double2* lng, const double2* in,
                double2* out, const double2* src, double m2, cudaStream_t s) {
    if (lng)
        apply_aos_kernel<true, EPI><<<blocks_for(g.vh), kBlock, 0, s>>>(g, P, fat, lng, in, out, src, m2);
    else
        apply_aos_kernel<false, EPI><<<blocks_for(g.vh), kBlock, 0, s>>>(g, P, fat, lng, in, out, src, m2);
}

bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// Sets the thread's create-error message (read with stag_last_error(NULL)).
void set_noalloc_error(const std::string& msg);

}  // namespace stag

using namespace stag;

extern "C" int stag_apply_A_noalloc(const double* links, const double* naik_long, const int32_t dims[4],
                                    double mass, const double* in_even, double* out_even, void* cuda_stream) {
    auto fail = [](int code, const std::string& msg) {
        set_noalloc_error(msg);
        return code;
    };
    if (!links || !in_even || !out_even || !dims) return fail(STAG_ERR_INVALID_ARG, "NULL argument");
    long long V = 1;
    for (int k = 0; k < 4; ++k) {
        if (dims[k] < 2 || dims[k] % 2)
            return fail(STAG_ERR_INVALID_ARG, "every lattice extent must be even and >= 2");
        V *= dims[k];
    }
    if (V / 2 > kNoallocMaxHalfSites)
        return fail(STAG_ERR_INVALID_ARG, "lattice too large for stag_apply_A_noalloc: V/2 = " +
                                              std::to_string(V / 2) + " sites exceeds its fixed work array of " +
                                              std::to_string(kNoallocMaxHalfSites) + " sites");
    if (!std::isfinite(mass)) return fail(STAG_ERR_INVALID_ARG, "mass must be finite");
    const size_t vec_bytes = (size_t)(V / 2) * 3 * sizeof(double2);
    const size_t link_bytes = (size_t)V * 4 * 9 * sizeof(double2);
    if (ranges_overlap(in_even, vec_bytes, out_even, vec_bytes))
        return fail(STAG_ERR_INVALID_ARG, "in and out must not overlap");
    if (ranges_overlap(links, link_bytes, out_even, vec_bytes) ||
        (naik_long && ranges_overlap(naik_long, link_bytes, out_even, vec_bytes)))
        return fail(STAG_ERR_INVALID_ARG, "out must not overlap the links");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices)
        return fail(STAG_ERR_CUDA, "no usable current CUDA device");
    if (!on_device(links, dev) || !on_device(in_even, dev) || !on_device(out_even, dev) ||
        (naik_long && !on_device(naik_long, dev)))
        return fail(STAG_ERR_INVALID_ARG,
                    "stag_apply_A_noalloc needs device memory of the current device for every array");
    double2* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_scratch_addr[dev] = nullptr;
                return fail(STAG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
            g_scratch_addr[dev] = static_cast<double2*>(p);
            g_scratch_ctx[dev] = ctx;
        }
        scratch = g_scratch_addr[dev];
    }
    Geom g{};
    g.lx = dims[0];
    g.ly = dims[1];
    g.lz = dims[2];
    g.lt = dims[3];
    g.lxh = g.lx / 2;
    g.vh = (int)(V / 2);
    g.vs = g.vh;
    for (int k = 0; k < 4; ++k) g.hop3[k] = 3 % dims[k];
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const double2* fat = reinterpret_cast<const double2*>(links);
    const double2* lng = reinterpret_cast<const double2*>(naik_long);
    const double2* in = reinterpret_cast<const double2*>(in_even);
    double2* out = reinterpret_cast<double2*>(out_even);
    launch_aos<false>(g, 1, fat, lng, in, scratch, nullptr, 0.0, s);   // scratch = D_oe in
    launch_aos<true>(g, 0, fat, lng, scratch, out, in, mass * mass, s);  // out = m^2 in - D_eo scratch
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(STAG_ERR_CUDA, std::string("stag_apply_A_noalloc: ") + cudaGetErrorString(e));
    return STAG_OK;
}
