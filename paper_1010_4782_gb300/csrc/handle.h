// handle.h - the library's handle (internal; the ABI sees an opaque pointer).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/stag.h"
#include "stag_internal.cuh"

namespace stag {
struct KernelStat {
    double ms = 0.0;
    long long launches = 0;
};
}  // namespace stag

struct stag_handle {
    stag::Geom g{};
    int device = 0;
    double mass = 0.0;
    bool naik = false;
    stag_options opt{};
    cudaStream_t user_stream = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev_in = nullptr;
    // links
    double2* fat64 = nullptr;
    double2* lng64 = nullptr;
    float4* fatff = nullptr;
    float4* lngff = nullptr;  // [2][4][6][vs] when long_recon = 12 (allocated at the nine-entry size)
    float2 lng_s = {0.f, 0.f};  // long_recon = 12: 1 / long_scale as float-float
    // vectors: 16 bytes per complex, [3][vs]
    double2 *x = nullptr, *r = nullptr, *ad = nullptr, *b = nullptr;
    void* d = nullptr;   // CG direction (F64 or FF)
    void* t = nullptr;   // odd-parity intermediate (F64 or FF)
    void* u = nullptr;   // scratch even vector (F64 or FF)
    float4* xff = nullptr;   // FF: solution increment since the last fold into x
    // mixed precision: low-precision links and inner vectors
    float2* fat32 = nullptr;
    float2* lng32 = nullptr;
    __half2* fat16 = nullptr;
    __half2* lng16 = nullptr;
    __nv_bfloat162* fatb16 = nullptr;
    __nv_bfloat162* lngb16 = nullptr;
    void* lo_d = nullptr;    // [3][vs] float2 (F32), __half2 (F16) or __nv_bfloat162 (BF16)
    void* lo_t = nullptr;
    void* lo_ad = nullptr;
    void* lo_r = nullptr;
    float2* lo_y = nullptr;  // solution increment since the last replacement, FP32
    double2* x_best = nullptr;  // mixed precision: iterate with the smallest true residual so far
    double* io_a = nullptr;  // ABI-layout staging [vh][3] complex
    double* io_b = nullptr;
    // reductions
    double* partials = nullptr;
    stag::CgScalars* scal = nullptr;
    stag::CgScalars* scal_host = nullptr;  // pinned
    // graphs
    cudaGraphExec_t graph = nullptr;
    // timing
    std::vector<cudaEvent_t> events;
    stag::KernelStat stats[STAG_KERNEL_COUNT];
    long long device_bytes = 0;
    // device buffers (opt.guard_bands: each lies between two guard bands of
    // kGuardBytes filled with kGuardByte): user pointer, allocation base, user bytes
    struct Alloc {
        void* user;
        void* base;
        size_t bytes;
    };
    std::vector<Alloc> allocs;
    long long launches = 0;  // kernels launched by this handle (graph replays counted per kernel)
    std::string err = "no error";
    // called after every block of CG iterations of the plain solver (training-pair snapshots)
    std::function<void()> block_hook;
};

namespace stag {
// Guard bands of opt.guard_bands: this many bytes on each side of every buffer,
// filled with this byte.
constexpr size_t kGuardBytes = 4096;
constexpr unsigned char kGuardByte = 0xA5;

// A scoped NVTX range (visible to profilers; no cost without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char* name);
    ~NvtxRange();
};

// Internal entry points of capi.cu used by the preconditioner code (pt.cu).
// They report failures by throwing HandleError with the handle's message set.
struct HandleError {
    int code;
};
// out = A in with native FP64 kernels on internal F64 SoA vectors (uses h->t).
void handle_apply_A_f64(stag_handle* h, const double2* in, double2* out);
// Plain CG (Fig. 1 with true-residual restarts) on the vectors already packed
// into h->b and h->x; returns the STAG_* status and fills info.
int handle_solve_packed(stag_handle* h, double bnorm2, double tol, long long max_it, stag_solve_info& info);
void handle_begin(stag_handle* h);
void handle_end(stag_handle* h);
bool handle_is_device_ptr(stag_handle* h, const void* p);
}  // namespace stag
