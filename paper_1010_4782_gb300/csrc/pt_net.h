// pt_net.h - the network object of the learned preconditioner (internal; the
// ABI sees an opaque pointer), shared by pt.cu (network, training) and fcg.cu
// (flexible CG).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "handle.h"
#include "pt_common.cuh"

namespace stag {

// Device state of one flexible-CG cycle beside the CG scalars it shares with
// the Dirac kernels' reduction epilogue (which computes (p, A p) and alpha).
// sc.delta_new holds (r, z).
struct FcgState {
    double rr;          // |r|^2 after the last update
    double best;        // least |r|^2 of the cycle
    double mark;        // best at its last drop by 10 % (of |r|)
    long long mark_it;  // cycle iteration of that drop
    int why;            // FCG_WHY_*: why the cycle stopped early
    int pad;
};
constexpr int FCG_WHY_NONE = 0;
constexpr int FCG_WHY_RZ = 1;     // (r, z) <= 0
constexpr int FCG_WHY_STALL = 2;  // the best |r| has not dropped by 10 % in 100 iterations

struct FcgDev {
    CgScalars sc;
    FcgState st;
};

}  // namespace stag

struct stag_ptnet {
    stag_handle* h = nullptr;
    stag::Geom g{};
    int prec = STAG_ARITH_BF16;  // activation storage of training and pairs: STAG_ARITH_BF16 or STAG_ARITH_F32
    int inf_prec = STAG_ARITH_BF16;  // activation storage when the network is applied
    size_t elem = 4;             // bytes per stored complex
    float2* links = nullptr;     // FP32 eta-folded fat links (transports and A)
    __half2* links16 = nullptr;  // the same / links16_scale in FP16 (two-hop inference with BF16 storage)
    float links16_scale = 1.f;   // a power of two near the largest link entry
    float2* lng = nullptr;       // FP32 eta-folded Naik links (A), or nullptr
    float2 *va = nullptr, *vt = nullptr, *vad = nullptr;  // FP32 [3][vs] vectors for A d
    std::vector<float2> w_host;  // weights, layer-major [9][C_out][C_in]
    float2* w = nullptr;         // device weights (FP32 master)
    bool use_tc = true;          // BF16 8 -> 8 forward layer on the tensor cores (pt_tc.cu)
    int inf_form = STAG_PTNET_COLLAPSED;  // how the network is evaluated when applied
    float2* coef = nullptr;      // collapsed form: k0, H[8][8] (pt_collapse)
    int* tc_err = nullptr;       // set by a tensor-core layer whose bounded wait ran out
    unsigned int* dot_counter = nullptr;  // last-block ticket of pt_dots_kernel
    double* dot_out = nullptr;            // its three sums
    float2* grad = nullptr;
    float *adam_m = nullptr, *adam_v = nullptr;
    long long adam_t = 0;
    void* act[stag::kLayers + 1] = {};  // activations (whole lattice)
    void* gact[stag::kLayers + 1] = {}; // gradients of activations
    float2* wpart = nullptr;      // weight-gradient partials
    double* red = nullptr;        // reduction partials
    std::vector<double> red_host;
    // training pairs: r and e slots (even sites, [3][vs]) and <e, A e>
    std::vector<void*> pairs_r, pairs_e;
    std::vector<double> pairs_eae;
    void* scratch_r = nullptr;  // slots for stag_ptnet_loss_grad
    void* scratch_e = nullptr;
    // stag_ptnet_apply's FP64 SoA vectors; fq also holds A x in flexible CG
    double2 *fr = nullptr, *fz = nullptr, *fq = nullptr;
    // flexible CG (fcg.cu): work vectors [3][vs] in the handle's arithmetic
    // (float-float float4 or FP64 double2, 16 bytes a complex either way)
    void *fcg_r = nullptr, *fcg_p = nullptr, *fcg_q = nullptr, *fcg_t = nullptr, *fcg_x = nullptr;
    stag::FcgDev* fcg_dev = nullptr;   // device state
    stag::FcgDev* fcg_host = nullptr;  // pinned copy read between graph replays
    cudaGraphExec_t fcg_graph = nullptr;
    int fcg_graph_key = -1;            // configuration the graph was captured for
    long long device_bytes = 0;
    std::string err = "no error";
};

namespace stag {

// Failure inside a network call: the message is in n->err.
struct PFail {
    int code;
};
[[noreturn]] void pfail(stag_ptnet* n, int code, const std::string& msg);
void pcheck(stag_ptnet* n, cudaError_t e, const char* what);
void* palloc(stag_ptnet* n, size_t bytes, const char* what);
inline cudaStream_t S(stag_ptnet* n) { return n->h->s; }
inline bool infer_bf16(const stag_ptnet* n) { return n->inf_prec == STAG_ARITH_BF16; }
// Fails with STAG_ERR_TIMEOUT if a tensor-core layer reported a bounded wait that ran out.
void check_tc(stag_ptnet* n);

// Collapsed form (STAG_PTNET_COLLAPSED): n->coef from the current weights
// (pt_collapse), then chi (act[2], [8][3][vs] on odd sites, stored in the
// inference precision) from r on even sites; every kernel returns at once
// while *skip is nonzero (skip nullable).  The even-site output is
// pt_out_site (pt_common.cuh).
void pt_collapse(stag_ptnet* n);
void launch_pt_chi(stag_ptnet* n, const float4* r, const int* skip);
void launch_pt_chi(stag_ptnet* n, const double2* r, const int* skip);

// act[3] (even sites) = M r for r on even sites ([3][vs]: float4 float-float
// or double2 FP64), with the inference precision and layers of n, unscaled
// (the network is linear and BF16 keeps FP32's exponent range).  Every kernel
// returns at once while *skip is nonzero (skip nullable).
void pt_network_from_vec(stag_ptnet* n, const float4* r, const int* skip);
void pt_network_from_vec(stag_ptnet* n, const double2* r, const int* skip);

}  // namespace stag
