// multi.cuh - types and launchers of the batched (many-system) kernels.
#pragma once

#include "stag_kernels.h"

namespace stag {

// One lattice (gauge field, mass) with nrhs right-hand sides; FP32 vectors are
// stored right-hand-side innermost: v[(colour * vs + site) * rpad + rhs].
struct MultiGroup {
    Geom g;
    const float2* fat;  // FP32 SoA links [2][4][9][vs], eta folded
    const float2* lng;  // or nullptr
    float2* d;          // search directions
    float2* t;          // odd-parity intermediate D_oe d
    float2* ad;         // A d
    float2* r;          // iterated residual (scaled by 1/sigma per RHS)
    float2* y;          // solution increment since the last replacement
    double m2;
    int nrhs;           // right-hand sides of this group
    int rpad;           // storage stride (nrhs rounded up to the largest block of RHS)
    int rhs0;           // global index of the group's first right-hand side (CG state)
    int prhs0;          // padded index of its first slot (partial sums, counters)
    int max_blocks;     // partial-sum stride per slot
};

struct MultiLaunch {
    const MultiGroup* groups;  // device array
    const int4* items;         // device array: (group, block in group, blocks in group, traversal:
                               // 0 contiguous runs of tiles, 1 resident sweep)
    CgScalars* scal;           // one per right-hand side, global index
    double* partials;          // [padded slots][max_blocks]
    unsigned int* counters;    // [padded slots], indexed by the group's first slot
    int out_parity;
    int phase;                 // 0: t = D_oe d;  1: Ad = m^2 d - D_eo t
};

enum MultiKernel { MK_DSLASH_PLAIN = 0, MK_DSLASH_CG = 1, MK_UPDATE_XR = 2, MK_UPDATE_D = 3, MK_DSLASH_AXPY = 4 };

// rb: right-hand sides per thread (1, 2, 4, 8; rpad / rb threads share a site, at most 32);
// bs: threads per block (64, 128, 256); mode: the items' traversal (0, 1, see multi.cu),
// which must be the same for every item of the launch
void launch_multi(MultiKernel k, const MultiLaunch& L, int nitems, int rb, int bs, int mode, cudaStream_t s);

// Blocks of the Dirac kernel of this shape that one SM holds at once (>= 1).
int multi_resident_blocks_per_sm(int rb, int bs);

// ----------------------------------------- device-side reliable updates (batch_dev.cu)
// Statuses a system ends with (the values of STAG_OK, STAG_ERR_NOT_CONVERGED, STAG_ERR_BREAKDOWN).
constexpr int STAG_STATUS_OK = 0;
constexpr int STAG_STATUS_NOT_CONVERGED = 3;
constexpr int STAG_STATUS_BREAKDOWN = 4;

// Phases of a system in a batched solve.
enum SysPhase { SYS_START = 0, SYS_RUNNING = 1, SYS_DUE = 2, SYS_CONFIRM = 3, SYS_REPLACE = 4, SYS_FINISHED = 5 };

// One system's fixed operands.
struct SysDev {
    Geom g;
    double m2;
    double2* x64;        // solution, FP64 SoA
    const double2* b64;  // source, FP64 SoA
    float4* u_ff;        // x as float-float
    float4* t_ff;        // D_oe u (float-float), or D_oe x (FP64, as double2) for the confirmation
    float4* ax;          // A x (float-float), or A x (FP64, as double2)
    float2* r;           // the group's RHS-innermost vectors and this system's slot
    float2* d;
    float2* y;
    int rpad, slot;
};

// One system's solve state (device; copied back at the end).
struct SysState {
    double bnorm2;       // |b|^2
    double tol;          // relative tolerance of the true residual
    double tol2;         // tol^2 |b|^2, the inner iteration's threshold
    double dtrue;        // last true |b - A x|^2 (float-float)
    double rel;          // last true |b - A x| / |b| (native FP64 once confirmed)
    double beta;         // beta of the pending replacement
    double rel_delta;    // replace once |r| < rel_delta * its maximum
    long long rel_interval;
    long long iters, max_iter;
    int phase, first, updates, status;
};

// A device-side list of systems: count, system indices, tile prefix (count + 1).
struct PassList {
    int* count;
    int* sys;
    int* prefix;
};

struct PassArgs {
    int n_sys;
    const SysDev* sys;
    SysState* state;
    CgScalars* scal;
    PassList fold, ff, confirm, replace;
    double* partials;  // one per tile of the largest list
    int* running;      // host-mapped: systems not finished
};

// The reliable-update pass (see batch_dev.cu) for every marked system, enqueued
// on s; oe/eo: each system's float-float and FP64 half-Dslash operands.
void enqueue_reliable_pass(const PassArgs& a, const SysDirac* oe_ff, const SysDirac* eo_ff, const SysDirac* oe_64,
                           const SysDirac* eo_64, int grid_dirac, int grid_vec, cudaStream_t s);

// single right-hand-side slot of a group's vectors
void launch_slot_set_residual(const Geom& g, const double2* r64, float2* r, float2* d, float2* y, int rpad, int slot,
                              double inv_sigma, double beta, bool first, cudaStream_t s);
void launch_slot_fold_y(const Geom& g, double2* x, float2* y, int rpad, int slot, double sigma, cudaStream_t s);
void launch_slot_put(const Geom& g, const double2* in, float2* out, int rpad, int slot, cudaStream_t s);
void launch_slot_get(const Geom& g, const float2* in, double2* out, int rpad, int slot, cudaStream_t s);

}  // namespace stag
