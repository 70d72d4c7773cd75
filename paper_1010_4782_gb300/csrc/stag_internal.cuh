// stag_internal.cuh - internal types of the sm_103a staggered even-odd CG library.
//
// Device layouts (structure of arrays, site index fastest, so consecutive
// threads of a warp touch consecutive 16-byte words):
//   links  (F64)  double2 [parity][mu][k = 3*row + col][vs]      eta folded in
//   links  (FF)   float4  [parity][mu][k][vs]                    (re_hi, re_lo, im_hi, im_lo)
//   vector (F64)  double2 [colour][vs]
//   vector (FF)   float4  [colour][vs]
// vs is V/2 rounded up to a multiple of 64; padding entries are zero.
// The half-lattice index of a site is its lexicographic index / 2, with x
// fastest (the same numbering as the ABI's [V/2][3] vectors).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stag {

constexpr int kBlock = 256;          // threads per block of every site kernel
constexpr int kMaxPartials = 1 << 20; // capacity of the per-block partial-sum buffer

struct Geom {
    int lx, ly, lz, lt;
    int lxh;        // lx / 2
    int vh;         // sites per parity
    int vs;         // padded plane stride (elements)
    int hop3[4];    // 3 mod L_mu, the Naik hop reduced to one period
};

// Device-resident CG state.  Written only by the last block of a reduction
// kernel; read by every block of the following kernels.
struct CgScalars {
    double delta_new;
    double delta_old;
    double pAp;        // Re(d^dag A d)
    double alpha;
    double beta;
    double threshold;  // stop once delta_new <= threshold
    double m2;         // m^2 of Eq. (3)
    double red_out;    // result of a stand-alone reduction
    long long iter;    // Fig. 1 iterations done since the last reset
    long long max_iter;
    int done;          // 1 once Fig. 1's loop condition is false
    int status;        // 0, or STAG_ERR_BREAKDOWN
    unsigned int counter; // blocks finished in the current reduction
    int pad;
    float2 m2_ff;      // m^2, alpha, beta as float-float pairs (hi, lo)
    float2 alpha_ff;
    float2 beta_ff;
    float2 pad2;
    // reliable updates of the mixed-precision solver
    double maxr;             // max |r| since the last residual replacement
    double rel_delta;        // replace once |r| < rel_delta * maxr
    long long iter_since;    // iterations since the last replacement
    long long rel_interval;  // ... or after this many iterations
};

// Host-side float-float split of a double: hi = fl32(a), lo = fl32(a - hi).
inline float2 host_ff_from_double(double a) {
    const float hi = (float)a;
    const float lo = (float)(a - (double)hi);
    return make_float2(hi, lo);
}

// -------------------------------------------------------------- geometry
__device__ __forceinline__ void site_coords(int i, int P, const Geom& g, int& x, int& y, int& z,
                                            int& t) {
    const int xh = i % g.lxh;
    int r = i / g.lxh;
    y = r % g.ly;
    r /= g.ly;
    z = r % g.lz;
    t = r / g.lz;
    x = 2 * xh + ((P + y + z + t) & 1);
}

__device__ __forceinline__ int site_index(int x, int y, int z, int t, const Geom& g) {
    return (((t * g.lz + z) * g.ly + y) * g.lx + x) >> 1;
}

__device__ __forceinline__ int wrap_up(int c, int k, int L) {
    c += k;
    return c >= L ? c - L : c;
}
__device__ __forceinline__ int wrap_dn(int c, int k, int L) {
    c -= k;
    return c < 0 ? c + L : c;
}

// ------------------------------------------------------- FP64 complex ops
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// acc += a * b
__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc -= conj(a) * b
__device__ __forceinline__ void cmsc_conj(double2& acc, double2 a, double2 b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// ------------------------------------------------------- FP32 complex ops
__device__ __forceinline__ void cmacf(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmscf_conj(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(-a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(-a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// ---------------------------------------------------- block reductions
// Sum of v over the block, deterministic (fixed shuffle tree), valid in thread 0.
template <int BS>
__device__ __forceinline__ double block_sum(double v, double* smem) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) smem[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = lane < BS / 32 ? smem[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Each block writes its partial; the last block to finish sums all partials
// in block order and returns true in every one of its threads, with the total
// in *total (valid in all threads of that block).  Other blocks return false.
template <int BS>
__device__ __forceinline__ bool grid_sum_last_block(double v, double* partials, unsigned int* counter,
                                                    double* total) {
    __shared__ double smem[BS / 32];
    __shared__ bool is_last;
    __shared__ double result;
    v = block_sum<BS>(v, smem);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = v;
        __threadfence();
        const unsigned int ticket = atomicAdd(counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += BS) s += __ldcg(partials + b);
    __syncthreads();  // smem reuse
    s = block_sum<BS>(s, smem);
    if (threadIdx.x == 0) {
        result = s;
        *counter = 0u;
    }
    __syncthreads();
    *total = result;
    return true;
}

// ------------------------------------------------------ launch helpers
inline int blocks_for(int n, int bs = kBlock) { return (n + bs - 1) / bs; }

}  // namespace stag
