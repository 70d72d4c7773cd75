// probe.cu - stag_measure_fma_rate: the fused multiply-add rate of this GPU,
// measured, for the arithmetic ceiling of the Dirac kernels' roofline.
//
// The paper's cost model (Sec. 2, text after Eq. (5)) counts each SU(3) x
// vector product of the Dslash as 36 real multiply-adds (9 complex ones).  In
// native FP64 a Naik site of the half-Dslash is therefore 16 x 36 = 576 DFMA.
// Whether that kernel is bound by HBM or by the FP64 pipe depends on the
// chip's DFMA rate, which this probe measures instead of assuming: every
// thread of a grid over all SMs runs kChains independent FMA chains (enough
// independent work to cover the pipe's latency) for a fixed number of steps,
// timed with CUDA events on a private stream after one warm-up launch, for
// two operand patterns; the faster one sets the rate.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/stag.h"

namespace stag {

void set_noalloc_error(const std::string& msg);  // thread-local message of stag_last_error(NULL)

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

// Two operand patterns, both with kChains independent chains per thread:
//  * ACC: acc_k <- x_k * y_(k+u) + acc_k, the pattern of a complex
//    multiply-accumulate (the Dirac kernels' inner step); on GB300 the FP64
//    pipe sustains about 19 % more DFMA per second with it;
//  * CHAIN: a_k <- a_k * m + c with one shared multiplier, which the FP32
//    pipes sustain best.
// x is small and y, m below 1, so the values stay bounded and normal.  The
// result is stored only if it equals `never` (a NaN passed at run time), which
// the compiler cannot rule out, so no FMA is dropped.
template <class T, bool ACC>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int steps, T m, T c, T never, T* out) {
    T acc[kChains], x[kChains], y[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        acc[k] = ACC ? (T)0 : (T)(threadIdx.x + k) * c;
        x[k] = (T)(threadIdx.x + k) * c;
        y[k] = m + (T)k * c;
    }
#pragma unroll 1
    for (int s = 0; s < steps; ++s) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if (ACC)
                    acc[k] = fma(x[k], y[(k + u) % kChains], acc[k]);
                else
                    acc[k] = fma(acc[k], m, c);
            }
        }
    }
    T sum = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) sum += acc[k];
    if (sum == never) *out = sum;
}

template <class T>
int measure(double* rate) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_noalloc_error("stag_measure_fma_rate: no usable CUDA device");
        return STAG_ERR_CUDA;
    }
    // about 6e10 FMA per launch in FP64 (~0.1 s at 0.6 T/s), 30x more in FP32
    const int steps = sizeof(T) == 8 ? 6000 : 180000;
    const int blocks = sms * kBlocksPerSm;  // full occupancy at 256 threads
    T* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(T));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;  // the faster of the two patterns
    for (int pattern = 0; pattern < 2 && e == cudaSuccess; ++pattern) {
        const T m = (T)0.5, c = (T)1e-7, never = (T)NAN;
        auto launch = [&](int n) {
            if (pattern)
                fma_chain_kernel<T, false><<<blocks, kThreads, 0, s>>>(n, (T)0.999999, (T)1e-6, never, out);
            else
                fma_chain_kernel<T, true><<<blocks, kThreads, 0, s>>>(n, m, c, never, out);
        };
        launch(steps / 10);  // warm-up
        cudaEventRecord(e0, s);
        launch(steps);
        cudaEventRecord(e1, s);
        e = cudaGetLastError();
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && (ms == 0.f || t < ms)) ms = t;
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    if (e != cudaSuccess || ms <= 0.f) {
        set_noalloc_error(std::string("stag_measure_fma_rate: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? STAG_ERR_OOM : STAG_ERR_CUDA;
    }
    const double fmas = (double)blocks * kThreads * kChains * 4.0 * steps;
    *rate = fmas / (ms * 1e-3);
    return STAG_OK;
}

}  // namespace
}  // namespace stag

extern "C" int stag_measure_fma_rate(int32_t bits, double* fma_per_second) {
    if (!fma_per_second || (bits != 32 && bits != 64)) {
        stag::set_noalloc_error("stag_measure_fma_rate: bits must be 32 or 64 and the output non-NULL");
        return STAG_ERR_INVALID_ARG;
    }
    return bits == 64 ? stag::measure<double>(fma_per_second) : stag::measure<float>(fma_per_second);
}
