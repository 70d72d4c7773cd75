// dd.cu - single-GPU emulation of the paper's multi-GPU domain decomposition
// (Sec. 4, Table 2).
//
// The lattice is cut into P slabs along t ("ranks").  Each rank stores its slab
// extended by G ghost t-slices on each side (G = 2 for the one-hop operator,
// 4 with the Naik term: the hop reach 1 or 3 rounded up to an even number, so
// that a site's parity - and eta, which never involves t - is the same in the
// rank's local coordinates as in the global ones).  A half-Dslash on a rank is
// then the library's Dirac kernel run over the rank's interior sites, one
// contiguous range of its local site numbering.  Before each half-Dslash the
// input's boundary slices (depth 1 or 3) are exchanged, in the steps of Sec. 4:
//   collect  - a kernel packs each rank's two boundary faces into a buffer;
//   D2H      - the buffers are copied to pinned host memory;
//   "MPI"    - host copies move each face to the neighbouring rank's buffer;
//   H2D      - the received faces are copied to the device;
//   unpack   - a kernel writes them into the ghost slices;
// or, in the device mode (the GPUDirect-style path the paper proposes in
// Sec. 5), by device-to-device copies between the ranks' buffers.  Every step
// is timed with CUDA events (host copies with the host clock).  All ranks share
// one GPU and one stream, so each step's total over the ranks is the work of the
// whole machine; divided by P it is the time of one rank on its own GPU.
//
// The CG solve follows Fig. 1 with the paper's host-driven structure: every
// dot product is a per-rank partial sum, gathered to the host and summed over
// the ranks (the global sum an MPI all-reduce would do).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/stag.h"
#include "handle.h"
#include "stag_kernels.h"

namespace stag {

// buf[c][k] <- v[c][s0 + k], k < n   (and the reverse)
__global__ void dd_pack_kernel(const double2* __restrict__ v, size_t vs, int s0, int n, double2* __restrict__ buf) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) buf[(size_t)c * n + k] = v[(size_t)c * vs + s0 + k];
}

__global__ void dd_unpack_kernel(const double2* __restrict__ buf, int n, double2* __restrict__ v, size_t vs, int s0) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) v[(size_t)c * vs + s0 + k] = buf[(size_t)c * n + k];
}

// per-block partials of Re<a, b> over sites [i0, i1)
__global__ void __launch_bounds__(kBlock) dd_dot_kernel(const double2* __restrict__ a, const double2* __restrict__ b,
                                                        size_t vs, int i0, int i1, double* __restrict__ partials) {
    const int i = i0 + blockIdx.x * kBlock + threadIdx.x;
    double acc = 0.0;
    if (i < i1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 x = a[(size_t)c * vs + i], y = b[(size_t)c * vs + i];
            acc = fma(x.x, y.x, fma(x.y, y.y, acc));
        }
    }
    __shared__ double sm[kBlock / 32];
    const double s = block_sum<kBlock>(acc, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// y = a x + y over sites [i0, i1)   (mode 0);   y = x + a y   (mode 1)
__global__ void __launch_bounds__(kBlock) dd_axpy_kernel(double a, const double2* __restrict__ x, double2* y, size_t vs,
                                                         int i0, int i1, int mode) {
    const int i = i0 + blockIdx.x * kBlock + threadIdx.x;
    if (i >= i1) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = (size_t)c * vs + i;
        const double2 xx = x[k], yy = y[k];
        y[k] = mode == 0 ? make_double2(fma(a, xx.x, yy.x), fma(a, xx.y, yy.y))
                         : make_double2(fma(a, yy.x, xx.x), fma(a, yy.y, xx.y));
    }
}

}  // namespace stag

using namespace stag;

enum { DD_CALC = 0, DD_COLLECT = 1, DD_D2H = 2, DD_MPI = 3, DD_H2D = 4, DD_SUM = 5, DD_PHASES = 6 };

struct stag_dd {
    stag_handle* h = nullptr;
    int P = 1;
    int depth = 1;  // hop reach
    int G = 2;      // ghost slices per side (even)
    int ltl = 0;    // interior t-slices per rank
    int v3h = 0;    // sites of one parity in a t-slice
    Geom gl{};      // a rank's extended local lattice
    std::vector<double2*> fat, lng;  // per rank
    std::vector<double2*> vin, vt, vout, x, r, d, b;  // per rank, [3][vs_l]
    std::vector<double2*> s_lo, s_hi, r_lo, r_hi;     // device face buffers per rank
    std::vector<double2*> hs_lo, hs_hi, hr_lo, hr_hi; // pinned host face buffers per rank
    double* partials = nullptr;
    std::vector<double> partials_host;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaStream_t cs = nullptr;                             // copy stream of the overlapped modes
    cudaEvent_t eo[3] = {nullptr, nullptr, nullptr};       // faces packed, faces on the host, faces in
    double phase[DD_PHASES] = {};
    long long bytes_exchanged = 0;
    std::string err = "no error";
};

namespace {

struct DFail {
    int code;
};

void dfail(stag_dd* dd, int code, const std::string& m) {
    dd->err = m;
    throw DFail{code};
}

void dcheck(stag_dd* dd, cudaError_t e, const char* what) {
    if (e != cudaSuccess)
        dfail(dd, e == cudaErrorMemoryAllocation ? STAG_ERR_OOM : STAG_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
T* dalloc(stag_dd* dd, size_t bytes, bool host = false) {
    void* p = nullptr;
    if (host)
        dcheck(dd, cudaMallocHost(&p, bytes), "allocate pinned buffer");
    else
        dcheck(dd, cudaMalloc(&p, bytes), "allocate");
    if (!host) dcheck(dd, cudaMemsetAsync(p, 0, bytes, dd->h->s), "clear");
    return static_cast<T*>(p);
}

cudaStream_t S(stag_dd* dd) { return dd->h->s; }
size_t vecb(const stag_dd* dd) { return (size_t)3 * dd->gl.vs * sizeof(double2); }
int interior0(const stag_dd* dd) { return dd->G * dd->v3h; }
int interior1(const stag_dd* dd) { return (dd->G + dd->ltl) * dd->v3h; }
int face_n(const stag_dd* dd) { return dd->depth * dd->v3h; }

// GPU phase timing: [start, stop) brackets on the handle's stream
void tstart(stag_dd* dd) { cudaEventRecord(dd->ev[0], S(dd)); }
void tstop(stag_dd* dd, int ph) {
    cudaEventRecord(dd->ev[1], S(dd));
    dcheck(dd, cudaEventSynchronize(dd->ev[1]), "phase timing");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, dd->ev[0], dd->ev[1]);
    dd->phase[ph] += ms;
}

// ghost slices of vectors v[rank] (parity of the vector is irrelevant: a face
// is a t-slice range of one parity's plane) from the neighbouring ranks
void exchange(stag_dd* dd, const std::vector<double2*>& v, int mode) {
    const int P = dd->P, n = face_n(dd);
    const size_t vs = (size_t)dd->gl.vs;
    const size_t fb = (size_t)3 * n * sizeof(double2);
    const int bl = blocks_for(n);
    // collect: the lowest and highest `depth` interior slices
    tstart(dd);
    for (int q = 0; q < P; ++q) {
        dd_pack_kernel<<<bl, kBlock, 0, S(dd)>>>(v[q], vs, interior0(dd), n, dd->s_lo[q]);
        dd_pack_kernel<<<bl, kBlock, 0, S(dd)>>>(v[q], vs, interior1(dd) - n, n, dd->s_hi[q]);
    }
    tstop(dd, DD_COLLECT);
    if (mode == STAG_DD_HOST) {
        tstart(dd);
        for (int q = 0; q < P; ++q) {
            cudaMemcpyAsync(dd->hs_lo[q], dd->s_lo[q], fb, cudaMemcpyDeviceToHost, S(dd));
            cudaMemcpyAsync(dd->hs_hi[q], dd->s_hi[q], fb, cudaMemcpyDeviceToHost, S(dd));
        }
        tstop(dd, DD_D2H);
        const auto t0 = std::chrono::steady_clock::now();
        for (int q = 0; q < P; ++q) {
            // rank q's lower ghost <- rank q-1's highest slices; upper ghost <- rank q+1's lowest
            std::memcpy(dd->hr_lo[q], dd->hs_hi[(q + P - 1) % P], fb);
            std::memcpy(dd->hr_hi[q], dd->hs_lo[(q + 1) % P], fb);
        }
        dd->phase[DD_MPI] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        tstart(dd);
        for (int q = 0; q < P; ++q) {
            cudaMemcpyAsync(dd->r_lo[q], dd->hr_lo[q], fb, cudaMemcpyHostToDevice, S(dd));
            cudaMemcpyAsync(dd->r_hi[q], dd->hr_hi[q], fb, cudaMemcpyHostToDevice, S(dd));
        }
        tstop(dd, DD_H2D);
    } else {
        tstart(dd);
        for (int q = 0; q < P; ++q) {
            cudaMemcpyAsync(dd->r_lo[q], dd->s_hi[(q + P - 1) % P], fb, cudaMemcpyDeviceToDevice, S(dd));
            cudaMemcpyAsync(dd->r_hi[q], dd->s_lo[(q + 1) % P], fb, cudaMemcpyDeviceToDevice, S(dd));
        }
        tstop(dd, DD_MPI);
    }
    tstart(dd);
    for (int q = 0; q < P; ++q) {
        dd_unpack_kernel<<<bl, kBlock, 0, S(dd)>>>(dd->r_lo[q], n, v[q], vs, interior0(dd) - n);
        dd_unpack_kernel<<<bl, kBlock, 0, S(dd)>>>(dd->r_hi[q], n, v[q], vs, interior1(dd));
    }
    tstop(dd, DD_COLLECT);
    dd->bytes_exchanged += 2LL * P * (long long)fb;
    dcheck(dd, cudaGetLastError(), "halo exchange");
}

// One half-Dslash on every rank with the face exchange overlapped with the
// interior (Sec. 5's proposal): after the faces are packed, the copies run on
// a second stream (and the host copies on the host thread) while the sites
// whose stencil stays inside the rank's own slab, t-slices
// [G + depth, G + ltl - depth), are computed; the boundary slices follow once
// the faces are unpacked.  Every site runs the same kernel as in the plain
// modes, so the result is bit-identical.  Timed as a whole (phase 0); the host
// copy time is also recorded (phase 3), though it is hidden.
void half_overlap(stag_dd* dd, int parity, const std::vector<double2*>& in, const std::vector<double2*>& out,
                  Epilogue epi, const std::vector<double2*>* src, double m2, bool host) {
    const int P = dd->P, n = face_n(dd);
    const size_t vs = (size_t)dd->gl.vs;
    const size_t fb = (size_t)3 * n * sizeof(double2);
    const int bl = blocks_for(n);
    const int v3h = dd->v3h, G = dd->G, ltl = dd->ltl;
    const int lo_end = std::min(G + dd->depth, G + ltl);
    const int hi_start = std::max(G + ltl - dd->depth, lo_end);
    auto dirac = [&](int q, int s0, int s1) {
        const LinkSet L{dd->fat[q], dd->lng[q], nullptr, nullptr};
        launch_dslash_f64_range(dd->gl, parity, L, in[q], out[q], epi, src ? (*src)[q] : nullptr, m2, s0 * v3h,
                                s1 * v3h, S(dd));
    };
    tstart(dd);
    for (int q = 0; q < P; ++q) {
        dd_pack_kernel<<<bl, kBlock, 0, S(dd)>>>(in[q], vs, interior0(dd), n, dd->s_lo[q]);
        dd_pack_kernel<<<bl, kBlock, 0, S(dd)>>>(in[q], vs, interior1(dd) - n, n, dd->s_hi[q]);
    }
    dcheck(dd, cudaEventRecord(dd->eo[0], S(dd)), "event");
    dcheck(dd, cudaStreamWaitEvent(dd->cs, dd->eo[0], 0), "stream wait");
    if (host) {
        for (int q = 0; q < P; ++q) {
            cudaMemcpyAsync(dd->hs_lo[q], dd->s_lo[q], fb, cudaMemcpyDeviceToHost, dd->cs);
            cudaMemcpyAsync(dd->hs_hi[q], dd->s_hi[q], fb, cudaMemcpyDeviceToHost, dd->cs);
        }
        dcheck(dd, cudaEventRecord(dd->eo[1], dd->cs), "event");
    } else {
        for (int q = 0; q < P; ++q) {
            cudaMemcpyAsync(dd->r_lo[q], dd->s_hi[(q + P - 1) % P], fb, cudaMemcpyDeviceToDevice, dd->cs);
            cudaMemcpyAsync(dd->r_hi[q], dd->s_lo[(q + 1) % P], fb, cudaMemcpyDeviceToDevice, dd->cs);
        }
    }
    for (int q = 0; q < P; ++q) dirac(q, lo_end, hi_start);  // interior, overlapping the copies
    if (host) {
        dcheck(dd, cudaEventSynchronize(dd->eo[1]), "faces to host");
        const auto t0 = std::chrono::steady_clock::now();
        for (int q = 0; q < P; ++q) {
            std::memcpy(dd->hr_lo[q], dd->hs_hi[(q + P - 1) % P], fb);
            std::memcpy(dd->hr_hi[q], dd->hs_lo[(q + 1) % P], fb);
        }
        dd->phase[DD_MPI] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        for (int q = 0; q < P; ++q) {
            cudaMemcpyAsync(dd->r_lo[q], dd->hr_lo[q], fb, cudaMemcpyHostToDevice, dd->cs);
            cudaMemcpyAsync(dd->r_hi[q], dd->hr_hi[q], fb, cudaMemcpyHostToDevice, dd->cs);
        }
    }
    dcheck(dd, cudaEventRecord(dd->eo[2], dd->cs), "event");
    dcheck(dd, cudaStreamWaitEvent(S(dd), dd->eo[2], 0), "stream wait");
    for (int q = 0; q < P; ++q) {
        dd_unpack_kernel<<<bl, kBlock, 0, S(dd)>>>(dd->r_lo[q], n, in[q], vs, interior0(dd) - n);
        dd_unpack_kernel<<<bl, kBlock, 0, S(dd)>>>(dd->r_hi[q], n, in[q], vs, interior1(dd));
    }
    for (int q = 0; q < P; ++q) {
        dirac(q, G, lo_end);
        if (hi_start < G + ltl) dirac(q, hi_start, G + ltl);
    }
    tstop(dd, DD_CALC);
    dd->bytes_exchanged += 2LL * P * (long long)fb;
    dcheck(dd, cudaGetLastError(), "overlapped half-Dslash");
}

// out[q] = A in[q] on every rank's interior (in is exchanged; uses vt)
void dd_apply(stag_dd* dd, const std::vector<double2*>& in, const std::vector<double2*>& out, int mode) {
    const double m2 = dd->h->mass * dd->h->mass;
    if (mode == STAG_DD_HOST_OVERLAP || mode == STAG_DD_DEVICE_OVERLAP) {
        const bool host = mode == STAG_DD_HOST_OVERLAP;
        half_overlap(dd, 1, in, dd->vt, EPI_PLAIN, nullptr, 0.0, host);
        half_overlap(dd, 0, dd->vt, out, EPI_AXPY, &in, m2, host);
        return;
    }
    exchange(dd, in, mode);
    tstart(dd);
    for (int q = 0; q < dd->P; ++q) {
        const LinkSet L{dd->fat[q], dd->lng[q], nullptr, nullptr};
        launch_dslash_f64_range(dd->gl, 1, L, in[q], dd->vt[q], EPI_PLAIN, nullptr, 0.0, interior0(dd),
                                interior1(dd), S(dd));
    }
    tstop(dd, DD_CALC);
    exchange(dd, dd->vt, mode);
    tstart(dd);
    for (int q = 0; q < dd->P; ++q) {
        const LinkSet L{dd->fat[q], dd->lng[q], nullptr, nullptr};
        launch_dslash_f64_range(dd->gl, 0, L, dd->vt[q], out[q], EPI_AXPY, in[q], m2, interior0(dd), interior1(dd),
                                S(dd));
    }
    tstop(dd, DD_CALC);
    dcheck(dd, cudaGetLastError(), "decomposed A");
}

// global Re<a, b>: per-rank partial sums, summed over the ranks on the host
double dd_dot(stag_dd* dd, const std::vector<double2*>& a, const std::vector<double2*>& b) {
    const int nb = blocks_for(dd->ltl * dd->v3h);
    tstart(dd);
    for (int q = 0; q < dd->P; ++q)
        dd_dot_kernel<<<nb, kBlock, 0, S(dd)>>>(a[q], b[q], dd->gl.vs, interior0(dd), interior1(dd),
                                                dd->partials + (size_t)q * nb);
    const size_t n = (size_t)dd->P * nb;
    dd->partials_host.resize(n);
    cudaMemcpyAsync(dd->partials_host.data(), dd->partials, n * sizeof(double), cudaMemcpyDeviceToHost, S(dd));
    tstop(dd, DD_SUM);
    double s = 0.0;
    for (size_t k = 0; k < n; ++k) s += dd->partials_host[k];
    return s;
}

void dd_axpy(stag_dd* dd, double a, const std::vector<double2*>& x, const std::vector<double2*>& y, int mode) {
    const int nb = blocks_for(dd->ltl * dd->v3h);
    for (int q = 0; q < dd->P; ++q)
        dd_axpy_kernel<<<nb, kBlock, 0, S(dd)>>>(a, x[q], y[q], dd->gl.vs, interior0(dd), interior1(dd), mode);
}

// global SoA vector (the handle's layout) <-> rank interiors
void scatter(stag_dd* dd, const double2* g, const std::vector<double2*>& v) {
    const size_t gvs = (size_t)dd->h->g.vs, lvs = (size_t)dd->gl.vs;
    const size_t n = (size_t)dd->ltl * dd->v3h;
    for (int q = 0; q < dd->P; ++q)
        for (int c = 0; c < 3; ++c)
            cudaMemcpyAsync(v[q] + c * lvs + interior0(dd), g + c * gvs + (size_t)q * n, n * sizeof(double2),
                            cudaMemcpyDeviceToDevice, S(dd));
}

void gather(stag_dd* dd, const std::vector<double2*>& v, double2* g) {
    const size_t gvs = (size_t)dd->h->g.vs, lvs = (size_t)dd->gl.vs;
    const size_t n = (size_t)dd->ltl * dd->v3h;
    for (int q = 0; q < dd->P; ++q)
        for (int c = 0; c < 3; ++c)
            cudaMemcpyAsync(g + c * gvs + (size_t)q * n, v[q] + c * lvs + interior0(dd), n * sizeof(double2),
                            cudaMemcpyDeviceToDevice, S(dd));
}

// a rank's extended links from the handle's packed (eta-folded) FP64 links
void copy_links(stag_dd* dd, const double2* src, double2* dst, int q) {
    const Geom& g = dd->h->g;
    const int lt_ext = dd->ltl + 2 * dd->G;
    for (int plane = 0; plane < 2 * 4 * 9; ++plane) {
        for (int te = 0; te < lt_ext; ++te) {
            const int tg = ((q * dd->ltl - dd->G + te) % g.lt + g.lt) % g.lt;
            cudaMemcpyAsync(dst + (size_t)plane * dd->gl.vs + (size_t)te * dd->v3h,
                            src + (size_t)plane * g.vs + (size_t)tg * dd->v3h, (size_t)dd->v3h * sizeof(double2),
                            cudaMemcpyDeviceToDevice, S(dd));
        }
    }
}

void destroy_dd(stag_dd* dd) {
    if (!dd) return;
    if (dd->h && dd->h->s) cudaStreamSynchronize(dd->h->s);
    for (auto* vec : {&dd->fat, &dd->lng, &dd->vin, &dd->vt, &dd->vout, &dd->x, &dd->r, &dd->d, &dd->b, &dd->s_lo,
                      &dd->s_hi, &dd->r_lo, &dd->r_hi})
        for (double2* p : *vec)
            if (p) cudaFree(p);
    for (auto* vec : {&dd->hs_lo, &dd->hs_hi, &dd->hr_lo, &dd->hr_hi})
        for (double2* p : *vec)
            if (p) cudaFreeHost(p);
    if (dd->partials) cudaFree(dd->partials);
    for (cudaEvent_t e : dd->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : dd->eo)
        if (e) cudaEventDestroy(e);
    if (dd->cs) {
        cudaStreamSynchronize(dd->cs);
        cudaStreamDestroy(dd->cs);
    }
    delete dd;
}

void report(stag_dd* dd, double* phase_ms) {
    if (phase_ms)
        for (int k = 0; k < DD_PHASES; ++k) phase_ms[k] = dd->phase[k];
}

}  // namespace

extern "C" {

int stag_dd_create(stag_dd** out, stag_handle* h, int32_t n_ranks) {
    if (out) *out = nullptr;
    if (!out || !h || n_ranks < 1) return STAG_ERR_INVALID_ARG;
    const Geom& g = h->g;
    const int depth = h->lng64 ? 3 : 1;
    const int G = depth == 1 ? 2 : 4;
    if (g.lt % n_ranks || (g.lt / n_ranks) % 2 || g.lt / n_ranks < depth) {
        h->err = "Lt must split into equal slabs of even extent >= the hop reach";
        return STAG_ERR_INVALID_ARG;
    }
    stag_dd* dd = new stag_dd();
    try {
        dd->h = h;
        dd->P = n_ranks;
        dd->depth = depth;
        dd->G = G;
        dd->ltl = g.lt / n_ranks;
        dd->v3h = g.lx * g.ly * g.lz / 2;
        Geom& l = dd->gl;
        l = g;
        l.lt = dd->ltl + 2 * G;
        l.vh = dd->v3h * l.lt;
        l.vs = (l.vh + 63) / 64 * 64;
        l.hop3[3] = 3 % l.lt;
        handle_begin(h);
        const size_t lb = (size_t)2 * 4 * 9 * l.vs * sizeof(double2);
        const size_t fb = (size_t)3 * depth * dd->v3h * sizeof(double2);
        for (int q = 0; q < n_ranks; ++q) {
            dd->fat.push_back(dalloc<double2>(dd, lb));
            copy_links(dd, h->fat64, dd->fat[q], q);
            dd->lng.push_back(h->lng64 ? dalloc<double2>(dd, lb) : nullptr);
            if (h->lng64) copy_links(dd, h->lng64, dd->lng[q], q);
            for (auto* vec : {&dd->vin, &dd->vt, &dd->vout, &dd->x, &dd->r, &dd->d, &dd->b})
                vec->push_back(dalloc<double2>(dd, vecb(dd)));
            for (auto* vec : {&dd->s_lo, &dd->s_hi, &dd->r_lo, &dd->r_hi}) vec->push_back(dalloc<double2>(dd, fb));
            for (auto* vec : {&dd->hs_lo, &dd->hs_hi, &dd->hr_lo, &dd->hr_hi})
                vec->push_back(dalloc<double2>(dd, fb, true));
        }
        dd->partials = dalloc<double>(dd, sizeof(double) * (size_t)n_ranks * blocks_for(dd->ltl * dd->v3h));
        dcheck(dd, cudaEventCreate(&dd->ev[0]), "event");
        dcheck(dd, cudaEventCreate(&dd->ev[1]), "event");
        dcheck(dd, cudaStreamCreateWithFlags(&dd->cs, cudaStreamNonBlocking), "stream");
        for (auto& e : dd->eo) dcheck(dd, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        dcheck(dd, cudaStreamSynchronize(S(dd)), "create");
        *out = dd;
        return STAG_OK;
    } catch (const DFail& f) {
        h->err = dd->err;
        destroy_dd(dd);
        return f.code;
    } catch (const HandleError& f) {
        destroy_dd(dd);
        return f.code;
    }
}

int stag_dd_apply_A(stag_dd* dd, const double* in_even, double* out_even, int32_t mode, double* phase_ms) {
    if (!dd || !in_even || !out_even || in_even == out_even) return STAG_ERR_INVALID_ARG;
    if (mode < STAG_DD_HOST || mode > STAG_DD_DEVICE_OVERLAP) return STAG_ERR_INVALID_ARG;
    stag_handle* h = dd->h;
    try {
        handle_begin(h);
        const Geom& g = h->g;
        const size_t ab = (size_t)3 * g.vh * sizeof(double2);
        std::memset(dd->phase, 0, sizeof(dd->phase));
        const double* src = in_even;
        if (!handle_is_device_ptr(h, src)) {
            dcheck(dd, cudaMemcpyAsync(h->io_a, src, ab, cudaMemcpyHostToDevice, S(dd)), "copy in");
            src = h->io_a;
        }
        launch_pack_vec(g, src, h->x, S(dd));
        scatter(dd, h->x, dd->vin);
        dd_apply(dd, dd->vin, dd->vout, mode);
        gather(dd, dd->vout, h->ad);
        const bool dev = handle_is_device_ptr(h, out_even);
        launch_unpack_vec(g, h->ad, dev ? out_even : h->io_b, S(dd));
        if (!dev) dcheck(dd, cudaMemcpyAsync(out_even, h->io_b, ab, cudaMemcpyDeviceToHost, S(dd)), "copy out");
        dcheck(dd, cudaGetLastError(), "apply");
        handle_end(h);
        report(dd, phase_ms);
        return STAG_OK;
    } catch (const DFail& f) {
        h->err = dd->err;
        return f.code;
    } catch (const HandleError& f) {
        return f.code;
    }
}

int stag_dd_cg_solve(stag_dd* dd, const double* b_even, double* x_even, double tol, int32_t max_iter, int32_t mode,
                     stag_solve_info* info, double* phase_ms) {
    if (!dd || !b_even || !x_even || b_even == x_even || !(tol > 0.0)) return STAG_ERR_INVALID_ARG;
    if (mode < STAG_DD_HOST || mode > STAG_DD_DEVICE_OVERLAP) return STAG_ERR_INVALID_ARG;
    stag_handle* h = dd->h;
    stag_solve_info inf{};
    int status = STAG_OK;
    const auto t0 = std::chrono::steady_clock::now();
    try {
        handle_begin(h);
        const Geom& g = h->g;
        const size_t ab = (size_t)3 * g.vh * sizeof(double2);
        std::memset(dd->phase, 0, sizeof(dd->phase));
        for (int k = 0; k < 2; ++k) {
            const double* src = k == 0 ? b_even : x_even;
            double* stage = k == 0 ? h->io_a : h->io_b;
            if (!handle_is_device_ptr(h, src)) {
                dcheck(dd, cudaMemcpyAsync(stage, src, ab, cudaMemcpyHostToDevice, S(dd)), "copy in");
                src = stage;
            }
            launch_pack_vec(g, src, k == 0 ? h->b : h->x, S(dd));
        }
        scatter(dd, h->b, dd->b);
        scatter(dd, h->x, dd->x);
        // Fig. 1: r = b - A x, d = r, delta = r^dag r
        const double bnorm2 = dd_dot(dd, dd->b, dd->b);
        const long long max_it = max_iter > 0 ? max_iter : 3LL * g.vh;
        long long it = 0;
        double rel = 0.0;
        if (bnorm2 > 0.0) {
            dd_apply(dd, dd->x, dd->vout, mode);
            for (int q = 0; q < dd->P; ++q)
                cudaMemcpyAsync(dd->r[q], dd->b[q], vecb(dd), cudaMemcpyDeviceToDevice, S(dd));
            dd_axpy(dd, -1.0, dd->vout, dd->r, 0);
            for (int q = 0; q < dd->P; ++q)
                cudaMemcpyAsync(dd->d[q], dd->r[q], vecb(dd), cudaMemcpyDeviceToDevice, S(dd));
            double delta = dd_dot(dd, dd->r, dd->r);
            const double thr = tol * tol * bnorm2;
            while (it < max_it && delta > thr) {
                dd_apply(dd, dd->d, dd->vout, mode);
                const double pap = dd_dot(dd, dd->d, dd->vout);
                if (!(pap > 0.0)) {
                    status = STAG_ERR_BREAKDOWN;
                    break;
                }
                const double alpha = delta / pap;
                dd_axpy(dd, alpha, dd->d, dd->x, 0);
                dd_axpy(dd, -alpha, dd->vout, dd->r, 0);
                const double dnew = dd_dot(dd, dd->r, dd->r);
                const double beta = dnew / delta;
                delta = dnew;
                dd_axpy(dd, beta, dd->r, dd->d, 1);  // d = r + beta d
                ++it;
            }
            // true residual with the decomposed operator
            dd_apply(dd, dd->x, dd->vout, mode);
            for (int q = 0; q < dd->P; ++q)
                cudaMemcpyAsync(dd->r[q], dd->b[q], vecb(dd), cudaMemcpyDeviceToDevice, S(dd));
            dd_axpy(dd, -1.0, dd->vout, dd->r, 0);
            rel = std::sqrt(dd_dot(dd, dd->r, dd->r) / bnorm2);
            if (status == STAG_OK && rel > tol) status = STAG_ERR_NOT_CONVERGED;
            inf.iter_rel_residual = std::sqrt(delta / bnorm2);
        }
        gather(dd, dd->x, h->x);
        const bool dev = handle_is_device_ptr(h, x_even);
        launch_unpack_vec(g, h->x, dev ? x_even : h->io_b, S(dd));
        if (!dev) dcheck(dd, cudaMemcpyAsync(x_even, h->io_b, ab, cudaMemcpyDeviceToHost, S(dd)), "copy x");
        dcheck(dd, cudaGetLastError(), "decomposed CG");
        handle_end(h);
        inf.iters = (int32_t)it;
        inf.true_rel_residual = rel;
        report(dd, phase_ms);
    } catch (const DFail& f) {
        h->err = dd->err;
        status = f.code;
    } catch (const HandleError& f) {
        status = f.code;
    }
    inf.status = status;
    inf.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return status;
}

int64_t stag_dd_bytes_exchanged(const stag_dd* dd) { return dd ? dd->bytes_exchanged : 0; }

int stag_dd_destroy(stag_dd* dd) {
    destroy_dd(dd);
    return STAG_OK;
}

}  // extern "C"
