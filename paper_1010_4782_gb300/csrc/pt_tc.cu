// pt_tc.cu - the 8 -> 8 layer of the parallel-transport network with its
// channel mixing on the tensor cores (tcgen05, sm_100 and later).
//
// The layer is psi'(x, o) = sum_p sum_i W[p][o][i] (T_p psi_i)(x) (paths and
// transports as in pt_common.cuh).  For a tile of 128 sites of one parity and
// each colour c it is the real matrix product
//     D_c[s][n] = sum_k A_c[s][k] B[n][k],   s < 128, n < 16, k < 144,
// with A_c[s][16 p + 2 i + h] the real (h = 0) or imaginary (h = 1) part of
// (T_p psi_i)(s)_c rounded to BF16, and B the real form of the complex weights
// (y = w x:  y_re = w_re x_re - w_im x_im,  y_im = w_im x_re + w_re x_im):
//     B[2o][16p+2i] = w_re,  B[2o][16p+2i+1] = -w_im,
//     B[2o+1][16p+2i] = w_im,  B[2o+1][16p+2i+1] = w_re,   w = W[p][o][i];
// D_c[s][2o + h] is then the real / imaginary part of psi'(s, o)_c.
//
// One thread per site.  K runs in nine phases, one per path: each thread
// transports its site's 8 channels along the path (FP32 links, FP32
// arithmetic) and writes them to one of two A buffers in shared memory; one
// thread issues the 3 colours' MMAs (M = 128, N = 16, K = 16, BF16 operands,
// FP32 accumulators in TMEM columns 16 c .. 16 c + 15) and commits them to the
// buffer's mbarrier.  The transport of the next path overlaps these MMAs; a
// buffer is rewritten only after the MMAs that read it have completed.  At the
// end each warp reads its 32 rows back with tcgen05.ld and stores them.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8 rows x 16 bytes core matrices; the leading byte offset (LBO) steps to the
// next core matrix along K, the stride byte offset (SBO) to the next group of
// 8 rows.  Waits are bounded; a wait that runs out sets *err, and the kernel
// issues no further MMAs.  It then still waits - in order on each barrier, with
// a longer limit - for every commit it has issued, so that TMEM is neither read
// nor freed under an MMA that may still be writing it, before it deallocates.
#include <cuda_bf16.h>

#include <cstdint>

#include "pt_common.cuh"

namespace stag {

namespace {

constexpr int kTileRows = 128;                    // sites per CTA (= MMA M)
constexpr int kAKGroups = 2;                      // one path = 16 K elements = 2 core matrices
constexpr int kASbo = kAKGroups * 128;            // 256 B between 8-row groups
constexpr int kAColour = (kTileRows / 8) * kASbo; // 4096 B per colour
constexpr int kABuf = 3 * kAColour;               // 12288 B per buffer
constexpr int kABytes = 2 * kABuf;                // two buffers
constexpr int kBKGroups = kPaths * 16 / 8;        // 18
constexpr int kBSbo = kBKGroups * 128;            // 2304 B
constexpr int kBBytes = 2 * kBSbo;                // 4608 B (N = 16: two 8-row groups)
constexpr int kTmemCols = 64;                     // 48 used: 3 colours x N = 16
constexpr long long kWaitLimit = 1LL << 22;   // try_wait polls before giving up
constexpr long long kDrainLimit = 1LL << 26;  // polls per outstanding commit after a give-up

// smem layout: [A 2 x 12288][B 4608][2 mbarriers 16][tmem address 4]
constexpr int kSmemBytes = kABytes + kBBytes + 32;

// tcgen05 instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((uint32_t)(kTileRows >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, LBO and SBO in
// 16-byte units (bits 0-13, 16-29, 32-45), descriptor version 1 (bits 46-47),
// base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// PHI (inference): instead of psi, store phi_p = sum_i W3[p][0][i] psi_i, the
// next layer's channel mixing done before its transports (T_p acts on colour,
// W3 on channels, so sum_i W3[p][0][i] T_p psi_i = T_p phi_p): on odd sites the
// 8 transported paths (channel p - 1), on even sites the identity path
// (channel 0).  w3: the next layer's weights [9][1][8].
template <class TI, class TO, bool PHI>
__global__ void __launch_bounds__(kTileRows) pt_mix8_tc_kernel(Geom g, const float2* __restrict__ links,
                                                              const float2* __restrict__ w,
                                                              const TI* __restrict__ in, TO* __restrict__ out,
                                                              const float2* __restrict__ w3, int* err,
                                                              const int* __restrict__ skip) {
    if (skip && *skip) return;  // the same value in every thread: the whole CTA leaves before any set-up
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ float2 sW3[kPaths * kHidden];  // PHI: the next layer's weights
    if constexpr (PHI) {
        for (int k = threadIdx.x; k < kPaths * kHidden; k += blockDim.x) sW3[k] = w3[k];
    }
    uint8_t* sA = smem;
    uint8_t* sB = smem + kABytes;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kABytes + kBBytes);  // one per A buffer
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kABytes + kBBytes + 16);
    const int tid = threadIdx.x, warp = tid >> 5;

    // TMEM columns for the accumulators (one warp allocates), the mbarrier,
    // and B from the complex weights W[p][o][i].
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < 16 * kPaths * 16; e += kTileRows) {
        const int n = e / (kPaths * 16), k = e % (kPaths * 16);
        const int o = n >> 1, ho = n & 1, p = k >> 4, i = (k & 15) >> 1, hi = k & 1;
        const float2 wv = w[(p * kHidden + o) * kHidden + i];
        const float v = ho == hi ? wv.x : (ho == 0 ? -wv.y : wv.y);
        *reinterpret_cast<__nv_bfloat16*>(sB + (n >> 3) * kBSbo + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) =
            __float2bfloat16_rn(v);
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int P = (int)(blockIdx.x & 1);
    const int i = (int)(blockIdx.x >> 1) * kTileRows + tid;
    const bool active = i < g.vh;
    const size_t vs = (size_t)g.vs;
    int x = 0, y = 0, z = 0, t = 0;
    if (active) site_coords(i, P, g, x, y, z, t);
    uint8_t* rowA = sA + (tid >> 3) * kASbo + (tid & 7) * 16;
    const uint32_t aBase = smem_u32(sA), bBase = smem_u32(sB);
    const uint32_t bar0 = smem_u32(bar), bar1 = smem_u32(bar + 1);
    bool ok = true;
    // Per buffer barrier: commits issued and completions seen so far (the same
    // in every thread).  A parity wait only tells the phase it names from the
    // one before it, so completions are always waited for in order.
    // (Scalars, not arrays indexed by b, so that they stay in registers.)
    int issued0 = 0, issued1 = 0, seen0 = 0, seen1 = 0;

    // waits for buffer b's next completion not yet seen; false after `limit` polls
    auto wait_next = [&](int b, long long limit) {
        int& seen = b ? seen1 : seen0;
        long long spins = 0;
        while (!mbar_try_wait(b ? bar1 : bar0, (uint32_t)(seen & 1)))
            if (++spins > limit) return false;
        ++seen;
        return true;
    };

    for (int p = 0; p < kPaths; ++p) {
        const int b = p & 1;
        if (p >= 2 && ok) {
            // the MMAs of path p - 2 read this buffer
            if (!wait_next(b, kWaitLimit)) {
                ok = false;
                atomicExch(err, 1);
            }
            fence_after_sync();
        }
        if (active) {
            int Pn = P, nb = i, d = 0;
            float2 U[9];
            if (p > 0) {
                const int mu = (p - 1) >> 1;
                d = (p - 1) & 1;
                const Hop hp = pt_hop(g, links, P, i, x, y, z, t, mu, d);
                Pn = hp.Pn;
                nb = hp.nb;
#pragma unroll
                for (int k = 0; k < 9; ++k) U[k] = __ldg(hp.u + k * vs);
            }
            uint8_t* row = rowA + b * kABuf;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t word[3][4];
                float2 vin[3][4];  // channels 4 h .. 4 h + 3, one 16-byte load per colour
#pragma unroll
                for (int c = 0; c < 3; ++c) ld4c(in + fidx(4 * h, c, Pn, nb, vs, kHidden), vin[c]);
#pragma unroll
                for (int ii = 0; ii < 4; ++ii) {
                    float2 v[3], tv[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) v[c] = vin[c][ii];
                    if (p > 0) {
                        pt_apply(U, d, v, tv);
                    } else {
#pragma unroll
                        for (int c = 0; c < 3; ++c) tv[c] = v[c];
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) word[c][ii] = pack_bf16x2(tv[c].x, tv[c].y);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    *reinterpret_cast<uint4*>(row + c * kAColour + h * 128) =
                        make_uint4(word[c][0], word[c][1], word[c][2], word[c][3]);
            }
        }
        fence_async_smem();
        fence_before_sync();
        ok = __syncthreads_and(ok ? 1 : 0) != 0;
        fence_after_sync();
        if (ok) {
            if (tid == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const uint64_t da = smem_desc(aBase + b * kABuf + c * kAColour, 128, kASbo);
                    const uint64_t db = smem_desc(bBase + p * kAKGroups * 128, 128, kBSbo);
                    mma_bf16(tmem + 16 * c, da, db, p > 0 ? 1u : 0u);
                }
                mma_commit(b ? bar1 : bar0);
            }
            if (b)
                ++issued1;
            else
                ++issued0;
        }
    }
    // Every issued commit must have arrived before TMEM is read or freed.
    // Normally only the last two paths' are outstanding.  After a wait that
    // ran out (here or above) the remaining ones are waited for with the
    // longer limit; if one of those runs out too, the kernel can no longer
    // tell when the MMAs end and deallocates anyway - its output is discarded
    // through *err.
#pragma unroll 1
    for (int b = 0; b < 2; ++b) {
        while ((b ? seen1 : seen0) < (b ? issued1 : issued0)) {
            if (wait_next(b, ok ? kWaitLimit : kDrainLimit)) continue;
            if (ok) {
                ok = false;
                atomicExch(err, 1);
                continue;
            }
            break;
        }
    }
    fence_after_sync();
    ok = __syncthreads_and(ok ? 1 : 0) != 0;

    // accumulators -> registers (warp w holds rows 32 w .. 32 w + 31) -> output
    // one colour at a time: 16 accumulators live (warp-collective loads, uniform loop)
#pragma unroll 1
    for (int c = 0; c < 3 && ok; ++c) {  // ok is the same in every thread here
        float dv[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16 * c, dv);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!active) continue;
        if constexpr (!PHI) {
#pragma unroll
            for (int o = 0; o < kHidden; o += 4)
                st4c(out + fidx(o, c, P, i, vs, kHidden), make_float2(dv[2 * o], dv[2 * o + 1]),
                     make_float2(dv[2 * o + 2], dv[2 * o + 3]), make_float2(dv[2 * o + 4], dv[2 * o + 5]),
                     make_float2(dv[2 * o + 6], dv[2 * o + 7]));
        } else if (P == 1) {
            float2 ph[kHidden];
#pragma unroll
            for (int q = 0; q < kHidden; ++q) {
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int o = 0; o < kHidden; ++o) {
                    const float2 m = cmulf(sW3[(q + 1) * kHidden + o], make_float2(dv[2 * o], dv[2 * o + 1]));
                    a.x += m.x;
                    a.y += m.y;
                }
                ph[q] = a;
            }
            st4c(out + fidx(0, c, P, i, vs, kHidden), ph[0], ph[1], ph[2], ph[3]);
            st4c(out + fidx(4, c, P, i, vs, kHidden), ph[4], ph[5], ph[6], ph[7]);
        } else {
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int o = 0; o < kHidden; ++o) {
                const float2 m = cmulf(sW3[o], make_float2(dv[2 * o], dv[2 * o + 1]));
                a.x += m.x;
                a.y += m.y;
            }
            stc(out + fidx(0, c, P, i, vs, kHidden), a);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

void launch_pt_mix8_tc(const Geom& g, const float2* links, const float2* w, const __nv_bfloat162* in,
                       __nv_bfloat162* out, const float2* w3, int* err, cudaStream_t s, const int* skip) {
    const int tiles = (g.vh + kTileRows - 1) / kTileRows;
    if (w3)
        pt_mix8_tc_kernel<__nv_bfloat162, __nv_bfloat162, true>
            <<<2 * tiles, kTileRows, kSmemBytes, s>>>(g, links, w, in, out, w3, err, skip);
    else
        pt_mix8_tc_kernel<__nv_bfloat162, __nv_bfloat162, false>
            <<<2 * tiles, kTileRows, kSmemBytes, s>>>(g, links, w, in, out, nullptr, err, skip);
}

// out(x) = phi_0(x) + sum_{p = 1..8} (T_p phi_p)(x) on even sites x, from the
// PHI output of pt_mix8_tc_kernel (the network's last layer, 8 -> 1).
__global__ void __launch_bounds__(256) pt_transport_sum_kernel(Geom g, const float2* __restrict__ links,
                                                               const __nv_bfloat162* __restrict__ phi,
                                                               __nv_bfloat162* __restrict__ out,
                                                               const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
    int x, y, z, t;
    site_coords(i, 0, g, x, y, z, t);
    float2 acc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = ldc(phi + fidx(0, c, 0, i, vs, kHidden));
#pragma unroll 1
    for (int p = 1; p < kPaths; ++p) {
        const int mu = (p - 1) >> 1, d = (p - 1) & 1;
        const Hop hp = pt_hop(g, links, 0, i, x, y, z, t, mu, d);
        float2 U[9], v[3], tv[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) U[k] = __ldg(hp.u + k * vs);
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = ldc(phi + fidx(p - 1, c, hp.Pn, hp.nb, vs, kHidden));
        pt_apply(U, d, v, tv);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            acc[c].x += tv[c].x;
            acc[c].y += tv[c].y;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) stc(out + fidx(0, c, 0, i, vs, 1), acc[c]);
}

void launch_pt_transport_sum(const Geom& g, const float2* links, const __nv_bfloat162* phi, __nv_bfloat162* out,
                             cudaStream_t s, const int* skip) {
    pt_transport_sum_kernel<<<(g.vh + 255) / 256, 256, 0, s>>>(g, links, phi, out, skip);
}

}  // namespace stag
