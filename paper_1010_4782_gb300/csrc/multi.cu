// multi.cu - kernels of the batched solver: many CG systems advanced by one
// launch per step.
//
// A batch holds groups; a group is one lattice (one gauge field, one mass) with
// R right-hand sides.  Each group's FP32 vectors are stored right-hand-side
// innermost, v[(colour * vs + site) * Rpad + rhs] as float2, so one thread can
// apply each link it loads to a block of RB right-hand sides (the link is read
// once for all of them - the multi-RHS form of Sec. 2's Dirac operation).
// Work items (group, block of the group, blocks of the group) are listed in a
// device table; blockIdx.x selects one, so a single launch covers lattices of
// any size mix.  A group's blocks take contiguous runs of site tiles.
//
// Per right-hand side the CG scalars (alpha, beta, delta, loop state) live in
// their own CgScalars; reductions are per right-hand side: per-block partials,
// and the last block of each group sums them in block order.
#include <cuda_fp16.h>

#include "ff.cuh"
#include "multi.cuh"

namespace stag {

__device__ __forceinline__ bool group_all_done(const MultiGroup& G, const CgScalars* scal) {
    for (int r = 0; r < G.nrhs; ++r)
        if (!scal[G.rhs0 + r].done) return false;
    return true;
}

// Two traversals of a group's site tiles by its nblk blocks (the work item's
// fourth field selects one):
//  * runs (0): block blk takes the contiguous tiles [tile_end(blk - 1),
//    tile_end(blk)), so that a block's consecutive tiles share their
//    neighbours' vectors in L2;
//  * sweep (1): nblk is the number of blocks that are resident at once, and
//    block blk takes the tiles blk, blk + nblk, blk + 2 nblk, ...  All blocks
//    then work on one narrow band of sites that moves through the lattice, so
//    the input vector's reuse window (t -/+ 3 slices) stays in L2.
__device__ __forceinline__ int tile_end(int blk, int ntiles, int nblk) {
    return (int)((long long)(blk + 1) * ntiles / nblk);
}

struct TileWalk {
    int first, end, step;
};

__device__ __forceinline__ TileWalk tile_walk(int4 w, int ntiles) {
    if (w.w) return TileWalk{w.y, ntiles, w.z};
    return TileWalk{tile_end(w.y - 1, ntiles, w.z), tile_end(w.y, ntiles, w.z), 1};
}

// Thread layout: right-hand sides are the fastest index.  TPS = rpad / RB
// threads share a site (lane % TPS selects RB consecutive right-hand sides), so
// the TPS lanes of a site issue identical link addresses - one transaction per
// warp - and read the site's vectors as one contiguous run.  A block holds
// SPB = BS / TPS sites and walks the group's site tiles with a stride of the
// number of blocks the group was given.
struct Lanes {
    int tps, spb, site_local, rlane, roff;
};

template <int RB, int BS>
__device__ __forceinline__ Lanes lanes_of(const MultiGroup& G) {
    Lanes l;
    l.tps = G.rpad / RB;
    l.spb = BS / l.tps;
    l.site_local = threadIdx.x / l.tps;
    l.rlane = threadIdx.x % l.tps;
    l.roff = l.rlane * RB;
    return l;
}

// Per-RHS block sums of v[RB] (lanes with equal rlane share right-hand sides):
// the sums for right-hand side roff + j end up in sm[roff + j] (all threads after return).
template <int RB, int BS>
__device__ __forceinline__ void block_sums_rhs(double (&v)[RB], const Lanes& l, double* sw /* [BS/32][32*RB] */,
                                               double* sm /* [32*RB] */, int rpad) {
    // over the sites inside the warp: lanes l, l+TPS, ... hold the same right-hand sides
#pragma unroll
    for (int j = 0; j < RB; ++j)
        for (int o = l.tps; o < 32; o <<= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane < l.tps) {
#pragma unroll
        for (int j = 0; j < RB; ++j) sw[w * (32 * RB) + l.roff + j] = v[j];
    }
    __syncthreads();
    // over the warps, in warp order
    for (int r = threadIdx.x; r < rpad; r += BS) {
        double s = 0.0;
        for (int k = 0; k < BS / 32; ++k) s += sw[k * (32 * RB) + r];
        sm[r] = s;
    }
    __syncthreads();
}

// Writes the block's per-RHS sums; in the last block of the group returns true
// with the grid sums (over the group's blocks, in block order) in tot[0..rpad).
template <int RB, int BS>
__device__ __forceinline__ bool multi_reduce(double (&v)[RB], const MultiGroup& G, const Lanes& l, int blk,
                                             int nblk, double* partials, unsigned int* counters, double* tot) {
    __shared__ double sw[(BS / 32) * 32 * RB];
    __shared__ double sm[32 * RB];
    __shared__ bool is_last;
    block_sums_rhs<RB, BS>(v, l, sw, sm, G.rpad);
    for (int r = threadIdx.x; r < G.rpad; r += BS) partials[(size_t)(G.prhs0 + r) * G.max_blocks + blk] = sm[r];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int ticket = atomicAdd(&counters[G.prhs0], 1u);
        is_last = (ticket == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    // one warp per right-hand side, fixed order inside each lane, fixed shuffle tree
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int r = w; r < G.rpad; r += BS / 32) {
        const double* p = partials + (size_t)(G.prhs0 + r) * G.max_blocks;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int b = lane;
        for (; b + 96 < nblk; b += 128) {
            s0 += __ldcg(p + b);
            s1 += __ldcg(p + b + 32);
            s2 += __ldcg(p + b + 64);
            s3 += __ldcg(p + b + 96);
        }
        for (; b < nblk; b += 32) s0 += __ldcg(p + b);
        double s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) tot[r] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) counters[G.prhs0] = 0u;
    return true;
}

__device__ __forceinline__ int nbr_index(const Geom& g, int x, int y, int z, int t, int mu, int h, bool up) {
    switch (mu) {
        case 0: x = up ? wrap_up(x, h, g.lx) : wrap_dn(x, h, g.lx); break;
        case 1: y = up ? wrap_up(y, h, g.ly) : wrap_dn(y, h, g.ly); break;
        case 2: z = up ? wrap_up(z, h, g.lz) : wrap_dn(z, h, g.lz); break;
        default: t = up ? wrap_up(t, h, g.lt) : wrap_dn(t, h, g.lt); break;
    }
    return site_index(x, y, z, t, g);
}

// 256-bit accesses (sm_100 and later) of four consecutive float2; p is 32-byte aligned.
__device__ __forceinline__ void ld256_nc(const float2* p, float2& a, float2& b, float2& c, float2& d) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(b.x), "=f"(b.y), "=f"(c.x), "=f"(c.y), "=f"(d.x), "=f"(d.y)
        : "l"(p));
}
__device__ __forceinline__ void ld256(const float2* p, float2& a, float2& b, float2& c, float2& d) {
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(b.x), "=f"(b.y), "=f"(c.x), "=f"(c.y), "=f"(d.x), "=f"(d.y)
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void st256(float2* p, float2 a, float2 b, float2 c, float2 d) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.x), "f"(a.y),
                 "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y), "f"(d.x), "f"(d.y)
                 : "memory");
}

// A thread's RB consecutive right-hand sides of one colour.  For RB >= 4 the
// offset is a multiple of 32 bytes (rpad >= 8 is a power of two and the lane
// offset is a multiple of RB), so the accesses are 256 bits wide.
template <int RB>
__device__ __forceinline__ void load_rb(float2 (&v)[RB], const float2* __restrict__ p) {
    if constexpr (RB == 1) {
        v[0] = __ldg(p);
    } else if constexpr (RB % 4 == 0) {
#pragma unroll
        for (int j = 0; j < RB; j += 4) ld256_nc(p + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < RB; j += 2) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(p + j));
            v[j] = make_float2(q.x, q.y);
            v[j + 1] = make_float2(q.z, q.w);
        }
    }
}

template <int RB>
__device__ __forceinline__ void load_rb_rw(float2 (&v)[RB], const float2* p) {
    if constexpr (RB == 1) {
        v[0] = *p;
    } else if constexpr (RB % 4 == 0) {
#pragma unroll
        for (int j = 0; j < RB; j += 4) ld256(p + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < RB; j += 2) {
            const float4 q = *reinterpret_cast<const float4*>(p + j);
            v[j] = make_float2(q.x, q.y);
            v[j + 1] = make_float2(q.z, q.w);
        }
    }
}

template <int RB>
__device__ __forceinline__ void store_rb(float2* p, const float2 (&v)[RB]) {
    if constexpr (RB == 1) {
        *p = v[0];
    } else if constexpr (RB % 4 == 0) {
#pragma unroll
        for (int j = 0; j < RB; j += 4) st256(p + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < RB; j += 2)
            *reinterpret_cast<float4*>(p + j) = make_float4(v[j].x, v[j].y, v[j + 1].x, v[j + 1].y);
    }
}

// acc[r][j] += U v (fwd, U at the output site) or -= U^dag v (bwd, U at the neighbour)
template <int RB, bool BWD>
__device__ __forceinline__ void multi_hop(float2 (&acc)[3][RB], const float2* __restrict__ u,
                                          const float2* __restrict__ in, int nb, size_t vs, int rpad, int roff,
                                          bool stream_links = false) {
    float2 U[9];
    // the links are read once: with stream_links they are loaded as streaming
    // (evict-first) data, so that they do not push the reused input vectors out of L2
#pragma unroll
    for (int k = 0; k < 9; ++k) U[k] = stream_links ? __ldcs(u + k * vs) : __ldg(u + k * vs);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 v[RB];
        load_rb<RB>(v, in + ((size_t)c * vs + nb) * rpad + roff);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int j = 0; j < RB; ++j) {
                if (BWD)
                    cmscf_conj(acc[r][j], U[3 * c + r], v[j]);
                else
                    cmacf(acc[r][j], U[3 * r + c], v[j]);
            }
        }
    }
}

// out = D in (EPI_PLAIN), m2 src - D in (EPI_AXPY), or the latter with per-RHS
// Re(src^dag out) -> alpha (EPI_CG).
// With eight right-hand sides per thread the compiler would use about 140
// registers, which leaves 12 warps per SM; the bound of 128 (16 warps per SM,
// spilling under 160 bytes a thread to L1) made both half-Dslash launches
// about 6 % faster on GB300 at 32^3 x 64 with 16 right-hand sides.  96
// registers (20 warps) spilled more and was slower.
template <int RB, int BS, int EPI, int MODE>
__global__ void __launch_bounds__(BS, (RB == 8 ? 512 / BS : 1)) multi_dslash_kernel(const MultiLaunch L) {
    const int4 w = L.items[blockIdx.x];  // (group, block in group, blocks in group, -)
    const MultiGroup& G = L.groups[w.x];
    if (group_all_done(G, L.scal)) return;
    const int blk = w.y, nblk = w.z;
    const Geom& g = G.g;
    const Lanes l = lanes_of<RB, BS>(G);
    const int P = L.out_parity, Q = 1 - L.out_parity;
    const size_t vs = (size_t)g.vs;
    const float2* in = L.phase == 0 ? G.d : G.t;  // phase 0: t = D d; phase 1: Ad = m2 d - D t
    float2* out = L.phase == 0 ? G.t : G.ad;
    const float m2 = (float)G.m2;
    const int ntiles = (g.vh + l.spb - 1) / l.spb;
    float dotf[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) dotf[j] = 0.f;
    constexpr bool kSweep = MODE != 0;
    const int tile0 = kSweep ? blk : tile_end(blk - 1, ntiles, nblk);
    const int tile1 = kSweep ? ntiles : tile_end(blk, ntiles, nblk);
    const int step = kSweep ? nblk : 1;
    for (int tile = tile0; tile < tile1; tile += step) {
        const int i = tile * l.spb + l.site_local;
        if (i >= g.vh) continue;
        float2 acc[3][RB];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < RB; ++j) acc[r][j] = make_float2(0.f, 0.f);
        int x, y, z, t;
        site_coords(i, P, g, x, y, z, t);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const int f1 = nbr_index(g, x, y, z, t, mu, 1, true);
            const int b1 = nbr_index(g, x, y, z, t, mu, 1, false);
            multi_hop<RB, false>(acc, G.fat + ((size_t)(P * 4 + mu) * 9) * vs + i, in, f1, vs, G.rpad, l.roff,
                                 kSweep);
            multi_hop<RB, true>(acc, G.fat + ((size_t)(Q * 4 + mu) * 9) * vs + b1, in, b1, vs, G.rpad, l.roff,
                                kSweep);
            if (G.lng) {
                const int h = g.hop3[mu];
                const int f3 = nbr_index(g, x, y, z, t, mu, h, true);
                const int b3 = nbr_index(g, x, y, z, t, mu, h, false);
                multi_hop<RB, false>(acc, G.lng + ((size_t)(P * 4 + mu) * 9) * vs + i, in, f3, vs, G.rpad,
                                     l.roff, kSweep);
                multi_hop<RB, true>(acc, G.lng + ((size_t)(Q * 4 + mu) * 9) * vs + b3, in, b3, vs, G.rpad,
                                    l.roff, kSweep);
            }
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            float2* o = out + ((size_t)r * vs + i) * G.rpad + l.roff;
            if constexpr (EPI == EPI_PLAIN) {
                store_rb<RB>(o, acc[r]);
            } else {
                float2 sv[RB], ov[RB];
                load_rb<RB>(sv, G.d + ((size_t)r * vs + i) * G.rpad + l.roff);
#pragma unroll
                for (int j = 0; j < RB; ++j) {
                    ov[j] = make_float2(fmaf(m2, sv[j].x, -acc[r][j].x), fmaf(m2, sv[j].y, -acc[r][j].y));
                    dotf[j] = fmaf(sv[j].x, ov[j].x, dotf[j]);
                    dotf[j] = fmaf(sv[j].y, ov[j].y, dotf[j]);
                }
                store_rb<RB>(o, ov);
            }
        }
    }
    if constexpr (EPI == EPI_CG) {
        __shared__ double tot[32 * RB];
        double dot[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j) dot[j] = (double)dotf[j];
        if (multi_reduce<RB, BS>(dot, G, l, blk, nblk, L.partials, L.counters, tot)) {
            for (int r = threadIdx.x; r < G.nrhs; r += BS) {
                CgScalars* sc = L.scal + G.rhs0 + r;
                if (sc->done) continue;
                sc->pAp = tot[r];
                const double alpha = sc->delta_new / tot[r];
                if (!(tot[r] > 0.0) || !isfinite(alpha)) {
                    sc->status = 4;
                    sc->done = 1;
                    sc->alpha_ff = make_float2(0.f, 0.f);
                } else {
                    sc->alpha = alpha;
                    sc->alpha_ff = ff_from_double(alpha);
                }
            }
        }
    }
}

// y += alpha d; r -= alpha Ad; per-RHS |r|^2 and the reliable-update decision
template <int RB, int BS>
__global__ void __launch_bounds__(BS) multi_update_xr_kernel(const MultiLaunch L) {
    const int4 w = L.items[blockIdx.x];
    const MultiGroup& G = L.groups[w.x];
    if (group_all_done(G, L.scal)) return;
    const int blk = w.y, nblk = w.z;
    const Geom& g = G.g;
    const Lanes l = lanes_of<RB, BS>(G);
    const size_t vs = (size_t)g.vs;
    float alpha[RB];
    bool live[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
        const int r = l.roff + j;
        live[j] = r < G.nrhs && !L.scal[G.rhs0 + r].done;
        alpha[j] = live[j] ? L.scal[G.rhs0 + r].alpha_ff.x : 0.f;
    }
    const int ntiles = (g.vh + l.spb - 1) / l.spb;
    float acc[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) acc[j] = 0.f;
    const TileWalk tw = tile_walk(w, ntiles);
    for (int tile = tw.first; tile < tw.end; tile += tw.step) {
        const int i = tile * l.spb + l.site_local;
        if (i >= g.vh) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = ((size_t)c * vs + i) * G.rpad + l.roff;
            float2 d[RB], a[RB], r[RB], y[RB];
            load_rb<RB>(d, G.d + k);
            load_rb<RB>(a, G.ad + k);
            load_rb_rw<RB>(r, G.r + k);
            load_rb_rw<RB>(y, G.y + k);
#pragma unroll
            for (int j = 0; j < RB; ++j) {
                y[j].x = fmaf(alpha[j], d[j].x, y[j].x);
                y[j].y = fmaf(alpha[j], d[j].y, y[j].y);
                r[j].x = fmaf(-alpha[j], a[j].x, r[j].x);
                r[j].y = fmaf(-alpha[j], a[j].y, r[j].y);
                acc[j] = fmaf(r[j].x, r[j].x, acc[j]);
                acc[j] = fmaf(r[j].y, r[j].y, acc[j]);
            }
            store_rb<RB>(G.y + k, y);
            store_rb<RB>(G.r + k, r);
        }
    }
    __shared__ double tot[32 * RB];
    double n2[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) n2[j] = (double)acc[j];
    if (multi_reduce<RB, BS>(n2, G, l, blk, nblk, L.partials, L.counters, tot)) {
        for (int r = threadIdx.x; r < G.nrhs; r += BS) {
            CgScalars* sc = L.scal + G.rhs0 + r;
            if (sc->done) continue;
            const double total = tot[r];
            sc->delta_old = sc->delta_new;
            sc->delta_new = total;
            sc->beta = total / sc->delta_old;
            sc->beta_ff = ff_from_double(sc->beta);
            sc->iter += 1;
            sc->iter_since += 1;
            const double rn = sqrt(total);
            if (!isfinite(total)) {
                sc->status = 4;
                sc->done = 1;
            } else if (total <= sc->threshold || rn < sc->rel_delta * sc->maxr ||
                       sc->iter_since >= sc->rel_interval || sc->iter >= sc->max_iter) {
                sc->done = 2;
            } else {
                sc->maxr = fmax(sc->maxr, rn);
            }
        }
    }
}

// d = r + beta d for the live right-hand sides
template <int RB, int BS>
__global__ void __launch_bounds__(BS) multi_update_d_kernel(const MultiLaunch L) {
    const int4 w = L.items[blockIdx.x];
    const MultiGroup& G = L.groups[w.x];
    if (group_all_done(G, L.scal)) return;
    const Geom& g = G.g;
    const Lanes l = lanes_of<RB, BS>(G);
    const size_t vs = (size_t)g.vs;
    float beta[RB];
    bool live[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
        const int r = l.roff + j;
        live[j] = r < G.nrhs && !L.scal[G.rhs0 + r].done;
        beta[j] = live[j] ? L.scal[G.rhs0 + r].beta_ff.x : 0.f;
    }
    const int ntiles = (g.vh + l.spb - 1) / l.spb;
    const TileWalk tw = tile_walk(w, ntiles);
    for (int tile = tw.first; tile < tw.end; tile += tw.step) {
        const int i = tile * l.spb + l.site_local;
        if (i >= g.vh) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = ((size_t)c * vs + i) * G.rpad + l.roff;
            float2 d[RB], r[RB];
            load_rb_rw<RB>(d, G.d + k);
            load_rb<RB>(r, G.r + k);
#pragma unroll
            for (int j = 0; j < RB; ++j)
                if (live[j]) d[j] = make_float2(fmaf(beta[j], d[j].x, r[j].x), fmaf(beta[j], d[j].y, r[j].y));
            store_rb<RB>(G.d + k, d);
        }
    }
}

// ------------------------------------------- single right-hand-side slots
// r_lo[slot] = r64 / sigma; d[slot] = r_lo (first) or r_lo + beta d[slot]; y[slot] = 0
__global__ void __launch_bounds__(kBlock) slot_set_residual_kernel(Geom g, const double2* __restrict__ r64,
                                                                   float2* r, float2* d, float2* y, int rpad,
                                                                   int slot, double inv_sigma, float beta,
                                                                   int first) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = ((size_t)c * vs + i) * rpad + slot;
        const double2 rr = r64[(size_t)c * vs + i];
        const float2 rl = make_float2((float)(rr.x * inv_sigma), (float)(rr.y * inv_sigma));
        r[k] = rl;
        if (first) {
            d[k] = rl;
        } else {
            const float2 dd = d[k];
            d[k] = make_float2(fmaf(beta, dd.x, rl.x), fmaf(beta, dd.y, rl.y));
        }
        y[k] = make_float2(0.f, 0.f);
    }
}

// x64 += sigma * y[slot]; y[slot] = 0
__global__ void __launch_bounds__(kBlock) slot_fold_y_kernel(Geom g, double2* __restrict__ x, float2* y, int rpad,
                                                             int slot, double sigma) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = ((size_t)c * vs + i) * rpad + slot;
        const float2 yy = y[k];
        double2 xx = x[(size_t)c * vs + i];
        xx.x = fma(sigma, (double)yy.x, xx.x);
        xx.y = fma(sigma, (double)yy.y, xx.y);
        x[(size_t)c * vs + i] = xx;
        y[k] = make_float2(0.f, 0.f);
    }
}

// F64 SoA vector -> slot of a RHS-innermost FP32 vector (for operator tests), and back
__global__ void __launch_bounds__(kBlock) slot_put_kernel(Geom g, const double2* __restrict__ in, float2* out,
                                                          int rpad, int slot) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 v = in[(size_t)c * vs + i];
        out[((size_t)c * vs + i) * rpad + slot] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void __launch_bounds__(kBlock) slot_get_kernel(Geom g, const float2* in, double2* __restrict__ out,
                                                          int rpad, int slot) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 v = in[((size_t)c * vs + i) * rpad + slot];
        out[(size_t)c * vs + i] = make_double2((double)v.x, (double)v.y);
    }
}

// ------------------------------------------------------------ launchers
template <int RB, int BS, int MODE>
static void launch_dslash_mode(MultiKernel k, const MultiLaunch& L, int nitems, cudaStream_t s) {
    switch (k) {
        case MK_DSLASH_PLAIN: multi_dslash_kernel<RB, BS, EPI_PLAIN, MODE><<<nitems, BS, 0, s>>>(L); break;
        case MK_DSLASH_CG: multi_dslash_kernel<RB, BS, EPI_CG, MODE><<<nitems, BS, 0, s>>>(L); break;
        default: multi_dslash_kernel<RB, BS, EPI_AXPY, MODE><<<nitems, BS, 0, s>>>(L); break;
    }
}

template <int RB, int BS>
static void launch_multi_rb_bs(MultiKernel k, const MultiLaunch& L, int nitems, int mode, cudaStream_t s) {
    switch (k) {
        case MK_UPDATE_XR: multi_update_xr_kernel<RB, BS><<<nitems, BS, 0, s>>>(L); break;
        case MK_UPDATE_D: multi_update_d_kernel<RB, BS><<<nitems, BS, 0, s>>>(L); break;
        default:
            if (mode)
                launch_dslash_mode<RB, BS, 1>(k, L, nitems, s);
            else
                launch_dslash_mode<RB, BS, 0>(k, L, nitems, s);
    }
}

template <int RB>
static void launch_multi_rb(MultiKernel k, const MultiLaunch& L, int nitems, int bs, int mode, cudaStream_t s) {
    switch (bs) {
        case 64: launch_multi_rb_bs<RB, 64>(k, L, nitems, mode, s); break;
        case 128: launch_multi_rb_bs<RB, 128>(k, L, nitems, mode, s); break;
        default: launch_multi_rb_bs<RB, 256>(k, L, nitems, mode, s); break;
    }
}

template <int RB>
static int resident_rb(int bs) {
    int n = 0;
    switch (bs) {
        case 64: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, multi_dslash_kernel<RB, 64, EPI_CG, 1>, 64, 0); break;
        case 128:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, multi_dslash_kernel<RB, 128, EPI_CG, 1>, 128, 0);
            break;
        default:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, multi_dslash_kernel<RB, 256, EPI_CG, 1>, 256, 0);
            break;
    }
    return n;
}

int multi_resident_blocks_per_sm(int rb, int bs) {
    int n = 0;
    switch (rb) {
        case 1: n = resident_rb<1>(bs); break;
        case 2: n = resident_rb<2>(bs); break;
        case 4: n = resident_rb<4>(bs); break;
        default: n = resident_rb<8>(bs); break;
    }
    cudaGetLastError();
    return n > 0 ? n : 1;
}

void launch_multi(MultiKernel k, const MultiLaunch& L, int nitems, int rb, int bs, int mode, cudaStream_t s) {
    if (nitems <= 0) return;
    switch (rb) {
        case 1: launch_multi_rb<1>(k, L, nitems, bs, mode, s); break;
        case 2: launch_multi_rb<2>(k, L, nitems, bs, mode, s); break;
        case 4: launch_multi_rb<4>(k, L, nitems, bs, mode, s); break;
        default: launch_multi_rb<8>(k, L, nitems, bs, mode, s); break;
    }
}

void launch_slot_set_residual(const Geom& g, const double2* r64, float2* r, float2* d, float2* y, int rpad, int slot,
                              double inv_sigma, double beta, bool first, cudaStream_t s) {
    slot_set_residual_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, r64, r, d, y, rpad, slot, inv_sigma, (float)beta,
                                                                  first ? 1 : 0);
}

void launch_slot_fold_y(const Geom& g, double2* x, float2* y, int rpad, int slot, double sigma, cudaStream_t s) {
    slot_fold_y_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, x, y, rpad, slot, sigma);
}

void launch_slot_put(const Geom& g, const double2* in, float2* out, int rpad, int slot, cudaStream_t s) {
    slot_put_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, in, out, rpad, slot);
}

void launch_slot_get(const Geom& g, const float2* in, double2* out, int rpad, int slot, cudaStream_t s) {
    slot_get_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, in, out, rpad, slot);
}

}  // namespace stag
