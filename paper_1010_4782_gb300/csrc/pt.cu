// pt.cu - learned preconditioner: a gauge-covariant parallel-transport network,
// its training on the GPU with the library's own forward / adjoint /
// weight-gradient kernels (flexible CG that uses it: fcg.cu).
//
// The paper's CG (Sec. 2, Fig. 1) has no preconditioner; this is an added form
// built on the same operator.  Network (the oracle in oracle/ptnet.py states
// the same definitions):
//   paths p = 0..8: identity, and p = 1 + 2 mu + s transporting from x + mu
//   (s = 0: U_mu(x) psi(x+mu)) or x - mu (s = 1: U_mu(x-mu)^dag psi(x-mu)) with the
//   operator's eta-folded fat links, so that sum_mu (T_{+mu} - T_{-mu}) = D;
//   layer: psi_l(x, o) = sum_p sum_i W_l[p][o][i] (T_p psi_{l-1, i})(x);
//   three layers with 1 -> 8 -> 8 -> 1 complex channels on the whole lattice;
//   input: the residual on even sites (zero on odd sites); output: the last
//   channel on even sites.  Linear and gauge covariant.
// Training pairs (r_k, e_k = x* - x_k) are snapshots of plain-CG solves of
// caller-supplied sources, scaled by 1/|r_k|; loss: the residual norm of the
// correction, L = |A d|^2 / |A e|^2 with d = M r - e (the least-squares
// polynomial-preconditioning objective: it weights the modes of A by lambda^2,
// so the network fits lambda M(lambda) ~ 1 on the bulk of the spectrum), A
// applied with the FP32 Dirac kernels; Adam on the real and imaginary parts of
// the weights, each step followed by the self-adjoint tie W3 = W1^dag,
// W2 = W2^dag (M Hermitian, as flexible CG's short recurrence assumes).  Activations are stored
// as BF16 (or FP32, for gradient checks) and every sum runs in FP32.
//
// Applying the network (stag_ptnet_apply, flexible CG) evaluates by default its
// exact two-hop form: with the input on even sites and the output read on
// even sites only paths of zero or two hops survive, so
// M r = k0 r + sum_{p,q >= 1} H[p][q] T_p T_q r (pt_collapse_kernel forms k0 and
// H from the weights; pt_chi_kernel and pt_out_site apply them).  The layered
// evaluation (apply_net, and every training pass) stays available.
//
// Gradients (Wirtinger, G = dL/d conj(W)):
//   output seed  g_3 = A (A d) / |A e|^2 on even sites, 0 on odd sites;
//   data         g_{l-1}(x, i) = sum_p sum_o conj(W_l[p][o][i]) (T_p^dag g_{l,o})(x),
//                T_{+mu}^dag = T_{-mu}, T_{-mu}^dag = T_{+mu};
//   weights      G_l[p][o][i] = sum_x sum_c conj((T_p psi_{l-1,i})(x)_c) g_{l,o}(x)_c.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <random>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/stag.h"
#include "ff.cuh"
#include "handle.h"
#include "pt_common.cuh"
#include "pt_net.h"
#include "stag_kernels.h"

namespace stag {

// Which sites and paths a layer launch covers.  The network's input is zero on
// odd sites and only its output's even sites are read, so:
//   SITES_ALL  - every site, every path;
//   EVEN_INPUT - the input is zero on odd sites: an even output site takes only
//                the identity path, an odd one only the transports;
//   EVEN_OUTPUT- only even output sites are computed (odd ones are left as they are).
enum LayerMode { SITES_ALL = 0, EVEN_INPUT = 1, EVEN_OUTPUT = 2 };

// One layer (ADJ = false) or its adjoint (ADJ = true; CIN / COUT are then the
// forward layer's output / input channel counts, w its forward weights).
// Blocks alternate between the parities over the same run of 256 site indices
// (block 2c: even sites, 2c + 1: odd sites of run c; EVEN_OUTPUT: run b, even),
// so that a link or an activation read by a site of one parity is read again,
// by its neighbour of the other parity, while it is still in L2.  The 8 -> 8
// layer is held to 128 registers (two blocks per SM), the others to 85 (three).
// skip (nullable): the kernel returns at once while *skip is nonzero.
template <int CIN, int COUT, class TI, class TO, bool ADJ, int MODE = SITES_ALL>
__global__ void __launch_bounds__(256, CIN * COUT >= 64 ? 2 : 3)
    pt_layer_kernel(Geom g, const float2* __restrict__ links, const float2* __restrict__ w,
                    const TI* __restrict__ in, TO* __restrict__ out, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ float2 sw[kPaths * CIN * COUT];
    for (int k = threadIdx.x; k < kPaths * CIN * COUT; k += blockDim.x) sw[k] = w[k];
    __syncthreads();
    const int P = MODE == EVEN_OUTPUT ? 0 : (int)(blockIdx.x & 1);
    const int i = (MODE == EVEN_OUTPUT ? (int)blockIdx.x : (int)(blockIdx.x >> 1)) * 256 + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
    int x, y, z, t;
    site_coords(i, P, g, x, y, z, t);
    const int p0 = (MODE == EVEN_INPUT && P == 1) ? 1 : 0;
    const int p1 = (MODE == EVEN_INPUT && P == 0) ? 1 : kPaths;
    float2 acc[COUT][3];
#pragma unroll
    for (int o = 0; o < COUT; ++o)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[o][c] = make_float2(0.f, 0.f);
    float2 vin[3][4];  // a group of 4 input channels (CIN a multiple of 4)
    for (int p = p0; p < p1; ++p) {
        int Pn = P, nb = i, d = 0;
        float2 U[9];
        if (p > 0) {
            const int mu = (p - 1) >> 1, s = (p - 1) & 1;
            d = ADJ ? 1 - s : s;
            const Hop hp = pt_hop(g, links, P, i, x, y, z, t, mu, d);
            Pn = hp.Pn;
            nb = hp.nb;
#pragma unroll
            for (int k = 0; k < 9; ++k) U[k] = __ldg(hp.u + k * vs);
        }
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) {
            float2 v[3], tv[3];
            if constexpr (CIN % 4 == 0) {
                if (ci % 4 == 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) ld4c(in + fidx(ci, c, Pn, nb, vs, CIN), vin[c]);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] = vin[c][ci % 4];
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] = ldc(in + fidx(ci, c, Pn, nb, vs, CIN));
            }
            if (p > 0) {
                pt_apply(U, d, v, tv);
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) tv[c] = v[c];
            }
#pragma unroll
            for (int o = 0; o < COUT; ++o) {
                const float2 wv = ADJ ? make_float2(sw[(p * CIN + ci) * COUT + o].x, -sw[(p * CIN + ci) * COUT + o].y)
                                      : sw[(p * COUT + o) * CIN + ci];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 m = cmulf(wv, tv[c]);
                    acc[o][c].x += m.x;
                    acc[o][c].y += m.y;
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if constexpr (COUT % 4 == 0) {
#pragma unroll
            for (int o = 0; o < COUT; o += 4)
                st4c(out + fidx(o, c, P, i, vs, COUT), acc[o][c], acc[o + 1][c], acc[o + 2][c], acc[o + 3][c]);
        } else {
#pragma unroll
            for (int o = 0; o < COUT; ++o) stc(out + fidx(o, c, P, i, vs, COUT), acc[o][c]);
        }
    }
}

// partials[blk][p][o][i] = sum over the block's sites of
// sum_c conj((T_p psi_i)(x)_c) g_o(x)_c, o in [o0, o0 + OC), path p = blockIdx.y.
// MODE EVEN_INPUT: psi is zero on odd sites (only even sites for p = 0, odd
// sites for p > 0 contribute); EVEN_OUTPUT: g is zero on odd sites.
template <int CIN, int OC, class T, int MODE = SITES_ALL>
__global__ void __launch_bounds__(256) pt_wgrad_kernel(Geom g, const float2* __restrict__ links,
                                                       const T* __restrict__ psi, const T* __restrict__ gout,
                                                       int cout, float2* __restrict__ partials) {
    const int p = blockIdx.y;
    const int o0 = blockIdx.z * OC;
    const size_t vs = (size_t)g.vs;
    float2 acc[OC][CIN];
#pragma unroll
    for (int oo = 0; oo < OC; ++oo)
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) acc[oo][ci] = make_float2(0.f, 0.f);
    const int n0 = (MODE == EVEN_INPUT && p > 0) ? g.vh : 0;
    const int n1 = ((MODE == EVEN_INPUT && p == 0) || MODE == EVEN_OUTPUT) ? g.vh : 2 * g.vh;
    for (int n = n0 + blockIdx.x * blockDim.x + threadIdx.x; n < n1; n += gridDim.x * blockDim.x) {
        const int P = n >= g.vh ? 1 : 0;
        const int i = n - P * g.vh;
        int x, y, z, t;
        site_coords(i, P, g, x, y, z, t);
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
        float2 gv[OC][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if constexpr (OC % 4 == 0) {
#pragma unroll
                for (int oo = 0; oo < OC; oo += 4) {
                    float2 q[4];
                    ld4c(gout + fidx(o0 + oo, c, P, i, vs, cout), q);
#pragma unroll
                    for (int k = 0; k < 4; ++k) gv[oo + k][c] = q[k];
                }
            } else {
#pragma unroll
                for (int oo = 0; oo < OC; ++oo) gv[oo][c] = ldc(gout + fidx(o0 + oo, c, P, i, vs, cout));
            }
        }
        float2 vin[3][4];
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) {
            float2 v[3], tv[3];
            if constexpr (CIN % 4 == 0) {
                if (ci % 4 == 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) ld4c(psi + fidx(ci, c, Pn, nb, vs, CIN), vin[c]);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] = vin[c][ci % 4];
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] = ldc(psi + fidx(ci, c, Pn, nb, vs, CIN));
            }
            if (p > 0) {
                pt_apply(U, d, v, tv);
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) tv[c] = v[c];
            }
#pragma unroll
            for (int oo = 0; oo < OC; ++oo)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 m = cmulf_conj(tv[c], gv[oo][c]);
                    acc[oo][ci].x += m.x;
                    acc[oo][ci].y += m.y;
                }
        }
    }
    __shared__ float2 sred[256 / 32][OC * CIN];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int oo = 0; oo < OC; ++oo)
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) {
            float2 v = acc[oo][ci];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
            }
            if (lane == 0) sred[wp][oo * CIN + ci] = v;
        }
    __syncthreads();
    for (int k = threadIdx.x; k < OC * CIN; k += blockDim.x) {
        float2 s = make_float2(0.f, 0.f);
        for (int q = 0; q < (int)(blockDim.x / 32); ++q) {
            s.x += sred[q][k].x;
            s.y += sred[q][k].y;
        }
        const int oo = k / CIN, ci = k % CIN;
        partials[(((size_t)blockIdx.x * kPaths + p) * cout + o0 + oo) * CIN + ci] = s;
    }
}

// grad[p][o][i] += sum over blocks of partials (block order)
__global__ void pt_wgrad_sum_kernel(const float2* __restrict__ partials, int nblk, int nw, float2* grad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nw) return;
    float2 s = make_float2(0.f, 0.f);
    for (int b = 0; b < nblk; ++b) {
        s.x += partials[(size_t)b * nw + k].x;
        s.y += partials[(size_t)b * nw + k].y;
    }
    grad[k].x += s.x;
    grad[k].y += s.y;
}

// act0 = embed(scale * r): even sites from an even-site vector, odd sites zero.
template <class TS, class T>
__global__ void __launch_bounds__(kBlock) pt_embed_kernel(Geom g, const TS* __restrict__ src, double scale,
                                                          T* __restrict__ act0) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 v;
        if constexpr (std::is_same<TS, double2>::value) {
            const double2 d = src[c * vs + i];
            v = make_float2((float)(d.x * scale), (float)(d.y * scale));
        } else {
            v = ldc(src + c * vs + i);
        }
        stc(act0 + fidx(0, c, 0, i, vs, 1), v);
        stc(act0 + fidx(0, c, 1, i, vs, 1), make_float2(0.f, 0.f));
    }
}

// out (FP64 even SoA) = scale * act3 on even sites
template <class T>
__global__ void __launch_bounds__(kBlock) pt_extract_kernel(Geom g, const T* __restrict__ act3, double scale,
                                                            double2* __restrict__ out) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 v = ldc(act3 + fidx(0, c, 0, i, vs, 1));
        out[c * vs + i] = make_double2(scale * (double)v.x, scale * (double)v.y);
    }
}

// d = act3 - e on even sites, as an FP32 SoA vector [3][vs]
template <class T>
__global__ void __launch_bounds__(kBlock) pt_diff_kernel(Geom g, const T* __restrict__ act3, const T* __restrict__ e,
                                                         float2* __restrict__ d) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 o = ldc(act3 + fidx(0, c, 0, i, vs, 1));
        const float2 t = ldc(e + c * vs + i);
        d[c * vs + i] = make_float2(o.x - t.x, o.y - t.y);
    }
}

// g3 = v * inv on even sites (0 on odd)
template <class T>
__global__ void __launch_bounds__(kBlock) pt_seed_kernel(Geom g, const float2* __restrict__ v, float inv,
                                                         T* __restrict__ g3) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 a = v[c * vs + i];
        stc(g3 + fidx(0, c, 0, i, vs, 1), make_float2(a.x * inv, a.y * inv));
        stc(g3 + fidx(0, c, 1, i, vs, 1), make_float2(0.f, 0.f));
    }
}

// FP32 copy [3][vs] of a slot
template <class T>
__global__ void __launch_bounds__(kBlock) pt_slot_f32_kernel(Geom g, const T* __restrict__ slot, float2* __restrict__ out) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c * vs + i] = ldc(slot + c * vs + i);
}

// per-block partials of Re<a, b> for FP32 [3][vs] vectors (FP64 sums)
__global__ void __launch_bounds__(kBlock) pt_dot_f32_kernel(Geom g, const float2* __restrict__ a,
                                                            const float2* __restrict__ b, double* __restrict__ partials) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    double acc = 0.0;
    if (i < g.vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 x = a[c * vs + i], y = b[c * vs + i];
            acc += (double)x.x * y.x + (double)x.y * y.y;
        }
    }
    __shared__ double sm[kBlock / 32];
    const double s = block_sum<kBlock>(acc, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// |v|^2 of an even-site vector (T, [3][vs]) -> per-block partials (FP64)
template <class T>
__global__ void __launch_bounds__(kBlock) pt_norm2_kernel(Geom g, const T* __restrict__ v, double* partials) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    double acc = 0.0;
    if (i < g.vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 a = ldc(v + c * vs + i);
            acc += (double)a.x * a.x + (double)a.y * a.y;
        }
    }
    __shared__ double sm[kBlock / 32];
    const double s = block_sum<kBlock>(acc, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// slot (T, even [3][vs]) = scale * v, v an FP64 or float-float SoA vector
template <class TS, class T>
__global__ void __launch_bounds__(kBlock) pt_store_slot_kernel(Geom g, const TS* __restrict__ v, double scale,
                                                               T* __restrict__ slot) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double2 d;
        if constexpr (std::is_same<TS, float4>::value)
            d = ff_to_complex(v[c * vs + i]);
        else
            d = v[c * vs + i];
        stc(slot + c * vs + i, make_float2((float)(d.x * scale), (float)(d.y * scale)));
    }
}

// slot = scale * (a - b), FP64 inputs
template <class T>
__global__ void __launch_bounds__(kBlock) pt_store_diff_kernel(Geom g, const double2* __restrict__ a,
                                                               const double2* __restrict__ b, double scale,
                                                               T* __restrict__ slot) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 x = a[c * vs + i], y = b[c * vs + i];
        stc(slot + c * vs + i, make_float2((float)((x.x - y.x) * scale), (float)((x.y - y.y) * scale)));
    }
}

// Adam on the real and imaginary parts: grad is sum_batch dL/dconj(W); dL/d(Re, Im) = 2 (Re, Im) / batch
__global__ void pt_adam_kernel(float* w, const float* grad, float* m, float* v, int n, float gscale, float lr,
                               float b1, float b2, float c1, float c2, float eps) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = grad[k] * gscale;
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// The path opposite to p (T_{+mu}^dag = T_{-mu}); p = 0 is its own.
__host__ __device__ __forceinline__ int rev_path(int p) { return p == 0 ? 0 : (((p - 1) ^ 1) + 1); }

// Self-adjoint tie: projects the weights onto W3[p][0][i] = conj(W1[rev p][i][0])
// and W2[p][o][i] = conj(W2[rev p][i][o]) (each weight and its partner's conjugate
// replaced by their mean), which makes M = E^dag L3 L2 L1 E Hermitian.  One
// block; every pair is handled by one thread.
__global__ void pt_tie_kernel(float2* w) {
    constexpr int H = kHidden;
    float2* w1 = w;                                   // [9][H][1]
    float2* w2 = w + kPaths * H;                      // [9][H][H]
    float2* w3 = w + kPaths * H + kPaths * H * H;     // [9][1][H]
    for (int k = threadIdx.x; k < kPaths * H; k += blockDim.x) {
        const int p = k / H, o = k % H;
        const int k3 = rev_path(p) * H + o;
        const float2 a = w1[k], b = w3[k3];
        const float2 m = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
        w1[k] = m;
        w3[k3] = make_float2(m.x, -m.y);
    }
    for (int k = threadIdx.x; k < kPaths * H * H; k += blockDim.x) {
        const int p = k / (H * H), o = (k / H) % H, i = k % H;
        const int kp = (rev_path(p) * H + i) * H + o;
        if (kp < k) continue;
        const float2 a = w2[k], b = w2[kp];
        const float2 m = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
        w2[k] = m;
        w2[kp] = make_float2(m.x, -m.y);
    }
}

// v = a fixed pseudo-random vector (start of the power iteration)
__global__ void pt_fill_kernel(Geom g, float2* v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        unsigned int h = (unsigned int)(c * vs + i) * 2654435761u + 12345u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        const float a = (float)(h & 0xffff) / 65536.f - 0.5f;
        const float b = (float)(h >> 16) / 65536.f - 0.5f;
        v[c * vs + i] = make_float2(a, b);
    }
}

// v = s * w
__global__ void pt_scale_kernel(Geom g, float2* v, const float2* w, float s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 a = w[c * vs + i];
        v[c * vs + i] = make_float2(s * a.x, s * a.y);
    }
}

// FP32 copy of the eta-folded FP64 links
__global__ void pt_links_kernel(const double2* __restrict__ in, float2* __restrict__ out, size_t n) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = make_float2((float)in[k].x, (float)in[k].y);
}

// largest |Re|, |Im| of the entries (as FP32 bits, atomically into *out; NaNs ignored)
__global__ void pt_absmax_kernel(const double2* __restrict__ in, size_t n, unsigned int* out) {
    float m = 0.f;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fmaxf(fabsf((float)in[k].x), fabsf((float)in[k].y)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// FP16 copy of the links divided by s
__global__ void pt_links16_kernel(const double2* __restrict__ in, __half2* __restrict__ out, size_t n, double inv_s) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = __floats2half2_rn((float)(in[k].x * inv_s), (float)(in[k].y * inv_s));
}

// ------------------------------------------------ collapsed inference form
// coef[0] = k0 = C[0][0][0], coef[1 + 8 (p - 1) + (q - 1)] = H[p][q] =
// C[p][q][0] + C[p][0][q] + C[0][p][q] with C[a][b][c] = sum_{o,i} W3[a][0][o]
// W2[b][o][i] W1[c][i][0]: the terms of the layer product T_a T_b T_c that
// take an even site to an even site (zero or two hops).  FP64 sums; H is
// multiplied by h_scale (s^2 for links stored divided by s).
__global__ void pt_collapse_kernel(const float2* __restrict__ w, float2* __restrict__ coef, double h_scale) {
    const int t = threadIdx.x;
    if (t >= kCollapsedCoefs) return;
    const float2* w1 = w;                                    // [9][8][1]
    const float2* w2 = w + kPaths * kHidden;                 // [9][8][8]
    const float2* w3 = w2 + kPaths * kHidden * kHidden;      // [9][1][8]
    auto C = [&](int a, int b, int c) {
        double re = 0.0, im = 0.0;
        for (int o = 0; o < kHidden; ++o) {
            const float2 x = w3[a * kHidden + o];
            for (int i = 0; i < kHidden; ++i) {
                const float2 y = w2[(b * kHidden + o) * kHidden + i], z = w1[c * kHidden + i];
                const double xyr = (double)x.x * y.x - (double)x.y * y.y;
                const double xyi = (double)x.x * y.y + (double)x.y * y.x;
                re += xyr * z.x - xyi * z.y;
                im += xyr * z.y + xyi * z.x;
            }
        }
        return make_double2(re, im);
    };
    double2 h;
    if (t == 0) {
        h = C(0, 0, 0);
    } else {
        const int p = 1 + (t - 1) / 8, q = 1 + (t - 1) % 8;
        const double2 a = C(p, q, 0), b = C(p, 0, q), c = C(0, p, q);
        h = make_double2(h_scale * (a.x + b.x + c.x), h_scale * (a.y + b.y + c.y));
    }
    coef[t] = make_float2((float)h.x, (float)h.y);
}

// chi on odd sites (pt_chi_site), stored as TS; links stored as L
template <class V, class TS, class L>
__global__ void __launch_bounds__(256, 2) pt_chi_kernel(Geom g, const L* __restrict__ links,
                                                        const float2* __restrict__ coef, const V* __restrict__ r,
                                                        TS* __restrict__ chi, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ float2 sH[64];
    for (int k = threadIdx.x; k < 64; k += blockDim.x) sH[k] = coef[1 + k];
    __syncthreads();
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
    float2 acc[8][3];
    pt_chi_site(g, links, sH, r, i, acc);
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int c = 0; c < 3; ++c) stc(chi + ((size_t)p * 3 + c) * vs + i, acc[p][c]);
}

// out (FP64, even sites) = k0 r + sum_p T_p chi_p
template <class TS, class L>
__global__ void __launch_bounds__(256) pt_out_kernel(Geom g, const L* __restrict__ links,
                                                     const float2* __restrict__ coef, const TS* __restrict__ chi,
                                                     const double2* __restrict__ r, double2* __restrict__ out) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
    float2 r0[3], z[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) r0[c] = ldc(r + c * vs + i);
    pt_out_site(g, links, coef[0], chi, i, r0, z);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c * vs + i] = make_double2(z[c].x, z[c].y);
}

// ------------------------------------------------ FP64 vector reductions
// Re(a, b), Re(a, c) (c nullable) and |b|^2: per-block partials, then the last
// block (atomic ticket) sums them in block order into out3[0..2].
__global__ void __launch_bounds__(kBlock) pt_dots_kernel(Geom g, const double2* __restrict__ a,
                                                          const double2* __restrict__ b, const double2* __restrict__ c,
                                                          double* __restrict__ partials, int nblk,
                                                          unsigned int* counter, double* out3) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const size_t vs = (size_t)g.vs;
    double ab = 0.0, ac = 0.0, bb = 0.0;
    if (i < g.vh) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double2 x = a[k * vs + i], y = b[k * vs + i];
            ab = fma(x.x, y.x, fma(x.y, y.y, ab));
            bb = fma(y.x, y.x, fma(y.y, y.y, bb));
            if (c) {
                const double2 zz = c[k * vs + i];
                ac = fma(x.x, zz.x, fma(x.y, zz.y, ac));
            }
        }
    }
    __shared__ double sm[kBlock / 32];
    const double s0 = block_sum<kBlock>(ab, sm);
    __syncthreads();
    const double s1 = block_sum<kBlock>(ac, sm);
    __syncthreads();
    const double s2 = block_sum<kBlock>(bb, sm);
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s0;
        partials[nblk + blockIdx.x] = s1;
        partials[2 * nblk + blockIdx.x] = s2;
        __threadfence();
        is_last = atomicAdd(counter, 1u) == (unsigned)nblk - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int bb2 = threadIdx.x; bb2 < nblk; bb2 += kBlock) s += __ldcg(partials + (size_t)k * nblk + bb2);
        __syncthreads();
        s = block_sum<kBlock>(s, sm);
        if (threadIdx.x == 0) out3[k] = s;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

}  // namespace stag

using namespace stag;

// =========================================================== the network
namespace stag {

void pfail(stag_ptnet* n, int code, const std::string& msg) {
    if (n) n->err = msg;
    throw PFail{code};
}

void pcheck(stag_ptnet* n, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    pfail(n, e == cudaErrorMemoryAllocation ? STAG_ERR_OOM : STAG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* palloc(stag_ptnet* n, size_t bytes, const char* what) {
    void* p = nullptr;
    pcheck(n, cudaMalloc(&p, bytes), what);
    n->device_bytes += (long long)bytes;
    pcheck(n, cudaMemsetAsync(p, 0, bytes, n->h->s), what);
    return p;
}

void check_tc(stag_ptnet* n) {
    int flag = 0;
    pcheck(n, cudaMemcpyAsync(&flag, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost, S(n)), "read error flag");
    pcheck(n, cudaStreamSynchronize(S(n)), "sync");
    if (flag) pfail(n, STAG_ERR_TIMEOUT, "tensor-core layer: a bounded wait on the MMA barrier ran out");
}

}  // namespace stag

namespace {

int layer_offset(int l) {  // complex weights before layer l (0-based)
    int off = 0;
    for (int k = 0; k < l; ++k) off += kPaths * kChan[k + 1] * kChan[k];
    return off;
}
int n_weights() { return layer_offset(kLayers); }

size_t field_bytes(const stag_ptnet* n, int ch) { return (size_t)ch * 3 * 2 * n->g.vs * sizeof(float2); }
size_t slot_bytes(const stag_ptnet* n) { return (size_t)3 * n->g.vs * n->elem; }
// blocks of a pt_layer_kernel launch over both parities (256 sites per block)
int site_blocks(const Geom& g) { return 2 * blocks_for(g.vh, 256); }

template <class T>
void layer_fwd(stag_ptnet* n, int l, const T* in, T* out) {
    const Geom& g = n->g;
    const float2* w = n->w + layer_offset(l);
    const int nb = site_blocks(g);
    if (l == 0)
        pt_layer_kernel<1, kHidden, T, T, false, EVEN_INPUT><<<nb, 256, 0, S(n)>>>(g, n->links, w, in, out, nullptr);
    else if (l == 1) {
        if constexpr (std::is_same<T, __nv_bfloat162>::value) {
            if (n->use_tc) {
                launch_pt_mix8_tc(g, n->links, w, in, out, nullptr, n->tc_err, S(n));
                return;
            }
        }
        pt_layer_kernel<kHidden, kHidden, T, T, false><<<nb, 256, 0, S(n)>>>(g, n->links, w, in, out, nullptr);
    } else
        pt_layer_kernel<kHidden, 1, T, T, false, EVEN_OUTPUT><<<blocks_for(g.vh), 256, 0, S(n)>>>(g, n->links, w, in,
                                                                                                  out, nullptr);
}

// gradient of layer l's input from the gradient of its output
template <class T>
void layer_adj(stag_ptnet* n, int l, const T* gout, T* gin) {
    const Geom& g = n->g;
    const float2* w = n->w + layer_offset(l);
    const int nb = site_blocks(g);
    if (l == 2)
        pt_layer_kernel<1, kHidden, T, T, true, EVEN_INPUT><<<nb, 256, 0, S(n)>>>(g, n->links, w, gout, gin, nullptr);
    else if (l == 1)
        pt_layer_kernel<kHidden, kHidden, T, T, true><<<nb, 256, 0, S(n)>>>(g, n->links, w, gout, gin, nullptr);
}

template <class T>
void layer_wgrad(stag_ptnet* n, int l, const T* psi, const T* gout) {
    const Geom& g = n->g;
    const int cin = kChan[l], cout = kChan[l + 1];
    const int nw = kPaths * cout * cin;
    if (l == 0) {
        dim3 grid(kWgradBlocks, kPaths, 1);
        pt_wgrad_kernel<1, kHidden, T, EVEN_INPUT><<<grid, 256, 0, S(n)>>>(g, n->links, psi, gout, cout, n->wpart);
    } else if (l == 1) {
        dim3 grid(kWgradBlocks, kPaths, kHidden / 4);
        pt_wgrad_kernel<kHidden, 4, T><<<grid, 256, 0, S(n)>>>(g, n->links, psi, gout, cout, n->wpart);
    } else {
        dim3 grid(kWgradBlocks, kPaths, 1);
        pt_wgrad_kernel<kHidden, 1, T, EVEN_OUTPUT><<<grid, 256, 0, S(n)>>>(g, n->links, psi, gout, cout, n->wpart);
    }
    pt_wgrad_sum_kernel<<<blocks_for(nw), kBlock, 0, S(n)>>>(n->wpart, kWgradBlocks, nw, n->grad + layer_offset(l));
}

double read_partials(stag_ptnet* n, int count) {
    n->red_host.resize(count);
    pcheck(n, cudaMemcpyAsync(n->red_host.data(), n->red, count * sizeof(double), cudaMemcpyDeviceToHost, S(n)),
           "read reduction");
    pcheck(n, cudaStreamSynchronize(S(n)), "sync");
    double s = 0.0;
    for (int k = 0; k < count; ++k) s += n->red_host[k];
    return s;
}

// vad = A va with the FP32 Dirac kernels (uses vt)
void apply_A_f32(stag_ptnet* n) {
    const Geom& g = n->g;
    const double m2 = n->h->mass * n->h->mass;
    launch_dslash_f32(g, 1, n->links, n->lng, n->va, n->vt, EPI_PLAIN, nullptr, 0.0, nullptr, nullptr, S(n));
    launch_dslash_f32(g, 0, n->links, n->lng, n->vt, n->vad, EPI_AXPY, n->va, m2, nullptr, nullptr, S(n));
}

// |A e|^2 of a slot
template <class T>
double slot_energy(stag_ptnet* n, const void* slot) {
    const Geom& g = n->g;
    pt_slot_f32_kernel<T><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, static_cast<const T*>(slot), n->va);
    apply_A_f32(n);
    pt_dot_f32_kernel<<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, n->vad, n->vad, n->red);
    return read_partials(n, blocks_for(g.vh));
}

template <class T>
double slot_norm2(stag_ptnet* n, const void* slot) {
    pt_norm2_kernel<T><<<blocks_for(n->g.vh), kBlock, 0, S(n)>>>(n->g, static_cast<const T*>(slot), n->red);
    return read_partials(n, blocks_for(n->g.vh));
}

// forward through all layers from act[0]
template <class T>
void forward(stag_ptnet* n) {
    for (int l = 0; l < kLayers; ++l) layer_fwd<T>(n, l, static_cast<const T*>(n->act[l]), static_cast<T*>(n->act[l + 1]));
}

// forward pass and loss |A d|^2 / |A e|^2 of one pair (eae = |A e|^2); with
// seed, leaves the output gradient A (A d) / |A e|^2 in gact[3]
template <class T>
double forward_energy(stag_ptnet* n, const void* r, const void* e, double eae, bool seed = false) {
    const Geom& g = n->g;
    pt_embed_kernel<T, T><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, static_cast<const T*>(r), 1.0, static_cast<T*>(n->act[0]));
    forward<T>(n);
    pt_diff_kernel<T><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, static_cast<const T*>(n->act[3]), static_cast<const T*>(e), n->va);
    apply_A_f32(n);
    pt_dot_f32_kernel<<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, n->vad, n->vad, n->red);
    if (seed) {
        pcheck(n, cudaMemcpyAsync(n->va, n->vad, (size_t)3 * g.vs * sizeof(float2), cudaMemcpyDeviceToDevice, S(n)), "copy");
        apply_A_f32(n);
        pt_seed_kernel<T><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, n->vad, (float)(1.0 / eae), static_cast<T*>(n->gact[3]));
    }
    pcheck(n, cudaGetLastError(), "forward");
    return read_partials(n, blocks_for(g.vh)) / eae;
}

// loss and accumulated weight gradients of one pair (slots r, e; <e, A e>); returns the loss
template <class T>
double sample_step(stag_ptnet* n, const void* r, const void* e, double eae) {
    const double loss = forward_energy<T>(n, r, e, eae, true);
    for (int l = kLayers - 1; l >= 0; --l) {
        layer_wgrad<T>(n, l, static_cast<const T*>(n->act[l]), static_cast<const T*>(n->gact[l + 1]));
        if (l > 0) layer_adj<T>(n, l, static_cast<const T*>(n->gact[l + 1]), static_cast<T*>(n->gact[l]));
    }
    pcheck(n, cudaGetLastError(), "training step");
    return loss;
}

// z = M(r) for FP64 vectors (scaled by 1/|r| on the way in, back on the way out)
template <class T>
void apply_net(stag_ptnet* n, const double2* r, double rnorm, double2* z) {
    const Geom& g = n->g;
    const double s = rnorm > 0.0 ? 1.0 / rnorm : 1.0;
    pt_embed_kernel<double2, T><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, r, s, static_cast<T*>(n->act[0]));
    bool fused = false;
    if constexpr (std::is_same<T, __nv_bfloat162>::value) {
        if (n->use_tc) {
            // the last layer's mixing in the tensor-core kernel's epilogue, then its transports
            layer_fwd<T>(n, 0, static_cast<const T*>(n->act[0]), static_cast<T*>(n->act[1]));
            launch_pt_mix8_tc(g, n->links, n->w + layer_offset(1), static_cast<const T*>(n->act[1]),
                              static_cast<T*>(n->act[2]), n->w + layer_offset(2), n->tc_err, S(n));
            launch_pt_transport_sum(g, n->links, static_cast<const T*>(n->act[2]), static_cast<T*>(n->act[3]), S(n));
            fused = true;
        }
    }
    if (!fused) forward<T>(n);
    pt_extract_kernel<T><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, static_cast<const T*>(n->act[3]), rnorm > 0.0 ? rnorm : 1.0, z);
}

void upload_weights(stag_ptnet* n) {
    pcheck(n, cudaMemcpyAsync(n->w, n->w_host.data(), n->w_host.size() * sizeof(float2), cudaMemcpyHostToDevice, S(n)),
           "upload weights");
}

void download_weights(stag_ptnet* n) {
    pcheck(n, cudaMemcpyAsync(n->w_host.data(), n->w, n->w_host.size() * sizeof(float2), cudaMemcpyDeviceToHost, S(n)),
           "download weights");
    pcheck(n, cudaStreamSynchronize(S(n)), "sync");
}

void destroy_net(stag_ptnet* n) {
    if (!n) return;
    if (n->h && n->h->s) cudaStreamSynchronize(n->h->s);
    for (void* p : {(void*)n->links, (void*)n->lng, (void*)n->va, (void*)n->vt, (void*)n->vad, (void*)n->w, (void*)n->grad, (void*)n->adam_m, (void*)n->adam_v,
                    (void*)n->wpart, (void*)n->red, n->scratch_r, n->scratch_e, (void*)n->fr, (void*)n->fz,
                    (void*)n->fq, (void*)n->tc_err, (void*)n->dot_counter, (void*)n->dot_out, n->fcg_r, n->fcg_p,
                    n->fcg_q, n->fcg_t, n->fcg_x, (void*)n->fcg_dev, (void*)n->coef, (void*)n->links16})
        if (p) cudaFree(p);
    if (n->fcg_host) cudaFreeHost(n->fcg_host);
    if (n->fcg_graph) cudaGraphExecDestroy(n->fcg_graph);
    for (int l = 0; l <= kLayers; ++l) {
        if (n->act[l]) cudaFree(n->act[l]);
        if (n->gact[l]) cudaFree(n->gact[l]);
    }
    for (void* p : n->pairs_r) cudaFree(p);
    for (void* p : n->pairs_e) cudaFree(p);
    delete n;
}

bool is_bf16(const stag_ptnet* n) { return n->prec == STAG_ARITH_BF16; }

// (Re<a,b>, Re<a,c>, |b|^2)
void dots(stag_ptnet* n, const double2* a, const double2* b, const double2* c, double out[3]) {
    const Geom& g = n->g;
    const int nb = blocks_for(g.vh);
    pt_dots_kernel<<<nb, kBlock, 0, S(n)>>>(g, a, b, c, n->red, nb, n->dot_counter, n->dot_out);
    pcheck(n, cudaGetLastError(), "dots");
    pcheck(n, cudaMemcpyAsync(out, n->dot_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, S(n)), "read dots");
    pcheck(n, cudaStreamSynchronize(S(n)), "sync");
}

// The network from a solver vector r (even sites) into act[3]: the first layer
// reads r directly (float-float or FP64, rounded to FP32 on load); the layers
// after it are those of apply_net.
template <class T, class V>
void network_from_vec(stag_ptnet* n, const V* r, const int* skip) {
    const Geom& g = n->g;
    const int nb = site_blocks(g);
    T* a1 = static_cast<T*>(n->act[1]);
    T* a2 = static_cast<T*>(n->act[2]);
    T* a3 = static_cast<T*>(n->act[3]);
    pt_layer_kernel<1, kHidden, V, T, false, EVEN_INPUT><<<nb, 256, 0, S(n)>>>(g, n->links, n->w, r, a1, skip);
    if constexpr (std::is_same<T, __nv_bfloat162>::value) {
        if (n->use_tc) {
            launch_pt_mix8_tc(g, n->links, n->w + layer_offset(1), a1, a2, n->w + layer_offset(2), n->tc_err, S(n),
                              skip);
            launch_pt_transport_sum(g, n->links, a2, a3, S(n), skip);
            return;
        }
    }
    pt_layer_kernel<kHidden, kHidden, T, T, false><<<nb, 256, 0, S(n)>>>(g, n->links, n->w + layer_offset(1), a1, a2,
                                                                          skip);
    pt_layer_kernel<kHidden, 1, T, T, false, EVEN_OUTPUT><<<blocks_for(g.vh), 256, 0, S(n)>>>(
        g, n->links, n->w + layer_offset(2), a2, a3, skip);
}

template <class V>
void network_from_vec_any(stag_ptnet* n, const V* r, const int* skip) {
    if (infer_bf16(n))
        network_from_vec<__nv_bfloat162>(n, r, skip);
    else
        network_from_vec<float2>(n, r, skip);
}

}  // namespace

namespace stag {
void pt_network_from_vec(stag_ptnet* n, const float4* r, const int* skip) { network_from_vec_any(n, r, skip); }
void pt_network_from_vec(stag_ptnet* n, const double2* r, const int* skip) { network_from_vec_any(n, r, skip); }

void pt_collapse(stag_ptnet* n) {
    const double s = infer_bf16(n) ? (double)n->links16_scale : 1.0;
    pt_collapse_kernel<<<1, 96, 0, S(n)>>>(n->w, n->coef, s * s);
}

template <class V>
void launch_pt_chi_any(stag_ptnet* n, const V* r, const int* skip) {
    const int nb = blocks_for(n->g.vh, 256);
    if (infer_bf16(n))
        pt_chi_kernel<V, __nv_bfloat162, __half2><<<nb, 256, 0, S(n)>>>(
            n->g, n->links16, n->coef, r, static_cast<__nv_bfloat162*>(n->act[2]), skip);
    else
        pt_chi_kernel<V, float2, float2><<<nb, 256, 0, S(n)>>>(n->g, n->links, n->coef, r,
                                                               static_cast<float2*>(n->act[2]), skip);
}
void launch_pt_chi(stag_ptnet* n, const float4* r, const int* skip) { launch_pt_chi_any(n, r, skip); }
void launch_pt_chi(stag_ptnet* n, const double2* r, const int* skip) { launch_pt_chi_any(n, r, skip); }
}  // namespace stag

namespace {
// z = M r (FP64 even-site vectors) in the collapsed form
void apply_collapsed(stag_ptnet* n, const double2* r, double2* z) {
    const Geom& g = n->g;
    pt_collapse(n);
    launch_pt_chi(n, r, nullptr);
    if (infer_bf16(n))
        pt_out_kernel<__nv_bfloat162, __half2><<<blocks_for(g.vh, 256), 256, 0, S(n)>>>(
            g, n->links16, n->coef, static_cast<const __nv_bfloat162*>(n->act[2]), r, z);
    else
        pt_out_kernel<float2, float2><<<blocks_for(g.vh, 256), 256, 0, S(n)>>>(
            g, n->links, n->coef, static_cast<const float2*>(n->act[2]), r, z);
}
}  // namespace

extern "C" {

int stag_ptnet_create(stag_ptnet** out, stag_handle* h, int32_t precision, uint64_t seed) {
    if (out) *out = nullptr;
    if (!out || !h) return STAG_ERR_INVALID_ARG;
    stag_ptnet* n = nullptr;
    try {
        if (precision != STAG_ARITH_BF16 && precision != STAG_ARITH_F32) {
            h->err = "ptnet precision must be STAG_ARITH_BF16 or STAG_ARITH_F32";
            return STAG_ERR_INVALID_ARG;
        }
        n = new stag_ptnet();
        n->h = h;
        n->g = h->g;
        n->prec = precision;
        n->inf_prec = precision;
        n->elem = precision == STAG_ARITH_BF16 ? sizeof(__nv_bfloat162) : sizeof(float2);
        handle_begin(h);
        const size_t nl = (size_t)2 * 4 * 9 * n->g.vs;
        n->links = static_cast<float2*>(palloc(n, nl * sizeof(float2), "allocate links"));
        pt_links_kernel<<<(int)((nl + 255) / 256), 256, 0, S(n)>>>(h->fat64, n->links, nl);
        if (h->lng64) {
            n->lng = static_cast<float2*>(palloc(n, nl * sizeof(float2), "allocate links"));
            pt_links_kernel<<<(int)((nl + 255) / 256), 256, 0, S(n)>>>(h->lng64, n->lng, nl);
        }
        const size_t fv = (size_t)3 * n->g.vs * sizeof(float2);
        n->va = static_cast<float2*>(palloc(n, fv, "allocate vectors"));
        n->vt = static_cast<float2*>(palloc(n, fv, "allocate vectors"));
        n->vad = static_cast<float2*>(palloc(n, fv, "allocate vectors"));
        const int nw = n_weights();
        n->w = static_cast<float2*>(palloc(n, nw * sizeof(float2), "allocate weights"));
        n->tc_err = static_cast<int*>(palloc(n, sizeof(int), "allocate error flag"));
        n->coef = static_cast<float2*>(palloc(n, kCollapsedCoefs * sizeof(float2), "allocate coefficients"));
        n->dot_counter = static_cast<unsigned int*>(palloc(n, sizeof(unsigned int), "allocate counter"));
        n->dot_out = static_cast<double*>(palloc(n, 3 * sizeof(double), "allocate sums"));
        {
            // FP16 links for the two-hop inference kernels, divided by s = the power of two
            // nearest the largest entry (so that they stay inside FP16's normal range)
            // dot_counter (zero until pt_dots_kernel uses it as its ticket) holds the maximum
            unsigned int* mx = n->dot_counter;
            pt_absmax_kernel<<<1024, 256, 0, S(n)>>>(h->fat64, nl, mx);
            unsigned int bits = 0;
            pcheck(n, cudaMemcpyAsync(&bits, mx, sizeof(bits), cudaMemcpyDeviceToHost, S(n)), "read link maximum");
            pcheck(n, cudaMemsetAsync(mx, 0, sizeof(unsigned int), S(n)), "reset counter");
            pcheck(n, cudaStreamSynchronize(S(n)), "sync");
            float amax;
            std::memcpy(&amax, &bits, sizeof(amax));
            n->links16_scale = (amax > 0.f && std::isfinite(amax)) ? std::exp2f(std::round(std::log2(amax))) : 1.f;
            n->links16 = static_cast<__half2*>(palloc(n, nl * sizeof(__half2), "allocate links"));
            pt_links16_kernel<<<(int)((nl + 255) / 256), 256, 0, S(n)>>>(h->fat64, n->links16, nl,
                                                                          1.0 / n->links16_scale);
        }
        n->grad = static_cast<float2*>(palloc(n, nw * sizeof(float2), "allocate gradients"));
        n->adam_m = static_cast<float*>(palloc(n, 2 * nw * sizeof(float), "allocate optimiser"));
        n->adam_v = static_cast<float*>(palloc(n, 2 * nw * sizeof(float), "allocate optimiser"));
        n->wpart = static_cast<float2*>(palloc(n, (size_t)kWgradBlocks * nw * sizeof(float2), "allocate partials"));
        n->red = static_cast<double*>(palloc(n, 3 * (size_t)blocks_for(2 * n->g.vs) * sizeof(double), "allocate partials"));
        for (int l = 0; l <= kLayers; ++l) {
            n->act[l] = palloc(n, field_bytes(n, kChan[l]), "allocate activations");
            n->gact[l] = palloc(n, field_bytes(n, kChan[l]), "allocate activations");
        }
        n->scratch_r = palloc(n, slot_bytes(n), "allocate slots");
        n->scratch_e = palloc(n, slot_bytes(n), "allocate slots");
        const size_t vb = (size_t)3 * n->g.vs * sizeof(double2);
        n->fr = static_cast<double2*>(palloc(n, vb, "allocate vectors"));
        n->fz = static_cast<double2*>(palloc(n, vb, "allocate vectors"));
        n->fq = static_cast<double2*>(palloc(n, vb, "allocate vectors"));
        static_assert(sizeof(float4) == sizeof(double2), "float-float and FP64 complex vectors share their size");
        for (void** v : {&n->fcg_r, &n->fcg_p, &n->fcg_q, &n->fcg_t, &n->fcg_x}) *v = palloc(n, vb, "allocate FCG vectors");
        n->fcg_dev = static_cast<FcgDev*>(palloc(n, sizeof(FcgDev), "allocate FCG state"));
        pcheck(n, cudaMallocHost(&n->fcg_host, sizeof(FcgDev)), "allocate FCG state");
        // initial weights: the least-squares degree-1 polynomial preconditioner
        // alpha + beta A_fat (A_fat: the one-hop part the transports can express),
        // minimising the integral of (1 - lambda p(lambda))^2 over [0, Lmax]:
        // alpha = 4 / Lmax, beta = -10 / (3 Lmax^2); Lmax = 1.25 times the Rayleigh
        // quotient after 100 power iterations of the FP32 operator (the quotient
        // approaches the largest eigenvalue from below, slowly when the top of the
        // spectrum is dense; lambda p(lambda) stays positive up to 1.2 Lmax).
        // Plus small seeded noise.
        pt_fill_kernel<<<blocks_for(n->g.vh), kBlock, 0, S(n)>>>(n->g, n->va);
        double lam = 1.0;
        for (int it = 0; it < 100; ++it) {
            apply_A_f32(n);
            pt_dot_f32_kernel<<<blocks_for(n->g.vh), kBlock, 0, S(n)>>>(n->g, n->va, n->vad, n->red);
            const double num = read_partials(n, blocks_for(n->g.vh));
            pt_dot_f32_kernel<<<blocks_for(n->g.vh), kBlock, 0, S(n)>>>(n->g, n->va, n->va, n->red);
            const double den = read_partials(n, blocks_for(n->g.vh));
            pt_dot_f32_kernel<<<blocks_for(n->g.vh), kBlock, 0, S(n)>>>(n->g, n->vad, n->vad, n->red);
            const double nrm = std::sqrt(read_partials(n, blocks_for(n->g.vh)));
            if (den > 0.0) lam = num / den;
            if (!(nrm > 0.0)) break;
            pt_scale_kernel<<<blocks_for(n->g.vh), kBlock, 0, S(n)>>>(n->g, n->va, n->vad, (float)(1.0 / nrm));
        }
        const double lmax = 1.25 * std::max(lam, 1e-6);
        const double alpha = 4.0 / lmax, beta = -10.0 / (3.0 * lmax * lmax);
        const double m2 = h->mass * h->mass;
        n->w_host.assign(nw, make_float2(0.f, 0.f));
        std::mt19937_64 rng(seed);
        std::normal_distribution<float> nd(0.f, 1.f);
        for (int l = 0; l < kLayers; ++l) {
            const int cin = kChan[l], cout = kChan[l + 1];
            const float sc = 1e-4f / std::sqrt((float)(kPaths * cin));  // symmetry breaking only
            for (int k = 0; k < kPaths * cin * cout; ++k)
                n->w_host[layer_offset(l) + k] = make_float2(sc * nd(rng), sc * nd(rng));
        }
        auto W = [&](int l, int p, int o, int i) -> float2& {
            return n->w_host[layer_offset(l) + (p * kChan[l + 1] + o) * kChan[l] + i];
        };
        // self-adjoint form M = L1^dag L2 L1: L1 = (r; D r), L2 = diag(alpha + beta m^2, beta),
        // L3 = L1^dag = (r, -D .): M r = (alpha + beta m^2) r - beta D D r = alpha r + beta A_fat r
        W(0, 0, 0, 0).x += 1.f;                       // channel 0: r
        W(1, 0, 0, 0).x += (float)(alpha + beta * m2);
        W(1, 0, 1, 1).x += (float)beta;
        W(2, 0, 0, 0).x += 1.f;                       // output: channel 0 ...
        for (int mu = 0; mu < 4; ++mu) {
            W(0, 1 + 2 * mu, 1, 0).x += 1.f;           // channel 1: D r
            W(0, 2 + 2 * mu, 1, 0).x -= 1.f;
            W(2, 1 + 2 * mu, 0, 1).x -= 1.f;           // ... - D (channel 1)
            W(2, 2 + 2 * mu, 0, 1).x += 1.f;
        }
        upload_weights(n);
        pt_tie_kernel<<<1, 256, 0, S(n)>>>(n->w);  // the noise, too
        pcheck(n, cudaGetLastError(), "ptnet create");
        handle_end(h);
        *out = n;
        return STAG_OK;
    } catch (const PFail& f) {
        destroy_net(n);
        return f.code;
    } catch (const HandleError& f) {
        destroy_net(n);
        return f.code;
    } catch (...) {
        destroy_net(n);
        return STAG_ERR_CUDA;
    }
}

int64_t stag_ptnet_num_weights(const stag_ptnet* n) { return n ? n_weights() : 0; }

int stag_ptnet_set_weights(stag_ptnet* n, const double* w, int64_t count) {
    if (!n || !w || count != n_weights()) return STAG_ERR_INVALID_ARG;
    try {
        for (int k = 0; k < n_weights(); ++k) n->w_host[k] = make_float2((float)w[2 * k], (float)w[2 * k + 1]);
        upload_weights(n);
        pcheck(n, cudaStreamSynchronize(S(n)), "sync");
        return STAG_OK;
    } catch (const PFail& f) {
        return f.code;
    }
}

int stag_ptnet_get_weights(stag_ptnet* n, double* w, int64_t count) {
    if (!n || !w || count != n_weights()) return STAG_ERR_INVALID_ARG;
    try {
        download_weights(n);
        for (int k = 0; k < n_weights(); ++k) {
            w[2 * k] = n->w_host[k].x;
            w[2 * k + 1] = n->w_host[k].y;
        }
        return STAG_OK;
    } catch (const PFail& f) {
        return f.code;
    }
}

int stag_ptnet_apply(stag_ptnet* n, const double* r_even, double* z_even) {
    if (!n || !r_even || !z_even) return STAG_ERR_INVALID_ARG;
    stag_handle* h = n->h;
    try {
        handle_begin(h);
        const Geom& g = n->g;
        const bool out_dev = handle_is_device_ptr(h, z_even);
        const double* src = r_even;
        if (!handle_is_device_ptr(h, r_even)) {
            pcheck(n, cudaMemcpyAsync(h->io_a, r_even, (size_t)3 * g.vh * sizeof(double2), cudaMemcpyHostToDevice, S(n)), "copy r");
            src = h->io_a;
        }
        launch_pack_vec(g, src, n->fr, S(n));
        if (n->inf_form == STAG_PTNET_COLLAPSED) {
            apply_collapsed(n, n->fr, n->fz);
        } else {
            double d3[3];
            dots(n, n->fr, n->fr, nullptr, d3);
            const double rn = std::sqrt(d3[0]);
            if (infer_bf16(n))
                apply_net<__nv_bfloat162>(n, n->fr, rn, n->fz);
            else
                apply_net<float2>(n, n->fr, rn, n->fz);
        }
        launch_unpack_vec(g, n->fz, out_dev ? z_even : h->io_b, S(n));
        if (!out_dev)
            pcheck(n, cudaMemcpyAsync(z_even, h->io_b, (size_t)3 * g.vh * sizeof(double2), cudaMemcpyDeviceToHost, S(n)), "copy z");
        pcheck(n, cudaGetLastError(), "ptnet apply");
        check_tc(n);
        handle_end(h);
        return STAG_OK;
    } catch (const PFail& f) {
        return f.code;
    } catch (const HandleError& f) {
        return f.code;
    }
}

int stag_ptnet_loss_grad(stag_ptnet* n, const double* r_even, const double* e_even, double* loss, double* grad) {
    if (!n || !r_even || !e_even) return STAG_ERR_INVALID_ARG;
    stag_handle* h = n->h;
    try {
        handle_begin(h);
        const Geom& g = n->g;
        for (int k = 0; k < 2; ++k) {
            const double* v = k == 0 ? r_even : e_even;
            if (!handle_is_device_ptr(h, v)) {
                pcheck(n, cudaMemcpyAsync(h->io_a, v, (size_t)3 * g.vh * sizeof(double2), cudaMemcpyHostToDevice, S(n)), "copy");
                v = h->io_a;
            }
            launch_pack_vec(g, v, n->fr, S(n));
            void* slot = k == 0 ? n->scratch_r : n->scratch_e;
            if (is_bf16(n))
                pt_store_slot_kernel<double2, __nv_bfloat162><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, n->fr, 1.0, static_cast<__nv_bfloat162*>(slot));
            else
                pt_store_slot_kernel<double2, float2><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, n->fr, 1.0, static_cast<float2*>(slot));
        }
        pcheck(n, cudaMemsetAsync(n->grad, 0, n_weights() * sizeof(float2), S(n)), "zero gradients");
        double L;
        if (is_bf16(n)) {
            const double eae = slot_energy<__nv_bfloat162>(n, n->scratch_e);
            L = sample_step<__nv_bfloat162>(n, n->scratch_r, n->scratch_e, eae);
        } else {
            const double eae = slot_energy<float2>(n, n->scratch_e);
            L = sample_step<float2>(n, n->scratch_r, n->scratch_e, eae);
        }
        if (loss) *loss = L;
        if (grad) {
            std::vector<float2> gh(n_weights());
            pcheck(n, cudaMemcpyAsync(gh.data(), n->grad, gh.size() * sizeof(float2), cudaMemcpyDeviceToHost, S(n)), "read gradients");
            pcheck(n, cudaStreamSynchronize(S(n)), "sync");
            for (int k = 0; k < n_weights(); ++k) {
                grad[2 * k] = gh[k].x;
                grad[2 * k + 1] = gh[k].y;
            }
        }
        handle_end(h);
        return STAG_OK;
    } catch (const PFail& f) {
        return f.code;
    } catch (const HandleError& f) {
        return f.code;
    }
}

int stag_ptnet_add_pairs(stag_ptnet* n, int32_t n_sources, const double* const* sources, int32_t stride,
                         double min_rel_residual, int32_t max_pairs, int32_t* n_pairs) {
    if (!n || !sources || n_sources < 1 || stride < 1 || max_pairs < 0) return STAG_ERR_INVALID_ARG;
    stag_handle* h = n->h;
    if (h->opt.inner != STAG_INNER_NONE) {
        h->err = "training pairs come from the plain CG solver (inner = NONE)";
        return STAG_ERR_INVALID_ARG;
    }
    const stag_options saved = h->opt;
    int code = STAG_OK;
    std::vector<double2*> xsnap;
    try {
        handle_begin(h);
        const Geom& g = n->g;
        const size_t vb = (size_t)3 * g.vs * sizeof(double2);
        // blocks of `stride` iterations: one snapshot per block
        if (h->graph) {
            cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
        }
        h->opt.check_interval = stride;
        for (int sidx = 0; sidx < n_sources && (int)n->pairs_r.size() < max_pairs; ++sidx) {
            const double* src = sources[sidx];
            if (!handle_is_device_ptr(h, src)) {
                pcheck(n, cudaMemcpyAsync(h->io_a, src, (size_t)3 * g.vh * sizeof(double2), cudaMemcpyHostToDevice, S(n)), "copy source");
                src = h->io_a;
            }
            launch_pack_vec(g, src, h->b, S(n));
            pcheck(n, cudaMemsetAsync(h->x, 0, vb, S(n)), "zero x");
            launch_norm2_diff(g, h->b, nullptr, h->scal, h->partials, S(n));
            pcheck(n, cudaMemcpyAsync(h->scal_host, h->scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, S(n)), "read");
            pcheck(n, cudaStreamSynchronize(S(n)), "sync");
            const double bnorm2 = h->scal_host->red_out;
            if (!(bnorm2 > 0.0)) continue;
            std::vector<std::pair<void*, double>> rs;  // (r slot, 1/|r|) of this solve
            const bool ff = h->fatff != nullptr && h->opt.arith == STAG_ARITH_FF;
            h->block_hook = [&]() {
                const double rel2 = h->scal_host->delta_new / bnorm2;
                if (h->scal_host->done || rel2 < min_rel_residual * min_rel_residual) return;
                if ((int)(n->pairs_r.size() + rs.size()) >= max_pairs) return;
                const double inv = 1.0 / std::sqrt(h->scal_host->delta_new);
                void* slot = palloc(n, slot_bytes(n), "allocate pair");
                if (is_bf16(n)) {
                    if (ff)
                        pt_store_slot_kernel<float4, __nv_bfloat162><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, reinterpret_cast<const float4*>(h->r), inv, static_cast<__nv_bfloat162*>(slot));
                    else
                        pt_store_slot_kernel<double2, __nv_bfloat162><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, h->r, inv, static_cast<__nv_bfloat162*>(slot));
                } else {
                    if (ff)
                        pt_store_slot_kernel<float4, float2><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, reinterpret_cast<const float4*>(h->r), inv, static_cast<float2*>(slot));
                    else
                        pt_store_slot_kernel<double2, float2><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, h->r, inv, static_cast<float2*>(slot));
                }
                double2* xs = static_cast<double2*>(palloc(n, vb, "allocate snapshot"));
                pcheck(n, cudaMemcpyAsync(xs, h->x, vb, cudaMemcpyDeviceToDevice, S(n)), "snapshot x");
                xsnap.push_back(xs);
                rs.push_back({slot, inv});
            };
            stag_solve_info info{};
            const int st = handle_solve_packed(h, bnorm2, 1e-10, 0, info);
            h->block_hook = nullptr;
            if (st != STAG_OK) pfail(n, st, "training-pair solve did not converge");
            // e_k = (x* - x_k) / |r_k|
            for (size_t k = 0; k < rs.size(); ++k) {
                void* slot = palloc(n, slot_bytes(n), "allocate pair");
                if (is_bf16(n))
                    pt_store_diff_kernel<__nv_bfloat162><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, h->x, xsnap[k], rs[k].second, static_cast<__nv_bfloat162*>(slot));
                else
                    pt_store_diff_kernel<float2><<<blocks_for(g.vh), kBlock, 0, S(n)>>>(g, h->x, xsnap[k], rs[k].second, static_cast<float2*>(slot));
                n->pairs_r.push_back(rs[k].first);
                n->pairs_e.push_back(slot);
                n->pairs_eae.push_back(is_bf16(n) ? slot_energy<__nv_bfloat162>(n, slot) : slot_energy<float2>(n, slot));
            }
            for (double2* p : xsnap) cudaFree(p);
            for (double2* p : xsnap) n->device_bytes -= (long long)vb;
            xsnap.clear();
        }
        pcheck(n, cudaGetLastError(), "training pairs");
        handle_end(h);
    } catch (const PFail& f) {
        code = f.code;
    } catch (const HandleError& f) {
        code = f.code;
    }
    h->block_hook = nullptr;
    for (double2* p : xsnap) cudaFree(p);
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->opt = saved;
    if (n_pairs) *n_pairs = (int32_t)n->pairs_r.size();
    return code;
}

int stag_ptnet_train(stag_ptnet* n, int32_t epochs, int32_t batch, double lr, uint64_t seed, double* epoch_loss) {
    if (!n || epochs < 0 || batch < 1 || !(lr > 0.0)) return STAG_ERR_INVALID_ARG;
    if (n->pairs_r.empty()) {
        n->err = "no training pairs";
        return STAG_ERR_INVALID_ARG;
    }
    try {
        handle_begin(n->h);
        const int np = (int)n->pairs_r.size();
        const int nw = n_weights();
        std::vector<int> order(np);
        std::iota(order.begin(), order.end(), 0);
        std::mt19937_64 rng(seed);
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        for (int ep = 0; ep < epochs; ++ep) {
            std::shuffle(order.begin(), order.end(), rng);
            double total = 0.0;
            for (int s0 = 0; s0 < np; s0 += batch) {
                const int s1 = std::min(np, s0 + batch);
                pcheck(n, cudaMemsetAsync(n->grad, 0, nw * sizeof(float2), S(n)), "zero gradients");
                for (int s = s0; s < s1; ++s) {
                    const int k = order[s];
                    total += is_bf16(n) ? sample_step<__nv_bfloat162>(n, n->pairs_r[k], n->pairs_e[k], n->pairs_eae[k])
                                        : sample_step<float2>(n, n->pairs_r[k], n->pairs_e[k], n->pairs_eae[k]);
                }
                n->adam_t += 1;
                const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
                pt_adam_kernel<<<blocks_for(2 * nw), kBlock, 0, S(n)>>>(reinterpret_cast<float*>(n->w),
                                                                        reinterpret_cast<const float*>(n->grad),
                                                                        n->adam_m, n->adam_v, 2 * nw,
                                                                        2.f / (float)(s1 - s0), (float)lr, b1, b2,
                                                                        c1, c2, eps);
                pt_tie_kernel<<<1, 256, 0, S(n)>>>(n->w);
            }
            if (epoch_loss) epoch_loss[ep] = total / np;
        }
        pcheck(n, cudaGetLastError(), "training");
        check_tc(n);
        download_weights(n);
        handle_end(n->h);
        return STAG_OK;
    } catch (const PFail& f) {
        return f.code;
    } catch (const HandleError& f) {
        return f.code;
    }
}

int stag_ptnet_dataset_loss(stag_ptnet* n, double* loss) {
    if (!n || !loss) return STAG_ERR_INVALID_ARG;
    if (n->pairs_r.empty()) return STAG_ERR_INVALID_ARG;
    try {
        handle_begin(n->h);
        double total = 0.0;
        for (size_t k = 0; k < n->pairs_r.size(); ++k)
            total += is_bf16(n) ? forward_energy<__nv_bfloat162>(n, n->pairs_r[k], n->pairs_e[k], n->pairs_eae[k])
                                : forward_energy<float2>(n, n->pairs_r[k], n->pairs_e[k], n->pairs_eae[k]);
        *loss = total / n->pairs_r.size();
        handle_end(n->h);
        return STAG_OK;
    } catch (const PFail& f) {
        return f.code;
    } catch (const HandleError& f) {
        return f.code;
    }
}

int stag_ptnet_set_inference_precision(stag_ptnet* n, int32_t precision) {
    if (!n || (precision != STAG_ARITH_BF16 && precision != STAG_ARITH_F32)) return STAG_ERR_INVALID_ARG;
    n->inf_prec = precision;
    return STAG_OK;
}

int stag_ptnet_set_inference_form(stag_ptnet* n, int32_t form) {
    if (!n || (form != STAG_PTNET_COLLAPSED && form != STAG_PTNET_LAYERED)) return STAG_ERR_INVALID_ARG;
    n->inf_form = form;
    return STAG_OK;
}

int stag_ptnet_use_tensor_cores(stag_ptnet* n, int32_t enable) {
    if (!n) return STAG_ERR_INVALID_ARG;
    n->use_tc = enable != 0;
    return STAG_OK;
}

int stag_ptnet_num_pairs(const stag_ptnet* n) { return n ? (int)n->pairs_r.size() : 0; }

const char* stag_ptnet_last_error(const stag_ptnet* n) { return n ? n->err.c_str() : "NULL network"; }

int stag_ptnet_destroy(stag_ptnet* n) {
    destroy_net(n);
    return STAG_OK;
}

}  // extern "C"
