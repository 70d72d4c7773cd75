// pack.cu - layout kernels: eta folding of the links (Sec. 2, after Eq. (5)),
// AoS -> structure-of-arrays transposition for coalesced access (Sec. 3.1),
// the low-precision link copies (FP32, FP16, BF16) of the mixed-precision solver, and the
// ABI <-> internal vector conversions.
#include "stag_kernels.h"
#include "ff.cuh"

namespace stag {

// One thread per (site, direction), direction fastest, so that a warp reads
// contiguous AoS links (the input may be host memory read over the host link).
// Reads the 9 complex entries of U_mu(x) (144 contiguous bytes), multiplies by
// eta_mu(x) and scatters them into the 9 planes of its parity.
__global__ void __launch_bounds__(kBlock) pack_links_kernel(Geom g, const double2* __restrict__ aos,
                                                            double2* __restrict__ soa64,
                                                            float4* __restrict__ soaff,
                                                            float2* __restrict__ soa32,
                                                            __half2* __restrict__ soa16,
                                                            __nv_bfloat162* __restrict__ soab16) {
    const long long V = 2LL * g.vh;
    const long long idx = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (idx >= 4 * V) return;
    const int mu = (int)(idx & 3);
    const int lex = (int)(idx >> 2);
    const int x = lex % g.lx;
    int r = lex / g.lx;
    const int y = r % g.ly;
    r /= g.ly;
    const int z = r % g.lz;
    const int t = r / g.lz;
    const int P = (x + y + z + t) & 1;
    const int cb = lex >> 1;
    int phase_sum = 0;
    if (mu >= 1) phase_sum += x;
    if (mu >= 2) phase_sum += y;
    if (mu >= 3) phase_sum += z;
    const double eta = (phase_sum & 1) ? -1.0 : 1.0;
    const double2* src = aos + ((size_t)lex * 4 + mu) * 9;
    const size_t vs = (size_t)g.vs;
    const size_t base = ((size_t)(P * 4 + mu) * 9) * vs + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 u = src[k];
        u.x *= eta;
        u.y *= eta;
        soa64[base + k * vs] = u;
        if (soaff) soaff[base + k * vs] = ff_from_complex(u);
        if (soa32) soa32[base + k * vs] = make_float2((float)u.x, (float)u.y);
        if (soa16) soa16[base + k * vs] = __floats2half2_rn((float)u.x, (float)u.y);
        if (soab16) soab16[base + k * vs] = __floats2bfloat162_rn((float)u.x, (float)u.y);
    }
}

void launch_pack_links(const Geom& g, const double* aos, double2* soa64, float4* soaff,
                       float2* soa32, __half2* soa16, __nv_bfloat162* soab16, cudaStream_t s) {
    const long long n = 8LL * g.vh;
    const int blocks = (int)((n + kBlock - 1) / kBlock);
    pack_links_kernel<<<blocks, kBlock, 0, s>>>(g, reinterpret_cast<const double2*>(aos), soa64,
                                                soaff, soa32, soa16, soab16);
}

// Links with the first two rows only ([parity][mu][6][vs], eta folded), in FP32
// and/or float-float: the third row of an SU(3) matrix (times a scale) is the
// conjugate cross product of the first two (Sec. 3.3), rebuilt in the Dirac
// kernel.  Direction fastest, as above.
__global__ void __launch_bounds__(kBlock) pack_links_rows2_kernel(Geom g, const double2* __restrict__ aos,
                                                                  float2* __restrict__ soa32r,
                                                                  float4* __restrict__ soaffr) {
    const long long V = 2LL * g.vh;
    const long long idx = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (idx >= 4 * V) return;
    const int mu = (int)(idx & 3);
    const int lex = (int)(idx >> 2);
    const int x = lex % g.lx;
    int r = lex / g.lx;
    const int y = r % g.ly;
    r /= g.ly;
    const int z = r % g.lz;
    const int t = r / g.lz;
    const int P = (x + y + z + t) & 1;
    const int cb = lex >> 1;
    int phase_sum = 0;
    if (mu >= 1) phase_sum += x;
    if (mu >= 2) phase_sum += y;
    if (mu >= 3) phase_sum += z;
    const double eta = (phase_sum & 1) ? -1.0 : 1.0;
    const double2* src = aos + ((size_t)lex * 4 + mu) * 9;
    const size_t vs = (size_t)g.vs;
    const size_t base = ((size_t)(P * 4 + mu) * 6) * vs + cb;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double2 u = make_double2(eta * src[k].x, eta * src[k].y);
        if (soa32r) soa32r[base + k * vs] = make_float2((float)u.x, (float)u.y);
        if (soaffr) soaffr[base + k * vs] = ff_from_complex(u);
    }
}

void launch_pack_links_rows2(const Geom& g, const double* aos, float2* soa32r, cudaStream_t s) {
    const long long n = 8LL * g.vh;
    pack_links_rows2_kernel<<<(int)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(
        g, reinterpret_cast<const double2*>(aos), soa32r, nullptr);
}

void launch_pack_links_ff_rows2(const Geom& g, const double* aos, float4* soaffr, cudaStream_t s) {
    const long long n = 8LL * g.vh;
    pack_links_rows2_kernel<<<(int)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(
        g, reinterpret_cast<const double2*>(aos), nullptr, soaffr);
}

// max over all links L (AoS, one thread per link) of the largest of
// |(L^dag L)_ij / c^2 - delta_ij| and |det L / c^3 - 1|: zero up to rounding
// exactly when every L / c is in SU(3).  A non-finite deviation counts as
// 1e30.  The maximum of non-negative floats is taken on their bit patterns.
__global__ void __launch_bounds__(kBlock) check_scaled_su3_kernel(long long nlinks, const double2* __restrict__ aos,
                                                                  double inv_c, unsigned int* __restrict__ maxdev) {
    const long long idx = (long long)blockIdx.x * kBlock + threadIdx.x;
    float dev = 0.f;
    if (idx < nlinks) {
        double2 u[9];
        double size = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            u[k] = make_double2(aos[idx * 9 + k].x * inv_c, aos[idx * 9 + k].y * inv_c);
            size += fabs(u[k].x) + fabs(u[k].y);
        }
        double d = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                double re = (i == j) ? -1.0 : 0.0, im = 0.0;  // sum_k conj(u_ki) u_kj - delta_ij
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double2 a = u[3 * k + i], b = u[3 * k + j];
                    re += a.x * b.x + a.y * b.y;
                    im += a.x * b.y - a.y * b.x;
                }
                d = fmax(d, sqrt(re * re + im * im));
            }
        }
        // det = u0 (u4 u8 - u5 u7) - u1 (u3 u8 - u5 u6) + u2 (u3 u7 - u4 u6)
        auto mul = [](double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
        auto sub2 = [](double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); };
        const double2 m0 = mul(u[0], sub2(mul(u[4], u[8]), mul(u[5], u[7])));
        const double2 m1 = mul(u[1], sub2(mul(u[3], u[8]), mul(u[5], u[6])));
        const double2 m2 = mul(u[2], sub2(mul(u[3], u[7]), mul(u[4], u[6])));
        const double dre = m0.x - m1.x + m2.x - 1.0, dim = m0.y - m1.y + m2.y;
        d = fmax(d, sqrt(dre * dre + dim * dim));
        // fmax drops NaN operands: entries that are non-finite or large enough to
        // overflow the products above fail through size
        dev = (d < 1e30 && size < 1e100) ? (float)d : 1e30f;
    }
    const unsigned int w = __reduce_max_sync(0xffffffffu, __float_as_uint(dev));
    if ((threadIdx.x & 31) == 0 && w != 0u) atomicMax(maxdev, w);
}

void launch_check_scaled_su3(const Geom& g, const double* aos, double c, unsigned int* maxdev, cudaStream_t s) {
    const long long n = 8LL * g.vh;  // V sites x 4 directions
    check_scaled_su3_kernel<<<(int)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(
        n, reinterpret_cast<const double2*>(aos), 1.0 / c, maxdev);
}

__global__ void __launch_bounds__(kBlock) pack_vec_kernel(Geom g, const double2* __restrict__ aos,
                                                          double2* __restrict__ soa) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vs) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        soa[c * vs + i] = i < g.vh ? aos[(size_t)i * 3 + c] : make_double2(0.0, 0.0);
}

__global__ void __launch_bounds__(kBlock) unpack_vec_kernel(Geom g, const double2* __restrict__ soa,
                                                            double2* __restrict__ aos) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.vh) return;
    const size_t vs = (size_t)g.vs;
#pragma unroll
    for (int c = 0; c < 3; ++c) aos[(size_t)i * 3 + c] = soa[c * vs + i];
}

void launch_pack_vec(const Geom& g, const double* aos, double2* soa, cudaStream_t s) {
    pack_vec_kernel<<<blocks_for(g.vs), kBlock, 0, s>>>(g, reinterpret_cast<const double2*>(aos), soa);
}

void launch_unpack_vec(const Geom& g, const double2* soa, double* aos, cudaStream_t s) {
    unpack_vec_kernel<<<blocks_for(g.vh), kBlock, 0, s>>>(g, soa, reinterpret_cast<double2*>(aos));
}

}  // namespace stag
