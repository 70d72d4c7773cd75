// stag_kernels.h - host-side launchers of the library's kernels (internal).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "stag_internal.cuh"

namespace stag {

enum Epilogue {
    EPI_PLAIN = 0,  // out = D_{P,1-P} in
    EPI_AXPY = 1,   // out = m2 * src - D_{P,1-P} in             (m2 from the launch)
    EPI_CG = 2      // out = scal->m2 * src - D in, + Re(src^dag out) -> scal->pAp, alpha
};

struct LinkSet {
    const double2* fat64;  // F64 SoA links (always present)
    const double2* lng64;  // nullptr: no Naik term
    const float4* fatff;   // FF SoA links (nullptr unless FF arithmetic is enabled)
    const float4* lngff;   // FF Naik links: [2][4][9][vs], or [2][4][6][vs] when lng_inv_scale_ff != 0
    float2 lng_inv_scale_ff = make_float2(0.f, 0.f);  // 1 / scale of the two-row Naik links, float-float
};

// ---- packing (pack.cu)
// AoS links [Lt][Lz][Ly][Lx][4][3][3] complex128 (device) -> SoA with eta folded,
// in FP64 and, where the pointer is not null, float-float, FP32, FP16 and BF16.
void launch_pack_links(const Geom& g, const double* aos, double2* soa64, float4* soaff,
                       float2* soa32, __half2* soa16, __nv_bfloat162* soab16, cudaStream_t s);
// AoS links -> float-float [2][4][6][vs]: the first two rows, eta folded
void launch_pack_links_ff_rows2(const Geom& g, const double* aos, float4* soaff_r, cudaStream_t s);
// max over the AoS links L of |L^dag L / c^2 - 1| and |det L / c^3 - 1| into *maxdev
// (a float's bits in an unsigned int, zeroed by the caller)
void launch_check_scaled_su3(const Geom& g, const double* aos, double c, unsigned int* maxdev, cudaStream_t s);
// AoS links -> FP32 [2][4][6][vs]: the first two rows, eta folded (12-parameter form)
void launch_pack_links_rows2(const Geom& g, const double* aos, float2* soa32r, cudaStream_t s);
// ABI vector [vh][3] complex128 (device) <-> F64 SoA [3][vs]
void launch_pack_vec(const Geom& g, const double* aos, double2* soa, cudaStream_t s);
void launch_unpack_vec(const Geom& g, const double2* soa, double* aos, cudaStream_t s);

// ---- Dirac kernels (dslash.cu)
void launch_dslash_f64(const Geom& g, int out_parity, const LinkSet& L, const double2* in,
                       double2* out, Epilogue epi, const double2* src, double m2,
                       CgScalars* scal, double* partials, cudaStream_t s);
// FP64 half-Dslash over output sites [i0, i1) only (no reduction epilogue)
void launch_dslash_f64_range(const Geom& g, int out_parity, const LinkSet& L, const double2* in, double2* out,
                             Epilogue epi, const double2* src, double m2, int i0, int i1, cudaStream_t s);
void launch_dslash_ff(const Geom& g, int out_parity, const LinkSet& L, const float4* in,
                      float4* out, Epilogue epi, const float4* src, double m2, CgScalars* scal,
                      double* partials, cudaStream_t s);

// One system's half-Dslash for launch_dslash_list: links, vectors and output in
// the arithmetic's layouts (FF: float4, F64: double2); nine-entry Naik links or none.
struct SysDirac {
    Geom g;
    int P;             // output parity
    const void* fat;   // [2][4][9][vs]
    const void* lng;   // [2][4][9][vs] or nullptr
    const void* in;    // [3][vs], parity 1-P
    void* out;         // [3][vs], parity P
    const void* src;   // [3][vs], parity P (EPI_AXPY)
    double m2;
    float2 m2_ff;
};
// The half-Dslash (EPI_PLAIN or EPI_AXPY) of the systems list[0 .. *count) (device
// arrays; prefix[j] = first tile of entry j in tiles of kBlock sites, prefix[*count] =
// all tiles) by `grid` blocks striding over the tiles; ff: float-float, else FP64.
void launch_dslash_list(bool ff, Epilogue epi, const SysDirac* sys, const int* list, const int* prefix,
                        const int* count, int grid, cudaStream_t s);

// low-precision Dirac kernels of the mixed-precision solver (same epilogues);
// lng_inv_scale != 0: the FP32 Naik links are two rows per link ([2][4][6][vs],
// eta folded) of scale x SU(3), lng_inv_scale = 1 / scale, the third row rebuilt
void launch_dslash_f32(const Geom& g, int out_parity, const float2* fat, const float2* lng,
                       const float2* in, float2* out, Epilogue epi, const float2* src, double m2,
                       CgScalars* scal, double* partials, cudaStream_t s, float lng_inv_scale = 0.f);
void launch_dslash_h16(const Geom& g, int out_parity, const __half2* fat, const __half2* lng,
                       const __half2* in, __half2* out, Epilogue epi, const __half2* src, double m2,
                       CgScalars* scal, double* partials, cudaStream_t s);
// FP32 with 12-parameter links ([2][4][6][vs], one-hop only): row 2 rebuilt in the kernel
void launch_dslash_f32r12(const Geom& g, int out_parity, const float2* fat_rows2, const float2* in, float2* out,
                          Epilogue epi, const float2* src, double m2, CgScalars* scal, double* partials,
                          cudaStream_t s);
// FP16-stored links, FP32 vectors and arithmetic
void launch_dslash_f32l16(const Geom& g, int out_parity, const __half2* fat, const __half2* lng, const float2* in,
                          float2* out, Epilogue epi, const float2* src, double m2, CgScalars* scal, double* partials,
                          cudaStream_t s);
void launch_dslash_b16(const Geom& g, int out_parity, const __nv_bfloat162* fat, const __nv_bfloat162* lng,
                       const __nv_bfloat162* in, __nv_bfloat162* out, Epilogue epi, const __nv_bfloat162* src,
                       double m2, CgScalars* scal, double* partials, cudaStream_t s);

// ---- CG vector kernels and reductions (blas.cu)
// kBlock-thread blocks that fill every SM of the current device once (grid of
// the grid-stride update kernels, whose grid reduction then has few partials)
int resident_wave_blocks();
// start of one run of Fig. 1 (iter = 0, done = 0, threshold, m^2, max_iter)
void launch_cg_reset(CgScalars* scal, double threshold, double m2, long long max_iter,
                     cudaStream_t s);
// FP64 vectors.  r = b - Ad; d = r; delta_new = delta_0 = |r|^2; done if converged
void launch_cg_init(const Geom& g, const double2* b, const double2* ad, double2* r, double2* d,
                    CgScalars* scal, double* partials, cudaStream_t s);
// x += alpha d; r -= alpha Ad; delta_old = delta_new; delta_new = |r|^2; beta; iter++; done
void launch_cg_update_xr(const Geom& g, double2* x, double2* r, const double2* d, const double2* ad,
                         CgScalars* scal, double* partials, cudaStream_t s);
// d = r + beta d
void launch_cg_update_d(const Geom& g, const double2* r, double2* d, CgScalars* scal, cudaStream_t s);
// float-float vectors: the same steps; x is accumulated in x_ff (zeroed by init)
void launch_cg_init_ff(const Geom& g, const double2* b, const double2* ad, float4* r, float4* d,
                       float4* xff, CgScalars* scal, double* partials, cudaStream_t s);
void launch_cg_update_xr_ff(const Geom& g, float4* xff, float4* r, const float4* d, const float4* ad,
                            CgScalars* scal, double* partials, cudaStream_t s);
void launch_cg_update_d_ff(const Geom& g, const float4* r, float4* d, CgScalars* scal, cudaStream_t s);
// x += x_ff (FP64), x_ff = 0
void launch_fold_x(const Geom& g, double2* x, float4* xff, cudaStream_t s);
// scal->red_out = |a - b|^2 (b may be nullptr: |a|^2)
void launch_norm2_diff(const Geom& g, const double2* a, const double2* b, CgScalars* scal,
                       double* partials, cudaStream_t s);
// ---- mixed-precision solver (blas_lo.cu)
// r = b - Ax (Ax FP64 or float-float); scal->red_out = |r|^2
void launch_residual(const Geom& g, const double2* b, const void* ax, bool ax_ff, double2* r,
                     CgScalars* scal, double* partials, cudaStream_t s);
// start of an inner run: delta, threshold (inner units), m^2, bounds of the replacement rule
void launch_lo_reset(CgScalars* scal, double delta, double threshold, double m2, long long max_iter,
                     long long rel_interval, double rel_delta, cudaStream_t s);
// r_lo = inv_sigma * r64; d_lo = r_lo (first) or r_lo + beta d_lo; y = 0
template <class V>
void launch_lo_set_residual(const Geom& g, const double2* r64, V* r, V* d, float2* y, double inv_sigma,
                            double beta, bool first, cudaStream_t s);
template <class V>
void launch_lo_update_xr(const Geom& g, float2* y, V* r, const V* d, const V* ad, CgScalars* scal,
                         double* partials, cudaStream_t s);
template <class V>
void launch_lo_update_d(const Geom& g, const V* r, V* d, CgScalars* scal, cudaStream_t s);
// out = scale * in, F64 SoA <-> low precision SoA
template <class V>
void launch_to_lo(const Geom& g, const double2* in, V* out, double scale, cudaStream_t s);
template <class V>
void launch_from_lo(const Geom& g, const V* in, double2* out, double scale, cudaStream_t s);
// x += sigma * y (FP64); y = 0
void launch_lo_fold_y(const Geom& g, double2* x, float2* y, double sigma, cudaStream_t s);

// F64 SoA vector <-> FF SoA vector
void launch_to_ff(const Geom& g, const double2* in, float4* out, cudaStream_t s);
void launch_from_ff(const Geom& g, const float4* in, double2* out, cudaStream_t s);

}  // namespace stag
