/*
 * stag.h - C ABI of the GB300 (sm_103a) staggered-fermion even-odd CG library.
 *
 * The library solves A x = b on the even sites of a 4-d periodic lattice with
 *     A = m^2 - D_eo D_oe                      (Sec. 2, Eq. (3) on even sites)
 *     D chi(x) = sum_mu U_mu(x) chi(x+mu) - U_mu(x-mu)^dag chi(x-mu)
 *              [+ sum_mu L_mu(x) chi(x+3mu) - L_mu(x-3mu)^dag chi(x-3mu)]
 *                                              (Sec. 2, Eqs. (4)-(5); Naik term optional)
 * with the staggered phase eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) multiplied
 * into every link by the library (Sec. 2, after Eq. (5)), by conjugate
 * gradient (Sec. 2, Fig. 1).  D carries no factor 1/2.
 *
 * Layouts (all complex numbers are interleaved (re, im) doubles):
 *   links   [Lt][Lz][Ly][Lx][mu=0..3 = x,y,z,t][3][3]   complex128, row-major 3x3,
 *           eta NOT folded in.  Size 4*V*9 complex = V*576 bytes.
 *   vectors [V/2][3] complex128 on the sites of one parity; sites are numbered
 *           in lexicographic order (x fastest), so the half-lattice index of a
 *           site is its lexicographic index / 2.  "Even" = (x+y+z+t) even.
 *
 * Pointers: every array argument may be host memory or device memory of the
 * current CUDA device; the library detects which (cudaPointerGetAttributes)
 * and stages host data through its own device buffers.  Arrays are owned by
 * the caller and are only accessed during the call.
 *
 * Streams: work is ordered after all work already enqueued on the stream set
 * with stag_set_stream (default: the legacy default stream), and every call
 * returns only after its work has completed.
 *
 * Errors: every call returns a STAG_* status; no C++ exception crosses the
 * ABI.  stag_last_error gives a message for the last failing call.  A handle
 * is not thread-safe.
 */
#ifndef STAG_H
#define STAG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    STAG_OK = 0,
    STAG_ERR_INVALID_ARG = 1,   /* bad pointer, extent, option or non-finite input */
    STAG_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    STAG_ERR_NOT_CONVERGED = 3, /* max_iter or max_restarts reached; x holds the last iterate */
    STAG_ERR_BREAKDOWN = 4,     /* d^dag A d <= 0 or non-finite inside CG */
    STAG_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
    STAG_ERR_OOM = 6            /* device allocation failed */
};

/* Arithmetic of the FP64-class Dirac kernels. */
enum {
    STAG_ARITH_F64 = 0, /* native FP64 fused multiply-add */
    STAG_ARITH_F32 = 2, /* FP32 links, vectors and arithmetic (stag_apply_A_prec only) */
    STAG_ARITH_F16 = 3, /* FP16-stored links and vectors, FP32 arithmetic (stag_apply_A_prec only) */
    STAG_ARITH_BF16 = 4, /* BF16-stored links and vectors (or network activations), FP32
                            arithmetic (stag_apply_A_prec and the learned preconditioner) */
    STAG_ARITH_FF = 1   /* float-float: each FP64 number held as an unevaluated sum of two
                           FP32 numbers (8 bytes, like FP64), products and sums formed with
                           error-free transformations (Dekker 1971; Knuth TAOCP vol. 2);
                           about 2^-48 relative rounding, FP32 pipelines */
};

/* Inner precision of the CG iteration.  NONE: the whole iteration in the
 * FP64-class arithmetic selected by `arith` (plain CG, Fig. 1).  F32 / F16 / BF16:
 * mixed-precision CG (the paper's stated next step, Sec. 5) - the iteration runs
 * on FP32 vectors and links (F32) or on FP16- or BF16-stored vectors and links
 * with FP32 arithmetic (F16, BF16), or on FP32 vectors with FP16-stored links
 * (F32_L16: the links carry most of the Dirac kernel's bytes, while the CG vectors
 * keep FP32's significand), and the iterated residual is replaced by the true residual
 * b - A x, computed in the FP64-class arithmetic, whenever it has dropped by
 * reliable_delta since the last replacement or after reliable_interval
 * iterations (reliable updates, Sleijpen & van der Vorst 1996).  x, b and the
 * CG scalars stay FP64. */
enum {
    STAG_INNER_NONE = 0,
    STAG_INNER_F32 = 1,
    STAG_INNER_F16 = 2,
    STAG_INNER_BF16 = 3,
    STAG_INNER_F32_L16 = 4  /* FP32 vectors and arithmetic, FP16-stored links */
};

/* Kernel ids for stag_kernel_stats. */
enum {
    STAG_KERNEL_DSLASH_OE = 0,  /* t = D_oe d (odd output)                               */
    STAG_KERNEL_DSLASH_EO = 1,  /* Ad = m^2 d - D_eo t (even output) + partial d^dag A d */
    STAG_KERNEL_UPDATE_XR = 2,  /* x += alpha d, r -= alpha Ad, partial r^dag r          */
    STAG_KERNEL_UPDATE_D = 3,   /* d = r + beta d                                        */
    STAG_KERNEL_COUNT = 4
};

typedef struct stag_handle stag_handle; /* opaque; owned by the library */

typedef struct {
    int32_t arith;          /* STAG_ARITH_*, Dirac arithmetic of the CG iteration (default F64) */
    int32_t check_interval; /* CG iterations between host convergence reads (default 32)     */
    int32_t max_restarts;   /* restarts of Fig. 1 from the current x when the true residual
                               exceeds tol (default 5)                                        */
    int32_t use_graphs;     /* capture check_interval iterations as one CUDA graph (default 1) */
    int32_t timing;         /* record CUDA events around every CG kernel (default 0);
                               disables graphs; read with stag_kernel_stats                    */
    int32_t inner;          /* STAG_INNER_*, precision of the CG iteration (default NONE)      */
    int32_t reliable_interval; /* mixed precision: most iterations between residual
                                  replacements (default 100)                                  */
    int32_t autotune;       /* batched solves: time the candidate RHS-block and block shapes and
                               keep the fastest (default 1); 0 = fixed shapes                  */
    double reliable_delta;  /* mixed precision: replace the residual once |r| < reliable_delta
                               times its maximum since the last replacement (default 0.1)     */
    int32_t link_recon;     /* 12: the FP32 inner iteration stores two rows of each link and
                               rebuilds the third as the conjugate cross product of the first
                               two, times eta (Sec. 3.3, Eq. for SU(3) reconstruction); needs
                               SU(3) links, the one-hop operator and inner = F32.  0 (default):
                               all nine entries.                                              */
    int32_t guard_bands;    /* 1: every device buffer of the handle lies between two guard bands
                               of 4096 bytes filled with a fixed byte, read back by
                               stag_check_guards (a check for writes past a buffer's ends,
                               for tests); 0 (default): none                                  */
    double long_scale;      /* long_recon = 12: the Naik links are long_scale x SU(3) (e.g. the
                               Naik coefficient times a product of SU(3) links); accepted for
                               1e-10 <= |long_scale| <= 1e18, where the float-float products
                               of two stored entries stay normal FP32 numbers               */
    int32_t long_recon;     /* 12: the float-float Dirac kernels store two rows of each Naik
                               link and rebuild the third as (eta / long_scale) times the
                               conjugate cross product of the first two (the 12-parameter
                               form of Sec. 3.3 for a scaled SU(3) matrix); with inner = F32
                               the FP32 Naik links of the mixed-precision iteration are two
                               rows too, the third rebuilt in FP32.  Needs arith = FF
                               and Naik links; stag_create_ex checks that every Naik link
                               divided by long_scale is unitary with determinant 1 (entries of
                               L^dag L / c^2 - 1 and det L / c^3 - 1 at most 1e-12) and fails
                               with STAG_ERR_INVALID_ARG otherwise.  The FP64 copy used for the
                               final residual check keeps all nine entries.  0 (default): all
                               nine entries.                                                  */
    int32_t reserved2;      /* 0 */
} stag_options;

typedef struct {
    int32_t iters;            /* CG iterations (all restarts)                              */
    int32_t restarts;         /* restarts of Fig. 1 after a true-residual check            */
    int32_t status;           /* the STAG_* status the call returned                       */
    int32_t reliable_updates; /* mixed precision: residual replacements                    */
    double true_rel_residual; /* |b - A x| / |b|, A applied in native FP64                 */
    double iter_rel_residual; /* sqrt(delta_new) / |b| of the last Fig. 1 iterate          */
    double time_ms;           /* wall time of the solve inside the call                     */
    int32_t fallbacks;        /* hand-overs to plain CG (flexible CG, mixed-precision safeguard) */
    int32_t reserved;
} stag_solve_info;

/* Fill *opt with the defaults.  Returns STAG_ERR_INVALID_ARG if opt is NULL. */
int stag_default_options(stag_options* opt);

/* Create a handle for the one-hop operator (Sec. 2, Eqs. (3)-(5)).
 * links: U_mu(x) in the link layout above (host or device), eta not folded;
 *        copied at create, so the caller may free it afterwards.
 * dims:  host array {Lx, Ly, Lz, Lt}; every extent even and >= 2, V/2 < 2^31.
 * mass:  the quark mass m of Eq. (3); must be finite.
 * On success *out holds a new handle (release with stag_destroy); on error
 * *out is NULL and the message is available from stag_last_error(NULL). */
int stag_create(stag_handle** out, const double* links, const int32_t dims[4], double mass);

/* As stag_create, with an optional Naik three-hop field (NULL = one-hop only)
 * and options (NULL = defaults).  fat plays the role of U in Eq. (5); naik_long
 * are the three-hop links L_mu(x) from x to x+3mu (eta not folded). */
int stag_create_ex(stag_handle** out, const double* fat, const double* naik_long,
                   const int32_t dims[4], double mass, const stag_options* opt);

/* Order the handle's work after the given cudaStream_t (NULL = legacy default stream). */
int stag_set_stream(stag_handle* h, void* cuda_stream);

/* Change m of Eq. (3); must be finite. */
int stag_set_mass(stag_handle* h, double mass);

/* Half of D (Sec. 2, Eq. (5)): out = D_{P,1-P} in, i.e. D restricted to output
 * sites of parity P = out_parity (0 even, 1 odd) acting on a vector of parity
 * 1-P.  in, out: [V/2][3] complex128, must not overlap.  Native FP64 arithmetic
 * unless the handle's arith is STAG_ARITH_FF. */
int stag_dslash(stag_handle* h, int32_t out_parity, const double* in, double* out);

/* out_even = A in_even = m^2 in - D_eo D_oe in (Sec. 2, Eq. (3)).  in, out:
 * [V/2][3] complex128 on even sites; must not overlap.  Arithmetic as for
 * stag_dslash. */
int stag_apply_A(stag_handle* h, const double* in_even, double* out_even);

/* As stag_apply_A (Sec. 2, Eq. (3)) in a chosen arithmetic: STAG_ARITH_F64
 * (always available), STAG_ARITH_FF (handle created with arith = FF),
 * STAG_ARITH_F32 / STAG_ARITH_F16 / STAG_ARITH_BF16 (handle created with inner =
 * F32 / F16 / BF16: the operator the mixed-precision iteration uses; FP16 vectors are scaled to unit
 * rms entries on the way in and back on the way out).  Returns
 * STAG_ERR_INVALID_ARG when the handle holds no links of that precision. */
int stag_apply_A_prec(stag_handle* h, int32_t arith, const double* in_even, double* out_even);

/* Solve A x = b by CG (Sec. 2, Fig. 1) to |b - A x| / |b| <= tol.
 * b_even: [V/2][3] source.  x_even: [V/2][3], on entry the initial guess (it
 * must be initialised, e.g. to zero), on exit the solution.
 * Fig. 1 runs until delta_new <= tol^2 |b|^2 (Fig. 1's eps^2 delta_0 when the
 * guess is zero) or max_iter total iterations (max_iter <= 0: N_dim = 3 V/2);
 * the true residual is then recomputed with native FP64 arithmetic and Fig. 1
 * restarts from the current x while it exceeds tol (at most max_restarts times).
 * Returns STAG_OK, STAG_ERR_NOT_CONVERGED (x holds the last iterate) or
 * STAG_ERR_BREAKDOWN; info (nullable) is filled in every case. */
int stag_cg_solve(stag_handle* h, const double* b_even, double* x_even, double tol,
                  int32_t max_iter, stag_solve_info* info);

/* Release the handle and its device memory.  NULL-safe. */
int stag_destroy(stag_handle* h);

/* Message of the last failing call on h (h = NULL: of the last failing create
 * on this thread).  Never NULL; valid until the next call on the handle. */
const char* stag_last_error(const stag_handle* h);

/* Accumulated CUDA-event time and launch count of one CG kernel (STAG_KERNEL_*),
 * recorded while the handle's timing option is on. */
int stag_kernel_stats(const stag_handle* h, int32_t kernel, double* total_ms, int64_t* launches);

/* Zero the kernel statistics. */
int stag_reset_stats(stag_handle* h);

/* Guard bands (opt.guard_bands = 1): *checked_bytes receives the bytes of all
 * the handle's guard bands and *bad_bytes those that no longer hold the fill
 * byte, i.e. were written by a kernel that ran past a buffer.  Synchronises the
 * handle's stream.  Returns STAG_ERR_INVALID_ARG when the handle has no guard
 * bands.  No counterpart in the paper: a test aid in place of a memory checker. */
int stag_check_guards(stag_handle* h, int64_t* checked_bytes, int64_t* bad_bytes);

/* Bytes of device memory the handle holds (0 for NULL). */
int64_t stag_device_bytes(const stag_handle* h);

/* Number of CUDA kernels the handle has launched since it was created (each
 * replay of a captured graph counts every kernel in it; 0 for NULL). */
int64_t stag_launch_count(const stag_handle* h);

/* ------------------------------------------------------------------ batches
 * Many independent systems A_k x_k = b_k (k = 0 .. n_sys-1) solved together.
 * No counterpart in the paper's single-system CG (Sec. 2, Fig. 1), whose method
 * each system follows.  Systems whose links (fat and Naik pointers), extents
 * and mass are equal share one packed field and run as right-hand sides of
 * multi-RHS Dirac kernels (each link is loaded once for a block of right-hand
 * sides); lattices of different sizes share every launch.  Each system runs the
 * mixed-precision CG (FP32 iteration, FP64 scalars) with its own reliable
 * updates in float-float arithmetic and a final true residual in native FP64.
 * The replacements are decided and applied on the device by a pass that
 * follows every iteration, so a system never waits for the host.  Blocks of
 * check_interval iterations of all systems, each with its pass, are one CUDA
 * graph; the host reads one word (the systems still running) per replay.  The
 * right-hand sides per thread and threads per block of each group are chosen
 * at create by timing the candidates' two Dirac launches of an iteration (the
 * D_oe and the reducing D_eo; the least sum wins; opt->autotune), cached per (extents,
 * Naik, RHS count) for the process and in the file STAG_AUTOTUNE_CACHE names;
 * STAG_AUTOTUNE_LOG names a file that receives every candidate's time.  The
 * candidates also include the traversals of a group's site tiles listed at
 * stag_batch_tuning. */
typedef struct stag_batch stag_batch;

/* fat, naik: n_sys link arrays (the link layout above; naik may be NULL, or
 * contain NULLs, for one-hop systems); dims: 4*n_sys extents; masses: n_sys.
 * Link arrays are copied at create.  opt: NULL = defaults, except
 * check_interval = 8; only check_interval, reliable_interval, reliable_delta
 * and autotune are used.  Besides the packed fields and the RHS vectors, the
 * batch holds three float-float work vectors per system for its true residuals. */
int stag_batch_create(stag_batch** out, int32_t n_sys, const double* const* fat, const double* const* naik,
                      const int32_t* dims, const double* masses, const stag_options* opt);

/* Order the batch's work after this cudaStream_t (NULL = legacy default stream). */
int stag_batch_set_stream(stag_batch* b, void* cuda_stream);

/* Solve every system to |b_k - A x_k| / |b_k| <= tol.  b[k], x[k]: [V_k/2][3]
 * complex128 (host or device); x[k] is the initial guess on entry.  max_iter
 * bounds each system's iterations (<= 0: unbounded).  infos (nullable): n_sys
 * entries; time_ms is the wall time of the whole batch.  Returns STAG_OK when
 * every system converged, else the first failing status. */
int stag_batch_solve(stag_batch* b, const double* const* bvec, double* const* xvec, double tol, int32_t max_iter,
                     stag_solve_info* infos);

/* out[k] = A_k in[k] with the batch's FP32 multi-RHS kernels (the operator of
 * the inner iteration; Sec. 2, Eq. (3)). */
int stag_batch_apply_A(stag_batch* b, const double* const* in, double* const* out);

/* The shapes the autotuner chose for system k's group and its measured D_oe time
 * (any output may be NULL); *traversal: how the blocks walk the site tiles
 * (0 contiguous runs per block, 1 a sweep by the blocks resident at once, all
 * on one narrow band of sites). */
int stag_batch_tuning(const stag_batch* b, int32_t system, int32_t* rhs_per_thread, int32_t* threads_per_block,
                      double* ms, int32_t* traversal);

/* Override the shape of system k's group (and so of every system in it):
 * rhs_per_thread in {1, 2, 4, 8}, at most the group's padded RHS count and at
 * least 1/32 of it (single-RHS groups: 1); threads_per_block in {64, 128, 256};
 * traversal in {0, 1}.  Returns STAG_ERR_INVALID_ARG for other values.
 * Used to run every candidate of the autotuner, e.g. in tests. */
int stag_batch_set_tuning(stag_batch* b, int32_t system, int32_t rhs_per_thread, int32_t threads_per_block,
                          int32_t traversal);

/* Message of the batch's last failing call (b = NULL: of the last failing create). */
const char* stag_batch_last_error(const stag_batch* b);

/* Bytes of device memory the batch holds (0 for NULL). */
int64_t stag_batch_device_bytes(const stag_batch* b);

/* Release the batch.  NULL-safe. */
int stag_batch_destroy(stag_batch* b);

/* ------------------------------------------------ learned preconditioner
 * A gauge-covariant parallel-transport network M used as the preconditioner
 * of flexible CG.  No counterpart in the paper, whose CG (Sec. 2, Fig. 1) is
 * unpreconditioned; it is built on the same operator.  Three linear layers
 * with 1 -> 8 -> 8 -> 1 complex channels on the whole lattice; each layer sums,
 * over nine paths p (the identity and the one-hop transports from x + mu with
 * U_mu(x) and from x - mu with U_mu(x - mu)^dag, eta-folded fat links, so that
 * sum_mu T_{+mu} - T_{-mu} = D of Eq. (5)), complex weights W[p][out][in]
 * times the transported inputs.  The residual enters on even sites (zero on
 * odd sites) and the output is read on even sites.  Weights: layer-major
 * [9][C_out][C_in], complex as interleaved doubles (stag_ptnet_num_weights
 * complex numbers).  The network keeps a pointer to its handle (whose field
 * and mass it uses); destroy it before the handle. */
typedef struct stag_ptnet stag_ptnet;

/* precision: STAG_ARITH_BF16 (activations stored as BF16, FP32 arithmetic) or
 * STAG_ARITH_F32.  The weights start as the least-squares degree-1 polynomial
 * preconditioner alpha + beta A_fat (alpha = 4/L, beta = -10/(3 L^2), L = 1.25
 * times the Rayleigh quotient after 100 power iterations; A_fat: m^2 - D^2 with
 * the one-hop links the transports use) written in the self-adjoint form
 * M = L1^dag L2 L1 (L1 = (r; D r), L2 = diag(alpha + beta m^2, beta)), plus small
 * noise seeded by `seed`, tied like the weights after a training step. */
int stag_ptnet_create(stag_ptnet** out, stag_handle* h, int32_t precision, uint64_t seed);
int64_t stag_ptnet_num_weights(const stag_ptnet* n);
int stag_ptnet_set_weights(stag_ptnet* n, const double* w, int64_t count);
int stag_ptnet_get_weights(stag_ptnet* n, double* w, int64_t count);

/* z_even = M(r_even) ([V/2][3] complex128, host or device). */
int stag_ptnet_apply(stag_ptnet* n, const double* r_even, double* z_even);

/* loss of one pair, the residual norm of the correction |A d|^2 / |A e|^2 with
 * d = M(r) - e (A applied with the FP32 Dirac kernels), and its gradient
 * dL/d conj(W) (complex, interleaved; nullable outputs). */
int stag_ptnet_loss_grad(stag_ptnet* n, const double* r_even, const double* e_even, double* loss, double* grad);

/* Training pairs from plain CG solves (the handle's solver, inner = NONE) of
 * the given sources to 1e-10: after every `stride` iterations, while the
 * iterated residual is above min_rel_residual * |b|, the residual r_k and, after
 * convergence, e_k = x* - x_k are stored, both scaled by 1/|r_k|; at most
 * max_pairs pairs in total.  *n_pairs: pairs stored so far. */
int stag_ptnet_add_pairs(stag_ptnet* n, int32_t n_sources, const double* const* sources, int32_t stride,
                         double min_rel_residual, int32_t max_pairs, int32_t* n_pairs);
int stag_ptnet_num_pairs(const stag_ptnet* n);

/* Adam (beta 0.9, 0.999) on the stored pairs: `epochs` passes in seeded random
 * order, mini-batches of `batch` pairs, learning rate lr; epoch_loss (nullable):
 * mean pair loss of each epoch.  After every step the weights are projected onto
 * the self-adjoint tie W3[p][0][i] = conj(W1[rev p][i][0]), W2[p][o][i] =
 * conj(W2[rev p][i][o]) (rev: the opposite path), so that M is Hermitian, as the
 * short recurrence of flexible CG assumes; weights set with
 * stag_ptnet_set_weights are used as given until the first step. */
int stag_ptnet_train(stag_ptnet* n, int32_t epochs, int32_t batch, double lr, uint64_t seed, double* epoch_loss);

/* Mean loss over the stored pairs. */
int stag_ptnet_dataset_loss(stag_ptnet* n, double* loss);

const char* stag_ptnet_last_error(const stag_ptnet* n);
int stag_ptnet_destroy(stag_ptnet* n);

/* Storage of the activations when the network is applied (stag_ptnet_apply,
 * stag_fcg_solve): STAG_ARITH_BF16 or STAG_ARITH_F32 (default: the precision
 * given at create).  Training and the stored pairs keep the create precision. */
int stag_ptnet_set_inference_precision(stag_ptnet* n, int32_t precision);

/* enable != 0 (the default): the BF16 8 -> 8 layer's forward pass mixes the
 * channels on the tensor cores (tcgen05: per tile of 128 sites and colour, the
 * real form of the complex mixing as a 128 x 144 by 144 x 16 BF16 product with
 * FP32 accumulation); 0: on the CUDA cores in FP32.  The transports are FP32
 * either way.  A tensor-core wait that runs out makes the next call that
 * applies the network return STAG_ERR_TIMEOUT. */
int stag_ptnet_use_tensor_cores(stag_ptnet* n, int32_t enable);

/* How the network is evaluated when it is applied (stag_ptnet_apply,
 * stag_fcg_solve); training always runs the layers.
 *  STAG_PTNET_COLLAPSED (the default): the layers are linear, the input is
 *    zero on odd sites and only the even-site output is read, so only paths of
 *    zero or two hops contribute and the network equals exactly
 *      M r = k0 r + sum_{p,q = 1..8} H[p][q] T_p T_q r,
 *    with C[a][b][c] = sum_{o,i} W3[a][0][o] W2[b][o][i] W1[c][i][0],
 *    k0 = C[0][0][0] and H[p][q] = C[p][q][0] + C[p][0][q] + C[0][p][q]
 *    (computed in FP64 from the weights at every call).  It is evaluated as
 *    chi_p = sum_q H[p][q] T_q r on odd sites (stored in the inference
 *    precision) and z = k0 r + sum_p T_p chi_p on even sites: 16 one-hop
 *    transports per pair of sites instead of 144, FP32 arithmetic.
 *  STAG_PTNET_LAYERED: the three layers as in training (inference precision
 *    for the activations, tensor cores per stag_ptnet_use_tensor_cores).
 * Both compute the same M up to rounding. */
enum { STAG_PTNET_COLLAPSED = 0, STAG_PTNET_LAYERED = 1 };
int stag_ptnet_set_inference_form(stag_ptnet* n, int32_t form);

/* Flexible CG (Notay 2000) with z_k = M(r_k): alpha = (r, z) / (p, A p),
 * x += alpha p, r -= alpha A p, beta = (z_new, r_new - r_old) / (r_old, z_old)
 * (formed as -alpha (z_new, A p) / (r_old, z_old), the same quantity),
 * p = z + beta p, with A and the vectors in the handle's FP64-class arithmetic
 * (float-float or FP64).  Every scalar stays on the device; blocks of
 * opt.check_interval iterations run as a CUDA graph and the host reads the
 * state between blocks.  When the iterated residual falls below tol |b| the
 * true residual is recomputed in native FP64 and decides convergence.  When
 * the smallest |r| so far has not dropped by 10 % within 100 iterations: if
 * this cycle reduced the true residual more than 100-fold, flexible CG
 * restarts from the true residual (info->restarts), otherwise plain CG
 * continues from the current x (info->fallbacks); (r, z) <= 0, (p, A p) <= 0
 * or a non-finite residual also hand over to plain CG.  The arguments and
 * return codes are those of stag_cg_solve. */
int stag_fcg_solve(stag_handle* h, stag_ptnet* n, const double* b_even, double* x_even, double tol,
                   int32_t max_iter, stag_solve_info* info);

/* ------------------------------------- emulated domain decomposition
 * The multi-GPU decomposition of Sec. 4 emulated on one GPU: the lattice is cut
 * into n_ranks slabs along t (Lt / n_ranks even and at least the hop reach, 1
 * or 3), each stored with ghost t-slices, and before every half-Dslash each
 * rank's boundary faces are packed ("boundary data collect"), exchanged and
 * unpacked into its neighbours' ghost slices.  STAG_DD_HOST stages the faces
 * through pinned host memory with host copies between the ranks' buffers (the
 * paper's GPU -> host -> MPI -> host -> GPU path); STAG_DD_DEVICE copies them
 * device to device (the direct path Sec. 5 proposes).  The _OVERLAP modes do
 * the same exchanges on a second stream (and the host copies on the host
 * thread) while each rank computes the sites whose stencil stays inside its own
 * slab, then the boundary slices (the overlap Sec. 5 proposes).  Native FP64
 * arithmetic.  phase_ms (nullable, 6 entries, summed over all ranks and calls
 * of the solve): [0] Dirac kernels, [1] face pack + unpack, [2] device -> host,
 * [3] exchange between ranks (host copies, or device copies in STAG_DD_DEVICE),
 * [4] host -> device, [5] global sums of the dot products; in the _OVERLAP
 * modes [0] is each whole half-Dslash (pack, exchange, Dirac, unpack) and [3]
 * the host copies hidden inside it.  The object keeps a pointer to its handle;
 * destroy it first. */
enum { STAG_DD_HOST = 0, STAG_DD_DEVICE = 1, STAG_DD_HOST_OVERLAP = 2, STAG_DD_DEVICE_OVERLAP = 3 };
typedef struct stag_dd stag_dd;
int stag_dd_create(stag_dd** out, stag_handle* h, int32_t n_ranks);
/* out_even = A in_even through the decomposition (bit-identical to stag_apply_A
 * with STAG_ARITH_F64). */
int stag_dd_apply_A(stag_dd* dd, const double* in_even, double* out_even, int32_t mode, double* phase_ms);
/* Fig. 1 CG with the decomposed operator; every dot product is a per-rank
 * partial sum gathered to the host and summed over the ranks; the true residual
 * is recomputed at the end (no restart).  Arguments and codes as stag_cg_solve. */
int stag_dd_cg_solve(stag_dd* dd, const double* b_even, double* x_even, double tol, int32_t max_iter,
                     int32_t mode, stag_solve_info* info, double* phase_ms);
/* Bytes of faces exchanged since create. */
int64_t stag_dd_bytes_exchanged(const stag_dd* dd);
int stag_dd_destroy(stag_dd* dd);

/* Measured fused multiply-add rate of the current device, in FMA per second:
 * bits = 64 for FP64 DFMA, 32 for FP32 FFMA.  A measurement helper for the
 * arithmetic ceiling of the Dirac kernels' roofline: the paper counts each
 * SU(3) x vector product of D as 36 real multiply-adds (Sec. 2, text after
 * Eq. (5)), so a native-FP64 Naik half-Dslash site is 576 DFMA.  Runs
 * independent FMA chains on every SM for about 0.1 s in two operand patterns
 * (a complex multiply-accumulate's and a shared-multiplier chain), timed with
 * CUDA events after one warm-up launch on a private stream, and reports the
 * faster (it allocates 8 bytes and synchronises that stream).  Returns STAG_ERR_INVALID_ARG for other bits or a
 * NULL output; the message is available from stag_last_error(NULL). */
int stag_measure_fma_rate(int32_t bits, double* fma_per_second);

/* Largest V/2 that stag_apply_A_noalloc accepts. */
#define STAG_NOALLOC_MAX_HALF_SITES 65536

/* out_even = A in_even = m^2 in - D_eo D_oe in, without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that must
 * not have the library allocate device memory (applications that hand out all
 * device memory from their own pool, or that cannot accept the device-wide
 * synchronisation an allocation or free may cause).  It needs no handle.
 * links, naik_long (NULL = one-hop only): the link layout above, eta not
 * folded; in_even, out_even: [V/2][3] complex128; out must not overlap in
 * or the links (any byte in common is rejected).  Every array must be device
 * memory of the current device (host pointers are rejected).  Native FP64
 * arithmetic.  The odd-site intermediate D_oe in is kept in a fixed
 * file-scope device array of STAG_NOALLOC_MAX_HALF_SITES sites (3 MiB) that
 * every GPU loading the library holds until the process exits; larger
 * lattices are rejected with STAG_ERR_INVALID_ARG.  The array is shared by
 * all calls: calls that overlap on the GPU (several host threads, or several
 * streams) race on it.
 * The guarantee of no allocation holds from the second call on each device.
 * CUDA loads a library's device code lazily, so the first call on a device
 * (or any earlier launch from this library there) loads the module: that
 * load allocates the array and the code, and may synchronise the device.
 * Make that first call at set-up time, before any stream capture.  The first
 * call in each CUDA context also looks up the array's device address and
 * caches it for that context; after a device reset (a new context) the next
 * call loads the module and looks the address up again.  Work is enqueued on
 * cuda_stream (NULL = legacy default stream) and the call returns after it
 * completes.  Errors are reported by status; the message is available from
 * stag_last_error(NULL). */
int stag_apply_A_noalloc(const double* links, const double* naik_long, const int32_t dims[4],
                         double mass, const double* in_even, double* out_even, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* STAG_H */
