"""Thin ctypes binding of the C ABI in include/stag.h (argument marshalling only).

Functions carry the ABI's names.  Array arguments may be torch tensors (CUDA
or CPU) or numpy arrays of complex128 (or float64 with a trailing (re, im)
axis); only their data pointers are passed.  Every computation runs inside
libstag.so; if the library cannot be loaded the call raises - there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

STAG_OK = 0
STAG_ERR_INVALID_ARG = 1
STAG_ERR_CUDA = 2
STAG_ERR_NOT_CONVERGED = 3
STAG_ERR_BREAKDOWN = 4
STAG_ERR_TIMEOUT = 5
STAG_ERR_OOM = 6

STAG_ARITH_F64 = 0
STAG_ARITH_FF = 1
STAG_ARITH_F32 = 2
STAG_ARITH_F16 = 3
STAG_ARITH_BF16 = 4

STAG_INNER_NONE = 0
STAG_INNER_F32 = 1
STAG_INNER_F16 = 2
STAG_INNER_BF16 = 3
STAG_INNER_F32_L16 = 4

STAG_PTNET_COLLAPSED = 0
STAG_PTNET_LAYERED = 1

STAG_DD_HOST = 0
STAG_DD_DEVICE = 1
STAG_DD_HOST_OVERLAP = 2
STAG_DD_DEVICE_OVERLAP = 3
DD_PHASES = ("dirac", "collect", "d2h", "exchange", "h2d", "global_sum")

STAG_KERNEL_DSLASH_OE = 0
STAG_KERNEL_DSLASH_EO = 1
STAG_KERNEL_UPDATE_XR = 2
STAG_KERNEL_UPDATE_D = 3
KERNEL_NAMES = ("dslash_oe", "dslash_eo_cg", "update_xr", "update_d")

EXPORTED = (
    "stag_default_options",
    "stag_create",
    "stag_create_ex",
    "stag_set_stream",
    "stag_set_mass",
    "stag_dslash",
    "stag_apply_A",
    "stag_apply_A_prec",
    "stag_cg_solve",
    "stag_destroy",
    "stag_last_error",
    "stag_kernel_stats",
    "stag_reset_stats",
    "stag_device_bytes",
    "stag_check_guards",
    "stag_launch_count",
    "stag_apply_A_noalloc",
    "stag_measure_fma_rate",
    "stag_batch_create",
    "stag_batch_set_stream",
    "stag_batch_solve",
    "stag_batch_apply_A",
    "stag_batch_tuning",
    "stag_batch_set_tuning",
    "stag_batch_last_error",
    "stag_batch_device_bytes",
    "stag_batch_destroy",
    "stag_ptnet_create",
    "stag_ptnet_num_weights",
    "stag_ptnet_set_weights",
    "stag_ptnet_get_weights",
    "stag_ptnet_apply",
    "stag_ptnet_loss_grad",
    "stag_ptnet_add_pairs",
    "stag_ptnet_num_pairs",
    "stag_ptnet_use_tensor_cores",
    "stag_ptnet_set_inference_form",
    "stag_ptnet_train",
    "stag_ptnet_dataset_loss",
    "stag_ptnet_last_error",
    "stag_ptnet_destroy",
    "stag_ptnet_set_inference_precision",
    "stag_fcg_solve",
    "stag_dd_create",
    "stag_dd_apply_A",
    "stag_dd_cg_solve",
    "stag_dd_bytes_exchanged",
    "stag_dd_destroy",
)


class stag_options(ctypes.Structure):
    _fields_ = [
        ("arith", ctypes.c_int32),
        ("check_interval", ctypes.c_int32),
        ("max_restarts", ctypes.c_int32),
        ("use_graphs", ctypes.c_int32),
        ("timing", ctypes.c_int32),
        ("inner", ctypes.c_int32),
        ("reliable_interval", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("reliable_delta", ctypes.c_double),
        ("link_recon", ctypes.c_int32),
        ("guard_bands", ctypes.c_int32),
        ("long_scale", ctypes.c_double),
        ("long_recon", ctypes.c_int32),
        ("reserved2", ctypes.c_int32),
    ]


class stag_solve_info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32),
        ("restarts", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("reliable_updates", ctypes.c_int32),
        ("true_rel_residual", ctypes.c_double),
        ("iter_rel_residual", ctypes.c_double),
        ("time_ms", ctypes.c_double),
        ("fallbacks", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class StagError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"stag error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return LIB


def load(path: str | None = None):
    """Load libstag.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build the CUDA library first (paper_1010_4782_gb300.build)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    H = ctypes.c_void_p
    i32 = ctypes.c_int32
    d = ctypes.c_double
    lib.stag_default_options.argtypes = [ctypes.POINTER(stag_options)]
    lib.stag_create.argtypes = [ctypes.POINTER(H), P, ctypes.POINTER(i32), d]
    lib.stag_create_ex.argtypes = [ctypes.POINTER(H), P, P, ctypes.POINTER(i32), d,
                                   ctypes.POINTER(stag_options)]
    lib.stag_set_stream.argtypes = [H, P]
    lib.stag_set_mass.argtypes = [H, d]
    lib.stag_dslash.argtypes = [H, i32, P, P]
    lib.stag_apply_A.argtypes = [H, P, P]
    lib.stag_apply_A_prec.argtypes = [H, i32, P, P]
    lib.stag_cg_solve.argtypes = [H, P, P, d, i32, ctypes.POINTER(stag_solve_info)]
    lib.stag_destroy.argtypes = [H]
    lib.stag_last_error.argtypes = [H]
    lib.stag_last_error.restype = ctypes.c_char_p
    lib.stag_kernel_stats.argtypes = [H, i32, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_int64)]
    lib.stag_reset_stats.argtypes = [H]
    lib.stag_check_guards.argtypes = [H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.stag_device_bytes.argtypes = [H]
    lib.stag_device_bytes.restype = ctypes.c_int64
    lib.stag_launch_count.argtypes = [H]
    lib.stag_launch_count.restype = ctypes.c_int64
    lib.stag_apply_A_noalloc.argtypes = [P, P, ctypes.POINTER(i32), d, P, P, P]
    lib.stag_measure_fma_rate.argtypes = [i32, ctypes.POINTER(d)]
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.stag_batch_create.argtypes = [ctypes.POINTER(H), i32, PP, PP, ctypes.POINTER(i32),
                                      ctypes.POINTER(d), ctypes.POINTER(stag_options)]
    lib.stag_batch_set_stream.argtypes = [H, P]
    lib.stag_batch_solve.argtypes = [H, PP, PP, d, i32, ctypes.POINTER(stag_solve_info)]
    lib.stag_batch_apply_A.argtypes = [H, PP, PP]
    lib.stag_batch_tuning.argtypes = [H, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(d),
                                      ctypes.POINTER(i32)]
    lib.stag_batch_set_tuning.argtypes = [H, i32, i32, i32, i32]
    lib.stag_batch_last_error.argtypes = [H]
    lib.stag_batch_last_error.restype = ctypes.c_char_p
    lib.stag_batch_device_bytes.argtypes = [H]
    lib.stag_batch_device_bytes.restype = ctypes.c_int64
    lib.stag_batch_destroy.argtypes = [H]
    lib.stag_ptnet_create.argtypes = [ctypes.POINTER(H), H, i32, ctypes.c_uint64]
    lib.stag_ptnet_num_weights.argtypes = [H]
    lib.stag_ptnet_num_weights.restype = ctypes.c_int64
    lib.stag_ptnet_set_weights.argtypes = [H, P, ctypes.c_int64]
    lib.stag_ptnet_get_weights.argtypes = [H, P, ctypes.c_int64]
    lib.stag_ptnet_apply.argtypes = [H, P, P]
    lib.stag_ptnet_loss_grad.argtypes = [H, P, P, ctypes.POINTER(d), P]
    lib.stag_ptnet_add_pairs.argtypes = [H, i32, PP, i32, d, i32, ctypes.POINTER(i32)]
    lib.stag_ptnet_num_pairs.argtypes = [H]
    lib.stag_ptnet_train.argtypes = [H, i32, i32, d, ctypes.c_uint64, P]
    lib.stag_ptnet_dataset_loss.argtypes = [H, ctypes.POINTER(d)]
    lib.stag_ptnet_last_error.argtypes = [H]
    lib.stag_ptnet_last_error.restype = ctypes.c_char_p
    lib.stag_ptnet_destroy.argtypes = [H]
    lib.stag_ptnet_set_inference_precision.argtypes = [H, i32]
    lib.stag_ptnet_use_tensor_cores.argtypes = [H, i32]
    lib.stag_ptnet_set_inference_form.argtypes = [H, i32]
    lib.stag_fcg_solve.argtypes = [H, H, P, P, d, i32, ctypes.POINTER(stag_solve_info)]
    lib.stag_dd_create.argtypes = [ctypes.POINTER(H), H, i32]
    lib.stag_dd_apply_A.argtypes = [H, P, P, i32, P]
    lib.stag_dd_cg_solve.argtypes = [H, P, P, d, i32, i32, ctypes.POINTER(stag_solve_info), P]
    lib.stag_dd_bytes_exchanged.argtypes = [H]
    lib.stag_dd_bytes_exchanged.restype = ctypes.c_int64
    lib.stag_dd_destroy.argtypes = [H]
    for name in EXPORTED:
        if name not in ("stag_last_error", "stag_device_bytes", "stag_launch_count", "stag_batch_last_error",
                        "stag_batch_device_bytes", "stag_ptnet_num_weights", "stag_ptnet_last_error",
                        "stag_dd_bytes_exchanged"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    """Data pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _check(code, h=None):
    if code != STAG_OK:
        raise StagError(code, stag_last_error(h))


def stag_default_options() -> stag_options:
    o = stag_options()
    _check(load().stag_default_options(ctypes.byref(o)))
    return o


def stag_create(links, dims, mass):
    h = ctypes.c_void_p()
    dd = (ctypes.c_int32 * 4)(*[int(v) for v in dims])
    _check(load().stag_create(ctypes.byref(h), _ptr(links), dd, float(mass)))
    return h


def stag_create_ex(fat, naik_long, dims, mass, options: stag_options | None = None):
    h = ctypes.c_void_p()
    dd = (ctypes.c_int32 * 4)(*[int(v) for v in dims])
    opt = ctypes.byref(options) if options is not None else None
    _check(load().stag_create_ex(ctypes.byref(h), _ptr(fat), _ptr(naik_long), dd, float(mass), opt))
    return h


def stag_set_stream(h, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(load().stag_set_stream(h, ctypes.c_void_p(raw or 0)), h)


def stag_set_mass(h, mass):
    _check(load().stag_set_mass(h, float(mass)), h)


def stag_dslash(h, out_parity, inp, out):
    _check(load().stag_dslash(h, int(out_parity), _ptr(inp), _ptr(out)), h)


def stag_apply_A(h, inp, out):
    _check(load().stag_apply_A(h, _ptr(inp), _ptr(out)), h)


def stag_apply_A_prec(h, arith, inp, out):
    _check(load().stag_apply_A_prec(h, int(arith), _ptr(inp), _ptr(out)), h)


def stag_cg_solve(h, b, x, tol, max_iter=0, raise_on_error=True):
    """Returns (status, info dict)."""
    info = stag_solve_info()
    code = load().stag_cg_solve(h, _ptr(b), _ptr(x), float(tol), int(max_iter), ctypes.byref(info))
    if raise_on_error and code not in (STAG_OK, STAG_ERR_NOT_CONVERGED):
        _check(code, h)
    return code, info.as_dict()


def stag_destroy(h):
    if h is not None:
        load().stag_destroy(h)


def stag_last_error(h=None) -> str:
    return load().stag_last_error(h).decode()


def stag_kernel_stats(h, kernel):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().stag_kernel_stats(h, int(kernel), ctypes.byref(ms), ctypes.byref(n)), h)
    return ms.value, n.value


def stag_reset_stats(h):
    _check(load().stag_reset_stats(h), h)


def stag_check_guards(h):
    """(guard-band bytes checked, bytes changed) of a handle created with guard_bands = 1."""
    checked, bad = ctypes.c_int64(), ctypes.c_int64()
    _check(load().stag_check_guards(h, ctypes.byref(checked), ctypes.byref(bad)), h)
    return checked.value, bad.value


def stag_device_bytes(h) -> int:
    return int(load().stag_device_bytes(h))


def stag_launch_count(h) -> int:
    return int(load().stag_launch_count(h))


def stag_apply_A_noalloc(links, naik_long, dims, mass, inp, out, stream=None):
    """A on even sites without device allocation (device arrays only; small lattices)."""
    dd = (ctypes.c_int32 * 4)(*[int(v) for v in dims])
    raw = getattr(stream, "cuda_stream", stream)
    _check(load().stag_apply_A_noalloc(_ptr(links), _ptr(naik_long), dd, float(mass), _ptr(inp), _ptr(out),
                                        ctypes.c_void_p(raw or 0)))


def stag_measure_fma_rate(bits):
    """Measured FMA per second of the current device (bits = 64: DFMA, 32: FFMA)."""
    rate = ctypes.c_double(0.0)
    _check(load().stag_measure_fma_rate(bits, ctypes.byref(rate)))
    return rate.value


def _ptr_array(arrs):
    return (ctypes.c_void_p * len(arrs))(*[_ptr(a) for a in arrs])


def stag_batch_create(fats, naiks, dims_list, masses, options: stag_options | None = None):
    """fats, naiks (None entries allowed), dims_list: per-system lists; returns a batch handle."""
    n = len(fats)
    h = ctypes.c_void_p()
    dd = (ctypes.c_int32 * (4 * n))(*[int(v) for dims in dims_list for v in dims])
    mm = (ctypes.c_double * n)(*[float(m) for m in masses])
    nk = _ptr_array(naiks) if naiks is not None else None
    opt = ctypes.byref(options) if options is not None else None
    code = load().stag_batch_create(ctypes.byref(h), n, _ptr_array(fats), nk, dd, mm, opt)
    if code != STAG_OK:
        raise StagError(code, stag_last_error(None))
    return h


def _bcheck(code, h):
    if code != STAG_OK:
        raise StagError(code, load().stag_batch_last_error(h).decode())


def stag_batch_set_stream(h, stream):
    raw = getattr(stream, "cuda_stream", stream)
    _bcheck(load().stag_batch_set_stream(h, ctypes.c_void_p(raw or 0)), h)


def stag_batch_solve(h, bs, xs, tol, max_iter=0):
    """Returns (status, [info dict per system])."""
    n = len(bs)
    infos = (stag_solve_info * n)()
    code = load().stag_batch_solve(h, _ptr_array(bs), _ptr_array(xs), float(tol), int(max_iter), infos)
    if code not in (STAG_OK, STAG_ERR_NOT_CONVERGED, STAG_ERR_BREAKDOWN):
        _bcheck(code, h)
    return code, [i.as_dict() for i in infos]


def stag_batch_apply_A(h, ins, outs):
    _bcheck(load().stag_batch_apply_A(h, _ptr_array(ins), _ptr_array(outs)), h)


def stag_batch_tuning(h, system):
    """(RHS per thread, threads per block, measured D_oe ms, traversal 0/1) of system's group."""
    rb = ctypes.c_int32()
    bs = ctypes.c_int32()
    ms = ctypes.c_double()
    sw = ctypes.c_int32()
    _bcheck(load().stag_batch_tuning(h, int(system), ctypes.byref(rb), ctypes.byref(bs), ctypes.byref(ms),
                                     ctypes.byref(sw)), h)
    return rb.value, bs.value, ms.value, sw.value


def stag_batch_set_tuning(h, system, rhs_per_thread, threads_per_block, traversal):
    _bcheck(load().stag_batch_set_tuning(h, int(system), int(rhs_per_thread), int(threads_per_block),
                                         int(traversal)), h)


def stag_batch_device_bytes(h) -> int:
    return int(load().stag_batch_device_bytes(h))


def stag_batch_destroy(h):
    if h is not None:
        load().stag_batch_destroy(h)


def _pcheck(code, net, h=None):
    if code != STAG_OK:
        msg = load().stag_ptnet_last_error(net).decode()
        if h is not None:
            msg += " / " + stag_last_error(h)
        raise StagError(code, msg)


def stag_ptnet_create(h, precision=STAG_ARITH_BF16, seed=0):
    n = ctypes.c_void_p()
    code = load().stag_ptnet_create(ctypes.byref(n), h, int(precision), int(seed))
    if code != STAG_OK:
        raise StagError(code, stag_last_error(h))
    return n


def stag_ptnet_weights(net):
    nw = int(load().stag_ptnet_num_weights(net))
    w = np.zeros(nw, dtype=np.complex128)
    _pcheck(load().stag_ptnet_get_weights(net, w.ctypes.data, nw), net)
    return w


def stag_ptnet_set_weights(net, w):
    w = np.ascontiguousarray(w, dtype=np.complex128)
    _pcheck(load().stag_ptnet_set_weights(net, w.ctypes.data, w.size), net)


def stag_ptnet_apply(net, r, z):
    _pcheck(load().stag_ptnet_apply(net, _ptr(r), _ptr(z)), net)


def stag_ptnet_loss_grad(net, r, e):
    nw = int(load().stag_ptnet_num_weights(net))
    loss = ctypes.c_double()
    g = np.zeros(nw, dtype=np.complex128)
    _pcheck(load().stag_ptnet_loss_grad(net, _ptr(r), _ptr(e), ctypes.byref(loss), g.ctypes.data), net)
    return loss.value, g


def stag_ptnet_add_pairs(net, sources, stride, min_rel_residual=1e-6, max_pairs=2000):
    npairs = ctypes.c_int32()
    _pcheck(load().stag_ptnet_add_pairs(net, len(sources), _ptr_array(sources), int(stride), float(min_rel_residual),
                                        int(max_pairs), ctypes.byref(npairs)), net)
    return npairs.value


def stag_ptnet_train(net, epochs, batch, lr, seed=0):
    losses = np.zeros(max(1, epochs), dtype=np.float64)
    _pcheck(load().stag_ptnet_train(net, int(epochs), int(batch), float(lr), int(seed), losses.ctypes.data), net)
    return losses[:epochs]


def stag_ptnet_dataset_loss(net):
    v = ctypes.c_double()
    _pcheck(load().stag_ptnet_dataset_loss(net, ctypes.byref(v)), net)
    return v.value


def stag_ptnet_set_inference_precision(net, precision):
    _pcheck(load().stag_ptnet_set_inference_precision(net, int(precision)), net)


def stag_ptnet_use_tensor_cores(net, enable):
    _pcheck(load().stag_ptnet_use_tensor_cores(net, int(bool(enable))), net)


def stag_ptnet_set_inference_form(net, form):
    _pcheck(load().stag_ptnet_set_inference_form(net, int(form)), net)


def stag_ptnet_destroy(net):
    if net is not None:
        load().stag_ptnet_destroy(net)


def stag_fcg_solve(h, net, b, x, tol, max_iter=0):
    info = stag_solve_info()
    code = load().stag_fcg_solve(h, net, _ptr(b), _ptr(x), float(tol), int(max_iter), ctypes.byref(info))
    if code not in (STAG_OK, STAG_ERR_NOT_CONVERGED):
        _check(code, h)
    return code, info.as_dict()


def stag_dd_create(h, n_ranks):
    dd = ctypes.c_void_p()
    _check(load().stag_dd_create(ctypes.byref(dd), h, int(n_ranks)), h)
    return dd


def stag_dd_apply_A(dd, h, inp, out, mode=STAG_DD_HOST):
    ph = np.zeros(6, dtype=np.float64)
    _check(load().stag_dd_apply_A(dd, _ptr(inp), _ptr(out), int(mode), ph.ctypes.data), h)
    return dict(zip(DD_PHASES, ph.tolist()))


def stag_dd_cg_solve(dd, h, b, x, tol, max_iter=0, mode=STAG_DD_HOST):
    info = stag_solve_info()
    ph = np.zeros(6, dtype=np.float64)
    code = load().stag_dd_cg_solve(dd, _ptr(b), _ptr(x), float(tol), int(max_iter), int(mode), ctypes.byref(info),
                                   ph.ctypes.data)
    if code not in (STAG_OK, STAG_ERR_NOT_CONVERGED):
        _check(code, h)
    return code, info.as_dict(), dict(zip(DD_PHASES, ph.tolist()))


def stag_dd_destroy(dd):
    if dd is not None:
        load().stag_dd_destroy(dd)


class Handle:
    """Owns one stag_handle; closes it on exit."""

    def __init__(self, fat, dims, mass, naik_long=None, options: stag_options | None = None,
                 stream=None):
        self.h = stag_create_ex(fat, naik_long, dims, mass, options)
        self.dims = tuple(int(v) for v in dims)
        if stream is not None:
            stag_set_stream(self.h, stream)

    def close(self):
        if self.h is not None:
            stag_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
