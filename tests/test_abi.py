"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point that include/stag.h declares, and rejects bad arguments
before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1010_4782_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(stag_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("stag_create", "stag_apply_A", "stag_cg_solve", "stag_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.EXPORTED) == set(_declared_functions())


def test_default_options(lib):
    o = binding.stag_default_options()
    assert o.arith in (binding.STAG_ARITH_F64, binding.STAG_ARITH_FF)
    assert o.check_interval == 32 and o.max_restarts == 5 and o.use_graphs == 1
    assert lib.stag_default_options(None) == binding.STAG_ERR_INVALID_ARG


@pytest.mark.parametrize("dims", [(4, 4, 3, 4), (0, 4, 4, 4), (4, 4, 4, -2), (1, 2, 2, 2)])
def test_create_rejects_bad_extents(lib, dims):
    links = np.zeros(16, dtype=np.complex128)
    with pytest.raises(binding.StagError) as e:
        binding.stag_create(links, dims, 0.1)
    assert e.value.code == binding.STAG_ERR_INVALID_ARG
    assert "even" in binding.stag_last_error(None)


def test_create_rejects_null_and_nonfinite_mass(lib):
    h = ctypes.c_void_p()
    dims = (ctypes.c_int32 * 4)(4, 4, 4, 4)
    assert lib.stag_create(ctypes.byref(h), None, dims, 0.1) == binding.STAG_ERR_INVALID_ARG
    assert not h.value
    links = np.zeros(4 ** 4 * 36, dtype=np.complex128)
    assert lib.stag_create(ctypes.byref(h), links.ctypes.data, dims, float("nan")) == \
        binding.STAG_ERR_INVALID_ARG
    assert lib.stag_create(ctypes.byref(h), links.ctypes.data, None, 0.1) == binding.STAG_ERR_INVALID_ARG


def test_null_handle_calls(lib):
    assert lib.stag_destroy(None) == binding.STAG_OK
    assert lib.stag_apply_A(None, None, None) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_cg_solve(None, None, None, 1e-10, 0, None) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_kernel_stats(None, 0, None, None) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_device_bytes(None) == 0
    assert isinstance(binding.stag_last_error(None), str)


def test_null_network_calls(lib):
    """Every network and flexible-CG entry point rejects a NULL network (or handle)
    before it touches a device; the inference setters also reject unknown values."""
    H = ctypes.c_void_p
    out = H()
    assert lib.stag_ptnet_create(ctypes.byref(out), None, binding.STAG_ARITH_BF16, 0) == binding.STAG_ERR_INVALID_ARG
    assert not out.value
    assert lib.stag_ptnet_create(None, None, binding.STAG_ARITH_BF16, 0) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_ptnet_destroy(None) == binding.STAG_OK
    assert lib.stag_ptnet_num_weights(None) == 0
    assert lib.stag_ptnet_apply(None, None, None) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_ptnet_set_weights(None, None, 720) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_ptnet_get_weights(None, None, 720) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_ptnet_train(None, 1, 16, 1e-3, 0, None) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_ptnet_dataset_loss(None, None) == binding.STAG_ERR_INVALID_ARG
    for form in (binding.STAG_PTNET_COLLAPSED, binding.STAG_PTNET_LAYERED, 2, -1):
        assert lib.stag_ptnet_set_inference_form(None, form) == binding.STAG_ERR_INVALID_ARG
    for prec in (binding.STAG_ARITH_BF16, binding.STAG_ARITH_F32, binding.STAG_ARITH_F64):
        assert lib.stag_ptnet_set_inference_precision(None, prec) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_ptnet_use_tensor_cores(None, 1) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_fcg_solve(None, None, None, None, 1e-10, 0, None) == binding.STAG_ERR_INVALID_ARG


@pytest.mark.parametrize("case", ["recon_7", "f64", "no_naik", "zero_scale", "nan_scale", "tiny_scale", "huge_scale",
                                  "link_recon_7"])
def test_create_rejects_bad_link_forms(lib, case):
    """Option checks of the 12-parameter link forms, all made before any device work."""
    dims = (4, 4, 4, 4)
    links = np.zeros(4 ** 4 * 36, dtype=np.complex128)
    o = binding.stag_default_options()
    o.arith, o.long_recon, o.long_scale = binding.STAG_ARITH_FF, 12, -1.0 / 24.0
    naik = links
    if case == "recon_7":
        o.long_recon = 7
    elif case == "f64":
        o.arith = binding.STAG_ARITH_F64
    elif case == "no_naik":
        naik = None
    elif case == "zero_scale":
        o.long_scale = 0.0
    elif case == "nan_scale":
        o.long_scale = float("nan")
    elif case == "tiny_scale":
        o.long_scale = -9e-11   # below 1e-10: float-float products of two entries would go subnormal
    elif case == "huge_scale":
        o.long_scale = 2e18     # above 1e18: such products approach the FP32 overflow
    else:
        o.long_recon, o.link_recon = 0, 7
    with pytest.raises(binding.StagError) as e:
        binding.stag_create_ex(links, naik, dims, 0.1, o)
    assert e.value.code == binding.STAG_ERR_INVALID_ARG
    assert "recon" in binding.stag_last_error(None)


def test_fma_probe_rejects_bad_arguments(lib):
    """stag_measure_fma_rate checks its arguments before touching a device."""
    import ctypes as ct

    rate = ct.c_double(0.0)
    assert lib.stag_measure_fma_rate(16, ct.byref(rate)) == binding.STAG_ERR_INVALID_ARG
    assert lib.stag_measure_fma_rate(64, None) == binding.STAG_ERR_INVALID_ARG


def test_guard_options_checked_before_device_work(lib):
    import ctypes as ct

    dims = (ct.c_int32 * 4)(4, 4, 4, 4)
    links = np.zeros(4 ** 4 * 36, dtype=np.complex128)
    o = binding.stag_default_options()
    assert o.guard_bands == 0
    o.guard_bands = 2
    h = ct.c_void_p()
    assert lib.stag_create_ex(ct.byref(h), links.ctypes.data, None, dims, ct.c_double(0.1),
                              ct.byref(o)) == binding.STAG_ERR_INVALID_ARG
    assert "guard" in binding.stag_last_error(None)
    checked, bad = ct.c_int64(), ct.c_int64()
    assert lib.stag_check_guards(None, ct.byref(checked), ct.byref(bad)) == binding.STAG_ERR_INVALID_ARG
