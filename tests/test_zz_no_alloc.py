"""stag_apply_A_noalloc: A on even sites for callers that cannot let the library
allocate device memory (their device memory comes from their own pool, or they
cannot accept the synchronisation an allocation may cause).

The entry point keeps its odd-site work vector in a fixed device array shared
by all calls.  Two calls in a row, on different lattices, must each agree with
stag_apply_A (the handle-based entry point) to the FP64 parity tolerance of the
other tests (1e-13, norm-wise and element-wise), so the second call cannot be
using anything the first left behind.  Oversized lattices and host pointers are
rejected.  This file is collected last and also passes when run alone.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1010_4782_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_4782_gb300 import build

    build.build()
    return binding.load()


def _reference(fat, lng, dims, mass, v):
    opt = binding.stag_default_options()
    opt.arith = binding.STAG_ARITH_F64
    with binding.Handle(torch.from_numpy(fat).cuda(), dims, mass,
                        naik_long=None if lng is None else torch.from_numpy(lng).cuda(), options=opt) as h:
        vt = torch.from_numpy(v).cuda()
        out = torch.empty_like(vt)
        binding.stag_apply_A(h.h, vt, out)
    return out.cpu().numpy()


def _noalloc(lib, fat_d, lng_d, dims, mass, v_d, out_d):
    dd = (ctypes.c_int32 * 4)(*dims)
    stream = torch.cuda.current_stream().cuda_stream
    return lib.stag_apply_A_noalloc(ctypes.c_void_p(fat_d.data_ptr()),
                                    None if lng_d is None else ctypes.c_void_p(lng_d.data_ptr()),
                                    dd, ctypes.c_double(mass), ctypes.c_void_p(v_d.data_ptr()),
                                    ctypes.c_void_p(out_d.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_matches_apply_A_on_two_calls(lib):
    cases = [((8, 8, 8, 16), True, 0.05, 3), ((6, 4, 2, 8), False, 0.3, 4)]
    for dims, naik, mass, seed in cases:
        if naik:
            fat, lng = inputs.asqtad_form_fields(dims, seeds=(seed, seed + 1, seed + 2))
        else:
            fat, lng = inputs.gauge_field(dims, seed), None
        v = inputs.gaussian_even_source(dims, seed + 10)
        ref = _reference(fat, lng, dims, mass, v)
        fat_d = torch.from_numpy(fat).cuda()
        lng_d = None if lng is None else torch.from_numpy(lng).cuda()
        v_d = torch.from_numpy(v).cuda()
        out_d = torch.full_like(v_d, float("nan"))
        assert _noalloc(lib, fat_d, lng_d, dims, mass, v_d, out_d) == binding.STAG_OK, \
            binding.stag_last_error(None)
        got = out_d.cpu().numpy()
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        elem = np.abs(got - ref).max() / np.abs(ref).max()
        assert rel <= TOL and elem <= TOL, (dims, rel, elem)


def test_noalloc_rejects_oversize_and_host_memory(lib):
    dims = (16, 16, 16, 34)  # V/2 = 69632 > 65536
    assert int(np.prod(dims)) // 2 > 65536
    fat = torch.zeros(4, dtype=torch.complex128, device="cuda")
    v = torch.zeros(4, dtype=torch.complex128, device="cuda")
    out = torch.zeros(4, dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, fat, None, dims, 0.1, v, out) == binding.STAG_ERR_INVALID_ARG
    assert "65536" in binding.stag_last_error(None)
    dims = (4, 4, 4, 4)
    fat_h = np.zeros((4, 4, 4, 4, 4, 3, 3), dtype=np.complex128)
    v_d = torch.zeros((128, 3), dtype=torch.complex128, device="cuda")
    out_d = torch.zeros_like(v_d)
    dd = (ctypes.c_int32 * 4)(*dims)
    code = lib.stag_apply_A_noalloc(ctypes.c_void_p(fat_h.ctypes.data), None, dd, ctypes.c_double(0.1),
                                    ctypes.c_void_p(v_d.data_ptr()), ctypes.c_void_p(out_d.data_ptr()), None)
    assert code == binding.STAG_ERR_INVALID_ARG
