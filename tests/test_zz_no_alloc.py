"""stag_apply_A_noalloc: A on even sites for callers that cannot let the library
allocate device memory (their device memory comes from their own pool, or they
cannot accept the synchronisation an allocation may cause).

The entry point keeps its odd-site work vector in a fixed device array shared
by all calls.  Calls in a row, on different lattices, must each agree with the
FP64 oracle's A (Eq. (3) on even sites) and with stag_apply_A (the
handle-based entry point) to the FP64 parity tolerance of the other tests
(1e-13, norm-wise and element-wise), so a later call cannot be using anything
an earlier one left behind.  The cases include the largest lattice the array
takes (V/2 = 65536) and a Naik lattice with an extent of 2, where the
three-hop wraps onto the one-hop neighbour.  A warmed call leaves the device's
free memory unchanged.  Oversized lattices, host pointers and overlapping
input and output are rejected.  This file is collected last and also passes
when run alone.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
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


def _close(got, ref):
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    elem = np.abs(got - ref).max() / np.abs(ref).max()
    return rel <= TOL and elem <= TOL, (rel, elem)


CASES = [((8, 8, 8, 16), True, 0.05, 3),
         ((6, 4, 2, 8), False, 0.3, 4),
         ((16, 16, 16, 32), True, 0.02, 5),   # V/2 = 65536: the largest lattice the array takes
         ((2, 4, 4, 6), True, 0.1, 6)]        # x extent 2: the Naik hop wraps onto the one-hop neighbour


def test_noalloc_matches_oracle_and_apply_A_on_calls_in_a_row(lib):
    assert int(np.prod(CASES[2][0])) // 2 == 65536
    for dims, naik, mass, seed in CASES:
        if naik:
            fat, lng = inputs.asqtad_form_fields(dims, seeds=(seed, seed + 1, seed + 2))
        else:
            fat, lng = inputs.gauge_field(dims, seed), None
        v = inputs.gaussian_even_source(dims, seed + 10)
        want = oracle.Operator(fat, lng, mass, dims).apply_A(v)
        ref = _reference(fat, lng, dims, mass, v)
        fat_d = torch.from_numpy(fat).cuda()
        lng_d = None if lng is None else torch.from_numpy(lng).cuda()
        v_d = torch.from_numpy(v).cuda()
        out_d = torch.full_like(v_d, float("nan"))
        assert _noalloc(lib, fat_d, lng_d, dims, mass, v_d, out_d) == binding.STAG_OK, \
            binding.stag_last_error(None)
        got = out_d.cpu().numpy()
        ok, err = _close(got, want)
        assert ok, ("vs oracle", dims, err)
        ok, err = _close(got, ref)
        assert ok, ("vs stag_apply_A", dims, err)


def test_noalloc_warmed_call_allocates_nothing(lib):
    dims = (8, 8, 8, 16)
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(40, 41, 42))
    v = inputs.gaussian_even_source(dims, 43)
    fat_d = torch.from_numpy(fat).cuda()
    lng_d = torch.from_numpy(lng).cuda()
    v_d = torch.from_numpy(v).cuda()
    out_d = torch.empty_like(v_d)
    assert _noalloc(lib, fat_d, lng_d, dims, 0.1, v_d, out_d) == binding.STAG_OK
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _noalloc(lib, fat_d, lng_d, dims, 0.1, v_d, out_d) == binding.STAG_OK
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    want = oracle.Operator(fat, lng, 0.1, dims).apply_A(v)
    ok, err = _close(out_d.cpu().numpy(), want)
    assert ok, err


def test_noalloc_rejects_oversize_overlap_and_host_memory(lib):
    dims = (16, 16, 16, 34)  # V/2 = 69632 > 65536
    assert int(np.prod(dims)) // 2 > 65536
    fat = torch.zeros(4, dtype=torch.complex128, device="cuda")
    v = torch.zeros(4, dtype=torch.complex128, device="cuda")
    out = torch.zeros(4, dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, fat, None, dims, 0.1, v, out) == binding.STAG_ERR_INVALID_ARG
    assert "65536" in binding.stag_last_error(None)
    dims = (4, 4, 4, 4)
    fat_d = torch.zeros((4, 4, 4, 4, 4, 3, 3), dtype=torch.complex128, device="cuda")
    fat_h = np.zeros((4, 4, 4, 4, 4, 3, 3), dtype=np.complex128)
    v_d = torch.zeros((128, 3), dtype=torch.complex128, device="cuda")
    out_d = torch.zeros_like(v_d)
    dd = (ctypes.c_int32 * 4)(*dims)
    code = lib.stag_apply_A_noalloc(ctypes.c_void_p(fat_h.ctypes.data), None, dd, ctypes.c_double(0.1),
                                    ctypes.c_void_p(v_d.data_ptr()), ctypes.c_void_p(out_d.data_ptr()), None)
    assert code == binding.STAG_ERR_INVALID_ARG
    # out starting 3 sites into in: the ranges share bytes, so the call is rejected
    buf = torch.zeros((131, 3), dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, fat_d, None, dims, 0.1, buf[:128], buf[3:]) == binding.STAG_ERR_INVALID_ARG
    assert "overlap" in binding.stag_last_error(None)
    # out inside the links
    assert _noalloc(lib, fat_d, None, dims, 0.1, v_d, fat_d.view(-1)[:384]) == binding.STAG_ERR_INVALID_ARG
