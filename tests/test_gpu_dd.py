"""Emulated domain decomposition (Sec. 4): the decomposed operator runs the same
Dirac kernel on the same neighbour values as stag_apply_A, so it must agree
bit for bit; the decomposed CG must meet the solver bars against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1010_4782_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_4782_gb300 import build

    build.build()
    binding.load()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _handle(fat, lng, dims, mass):
    opt = binding.stag_default_options()
    opt.arith = binding.STAG_ARITH_F64
    return binding.Handle(_dev(fat), dims, mass, naik_long=None if lng is None else _dev(lng), options=opt)


@pytest.mark.parametrize("mode", [binding.STAG_DD_HOST, binding.STAG_DD_DEVICE, binding.STAG_DD_HOST_OVERLAP,
                                  binding.STAG_DD_DEVICE_OVERLAP])
@pytest.mark.parametrize("naik,dims,ranks", [(False, (4, 4, 6, 8), 1), (False, (4, 4, 6, 8), 4),
                                             (True, (6, 4, 4, 16), 2), (True, (6, 4, 4, 24), 4),
                                             (False, (8, 8, 8, 16), 8)])
def test_decomposed_A_is_bit_identical(naik, dims, ranks, mode):
    if naik:
        fat, lng = inputs.asqtad_form_fields(dims, seeds=(121, 122, 123))
    else:
        fat, lng = inputs.gauge_field(dims, 121), None
    v = _dev(inputs.gaussian_even_source(dims, 124))
    with _handle(fat, lng, dims, 0.07) as h:
        ref = torch.empty_like(v)
        binding.stag_apply_A(h.h, v, ref)
        dd = binding.stag_dd_create(h.h, ranks)
        try:
            out = torch.empty_like(v)
            ph = binding.stag_dd_apply_A(dd, h.h, v, out, mode)
        finally:
            binding.stag_dd_destroy(dd)
    assert torch.equal(out, ref)
    assert ph["dirac"] > 0
    if mode == binding.STAG_DD_HOST:
        assert ph["collect"] > 0 and ph["d2h"] > 0 and ph["h2d"] > 0
    elif mode == binding.STAG_DD_DEVICE:
        assert ph["collect"] > 0 and ph["d2h"] == 0 and ph["h2d"] == 0
    else:  # overlapped: one timing per half-Dslash
        assert ph["collect"] == 0 and ph["d2h"] == 0 and ph["h2d"] == 0


def test_decomposed_cg_solve():
    dims, m, tol = (6, 4, 4, 24), 0.05, 1e-10
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(131, 132, 133))
    b = inputs.gaussian_even_source(dims, 0)
    op = oracle.Operator(fat, lng, m, dims)
    ref = oracle.solve(op.apply_A, b, tol=1e-13, max_iter=200000, max_restarts=20)["x"]
    xs_modes = {}
    with _handle(fat, lng, dims, m) as h:
        dd = binding.stag_dd_create(h.h, 4)
        try:
            for mode in (binding.STAG_DD_HOST, binding.STAG_DD_HOST_OVERLAP):
                x = torch.zeros_like(_dev(b))
                code, info, ph = binding.stag_dd_cg_solve(dd, h.h, _dev(b), x, tol, mode=mode)
                assert code == binding.STAG_OK, info
                assert info["true_rel_residual"] <= tol
                assert ph["global_sum"] > 0
                xs_modes[mode] = x.cpu().numpy().reshape(-1)
        finally:
            binding.stag_dd_destroy(dd)
    xs = xs_modes[binding.STAG_DD_HOST]
    assert np.linalg.norm(xs - ref) / np.linalg.norm(ref) <= 1e-8
    # the overlapped exchange changes the schedule, not the arithmetic
    assert np.array_equal(xs_modes[binding.STAG_DD_HOST_OVERLAP], xs)


def test_decomposition_rejects_bad_splits():
    dims = (4, 4, 4, 6)
    fat = inputs.gauge_field(dims, 1)
    with _handle(fat, None, dims, 0.1) as h:
        with pytest.raises(binding.StagError):
            binding.stag_dd_create(h.h, 4)   # 6 / 4 not integral
        with pytest.raises(binding.StagError):
            binding.stag_dd_create(h.h, 6)   # slabs of one t-slice: odd extent
