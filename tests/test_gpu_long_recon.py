"""Float-float Dirac kernels with two-row Naik links (option long_recon = 12).

The Naik links of the asqtad-form fields are c x SU(3) with c = -1/24; the
kernel stores their first two rows and rebuilds the third as
(eta / c) conj(row0 x row1) (Sec. 3.3's 12-parameter form for a scaled SU(3)
matrix).  Same bars as the nine-entry float-float kernels: the rebuilt entries
carry a few float-float roundings (about 2^-48 each) and the stored SU(3)
matrices are unitary to FP64 rounding, so
  * operator parity: norm and elem <= 1e-13 against the FP64 oracle (worst
    element error measured on GB300: 4.0e-14);
  * solves: true residual <= 1e-10, |x - x_oracle| / |x_oracle| <= 1e-8, and the
    iteration count of the nine-entry float-float solve within 2.
Links that are not c x SU(3) (the fat links, or the right matrices with the
wrong sign of c, whose determinant is then -1) must be rejected at creation.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1010_4782_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

TOL_OP, TOL_ELEM = 1e-13, 1e-13
C = inputs.NAIK_COEFF


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_4782_gb300 import build

    build.build()
    binding.load()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _handle(fat, lng, dims, mass, long_recon=12, long_scale=C):
    opt = binding.stag_default_options()
    opt.arith = binding.STAG_ARITH_FF
    opt.long_recon = long_recon
    opt.long_scale = long_scale
    return binding.Handle(_dev(fat), dims, mass, naik_long=_dev(lng), options=opt)


def _close(got, ref):
    got, ref = np.asarray(got).reshape(-1), np.asarray(ref).reshape(-1)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    elem = np.abs(got - ref).max() / np.abs(ref).max()
    assert rel <= TOL_OP and elem <= TOL_ELEM, (rel, elem)


DIMS = [(4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 2, 8), (10, 6, 4, 12), (8, 8, 8, 16)]


@pytest.mark.parametrize("dims", DIMS)
def test_dslash_half_parity(dims):
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(7, 8, 9))
    op = oracle.Operator(fat, lng, 0.1, dims)
    with _handle(fat, lng, dims, 0.1) as h:
        for p_out in (0, 1):
            v = inputs.gaussian_vector(op.n_half, 100 + p_out)
            out = torch.empty((op.n_half, 3), dtype=torch.complex128, device="cuda")
            binding.stag_dslash(h.h, p_out, _dev(v), out)
            _close(out.cpu().numpy(), op.dslash_half(v, p_out))


@pytest.mark.parametrize("dims", DIMS)
def test_apply_A_parity(dims):
    mass = 0.05
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(17, 18, 19))
    op = oracle.Operator(fat, lng, mass, dims)
    v = inputs.gaussian_even_source(dims, 3)
    with _handle(fat, lng, dims, mass) as h:
        out = torch.empty_like(_dev(v))
        binding.stag_apply_A(h.h, _dev(v), out)
        _close(out.cpu().numpy(), op.apply_A(v))


@pytest.mark.parametrize("dims,mass", [((8, 8, 8, 16), 0.05), ((6, 4, 2, 8), 0.02), ((10, 6, 4, 12), 0.031)])
def test_solve_matches_oracle_and_nine_entry_iterations(dims, mass):
    tol = 1e-10
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(11, 12, 13))
    b = inputs.gaussian_even_source(dims, 0)
    op = oracle.Operator(fat, lng, mass, dims)
    x_ref = oracle.solve(op.apply_A, b, tol=1e-13, max_iter=200000, max_restarts=20)["x"]
    iters = {}
    for recon in (0, 12):
        with _handle(fat, lng, dims, mass, long_recon=recon) as h:
            x = torch.zeros_like(_dev(b))
            code, info = binding.stag_cg_solve(h.h, _dev(b), x, tol)
        assert code == binding.STAG_OK and info["true_rel_residual"] <= tol, info
        xs = x.cpu().numpy().reshape(-1)
        r = b.reshape(-1) - op.apply_A(xs).reshape(-1)
        assert np.linalg.norm(r) <= tol * np.linalg.norm(b) * 1.01
        assert np.linalg.norm(xs - x_ref) / np.linalg.norm(x_ref) <= 1e-8
        iters[recon] = info["iters"]
    assert abs(iters[12] - iters[0]) <= 2, iters


@pytest.mark.parametrize("which", ["fat_links", "wrong_sign", "wrong_size"])
def test_rejects_links_that_are_not_scaled_su3(which):
    dims = (4, 4, 4, 4)
    fat, lng = inputs.asqtad_form_fields(dims)
    links, scale = {"fat_links": (fat, C), "wrong_sign": (lng, -C), "wrong_size": (lng, 2 * C)}[which]
    with pytest.raises(binding.StagError) as e:
        _handle(fat, links, dims, 0.1, long_scale=scale)
    assert e.value.code == binding.STAG_ERR_INVALID_ARG
    assert "SU(3)" in binding.stag_last_error(None)


@pytest.mark.parametrize("scale", [1.5e-10, -1.5e-10, 8e17, -8e17])
def test_parity_at_the_ends_of_the_scale_range(scale):
    """Naik links c x SU(3) with |c| near the ends of the accepted range 1e-10 .. 1e18.  The
    fat links and the mass are scaled by the same factor k = |c| / (1/24), so the Naik term
    keeps its usual weight in D; the rebuilt third row, whose float-float products are of
    size c^2, must still meet the bars against the oracle (both half-Dslash parities, and A
    where k^2 stays inside the FP32 range)."""
    dims = (6, 4, 2, 8)
    k = abs(scale / C)
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(27, 28, 29))
    fat, lng = fat * k, lng * (scale / C)
    mass = 0.1 * k
    op = oracle.Operator(fat, lng, mass, dims)
    with _handle(fat, lng, dims, mass, long_scale=scale) as h:
        for p_out in (0, 1):
            v = inputs.gaussian_vector(op.n_half, 200 + p_out)
            out = torch.empty((op.n_half, 3), dtype=torch.complex128, device="cuda")
            binding.stag_dslash(h.h, p_out, _dev(v), out)
            _close(out.cpu().numpy(), op.dslash_half(v, p_out))
        if k < 1.0:
            v = inputs.gaussian_even_source(dims, 5)
            out = torch.empty_like(_dev(v))
            binding.stag_apply_A(h.h, _dev(v), out)
            _close(out.cpu().numpy(), op.apply_A(v))
