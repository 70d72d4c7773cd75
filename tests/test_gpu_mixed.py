"""Mixed-precision reliable-update CG (the paper's stated next step, Sec. 5) and
the low-precision operators it runs on, against the FP64 oracle.

Operator tolerances (relative, norm-wise / element-wise against max |ref|):
  * FP32 links, vectors and arithmetic: 2e-6 / 1e-5.  Each of the up to 96
    products per component carries 2^-24 = 6e-8 rounding, and the odd
    intermediate is rounded to FP32 once more.
  * FP16-stored links and vectors (FP32 arithmetic): 2e-3 / 2e-2.  Storage
    rounding is 2^-11 = 4.9e-4 relative per entry (links, input, intermediate,
    output), averaged over the sums.
  * BF16-stored links and vectors (FP32 arithmetic): 1.6e-2 / 1.6e-1, the FP16
    bounds scaled by the ratio of unit roundoffs 2^-8 / 2^-11 = 8.
Solves must meet the same bars as the FP64 solver: true residual <= 1e-10 and
|x - x_oracle| / |x_oracle| <= 1e-8 against an oracle solution taken to 1e-13.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1010_4782_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

OP_TOL = {binding.STAG_ARITH_F32: (2e-6, 1e-5), binding.STAG_ARITH_F16: (2e-3, 2e-2),
          binding.STAG_ARITH_BF16: (1.6e-2, 1.6e-1)}
INNER_OF = {binding.STAG_ARITH_F32: binding.STAG_INNER_F32, binding.STAG_ARITH_F16: binding.STAG_INNER_F16,
            binding.STAG_ARITH_BF16: binding.STAG_INNER_BF16}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_4782_gb300 import build

    build.build()
    binding.load()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _fields(dims, naik, seed):
    if naik:
        return inputs.asqtad_form_fields(dims, seeds=(seed, seed + 1, seed + 2))
    return inputs.gauge_field(dims, seed), None


def _handle(fat, lng, dims, mass, arith=binding.STAG_ARITH_FF, inner=binding.STAG_INNER_NONE, **kw):
    opt = binding.stag_default_options()
    opt.arith = arith
    opt.inner = inner
    for k, v in kw.items():
        setattr(opt, k, v)
    return binding.Handle(_dev(fat), dims, mass, naik_long=None if lng is None else _dev(lng), options=opt)


@pytest.mark.parametrize("prec", [binding.STAG_ARITH_F32, binding.STAG_ARITH_F16, binding.STAG_ARITH_BF16])
@pytest.mark.parametrize("naik", [False, True])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (10, 6, 4, 12), (8, 8, 8, 16)])
def test_low_precision_operator(dims, naik, prec):
    mass = 0.05
    fat, lng = _fields(dims, naik, 61)
    ref = oracle.Operator(fat, lng, mass, dims).apply_A(v := inputs.gaussian_even_source(dims, 62))
    with _handle(fat, lng, dims, mass, inner=INNER_OF[prec]) as h:
        out = torch.empty_like(_dev(v))
        binding.stag_apply_A_prec(h.h, prec, _dev(v), out)
    got = out.cpu().numpy()
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    elem = np.abs(got - ref).max() / np.abs(ref).max()
    tn, te = OP_TOL[prec]
    assert rel <= tn and elem <= te, (rel, elem)


def test_apply_A_prec_fp64_classes_match_apply_A():
    dims = (6, 4, 2, 8)
    fat, lng = _fields(dims, True, 63)
    v = _dev(inputs.gaussian_even_source(dims, 64))
    with _handle(fat, lng, dims, 0.1, arith=binding.STAG_ARITH_FF) as h:
        a, b = torch.empty_like(v), torch.empty_like(v)
        binding.stag_apply_A(h.h, v, a)
        binding.stag_apply_A_prec(h.h, binding.STAG_ARITH_FF, v, b)
        assert torch.equal(a, b)
        c = torch.empty_like(v)
        binding.stag_apply_A_prec(h.h, binding.STAG_ARITH_F64, v, c)
        ref = oracle.Operator(fat, lng, 0.1, dims).apply_A(v.cpu().numpy())
        assert np.linalg.norm(c.cpu().numpy() - ref) <= 1e-13 * np.linalg.norm(ref)
        with pytest.raises(binding.StagError) as e:
            binding.stag_apply_A_prec(h.h, binding.STAG_ARITH_F32, v, c)
        assert e.value.code == binding.STAG_ERR_INVALID_ARG


def _oracle_x(fat, lng, mass, dims, b):
    op = oracle.Operator(fat, lng, mass, dims)
    return op, oracle.solve(op.apply_A, b, tol=1e-13, max_iter=200000, max_restarts=20)["x"]


CASES = [((4, 4, 4, 4), False, 0.1, 1),     # the config-1 system
         ((8, 8, 8, 16), True, 0.05, 11),
         ((10, 6, 4, 12), True, 0.031, 13),
         ((8, 8, 8, 8), False, 0.02, 17)]


@pytest.mark.parametrize("arith", [binding.STAG_ARITH_FF, binding.STAG_ARITH_F64])
@pytest.mark.parametrize("inner", [binding.STAG_INNER_F32, binding.STAG_INNER_F16, binding.STAG_INNER_BF16,
                                   binding.STAG_INNER_F32_L16])
@pytest.mark.parametrize("case", CASES)
def test_mixed_solve(case, inner, arith):
    dims, naik, mass, seed = case
    tol = 1e-10
    fat, lng = (inputs.gauge_field(dims, seed), None) if not naik else _fields(dims, True, seed)
    b = inputs.gaussian_even_source(dims, 0)
    op, x_ref = _oracle_x(fat, lng, mass, dims, b)
    with _handle(fat, lng, dims, mass, arith=arith, inner=inner) as h:
        x = torch.zeros_like(_dev(b))
        code, info = binding.stag_cg_solve(h.h, _dev(b), x, tol, max_iter=20000)
    assert code == binding.STAG_OK, info
    assert info["true_rel_residual"] <= tol
    assert info["reliable_updates"] >= 1
    xs = x.cpu().numpy().reshape(-1)
    r = b.reshape(-1) - op.apply_A(xs).reshape(-1)
    assert np.linalg.norm(r) <= tol * np.linalg.norm(b) * 1.01
    assert np.linalg.norm(xs - x_ref) / np.linalg.norm(x_ref) <= 1e-8


def test_mixed_fp32_iteration_count_close_to_fp64():
    """FP32 vectors cost at most 30 % more iterations than FP64-class CG with FP32
    links, and at most 50 % more with FP16-stored links: rounding the links to FP16
    (2^-11 relative) perturbs the inner operator by ~5e-4, so each inner cycle
    gets less far before its residual is replaced (measured: +33 % on this system)."""
    dims, mass = (8, 8, 8, 16), 0.05
    fat, lng = _fields(dims, True, 11)
    b = _dev(inputs.gaussian_even_source(dims, 0))
    its = {}
    for inner in (binding.STAG_INNER_NONE, binding.STAG_INNER_F32, binding.STAG_INNER_F32_L16):
        with _handle(fat, lng, dims, mass, inner=inner) as h:
            x = torch.zeros_like(b)
            code, info = binding.stag_cg_solve(h.h, b, x, 1e-10)
            assert code == binding.STAG_OK
            its[inner] = info["iters"]
    assert its[binding.STAG_INNER_F32] <= 1.3 * its[binding.STAG_INNER_NONE]
    assert its[binding.STAG_INNER_F32_L16] <= 1.5 * its[binding.STAG_INNER_NONE], its


def test_mixed_rejects_bad_options():
    dims = (4, 4, 4, 4)
    fat, _ = _fields(dims, False, 1)
    with pytest.raises(binding.StagError):
        _handle(fat, None, dims, 0.1, inner=binding.STAG_INNER_F32, reliable_delta=1.5)
    with pytest.raises(binding.StagError):
        _handle(fat, None, dims, 0.1, inner=7)


# ---- 12-parameter links (Sec. 3.3): two stored rows, the third rebuilt in the kernel

def _recon_handle(fat, dims, mass):
    return _handle(fat, None, dims, mass, inner=binding.STAG_INNER_F32, link_recon=12)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (10, 6, 4, 12), (8, 8, 8, 16)])
def test_recon12_operator(dims):
    """SU(3) links (exp(0.3 i H)) rebuilt from two rows: the FP32 bound of the
    full-link operator holds (the rebuilt row carries a few FP32 roundings)."""
    mass = 0.05
    fat = inputs.gauge_field(dims, 71)
    v = inputs.gaussian_even_source(dims, 72)
    ref = oracle.Operator(fat, None, mass, dims).apply_A(v)
    with _recon_handle(fat, dims, mass) as h:
        out = torch.empty_like(_dev(v))
        binding.stag_apply_A_prec(h.h, binding.STAG_ARITH_F32, _dev(v), out)
    got = out.cpu().numpy()
    tn, te = OP_TOL[binding.STAG_ARITH_F32]
    assert np.linalg.norm(got - ref) <= tn * np.linalg.norm(ref)
    assert np.abs(got - ref).max() <= te * np.abs(ref).max()


@pytest.mark.parametrize("case", [((4, 4, 4, 4), 0.1, 1), ((8, 8, 8, 8), 0.02, 17)])
def test_recon12_mixed_solve(case):
    dims, mass, seed = case
    tol = 1e-10
    fat = inputs.gauge_field(dims, seed)
    b = inputs.gaussian_even_source(dims, 0)
    op, x_ref = _oracle_x(fat, None, mass, dims, b)
    with _recon_handle(fat, dims, mass) as h:
        x = torch.zeros_like(_dev(b))
        code, info = binding.stag_cg_solve(h.h, _dev(b), x, tol, max_iter=20000)
    assert code == binding.STAG_OK and info["true_rel_residual"] <= tol, info
    assert info["fallbacks"] == 0
    xs = x.cpu().numpy().reshape(-1)
    assert np.linalg.norm(xs - x_ref) / np.linalg.norm(x_ref) <= 1e-8


def test_recon12_rejects_naik_and_other_inner():
    dims = (4, 4, 4, 4)
    fat, lng = _fields(dims, True, 3)
    with pytest.raises(binding.StagError):
        _handle(fat, lng, dims, 0.1, inner=binding.STAG_INNER_F32, link_recon=12)
    with pytest.raises(binding.StagError):
        _handle(fat, None, dims, 0.1, inner=binding.STAG_INNER_F16, link_recon=12)
    with pytest.raises(binding.StagError):
        _handle(fat, None, dims, 0.1, inner=binding.STAG_INNER_F32, link_recon=8)


# ---- two-row Naik links (long_recon = 12) in the FP32 iteration: the asqtad Naik links
# are c x SU(3) (c = -1/24), so the 12-parameter form of Sec. 3.3 applies with the third
# row rebuilt as (eta / c) conj(row0 x row1), in FP32

def _long_recon_handle(fat, lng, dims, mass):
    return _handle(fat, lng, dims, mass, inner=binding.STAG_INNER_F32, long_recon=12,
                   long_scale=inputs.NAIK_COEFF)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (10, 6, 4, 12), (8, 8, 8, 16)])
def test_long_recon12_fp32_operator(dims):
    """The FP32 operator with two-row Naik links meets the FP32 bars of the nine-entry
    operator against the oracle (the rebuilt row carries a few FP32 roundings of
    entries of size |c|)."""
    mass = 0.05
    fat, lng = _fields(dims, True, 81)
    v = inputs.gaussian_even_source(dims, 82)
    ref = oracle.Operator(fat, lng, mass, dims).apply_A(v)
    with _long_recon_handle(fat, lng, dims, mass) as h:
        out = torch.empty_like(_dev(v))
        binding.stag_apply_A_prec(h.h, binding.STAG_ARITH_F32, _dev(v), out)
    got = out.cpu().numpy()
    tn, te = OP_TOL[binding.STAG_ARITH_F32]
    assert np.linalg.norm(got - ref) <= tn * np.linalg.norm(ref)
    assert np.abs(got - ref).max() <= te * np.abs(ref).max()


@pytest.mark.parametrize("case", [((8, 8, 8, 16), 0.05, 11), ((10, 6, 4, 12), 0.031, 13)])
def test_long_recon12_fp32_mixed_solve(case):
    """Mixed FP32 solves with two-row Naik links in both the FP32 iteration and the
    float-float true residuals: the oracle's solution to 1e-8, no fallback, and the
    iteration count of the nine-entry mixed solve within 2 %."""
    dims, mass, seed = case
    tol = 1e-10
    fat, lng = _fields(dims, True, seed)
    b = inputs.gaussian_even_source(dims, 0)
    op, x_ref = _oracle_x(fat, lng, mass, dims, b)
    its = {}
    for recon in (0, 12):
        h = _long_recon_handle(fat, lng, dims, mass) if recon else _handle(fat, lng, dims, mass,
                                                                          inner=binding.STAG_INNER_F32)
        with h:
            x = torch.zeros_like(_dev(b))
            code, info = binding.stag_cg_solve(h.h, _dev(b), x, tol, max_iter=20000)
        assert code == binding.STAG_OK and info["true_rel_residual"] <= tol, info
        assert info["fallbacks"] == 0
        xs = x.cpu().numpy().reshape(-1)
        assert np.linalg.norm(xs - x_ref) / np.linalg.norm(x_ref) <= 1e-8
        its[recon] = info["iters"]
    assert abs(its[12] - its[0]) <= max(2, 0.02 * its[0]), its
