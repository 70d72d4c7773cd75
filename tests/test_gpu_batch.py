"""Batched solves (stag_batch_*): right-hand sides sharing a field plus lattices of
uneven size, advanced together by multi-RHS FP32 kernels with FP64-class reliable
updates, against the FP64 oracle.

Operator tolerance (FP32 multi-RHS kernels): norm-wise 2e-6, element-wise 1e-5
(2^-24 rounding per product, 96 products per component).  Solves: true residual
<= 1e-10 and |x - x_oracle| / |x_oracle| <= 1e-8 (oracle solution to 1e-13).
"""
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


def _systems():
    """A 5-RHS group on one 8^4 asqtad field (a partly filled RHS chunk) and
    three single-RHS lattices of different sizes and operators."""
    systems = []
    fat, lng = inputs.asqtad_form_fields((8, 8, 8, 8), seeds=(71, 72, 73))
    fat_d, lng_d = _dev(fat), _dev(lng)
    for k in range(5):
        systems.append(dict(dims=(8, 8, 8, 8), fat=fat, lng=lng, fat_d=fat_d, lng_d=lng_d, mass=0.03,
                            b=inputs.gaussian_even_source((8, 8, 8, 8), 100 + k)))
    for dims, naik, mass, seed in (((4, 4, 4, 4), False, 0.1, 74), ((6, 4, 2, 8), True, 0.05, 75),
                                   ((8, 8, 8, 16), True, 0.04, 78)):
        if naik:
            f, l = inputs.asqtad_form_fields(dims, seeds=(seed, seed + 10, seed + 20))
        else:
            f, l = inputs.gauge_field(dims, seed), None
        systems.append(dict(dims=dims, fat=f, lng=l, fat_d=_dev(f), lng_d=None if l is None else _dev(l),
                            mass=mass, b=inputs.gaussian_even_source(dims, seed)))
    return systems


@pytest.fixture(scope="module")
def systems():
    return _systems()


def _batch(systems, **kw):
    opt = binding.stag_default_options()
    for k, v in kw.items():
        setattr(opt, k, v)
    return binding.stag_batch_create([s["fat_d"] for s in systems], [s["lng_d"] for s in systems],
                                     [s["dims"] for s in systems], [s["mass"] for s in systems], opt)


def test_batch_groups_and_tuning(systems):
    bt = _batch(systems)
    try:
        rb, bs, ms, sw = binding.stag_batch_tuning(bt, 0)
        assert rb in (1, 2, 4, 8) and bs in (64, 128, 256) and ms > 0 and sw in (0, 1)
        assert binding.stag_batch_tuning(bt, 4)[:2] == (rb, bs)  # same group
        rb1, bs1, _, sw1 = binding.stag_batch_tuning(bt, 5)
        assert rb1 == 1 and bs1 in (64, 128, 256) and sw1 in (0, 1)
        # shapes outside the candidates are rejected
        for bad in ((0, 3, 64, 0), (0, 16, 64, 0), (5, 2, 64, 0), (0, 2, 96, 0), (0, 2, 64, 2)):
            with pytest.raises(binding.StagError):
                binding.stag_batch_set_tuning(bt, *bad)
        assert binding.stag_batch_device_bytes(bt) > 0
    finally:
        binding.stag_batch_destroy(bt)


# every candidate of the autotuner for the 5-RHS group (padded to 8): RB RHS per thread
# (8 / RB threads per site; RB >= 4 uses the 256-bit accesses), threads per block, and the
# four traversals; the single-RHS groups run every block size and traversal alongside
SHAPES = [(rb, bs, sw) for sw in (0, 1) for rb in (1, 2, 4, 8) for bs in (64, 128, 256)]


@pytest.fixture(scope="module")
def operator_refs(systems):
    ins = [inputs.gaussian_even_source(s["dims"], 200 + k) for k, s in enumerate(systems)]
    refs = [oracle.Operator(s["fat"], s["lng"], s["mass"], s["dims"]).apply_A(v) for s, v in zip(systems, ins)]
    return ins, refs


@pytest.mark.parametrize("rb,bs,sweep", SHAPES)
def test_batch_operator_parity(systems, operator_refs, rb, bs, sweep):
    ins_h, refs = operator_refs
    bt = _batch(systems, autotune=0)
    try:
        binding.stag_batch_set_tuning(bt, 0, rb, bs, sweep)
        for k in (5, 6, 7):
            binding.stag_batch_set_tuning(bt, k, 1, bs, sweep)
        assert binding.stag_batch_tuning(bt, 0)[::3] == (rb, sweep)
        ins = [_dev(v) for v in ins_h]
        outs = [torch.full_like(v, float("nan")) for v in ins]
        binding.stag_batch_apply_A(bt, ins, outs)
    finally:
        binding.stag_batch_destroy(bt)
    for s, o, ref in zip(systems, outs, refs):
        got = o.cpu().numpy()
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        elem = np.abs(got - ref).max() / np.abs(ref).max()
        assert rel <= 2e-6 and elem <= 1e-5, (s["dims"], rel, elem)


@pytest.mark.parametrize("autotune,sweep", [(1, None), (0, 0), (0, 1)])
def test_batch_solve(systems, autotune, sweep):
    tol = 1e-10
    bt = _batch(systems, autotune=autotune, check_interval=8)
    try:
        if sweep is not None:  # the fixed shapes, with each traversal of the site tiles
            binding.stag_batch_set_tuning(bt, 0, 4, 128, sweep)
            for k in (5, 6, 7):
                binding.stag_batch_set_tuning(bt, k, 1, 128, sweep)
        bs = [_dev(s["b"]) for s in systems]
        xs = [torch.zeros_like(b) for b in bs]
        code, infos = binding.stag_batch_solve(bt, bs, xs, tol, max_iter=20000)
    finally:
        binding.stag_batch_destroy(bt)
    assert code == binding.STAG_OK, infos
    for s, x, info in zip(systems, xs, infos):
        assert info["status"] == binding.STAG_OK and info["true_rel_residual"] <= tol, info
        assert info["reliable_updates"] >= 1
        op = oracle.Operator(s["fat"], s["lng"], s["mass"], s["dims"])
        ref = oracle.solve(op.apply_A, s["b"], tol=1e-13, max_iter=200000, max_restarts=20)["x"]
        xs_ = x.cpu().numpy().reshape(-1)
        r = s["b"].reshape(-1) - op.apply_A(xs_).reshape(-1)
        assert np.linalg.norm(r) <= tol * np.linalg.norm(s["b"]) * 1.01
        assert np.linalg.norm(xs_ - ref) / np.linalg.norm(ref) <= 1e-8


def test_batch_host_vectors_and_determinism(systems):
    sub = systems[:2] + systems[5:6]
    bt = _batch(sub)
    try:
        bs = [s["b"] for s in sub]                     # host arrays
        x1 = [np.zeros_like(b) for b in bs]
        x2 = [np.zeros_like(b) for b in bs]
        c1, _ = binding.stag_batch_solve(bt, bs, x1, 1e-10)
        c2, _ = binding.stag_batch_solve(bt, bs, x2, 1e-10)
    finally:
        binding.stag_batch_destroy(bt)
    assert c1 == c2 == binding.STAG_OK
    for a, b in zip(x1, x2):
        assert np.array_equal(a, b)


def test_batch_zero_source_and_bad_args(systems):
    s = systems[5]
    bt = _batch([s])
    try:
        b = torch.zeros_like(_dev(s["b"]))
        x = torch.ones_like(b)
        code, infos = binding.stag_batch_solve(bt, [b], [x], 1e-10)
        assert code == binding.STAG_OK and infos[0]["iters"] == 0
        assert torch.count_nonzero(x) == 0
    finally:
        binding.stag_batch_destroy(bt)
    with pytest.raises(binding.StagError):
        binding.stag_batch_create([s["fat_d"]], [None], [(4, 4, 3, 4)], [0.1])


def test_batch_breakdown_and_budget_end_only_their_systems(systems):
    """The device-side reliable-update pass ends a system on a CG breakdown (free field at
    m = 0 with a constant source: a zero mode of A, so d^dag A d = 0) and on an exhausted
    iteration budget, while the other systems of the same batch converge to the oracle."""
    tol = 1e-10
    dims0 = (4, 4, 4, 4)
    unit = np.zeros((4, 4, 4, 4, 4, 3, 3), dtype=np.complex128)
    unit[..., 0, 0] = unit[..., 1, 1] = unit[..., 2, 2] = 1.0
    b0 = np.zeros((128, 3), dtype=np.complex128)
    b0[:, 0] = 1.0
    good = systems[5]
    bt = binding.stag_batch_create([_dev(unit), good["fat_d"]], [None, good["lng_d"]], [dims0, good["dims"]],
                                   [0.0, good["mass"]])
    try:
        bs = [_dev(b0), _dev(good["b"])]
        xs = [torch.zeros_like(b) for b in bs]
        code, infos = binding.stag_batch_solve(bt, bs, xs, tol, max_iter=20000)
    finally:
        binding.stag_batch_destroy(bt)
    assert code == binding.STAG_ERR_BREAKDOWN
    assert infos[0]["status"] == binding.STAG_ERR_BREAKDOWN
    assert infos[1]["status"] == binding.STAG_OK and infos[1]["true_rel_residual"] <= tol, infos[1]
    op = oracle.Operator(good["fat"], good["lng"], good["mass"], good["dims"])
    ref = oracle.solve(op.apply_A, good["b"], tol=1e-13, max_iter=200000, max_restarts=20)["x"]
    x1 = xs[1].cpu().numpy().reshape(-1)
    assert np.linalg.norm(x1 - ref) / np.linalg.norm(ref) <= 1e-8

    # an iteration budget of 7: every system stops after exactly 7 iterations, not converged
    sub = systems[:2] + systems[5:6]
    bt = _batch(sub)
    try:
        bs = [_dev(s["b"]) for s in sub]
        xs = [torch.zeros_like(b) for b in bs]
        code, infos = binding.stag_batch_solve(bt, bs, xs, tol, max_iter=7)
    finally:
        binding.stag_batch_destroy(bt)
    assert code == binding.STAG_ERR_NOT_CONVERGED
    for x, info in zip(xs, infos):
        assert info["status"] == binding.STAG_ERR_NOT_CONVERGED and info["iters"] == 7, info
        assert 1e-10 < info["true_rel_residual"] < 1.0
        assert torch.isfinite(x).all() and x.abs().sum() > 0
