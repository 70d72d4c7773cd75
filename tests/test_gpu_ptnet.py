"""Learned preconditioner on the GPU against the oracle (oracle/ptnet.py).

Tolerances: FP32 activations - forward 2e-6 (three layers of FP32 sums),
loss 1e-5 and gradients vs FP64 central differences of the
oracle's loss 1e-3 relative to the largest checked component; BF16
activations - forward 2e-2 (2^-8 storage rounding per layer).
Flexible CG meets the solver bars: true residual <= 1e-10, x within 1e-8 of the
oracle solution.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import ptnet
from paper_1010_4782_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

CHANS = (1, 8, 8, 1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_4782_gb300 import build

    build.build()
    binding.load()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _split(wflat):
    out, off = [], 0
    for ci, co in zip(CHANS[:-1], CHANS[1:]):
        n = 9 * co * ci
        out.append(wflat[off:off + n].reshape(9, co, ci))
        off += n
    return out


def _random_flat(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    n = sum(9 * co * ci for ci, co in zip(CHANS[:-1], CHANS[1:]))
    return scale * (rng.standard_normal(n) + 1j * rng.standard_normal(n))


def _handle(fat, lng, dims, mass, arith=binding.STAG_ARITH_FF):
    opt = binding.stag_default_options()
    opt.arith = arith
    return binding.Handle(_dev(fat), dims, mass, naik_long=None if lng is None else _dev(lng), options=opt)


FORMS = (binding.STAG_PTNET_COLLAPSED, binding.STAG_PTNET_LAYERED)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("prec,tol", [(binding.STAG_ARITH_F32, 2e-6), (binding.STAG_ARITH_BF16, 2e-2)])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (10, 6, 4, 12)])
def test_forward_parity(dims, prec, tol, form):
    """The applied network (both inference forms) against the oracle's layers."""
    fat = inputs.gauge_field(dims, 81)
    w = _random_flat(82)
    r = inputs.gaussian_even_source(dims, 83)
    ref = ptnet.PTNet(fat, dims, _split(w)).apply(r)
    with _handle(fat, None, dims, 0.1) as h:
        net = binding.stag_ptnet_create(h.h, prec, 1)
        try:
            binding.stag_ptnet_set_inference_form(net, form)
            binding.stag_ptnet_set_weights(net, w)
            z = torch.empty_like(_dev(r))
            binding.stag_ptnet_apply(net, _dev(r), z)
        finally:
            binding.stag_ptnet_destroy(net)
    got = z.cpu().numpy()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("c", [1e5, 1e-6])
def test_two_hop_form_with_links_far_from_one(c):
    """The two-hop form with BF16 storage reads FP16 links divided by a power of two
    near their largest entry.  Links scaled by 1e5 (beyond FP16's range) and by 1e-6
    (FP16 subnormals unscaled), against the oracle at the BF16 bound.  The first
    layer's identity path is zero, so k0 = 0 and the output is the two-hop part
    alone (which, at 1e-6, would otherwise sit below the FP32 rounding of k0 r)."""
    dims = (6, 4, 2, 8)
    fat = inputs.gauge_field(dims, 81) * c
    w = _random_flat(82)
    w[:8] = 0.0   # W1[0][:][0]
    r = inputs.gaussian_even_source(dims, 83)
    ref = ptnet.PTNet(fat, dims, _split(w)).apply(r)
    with _handle(fat, None, dims, 0.1) as h:
        net = binding.stag_ptnet_create(h.h, binding.STAG_ARITH_BF16, 1)
        try:
            binding.stag_ptnet_set_weights(net, w)
            z = torch.empty_like(_dev(r))
            binding.stag_ptnet_apply(net, _dev(r), z)
        finally:
            binding.stag_ptnet_destroy(net)
    got = z.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 2e-2 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (10, 6, 4, 12), (8, 8, 8, 16)])
def test_tensor_core_layer_matches_cuda_cores_and_oracle(dims):
    """The BF16 network with its 8 -> 8 channel mixing on the tensor cores against
    the same network on the CUDA cores and the FP64 oracle, on lattices of 1, 11.25
    (ragged) and 32 tiles of 128 sites per parity.  Both BF16 paths round the
    stored activations (2^-9 relative); the tensor-core path also rounds the
    transported inputs of the mixing, so the bound is that of the BF16 parity test."""
    fat = inputs.gauge_field(dims, 84)
    w = _random_flat(85)
    r = inputs.gaussian_even_source(dims, 86)
    ref = ptnet.PTNet(fat, dims, _split(w)).apply(r)
    outs = {}
    with _handle(fat, None, dims, 0.1) as h:
        net = binding.stag_ptnet_create(h.h, binding.STAG_ARITH_BF16, 1)
        try:
            binding.stag_ptnet_set_inference_form(net, binding.STAG_PTNET_LAYERED)
            binding.stag_ptnet_set_weights(net, w)
            for tc in (True, False):
                binding.stag_ptnet_use_tensor_cores(net, tc)
                z = torch.empty_like(_dev(r))
                binding.stag_ptnet_apply(net, _dev(r), z)
                outs[tc] = z.cpu().numpy()
        finally:
            binding.stag_ptnet_destroy(net)
    for tc, got in outs.items():
        assert np.linalg.norm(got - ref) <= 2e-2 * np.linalg.norm(ref), tc
    assert np.linalg.norm(outs[True] - outs[False]) <= 2e-2 * np.linalg.norm(ref)
    assert np.linalg.norm(outs[True] - outs[False]) > 0.0   # the two paths really differ


@pytest.mark.parametrize("form", FORMS)
def test_network_weights_reproducing_A(form):
    """Layer 1: (r, D r); layer 2: m^2 r - D(D r); layer 3: identity => the network is A."""
    dims, m = (4, 6, 4, 8), 0.3
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(84, 85, 86))
    w1 = np.zeros((9, 8, 1), complex)
    w2 = np.zeros((9, 8, 8), complex)
    w3 = np.zeros((9, 1, 8), complex)
    w1[0, 0, 0] = 1
    w2[0, 0, 0] = m ** 2
    w3[0, 0, 0] = 1
    for mu in range(4):
        w1[1 + 2 * mu, 1, 0], w1[2 + 2 * mu, 1, 0] = 1, -1
        w2[1 + 2 * mu, 0, 1], w2[2 + 2 * mu, 0, 1] = -1, 1
    w = np.concatenate([w1.ravel(), w2.ravel(), w3.ravel()])
    v = inputs.gaussian_even_source(dims, 87)
    with _handle(fat, None, dims, m) as h:   # one-hop operator
        net = binding.stag_ptnet_create(h.h, binding.STAG_ARITH_F32, 1)
        try:
            binding.stag_ptnet_set_inference_form(net, form)
            binding.stag_ptnet_set_weights(net, w)
            z = torch.empty_like(_dev(v))
            binding.stag_ptnet_apply(net, _dev(v), z)
            a = torch.empty_like(z)
            binding.stag_apply_A(h.h, _dev(v), a)
        finally:
            binding.stag_ptnet_destroy(net)
    assert torch.linalg.vector_norm(z - a) <= 2e-6 * torch.linalg.vector_norm(a)


def test_gradient_matches_oracle_finite_differences():
    dims = (4, 4, 4, 4)
    fat = inputs.gauge_field(dims, 91)
    w = _random_flat(92, 0.2)
    r = inputs.gaussian_even_source(dims, 93)
    e = inputs.gaussian_even_source(dims, 94)
    with _handle(fat, None, dims, 0.1) as h:
        net = binding.stag_ptnet_create(h.h, binding.STAG_ARITH_F32, 1)
        try:
            binding.stag_ptnet_set_weights(net, w)
            loss, grad = binding.stag_ptnet_loss_grad(net, _dev(r), _dev(e))
        finally:
            binding.stag_ptnet_destroy(net)
    onet = ptnet.PTNet(fat, dims, _split(w))
    A = oracle.Operator(fat, None, 0.1, dims).apply_A
    assert loss == pytest.approx(onet.loss(r, e, A), rel=1e-5)
    rng = np.random.default_rng(95)
    idx = np.concatenate([rng.choice(72, 6, replace=False), 72 + rng.choice(576, 10, replace=False),
                          648 + rng.choice(72, 6, replace=False)])
    fd, gpu = [], []
    for k in idx:
        for part in (1.0, 1j):
            hstep = 1e-6
            wp, wm = w.copy(), w.copy()
            wp[k] += hstep * part
            wm[k] -= hstep * part
            lp = ptnet.PTNet(fat, dims, _split(wp)).loss(r, e, A)
            lm = ptnet.PTNet(fat, dims, _split(wm)).loss(r, e, A)
            fd.append((lp - lm) / (2 * hstep))
            gpu.append(2 * (grad[k].real if part == 1.0 else grad[k].imag))
    fd, gpu = np.array(fd), np.array(gpu)
    assert np.abs(fd - gpu).max() <= 1e-3 * np.abs(fd).max()


def _poor_start():
    """0.1 * identity through channel 0 - a deliberately poor starting point."""
    w = _random_flat(111, 0.002)
    w1, w2, w3 = _split(w.copy())
    w1[0, 0, 0] += 1
    w2[0, 0, 0] += 1
    w3[0, 0, 0] += 0.1
    return np.concatenate([w1.ravel(), w2.ravel(), w3.ravel()])


@pytest.fixture(scope="module")
def trained():
    """8^4 asqtad-form field, m = 0.05: pairs from plain-CG solves; one BF16 network from
    the library's polynomial start, one from a poor start, both trained on the pairs."""
    dims, m = (8, 8, 8, 8), 0.05
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(101, 102, 103))
    h = _handle(fat, lng, dims, m)
    sources = [_dev(inputs.gaussian_even_source(dims, 200 + k)) for k in range(4)]
    out = dict(dims=dims, m=m, fat=fat, lng=lng, h=h)
    for name, weights in (("poly", None), ("poor", _poor_start())):
        net = binding.stag_ptnet_create(h.h, binding.STAG_ARITH_BF16, 7)
        if weights is not None:
            binding.stag_ptnet_set_weights(net, weights)
        npairs = binding.stag_ptnet_add_pairs(net, sources, stride=2, min_rel_residual=0.05, max_pairs=400)
        before = binding.stag_ptnet_dataset_loss(net)
        losses = binding.stag_ptnet_train(net, epochs=6, batch=8, lr=3e-3, seed=1)
        after = binding.stag_ptnet_dataset_loss(net)
        out[name] = dict(net=net, npairs=npairs, before=before, after=after, losses=losses)
    yield out
    for name in ("poly", "poor"):
        binding.stag_ptnet_destroy(out[name]["net"])
    h.close()


def test_training_reduces_loss_from_a_poor_start(trained):
    t = trained["poor"]
    assert t["npairs"] >= 100
    assert t["after"] < 0.8 * t["before"], (t["before"], t["after"], t["losses"])
    assert np.all(np.isfinite(t["losses"]))


def test_training_keeps_the_polynomial_start(trained):
    t = trained["poly"]
    assert t["after"] <= 1.001 * t["before"], (t["before"], t["after"], t["losses"])


def _tie_error(w):
    ws = _split(w)
    return max(np.abs(a - b).max() for a, b in zip(ptnet.tie(ws), ws))


def test_training_keeps_the_network_self_adjoint(trained):
    """After training (and from the polynomial start) the weights satisfy the tie
    W3 = W1^dag, W2 = W2^dag of the oracle, and the GPU network is Hermitian."""
    for name in ("poly", "poor"):
        w = binding.stag_ptnet_weights(trained[name]["net"])
        assert _tie_error(w) <= 1e-6 * np.abs(w).max(), name
    dims, net = trained["dims"], trained["poly"]["net"]
    u = _dev(inputs.gaussian_even_source(dims, 700))
    v = _dev(inputs.gaussian_even_source(dims, 701))
    mu, mv = torch.empty_like(u), torch.empty_like(v)
    binding.stag_ptnet_set_inference_precision(net, binding.STAG_ARITH_F32)
    try:
        binding.stag_ptnet_apply(net, u, mu)
        binding.stag_ptnet_apply(net, v, mv)
    finally:
        binding.stag_ptnet_set_inference_precision(net, binding.STAG_ARITH_BF16)
    lhs = torch.vdot(u.reshape(-1), mv.reshape(-1)).item()
    rhs = torch.vdot(mu.reshape(-1), v.reshape(-1)).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


def test_fcg_with_trained_network_gains_over_plain_cg(trained):
    dims, m, h, net = trained["dims"], trained["m"], trained["h"], trained["poly"]["net"]
    op = oracle.Operator(trained["fat"], trained["lng"], m, dims)
    it_fcg, it_cg = [], []
    for k in range(3):
        b = inputs.gaussian_even_source(dims, 500 + k)   # fresh sources
        x = torch.zeros_like(_dev(b))
        code, info = binding.stag_fcg_solve(h.h, net, _dev(b), x, 1e-10, max_iter=20000)
        assert code == binding.STAG_OK, info
        assert info["true_rel_residual"] <= 1e-10
        xs = x.cpu().numpy().reshape(-1)
        ref = oracle.solve(op.apply_A, b, tol=1e-13, max_iter=200000, max_restarts=20)["x"]
        assert np.linalg.norm(xs - ref) / np.linalg.norm(ref) <= 1e-8
        it_fcg.append((info["iters"], info["fallbacks"]))
        x2 = torch.zeros_like(x)
        code, info2 = binding.stag_cg_solve(h.h, _dev(b), x2, 1e-10)
        it_cg.append(info2["iters"])
    assert all(rs == 0 for _, rs in it_fcg), it_fcg  # no fallback to plain CG
    # at least 20 % fewer iterations than CG without the network
    assert sum(i for i, _ in it_fcg) < 0.8 * sum(it_cg), (it_fcg, it_cg)


def test_training_gains_over_the_untrained_network(trained):
    """What training buys, separated from the polynomial start: on the same fresh sources,
    flexible CG with the trained network needs fewer iterations than with the same
    network untrained (a fresh network from the same seed: the polynomial start)."""
    dims, h, net = trained["dims"], trained["h"], trained["poly"]["net"]
    net0 = binding.stag_ptnet_create(h.h, binding.STAG_ARITH_BF16, 7)
    its = {"trained": 0, "untrained": 0}
    try:
        for k in range(4):
            b = _dev(inputs.gaussian_even_source(dims, 900 + k))
            for name, nt in (("trained", net), ("untrained", net0)):
                x = torch.zeros_like(b)
                code, info = binding.stag_fcg_solve(h.h, nt, b, x, 1e-10, max_iter=20000)
                assert code == binding.STAG_OK and info["fallbacks"] == 0, (name, info)
                its[name] += info["iters"]
    finally:
        binding.stag_ptnet_destroy(net0)
    assert its["trained"] < its["untrained"], its


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("arith", [binding.STAG_ARITH_FF, binding.STAG_ARITH_F64])
@pytest.mark.parametrize("prec,tc,tol", [(binding.STAG_ARITH_F32, False, 1e-5),
                                         (binding.STAG_ARITH_BF16, True, 5e-2)])
def test_fcg_iterates_match_oracle(arith, prec, tc, tol, form):
    """Ten flexible-CG iterations from x = 0 (the iteration budget ends the solve)
    against the oracle's flexible CG with the same network weights, in both forms of
    the solver's arithmetic, with the iteration captured in graphs of three (so the
    budget ends inside a graph) and enqueued directly, with the network collapsed
    or layered.  The two launch modes run the same kernels in the same order:
    bit-identical x.  The bound is the network's: FP32 storage (2^-24 per stored
    value, amplified by ten iterations) or BF16 (2^-9 per stored value; the layered
    form with the tensor-core layer)."""
    dims, m, k = (4, 6, 4, 8), 0.05, 10
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(91, 92, 93))
    b = inputs.gaussian_even_source(dims, 94)
    xs = {}
    for graphs in (1, 0):
        opt = binding.stag_default_options()
        opt.arith = arith
        opt.use_graphs = graphs
        opt.check_interval = 3
        with binding.Handle(_dev(fat), dims, m, naik_long=_dev(lng), options=opt) as h:
            net = binding.stag_ptnet_create(h.h, prec, 3)
            try:
                binding.stag_ptnet_set_inference_form(net, form)
                binding.stag_ptnet_use_tensor_cores(net, tc)
                w = binding.stag_ptnet_weights(net)
                x = torch.zeros_like(_dev(b))
                code, info = binding.stag_fcg_solve(h.h, net, _dev(b), x, 1e-10, max_iter=k)
            finally:
                binding.stag_ptnet_destroy(net)
        assert code == binding.STAG_ERR_NOT_CONVERGED, info
        assert info["iters"] == k and info["fallbacks"] == 0 and info["restarts"] == 0, info
        xs[graphs] = x.cpu().numpy().reshape(-1)
    assert np.array_equal(xs[0], xs[1])
    op = oracle.Operator(fat, lng, m, dims)
    ref, its = ptnet.fcg(op.apply_A, ptnet.PTNet(fat, dims, _split(w)).apply, b, tol=1e-10, max_iter=k)
    assert its == k
    err = np.linalg.norm(xs[1] - ref) / np.linalg.norm(ref)
    assert err <= tol, err


def test_fcg_falls_back_to_plain_cg(trained):
    """A network with zero weights gives z = 0: flexible CG hands over to plain CG, which converges."""
    dims, m = (4, 4, 4, 4), 0.1
    fat = inputs.gauge_field(dims, 1)
    with _handle(fat, None, dims, m) as h:
        net = binding.stag_ptnet_create(h.h, binding.STAG_ARITH_BF16, 1)
        try:
            binding.stag_ptnet_set_weights(net, np.zeros(720, complex))
            b = _dev(inputs.gaussian_even_source(dims, 0))
            x = torch.zeros_like(b)
            code, info = binding.stag_fcg_solve(h.h, net, b, x, 1e-10)
        finally:
            binding.stag_ptnet_destroy(net)
    assert code == binding.STAG_OK and info["fallbacks"] >= 1 and info["true_rel_residual"] <= 1e-10
