"""Pins of the parallel-transport network and flexible-CG oracle.

Choices of weights that make the network reproduce the oracle's D (Eq. (5))
and A = m^2 - D^2 (Eq. (3)) pin its transports, embedding and restriction;
gauge covariance and linearity pin the rest; flexible CG reduces to Fig. 1's
CG with the identity preconditioner and to one step with the exact inverse.
"""
import numpy as np
import pytest

import oracle
from oracle import ptnet
from paper_1010_4782_gb300 import inputs


def _d_weights(c_out, c_in, o, i, sign=1.0):
    w = np.zeros((9, c_out, c_in), dtype=np.complex128)
    for mu in range(4):
        w[1 + 2 * mu, o, i] = sign
        w[2 + 2 * mu, o, i] = -sign
    return w


def test_one_layer_reproduces_D():
    dims = (4, 6, 4, 8)
    fat = inputs.random_links(dims, 3)
    net = ptnet.PTNet(fat, dims, [_d_weights(1, 1, 0, 0)])
    r = inputs.gaussian_even_source(dims, 1)
    got = net.activations(r)[1][0]
    op = oracle.Operator(fat, None, 0.1, dims)
    ref = op.D(oracle.embed(r, dims, 0))
    assert np.allclose(got, ref, rtol=0, atol=1e-13)


def test_three_layers_reproduce_A():
    """layer 1: (r, D r); layer 2: m^2 r - D (D r); layer 3: identity  =>  M = A on even sites."""
    dims = (4, 4, 6, 4)
    m = 0.3
    fat = inputs.gauge_field(dims, 5)
    w1 = np.zeros((9, 2, 1), dtype=np.complex128)
    w1[0, 0, 0] = 1.0
    w1 += _d_weights(2, 1, 1, 0)
    w2 = np.zeros((9, 1, 2), dtype=np.complex128)
    w2[0, 0, 0] = m ** 2
    w2 += _d_weights(1, 2, 0, 1, sign=-1.0)
    w3 = np.zeros((9, 1, 1), dtype=np.complex128)
    w3[0, 0, 0] = 1.0
    net = ptnet.PTNet(fat, dims, [w1, w2, w3])
    r = inputs.gaussian_even_source(dims, 2)
    ref = oracle.Operator(fat, None, m, dims).apply_A(r)
    assert np.linalg.norm(net.apply(r) - ref) <= 1e-13 * np.linalg.norm(ref)


def _random_weights(seed, chans=(1, 8, 8, 1)):
    rng = np.random.default_rng(seed)
    return [0.3 * (rng.standard_normal((9, co, ci)) + 1j * rng.standard_normal((9, co, ci)))
            for ci, co in zip(chans[:-1], chans[1:])]


def test_layers_equal_the_two_hop_form():
    """With the input on even sites and the output read on even sites, only the
    layer paths with zero or two hops contribute, so the three linear layers equal
    k0 + sum_{p,q >= 1} H[p][q] T_p T_q with C[a][b][c] = W3[a] W2[b] W1[c]
    (channel contractions), k0 = C[0][0][0], H[p][q] = C[p][q][0] + C[p][0][q] +
    C[0][p][q].  This is the form the library evaluates when it applies the
    network; here it is checked against the oracle's layers, on a ragged lattice
    and for random, untied weights."""
    dims = (4, 6, 4, 8)
    fat = inputs.gauge_field(dims, 81)
    w1, w2, w3 = _random_weights(3)
    net = ptnet.PTNet(fat, dims, [w1, w2, w3])
    r = inputs.gaussian_even_source(dims, 83)
    C = np.einsum("ao,boi,ci->abc", w3[:, 0, :], w2, w1[:, :, 0])
    psi = oracle.embed(r, dims, 0)
    out = C[0, 0, 0] * psi
    for p in range(1, 9):
        chi = sum((C[p, q, 0] + C[p, 0, q] + C[0, p, q]) * ptnet.transport(net.u, psi, q) for q in range(1, 9))
        out = out + ptnet.transport(net.u, chi, p)
    got = oracle.restrict(out, dims, 0)
    ref = net.apply(r)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    # a term with an odd number of hops (here the one-hop part of layer 1) is zero on even sites
    odd = ptnet.transport(net.u, psi, 1)
    assert np.abs(oracle.restrict(odd, dims, 0)).max() == 0.0


def test_network_gauge_covariant_and_linear():
    dims = (4, 4, 4, 6)
    fat = inputs.gauge_field(dims, 7)
    ws = _random_weights(8)
    g = inputs.gauge_transform(dims, 9)
    fat_t = np.empty_like(fat)
    for mu in range(4):
        fat_t[..., mu, :, :] = g @ fat[..., mu, :, :] @ oracle.dagger(oracle.shift(g, mu, 1))
    r1 = inputs.gaussian_even_source(dims, 10)
    r2 = inputs.gaussian_even_source(dims, 11)
    net = ptnet.PTNet(fat, dims, ws)
    net_t = ptnet.PTNet(fat_t, dims, ws)
    g_e = g.reshape(-1, 3, 3)[oracle.sites_of_parity(dims, 0)]
    lhs = net_t.apply(oracle.matvec(g_e, r1))
    rhs = oracle.matvec(g_e, net.apply(r1))
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    lin = net.apply(a * r1 + b * r2) - (a * net.apply(r1) + b * net.apply(r2))
    assert np.linalg.norm(lin) <= 1e-13 * np.linalg.norm(net.apply(r1))


def _vdot(a, b):
    return np.vdot(np.asarray(a).reshape(-1), np.asarray(b).reshape(-1))


def test_tied_network_is_hermitian_and_untied_is_not():
    dims = (4, 4, 6, 4)
    fat = inputs.asqtad_form_fields(dims, seeds=(21, 22, 23))[0]
    u = inputs.gaussian_even_source(dims, 24)
    v = inputs.gaussian_even_source(dims, 25)
    ws = _random_weights(26)
    tied = ptnet.tie(ws)
    net = ptnet.PTNet(fat, dims, tied)
    lhs, rhs = _vdot(u, net.apply(v)), _vdot(net.apply(u), v)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    raw = ptnet.PTNet(fat, dims, ws)
    lhs, rhs = _vdot(u, raw.apply(v)), _vdot(raw.apply(u), v)
    assert abs(lhs - rhs) > 1e-3 * abs(lhs)
    # a projection: tying tied weights changes nothing
    again = ptnet.tie(tied)
    assert all(np.array_equal(a, b) for a, b in zip(again, tied))
    # rev pairs +mu with -mu
    assert [ptnet.rev(p) for p in range(9)] == [0, 2, 1, 4, 3, 6, 5, 8, 7]


def test_tied_degree_one_polynomial_is_a_plus_b_times_A_minus_m2():
    """W_1 = (identity; D), W_2 = diag(a, b) on the identity path, tied:
    M = E^dag (a + b D^dag D) E = a + b (A - m^2) on even sites, by Eq. (3) and D^dag = -D."""
    dims = (4, 6, 4, 4)
    m, a, b = 0.2, 0.7, -0.3
    fat = inputs.gauge_field(dims, 27)
    w1 = np.zeros((9, 2, 1), dtype=np.complex128)
    w1[0, 0, 0] = 1.0
    w1 += _d_weights(2, 1, 1, 0)
    w2 = np.zeros((9, 2, 2), dtype=np.complex128)
    w2[0, 0, 0] = a
    w2[0, 1, 1] = b
    w3 = ptnet.adjoint_weights(w1)
    tied = ptnet.tie([w1, w2, w3])
    assert all(np.allclose(x, y, rtol=0, atol=1e-15) for x, y in zip(tied, [w1, w2, w3]))
    net = ptnet.PTNet(fat, dims, [w1, w2, w3])
    r = inputs.gaussian_even_source(dims, 28)
    ar = oracle.Operator(fat, None, m, dims).apply_A(r)
    ref = a * r + b * (ar - m * m * r)
    assert np.linalg.norm(net.apply(r) - ref) <= 1e-13 * np.linalg.norm(ref)


def test_loss_definition():
    """The loss is >= 0, zero for a pair whose target is the network's own output, and
    |A (M r - e)|^2 / |A e|^2."""
    dims = (2, 2, 2, 4)
    fat = inputs.gauge_field(dims, 12)
    op = oracle.Operator(fat, None, 0.5, dims)
    net = ptnet.PTNet(fat, dims, _random_weights(13))
    r = inputs.gaussian_even_source(dims, 14)
    e = inputs.gaussian_even_source(dims, 15)
    assert net.loss(r, e, op.apply_A) > 0.0
    # a pair whose target is exactly the network's output has zero loss
    assert net.loss(r, net.apply(r), op.apply_A) == pytest.approx(0.0, abs=1e-28)
    ad = op.apply_A(net.apply(r) - e)
    ae = op.apply_A(e)
    ref = np.vdot(ad, ad).real / np.vdot(ae, ae).real
    assert net.loss(r, e, op.apply_A) == pytest.approx(ref, rel=1e-14)


def test_fcg_identity_is_cg_and_exact_inverse_is_one_step():
    dims = (4, 4, 4, 4)
    op = oracle.Operator(inputs.gauge_field(dims, 1), None, 0.2, dims)
    b = inputs.gaussian_even_source(dims, 0).reshape(-1)
    x_f, it_f = ptnet.fcg(op.apply_A, lambda r: r, b, tol=1e-10)
    x_c, it_c, _, _ = oracle.cg_fig1(op.apply_A, b, np.zeros_like(b), 1e-10, 10000)
    assert it_f == it_c
    assert np.linalg.norm(x_f - x_c) <= 1e-9 * np.linalg.norm(x_c)
    n = b.size
    a = np.stack([op.apply_A(np.eye(1, n, k).reshape(-1, 3)).reshape(-1) for k in range(n)], axis=1)
    ainv = np.linalg.inv(a)
    x1, it1 = ptnet.fcg(op.apply_A, lambda r: ainv @ r, b, tol=1e-10)
    assert it1 <= 1
    assert np.linalg.norm(a @ x1 - b) <= 1e-10 * np.linalg.norm(b)


def test_fcg_beta_from_the_applied_operator():
    """The library forms the Polak-Ribiere beta as -alpha (z_new, A p) / (r, z), which
    equals (z_new, r_new - r) / (r, z) because r_new - r = -alpha A p.  Flexible CG
    written that way reproduces the oracle's iterates, with a network preconditioner
    (tied, so that (r, z) > 0) whose z is not a fixed polynomial of A."""
    dims = (4, 6, 4, 8)
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(91, 92, 93))
    op = oracle.Operator(fat, lng, 0.05, dims)
    net = ptnet.PTNet(fat, dims, ptnet.tie(_random_weights(5)))
    b = inputs.gaussian_even_source(dims, 94).reshape(-1)
    k = 12

    def apply_a(v):
        return op.apply_A(v.reshape(-1, 3)).reshape(-1)

    def apply_m(v):
        return net.apply(v.reshape(-1, 3)).reshape(-1)

    ref, its = ptnet.fcg(apply_a, apply_m, b, tol=1e-10, max_iter=k)
    assert its == k
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_m(r)
    p = z.copy()
    rz = np.vdot(r, z).real
    for _ in range(k):
        q = apply_a(p)
        alpha = rz / np.vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        z = apply_m(r)
        beta = -alpha * np.vdot(z, q).real / rz
        rz = np.vdot(r, z).real
        p = z + beta * p
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


# ----------------------------------------------------- loss: free-field closed forms
def _unit_links(dims):
    lx, ly, lz, lt = dims
    u = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def _plane_wave_even(dims, n, colour):
    """exp(i p.x) e_colour on even sites, p_mu = 2 pi n_mu / L_mu, and
    lambda = m^2 + 4 sum sin^2 p_mu without the m^2 (the free-field spectrum of
    A = m^2 - D^2 for the paper's D, Eqs. (3)-(5), no factor 1/2)."""
    x, y, z, t = oracle.coordinates(dims)
    p = [2 * np.pi * n[mu] / dims[mu] for mu in range(4)]
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    full = np.zeros(phase.shape + (3,), dtype=np.complex128)
    full[..., colour] = phase
    return oracle.restrict(full, dims, 0), 4.0 * float(np.sum(np.sin(p) ** 2))


def _scalar_net(fat, dims, c):
    """Three one-channel layers on the identity path: M = c * identity."""
    w1 = np.zeros((9, 1, 1), dtype=np.complex128)
    w1[0, 0, 0] = c
    one = np.zeros((9, 1, 1), dtype=np.complex128)
    one[0, 0, 0] = 1.0
    return ptnet.PTNet(fat, dims, [w1, one, one.copy()])


LOSS_CASES = [((0, 0, 0, 0), 0.5), ((1, 0, 0, 0), 0.3), ((1, 2, 0, 1), 0.1), ((2, 1, 3, 5), 0.7)]


@pytest.mark.parametrize("n,m", LOSS_CASES)
def test_loss_closed_form_single_plane_wave(n, m):
    """Free field, residual r = v a plane wave with A v = lambda v, target e = v / lambda
    (the exact correction).  With M = c * identity, A (M r - e) = (c lambda - 1) v and
    A e = v, so L = (c lambda - 1)^2: (lambda - 1)^2 for c = 1 and 1 for c = 0.  The
    cases have lambda from 0.25 to about 14, so normalising by |e|^2 (a factor lambda^2),
    putting |d|^2 in the numerator (a factor 1 / lambda^2) or dropping the square all
    change the value."""
    dims = (4, 6, 4, 8)
    op = oracle.Operator(_unit_links(dims), None, m, dims)
    v, lam_free = _plane_wave_even(dims, n, 1)
    lam = m * m + lam_free
    e = v / lam
    for c in (1.0, 0.0, 0.37, -0.8):
        net = _scalar_net(_unit_links(dims), dims, c)
        want = (c * lam - 1.0) ** 2
        assert net.loss(v, e, op.apply_A) == pytest.approx(want, rel=1e-12, abs=1e-24)
    assert lam != pytest.approx(1.0)


def test_loss_closed_form_two_plane_waves_and_polynomial_network():
    """Free field, r = v1 + v2 (orthogonal plane waves, eigenvalues l1 != l2), e = v1 / l1 +
    v2 / l2.  The tied degree-1 network M = a + b (A - m^2) (a pinned form) maps v_k to
    (a + b (l_k - m^2)) v_k, so with g_k = (a + b (l_k - m^2)) l_k - 1:
        L = (g1^2 |v1|^2 + g2^2 |v2|^2) / (|v1|^2 + |v2|^2).
    A wrong weighting of the two modes (|e|^2 or |d|^2 norms) changes this value."""
    dims = (4, 4, 6, 4)
    m, a, b = 0.25, 0.6, -0.07
    fat = _unit_links(dims)
    op = oracle.Operator(fat, None, m, dims)
    v1, f1 = _plane_wave_even(dims, (1, 0, 0, 0), 0)
    v2, f2 = _plane_wave_even(dims, (1, 1, 2, 1), 2)
    l1, l2 = m * m + f1, m * m + f2
    assert abs(l1 - l2) > 1.0
    w1 = np.zeros((9, 2, 1), dtype=np.complex128)
    w1[0, 0, 0] = 1.0
    w1 += _d_weights(2, 1, 1, 0)
    w2 = np.zeros((9, 2, 2), dtype=np.complex128)
    w2[0, 0, 0] = a
    w2[0, 1, 1] = b
    net = ptnet.PTNet(fat, dims, [w1, w2, ptnet.adjoint_weights(w1)])
    g1 = (a + b * f1) * l1 - 1.0
    g2 = (a + b * f2) * l2 - 1.0
    n1, n2 = np.vdot(v1, v1).real, np.vdot(v2, v2).real
    want = (g1 * g1 * n1 + g2 * g2 * n2) / (n1 + n2)
    got = net.loss(v1 + v2, v1 / l1 + v2 / l2, op.apply_A)
    assert got == pytest.approx(want, rel=1e-12)
    # the same pair under the two plausible wrong normalisations differs from the pin
    ne = np.vdot(v1 / l1 + v2 / l2, v1 / l1 + v2 / l2).real
    wrong_e_norm = (g1 * g1 * n1 + g2 * g2 * n2) / ne
    assert abs(wrong_e_norm - want) > 0.1 * want
