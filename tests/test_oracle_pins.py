"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each checks a closed form,
an invariant, a special case that reduces to a library routine, or brute
force on a tiny lattice (Sec. 2, Eqs. (3)-(5) and Fig. 1).
"""
import numpy as np
import pytest

import oracle
from paper_1010_4782_gb300 import inputs


def _unit_links(dims, c=1.0):
    lx, ly, lz, lt = dims
    u = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = c
    return u


def _plane_wave_even(dims, n, colour):
    """exp(i p.x) e_colour on even sites, p_mu = 2 pi n_mu / L_mu."""
    x, y, z, t = oracle.coordinates(dims)
    p = [2 * np.pi * n[mu] / dims[mu] for mu in range(4)]
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    full = np.zeros(phase.shape + (3,), dtype=np.complex128)
    full[..., colour] = phase
    return oracle.restrict(full, dims, 0), np.array(p)


# ---------------------------------------------------------------- free field
@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (2, 4, 4, 6), (6, 4, 2, 8)])
def test_free_field_one_hop_eigenvalues(dims):
    """U = 1: plane waves are eigenvectors, lambda = m^2 + 4 sum sin^2 p_mu (paper's D, no 1/2)."""
    m = 0.37
    op = oracle.Operator(_unit_links(dims), None, m, dims)
    rng = np.random.default_rng(5)
    for _ in range(6):
        n = [int(rng.integers(0, dims[mu])) for mu in range(4)]
        v, p = _plane_wave_even(dims, n, int(rng.integers(0, 3)))
        lam = m ** 2 + 4.0 * np.sum(np.sin(p) ** 2)
        av = op.apply_A(v)
        assert np.linalg.norm(av - lam * v) <= 1e-13 * lam * np.linalg.norm(v)


@pytest.mark.parametrize("dims", [(8, 6, 4, 10), (4, 4, 4, 4), (6, 6, 8, 2)])
def test_free_field_naik_eigenvalues(dims):
    """fat = c1, long = c3: lambda = m^2 + 4 sum (c1 sin p + c3 sin 3p)^2."""
    m = 0.21
    c1, c3 = 0.6 + 0.4, -1.0 / 24.0
    op = oracle.Operator(_unit_links(dims, c1), _unit_links(dims, c3), m, dims)
    rng = np.random.default_rng(7)
    for _ in range(6):
        n = [int(rng.integers(0, dims[mu])) for mu in range(4)]
        v, p = _plane_wave_even(dims, n, int(rng.integers(0, 3)))
        lam = m ** 2 + 4.0 * np.sum((c1 * np.sin(p) + c3 * np.sin(3 * p)) ** 2)
        av = op.apply_A(v)
        assert np.linalg.norm(av - lam * v) <= 1e-13 * lam * np.linalg.norm(v)


def test_free_field_distinguishes_axes():
    """A wave along one axis only: an axis mix-up would change lambda."""
    dims = (4, 6, 8, 10)
    m = 0.1
    op = oracle.Operator(_unit_links(dims), None, m, dims)
    for mu in range(4):
        n = [0, 0, 0, 0]
        n[mu] = 1
        v, _ = _plane_wave_even(dims, n, 0)
        lam = m ** 2 + 4.0 * np.sin(2 * np.pi / dims[mu]) ** 2
        assert np.allclose(op.apply_A(v), lam * v, rtol=0, atol=1e-13)


# ----------------------------------------------------------- anti-Hermiticity
@pytest.mark.parametrize("naik", [False, True])
def test_dslash_anti_hermitian(naik):
    """<x, D y> = -<D x, y> for arbitrary (non-unitary) complex links."""
    dims = (4, 6, 4, 8)
    fat = inputs.random_links(dims, 3)
    lng = inputs.random_links(dims, 4, 0.5) if naik else None
    op = oracle.Operator(fat, lng, 0.1, dims)
    rng = np.random.default_rng(9)
    shape = (dims[3], dims[2], dims[1], dims[0], 3)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    b = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    lhs = np.vdot(a, op.D(b))
    rhs = -np.vdot(op.D(a), b)
    scale = np.linalg.norm(a) * np.linalg.norm(op.D(b))
    assert abs(lhs - rhs) <= 1e-14 * scale


@pytest.mark.parametrize("naik", [False, True])
def test_A_hermitian_positive(naik):
    dims = (4, 4, 6, 4)
    m = 0.3
    fat = inputs.random_links(dims, 21)
    lng = inputs.random_links(dims, 22, 0.3) if naik else None
    op = oracle.Operator(fat, lng, m, dims)
    u = inputs.gaussian_even_source(dims, 1)
    v = inputs.gaussian_even_source(dims, 2)
    lhs = np.vdot(u, op.apply_A(v))
    rhs = np.vdot(op.apply_A(u), v)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    q = np.vdot(u, op.apply_A(u))
    assert abs(q.imag) <= 1e-13 * abs(q.real)
    assert q.real >= m ** 2 * np.vdot(u, u).real


# ------------------------------------------------------------ gauge covariance
@pytest.mark.parametrize("naik", [False, True])
def test_gauge_covariance(naik):
    """U'(x) = g(x) U(x) g(x+mu)^dag, L'(x) = g(x) L(x) g(x+3mu)^dag, chi' = g chi => D' chi' = g D chi."""
    dims = (4, 6, 8, 4)
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(31, 32, 33))
    if not naik:
        lng = None
    g = inputs.gauge_transform(dims, 34)
    fat_t = np.empty_like(fat)
    lng_t = None if lng is None else np.empty_like(lng)
    for mu in range(4):
        g1 = oracle.shift(g, mu, 1)
        fat_t[..., mu, :, :] = g @ fat[..., mu, :, :] @ oracle.dagger(g1)
        if lng is not None:
            g3 = oracle.shift(g, mu, 3)
            lng_t[..., mu, :, :] = g @ lng[..., mu, :, :] @ oracle.dagger(g3)
    op = oracle.Operator(fat, lng, 0.05, dims)
    op_t = oracle.Operator(fat_t, lng_t, 0.05, dims)
    rng = np.random.default_rng(11)
    shape = (dims[3], dims[2], dims[1], dims[0], 3)
    chi = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    lhs = op_t.D(oracle.matvec(g, chi))
    rhs = oracle.matvec(g, op.D(chi))
    assert np.linalg.norm(lhs - rhs) <= 1e-14 * np.linalg.norm(rhs)
    # and A on even sites
    v = inputs.gaussian_even_source(dims, 12)
    g_e = g.reshape(-1, 3, 3)[oracle.sites_of_parity(dims, 0)]
    lhs = op_t.apply_A(oracle.matvec(g_e, v))
    rhs = oracle.matvec(g_e, op.apply_A(v))
    assert np.linalg.norm(lhs - rhs) <= 1e-14 * np.linalg.norm(rhs)


# ------------------------------------------------------ dense brute force + CG
def _dense_A(op):
    n = op.n_half * 3
    cols = [op.apply_A(np.eye(1, n, k, dtype=np.complex128).reshape(-1, 3)).reshape(-1)
            for k in range(n)]
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("dims,naik,m", [((2, 2, 2, 2), False, 0.1),
                                         ((4, 4, 4, 4), False, 0.1),
                                         ((4, 4, 4, 4), True, 0.05),
                                         ((2, 4, 2, 6), True, 0.2)])
def test_dense_bruteforce_and_cg(dims, naik, m):
    """Dense A is Hermitian with lambda_min >= m^2; CG x matches LAPACK's solve within kappa*tol."""
    if naik:
        fat, lng = inputs.asqtad_form_fields(dims, seeds=(41, 42, 43))
    else:
        fat, lng = inputs.gauge_field(dims, 1), None
    op = oracle.Operator(fat, lng, m, dims)
    a = _dense_A(op)
    assert np.abs(a - a.conj().T).max() <= 1e-13 * np.abs(a).max()
    w = np.linalg.eigvalsh(a)
    assert w[0] >= m ** 2 * (1 - 1e-12)
    b = inputs.gaussian_even_source(dims, 0).reshape(-1)
    x_ref = np.linalg.solve(a, b)
    tol = 1e-10
    # Fig. 1 caps at N_dim steps; in floating point an ill-conditioned tiny system needs more
    res = oracle.solve(op.apply_A, b, tol=tol, max_iter=20 * b.size)
    assert res["true_rel_residual"] <= tol
    kappa = w[-1] / w[0]
    err = np.linalg.norm(res["x"] - x_ref) / np.linalg.norm(x_ref)
    assert err <= max(kappa * tol, 1e-14) * 2
    # true residual computed with the dense matrix, not with apply_A
    r = b - a @ res["x"]
    assert np.linalg.norm(r) <= 1.01 * tol * np.linalg.norm(b)


def test_cg_on_dense_hpd_matrix_matches_lapack():
    """Fig. 1 alone, on a random HPD matrix: converges within n steps to LAPACK's answer."""
    rng = np.random.default_rng(3)
    n = 40
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    lam = np.linspace(1.0, 30.0, n)
    a = (q * lam) @ q.conj().T
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, hist, _ = oracle.cg_fig1(lambda v: a @ v, b, np.zeros(n), 1e-12, n)
    assert it <= n
    assert np.linalg.norm(x - np.linalg.solve(a, b)) <= 1e-10 * np.linalg.norm(x)
    # residual history is r^dag r of the iterates (delta_new of Fig. 1)
    assert hist[0] == pytest.approx(np.vdot(b, b).real)


def test_cg_lanczos_extremes():
    """The alpha/beta of Fig. 1 build the Lanczos tridiagonal; its extreme Ritz values
    bracket-converge to A's extreme eigenvalues (dense 2^4 lattice)."""
    dims = (2, 2, 2, 2)
    op = oracle.Operator(inputs.gauge_field(dims, 5), None, 0.3, dims)
    a = _dense_A(op)
    w = np.linalg.eigvalsh(a)
    b = inputs.gaussian_even_source(dims, 6).reshape(-1)
    _, it, _, co = oracle.cg_fig1(op.apply_A, b, np.zeros_like(b), 1e-13, 10 * b.size)
    k = len(co)
    t = np.zeros((k, k))
    for j, (al, be) in enumerate(co):
        t[j, j] = 1.0 / al + (co[j - 1][1] / co[j - 1][0] if j > 0 else 0.0)
        if j + 1 < k:
            t[j, j + 1] = t[j + 1, j] = np.sqrt(be) / al
    ritz = np.linalg.eigvalsh(t)
    assert ritz[0] >= w[0] * (1 - 1e-9) and ritz[0] <= w[0] * (1 + 1e-6)
    assert ritz[-1] <= w[-1] * (1 + 1e-9) and ritz[-1] >= w[-1] * (1 - 1e-6)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_cg_plane_wave_sources_converge_in_k_steps(k):
    """Free field: a source made of k plane waves with distinct eigenvalues needs <= k CG steps."""
    dims = (4, 6, 8, 10)
    m = 0.2
    op = oracle.Operator(_unit_links(dims), None, m, dims)
    modes = [(1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (1, 1, 0, 0)][:k]
    b = np.zeros((op.n_half, 3), dtype=np.complex128)
    lams = []
    for j, n in enumerate(modes):
        v, p = _plane_wave_even(dims, n, j % 3)
        b += (1.0 + j) * v
        lams.append(m ** 2 + 4 * np.sum(np.sin(p) ** 2))
    assert len(set(np.round(lams, 12))) == k
    x, it, _, _ = oracle.cg_fig1(op.apply_A, b, np.zeros_like(b), 1e-12, 100)
    assert it <= k
    if k == 1:
        assert np.allclose(x.reshape(-1, 3), b / lams[0], rtol=0, atol=1e-13)


def test_large_mass_limit():
    """m^2 >> |D|^2: A ~ m^2, x ~ b/m^2 and CG needs only a few steps."""
    dims = (4, 4, 4, 4)
    m = 40.0
    op = oracle.Operator(inputs.gauge_field(dims, 1), None, m, dims)
    b = inputs.gaussian_even_source(dims, 0)
    res = oracle.solve(op.apply_A, b, tol=1e-12)
    assert res["iters"] <= 12
    # |D| <= 8 for unitary links, so |x - b/m^2| / |b/m^2| <= 64 / m^2
    rel = np.linalg.norm(res["x"].reshape(-1, 3) - b / m ** 2) / np.linalg.norm(b / m ** 2)
    assert rel <= 64.0 / m ** 2


# -------------------------------------------------- single-site oracle forms
@pytest.mark.parametrize("naik", [False, True])
def test_site_forms_match_lattice_forms(naik):
    """The per-site D and A (explicit neighbour indexing) agree with the rolled-array forms."""
    dims = (4, 6, 4, 8)
    fat = inputs.random_links(dims, 51)
    lng = inputs.random_links(dims, 52, 0.4) if naik else None
    m = 0.13
    op = oracle.Operator(fat, lng, m, dims)
    v = inputs.gaussian_even_source(dims, 53)
    av = op.apply_A(v)
    rng = np.random.default_rng(54)
    for idx in rng.integers(0, op.n_half, 12):
        s = oracle.even_site_coords(dims, int(idx))
        got = oracle.apply_A_at(fat, lng, m, v, s, dims)
        assert np.allclose(got, av[idx], rtol=0, atol=1e-12 * np.abs(av).max())


def test_even_site_numbering():
    """Even sites in lexicographic order: half-lattice number = lexicographic number // 2."""
    dims = (6, 4, 2, 4)
    ev = oracle.sites_of_parity(dims, 0)
    assert np.array_equal(ev // 2, np.arange(ev.size))
    od = oracle.sites_of_parity(dims, 1)
    assert np.array_equal(od // 2, np.arange(od.size))


def test_rejects_odd_extent():
    with pytest.raises(ValueError):
        oracle.check_dims((4, 4, 3, 4))


def test_gauge_field_is_su3():
    """The seeded links U = exp(0.3 i H), H Hermitian and traceless, are SU(3) to
    rounding: U^dag U = 1 and det U = 1.  The 12-parameter form (Sec. 3.3) relies
    on it: the third row of an SU(3) matrix is the conjugate cross product of the
    first two."""
    dims = (4, 2, 6, 4)
    u = inputs.gauge_field(dims, 3).reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.abs(np.conj(np.swapaxes(u, -1, -2)) @ u - eye).max() < 1e-13
    assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-13
    row2 = np.conj(np.cross(u[:, 0, :], u[:, 1, :]))
    assert np.abs(row2 - u[:, 2, :]).max() < 1e-13
    # the asqtad-form fat links are not unitary (the 12-parameter form does not apply)
    fat, _ = inputs.asqtad_form_fields(dims)
    f = fat.reshape(-1, 3, 3)
    assert np.abs(np.conj(np.swapaxes(f, -1, -2)) @ f - eye).max() > 1e-3


def test_naik_links_are_scaled_su3_with_eta_folded():
    """The asqtad-form Naik links are c U with c = -1/24 and U in SU(3).  After
    eta is folded in (L' = eta L), the third row is (eta / c) conj(row0' x row1'),
    since eta^2 = 1: the identity behind the two-row float-float Naik links.
    With the opposite sign of c the rebuilt row has the wrong sign (det(-U) = -1
    for 3x3), which is why the library checks det L / c^3 = 1 and not only
    unitarity."""
    dims = (4, 6, 2, 4)
    _, lng = inputs.asqtad_form_fields(dims)
    c = inputs.NAIK_COEFF
    folded = oracle.fold_eta(lng, dims)                              # [t][z][y][x][mu][3][3]
    e = np.moveaxis(oracle.eta(dims), 0, -1)[..., None]              # [t][z][y][x][mu][1]
    rebuilt = (e / c) * np.conj(np.cross(folded[..., 0, :], folded[..., 1, :]))
    assert np.abs(rebuilt - folded[..., 2, :]).max() < 1e-15
    assert np.abs(e).min() == 1.0 and (e < 0).any() and (e > 0).any()
    u = (lng / c).reshape(-1, 3, 3)
    assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-13
    assert np.abs(np.linalg.det(lng.reshape(-1, 3, 3) / -c) + 1.0).max() < 1e-13
    wrong = (e / -c) * np.conj(np.cross(folded[..., 0, :], folded[..., 1, :]))
    assert np.abs(wrong + folded[..., 2, :]).max() < 1e-15
