"""FP64 CPU oracle of the staggered even-odd CG solve.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the package
smoke check and the benchmark's CPU-baseline / reference leg may import or
run anything in this directory.  It shares no code with the CUDA library
(no kernels, headers, index helpers or table generators) and never reads
values produced by it.

What it computes (Kim & Lee, "Multi GPU Performance of Conjugate Gradient
Algorithm with Staggered Fermions", Lattice 2010):

  * Sec. 2, Eqs. (4)-(5): the staggered Dirac operator
        D chi(x) = sum_mu  U_mu(x) chi(x+mu) - U_mu(x-mu)^dag chi(x-mu),
    with the staggered phase eta_mu(x) multiplied into U_mu(x) beforehand
    (Sec. 2, text after Eq. (5)).  There is no factor 1/2.
    Optional Naik three-hop term (not in the paper; the asqtad-form reading):
        + sum_mu  L_mu(x) chi(x+3mu) - L_mu(x-3mu)^dag chi(x-3mu),
    with eta_mu(x) multiplied into L_mu(x) the same way.
  * Sec. 2, Eq. (3): A = -D^2 + m^2.  D connects only sites of opposite
    parity, so on even sites A chi_e = m^2 chi_e - D_eo D_oe chi_e.
  * Sec. 2, Fig. 1: the conjugate-gradient recurrence, run literally.

Readings where the paper is silent (each is listed in the design notes):
  * eta_mu(x) = (-1)^(sum_{nu<mu} x_nu) with axis order (x, y, z, t):
    eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z).
  * periodic boundaries in all four directions; every extent must be even.
  * d^dag A d is taken as its real part (A is Hermitian).
  * the stopping threshold of Fig. 1, eps^2 delta_0, is applied as
    tol^2 |b|^2 (identical when the initial guess is zero); the outer
    driver then recomputes the true residual b - A x and restarts Fig. 1
    from the current x while it exceeds tol.

Array layouts:
  * lattice fields are [Lt, Lz, Ly, Lx, ...]: x is the fastest coordinate;
  * links are [Lt, Lz, Ly, Lx, 4, 3, 3] complex, direction mu = 0..3 is
    x, y, z, t; eta is NOT folded in the inputs (the oracle folds it);
  * even-site vectors are [V/2, 3] complex: the sites with x+y+z+t even
    in lexicographic order (x fastest).
"""
from __future__ import annotations

import numpy as np

# direction mu (x, y, z, t) -> axis of a [Lt, Lz, Ly, Lx] array
_AXIS = (3, 2, 1, 0)


# ---------------------------------------------------------------- geometry
def check_dims(dims):
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4 or any(d < 2 or d % 2 for d in dims):
        raise ValueError(f"lattice extents must be four even numbers >= 2, got {dims}")
    return dims


def coordinates(dims):
    """Integer arrays (x, y, z, t), each of shape [Lt, Lz, Ly, Lx]."""
    lx, ly, lz, lt = check_dims(dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly),
                             np.arange(lx), indexing="ij")
    return x, y, z, t


def parity(dims):
    """(x + y + z + t) mod 2 for every site, shape [Lt, Lz, Ly, Lx]."""
    x, y, z, t = coordinates(dims)
    return (x + y + z + t) % 2


def sites_of_parity(dims, p):
    """Lexicographic site numbers (x fastest) of the sites of parity p, in order."""
    return np.flatnonzero(parity(dims).ravel() == p)


def eta(dims):
    """Staggered phases eta_mu(x) = (-1)^(sum_{nu<mu} x_nu); shape [4, Lt, Lz, Ly, Lx]."""
    x, y, z, t = coordinates(dims)
    c = [np.zeros_like(x), x, x + y, x + y + z]
    return np.stack([np.where(ci % 2 == 0, 1.0, -1.0) for ci in c])


def fold_eta(links, dims):
    """U_mu(x) -> eta_mu(x) U_mu(x) (Sec. 2, after Eq. (5))."""
    e = np.moveaxis(eta(dims), 0, -1)          # [Lt, Lz, Ly, Lx, 4]
    return links * e[..., None, None]


def shift(field, mu, k):
    """Field value at x + k*mu_hat, stored at x (periodic)."""
    return np.roll(field, -k, axis=_AXIS[mu])


def dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))


def matvec(m, v):
    return np.einsum("...ab,...b->...a", m, v)


# ---------------------------------------------------------------- operator
def dslash(fat_folded, long_folded, chi):
    """D chi on the whole lattice, Eq. (5) (+ Naik term when long_folded is not None).

    fat_folded / long_folded: [Lt, Lz, Ly, Lx, 4, 3, 3] with eta folded in.
    chi: [Lt, Lz, Ly, Lx, 3].
    """
    out = np.zeros_like(chi)
    for mu in range(4):
        u = fat_folded[..., mu, :, :]
        out += matvec(u, shift(chi, mu, +1))
        out -= matvec(dagger(shift(u, mu, -1)), shift(chi, mu, -1))
        if long_folded is not None:
            w = long_folded[..., mu, :, :]
            out += matvec(w, shift(chi, mu, +3))
            out -= matvec(dagger(shift(w, mu, -3)), shift(chi, mu, -3))
    return out


def embed(v, dims, p):
    """Half-lattice vector of parity p ([V/2, 3]) -> full lattice field, zero elsewhere."""
    lx, ly, lz, lt = check_dims(dims)
    full = np.zeros((lt * lz * ly * lx, 3), dtype=np.complex128)
    full[sites_of_parity(dims, p)] = v
    return full.reshape(lt, lz, ly, lx, 3)


def restrict(field, dims, p):
    """Full lattice field -> its values on the sites of parity p, [V/2, 3]."""
    return field.reshape(-1, 3)[sites_of_parity(dims, p)]


class Operator:
    """A = m^2 - D_eo D_oe on even sites for one gauge field (eta folded here)."""

    def __init__(self, fat, long=None, mass=0.1, dims=None):
        if dims is None:
            lt, lz, ly, lx = fat.shape[:4]
            dims = (lx, ly, lz, lt)
        self.dims = check_dims(dims)
        self.mass = float(mass)
        self.fat = fold_eta(np.asarray(fat, dtype=np.complex128), self.dims)
        self.long = None if long is None else fold_eta(np.asarray(long, dtype=np.complex128), self.dims)
        self.n_half = int(np.prod(self.dims)) // 2

    def D(self, chi):
        return dslash(self.fat, self.long, chi)

    def dslash_half(self, v, out_parity):
        """D restricted to parity out_parity <- 1 - out_parity, on [V/2, 3] vectors."""
        chi = embed(v, self.dims, 1 - out_parity)
        return restrict(self.D(chi), self.dims, out_parity)

    def apply_A(self, v_even):
        """A v = m^2 v - D_eo D_oe v on even sites (Eq. (3) restricted to even sites)."""
        v_even = np.asarray(v_even, dtype=np.complex128).reshape(self.n_half, 3)
        chi = embed(v_even, self.dims, 0)
        dd = self.D(self.D(chi))
        return self.mass ** 2 * v_even - restrict(dd, self.dims, 0)


# ------------------------------------------------------- single-site forms
def _site(dims, x, y, z, t):
    lx, ly, lz, lt = dims
    return (x % lx, y % ly, z % lz, t % lt)


def _step(dims, s, mu, k):
    c = list(s)
    c[mu] += k
    return _site(dims, *c)


def _eta_at(s, mu):
    return -1.0 if sum(s[:mu]) % 2 else 1.0


def _link(links, s, mu):
    x, y, z, t = s
    return links[t, z, y, x, mu]


def dslash_at(fat, long, chi_at, s, dims):
    """(D chi)(s) for one site s = (x, y, z, t), from raw (un-folded) links.

    chi_at(site) returns the 3-vector chi(site).  Eq. (5) with eta_mu
    multiplied into each link at the link's own site, plus the Naik term.
    """
    dims = check_dims(dims)
    out = np.zeros(3, dtype=np.complex128)
    terms = [(fat, 1)] + ([(long, 3)] if long is not None else [])
    for links, k in terms:
        for mu in range(4):
            fwd = _step(dims, s, mu, +k)
            bwd = _step(dims, s, mu, -k)
            u_f = _eta_at(s, mu) * _link(links, s, mu)
            u_b = _eta_at(bwd, mu) * _link(links, bwd, mu)
            out += u_f @ chi_at(fwd)
            out -= np.conj(u_b.T) @ chi_at(bwd)
    return out


def apply_A_at(fat, long, mass, v_even, s, dims):
    """(A v)(s) for one even site s: m^2 v(s) - (D D v)(s)."""
    dims = check_dims(dims)
    lx, ly, lz, lt = dims

    def v_at(site):
        x, y, z, t = site
        if (x + y + z + t) % 2:
            return np.zeros(3, dtype=np.complex128)
        return v_even[(((t * lz + z) * ly + y) * lx + x) // 2]

    def dv_at(site):
        return dslash_at(fat, long, v_at, site, dims)

    return mass ** 2 * v_at(s) - dslash_at(fat, long, dv_at, s, dims)


def even_site_coords(dims, index):
    """Coordinates (x, y, z, t) of the even site with half-lattice number `index`."""
    lx, ly, lz, lt = check_dims(dims)
    lex = int(sites_of_parity(dims, 0)[index])
    x = lex % lx
    y = (lex // lx) % ly
    z = (lex // (lx * ly)) % lz
    t = lex // (lx * ly * lz)
    return (x, y, z, t)


# ---------------------------------------------------------------------- CG
def cg_fig1(apply_A, b, x0, eps, n_dim, threshold=None):
    """Fig. 1 conjugate gradient, run literally.

    Stops when i reaches n_dim or delta_new <= eps^2 delta_0 (or, when
    `threshold` is given, delta_new <= threshold).  Returns
    (x, iterations, history of delta_new, list of (alpha, beta)).
    """
    x = np.array(x0, dtype=np.complex128).reshape(-1)
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    r = b - apply_A(x).reshape(-1)
    d = r.copy()
    delta_new = float(np.vdot(r, r).real)
    delta_0 = delta_new
    stop = eps ** 2 * delta_0 if threshold is None else threshold
    hist = [delta_new]
    coeffs = []
    i = 0
    while i < n_dim and delta_new > stop:
        ad = apply_A(d).reshape(-1)
        alpha = delta_new / float(np.vdot(d, ad).real)
        x = x + alpha * d
        r = r - alpha * ad
        delta_old = delta_new
        delta_new = float(np.vdot(r, r).real)
        beta = delta_new / delta_old
        d = r + beta * d
        hist.append(delta_new)
        coeffs.append((alpha, beta))
        i += 1
    return x, i, hist, coeffs


def solve(apply_A, b, x0=None, tol=1e-10, max_iter=None, max_restarts=5):
    """Solve A x = b to a true relative residual |b - A x| / |b| <= tol.

    Runs Fig. 1 with the threshold tol^2 |b|^2, then recomputes the true
    residual; while it exceeds tol, restarts Fig. 1 from the current x.
    Returns dict(x, iters, restarts, true_rel_residual, history).
    """
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    bnorm2 = float(np.vdot(b, b).real)
    if max_iter is None or max_iter <= 0:
        max_iter = n
    iters, restarts, hist = 0, 0, []
    rel = np.inf
    if bnorm2 == 0.0:
        return dict(x=np.zeros(n, dtype=np.complex128), iters=0, restarts=0,
                    true_rel_residual=0.0, history=[0.0])
    while True:
        x, it, h, _ = cg_fig1(apply_A, b, x, 1.0, max_iter - iters,
                              threshold=tol ** 2 * bnorm2)
        iters += it
        hist.extend(h)
        r = b - apply_A(x).reshape(-1)
        rel = float(np.sqrt(np.vdot(r, r).real / bnorm2))
        if rel <= tol or iters >= max_iter or restarts >= max_restarts:
            break
        restarts += 1
    return dict(x=x, iters=iters, restarts=restarts, true_rel_residual=rel, history=hist)
