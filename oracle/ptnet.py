"""FP64 CPU oracle of the learned preconditioner and flexible CG.

TEST INFRASTRUCTURE, NOT PRODUCT CODE (see oracle/staggered.py).

Not in the paper, whose CG (Sec. 2, Fig. 1) is unpreconditioned; the design
is a gauge-covariant parallel-transport convolution network used as the
preconditioner of flexible CG.  Definitions:

  * paths p = 0..8: p = 0 is the identity; p = 1 + 2 mu + s transports from
    x + mu (s = 0) or x - mu (s = 1) with the eta-folded links of the operator:
        (T_{+mu} psi)(x) = U_mu(x) psi(x + mu),
        (T_{-mu} psi)(x) = U_mu(x - mu)^dag psi(x - mu),
    so that sum_mu (T_{+mu} - T_{-mu}) = D of Eq. (5).
  * layer l: psi_l(x, o) = sum_p sum_i W_l[p, o, i] (T_p psi_{l-1, i})(x),
    complex weights W_l of shape [9, C_l, C_{l-1}], no bias, no nonlinearity
    (a linear, gauge-covariant map).
  * the network: the residual r (even sites) is embedded on the full lattice
    (zero on odd sites), passed through the layers, and the last layer's
    single channel is restricted to even sites: M(r).
  * loss of a pair (r, e): the residual norm of the correction, i.e. the
    error d = M(r) - e in the norm |A .|:
        L = |A d|^2 / |A e|^2.
  * self-adjoint tie: with E the embedding of even-site vectors and L_l the
    layers, M = E^dag L_3 L_2 L_1 E is Hermitian when L_3 = L_1^dag and
    L_2 = L_2^dag.  The adjoint of a layer has the weights
    W^dag[p][i][o] = conj(W[rev(p)][o][i]), rev(p) the path in the opposite
    direction (T_{+mu}^dag = T_{-mu}), so the tie is
        W_3[p][0][i] = conj(W_1[rev(p)][i][0]),
        W_2[p][o][i] = conj(W_2[rev(p)][i][o]);
    `tie` projects arbitrary weights onto these relations (the mean of each
    weight and its partner's conjugate).
  * flexible CG (Notay 2000): z_k = M(r_k), p_0 = z_0,
    alpha = (r_k, z_k) / (p_k, A p_k), x += alpha p, r -= alpha A p,
    beta = (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k), p = z_{k+1} + beta p.
"""
from __future__ import annotations

import numpy as np

from . import staggered as st

N_PATHS = 9


def path_of(p):
    """(mu, s) of path p >= 1: transport from x + mu (s = 0) or x - mu (s = 1)."""
    return (p - 1) // 2, (p - 1) % 2


def rev(p):
    """The path opposite to p (p = 0 is its own)."""
    if p == 0:
        return 0
    mu, s = path_of(p)
    return 1 + 2 * mu + (1 - s)


def adjoint_weights(w):
    """Weights of the adjoint of a layer with weights w [9, C_out, C_in]: [9, C_in, C_out]."""
    w = np.asarray(w, dtype=np.complex128)
    return np.stack([np.conj(w[rev(p)]).T for p in range(N_PATHS)])


def tie(weights):
    """Project [W_1, W_2, W_3] onto the self-adjoint form W_3 = W_1^dag, W_2 = W_2^dag."""
    w1, w2, w3 = (np.asarray(w, dtype=np.complex128) for w in weights)
    w1t = 0.5 * (w1 + adjoint_weights(w3))
    w2t = 0.5 * (w2 + adjoint_weights(w2))
    return [w1t, w2t, adjoint_weights(w1t)]


def transport(u_folded, psi, p):
    """(T_p psi)(x) for a field psi [Lt, Lz, Ly, Lx, 3] (or with leading channel axes)."""
    if p == 0:
        return psi
    mu, s = path_of(p)
    u = u_folded[..., mu, :, :]
    if s == 0:
        return st.matvec(u, st.shift(psi, mu, +1))
    return st.matvec(st.dagger(st.shift(u, mu, -1)), st.shift(psi, mu, -1))


def layer(u_folded, w, psi):
    """psi: [C_in, Lt, Lz, Ly, Lx, 3]; w: [9, C_out, C_in] complex -> [C_out, ...]."""
    out = np.zeros((w.shape[1],) + psi.shape[1:], dtype=np.complex128)
    for p in range(N_PATHS):
        t = np.stack([transport(u_folded, psi[i], p) for i in range(psi.shape[0])])
        out += np.einsum("oi,i...->o...", w[p], t)
    return out


class PTNet:
    """The network for one gauge field (eta folded here); weights: list of [9, C_out, C_in]."""

    def __init__(self, fat, dims, weights):
        self.dims = st.check_dims(dims)
        self.u = st.fold_eta(np.asarray(fat, dtype=np.complex128), self.dims)
        self.weights = [np.asarray(w, dtype=np.complex128) for w in weights]

    def activations(self, r_even):
        psi = st.embed(np.asarray(r_even, dtype=np.complex128).reshape(-1, 3), self.dims, 0)[None]
        acts = [psi]
        for w in self.weights:
            psi = layer(self.u, w, psi)
            acts.append(psi)
        return acts

    def apply(self, r_even):
        return st.restrict(self.activations(r_even)[-1][0], self.dims, 0)

    def loss(self, r_even, e_even, apply_A):
        """|A d|^2 / |A e|^2 with d = M(r) - e; apply_A acts on [V/2, 3] vectors."""
        e = np.asarray(e_even, dtype=np.complex128).reshape(-1, 3)
        ad = apply_A(self.apply(r_even) - e)
        ae = apply_A(e)
        return float(np.vdot(ad, ad).real / np.vdot(ae, ae).real)


def fcg(apply_A, precond, b, x0=None, tol=1e-10, max_iter=10000):
    """Flexible CG as defined above; stops at |r| <= tol |b| (iterated residual).

    Returns (x, iterations)."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    r = b - apply_A(x).reshape(-1)
    z = precond(r).reshape(-1)
    p = z.copy()
    rz = np.vdot(r, z).real
    bn = np.linalg.norm(b)
    k = 0
    while k < max_iter and np.linalg.norm(r) > tol * bn:
        q = apply_A(p).reshape(-1)
        alpha = rz / np.vdot(p, q).real
        x = x + alpha * p
        r_new = r - alpha * q
        z_new = precond(r_new).reshape(-1)
        beta = np.vdot(z_new, r_new - r).real / rz
        rz = np.vdot(r_new, z_new).real
        p = z_new + beta * p
        r, z = r_new, z_new
        k += 1
    return x, k
