"""Seeded synthetic inputs for the staggered even-odd CG solver.

This module generates input data only: gauge fields, sources and random
gauge transformations.  It contains none of the solver's arithmetic (no
Dirac operator, no eta phases, no CG) and is shared by the oracle-based
tests and by the CUDA path's tests and benchmark, which both receive the
same arrays.

Layouts (the library's ABI layouts):
  * gauge field: complex128 array [Lt, Lz, Ly, Lx, 4, 3, 3]; direction index
    mu = 0, 1, 2, 3 is x, y, z, t; x is the fastest lattice coordinate.
    Eta phases are NOT folded in.
  * even-site vector: complex128 array [V/2, 3]; even sites
    ((x + y + z + t) even) in lexicographic order, x fastest.

The gauge links follow the synthetic recipe used in place of the MILC
ensemble of the paper (Sec. 2, 28^3 x 96): U = exp(i eps H) with H a
Gaussian Hermitian traceless 3x3 matrix (entries re, im ~ N(0, 1) before
Hermitisation) and eps = 0.3; the asqtad-form operator uses fat links
0.6 U_a + 0.4 U_b and Naik links -(1/24) U_c from three independent fields.
"""
from __future__ import annotations

import numpy as np
import torch

__all__ = [
    "volume",
    "su3_matrices",
    "gauge_field",
    "asqtad_form_fields",
    "random_links",
    "gaussian_even_source",
    "gaussian_vector",
    "gauge_transform",
    "DEFAULT_EPS",
    "NAIK_COEFF",
    "FAT_COEFFS",
]

DEFAULT_EPS = 0.3
FAT_COEFFS = (0.6, 0.4)
NAIK_COEFF = -1.0 / 24.0
# seeds of the three independent fields of the asqtad-form operator
ASQTAD_SEEDS = (11, 12, 13)
_CHUNK = 1 << 20


def volume(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def _hermitian_traceless(rng: np.random.Generator, n: int) -> np.ndarray:
    m = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    h = 0.5 * (m + np.conj(np.swapaxes(m, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h[:, 0, 0] -= tr
    h[:, 1, 1] -= tr
    h[:, 2, 2] -= tr
    return h


def su3_matrices(rng: np.random.Generator, n: int, eps: float = DEFAULT_EPS) -> np.ndarray:
    """n matrices exp(i eps H), H Gaussian Hermitian traceless; shape [n, 3, 3]."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        h = _hermitian_traceless(rng, e - s)
        out[s:e] = torch.linalg.matrix_exp(torch.from_numpy(1j * eps * h)).numpy()
    return out


def gauge_field(dims, seed: int, eps: float = DEFAULT_EPS) -> np.ndarray:
    """SU(3) gauge field [Lt, Lz, Ly, Lx, 4, 3, 3], links exp(i eps H)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    u = su3_matrices(rng, volume(dims) * 4, eps)
    return u.reshape(lt, lz, ly, lx, 4, 3, 3)


def asqtad_form_fields(dims, seeds=ASQTAD_SEEDS, eps: float = DEFAULT_EPS):
    """(fat, long): fat = 0.6 U_a + 0.4 U_b (not unitary), long = -(1/24) U_c."""
    fat = gauge_field(dims, seeds[0], eps)
    fat *= FAT_COEFFS[0]
    ub = gauge_field(dims, seeds[1], eps)
    fat += FAT_COEFFS[1] * ub
    del ub
    lng = gauge_field(dims, seeds[2], eps)
    lng *= NAIK_COEFF
    return fat, lng


def random_links(dims, seed: int, scale: float = 1.0) -> np.ndarray:
    """General complex (non-unitary) links, entries re, im ~ N(0, scale^2)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    shape = (lt, lz, ly, lx, 4, 3, 3)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def gaussian_even_source(dims, seed: int = 0) -> np.ndarray:
    """Even-site source [V/2, 3], re and im ~ N(0, 1)."""
    vh = volume(dims) // 2
    rng = np.random.default_rng(seed)
    return rng.standard_normal((vh, 3)) + 1j * rng.standard_normal((vh, 3))


def gaussian_vector(n_sites: int, seed: int) -> np.ndarray:
    """Colour vectors [n_sites, 3], re and im ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_sites, 3)) + 1j * rng.standard_normal((n_sites, 3))


def gauge_transform(dims, seed: int, eps: float = 1.0) -> np.ndarray:
    """Random SU(3) matrix per site, [Lt, Lz, Ly, Lx, 3, 3]."""
    lx, ly, lz, lt = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    return su3_matrices(rng, volume(dims), eps).reshape(lt, lz, ly, lx, 3, 3)
