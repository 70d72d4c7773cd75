"""Byte and flop accounting of the staggered Dirac operator (Sec. 2).

Per output site of one half-Dslash (D restricted to one parity):
  * the paper's convention (Sec. 2: 1584 bytes and 576 flops per site for
    D chi(x)): every link and every neighbour vector is read once per
    output site, plus the output write;
  * compulsory bytes: each link and each output once, and each input
    vector once per site (every input site is the neighbour of 8 or 16
    output sites, so the re-reads are cache hits, not compulsory traffic).
Flops: a 3x3 complex matrix times a colour vector is 9 complex
multiplications (6 flops) and 6 complex additions (2 flops) = 66 flops;
adding it into the site's sum is 6 more, so 72 flops per hop.
Sizes are those of FP64 (a float-float number occupies the same 8 bytes).
"""
from __future__ import annotations

LINK_BYTES_F64 = 9 * 16      # 3x3 complex128
VECTOR_BYTES_F64 = 3 * 16    # colour vector, complex128
FLOPS_PER_HOP = 66 + 6


def hops(naik: bool) -> int:
    return 16 if naik else 8


def paper_bytes_per_site(naik: bool = False, elem_bytes: int = 8) -> int:
    """Sec. 2: links + neighbour vectors + output, nothing cached (1584 B one-hop, FP64)."""
    s = elem_bytes / 8
    return int(hops(naik) * (LINK_BYTES_F64 + VECTOR_BYTES_F64) * s + VECTOR_BYTES_F64 * s)


def compulsory_bytes_per_site(naik: bool = False, elem_bytes: int = 8, long_entries: int = 9) -> int:
    """Each link once, the input vector once, the output once (1248 B one-hop, FP64).
    long_entries = 6: the Naik links stored as two rows (Sec. 3.3), 2016 B with Naik."""
    s = elem_bytes / 8
    links = 8 * LINK_BYTES_F64 + (8 * LINK_BYTES_F64 * long_entries // 9 if naik else 0)
    return int(links * s + 2 * VECTOR_BYTES_F64 * s)


def multi_rhs_bytes_per_site(nrhs: int, naik: bool = True) -> int:
    """Multi-RHS half-Dslash in FP32: each FP32 link once (72 B) and, per
    right-hand side, its input vector once and its output once (24 + 24 B).
    16 RHS with Naik: 16 x 72 + 16 x 48 = 1920 B."""
    return hops(naik) * (LINK_BYTES_F64 // 2) + nrhs * 2 * (VECTOR_BYTES_F64 // 2)


def flops_per_site(naik: bool = False) -> int:
    """Sec. 2: 576 flops per site for the one-hop D chi(x)."""
    return hops(naik) * FLOPS_PER_HOP


def fma_per_site(naik: bool = False) -> int:
    """Fused multiply-adds of one output site in real arithmetic: a 3x3 complex
    matrix times a colour vector accumulated into the site's sum is 9 complex
    multiply-adds = 36 real FMAs per hop (288 one-hop, 576 with Naik)."""
    return hops(naik) * 9 * 4


def half_sites(dims) -> int:
    lx, ly, lz, lt = dims
    return lx * ly * lz * lt // 2


def dslash_totals(dims, naik: bool = False):
    """(flops, paper-convention bytes, compulsory bytes) of one half-Dslash over all sites of a parity."""
    n = half_sites(dims)
    return n * flops_per_site(naik), n * paper_bytes_per_site(naik), n * compulsory_bytes_per_site(naik)
