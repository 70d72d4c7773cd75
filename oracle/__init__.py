"""FP64 CPU oracle (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's
CPU-baseline / reference leg may import this package.  See
oracle/staggered.py for what it computes and the passages it follows.
"""
from .staggered import (  # noqa: F401
    Operator,
    apply_A_at,
    cg_fig1,
    check_dims,
    coordinates,
    dagger,
    dslash,
    dslash_at,
    embed,
    eta,
    even_site_coords,
    fold_eta,
    matvec,
    parity,
    restrict,
    shift,
    sites_of_parity,
    solve,
)
