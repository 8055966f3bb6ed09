"""FP64 CPU oracle for the exact 2D DCT -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library does not, and the two share no
code: the oracle builds its own cosine tables on the CPU.

Parity: pinned.  Every function here is checked by the ``-m "not gpu"`` tests
against brute force, SciPy's DCT, closed forms and invariants.
"""
from .oracle import (  # noqa: F401
    NORM_ORTHO,
    NORM_NONE,
    build,
    forward,
    inverse,
    roundtrip,
    spectral,
    bruteforce,
    matrix,
    cospi_frac,
    set_fault,
    default_threads,
)
from .check import metrics, accept, boundary_metrics, ERR_REL_TOL, MAX_ABS_TOL  # noqa: F401
