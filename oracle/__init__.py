"""Oracle for the FFT pressure-projection path: TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded FP64 CPU statement of what the projection step of
FluTAS (arXiv 2204.08834, Sec. 3.3 "Pressure correction algorithm" and Sec. 3.3.1
"Poisson solver") computes.  It shares no code with the CUDA library and imports
nothing from the product package; only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import it.  The product
path never calls it and has no CPU fallback.

The volume-of-fluid step (MTHINC reconstruction and directional-split advection, Sec. 3.1
and Appendix A) is in oracle/vof.py (`from oracle import vof`).

Pins (see tests/test_oracle_*.py): single Fourier modes against the closed-form
discrete eigenvalues, a dense (bordered) LU solve of the assembled 7-point
operator on grids of 8^3 or smaller, brute-force DFT sums for the spectral steps,
a dense solve for the Thomas sweep, the adjointness D = -G^T, the exact action of
the stretched-z operator on a linear field, zero-mean p, divergence-free velocity
after correction, and the Dodd-Ferrante fixed point.  Parity with the paper's own
program output is unpinned: the paper prints no solver values.
"""

from .projection import (  # noqa: F401
    Grid,
    make_grid,
    grad,
    div,
    lap,
    face_density,
    min_density,
    p_hat,
    rhs,
    volume_mean,
    solve,
    tridiag_z,
    z_coefficients,
    eigenvalues,
    correct,
    project,
    residual,
    rel_residual,
    div_rel,
)
