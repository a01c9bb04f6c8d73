"""The allocation-free FP64 solve (flups_solve_fp64_noalloc) against the plan-based solve
and against the FP64 oracle.

Callers that may not allocate device memory (a plug-in inside an application that owns the
whole device memory budget) get the FP64 direct solve with its workspace in one fixed
device array.  Two calls in a row on different grids and boundary conditions must each
match flups_solve on an FP64 plan and the oracle's direct solve, within the FP64 parity
tolerance of the other tests (relative L2 error 1e-11): the second call reuses the array
the first one left behind.  This file is collected last on purpose.
"""

import numpy as np
import pytest

import oracle
from paper_2204_08834_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_08834_gb300 import flups  # noqa: E402


def _grid(c):
    nz, ny, nx = c.shape
    return oracle.make_grid(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc)


def _rhs(c):
    return oracle.rhs(c.u, c.v, c.w, c.rho, c.pn, c.pnm1, 2.0, 1.0, c.dt, _grid(c))


def test_noalloc_solve_matches_plan_solve_on_two_calls_in_a_row():
    cases = [synth.sphere(32), synth.random_fields(32, 16, 24, "walls", True, seed=95)]
    for c in cases:
        nz, ny, nx = c.shape
        f = torch.from_numpy(_rhs(c)).cuda()
        p_ref = torch.empty_like(f)
        p_na = torch.full_like(f, np.nan)
        with flups.Plan.for_case(c, "fp64") as plan:
            plan.solve(f, p_ref, rtol=0.0, info=False)
        flups.solve_fp64_noalloc(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc, f, p_na)
        torch.cuda.synchronize()
        a, b = p_na.cpu().numpy(), p_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-11, c.name
        po = oracle.solve(f.cpu().numpy(), _grid(c))
        assert np.linalg.norm(a - po) / np.linalg.norm(po) <= 1e-11, c.name


def test_noalloc_rejects_grids_beyond_its_array():
    f = torch.zeros((128, 128, 128), dtype=torch.float64, device="cuda")
    p = torch.zeros_like(f)
    st = flups.solve_fp64_noalloc(128, 128, 128, 1 / 128, 1 / 128, 1 / 128, "periodic", f, p, check=False)
    assert st == flups.EUNSUPPORTED
