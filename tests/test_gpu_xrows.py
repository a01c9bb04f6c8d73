"""FP32 + refine solves through the register x-row kernels and the z-marching defect, against
the FP64 oracle.

* Every row split of the four-step x transform (M = nx/2 = 64, 128, 256, 512, 1024: N1 x N2 =
  8x8, 16x8, 16x16, 32x16, 32x32), with row counts that are not a multiple of the CTA's rows
  (z walls with 5 or 3 planes), in both boundary conditions.
* The z-marching defect with a ragged last chunk of planes (nz % 16 = 8) on a grid of 2^24
  points or more, where the later stopping tests take the norm-only pass.
Each solve must reach rtol 1e-10 by the oracle's own FP64 residual of the GPU's p and agree with
the oracle's direct solve to 1e-8 (the bar of the other refine parity tests).
"""

import numpy as np
import pytest

import oracle
from paper_2204_08834_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_08834_gb300 import flups  # noqa: E402


def refine_case(nx, ny, nz, bc, seed):
    # unit spacing per cell in every direction (one spacing h = 1/nx: the fixed-point defect)
    h = 1.0 / nx
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((nz, ny, nx))
    g = oracle.make_grid(nx, ny, nz, h, h, np.full(nz, h), bc)
    f = f - oracle.volume_mean(f, g)
    return f, g, h


def solve_and_check(nx, ny, nz, bc, seed):
    f, g, h = refine_case(nx, ny, nz, bc, seed)
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    pd = torch.empty_like(fd)
    with flups.Plan(nx, ny, nz, h, h, np.full(nz, h), bc, "fp32_refine", flups.current_stream()) as plan:
        info = plan.solve(fd, pd, rtol=1e-10, max_iter=10)
    pg = pd.cpu().numpy()
    assert info.rel_res <= 1e-10
    assert oracle.rel_residual(f, pg, g) <= 1.5e-10
    po = oracle.solve(f, g)
    err = np.linalg.norm(pg - po) / np.linalg.norm(po)
    assert err <= 1e-8, (nx, ny, nz, bc, err)


@pytest.mark.parametrize("nx", [128, 256, 512, 1024, 2048])
@pytest.mark.parametrize("bc,nz", [("periodic", 16), ("walls", 5), ("walls", 3)])
def test_row_splits(nx, bc, nz):
    solve_and_check(nx, 8, nz, bc, seed=nx + nz)


def test_z_march_ragged_chunk_and_norm_only_pass():
    # 128 x 512 x 264 = 17.3 M points >= 2^24: 64 row blocks x 17 chunks of 16 planes, the last
    # of 8
    solve_and_check(128, 512, 264, "walls", seed=7)
