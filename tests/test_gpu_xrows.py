"""FP32 + refine solves through the register x-row kernels and the z-marching defect, against
the FP64 oracle.

* Every row split of the four-step x transform (M = nx/2 = 64, 128, 256, 512, 1024: N1 x N2 =
  8x8, 16x8, 16x16, 32x16, 32x32), with row counts that are not a multiple of the CTA's rows
  (z walls with 5 or 3 planes), in both boundary conditions.
* The z-marching defect with a ragged last chunk of planes (nz % 16 = 8) on a grid of 2^24
  points or more, where the later stopping tests take the norm-only pass.
* The first FP32 iterate held in binary32 until the first update, including solves that stop
  at their first defect (host-driven and fixed-sequence).
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


@pytest.mark.parametrize("bc,nz", [("periodic", 32), ("walls", 24)])
def test_first_iterate_kept_in_binary32(bc, nz):
    # one-spacing grids keep the first FP32 iterate in binary32 until the first update: a solve
    # that stops at its first defect (loose rtol, or max_iter = 1) must still return that iterate
    # in p whatever p held before, the graph-capturable sequence the same p, and a full solve the
    # oracle's p
    nx, ny = 128, 64
    f, g, h = refine_case(nx, ny, nz, bc, seed=11)
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    po = oracle.solve(f, g)
    with flups.Plan(nx, ny, nz, h, h, np.full(nz, h), bc, "fp32_refine", flups.current_stream()) as plan:
        p1 = torch.full_like(fd, float("nan"))
        info = plan.solve(fd, p1, rtol=1e-3, max_iter=10)
        assert info.iters == 1 and 1e-9 < info.rel_res <= 1e-3
        a1 = p1.cpu().numpy()
        assert np.all(a1.astype(np.float32).astype(np.float64) == a1)     # a binary32 iterate
        assert np.linalg.norm(a1 - po) / np.linalg.norm(po) <= 1e-4
        assert abs(oracle.rel_residual(f, a1, g) - info.rel_res) <= 1e-3 * info.rel_res
        p2 = torch.full_like(fd, float("nan"))
        st, info2 = plan.solve(fd, p2, rtol=1e-14, max_iter=1, check=False)
        assert st == flups.ENOCONV and info2.iters == 1
        assert torch.equal(p2, p1)
        p3 = torch.full_like(fd, float("nan"))
        plan.solve_graphable(fd, p3, rtol=1e-3, max_iter=4)
        r3 = plan.solve_result(rtol=1e-3)
        assert r3.rel_res == info.rel_res and torch.equal(p3, p1)
        p4 = torch.full_like(fd, float("nan"))
        plan.solve_graphable(fd, p4, rtol=1e-10, max_iter=4)
        r4 = plan.solve_result(rtol=1e-10)
        a4 = p4.cpu().numpy()
        assert r4.rel_res <= 1e-10 and oracle.rel_residual(f, a4, g) <= 1.5e-10
        assert np.linalg.norm(a4 - po) / np.linalg.norm(po) <= 1e-8
