"""Batched ensembles of mixed-size FP32-refine solves in one CUDA graph launch.

* The graph-capturable solve (fixed kernel sequence, device-side early exit) must give
  exactly the bits of the host-driven flups_solve on the same plan.
* Every ensemble member must solve the oracle's own equation to rel. residual <= rtol
  (checked by the oracle's FP64 residual of the GPU's p) and agree with the member's
  oracle direct solve; a graph replay must reproduce the first launch bit for bit.
* The mixed-size ensemble of 64 members {32, 48, 64, 96, 128}^3 (periodic and z walls,
  density ratios in [1, 20]) at full size.
* Ensembles whose members all have transform lengths 8 2^a or 12 2^a run one kernel per stage
  for all members (7 max_iter + 3 graph kernels whatever the member count: 10 for the first
  solve and defect test, then per iteration a conditional node's 6 and the kernel that sets
  its condition); an ensemble with a shorter length captures each member's own kernel
  sequence instead, and must solve to the same bar.
"""

import numpy as np
import pytest

import oracle
from paper_2204_08834_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_08834_gb300 import flups  # noqa: E402


def grid_of(c):
    nz, ny, nx = c.shape
    return oracle.make_grid(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc)


def member_rhs(c):
    return oracle.rhs(c.u, c.v, c.w, c.rho, c.pn, c.pnm1, 2.0, 1.0, c.dt, grid_of(c))


def spec(c):
    nz, ny, nx = c.shape
    return (nx, ny, nz, c.dx, c.dy, c.dzf, c.bc)


@pytest.mark.parametrize("case,rtol", [("sphere32", 1e-10), ("walls48", 1e-10), ("sphere32", 1e-15)])
def test_graphable_solve_equals_host_loop(case, rtol):
    """Same bits as the host-driven loop; rtol 1e-15 makes the graph-capturable solve find the
    defect above rtol after its second FP32 solve, so its norm-only stopping test is followed by
    the fused defect pass and further solves."""
    c = synth.sphere(32) if case == "sphere32" else synth.random_fields(48, 24, 20, "walls", True, seed=99)
    f = torch.from_numpy(member_rhs(c)).cuda()
    p1 = torch.empty_like(f)
    p2 = torch.full_like(f, np.nan)
    with flups.Plan.for_case(c, "fp32_refine") as plan:
        st, info = plan.solve(f, p1, rtol=rtol, max_iter=6, check=False)
        plan.solve_graphable(f, p2, rtol=rtol, max_iter=6)
        st2, res = plan.solve_result(rtol=rtol, check=False)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)
    assert res.rel_res == info.rel_res
    if rtol < 1e-14:
        assert info.iters >= 3


@pytest.mark.parametrize("rtol", [1e-10, 1e-15])
def test_graphable_solve_equals_host_loop_at_2_24_points(rtol):
    """At 2^24 points with one spacing both solves take the norm-only stopping test from the
    second FP32 solve on; rtol 1e-15 makes that test fail, so the fused defect pass and further
    solves follow it.  Same bits and the same final defect norm either way."""
    n = 256
    h = 1.0 / n
    f = torch.from_numpy(np.random.default_rng(7).standard_normal((n, n, n))).cuda()
    p1 = torch.empty_like(f)
    p2 = torch.full_like(f, np.nan)
    with flups.Plan(n, n, n, h, h, h, "periodic", "fp32_refine") as plan:
        st, info = plan.solve(f, p1, rtol=rtol, max_iter=5, check=False)
        plan.solve_graphable(f, p2, rtol=rtol, max_iter=5)
        st2, res = plan.solve_result(rtol=rtol, check=False)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)
    assert res.rel_res == info.rel_res and st2 == st
    assert info.iters >= (3 if rtol < 1e-14 else 2)
    if rtol > 1e-14:
        assert st == flups.OK and info.rel_res <= rtol


def small_members():
    cases = []
    for m in range(10):
        n = (32, 48, 64)[m % 3]
        c = synth.emulsion(n, ratio=1.0 + 2.0 * m, ndrops=4, rmin_cells=2.0, rmax_cells=4.0, seed=200 + m)
        if m % 2:
            c["bc"] = "walls"
            c["w"][-1] = 0.0
        cases.append(c)
    return cases


def test_batch_members_match_oracle_and_replay():
    cases = small_members()
    fs = [torch.from_numpy(member_rhs(c)).cuda() for c in cases]
    ps = [torch.empty_like(f) for f in fs]
    with flups.Batch([spec(c) for c in cases], nstreams=4, autotune=True) as b:
        infos = b.solve(fs, ps, rtol=1e-10, max_iter=5)
        first = [p.clone() for p in ps]
        assert b.graph_kernels > 0
        for p in ps:
            p.fill_(0.0)
        b.solve(fs, ps, rtol=1e-10, max_iter=5)          # replay of the captured graph
        torch.cuda.synchronize()
        for a, bb in zip(first, ps):
            assert torch.equal(a, bb)
        for m in range(len(cases)):
            cta, rv = b.tuning(m)
            assert cta in (256, 512, 1024) and rv in (0, 1)
    for c, f, p, inf in zip(cases, fs, ps, infos):
        g = grid_of(c)
        fo = f.cpu().numpy()
        pg = p.cpu().numpy()
        assert inf.rel_res <= 1e-10
        assert oracle.rel_residual(fo, pg, g) <= 1.5e-10
        po = oracle.solve(fo, g)
        assert np.linalg.norm(pg - po) / np.linalg.norm(po) <= 1e-8


@pytest.mark.slow
def test_mixed_size_ensemble_of_64():
    cases = [synth.ensemble_member(m) for m in range(64)]
    assert sorted({c.shape[0] for c in cases}) == [32, 48, 64, 96, 128]
    fs = [torch.from_numpy(member_rhs(c)).cuda() for c in cases]
    ps = [torch.empty_like(f) for f in fs]
    with flups.Batch([spec(c) for c in cases], nstreams=8, autotune=True) as b:
        infos = b.solve(fs, ps, rtol=1e-10, max_iter=5)
    for m, (c, f, p, inf) in enumerate(zip(cases, fs, ps, infos)):
        assert inf.rel_res <= 1e-10, c.name
        fo, pg = f.cpu().numpy(), p.cpu().numpy()
        assert oracle.rel_residual(fo, pg, grid_of(c)) <= 1.5e-10, c.name
        if m % 7 == 0:      # a sample of ten members (every size, both z treatments): p itself
            po = oracle.solve(fo, grid_of(c))
            assert np.linalg.norm(pg - po) / np.linalg.norm(po) <= 1e-8, c.name


def test_stage_kernels_graph_size_and_per_member_fallback():
    cases = small_members()[:4]
    fs = [torch.from_numpy(member_rhs(c)).cuda() for c in cases]
    ps = [torch.empty_like(f) for f in fs]
    with flups.Batch([spec(c) for c in cases], nstreams=4, autotune=False) as b:
        b.solve(fs, ps, rtol=1e-10, max_iter=5)
        assert b.graph_kernels == 7 * 5 + 3          # one kernel per stage for all members
    # a member of nx = 8 (a 4-point complex x transform) takes the per-member sequences
    small = synth.random_fields(8, 16, 12, "walls", False, seed=97)
    cases2 = [cases[0], small]
    fs2 = [torch.from_numpy(member_rhs(c)).cuda() for c in cases2]
    ps2 = [torch.empty_like(f) for f in fs2]
    with flups.Batch([spec(c) for c in cases2], nstreams=2, autotune=False) as b:
        infos = b.solve(fs2, ps2, rtol=1e-10, max_iter=5)
        assert b.graph_kernels > 7 * 5 + 3
    for c, f, p, inf in zip(cases2, fs2, ps2, infos):
        g = grid_of(c)
        fo, pg = f.cpu().numpy(), p.cpu().numpy()
        assert inf.rel_res <= 1e-10
        assert oracle.rel_residual(fo, pg, g) <= 1.5e-10
        po = oracle.solve(fo, g)
        assert np.linalg.norm(pg - po) / np.linalg.norm(po) <= 1e-8
