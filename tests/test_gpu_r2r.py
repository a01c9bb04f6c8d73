"""GPU parity of the Poisson solve with Neumann or Dirichlet ends in x and/or y (Sec. 3.3.1,
cosine/sine series; oracle/r2r.py, readings E1-E4) against the FP64 oracle.

Tolerance: both sides are FP64 eigen-expansion solves (GPU: Makhoul's construction around the
library's FFTs; oracle: scipy's DCT/DST), so p agrees to the rounding of the transforms
amplified by the condition number of the smallest retained mode: relative L2 error <= 1e-11
(as the periodic FP64 solve), and the oracle's residual of the GPU's p <= 1e-12.
"""

import itertools
import zlib

import numpy as np
import pytest

import oracle
from oracle import r2r

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_08834_gb300 import flups  # noqa: E402

NAME = {"P": "periodic", "NN": "neumann", "DD": "dirichlet", "ND": "neumann_dirichlet", "DN": "dirichlet_neumann"}
ENDS = [e for e in itertools.product(r2r.KINDS, repeat=2) if e != ("P", "P")]


def run(f, nx, ny, nz, dx, dy, dzf, bcz, bcx, bcy, prec="fp64", rtol=0.0):
    with flups.Plan(nx, ny, nz, dx, dy, dzf, bcz, prec, flups.current_stream(), bcx=NAME[bcx], bcy=NAME[bcy]) as plan:
        fd = torch.from_numpy(f).cuda()
        p = torch.empty_like(fd)
        info = plan.solve(fd, p, rtol=rtol, max_iter=12)
        torch.cuda.synchronize()
        return p.cpu().numpy(), info


@pytest.mark.parametrize("bcz", ["periodic", "walls"])
@pytest.mark.parametrize("shape", [(8, 16, 32), (16, 32, 8), (8, 8, 64)])
@pytest.mark.parametrize("bcx,bcy", ENDS)
def test_solve_with_ends_matches_oracle(bcx, bcy, shape, bcz):
    nz, ny, nx = shape
    dx, dy = 1.0 / nx, 1.3 / ny
    if bcz == "periodic":
        dzf = 0.7 / nz
    else:
        beta = 1.5
        zf = 0.5 * (1 + np.tanh(beta * (2 * np.arange(nz + 1) / nz - 1)) / np.tanh(beta))
        dzf = np.diff(zf)
    g = oracle.make_grid(nx, ny, nz, dx, dy, dzf, bcz)
    f = np.random.default_rng(zlib.crc32(repr((bcx, bcy, shape, bcz)).encode())).standard_normal(shape)
    po = r2r.solve(f, g, bcx, bcy)
    p, _ = run(f, nx, ny, nz, dx, dy, dzf, bcz, bcx, bcy)
    err = np.linalg.norm(p - po) / np.linalg.norm(po)
    assert err <= 1e-11, err
    assert r2r.rel_residual(f, p, g, bcx, bcy) <= 1e-12
    # FP32 transforms with FP64 defect correction to 1e-10: the oracle's residual of the GPU's p
    # meets rtol, and p is within the residual times the conditioning of the smallest mode
    p32, info = run(f, nx, ny, nz, dx, dy, dzf, bcz, bcx, bcy, "fp32_refine", 1e-10)
    assert info.rel_res <= 1e-10
    assert r2r.rel_residual(f, p32, g, bcx, bcy) <= 1e-10
    assert np.linalg.norm(p32 - po) / np.linalg.norm(po) <= 1e-7


@pytest.mark.parametrize("bcx,bcy", [("ND", "DN"), ("DN", "NN")])
def test_single_mixed_mode(bcx, bcy):
    """Mixed ends: cos/sin(pi (2k+1)(2i+1)/(4n)) modes with eigenvalues -4 sin^2(pi (2k+1)/(4n))/h^2."""
    nz, ny, nx = 8, 16, 32
    dx, dy, dz = 0.1, 0.07, 0.2
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    kx, ky = 6, 2

    def mode(bc, kk, ii, n):
        if bc == "ND":
            return np.cos(np.pi * (2 * kk + 1) * (2 * ii + 1) / (4 * n))
        if bc == "DN":
            return np.sin(np.pi * (2 * kk + 1) * (2 * ii + 1) / (4 * n))
        return np.cos(np.pi * kk * (2 * ii + 1) / (2 * n))
    f = mode(bcx, kx, i, nx)[None, None, :] * mode(bcy, ky, j, ny)[None, :, None] * np.ones((nz, 1, 1))
    lx = -4 * np.sin(np.pi * (2 * kx + 1) / (4 * nx)) ** 2 / dx ** 2
    ly = (-4 * np.sin(np.pi * (2 * ky + 1) / (4 * ny)) ** 2 if bcy != "NN" else -4 * np.sin(np.pi * ky / (2 * ny)) ** 2) / dy ** 2
    p, _ = run(f, nx, ny, nz, dx, dy, dz, "periodic", bcx, bcy)
    assert np.max(np.abs(p - f / (lx + ly))) <= 1e-12 * np.max(np.abs(f / (lx + ly)))


def test_single_mode_with_ends():
    """A cosine mode in x (Neumann) times a sine mode in y (Dirichlet) times a Fourier mode in z:
    p = f / (lam_x + lam_y + lam_z) exactly, with the closed-form eigenvalues."""
    nz, ny, nx = 8, 16, 32
    dx, dy, dz = 0.1, 0.07, 0.2
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    kx, ky, kz = 5, 3, 2
    f = (np.cos(np.pi * kx * (2 * i + 1) / (2 * nx))[None, None, :]
         * np.sin(np.pi * (ky + 1) * (2 * j + 1) / (2 * ny))[None, :, None]
         * np.cos(2 * np.pi * kz * k / nz + 0.3)[:, None, None])
    lam = (-4 * np.sin(np.pi * kx / (2 * nx)) ** 2 / dx ** 2 - 4 * np.sin(np.pi * (ky + 1) / (2 * ny)) ** 2 / dy ** 2
           - 4 * np.sin(np.pi * kz / nz) ** 2 / dz ** 2)
    p, _ = run(f, nx, ny, nz, dx, dy, dz, "periodic", "NN", "DD")
    assert np.max(np.abs(p - f / lam)) <= 1e-12 * np.max(np.abs(f / lam))


def test_periodic_ends_through_the_new_entry_point_equal_the_old():
    nz, ny, nx = 8, 16, 32
    f = np.random.default_rng(5).standard_normal((nz, ny, nx))
    p1, _ = run(f, nx, ny, nz, 0.1, 0.1, 0.1, "periodic", "P", "P")
    with flups.Plan(nx, ny, nz, 0.1, 0.1, 0.1, "periodic", "fp64", flups.current_stream()) as plan:
        fd = torch.from_numpy(f).cuda()
        p = torch.empty_like(fd)
        plan.solve(fd, p, rtol=0.0)
        p2 = p.cpu().numpy()
    assert np.array_equal(p1, p2)


def test_unsupported_uses_of_plans_with_ends():
    with flups.Plan(32, 16, 8, 0.1, 0.1, 0.1, "periodic", "fp32_refine", bcx="neumann") as plan:
        z = torch.zeros((8, 16, 32), dtype=torch.float64, device="cuda")
        with pytest.raises(flups.FlupsError) as e:
            plan.solve_graphable(z, z.clone(), rtol=1e-10, max_iter=3)
        assert e.value.status == flups.EUNSUPPORTED
    with flups.Plan(32, 16, 8, 0.1, 0.1, 0.1, "periodic", "fp64", bcx="neumann") as plan:
        z = torch.zeros((8, 16, 32), dtype=torch.float64, device="cuda")
        with pytest.raises(flups.FlupsError) as e:
            plan.set_density(z + 1.0)
        assert e.value.status == flups.EUNSUPPORTED
        with pytest.raises(flups.FlupsError) as e:
            plan.rhs(z, z, z, z, z, 2.0, 1.0, 1e-3, z.clone())
        assert e.value.status == flups.EUNSUPPORTED


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_walls_solve_removes_the_mean_of_f(prec):
    """z walls, periodic x and y, f with a large mean: the solve returns L^-1 (f - <f>_V) with zero
    mean (R3) in both precisions (the singular column subtracts the mean before dropping its
    first row)."""
    nz, ny, nx = 12, 16, 32
    beta = 1.5
    zf = 0.5 * (1 + np.tanh(beta * (2 * np.arange(nz + 1) / nz - 1)) / np.tanh(beta))
    dzf = np.diff(zf)
    g = oracle.make_grid(nx, ny, nz, 1 / nx, 1 / ny, dzf, "walls")
    f = np.random.default_rng(8).standard_normal((nz, ny, nx)) + 3.7
    with flups.Plan(nx, ny, nz, 1 / nx, 1 / ny, dzf, "walls", prec, flups.current_stream()) as plan:
        fd = torch.from_numpy(f).cuda()
        p = torch.empty_like(fd)
        plan.solve(fd, p, rtol=1e-12 if prec == "fp32_refine" else 0.0, max_iter=12)
        p = p.cpu().numpy()
    po = oracle.solve(f, g)
    assert np.linalg.norm(p - po) / np.linalg.norm(po) <= (1e-11 if prec == "fp64" else 1e-9)


@pytest.mark.slow
def test_fullsize_closed_box_512x512x256():
    """The measured workload (Neumann ends in x and y, stretched z walls, f ~ N(0,1) seed 60): the
    oracle's residual of the GPU's p (FP32+refine to 1e-10, and FP64 direct), and both against
    the oracle's own solve at full size."""
    from paper_2204_08834_gb300 import synth
    nx, ny, nz = 512, 512, 256
    dzf = synth.stretched_dzf(nz, 1.0, 1.5)
    g = oracle.make_grid(nx, ny, nz, 2.0 / nx, 2.0 / ny, dzf, "walls")
    f = np.random.default_rng(60).standard_normal((nz, ny, nx))
    p32, info = run(f, nx, ny, nz, 2.0 / nx, 2.0 / ny, dzf, "walls", "NN", "NN", "fp32_refine", 1e-10)
    torch.cuda.empty_cache()
    p64, _ = run(f, nx, ny, nz, 2.0 / nx, 2.0 / ny, dzf, "walls", "NN", "NN")
    torch.cuda.empty_cache()
    assert info.rel_res <= 1e-10
    assert r2r.rel_residual(f, p32, g, "NN", "NN") <= 1e-10
    assert r2r.rel_residual(f, p64, g, "NN", "NN") <= 1e-12
    po = r2r.solve(f, g, "NN", "NN")
    assert np.linalg.norm(p64 - po) / np.linalg.norm(po) <= 1e-11
    assert np.linalg.norm(p32 - po) / np.linalg.norm(po) <= 1e-7
