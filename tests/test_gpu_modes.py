"""GPU solves of single Fourier modes against the closed form (Sec. 3.3.1: the eigen-expansion
diagonalises L, so a mode of the discrete operator is returned exactly up to rounding).

For p = cos(2 pi (ax i/nx + ay j/ny + az k/nz)) on a periodic grid, or
p = cos(2 pi (ax i/nx + ay j/ny)) cos(pi az (k + 1/2)/nz) with walls and uniform dz, the
right-hand side f = lam p with lam = sum_d (2 cos(theta_d) - 2)/h_d^2 (theta = 2 pi a/n
periodic, pi a/n Neumann) has zero mean for any nonzero mode, so the solve must return p.
Tolerance (rounding of a direct solve, amplified by the condition of the mode):
C eps cond with cond = (sum_d 4/h_d^2)/|lam| and C = max(64, 8 log2 N) for N grid points
(the rounding error of an N-point transform grows like log N; 64 covers the oracle's small
pins).  FP32 + FP64 refinement (to rtol = 1e-13, or 32 eps cond where the FP64 defect of the
mode cannot go lower) adds 4 rtol max(cond, |lam|/lam_min): the defect left at rtol may sit
in the smoothest mode.
Cases include the Nyquist modes, (0, 0, az), and lengths 3 * 2^a; the 512-long columns go
through the register four-step column kernels, the walls cases through the tiled partitioned
Thomas kernel.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_08834_gb300 import flups  # noqa: E402

EPS = np.finfo(np.float64).eps


def mode_case(nx, ny, nz, ax, ay, az, bc):
    dx, dy, dz = 1.0 / nx, 1.3 / ny, 0.7 / nz
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    lam = (2 * np.cos(2 * np.pi * ax / nx) - 2) / dx ** 2 + (2 * np.cos(2 * np.pi * ay / ny) - 2) / dy ** 2
    # phases reduced exactly in integers (a phase of many turns formed in floating point
    # carries an error of that many ulps into the "exact" mode)
    if bc == "periodic":
        n = nx * ny * nz
        turns = (ax * i * (ny * nz) + ay * j * (nx * nz) + az * k * (nx * ny)) % n
        p = np.cos(2 * np.pi * turns / n)
        lam += (2 * np.cos(2 * np.pi * az / nz) - 2) / dz ** 2
    else:
        n = nx * ny
        turns = (ax * i * ny + ay * j * nx) % n
        zt = (az * (2 * k + 1)) % (4 * nz)
        p = np.cos(2 * np.pi * turns / n) * np.cos(2 * np.pi * zt / (4 * nz))
        lam += (2 * np.cos(np.pi * az / nz) - 2) / dz ** 2
    cond = (4 / dx ** 2 + 4 / dy ** 2 + 4 / dz ** 2) / abs(lam)
    # smallest nonzero |eigenvalue| of L: a defect of size rtol |lam| |p| left in the
    # smoothest mode moves p by up to rtol |lam| / lam_min
    lmin = min(4 * np.sin(np.pi / nx) ** 2 / dx ** 2, 4 * np.sin(np.pi / ny) ** 2 / dy ** 2,
               4 * np.sin(np.pi / (nz if bc == "periodic" else 2 * nz)) ** 2 / dz ** 2)
    return np.ascontiguousarray(p), lam * p, abs(lam) / lmin, cond


CASES = [
    # (nx, ny, nz, bc, modes)
    (32, 48, 64, "periodic", [(1, 0, 0), (0, 0, 1), (16, 24, 32), (3, 5, 7), (0, 24, 0), (0, 0, 32)]),
    (16, 512, 512, "periodic", [(0, 0, 1), (8, 256, 256), (1, 3, 200), (0, 1, 0)]),
    (96, 24, 48, "periodic", [(48, 12, 24), (5, 0, 1), (0, 0, 24)]),
    (32, 32, 24, "walls", [(0, 0, 1), (16, 16, 23), (2, 3, 5), (0, 1, 0), (1, 0, 0)]),
    (64, 16, 256, "walls", [(0, 0, 1), (32, 8, 255), (7, 1, 100)]),
    (48, 96, 30, "walls", [(24, 48, 29), (1, 1, 1)]),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("nx,ny,nz,bc,modes", CASES)
def test_single_modes(nx, ny, nz, bc, modes, prec):
    with flups.Plan(nx, ny, nz, 1.0 / nx, 1.3 / ny, np.full(nz, 0.7 / nz), bc, prec,
                    flups.current_stream()) as plan:
        for ax, ay, az in modes:
            p_exact, f, spread, cond = mode_case(nx, ny, nz, ax, ay, az, bc)
            # the FP64 defect of a smooth mode cannot go below about eps cond (reading c10)
            rtol = max(1e-13, 32 * EPS * cond)
            fd = torch.from_numpy(f).cuda()
            pd = torch.empty_like(fd)
            info = plan.solve(fd, pd, rtol=rtol if prec == "fp32_refine" else 0.0, max_iter=12,
                              info=prec == "fp32_refine")
            pg = pd.cpu().numpy()
            err = np.linalg.norm(pg - p_exact) / np.linalg.norm(p_exact)
            C = max(64.0, 8.0 * np.log2(nx * ny * nz))
            tol = C * EPS * cond + (4 * rtol * max(cond, spread) if prec == "fp32_refine" else 0.0)
            assert err <= tol, (ax, ay, az, err, tol)
            if prec == "fp32_refine":
                assert info.rel_res <= rtol
