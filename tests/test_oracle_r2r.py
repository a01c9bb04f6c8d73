"""Pins of the Neumann/Dirichlet-end Poisson oracle (Sec. 3.3.1 eigen-expansion, readings E1-E4
in oracle/r2r.py) against constructions that do not use the oracle: an operator assembled
cell by cell from the ghost rules, dense solves, explicit cosine/sine sums, closed-form modes."""

import itertools

import numpy as np
import pytest

from oracle import projection as P
from oracle import r2r

KINDS = r2r.KINDS


def dense_operator(g, bcx, bcy):
    """The 7-point operator as a dense matrix, assembled by looping over cells: each
    neighbour across a periodic face wraps, across a Neumann face it is the cell itself,
    across a Dirichlet face it is minus the cell itself (ghost rules of oracle/r2r.py)."""
    nx, ny, nz = g.nx, g.ny, g.nz
    n = nx * ny * nz
    A = np.zeros((n, n))

    def idx(i, j, k):
        return (k * ny + j) * nx + i

    def neighbour(bc, m, n_, step):
        """(index, sign) of the neighbour of m in direction step along a line of n_ cells."""
        t = m + step
        if 0 <= t < n_:
            return t, 1.0
        if bc == "P":
            return t % n_, 1.0
        end = bc[0] if t < 0 else bc[1]
        return m, (1.0 if end == "N" else -1.0)

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = idx(i, j, k)
                for bc, h, axis in ((bcx, g.dx, 0), (bcy, g.dy, 1)):
                    for step in (-1, 1):
                        if axis == 0:
                            t, s = neighbour(bc, i, nx, step)
                            A[r, idx(t, j, k)] += s / h ** 2
                        else:
                            t, s = neighbour(bc, j, ny, step)
                            A[r, idx(i, t, k)] += s / h ** 2
                    A[r, r] -= 2.0 / h ** 2
                # z: flux form with dzf, dzc (periodic or Neumann walls)
                for step in (-1, 1):
                    t = k + step
                    if g.bc == "walls" and not 0 <= t < nz:
                        continue
                    t %= nz
                    dzc = g.dzc[k] if step == 1 else g.dzc[(k - 1) % nz]
                    cf = 1.0 / (g.dzf[k] * dzc)
                    A[r, idx(i, j, t)] += cf
                    A[r, r] -= cf
    return A


def grid(bcz, nx=4, ny=4, nz=4):
    dz = 0.25 if bcz == "periodic" else np.array([0.2, 0.3, 0.25, 0.15])[:nz]
    return P.make_grid(nx, ny, nz, 0.3, 0.2, dz, bcz)


@pytest.mark.parametrize("bcz", ["periodic", "walls"])
@pytest.mark.parametrize("bcx,bcy", list(itertools.product(KINDS, KINDS)))
def test_lap_equals_assembled_operator(bcx, bcy, bcz):
    g = grid(bcz)
    p = np.random.default_rng(1).standard_normal((g.nz, g.ny, g.nx))
    A = dense_operator(g, bcx, bcy)
    assert np.max(np.abs(r2r.lap(p, g, bcx, bcy).ravel() - A @ p.ravel())) < 1e-10 * np.max(np.abs(A))


@pytest.mark.parametrize("bcz", ["periodic", "walls"])
@pytest.mark.parametrize("bcx,bcy", list(itertools.product(KINDS, KINDS)))
def test_solve_equals_dense_solve(bcx, bcy, bcz):
    g = grid(bcz)
    rng = np.random.default_rng(2)
    f = rng.standard_normal((g.nz, g.ny, g.nx))
    A = dense_operator(g, bcx, bcy)
    n = A.shape[0]
    wts = np.repeat(g.dzf, g.nx * g.ny)
    sing = bcx in ("P", "NN") and bcy in ("P", "NN")
    if sing:      # bordered system: A p + mu 1 = f - <f>, sum(dzf p) = 0
        fm = f.ravel() - np.sum(f.ravel() * wts) / np.sum(wts)
        B = np.zeros((n + 1, n + 1))
        B[:n, :n] = A
        B[:n, n] = 1.0
        B[n, :n] = wts
        x = np.linalg.solve(B, np.concatenate([fm, [0.0]]))[:n]
    else:
        assert np.linalg.matrix_rank(A) == n
        x = np.linalg.solve(A, f.ravel())
    p = r2r.solve(f, g, bcx, bcy)
    assert np.max(np.abs(p.ravel() - x)) < 1e-10 * max(1.0, np.max(np.abs(x)))


@pytest.mark.parametrize("bc", ["NN", "DD", "ND", "DN"])
def test_single_modes_and_eigenvalues_closed_form(bc):
    n, h = 12, 0.37
    i = np.arange(n)
    lam = r2r.eigenvalues(n, h, bc)
    for k in range(n):
        if bc == "NN":
            v = np.cos(np.pi * k * (2 * i + 1) / (2 * n))
            ref = -4 * np.sin(np.pi * k / (2 * n)) ** 2 / h ** 2
        elif bc == "DD":
            v = np.sin(np.pi * (k + 1) * (2 * i + 1) / (2 * n))
            ref = -4 * np.sin(np.pi * (k + 1) / (2 * n)) ** 2 / h ** 2
        elif bc == "ND":
            v = np.cos(np.pi * (2 * k + 1) * (2 * i + 1) / (4 * n))
            ref = -4 * np.sin(np.pi * (2 * k + 1) / (4 * n)) ** 2 / h ** 2
        else:
            v = np.sin(np.pi * (2 * k + 1) * (2 * i + 1) / (4 * n))
            ref = -4 * np.sin(np.pi * (2 * k + 1) / (4 * n)) ** 2 / h ** 2
        a = np.broadcast_to(v, (2, 3, n)).copy()
        assert np.max(np.abs(r2r.second_difference(a, bc, h, 2) - ref * a)) < 1e-10 / h ** 2
        assert abs(lam[k] - ref) < 1e-10 / h ** 2
    # the 1-D operator's spectrum (dense, assembled from the ghost rules) is the same set
    g1 = P.make_grid(n, 1, 1, h, 1.0, 1.0, "periodic")
    A = dense_operator(g1, bc, "P")
    ev = np.sort(np.linalg.eigvals(A).real)
    assert np.allclose(ev, np.sort(lam), atol=1e-9 / h ** 2)


@pytest.mark.parametrize("bc", ["NN", "DD", "ND", "DN"])
def test_library_transform_kind_is_the_eigenvector_projection(bc):
    """forward(x)_k equals 2 sum_i x_i v_k(i) with the eigenvectors of E1 (explicit sums)."""
    n = 10
    x = np.random.default_rng(3).standard_normal(n)
    i = np.arange(n)
    X = r2r.forward(x[None, None, :], bc, 2, True)[0, 0]
    for k in range(n):
        if bc == "NN":
            v = np.cos(np.pi * k * (2 * i + 1) / (2 * n))
        elif bc == "DD":
            v = np.sin(np.pi * (k + 1) * (2 * i + 1) / (2 * n))
        elif bc == "ND":
            v = np.cos(np.pi * (2 * k + 1) * (2 * i + 1) / (4 * n))
        else:
            v = np.sin(np.pi * (2 * k + 1) * (2 * i + 1) / (4 * n))
        assert abs(X[k] - 2 * np.dot(x, v)) < 1e-12
    assert np.allclose(r2r.backward(X[None, None, :], bc, 2, n, True)[0, 0], x, atol=1e-13)


@pytest.mark.parametrize("bcz", ["periodic", "walls"])
def test_periodic_ends_reduce_to_the_projection_oracle(bcz):
    g = grid(bcz, 8, 8, 4)
    f = np.random.default_rng(4).standard_normal((g.nz, g.ny, g.nx))
    assert np.max(np.abs(r2r.solve(f, g, "P", "P") - P.solve(f, g))) < 1e-12


def test_nonsingular_solve_keeps_the_mean():
    """With a Dirichlet end, f's mean is part of the problem: L p = f holds exactly."""
    g = grid("walls", 8, 6, 4)
    f = np.ones((g.nz, g.ny, g.nx))
    for bcx, bcy in (("DD", "P"), ("ND", "NN"), ("P", "DN")):
        p = r2r.solve(f, g, bcx, bcy)
        assert np.max(np.abs(r2r.lap(p, g, bcx, bcy) - f)) < 1e-10
