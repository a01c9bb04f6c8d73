"""Pins of the FP64 oracle against facts fixed by mathematics (CPU only).

Each test checks the oracle against something other than itself: closed-form
eigenvalues of the discrete operators, a dense LU solve of the operator assembled by
brute force (unit vectors), explicit DFT sums, an explicitly looped variable-coefficient
operator, and the invariants the direct method must satisfy (Sec. 3.1: with a direct
Poisson solver the discrete divergence vanishes to machine precision).
"""

import itertools

import numpy as np
import pytest

import oracle
from paper_2204_08834_gb300 import synth

EPS = np.finfo(np.float64).eps


def rand(shape, seed):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(shape)


def grid(nx, ny, nz, bc, stretched=False, dx=None, dy=None):
    dx = dx or 1.0 / nx
    dy = dy or 1.3 / ny
    dzf = synth.stretched_dzf(nz, 0.9, 1.5) if stretched else 0.7 / nz
    return oracle.make_grid(nx, ny, nz, dx, dy, dzf, bc)


# --------------------------------------------------------------- operator pins

def test_face_density_orientation():
    """Face i+1/2 sits between cells i and i+1 (MAC grid, Sec. 3)."""
    g = grid(4, 5, 6, "walls")
    i = np.arange(4.0)[None, None, :] * np.ones((6, 5, 1))
    j = np.arange(5.0)[None, :, None] * np.ones((6, 1, 4))
    k = np.arange(6.0)[:, None, None] * np.ones((1, 5, 4))
    rx, _, _ = oracle.face_density(i, g)
    _, ry, _ = oracle.face_density(j, g)
    _, _, rz = oracle.face_density(k, g)
    assert np.allclose(rx[..., :3], i[..., :3] + 0.5) and np.allclose(rx[..., 3], 1.5)
    assert np.allclose(ry[:, :4], j[:, :4] + 0.5) and np.allclose(ry[:, 4], 2.0)
    assert np.allclose(rz[:5], k[:5] + 0.5)


@pytest.mark.parametrize("bc", ["periodic", "walls"])
@pytest.mark.parametrize("stretched", [False, True])
def test_adjoint_div_grad(bc, stretched):
    """sum_cells dzf p (D u) = - sum_faces (face volume) u (G p): D = -G^T, which fixes the
    relative index shift and sign of every difference."""
    if bc == "periodic" and stretched:
        pytest.skip("periodic z is uniform")
    g = grid(6, 5, 7, bc, stretched)
    p = rand(g.dzf.shape + (5, 6), 1)
    u, v, w = (rand(p.shape, s) for s in (2, 3, 4))
    if bc == "walls":
        w[-1] = 0.0
    lhs = np.sum(g.dzf[:, None, None] * p * oracle.div(u, v, w, g))
    gx, gy, gz = oracle.grad(p, g)
    dzc = g.dzc.copy()
    if bc == "walls":
        dzc[-1] = 0.0
    rhs_ = -(np.sum(g.dzf[:, None, None] * (u * gx + v * gy)) + np.sum(dzc[:, None, None] * w * gz))
    assert abs(lhs - rhs_) <= 1e-12 * np.sum(np.abs(g.dzf[:, None, None] * p * oracle.div(u, v, w, g)))


def test_lap_of_linear_z_on_stretched_walls():
    """On any z grid with centres midway between faces, G_z z_c = 1 on interior faces,
    so L z_c = +1/dzf_0 in the bottom cell, -1/dzf_{nz-1} in the top one, 0 elsewhere."""
    g = grid(4, 4, 9, "walls", stretched=True)
    zf = np.concatenate(([0.0], np.cumsum(g.dzf)))
    zc = 0.5 * (zf[:-1] + zf[1:])
    p = np.broadcast_to(zc[:, None, None], (9, 4, 4)).copy()
    L = oracle.lap(p, g)
    want = np.zeros(9)
    want[0], want[-1] = 1.0 / g.dzf[0], -1.0 / g.dzf[-1]
    assert np.allclose(L, want[:, None, None], rtol=0, atol=1e-12 / g.dzf.min())


def _mode_periodic(nx, ny, nz, ax, ay, az):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.cos(2 * np.pi * (ax * i / nx + ay * j / ny + az * k / nz))


def _lam(a, n, h, neumann=False):
    th = (np.pi if neumann else 2 * np.pi) * a / n
    return (2 * np.cos(th) - 2) / h ** 2


@pytest.mark.parametrize("dims,modes", [
    ((8, 8, 8), [(1, 0, 0), (0, 1, 0), (0, 0, 1), (4, 4, 4), (3, 2, 1), (0, 0, 4)]),
    ((16, 6, 10), [(8, 3, 5), (1, 1, 1), (7, 0, 2), (0, 3, 0)]),
])
def test_single_mode_periodic(dims, modes):
    """p = cos(2 pi (ax i/nx + ay j/ny + az k/nz)) is an eigenvector of L with
    lambda = sum_d (2 cos(2 pi a_d / n_d) - 2) / h_d^2; the solve must return it exactly."""
    nx, ny, nz = dims
    g = grid(nx, ny, nz, "periodic")
    for ax, ay, az in modes:
        p = _mode_periodic(nx, ny, nz, ax, ay, az)
        lam = _lam(ax, nx, g.dx) + _lam(ay, ny, g.dy) + _lam(az, nz, g.dzf[0])
        assert np.allclose(oracle.lap(p, g), lam * p, atol=1e-12 * abs(lam))
        cond = (4 / g.dx ** 2 + 4 / g.dy ** 2 + 4 / g.dzf[0] ** 2) / abs(lam)
        err = np.max(np.abs(oracle.solve(lam * p, g) - p))
        assert err <= 64 * EPS * cond, (ax, ay, az, err)


@pytest.mark.parametrize("modes", [[(1, 0, 1), (0, 0, 1), (2, 3, 5), (4, 0, 7), (0, 2, 0)]])
def test_single_mode_walls_uniform(modes):
    """With Neumann walls and uniform dz, cos(pi az (k+1/2)/nz) is the z eigenvector with
    lambda_z = (2 cos(pi az/nz) - 2)/dz^2."""
    nx, ny, nz = 8, 6, 8
    g = grid(nx, ny, nz, "walls")
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for ax, ay, az in modes:
        p = np.cos(2 * np.pi * (ax * i / nx + ay * j / ny)) * np.cos(np.pi * az * (k + 0.5) / nz)
        lam = _lam(ax, nx, g.dx) + _lam(ay, ny, g.dy) + _lam(az, nz, g.dzf[0], neumann=True)
        assert np.allclose(oracle.lap(p, g), lam * p, atol=1e-12 * abs(lam))
        cond = (4 / g.dx ** 2 + 4 / g.dy ** 2 + 4 / g.dzf[0] ** 2) / abs(lam)
        err = np.max(np.abs(oracle.solve(lam * p, g) - p))
        assert err <= 64 * EPS * cond, (ax, ay, az, err)


# ---------------------------------------------------------------- dense LU pins

def dense_operator(g):
    """Matrix of L assembled by applying the oracle operator to unit vectors (brute force)."""
    n = g.nx * g.ny * g.nz
    A = np.empty((n, n))
    e = np.zeros(n)
    for c in range(n):
        e[c] = 1.0
        A[:, c] = oracle.lap(e.reshape(g.nz, g.ny, g.nx), g).ravel()
        e[c] = 0.0
    return A


def bordered_solve(A, f, wts):
    """Solve [A 1; w^T 0][p; mu] = [f - <f>_w; 0] with LAPACK's partial-pivoting LU."""
    n = A.shape[0]
    B = np.zeros((n + 1, n + 1))
    B[:n, :n] = A
    B[:n, n] = 1.0
    B[n, :n] = wts
    fm = f - np.sum(wts * f) / np.sum(wts)
    x = np.linalg.solve(B, np.concatenate((fm, [0.0])))
    return x[:n], x[n]


@pytest.mark.parametrize("dims,bc,stretched", [
    ((4, 4, 4), "periodic", False),
    ((6, 6, 6), "periodic", False),
    ((8, 8, 8), "periodic", False),
    ((4, 6, 8), "periodic", False),
    ((4, 4, 4), "walls", False),
    ((6, 6, 6), "walls", True),
    ((8, 8, 8), "walls", True),
    ((4, 6, 8), "walls", True),
    ((6, 4, 3), "walls", True),
])
def test_solve_matches_dense_lu(dims, bc, stretched):
    """The eigen-expansion solve equals the dense bordered LU solution (null space pinned by
    zero volume-weighted mean) to round-off."""
    nx, ny, nz = dims
    g = grid(nx, ny, nz, bc, stretched)
    A = dense_operator(g)
    wts = np.broadcast_to(g.dzf[:, None, None], (nz, ny, nx)).ravel()
    f = rand((nz, ny, nx), 7)
    p_lu, mu = bordered_solve(A, f.ravel(), wts)
    assert abs(mu) < 1e-10 * np.max(np.abs(f))
    p = oracle.solve(f, g)
    assert np.max(np.abs(p.ravel() - p_lu)) <= 1e-11 * np.max(np.abs(p_lu))
    assert abs(oracle.volume_mean(p, g)) <= 1e-14 * np.max(np.abs(p))


def test_dense_operator_rank_and_null_space():
    """L has exactly the constants as null space and the volume weights as left null vector."""
    g = grid(4, 4, 6, "walls", stretched=True)
    A = dense_operator(g)
    s = np.linalg.svd(A, compute_uv=False)
    assert s[-1] < 1e-10 * s[0] and s[-2] > 1e-6 * s[0]
    wts = np.broadcast_to(g.dzf[:, None, None], (6, 4, 4)).ravel()
    assert np.max(np.abs(wts @ A)) < 1e-10 * s[0]
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) < 1e-10 * s[0]


# ------------------------------------------------------- spectral-step pins

def test_forward_steps_are_explicit_dft_sums():
    """Steps 1 and 3 (forward along x, then y) equal the explicit sums
    F(kx, ky) = sum_{i,j} f(i, j) exp(-2 pi i (kx i/nx + ky j/ny)) (sign R7)."""
    nx, ny = 6, 4
    f = rand((ny, nx), 3)
    F = np.fft.fft(np.fft.rfft(f, axis=1), axis=0)
    for ky, kx in itertools.product(range(ny), range(nx // 2 + 1)):
        s = 0j
        for j, i in itertools.product(range(ny), range(nx)):
            s += f[j, i] * np.exp(-2j * np.pi * (kx * i / nx + ky * j / ny))
        assert abs(F[ky, kx] - s) < 1e-12


@pytest.mark.parametrize("n", [2, 3, 4, 6, 8, 12, 16, 48, 96])
def test_transform_lengths_of_the_path_are_explicit_dft_sums(n):
    """Every length the GPU path factors (radix 2, 3, 4, 8, the ensemble's 48 and 96): the
    library's real and complex forward transforms and their inverses equal the O(n^2) sums."""
    x = rand((n,), 7 + n)
    z = x + 1j * rand((n,), 8 + n)
    k = np.arange(n)
    W = np.exp(-2j * np.pi * np.outer(k, k) / n)
    assert np.max(np.abs(np.fft.fft(z) - W @ z)) < 1e-12 * n
    assert np.max(np.abs(np.fft.rfft(x) - (W @ x)[: n // 2 + 1])) < 1e-12 * n
    assert np.max(np.abs(np.fft.ifft(z) - (W.conj() @ z) / n)) < 1e-13 * n
    assert np.max(np.abs(np.fft.irfft(np.fft.rfft(x), n=n) - x)) < 1e-13 * n


def test_eigenvalues_match_dft_of_stencil():
    """(2 cos(2 pi k/n) - 2)/h^2 is the DFT of the periodic 3-point stencil."""
    n, h = 12, 0.3
    col = np.zeros(n)
    col[0], col[1], col[-1] = -2 / h ** 2, 1 / h ** 2, 1 / h ** 2
    lam = np.array([sum(col[m] * np.exp(-2j * np.pi * k * m / n) for m in range(n)) for k in range(n)])
    assert np.allclose(lam.real, oracle.eigenvalues(n, h)) and np.allclose(lam.imag, 0)


def test_thomas_matches_dense_per_column():
    """Gauss elimination along z equals a dense solve of each column's tridiagonal system,
    including the singular (0, 0) column solved with zero volume-weighted mean (R4)."""
    g = grid(6, 4, 9, "walls", stretched=True)
    a, b, c = oracle.z_coefficients(g)
    lx = oracle.eigenvalues(6, g.dx)[:4]
    ly = oracle.eigenvalues(4, g.dy)
    lam = ly[:, None] + lx[None, :]
    F = rand((9, 4, 4), 5) + 1j * rand((9, 4, 4), 6)
    # compatibility of the singular column
    F[:, 0, 0] -= np.sum(F[:, 0, 0] * g.dzf) / np.sum(g.dzf)
    P = oracle.tridiag_z(F, lam, g)
    T = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    for ky, kx in itertools.product(range(4), range(4)):
        M = T + lam[ky, kx] * np.eye(9)
        if (ky, kx) == (0, 0):
            B = np.zeros((10, 10), dtype=complex)
            B[:9, :9] = M
            B[:9, 9] = 1.0
            B[9, :9] = g.dzf
            want = np.linalg.solve(B, np.concatenate((F[:, 0, 0], [0])))[:9]
        else:
            want = np.linalg.solve(M, F[:, ky, kx])
        assert np.allclose(P[:, ky, kx], want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


# ------------------------------------------------------------- invariants

def _case(bc, n=12, stretched=True):
    c = synth.sphere(n)
    if bc == "walls":
        c["w"][-1] = 0.0
        dzf = synth.stretched_dzf(n, 1.0, 1.5) if stretched else np.full(n, 1.0 / n)
        return c, oracle.make_grid(n, n, n, c.dx, c.dy, dzf, "walls")
    return c, oracle.make_grid(n, n, n, c.dx, c.dy, c.dzf, "periodic")


@pytest.mark.parametrize("bc", ["periodic", "walls"])
def test_projection_divergence_free_and_zero_mean(bc):
    """After the correction D u^{n+1} = 0 to machine precision (Sec. 3.1: a direct solve
    conserves mass to machine precision); <p>_V = 0 (R3)."""
    c, g = _case(bc)
    f, p, u1, v1, w1 = oracle.project(c.u, c.v, c.w, c.rho, c.pn, c.pnm1, 2.0, 1.0, c.dt, g)
    assert oracle.div_rel(u1, v1, w1, c.u, c.v, c.w, g) < 1e-12
    assert abs(oracle.volume_mean(p, g)) < 1e-14 * np.max(np.abs(p))
    assert oracle.rel_residual(f, p, g) < 1e-13
    if bc == "walls":
        assert np.all(w1[-1] == 0.0)


@pytest.mark.parametrize("bc", ["periodic", "walls"])
def test_constant_density_makes_p_hat_irrelevant(bc):
    """rho = const gives rho_0 = rho, so the splitting term vanishes (textbook projection)."""
    c, g = _case(bc)
    rho = np.full_like(c.rho, 3.0)
    a = oracle.project(c.u, c.v, c.w, rho, c.pn, c.pnm1, 2.0, 1.0, c.dt, g)
    b = oracle.project(c.u, c.v, c.w, rho, 0 * c.pn, 0 * c.pnm1, 2.0, 1.0, c.dt, g)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.allclose(a[0], (3.0 / c.dt) * oracle.div(c.u, c.v, c.w, g))


def test_linearity_in_velocity_and_p_hat():
    c, g = _case("walls", n=8)
    args = (c.rho,)
    f1 = oracle.rhs(c.u, c.v, c.w, *args, c.pn, c.pnm1, 2.0, 1.0, c.dt, g)
    f2 = oracle.rhs(2 * c.u, 2 * c.v, 2 * c.w, *args, 2 * c.pn, 2 * c.pnm1, 2.0, 1.0, c.dt, g)
    assert np.allclose(f2, 2 * f1, rtol=1e-14, atol=1e-13 * np.max(np.abs(f1)))
    p1 = oracle.solve(f1, g)
    assert np.allclose(oracle.solve(2 * f1, g), 2 * p1, atol=1e-13 * np.max(np.abs(p1)))


def varcoef_dense(rho, g):
    """Dense matrix of D((1/rho_f) G p), written with explicit index loops (independent of
    the oracle's vectorised operators): rho_f = (rho_a + rho_b)/2 on each face (R2)."""
    nz, ny, nx = rho.shape
    n = nx * ny * nz
    A = np.zeros((n, n))

    def idx(k, j, i):
        return (k * ny + (j % ny)) * nx + (i % nx)

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = idx(k, j, i)
                for (dj, di, h) in ((0, 1, g.dx), (0, -1, g.dx), (1, 0, g.dy), (-1, 0, g.dy)):
                    nb = idx(k, j + dj, i + di)
                    cf = 1.0 / (0.5 * (rho[k, j, i] + rho.ravel()[nb])) / (h * h)
                    A[r, nb] += cf
                    A[r, r] -= cf
                for dk in (1, -1):
                    kk = k + dk
                    if g.bc == "periodic":
                        kk %= nz
                    elif kk < 0 or kk >= nz:
                        continue
                    dzc = 0.5 * (g.dzf[k] + g.dzf[kk])
                    cf = 1.0 / (0.5 * (rho[k, j, i] + rho[kk, j, i])) / (g.dzf[k] * dzc)
                    A[r, idx(kk, j, i)] += cf
                    A[r, r] -= cf
    return A


@pytest.mark.parametrize("bc", ["periodic", "walls"])
def test_dodd_ferrante_fixed_point(bc):
    """If p_hat is the exact variable-coefficient pressure p_ex, D((1/rho_f) G p_ex) = D u**/dt,
    the split solve returns p_ex and u^{n+1} = u** - dt (1/rho_f) G p_ex (reading R1).
    The opposite sign of the splitting term (the literal reading of Eq. us_predic) fails."""
    n = 6
    c, g = _case(bc, n=n)
    rho = 1.0 + 9.0 * (rand((n, n, n), 9) > 0.3)
    A = varcoef_dense(rho, g)
    wts = np.broadcast_to(g.dzf[:, None, None], (n, n, n)).ravel()
    p_ex, _ = bordered_solve(A, (oracle.div(c.u, c.v, c.w, g) / c.dt).ravel(), wts)
    p_ex = p_ex.reshape(n, n, n)
    zero = np.zeros_like(p_ex)
    f, p, u1, v1, w1 = oracle.project(c.u, c.v, c.w, rho, p_ex, zero, 1.0, 0.0, c.dt, g)
    assert np.max(np.abs(p - p_ex)) < 1e-10 * np.max(np.abs(p_ex))
    gx, gy, gz = oracle.grad(p_ex, g)
    rx, ry, rz = oracle.face_density(rho, g)
    assert np.allclose(u1, c.u - c.dt * gx / rx, atol=1e-12 * np.max(np.abs(c.u)))
    assert np.allclose(v1, c.v - c.dt * gy / ry, atol=1e-12 * np.max(np.abs(c.v)))
    w_ex = c.w - c.dt * gz / rz
    if bc == "walls":
        w_ex[-1] = 0.0
    assert np.allclose(w1, w_ex, atol=1e-12 * np.max(np.abs(c.w)))
    # p_hat = 2 p^n - p^{n-1} at constant dt (Sec. 3.3): a pressure steady in time
    # extrapolates to itself, so p^n = p^{n-1} = p_ex is a fixed point too
    f2, p2, _, _, _ = oracle.project(c.u, c.v, c.w, rho, p_ex, p_ex, 2.0, 1.0, c.dt, g)
    assert np.max(np.abs(p2 - p_ex)) < 1e-10 * np.max(np.abs(p_ex))
    # negative control: flip the sign of the splitting term in the right-hand side
    rho0 = rho.min()
    hx, hy, hz = oracle.grad(p_ex, g)
    wrong = (rho0 / c.dt) * oracle.div(c.u, c.v, c.w, g) - oracle.div(
        (1 - rho0 / rx) * hx, (1 - rho0 / ry) * hy, (1 - rho0 / rz) * hz, g)
    assert np.max(np.abs(oracle.solve(wrong, g) - p_ex)) > 1e-3 * np.max(np.abs(p_ex))


def test_p_hat_linear_extrapolation():
    """p_hat = (1 + r) p^n - r p^{n-1}, r = dt^{n+1}/dt^n, extrapolates a pressure linear in
    time exactly: p(t) = q + t s sampled at t = -dt_n, 0 gives p(dt_{n+1}) (Sec. 3.3)."""
    q, s_, dtn, dtn1 = 1.7, -0.3, 0.2, 0.5
    r = dtn1 / dtn
    assert np.isclose(oracle.p_hat(q, q - dtn * s_, 1 + r, r), q + dtn1 * s_, rtol=1e-15)


def test_min_density():
    rho = np.array([[[3.0, 2.5], [7.0, 4.0]]])
    assert oracle.min_density(rho) == 2.5


def test_periodic_rejects_stretched_z():
    with pytest.raises(ValueError):
        oracle.make_grid(4, 4, 4, 0.25, 0.25, synth.stretched_dzf(4, 1.0, 1.5), "periodic")
