"""Plain FP64 statement of the FluTAS projection step (oracle; test infrastructure only).

Paper: Crialesi-Esposito et al., "FluTAS: A GPU-accelerated finite difference code for
multiphase flows", arXiv 2204.08834.

What is followed, and where:
  * MAC grid, cell-centred scalars, face-centred velocities ............ Sec. 3 (opening)
  * one-fluid density, rho_0 = min rho, extrapolated p_hat ............. Eq. material_prop; Sec. 3.3
  * split right-hand side, correction and pressure update ............. Sec. 3.3, Eqs. us_predic,
                                                                          poisson, corr, p_upt
  * Poisson solve: Fourier along x and y, Gauss elimination along z,
    step order forward-x, forward-y, z-solve, backward-y, backward-x ... Sec. 3.3.1 (nine-step list)
  * a third Fourier expansion along z when z is periodic .............. Sec. 3.3 (eigen-expansion
                                                                          for any homogeneous BCs)

Readings of the paper taken here (the paper is silent or garbled on these):
  R1  Eq. us_predic prints "(1 - rho0/rho grad p_hat)"; the splitting term is read as
      u* = u** - dt[(1/rho - 1/rho0) grad p_hat + grad p^n / rho0], which after substituting
      p^{n+1} = p^n + psi gives the non-incremental form solved here:
          L p = (rho0/dt) D u** + D[(1 - rho0/rho_f) G p_hat],
          u^{n+1} = u** - (dt/rho0) [G p - (1 - rho0/rho_f) G p_hat].
      (The arguments called u, v, w below are the paper's u**.)
  R2  Face density rho_f is the arithmetic mean of the two adjacent cell densities.
  R3  p is defined up to a constant; the solve returns the solution with zero
      volume-weighted mean, after removing the volume-weighted mean of f.
  R4  For z walls the (kx, ky) = (0, 0) tridiagonal system is singular: row 0 is dropped,
      P_0 is pinned to 0, and the column is shifted to zero volume-weighted mean.
  R5  z walls: homogeneous Neumann for p (G_z = 0 on both wall faces), w = 0 on both wall
      faces; w[k] sits on the top face of cell k, so w[nz-1] is the top wall face.
  R6  Stretched z: cell-centre spacing dzc_k = (dzf_k + dzf_{k+1}) / 2.
  R7  Forward transform sign exp(-2 pi i k n / N); 1/N on the inverse (no effect on p).

Layout: every field is a C-contiguous float64 array of shape (nz, ny, nx), x fastest.
u[k, j, i] lives on the x-face i+1/2, v[k, j, i] on the y-face j+1/2, w[k, j, i] on the
z-face k+1/2.  x and y are always periodic; z is 'periodic' (uniform dz) or 'walls'.
"""

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dzf: np.ndarray  # (nz,) cell widths along z
    dzc: np.ndarray  # (nz,) centre-to-centre spacing k -> k+1 (last entry unused with walls)
    bc: str          # 'periodic' or 'walls' (z only)


def make_grid(nx, ny, nz, dx, dy, dzf, bc):
    """Build the grid; dzf may be a scalar (uniform) or an array of nz widths (R6)."""
    if bc not in ("periodic", "walls"):
        raise ValueError("bc must be 'periodic' or 'walls'")
    dzf = np.broadcast_to(np.asarray(dzf, dtype=np.float64), (nz,)).copy()
    if bc == "periodic" and not np.all(dzf == dzf[0]):
        raise ValueError("a periodic z direction needs uniform dz")
    dzc = np.empty(nz)
    dzc[:-1] = 0.5 * (dzf[:-1] + dzf[1:])
    dzc[-1] = 0.5 * (dzf[-1] + dzf[0]) if bc == "periodic" else np.nan
    return Grid(nx, ny, nz, float(dx), float(dy), dzf, dzc, bc)


# ---------------------------------------------------------------- MAC operators (Sec. 3)

def grad(p, g):
    """Face gradients (G_x p, G_y p, G_z p); G_z = 0 on the top wall face (R5)."""
    gx = (np.roll(p, -1, axis=2) - p) / g.dx
    gy = (np.roll(p, -1, axis=1) - p) / g.dy
    if g.bc == "periodic":
        gz = (np.roll(p, -1, axis=0) - p) / g.dzc[:, None, None]
    else:
        gz = np.zeros_like(p)
        gz[:-1] = (p[1:] - p[:-1]) / g.dzc[:-1, None, None]
    return gx, gy, gz


def div(u, v, w, g):
    """Cell divergence D(u, v, w); with walls both wall-face w values are taken as 0 (R5)."""
    d = (u - np.roll(u, 1, axis=2)) / g.dx + (v - np.roll(v, 1, axis=1)) / g.dy
    if g.bc == "periodic":
        dz = w - np.roll(w, 1, axis=0)
    else:
        wt = w.copy()
        wt[-1] = 0.0
        wb = np.zeros_like(w)
        wb[1:] = wt[:-1]
        dz = wt - wb
    return d + dz / g.dzf[:, None, None]


def lap(p, g):
    """L p = D G p, the 7-point operator the direct solver inverts."""
    return div(*grad(p, g), g)


# ------------------------------------------------------- density terms (Sec. 3.3, R2)

def min_density(rho):
    """rho_0: the minimum density in the domain (Sec. 3.3)."""
    return float(np.min(rho))


def face_density(rho, g):
    """Arithmetic-mean face densities (R2); the top wall face copies the cell value (unused)."""
    rx = 0.5 * (rho + np.roll(rho, -1, axis=2))
    ry = 0.5 * (rho + np.roll(rho, -1, axis=1))
    if g.bc == "periodic":
        rz = 0.5 * (rho + np.roll(rho, -1, axis=0))
    else:
        rz = rho.copy()
        rz[:-1] = 0.5 * (rho[:-1] + rho[1:])
    return rx, ry, rz


def p_hat(pn, pnm1, c1, c2):
    """Extrapolated pressure p_hat = c1 p^n - c2 p^{n-1} (Sec. 3.3: c1 = 1 + r, c2 = r)."""
    return c1 * pn - c2 * pnm1


def rhs(u, v, w, rho, pn, pnm1, c1, c2, dt, g, rho0=None):
    """f = (rho0/dt) D u** + D[(1 - rho0/rho_f) G p_hat]   (Eqs. us_predic + poisson, R1)."""
    if rho0 is None:
        rho0 = min_density(rho)
    ph = p_hat(pn, pnm1, c1, c2)
    hx, hy, hz = grad(ph, g)
    rx, ry, rz = face_density(rho, g)
    split = div((1.0 - rho0 / rx) * hx, (1.0 - rho0 / ry) * hy, (1.0 - rho0 / rz) * hz, g)
    return (rho0 / dt) * div(u, v, w, g) + split


def volume_mean(a, g):
    """Volume-weighted mean <a>_V = sum(a dzf) / (nx ny sum dzf)  (R3)."""
    return float(np.sum(a * g.dzf[:, None, None]) / (g.nx * g.ny * np.sum(g.dzf)))


# ------------------------------------------------------------ Poisson solve (Sec. 3.3.1)

def eigenvalues(n, h):
    """Eigenvalues (2 cos(2 pi k / n) - 2) / h^2, k = 0..n-1, of the periodic 3-point operator."""
    k = np.arange(n)
    return (2.0 * np.cos(2.0 * np.pi * k / n) - 2.0) / (h * h)


def z_coefficients(g):
    """Sub-, main- and super-diagonals (a_k, b_k, c_k) of the z part of L with walls (R5, R6)."""
    nz = g.nz
    a = np.zeros(nz)
    c = np.zeros(nz)
    a[1:] = 1.0 / (g.dzf[1:] * g.dzc[:-1])
    c[:-1] = 1.0 / (g.dzf[:-1] * g.dzc[:-1])
    return a, -(a + c), c


def tridiag_z(F, lam_xy, g):
    """Gauss elimination (Thomas) along z for every (ky, kx) column (Sec. 3.3.1, step 5).

    Column (ky, kx) solves a_k P_{k-1} + (b_k + lam_xy) P_k + c_k P_{k+1} = F_k.
    The singular (0, 0) column follows R4.
    """
    nz = g.nz
    a, b, c = z_coefficients(g)
    lam = lam_xy.copy()
    lam[0, 0] = -1.0  # placeholder so the vectorised sweep stays finite; column redone below
    cp = np.zeros((nz,) + lam.shape)
    dp = np.zeros_like(F)
    m = b[0] + lam
    cp[0] = c[0] / m
    dp[0] = F[0] / m
    for k in range(1, nz):
        m = (b[k] + lam) - a[k] * cp[k - 1]
        cp[k] = c[k] / m
        dp[k] = (F[k] - a[k] * dp[k - 1]) / m
    P = np.empty_like(F)
    P[nz - 1] = dp[nz - 1]
    for k in range(nz - 2, -1, -1):
        P[k] = dp[k] - cp[k] * P[k + 1]

    # (kx, ky) = (0, 0): P_0 = 0, rows 1..nz-1, then zero volume-weighted mean (R4).
    f00 = F[:, 0, 0]
    q = np.zeros(nz, dtype=F.dtype)
    if nz > 1:
        cs = np.zeros(nz)
        ds = np.zeros(nz, dtype=F.dtype)
        cs[1] = c[1] / b[1]
        ds[1] = f00[1] / b[1]
        for k in range(2, nz):
            m = b[k] - a[k] * cs[k - 1]
            cs[k] = c[k] / m
            ds[k] = (f00[k] - a[k] * ds[k - 1]) / m
        q[nz - 1] = ds[nz - 1]
        for k in range(nz - 2, 0, -1):
            q[k] = ds[k] - cs[k] * q[k + 1]
    q -= np.sum(q * g.dzf) / np.sum(g.dzf)
    P[:, 0, 0] = q
    return P


def _library_transforms(workers):
    """The FFT routines the solve calls: numpy's (one thread), or with `workers` scipy.fft's
    on that many host threads (the batched 1-D transforms split over threads; used only to
    time the oracle on all cores)."""
    if workers is None:
        return np.fft.rfft, np.fft.fft, np.fft.ifft, np.fft.irfft
    import scipy.fft as sfft

    return (lambda a, axis: sfft.rfft(a, axis=axis, workers=workers),
            lambda a, axis: sfft.fft(a, axis=axis, workers=workers),
            lambda a, axis: sfft.ifft(a, axis=axis, workers=workers),
            lambda a, n, axis: sfft.irfft(a, n=n, axis=axis, workers=workers))


def solve(f, g, workers=None):
    """p with L p = f - <f>_V and <p>_V = 0, by the eigen-expansion direct method (Sec. 3.3.1).

    Steps in the paper's order: forward transform along x, forward along y, the z solve
    (Gauss elimination with walls, a third transform when z is periodic), backward
    along y, backward along x.  `workers` (timing only) runs the transforms on that many
    host threads.
    """
    rfft, fft, ifft, irfft = _library_transforms(workers)
    f = f - volume_mean(f, g)
    F = rfft(f, axis=2)                               # step 1: forward along x (kx = 0..nx/2)
    F = fft(F, axis=1)                                # step 3: forward along y
    lx = eigenvalues(g.nx, g.dx)[: g.nx // 2 + 1]
    ly = eigenvalues(g.ny, g.dy)
    lam_xy = ly[:, None] + lx[None, :]
    if g.bc == "periodic":
        F = fft(F, axis=0)                            # z transform (periodic z)
        lam = eigenvalues(g.nz, g.dzf[0])[:, None, None] + lam_xy[None]
        lam[0, 0, 0] = 1.0
        P = F / lam
        P[0, 0, 0] = 0.0                              # zero mean (R3)
        P = ifft(P, axis=0)
    else:
        P = tridiag_z(F, lam_xy, g)                   # step 5: Gauss elimination along z
    P = ifft(P, axis=1)                               # step 7: backward along y
    return irfft(P, n=g.nx, axis=2)                   # step 9: backward along x


# ---------------------------------------------------------- correction (Sec. 3.3, R1)

def correct(u, v, w, p, pn, pnm1, rho, c1, c2, dt, g, rho0=None):
    """u^{n+1} = u** - (dt/rho0)[G p - (1 - rho0/rho_f) G p_hat]  (Eqs. us_predic + corr, R1).

    With walls the top wall face gets w = 0 (R5).
    """
    if rho0 is None:
        rho0 = min_density(rho)
    ph = p_hat(pn, pnm1, c1, c2)
    gx, gy, gz = grad(p, g)
    hx, hy, hz = grad(ph, g)
    rx, ry, rz = face_density(rho, g)
    s = dt / rho0
    u1 = u - s * (gx - (1.0 - rho0 / rx) * hx)
    v1 = v - s * (gy - (1.0 - rho0 / ry) * hy)
    w1 = w - s * (gz - (1.0 - rho0 / rz) * hz)
    if g.bc == "walls":
        w1[-1] = 0.0
    return u1, v1, w1


def project(u, v, w, rho, pn, pnm1, c1, c2, dt, g):
    """One projection: rhs, solve, correct.  Returns (f, p, u1, v1, w1)."""
    rho0 = min_density(rho)
    f = rhs(u, v, w, rho, pn, pnm1, c1, c2, dt, g, rho0)
    p = solve(f, g)
    u1, v1, w1 = correct(u, v, w, p, pn, pnm1, rho, c1, c2, dt, g, rho0)
    return f, p, u1, v1, w1


# ------------------------------------------------------------------------ norms

def residual(f, p, g):
    """r = (f - <f>_V) - L p."""
    return (f - volume_mean(f, g)) - lap(p, g)


def rel_residual(f, p, g):
    """||f - <f>_V - L p||_2 / ||f - <f>_V||_2."""
    fm = f - volume_mean(f, g)
    return float(np.linalg.norm(residual(f, p, g)) / np.linalg.norm(fm))


def div_rel(u1, v1, w1, u, v, w, g):
    """max |D u^{n+1}| * h_min / max |u**|, the relative discrete divergence."""
    h = min(g.dx, g.dy, float(np.min(g.dzf)))
    umax = max(np.max(np.abs(u)), np.max(np.abs(v)), np.max(np.abs(w)))
    return float(np.max(np.abs(div(u1, v1, w1, g))) * h / umax)
