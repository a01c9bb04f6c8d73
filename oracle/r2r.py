"""Poisson solve with homogeneous Neumann/Dirichlet ends in x and y (oracle; test infrastructure only).

Sec. 3.3.1: the eigen-expansion along x and y works for any combination of homogeneous
boundary conditions, with cosine/sine series computed by FFTs plus pre/post-processing (the
Makhoul construction the paper cites for the GPU).  This module states the solve with those
series taken from a library (scipy.fft dct/dst, FFTW's REDFT/RODFT kinds), in the paper's step
order: forward along x, forward along y, the z solve, backward along y, backward along x.

Boundary conditions per direction x, y: 'P' periodic, or two letters for the low end (face
-1/2) and the high end (face n-1/2), each 'N' (homogeneous Neumann, ghost cell p_{-1} = p_0)
or 'D' (homogeneous Dirichlet on the boundary face, ghost p_{-1} = -p_0).  z is periodic or
walls (Neumann) as in oracle/projection.py.

Readings (E1-E4):
  E1  Cell-centred p with the boundary on the outer cell faces, so the ghost rules above give
      the eigenvectors cos(pi k (2i+1)/(2n)) (NN), sin(pi (k+1)(2i+1)/(2n)) (DD),
      cos(pi (2k+1)(2i+1)/(4n)) (ND) and sin(pi (2k+1)(2i+1)/(4n)) (DN): the DCT-II, DST-II,
      DCT-IV and DST-IV kinds.
  E2  Eigenvalues of the 3-point operator: -4 sin^2(pi k/(2n))/h^2 (NN), -4 sin^2(pi (k+1)/(2n))/h^2
      (DD), -4 sin^2(pi (2k+1)/(4n))/h^2 (ND, DN).
  E3  The operator is singular only when no end is Dirichlet (x, y each 'P' or 'NN', z periodic
      or walls); then R3/R4 of oracle/projection.py apply (mean of f removed, zero-mean p).
      Otherwise the solve is plain: f is used as given and p is unique.
  E4  Only the Poisson solve (and its residual) takes these ends; the projection stencils of
      oracle/projection.py stay periodic in x and y.
"""

import numpy as np
import scipy.fft as sfft

from . import projection as P

KINDS = ("P", "NN", "DD", "ND", "DN")


def _check(bc):
    if bc not in KINDS:
        raise ValueError(f"x/y boundary must be one of {KINDS}")


def ghost_signs(bc):
    """(s_lo, s_hi): ghost = s * adjacent interior value (+1 Neumann, -1 Dirichlet)."""
    return (1.0 if bc[0] == "N" else -1.0), (1.0 if bc[1] == "N" else -1.0)


def second_difference(p, bc, h, axis):
    """(p_{i-1} - 2 p_i + p_{i+1}) / h^2 along `axis` with periodic wrap or the ghost rules."""
    if bc == "P":
        return (np.roll(p, 1, axis=axis) - 2.0 * p + np.roll(p, -1, axis=axis)) / (h * h)
    s_lo, s_hi = ghost_signs(bc)
    pm = np.roll(p, 1, axis=axis)
    pp = np.roll(p, -1, axis=axis)
    n = p.shape[axis]
    idx0 = [slice(None)] * 3
    idxn = [slice(None)] * 3
    idx0[axis] = 0
    idxn[axis] = n - 1
    pm[tuple(idx0)] = s_lo * p[tuple(idx0)]
    pp[tuple(idxn)] = s_hi * p[tuple(idxn)]
    return (pm - 2.0 * p + pp) / (h * h)


def lap(p, g, bcx, bcy):
    """The 7-point operator with the given x/y ends and g's z treatment."""
    _check(bcx)
    _check(bcy)
    zero = np.zeros_like(p)
    lz = P.div(zero, zero, P.grad(p, g)[2], g)               # the z part, periodic or walls
    return second_difference(p, bcx, g.dx, 2) + second_difference(p, bcy, g.dy, 1) + lz


def eigenvalues(n, h, bc):
    """Eigenvalues of the 3-point operator along one direction, in transform order (E2)."""
    k = np.arange(n)
    if bc == "P":
        return P.eigenvalues(n, h)
    if bc == "NN":
        return -4.0 * np.sin(np.pi * k / (2 * n)) ** 2 / (h * h)
    if bc == "DD":
        return -4.0 * np.sin(np.pi * (k + 1) / (2 * n)) ** 2 / (h * h)
    return -4.0 * np.sin(np.pi * (2 * k + 1) / (4 * n)) ** 2 / (h * h)


def forward(a, bc, axis, real_input):
    """Forward series along `axis`: real FFT (x, periodic), complex FFT (y, periodic) or the
    cosine/sine kind of E1 (real and imaginary parts transformed alike)."""
    if bc == "P":
        return np.fft.rfft(a, axis=axis) if real_input else np.fft.fft(a, axis=axis)
    typ = 2 if bc in ("NN", "DD") else 4
    return (sfft.dct if bc[0] == "N" else sfft.dst)(a, type=typ, axis=axis)


def backward(a, bc, axis, n, real_output):
    if bc == "P":
        return np.fft.irfft(a, n=n, axis=axis) if real_output else np.fft.ifft(a, axis=axis)
    typ = 2 if bc in ("NN", "DD") else 4
    return (sfft.idct if bc[0] == "N" else sfft.idst)(a, type=typ, axis=axis)


def singular(g, bcx, bcy):
    """No Dirichlet end anywhere (E3)."""
    return bcx in ("P", "NN") and bcy in ("P", "NN")


def solve(f, g, bcx, bcy):
    """p with L p = f (minus <f>_V and with <p>_V = 0 when L is singular), eigen-expansion."""
    _check(bcx)
    _check(bcy)
    sing = singular(g, bcx, bcy)
    if sing:
        f = f - P.volume_mean(f, g)
    F = forward(f, bcx, 2, True)                               # forward along x
    F = forward(F, bcy, 1, False)                              # forward along y
    lx = eigenvalues(g.nx, g.dx, bcx)
    if bcx == "P":
        lx = lx[: g.nx // 2 + 1]
    ly = eigenvalues(g.ny, g.dy, bcy)
    lam_xy = ly[:, None] + lx[None, :]
    if g.bc == "periodic":
        F = np.fft.fft(F, axis=0)
        lam = P.eigenvalues(g.nz, g.dzf[0])[:, None, None] + lam_xy[None]
        if sing:
            lam[0, 0, 0] = 1.0
        Pk = F / lam
        if sing:
            Pk[0, 0, 0] = 0.0
        Pk = np.fft.ifft(Pk, axis=0)
    elif sing:
        Pk = P.tridiag_z(F, lam_xy, g)                         # (0, 0) column by R4
    else:
        Pk = thomas_z(F, lam_xy, g)
    Pk = backward(Pk, bcy, 1, g.ny, False)                     # backward along y
    if bcx != "P":
        Pk = np.real(Pk)                                       # the x coefficients are real
    return backward(Pk, bcx, 2, g.nx, True)                    # backward along x


def thomas_z(F, lam_xy, g):
    """Gauss elimination along z for every column of a nonsingular system (no special column)."""
    nz = g.nz
    a, b, c = P.z_coefficients(g)
    cp = np.zeros((nz,) + lam_xy.shape)
    dp = np.zeros_like(F)
    m = b[0] + lam_xy
    cp[0] = c[0] / m
    dp[0] = F[0] / m
    for k in range(1, nz):
        m = (b[k] + lam_xy) - a[k] * cp[k - 1]
        cp[k] = c[k] / m
        dp[k] = (F[k] - a[k] * dp[k - 1]) / m
    X = np.empty_like(F)
    X[nz - 1] = dp[nz - 1]
    for k in range(nz - 2, -1, -1):
        X[k] = dp[k] - cp[k] * X[k + 1]
    return X


def rel_residual(f, p, g, bcx, bcy):
    """||f' - L p|| / ||f'||, f' = f - <f>_V when L is singular, else f."""
    fm = f - P.volume_mean(f, g) if singular(g, bcx, bcy) else f
    return float(np.linalg.norm(fm - lap(p, g, bcx, bcy)) / np.linalg.norm(fm))
