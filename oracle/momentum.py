"""Oracle of the momentum predictor (test infrastructure only), FP64, triply periodic MAC grid.

Sec. 3.3, Eq. uss_predic: u** = u^n + dt (f1 M^n - f2 M^{n-1}) + dt g, with the second-order
Adams-Bashforth coefficients f1 = 1 + dt/(2 dt_prev), f2 = dt/(2 dt_prev) (Eq. tmp uses the same
pair), and M = -div(u u) + nu lap(u): convection in divergence form and diffusion, both with
second-order central differences (single phase: constant density and viscosity, so the
surface-tension term vanishes and the buoyancy term is the constant g).

Readings (M1-M3):
  M1  u[k][j][i] sits on the x face i+1/2 of cell (i, j, k), v on the y face j+1/2, w on the z
      face k+1/2 (the layout of the projection).  Products are formed from two-point averages:
      (u u) at cell centres from the averages of the two x faces, (u v) at the (i+1/2, j+1/2)
      edge from u averaged in y and v averaged in x, and likewise for (u w) and (v w).
  M2  The first step (no M^{n-1}) is forward Euler: f1 = 1, f2 = 0 (dt_prev <= 0).
  M3  Only triply periodic grids with uniform spacing in each direction are covered.
  M4  With constant viscosity mu and density rho (single phase), the viscous term of Eq. mom_con,
      div[mu (grad u + grad u^T)] / rho, is taken as nu lap(u), nu = mu / rho: the transposed part
      is nu grad(div u), which vanishes for the discretely solenoidal u^n that the projection
      returns (the MAC difference operators commute).
"""

import numpy as np


def sh(a, d, axis):
    """a shifted so that sh(a, +1, axis)[i] = a[i + 1] (periodic)."""
    return np.roll(a, -d, axis=axis)


AX = {"x": 2, "y": 1, "z": 0}


def convection(u, v, w, dx, dy, dz):
    """-div(u u) for the three velocity components (divergence form, central)."""
    X, Y, Z = AX["x"], AX["y"], AX["z"]
    # centres: averages of the two faces of each cell in the component's own direction
    uc = 0.5 * (sh(u, -1, X) + u)          # u at cell centre i (faces i-1/2, i+1/2)
    vc = 0.5 * (sh(v, -1, Y) + v)
    wc = 0.5 * (sh(w, -1, Z) + w)
    # edges
    u_y = 0.5 * (u + sh(u, 1, Y))          # u at (i+1/2, j+1/2)
    v_x = 0.5 * (v + sh(v, 1, X))          # v at (i+1/2, j+1/2)
    u_z = 0.5 * (u + sh(u, 1, Z))          # u at (i+1/2, k+1/2)
    w_x = 0.5 * (w + sh(w, 1, X))          # w at (i+1/2, k+1/2)
    v_z = 0.5 * (v + sh(v, 1, Z))          # v at (j+1/2, k+1/2)
    w_y = 0.5 * (w + sh(w, 1, Y))          # w at (j+1/2, k+1/2)
    uu, vv, ww = uc * uc, vc * vc, wc * wc
    uv, uw, vw = u_y * v_x, u_z * w_x, v_z * w_y
    cu = -((sh(uu, 1, X) - uu) / dx + (uv - sh(uv, -1, Y)) / dy + (uw - sh(uw, -1, Z)) / dz)
    cv = -((uv - sh(uv, -1, X)) / dx + (sh(vv, 1, Y) - vv) / dy + (vw - sh(vw, -1, Z)) / dz)
    cw = -((uw - sh(uw, -1, X)) / dx + (vw - sh(vw, -1, Y)) / dy + (sh(ww, 1, Z) - ww) / dz)
    return cu, cv, cw


def laplacian(a, dx, dy, dz):
    X, Y, Z = AX["x"], AX["y"], AX["z"]
    return ((sh(a, 1, X) - 2 * a + sh(a, -1, X)) / dx ** 2 + (sh(a, 1, Y) - 2 * a + sh(a, -1, Y)) / dy ** 2
            + (sh(a, 1, Z) - 2 * a + sh(a, -1, Z)) / dz ** 2)


def rhs(u, v, w, nu, dx, dy, dz):
    """M = -div(u u) + nu lap(u), per component."""
    cu, cv, cw = convection(u, v, w, dx, dy, dz)
    return (cu + nu * laplacian(u, dx, dy, dz), cv + nu * laplacian(v, dx, dy, dz),
            cw + nu * laplacian(w, dx, dy, dz))


def ab2_coefficients(dt, dt_prev):
    if dt_prev is None or dt_prev <= 0.0:
        return 1.0, 0.0
    r = dt / dt_prev
    return 1.0 + 0.5 * r, 0.5 * r


def predictor(u, v, w, m_prev, nu, g, dt, dt_prev, dx, dy, dz):
    """(u**, v**, w**), M^n for the velocity u^n, the previous M (or None) and gravity g."""
    m = rhs(u, v, w, nu, dx, dy, dz)
    f1, f2 = ab2_coefficients(dt, dt_prev if m_prev is not None else None)
    out = []
    for a, mn, q, gq in zip((u, v, w), m, m_prev if m_prev is not None else (0.0, 0.0, 0.0), g):
        out.append(a + dt * (f1 * mn - f2 * q) + dt * gq)
    return tuple(out), m


def taylor_green(nx, ny, nz, t=0.0, nu=0.0, L=2 * np.pi):
    """2-D Taylor-Green vortex on the MAC grid of an L-periodic box (uniform in z):
    u = sin x cos y e^{-2 nu t}, v = -cos x sin y e^{-2 nu t}, w = 0."""
    dx, dy = L / nx, L / ny
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dy
    xf, yf = xc + 0.5 * dx, yc + 0.5 * dy
    d = np.exp(-2.0 * nu * t)
    u = np.broadcast_to(np.sin(xf)[None, None, :] * np.cos(yc)[None, :, None] * d, (nz, ny, nx)).copy()
    v = np.broadcast_to(-np.cos(xc)[None, None, :] * np.sin(yf)[None, :, None] * d, (nz, ny, nx)).copy()
    w = np.zeros((nz, ny, nx))
    return u, v, w
