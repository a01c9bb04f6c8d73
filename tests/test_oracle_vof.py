"""Pins of the VoF oracle (MTHINC reconstruction and split advection, Sec. 3.1 and App. A)
against mathematics, not against the oracle itself.

  * the exact line integral (App. A.1.2, log cosh antiderivative) against a 64-point
    Gauss-Legendre quadrature of tanh;
  * d_th against the paper's quartic in D = exp(2 beta d_th) (coefficients from the elementary
    symmetric polynomials, reading V5): D is a root, and the only positive one;
  * a plane through the cell centre at phi = 1/2 has T(centre) + d_th = 0;
  * the complement 1 - phi reconstructs with n -> -n and d_th -> -d_th;
  * Youngs' gradient of a linear field is exact (cell units) and its curvature tensor zero;
  * the curvature of a sphere of radius R cells is 2/R (sign of reading V2);
  * the split step conserves sum(phi) to rounding for any velocity (divergence correction,
    Eq. vof_corr_step), leaves phi unchanged at zero velocity and keeps phi = 1 under a
    solenoidal velocity;
  * at CFL 1 in every direction the step is an exact shift by one cell (each face carries the
    whole upwind cell, because d_th makes the cell integral of H equal phi).
"""

import numpy as np
import pytest

from oracle import vof


def sphere_phi(n, centre, radius, width=0.75):
    x = np.arange(n) + 0.5
    r = np.sqrt((x[None, None, :] - centre[0]) ** 2 + (x[None, :, None] - centre[1]) ** 2
                + (x[:, None, None] - centre[2]) ** 2)
    return 0.5 * (1.0 - np.tanh((r - radius) / width))


def test_line_integral_matches_quadrature():
    rng = np.random.default_rng(1)
    xg, wg = np.polynomial.legendre.leggauss(64)
    for _ in range(50):
        a = rng.uniform(0.58, 1.0) * rng.choice([-1, 1])
        g, d, beta = rng.uniform(-2, 2), rng.uniform(-3, 3), rng.uniform(0.5, 4.0)
        s0, s1 = sorted(rng.uniform(0, 1, 2))
        s = 0.5 * (s1 - s0) * xg + 0.5 * (s1 + s0)
        ref = 0.5 * (s1 - s0) * np.sum(wg * 0.5 * (1 + np.tanh(beta * (a * s + g + d))))
        assert abs(vof.line_integral(a, g, d, beta, s0, s1) - ref) <= 1e-13


@pytest.mark.parametrize("beta", [1.0, 2.0, 3.0])
def test_dth_is_the_positive_root_of_the_quartic(beta):
    phi = sphere_phi(20, (10.2, 9.7, 10.4), 5.3)
    rec = vof.reconstruct(phi, beta)
    live = ~rec["uniform"] & (phi > 1e-4) & (phi < 1 - 1e-4)
    al = vof.quartic_coefficients(rec, beta)
    D = np.exp(2.0 * beta * rec["d"])
    val = sum(al[k] * D ** k for k in range(5))
    scale = sum(np.abs(al[k] * D ** k) for k in range(5))
    assert np.max(np.abs(val / scale)[live]) <= 1e-10
    # the only positive root: the sign of the quartic changes at D and nowhere else on a grid
    cells = np.argwhere(live)[:40]
    for c in map(tuple, cells):
        coef = [al[k][c] for k in range(4, -1, -1)]
        roots = np.roots(coef)
        pos = [z.real for z in roots if abs(z.imag) <= 1e-8 * abs(z) and z.real > 0]
        assert len(pos) == 1 and abs(pos[0] - D[c]) <= 1e-6 * D[c], (c, pos, D[c])


def test_plane_through_the_centre():
    """phi = 1/2 cut by a plane through the cell centre: by symmetry T(1/2,1/2,1/2) + d = 0."""
    n = 16
    x = np.arange(n) + 0.5
    nrm = np.array([0.6, 0.48, 0.64])
    nrm /= np.linalg.norm(nrm)
    s = (nrm[0] * (x[None, None, :] - 8.5) + nrm[1] * (x[None, :, None] - 8.5) + nrm[2] * (x[:, None, None] - 8.5))
    phi = 0.5 * (1 + np.tanh(0.5 * s))      # a function of the distance to the plane only
    rec = vof.reconstruct(phi, 2.0)
    c = (8, 8, 8)
    assert abs(phi[c] - 0.5) <= 1e-15
    t = vof.t_value(rec["q"], rec["r"], rec["L"], (0.5, 0.5, 0.5))
    assert abs(t[c] + rec["d"][c]) <= 1e-12
    assert np.allclose([rec["n"][a][c] for a in range(3)], nrm, atol=5e-3)   # Youngs, O(h^2) off


def test_complement_flips_normal_and_dth():
    phi = sphere_phi(16, (8.3, 7.9, 8.1), 4.2)
    a = vof.reconstruct(phi, 2.0)
    b = vof.reconstruct(1.0 - phi, 2.0)
    live = ~a["uniform"]
    for k in range(3):
        assert np.max(np.abs(a["n"][k] + b["n"][k])[live]) <= 1e-9
    # cells whose two largest normal components tie to rounding may pick another case (V7);
    # near phi = 0 or 1 the complement 1 - phi itself carries eps / phi of relative rounding
    same = live & (a["p"] == b["p"]) & (phi > 1e-4) & (phi < 1 - 1e-4)
    assert same.sum() >= 1000
    assert np.max(np.abs(a["d"] + b["d"])[same]) <= 1e-10


def test_youngs_linear_field_is_exact():
    n = 12
    x = np.arange(n, dtype=float)
    phi = 0.3 * x[None, None, :] - 0.2 * x[None, :, None] + 0.7 * x[:, None, None]
    m, nn, K = vof.youngs(phi)
    inner = (slice(2, -2),) * 3        # away from the periodic wrap
    for a, g in enumerate((0.3, -0.2, 0.7)):
        assert np.max(np.abs(m[a][inner] - g)) <= 1e-14
    for v in K.values():
        assert np.max(np.abs(v[inner])) <= 1e-14


def test_sphere_curvature():
    R = 8.0
    phi = sphere_phi(32, (16.1, 15.8, 16.3), R)
    kap = vof.curvature(phi)
    band = (phi > 0.3) & (phi < 0.7)
    assert abs(np.mean(kap[band]) * R / 2.0 - 1.0) <= 0.03


def random_velocity(shape, seed, cfl, h=1.0, dt=1.0):
    r = np.random.default_rng(seed)
    return [r.uniform(-cfl, cfl, shape) * h / dt for _ in range(3)]


def test_mass_conservation_any_velocity():
    phi = sphere_phi(16, (8.2, 7.7, 8.4), 4.5)
    u, v, w = random_velocity(phi.shape, 3, 0.45)
    out, _ = vof.vof_step(phi, u, v, w, 1.0, 2.0, 1.0, 1.0, 1.0)
    assert abs(out.sum() - phi.sum()) <= 1e-13 * phi.sum()


def test_zero_velocity_and_uniform_field():
    phi = sphere_phi(12, (6.2, 5.7, 6.4), 3.5)
    z = np.zeros_like(phi)
    out, _ = vof.vof_step(phi, z, z, z, 1.0, 2.0, 1.0, 1.0, 1.0)
    assert np.array_equal(out, phi)
    # phi = 1 under a discretely solenoidal velocity (curl of a random potential)
    r = np.random.default_rng(4)
    A = [r.standard_normal(phi.shape) for _ in range(3)]
    sh = vof.sh
    # A_x on the (j+1/2, k+1/2) edges, A_y on (i+1/2, k+1/2), A_z on (i+1/2, j+1/2): backward
    # differences of the edge values give face velocities with zero MAC divergence
    u = (A[2] - sh(A[2], -1, 1)) - (A[1] - sh(A[1], -1, 2))
    v = (A[0] - sh(A[0], -1, 2)) - (A[2] - sh(A[2], -1, 0))
    w = (A[1] - sh(A[1], -1, 0)) - (A[0] - sh(A[0], -1, 1))
    div = (u - sh(u, -1, 0)) + (v - sh(v, -1, 1)) + (w - sh(w, -1, 2))
    assert np.max(np.abs(div)) <= 1e-13
    s = 0.4 / max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    one = np.ones_like(phi)
    out, _ = vof.vof_step(one, s * u, s * v, s * w, 1.0, 2.0, 1.0, 1.0, 1.0)
    assert np.max(np.abs(out - 1.0)) <= 1e-14


@pytest.mark.parametrize("signs", [(1, 1, 1), (-1, 1, -1)])
def test_cfl_one_is_an_exact_shift(signs):
    phi = sphere_phi(12, (6.3, 5.6, 6.2), 3.4)
    one = np.ones_like(phi)
    vel = [s * one for s in signs]
    out, _ = vof.vof_step(phi, *vel, 1.0, 2.0, 1.0, 1.0, 1.0)
    ref = phi
    for a, s in enumerate(signs):
        ref = np.roll(ref, s, axis=vof.axis(a))
    assert np.max(np.abs(out - ref)) <= 1e-14


def test_polynomial_has_the_imposed_gradient_and_hessian():
    """Eq. constrain: grad T = n and grad grad T = K at the cell centre on the kept terms (V3);
    every second derivative involving the exact direction p is zero (T linear along p)."""
    phi = sphere_phi(16, (8.3, 7.9, 8.1), 4.2)
    rec = vof.reconstruct(phi, 2.0)
    live = ~rec["uniform"]
    q, r, L = rec["q"], rec["r"], rec["L"]
    h = 1e-4

    def T(dx):
        return vof.t_value(q, r, L, tuple(0.5 + dx[a] for a in range(3)))

    e = np.eye(3) * h
    for a in range(3):
        grad = (T(e[a]) - T(-e[a])) / (2 * h)
        assert np.max(np.abs(grad - rec["n"][a])[live]) <= 1e-9
        for b in range(3):
            hess = (T(e[a] + e[b]) - T(e[a] - e[b]) - T(-e[a] + e[b]) + T(-e[a] - e[b])) / (4 * h * h)
            kab = rec["K"][(min(a, b), max(a, b))]
            kept = (rec["p"] != a) & (rec["p"] != b)
            ref = np.where(kept, kab, 0.0)
            assert np.max(np.abs(hess - ref)[live]) <= 1e-5, (a, b)


def test_quadrature_in_the_small_beta_limit():
    """For beta -> 0, H = 1/2 + beta (T + d)/2 + O(beta^3): the box quadrature (exact along p,
    two-point Gauss-Legendre elsewhere, exact for cubics) must give 1/2 + beta/2 times the exact
    integral of T + d over the box (T quadratic; closed-form moments of a box)."""
    rng = np.random.default_rng(5)
    shape = (4, 4, 4)
    # beta = 1e-3: the tanh truncation is (beta T)^2 / 3 ~ 1e-6 relative and the rounding of the
    # log cosh difference ~ 1e-8; a wrong Gauss node errs by percents on the quadratic terms
    beta = 1e-3
    for p in range(3):
        K = {(a, b): rng.uniform(-0.5, 0.5, shape) for a in range(3) for b in range(a, 3)}
        nv = rng.standard_normal((3,) + shape)
        nv[p] = 3.0 + np.abs(nv[p])                  # p is the largest component
        nv /= np.linalg.norm(nv, axis=0)
        pp, q, r, L = vof.polynomial(list(nv), K)
        assert np.all(pp == p)
        lo = [rng.uniform(0, 0.4, shape) for _ in range(3)]
        hi = [lo[a] + rng.uniform(0.1, 0.6, shape) for a in range(3)]
        d = rng.uniform(-0.5, 0.5, shape)
        rec = {"p": pp, "q": q, "r": r, "L": L, "d": d}
        V = vof.box_integral(rec, lo, hi, beta)

        def mom(a, k):                               # integral of x_a^k over [lo_a, hi_a]
            return (hi[a] ** (k + 1) - lo[a] ** (k + 1)) / (k + 1)

        vol = mom(0, 0) * mom(1, 0) * mom(2, 0)
        IT = sum(q[a] * mom(a, 2) * vol / mom(a, 0) + L[a] * mom(a, 1) * vol / mom(a, 0) for a in range(3))
        for (a, b), v in r.items():
            c = [x for x in range(3) if x not in (a, b)][0]
            IT = IT + v * mom(a, 1) * mom(b, 1) * mom(c, 0)
        ref = 0.5 * vol + 0.5 * beta * (IT + d * vol)
        assert np.max(np.abs((V - ref) / (0.5 * beta * vol))) <= 1e-5, p
