"""Pins of the momentum-predictor oracle (Sec. 3.3, Eq. uss_predic) against closed forms and
invariants that do not come from the oracle itself."""

import itertools

import numpy as np
import pytest

from oracle import momentum as M
from oracle import projection as P

L = 2 * np.pi


def plane_taylor_green(n, a, b):
    """Taylor-Green vortex in the (a, b) plane of an L-periodic box with n = (nz, ny, nx) cells:
    q_a = sin(a) cos(b), q_b = -cos(a) sin(b), third component 0, each component sampled at its
    own face positions (face along its own axis, centres along the others)."""
    axis = {"x": 2, "y": 1, "z": 0}
    h = {k: L / n[axis[k]] for k in "xyz"}

    def coords(k, face):
        c = (np.arange(n[axis[k]]) + 0.5) * h[k]
        c = c + 0.5 * h[k] if face else c
        shape = [1, 1, 1]
        shape[axis[k]] = -1
        return c.reshape(shape)

    qa = np.sin(coords(a, True)) * np.cos(coords(b, False)) * np.ones(n)
    qb = -np.cos(coords(a, False)) * np.sin(coords(b, True)) * np.ones(n)
    comp = {a: qa, b: qb}
    zero = np.zeros(n)
    return [comp.get(k, zero) for k in "xyz"], h, coords


def closed_form_rhs(a, b, h, coords, nu):
    """M for the plane vortex, derived by hand from Eq. uss_predic's convection (divergence form,
    two-point averages) and diffusion (7-point Laplacian) on the MAC grid:
      M_a = -1/2 sin(2 a_f) [c_a^2 s_a (1 + cos 2 b_c) - c_a c_b s_b cos 2 b_c] - nu (lam_a + lam_b) q_a,
      M_b = -1/2 sin(2 b_f) [c_b^2 s_b (1 + cos 2 a_c) - c_a c_b s_a cos 2 a_c] - nu (lam_a + lam_b) q_b,
    with c = cos(h/2), s = sin(h)/h, lam = 4 sin^2(h/2)/h^2, a_f a face and a_c a centre coordinate."""
    ca, cb = np.cos(h[a] / 2), np.cos(h[b] / 2)
    sa, sb = np.sin(h[a]) / h[a], np.sin(h[b]) / h[b]
    lam = 4 * np.sin(h[a] / 2) ** 2 / h[a] ** 2 + 4 * np.sin(h[b] / 2) ** 2 / h[b] ** 2
    af, ac, bf, bc = coords(a, True), coords(a, False), coords(b, True), coords(b, False)
    qa = np.sin(af) * np.cos(bc)
    qb = -np.cos(ac) * np.sin(bf)
    ma = -0.5 * np.sin(2 * af) * (ca * ca * sa * (1 + np.cos(2 * bc)) - ca * cb * sb * np.cos(2 * bc)) - nu * lam * qa
    mb = -0.5 * np.sin(2 * bf) * (cb * cb * sb * (1 + np.cos(2 * ac)) - ca * cb * sa * np.cos(2 * ac)) - nu * lam * qb
    return ma, mb


@pytest.mark.parametrize("a,b", list(itertools.permutations("xyz", 2)))
def test_taylor_green_rhs_closed_form_every_plane(a, b):
    n = (8, 12, 16)                          # unequal spacings in the three directions
    (u, v, w), h, coords = plane_taylor_green(n, a, b)
    nu = 0.037
    m = dict(zip("xyz", M.rhs(u, v, w, nu, h["x"], h["y"], h["z"])))
    ma, mb = closed_form_rhs(a, b, h, coords, nu)
    third = ({"x", "y", "z"} - {a, b}).pop()
    assert np.max(np.abs(m[a] - ma)) < 1e-13
    assert np.max(np.abs(m[b] - mb)) < 1e-13
    assert np.max(np.abs(m[third])) < 1e-13


def test_laplacian_single_mode_eigenvalue():
    rng = np.random.default_rng(3)
    nz, ny, nx = 8, 16, 12
    hx, hy, hz = 0.3, 0.17, 0.41
    x = (np.arange(nx) + 0.5) * hx
    y = np.arange(ny) * hy
    z = (np.arange(nz) + 0.25) * hz
    for _ in range(4):
        kx, ky, kz = (2 * np.pi * rng.integers(0, n) / (n * h) for n, h in ((nx, hx), (ny, hy), (nz, hz)))
        px, py, pz = rng.uniform(0, 2 * np.pi, 3)
        a = (np.cos(kx * x + px)[None, None, :] * np.cos(ky * y + py)[None, :, None]
             * np.cos(kz * z + pz)[:, None, None])
        lam = sum(4 * np.sin(k * h / 2) ** 2 / h ** 2 for k, h in ((kx, hx), (ky, hy), (kz, hz)))
        assert np.max(np.abs(M.laplacian(a, hx, hy, hz) + lam * a)) < 1e-12 * max(lam, 1.0)


def solenoidal_field(rng, n, hx, hy, hz):
    """Discrete curl of a random edge-centred vector potential: discretely divergence-free."""
    def d(a, ax):
        return a - np.roll(a, 1, axis=ax)
    px, py, pz = (rng.standard_normal(n) for _ in range(3))
    u = d(pz, 1) / hy - d(py, 0) / hz
    v = d(px, 0) / hz - d(pz, 2) / hx
    w = d(py, 2) / hx - d(px, 1) / hy
    div = d(u, 2) / hx + d(v, 1) / hy + d(w, 0) / hz
    assert np.max(np.abs(div)) < 1e-12 * np.max(np.abs(u))
    return u, v, w


def test_convection_conserves_momentum_and_kinetic_energy():
    """The central divergence form on a staggered grid conserves momentum for any field and
    kinetic energy for a discretely divergence-free one (Morinishi et al., JCP 143, 1998)."""
    rng = np.random.default_rng(5)
    hx, hy, hz = 0.3, 0.2, 0.25
    u, v, w = solenoidal_field(rng, (8, 12, 16), hx, hy, hz)
    cu, cv, cw = M.convection(u, v, w, hx, hy, hz)
    scale = np.abs(cu).sum() + np.abs(cv).sum() + np.abs(cw).sum()
    for c in (cu, cv, cw):
        assert abs(c.sum()) < 1e-13 * scale
    e = (u * cu).sum() + (v * cv).sum() + (w * cw).sum()
    s = np.abs(u * cu).sum() + np.abs(v * cv).sum() + np.abs(w * cw).sum()
    assert abs(e) < 1e-14 * s
    # the same check fails on a field that is not solenoidal, so it has teeth
    u2, v2, w2 = (rng.standard_normal((8, 12, 16)) for _ in range(3))
    c2 = M.convection(u2, v2, w2, hx, hy, hz)
    e2 = sum((q * c).sum() for q, c in zip((u2, v2, w2), c2))
    s2 = sum(np.abs(q * c).sum() for q, c in zip((u2, v2, w2), c2))
    assert abs(e2) > 1e-3 * s2


def test_diffusion_dissipates():
    rng = np.random.default_rng(6)
    a = rng.standard_normal((8, 8, 8))
    assert (a * M.laplacian(a, 0.1, 0.2, 0.3)).sum() < 0


def test_uniform_flow_has_no_rhs_and_gravity_is_a_constant_acceleration():
    n = (4, 6, 8)
    u, v, w = (np.full(n, c) for c in (0.7, -1.3, 2.1))
    for m in M.rhs(u, v, w, 0.2, 0.1, 0.2, 0.3):
        assert np.max(np.abs(m)) < 1e-12
    g = (0.5, -9.81, 3.0)
    (us, vs, ws), _ = M.predictor(u, v, w, None, 0.2, g, 1e-2, 0.0, 0.1, 0.2, 0.3)
    for q, q0, gq in zip((us, vs, ws), (0.7, -1.3, 2.1), g):
        assert np.max(np.abs(q - (q0 + 1e-2 * gq))) < 1e-14


def test_ab2_coefficients_textbook_and_exact_for_linear_forcing():
    assert M.ab2_coefficients(0.1, 0.1) == (1.5, 0.5)
    assert M.ab2_coefficients(0.1, 0.0) == (1.0, 0.0)      # first step: forward Euler
    # variable steps: AB2 integrates a forcing linear in time exactly
    fa, fb = 0.7, -2.3
    for dt_prev, dt in ((0.1, 0.05), (0.03, 0.11), (0.2, 0.2)):
        t = 1.9
        f1, f2 = M.ab2_coefficients(dt, dt_prev)
        step = dt * (f1 * (fa + fb * t) - f2 * (fa + fb * (t - dt_prev)))
        exact = fa * dt + fb * ((t + dt) ** 2 - t ** 2) / 2
        assert abs(step - exact) < 1e-14 * abs(exact)


def test_predictor_uses_previous_rhs_with_ab2_weights():
    """With M^{n-1} = M^n the AB2 update reduces to one Euler step with M^n (f1 - f2 = 1)."""
    rng = np.random.default_rng(7)
    u, v, w = solenoidal_field(rng, (4, 8, 8), 0.25, 0.25, 0.25)
    m = M.rhs(u, v, w, 0.05, 0.25, 0.25, 0.25)
    (a, b, c), m2 = M.predictor(u, v, w, m, 0.05, (0, 0, 0), 0.013, 0.021, 0.25, 0.25, 0.25)
    (a0, b0, c0), _ = M.predictor(u, v, w, None, 0.05, (0, 0, 0), 0.013, 0.0, 0.25, 0.25, 0.25)
    for x, y in zip((a, b, c), (a0, b0, c0)):
        assert np.max(np.abs(x - y)) < 1e-14
    for x, y in zip(m, m2):
        assert np.array_equal(x, y)


def taylor_green_error(n, nu, t_end, cfl=0.25):
    """Run predictor + projection (constant density 1) on the 2-D vortex; max error against the
    closed-form decay u = sin x cos y exp(-2 nu t)."""
    h = L / n
    steps = int(np.ceil(t_end / (cfl * h)))
    dt = t_end / steps
    g = P.make_grid(n, n, 2, h, h, h, "periodic")
    u, v, w = M.taylor_green(n, n, 2)
    rho = np.ones_like(u)
    zero = np.zeros_like(u)
    m_prev = None
    for _ in range(steps):
        (us, vs, ws), m_prev = M.predictor(u, v, w, m_prev, nu, (0, 0, 0), dt, dt, h, h, h)
        _, _, u, v, w = P.project(us, vs, ws, rho, zero, zero, 0.0, 0.0, dt, g)
    ue, ve, we = M.taylor_green(n, n, 2, t=t_end, nu=nu)
    return max(np.max(np.abs(u - ue)), np.max(np.abs(v - ve)), np.max(np.abs(w - we)))


def test_taylor_green_decay_second_order():
    """A full time step (Eq. uss_predic, then Eqs. poisson and corr) converges to the closed-form
    Taylor-Green decay at second order in h with dt proportional to h."""
    e16 = taylor_green_error(16, 0.1, 0.5)
    e32 = taylor_green_error(32, 0.1, 0.5)
    assert e32 < 5e-3
    assert 3.2 < e16 / e32 < 4.8
