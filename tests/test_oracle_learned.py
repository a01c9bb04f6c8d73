"""Pins of the learned-p_hat oracle (CPU): the variable-coefficient solve against a dense
solve of an independently looped operator and the constant-density limit; the conv net
against finite differences, periodic shift equivariance and single-tap kernels; Adam against
its closed form on the first step; the density feature against the split coefficient that
oracle.correct applies, and the predictor's zero-net limit against oracle.p_hat."""

import numpy as np
import pytest

import oracle
from oracle import learned as L
from paper_2204_08834_gb300 import synth

from test_oracle_pins import bordered_solve, varcoef_dense


def grid_of(c):
    nz, ny, nx = c.shape
    return oracle.make_grid(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc)


@pytest.mark.parametrize("bc", ["periodic", "walls"])
def test_varcoef_solve_matches_dense(bc):
    """PCG equals a dense solve of rho0 D((1/rho_f) G p) = f (explicit index loops)."""
    c = synth.random_fields(6, 6, 6, bc, stretched=(bc == "walls"), lx=1.0, ly=1.0, lz=1.0, seed=5)
    g = grid_of(c)
    rho = 1.0 + 19.0 * (np.random.default_rng(3).random(c.shape) > 0.5)
    f = np.random.default_rng(4).standard_normal(c.shape)
    p, it, rel = L.varcoef_solve(f, rho, g, rtol=1e-13)
    assert rel <= 1e-13
    A = rho.min() * varcoef_dense(rho, g)
    wts = np.broadcast_to(g.dzf[:, None, None], c.shape).ravel()
    p_lu, _ = bordered_solve(A, f.ravel(), wts)
    assert np.max(np.abs(p.ravel() - p_lu)) <= 1e-10 * np.max(np.abs(p_lu))


def test_varcoef_constant_density_is_poisson():
    """rho = const: A = L, one preconditioned step solves it exactly."""
    c = synth.sphere(8)
    g = grid_of(c)
    f = np.random.default_rng(5).standard_normal(c.shape)
    p, it, rel = L.varcoef_solve(f, np.full(c.shape, 2.0), g, rtol=1e-13)
    assert it == 1
    assert np.allclose(p, oracle.solve(f, g), atol=1e-12 * np.max(np.abs(p)))


def test_split_solve_fixed_point_with_exact_pressure():
    """p_hat = p_ex (the variable-coefficient pressure) makes the split solve exact."""
    c = synth.sphere(12)
    g = grid_of(c)
    rho0 = c.rho.min()
    f0 = oracle.rhs(c.u, c.v, c.w, c.rho, 0 * c.pn, 0 * c.pn, 0.0, 0.0, c.dt, g)
    p_ex, _, _ = L.varcoef_solve(f0, c.rho, g, rtol=1e-13)
    f = oracle.rhs(c.u, c.v, c.w, c.rho, p_ex, 0 * p_ex, 1.0, 0.0, c.dt, g, rho0)
    p = oracle.solve(f, g)
    assert np.max(np.abs(p - p_ex)) <= 1e-9 * np.max(np.abs(p_ex))


def small_net(rng, widths=(3, 2, 1)):
    return [(rng.standard_normal((widths[i + 1], widths[i], 27)) * 0.3, rng.standard_normal(widths[i + 1]) * 0.1)
            for i in range(len(widths) - 1)]


def test_conv_backward_matches_finite_differences():
    """Central differences (h = 1e-6) of the MSE loss of a 2-layer, 2-channel net at 6^3."""
    rng = np.random.default_rng(7)
    params = small_net(rng)
    rho = 1.0 + rng.random((6, 6, 6))
    pn, pnm1, pt = (rng.standard_normal((6, 6, 6)) for _ in range(3))
    loss, grads = L.loss_and_grads(params, rho, pn, pnm1, pt, 1.0)
    h = 1e-6
    for li, (w, b) in enumerate(params):
        for idx in [(0, 0, 0), (1, 2, 13), (0, 1, 26)] if li == 0 else [(0, 0, 5), (0, 1, 20)]:
            w[idx] += h
            lp, _ = L.loss_and_grads(params, rho, pn, pnm1, pt, 1.0)
            w[idx] -= 2 * h
            lm, _ = L.loss_and_grads(params, rho, pn, pnm1, pt, 1.0)
            w[idx] += h
            assert abs((lp - lm) / (2 * h) - grads[li][0][idx]) <= 1e-6 * max(1.0, abs(grads[li][0][idx]))
        b[0] += h
        lp, _ = L.loss_and_grads(params, rho, pn, pnm1, pt, 1.0)
        b[0] -= 2 * h
        lm, _ = L.loss_and_grads(params, rho, pn, pnm1, pt, 1.0)
        b[0] += h
        assert abs((lp - lm) / (2 * h) - grads[li][1][0]) <= 1e-6 * max(1.0, abs(grads[li][1][0]))


def test_conv_single_tap_is_a_shift_and_equivariant():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((1, 5, 6, 7))
    w = np.zeros((1, 1, 27))
    w[0, 0, L.TAPS.index((1, 0, -1))] = 1.0
    y = L.conv3(x, w, np.zeros(1))
    assert np.array_equal(y[0], np.roll(x[0], (-1, 0, 1), axis=(0, 1, 2)))
    params = small_net(rng, (1, 3, 1))
    ya, _ = L.forward(params, x)
    yb, _ = L.forward(params, np.roll(x, 2, axis=-1))
    assert np.allclose(np.roll(ya, 2, axis=-1), yb, atol=1e-12)


def test_adam_first_step_moves_by_lr_times_sign():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    L.adam_update(p, g, m, v, 1, 0.01)
    assert np.allclose(p, np.array([1.0, -2.0, 3.0]) - 0.01 * np.sign(g), atol=1e-7)


def test_bf16_rounding_against_float32_bits():
    """bf16() against rounding the float32 bit pattern (exact float32 inputs), plus ties."""
    rng = np.random.default_rng(9)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))).astype(np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)
    assert np.array_equal(L.bf16(x.astype(np.float64)), rounded.astype(np.float64))
    assert L.bf16(1.0 + 2.0 ** -8) == 1.0                     # tie -> even
    assert L.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # tie -> even (upwards)
    assert L.bf16(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7


def test_splitting_error_vanishes_for_exact_pressure_and_constant_density():
    c = synth.sphere(12)
    g = grid_of(c)
    e_p, e_u, e_du, ps, p_ex = L.split_error(c.u, c.v, c.w, c.rho, c.pn, c.dt, g)
    assert e_p > 1e-3 and e_du > e_u > 0.0                    # a random p_hat is far off
    e_p0, e_u0, e_du0, _, _ = L.split_error(c.u, c.v, c.w, c.rho, p_ex, c.dt, g, p_ex)
    assert e_p0 <= 1e-10 and e_u0 <= 1e-10 and e_du0 <= 1e-10
    # u_ex is divergence free
    z = np.zeros_like(p_ex)
    ue = oracle.correct(c.u, c.v, c.w, p_ex, p_ex, z, c.rho, 1.0, 0.0, c.dt, g)
    assert np.max(np.abs(oracle.div(*ue, g))) <= 1e-9 * np.max(np.abs(oracle.div(c.u, c.v, c.w, g)))
    # constant density: the split is exact whatever p_hat is
    rho1 = np.full(c.shape, 3.0)
    e_p1, e_u1, e_du1, _, _ = L.split_error(c.u, c.v, c.w, rho1, c.pn, c.dt, g)
    assert e_p1 <= 1e-12 and e_u1 <= 1e-12


def test_rounded_forward_backward_stay_close_to_fp64():
    """With bf16 rounding points the net stays within a few bf16 ulps of the FP64 net
    (a structural check that rnd is applied to values, not to indices)."""
    rng = np.random.default_rng(11)
    params = small_net(rng, (3, 4, 4, 1))
    rho = 1.0 + 9.0 * (rng.random((6, 6, 6)) > 0.7)
    pn, pnm1, pt = (rng.standard_normal((6, 6, 6)) for _ in range(3))
    l0, g0 = L.loss_and_grads(params, rho, pn, pnm1, pt, 1.0)
    l1, g1 = L.loss_and_grads(params, rho, pn, pnm1, pt, 1.0, rnd=L.bf16)
    assert abs(l1 - l0) <= 2e-2 * l0
    for (a, _), (b, _) in zip(g0, g1):
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(a)


def test_density_feature_is_the_split_coefficient_of_the_correction():
    """The density feature (reading L2) is the factor the split puts in front of G p_hat:
    oracle.correct with p = 0, u** = 0 gives u = (dt/rho0)(1 - rho0/rho_f) G_x p_hat, and at
    x faces between two cells of equal density that ratio must equal the cells' feature."""
    n = 8
    g = oracle.make_grid(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, "periodic")
    rho = np.ones((n, n, n))
    rho[:, :, 2:6] = 3.0                                    # a slab of density 3 in 1
    rho[:, 5:, 3:5] = 7.0                                   # and a block of density 7 in it
    x = (np.arange(n) + 0.5) / n
    ph = np.broadcast_to(np.sin(2 * np.pi * x), (n, n, n)).copy()
    zero = np.zeros_like(rho)
    dt = 0.01
    u1, _, _ = oracle.correct(zero, zero, zero, zero, ph, zero, rho, 1.0, 0.0, dt, g)
    gx = (np.roll(ph, -1, axis=2) - ph) / g.dx
    same = (rho == np.roll(rho, -1, axis=2)) & (np.abs(gx) > 1e-3)
    ratio = u1[same] / (dt / oracle.min_density(rho) * gx[same])
    feat, _ = L.features(rho, ph, ph, oracle.min_density(rho))
    assert same.sum() > 100
    assert np.max(np.abs(ratio - feat[0][same])) < 1e-12
    assert {round(v, 12) for v in feat[0][same]} == {0.0, round(2 / 3, 12), round(6 / 7, 12)}


def test_zero_net_predicts_the_method_extrapolation_and_a_bias_net_adds_s_times_it():
    """All weights zero: the prediction is the method's own p_hat = 2 p^n - p^{n-1} (Sec. 3.3,
    constant dt, as oracle.p_hat); a last-layer bias c alone adds s c with s = rms(p^n)."""
    rng = np.random.default_rng(4)
    shape = (4, 6, 8)
    rho = 1.0 + rng.random(shape)
    pn, pnm1 = rng.standard_normal(shape), rng.standard_normal(shape)
    layers = [(np.zeros((co, ci, 27)), np.zeros(co)) for ci, co in ((3, 16), (16, 16), (16, 16), (16, 1))]
    base = oracle.p_hat(pn, pnm1, 2.0, 1.0)
    assert np.array_equal(L.predict(layers, rho, pn, pnm1, 1.0), base)
    layers[-1] = (layers[-1][0], np.array([0.25]))
    s = np.linalg.norm(pn) / np.sqrt(pn.size)
    assert np.allclose(L.predict(layers, rho, pn, pnm1, 1.0), base + 0.25 * s, rtol=0, atol=1e-14)
