"""GPU parity of the momentum predictor (Sec. 3.3, Eq. uss_predic) against the FP64 oracle.

Tolerances, with U = max(|u|, |v|, |w|), h the smallest spacing and S = U^2/h + nu U/h^2 the
scale of M:
  * FLUPS_MOM_FP64: both sides are binary64 with different rounding orders (the kernel sums
    the unscaled flux products, the oracle averages first) -> |M - M_or| <= 2^-40 S.
  * FLUPS_MOM_PAIR: every velocity is held as A + a with |a - exact| <= 2^-44 U, products
    carry ~q^2 = 2^-40 U^2 of rounding in their low parts and six of them enter each flux
    divergence, scaled by 1/(4h): about 2^-38 S; the check allows 2^-34 S.
  * u**: dt (|f1| + |f2|) times the M bound (the state M^{n-1} of each side comes from its
    own first step) plus 2^-50 max|u^n + dt g| for the final binary64 additions.
"""

import numpy as np
import pytest

import oracle
from oracle import momentum as om
from paper_2204_08834_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_08834_gb300 import flups  # noqa: E402

G = (0.1, -9.81, 0.3)
TOL = {flups.MOM_FP64: 2.0 ** -40, flups.MOM_PAIR: 2.0 ** -34}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def state_to_f64(st):
    a = host(st).astype(np.float64)
    return a[..., 0] + a[..., 1]          # [3][nz][ny][nx]


def run_two_steps(shape, h, fields1, fields2, nu, dt1, dt2, arith):
    """Two predictor calls (Euler, then AB2 with the state of the first); returns GPU and oracle
    (u**, M) of both calls."""
    nz, ny, nx = shape
    hx, hy, hz = h
    out = {}
    with flups.Plan(nx, ny, nz, hx, hy, hz, "periodic", "fp32_refine", flups.current_stream()) as plan:
        st = flups.momentum_state(nz, ny, nx)
        for call, (flds, dt, dtp) in enumerate(((fields1, dt1, 0.0), (fields2, dt2, dt1))):
            d = [dev(q) for q in flds]
            o = [torch.empty_like(d[0]) for _ in range(3)]
            plan.momentum_predict(*d, *o, st, nu, G, dt, dtp, arith)
            out[call] = ([host(q) for q in o], state_to_f64(st))
    m_prev = None
    ref = {}
    for call, (flds, dt, dtp) in enumerate(((fields1, dt1, 0.0), (fields2, dt2, dt1))):
        us, m = om.predictor(*flds, m_prev, nu, G, dt, dtp, hx, hy, hz)
        ref[call] = (us, m)
        m_prev = m
    return out, ref


def check(out, ref, flds, nu, h, dts, arith):
    hmin = min(h)
    U = max(np.max(np.abs(q)) for fl in flds for q in fl)
    S = U * U / hmin + nu * U / hmin ** 2
    worst = []
    for call in (0, 1):
        (us, m), (us_r, m_r) = out[call], ref[call]
        dt = dts[call]
        f1, f2 = om.ab2_coefficients(dt, dts[0] if call else 0.0)
        em = max(np.max(np.abs(m[q] - m_r[q])) for q in range(3))
        assert em <= TOL[arith] * S, (call, em / S)
        tol_u = dt * (abs(f1) + abs(f2)) * TOL[arith] * S + 2.0 ** -50 * (U + dt * max(map(abs, G)))
        eu = max(np.max(np.abs(us[q] - us_r[q])) for q in range(3))
        assert eu <= tol_u, (call, eu, tol_u)
        worst.append(em / S)
    return max(worst)


CASES = [((8, 8, 8), 0), ((8, 16, 16), 1), ((16, 8, 32), 2), ((32, 16, 64), 3), ((16, 32, 128), 4)]


@pytest.mark.parametrize("arith", [flups.MOM_PAIR, flups.MOM_FP64])
@pytest.mark.parametrize("shape,seed", CASES)
def test_predictor_matches_oracle(shape, seed, arith):
    nz, ny, nx = shape
    h = 1.0 / nx
    rng = np.random.default_rng(100 + seed)
    f1 = synth.solenoidal_velocity(nx, seed=200 + seed, nz=nz, ny=ny)
    f1 = tuple(q + c for q, c in zip(f1, (0.3, -0.2, 0.1)))
    f2 = tuple(q + 0.1 * rng.standard_normal(shape) for q in f1)   # not solenoidal: M is defined anyway
    nu = 0.01
    dt1 = 0.2 * h
    dt2 = 0.17 * h
    out, ref = run_two_steps(shape, (h, h, h), f1, f2, nu, dt1, dt2, arith)
    err = check(out, ref, (f1, f2), nu, (h, h, h), (dt1, dt2), arith)
    print(f"{shape} arith={arith}: max |M - M_or| / S = {err:.3g} (2^{np.log2(max(err, 1e-300)):.1f})")


def test_fp64_arith_on_unequal_spacings():
    shape = (16, 8, 32)
    h = (0.031, 0.047, 0.052)
    rng = np.random.default_rng(7)
    f1 = tuple(rng.standard_normal(shape) for _ in range(3))
    f2 = tuple(rng.standard_normal(shape) for _ in range(3))
    out, ref = run_two_steps(shape, h, f1, f2, 0.02, 0.003, 0.0025, flups.MOM_FP64)
    check(out, ref, (f1, f2), 0.02, h, (0.003, 0.0025), flups.MOM_FP64)


@pytest.mark.parametrize("scale,h", [(0.0, 1.0 / 32), (1e-20, 1.0 / 32), (2.0 ** 59, 1.0)])
def test_zero_tiny_and_huge_velocities(scale, h):
    """U = 0 takes the pair path with any quantum; U outside the pair range (2^-40 .. 2^60 and
    the spacing limits) makes the same launch run the binary64 path.  The huge case uses unit
    spacing so that M (~2 U^2/h) still fits the binary32 pairs of the state (|M| < 2^127)."""
    shape = (8, 16, 32)
    rng = np.random.default_rng(9)
    f1 = tuple(scale * rng.standard_normal(shape) for _ in range(3))
    f2 = tuple(scale * rng.standard_normal(shape) for _ in range(3))
    dt = 1e-3
    out, ref = run_two_steps(shape, (h, h, h), f1, f2, 0.01, dt, dt, flups.MOM_PAIR)
    if scale == 0.0:
        for call in (0, 1):
            us, m = out[call]
            assert all(np.all(q == 0.0) for q in m)
            for q, gq in zip(us, G):
                assert np.max(np.abs(q - dt * gq)) <= 2.0 ** -44 * abs(dt * gq)
    else:
        # outside the pair range the kernel is binary64: hold it to the binary64 bound
        check(out, ref, (f1, f2), 0.01, (h, h, h), (dt, dt), flups.MOM_FP64)


def test_single_spike_sets_the_quantum():
    """One velocity 1e6 times the rest: the quantum follows the maximum, the error bound is
    relative to it, and the small values still carry |a| <= q/2 accurately."""
    shape = (8, 16, 32)
    h = 1.0 / 32
    rng = np.random.default_rng(11)
    f1 = [rng.standard_normal(shape) for _ in range(3)]
    f1[1][3, 5, 7] = 1e6
    f2 = [q.copy() for q in f1]
    out, ref = run_two_steps(shape, (h, h, h), f1, f2, 0.01, 1e-8, 1e-8, flups.MOM_PAIR)
    check(out, ref, (f1, f2), 0.01, (h, h, h), (1e-8, 1e-8), flups.MOM_PAIR)


def test_nonfinite_input_propagates():
    shape = (8, 8, 32)
    u = np.zeros(shape)
    u[2, 3, 4] = np.nan
    with flups.Plan(32, 8, 8, 1 / 32, 1 / 32, 1 / 32) as plan:
        d = [dev(u), dev(np.zeros(shape)), dev(np.zeros(shape))]
        o = [torch.empty_like(d[0]) for _ in range(3)]
        st = flups.momentum_state(*shape)
        plan.momentum_predict(*d, *o, st, 0.01, G, 1e-3, 0.0, flups.MOM_PAIR)
        assert np.isnan(host(o[0])[2, 3, 4])


def test_argument_errors():
    shape = (8, 8, 32)
    z = dev(np.zeros(shape))
    o = [torch.empty_like(z) for _ in range(3)]
    st = flups.momentum_state(*shape)
    with flups.Plan(32, 8, 8, 1 / 32, 1 / 32, 1 / 32) as plan:
        for kw in ({"dt": 0.0}, {"nu": -1.0}, {"dt": float("nan")}):
            args = {"nu": 0.01, "dt": 1e-3}
            args.update(kw)
            with pytest.raises(flups.FlupsError) as e:
                plan.momentum_predict(z, z, z, *o, st, args["nu"], G, args["dt"], 0.0)
            assert e.value.status == flups.EINVAL
        with pytest.raises(flups.FlupsError) as e:           # output aliases an input
            plan.momentum_predict(z, z, z, z, o[1], o[2], st, 0.01, G, 1e-3, 0.0)
        assert e.value.status == flups.EINVAL
    with flups.Plan(32, 8, 8, 1 / 32, 1 / 16, 1 / 32) as plan:   # unequal spacings
        with pytest.raises(flups.FlupsError) as e:
            plan.momentum_predict(z, z, z, *o, st, 0.01, G, 1e-3, 0.0, flups.MOM_PAIR)
        assert e.value.status == flups.EUNSUPPORTED
        plan.momentum_predict(z, z, z, *o, st, 0.01, G, 1e-3, 0.0, flups.MOM_FP64)
    with flups.Plan(32, 8, 8, 1 / 32, 1 / 32, 1 / 32, "walls") as plan:
        with pytest.raises(flups.FlupsError) as e:
            plan.momentum_predict(z, z, z, *o, st, 0.01, G, 1e-3, 0.0, flups.MOM_FP64)
        assert e.value.status == flups.EUNSUPPORTED


def test_graph_replay_and_determinism():
    shape = (16, 32, 64)
    h = 1.0 / 64
    f = synth.solenoidal_velocity(64, seed=5, nz=16, ny=32)
    with flups.Plan(64, 32, 16, h, h, h, stream=flups.current_stream()) as plan:
        d = [dev(q) for q in f]
        o = [torch.empty_like(d[0]) for _ in range(3)]
        st = flups.momentum_state(*shape)
        plan.momentum_predict(*d, *o, st, 0.01, G, 0.1 * h, 0.0)
        first = [host(q) for q in o] + [host(st)]
        plan.momentum_predict(*d, *o, st, 0.01, G, 0.1 * h, 0.0)
        again = [host(q) for q in o] + [host(st)]
        assert all(np.array_equal(a, b) for a, b in zip(first, again))
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            plan.set_stream(s.cuda_stream)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                plan.momentum_predict(*d, *o, st, 0.01, G, 0.1 * h, 0.0)
        torch.cuda.current_stream().wait_stream(s)
        plan.set_stream(flups.current_stream())
        for q in o:
            q.zero_()
        g.replay()
        replay = [host(q) for q in o] + [host(st)]
        assert all(np.array_equal(a, b) for a, b in zip(first, replay))


def gpu_taylor_green(n, nu, t_end, arith, cfl=0.25, nz=8):
    """Predictor + projection on the GPU for the 2-D vortex (density 1, FP32+refine solve to
    rtol 1e-12); returns the final (u, v, w), the step count and dt."""
    h = 2 * np.pi / n
    steps = int(np.ceil(t_end / (cfl * h)))
    dt = t_end / steps
    u0 = synth.taylor_green(n, n, nz)
    with flups.Plan(n, n, nz, h, h, h, "periodic", "fp32_refine", flups.current_stream()) as plan:
        d = [dev(q) for q in u0]
        o = [torch.empty_like(d[0]) for _ in range(3)]
        zero = torch.zeros_like(d[0])
        f = torch.empty_like(d[0])
        p = torch.empty_like(d[0])
        plan.set_density(torch.ones_like(d[0]))
        st = flups.momentum_state(nz, n, n)
        for s in range(steps):
            plan.momentum_predict(*d, *o, st, nu, (0.0, 0.0, 0.0), dt, dt if s else 0.0, arith)
            plan.rhs(*o, zero, zero, 0.0, 0.0, dt, f)
            plan.solve(f, p, rtol=1e-12, max_iter=12)
            plan.correct(p, zero, zero, 0.0, 0.0, dt, *o)
            d = o + []
            o = [torch.empty_like(d[0]) for _ in range(3)]
        return [host(q) for q in d], steps, dt


def oracle_taylor_green(n, nu, steps, dt, nz=8):
    h = 2 * np.pi / n
    g = oracle.make_grid(n, n, nz, h, h, h, "periodic")
    u, v, w = synth.taylor_green(n, n, nz)
    rho = np.ones_like(u)
    zero = np.zeros_like(u)
    m_prev = None
    for _ in range(steps):
        (us, vs, ws), m_prev = om.predictor(u, v, w, m_prev, nu, (0, 0, 0), dt, dt, h, h, h)
        _, _, u, v, w = oracle.project(us, vs, ws, rho, zero, zero, 0.0, 0.0, dt, g)
    return u, v, w


@pytest.mark.parametrize("arith", [flups.MOM_PAIR, flups.MOM_FP64])
def test_taylor_green_time_steps_match_oracle_and_decay(arith):
    """A full time step on the GPU (predictor, rhs, solve, correct) follows the oracle's time
    stepping and converges to the closed-form decay u = sin x cos y exp(-2 nu t) at second
    order."""
    nu, t_end = 0.1, 0.5
    errs = []
    for n in (32, 64):
        (u, v, w), steps, dt = gpu_taylor_green(n, nu, t_end, arith)
        if n == 32:
            uo, vo, wo = oracle_taylor_green(n, nu, steps, dt)
            diff = max(np.max(np.abs(u - uo)), np.max(np.abs(v - vo)), np.max(np.abs(w - wo)))
            assert diff <= 1e-10, diff
        ue, ve, we = synth.taylor_green(n, n, 8, amplitude=np.exp(-2 * nu * t_end))
        errs.append(max(np.max(np.abs(u - ue)), np.max(np.abs(v - ve)), np.max(np.abs(w - we))))
    assert errs[1] < 1e-3
    assert 3.2 < errs[0] / errs[1] < 4.8, errs


def blocks_of(a, starts, b):
    """Periodic (b+2)^3 blocks of a with one-cell halos, origins `starts`."""
    nz, ny, nx = a.shape
    out = []
    for k0, j0, i0 in starts:
        kk = np.arange(k0 - 1, k0 + b + 1) % nz
        jj = np.arange(j0 - 1, j0 + b + 1) % ny
        ii = np.arange(i0 - 1, i0 + b + 1) % nx
        out.append(a[np.ix_(kk, jj, ii)])
    return out


@pytest.mark.slow
@pytest.mark.parametrize("arith", [flups.MOM_PAIR, flups.MOM_FP64])
def test_fullsize_512_sampled(arith):
    """The 512^3 workload in the launch configuration the benchmark times: M and u** on eight
    sampled 8^3 blocks (two on the periodic seams) against the oracle on the same blocks."""
    n = 512
    h = 1.0 / n
    f = synth.solenoidal_velocity(n, seed=50)
    nu, dt = 1e-3, 0.5 * h / max(np.max(np.abs(q)) for q in f)
    b = 8
    starts = [(0, 0, 0), (n - 4, 17, n - 3), (100, 200, 300), (255, 256, 257), (511, 3, 128), (64, 511, 9),
              (400, 100, 504), (37, 388, 222)]
    with flups.Plan(n, n, n, h, h, h, "periodic", "fp32_refine", flups.current_stream()) as plan:
        d = [dev(q) for q in f]
        o = [torch.empty_like(d[0]) for _ in range(3)]
        st = flups.momentum_state(n, n, n)
        plan.momentum_predict(*d, *o, st, nu, G, dt, 0.0, arith)
        torch.cuda.synchronize()
        m = state_to_f64(st)
        us = [host(q) for q in o]
        del d, o, st
    torch.cuda.empty_cache()
    U = max(np.max(np.abs(q)) for q in f)
    S = U * U / h + nu * U / h ** 2
    fb = [blocks_of(q, starts, b) for q in f]
    for s, (k0, j0, i0) in enumerate(starts):
        ub, vb, wb = fb[0][s], fb[1][s], fb[2][s]
        (usr, vsr, wsr), mr = om.predictor(ub, vb, wb, None, nu, G, dt, 0.0, h, h, h)
        kk = np.arange(k0, k0 + b) % n
        jj = np.arange(j0, j0 + b) % n
        ii = np.arange(i0, i0 + b) % n
        for q in range(3):
            got = m[q][np.ix_(kk, jj, ii)]
            assert np.max(np.abs(got - mr[q][1:-1, 1:-1, 1:-1])) <= TOL[arith] * S
            gu = us[q][np.ix_(kk, jj, ii)]
            assert np.max(np.abs(gu - (usr, vsr, wsr)[q][1:-1, 1:-1, 1:-1])) <= dt * TOL[arith] * S + 2.0 ** -50 * (
                U + dt * 10)
