"""GPU parity: every step of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (derived from the arithmetic, stated per check):
  * rhs, correct: FP64 stencils with a different rounding order and a Newton-refined
    reciprocal for 1/rho_f -> max |diff| <= 1e-12 * max |reference|.
  * FP64 direct solve: both sides are FP64 eigen-expansion solves with different FFT
    rounding orders -> relative L2 error of p <= 1e-11.
  * FP32+refine: the FP64 residual ||f - <f> - L p|| / ||f - <f>|| recomputed by the oracle
    from the GPU's p must be <= rtol (1e-10; 1e-12 for the divergence gate), and p must
    match the oracle's direct solution to 1e-8 relative (residual 1e-10 times the
    condition number of the smallest retained mode, at most ~1e2 on these grids).
  * divergence after correction: div_rel <= 1e-12 (direct-solver mass conservation,
    Sec. 3.1), run with rtol = 1e-12.
"""

import numpy as np
import pytest

import oracle
from paper_2204_08834_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_08834_gb300 import flups  # noqa: E402


def grid_of(c):
    nz, ny, nx = c.shape
    return oracle.make_grid(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = {
    "sphere16": lambda: synth.sphere(16),
    "sphere32": lambda: synth.sphere(32),
    "aniso_per_32x16x8": lambda: synth.random_fields(32, 16, 8, "periodic"),
    "aniso_per_8x64x16": lambda: synth.random_fields(8, 64, 16, "periodic", seed=91),
    "walls_uniform_16x8x12": lambda: synth.random_fields(16, 8, 12, "walls", False, seed=92),
    "walls_str_32x32x24": lambda: synth.random_fields(32, 32, 24, "walls", True, seed=93),
    "walls_str_64x16x2": lambda: synth.random_fields(64, 16, 2, "walls", True, seed=94),
    "two_layer_64x64x40": lambda: synth.two_layer(64, 64, 40),
    "emulsion64": lambda: synth.emulsion(64, ndrops=20),
    # one spacing in x, y and z with walls: the exact fixed-point defect applies
    "walls_cubic_32x16x24": lambda: synth.random_fields(32, 16, 24, "walls", False, lx=1.0, ly=0.5, lz=0.75,
                                                        seed=96),
    # lengths 3 * 2^a (radix-3 passes): the 48 and 96 members of the ensemble
    "per_48x24x96": lambda: synth.random_fields(48, 24, 96, "periodic", seed=97),
    "walls_str_96x48x30": lambda: synth.random_fields(96, 48, 30, "walls", True, seed=98),
    "emulsion48": lambda: synth.emulsion(48, ndrops=6, rmin_cells=2.0, rmax_cells=5.0),
    # long periodic columns: the four-step column transforms of every length they take
    # (y 256 and z 512 with 8-column tiles; y 1024 and z 128 with 4-column tiles)
    "per_16x256x512": lambda: synth.random_fields(16, 256, 512, "periodic", seed=99),
    "per_8x1024x128": lambda: synth.random_fields(8, 1024, 128, "periodic", seed=100),
    "per_32x128x1024": lambda: synth.random_fields(32, 128, 1024, "periodic", seed=101),
}
_cache = {}


def case(name):
    if name not in _cache:
        c = CASES[name]()
        g = grid_of(c)
        _cache[name] = (c, g, oracle.project(c.u, c.v, c.w, c.rho, c.pn, c.pnm1, 2.0, 1.0, c.dt, g))
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_set_density_rho0_is_min(name):
    c, g, _ = case(name)
    with flups.Plan.for_case(c, "fp64") as plan:
        plan.set_density(dev(c.rho))
        assert plan.rho0() == np.min(c.rho)
        plan.set_density(dev(c.rho), rho0=0.5)
        assert plan.rho0() == 0.5


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_matches_oracle(name):
    c, g, (fo, po, uo, vo, wo) = case(name)
    d = {k: dev(c[k]) for k in ("u", "v", "w", "rho", "pn", "pnm1")}
    f = torch.empty_like(d["u"])
    with flups.Plan.for_case(c, "fp32_refine") as plan:
        plan.set_density(d["rho"])
        plan.rhs(d["u"], d["v"], d["w"], d["pn"], d["pnm1"], 2.0, 1.0, c.dt, f)
        fg = host(f)
    assert np.max(np.abs(fg - fo)) <= 1e-12 * np.max(np.abs(fo))
    # p_nm1 = NULL means p_hat = c1 p^n
    with flups.Plan.for_case(c, "fp64") as plan:
        plan.set_density(d["rho"])
        plan.rhs(d["u"], d["v"], d["w"], d["pn"], None, 1.0, 0.0, c.dt, f)
        fg1 = host(f)
    fo1 = oracle.rhs(c.u, c.v, c.w, c.rho, c.pn, 0 * c.pn, 1.0, 0.0, c.dt, g)
    assert np.max(np.abs(fg1 - fo1)) <= 1e-12 * np.max(np.abs(fo1))


@pytest.mark.parametrize("name", list(CASES))
def test_solve_fp64_matches_oracle(name):
    c, g, (fo, po, _, _, _) = case(name)
    f = dev(fo)
    p = torch.empty_like(f)
    with flups.Plan.for_case(c, "fp64") as plan:
        info = plan.solve(f, p, rtol=1e-12)
        pg = host(p)
    err = np.linalg.norm(pg - po) / np.linalg.norm(po)
    assert err <= 1e-11, err
    assert info.iters == 1 and info.rel_res <= 1e-12
    assert oracle.rel_residual(fo, pg, g) <= 1e-12
    assert abs(oracle.volume_mean(pg, g)) <= 1e-13 * np.max(np.abs(pg))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("rtol", [1e-10, 1e-12])
def test_solve_refine_matches_oracle(name, rtol):
    c, g, (fo, po, _, _, _) = case(name)
    f = dev(fo)
    p = torch.empty_like(f)
    with flups.Plan.for_case(c, "fp32_refine") as plan:
        info = plan.solve(f, p, rtol=rtol, max_iter=10)
        pg = host(p)
    assert info.rel_res <= rtol
    hist = info.history()
    assert all(b < a for a, b in zip(hist, hist[1:])), hist
    assert oracle.rel_residual(fo, pg, g) <= 1.5 * rtol
    err = np.linalg.norm(pg - po) / np.linalg.norm(po)
    assert err <= 1e-8 if rtol >= 1e-10 else err <= 1e-10, err
    # the first iterate's FP32 constant is removed in the first FP64 update
    assert abs(oracle.volume_mean(pg, g)) <= 1e-12 * np.max(np.abs(pg))


@pytest.mark.parametrize("name", list(CASES))
def test_correct_matches_oracle(name):
    c, g, (fo, po, uo, vo, wo) = case(name)
    d = {k: dev(c[k]) for k in ("u", "v", "w", "rho", "pn", "pnm1")}
    with flups.Plan.for_case(c, "fp64") as plan:
        plan.set_density(d["rho"])
        plan.correct(dev(po), d["pn"], d["pnm1"], 2.0, 1.0, c.dt, d["u"], d["v"], d["w"])
        for key, ref in (("u", uo), ("v", vo), ("w", wo)):
            got = host(d[key])
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), key
    if c.bc == "walls":
        assert np.all(host(d["w"])[-1] == 0.0)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_projection_divergence_free(name, prec):
    """Full GPU projection (set_density, rhs, solve, correct) leaves D u^{n+1} = 0."""
    c, g, _ = case(name)
    d = {k: dev(c[k]) for k in ("u", "v", "w", "rho", "pn", "pnm1")}
    f = torch.empty_like(d["u"])
    p = torch.empty_like(d["u"])
    # D u^{n+1} = (dt/rho0)(f - <f> - L p) pointwise, and the max-norm divergence can exceed
    # the L2 relative residual by an O(1) factor, so the refinement runs to 1e-13 here.
    with flups.Plan.for_case(c, prec) as plan:
        plan.set_density(d["rho"])
        plan.rhs(d["u"], d["v"], d["w"], d["pn"], d["pnm1"], 2.0, 1.0, c.dt, f)
        plan.solve(f, p, rtol=1e-13, max_iter=10)
        plan.correct(p, d["pn"], d["pnm1"], 2.0, 1.0, c.dt, d["u"], d["v"], d["w"])
        u1, v1, w1 = host(d["u"]), host(d["v"]), host(d["w"])
    assert oracle.div_rel(u1, v1, w1, c.u, c.v, c.w, g) <= 1e-12


def test_project_host_matches_device_path():
    c, g, (fo, po, uo, vo, wo) = case("walls_str_32x32x24")
    u, v, w = c.u.copy(), c.v.copy(), c.w.copy()
    p = np.empty_like(u)
    with flups.Plan.for_case(c, "fp32_refine") as plan:
        # refinement past the divergence gate, as in test_projection_divergence_free
        info = plan.project_host(u, v, w, c.rho, c.pn, c.pnm1, 2.0, 1.0, c.dt, p, rtol=1e-13)
    assert info.rel_res <= 1e-13
    assert np.linalg.norm(p - po) / np.linalg.norm(po) <= 1e-10
    assert np.max(np.abs(u - uo)) <= 1e-10 * np.max(np.abs(uo))
    assert oracle.div_rel(u, v, w, c.u, c.v, c.w, g) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_solve_host_equals_device_solve(prec):
    c, g, (fo, po, _, _, _) = case("emulsion64")
    fh = torch.empty(c.shape, dtype=torch.float64, pin_memory=True).numpy()
    np.copyto(fh, fo)
    ph = np.full(c.shape, np.nan)
    fd = dev(fo)
    pd = torch.empty_like(fd)
    with flups.Plan.for_case(c, prec) as plan:
        i1 = plan.solve_host(fh, ph, rtol=1e-10, max_iter=12)
        i2 = plan.solve(fd, pd, rtol=1e-10, max_iter=12)
    assert np.array_equal(ph, host(pd))
    assert i1.iters == i2.iters
    assert np.linalg.norm(ph - po) / np.linalg.norm(po) <= (1e-11 if prec == "fp64" else 1e-8)


def test_project_host_equals_device_path_bitwise_at_2_24_points():
    """The host-buffer projection (inputs on the plan's copy stream, rho first; p copied back
    while the correction runs) returns the bits of the device-resident sequence, call after
    call, also after a call that failed (refinement stopped by max_iter)."""
    n = 256
    h, dt = 1.0 / n, 1e-3
    rng = np.random.default_rng(11)
    u, v, w = (rng.standard_normal((n, n, n)) for _ in range(3))
    rho = np.where(rng.random((n, n, n)) < 0.05, 10.0, 1.0)
    pn, pm = (0.01 * rng.standard_normal((n, n, n)) for _ in range(2))
    with flups.Plan(n, n, n, h, h, h, "periodic", "fp32_refine") as plan:
        d = {k: dev(a) for k, a in (("u", u), ("v", v), ("w", w), ("rho", rho), ("pn", pn), ("pm", pm))}
        f = torch.empty_like(d["u"])
        p = torch.empty_like(f)
        plan.set_density(d["rho"])
        plan.rhs(d["u"], d["v"], d["w"], d["pn"], d["pm"], 2.0, 1.0, dt, f)
        info = plan.solve(f, p, rtol=1e-10, max_iter=6)
        plan.correct(p, d["pn"], d["pm"], 2.0, 1.0, dt, d["u"], d["v"], d["w"])
        ref = [host(t) for t in (p, d["u"], d["v"], d["w"])]
        del d, f, p
        uh, vh, wh, ph = u.copy(), v.copy(), w.copy(), np.zeros_like(u)
        with pytest.raises(flups.FlupsError) as e:
            plan.project_host(uh, vh, wh, rho, pn, pm, 2.0, 1.0, dt, ph, rtol=1e-30, max_iter=1)
        assert e.value.status == flups.ENOCONV
        assert np.array_equal(uh, u) and not ph.any()      # nothing copied back on failure
        for _ in range(2):
            uh, vh, wh, ph = u.copy(), v.copy(), w.copy(), np.empty_like(u)
            inf = plan.project_host(uh, vh, wh, rho, pn, pm, 2.0, 1.0, dt, ph, rtol=1e-10, max_iter=6)
            assert inf.iters == info.iters and inf.rel_res == info.rel_res
            for a, b in zip((ph, uh, vh, wh), ref):
                assert np.array_equal(a, b)


@pytest.mark.parametrize("frac", [7.5, 100.0])
def test_refine_integer_defect_and_its_fp64_fallbacks(frac):
    """On a grid whose spacing is a power of two the defect is formed in 64-bit integers at the
    fixed-point scale of p, whose bound is B = 2^e with e the frexp exponent of max|p|: h^2 f
    must stay below 8 B.  f = c + g with h^2 <f> = 7.5 B puts the points where h^2 g > B/2
    past that bound (those points take the FP64 form, their neighbours the integer form);
    h^2 <f> = 100 B sends every point to the FP64 form.  Both refine to rtol against the
    oracle."""
    n = 32
    h = 1.0 / n
    g = oracle.make_grid(n, n, n, h, h, h, "periodic")
    gz = np.random.default_rng(21).standard_normal((n, n, n))
    gz -= oracle.volume_mean(gz, g)
    po = oracle.solve(gz, g)
    m, ex = np.frexp(np.max(np.abs(po)))
    assert 0.5005 < m < 0.9995                        # the FP32 iterate has the same exponent
    B = 2.0 ** ex
    f = gz + frac * B / h ** 2
    if frac < 8:
        over = h ** 2 * f >= 8 * B
        assert 0 < over.sum() < over.size // 2        # some points past the bound, most below
    p = torch.empty(n, n, n, dtype=torch.float64, device="cuda")
    with flups.Plan(n, n, n, h, h, h, "periodic", "fp32_refine") as plan:
        info = plan.solve(dev(f), p, rtol=1e-10, max_iter=10)
    pg = host(p)
    assert info.rel_res <= 1e-10
    assert oracle.rel_residual(f, pg, g) <= 1.5e-10
    assert np.linalg.norm(pg - po) / np.linalg.norm(po) <= 1e-8


def test_refine_reports_noconv():
    c, g, (fo, _, _, _, _) = case("sphere32")
    f = dev(fo)
    p = torch.empty_like(f)
    with flups.Plan.for_case(c, "fp32_refine") as plan:
        st, info = plan.solve(f, p, rtol=1e-14, max_iter=1, check=False)
    assert st == flups.ENOCONV and info.iters == 1 and info.rel_res > 1e-14


def test_bad_density_is_reported():
    c, g, _ = case("sphere16")
    rho = c.rho.copy()
    rho[3, 4, 5] = np.nan
    rho[1, 1, 1] = -1.0
    with flups.Plan.for_case(c, "fp32_refine") as plan:
        plan.set_density(dev(rho))
        with pytest.raises(flups.FlupsError) as e:
            plan.rho0()
        assert e.value.status == flups.ENONFINITE
        # the documented error exit reports the same latched state without reading rho0
        assert plan.sync(check=False) == flups.ENONFINITE
        plan.set_density(dev(c.rho))
        assert plan.sync(check=False) == flups.OK


def test_state_errors():
    c, g, _ = case("sphere16")
    d = dev(c.u)
    with flups.Plan.for_case(c, "fp64") as plan:
        with pytest.raises(flups.FlupsError) as e:
            plan.rhs(d, d, d, d, None, 1.0, 0.0, 1e-3, torch.empty_like(d))
        assert e.value.status == flups.ESTATE
        with pytest.raises(flups.FlupsError) as e:
            plan.solve(d, d)
        assert e.value.status == flups.EINVAL


def test_solve_zero_rhs_gives_zero():
    c, g, _ = case("walls_uniform_16x8x12")
    f = torch.zeros((12, 8, 16), dtype=torch.float64, device="cuda")
    p = torch.full_like(f, 7.0)
    with flups.Plan.for_case(c, "fp64") as plan:
        plan.solve(f, p, rtol=0.0, info=False)
        assert np.all(host(p) == 0.0)


def test_profiling_reports_every_launched_kernel():
    c, g, (fo, _, _, _, _) = case("sphere32")
    d = {k: dev(c[k]) for k in ("u", "v", "w", "rho", "pn", "pnm1")}
    f = torch.empty_like(d["u"])
    p = torch.empty_like(d["u"])
    with flups.Plan.for_case(c, "fp32_refine") as plan:
        plan.set_profiling(True)
        plan.set_density(d["rho"])
        plan.rhs(d["u"], d["v"], d["w"], d["pn"], d["pnm1"], 2.0, 1.0, c.dt, f)
        info = plan.solve(f, p, rtol=1e-10)
        plan.correct(p, d["pn"], d["pnm1"], 2.0, 1.0, c.dt, d["u"], d["v"], d["w"])
        prof = plan.profile()
    for k in ("k_rho_tiles", "k_rho_finalize", "k_face_coeffs", "k_rhs", "k_correct", "k_xfwd_f32", "k_xfwd_residual32",
              "k_ycol32", "k_zper32", "k_xinv32"):
        assert k in prof and prof[k][0] > 0.0, k
    assert prof["k_xfwd_residual32"][1] == info.iters
    # the first inverse x pass writes p, each later one adds the correction to it
    assert info.iters >= 2
    assert prof["k_xinv32"][1] == 1
    assert prof["k_xinv_acc32"][1] == info.iters - 1


def test_bounded_device_wait_reports_timeout():
    """A device-side wait on a barrier nothing arrives at gives up and returns ETIMEOUT; the
    context stays usable (a solve right after still matches the oracle)."""
    assert flups.selftest_wait_timeout(4096) == flups.ETIMEOUT
    assert flups.selftest_wait_timeout(1) == flups.ETIMEOUT
    c = synth.sphere(16)
    f = oracle.rhs(c.u, c.v, c.w, c.rho, c.pn, c.pnm1, 2.0, 1.0, c.dt, grid_of(c))
    fd = torch.from_numpy(f).cuda()
    p = torch.empty_like(fd)
    with flups.Plan.for_case(c, "fp64") as plan:
        plan.solve(fd, p, rtol=1e-12)
    po = oracle.solve(f, grid_of(c))
    assert np.max(np.abs(p.cpu().numpy() - po)) <= 1e-10 * np.max(np.abs(po))
