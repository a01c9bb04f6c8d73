"""GPU VoF step (flups_vof_step: MTHINC reconstruction and split advection, Sec. 3.1 and
App. A) against the FP64 oracle (oracle/vof.py).

Each split is compared with the oracle's split of the same input: phi^x with the oracle's x
split of phi^n, phi^y with its y split of the GPU's phi^x, phi^z with its z split of the GPU's
phi^y, and phi^{n+1} with the correction formula on the GPU's stages.  Both sides then
reconstruct from identical arrays, and both take the case decision (the largest Youngs
gradient component) and the uniform-cell test in binary32 from sums rounded in the same order,
so the integer decisions agree.
Tolerance of a split (derived from the arithmetic): the GPU's reconstruction and fluxes run in
FP32; a flux is a fraction of a cell volume at most |c| <= 1, so each face flux carries about
1e-6 of rounding (FP32 d_th solve, softplus differences of arguments up to ~40), i.e. at most
a few 1e-6 on phi per split; 2e-5 absolute bounds it, with a mean below 5e-7.  The FP64
updates conserve sum(phi) to rounding for any velocity; zero velocity leaves phi unchanged
bit for bit; a CFL of exactly 1 shifts phi by one cell up to the FP32 cell integral (5e-6).
A full (or empty) domain stays full (empty) to FP64 rounding under a discretely solenoidal
velocity: the flux of a uniform cell is phi u dt / h in FP64, the number the update divides out.
"""

import numpy as np
import pytest

from oracle import vof as ov
from paper_2204_08834_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_08834_gb300 import flups  # noqa: E402


def sphere_phi(n, centre, radius, width=0.75):
    x = np.arange(n) + 0.5
    r = np.sqrt((x[None, None, :] - centre[0]) ** 2 + (x[None, :, None] - centre[1]) ** 2
                + (x[:, None, None] - centre[2]) ** 2)
    return 0.5 * (1.0 - np.tanh((r - radius) / width))


def droplets_phi(n, seed):
    rng = np.random.default_rng(seed)
    phi = np.zeros((n, n, n))
    for _ in range(4):
        c = rng.uniform(0, n, 3)
        rad = rng.uniform(3.0, n / 5)
        x = np.arange(n) + 0.5
        dd = [np.minimum(np.abs(x - c[a]), n - np.abs(x - c[a])) for a in range(3)]
        r = np.sqrt(dd[0][None, None, :] ** 2 + dd[1][None, :, None] ** 2 + dd[2][:, None, None] ** 2)
        phi = np.maximum(phi, 0.5 * (1.0 - np.tanh((r - rad) / 0.75)))
    return phi


def solenoidal(shape, seed, cfl, h, dt):
    vel = synth.solenoidal_velocity(shape[2], seed=seed, nz=shape[0], ny=shape[1])
    umax = max(float(np.max(np.abs(q))) for q in vel)
    return [np.ascontiguousarray(q * (cfl * h / dt / umax)) for q in vel]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_step(phi, vel, dt, h, beta):
    nz, ny, nx = phi.shape
    d = dev(phi)
    st = torch.empty((3,) + phi.shape, dtype=torch.float64, device="cuda")
    with flups.Plan(nx, ny, nz, h, h, np.full(nz, h), "periodic", "fp32_refine", flups.current_stream()) as plan:
        plan.vof_step(d, *[dev(v) for v in vel], dt, beta, st)
        st_ = plan.sync(check=False)
    return d.cpu().numpy(), st.cpu().numpy(), st_


@pytest.mark.parametrize("case", ["sphere32", "droplets48", "aniso"])
def test_splits_match_oracle(case):
    beta, dt = 2.0, 1.0
    if case == "sphere32":
        phi, h = sphere_phi(32, (15.6, 16.3, 16.1), 7.3), 1.0
    elif case == "droplets48":
        phi, h = droplets_phi(48, 7), 1.0 / 48
    else:
        phi, h = droplets_phi(32, 9)[:16, :24, :], 0.5
    vel = solenoidal(phi.shape, 11, 0.45, h, dt)
    out, st, status = gpu_step(phi, vel, dt, h, beta)
    assert status == flups.OK
    src = phi
    for a in range(3):
        ref = ov.split(src, vel[a], dt, h, a, beta)
        err = np.abs(st[a] - ref)
        assert np.max(err) <= 2e-5, (a, np.max(err))
        assert np.mean(err) <= 5e-7, (a, np.mean(err))
        src = st[a]
    fin = st[2].copy()
    for a in range(3):
        fin = fin - dt / h * st[a] * (vel[a] - ov.sh(vel[a], -1, a))
    assert np.max(np.abs(out - fin)) <= 1e-14
    assert abs(out.sum() - phi.sum()) <= 1e-12 * phi.sum()


def test_mass_conserved_for_any_velocity():
    phi = droplets_phi(32, 3)
    rng = np.random.default_rng(5)
    vel = [rng.uniform(-0.45, 0.45, phi.shape) for _ in range(3)]     # divergent
    out, _, status = gpu_step(phi, vel, 1.0, 1.0, 2.0)
    assert status == flups.OK
    assert abs(out.sum() - phi.sum()) <= 1e-12 * phi.sum()


def test_zero_velocity_and_cfl_one():
    phi = sphere_phi(16, (8.2, 7.7, 8.4), 4.5)
    z = np.zeros_like(phi)
    out, _, _ = gpu_step(phi, [z, z, z], 1.0, 1.0, 2.0)
    assert np.array_equal(out, phi)
    one = np.ones_like(phi)
    out, _, _ = gpu_step(phi, [one, -one, one], 1.0, 1.0, 2.0)
    ref = np.roll(np.roll(np.roll(phi, 1, axis=2), -1, axis=1), 1, axis=0)
    assert np.max(np.abs(out - ref)) <= 5e-6


def test_full_and_empty_domains_stay_so():
    vel = solenoidal((24, 16, 32), 13, 0.45, 1.0, 1.0)
    for val in (0.0, 1.0):
        phi = np.full((24, 16, 32), val)
        out, st, status = gpu_step(phi, vel, 1.0, 1.0, 2.0)
        assert status == flups.OK
        assert np.max(np.abs(out - val)) <= 1e-13, val
        assert np.max(np.abs(st - val)) <= 1e-13, val


def test_cfl_above_one_is_reported():
    phi = sphere_phi(16, (8.2, 7.7, 8.4), 4.5)
    z = np.zeros_like(phi)
    u = np.full_like(phi, 1.5)
    _, _, status = gpu_step(phi, [u, z, z], 1.0, 1.0, 2.0)
    assert status == flups.EINVAL


def test_unsupported_grids():
    with flups.Plan(32, 32, 24, 1.0, 1.0, np.full(24, 1.0), "walls", "fp32_refine", flups.current_stream()) as plan:
        t = torch.zeros((24, 32, 32), dtype=torch.float64, device="cuda")
        with pytest.raises(flups.FlupsError) as e:
            plan.vof_step(t, t, t, t, 0.1)
        assert e.value.status == flups.EUNSUPPORTED
