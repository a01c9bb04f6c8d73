"""Learned splitting pressure: data generation, training and evaluation on the GPU.

Host orchestration only: every arithmetic step runs in libflups' kernels (flups.Plan for the
exact variable-coefficient solves and the split projection, flups.PNet for the net).

Workload (64^3 training windows, 128^3 inference windows, see synth.learned_window): per
window a fixed droplet field of density ratio 20 and a velocity predictor that follows an
AR(1) series; the pressures p^m of the series are exact variable-coefficient solves
(flups_varcoef_solve to 1e-12).  A sample is (rho, p^{m-1}, p^m -> p^{m+1}).

The splitting error of a predictor p_hat at step n+1 (u** = u^{n+1} of the series):
p_split = split solve with p_hat, u_split its corrected velocity; against p_ex = p^{n+1} and
u_ex = u** - (dt/rho_f) G p_ex:  e_p = ||p_split - p_ex|| / ||p_ex||,
e_u = ||u_split - u_ex|| / ||u_ex||, and relative to the pressure correction itself
e_du = ||u_split - u_ex|| / ||u_ex - u**||.
"""

import numpy as np

from . import flups, synth

LAYERS = [(3, 16), (16, 16), (16, 16), (16, 1)]


def init_params(seed=40):
    """He-normal weights (std sqrt(2 / (27 in))), last layer scaled by 0.1, zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for li, (cin, cout) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (27 * cin)) * (0.1 if li == len(LAYERS) - 1 else 1.0)
        out.append((rng.standard_normal((cout, cin, 27)) * std).ravel())
        out.append(np.zeros(cout))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == flups.PNET_NPARAMS
    return p


def split_params(params):
    """Flat parameter vector -> [(W (out, in, 27), b (out,))] as float64."""
    p = np.asarray(params, dtype=np.float64)
    res, o = [], 0
    for cin, cout in LAYERS:
        w = p[o:o + cout * cin * 27].reshape(cout, cin, 27)
        o += cout * cin * 27
        b = p[o:o + cout]
        o += cout
        res.append((w, b))
    return res


class Window:
    """One window on the device: rho, rho0, the velocity predictors (optional) and p^m."""

    def __init__(self, rho, rho0, p, vel=None):
        self.rho, self.rho0, self.p, self.vel = rho, rho0, p, vel


def make_window(kind, w, steps, keep_velocity=False, n=None, rtol=1e-12, device="cuda"):
    """Builds window w of `kind` ("train" / "infer"): `steps` exact pressures on the GPU."""
    import torch
    rho_h, vseed, n, dt = synth.learned_window(kind, w, n)
    dzf = np.full(n, 1.0 / n)
    rho = torch.from_numpy(rho_h).to(device)
    zero = torch.zeros_like(rho)
    f = torch.empty_like(rho)
    ps, vel = [], []
    with flups.Plan(n, n, n, 1.0 / n, 1.0 / n, dzf, "periodic", "fp64", flups.current_stream()) as plan:
        plan.set_density(rho)
        rho0 = plan.rho0()
        for uvw in synth.velocity_series(n, steps, vseed):
            u, v, ww = (torch.from_numpy(a).to(device) for a in uvw)
            plan.rhs(u, v, ww, zero, None, 0.0, 0.0, dt, f)
            p = torch.empty_like(rho)
            plan.varcoef_solve(rho, f, p, rtol=rtol, max_iter=2000)
            ps.append(p)
            if keep_velocity:
                vel.append((u, v, ww))
    return Window(rho, rho0, ps, vel if keep_velocity else None), dt


def samples(windows):
    """(window index, m) of every sample (p^{m-1}, p^m -> p^{m+1})."""
    return [(i, m) for i, win in enumerate(windows) for m in range(1, len(win.p) - 1)]


def train(net, windows, steps, lr=1e-3, seed=41, log_every=0):
    """`steps` Adam steps on samples drawn uniformly (seeded) from the windows; returns losses."""
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = samples(windows)
    losses = []
    for s in range(steps):
        i, m = idx[rng.integers(len(idx))]
        win = windows[i]
        want = log_every and (s % log_every == 0 or s == steps - 1)
        loss = net.train_step(win.rho, win.rho0, win.p[m], win.p[m - 1], win.p[m + 1], lr, want_loss=bool(want))
        if want:
            losses.append((s, loss))
    return losses


def eval_losses(net, windows):
    """Mean loss of the net and of the linear extrapolation (y = 0) over every sample; the
    latter is evaluated on the host (a reported baseline, not part of the path)."""
    net_l, lin_l = [], []
    host = [[p.cpu().numpy() for p in win.p] for win in windows]
    for i, m in samples(windows):
        win = windows[i]
        net_l.append(net.eval_loss(win.rho, win.rho0, win.p[m], win.p[m - 1], win.p[m + 1]))
        pm1, pn, pp1 = host[i][m - 1], host[i][m], host[i][m + 1]
        t = pp1 - 2.0 * pn + pm1
        lin_l.append(float(np.mean(t * t) / np.mean(pn * pn)))
    return float(np.mean(net_l)), float(np.mean(lin_l))


def splitting_errors(win, m, dt, pn, pnm1, c1, c2, plan):
    """(e_p, e_u, e_du) of the split projection of step m with p_hat = c1 pn - c2 pnm1."""
    import torch
    u, v, w = win.vel[m]
    f = torch.empty_like(u)
    p = torch.empty_like(u)
    plan.rhs(u, v, w, pn, pnm1, c1, c2, dt, f)
    plan.solve(f, p, rtol=1e-13, max_iter=8)
    us, vs, ws = u.clone(), v.clone(), w.clone()
    plan.correct(p, pn, pnm1, c1, c2, dt, us, vs, ws)
    pe = win.p[m]
    ue, ve, we = u.clone(), v.clone(), w.clone()
    plan.correct(pe, pe, None, 1.0, 0.0, dt, ue, ve, we)
    h = lambda a: a.cpu().numpy()
    pe_h = h(pe)
    e_p = np.linalg.norm(h(p) - pe_h) / np.linalg.norm(pe_h)
    num = sum(np.linalg.norm(h(a) - h(b)) ** 2 for a, b in ((us, ue), (vs, ve), (ws, we)))
    den_u = sum(np.linalg.norm(h(a)) ** 2 for a in (ue, ve, we))
    den_du = sum(np.linalg.norm(h(a) - h(b)) ** 2 for a, b in ((ue, u), (ve, v), (we, w)))
    return float(e_p), float(np.sqrt(num / den_u)), float(np.sqrt(num / den_du))


def compare_predictors(net, win, dt, plan):
    """Splitting errors of the learned and the linear predictors at every step m >= 2."""
    import torch
    out = {"net": [], "lin": []}
    p_hat = torch.empty_like(win.rho)
    for m in range(2, len(win.p)):
        net.predict(win.rho, win.rho0, win.p[m - 1], win.p[m - 2], p_hat)
        out["net"].append(splitting_errors(win, m, dt, p_hat, None, 1.0, 0.0, plan))
        out["lin"].append(splitting_errors(win, m, dt, win.p[m - 1], win.p[m - 2], 2.0, 1.0, plan))
    return out
