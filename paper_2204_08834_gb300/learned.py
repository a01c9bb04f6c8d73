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

import json
import struct

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


def train(net, windows, steps, lr=1e-3, seed=41, log_every=0, start=0):
    """`steps` Adam steps on samples drawn uniformly (seeded) from the windows; returns losses.
    `start` > 0 continues a run that stopped after `start` steps (restored from a checkpoint):
    the same seed then draws the samples the uninterrupted run would have drawn."""
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = samples(windows)
    for _ in range(start):
        rng.integers(len(idx))
    losses = []
    for s in range(start, start + steps):
        i, m = idx[rng.integers(len(idx))]
        win = windows[i]
        want = log_every and (s % log_every == 0 or s == start + steps - 1)
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


# ------------------------------------------------------- checkpoints and saved datasets
#
# File layout: the 8 bytes b"FLUPSARR", the header length as a little-endian uint64, a UTF-8
# JSON header {"version": 1, "arrays": [{"name", "dtype", "shape", "offset", "nbytes"}, ...],
# "meta": {...}}, then the arrays' raw little-endian bytes, offsets counted from the end of
# the header.

ARRAY_MAGIC = b"FLUPSARR"


def write_arrays(path, arrays, meta=None):
    """Named arrays (dict name -> ndarray) and a JSON-able `meta` dict in one file."""
    entries, blobs, off = [], [], 0
    for name, a in arrays.items():
        a = np.ascontiguousarray(a)
        le = a.astype(a.dtype.newbyteorder("<"), copy=False)
        b = le.tobytes()
        entries.append({"name": name, "dtype": le.dtype.str, "shape": list(a.shape), "offset": off,
                        "nbytes": len(b)})
        blobs.append(b)
        off += len(b)
    hdr = json.dumps({"version": 1, "arrays": entries, "meta": meta or {}}).encode()
    with open(path, "wb") as fh:
        fh.write(ARRAY_MAGIC)
        fh.write(struct.pack("<Q", len(hdr)))
        fh.write(hdr)
        for b in blobs:
            fh.write(b)


def read_arrays(path):
    """(dict name -> ndarray in native byte order, meta) of a file written by write_arrays."""
    with open(path, "rb") as fh:
        if fh.read(8) != ARRAY_MAGIC:
            raise ValueError(f"{path}: not an array file")
        raw = fh.read(8)
        if len(raw) != 8:
            raise ValueError(f"{path}: truncated header")
        (n,) = struct.unpack("<Q", raw)
        hdr = fh.read(n)
        if len(hdr) != n:
            raise ValueError(f"{path}: truncated header")
        hdr = json.loads(hdr.decode())
        data = fh.read()
    if hdr.get("version") != 1:
        raise ValueError(f"{path}: unknown version {hdr.get('version')}")
    out = {}
    for e in hdr["arrays"]:
        dt = np.dtype(e["dtype"])
        count = int(np.prod(e["shape"], dtype=np.int64))
        if e["offset"] + e["nbytes"] > len(data) or count * dt.itemsize != e["nbytes"]:
            raise ValueError(f"{path}: array {e['name']} truncated or inconsistent")
        a = np.frombuffer(data, dtype=dt, count=count, offset=e["offset"]).reshape(e["shape"])
        out[e["name"]] = a.astype(dt.newbyteorder("="))
    return out, hdr["meta"]


def save_checkpoint(net, path, meta=None):
    """The whole training state of a flups.PNet: FP32 master parameters, Adam moments, step
    count (in meta["step"]) and the caller's `meta` (learning rate, seed, ...)."""
    m, v, step = net.adam_state()
    write_arrays(path, {"params": net.params(), "m": m, "v": v},
                 dict(meta or {}, kind="pnet-checkpoint", step=step, nparams=flups.PNET_NPARAMS))


def load_checkpoint(path):
    """(arrays, meta) of a checkpoint written by save_checkpoint."""
    arrays, meta = read_arrays(path)
    if meta.get("kind") != "pnet-checkpoint" or meta.get("nparams") != flups.PNET_NPARAMS:
        raise ValueError(f"{path}: not a checkpoint of this net")
    return arrays, meta


def restore(net, arrays, meta):
    """Puts a loaded checkpoint into `net`; training then continues as if never stopped."""
    net.set_params(arrays["params"])
    net.set_adam_state(arrays["m"], arrays["v"], meta["step"])


def save_windows(path, windows, dt):
    """A dataset of windows (density and the exact pressure series; FP64) with dt."""
    arrays, info = {}, []
    for i, win in enumerate(windows):
        arrays[f"w{i}/rho"] = win.rho.cpu().numpy()
        for m, p in enumerate(win.p):
            arrays[f"w{i}/p{m}"] = p.cpu().numpy()
        info.append({"rho0": win.rho0, "steps": len(win.p)})
    write_arrays(path, arrays, {"kind": "learned-windows", "dt": dt, "windows": info})


def load_windows(path, device="cuda"):
    """(windows, dt) of a dataset written by save_windows, on `device`."""
    import torch
    arrays, meta = read_arrays(path)
    if meta.get("kind") != "learned-windows":
        raise ValueError(f"{path}: not a saved dataset")
    wins = []
    for i, wi in enumerate(meta["windows"]):
        rho = torch.from_numpy(arrays[f"w{i}/rho"]).to(device)
        ps = [torch.from_numpy(arrays[f"w{i}/p{m}"]).to(device) for m in range(wi["steps"])]
        wins.append(Window(rho, wi["rho0"], ps))
    return wins, meta["dt"]
