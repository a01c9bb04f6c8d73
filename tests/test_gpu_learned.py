"""Learned splitting pressure on the GPU against the oracle.

* flups_varcoef_solve (PCG) against the oracle's PCG on the same equation, periodic and
  stretched walls, FP64 and FP32-refine preconditioners; the split fixed point on the GPU.
* The conv net's forward pass, gradients and Adam steps against the FP64 oracle net with the
  same bfloat16 rounding points (weights, every layer's input, every layer's output gradient).
  What is left is FP32 accumulation order and the rare bfloat16 rounding flips it causes, so
  each output is held to 4e-3 of max|y| (one flipped activation moves an output by about
  2^-8 |w a| ~ 1e-3 max|y|) and the mean error to 1e-4 max|y|; gradients to 1e-2 relative
  L2 per layer.
* Full-size inference (128^3): sampled outputs against the oracle on the 9^3 receptive-field
  patch around each sample (periodic wrap contaminates only cells within 4 of the patch edge).
* Training: the learned p_hat beats the linear extrapolation on held-out windows.
"""

import numpy as np
import pytest

import oracle
from oracle import learned as L
from paper_2204_08834_gb300 import learned, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_08834_gb300 import flups  # noqa: E402


def grid_of(c):
    nz, ny, nx = c.shape
    return oracle.make_grid(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ----------------------------------------------------------------- exact solve

VC_CASES = {
    "sphere16": lambda: synth.sphere(16),
    "walls_str_16x16x12": lambda: synth.random_fields(16, 16, 12, "walls", True, ratio=20.0, seed=3),
    "emulsion32_r20": lambda: synth.emulsion(32, ratio=20.0, ndrops=6, rmin_cells=2.0, rmax_cells=4.0, seed=7),
}


@pytest.mark.parametrize("name,prec", [("sphere16", "fp64"), ("sphere16", "fp32_refine"),
                                       ("walls_str_16x16x12", "fp64"), ("emulsion32_r20", "fp32_refine")])
def test_varcoef_solve_matches_oracle(name, prec):
    c = VC_CASES[name]()
    g = grid_of(c)
    z = np.zeros(c.shape)
    f = oracle.rhs(c.u, c.v, c.w, c.rho, z, z, 0.0, 0.0, c.dt, g)
    p_o, it_o, rel_o = L.varcoef_solve(f, c.rho, g, rtol=1e-12)
    rho, fd = dev(c.rho), dev(f)
    p = torch.empty_like(fd)
    with flups.Plan.for_case(c, prec) as plan:
        plan.set_density(rho)
        info = plan.varcoef_solve(rho, fd, p, rtol=1e-12, max_iter=500)
    ph = p.cpu().numpy()
    assert info.rel_res <= 1e-12
    assert abs(info.iters - it_o) <= 2, (info.iters, it_o)
    assert np.linalg.norm(ph - p_o) / np.linalg.norm(p_o) <= 1e-10
    assert abs(oracle.volume_mean(ph, g)) <= 1e-13 * np.max(np.abs(ph))
    # the oracle's variable-coefficient residual of the GPU's p
    r = f - oracle.volume_mean(f, g) - L.varcoef_apply(ph, c.rho, g)
    assert np.linalg.norm(r) <= 2e-12 * np.linalg.norm(f - oracle.volume_mean(f, g))


def test_split_fixed_point_on_gpu():
    """p_hat = p_ex: the GPU's split rhs + solve return p_ex, and correct gives the exactly
    projected velocity (divergence free)."""
    c = VC_CASES["emulsion32_r20"]()
    g = grid_of(c)
    d = {k: dev(c[k]) for k in ("u", "v", "w", "rho")}
    zero = torch.zeros_like(d["u"])
    f = torch.empty_like(zero)
    pex = torch.empty_like(zero)
    p = torch.empty_like(zero)
    with flups.Plan.for_case(c, "fp64") as plan:
        plan.set_density(d["rho"])
        plan.rhs(d["u"], d["v"], d["w"], zero, None, 0.0, 0.0, c.dt, f)
        plan.varcoef_solve(d["rho"], f, pex, rtol=1e-13, max_iter=500)
        plan.rhs(d["u"], d["v"], d["w"], pex, None, 1.0, 0.0, c.dt, f)
        plan.solve(f, p, rtol=0.0)
        plan.correct(p, pex, None, 1.0, 0.0, c.dt, d["u"], d["v"], d["w"])
    pe, ph = pex.cpu().numpy(), p.cpu().numpy()
    assert np.linalg.norm(ph - pe) / np.linalg.norm(pe) <= 1e-10
    div = oracle.div(d["u"].cpu().numpy(), d["v"].cpu().numpy(), d["w"].cpu().numpy(), g)
    assert np.max(np.abs(div)) <= 1e-9 * np.max(np.abs(oracle.div(c.u, c.v, c.w, g)))


def test_varcoef_requires_density():
    c = synth.sphere(16)
    x = dev(c.u)
    with flups.Plan.for_case(c, "fp64") as plan:
        st, _ = plan.varcoef_solve(x, x.clone(), torch.empty_like(x), check=False)
    assert st == flups.ESTATE


# ----------------------------------------------------------------- conv net

def net_inputs(shape, seed):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 19.0 * (rng.random(shape) > 0.6)
    pn = rng.standard_normal(shape)
    pnm1 = pn + 0.3 * rng.standard_normal(shape)
    pnext = 2.0 * pn - pnm1 + 0.2 * rng.standard_normal(shape)
    return rho, pn, pnm1, pnext


def rand_params(seed):
    p = learned.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    o = 0
    for cin, cout in learned.LAYERS:
        o += cout * cin * 27
        p[o:o + cout] = (0.1 * rng.standard_normal(cout)).astype(np.float32)
        o += cout
    p[o - 27 * 16 - 1:o - 1] *= 10.0        # a last layer of ordinary size
    return p


def oracle_layers(params):
    return [(L.bf16(w), b) for w, b in learned.split_params(params)]


def check_close(y_gpu, y_ref, what):
    scale = np.max(np.abs(y_ref))
    err = np.abs(y_gpu - y_ref)
    assert np.max(err) <= 4e-3 * scale, (what, np.max(err) / scale)
    assert np.mean(err) <= 1e-4 * scale, (what, np.mean(err) / scale)


# nx = 32: mma.sync kernels; nx = 64: mma.sync for the 16-channel layers, the row-pair tcgen05
# kernel for the output layer; nx = 128, 256: tcgen05 kernels (tensor-memory accumulators; z
# chunks of 4, 8 and 16 planes; at nz = 32 two chunks of 16 whose 18 input planes wrap the
# 8-slot ring twice)
@pytest.mark.parametrize("shape", [(8, 16, 32), (12, 8, 64), (4, 8, 128), (8, 8, 256), (32, 8, 128)])
def test_forward_matches_oracle(shape):
    rho, pn, pnm1, _ = net_inputs(shape, 5)
    params = rand_params(50)
    nz, ny, nx = shape
    ph = torch.empty(shape, dtype=torch.float64, device="cuda")
    with flups.PNet(nx, ny, nz, params) as net:
        net.predict(dev(rho), 1.0, dev(pn), dev(pnm1), ph)
        assert net.launches > 0
    x, s = L.features(rho, pn, pnm1, 1.0)
    y_o, _ = L.forward(oracle_layers(params), x, rnd=L.bf16)
    y_g = (ph.cpu().numpy() - (2.0 * pn - pnm1)) / s
    check_close(y_g, y_o[0], "y")


def test_zero_pressure_uses_unit_scale():
    shape = (4, 8, 32)
    rho, _, _, _ = net_inputs(shape, 6)
    z = np.zeros(shape)
    params = rand_params(51)
    ph = torch.empty(shape, dtype=torch.float64, device="cuda")
    with flups.PNet(32, 8, 4, params) as net:
        net.predict(dev(rho), 1.0, dev(z), dev(z), ph)
    y_o, _ = L.forward(oracle_layers(params), L.features(rho, z, z, 1.0)[0], rnd=L.bf16)
    check_close(ph.cpu().numpy(), y_o[0], "y")


@pytest.mark.parametrize("shape", [(8, 16, 32), (12, 8, 64), (4, 8, 128), (32, 8, 128)])
def test_gradients_match_oracle(shape):
    rho, pn, pnm1, pnext = net_inputs(shape, 7)
    params = rand_params(52)
    nz, ny, nx = shape
    with flups.PNet(nx, ny, nz, params) as net:
        loss = net.train_step(dev(rho), 1.0, dev(pn), dev(pnm1), dev(pnext), 0.0)
        grads = net.grads()
        assert np.array_equal(net.params(), params)            # lr = 0 leaves the weights alone
    loss_o, grads_o = L.loss_and_grads(oracle_layers(params), rho, pn, pnm1, pnext, 1.0, rnd=L.bf16)
    assert abs(loss - loss_o) <= 1e-3 * loss_o
    for li, (gw, gb) in enumerate(learned.split_params(grads)):
        ow, ob = grads_o[li]
        assert np.linalg.norm(gw - ow) <= 1e-2 * np.linalg.norm(ow), li
        assert np.linalg.norm(gb - ob) <= 1e-2 * np.linalg.norm(ob) + 1e-30, li
        # element by element: every weight and bias gradient within 2 % of the layer's largest
        # (bf16 operands rounded from FP32 on the GPU and from FP64 in the oracle can round
        # apart by one bf16 unit, 2^-8, at a few points; the sums over points are FP32 on the
        # GPU), and the mean difference a tenth of that
        for what, a, o in (("w", gw, ow), ("b", gb, ob)):
            scale = np.max(np.abs(o))
            d = np.abs(np.asarray(a, dtype=np.float64) - o)
            assert np.max(d) <= 2e-2 * scale + 1e-30, (li, what, np.max(d) / scale)
            assert np.mean(d) <= 2e-3 * scale + 1e-30, (li, what, np.mean(d) / scale)


def test_adam_steps_match_oracle():
    shape = (4, 8, 32)
    rho, pn, pnm1, pnext = net_inputs(shape, 8)
    params = rand_params(53)
    ref = params.astype(np.float64)
    m, v = np.zeros_like(ref), np.zeros_like(ref)
    lr = 1e-2
    with flups.PNet(32, 8, 4, params) as net:
        for step in (1, 2, 3):
            before = net.params().astype(np.float64)
            net.train_step(dev(rho), 1.0, dev(pn), dev(pnm1), dev(pnext), lr, want_loss=False)
            g = net.grads().astype(np.float64)
            L.adam_update(ref, g, m, v, step, lr)
            after = net.params().astype(np.float64)
            assert np.max(np.abs(after - ref)) <= 1e-5 * lr + 2e-7 * np.max(np.abs(before)), step
            ref = after.copy()                              # continue from the GPU's FP32 state


def test_checkpoint_resume_equals_uninterrupted_training(tmp_path):
    """Parameters, Adam moments and step count saved after two steps and restored into a fresh
    net (created with other weights) continue exactly like the uninterrupted run: the same
    losses and the same state, bit for bit."""
    shape = (4, 8, 32)
    batches = [tuple(dev(a) for a in net_inputs(shape, 60 + k)) for k in range(4)]
    params = rand_params(54)
    lr = 1e-2

    def step(net, b):
        rho, pn, pnm1, pnext = b
        return net.train_step(rho, 1.0, pn, pnm1, pnext, lr)

    with flups.PNet(32, 8, 4, params) as a:
        la = [step(a, b) for b in batches]
        pa, (ma, va, sa) = a.params(), a.adam_state()
    path = tmp_path / "ckpt.bin"
    with flups.PNet(32, 8, 4, params) as b:
        lb = [step(b, x) for x in batches[:2]]
        learned.save_checkpoint(b, path, meta={"lr": lr})
    arrays, meta = learned.load_checkpoint(path)
    assert meta["step"] == 2 and meta["lr"] == lr
    with flups.PNet(32, 8, 4, learned.init_params(99)) as c:
        learned.restore(c, arrays, meta)
        assert c.adam_state()[2] == 2
        lc = [step(c, x) for x in batches[2:]]
        pc, (mc, vc, sc) = c.params(), c.adam_state()
    assert lb == la[:2] and lc == la[2:]
    assert np.array_equal(pc, pa) and np.array_equal(mc, ma) and np.array_equal(vc, va)
    assert sa == sc == 4


def test_adam_state_rejects_invalid_moments():
    m = np.zeros(flups.PNET_NPARAMS, np.float32)
    v = np.zeros(flups.PNET_NPARAMS, np.float32)
    with flups.PNet(32, 8, 4, rand_params(55)) as net:
        for mm, vv, st in ((m, -np.ones_like(v), 1), (np.full_like(m, np.nan), v, 1), (m, v, -1)):
            with pytest.raises(flups.FlupsError) as e:
                net.set_adam_state(mm, vv, st)
            assert e.value.status == flups.EINVAL


@pytest.mark.slow
def test_fullsize_inference_sampled():
    """128^3 inference window (ratio 20, 50 droplets): 48 sampled outputs against the oracle."""
    rho, _, n, _ = synth.learned_window("infer", 0)
    rng = np.random.default_rng(12)
    pn = synth.smooth_noise(rng, n, 2.0)
    pnm1 = pn + 0.1 * synth.smooth_noise(rng, n, 2.0)
    params = rand_params(54)
    rho0 = float(rho.min())
    ph = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    with flups.PNet(n, n, n, params) as net:
        net.predict(dev(rho), rho0, dev(pn), dev(pnm1), ph)
    php = ph.cpu().numpy()
    s = float(np.sqrt(np.mean(pn * pn)))
    layers = oracle_layers(params)
    pts = rng.integers(0, n, size=(48, 3))
    # bias the sample towards droplet interfaces, where the density feature varies
    iface = np.argwhere((rho > 1.5) & (rho < 19.5))
    pts[:24] = iface[rng.integers(0, len(iface), 24)]
    yg, yo = [], []
    for k, j, i in pts:
        sl = np.ix_((np.arange(k - 4, k + 5)) % n, (np.arange(j - 4, j + 5)) % n, (np.arange(i - 4, i + 5)) % n)
        x, _ = L.features(rho[sl], pn[sl], pnm1[sl], rho0, s)
        y, _ = L.forward(layers, x, rnd=L.bf16)
        yo.append(y[0, 4, 4, 4])
        yg.append((php[k, j, i] - (2.0 * pn[k, j, i] - pnm1[k, j, i])) / s)
    check_close(np.array(yg), np.array(yo), "y128")


# ----------------------------------------------------------------- training

@pytest.mark.slow
def test_training_beats_linear_extrapolation():
    """64^3 windows of the learned workload: 3 windows x 8 steps for training, a held-out
    window for validation; after 300 Adam steps the learned p_hat has a lower loss and a
    lower splitting error than 2 p^n - p^{n-1} on the held-out window."""
    train_w = [learned.make_window("train", w, 8)[0] for w in range(3)]
    held, dt = learned.make_window("train", 3, 8, keep_velocity=True)
    with flups.PNet(64, 64, 64, learned.init_params()) as net:
        learned.train(net, train_w, 300, lr=2e-3)
        l_net, l_lin = learned.eval_losses(net, [held])
        assert l_net < 0.8 * l_lin, (l_net, l_lin)
        with flups.Plan(64, 64, 64, 1 / 64, 1 / 64, np.full(64, 1 / 64), "periodic", "fp64",
                        flups.current_stream()) as plan:
            plan.set_density(held.rho)
            res = learned.compare_predictors(net, held, dt, plan)
    e_net = np.mean([e[0] for e in res["net"]])
    e_lin = np.mean([e[0] for e in res["lin"]])
    assert e_net < e_lin, (e_net, e_lin)
