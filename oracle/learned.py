"""Oracle for the learned splitting pressure (test infrastructure only).

Two plain FP64 pieces:

* The exact variable-coefficient pressure the split method approximates (Sec. 3.3: the
  split replaces 1/rho by 1/rho0 plus a correction built from p_hat).  p_ex solves
      A p = D((rho0/rho_f) G p) = f,   <p>_V = 0,
  with f = (rho0/dt) D u** (the split right-hand side without the p_hat term), by
  preconditioned conjugate gradients in the volume-weighted inner product; the
  preconditioner is the constant-coefficient direct solve L^{-1} (rho0/rho_f <= 1, so
  L^{-1} A is well conditioned).  With p_hat = p_ex the split solve returns p_ex
  (the Dodd-Ferrante fixed point), so ||p_split(p_hat) - p_ex|| measures the splitting error
  of a predicted p_hat.
* A small periodic 3-D convolutional net (3x3x3 kernels, ReLU between layers) that maps
  (1 - rho0/rho, p^n/s, p^{n-1}/s) to a correction y, p_hat = 2 p^n - p^{n-1} + s y with
  s = rms(p^n): forward, backward (explicit chain rule) and the Adam update, in FP64.
  The density feature 1 - rho0/rho is the coefficient the split puts in front of G p_hat.
  An optional rounding function `rnd` is applied where a reduced-precision implementation
  stores values: each layer's input (features, hidden activations) on the way forward and
  each layer's output gradient on the way back; with rnd=None everything stays FP64.
* The splitting error of a p_hat (the measure the linear extrapolation is judged by):
  e_p = ||p_split - p_ex|| / ||p_ex||, e_u = ||u_split - u_ex|| / ||u_ex|| and, relative to
  the size of the pressure correction, e_du = ||u_split - u_ex|| / ||u_ex - u**||, with
  u_ex = u** - (dt/rho_f) G p_ex the exactly projected velocity.

Parity of the learned predictor with the paper is unpinned: the paper has no learned p_hat.
"""

import numpy as np

from .projection import correct, div, face_density, grad, min_density, rhs, solve, volume_mean


# ------------------------------------------------------- variable-coefficient solve

def varcoef_apply(p, rho, g, rho0=None):
    """A p = D((rho0/rho_f) G p); the top wall face carries no flux (G_z = 0 there)."""
    if rho0 is None:
        rho0 = min_density(rho)
    gx, gy, gz = grad(p, g)
    rx, ry, rz = face_density(rho, g)
    return div(rho0 / rx * gx, rho0 / ry * gy, rho0 / rz * gz, g)


def wdot(a, b, g):
    """Volume-weighted inner product sum(dzf a b); A is symmetric in it."""
    return float(np.sum(g.dzf[:, None, None] * a * b))


def varcoef_solve(f, rho, g, rtol=1e-12, maxit=500):
    """PCG for A p = f - <f>_V, <p>_V = 0, preconditioner M^{-1} r = L^{-1} r (c13 reading).

    Returns (p, iterations, relative residual ||r||_w / ||f - <f>||_w)."""
    rho0 = min_density(rho)
    b = f - volume_mean(f, g)
    nb = np.sqrt(wdot(b, b, g))
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = solve(r, g)
    d = z.copy()
    rz = wdot(r, z, g)
    for it in range(1, maxit + 1):
        q = varcoef_apply(d, rho, g, rho0)
        alpha = rz / wdot(d, q, g)
        x += alpha * d
        r -= alpha * q
        rel = np.sqrt(wdot(r, r, g)) / nb
        if rel <= rtol:
            return x - volume_mean(x, g), it, rel
        z = solve(r, g)
        rz_new = wdot(r, z, g)
        d = z + (rz_new / rz) * d
        rz = rz_new
    return x - volume_mean(x, g), maxit, rel


# ----------------------------------------------------------------------- conv net

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x, dz, dy, dx):
    """s[..., k, j, i] = x[..., k+dz, j+dy, i+dx] (periodic)."""
    return np.roll(x, (-dz, -dy, -dx), axis=(-3, -2, -1))


def conv3(x, w, b):
    """y[o] = b[o] + sum_{i, tap} w[o, i, tap] x[i](v + tap) with x (Cin, nz, ny, nx),
    w (Cout, Cin, 27) in TAPS order (dz slowest, dx fastest)."""
    y = np.broadcast_to(b[:, None, None, None], (w.shape[0],) + x.shape[1:]).astype(np.float64).copy()
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += np.einsum("oi,izyx->ozyx", w[:, :, t], shift(x, dz, dy, dx))
    return y


def conv3_back(x, w, dy_):
    """Gradients of conv3: (dx, dw, db) for upstream gradient dy_ (Cout, nz, ny, nx)."""
    dx = np.zeros_like(x, dtype=np.float64)
    dw = np.zeros_like(w, dtype=np.float64)
    for t, (dz, dyy, dxx) in enumerate(TAPS):
        xs = shift(x, dz, dyy, dxx)
        dw[:, :, t] = np.einsum("ozyx,izyx->oi", dy_, xs)
        # y(v) gets x(v + tap): x(u) feeds y(u - tap)
        dx += np.einsum("oi,ozyx->izyx", w[:, :, t], shift(dy_, -dz, -dyy, -dxx))
    db = dy_.sum(axis=(1, 2, 3))
    return dx, dw, db


def bf16(a):
    """Round to the nearest bfloat16 (8 significant bits), ties to even, straight from FP64."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def _id(a):
    return a


def features(rho, pn, pnm1, rho0, s=None):
    """Net input and its scale s = rms(p^n) (1 when p^n = 0); s may be given (a patch of a
    larger field uses the field's s)."""
    if s is None:
        s = float(np.sqrt(np.mean(pn * pn)))
        s = s if s > 0.0 else 1.0
    return np.stack([1.0 - rho0 / rho, pn / s, pnm1 / s]), s


def forward(params, x, rnd=None):
    """params: list of (w, b); ReLU after every layer except the last.
    Returns (y, acts) with acts[l] the (rounded) input of layer l."""
    rnd = rnd or _id
    acts = []
    a = x
    for li, (w, b) in enumerate(params):
        a = rnd(a)
        acts.append(a)
        a = conv3(a, w, b)
        if li < len(params) - 1:
            a = np.maximum(a, 0.0)
    return a, acts


def backward(params, acts, dy_, rnd=None):
    """Gradients (dw, db) per layer for the upstream gradient dy_ of the last layer's output;
    the gradient of each layer's output is rounded by rnd before it is used."""
    rnd = rnd or _id
    grads = [None] * len(params)
    g = dy_
    for li in range(len(params) - 1, -1, -1):
        w, b = params[li]
        if li < len(params) - 1:
            g = g * (acts[li + 1] > 0.0)
        g = rnd(g)
        dx, dw, db = conv3_back(acts[li], w, g)
        grads[li] = (dw, db)
        g = dx
    return grads


def predict(params, rho, pn, pnm1, rho0, rnd=None, s=None):
    """p_hat = 2 p^n - p^{n-1} + s y(features)."""
    x, s = features(rho, pn, pnm1, rho0, s)
    y, _ = forward(params, x, rnd)
    return 2.0 * pn - pnm1 + s * y[0]


def loss_and_grads(params, rho, pn, pnm1, ptarget, rho0, rnd=None):
    """MSE between y and the scaled correction (ptarget - (2 p^n - p^{n-1}))/s."""
    x, s = features(rho, pn, pnm1, rho0)
    y, acts = forward(params, x, rnd)
    t = (ptarget - (2.0 * pn - pnm1)) / s
    e = y[0] - t
    n = e.size
    loss = float(np.mean(e * e))
    dy_ = (2.0 / n) * e[None]
    return loss, backward(params, acts, dy_, rnd)


def adam_update(param, grad_, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba), in place; step counts from 1."""
    m *= b1
    m += (1.0 - b1) * grad_
    v *= b2
    v += (1.0 - b2) * grad_ * grad_
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    param -= lr * mh / (np.sqrt(vh) + eps)


# ------------------------------------------------------------------ splitting error

def split_error(u, v, w, rho, p_hat, dt, g, p_ex=None):
    """(e_p, e_u, e_du, p_split, p_ex) for the split projection with predictor p_hat."""
    rho0 = min_density(rho)
    z = np.zeros_like(p_hat)
    if p_ex is None:
        f0 = rhs(u, v, w, rho, z, z, 0.0, 0.0, dt, g, rho0)
        p_ex, _, _ = varcoef_solve(f0, rho, g, rtol=1e-13)
    f = rhs(u, v, w, rho, p_hat, z, 1.0, 0.0, dt, g, rho0)
    ps = solve(f, g)
    us = correct(u, v, w, ps, p_hat, z, rho, 1.0, 0.0, dt, g)
    ue = correct(u, v, w, p_ex, p_ex, z, rho, 1.0, 0.0, dt, g)
    e_p = np.linalg.norm(ps - p_ex) / np.linalg.norm(p_ex)
    num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(us, ue))
    den_u = sum(np.linalg.norm(a) ** 2 for a in ue)
    den_du = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(ue, (u, v, w)))
    return float(e_p), float(np.sqrt(num / den_u)), float(np.sqrt(num / den_du)), ps, p_ex
