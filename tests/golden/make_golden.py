"""Writes the golden fixtures of this folder from the FP64 oracle alone: oracle/ for every value,
the seeded input generators (paper_2204_08834_gb300.synth, numpy's PCG64) for the inputs, and
nothing from the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py

Each fixture is a small JSON text file: how its inputs are generated, the oracle function and
the passage of the paper it follows, and the values at fixed sample positions (flat C-order
indices of the [nz][ny][nx] arrays) plus a few whole-array norms.  tests/test_golden.py
recomputes them and fails if the oracle has drifted.
"""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import learned as OL  # noqa: E402
from oracle import momentum as OM  # noqa: E402
from oracle import r2r as OR  # noqa: E402
from paper_2204_08834_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
NSAMPLES = 12


def samples(a, seed):
    idx = np.random.default_rng(seed).choice(a.size, size=min(NSAMPLES, a.size), replace=False)
    idx = np.sort(idx)
    return {"idx": [int(i) for i in idx], "val": [float(a.ravel()[i]) for i in idx], "norm2": float(np.linalg.norm(a))}


def grid_of(c):
    nz, ny, nx = c.shape
    return oracle.make_grid(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc)


def projection_case(name, make, inputs):
    c = make()
    g = grid_of(c)
    f, p, u1, v1, w1 = oracle.project(c.u, c.v, c.w, c.rho, c.pn, c.pnm1, 2.0, 1.0, c.dt, g)
    return {"case": name, "inputs": inputs,
            "computes": "oracle.project with c1 = 2, c2 = 1: f (Eqs. us_predic + poisson), p (the Sec. 3.3.1 "
                        "direct solve of L p = f - <f>, <p> = 0), u, v, w at t^{n+1} (Eq. corr)",
            "values": {"f": samples(f, 1), "p": samples(p, 2), "u1": samples(u1, 3), "v1": samples(v1, 4),
                       "w1": samples(w1, 5)},
            "scalars": {"rho0": oracle.min_density(c.rho), "rel_residual": oracle.rel_residual(f, p, g)}}


def ends_case():
    nx, ny, nz = 6, 8, 4
    f = np.random.default_rng(70).standard_normal((nz, ny, nx))
    g = oracle.make_grid(nx, ny, nz, 0.3, 0.2, np.array([0.2, 0.3, 0.25, 0.15]), "walls")
    out = {"case": "ends_ND_DN_6x8x4_walls",
           "inputs": "f = numpy default_rng(70).standard_normal((4, 8, 6)); dx 0.3, dy 0.2, z walls with "
                     "dzf (0.2, 0.3, 0.25, 0.15); x ends Neumann-low/Dirichlet-high, y ends Dirichlet/Neumann",
           "computes": "oracle.r2r.solve: L p = f with homogeneous Neumann/Dirichlet ends (Sec. 3.3.1 "
                       "eigen-expansion with cosine/sine series; readings E1-E4)",
           "values": {"p": samples(OR.solve(f, g, "ND", "DN"), 6), "p_NN_DD": samples(OR.solve(f, g, "NN", "DD"), 7)}}
    return out


def momentum_case():
    u, v, w = synth.solenoidal_velocity(8, seed=51)
    h = 1.0 / 8
    gvec = (0.0, 0.0, -1.0)
    (u1, v1, w1), m0 = OM.predictor(u, v, w, None, 1e-2, gvec, 2e-3, None, h, h, h)
    (u2, v2, w2), m1 = OM.predictor(u1, v1, w1, m0, 1e-2, gvec, 2e-3, 3e-3, h, h, h)
    return {"case": "momentum_solenoidal_8",
            "inputs": "synth.solenoidal_velocity(8, seed=51); nu 1e-2, g (0, 0, -1), h 1/8; a forward-Euler "
                      "step of dt 2e-3, then an AB2 step of dt 2e-3 after dt_prev 3e-3",
            "computes": "oracle.momentum.predictor (Sec. 3.3 Eq. uss_predic with the AB2 weights of Sec. 3.2; "
                        "readings M1-M4): u** of both steps and M of the second",
            "values": {"u1": samples(u1, 8), "w1": samples(w1, 9), "u2": samples(u2, 10), "v2": samples(v2, 11),
                       "w2": samples(w2, 12), "Mu": samples(m1[0], 13), "Mw": samples(m1[2], 14)}}


def learned_case():
    rng = np.random.default_rng(80)
    shape = (4, 8, 8)
    rho = 1.0 + 19.0 * (rng.random(shape) > 0.7)
    pn = rng.standard_normal(shape)
    pnm1 = pn + 0.3 * rng.standard_normal(shape)
    pnext = 2.0 * pn - pnm1 + 0.2 * rng.standard_normal(shape)
    layers = []
    for cin, cout in ((3, 16), (16, 16), (16, 16), (16, 1)):
        layers.append((rng.standard_normal((cout, cin, 27)) * np.sqrt(2.0 / (27 * cin)),
                       0.1 * rng.standard_normal(cout)))
    ph = OL.predict(layers, rho, pn, pnm1, 1.0)
    loss, grads = OL.loss_and_grads(layers, rho, pn, pnm1, pnext, 1.0)
    return {"case": "learned_net_4x8x8",
            "inputs": "numpy default_rng(80): rho = 1 + 19 (U > 0.7), p^n ~ N(0,1), p^{n-1} = p^n + 0.3 N, "
                      "p^{n+1} = 2 p^n - p^{n-1} + 0.2 N, then the four layers' weights N * sqrt(2/(27 in)) "
                      "and biases 0.1 N, drawn in that order",
            "computes": "oracle.learned.predict and loss_and_grads in FP64 (not in the paper: a learned "
                        "correction to the p_hat extrapolation of Sec. 3.3; readings L2, L3): p_hat, the loss "
                        "and the first layer's weight gradient",
            "values": {"p_hat": samples(ph, 15), "dW1": samples(grads[0][0], 16)},
            "scalars": {"loss": loss}}


def main():
    cases = [
        projection_case("projection_sphere8", lambda: synth.sphere(8),
                        "synth.sphere(8): one sphere of density 10 in 1, periodic unit box, u** and p ~ U[-1, 1]"),
        projection_case("projection_walls_stretched_8x6x5",
                        lambda: synth.random_fields(8, 6, 5, "walls", True, seed=95),
                        "synth.random_fields(8, 6, 5, 'walls', stretched=True, seed=95)"),
        ends_case(), momentum_case(), learned_case(),
    ]
    for c in cases:
        c["generated_by"] = "tests/golden/make_golden.py (FP64 oracle only)"
        with open(os.path.join(HERE, c["case"] + ".json"), "w") as fh:
            json.dump(c, fh, indent=1, sort_keys=True)
            fh.write("\n")
        print("wrote", c["case"])


if __name__ == "__main__":
    main()
