"""Momentum-predictor micro-benchmark: flups_momentum_predict on an n^3 periodic grid.

  python -m paper_2204_08834_gb300.microbench.momentum [n] [reps] [arith]

Solenoidal random velocity (rms 1), nu = 1e-3, dt at CFL 0.5; one Euler call to fill the
M state, then `reps` AB2 calls timed with CUDA events.  arith: "pair" (default) or "fp64".
"""

import sys

import numpy as np


def main(n=256, reps=3, arith="pair"):
    import torch

    from paper_2204_08834_gb300 import flups, synth

    h = 1.0 / n
    vel = synth.solenoidal_velocity(n, seed=50)
    dt = 0.5 * h / max(float(np.max(np.abs(q))) for q in vel)
    d = [torch.from_numpy(q).cuda() for q in vel]
    o = [torch.empty_like(d[0]) for _ in range(3)]
    st = flups.momentum_state(n, n, n)
    a = flups.MOM_PAIR if arith == "pair" else flups.MOM_FP64
    with flups.Plan(n, n, n, h, h, h, "periodic", "fp32_refine", flups.current_stream()) as plan:
        plan.momentum_predict(*d, *o, st, 1e-3, (0.0, 0.0, -1.0), dt, 0.0, a)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.momentum_predict(*d, *o, st, 1e-3, (0.0, 0.0, -1.0), dt, dt, a)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
    print(f"n={n} arith={arith} predictor {ms:.4f} ms ({n ** 3 / ms / 1e3:.1f} Mpts/s)")


if __name__ == "__main__":
    args = sys.argv[1:]
    main(int(args[0]) if args else 256, int(args[1]) if len(args) > 1 else 3, args[2] if len(args) > 2 else "pair")
