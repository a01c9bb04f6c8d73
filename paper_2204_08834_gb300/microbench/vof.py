"""VoF step micro-benchmark (flups_vof_step: MTHINC reconstruction, split advection).

  python -m paper_2204_08834_gb300.microbench.vof [n] [steps]

An n^3 periodic box (unit length) of 30 droplets (r U[4,12] cells, tanh profile 1.5 cells
wide, seed 70) in the solenoidal velocity field of synth.solenoidal_velocity (seed 71) at CFL
0.5, beta_th = 2.  One warm-up step, then `steps` steps timed with CUDA events; prints the time
per step and the change of sum(phi).  With steps = 0 only the warm-up step runs.
"""

import json
import sys

import numpy as np


def droplets(n, count=30, seed=70):
    rng = np.random.default_rng(seed)
    x = np.arange(n) + 0.5
    phi = np.zeros((n, n, n))
    for _ in range(count):
        c = rng.uniform(0, n, 3)
        rad = rng.uniform(4.0, 12.0)
        dd = [np.minimum(np.abs(x - c[a]), n - np.abs(x - c[a])) for a in range(3)]
        r = np.sqrt(dd[0][None, None, :] ** 2 + dd[1][None, :, None] ** 2 + dd[2][:, None, None] ** 2)
        phi = np.maximum(phi, 0.5 * (1.0 - np.tanh((r - rad) / 0.75)))
    return phi


def main(n=256, steps=3):
    import torch

    from paper_2204_08834_gb300 import flups, synth

    h = 1.0 / n
    phi = torch.from_numpy(droplets(n)).cuda()
    vel = synth.solenoidal_velocity(n, seed=71)
    U = max(float(np.max(np.abs(q))) for q in vel)
    dt = 0.5 * h / U
    v = [torch.from_numpy(q).cuda() for q in vel]
    with flups.Plan(n, n, n, h, h, np.full(n, h), "periodic", "fp32_refine", flups.current_stream()) as plan:
        plan.vof_step(phi, *v, dt, 2.0)
        out = {"n": n, "steps": steps}
        if steps > 0:
            m0 = float(phi.sum())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                plan.vof_step(phi, *v, dt, 2.0)
            e1.record()
            torch.cuda.synchronize()
            out["ms_per_step"] = round(e0.elapsed_time(e1) / steps, 4)
            out["mass_rel_change"] = (float(phi.sum()) - m0) / m0
        plan.sync()
    print(json.dumps(out))


if __name__ == "__main__":
    a = sys.argv[1:]
    main(int(a[0]) if a else 256, int(a[1]) if len(a) > 1 else 3)
