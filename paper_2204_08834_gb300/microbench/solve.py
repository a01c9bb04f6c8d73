"""Poisson solve micro-benchmark on one grid, x and y periodic (the kernels of flups_solve).

  python -m paper_2204_08834_gb300.microbench.solve NXxNYxNZ[xwalls] [prec] [reps]

f ~ N(0,1) seeded on a unit-spacing-per-cell grid (h = 1/nx in x, y and, periodic, z; walls:
tanh-stretched z with beta 1.5 over a unit height); one warm-up solve, then `reps` solves
timed with CUDA events, printed with the library's per-kernel times of one more solve.  prec
is "fp32_refine" (to rel. residual 1e-10) or "fp64".  With reps = 0 only the warm-up solve
runs (a short command for profilers).
"""

import json
import sys

import numpy as np


def main(spec="512x256x512", prec="fp32_refine", reps=3):
    import torch

    from paper_2204_08834_gb300 import flups, synth

    a = spec.split("x")
    nx, ny, nz = int(a[0]), int(a[1]), int(a[2])
    bc = a[3] if len(a) > 3 else "periodic"
    h = 1.0 / nx
    dzf = synth.stretched_dzf(nz, 1.0, 1.5) if bc == "walls" else np.full(nz, h)
    f = torch.from_numpy(np.random.default_rng(61).standard_normal((nz, ny, nx))).cuda()
    p = torch.empty_like(f)
    rtol = 1e-10 if prec == "fp32_refine" else 0.0
    with flups.Plan(nx, ny, nz, h, h, dzf, bc, prec, flups.current_stream()) as plan:
        info = plan.solve(f, p, rtol=rtol, max_iter=12)
        out = {"grid": [nx, ny, nz], "bc": bc, "prec": prec, "iters": info.iters, "rel_res": info.rel_res}
        if reps > 0:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                plan.solve(f, p, rtol=rtol, max_iter=12)
            e1.record()
            torch.cuda.synchronize()
            out["ms_per_solve"] = round(e0.elapsed_time(e1) / reps, 4)
            plan.set_profiling(True)
            plan.solve(f, p, rtol=rtol, max_iter=12)
            out["kernels_ms"] = {k: round(ms, 4) for k, (ms, n) in plan.profile().items()}
            plan.set_profiling(False)
        torch.cuda.synchronize()
    print(json.dumps(out))


if __name__ == "__main__":
    args = sys.argv[1:]
    main(args[0] if args else "512x256x512", args[1] if len(args) > 1 else "fp32_refine",
         int(args[2]) if len(args) > 2 else 3)
