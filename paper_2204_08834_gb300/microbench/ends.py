"""Closed-box Poisson solve micro-benchmark: Neumann ends in x and y, z walls (tanh-stretched).

  python -m paper_2204_08834_gb300.microbench.ends [nx] [nz] [prec] [reps]

f ~ N(0,1) seeded; one warm-up solve, then `reps` solves timed with CUDA events.  prec is
"fp32_refine" (to rel. residual 1e-10) or "fp64".
"""

import sys

import numpy as np


def main(nx=256, nz=128, prec="fp32_refine", reps=2):
    import torch

    from paper_2204_08834_gb300 import flups, synth

    dzf = synth.stretched_dzf(nz, 1.0, 1.5)
    f = torch.from_numpy(np.random.default_rng(60).standard_normal((nz, nx, nx))).cuda()
    p = torch.empty_like(f)
    rtol = 1e-10 if prec == "fp32_refine" else 0.0
    with flups.Plan(nx, nx, nz, 2.0 / nx, 2.0 / nx, dzf, "walls", prec, flups.current_stream(), bcx="neumann",
                    bcy="neumann") as plan:
        info = plan.solve(f, p, rtol=rtol, max_iter=12)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            info = plan.solve(f, p, rtol=rtol, max_iter=12)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
    print(f"closed box {nx}x{nx}x{nz} {prec}: {ms:.4f} ms per solve, iters {info.iters}, rel_res {info.rel_res:.3g}")


if __name__ == "__main__":
    a = sys.argv[1:]
    main(int(a[0]) if a else 256, int(a[1]) if len(a) > 1 else 128, a[2] if len(a) > 2 else "fp32_refine",
         int(a[3]) if len(a) > 3 else 2)
