"""Mixed-size ensemble micro-benchmark: flups_batch_solve of the 64-member ensemble.

  python -m paper_2204_08834_gb300.microbench.ensemble [reps]

The members of synth.ensemble_member (sizes {32, 48, 64, 96, 128}^3, periodic for even m, z walls
for odd m), right-hand sides by the oracle's rhs of each member's fields; one captured solve
(rtol 1e-10, at most 3 FP32 solves), then `reps` graph replays timed with CUDA events.  With
reps = 0 only the capture and first launch run (a short command for profilers).
"""

import json
import sys


def main(reps=5):
    import torch

    import oracle
    from paper_2204_08834_gb300 import flups, synth

    cases = [synth.ensemble_member(m) for m in range(64)]
    fs = []
    for c in cases:
        nz, ny, nx = c.shape
        g = oracle.make_grid(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc)
        fs.append(torch.from_numpy(oracle.rhs(c.u, c.v, c.w, c.rho, c.pn, c.pnm1, 2.0, 1.0, c.dt, g)).cuda())
    ps = [torch.empty_like(f) for f in fs]
    specs = [(c.shape[2], c.shape[1], c.shape[0], c.dx, c.dy, c.dzf, c.bc) for c in cases]
    pts = sum(c.npts for c in cases)
    with flups.Batch(specs, nstreams=8, autotune=False) as b:
        infos = b.solve(fs, ps, rtol=1e-10, max_iter=3)
        out = {"members": len(cases), "points": pts, "graph_kernels": int(b.graph_kernels),
               "max_rel_res": max(i.rel_res for i in infos)}
        if reps > 0:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                b.solve(fs, ps, rtol=1e-10, max_iter=3, info=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out["ms_per_launch"] = round(ms, 4)
            out["mpts_per_s"] = round(pts / ms / 1e3, 1)
        torch.cuda.synchronize()
    print(json.dumps(out))


if __name__ == "__main__":
    main(*(int(a) for a in sys.argv[1:2]))
