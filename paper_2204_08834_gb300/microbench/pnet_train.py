"""Learned-p_hat training micro-benchmark: flups_pnet_train_step on an n^3 periodic grid.

  python -m paper_2204_08834_gb300.microbench.pnet_train [n] [reps]

Random density (ratio 20) and pressures, He-initialised weights; one warm-up step, then `reps`
Adam steps (learning rate 1e-3, no loss read back) timed with CUDA events, printed with the
per-kernel-group times of one more step.  n must be a multiple of 32; with reps = 0 only the
warm-up step runs (a short command for profilers).
"""

import sys

import numpy as np


def main(n=64, reps=20):
    import torch

    from paper_2204_08834_gb300 import flups, learned

    rng = np.random.default_rng(4)
    rho = torch.from_numpy(1.0 + 19.0 * (rng.random((n, n, n)) > 0.9)).cuda()
    pn = torch.from_numpy(rng.standard_normal((n, n, n))).cuda()
    pm = torch.from_numpy(rng.standard_normal((n, n, n))).cuda()
    pnext = torch.from_numpy(rng.standard_normal((n, n, n))).cuda()
    with flups.PNet(n, n, n, learned.init_params()) as net:
        loss = net.train_step(rho, 1.0, pn, pm, pnext, 1e-3)
        out = f"n={n} loss {loss:.5f}"
        if reps > 0:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                net.train_step(rho, 1.0, pn, pm, pnext, 1e-3, want_loss=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            net.set_profiling(True)
            net.train_step(rho, 1.0, pn, pm, pnext, 1e-3, want_loss=False)
            prof = net.profile()
            out += (f" train step {ms:.4f} ms ({n ** 3 / ms / 1e3:.1f} Mpts/s); "
                    + ", ".join(f"{k} {v[0]:.4f} ms" for k, v in prof.items()))
        torch.cuda.synchronize()
    print(out)


if __name__ == "__main__":
    main(*(int(a) for a in sys.argv[1:3]))
