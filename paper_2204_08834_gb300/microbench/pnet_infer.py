"""Learned-p_hat inference micro-benchmark: flups_pnet_predict on an n^3 periodic grid.

  python -m paper_2204_08834_gb300.microbench.pnet_infer [n] [reps]

Random density (ratio 20) and pressures, He-initialised weights; prints the mean time of
one inference (CUDA events) and the per-kernel-group times.  n must be a multiple of 32.
"""

import sys

import numpy as np


def main(n=192, reps=3):
    import torch

    from paper_2204_08834_gb300 import flups, learned

    rng = np.random.default_rng(3)
    rho = torch.from_numpy(1.0 + 19.0 * (rng.random((n, n, n)) > 0.9)).cuda()
    pn = torch.from_numpy(rng.standard_normal((n, n, n))).cuda()
    pm = torch.from_numpy(rng.standard_normal((n, n, n))).cuda()
    ph = torch.empty_like(pn)
    with flups.PNet(n, n, n, learned.init_params()) as net:
        net.predict(rho, 1.0, pn, pm, ph)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            net.predict(rho, 1.0, pn, pm, ph)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        net.set_profiling(True)
        net.predict(rho, 1.0, pn, pm, ph)
        prof = net.profile()
    print(f"n={n} predict {ms:.4f} ms ({n ** 3 / ms / 1e3:.1f} Mpts/s); "
          + ", ".join(f"{k} {v[0]:.4f} ms" for k, v in prof.items()))


if __name__ == "__main__":
    main(*(int(a) for a in sys.argv[1:3]))
