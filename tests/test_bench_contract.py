"""The bench's reference arm (the FP64 oracle, timed on the host cores) prints one JSON line
with the keys of the bench contract; it needs no GPU."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl")


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=900, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert all(k in d for k in KEYS), [k for k in KEYS if k not in d]
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    # the bench raises W to the contract's minimum of three untimed warm-up steps
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3 and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_solve_byte_accounting():
    # compulsory bytes per point of the FP32 solve's passes: with the binary32 first iterate the
    # first inverse writes 4 B instead of 8 and the first defect and update read 4 B of p instead
    # of 8 (the first defect also writes f's fixed point, 8 B); later launches of those kernels
    # keep the binary64 figures
    import types

    import numpy as np

    sys.path.insert(0, ROOT)
    import bench

    def case(nx, ny, nz, h, dzf=None):
        return types.SimpleNamespace(shape=(nz, ny, nx), dx=h, dy=h, dzf=np.full(nz, h) if dzf is None else dzf)

    assert bench.p32_first(case(512, 512, 512, 1 / 512))
    assert bench.p32_first(case(128, 8, 4, 1 / 128))
    assert not bench.p32_first(case(32, 16, 8, 1 / 32))              # M = 16: no register x rows
    assert not bench.p32_first(case(2048, 8, 8, 1 / 2048))           # M = 1024: no z-marching defect
    assert not bench.p32_first(case(512, 12, 8, 1 / 512))            # ny not a multiple of 8
    assert not bench.p32_first(case(512, 512, 4, 1 / 512, np.array([1, 2, 1, 2]) / 512))   # stretched z
    assert bench.solve_bytes_per_point("k_xinv32", 1.0, True) == 8
    assert bench.solve_bytes_per_point("k_xinv32", 1.0, False) == 12
    assert bench.solve_bytes_per_point("k_xfwd_residual32", 1.0, True) == 24
    assert bench.solve_bytes_per_point("k_xfwd_residual32", 2.0, True) == 22      # (24 + 20) / 2
    assert bench.solve_bytes_per_point("k_xinv_acc32", 1.0, True) == 16
    assert bench.solve_bytes_per_point("k_xinv_acc32", 3.0, True) == (16 + 2 * 20) / 3
    assert bench.solve_bytes_per_point("k_ycol32", 4.0, True) == 8
    # two FP32 solves with three defect passes (the bench's 512^3 solve): 124 B/point
    per_solve = {"k_xfwd_f32": 1, "k_xfwd_residual32": 1, "k_xres_norm32": 1, "k_ycol32": 4, "k_zper32": 2,
                 "k_xinv32": 1, "k_xinv_acc32": 1}
    total = sum(bench.solve_bytes_per_point(k, n, True) * n for k, n in per_solve.items())
    assert total == 124
