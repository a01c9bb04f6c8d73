"""The C ABI library (CPU-only checks): it builds, loads, exports every entry point that
include/flups.h declares, and rejects bad arguments before touching the GPU."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2204_08834_gb300 import build, flups

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return flups.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "flups.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(flups_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(flups.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for s in range(9):
        assert flups.status_string(s).startswith("FLUPS_")
    assert "unknown" in flups.status_string(99)


def _create(lib, nx, ny, nz, dzf, bc=0, prec=1, dx=0.1, dy=0.1):
    h = ctypes.c_void_p()
    dz = np.ascontiguousarray(np.broadcast_to(np.asarray(dzf, float), (max(nz, 1),)))
    st = lib.flups_plan_create(ctypes.byref(h), nx, ny, nz, dx, dy,
                               dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), bc, prec, None)
    return st, h


@pytest.mark.parametrize("nx,ny,nz,bc,want", [
    (12, 16, 16, 0, flups.EUNSUPPORTED),   # nx = 3*4: radix-3 sizes start at 24
    (16, 4, 16, 0, flups.EUNSUPPORTED),    # ny below 8
    (16, 16, 40, 0, flups.EUNSUPPORTED),   # periodic nz must be 2^a or 3*2^a
    (20, 16, 16, 0, flups.EUNSUPPORTED),   # nx = 5*4
    (16, 16, 1, 1, flups.EUNSUPPORTED),    # walls need nz >= 2
    (8192, 16, 16, 0, flups.EUNSUPPORTED),
    (16, 16, 16, 7, flups.EINVAL),         # unknown bc
])
def test_plan_rejects_bad_sizes(lib, nx, ny, nz, bc, want):
    st, h = _create(lib, nx, ny, nz, 1.0 / max(nz, 1), bc=bc)
    assert st == want and not h.value


def test_plan_rejects_bad_spacing(lib):
    assert _create(lib, 16, 16, 16, 0.1, dx=0.0)[0] == flups.EINVAL
    assert _create(lib, 16, 16, 16, 0.1, dy=float("nan"))[0] == flups.EINVAL
    assert _create(lib, 16, 16, 16, [0.1] * 15 + [-0.1], bc=1)[0] == flups.EINVAL
    assert _create(lib, 16, 16, 16, np.linspace(0.05, 0.1, 16), bc=0)[0] == flups.EINVAL  # periodic, stretched
    assert _create(lib, 16, 16, 16, 0.1, prec=5)[0] == flups.EINVAL
    h = ctypes.c_void_p()
    assert lib.flups_plan_create(ctypes.byref(h), 16, 16, 16, 0.1, 0.1, None, 0, 0, None) == flups.EINVAL
    assert lib.flups_plan_create(None, 16, 16, 16, 0.1, 0.1, None, 0, 0, None) == flups.EINVAL


def test_null_plan_calls_are_rejected(lib):
    assert lib.flups_plan_destroy(None) == flups.EINVAL
    assert lib.flups_set_density(None, None, 0.0) == flups.EINVAL
    assert lib.flups_solve(None, None, None, 1e-10, 4, None) == flups.EINVAL
    assert lib.flups_rhs(None, None, None, None, None, None, 2.0, 1.0, 1e-3, None) == flups.EINVAL
    assert lib.flups_correct(None, None, None, None, 2.0, 1.0, 1e-3, None, None, None) == flups.EINVAL
    assert lib.flups_workspace_bytes(None) == 0


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(flups, "_lib", None)
    monkeypatch.setattr(flups, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        flups.lib()


def test_pnet_create_rejects_bad_sizes_and_params(lib):
    """Size and parameter checks of flups_pnet_create happen before any GPU work."""
    params = np.zeros(flups.PNET_NPARAMS, np.float32)
    pp = params.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    h = ctypes.c_void_p()
    for nx, ny, nz in ((16, 8, 4), (48, 8, 4), (32, 12, 4), (32, 8, 6), (32, 8, 2)):
        assert lib.flups_pnet_create(ctypes.byref(h), nx, ny, nz, pp, None) == flups.EUNSUPPORTED, (nx, ny, nz)
    assert lib.flups_pnet_create(ctypes.byref(h), 32, 8, 4, None, None) == flups.EINVAL
    bad = params.copy()
    bad[7] = np.nan
    assert lib.flups_pnet_create(ctypes.byref(h), 32, 8, 4, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                 None) == flups.EINVAL
    assert lib.flups_pnet_create(None, 32, 8, 4, pp, None) == flups.EINVAL


def test_null_handles_are_rejected(lib):
    assert lib.flups_varcoef_solve(None, None, None, None, 1e-12, 10, None) == flups.EINVAL
    for fn in ("flups_pnet_destroy", "flups_pnet_set_profiling"):
        args = (None,) if fn == "flups_pnet_destroy" else (None, 1)
        assert getattr(lib, fn)(*args) == flups.EINVAL
    assert lib.flups_pnet_predict(None, None, 1.0, None, None, None) == flups.EINVAL
    assert lib.flups_pnet_launch_count(None) == 0
    assert lib.flups_pnet_get_adam(None, None, None, None) == flups.EINVAL
    assert lib.flups_pnet_set_adam(None, None, None, 0) == flups.EINVAL
    assert lib.flups_pnet_kernel_name(99).decode() == "unknown"
    assert lib.flups_selftest_wait_timeout(None, 0) == flups.EINVAL


def test_plan_with_ends_rejects_bad_ends(lib):
    h = ctypes.c_void_p()
    dz = np.full(16, 0.1)
    for bcx, bcy in ((5, 0), (0, -1), (9, 9)):
        st = lib.flups_plan_create_bc(ctypes.byref(h), 16, 16, 16, 0.1, 0.1,
                                      dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), bcx, bcy, 0, 1, None)
        assert st == flups.EINVAL
        assert not h.value


def test_momentum_predict_rejects_null_plan(lib):
    assert lib.flups_momentum_predict(None, None, None, None, None, None, None, None, 0.01, 0.0, 0.0, 0.0,
                                      1e-3, 0.0, 0) == flups.EINVAL
