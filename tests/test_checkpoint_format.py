"""The array container behind net checkpoints and saved datasets (host logic, no GPU)."""

import struct

import numpy as np
import pytest

from paper_2204_08834_gb300 import learned


def test_round_trip_keeps_names_dtypes_shapes_values_and_meta(tmp_path):
    rng = np.random.default_rng(3)
    arrays = {"params": rng.standard_normal(15601).astype(np.float32),
              "w0/rho": rng.random((4, 3, 8)),
              "big": rng.standard_normal((2, 5)).astype(">f8"),     # big-endian in memory
              "empty": np.zeros((0, 3), np.float32)}
    meta = {"kind": "x", "step": 7, "lr": 1e-3, "windows": [{"rho0": 1.0, "steps": 3}]}
    path = tmp_path / "a.bin"
    learned.write_arrays(path, arrays, meta)
    got, m = learned.read_arrays(path)
    assert m == meta and list(got) == list(arrays)
    for k, a in arrays.items():
        assert got[k].shape == a.shape and got[k].dtype == a.dtype.newbyteorder("=")
        assert np.array_equal(got[k], a)


def test_file_is_little_endian_with_the_stated_header(tmp_path):
    path = tmp_path / "b.bin"
    learned.write_arrays(path, {"x": np.array([1.0, -2.5], np.float32)}, {"k": 1})
    raw = path.read_bytes()
    assert raw[:8] == learned.ARRAY_MAGIC
    (n,) = struct.unpack("<Q", raw[8:16])
    assert raw[16 + n:] == struct.pack("<2f", 1.0, -2.5)


def test_bad_files_are_rejected(tmp_path):
    good = tmp_path / "g.bin"
    learned.write_arrays(good, {"x": np.arange(10.0)}, {})
    raw = good.read_bytes()
    for name, data in (("magic", b"NOTFLUPS" + raw[8:]), ("short", raw[:12]), ("cut", raw[:-8])):
        p = tmp_path / f"{name}.bin"
        p.write_bytes(data)
        with pytest.raises(ValueError):
            learned.read_arrays(p)


def test_checkpoint_loader_checks_kind(tmp_path):
    p = tmp_path / "c.bin"
    learned.write_arrays(p, {"params": np.zeros(3, np.float32)}, {"kind": "learned-windows"})
    with pytest.raises(ValueError):
        learned.load_checkpoint(p)
