"""The stored golden fixtures (tests/golden/*.json, written by tests/golden/make_golden.py from
the FP64 oracle alone) against the oracle as it is now: any change to the oracle's arithmetic
shows up here, and must name the passage of the paper that justifies it."""

import glob
import importlib.util
import json
import os

import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
MG = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(MG)

FIXTURES = sorted(glob.glob(os.path.join(HERE, "*.json")))


def fresh():
    cases = {
        "projection_sphere8": lambda: MG.projection_case("projection_sphere8", lambda: MG.synth.sphere(8), ""),
        "projection_walls_stretched_8x6x5": lambda: MG.projection_case(
            "projection_walls_stretched_8x6x5", lambda: MG.synth.random_fields(8, 6, 5, "walls", True, seed=95), ""),
        "ends_ND_DN_6x8x4_walls": MG.ends_case,
        "momentum_solenoidal_8": MG.momentum_case,
        "learned_net_4x8x8": MG.learned_case,
    }
    return cases


def test_every_fixture_is_present_and_cites_its_passage():
    names = {os.path.basename(p)[:-5] for p in FIXTURES}
    assert names == set(fresh())
    for p in FIXTURES:
        d = json.load(open(p))
        assert d["generated_by"].startswith("tests/golden/make_golden.py")
        assert "Sec." in d["computes"] and d["inputs"]


@pytest.mark.parametrize("path", FIXTURES, ids=lambda p: os.path.basename(p)[:-5])
def test_oracle_reproduces_the_fixture(path):
    stored = json.load(open(path))
    now = fresh()[stored["case"]]()
    assert set(now["values"]) == set(stored["values"])
    for key, s in stored["values"].items():
        n = now["values"][key]
        assert n["idx"] == s["idx"], key
        scale = max(max(abs(x) for x in s["val"]), 1e-300)
        for a, b in zip(n["val"], s["val"]):
            assert abs(a - b) <= 1e-12 * scale, (key, a, b)
        assert abs(n["norm2"] - s["norm2"]) <= 1e-12 * s["norm2"], key
    for key, s in stored.get("scalars", {}).items():
        if key == "rel_residual":        # a round-off level number: only its size is fixed
            assert now["scalars"][key] <= 1e-13
        else:
            assert abs(now["scalars"][key] - s) <= 1e-12 * abs(s), key
