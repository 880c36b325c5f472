"""The stored oracle results (tests/golden/ctmrg_w<k>.json, which the GPU parity tests compare
against) are what the committed oracle computes now: the two small workloads (real D=2, chi=16;
complex D=3, chi=27) are recomputed by the golden script and compared checkpoint by checkpoint."""
import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _make_golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("k", [1, 6])
def test_stored_results_match_the_oracle(k):
    with open(os.path.join(HERE, "golden", f"ctmrg_w{k}.json")) as f:
        stored = json.load(f)
    now = _make_golden().compute(k)
    for key in ("d", "D", "chi", "moves", "seed", "n"):
        assert now[key] == stored[key], key
    assert sorted(now["checkpoints"]) == sorted(stored["checkpoints"])
    for m, snap in stored["checkpoints"].items():
        got = now["checkpoints"][m]
        assert got["energy"] == pytest.approx(snap["energy"], abs=1e-12), m
        np.testing.assert_allclose(got["rho_re"], snap["rho_re"], atol=1e-12, err_msg=m)
        np.testing.assert_allclose(got["rho_im"], snap["rho_im"], atol=1e-12, err_msg=m)
        np.testing.assert_allclose(got["corner_spectrum"], snap["corner_spectrum"], atol=1e-12, err_msg=m)
        if snap["s_err"] is not None:
            assert got["s_err"] == pytest.approx(snap["s_err"], abs=1e-12), m
    for g_now, g_st in zip(now["gaps"], stored["gaps"]):
        assert (g_now is None) == (g_st is None)
        if g_st is not None:
            assert g_now == pytest.approx(g_st, rel=1e-6, abs=1e-12)
