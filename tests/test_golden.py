"""The oracle reproduces its stored small-case outputs (CPU only).

tests/golden/oracle_small2d.json was written by tests/golden/make_golden.py, which calls
only the oracle.  The stored values also satisfy the dot-product test by themselves.
"""
import importlib.util
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    with open(os.path.join(HERE, "golden", "oracle_small2d.json")) as f:
        stored = json.load(f)
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return stored, mod


def _close(a, b, tol=1e-10):
    return abs(a - b) <= tol * max(abs(a), abs(b), 1e-300)


def test_stored_values_satisfy_the_dot_test():
    stored, _ = _load()
    a, b = stored["dot_Fdm_r"], stored["dot_dm_Fadj_r"]
    assert abs(a - b) / max(abs(a), abs(b)) < 1e-12


def test_oracle_reproduces_the_stored_values():
    stored, mod = _load()
    now = mod.compute()
    assert now["spec"] == stored["spec"]
    for key in ("born_norm", "hdm_norm", "dot_Fdm_r", "dot_dm_Fadj_r"):
        assert _close(now[key], stored[key]), key
    for s_now, s_old in zip(now["born_samples"] + now["hdm_samples"], stored["born_samples"] + stored["hdm_samples"]):
        assert s_now[:-1] == s_old[:-1] and _close(s_now[-1], s_old[-1]), (s_now, s_old)
