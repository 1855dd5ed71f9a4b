"""The oracle reproduces its stored regression fixture (see
tests/golden/README.md: a guard against unintended changes of its
arithmetic, not an independent pin)."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_its_regression_fixture():
    spec = importlib.util.spec_from_file_location("mk", os.path.join(HERE, "golden", "make_oracle_regression.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(HERE, "golden", "oracle_regression.json")) as f:
        ref = json.load(f)
    got = mk.compute()
    for k in ("energy", "gradient", "q1", "qdot1"):
        a, b = np.array(got[k]), np.array(ref[k])
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(b).max(), err_msg=k)
    assert got["n_active"] == ref["n_active"] > 0
