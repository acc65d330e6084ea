"""The oracle still reproduces its committed regression fixture (tests/golden)."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_regression_fixture():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    now = mg.compute()
    with open(os.path.join(HERE, "golden", "oracle_tiny.json")) as fh:
        ref = json.load(fh)
    for k, v in ref.items():
        if isinstance(v, str):
            continue
        np.testing.assert_allclose(np.asarray(now[k]), np.asarray(v), rtol=1e-12, atol=1e-300, err_msg=k)
