import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# measured errors of the parity tests: (test id, key, error, bound), reported at the end of the run
_MEASURED = []


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libfm.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def synth():
    from paper_2504_07090_gb300 import synth as s
    return s


@pytest.fixture
def check_err(request):
    """check_err(err, bound, key): record a measured relative error under `key`
    ("<form> <quantity> <precision>"), then assert it is below its bound."""
    def _check(err, bound, key, case=""):
        _MEASURED.append((request.node.nodeid, key, case, float(err), float(bound)))
        assert err < bound, f"{key} [{case}]: measured {err:.3e}, bound {bound:.1e}"
        return err
    return _check


def pytest_terminal_summary(terminalreporter):
    """One line per (form, quantity, precision): the largest measured error, its case and the
    bound it was held to; the full list goes to $FM_ERR_LOG (JSON lines) when that is set."""
    if not _MEASURED:
        return
    agg = {}
    for nodeid, key, case, err, bound in _MEASURED:
        a = agg.setdefault(key, [0.0, "", bound, 0])
        if err >= a[0]:
            a[0], a[1] = err, case
        a[2] = max(a[2], bound)
        a[3] += 1
    tr = terminalreporter
    tr.write_sep("-", "measured relative errors vs the FP64 oracle (max over cases)")
    for key in sorted(agg):
        e, c, b, n = agg[key]
        tr.write_line(f"{key:<40s} max {e:.2e} ({c}; bound {b:.0e}; {n} checks)")
    path = os.environ.get("FM_ERR_LOG")
    if path:
        with open(path, "w") as fh:
            for nodeid, key, case, err, bound in _MEASURED:
                fh.write(json.dumps({"test": nodeid, "key": key, "case": case, "err": err, "bound": bound}) + "\n")
