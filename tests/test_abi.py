"""libfm.so builds, loads and exports every entry point include/fm.h declares (no GPU
needed); argument validation rejects bad input before touching the device."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fm.h")).read()
    return sorted(set(re.findall(r"^FM_API\s+[^(]*?\b(fm_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_07090_gb300 import build
    build.build()
    from paper_2504_07090_gb300 import fm
    return fm.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2504_07090_gb300 import fm
    decl = _declared()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(fm.EXPORTS) == decl


def test_invalid_config_rejected_before_device_work(lib):
    import ctypes
    from paper_2504_07090_gb300 import fm, synth
    p = synth.config("tiny")
    cfg, keep = fm.make_config(p, "fp32")
    h = ctypes.c_void_p()
    assert lib.fm_create(None, ctypes.byref(h)) == fm.FM_ERR_INVALID_ARG
    bad = fm.FmConfig.from_buffer_copy(cfg)
    bad.n_ant = 1
    assert lib.fm_create(ctypes.byref(bad), ctypes.byref(h)) == fm.FM_ERR_INVALID_ARG
    assert "n_ant" in fm.last_error()
    bad = fm.FmConfig.from_buffer_copy(cfg)
    bad.sigma_noise = -1.0
    assert lib.fm_create(ctypes.byref(bad), ctypes.byref(h)) == fm.FM_ERR_INVALID_ARG
    bad = fm.FmConfig.from_buffer_copy(cfg)
    bad.precision = 9
    assert lib.fm_create(ctypes.byref(bad), ctypes.byref(h)) == fm.FM_ERR_INVALID_ARG
    bad = fm.FmConfig.from_buffer_copy(cfg)
    bad.dec_max = bad.dec_min
    assert lib.fm_create(ctypes.byref(bad), ctypes.byref(h)) == fm.FM_ERR_INVALID_ARG
    assert h.value is None
    # calls on a NULL handle are rejected too
    assert lib.fm_forward(None, None, None, None) == fm.FM_ERR_INVALID_ARG
    assert lib.fm_num_params(None) == -1
    assert lib.fm_destroy(None) == fm.FM_OK


def test_batch_and_diagnostic_arguments_rejected_before_device_work(lib):
    import ctypes
    from paper_2504_07090_gb300 import fm
    out = ctypes.c_void_p()
    # batches: no handles, a NULL handle, n_steps out of range
    assert lib.fm_batch_create(0, None, None, None, None, None, 20, ctypes.byref(out)) == fm.FM_ERR_INVALID_ARG
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.fm_batch_create(1, arr, arr, arr, arr, arr, 20, ctypes.byref(out)) == fm.FM_ERR_INVALID_ARG
    assert lib.fm_batch_create(1, arr, arr, arr, arr, arr, 0, ctypes.byref(out)) == fm.FM_ERR_INVALID_ARG
    assert out.value is None
    assert lib.fm_batch_leapfrog(None, None, None, None) == fm.FM_ERR_INVALID_ARG
    assert lib.fm_batch_destroy(None) == fm.FM_OK
    assert lib.fm_create_batch(0, None, None) == fm.FM_ERR_INVALID_ARG
    # the bounded-wait diagnostic: status pointer required, limit within the kernels' own
    dummy = ctypes.c_int(0)
    assert lib.fm_diag_bounded_wait(1000, None, None) == fm.FM_ERR_INVALID_ARG
    assert lib.fm_diag_bounded_wait(0, ctypes.byref(dummy), None) == fm.FM_ERR_INVALID_ARG
    assert lib.fm_diag_bounded_wait(5_000_000_000, ctypes.byref(dummy), None) == fm.FM_ERR_INVALID_ARG
