"""fm_sky_pixels_noalloc, the entry point for callers that cannot allocate device
memory at call time, called through the C ABI twice in a row: each result matches the
allocating fm_sky_pixels of a handle on the same geometry (relative l2 < 1e-6, FP32),
the second call shows that a reused scratch array does not leak the first call's data,
and sizes beyond the fixed scratch are rejected without launching anything."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    import oracle
    from paper_2504_07090_gb300 import build, fm, synth
    build.build()
    lib = fm.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    results = []
    for name, seed in (("small", 1), ("mid", 2)):
        p = synth.config(name)
        o = oracle.Oracle(p)                      # basis tables of the geometry (test side)
        h = fm.ForwardModel(p, "fp32")
        theta = torch.tensor(np.random.default_rng(seed).standard_normal(h.n_params), dtype=torch.float32,
                             device="cuda")
        want = h.sky_pixels(theta)
        phi = torch.tensor(o.phi, dtype=torch.float32, device="cuda").contiguous()
        leg = torch.tensor(o.leg, dtype=torch.float32, device="cuda").contiguous()
        a = theta[: h.n_sky].contiguous()
        x = torch.full((p.n_freq * p.n_pix,), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.fm_sky_pixels_noalloc(p.n_freq, p.n_ra, p.n_dec, p.n_mode_ra, p.n_mode_dec, _dev(phi), _dev(leg),
                                       _dev(a), _dev(x), stream)
        assert st == fm.FM_OK, fm.last_error()
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(x.double() - want.double()) / torch.linalg.norm(want.double()))
        results.append(err)
        assert err < 1e-6, (name, err)
        h.close()
    assert len(results) == 2


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2504_07090_gb300 import build, fm
    build.build()
    lib = fm.load()
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    n0 = fm.kernel_launches()
    st = lib.fm_sky_pixels_noalloc(64, 4096, 8, 8, 16, _dev(dummy), _dev(dummy), _dev(dummy), _dev(dummy),
                                   ctypes.c_void_p(0))
    assert st == fm.FM_ERR_INVALID_ARG
    assert "exceeds" in fm.last_error()
    assert fm.kernel_launches() == n0
