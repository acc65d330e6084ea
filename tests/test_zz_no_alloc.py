"""fm_sky_pixels_noalloc, the entry point for callers that cannot allocate device
memory at call time, called through the C ABI three times in a row: each result matches
the allocating fm_sky_pixels of a handle on the same geometry (relative l2 < 1e-6, FP32).
The calls go from the largest scratch footprint to the smallest (n_freq * n_ra *
n_mode_dec = 4480, then 2208 with a different n_mode_dec, then 153), so every later call
reads a region the earlier ones left filled: a result that picked up any of that data
would fail.  Sizes beyond the fixed scratch, and beyond the launch grid, are rejected
without launching anything."""
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
    for name, seed in (("mid", 2), ("small", 1), ("tiny", 3)):
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
        print(f"fm_sky_pixels_noalloc {name}: relative l2 vs fm_sky_pixels {err:.2e}")
        assert err < 1e-6, (name, err)
        h.close()
    assert len(results) == 3


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
    # within the scratch but past the launch grid: 70000 channels of one 1 x 1 map
    st = lib.fm_sky_pixels_noalloc(70000, 1, 1, 1, 1, _dev(dummy), _dev(dummy), _dev(dummy), _dev(dummy),
                                   ctypes.c_void_p(0))
    assert st == fm.FM_ERR_INVALID_ARG
    assert "grid limits" in fm.last_error()
    assert fm.kernel_launches() == n0
