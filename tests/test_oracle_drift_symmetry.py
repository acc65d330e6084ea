"""Symmetries of the drift-scan workloads that the hour-angle form of the contraction
relies on, checked on the oracle's own geometry and visibilities (no GPU).

1. With LSTs spaced by k RA pixels, pixel (r, d) at LST t points where pixel (r - k, d)
   pointed at LST t - 1 (the direction depends on the hour angle LST - RA only, Sec. 2.1);
   with a spacing of k / q pixels the same holds for a shift of q LSTs and k pixels.
2. With one beam for all antennas (Sec. 3.4), baselines with equal vectors have equal
   visibilities and reversed vectors give the complex conjugate (Eq. rime_discrete)."""
import numpy as np
import pytest

import oracle
from paper_2504_07090_gb300 import synth


@pytest.mark.parametrize("name,k", [("ha7", 2), ("ha37", 1), ("harand", 1), ("cfg1", 1)])
def test_directions_shift_by_k_pixels_per_lst(name, k):
    p = synth.config(name)
    dra = (p.ra_max - p.ra_min) / p.n_ra
    assert abs((p.lst_rad[1] - p.lst_rad[0]) / dra - k) < 1e-9
    o = oracle.Oracle(p)
    s = o.s.reshape(o.T, o.D, o.R, 3)
    a = s[1:, :, k:, :]
    b = s[:-1, :, :-k, :]
    assert np.max(np.abs(a - b)) < 1e-12
    # and not for a shift by a different number of pixels
    assert np.max(np.abs(s[1:, :, k + 1:, :] - s[:-1, :, : o.R - k - 1, :])) > 1e-4


@pytest.mark.parametrize("name,k,q", [("hafrac2", 5, 2), ("hafrac4", 3, 4), ("hachunk", 1, 2)])
def test_directions_shift_by_k_pixels_per_q_lsts(name, k, q):
    """LST step of k / q pixels: pixel (r, d) at LST t points where pixel (r - k, d) pointed at
    LST t - q (the hour angle t k / q - r is unchanged), and no shift by fewer LSTs does so."""
    p = synth.config(name)
    dra = (p.ra_max - p.ra_min) / p.n_ra
    assert abs((p.lst_rad[1] - p.lst_rad[0]) / dra * q - k) < 1e-9
    o = oracle.Oracle(p)
    s = o.s.reshape(o.T, o.D, o.R, 3)
    assert np.max(np.abs(s[q:, :, k:, :] - s[:-q, :, :-k, :])) < 1e-12
    for tq in range(1, q):
        # a shift of tq < q LSTs moves the hour angle by tq k / q pixels, not a whole number
        kk = (tq * k) // q
        assert np.max(np.abs(s[tq:, :, kk:, :] - s[:-tq, :, : o.R - kk, :])) > 1e-4


def _groups(ant):
    A = ant.shape[0]
    reps, out = [], []
    for i in range(A):
        for j in range(i + 1, A):
            v = ant[i] - ant[j]
            for u, r in enumerate(reps):
                if np.max(np.abs(v - r)) < 1e-9:
                    out.append((u, 0))
                    break
                if np.max(np.abs(v + r)) < 1e-9:
                    out.append((u, 1))
                    break
            else:
                reps.append(v)
                out.append((len(reps) - 1, 0))
    return len(reps), out


@pytest.mark.parametrize("name,n_groups", [("ha7", 9), ("ha37", 63), ("harand", 66)])
def test_redundant_baselines_have_equal_or_conjugate_visibilities(name, n_groups):
    p = synth.config(name)
    o = oracle.Oracle(p)
    U, memb = _groups(p.ant_enu)
    assert U == n_groups
    x = np.random.default_rng(5).standard_normal((o.F, o.npix)) + 3.0
    V = o.vis(x)                                   # [F][T][B] complex
    first = {}
    for b, (u, cj) in enumerate(memb):
        vb = np.conj(V[..., b]) if cj else V[..., b]
        if u not in first:
            first[u] = vb
        else:
            assert np.max(np.abs(vb - first[u])) < 1e-12 * np.max(np.abs(first[u]))
