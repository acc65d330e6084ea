"""Pins of the oracle's modified Airy beam (Eq. airy) and of J1 behind it:

- J1 from Bessel's integral equals scipy.special.j1 (a library routine) over [0, 60];
- the power beam (2 J1(x) / x)^2 is 1 at the zenith, 1/2 at x = 1.6163 (half power), 0 at
  the first zero of J1 (x = 3.8317) and below the horizon;
- the effective diameter is D_ns toward north and south and D_ew toward east and west, and
  the beam is even in each of the east and north components;
- a point source under the Airy beam gives one fringe of amplitude S A (closed form), and
  the beam enters the visibilities of any sky linearly."""
import math

import numpy as np
import pytest

import oracle
from paper_2504_07090_gb300 import synth

C = 299792458.0


def test_j1_equals_library_routine():
    sp = pytest.importorskip("scipy.special")
    xs = np.concatenate([np.linspace(0.0, 60.0, 601), [1e-6, 3.8317059702075125, 7.0155866698156187]])
    got = np.array([oracle.bessel_j1(x) for x in xs])
    np.testing.assert_allclose(got, sp.j1(xs), rtol=0, atol=2e-15)
    assert oracle.bessel_j1(-2.5) == pytest.approx(-oracle.bessel_j1(2.5), abs=1e-15)


def _airy_problem(dew=12.0, dns=14.0):
    p = synth.with_airy_beam(synth.config("small"), dew, dns)
    return p, oracle.Oracle(p)


def _dir(za, az):
    """unit (east, north, up) at zenith angle za, azimuth az from north through east"""
    return math.sin(za) * math.sin(az), math.sin(za) * math.cos(az), math.cos(za)


def test_airy_power_beam_landmarks():
    nu = 150e6
    p, o = _airy_problem(14.0, 14.0)
    assert o.beam_dir(nu, 0.0, 0.0, 1.0) == 1.0
    # the limit 2 J1(x) / x -> 1 - x^2 / 8 near the zenith (x down to 1e-15)
    for za in (1e-15 * C / (math.pi * 14.0 * nu), 1e-6, 2e-4):
        x = math.pi * 14.0 * nu * math.sin(za) / C
        assert o.beam_dir(nu, *_dir(za, 0.3)) == pytest.approx((1.0 - x * x / 8.0 + x ** 4 / 192.0) ** 2, abs=1e-14)
    # x = pi D nu sin(za) / c
    for x, want in ((1.616339948310703, 0.5), (3.8317059702075125, 0.0)):
        za = math.asin(x * C / (math.pi * 14.0 * nu))
        assert o.beam_dir(nu, *_dir(za, 0.7)) == pytest.approx(want, abs=1e-12)
    assert o.beam_dir(nu, 0.6, 0.8, 0.0) == 0.0
    assert o.beam_dir(nu, 0.6, 0.0, -0.8) == 0.0


def test_airy_squash_and_symmetry():
    nu = 160e6
    p, o = _airy_problem(12.0, 14.0)
    za = 0.15
    north, east = o.beam_dir(nu, *_dir(za, 0.0)), o.beam_dir(nu, *_dir(za, math.pi / 2))
    for d, a in ((14.0, north), (12.0, east)):
        x = math.pi * d * nu * math.sin(za) / C
        assert a == pytest.approx((2.0 * oracle.bessel_j1(x) / x) ** 2, abs=1e-14)
    assert east > north          # the smaller aperture gives the wider beam
    e, n, u = _dir(0.2, 0.9)
    for se, sn in ((1, -1), (-1, 1), (-1, -1)):
        assert o.beam_dir(nu, se * e, sn * n, u) == pytest.approx(o.beam_dir(nu, e, n, u), abs=1e-15)


def test_point_source_under_airy_beam_is_one_fringe():
    p, o = _airy_problem()
    f, t, pix, S = 2, 3, 21 * 46 // 2 + 7, 3.5
    x = np.zeros(o.npix)
    d = pix // p.n_ra
    x[pix] = S / o.domega[d]
    V = o.vis_ft(f, t, x)
    s = o.s[t, pix]
    A = o.beam_dir(p.freq_hz[f], *s)
    assert A > 0.01
    b = p.ant_enu[o.bl_i] - p.ant_enu[o.bl_j]
    want = S * A * np.exp(-2j * np.pi * p.freq_hz[f] * (b @ s) / C)
    np.testing.assert_allclose(V, want, rtol=1e-12, atol=1e-12 * S)


def test_airy_beam_multiplies_the_sky():
    # V is linear in the beam-weighted sky: the Airy visibilities of x equal the isotropic
    # visibilities of A x (the beam moved into the sky, pixel by pixel)
    p, o = _airy_problem()
    pi = synth.with_isotropic_beam(synth.config("small"))
    oi = oracle.Oracle(pi)
    f, t = 1, 2
    x = np.random.default_rng(3).standard_normal(o.npix)
    A = np.array([o.beam_dir(p.freq_hz[f], *o.s[t, k]) for k in range(o.npix)])
    np.testing.assert_allclose(o.vis_ft(f, t, x), oi.vis_ft(f, t, A * x), rtol=1e-11, atol=1e-11 * np.abs(x).sum())
