"""Pins of the oracle's geometry, basis, beam and fringe against facts fixed outside it.

Each test names what it pins: a closed form, a textbook identity, a library routine,
or an invariant that a plausible slip (wrong sign, swapped index, wrong constant)
would break.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle
from paper_2504_07090_gb300 import synth

C = 299792458.0


def _problem(**kw):
    base = dict(name="t", ant_enu=np.array([[0.0, 0.0, 0.0], [14.6, 0.0, 0.0]]),
                freq_hz=np.array([150e6]), lst_rad=np.array([0.3]), lat_rad=synth.LATITUDE_RAD,
                n_ra=8, n_dec=4, ra_min=0.0, ra_max=0.4, dec_min=-0.7, dec_max=-0.3,
                n_mode_ra=1, n_mode_dec=1, n_gain=1)
    base.update(kw)
    return synth.Problem(**base)


def _enu_by_projection(ra, dec, lst, lat):
    """Topocentric direction by projecting onto local axes built as vectors
    (zenith on the meridian at declination lat; north = pole projected on the horizon;
    east = north x up) -- a derivation independent of the oracle's trig closed form."""
    H = lst - ra
    e_h = np.array([math.cos(dec) * math.cos(H), -math.cos(dec) * math.sin(H), math.sin(dec)])
    up = np.array([math.cos(lat), 0.0, math.sin(lat)])
    pole = np.array([0.0, 0.0, 1.0])
    north = pole - (pole @ up) * up
    north /= np.linalg.norm(north)
    east = np.cross(north, up)
    return np.array([e_h @ east, e_h @ north, e_h @ up])


def test_topocentric_matches_vector_projection_and_unit_norm():
    p = _problem(n_ra=7, n_dec=5, ra_min=-1.0, ra_max=1.5, dec_min=-1.2, dec_max=0.4,
                 lst_rad=np.array([0.1, 0.9, -2.0]))
    o = oracle.Oracle(p)
    for t, lst in enumerate(p.lst_rad):
        for d in range(p.n_dec):
            for r in range(p.n_ra):
                ref = _enu_by_projection(o.ra_c[r], o.dec_c[d], lst, p.lat_rad)
                np.testing.assert_allclose(o.s[t, d * p.n_ra + r], ref, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(o.s, axis=-1), 1.0, atol=1e-14)


def test_zenith_and_south_pole_altitude():
    lat = synth.LATITUDE_RAD
    # a cell centred on the zenith at transit: s = (0, 0, 1)
    p = _problem(n_ra=1, n_dec=1, ra_min=0.3 - 0.01, ra_max=0.3 + 0.01, dec_min=lat - 0.01, dec_max=lat + 0.01)
    o = oracle.Oracle(p)
    np.testing.assert_allclose(o.s[0, 0], [0.0, 0.0, 1.0], atol=1e-15)
    # the south celestial pole stands due south at altitude |latitude| (textbook fact)
    p = _problem(n_ra=1, n_dec=1, ra_min=0.0, ra_max=0.2, dec_min=-math.pi / 2, dec_max=-math.pi / 2 + 2e-9)
    o = oracle.Oracle(p)
    s = o.s[0, 0]
    assert abs(math.asin(s[2]) - abs(lat)) < 1e-8
    assert s[1] < 0 and abs(s[0]) < 1e-8


def test_cell_solid_angles_exact():
    # full sphere sums to 4 pi; one cell equals the integral of cos(dec) over it
    p = _problem(n_ra=36, n_dec=18, ra_min=0.0, ra_max=2 * math.pi, dec_min=-math.pi / 2, dec_max=math.pi / 2)
    o = oracle.Oracle(p)
    assert abs(o.domega.sum() * p.n_ra - 4 * math.pi) < 1e-12
    from scipy.integrate import quad
    dd = math.pi / 18
    for d in (0, 5, 9, 17):
        lo = -math.pi / 2 + d * dd
        ref = (2 * math.pi / 36) * quad(math.cos, lo, lo + dd)[0]
        assert abs(o.domega[d] - ref) < 1e-14


def test_dec_basis_is_numpy_legendre():
    p = _problem(n_ra=4, n_dec=13, n_mode_ra=2, n_mode_dec=9)
    o = oracle.Oracle(p)
    dhat = 2.0 * (o.dec_c - p.dec_min) / (p.dec_max - p.dec_min) - 1.0
    for n in range(9):
        np.testing.assert_allclose(o.leg[:, n], npleg.legval(dhat, np.eye(9)[n]), atol=1e-13)


def test_ra_basis_orthogonal_and_at_its_wavenumber():
    # cos/sin periodic over the span: discrete orthogonality on the uniform grid and the
    # FFT puts each function's power at its own wavenumber (App. A.2 azimuthal condition)
    M, R = 16, 24
    p = _problem(n_ra=R, n_dec=2, n_mode_ra=M, n_mode_dec=1)
    o = oracle.Oracle(p)
    gram = o.phi.T @ o.phi
    want = np.full(M, R / 2.0)
    want[0] = R
    np.testing.assert_allclose(gram, np.diag(want), atol=1e-10)
    spec = np.abs(np.fft.rfft(o.phi, axis=0))
    for m in range(M):
        k = 0 if m == 0 else (M // 2 if m == M - 1 else (m + 1) // 2)
        assert int(np.argmax(spec[:, m])) == k


def test_gain_frequency_basis_is_numpy_legendre():
    p = _problem(freq_hz=np.linspace(140e6, 160e6, 7), n_gain=4)
    o = oracle.Oracle(p)
    nhat = np.linspace(-1, 1, 7)
    for k in range(4):
        np.testing.assert_allclose(o.gleg[:, k], npleg.legval(nhat, np.eye(4)[k]), atol=1e-14)


def test_beam_half_power_at_half_fwhm_and_horizon():
    p = _problem()
    o = oracle.Oracle(p)
    for nu in (120e6, 150e6, 180e6):
        fwhm = synth.BEAM_FWHM_REF_RAD * 150e6 / nu
        assert abs(o.beam(nu, 1.0) - 1.0) < 1e-15
        assert abs(o.beam(nu, math.cos(fwhm / 2)) - 0.5) < 1e-12       # definition of FWHM
    assert o.beam(150e6, 0.0) == 0.0 and o.beam(150e6, -0.3) == 0.0
    iso = oracle.Oracle(synth.with_isotropic_beam(p))
    assert iso.beam(150e6, 1e-3) == 1.0


def test_point_source_gives_pure_fringe():
    # one source of flux S in one pixel: V_pq = S A exp(-2 pi i nu (r_p - r_q).s / c)
    ants = np.array([[0.0, 0.0, 0.0], [14.6, 0.0, 0.0], [7.3, 12.64, 0.0], [-3.0, 5.0, 0.4]])
    p = _problem(ant_enu=ants, n_ra=9, n_dec=7, ra_min=0.0, ra_max=0.6, dec_min=-0.8, dec_max=-0.3,
                 freq_hz=np.array([121e6, 173e6]), lst_rad=np.array([0.2, 0.45]))
    o = oracle.Oracle(p)
    S = 3.7
    for f, nu in enumerate(p.freq_hz):
        for t, lst in enumerate(p.lst_rad):
            for pix in (0, 31, 62):
                d, r = divmod(pix, p.n_ra)
                x = np.zeros(o.npix)
                x[pix] = S / o.domega[d]
                V = o.vis_ft(f, t, x)
                s = _enu_by_projection(o.ra_c[r], o.dec_c[d], lst, p.lat_rad)
                za = math.acos(s[2])
                sig = synth.BEAM_FWHM_REF_RAD * 150e6 / nu / math.sqrt(8 * math.log(2))
                amp = S * math.exp(-za * za / (2 * sig * sig))
                for b, (i, j) in enumerate(zip(o.bl_i, o.bl_j)):
                    tau = (ants[i] - ants[j]) @ s / C            # geometric delay of the baseline
                    want = amp * np.exp(-2j * math.pi * nu * tau)
                    assert abs(V[b] - want) < 1e-12 * max(1.0, amp)


def test_uniform_sky_isotropic_beam_gives_sinc():
    # hemisphere integral of exp(-i k b.s) for a horizontal baseline is 2 pi sin(kb)/(kb);
    # antipodal cell pairs make Re V half the full-sphere midpoint sum (error O(h^2)) and
    # the autocorrelation exactly 2 pi
    b = 14.6
    k = 2 * math.pi * 150e6 / C
    want = 2 * math.pi * math.sin(k * b) / (k * b)
    errs = []
    for nra, ndec in ((360, 180), (720, 360)):
        p = _problem(ant_enu=np.array([[0.0, 0.0, 0.0], [b, 0.0, 0.0], [b, 0.0, 0.0]]), n_ra=nra, n_dec=ndec,
                     ra_min=0.0, ra_max=2 * math.pi, dec_min=-math.pi / 2, dec_max=math.pi / 2,
                     beam_fwhm_ref_rad=0.0)
        o = oracle.Oracle(p)
        V = o.vis_ft(0, 0, np.ones(o.npix))
        h = math.pi / ndec
        assert abs(V[0].real - V[1].real) < 1e-13
        assert abs(V[2] - 2 * math.pi) < 1e-11                   # zero-length baseline: 2 pi
        assert abs(V[0].imag) < 2.0 * h                          # horizon staircase -> 0
        errs.append(abs(V[0].real - want))
    assert errs[1] < 1e-4
    assert errs[0] / errs[1] > 3.5                               # second-order convergence


def test_linearity_and_hermitian_reversal():
    p = synth.config("tiny")
    o = oracle.Oracle(p)
    rng = np.random.default_rng(1)
    x1, x2 = rng.standard_normal((2, o.npix))
    v1, v2, v12 = o.vis_ft(1, 2, x1), o.vis_ft(1, 2, x2), o.vis_ft(1, 2, x1 - 2.5 * x2)
    np.testing.assert_allclose(v12, v1 - 2.5 * v2, atol=1e-12 * np.abs(v1).max())
    # reversing the antenna order turns every pair (p, q) into (q, p): b -> -b, V -> conj V
    rev = synth.Problem(**{**p.__dict__, "ant_enu": p.ant_enu[::-1].copy()})
    orv = oracle.Oracle(rev)
    vr = orv.vis_ft(1, 2, x1)
    A = p.n_ant
    for b, (i, j) in enumerate(zip(o.bl_i, o.bl_j)):
        ir, jr = A - 1 - j, A - 1 - i
        br = [k for k, (a, c) in enumerate(zip(orv.bl_i, orv.bl_j)) if a == ir and c == jr][0]
        assert abs(vr[br] - np.conj(v1[b])) < 1e-12 * abs(v1).max()


def test_separable_mode_transform_equals_matrix_product():
    # x = P_dec a Phi_ra^T (Eq. fg_separable) computed with a library matmul
    p = synth.config("small")
    o = oracle.Oracle(p)
    a = np.random.default_rng(2).standard_normal(o.nk)
    x = o.sky_f(a).reshape(p.n_dec, p.n_ra)
    ref = o.leg @ a.reshape(p.n_mode_ra, p.n_mode_dec).T @ o.phi.T
    np.testing.assert_allclose(x, ref, atol=1e-11 * np.abs(ref).max())
    # and the adjoint is its transpose: <x(a), y> = <a, x^T(y)>
    y = np.random.default_rng(3).standard_normal(o.npix)
    assert abs(x.reshape(-1) @ y - a @ o.sky_adjoint_f(y)) < 1e-10 * abs(x.reshape(-1) @ y)
