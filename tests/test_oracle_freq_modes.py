"""Pins of the oracle's Legendre-in-frequency sky compression (Eq. fg_legendre, Eq. eor_model):
a(nu_f) = sum_k X_k(nu_f) a~_k with X_k the Legendre polynomial P_k of the band-normalised
frequency nu^ in [-1, 1].

What fixes the answers here without the oracle's own expansion:
- X against the explicit polynomials P_0 = 1, P_1 = x, P_2 = (3x^2 - 1)/2, P_3 = (5x^3 - 3x)/2 and
  the endpoint values P_k(1) = 1, P_k(-1) = (-1)^k;
- the per-channel problem (no compression) as the second route: a spectrum that is flat, or
  linear in nu^, gives the per-channel model of that spectrum, and with K = n_freq the
  compressed U is the per-channel U composed with the (explicit) design matrix, so its gradient
  is X^T times the per-channel gradient (chain rule);
- exactness facts: the model stays linear in the compressed sky coefficients, so central
  differences of U along them are exact up to rounding; the Jacobian built column by column
  from the forward sum gives the Gauss-Newton products and blocks by brute force.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from paper_2504_07090_gb300 import synth


def _nuhat(freq):
    f = np.asarray(freq, dtype=np.float64)
    return 2.0 * (f - f.min()) / (f.max() - f.min()) - 1.0


def _explicit_legendre(x, K):
    polys = [np.ones_like(x), x, (3 * x ** 2 - 1) / 2, (5 * x ** 3 - 3 * x) / 2]
    return np.stack(polys[:K], axis=1)


def _setup(name="tiny", K=2, noise=True):
    p = synth.with_freq_modes(synth.config(name), K)
    tr = synth.draw_truth(p)
    o = oracle.Oracle(p)
    m = o.model(tr.theta)
    o.sigma = p.sigma = 0.01 * float(np.mean(np.abs(m)))
    d = m + (p.sigma * (tr.noise[..., 0] + 1j * tr.noise[..., 1]) if noise else 0.0)
    mu, lam = synth.prior_for(p, tr.theta)
    return p, o, tr.theta.copy(), d, mu, lam


def _per_channel(p):
    o0 = oracle.Oracle(replace(p, n_freq_modes=0))
    return o0


def _params_per_channel(o, a_f, gains):
    return np.concatenate([np.asarray(a_f).reshape(-1), gains])


@pytest.mark.parametrize("name,K", [("tiny", 3), ("small", 4), ("small", 2)])
def test_design_matrix_is_legendre_of_normalised_frequency(name, K):
    p = synth.with_freq_modes(synth.config(name), K)
    o = oracle.Oracle(p)
    x = _nuhat(p.freq_hz)
    np.testing.assert_allclose(o.Xf, _explicit_legendre(x, K), rtol=0, atol=1e-14)
    lo, hi = int(np.argmin(p.freq_hz)), int(np.argmax(p.freq_hz))
    np.testing.assert_array_equal(o.Xf[hi], np.ones(K))
    np.testing.assert_array_equal(o.Xf[lo], (-1.0) ** np.arange(K))
    assert o.n_sky == K * o.nk and o.n_par == K * o.nk + 2 * o.A * o.NG


def test_flat_and_linear_spectra_reduce_to_the_per_channel_model():
    p, o, th, d, mu, lam = _setup("small", 3)
    o0 = _per_channel(p)
    gains = th[o.n_sky:]
    rng = np.random.default_rng(3)
    b = th[: o.nk] * (1.0 + 0.1 * rng.standard_normal(o.nk))
    x = _nuhat(p.freq_hz)
    flat = np.zeros(o.n_sky)
    flat[: o.nk] = b
    m_flat = o.model(np.concatenate([flat, gains]))
    m_ref = o0.model(_params_per_channel(o0, np.tile(b, (o.F, 1)), gains))
    np.testing.assert_allclose(m_flat, m_ref, rtol=0, atol=1e-12 * np.abs(m_ref).max())
    lin = np.zeros(o.n_sky)
    lin[o.nk: 2 * o.nk] = b
    m_lin = o.model(np.concatenate([lin, gains]))
    m_ref = o0.model(_params_per_channel(o0, x[:, None] * b[None, :], gains))
    np.testing.assert_allclose(m_lin, m_ref, rtol=0, atol=1e-12 * np.abs(m_ref).max())


def test_full_rank_compression_is_a_change_of_basis():
    # K = n_freq: U_K(a~, gamma) = U_0(X a~, gamma), so grad_a~ = X^T grad_a and the gain
    # gradient is unchanged; the model is the per-channel model of X a~
    p, o, th, d, mu, lam = _setup("tiny", 3)
    o0 = _per_channel(p)
    X = _explicit_legendre(_nuhat(p.freq_hz), 3)
    th = th + 0.02 * np.abs(th).mean() * np.random.default_rng(4).standard_normal(o.n_par)
    a_f = X @ th[: o.n_sky].reshape(3, o.nk)
    th0 = _params_per_channel(o0, a_f, th[o.n_sky:])
    np.testing.assert_allclose(o.model(th), o0.model(th0), rtol=0, atol=1e-12 * np.abs(o0.model(th0)).max())
    c, U, g = o.chi2_grad(th, d)
    c0, U0, g0 = o0.chi2_grad(th0, d)
    assert abs(c - c0) <= 1e-12 * c0
    g_sky = X.T @ g0[: o0.n_sky].reshape(o.F, o.nk)
    np.testing.assert_allclose(g[: o.n_sky], g_sky.reshape(-1), rtol=0, atol=1e-11 * np.abs(g_sky).max())
    np.testing.assert_allclose(g[o.n_sky:], g0[o0.n_sky:], rtol=0, atol=1e-11 * np.abs(g0[o0.n_sky:]).max())


def test_gradient_matches_exact_central_differences():
    p, o, th, d, mu, lam = _setup("tiny", 2)
    rng = np.random.default_rng(5)
    sc = np.abs(th[: o.n_sky]).mean()
    th = th.copy()
    th[: o.n_sky] += 0.02 * sc * rng.standard_normal(o.n_sky)
    _, _, g = o.chi2_grad(th, d, mu, lam)
    for k in rng.choice(o.n_sky, 8, replace=False):
        h = 0.3 * sc
        e = np.zeros(o.n_par)
        e[k] = h
        fd = (o.chi2_grad(th + e, d, mu, lam)[1] - o.chi2_grad(th - e, d, mu, lam)[1]) / (2 * h)
        assert abs(fd - g[k]) < 1e-7 * max(abs(g).max() / 100, abs(g[k]))
    for k in o.n_sky + rng.choice(o.n_par - o.n_sky, 4, replace=False):
        errs = []
        for h in (1e-2, 5e-3):
            e = np.zeros(o.n_par)
            e[k] = h
            fd = (o.chi2_grad(th + e, d, mu, lam)[1] - o.chi2_grad(th - e, d, mu, lam)[1]) / (2 * h)
            errs.append(abs(fd - g[k]))
        assert errs[1] < 1e-4 * abs(g).max() + 1e-9
        assert errs[1] < errs[0] / 3.0 or errs[0] < 1e-9 * abs(g).max()


def test_jacobian_gn_products_and_blocks_by_brute_force():
    p, o, th, d, mu, lam = _setup("tiny", 2)
    J = o.jacobian(th)
    sc = np.abs(th[: o.n_sky]).mean()
    rng = np.random.default_rng(6)
    for k in rng.choice(o.n_sky, 6, replace=False):
        h = 0.5 * sc
        e = np.zeros(o.n_par)
        e[k] = h
        fd = (o.model(th + e) - o.model(th - e)).reshape(-1) / (2 * h)
        assert np.abs(fd - J[:, k]).max() < 1e-9 * np.abs(J).max()
    H = (J.conj().T @ J).real / o.sigma ** 2 + np.diag(lam)
    v = rng.standard_normal(o.n_par)
    np.testing.assert_allclose(o.hvp(th, d, v, lam, full=False), H @ v, rtol=0, atol=1e-10 * np.abs(H @ v).max())
    bs = 4
    blocks, Hg = o.gn_blocks(th, lam, bs)
    assert sorted(blocks) == list(range(o.K * o.nk // bs))
    for blk, Hb in blocks.items():
        l, j0 = divmod(blk, o.nk // bs)
        s = l * o.nk + j0 * bs
        np.testing.assert_allclose(Hb, H[s:s + bs, s:s + bs], rtol=0, atol=1e-10 * np.abs(H).max())
    np.testing.assert_allclose(Hg, H[o.n_sky:, o.n_sky:], rtol=0, atol=1e-10 * np.abs(Hg).max())
    # the orders couple (X_l X_l' summed over channels is not zero on a discrete band): the
    # block-diagonal mass matrix leaves those cross blocks out
    cross = H[: o.nk, o.nk: 2 * o.nk]
    assert np.abs(cross).max() > 1e-6 * np.abs(H[: o.nk, : o.nk]).max()


def test_synth_compressed_problem():
    p = synth.with_freq_modes(synth.config("small"), 3)
    assert p.n_freq_modes == 3 and p.n_sky_rows == 3 and p.n_sky_params == 3 * p.n_modes
    tr = synth.draw_truth(p)
    assert tr.theta.shape == (p.n_params,) and np.isfinite(tr.theta).all()
    sky = tr.theta[: p.n_sky_params].reshape(3, p.n_modes)
    # smooth spectra: the orders fall off
    r = np.sqrt(np.mean(sky ** 2, axis=1))
    assert r[0] > r[1] > r[2] > 0
    mu, lam = synth.prior_for(p, tr.theta)
    assert lam.shape == (p.n_params,) and (lam > 0).all()
    with pytest.raises(ValueError):
        synth.with_freq_modes(synth.config("small"), p.n_freq + 1)
    assert synth.with_freq_modes(p, 0).n_sky_params == p.n_freq * p.n_modes
