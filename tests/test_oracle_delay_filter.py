"""Pins of the delay filter (Eq. rime_filter, Eq. gpr, Eq. filtered_noise) in the oracle.

- C_noise = eps I commutes with C_fg, so F = I - C (C + eps I)^-1 = eps (C + eps I)^-1: built
  here a second way, from the eigendecomposition of C (F = V diag(eps / (l + eps)) V^T);
- a pure delay mode exp(2 pi i nu tau) inside the rejection band |tau| < tau_max is removed
  to below 1e-3 of its amplitude, one well outside it passes nearly unchanged;
- with F = I and unit weights the filtered chi^2 and gradient are the unfiltered ones;
- the filtered gradient matches central differences of the filtered U along sky directions
  (exact: U is quadratic in the sky modes) and, with gains, falls as h^2."""
import numpy as np

import oracle
from paper_2504_07090_gb300 import synth


def _band(n=64, lo=140e6, hi=160e6):
    return np.linspace(lo, hi, n)


def test_filter_equals_its_eigen_form_and_is_symmetric():
    nu = _band()
    Fm = oracle.delay_filter(nu, 250e-9, 1e-8)
    C = np.sinc(2.0 * 250e-9 * (nu[:, None] - nu[None, :]))
    w, V = np.linalg.eigh(C)
    Fe = V @ np.diag(1e-8 / (w + 1e-8)) @ V.T
    assert np.max(np.abs(Fm - Fe)) < 1e-6
    assert np.max(np.abs(Fm - Fm.T)) < 1e-6


def test_delay_modes_inside_the_band_are_removed_and_outside_pass():
    nu = _band()
    Fm = oracle.delay_filter(nu, 250e-9, 1e-8)
    for tau in (0.0, 60e-9, -120e-9):
        y = np.exp(2j * np.pi * nu * tau)
        assert np.linalg.norm(Fm @ y) / np.linalg.norm(y) < 1e-3, tau
    for tau in (1.2e-6, -1.6e-6):
        y = np.exp(2j * np.pi * nu * tau)
        assert abs(np.linalg.norm(Fm @ y) / np.linalg.norm(y) - 1.0) < 0.05, tau


def _case():
    p = synth.config("small")
    tr = synth.draw_truth(p)
    o = oracle.Oracle(p)
    m = o.model(tr.theta)
    p.sigma = o.sigma = 0.01 * float(np.mean(np.abs(m)))
    d = m + p.sigma * (tr.noise[..., 0] + 1j * tr.noise[..., 1])
    mu, lam = synth.prior_for(p, tr.theta)
    th = tr.theta * (1.0 + 0.01 * np.random.default_rng(3).standard_normal(tr.theta.shape))
    return p, o, th, d, mu, lam


def test_identity_filter_reduces_to_the_plain_likelihood():
    p, o, th, d, mu, lam = _case()
    c1, U1, g1 = o.chi2_grad(th, d, mu, lam)
    c2, U2, g2 = o.chi2_grad_filtered(th, d, np.eye(p.n_freq), mu, lam)
    assert abs(c1 - c2) <= 1e-12 * c1 and abs(U1 - U2) <= 1e-12 * U1
    np.testing.assert_allclose(g2, g1, rtol=0, atol=1e-10 * np.max(np.abs(g1)))


def test_filtered_gradient_matches_central_differences():
    p, o, th, d, mu, lam = _case()
    Fm = oracle.delay_filter(p.freq_hz, 250e-9, 1e-8)
    _, U0, g = o.chi2_grad_filtered(th, d, Fm, mu, lam)
    rng = np.random.default_rng(4)
    # sky direction: exact for any step
    v = np.zeros(o.n_par)
    v[: o.n_sky] = rng.standard_normal(o.n_sky)
    h = 1e-3 * np.linalg.norm(th[: o.n_sky]) / np.linalg.norm(v)
    fd = (o.chi2_grad_filtered(th + h * v, d, Fm, mu, lam)[1] - o.chi2_grad_filtered(th - h * v, d, Fm, mu, lam)[1]) / (2 * h)
    assert abs(fd - g @ v) <= 1e-8 * abs(g @ v) + 1e-9 * abs(U0)
    # gain direction: O(h^2)
    v = np.zeros(o.n_par)
    v[o.n_sky:] = rng.standard_normal(o.n_par - o.n_sky)
    errs = []
    for h in (2e-4, 1e-4):
        fd = (o.chi2_grad_filtered(th + h * v, d, Fm, mu, lam)[1] - o.chi2_grad_filtered(th - h * v, d, Fm, mu, lam)[1]) / (2 * h)
        errs.append(abs(fd - g @ v))
    assert 3.0 < errs[0] / errs[1] < 5.0          # second order: the error falls as h^2
    assert errs[1] < 1e-4 * abs(g @ v)


def test_filtered_noise_gives_the_expected_chi2_at_truth():
    # at the truth the filtered residual is the filtered noise: E[chi^2] = 2 N_vis with the
    # diagonal of F N F^T (Eq. filtered_noise) in the denominator
    p = synth.config("small")
    tr = synth.draw_truth(p)
    o = oracle.Oracle(p)
    m = o.model(tr.theta)
    p.sigma = o.sigma = 0.01 * float(np.mean(np.abs(m)))
    d = m + p.sigma * (tr.noise[..., 0] + 1j * tr.noise[..., 1])
    Fm = oracle.delay_filter(p.freq_hz, 250e-9, 1e-8)
    chi2, _, _ = o.chi2_grad_filtered(tr.theta, d, Fm)
    n = 2 * p.n_vis
    assert abs(chi2 - n) < 6.0 * np.sqrt(2.0 * n)
