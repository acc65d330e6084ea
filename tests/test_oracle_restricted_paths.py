"""Pins of the oracle entry points that the full-size parity tests lean on:

- orc_vis_one, one visibility of Eq. rime_discrete at a time, equals the pinned
  per-(channel, LST) sum orc_vis_ft element by element (same terms, same order);
- chi2_grad / hvp / model restricted to a list of (channel, LST) pairs: chi^2 of
  Eq. likelihood is a sum over (channel, LST, baseline) and the gradient and HVP are sums
  of per-pair terms, so a restricted call over every pair equals the full call without the
  prior of Eq. posterior, and two restricted calls over a partition of the pairs add up to
  it; the restricted model is the full model on its pairs and zero elsewhere."""
import numpy as np
import pytest

import oracle
from paper_2504_07090_gb300 import synth


def _case(name):
    p = synth.config(name)
    tr = synth.draw_truth(p)
    o = oracle.Oracle(p)
    m = o.model(tr.theta)
    p.sigma = o.sigma = 0.01 * float(np.mean(np.abs(m)))
    d = m + p.sigma * (tr.noise[..., 0] + 1j * tr.noise[..., 1])
    mu, lam = synth.prior_for(p, tr.theta)
    rng = np.random.default_rng(5)
    th = tr.theta * (1.0 + 0.01 * rng.standard_normal(tr.theta.shape))
    return p, o, th, d, mu, lam


@pytest.mark.parametrize("name", ["small", "ha37"])
def test_vis_one_equals_vis_ft_element_by_element(name):
    p = synth.config(name)
    tr = synth.draw_truth(p)
    o = oracle.Oracle(p)
    a, _ = o.split(tr.theta)
    for f in range(p.n_freq):
        x_f = o.sky_f(a[f])
        for t in range(p.n_lst):
            V = o.vis_ft(f, t, x_f)
            one = np.array([o.vis_one(f, t, b, x_f) for b in range(p.n_bl)])
            assert np.array_equal(one, V), (f, t)


def test_vis_one_at_cfg1_equals_vis_ft():
    # the full-size geometry of the sampled checks (37 antennas, 24,576 pixels), a few pairs
    p = synth.config("cfg1")
    tr = synth.draw_truth(p)
    o = oracle.Oracle(p)
    a, _ = o.split(tr.theta)
    rng = np.random.default_rng(1)
    for f, t in ((0, 0), (37, 59), (63, 17)):
        x_f = o.sky_f(a[f])
        V = o.vis_ft(f, t, x_f)
        for b in rng.integers(0, p.n_bl, 6):
            assert o.vis_one(f, t, int(b), x_f) == V[b]


@pytest.mark.parametrize("name", ["small", "ha37"])
def test_restricted_chi2_grad_over_all_pairs_is_the_full_call_without_prior(name):
    p, o, th, d, mu, lam = _case(name)
    chi2, U, g = o.chi2_grad(th, d, mu, lam)
    pu, pg = o.prior_terms(th, mu, lam)
    assert pu > 0 and np.linalg.norm(pg) > 0
    pairs = [(f, t) for t in range(p.n_lst) for f in range(p.n_freq)]    # another order
    c2, U2, g2 = o.chi2_grad(th, d, mu, lam, fts=pairs)
    assert abs(c2 - chi2) <= 1e-12 * chi2
    assert abs(U2 - (U - pu)) <= 1e-12 * U
    np.testing.assert_allclose(g2, g - pg, rtol=0, atol=1e-10 * np.max(np.abs(g)))


@pytest.mark.parametrize("name", ["small", "ha37"])
def test_restricted_calls_over_a_partition_add_up(name):
    p, o, th, d, mu, lam = _case(name)
    rng = np.random.default_rng(9)
    pairs = [(f, t) for f in range(p.n_freq) for t in range(p.n_lst)]
    pick = rng.random(len(pairs)) < 0.4
    A = [q for q, k in zip(pairs, pick) if k]
    B = [q for q, k in zip(pairs, pick) if not k]
    cA, UA, gA = o.chi2_grad(th, d, fts=A)
    cB, UB, gB = o.chi2_grad(th, d, fts=B)
    c, U, g = o.chi2_grad(th, d)
    assert abs(cA + cB - c) <= 1e-12 * c
    np.testing.assert_allclose(gA + gB, g, rtol=0, atol=1e-10 * np.max(np.abs(g)))
    # each part is nonzero and differs from the whole
    assert 0 < cA < c and 0 < cB < c
    v = np.random.default_rng(10).standard_normal(o.n_par)
    for full in (True, False):
        hA = o.hvp(th, d, v, full=full, fts=A)
        hB = o.hvp(th, d, v, full=full, fts=B)
        h = o.hvp(th, d, v, full=full)
        np.testing.assert_allclose(hA + hB, h, rtol=0, atol=1e-10 * np.max(np.abs(h)))


def test_restricted_model_is_the_full_model_on_its_pairs():
    p, o, th, d, mu, lam = _case("small")
    full = o.model(th)
    pairs = [(1, 2), (4, 0), (5, 4)]
    part = o.model(th, fts=pairs)
    for f in range(p.n_freq):
        for t in range(p.n_lst):
            if (f, t) in pairs:
                assert np.array_equal(part[f, t], full[f, t])
            else:
                assert not np.any(part[f, t])
