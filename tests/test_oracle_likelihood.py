"""Pins of the oracle's likelihood, gradient, HVP, Jacobian, GN blocks and leapfrog.

Exactness facts used: the model is linear in the sky modes, so chi^2 is exactly
quadratic along sky directions and a central difference of U (or of grad U) there is
exact up to rounding; along gain directions it is a polynomial, so the central
difference error falls as h^2.  Brute force: the explicit Jacobian built column by
column from the forward sum.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2504_07090_gb300 import synth


def _setup(name="tiny", noise=True, seed=None):
    p = synth.config(name)
    tr = synth.draw_truth(p, seed)
    o = oracle.Oracle(p)
    m = o.model(tr.theta)
    sigma = 0.01 * float(np.mean(np.abs(m)))
    o.sigma = sigma
    nz = tr.noise[..., 0] + 1j * tr.noise[..., 1]
    d = m + (sigma * nz if noise else 0.0)
    mu, lam = synth.prior_for(p, tr.theta)
    return p, o, tr.theta.copy(), d, mu, lam


def _scales(o, theta):
    a, _ = o.split(theta)
    s = np.empty(o.n_par)
    s[: o.n_sky] = np.repeat(np.sqrt(np.mean(a ** 2, axis=1)), o.nk)
    s[o.n_sky:] = 1.0
    return s


def test_chi2_zero_at_truth_and_noise_expectation():
    p, o, th, d, mu, lam = _setup("tiny", noise=False)
    c, U, g = o.chi2_grad(th, d, mu, lam)
    assert c == 0.0 and U == 0.0
    # with noise: chi^2 ~ chi-square with 2 N_vis dof (sigma per real component)
    p, o, th, d, mu, lam = _setup("small", noise=True)
    c, _, _ = o.chi2_grad(th, d)
    n = 2 * p.n_vis
    assert abs(c - n) < 5 * math.sqrt(2 * n)


def test_gradient_matches_central_differences():
    p, o, th, d, mu, lam = _setup("tiny")
    th = th + 0.02 * _scales(o, th) * np.random.default_rng(5).standard_normal(o.n_par)
    _, U0, g = o.chi2_grad(th, d, mu, lam)
    sc = _scales(o, th)
    rng = np.random.default_rng(6)
    # sky entries: U is quadratic along them, central difference is exact
    for k in rng.choice(o.n_sky, 8, replace=False):
        h = 0.3 * sc[k]
        e = np.zeros(o.n_par); e[k] = h
        fd = (o.chi2_grad(th + e, d, mu, lam)[1] - o.chi2_grad(th - e, d, mu, lam)[1]) / (2 * h)
        assert abs(fd - g[k]) < 1e-7 * max(abs(g).max() / 100, abs(g[k]))
    # gain entries: error O(h^2) -- halving h quarters it
    for k in o.n_sky + rng.choice(o.n_par - o.n_sky, 6, replace=False):
        errs = []
        for h in (1e-2, 5e-3):
            e = np.zeros(o.n_par); e[k] = h
            fd = (o.chi2_grad(th + e, d, mu, lam)[1] - o.chi2_grad(th - e, d, mu, lam)[1]) / (2 * h)
            errs.append(abs(fd - g[k]))
        assert errs[1] < 1e-4 * abs(g).max() + 1e-9
        assert errs[1] < errs[0] / 3.0 or errs[0] < 1e-9 * abs(g).max()


def test_adjoint_dot_product():
    # <J v, u> = <v, J^H u> for the sky block: J v is the model with sky v (gains fixed),
    # J^H u is the gradient when the residual equals sigma^2 u
    p, o, th, d, mu, lam = _setup("small")
    rng = np.random.default_rng(7)
    v = np.zeros(o.n_par)
    v[: o.n_sky] = rng.standard_normal(o.n_sky)
    v[o.n_sky:] = th[o.n_sky:]
    Jv = o.model(v)
    u = rng.standard_normal(Jv.shape) + 1j * rng.standard_normal(Jv.shape)
    m0 = o.model(th)
    dd = m0 - o.sigma ** 2 * u                     # residual r = sigma^2 u
    _, _, g = o.chi2_grad(th, dd)
    lhs = float(np.sum((np.conj(Jv) * u).real))
    g_th = o.chi2_grad(th, dd)[2]
    # gradient w.r.t. sky at theta uses the model at th; J is taken at th's gains
    rhs = float(v[: o.n_sky] @ g_th[: o.n_sky])
    assert abs(lhs - rhs) < 1e-11 * (abs(lhs) + 1.0)


def test_jacobian_columns_match_model_differences():
    p, o, th, d, mu, lam = _setup("tiny")
    J = o.jacobian(th)
    rng = np.random.default_rng(8)
    sc = _scales(o, th)
    for k in list(rng.choice(o.n_sky, 5, replace=False)) + list(o.n_sky + rng.choice(o.n_par - o.n_sky, 5, replace=False)):
        h = 0.5 * sc[k] if k < o.n_sky else 1e-4
        e = np.zeros(o.n_par); e[k] = h
        fd = (o.model(th + e) - o.model(th - e)).reshape(-1) / (2 * h)
        tol = 1e-9 if k < o.n_sky else 1e-6
        assert np.abs(fd - J[:, k]).max() < tol * np.abs(J).max()


def test_hvp_full_matches_gradient_differences_and_gn_at_zero_residual():
    p, o, th, d, mu, lam = _setup("tiny")
    rng = np.random.default_rng(9)
    sc = _scales(o, th)
    v = rng.standard_normal(o.n_par) * sc
    v_sky = v.copy(); v_sky[o.n_sky:] = 0.0
    Hv = o.hvp(th, d, v_sky, lam, full=True)
    h = 0.5
    fd = (o.chi2_grad(th + h * v_sky, d, mu, lam)[2] - o.chi2_grad(th - h * v_sky, d, mu, lam)[2]) / (2 * h)
    assert np.abs(fd - Hv).max() < 1e-8 * np.abs(Hv).max()          # exact: grad is quadratic in a
    v_g = np.zeros(o.n_par); v_g[o.n_sky:] = v[o.n_sky:]
    Hg = o.hvp(th, d, v_g, lam, full=True)
    errs = []
    for h in (1e-3, 5e-4):
        fd = (o.chi2_grad(th + h * v_g, d, mu, lam)[2] - o.chi2_grad(th - h * v_g, d, mu, lam)[2]) / (2 * h)
        errs.append(np.abs(fd - Hg).max())
    assert errs[1] < 1e-5 * np.abs(Hg).max()
    assert errs[1] < errs[0] / 3.0
    # GN == full when the residual is zero
    d0 = o.model(th)
    np.testing.assert_allclose(o.hvp(th, d0, v, lam, full=False), o.hvp(th, d0, v, lam, full=True),
                               rtol=0, atol=1e-10 * np.abs(o.hvp(th, d0, v, lam, full=True)).max())
    # but not at a nonzero residual (the curvature terms matter)
    diff = np.abs(o.hvp(th, d, v, lam, full=False) - o.hvp(th, d, v, lam, full=True)).max()
    assert diff > 1e-6 * np.abs(Hg).max()


def test_gn_hvp_and_blocks_equal_explicit_jacobian_products():
    p, o, th, d, mu, lam = _setup("tiny")
    J = o.jacobian(th)
    H = (J.conj().T @ J).real / o.sigma ** 2 + np.diag(lam)
    v = np.random.default_rng(10).standard_normal(o.n_par)
    np.testing.assert_allclose(o.hvp(th, d, v, lam, full=False), H @ v, rtol=0, atol=1e-10 * np.abs(H @ v).max())
    bs = 4
    blocks, Hg = o.gn_blocks(th, lam, bs)
    for blk, Hb in blocks.items():
        f, j0 = divmod(blk, o.nk // bs)
        s = f * o.nk + j0 * bs
        np.testing.assert_allclose(Hb, H[s:s + bs, s:s + bs], rtol=0, atol=1e-10 * np.abs(H).max())
    np.testing.assert_allclose(Hg, H[o.n_sky:, o.n_sky:], rtol=0, atol=1e-10 * np.abs(Hg).max())


def _mass(o, th, lam, bs=4):
    blocks, Hg = o.gn_blocks(th, lam, bs)
    out = []
    for blk in sorted(blocks):
        f, j0 = divmod(blk, o.nk // bs)
        s = f * o.nk + j0 * bs
        L, _ = oracle.cholesky_with_inflation(blocks[blk] - np.diag(lam[s:s + bs]), lam[s:s + bs])
        out.append((s, L))
    L, _ = oracle.cholesky_with_inflation(Hg - np.diag(lam[o.n_sky:]), lam[o.n_sky:])
    out.append((o.n_sky, L))
    return oracle.BlockCholesky(out)


def test_block_cholesky_algebra():
    p, o, th, d, mu, lam = _setup("tiny")
    mass = _mass(o, th, lam)
    Mfull = np.zeros((o.n_par, o.n_par))
    for s, L in mass.blocks:
        n = L.shape[0]
        Mfull[s:s + n, s:s + n] = L @ L.T
    p0 = np.random.default_rng(11).standard_normal(o.n_par)
    p_ = mass.mul_lower(p0)
    z = mass.solve_lower(p_)
    np.testing.assert_allclose(z, p0, atol=1e-9 * np.abs(p0).max())
    # K = z^T z / 2 equals p^T M^-1 p / 2 and the drift equals M^-1 p (library solve)
    minv_p = np.linalg.solve(Mfull, p_)
    assert abs(0.5 * z @ z - 0.5 * p_ @ minv_p) < 1e-9 * abs(p_ @ minv_p)
    np.testing.assert_allclose(mass.solve_upper_t(z), minv_p, rtol=1e-7, atol=1e-12 * np.abs(minv_p).max())


def _grad_fn(o, d, mu, lam):
    def fn(q):
        _, U, g = o.chi2_grad(q, d, mu, lam)
        return U, g
    return fn


def test_leapfrog_reversible_and_second_order():
    p, o, th, d, mu, lam = _setup("tiny")
    mass = _mass(o, th, lam)
    fn = _grad_fn(o, d, mu, lam)
    p0 = mass.mul_lower(np.random.default_rng(12).standard_normal(o.n_par))
    q1, p1, H0, H1, acc = oracle.leapfrog(fn, th, p0, 0.1, 10, 0.0, mass)
    assert acc
    q2, p2, _, _, _ = oracle.leapfrog(fn, q1, -p1, 0.1, 10, 0.0, mass)
    sc = _scales(o, th)
    assert np.abs((q2 - th) / sc).max() < 1e-8
    assert np.abs(p2 + p0).max() < 1e-8 * np.abs(p0).max()
    # energy error of a fixed-length trajectory falls as eps^2
    dH = []
    for eps, n in ((0.2, 10), (0.1, 20), (0.05, 40)):
        _, _, a, b, _ = oracle.leapfrog(fn, th, p0, eps, n, 0.0, mass)
        dH.append(abs(b - a))
    s1, s2 = math.log2(dH[0] / dH[1]), math.log2(dH[1] / dH[2])
    assert 1.7 < s1 < 2.4 and 1.7 < s2 < 2.4


def test_metropolis_rule_uses_u_against_exp_delta_h():
    p, o, th, d, mu, lam = _setup("tiny")
    mass = _mass(o, th, lam)
    fn = _grad_fn(o, d, mu, lam)
    p0 = mass.mul_lower(np.random.default_rng(13).standard_normal(o.n_par))
    _, _, H0, H1, _ = oracle.leapfrog(fn, th, p0, 0.4, 5, 0.0, mass)
    a = math.exp(min(0.0, H0 - H1))
    if a < 1.0:
        assert oracle.leapfrog(fn, th, p0, 0.4, 5, a * 0.999, mass)[4]
        q, _, _, _, acc = oracle.leapfrog(fn, th, p0, 0.4, 5, min(a * 1.001, 0.9999999), mass)
        assert not acc and np.array_equal(q, th)
    else:
        assert oracle.leapfrog(fn, th, p0, 0.4, 5, 0.999999, mass)[4]


def test_global_gain_phase_is_a_gauge_and_gain_scale_is_quadratic():
    # m_pq = g_p conj(g_q) V_pq: one common phase on every gain cancels, a common real
    # factor c scales every model visibility by c^2 (a dropped conjugate breaks both)
    p, o, th, d, mu, lam = _setup("tiny")
    a, gam = o.split(th)
    m0 = o.model(th)
    for phase in (0.3, -1.9):
        th2 = th.copy()
        g2 = th2[o.n_sky:].reshape(o.A, o.NG, 2)
        gc = (gam[..., 0] + 1j * gam[..., 1]) * np.exp(1j * phase)
        g2[..., 0], g2[..., 1] = gc.real, gc.imag
        np.testing.assert_allclose(o.model(th2), m0, atol=1e-12 * np.abs(m0).max())
    th3 = th.copy()
    th3[o.n_sky:] *= 1.7
    np.testing.assert_allclose(o.model(th3), 1.7 ** 2 * m0, atol=1e-12 * np.abs(m0).max())


def test_prior_inflation_takes_the_first_spd_factor():
    # M = H_lik + c diag(lam) for the first c in 1, 1.1, 1.21, ... that is SPD: with
    # H_lik = diag(-2, 1) and lam = 1 that needs c > 2, first reached at c = 1.1^8
    H = np.diag([-2.0, 1.0])
    lam = np.array([1.0, 1.0])
    L, c = oracle.cholesky_with_inflation(H, lam)
    want = 1.0
    for _ in range(8):
        want *= 1.1
    assert c == want and want > 2.0 and want / 1.1 < 2.0
    np.testing.assert_allclose(L @ L.T, H + c * np.diag(lam), rtol=1e-14)
    # an SPD H_lik is factorised with c = 1 (no inflation)
    L1, c1 = oracle.cholesky_with_inflation(np.array([[4.0, 1.0], [1.0, 3.0]]), lam)
    assert c1 == 1.0
    np.testing.assert_allclose(L1 @ L1.T, [[5.0, 1.0], [1.0, 4.0]], rtol=1e-14)
