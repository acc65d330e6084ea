"""Legendre-in-frequency sky compression (fm_config.n_freq_modes; Eq. fg_legendre) through the
CUDA path against the oracle: visibilities, chi^2 and gradient, the Gauss-Newton and full HVPs,
the mass-matrix blocks, a leapfrog trajectory, the filtered likelihood, and the exact central
differences of the device U along compressed sky directions.  Cases: the direct FP64 / FP32
sums on `small` (6 channels onto 3 orders) and the hour-angle split forms on ha37 / ha37m
(3 channels onto 2 orders)."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from gpu_cases import bound, handle, key, make_case, perturbed, quant, rel_l2

pytestmark = pytest.mark.gpu

CASES = [("small", 3, "fp64"), ("small", 3, "fp32"), ("ha37", 2, "fp16x3"), ("ha37", 2, "bf16x3"),
         ("small", 6, "fp32")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_07090_gb300 import build
    build.build()


def _t(a, h):
    import torch
    return torch.tensor(np.asarray(a), dtype=h.dtype, device="cuda").contiguous()


def _form(h):
    return h.contraction_info()["form"]


def test_handle_sizes_and_validation():
    from paper_2504_07090_gb300 import fm, synth
    p, o, th, d, mu, lam = make_case("small", freq_modes=3)
    h = handle(p, "fp32")
    assert h.n_params == o.n_par == 3 * p.n_modes + 2 * p.n_ant * p.n_gain
    bad = replace(synth.config("small"), n_freq_modes=p.n_freq + 1)
    with pytest.raises(fm.FmError) as e:
        fm.ForwardModel(bad, "fp32")
    assert e.value.status == fm.FM_ERR_INVALID_ARG


@pytest.mark.parametrize("name,K,prec", CASES)
def test_vis_chi2_gradient_match_oracle(name, K, prec, check_err):
    p, o, th, d, mu, lam = make_case(name, freq_modes=K)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    form = _form(h)
    if name.startswith("ha"):
        assert form == "hour_angle"
    th = quant(prec, perturbed(o, th, 0.01, 3))
    t = _t(th, h)
    V = h.forward(t).double().cpu().numpy()
    check_err(rel_l2(V[..., 0] + 1j * V[..., 1], o.model(th)), bound(form, "V", prec, name),
              key(form, "V_K", prec), f"{name} K{K}")
    chi2, U, g = o.chi2_grad(th, d, mu, lam)
    scal, grad = h.chi2_grad(t)
    scal = scal.cpu().numpy()
    # |chi2' - chi2| <= 2 sqrt(chi2) |dm| / sigma + |dm|^2 / sigma^2 with |dm| <= tol_V |m| (x2 margin)
    dm = bound(form, "V", prec, name) * np.linalg.norm(o.model(th)) / o.sigma
    cb = 2.0 * (2.0 * np.sqrt(chi2) * dm + dm * dm) + 1e-12 * chi2
    check_err(abs(scal[0] - chi2) / chi2, cb / chi2, key(form, "chi2_K", prec), f"{name} K{K}")
    assert abs(scal[1] - U) < 0.5 * cb + 1e-12 * U
    check_err(rel_l2(grad.cpu().numpy(), g), bound(form, "grad", prec, name), key(form, "grad_K", prec),
              f"{name} K{K}")
    x = h.sky_pixels(t).double().cpu().numpy().reshape(o.F, -1)
    a, _ = o.split(th)
    check_err(rel_l2(x, o.sky(a)), 1e-12 if prec == "fp64" else 1e-6, key("modes", "x_K", prec), f"{name} K{K}")
    h.sync_status()


@pytest.mark.parametrize("name,K,prec", CASES[:4])
@pytest.mark.parametrize("full", [False, True])
def test_hvp_matches_oracle(name, K, prec, full, check_err):
    p, o, th, d, mu, lam = make_case(name, freq_modes=K)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    th = quant(prec, perturbed(o, th, 0.01, 4))
    v = quant(prec, np.random.default_rng(5).standard_normal(o.n_par) * np.abs(th).mean())
    want = o.hvp(th, d, v, lam, full=full)
    got = h.hvp(_t(th, h), _t(v, h), full=full).cpu().numpy()
    form = _form(h)
    check_err(rel_l2(got, want), bound(form, "grad", prec, name), key(form, "hvp_full_K" if full else "hvp_gn_K", prec),
              f"{name} K{K}")


@pytest.mark.parametrize("prec,name,K,bs", [("fp64", "small", 3, 64), ("fp32", "small", 3, 64),
                                            ("fp32", "small", 3, 1), ("fp16x3", "ha37m", 2, 64)])
def test_gn_blocks_match_oracle(prec, name, K, bs, check_err):
    p, o, th, d, mu, lam = make_case(name, freq_modes=K)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    th = quant(prec, perturbed(o, th, 0.01, 5))
    h.build_precond(_t(th, h), bs)
    got = h.precond_blocks().cpu().numpy()
    if bs == 1:
        J = o.jacobian(th)
        diag = np.sum(np.abs(J) ** 2, axis=0) / o.sigma ** 2 + lam
        sky, gain = diag[: o.n_sky], diag[o.n_sky:]
    else:
        blocks, gain = o.gn_blocks(th, lam, bs)
        sky = np.stack([blocks[k] for k in sorted(blocks)])
    n_sky = sky.size
    tol = 1e-10 if prec == "fp64" else 1e-4
    check_err(rel_l2(got[:n_sky], sky.reshape(-1)), tol, key("precond", "gn_sky_K", prec), f"{name} K{K} bs{bs}")
    check_err(rel_l2(got[n_sky:], gain.reshape(-1)), tol, key("precond", "gn_gain_K", prec), f"{name} K{K} bs{bs}")


def _oracle_mass(o, th, lam, bs):
    blocks, Hg = o.gn_blocks(th, lam, bs)
    out = []
    for blk in sorted(blocks):
        l, j0 = divmod(blk, o.nk // bs)
        s = l * o.nk + j0 * bs
        L, _ = oracle.cholesky_with_inflation(blocks[blk] - np.diag(lam[s:s + bs]), lam[s:s + bs])
        out.append((s, L))
    L, _ = oracle.cholesky_with_inflation(Hg - np.diag(lam[o.n_sky:]), lam[o.n_sky:])
    out.append((o.n_sky, L))
    return oracle.BlockCholesky(out)


@pytest.mark.parametrize("name,K,prec,eps,prior", [("small", 3, "fp64", 0.1, (0.05, 0.05)),
                                                   ("small", 3, "fp32", 0.1, (0.05, 0.05)),
                                                   ("ha37m", 2, "fp16x3", 0.01, (0.005, 0.005))])
def test_leapfrog_trajectory_matches_oracle(name, K, prec, eps, prior, check_err):
    p, o, th, d, mu, lam = make_case(name, prior=prior, freq_modes=K)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    q0 = quant(prec, perturbed(o, th, 0.005, 6))
    mass = _oracle_mass(o, q0, lam, 64)
    p0 = quant(prec, mass.mul_lower(np.random.default_rng(7).standard_normal(o.n_par)))
    n = 20

    def fn(q):
        _, U, g = o.chi2_grad(q, d, mu, lam)
        return U, g

    qw, pw, H0, H1, acc = oracle.leapfrog(fn, q0, p0, eps, n, 0.0, mass)
    tq, tp = _t(q0, h), _t(p0, h)
    h.build_precond(tq, 64)
    hout, aout = h.leapfrog(tq, tp, eps, n, 0.0)
    hh = hout.cpu().numpy()
    exact = prec == "fp64"
    form = _form(h)
    tol_q = 1e-9 if exact else (1e-4 if name == "small" else 2e-4)
    check_err(rel_l2(tq.cpu().numpy() - q0, qw - q0), tol_q, key(form, "lf_q_K", prec), f"{name} K{K}")
    check_err(rel_l2(tp.cpu().numpy(), pw), tol_q, key(form, "lf_p_K", prec), f"{name} K{K}")
    check_err(abs(hh[0] - H0) / abs(H0), 1e-12 if exact else 1e-5, key(form, "H0_K", prec), f"{name} K{K}")
    e_dh = abs((hh[1] - hh[0]) - (H1 - H0)) / max(1.0, abs(H1 - H0))
    # the split modes' energy change: an absolute error of order one (the bound and its
    # derivation as in the uncompressed trajectory test)
    check_err(e_dh, 1e-9 if exact else (2e-2 if form == "direct" else 3.0), key(form, "dH_K", prec), f"{name} K{K}")
    assert int(aout.item()) == 1


# chi^2 bounds as for the uncompressed filter on cfg0; gradient bounds relative to the terms'
# size (below), a little above the measured 1.2e-9 (FP64), 1.3e-8 (FP32), 2.0e-8 (FP16 split)
FILTER_K_BOUNDS = {"fp64": (1e-7, 1e-8), "fp32": (1e-5, 1e-7), "fp16x3": (5e-6, 1e-7)}


@pytest.mark.parametrize("prec", list(FILTER_K_BOUNDS))
def test_filtered_likelihood_with_compression(prec, check_err):
    tau, eps = 250e-9, 1e-8
    p, o, th, d, mu, lam = make_case("cfg0", freq_modes=3)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    h.set_delay_filter(tau, eps)
    th = quant(prec, perturbed(o, th, 0.01, 8))
    Fm = oracle.delay_filter(p.freq_hz, tau, eps)
    chi2, U, g = o.chi2_grad_filtered(th, d, Fm, mu, lam)
    scal, grad = h.chi2_grad(_t(th, h))
    form = _form(h)
    b_c, b_g = FILTER_K_BOUNDS[prec]
    check_err(abs(float(scal[0]) - chi2) / chi2, b_c, key(form, "filtered_chi2_K", prec), "cfg0 K3")
    # The filter removes the spectra that three Legendre orders (and the gains' four) can
    # make, so the gradient J^T F^T (r~ / N~) is a sum that cancels: here to 4e-5 of its terms.
    # A filter that differs by dF (the two sides build it by different factorisations; FP32
    # rounds it) moves it by J^T dF^T (r~ / N~), whose size is set by the terms
    # J^T (r~ / N~) without the last F^T; the error is measured against their norm.
    r = o.model(th) - d
    rt = np.einsum("fg,gtb->ftb", Fm, r)
    ntil = o.sigma ** 2 * np.sum(Fm * Fm, axis=1)
    terms = o.grad_from_weights(th, rt / ntil[:, None, None])
    err = float(np.linalg.norm(grad.double().cpu().numpy() - g) / np.linalg.norm(terms))
    check_err(err, b_g, key(form, "filtered_grad_K_terms", prec), "cfg0 K3")
    h.sync_status()


def test_central_differences_of_device_u(check_err):
    # the model is linear in the compressed sky coefficients: U is quadratic along them and
    # a central difference of the device's own U is exact up to its rounding
    prec = "fp16x3"
    p, o, th, d, mu, lam = make_case("ha37", freq_modes=2)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    th = quant(prec, perturbed(o, th, 0.01, 9))
    scal, grad = h.chi2_grad(_t(th, h))
    U0 = float(scal[1].item())
    g = grad.double().cpu().numpy()
    rng = np.random.default_rng(10)
    errs = []
    for _ in range(6):
        v = np.zeros(o.n_par)
        v[: o.n_sky] = g[: o.n_sky] / np.linalg.norm(g[: o.n_sky]) + rng.standard_normal(o.n_sky) / np.sqrt(o.n_sky)
        v /= np.linalg.norm(v)
        gv = float(g @ v)
        hs = 0.01 * abs(U0) / abs(gv)
        up = float(h.chi2_grad(_t(th + hs * v, h))[0][1].item())
        dn = float(h.chi2_grad(_t(th - hs * v, h))[0][1].item())
        errs.append(abs((up - dn) / (2 * hs) - gv) / abs(gv))
    check_err(max(errs), 1e-4, key("hour_angle", "fd_sky_K", prec), "ha37 K2")
