"""Parity at the full benchmark size (cfg1: 37 antennas, 64 channels, 60 LSTs, 24,576
pixels, 16,384 modes per channel), in the launch configuration bench.py times:

- every visibility of one channel (60 LSTs x 666 baselines) against the oracle's
  per-baseline sum, and sampled visibilities of three more channels computed one by one;
- the complete sky gradient of one channel (all LSTs) against the oracle's adjoint, with
  the data of the other channels zero (sky modes are per channel, so that slice of the
  gradient depends on this channel alone);
- on a two-channel sub-band of the same geometry (same array, pixel grid, LSTs and modes;
  every kernel runs its cfg1 tiling with fewer channels), the whole gradient including the
  gain coefficients, and the Gauss-Newton and full HVPs.

Gradients are compared away from the truth (sky modes perturbed by 1 % of the channel
rms).  At the truth the residual is pure noise, the true gradient is its incoherent
projection, and any model error eps adds a coherent bias of relative size about
eps |m|/sigma sqrt(N_vis) -- at cfg1 that is percent level even for FP32 -- so the
relative metric there measures the noise, not the kernels."""
import numpy as np
import pytest

import oracle
from gpu_cases import as_complex, bound, key, quant, rel_l2

pytestmark = pytest.mark.gpu

FORM = {"fp32": "direct", "fp16x3": "hour_angle", "bf16x3": "hour_angle"}


def _perturbed(o, theta, frac, seed, gains=0.0):
    a, _ = o.split(theta)
    sc = np.zeros(o.n_par)
    sc[: o.n_sky] = np.repeat(np.sqrt(np.mean(a ** 2, axis=1)), o.nk)
    sc[o.n_sky:] = gains
    return theta + frac * sc * np.random.default_rng(seed).standard_normal(o.n_par)


@pytest.fixture(scope="module")
def cfg1():
    from paper_2504_07090_gb300 import build, synth
    build.build()
    p = synth.config("cfg1")
    tr = synth.draw_truth(p)
    o = oracle.Oracle(p)
    return p, o, tr


@pytest.fixture(scope="module")
def channel_model(cfg1):
    """Oracle model visibilities of one channel at the truth (float32-rounded parameters)."""
    p, o, tr = cfg1
    f0 = int(np.random.default_rng(3).integers(p.n_freq))
    th = quant("fp32", tr.theta)
    return f0, o.model(th, fts=[(f0, t) for t in range(p.n_lst)])[f0]


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3", "fp32"])
def test_cfg1_visibilities(cfg1, channel_model, prec, check_err):
    import torch
    from paper_2504_07090_gb300 import fm
    p, o, tr = cfg1
    th = quant(prec, tr.theta)
    h = fm.ForwardModel(p, prec, sigma=1.0)
    assert h.contraction_info()["form"] == FORM[prec]
    V = as_complex(h.forward(torch.tensor(th, dtype=torch.float32, device="cuda")))
    f0, m0 = channel_model
    check_err(rel_l2(V[f0], m0), bound(FORM[prec], "V", prec, "cfg1"), key(FORM[prec], "V", prec),
              f"cfg1 channel {f0}")
    # sampled visibilities of three other channels, one by one
    rng = np.random.default_rng(4)
    a, gam = o.split(th)
    g = o.gains(gam)
    got, want = [], []
    for f in rng.choice([k for k in range(p.n_freq) if k != f0], 3, replace=False):
        x_f = o.sky_f(a[f])
        for _ in range(8):
            t, b = int(rng.integers(p.n_lst)), int(rng.integers(p.n_bl))
            want.append(o.vis_one(int(f), t, b, x_f) * g[f, o.bl_i[b]] * np.conj(g[f, o.bl_j[b]]))
            got.append(V[f, t, b])
    check_err(rel_l2(np.array(got), np.array(want)), bound(FORM[prec], "V", prec, "cfg1"),
              key(FORM[prec], "V", prec), "cfg1 sampled")
    h.close()


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3", "fp32"])
def test_cfg1_one_channel_gradient(cfg1, channel_model, prec, check_err):
    import torch
    from paper_2504_07090_gb300 import fm
    p, o, tr = cfg1
    f0, m0 = channel_model
    # data of channel f0: oracle model plus seeded noise of 1 % of its mean |V| (other channels 0)
    sigma = 0.01 * float(np.mean(np.abs(m0)))
    p.sigma = sigma
    o.sigma = sigma
    d_full = np.zeros((p.n_freq, p.n_lst, p.n_bl), dtype=np.complex128)
    d_full[f0] = m0 + sigma * (tr.noise[f0, ..., 0] + 1j * tr.noise[f0, ..., 1])
    d_full = quant(prec, d_full)
    h = fm.ForwardModel(p, prec, sigma=sigma)
    h.set_data(torch.tensor(np.stack([d_full.real, d_full.imag], -1), dtype=torch.float32, device="cuda").contiguous())
    th_eval = quant(prec, _perturbed(o, quant(prec, tr.theta), 0.01, 6))
    _, grad = h.chi2_grad(torch.tensor(th_eval, dtype=torch.float32, device="cuda"))
    chi2, U, g = o.chi2_grad(th_eval, d_full, fts=[(f0, t) for t in range(p.n_lst)])
    sl = slice(f0 * o.nk, (f0 + 1) * o.nk)
    check_err(rel_l2(grad.cpu().numpy()[sl], g[sl]), bound(FORM[prec], "grad", prec, "cfg1"),
              key(FORM[prec], "grad", prec), f"cfg1 channel {f0} sky")
    h.close()


@pytest.fixture(scope="module")
def subband(cfg1):
    """Channels 20 and 21 of cfg1 as a problem of its own, with oracle data and prior."""
    from dataclasses import replace
    from paper_2504_07090_gb300 import synth
    p1, _, tr1 = cfg1
    p = replace(p1, name="cfg1 sub-band", freq_hz=p1.freq_hz[20:22].copy())
    nk = p.n_modes
    theta = np.concatenate([tr1.theta[20 * nk:22 * nk], tr1.theta[p1.n_sky_params:]])
    theta = quant("fp32", theta)
    o = oracle.Oracle(p)
    m = o.model(theta)
    p.sigma = o.sigma = 0.01 * float(np.mean(np.abs(m)))
    d = quant("fp32", m + p.sigma * (tr1.noise[20:22, ..., 0] + 1j * tr1.noise[20:22, ..., 1]))
    mu, lam = synth.prior_for(p, theta)
    mu, lam = quant("fp32", mu, lam)
    th = quant("fp32", _perturbed(o, theta, 0.01, 7, gains=0.01))
    v = quant("fp32", _perturbed(o, np.zeros_like(theta), 1.0, 8, gains=0.01))
    return p, o, th, d, mu, lam, v


def test_cfg1_subband_gradient_and_hvp(subband, check_err):
    import torch
    from gpu_cases import handle
    p, o, th, d, mu, lam, v = subband
    prec = "fp16x3"
    h = handle(p, prec, d, mu, lam)
    assert h.contraction_info()["form"] == "hour_angle"
    tt = torch.tensor(th, dtype=torch.float32, device="cuda")
    _, grad = h.chi2_grad(tt)
    chi2, U, g = o.chi2_grad(th, d, mu, lam)
    grad = grad.cpu().numpy()
    cb = bound("hour_angle", "grad", prec, "cfg1 sub-band")
    check_err(rel_l2(grad, g), cb, key("hour_angle", "grad", prec), "cfg1 sub-band")
    check_err(rel_l2(grad[o.n_sky:], g[o.n_sky:]), cb, key("hour_angle", "grad_gains", prec), "cfg1 sub-band")
    hv = h.hvp(tt, torch.tensor(v, dtype=torch.float32, device="cuda"), full=False).cpu().numpy()
    check_err(rel_l2(hv, o.hvp(th, d, v, lam, full=False)), cb, key("hour_angle", "hvp_gn", prec), "cfg1 sub-band")
    h.close()
