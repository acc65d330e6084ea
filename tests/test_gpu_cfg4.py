"""The largest workload (cfg4: 127-antenna hexagon, 8001 baselines in 234 fringe groups,
128 channels 120-180 MHz, 120 LSTs run as two hour-angle passes of 64 and 56, 256 x 384
pixels, 256 x 256 modes per channel) in the launch configuration bench.py times:

- visibilities sampled over channels, both LST passes and baselines, each summed one by one
  by the FP64 oracle (the whole-channel oracle takes minutes at this size);
- central differences of the device's own U along sky directions against its gradient (U is
  quadratic in the sky modes, so the difference is exact for any step)."""
import numpy as np
import pytest

import oracle
from gpu_cases import bound, key, quant, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg4():
    import torch
    from paper_2504_07090_gb300 import build, fm, synth
    build.build()
    p = synth.config("cfg4")
    tr = synth.draw_truth(p)
    h = fm.ForwardModel(p, "fp16x3", sigma=1.0)
    th = quant("fp16x3", tr.theta)
    V = h.forward(torch.tensor(th, dtype=torch.float32, device="cuda"))
    yield p, tr, th, h, V
    h.close()


def test_cfg4_runs_the_hour_angle_form_in_two_passes(cfg4):
    p, tr, th, h, V = cfg4
    info = h.contraction_info()
    assert info["form"] == "hour_angle" and info["fringes"] == 234
    assert p.n_lst == 120 and p.n_bl == 8001


def test_cfg4_sampled_visibilities(cfg4, check_err):
    import torch
    p, tr, th, h, V = cfg4
    o = oracle.Oracle(p)
    a, gam = o.split(th)
    g = o.gains(gam)
    rng = np.random.default_rng(11)
    idx, want = [], []
    for f in rng.choice(p.n_freq, 4, replace=False):
        x_f = o.sky_f(a[f])
        for k in range(10):
            t = int(rng.integers(64)) if k % 2 == 0 else 64 + int(rng.integers(56))    # both passes
            b = int(rng.integers(p.n_bl))
            idx.append((int(f), t, b))
            want.append(o.vis_one(int(f), t, b, x_f) * g[f, o.bl_i[b]] * np.conj(g[f, o.bl_j[b]]))
    ii = torch.tensor(idx, dtype=torch.long, device="cuda")
    got = V[ii[:, 0], ii[:, 1], ii[:, 2]].double().cpu().numpy()
    check_err(rel_l2(got[:, 0] + 1j * got[:, 1], np.array(want)), bound("hour_angle", "V", "fp16x3", "cfg1"),
              key("hour_angle", "V", "fp16x3"), "cfg4 sampled")


def test_cfg4_central_differences_of_device_u(cfg4, check_err):
    import torch
    from paper_2504_07090_gb300 import fm, synth
    p, tr, th, h0, V = cfg4
    sigma = 0.01 * float(torch.linalg.norm(V, dim=-1).mean())
    h = fm.ForwardModel(p, "fp16x3", sigma=sigma)
    h.set_data((V + sigma * torch.tensor(tr.noise, dtype=torch.float32, device="cuda")).contiguous())
    mu, lam = synth.prior_for(p, tr.theta)
    h.set_prior(torch.tensor(mu, dtype=torch.float32, device="cuda"), torch.tensor(lam, dtype=torch.float32, device="cuda"))
    n_sky = p.n_sky_params
    a = tr.theta[:n_sky].reshape(p.n_freq, -1)
    sc = np.zeros(p.n_params)
    sc[:n_sky] = np.repeat(np.sqrt(np.mean(a ** 2, axis=1)), p.n_modes)
    th1 = quant("fp16x3", th + 0.01 * sc * np.random.default_rng(12).standard_normal(p.n_params))
    dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")   # noqa: E731
    scal, grad = h.chi2_grad(dev(th1))
    U0 = float(scal[1].item())
    gv_all = grad.double().cpu().numpy()
    gs = np.zeros(p.n_params)
    gs[:n_sky] = gv_all[:n_sky] / np.linalg.norm(gv_all[:n_sky])
    rng = np.random.default_rng(13)
    errs = []
    for _ in range(4):
        r = np.zeros(p.n_params)
        r[:n_sky] = rng.standard_normal(n_sky)
        v = gs + r / np.linalg.norm(r)
        v /= np.linalg.norm(v)
        gv = float(gv_all @ v)
        hs = 0.01 * abs(U0) / abs(gv)
        up = float(h.chi2_grad(dev(th1 + hs * v))[0][1].item())
        dn = float(h.chi2_grad(dev(th1 - hs * v))[0][1].item())
        errs.append(abs((up - dn) / (2.0 * hs) - gv) / abs(gv))
    check_err(max(errs), 1e-4, key("hour_angle", "fd_sky", "fp16x3"), "cfg4")
    h.close()
