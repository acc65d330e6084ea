"""Launch grids of the hour-angle contraction kernels and their autotuner (the batched
schedule of independent problems):

- fewer CTAs re-partition the forward's work units: the results stay within the parity bounds
  against the FP64 oracle and within FP32 rounding of the default grid's;
- the grids are validated (at most one CTA per SM; the direct form has none);
- the tuner times each problem shape once, caches the times by shape in JSON, picks per
  problem the fewest CTAs within the slack of the best, and a second call reads the cache."""
import json

import numpy as np
import pytest

from gpu_cases import bound, handle, key, make_case, perturbed, quant, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_07090_gb300 import build
    build.build()


def _t(a, h):
    import torch
    return torch.tensor(np.asarray(a), dtype=h.dtype, device="cuda").contiguous()


@pytest.mark.parametrize("grids", [(19, 38), (8, 152), (1, 1)])
def test_smaller_grids_keep_parity(grids, check_err):
    prec = "fp16x3"
    p, o, th, d, mu, lam = make_case("ha37")
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    th = quant(prec, perturbed(o, th, 0.01, 2))
    t = _t(th, h)
    V0 = h.forward(t).clone()
    _, g0 = h.chi2_grad(t)
    g0 = g0.clone()
    h.set_launch_grids(*grids)
    assert h.launch_grids()[0] == grids[0]
    V1 = h.forward(t)
    _, g1 = h.chi2_grad(t)
    V1n = V1.double().cpu().numpy()
    check_err(rel_l2(V1n[..., 0] + 1j * V1n[..., 1], o.model(th)), bound("hour_angle", "V", prec, "ha37"),
              key("hour_angle", "V_grid", prec), f"ha37 grids {grids}")
    _, _, g = o.chi2_grad(th, d, mu, lam)
    check_err(rel_l2(g1.cpu().numpy(), g), bound("hour_angle", "grad", prec, "ha37"),
              key("hour_angle", "grad_grid", prec), f"ha37 grids {grids}")
    assert rel_l2(V1.cpu().numpy(), V0.cpu().numpy()) < 1e-6
    assert rel_l2(g1.cpu().numpy(), g0.cpu().numpy()) < 1e-5


def test_grids_are_validated():
    import torch
    from paper_2504_07090_gb300 import fm
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    p, o, th, d, mu, lam = make_case("ha37")
    h = handle(p, "fp16x3")
    with pytest.raises(fm.FmError) as e:
        h.set_launch_grids(sm + 1, 0)
    assert e.value.status == fm.FM_ERR_INVALID_ARG
    h.set_launch_grids(0, 0)
    g_f, g_a = h.launch_grids()
    assert 1 <= g_f <= sm and 1 <= g_a <= sm
    p2, *_ = make_case("small")
    h2 = handle(p2, "fp32")
    with pytest.raises(fm.FmError) as e:
        h2.set_launch_grids(8, 8)
    assert e.value.status == fm.FM_ERR_UNSUPPORTED


def test_tuner_caches_by_shape(tmp_path):
    import torch
    from paper_2504_07090_gb300 import autotune
    models, thetas = [], []
    for name in ("ha37", "ha37", "ha7"):
        p, o, th, d, mu, lam = make_case(name)
        d, mu, lam = quant("fp16x3", d, mu, lam)
        h = handle(p, "fp16x3", d, mu, lam)
        models.append(h)
        thetas.append(_t(quant("fp16x3", th), h))
    path = str(tmp_path / "grids.json")
    tables, timed = autotune.shape_times(models, thetas, path, candidates=(4, 16, 152), reps=2)
    assert timed == 2                       # two distinct shapes among three problems
    cache = json.load(open(path))
    assert set(cache) == {autotune.shape_key(models[0]), autotune.shape_key(models[2])}
    for tab in tables:
        assert set(tab) == {"4", "16", "152"} and all(v > 0 for v in tab.values())
    chosen = autotune.apply(models, tables, 1.25)
    for g, tab in zip(chosen, tables):
        assert g == autotune.choose(tab, 1.25) and tab[str(g)] <= 1.25 * min(tab.values())
        assert all(int(c) >= g for c, v in tab.items() if v <= 1.25 * min(tab.values()))
    assert models[0].launch_grids()[0] == chosen[0]
    _, timed2 = autotune.shape_times(models, thetas, path, candidates=(4, 16, 152), reps=2)
    assert timed2 == 0
    torch.cuda.synchronize()
