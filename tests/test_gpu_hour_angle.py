"""Hour-angle form of the tensor-core contraction (drift scans whose LST step is k / q RA
pixels, q <= 4) against the FP64 oracle, element by element.

ha7: 7-antenna hexagon, LST step 2 pixels (9 baseline groups); hachunk: a 91-antenna hexagon
(165 groups, a 29-antenna table) over 70 LSTs (two passes of at most 64); ha37: the 37-antenna
hexagon, step 1 (63 groups, 666 baselines); harand: 12 antennas at random 3-D offsets
(66 groups: two forward M-tiles, three adjoint K chunks); hafrac2: step 2.5 pixels (cells of
half a pixel, 5 per step); hafrac4: 19-antenna hexagon, step 0.75 pixel (cells of a quarter
pixel, 3 per step).  Each runs with baseline grouping on and off (FM_HA_GROUPS=0: every
baseline its own group, 11 M-tiles and 21 K chunks for ha37).  Every error is held to the
hour-angle bound of its precision (gpu_cases.BOUNDS) and recorded in the run's summary."""
import numpy as np
import pytest

from gpu_cases import as_complex, bound, handle, key, make_case, perturbed, quant, rel_l2

pytestmark = pytest.mark.gpu

# groups, baselines, LST step in hour-angle cells k, cells per RA pixel q
CASES = {"ha7": (9, 21, 2, 1), "ha37": (63, 666, 1, 1), "harand": (66, 66, 1, 1), "hafrac2": (9, 21, 5, 2),
         "hafrac4": (30, 171, 3, 4), "hachunk": (165, 4095, 1, 2)}
# hachunk has 91 antennas: with every baseline its own group the table would need all of
# them (more than its 63 entries), so it runs grouped only
PRECS = ["bf16x1", "bf16x3", "fp16x1", "fp16x3"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2504_07090_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _t(a, h):
    import torch
    return torch.tensor(np.asarray(a), dtype=h.dtype, device="cuda").contiguous()


def _groups(monkeypatch, on, name=None):
    if not on and name == "hachunk":
        pytest.skip("91 antennas: the hour-angle form needs baseline grouping")
    monkeypatch.setenv("FM_HA_GROUPS", "1" if on else "0")


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("grouped", [True, False])
def test_handle_runs_the_hour_angle_form(name, grouped, monkeypatch):
    _groups(monkeypatch, grouped, name)
    p, o, th, d, mu, lam = make_case(name)
    info = handle(p, "fp16x3").contraction_info()
    ng, nb, k, q = CASES[name]
    assert info["form"] == "hour_angle"
    assert info["fringes"] == (ng if grouped else nb)
    assert info["lst_step_cells"] == k
    assert info["hour_angle_cells"] % 128 == 0
    assert info["hour_angle_cells"] >= (p.n_ra - 1) * q + (p.n_lst - 1) * k + 1


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("grouped", [True, False])
def test_forward_pixels_matches_oracle(name, prec, grouped, monkeypatch, check_err):
    _groups(monkeypatch, grouped, name)
    p, o, th, d, mu, lam = make_case(name)
    h = handle(p, prec)
    a, _ = o.split(th)
    x = quant(prec, o.sky(a))
    got = as_complex(h.forward_pixels(_t(x, h)))
    case = name + ("" if grouped else " ungrouped")
    check_err(rel_l2(got, o.vis(x)), bound("hour_angle", "V", prec, name), key("hour_angle", "V", prec), case)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("grouped", [True, False])
def test_chi2_and_gradient_match_oracle(name, prec, grouped, monkeypatch, check_err):
    _groups(monkeypatch, grouped, name)
    p, o, th, d, mu, lam = make_case(name)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    th = quant(prec, perturbed(o, th, 0.01, 2))
    chi2, U, g = o.chi2_grad(th, d, mu, lam)
    scal, grad = h.chi2_grad(_t(th, h))
    scal = scal.cpu().numpy()
    dm = bound("hour_angle", "V", prec, name) * np.linalg.norm(o.model(th)) / o.sigma
    cb = 2.0 * (2.0 * np.sqrt(chi2) * dm + dm * dm) + 1e-12 * chi2
    case = name + ("" if grouped else " ungrouped")
    check_err(abs(scal[0] - chi2) / chi2, cb / chi2, key("hour_angle", "chi2", prec), case)
    check_err(rel_l2(grad.cpu().numpy(), g), bound("hour_angle", "grad", prec, name), key("hour_angle", "grad", prec),
              case)
    h.sync_status()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("full", [True, False])
def test_hvp_matches_oracle(prec, full, check_err):
    p, o, th, d, mu, lam = make_case("ha37")
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    th = quant(prec, perturbed(o, th, 0.01, 3))
    v = quant(prec, perturbed(o, np.zeros_like(th), 1.0, 4))
    got = h.hvp(_t(th, h), _t(v, h), full=full).cpu().numpy()
    check_err(rel_l2(got, o.hvp(th, d, v, lam, full=full)), bound("hour_angle", "grad", prec, "ha37"),
              key("hour_angle", "hvp_full" if full else "hvp_gn", prec), "ha37")


def test_repeat_runs_are_bitwise_identical():
    p, o, th, d, mu, lam = make_case("ha37")
    h = handle(p, "fp16x3", d, mu, lam)
    t = _t(th, h)
    s1, g1 = h.chi2_grad(t)
    s1, g1 = s1.clone(), g1.clone()
    s2, g2 = h.chi2_grad(t)
    assert bool((s1 == s2).all()) and bool((g1 == g2).all())


# With one pass over the LSTs the chi^2 epilogue forms V itself from the forward's partial
# sums, with the roundings of the kernel that otherwise finishes V (FM_HA_FUSED_CHI2=0): the
# two routes give the same bits, and the fused one launches one kernel fewer.  harand has two
# forward M-tiles, hafrac2 cells of half a pixel.
@pytest.mark.parametrize("name", ["ha37", "harand", "hafrac2"])
@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3"])
def test_fused_chi2_epilogue_equals_the_finished_forward(name, prec, monkeypatch):
    from paper_2504_07090_gb300 import fm
    p, o, th, d, mu, lam = make_case(name)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    t = _t(quant(prec, perturbed(o, th, 0.01, 2)), h)
    out = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("FM_HA_FUSED_CHI2", fused)
        n0 = fm.kernel_launches()
        s, g = h.chi2_grad(t)
        out[fused] = (s.clone(), g.clone(), fm.kernel_launches() - n0)
    (s1, g1, n1), (s0, g0, n0) = out["1"], out["0"]
    assert bool((s1 == s0).all()) and bool((g1 == g0).all())
    assert n1 == n0 - 1


def test_antenna_form_is_used_when_disabled(monkeypatch, check_err):
    monkeypatch.setenv("FM_HA", "0")
    p, o, th, d, mu, lam = make_case("ha37")
    h = handle(p, "fp16x3")
    assert h.contraction_info()["form"] == "antenna"
    a, _ = o.split(th)
    x = quant("fp16x3", o.sky(a))
    check_err(rel_l2(as_complex(h.forward_pixels(_t(x, h))), o.vis(x)), bound("antenna", "V", "fp16x3", "ha37"),
              key("antenna", "V", "fp16x3"), "ha37")


def test_non_commensurate_grid_keeps_the_antenna_form():
    p, o, th, d, mu, lam = make_case("ant37")
    assert handle(p, "fp16x3").contraction_info()["form"] == "antenna"
