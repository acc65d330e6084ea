"""CUDA path vs the FP64 oracle, element by element, on seeded inputs that span several
tiles with ragged tails.  Errors are relative l2 over the whole output vector, each held
to the bound of its contraction form and precision (gpu_cases.BOUNDS) and recorded in the
run's summary of measured errors.

The small cases run the direct CUDA-core sum for FP64 / FP32 and the antenna form on the
tensor cores for the split precisions.  The split-precision operand rounding (2^-9 BF16,
2^-12 FP16 per product; about 2^-17 and 2^-22 after the hi/lo split) is amplified by the
cancellation of the fringe sum, and the gradient amplifies visibility errors by
|m| / |m - d| (about 100 at a noise level of 1 % of |V|).  The chi^2 check uses the
bound implied by the visibility bound."""
import numpy as np
import pytest

from gpu_cases import as_complex, bound, form_of, handle, key, make_case, perturbed, quant, rel_l2

pytestmark = pytest.mark.gpu
CASES = ["tiny", "small", "mid"]
PRECS = ["fp64", "fp32", "bf16x1", "bf16x3", "fp16x1", "fp16x3"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2504_07090_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _t(a, h):
    import torch
    return torch.tensor(np.asarray(a), dtype=h.dtype, device="cuda").contiguous()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", PRECS)
def test_forward_pixels_matches_oracle(name, prec, check_err):
    p, o, th, d, mu, lam = make_case(name)
    h = handle(p, prec)
    a, _ = o.split(th)
    x = quant(prec, o.sky(a))
    got = as_complex(h.forward_pixels(_t(x, h)))
    want = o.vis(x)
    f = form_of(prec)
    check_err(rel_l2(got, want), bound(f, "V", prec, name), key(f, "V", prec), name)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", PRECS)
def test_forward_model_matches_oracle(name, prec, check_err):
    p, o, th, d, mu, lam = make_case(name)
    h = handle(p, prec)
    th = quant(prec, perturbed(o, th, 0.02, 1))
    got = as_complex(h.forward(_t(th, h)))
    f = form_of(prec)
    check_err(rel_l2(got, o.model(th)), bound(f, "V", prec, name), key(f, "V", prec), name)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", PRECS)
def test_chi2_and_gradient_match_oracle(name, prec, check_err):
    p, o, th, d, mu, lam = make_case(name)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    th = quant(prec, perturbed(o, th, 0.01, 2))
    chi2, U, g = o.chi2_grad(th, d, mu, lam)
    scal, grad = h.chi2_grad(_t(th, h))
    scal = scal.cpu().numpy()
    # |chi2' - chi2| <= 2 sqrt(chi2) |dm| / sigma + |dm|^2 / sigma^2 with |dm| <= tol_V |m| (x2 margin)
    f = form_of(prec)
    dm = bound(f, "V", prec, name) * np.linalg.norm(o.model(th)) / o.sigma
    cb = 2.0 * (2.0 * np.sqrt(chi2) * dm + dm * dm) + 1e-12 * chi2
    assert abs(scal[0] - chi2) < cb
    assert abs(scal[1] - U) < 0.5 * cb + 1e-12 * U
    check_err(abs(scal[0] - chi2) / chi2, cb / chi2, key(f, "chi2", prec), name)
    check_err(rel_l2(grad.cpu().numpy(), g), bound(f, "grad", prec, name), key(f, "grad", prec), name)
    h.sync_status()


@pytest.mark.parametrize("name", ["tiny", "small"])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("full", [True, False])
def test_hvp_matches_oracle(name, prec, full, check_err):
    p, o, th, d, mu, lam = make_case(name)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    th = quant(prec, perturbed(o, th, 0.01, 3))
    v = quant(prec, perturbed(o, np.zeros_like(th), 1.0, 4))
    want = o.hvp(th, d, v, lam, full=full)
    got = h.hvp(_t(th, h), _t(v, h), full=full).cpu().numpy()
    f = form_of(prec)
    check_err(rel_l2(got, want), bound(f, "grad", prec, name), key(f, "hvp_full" if full else "hvp_gn", prec), name)


def test_gradient_without_data_is_a_state_error():
    from paper_2504_07090_gb300 import fm
    p, o, th, d, mu, lam = make_case("tiny")
    h = handle(p, "fp32")
    with pytest.raises(fm.FmError) as e:
        h.chi2_grad(_t(th, h))
    assert e.value.status == fm.FM_ERR_STATE


def test_repeat_runs_are_bitwise_identical():
    p, o, th, d, mu, lam = make_case("mid")
    h = handle(p, "fp32", d, mu, lam)
    t = _t(th, h)
    s1, g1 = h.chi2_grad(t)
    s1, g1 = s1.clone(), g1.clone()
    s2, g2 = h.chi2_grad(t)
    assert bool((s1 == s2).all()) and bool((g1 == g2).all())


@pytest.mark.parametrize("name", ["small", "ha37"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "fp16x3", "fp16x1"])
def test_sky_pixels_match_oracle(prec, name, check_err):
    # the split precisions run the mode -> pixel transform on the tensor cores (FP16
    # three-term split, about 2^-22 per product)
    p, o, th, d, mu, lam = make_case(name)
    h = handle(p, prec)
    th = quant(prec, th)
    a, _ = o.split(th)
    got = h.sky_pixels(_t(th, h)).cpu().numpy().reshape(p.n_freq, -1)
    check_err(rel_l2(got, o.sky(a)), 1e-12 if prec == "fp64" else 1e-6, key("modes", "x", prec), name)


@pytest.mark.parametrize("rch,sub", [("1", "32"), ("3", "4"), ("4", "7")])
@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3", "fp16x1"])
def test_37_antennas_with_channel_recurrence_groups(prec, rch, sub, monkeypatch, check_err):
    # the cfg1 array on a small grid: two K atoms in the adjoint tiles, the frequency
    # recurrence forced to groups of 1, 3 (ragged last group) and 4 channels, and the
    # accumulation restarted every 4 or 7 stages (several partials, ragged last one)
    monkeypatch.setenv("FM_TC_CHANNELS_PER_TASK", rch)
    monkeypatch.setenv("FM_TC_STAGES_PER_PARTIAL", sub)
    p, o, th, d, mu, lam = make_case("ant37")
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    th = quant(prec, perturbed(o, th, 0.01, 12))
    got = as_complex(h.forward(_t(th, h)))
    case = f"ant37 r{rch} s{sub}"
    check_err(rel_l2(got, o.model(th)), bound("antenna", "V", prec, "ant37"), key("antenna", "V", prec), case)
    chi2, U, g = o.chi2_grad(th, d, mu, lam)
    _, grad = h.chi2_grad(_t(th, h))
    check_err(rel_l2(grad.cpu().numpy(), g), bound("antenna", "grad", prec, "ant37"), key("antenna", "grad", prec),
              case)
