"""The modified Airy beam (Eq. airy, power beam (2 J1(x) / x)^2, D_ew = 12 m, D_ns = 14 m)
through every contraction form against the oracle, whose J1 comes from Bessel's integral
while the library's comes from the power series and Hankel's expansion: visibilities, chi^2
gradient at a 1 % perturbation, and the Gauss-Newton diagonal of the mass matrix.  Bounds are
those of the form and precision with the Gaussian beam."""
import numpy as np
import pytest

import oracle
from gpu_cases import bound, handle, key, perturbed, quant, rel_l2
from paper_2504_07090_gb300 import synth

pytestmark = pytest.mark.gpu

# (case, precision, form)
CASES = [("small", "fp64", "direct"), ("small", "fp32", "direct"), ("ant37", "fp16x3", "antenna"),
         ("ha37", "fp16x3", "hour_angle"), ("ha37", "bf16x3", "hour_angle")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_07090_gb300 import build
    build.build()


def _t(a, h):
    import torch
    return torch.tensor(np.asarray(a), dtype=h.dtype, device="cuda").contiguous()


def _case(name):
    p = synth.with_airy_beam(synth.config(name))
    tr = synth.draw_truth(p)
    o = oracle.Oracle(p)
    m = o.model(tr.theta)
    p.sigma = o.sigma = 0.01 * float(np.mean(np.abs(m)))
    d = m + p.sigma * (tr.noise[..., 0] + 1j * tr.noise[..., 1])
    mu, lam = synth.prior_for(p, tr.theta)
    return p, o, tr.theta.copy(), d, mu, lam


@pytest.mark.parametrize("name,prec,form", CASES)
def test_airy_visibilities_and_gradient_match_oracle(name, prec, form, check_err):
    p, o, th, d, mu, lam = _case(name)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    assert h.contraction_info()["form"] == form
    thq = quant(prec, perturbed(o, th, 0.02, 1))
    V = h.forward(_t(thq, h)).double().cpu().numpy()
    check_err(rel_l2(V[..., 0] + 1j * V[..., 1], o.model(thq)), bound(form, "V", prec, name),
              key(form, "airy_V", prec), name)
    th1 = quant(prec, perturbed(o, th, 0.01, 2))
    _, _, g = o.chi2_grad(th1, d, mu, lam)
    _, grad = h.chi2_grad(_t(th1, h))
    check_err(rel_l2(grad.cpu().numpy(), g), bound(form, "grad", prec, name), key(form, "airy_grad", prec), name)
    h.sync_status()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_airy_gn_diagonal_matches_oracle(prec, check_err):
    p, o, th, d, mu, lam = _case("tiny")
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    th = quant(prec, perturbed(o, th, 0.01, 5))
    h.build_precond(_t(th, h), 1)
    got = h.precond_blocks().cpu().numpy()
    J = o.jacobian(th)
    diag = np.sum(np.abs(J) ** 2, axis=0) / o.sigma ** 2 + lam
    check_err(rel_l2(got, diag), 1e-10 if prec == "fp64" else 1e-4, key("precond", "airy_gn_diag", prec), "tiny")
