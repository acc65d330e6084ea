"""The device-side HMC chain (fm_hmc_chain: Philox momentum draws, p = L z, leapfrog,
Metropolis test and the adaptive step size of App. B in one captured graph per iteration),
replayed on the host:

- the generator: fm_draw_accept_uniform equals the oracle's Philox4x32-10 bit for bit, and
  fm_draw_normal equals its Box-Muller normals to FP32 rounding;
- the first iteration equals the oracle's trajectory from the same draw (z from the
  oracle's generator, p = L z with the oracle's mass matrix, the oracle's accept uniform);
- over 50 iterations on two chains (thresholds 0.2 and 0.95) the recorded step sizes
  follow the rule eps <- eps / 1.2 (a < a_min) or min(eps0, 1.2 eps) exactly, every accept
  decision is u < a with the oracle's uniform, and the state continues across calls."""
import math

import numpy as np
import pytest

import oracle
from oracle import philox
from gpu_cases import handle, make_case, perturbed, quant, rel_l2

pytestmark = pytest.mark.gpu
SEED = 0x5EED2504_07090


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_07090_gb300 import build
    build.build()


def _t(a, h):
    import torch
    return torch.tensor(np.asarray(a), dtype=h.dtype, device="cuda").contiguous()


def test_draws_match_the_oracle_generator():
    import torch
    from paper_2504_07090_gb300 import fm
    for it in (0, 7, (1 << 32) + 5):
        u = fm.draw_accept_uniform(SEED, it, 64).cpu().numpy()
        want = np.array([philox.accept_uniform(SEED, it + k) for k in range(64)])
        assert np.array_equal(u, want)
        for dt in (torch.float32, torch.float64):
            z = fm.draw_normal(SEED, it, 10_003, dt).double().cpu().numpy()
            np.testing.assert_allclose(z, philox.normals(SEED, it, 10_003), rtol=2e-6, atol=2e-6)


def _setup(name, prec, prior=(0.05, 0.05)):
    p, o, th, d, mu, lam = make_case(name, prior=prior)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    q0 = quant(prec, perturbed(o, th, 0.005, 6))
    tq = _t(q0, h)
    h.build_precond(tq, 64)
    return p, o, d, mu, lam, h, q0, tq


def _oracle_mass(o, th, lam, bs=64):
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


# ha37m with the tight priors of the leapfrog parity test (a well-conditioned mass matrix)
@pytest.mark.parametrize("name,prec,eps0,prior", [("small", "fp32", 0.1, (0.05, 0.05)),
                                                  ("ha37m", "fp16x3", 0.01, (0.005, 0.005))])
def test_first_iteration_is_the_oracle_trajectory(name, prec, eps0, prior, check_err):
    import torch
    p, o, d, mu, lam, h, q0, tq = _setup(name, prec, prior)
    it0 = 3
    state = torch.tensor([eps0, float(it0)], dtype=torch.float64, device="cuda")
    trace = torch.zeros((1, 5), dtype=torch.float64, device="cuda")
    h.hmc_chain(tq, 1, 20, eps0, 0.2, SEED, state, trace)
    tr = trace.cpu().numpy()[0]
    mass = _oracle_mass(o, q0, lam)
    z = philox.normals(SEED, it0, o.n_par)
    u = philox.accept_uniform(SEED, it0)

    def fn(q):
        _, U, g = o.chi2_grad(q, d, mu, lam)
        return U, g

    qw, pw, H0, H1, acc = oracle.leapfrog(fn, q0, mass.mul_lower(z), eps0, 20, u, mass)
    assert tr[0] == eps0
    check_err(abs(tr[1] - H0) / abs(H0), 1e-5, f"chain H0 {prec}", name)
    assert int(tr[3]) == int(acc)
    if acc:
        # the bounds of the leapfrog parity test (ha37m: 1.3e-4 from the FP32 state)
        check_err(rel_l2(tq.cpu().numpy() - q0, qw - q0), 1e-4 if name == "small" else 2e-4, f"chain q {prec}", name)
    else:
        assert np.array_equal(tq.cpu().numpy(), _t(q0, h).cpu().numpy())
    assert state.cpu().numpy()[1] == it0 + 1


@pytest.mark.parametrize("a_min", [0.2, 0.95])
def test_step_rule_and_accept_decisions_over_50_iterations(a_min):
    import torch
    name, prec, eps0 = "small", "fp32", 0.1
    p, o, d, mu, lam, h, q0, tq = _setup(name, prec)
    state = torch.tensor([eps0, 0.0], dtype=torch.float64, device="cuda")
    traces = []
    for n in (20, 30):                  # two calls: the chain and its graph continue
        tr = torch.full((n, 5), float("nan"), dtype=torch.float64, device="cuda")
        h.hmc_chain(tq, n, 20, eps0, a_min, SEED + 1, state, tr)
        traces.append(tr.cpu().numpy())
    rec = np.concatenate(traces)
    st = state.cpu().numpy()
    assert st[1] == 50.0
    eps = eps0
    shrinks = 0
    for k in range(50):
        e_used, H0, H1, acc, a = rec[k]
        assert e_used == eps, k
        a_host = philox.acceptance_probability(H0, H1)
        assert abs(a - a_host) <= 1e-15 * max(1.0, a_host)
        u = philox.accept_uniform(SEED + 1, k)
        if math.isfinite(H0) and math.isfinite(H1):
            assert int(acc) == int(H1 <= H0 or u < math.exp(H0 - H1)), k
        else:
            assert int(acc) == 0
        nxt = philox.adapt_step(eps, eps0, a, a_min)
        shrinks += nxt < eps
        eps = nxt
    assert st[0] == eps
    assert 0 < rec[:, 3].sum() <= 50
    if a_min > 0.9:
        assert shrinks > 0            # the high threshold exercises the shrinking branch
    h.sync_status()
