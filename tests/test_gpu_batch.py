"""Batched trajectories over independent problems (fm_batch_*): one CUDA graph launch runs
one leapfrog trajectory per handle.  Every chain must reproduce, bit for bit, fm_leapfrog on
its own handle with the same step and accept uniform (the chains share no state and every
reduction runs in a fixed order), over two launches of the same graph with different
parameters; the first chain is also held to the FP64 oracle trajectory."""
import numpy as np
import pytest

import oracle
from gpu_cases import handle, make_case, perturbed, quant, rel_l2

pytestmark = pytest.mark.gpu

# (workload, precision): the direct CUDA-core form, the hour-angle form (LST step of two RA
# pixels) and the antenna form on the tensor cores
CHAINS = [("small", "fp32"), ("ha7", "fp16x3"), ("mid", "bf16x3")]
N_STEPS = 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_07090_gb300 import build
    build.build()


def _t(a, h):
    import torch
    return torch.tensor(np.asarray(a), dtype=h.dtype, device="cuda").contiguous()


def _chain(name, prec, seed):
    p, o, th, d, mu, lam = make_case(name)
    d, mu, lam = quant(prec, d, mu, lam)
    h = handle(p, prec, d, mu, lam)
    q0 = quant(prec, perturbed(o, th, 0.005, seed))
    tq = _t(q0, h)
    h.build_precond(tq, 64 if o.nk % 64 == 0 else 1)      # 64-blocks, or the diagonal
    z = _t(np.random.default_rng(seed + 100).standard_normal(o.n_par), h)
    p0 = h.precond_apply(0, z)                      # momentum L z
    return dict(h=h, o=o, d=d, mu=mu, lam=lam, q0=tq.clone(), p0=p0.clone())


@pytest.fixture(scope="module")
def chains():
    return [_chain(n, pr, 11 + k) for k, (n, pr) in enumerate(CHAINS)]


def _oracle_mass(o, th, lam, bs):
    """The oracle's block Cholesky factor of the GN mass matrix at th (block size bs)."""
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


def _single(c, eps, u):
    q, p = c["q0"].clone(), c["p0"].clone()
    hout, aout = c["h"].leapfrog(q, p, eps, N_STEPS, u)
    return q, p, hout.clone(), aout.clone()


def test_batch_matches_single_trajectories(chains):
    import torch
    from paper_2504_07090_gb300 import fm
    qs = [c["q0"].clone() for c in chains]
    ps = [c["p0"].clone() for c in chains]
    b = fm.Batch([c["h"] for c in chains], qs, ps, N_STEPS)
    assert b.kernels() > 0
    for eps, u in (([0.05, 0.08, 0.06], [0.3, 0.6, 0.9]), ([0.03, 0.1, 0.04], [0.999, 0.0, 0.5])):
        for k, c in enumerate(chains):                 # same starting point for every launch
            qs[k].copy_(c["q0"])
            ps[k].copy_(c["p0"])
        hb, ab = b.run(eps, u)
        torch.cuda.synchronize()
        for k, c in enumerate(chains):
            q, p, h1, a1 = _single(c, eps[k], u[k])
            torch.cuda.synchronize()
            assert torch.equal(qs[k], q), CHAINS[k]
            assert torch.equal(ps[k], p), CHAINS[k]
            assert torch.equal(hb[k], h1), CHAINS[k]
            assert torch.equal(ab[k], a1), CHAINS[k]
    b.close()


def test_batch_first_chain_matches_oracle(chains):
    import torch
    from paper_2504_07090_gb300 import fm
    c = chains[0]
    o, d, mu, lam = c["o"], c["d"], c["mu"], c["lam"]
    q0 = c["q0"].cpu().double().numpy()
    p0 = c["p0"].cpu().double().numpy()
    mass = _oracle_mass(o, q0, lam, 64)
    # 20 steps of 0.05 (stable for this start; the oracle's H1 stays within 0.1% of H0) move q
    # well past its FP32 rounding
    eps, n = 0.05, 20

    def fn(q):
        _, U, g = o.chi2_grad(q, d, mu, lam)
        return U, g

    qw, pw, H0, H1, acc = oracle.leapfrog(fn, q0, p0, eps, n, 0.0, mass)
    qs = [x["q0"].clone() for x in chains]
    ps = [x["p0"].clone() for x in chains]
    b = fm.Batch([x["h"] for x in chains], qs, ps, n)
    hb, ab = b.run([eps, 0.05, 0.05], [0.0, 0.0, 0.0])
    torch.cuda.synchronize()
    hh = hb[0].cpu().numpy()
    assert abs(hh[0] - H0) < 2e-3 * abs(H0) + 0.05
    assert abs((hh[1] - hh[0]) - (H1 - H0)) < 0.05 * max(1.0, abs(H1 - H0)) + 0.05
    assert int(ab[0].item()) == int(acc)
    # q is stored in FP32 (entries up to 1.4e5, rounded at every drift): relative to the
    # displacement of 20 steps of 0.05 the rounding is about twice what it is for the single
    # trajectory test's 20 steps of 0.1 (held to 1e-4 there)
    assert rel_l2(qs[0].cpu().numpy() - q0, qw - q0) < 3e-4
    assert rel_l2(ps[0].cpu().numpy(), pw) < 1e-4
    b.close()


def test_handles_of_different_sizes_coexist():
    """A handle created after a larger one (smaller tiles, smaller shared-memory needs) must
    not break the larger handle's launches: per-kernel launch limits are process-wide."""
    import torch
    big_p, big_o, big_th, *_ = make_case("mid")
    small_p, *_ = make_case("ha37")
    big = handle(big_p, "fp16x3")
    v1 = big.forward(torch.tensor(big_th, dtype=torch.float32, device="cuda")).clone()
    small = handle(small_p, "fp16x3")
    v2 = big.forward(torch.tensor(big_th, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(v1, v2)
    small.close()
    big.close()
