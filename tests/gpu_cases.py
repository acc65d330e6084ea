"""Shared set-up of GPU parity cases: seeded inputs, oracle expectations, a handle."""
import numpy as np

import oracle
from paper_2504_07090_gb300 import synth


# Relative l2 tolerances (visibilities / gradients and HVPs) per precision; the reasoning
# behind each is in the docstring of test_gpu_parity.py.
TOL_VIS = {"fp64": 1e-10, "fp32": 1e-5, "bf16x1": 1e-2, "bf16x3": 2e-5, "fp16x1": 2e-3, "fp16x3": 1e-5}
TOL_GRAD = {"fp64": 1e-10, "fp32": 1e-4, "bf16x1": 1e-1, "bf16x3": 3e-4, "fp16x1": 5e-3, "fp16x3": 3e-4}


def rel_l2(a, b) -> float:
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def as_complex(t) -> np.ndarray:
    a = t.detach().cpu().double().numpy()
    return a[..., 0] + 1j * a[..., 1]


def to_pairs(z: np.ndarray) -> np.ndarray:
    return np.stack([z.real, z.imag], axis=-1)


def make_case(name: str, noise: bool = True):
    """Problem, oracle, truth, data d (oracle model + seeded noise), prior."""
    p = synth.config(name)
    tr = synth.draw_truth(p)
    o = oracle.Oracle(p)
    m = o.model(tr.theta)
    p.sigma = 0.01 * float(np.mean(np.abs(m)))
    o.sigma = p.sigma
    d = m + (p.sigma * (tr.noise[..., 0] + 1j * tr.noise[..., 1]) if noise else 0.0)
    mu, lam = synth.prior_for(p, tr.theta)
    return p, o, tr.theta.copy(), d, mu, lam


def perturbed(o, theta: np.ndarray, frac: float, seed: int) -> np.ndarray:
    a, _ = o.split(theta)
    sc = np.empty(o.n_par)
    sc[: o.n_sky] = np.repeat(np.sqrt(np.mean(a ** 2, axis=1)), o.nk)
    sc[o.n_sky:] = 1.0
    return theta + frac * sc * np.random.default_rng(seed).standard_normal(o.n_par)


def handle(p, precision: str, d=None, mu=None, lam=None):
    import torch
    from paper_2504_07090_gb300 import fm
    h = fm.ForwardModel(p, precision)
    dt = h.dtype
    if d is not None:
        h.set_data(torch.tensor(to_pairs(d), dtype=dt, device="cuda").contiguous())
    if lam is not None:
        h.set_prior(torch.tensor(mu, dtype=dt, device="cuda"), torch.tensor(lam, dtype=dt, device="cuda"))
    return h


def quant(prec: str, *arrays):
    """The values the device actually receives: float32-rounded for the FP32-storage paths."""
    out = []
    for a in arrays:
        if a is None or prec == "fp64":
            out.append(a)
        elif np.iscomplexobj(a):
            out.append(a.real.astype(np.float32).astype(np.float64) + 1j * a.imag.astype(np.float32).astype(np.float64))
        else:
            out.append(np.asarray(a).astype(np.float32).astype(np.float64))
    return out if len(out) > 1 else out[0]
