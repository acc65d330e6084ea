"""Writes tests/golden/oracle_tiny.json: a regression fixture of the FP64 oracle on the
seeded 'tiny' workload.  It calls only the oracle (and the seeded input generator), so
the stored values never come from the CUDA path.  A change to these numbers must come
with a change to the oracle's arithmetic whose commit message names the passage of the
paper that justifies it."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2504_07090_gb300 import synth  # noqa: E402


def compute():
    p = synth.config("tiny")
    tr = synth.draw_truth(p)
    o = oracle.Oracle(p)
    m = o.model(tr.theta)
    o.sigma = 0.01 * float(np.mean(np.abs(m)))
    d = m + o.sigma * (tr.noise[..., 0] + 1j * tr.noise[..., 1])
    mu, lam = synth.prior_for(p, tr.theta)
    th = tr.theta + 0.01 * synth.random_vectors(o.n_par, 1, 3)[0] * np.abs(tr.theta).mean()
    chi2, U, g = o.chi2_grad(th, d, mu, lam)
    v = synth.random_vectors(o.n_par, 1, 4)[0]
    hv = o.hvp(th, d, v, lam, full=True)
    return {
        "workload": "tiny (3 antennas, 3 channels, 4 LSTs, 5x17 pixels, 4x3 modes)",
        "sigma": o.sigma,
        "model_f1_t2": [[z.real, z.imag] for z in o.model(th)[1, 2]],
        "chi2": chi2, "U": U,
        "grad_first8": g[:8].tolist(), "grad_gain": g[o.n_sky:].tolist(),
        "hvp_first8": hv[:8].tolist(), "hvp_norm": float(np.linalg.norm(hv)),
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_tiny.json"), "w") as fh:
        json.dump(compute(), fh, indent=1)
