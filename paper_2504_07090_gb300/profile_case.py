"""Run one chi-squared gradient evaluation under an NVTX range, for a profiler.

Usage: ``python -m paper_2504_07090_gb300.profile_case [config] [precision]``
(defaults ``cfg1 fp16x3``).  Builds the handle for the named synthetic workload,
sets the noiseless model of the drawn truth as data, runs one untimed warm-up
evaluation of chi^2 and its gradient (Eq. 8 and its adjoint), and then one more
inside the NVTX range ``prof``, so that a profiler filtered on that range sees
exactly one forward and one adjoint launch of the hot path.
"""
import sys

import torch

from . import fm, synth


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    name = argv[0] if len(argv) > 0 else "cfg1"
    prec = argv[1] if len(argv) > 1 else "fp16x3"
    fm.load()
    p = synth.config(name)
    truth = synth.draw_truth(p)
    h = fm.ForwardModel(p, prec, sigma=1.0)
    theta = torch.tensor(truth.theta, dtype=torch.float32, device="cuda")
    h.set_data(h.forward(theta).contiguous())
    h.chi2_grad(theta)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("prof")
    h.chi2_grad(theta)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(f"profiled one chi2_grad: {name} {prec} params={p.n_params}")


if __name__ == "__main__":
    main()
