"""GB300-native forward model, adjoint, Hessian-vector products, preconditioner and
leapfrog for the 21 cm visibility model of arXiv:2504.07090.

Importing the package loads nothing; ``paper_2504_07090_gb300.fm`` binds the CUDA
library ``libfm.so`` (built by ``paper_2504_07090_gb300.build``) and fails loudly when
it is missing.  ``synth`` draws seeded synthetic inputs.
"""
__all__ = ["synth", "fm", "build"]
