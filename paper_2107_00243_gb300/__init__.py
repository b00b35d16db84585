"""GB300-native preconditioned GP log-marginal-likelihood estimator.

The compute path lives in a CUDA shared library (``csrc/``, C ABI declared in
``include/gp.h``); ``gp`` holds its thin Python binding and ``autograd`` the
``torch.autograd.Function`` on top of it.  ``workloads`` draws seeded synthetic
inputs.
"""
