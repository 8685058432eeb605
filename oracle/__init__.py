"""fkski CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU definitions of everything the GPU path computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``
may import this package.  It shares no code with the CUDA library and never imports it.

Layout:
  fkski_oracle.c  -- per-point arithmetic in C (cell keys as an exact float sequence, Keys
                     weights, W^T W / W^T y / y^T y by explicit per-point sums, stable counting
                     sort, probe signs); built by ``build()`` into ``liboracle.so``.
  core.py         -- numpy/scipy definitions on top: K_G (dense and Kronecker/BTTB), explicit W,
                     n-space CG (Alg. 1), SKI/GSGP inference (Def. 1, Fact 2), log-likelihood,
                     stochastic Lanczos quadrature and the hyperparameter gradient.

Parity status of each function is stated in core.py's header.
"""
from .lib import build, lib_path  # noqa: F401
from .core import *  # noqa: F401,F403
