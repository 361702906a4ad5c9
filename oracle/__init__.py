"""FP64 CPU oracle for the source-extended elastic FWI hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link
this package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference arm use it.  It shares no code with the CUDA library
(``paper_2305_14130_gb300``); both read their inputs from ``workloads``.

Modules
-------
elastic    forward modelling (eqs. 1-3), L2 misfit (eq. 4 / first term of
           eq. 8), exact discrete adjoint and per-source gradient (eq. 6).
extension  zone-of-influence weights (eq. 10), the footprint operator W
           (eq. 11), the weighted collapse S_w (eq. 12) and the
           inter-component consistency term of eq. 8 with its gradient.
hessian    the pseudo-Hessian of the paper's illumination-compensation
           comparison (zero-lag auto-correlation of |v| summed over shots)
           and its clipped, scaled inverse.
lbfgs      the optimizer (l-BFGS, strong-Wolfe line search, eq. 13 rate).
"""
from . import elastic, extension, hessian  # noqa: F401
