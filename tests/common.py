"""Helpers shared by tests: FP32-rounded problems and error measures."""
import copy

import numpy as np


def f32(a):
    """Round to float32 and back: the values the CUDA path actually sees (C-contiguous,
    also for broadcast views)."""
    return np.array(a, dtype=np.float32, order="C").astype(np.float64, order="C")


def rounded(problem):
    """Copy of a workloads.Problem whose float inputs are float32-representable."""
    p = copy.deepcopy(problem)
    a = p.acq
    a.wavelet = f32(a.wavelet)
    a.ref_vp, a.ref_vs, a.ref_rho = f32(a.ref_vp), f32(a.ref_vs), f32(a.ref_rho)
    p.vp, p.vs, p.rho = f32(p.vp), f32(p.vs), f32(p.rho)
    for k in ("true_vp", "true_vs", "true_rho"):
        if getattr(p, k) is not None:
            setattr(p, k, f32(getattr(p, k)))
    return p


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))
