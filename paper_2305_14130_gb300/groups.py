"""Extended problems whose shots do not fit one plan: the data term and its
gradient for every component, with the shots run in groups, one plan per
group, created, used and destroyed in turn.

Each component (shot) of the extended model is independent through the
forward, adjoint and imaging steps (eq. 6 applied to each m_s), so a group
is an independent slice of the problem: the gradient rows of its shots are
those a single plan holding every shot would produce.  This module only
slices the acquisition and the device tensors and sums the groups' misfits;
all arithmetic runs in the library's kernels.  The consistency term couples
the groups through per-pixel sums over all components; evaluate it with any
of the plans through ``Plan.regularization_grad`` on the full [ns, nz, nx]
model (``efwi_regularization_grad_n``).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import Plan


def group_acquisition(acq, shots):
    """The acquisition restricted to `shots` (their sources, wavelets, moment
    tensors or forces, windows and traces) and the indices of their traces."""
    shots = [int(s) for s in shots]
    ptr, idx = [0], []
    for s in shots:
        lo, hi = int(acq.tr_ptr[s]), int(acq.tr_ptr[s + 1])
        idx.extend(range(lo, hi))
        ptr.append(ptr[-1] + hi - lo)
    idx = np.asarray(idx, np.int64)
    sel = lambda v: None if v is None else np.asarray(v)[shots]
    sub = dict(src_xz=np.asarray(acq.src_xz)[shots], mt=np.asarray(acq.mt)[shots],
               wavelet=np.asarray(acq.wavelet)[shots], tr_ptr=np.asarray(ptr, np.int32),
               ch_xz=np.asarray(acq.ch_xz).reshape(-1, 2)[idx], ch_t=np.asarray(acq.ch_t).reshape(-1, 2)[idx],
               win=sel(getattr(acq, "win", None)), force=sel(getattr(acq, "force", None)))
    return dataclasses.replace(acq, **sub), idx


def grouped_gradient(acq, vp, vs, rho, d_obs, group_size, out=None, times=None, **plan_kwargs):
    """phi_data (float) and the gradients (g_vp, g_vs, g_rho) [ns, nz, nx] of every
    component, the shots taken group_size at a time (one plan per group).

    vp, vs, rho: device [ns, nz, nx] float32; d_obs: device [ntr, nt].  plan_kwargs
    go to every group's Plan (checkpoint store, stencil, ...).  When `times` is a
    list, the seconds of each group's gradient call (after its plan exists) are
    appended to it."""
    ns = int(np.asarray(acq.src_xz).shape[0])
    if out is None:
        out = tuple(torch.empty_like(vp) for _ in range(3))
    phi = 0.0
    for s0 in range(0, ns, group_size):
        shots = list(range(s0, min(ns, s0 + group_size)))
        gacq, idx = group_acquisition(acq, shots)
        plan = Plan(gacq, **plan_kwargs)
        try:
            sl = slice(shots[0], shots[-1] + 1)
            tr = torch.as_tensor(idx, device=d_obs.device)
            dg = d_obs.index_select(0, tr) if len(idx) else d_obs[:0]
            m = [t[sl] for t in (vp, vs, rho)]
            g = [t[sl] for t in out]
            start = end = None
            if times is not None:
                start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                start.record()
            p, *_ = plan.gradient(*m, dg, out=tuple(g))
            if times is not None:
                end.record()
                end.synchronize()
                times.append(start.elapsed_time(end) / 1e3)
            phi += float(p.item())
            plan.sync_status()
        finally:
            plan.close()
    return phi, out
