"""Extended problems whose shots do not fit one plan: the data term and its
gradient for every component, with the shots run in groups through one plan
at a time.

Each component (shot) of the extended model is independent through the
forward, adjoint and imaging steps (eq. 6 applied to each m_s), so a group
is an independent slice of the problem: the gradient rows of its shots are
those a single plan holding every shot would produce.  Groups of the same shape
share one plan, rebound to each group's sources and receivers.  This module only
slices the acquisition and the device tensors and sums the groups' misfits;
all arithmetic runs in the library's kernels.  The consistency term couples
the groups through per-pixel sums over all components; evaluate it with any
of the plans through ``Plan.regularization_grad`` on the full [ns, nz, nx]
model (``efwi_regularization_grad_n``).
"""
from __future__ import annotations

import ctypes as C
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


def _shape(acq, shots):
    """What a plan's workspace depends on besides the grid: shots, traces per shot, windows."""
    win = getattr(acq, "win", None)
    ptr = np.asarray(acq.tr_ptr)
    return (len(shots), tuple(int(ptr[s + 1] - ptr[s]) for s in shots),
            None if win is None else tuple(tuple(int(v) for v in np.asarray(win)[s]) for s in shots),
            getattr(acq, "force", None) is None)


def grouped_gradient(acq, vp, vs, rho, d_obs, group_size, out=None, times=None, reuse=True, stats=None,
                     **plan_kwargs):
    """phi_data (float) and the gradients (g_vp, g_vs, g_rho) [ns, nz, nx] of every
    component, the shots taken group_size at a time.

    vp, vs, rho: device [ns, nz, nx] float32; d_obs: device [ntr, nt].  plan_kwargs
    go to the group plans (checkpoint store, stencil, ...).  With reuse, a group of
    the same shape as the previous one rebinds the previous group's plan to its
    sources and receivers (no new workspace, no new tuning); otherwise every group
    creates its own plan.  When `times` is a list, the seconds of each group's
    gradient call are appended to it; `stats` (a dict) receives the seconds spent
    creating plans ("create_s") and rebinding them ("rebind_s")."""
    import time
    ns = int(np.asarray(acq.src_xz).shape[0])
    if out is None:
        out = tuple(torch.empty_like(vp) for _ in range(3))
    if stats is not None:
        stats.setdefault("create_s", 0.0)
        stats.setdefault("rebind_s", 0.0)
    phi = 0.0
    plan, shape = None, None
    try:
        for s0 in range(0, ns, group_size):
            shots = list(range(s0, min(ns, s0 + group_size)))
            gacq, idx = group_acquisition(acq, shots)
            sh = _shape(acq, shots)
            t0 = time.perf_counter()
            if plan is not None and reuse and sh == shape:
                plan.rebind(gacq)
                key = "rebind_s"
            else:
                if plan is not None:
                    plan.close()
                plan = Plan(gacq, **plan_kwargs)
                shape = sh
                key = "create_s"
            torch.cuda.synchronize()
            if stats is not None:
                stats[key] += time.perf_counter() - t0
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
        if plan is not None:
            plan.close()
    return phi, out


class GroupSet:
    """The shot groups of an extended problem held on the device (efwi_groups_*):
    every group's acquisition (each of the plan's shape, as for ``Plan.rebind``) is
    uploaded once, so that binding the plan to group k is device-to-device copies.
    ``objective`` evaluates eq. 8 over all groups' components (eager);
    ``device_objective`` gives the same objective to
    ``LBFGS.iterate_device``, whose line search replays it from a CUDA graph."""

    def __init__(self, plan, acqs):
        from . import _abi
        self._lib = _abi.load()
        self.plan = plan
        self.ngroups = len(acqs)
        self.ns_total = plan.ns * self.ngroups
        descs = (_abi.PlanDesc * self.ngroups)()
        self._keep = []
        for k, a in enumerate(acqs):
            d, keep = plan._desc(a)
            descs[k] = d
            self._keep.append(keep)
        h = C.c_void_p()
        _abi.check(self._lib.efwi_groups_create(C.byref(h), plan._h, descs, self.ngroups), None)
        self._h = h
        self._ctx = []

    def close(self):
        if getattr(self, "_h", None):
            self._lib.efwi_groups_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bind(self, k):
        from . import _abi
        _abi.check(self._lib.efwi_groups_bind(self._h, int(k), _stream()), None)

    def objective(self, x, d_obs, eta, b=None, bp=None, sink=None, phi=None, g=None):
        """(phi [float64 CUDA scalar], g) of eq. 8 at x [3, ngroups * ns, nz, nx]
        (d_obs [ngroups, ntr, nt]); b, bp, sink [ngroups * ns, nz, nx]."""
        from . import _abi
        if phi is None:
            phi = torch.empty((), dtype=torch.float64, device=x.device)
        if g is None:
            g = torch.empty_like(x)
        e = (C.c_double * 3)(*[float(v) for v in eta])
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        _abi.check(self._lib.efwi_groups_objective(self._h, ptr(x), ptr(d_obs), e, ptr(b), ptr(bp), ptr(sink),
                                                   ptr(phi), ptr(g), _stream()), None)
        return phi, g

    def device_objective(self, d_obs, eta, b=None, bp=None, sink=None):
        """The objective as an efwi_device_objective_fn and its context (kept alive
        with this set) for LBFGS.iterate_device."""
        from . import _abi
        ctx = _abi.GroupsObjectiveCtx(self._h, C.c_void_p(d_obs.data_ptr()), (C.c_double * 3)(*map(float, eta)),
                                      None if b is None else C.c_void_p(b.data_ptr()),
                                      None if bp is None else C.c_void_p(bp.data_ptr()),
                                      None if sink is None else C.c_void_p(sink.data_ptr()))
        self._ctx.append((ctx, d_obs, b, bp, sink))
        fn = C.cast(self._lib.efwi_groups_objective_fn, C.c_void_p)
        return _DeviceObjective(fn, C.cast(C.pointer(ctx), C.c_void_p))


class _DeviceObjective:
    def __init__(self, fn, ctx):
        self.fn, self.ctx = fn, ctx


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)
