"""Source-extended elastic FWI with DAS data on one GB300 (sm_103a).

Python side of the C ABI declared in ``include/efwi.h``: it only marshals
arguments (torch CUDA tensors -> device pointers, the current torch stream ->
cudaStream_t).  Every step of the computation runs in the CUDA kernels of
``_lib/libefwi_gb300.so``; there is no CPU fallback, and a missing library
raises at first use.

Method (Bader, Clapp, Nihei, Biondi, "Source footprint elimination in
full-waveform inversion by model extension"):
  * forward modelling d_s = K_r u_s(m_s) with one model component per source
    (eqs. 1-3, first term of eq. 8), DAS axial strain as K_r;
  * misfit 1/2 sum ||d_s - d_obs_s||^2 and its gradient per component by the
    adjoint-state method (eqs. 4, 6);
  * zone-of-influence weights (eq. 10) and the consistency term
    1/2 eta^2 ||(I - S^T S_w) W m~||^2 with its gradient (eqs. 8, 11, 12).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import EfwiError, STORE, EXEC, STENCIL, OVERLAP, ADJ_FORM, CKPT_AUTO

__all__ = ["Plan", "zoi_weights", "collapse", "EfwiError", "load_library", "DataMisfit", "Consistency",
           "ExtendedFWI", "extended_objective"]


from .autograd import DataMisfit, Consistency, ExtendedFWI, extended_objective  # noqa: E402


def load_library():
    return _abi.load()


def _ptr(t, name, numel=None, dtype=torch.float32, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _np(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


class Plan:
    """A problem (grid, sources, DAS geometry, windows) bound to device workspace.

    ``acq`` is any object with the attributes of ``efwi_plan_desc`` (see
    include/efwi.h): nx, nz, dx, dz, nt, dt, npml, pml_R, pml_vmax, pml_f0,
    src_xz, mt, wavelet, tr_ptr, ch_xz, ch_t, gauge, das_mode, win,
    ref_vp, ref_vs, ref_rho.

    ``ckpt_interval``: 0 = ceil(sqrt(nt)) steps per checkpoint, >= nt = every
    step stored, "auto" = every step stored when the snapshots fit the free
    device memory, else ceil(sqrt(nt)) with as many stored final steps as fit.
    ``stored_steps``: with an interval K < nt, the forward pass also keeps the
    velocities of the final stored_steps steps (rounded down to leave whole
    K-step segments before them), which the adjoint then reads without a
    recompute.  ``snap_store``: precision of those stored forward
    velocities ("fp32", "fp16", "bf16"; the latter two need exec="batched").
    ``adj_form``: the adjoint step's stress variable -- "scaled" (F = dt C
    sigma^; per-thread loads or TMA staging; needs Vp > Vs
    on the imaging area), "stress" (sigma^ itself, every staging) or "auto"
    (scaled with exec="batched" unless the requested adjoint staging exists in
    the stress form only).
    """

    def __init__(self, acq, exec: str = "batched", ckpt_interval=0, ckpt_store: str = "fp32",
                 tile=(0, 0), stencil: str = "auto", adj_tile=(0, 0), adj_stencil: str = "auto",
                 overlap: str = "auto", snap_store: str = "fp32", stored_steps: int = 0, adj_form: str = "auto"):
        lib = _abi.load()
        self._opts = dict(exec=exec, ckpt_interval=ckpt_interval, ckpt_store=ckpt_store, tile=tile, stencil=stencil,
                          adj_tile=adj_tile, adj_stencil=adj_stencil, overlap=overlap, snap_store=snap_store,
                          stored_steps=stored_steps, adj_form=adj_form)
        d, keep = self._desc(acq)
        self.exec, self.ckpt_store, self.snap_store = exec, ckpt_store, snap_store
        h = C.c_void_p()
        torch.cuda.init()
        rc = lib.efwi_plan_create(C.byref(h), C.byref(d))
        _abi.check(rc, None)
        self._h = h
        self._lib = lib
        self.model_numel = self.ns * self.nz * self.nx
        self.data_shape = (self.ntr, self.nt)

    def _desc(self, acq):
        """efwi_plan_desc of an acquisition with this plan's options, and the host
        arrays it points into (kept alive by the caller until the call returns)."""
        a = acq
        o = self._opts
        self.nx, self.nz, self.nt = int(a.nx), int(a.nz), int(a.nt)
        self.ns = int(np.asarray(a.src_xz).shape[0])
        self.ntr = int(np.asarray(a.ch_xz).reshape(-1, 2).shape[0])
        keep = dict(
            src=_np(a.src_xz, np.float64), mt=_np(a.mt, np.float64), wav=_np(a.wavelet, np.float32),
            ptr=_np(a.tr_ptr, np.int32), ch=_np(np.asarray(a.ch_xz).reshape(-1, 2), np.float64),
            cht=_np(np.asarray(a.ch_t).reshape(-1, 2), np.float64),
            rvp=_np(a.ref_vp, np.float32), rvs=_np(a.ref_vs, np.float32), rrho=_np(a.ref_rho, np.float32))
        win = getattr(a, "win", None)
        keep["win"] = None if win is None else _np(win, np.int32)
        force = getattr(a, "force", None)
        keep["force"] = None if force is None else _np(np.asarray(force).reshape(-1, 2), np.float64)
        if keep["force"] is not None and keep["force"].shape != (self.ns, 2):
            raise ValueError("force must be [ns, 2]")
        if keep["wav"].shape != (self.ns, self.nt + 1):
            raise ValueError("wavelet must be [ns, nt+1]")
        P = lambda arr, typ: arr.ctypes.data_as(C.POINTER(typ)) if arr is not None and arr.size else None
        d = _abi.PlanDesc()
        d.nx, d.nz, d.dx, d.dz = self.nx, self.nz, float(a.dx), float(a.dz)
        d.nt, d.dt = self.nt, float(a.dt)
        d.npml = int(getattr(a, "npml", 20))
        d.pml_R = float(getattr(a, "pml_R", 1e-3))
        d.pml_vmax = float(getattr(a, "pml_vmax", 0.0))
        d.pml_f0 = float(getattr(a, "pml_f0", 0.0))
        d.ns = self.ns
        d.src_xz, d.mt, d.wavelet = P(keep["src"], C.c_double), P(keep["mt"], C.c_double), P(keep["wav"], C.c_float)
        d.ntr, d.tr_ptr = self.ntr, P(keep["ptr"], C.c_int)
        d.ch_xz, d.ch_t = P(keep["ch"], C.c_double), P(keep["cht"], C.c_double)
        d.gauge = float(a.gauge)
        d.das_mode = int(getattr(a, "das_mode", 0))
        d.win = P(keep["win"], C.c_int)
        d.ref_vp, d.ref_vs, d.ref_rho = P(keep["rvp"], C.c_float), P(keep["rvs"], C.c_float), P(keep["rrho"], C.c_float)
        d.ckpt_interval = CKPT_AUTO if o["ckpt_interval"] == "auto" else int(o["ckpt_interval"])
        d.snap_store = STORE[o["snap_store"]]
        d.stored_steps = int(o["stored_steps"])
        d.ckpt_store = STORE[o["ckpt_store"]]
        d.exec = EXEC[o["exec"]]
        d.tile_x, d.tile_z = int(o["tile"][0]), int(o["tile"][1])
        d.stencil = STENCIL[o["stencil"]]
        d.adj_tile_x, d.adj_tile_z = int(o["adj_tile"][0]), int(o["adj_tile"][1])
        d.adj_stencil = STENCIL[o["adj_stencil"]]
        d.overlap = OVERLAP[o["overlap"]]
        d.force = P(keep["force"], C.c_double)
        d.adj_form = ADJ_FORM[o["adj_form"]]
        return d, keep

    def rebind(self, acq):
        """Bind the plan to another acquisition of the same shape (the next shot
        group of an extended problem): new sources, wavelets and receivers on the
        same grid, windows and trace counts, with no re-allocation or re-tuning
        (efwi_plan_rebind)."""
        d, keep = self._desc(acq)
        self._check(self._lib.efwi_plan_rebind(self._h, C.byref(d), _stream()))

    # -- lifecycle -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.efwi_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        _abi.check(rc, self._h)

    def info(self) -> dict:
        i = _abi.PlanInfo()
        self._check(self._lib.efwi_plan_info(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in _abi.PlanInfo._fields_}

    # -- calls -------------------------------------------------------------------
    def _model(self, vp, vs, rho):
        n = self.model_numel
        return _ptr(vp, "vp", n), _ptr(vs, "vs", n), _ptr(rho, "rho", n)

    def forward(self, vp, vs, rho, out=None):
        """Modelled DAS data [ntr, nt] of the extended model (each [ns, nz, nx])."""
        m = self._model(vp, vs, rho)
        if out is None:
            out = torch.empty(self.data_shape, dtype=torch.float32, device=vp.device)
        self._check(self._lib.efwi_forward(self._h, *m, _ptr(out, "out", self.ntr * self.nt), _stream()))
        return out

    def gradient(self, vp, vs, rho, d_obs, mask=None, out=None, return_data=False):
        """(phi_data [device float64 scalar], g_vp, g_vs, g_rho[, d]) of the data term."""
        m = self._model(vp, vs, rho)
        dev = vp.device
        if out is None:
            out = tuple(torch.empty_like(vp) for _ in range(3))
        phi = torch.empty((), dtype=torch.float64, device=dev)
        dmod = torch.empty(self.data_shape, dtype=torch.float32, device=dev) if return_data else None
        self._check(self._lib.efwi_adjoint_gradient(
            self._h, *m, _ptr(d_obs, "d_obs", self.ntr * self.nt), _ptr(phi, "phi", 1, torch.float64),
            _ptr(out[0], "g_vp", self.model_numel), _ptr(out[1], "g_vs", self.model_numel),
            _ptr(out[2], "g_rho", self.model_numel), _ptr(mask, "mask", self.nz * self.nx, allow_none=True),
            _ptr(dmod, "d_out", self.ntr * self.nt, allow_none=True), _stream()))
        return (phi, *out, dmod) if return_data else (phi, *out)

    def set_zoi(self, zoi):
        """Zone-of-influence weights of the plan's sources held by the plan
        (efwi_plan_set_zoi): afterwards b, bp, sink may be None in
        regularization_grad and extended_objective."""
        z, keep = _zoi_desc(zoi)
        self._check(self._lib.efwi_plan_set_zoi(self._h, C.byref(z), _stream()))

    def regularization_grad(self, m, b, bp, sink, eta, g=None):
        """phi_reg (device float64) and g += eta^2 A^T A m for one parameter field
        (b, bp, sink None: the weights set with set_zoi).

        m may hold any number of components [ns', nz, nx] on the plan's grid (for
        shot groups: every component of the extended problem, evaluated with the
        plan of one group)."""
        ns = m.shape[0] if m.dim() == 3 else self.ns
        if ns != self.ns:
            n = ns * self.nz * self.nx
            if g is None:
                g = torch.zeros_like(m)
            phi = torch.empty((), dtype=torch.float64, device=m.device)
            self._check(self._lib.efwi_regularization_grad_n(
                self._h, int(ns), _ptr(m, "m", n), _ptr(b, "b", n), _ptr(bp, "bp", n),
                _ptr(sink, "sink", n, torch.uint8), float(eta), _ptr(phi, "phi", 1, torch.float64),
                _ptr(g, "g", n), _stream()))
            return phi, g
        n = self.model_numel
        if g is None:
            g = torch.zeros_like(m)
        phi = torch.empty((), dtype=torch.float64, device=m.device)
        self._check(self._lib.efwi_regularization_grad(
            self._h, _ptr(m, "m", n), _ptr(b, "b", n, allow_none=True), _ptr(bp, "bp", n, allow_none=True),
            _ptr(sink, "sink", n, torch.uint8, allow_none=True), float(eta), _ptr(phi, "phi", 1, torch.float64), _ptr(g, "g", n), _stream()))
        return phi, g

    def extended_objective(self, vp, vs, rho, d_obs, eta, b, bp, sink):
        """(phi_data, phi_reg) of eq. 8 as device float64 scalars."""
        n = self.model_numel
        m = self._model(vp, vs, rho)
        pd = torch.empty((), dtype=torch.float64, device=vp.device)
        pr = torch.empty((), dtype=torch.float64, device=vp.device)
        e = (C.c_double * 3)(*[float(x) for x in eta])
        self._check(self._lib.efwi_extended_objective(
            self._h, *m, _ptr(d_obs, "d_obs", self.ntr * self.nt), e, _ptr(b, "b", n, allow_none=True),
            _ptr(bp, "bp", n, allow_none=True),
            _ptr(sink, "sink", n, torch.uint8, allow_none=True), _ptr(pd, "phi_data", 1, torch.float64),
            _ptr(pr, "phi_reg", 1, torch.float64), _stream()))
        return pd, pr

    def pseudo_hessian(self, vp, vs, rho, eps=1e-3, inverse=True):
        """(h, h_inv) [nz, nx]: zero-lag auto-correlation of |v| summed over the
        shots, and its clipped, scaled inverse (None unless inverse)."""
        m = self._model(vp, vs, rho)
        h = torch.empty((self.nz, self.nx), dtype=torch.float32, device=vp.device)
        hi = torch.empty_like(h) if inverse else None
        self._check(self._lib.efwi_pseudo_hessian(self._h, *m, float(eps), _ptr(h, "h", self.nz * self.nx),
                                                  _ptr(hi, "h_inv", self.nz * self.nx, allow_none=True),
                                                  _stream()))
        return h, hi

    def sync_status(self):
        """Synchronise the current stream; raise on device-side failures of earlier calls."""
        self._check(self._lib.efwi_sync_status(self._h, _stream()))

    def prof_enable(self, every: int):
        self._check(self._lib.efwi_prof_enable(self._h, int(every)))

    def prof_read(self, kernel: str = "step"):
        """(summed ms, launches timed) of the 'step' (forward) or 'adj' stencil kernel."""
        ms = C.c_double()
        cnt = C.c_longlong()
        k = {"step": 0, "adj": 1}[kernel]
        self._check(self._lib.efwi_prof_read(self._h, k, C.byref(ms), C.byref(cnt)))
        return ms.value, cnt.value


def _zoi_desc(zoi):
    """efwi_zoi_desc of a zone-of-influence description and the arrays it points into."""
    act = _np(zoi.active_x, np.float64)
    tap = _np(zoi.taper, np.float64)
    sxz = _np(zoi.sink_xz, np.float64)
    axes = _np(np.stack([np.asarray(zoi.sink_ax, np.float64), np.asarray(zoi.sink_az, np.float64)], axis=1),
               np.float64)
    PD = C.POINTER(C.c_double)
    z = _abi.ZoiDesc(act.ctypes.data_as(PD), tap.ctypes.data_as(PD), sxz.ctypes.data_as(PD),
                     axes.ctypes.data_as(PD), float(zoi.n), float(zoi.nu))
    return z, (act, tap, sxz, axes)


def zoi_weights(ns, nx, nz, dx, dz, zoi, device="cuda"):
    """b, b' [ns, nz, nx] float32 and the sinkhole flags (uint8) of eq. 10 on the device."""
    lib = _abi.load()
    z, keep = _zoi_desc(zoi)
    b = torch.empty((ns, nz, nx), dtype=torch.float32, device=device)
    bp = torch.empty_like(b)
    sink = torch.empty((ns, nz, nx), dtype=torch.uint8, device=device)
    _abi.check(lib.efwi_zoi_weights(int(ns), int(nx), int(nz), float(dx), float(dz), C.byref(z),
                                    C.c_void_p(b.data_ptr()), C.c_void_p(bp.data_ptr()),
                                    C.c_void_p(sink.data_ptr()), _stream()))
    return b, bp, sink


def collapse(x, b, bp, sink, out=None):
    """S_w W x~ of an extended field x [ns, nz, nx] (eq. 9 for a model, eq. 15 for
    per-source gradients): one physical field [nz, nx], computed on the device."""
    lib = _abi.load()
    ns, nz, nx = x.shape
    for t, dt in ((x, torch.float32), (b, torch.float32), (bp, torch.float32), (sink, torch.uint8)):
        if t.dtype != dt or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != (ns, nz, nx):
            raise ValueError("collapse: x, b, bp (float32) and sink (uint8) must be contiguous CUDA [ns, nz, nx]")
    if out is None:
        out = torch.empty((nz, nx), dtype=torch.float32, device=x.device)
    _abi.check(lib.efwi_collapse(int(ns), int(nx), int(nz), C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()),
                                 C.c_void_p(bp.data_ptr()), C.c_void_p(sink.data_ptr()), C.c_void_p(out.data_ptr()),
                                 _stream()))
    return out
