"""l-BFGS with a strong-Wolfe line search on the device (the paper's solver),
stopping on the convergence rate of eq. 13.

Thin binding of the ``efwi_lbfgs_*`` C-ABI: every vector operation runs in the
library's CUDA kernels; this module only marshals pointers and wraps the
objective as the C callback.  The objective is a Python callable

    phi = objective(x, g)

that receives the trial point ``x`` (float32 CUDA vector of n elements, read
only) and writes its gradient into ``g`` (same shape), returning phi as a
Python float.  Both are views of device memory owned by the caller or by the
l-BFGS handle, valid only during the call.

``extended_fwi_objective`` builds that callable for the extended misfit of
eq. 8 over the packed model (Vp, Vs, rho), each [ns, nz, nx].
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _abi

STOP = {0: "max_iter", 1: "rate", 2: "no_step"}


class _DevView:
    """__cuda_array_interface__ of a raw float32 device pointer (no copy)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3,
                                         "strides": None}


def _as_tensor(ptr, n):
    return torch.as_tensor(_DevView(ptr, n), device="cuda")


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _vec(t, n, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
            and t.numel() == n):
        raise ValueError(f"{name}: contiguous float32 CUDA tensor of {n} elements expected")
    return C.c_void_p(t.data_ptr())


def _info(i):
    return {"phi": i.phi, "phi_prev": i.phi_prev, "rate": i.rate, "alpha": i.alpha, "evals": i.evals,
            "iters": i.iters, "pairs": i.pairs, "ls_failed": bool(i.ls_failed), "stop": STOP.get(i.stop, i.stop)}


class LBFGS:
    """Device l-BFGS over n-element float32 vectors with m stored pairs."""

    def __init__(self, n: int, m: int = 5, c1: float = 1e-4, c2: float = 0.9, max_ls: int = 20):
        self._lib = _abi.load()
        self.n = int(n)
        h = C.c_void_p()
        _abi.check(self._lib.efwi_lbfgs_create(C.byref(h), self.n, int(m), float(c1), float(c2), int(max_ls)))
        self._h = h
        self._err = None

    def close(self):
        if self._h:
            self._lib.efwi_lbfgs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        _abi.check(self._lib.efwi_lbfgs_reset(self._h))

    def set_step0(self, length: float):
        """Length of the first trial step without stored pairs (0: min(1, 1/||d||))."""
        _abi.check(self._lib.efwi_lbfgs_set_step0(self._h, float(length)))

    def push(self, s, y) -> bool:
        """Stores the pair (s, y) when s^T y > 0; returns whether it was stored."""
        acc = C.c_int()
        _abi.check(self._lib.efwi_lbfgs_push(self._h, _vec(s, self.n, "s"), _vec(y, self.n, "y"), C.byref(acc),
                                             _stream()))
        return bool(acc.value)

    def set_h0(self, diag=None):
        """Positive diagonal initial inverse Hessian (e.g. the clipped, scaled inverse
        pseudo-Hessian, flattened like the model vector); None returns to gamma I.
        Forgets the stored pairs."""
        p = None if diag is None else _vec(diag, self.n, "diag")
        _abi.check(self._lib.efwi_lbfgs_set_h0(self._h, p, _stream()))

    def state(self):
        """The stored pairs (S, Y), device tensors [pairs, n], oldest first: save them
        to resume the inversion with load_state."""
        k = C.c_int()
        _abi.check(self._lib.efwi_lbfgs_export(self._h, C.byref(k), None, None, _stream()))
        S = torch.empty((k.value, self.n), dtype=torch.float32, device="cuda")
        Y = torch.empty_like(S)
        if k.value:
            _abi.check(self._lib.efwi_lbfgs_export(self._h, C.byref(k), C.c_void_p(S.data_ptr()),
                                                   C.c_void_p(Y.data_ptr()), _stream()))
        return S, Y

    def load_state(self, S, Y):
        """Replaces the history with the pairs of state() (set a diagonal H_0 first if
        one is used); the directions then equal the saved handle's bit for bit."""
        self.reset()
        for s, y in zip(S, Y):
            if not self.push(s.contiguous(), y.contiguous()):
                raise ValueError("a saved pair has s^T y <= 0")

    def direction(self, g, d=None):
        """d = -H g from the stored pairs (two-loop recursion)."""
        if d is None:
            d = torch.empty_like(g)
        _abi.check(self._lib.efwi_lbfgs_direction(self._h, _vec(g, self.n, "g"), _vec(d, self.n, "d"), _stream()))
        return d

    def _callback(self, objective):
        n = self.n

        def fn(ctx, xp, phip, gp, stream):
            try:
                phip[0] = float(objective(_as_tensor(xp, n), _as_tensor(gp, n)))
                return 0
            except Exception as e:          # reported after the C call returns
                self._err = e
                return 1
        return _abi.OBJECTIVE_FN(fn)

    def _raise(self, code):
        if self._err is not None:
            e, self._err = self._err, None
            raise e
        _abi.check(code)

    def iterate(self, x, phi: float, g, objective):
        """One iteration from (x, phi, g), all updated in place; returns (phi, info)."""
        cb = self._callback(objective)
        p = C.c_double(phi)
        info = _abi.LbfgsInfo()
        rc = self._lib.efwi_lbfgs_iterate(self._h, _vec(x, self.n, "x"), C.byref(p), _vec(g, self.n, "g"), cb, None,
                                          C.byref(info), _stream())
        self._raise(rc)
        return p.value, _info(info)

    def iterate_device(self, x, phi, g, objective):
        """One iteration whose line search runs on the device from a CUDA graph
        (efwi_lbfgs_iterate_device).  phi: float64 CUDA scalar (updated in place),
        x and g updated in place; objective: a device objective with the attributes
        ``fn`` (address of a C efwi_device_objective_fn) and ``ctx`` (its context),
        e.g. ``groups.GroupSet.device_objective(...)``.  Returns info."""
        if not (isinstance(phi, torch.Tensor) and phi.is_cuda and phi.dtype == torch.float64 and phi.numel() == 1):
            raise ValueError("phi: float64 CUDA scalar expected")
        info = _abi.LbfgsInfo()
        rc = self._lib.efwi_lbfgs_iterate_device(self._h, _vec(x, self.n, "x"), C.c_void_p(phi.data_ptr()),
                                                 _vec(g, self.n, "g"), objective.fn, objective.ctx, C.byref(info),
                                                 _stream())
        _abi.check(rc)
        return _info(info)

    def run(self, x, objective, max_iter: int = 100, min_rate: float = 1e-3, g=None):
        """Iterates from x (updated in place) until max_iter, a rate of eq. 13
        below min_rate or a failed line search; returns (g, info)."""
        if g is None:
            g = torch.empty_like(x)
        cb = self._callback(objective)
        info = _abi.LbfgsInfo()
        rc = self._lib.efwi_lbfgs_run(self._h, _vec(x, self.n, "x"), _vec(g, self.n, "g"), cb, None, int(max_iter),
                                      float(min_rate), C.byref(info), _stream())
        self._raise(rc)
        return g, _info(info)


def extended_fwi_objective(plan, d_obs, b, bp, sink, eta, mask=None):
    """phi = phi_data + sum_p phi_reg,p (eq. 8) over the packed model x = (Vp, Vs, rho)
    [3 * ns * nz * nx]; writes the packed gradient into g."""
    shape = (3, plan.ns, plan.nz, plan.nx)

    def objective(x, g):
        m = x.view(shape)
        gg = g.view(shape)
        phi_d, *_ = plan.gradient(m[0], m[1], m[2], d_obs, mask=mask, out=(gg[0], gg[1], gg[2]))
        phi = phi_d
        for k in range(3):
            phi_r, _ = plan.regularization_grad(m[k], b, bp, sink, eta[k], g=gg[k])
            phi = phi + phi_r
        return float(phi.item())
    return objective


def pseudo_hessian_h0(plan, x, eps=1e-3):
    """Diagonal initial inverse Hessian for the packed model x = (Vp, Vs, rho)
    [3 * ns * nz * nx]: the clipped, scaled inverse pseudo-Hessian of the model
    x (efwi_pseudo_hessian), the same [nz, nx] map for every parameter and
    component.  Pass it to LBFGS.set_h0."""
    shape = (3, plan.ns, plan.nz, plan.nx)
    m = x.view(shape)
    _, hinv = plan.pseudo_hessian(m[0], m[1], m[2], eps=eps)
    return hinv.expand(shape).contiguous().view(-1)
