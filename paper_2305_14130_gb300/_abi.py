"""ctypes declarations of the C ABI in include/efwi.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

EFWI_OK = 0
STATUS = {0: "EFWI_OK", -1: "EFWI_ERR_ARG", -2: "EFWI_ERR_CFL", -3: "EFWI_ERR_OOM", -4: "EFWI_ERR_CUDA",
          -5: "EFWI_ERR_TIMEOUT", -6: "EFWI_ERR_NAN", -7: "EFWI_ERR_NOT_IMPLEMENTED"}
DAS_STRAIN, DAS_STRAIN_RATE, DAS_VELOCITY = 0, 1, 2
STORE = {"fp32": 0, "fp16": 1, "bf16": 2}
EXEC = {"plain": 0, "batched": 1}
STENCIL = {"auto": 0, "loads": 1, "tma": 2, "tma_pairs": 3, "tma_staged": 4}
OVERLAP = {"auto": 0, "off": 1, "on": 2}
ADJ_FORM = {"auto": 0, "stress": 1, "scaled": 2}
CKPT_AUTO = -1

PD = C.POINTER(C.c_double)
PF = C.POINTER(C.c_float)
PI = C.POINTER(C.c_int)


class PlanDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dz", C.c_double),
                ("nt", C.c_int), ("dt", C.c_double), ("npml", C.c_int), ("pml_R", C.c_double),
                ("pml_vmax", C.c_double), ("pml_f0", C.c_double), ("ns", C.c_int),
                ("src_xz", PD), ("mt", PD), ("wavelet", PF), ("ntr", C.c_int), ("tr_ptr", PI),
                ("ch_xz", PD), ("ch_t", PD), ("gauge", C.c_double), ("das_mode", C.c_int), ("win", PI),
                ("ref_vp", PF), ("ref_vs", PF), ("ref_rho", PF), ("ckpt_interval", C.c_int),
                ("ckpt_store", C.c_int), ("exec", C.c_int), ("tile_x", C.c_int), ("tile_z", C.c_int),
                ("stencil", C.c_int), ("adj_tile_x", C.c_int), ("adj_tile_z", C.c_int), ("adj_stencil", C.c_int),
                ("overlap", C.c_int), ("force", PD), ("snap_store", C.c_int),
                ("stored_steps", C.c_int), ("adj_form", C.c_int)]


class PlanInfo(C.Structure):
    _fields_ = [("ckpt_interval", C.c_int), ("n_ckpt", C.c_int), ("tile_x", C.c_int), ("tile_z", C.c_int),
                ("adj_tile_x", C.c_int), ("adj_tile_z", C.c_int), ("stencil", C.c_int),
                ("stages", C.c_int), ("adj_stencil", C.c_int), ("adj_stages", C.c_int),
                ("overlap_fwd_blocks", C.c_int), ("overlap_adj_blocks", C.c_int),
                ("workspace_bytes", C.c_size_t), ("padded_cells", C.c_longlong),
                ("physical_cells", C.c_longlong), ("launches", C.c_longlong), ("layout", C.c_int),
                ("staged_stores", C.c_int), ("adj_persistent", C.c_int), ("snap_store", C.c_int),
                ("prefetch", C.c_int), ("stored_steps", C.c_int), ("adj_form", C.c_int),
                ("adj_layout", C.c_int)]


class ZoiDesc(C.Structure):
    _fields_ = [("active_x", PD), ("taper", PD), ("sink_xz", PD), ("sink_axes", PD),
                ("n", C.c_double), ("nu", C.c_double)]


class GroupsObjectiveCtx(C.Structure):
    _fields_ = [("groups", C.c_void_p), ("d_obs", C.c_void_p), ("eta", C.c_double * 3), ("b", C.c_void_p),
                ("bp", C.c_void_p), ("sink", C.c_void_p)]


class LbfgsInfo(C.Structure):
    _fields_ = [("phi", C.c_double), ("phi_prev", C.c_double), ("rate", C.c_double), ("alpha", C.c_double),
                ("evals", C.c_int), ("iters", C.c_int), ("pairs", C.c_int), ("ls_failed", C.c_int), ("stop", C.c_int)]


VP = C.c_void_p
# int fn(void *ctx, const float *x, double *phi, float *g, cudaStream_t stream)
OBJECTIVE_FN = C.CFUNCTYPE(C.c_int, VP, VP, C.POINTER(C.c_double), VP, VP)
SIGNATURES = {
    "efwi_plan_create": (C.c_int, [C.POINTER(VP), C.POINTER(PlanDesc)]),
    "efwi_plan_destroy": (C.c_int, [VP]),
    "efwi_plan_rebind": (C.c_int, [VP, C.POINTER(PlanDesc), VP]),
    "efwi_plan_set_zoi": (C.c_int, [VP, C.POINTER(ZoiDesc), VP]),
    "efwi_last_error": (C.c_char_p, [VP]),
    "efwi_plan_info": (C.c_int, [VP, C.POINTER(PlanInfo)]),
    "efwi_sync_status": (C.c_int, [VP, VP]),
    "efwi_forward": (C.c_int, [VP, VP, VP, VP, VP, VP]),
    "efwi_adjoint_gradient": (C.c_int, [VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP]),
    "efwi_zoi_weights": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.POINTER(ZoiDesc),
                                   VP, VP, VP, VP]),
    "efwi_regularization_grad": (C.c_int, [VP, VP, VP, VP, VP, C.c_double, VP, VP, VP]),
    "efwi_regularization_grad_n": (C.c_int, [VP, C.c_int, VP, VP, VP, VP, C.c_double, VP, VP, VP]),
    "efwi_collapse": (C.c_int, [C.c_int, C.c_int, C.c_int, VP, VP, VP, VP, VP, VP]),
    "efwi_lbfgs_create": (C.c_int, [C.POINTER(VP), C.c_longlong, C.c_int, C.c_double, C.c_double, C.c_int]),
    "efwi_lbfgs_destroy": (C.c_int, [VP]),
    "efwi_lbfgs_reset": (C.c_int, [VP]),
    "efwi_lbfgs_set_step0": (C.c_int, [VP, C.c_double]),
    "efwi_lbfgs_push": (C.c_int, [VP, VP, VP, C.POINTER(C.c_int), VP]),
    "efwi_lbfgs_direction": (C.c_int, [VP, VP, VP, VP]),
    "efwi_lbfgs_set_h0": (C.c_int, [VP, VP, VP]),
    "efwi_lbfgs_export": (C.c_int, [VP, C.POINTER(C.c_int), VP, VP, VP]),
    "efwi_lbfgs_iterate": (C.c_int, [VP, VP, C.POINTER(C.c_double), VP, OBJECTIVE_FN, VP, C.POINTER(LbfgsInfo), VP]),
    "efwi_lbfgs_run": (C.c_int, [VP, VP, VP, OBJECTIVE_FN, VP, C.c_int, C.c_double, C.POINTER(LbfgsInfo), VP]),
    "efwi_lbfgs_iterate_device": (C.c_int, [VP, VP, VP, VP, VP, VP, C.POINTER(LbfgsInfo), VP]),
    "efwi_groups_create": (C.c_int, [C.POINTER(VP), VP, C.POINTER(PlanDesc), C.c_int]),
    "efwi_groups_destroy": (C.c_int, [VP]),
    "efwi_groups_bind": (C.c_int, [VP, C.c_int, VP]),
    "efwi_groups_objective": (C.c_int, [VP, VP, VP, C.POINTER(C.c_double), VP, VP, VP, VP, VP, VP]),
    "efwi_groups_objective_fn": (C.c_int, [VP, VP, VP, VP, VP]),
    "efwi_regularization_grad_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, VP, VP, VP, VP, C.c_double, VP, VP,
                                                    VP]),
    "efwi_extended_objective": (C.c_int, [VP, VP, VP, VP, VP, PD, VP, VP, VP, VP, VP, VP]),
    "efwi_pseudo_hessian": (C.c_int, [VP, VP, VP, VP, C.c_double, VP, VP, VP]),
    "efwi_prof_enable": (C.c_int, [VP, C.c_int]),
    "efwi_selftest_timeout": (C.c_int, [VP, C.c_longlong, VP]),
    "efwi_selftest_store": (C.c_int, [C.c_int, C.c_longlong, VP, VP, VP, VP, VP]),
    "efwi_selftest_kahan": (C.c_int, [C.c_longlong, C.c_int, VP, VP, VP, VP]),
    "efwi_prof_read": (C.c_int, [VP, C.c_int, PD, C.POINTER(C.c_longlong)]),
}

_lib = None


def load(path: str = LIB):
    """Load libefwi_gb300.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2305_14130_gb300.build.build() "
                           "(the CUDA path has no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class EfwiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def check(code, plan_handle=None):
    if code != EFWI_OK:
        msg = _lib.efwi_last_error(plan_handle)
        raise EfwiError(code, msg.decode() if msg else "")
