"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a,
loads, exports every entry point include/efwi.h declares, its structs match
the ctypes binding, and argument validation answers before any device call."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "efwi.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2305_14130_gb300 import build, _abi
    build.build()
    return _abi.load()


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(efwi_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 11
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (efwi_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_struct_layouts_match_binding(tmp_path):
    from paper_2305_14130_gb300 import _abi
    prog = tmp_path / "layout.c"
    fields = [f for f, _ in _abi.PlanDesc._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "efwi.h"', 'int main(void) {',
             'printf("%zu\\n", sizeof(efwi_plan_desc));']
    lines += [f'printf("%zu\\n", offsetof(efwi_plan_desc, {f}));' for f in fields]
    lines += ['printf("%zu\\n", sizeof(efwi_lbfgs_info_t));']
    lines += [f'printf("%zu\\n", offsetof(efwi_lbfgs_info_t, {f}));' for f, _ in _abi.LbfgsInfo._fields_]
    lines += ['printf("%zu\\n", sizeof(efwi_plan_info_t));', 'printf("%zu\\n", sizeof(efwi_zoi_desc));',
              'printf("%zu\\n", sizeof(efwi_groups_objective_ctx));',
              'printf("%zu\\n", offsetof(efwi_groups_objective_ctx, sink));', 'return 0; }']
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == C.sizeof(_abi.PlanDesc)
    for f, off in zip(fields, vals[1:1 + len(fields)]):
        assert getattr(_abi.PlanDesc, f).offset == off, f
    lb = vals[1 + len(fields):1 + len(fields) + 1 + len(_abi.LbfgsInfo._fields_)]
    assert lb[0] == C.sizeof(_abi.LbfgsInfo)
    for (f, _), off in zip(_abi.LbfgsInfo._fields_, lb[1:]):
        assert getattr(_abi.LbfgsInfo, f).offset == off, f
    assert vals[-4] == C.sizeof(_abi.PlanInfo)
    assert vals[-3] == C.sizeof(_abi.ZoiDesc)
    assert vals[-2] == C.sizeof(_abi.GroupsObjectiveCtx)
    assert vals[-1] == _abi.GroupsObjectiveCtx.sink.offset


def _desc(p, **over):
    """A filled PlanDesc plus the numpy arrays it points into."""
    from paper_2305_14130_gb300 import _abi
    a = p.acq
    keep = [np.ascontiguousarray(a.src_xz, np.float64), np.ascontiguousarray(a.mt, np.float64),
            np.ascontiguousarray(a.wavelet, np.float32), np.ascontiguousarray(a.tr_ptr, np.int32),
            np.ascontiguousarray(a.ch_xz, np.float64), np.ascontiguousarray(a.ch_t, np.float64),
            np.ascontiguousarray(a.ref_vp, np.float32), np.ascontiguousarray(a.ref_vs, np.float32),
            np.ascontiguousarray(a.ref_rho, np.float32)]
    P = lambda x, t: x.ctypes.data_as(C.POINTER(t))
    d = _abi.PlanDesc(nx=a.nx, nz=a.nz, dx=a.dx, dz=a.dz, nt=a.nt, dt=a.dt, npml=a.npml, pml_R=a.pml_R,
                      pml_vmax=0.0, pml_f0=a.pml_f0, ns=a.ns, src_xz=P(keep[0], C.c_double),
                      mt=P(keep[1], C.c_double), wavelet=P(keep[2], C.c_float), ntr=a.ntr,
                      tr_ptr=P(keep[3], C.c_int), ch_xz=P(keep[4], C.c_double), ch_t=P(keep[5], C.c_double),
                      gauge=a.gauge, das_mode=a.das_mode, win=None, ref_vp=P(keep[6], C.c_float),
                      ref_vs=P(keep[7], C.c_float), ref_rho=P(keep[8], C.c_float), ckpt_interval=0,
                      ckpt_store=0, exec=1, tile_x=0, tile_z=0)
    for k, v in over.items():
        setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("over,code,msg", [
    ({"nx": 0}, -1, "positive"),
    ({"dt": 1e-2}, -2, "CFL"),
    ({"das_mode": 7}, -1, "das_mode"),
    ({"ckpt_store": 9}, -1, "ckpt_store"),
    ({"npml": 0}, -1, "npml"),
    ({"tile_x": 8, "tile_z": 0}, -1, "tile"),
    ({"ckpt_interval": -2}, -1, "ckpt_interval"),
    ({"snap_store": 5}, -1, "snap_store"),
    ({"snap_store": 1, "exec": 0}, -1, "EXEC_BATCHED"),
    ({"snap_store": 2, "overlap": 2}, -1, "FP32 snapshots"),
    ({"stored_steps": -1}, -1, "stored_steps"),
    ({"stored_steps": 10, "overlap": 2}, -1, "forced overlap"),
    ({"adj_form": 3}, -1, "adj_form"),
    ({"adj_form": 2, "exec": 0}, -1, "scaled-stress"),
    ({"adj_form": 2, "adj_stencil": 3}, -1, "scaled-stress"),
])
def test_plan_create_rejects_bad_descriptions(lib, over, code, msg):
    d, keep = _desc(W.tiny(), **over)
    h = C.c_void_p()
    assert lib.efwi_plan_create(C.byref(h), C.byref(d)) == code
    assert not h.value
    assert msg in lib.efwi_last_error(None).decode()


def test_plan_create_rejects_positions_outside_window(lib):
    p = W.tiny()
    p.acq.src_xz = p.acq.src_xz.copy()
    p.acq.src_xz[1, 0] = -3.0
    d, keep = _desc(p)
    h = C.c_void_p()
    assert lib.efwi_plan_create(C.byref(h), C.byref(d)) == -1
    assert "source 1" in lib.efwi_last_error(None).decode()
    p = W.tiny()
    p.acq.ch_xz = p.acq.ch_xz.copy()
    p.acq.ch_xz[3, 1] = 1e4
    d, keep = _desc(p)
    assert lib.efwi_plan_create(C.byref(h), C.byref(d)) == -1
    assert "trace 3" in lib.efwi_last_error(None).decode()


def test_collapse_rejects_bad_arguments(lib):
    """Argument checks happen on the host, before any launch."""
    p = C.c_void_p(16)
    assert lib.efwi_collapse(0, 4, 4, p, p, p, p, p, None) == -1
    assert "ns, nx and nz" in lib.efwi_last_error(None).decode()
    assert lib.efwi_collapse(2, 4, 4, None, p, p, p, p, None) == -1
    assert "NULL" in lib.efwi_last_error(None).decode()


def test_lbfgs_rejects_bad_arguments(lib):
    """Argument checks of the l-BFGS handle happen before any allocation."""
    h = C.c_void_p()
    assert lib.efwi_lbfgs_create(C.byref(h), 0, 5, 1e-4, 0.9, 20) == -1
    assert lib.efwi_lbfgs_create(C.byref(h), 100, 0, 1e-4, 0.9, 20) == -1
    assert lib.efwi_lbfgs_create(C.byref(h), 100, 5, 0.9, 1e-4, 20) == -1
    assert "c1 < c2" in lib.efwi_last_error(None).decode()
    assert lib.efwi_lbfgs_create(C.byref(h), 100, 5, 1e-4, 0.9, 0) == -1
    assert not h.value
    assert lib.efwi_lbfgs_destroy(None) == 0
    assert lib.efwi_lbfgs_reset(None) == -1
    assert lib.efwi_lbfgs_set_step0(None, 1.0) == -1


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.efwi_plan_create(C.byref(h), None) == -1
    assert lib.efwi_plan_create(None, None) == -1
    assert lib.efwi_plan_destroy(None) == 0
    assert lib.efwi_forward(None, None, None, None, None, None) == -1
    assert lib.efwi_pseudo_hessian(None, None, None, None, 1e-3, None, None, None) == -1


def test_enum_values_match_binding(tmp_path):
    """Every status code and enum value the binding (and the workloads' DAS modes)
    passes across the ABI equals the header's, read by compiling against it."""
    from paper_2305_14130_gb300 import _abi
    import workloads as W
    names = list(_abi.STATUS.values())
    names += [f"EFWI_STORE_{k.upper()}" for k in _abi.STORE] + [f"EFWI_EXEC_{k.upper()}" for k in _abi.EXEC]
    names += [f"EFWI_STENCIL_{k.upper()}" for k in _abi.STENCIL] + [f"EFWI_OVERLAP_{k.upper()}" for k in _abi.OVERLAP]
    names += [f"EFWI_ADJ_FORM_{k.upper()}" for k in _abi.ADJ_FORM]
    names += ["EFWI_DAS_STRAIN", "EFWI_DAS_STRAIN_RATE", "EFWI_DAS_VELOCITY", "EFWI_CKPT_AUTO"]
    prog = tmp_path / "enums.c"
    prog.write_text("\n".join(['#include <stdio.h>', '#include "efwi.h"', 'int main(void) {']
                              + [f'printf("%d\\n", (int){n});' for n in names] + ['return 0; }']))
    exe = tmp_path / "enums"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = dict(zip(names, (int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.split())))
    for code, n in _abi.STATUS.items():
        assert got[n] == code, n
    for table, prefix in ((_abi.STORE, "STORE"), (_abi.EXEC, "EXEC"), (_abi.STENCIL, "STENCIL"),
                          (_abi.OVERLAP, "OVERLAP"), (_abi.ADJ_FORM, "ADJ_FORM")):
        for k, v in table.items():
            assert got[f"EFWI_{prefix}_{k.upper()}"] == v, k
    assert (got["EFWI_DAS_STRAIN"], got["EFWI_DAS_STRAIN_RATE"], got["EFWI_DAS_VELOCITY"]) == \
        (W.STRAIN, W.STRAIN_RATE, W.VELOCITY) == (_abi.DAS_STRAIN, _abi.DAS_STRAIN_RATE, _abi.DAS_VELOCITY)
    assert got["EFWI_CKPT_AUTO"] == _abi.CKPT_AUTO
