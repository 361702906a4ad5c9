"""GPU test of efwi_regularization_grad_noalloc, the allocation-free entry point.

It is meant for callers that cannot let the library allocate device memory
(they own all device memory through their own pool or budget) or that want
the consistency-term gradient without creating a plan.  The test calls it
through the C ABI twice in a row (its static scratch array keeps the previous
call's contents) and compares each result with the plan-based
efwi_regularization_grad, within the regularization parity tolerances used by
the other GPU tests.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W
from oracle import extension as X

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def efwi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_14130_gb300 as m
    return m


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _noalloc(lib, ns, nx, nz, m, b, bp, sink, eta, g):
    phi = torch.empty((), dtype=torch.float64, device="cuda")
    rc = lib.efwi_regularization_grad_noalloc(ns, nx, nz, _ptr(m), _ptr(b), _ptr(bp), _ptr(sink), float(eta),
                                              _ptr(phi), _ptr(g),
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, phi


@pytest.mark.parametrize("ns,nz,nx", [(5, 37, 53), (6, 256, 1024)])
def test_noalloc_matches_plan_entry_point_twice(efwi, ns, nz, nx):
    from paper_2305_14130_gb300 import _abi
    lib = _abi.load()
    p = W.tiny(nx=nx, nz=nz, ns=ns, nt=4, npml=3, nch=2)
    b, bp, sink = X.zoi_weights(p.zoi, nx, nz, p.acq.dx, p.acq.dz)
    rng = np.random.default_rng(11)
    dev = lambda a, dt=np.float32: torch.tensor(np.asarray(a, dt), device="cuda")
    db, dbp, dsink = dev(b), dev(bp), dev(sink, np.uint8)
    plan = efwi.Plan(p.acq, exec="plain")
    for call in range(2):
        m = dev(3000 + 100 * rng.standard_normal((ns, nz, nx)))
        g0 = dev(rng.standard_normal((ns, nz, nx)))
        eta = 0.3 + 0.2 * call
        phi_ref, g_ref = plan.regularization_grad(m, db, dbp, dsink, eta, g=g0.clone())
        g = g0.clone()
        rc, phi = _noalloc(lib, ns, nx, nz, m, db, dbp, dsink, eta, g)
        assert rc == 0, lib.efwi_last_error(None)
        torch.cuda.synchronize()
        assert abs(phi.item() - phi_ref.item()) <= 1e-10 * phi_ref.item()
        num = torch.linalg.vector_norm((g - g0).double() - (g_ref - g0).double())
        den = torch.linalg.vector_norm((g_ref - g0).double())
        assert float(num / den) <= 1e-5
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(efwi):
    from paper_2305_14130_gb300 import _abi
    lib = _abi.load()
    t = torch.zeros(8, device="cuda")
    s = torch.zeros(8, dtype=torch.uint8, device="cuda")
    rc, _ = _noalloc(lib, 1, 1025, 1024, t, t, t, s, 1.0, t)
    assert rc == -1
    assert b"1048576-pixel limit" in lib.efwi_last_error(None)
