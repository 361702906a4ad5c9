"""GPU tests of efwi_regularization_grad_noalloc, the allocation-free entry point.

It serves callers that cannot let a library allocate device memory (they hand
out all device memory through their own pool or budget) and callers that want
the consistency-term gradient without creating a plan.  The tests call it
through the C ABI twice in a row (its static scratch array keeps the previous
call's contents) and check

* that the gradient equals the plan-based efwi_regularization_grad bit for bit
  (both evaluate every pixel with the same per-pixel routine) and phi_reg
  within the reduction-order tolerance;
* both results against the FP64 oracle of the consistency term;
* that the calls leave the device's free memory unchanged, at sizes far apart;
* that sizes beyond the scratch are refused.

This file is collected last on purpose.
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


def _noalloc(lib, ns, nx, nz, m, b, bp, sink, eta, g, phi=None):
    if phi is None:
        phi = torch.empty((), dtype=torch.float64, device="cuda")
    rc = lib.efwi_regularization_grad_noalloc(ns, nx, nz, _ptr(m), _ptr(b), _ptr(bp), _ptr(sink), float(eta),
                                              _ptr(phi), _ptr(g),
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, phi


def _weights(ns, nz, nx):
    p = W.tiny(nx=nx, nz=nz, ns=ns, nt=4, npml=3, nch=2)
    b, bp, sink = X.zoi_weights(p.zoi, nx, nz, p.acq.dx, p.acq.dz)
    # the device works on FP32 weights; the oracle gets the same rounded values
    return p, np.float32(b).astype(np.float64), np.float32(bp).astype(np.float64), sink


@pytest.mark.parametrize("ns,nz,nx", [(5, 37, 53), (6, 256, 1024)])
def test_noalloc_matches_plan_entry_point_and_oracle_twice(efwi, ns, nz, nx):
    from paper_2305_14130_gb300 import _abi
    lib = _abi.load()
    p, b, bp, sink = _weights(ns, nz, nx)
    assert sink.any() and not sink.all()
    rng = np.random.default_rng(11)
    dev = lambda a, dt=np.float32: torch.tensor(np.asarray(a, dt), device="cuda")
    db, dbp, dsink = dev(b), dev(bp), dev(sink, np.uint8)
    plan = efwi.Plan(p.acq, exec="plain")
    for call in range(2):
        m32 = np.float32(3000 + 100 * rng.standard_normal((ns, nz, nx)))
        g0_32 = np.float32(rng.standard_normal((ns, nz, nx)))
        m, g0 = dev(m32), dev(g0_32)
        eta = 0.3 + 0.2 * call
        phi_ref, g_ref = plan.regularization_grad(m, db, dbp, dsink, eta, g=g0.clone())
        g = g0.clone()
        rc, phi = _noalloc(lib, ns, nx, nz, m, db, dbp, dsink, eta, g)
        assert rc == 0, lib.efwi_last_error(None)
        torch.cuda.synchronize()
        # same per-pixel routine on the same inputs: the same bits; phi differs only by
        # the order of the FP64 block sums
        assert torch.equal(g, g_ref)
        assert abs(phi.item() - phi_ref.item()) <= 1e-10 * phi_ref.item()
        # the FP64 oracle of the consistency term (eqs. 8, 11, 12)
        phi_o, g_o = X.regularization(m32.astype(np.float64), b, bp, sink, eta)
        assert abs(phi.item() - phi_o) <= 1e-10 * phi_o
        inc = g.double().cpu().numpy() - g0_32.astype(np.float64)
        assert np.linalg.norm(inc - g_o) <= 1e-5 * np.linalg.norm(g_o)
    plan.close()


def test_noalloc_allocates_no_device_memory(efwi):
    from paper_2305_14130_gb300 import _abi
    lib = _abi.load()
    cases = []
    for ns, nz, nx in [(3, 37, 53), (2, 1024, 1024)]:
        p, b, bp, sink = _weights(ns, nz, nx)
        dev = lambda a, dt=np.float32: torch.tensor(np.asarray(a, dt), device="cuda")
        m = dev(np.full((ns, nz, nx), 2500.0) + np.arange(ns)[:, None, None])
        cases.append((ns, nx, nz, m, dev(b), dev(bp), dev(sink, np.uint8), torch.zeros_like(m),
                      torch.empty((), dtype=torch.float64, device="cuda")))
    # a first call may load the module; everything the calls use exists before the count
    for ns, nx, nz, m, b, bp, sink, g, phi in cases:
        assert _noalloc(lib, ns, nx, nz, m, b, bp, sink, 0.5, g, phi)[0] == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for ns, nx, nz, m, b, bp, sink, g, phi in cases:
            assert _noalloc(lib, ns, nx, nz, m, b, bp, sink, 0.5, g, phi)[0] == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_scratch(efwi):
    from paper_2305_14130_gb300 import _abi
    lib = _abi.load()
    t = torch.zeros(8, device="cuda")
    s = torch.zeros(8, dtype=torch.uint8, device="cuda")
    rc, _ = _noalloc(lib, 1, 1025, 1024, t, t, t, s, 1.0, t)
    assert rc == -1
    assert b"1048576-pixel limit" in lib.efwi_last_error(None)
