"""GPU tests of failure detection, made without faulting, trapping or hanging the
GPU: a bounded device wait that runs out (a barrier nothing completes, a budget of
about a millisecond), a model with a non-finite or non-positive value, and a forced
workspace-allocation failure.  Each is reported as a status code, and the plan (or
the next plan) works normally afterwards."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W
from common import rel_l2, rounded

pytestmark = pytest.mark.gpu
ERR_OOM, ERR_TIMEOUT, ERR_NAN = -3, -5, -6


@pytest.fixture(scope="module")
def efwi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_14130_gb300 as m
    return m


def dev(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a, np.float32)), device="cuda")


def _problem():
    p = rounded(W.tiny(nx=40, nz=30, ns=2, nt=40, npml=5))
    return p, [dev(v) for v in (p.vp, p.vs, p.rho)]


def test_bounded_wait_runs_out_and_is_reported(efwi):
    p, m = _problem()
    plan = efwi.Plan(p.acq, exec="batched")
    d0 = plan.forward(*m).clone()
    lib = efwi.load_library()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.efwi_selftest_timeout(plan._h, 1 << 21, stream) == 0
    with pytest.raises(efwi.EfwiError) as e:
        plan.sync_status()
    assert e.value.code == ERR_TIMEOUT and "bounded wait" in str(e.value)
    plan.sync_status()                                    # the flag was cleared
    assert torch.equal(plan.forward(*m), d0)              # and the plan still works
    plan.sync_status()
    assert lib.efwi_selftest_timeout(plan._h, 0, stream) == -1
    plan.close()


@pytest.mark.parametrize("bad", ["nan_vp", "inf_vs", "zero_rho"])
def test_invalid_model_is_reported(efwi, bad):
    p, m = _problem()
    plan = efwi.Plan(p.acq, exec="batched")
    d_obs = plan.forward(*m).clone()
    plan.sync_status()
    k, val = {"nan_vp": (0, float("nan")), "inf_vs": (1, float("inf")), "zero_rho": (2, 0.0)}[bad]
    mb = [t.clone() for t in m]
    mb[k][1, 12, 17] = val
    plan.gradient(*mb, d_obs)
    with pytest.raises(efwi.EfwiError) as e:
        plan.sync_status()
    assert e.value.code == ERR_NAN
    phi, *g = plan.gradient(*m, d_obs)                    # a valid model afterwards: no error,
    plan.sync_status()                                    # zero residual, zero gradient
    assert float(phi.item()) == 0.0 and all(float(t.abs().max()) == 0.0 for t in g)
    plan.close()


def test_forced_allocation_failure(efwi, monkeypatch):
    p, m = _problem()
    monkeypatch.setenv("EFWI_TEST_FAIL_ALLOC", "4")
    with pytest.raises(efwi.EfwiError) as e:
        efwi.Plan(p.acq, exec="batched")
    assert e.value.code == ERR_OOM and "EFWI_TEST_FAIL_ALLOC" in str(e.value)
    monkeypatch.delenv("EFWI_TEST_FAIL_ALLOC")
    plan = efwi.Plan(p.acq, exec="batched")               # nothing left behind
    d = plan.forward(*m)
    plan.sync_status()
    from oracle import elastic as E
    assert rel_l2(d.cpu().numpy(), E.forward(p.acq, p.vp, p.vs, p.rho)) <= 1e-4
    plan.close()


def test_zero_shear_modulus_is_reported_by_gradients(efwi):
    """A gradient divides by the shear modulus (the chain rule through the harmonic
    mean mu_xz, and the scaled-stress adjoint's conversion of its sums): a cell with
    Vs = 0 on the physical grid is reported by a gradient call, in either adjoint
    form, and not by forward modelling, which needs no mu > 0."""
    p, m = _problem()
    mb = [t.clone() for t in m]
    mb[1][0, 14, 20] = 0.0
    for form in ("scaled", "stress"):
        plan = efwi.Plan(p.acq, exec="batched", adj_form=form)
        d_obs = plan.forward(*m).clone()
        plan.forward(*mb)
        plan.sync_status()
        plan.gradient(*mb, d_obs)
        with pytest.raises(efwi.EfwiError) as e:
            plan.sync_status()
        assert e.value.code == ERR_NAN and "mu > 0" in str(e.value)
        phi, *g = plan.gradient(*m, d_obs)                # the valid model afterwards: no error
        plan.sync_status()
        assert float(phi.item()) == 0.0
        plan.close()
