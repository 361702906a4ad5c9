"""Shot groups through one plan (efwi_plan_rebind): an extended problem whose
sources do not fit one plan runs group by group, each group a slice of the
problem (every component is independent through eqs. 1-6).  A plan bound to
the next group's sources and receivers must give what a fresh plan gives."""
import copy
import dataclasses

import numpy as np
import pytest
import torch

import workloads as W
from common import f32, rounded
from oracle import elastic as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def efwi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_14130_gb300 as m
    return m


def dev(a, dtype=np.float32):
    return torch.tensor(np.ascontiguousarray(np.asarray(a, dtype)), device="cuda")


def observed(p):
    ns = p.acq.ns
    return f32(E.forward(p.acq, *(np.repeat(m[None], ns, 0) for m in (p.true_vp, p.true_vs, p.true_rho))))


@pytest.mark.parametrize("snap", ["fp32", "fp16"])
def test_rebound_groups_equal_one_plan(efwi, snap):
    from paper_2305_14130_gb300.groups import grouped_gradient
    p = rounded(W.tiny(nx=48, nz=26, ns=6, nt=50, npml=4))
    d_obs = dev(observed(p))
    m = (dev(p.vp), dev(p.vs), dev(p.rho))
    plan = efwi.Plan(p.acq, exec="batched", snap_store=snap)
    phi, *g = plan.gradient(*m, d_obs)
    plan.close()
    stats = {}
    phi_g, gg = grouped_gradient(p.acq, *m, d_obs, 2, exec="batched", snap_store=snap, stats=stats)
    assert stats["rebind_s"] > 0                 # groups 2 and 3 rebound the first group's plan
    assert phi_g == pytest.approx(float(phi.item()), rel=1e-12)
    for a, b in zip(g, gg):
        assert torch.equal(a, b)


def test_rebind_with_a_new_gather_shape(efwi):
    """Receivers moved so that the adjoint-source gather changes shape: the plan
    drops its captured time loops and captures them again; results equal a fresh
    plan's.  Moving them back restores the first results bit for bit."""
    p = rounded(W.tiny(nx=40, nz=30, ns=2, nt=40, npml=5))
    d_obs = dev(observed(p))
    m = (dev(p.vp), dev(p.vs), dev(p.rho))
    moved = copy.deepcopy(p.acq)
    moved.ch_xz = np.asarray(moved.ch_xz).copy()
    moved.ch_xz[:, 0] += 0.37 * p.acq.dx           # off the grid points: other corners
    plan = efwi.Plan(p.acq, exec="batched")
    first = [t.clone() for t in plan.gradient(*m, d_obs, return_data=True)]
    plan.rebind(moved)
    second = [t.clone() for t in plan.gradient(*m, d_obs, return_data=True)]
    fresh = efwi.Plan(moved, exec="batched")
    ref = [t.clone() for t in fresh.gradient(*m, d_obs, return_data=True)]
    fresh.close()
    for a, b in zip(second, ref):
        assert torch.equal(a, b)
    plan.rebind(p.acq)
    third = [t.clone() for t in plan.gradient(*m, d_obs, return_data=True)]
    for a, b in zip(first, third):
        assert torch.equal(a, b)
    plan.sync_status()
    plan.close()


def test_rebind_rejects_another_shape(efwi):
    p = rounded(W.tiny(nx=40, nz=30, ns=2, nt=40, npml=5))
    plan = efwi.Plan(p.acq, exec="batched")
    other = dataclasses.replace(copy.deepcopy(p.acq), nt=39)
    other.wavelet = np.asarray(other.wavelet)[:, :40]
    with pytest.raises(efwi.EfwiError):
        plan.rebind(other)
    forced = W.with_forces(copy.deepcopy(p)).acq
    with pytest.raises(efwi.EfwiError):
        plan.rebind(forced)
    # the plan is unchanged and still usable
    d_obs = dev(observed(p))
    m = (dev(p.vp), dev(p.vs), dev(p.rho))
    a = [t.clone() for t in plan.gradient(*m, d_obs)]
    fresh = efwi.Plan(p.acq, exec="batched")
    b = [t.clone() for t in fresh.gradient(*m, d_obs)]
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    fresh.close()
    plan.close()
