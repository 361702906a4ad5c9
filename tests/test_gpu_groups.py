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
from common import f32, rel_l2, rounded
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


def _three_groups():
    """A 6-source tiny extended problem as 3 groups of 2 sources (same receivers)."""
    from paper_2305_14130_gb300.groups import group_acquisition
    p = rounded(W.tiny(nx=40, nz=30, ns=6, nt=60, npml=6))
    acqs = [group_acquisition(p.acq, [2 * k, 2 * k + 1])[0] for k in range(3)]
    return p, acqs


def test_group_set_objective_equals_rebound_plans(efwi):
    """efwi_groups_objective (groups bound by device copies, eq. 8 over all six
    components) against the host path: grouped_gradient through a rebound plan and
    the consistency term of all components."""
    from paper_2305_14130_gb300.groups import GroupSet, grouped_gradient
    p, acqs = _three_groups()
    acq = p.acq
    d_obs = dev(observed(p))
    x = torch.stack([dev(p.vp), dev(p.vs), dev(p.rho)]).contiguous()     # [3, 6, nz, nx]
    b, bp, sink = efwi.zoi_weights(6, acq.nx, acq.nz, acq.dx, acq.dz, p.zoi)
    eta = (1e-4, 2e-4, 3e-4)
    plan = efwi.Plan(acqs[0], exec="batched")
    gs = GroupSet(plan, acqs)
    phi, g = gs.objective(x, d_obs.view(3, -1, acq.nt), eta, b, bp, sink)
    torch.cuda.synchronize()
    phi_d, gg = grouped_gradient(acq, x[0], x[1], x[2], d_obs, 2, exec="batched")
    phi_ref = phi_d
    for k in range(3):
        r, _ = plan.regularization_grad(x[k], b, bp, sink, eta[k], g=gg[k])
        phi_ref += float(r.item())
    for k in range(3):
        assert torch.equal(g[k], gg[k])
    assert phi.item() == pytest.approx(phi_ref, rel=1e-12)
    gs.close()
    plan.close()


@pytest.mark.parametrize("step0", [0.0, 1e-3, 1.0])
def test_device_line_search_matches_host_line_search(efwi, step0):
    """Three l-BFGS iterations of the 6-source problem in groups: the line search as a
    device state machine replayed from a CUDA graph (efwi_lbfgs_iterate_device)
    against the host line search (efwi_lbfgs_iterate) on the same objective: the same
    accepted steps and evaluation counts, the same iterates and objective values.
    A first trial of the model's own length (step0 = 1) makes the modelling
    unstable; both searches must back off from the non-finite trial alike."""
    from paper_2305_14130_gb300.groups import GroupSet
    from paper_2305_14130_gb300.optim import LBFGS
    p, acqs = _three_groups()
    acq = p.acq
    d_obs = dev(observed(p)).view(3, -1, acq.nt).contiguous()
    b, bp, sink = efwi.zoi_weights(6, acq.nx, acq.nz, acq.dx, acq.dz, p.zoi)
    eta = (1e-3, 1e-3, 1e-3)
    plan = efwi.Plan(acqs[0], exec="batched")
    gs = GroupSet(plan, acqs)
    x0 = torch.stack([dev(p.vp), dev(p.vs), dev(p.rho)]).contiguous().view(-1)
    n = x0.numel()
    shape = (3, 6, acq.nz, acq.nx)

    def host_objective(xv, gv):
        ph, _ = gs.objective(xv.view(shape), d_obs, eta, b, bp, sink, g=gv.view(shape))
        return float(ph.item())

    xh, gh = x0.clone(), torch.empty_like(x0)
    phih = host_objective(xh, gh)
    xd, gd = x0.clone(), torch.empty_like(x0)
    phid = torch.empty((), dtype=torch.float64, device="cuda")
    gs.objective(xd.view(shape), d_obs, eta, b, bp, sink, phi=phid, g=gd.view(shape))
    oh, od = LBFGS(n, m=5), LBFGS(n, m=5)
    if step0:                                   # first trial: a fraction of the model norm
        for o in (oh, od):
            o.set_step0(step0 * float(torch.linalg.vector_norm(x0)))
    dobj = gs.device_objective(d_obs, eta, b, bp, sink)
    done = 0
    for it in range(4):
        phih, ih = oh.iterate(xh, phih, gh, host_objective)
        idv = od.iterate_device(xd, phid, gd, dobj)
        torch.cuda.synchronize()
        print(f"iteration {it}: host alpha {ih['alpha']:.6g} evals {ih['evals']} phi {phih:.9e} "
              f"failed {ih['ls_failed']}; device alpha {idv['alpha']:.6g} evals {idv['evals']} "
              f"phi {phid.item():.9e} failed {idv['ls_failed']}")
        assert idv["ls_failed"] == ih["ls_failed"] and idv["evals"] == ih["evals"]
        if ih["ls_failed"]:
            break
        assert idv["pairs"] == ih["pairs"]
        assert idv["alpha"] == pytest.approx(ih["alpha"], rel=1e-9)
        assert phid.item() == pytest.approx(phih, rel=1e-9)
        assert idv["rate"] == pytest.approx(ih["rate"], rel=1e-6, abs=1e-12)
        assert rel_l2(xd.cpu().numpy(), xh.cpu().numpy()) <= 1e-7
        assert phih < ih["phi_prev"]
        done += 1
    assert done >= 2
    oh.close()
    od.close()
    gs.close()
    plan.close()
