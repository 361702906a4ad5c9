"""GPU: the torch.autograd path, finite differences and properties at full size.

* DataMisfit / Consistency backpropagate exactly the kernels' gradients and
  match the FP64 oracle gradient (rel-L2 <= 1e-4);
* central finite differences of phi_ext through the library agree with
  <grad, dm> (FP32 time stepping: tolerance 1e-2) on a tiny grid and on the
  full 1000x300, 32-shot, nt = 4000 workload in the bench's configuration;
* a window covering the whole grid reproduces the unwindowed result bit for
  bit; one source and no traces are handled.
"""
import copy

import numpy as np
import pytest
import torch

import workloads as W
from common import f32, rel_l2, rounded
from oracle import elastic as E
from oracle import extension as X

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


def test_autograd_matches_kernels_and_oracle(efwi):
    from paper_2305_14130_gb300.autograd import extended_objective
    p = rounded(W.tiny(nx=40, nz=30, ns=3, nt=60, npml=6))
    d_obs = observed(p)
    acq = p.acq
    bo, bpo, sinko = X.zoi_weights(p.zoi, acq.nx, acq.nz, acq.dx, acq.dz)
    bo, bpo = f32(bo), f32(bpo)
    eta = (2e-4, 3e-4, 5e-4)
    plan = efwi.Plan(acq, exec="batched")
    vp, vs, rho = (dev(m).requires_grad_() for m in (p.vp, p.vs, p.rho))
    phi = extended_objective(plan, vp, vs, rho, dev(d_obs), eta, dev(bo), dev(bpo), dev(sinko, np.uint8))
    phi.backward()
    phi_o, gvp_o, gvs_o, grho_o = E.gradient(acq, p.vp, p.vs, p.rho, d_obs)
    regs = [X.regularization(m, bo, bpo, sinko, e) for m, e in zip((p.vp, p.vs, p.rho), eta)]
    assert abs(phi.item() - (phi_o + sum(r[0] for r in regs))) <= 1e-4 * phi.item()
    for g, go, r in zip((vp.grad, vs.grad, rho.grad), (gvp_o, gvs_o, grho_o), regs):
        assert rel_l2(g.cpu().numpy(), go + r[1]) <= 1e-4
    plan.close()


def _fd(plan, efwi, ms, d_obs, eta, zoi_dev, direction, h):
    from paper_2305_14130_gb300.autograd import extended_objective
    vals = []
    for sgn in (1.0, -1.0):
        pert = [m + sgn * h * d for m, d in zip(ms, direction)]
        vals.append(extended_objective(plan, *pert, d_obs, eta, *zoi_dev).item())
    return (vals[0] - vals[1]) / (2 * h)


def test_finite_difference_tiny(efwi):
    from paper_2305_14130_gb300.autograd import extended_objective
    p = rounded(W.tiny(nx=40, nz=30, ns=2, nt=60, npml=6))
    d_obs = dev(observed(p))
    acq = p.acq
    zoi_dev = efwi.zoi_weights(acq.ns, acq.nx, acq.nz, acq.dx, acq.dz, p.zoi)
    eta = (1e-4, 1e-4, 1e-4)
    plan = efwi.Plan(acq, exec="batched")
    ms = [dev(m).requires_grad_() for m in (p.vp, p.vs, p.rho)]
    extended_objective(plan, *ms, d_obs, eta, *zoi_dev).backward()
    rng = np.random.default_rng(3)
    direction = [dev(rng.standard_normal(m.shape)) * m.detach().abs().max() for m in ms]
    an = sum(float(torch.sum(m.grad.double() * d.double())) for m, d in zip(ms, direction))
    with torch.no_grad():
        fd = _fd(plan, efwi, [m.detach() for m in ms], d_obs, eta, zoi_dev, direction, 1e-3)
    assert abs(fd - an) <= 1e-2 * abs(an), (fd, an)
    plan.close()


def test_finite_difference_full_size(efwi):
    """32 shots, 1000x300, nt=4000: FD of phi_ext along a smooth perturbation in the layer."""
    from paper_2305_14130_gb300.autograd import extended_objective
    p = rounded(W.guided_wave_1000x300())
    acq = p.acq
    plan = efwi.Plan(acq, exec="batched")
    ns = acq.ns
    tv = lambda m: dev(np.repeat(np.asarray(m)[None], ns, 0))
    d_obs = plan.forward(tv(p.true_vp), tv(p.true_vs), tv(p.true_rho)).clone()
    zoi_dev = efwi.zoi_weights(ns, acq.nx, acq.nz, acq.dx, acq.dz, p.zoi)
    ms = [dev(m).requires_grad_() for m in (p.vp, p.vs, p.rho)]
    extended_objective(plan, *ms, d_obs, p.eta, *zoi_dev).backward()
    bump = W.gaussian_bump(acq.nx, acq.nz, 500, 150, 60, 12)
    rng = np.random.default_rng(4)
    direction = [dev(np.repeat(bump[None], ns, 0) * (1 + 0.1 * rng.standard_normal((ns, 1, 1)))) * s
                 for s in (40.0, 30.0, 20.0)]
    an = sum(float(torch.sum(m.grad.double() * d.double())) for m, d in zip(ms, direction))
    with torch.no_grad():
        fd = _fd(plan, efwi, [m.detach() for m in ms], d_obs, p.eta, zoi_dev, direction, 1e-2)
    assert abs(fd - an) <= 1e-2 * abs(an), (fd, an)
    plan.sync_status()
    plan.close()


def test_full_window_reproduces_unwindowed(efwi):
    p = rounded(W.tiny(nx=45, nz=31, ns=2, nt=50, npml=5))
    d_obs = observed(p)
    args = (dev(p.vp), dev(p.vs), dev(p.rho), dev(d_obs))
    a = [t.clone() for t in efwi.Plan(p.acq, exec="batched").gradient(*args, return_data=True)]
    q = copy.deepcopy(p)
    q.acq.win = np.array([[0, p.acq.nx]] * p.acq.ns, np.int32)
    b = [t.clone() for t in efwi.Plan(q.acq, exec="batched").gradient(*args, return_data=True)]
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_single_source_and_no_traces(efwi):
    p = rounded(W.tiny(nx=40, nz=30, ns=1, nt=40, npml=5))
    d_obs = observed(p)
    plan = efwi.Plan(p.acq, exec="batched")
    phi, gvp, gvs, grho = plan.gradient(dev(p.vp), dev(p.vs), dev(p.rho), dev(d_obs))
    phi_o, gvp_o, _, _ = E.gradient(p.acq, p.vp, p.vs, p.rho, d_obs)
    assert abs(phi.item() - phi_o) <= 1e-4 * phi_o
    assert rel_l2(gvp.cpu().numpy(), gvp_o) <= 1e-4
    plan.close()
    q = copy.deepcopy(p)
    q.acq.tr_ptr = np.array([0, 0], np.int32)
    q.acq.ch_xz = np.zeros((0, 2))
    q.acq.ch_t = np.zeros((0, 2))
    plan = efwi.Plan(q.acq, exec="batched")
    d = plan.forward(dev(p.vp), dev(p.vs), dev(p.rho))
    phi, gvp, gvs, grho = plan.gradient(dev(p.vp), dev(p.vs), dev(p.rho), torch.zeros((0, q.acq.nt), device="cuda"))
    torch.cuda.synchronize()
    assert d.shape == (0, q.acq.nt)
    assert phi.item() == 0.0 and not gvp.any() and not gvs.any() and not grho.any()
    plan.close()


def test_extended_fwi_function_matches_the_two_terms(efwi):
    """ExtendedFWI.apply (eq. 8 in one Function, with the plan's zone-of-influence
    weights) gives the objective and gradients of DataMisfit + Consistency."""
    from paper_2305_14130_gb300.autograd import extended_objective
    p = rounded(W.tiny(nx=40, nz=30, ns=3, nt=60, npml=6))
    d_obs = dev(observed(p))
    acq = p.acq
    eta = (2e-4, 3e-4, 5e-4)
    plan = efwi.Plan(acq, exec="batched")
    plan.set_zoi(p.zoi)
    b, bp, sink = efwi.zoi_weights(acq.ns, acq.nx, acq.nz, acq.dx, acq.dz, p.zoi)
    a = [dev(m).requires_grad_() for m in (p.vp, p.vs, p.rho)]
    phi_a = efwi.ExtendedFWI.apply(*a, plan, d_obs, eta)
    phi_a.backward()
    c = [dev(m).requires_grad_() for m in (p.vp, p.vs, p.rho)]
    phi_c = extended_objective(plan, *c, d_obs, eta, b, bp, sink)
    phi_c.backward()
    assert phi_a.item() == pytest.approx(phi_c.item(), rel=1e-12)
    for x, y in zip(a, c):
        assert rel_l2(x.grad.cpu().numpy(), y.grad.cpu().numpy()) <= 1e-6
    plan.close()
