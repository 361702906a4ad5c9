"""GPU parity of the pseudo-Hessian (efwi_pseudo_hessian) against the FP64
oracle: the zero-lag auto-correlation of |v| summed over shots and its
clipped, scaled inverse, through the C ABI.  Acceptance: relative L2 <= 1e-4
(FP32 time stepping, Kahan-compensated FP32 accumulation over time,
FP64 sum over shots)."""
import numpy as np
import pytest
import torch

import workloads as W
from common import rel_l2, rounded
from oracle import hessian as PH

pytestmark = pytest.mark.gpu
TOL = 1e-4
EPS = 0.02


@pytest.fixture(scope="module")
def efwi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_14130_gb300 as m
    return m


def dev(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a, np.float32)), device="cuda")


CASES = {
    "windows": lambda: W.tiny(nx=48, nz=26, ns=3, nt=60, npml=4, win=[[0, 30], [9, 37], [20, 28]]),
    "force": lambda: W.with_forces(W.tiny(nx=41, nz=30, ns=3, nt=70, npml=5, win=[[0, 34], [5, 36], [11, 30]])),
    "full_width": lambda: W.tiny(nx=45, nz=33, ns=2, nt=50, npml=6),
}


@pytest.mark.parametrize("exec_", ["plain", "batched"])
@pytest.mark.parametrize("name", list(CASES))
def test_pseudo_hessian_matches_oracle(efwi, name, exec_):
    p = rounded(CASES[name]())
    H = PH.pseudo_hessian(p.acq, p.vp, p.vs, p.rho)
    Pinv = PH.inverse_pseudo_hessian(H, EPS)
    plan = efwi.Plan(p.acq, exec=exec_)
    h, hi = plan.pseudo_hessian(dev(p.vp), dev(p.vs), dev(p.rho), eps=EPS)
    plan.sync_status()
    plan.close()
    h, hi = h.cpu().numpy(), hi.cpu().numpy()
    assert rel_l2(h, H) <= TOL, rel_l2(h, H)
    assert rel_l2(hi, Pinv) <= TOL, rel_l2(hi, Pinv)
    win = p.acq.windows()
    covered = np.zeros(p.acq.nx, bool)
    for x0, w in win:
        covered[x0:x0 + w] = True
    assert np.all(h[:, ~covered] == 0.0)


def test_repeat_calls_and_gradient_in_between_are_bitwise_identical(efwi):
    """The compensated sum reuses the imaging workspace: a gradient call in
    between, and the replayed CUDA graph, leave the result unchanged."""
    p = rounded(CASES["windows"]())
    plan = efwi.Plan(p.acq, exec="batched")
    m = (dev(p.vp), dev(p.vs), dev(p.rho))
    a = [t.clone() for t in plan.pseudo_hessian(*m, eps=EPS)]
    plan.gradient(*m, torch.zeros((p.acq.ntr, p.acq.nt), device="cuda"))
    b = [t.clone() for t in plan.pseudo_hessian(*m, eps=EPS)]
    plan.sync_status()
    plan.close()
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_guided_wave_single_shot_full_grid(efwi):
    """One shot of the 1000x300 waveguide workload on its full grid, 120 steps."""
    import copy
    p = rounded(W.guided_wave_1000x300(ns=1, nt=120))
    acq = copy.deepcopy(p.acq)
    H = PH.pseudo_hessian(acq, p.vp, p.vs, p.rho)
    plan = efwi.Plan(acq, exec="batched")
    h, hi = plan.pseudo_hessian(dev(p.vp), dev(p.vs), dev(p.rho), eps=EPS)
    plan.sync_status()
    plan.close()
    h = h.cpu().numpy()
    assert rel_l2(h, H) <= TOL, rel_l2(h, H)
    assert rel_l2(hi.cpu().numpy(), PH.inverse_pseudo_hessian(H, EPS)) <= TOL


def test_guided_wave_32_shots_properties(efwi):
    """The 32-shot, 4000-step waveguide workload: h >= 0 and finite, the inverse
    lies in [eps, 1], equals eps at the maximum of h and 1 where h is clipped."""
    p = rounded(W.guided_wave_1000x300())
    plan = efwi.Plan(p.acq, exec="batched")
    h, hi = plan.pseudo_hessian(dev(p.vp), dev(p.vs), dev(p.rho), eps=EPS)
    plan.sync_status()
    plan.close()
    h, hi = h.double().cpu().numpy(), hi.double().cpu().numpy()
    assert np.all(np.isfinite(h)) and np.all(h >= 0.0) and h.max() > 0.0
    assert np.all((hi >= EPS * (1 - 1e-6)) & (hi <= 1.0))
    assert abs(hi.flat[np.argmax(h)] - EPS) <= 1e-6 * EPS
    assert np.all(hi[h <= EPS * h.max() * (1 - 1e-6)] == 1.0)
