"""Gradient schedules between sqrt(nt) checkpointing and full storage.

With ``stored_steps`` the forward pass keeps the velocities of the final steps
itself; the adjoint reads those and recomputes only the segments before them
from their checkpoints.  With FP32 checkpoints a recompute reproduces the
forward pass bit for bit and the imaging sums are folded at the same segment
ends, so every such schedule must give the sqrt(nt) schedule's results bit for
bit (eq. 6 sums the same products in the same order).  With reduced-precision
checkpoints the stored steps are more accurate than recomputed ones; the
result is checked against the FP64 oracle instead.
"""
import copy

import numpy as np
import pytest
import torch

import workloads as W
from common import f32, rel_l2, rounded
from oracle import elastic as E

pytestmark = pytest.mark.gpu
TOL = 1e-4
CKPT_BOUND = {"fp16": 2.0 ** -12, "bf16": 2.0 ** -9}


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


def effective(nt, K, S):
    """Stored steps a plan keeps for a request of S: the recomputed steps are rounded
    up to whole K-step segments."""
    if S <= 0:
        return 0
    split = min(nt, -(-max(0, nt - S) // K) * K)
    return nt - split


@pytest.fixture(scope="module")
def windows():
    p = rounded(W.tiny(nx=48, nz=26, ns=3, nt=90, npml=4, win=[[0, 30], [9, 37], [20, 28]]))
    return p, observed(p)


@pytest.mark.parametrize("exec_,snap", [("batched", "fp32"), ("batched", "fp16"), ("plain", "fp32")])
def test_stored_steps_equal_the_sqrt_schedule(efwi, windows, exec_, snap):
    p, d_obs = windows
    nt, K = p.acq.nt, 7
    args = (dev(p.vp), dev(p.vs), dev(p.rho), dev(d_obs))
    plan = efwi.Plan(p.acq, exec=exec_, ckpt_interval=K, snap_store=snap)
    ref = [t.clone() for t in plan.gradient(*args, return_data=True)]
    assert plan.info()["stored_steps"] == 0
    plan.close()
    for S in (1, 6, 7, 20, 45, 84, 85):
        plan = efwi.Plan(p.acq, exec=exec_, ckpt_interval=K, snap_store=snap, stored_steps=S)
        info = plan.info()
        want = effective(nt, K, S)
        assert info["stored_steps"] == want, S
        assert info["ckpt_interval"] == K and info["n_ckpt"] == (nt - want + K - 1) // K
        out = [t.clone() for t in plan.gradient(*args, return_data=True)]
        again = [t.clone() for t in plan.gradient(*args, return_data=True)]    # graph replay
        plan.sync_status()
        plan.close()
        for a, b, c in zip(ref, out, again):
            assert torch.equal(a, b), S
            assert torch.equal(b, c), S


def test_every_step_requested_is_full_storage(efwi, windows):
    """stored_steps >= nt - (nt mod K) leaves no segment to recompute: the plan runs the
    full-storage schedule (its Kahan folds group the sums differently)."""
    p, d_obs = windows
    nt, K = p.acq.nt, 7
    args = (dev(p.vp), dev(p.vs), dev(p.rho), dev(d_obs))
    outs = []
    for kw in (dict(ckpt_interval=K), dict(ckpt_interval=K, stored_steps=nt), dict(ckpt_interval=nt)):
        plan = efwi.Plan(p.acq, exec="batched", **kw)
        if "stored_steps" in kw or kw["ckpt_interval"] == nt:
            info = plan.info()
            assert info["ckpt_interval"] == nt and info["stored_steps"] == nt and info["n_ckpt"] == 1
        outs.append([t.clone() for t in plan.gradient(*args)])
        plan.close()
    for a, b in zip(outs[1], outs[2]):
        assert torch.equal(a, b)
    assert torch.equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1:], outs[1][1:]):
        assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("ckpt", ["fp16", "bf16"])
def test_stored_steps_with_reduced_checkpoints_against_oracle(efwi, windows, ckpt):
    p, d_obs = windows
    phi_o, gvp_o, gvs_o, grho_o = E.gradient(p.acq, p.vp, p.vs, p.rho, d_obs)
    args = (dev(p.vp), dev(p.vs), dev(p.rho), dev(d_obs))
    errs = {}
    for S in (0, 42):
        plan = efwi.Plan(p.acq, exec="batched", ckpt_interval=9, ckpt_store=ckpt, stored_steps=S)
        phi, gvp, gvs, grho = plan.gradient(*args)
        plan.sync_status()
        plan.close()
        e = [rel_l2(g.cpu().numpy(), go) for g, go in ((gvp, gvp_o), (gvs, gvs_o), (grho, grho_o))]
        errs[S] = e
        print(f"{ckpt} checkpoints, stored_steps {S}: g errors vs FP64 oracle {['%.2e' % x for x in e]}")
        assert abs(phi.item() - phi_o) / phi_o <= TOL
        assert max(e) <= CKPT_BOUND[ckpt]


def test_stored_steps_skip_the_overlapped_schedule(efwi, windows):
    p, _ = windows
    plan = efwi.Plan(p.acq, exec="batched", ckpt_interval=7, stored_steps=30, overlap="auto")
    info = plan.info()
    assert info["overlap_fwd_blocks"] == 0 and info["stored_steps"] == effective(p.acq.nt, 7, 30)
    plan.close()
    with pytest.raises(efwi.EfwiError):
        efwi.Plan(p.acq, exec="batched", ckpt_interval=7, stored_steps=30, overlap="on")


def test_guided_wave_stored_steps_bitwise(efwi):
    """1000x300 grid, 32 shots, 400 steps, the bench's kernels: half the steps kept by
    the forward pass give the sqrt(nt) schedule's gradient bit for bit."""
    p = rounded(W.guided_wave_1000x300())
    acq = copy.deepcopy(p.acq)
    acq.nt = 400
    acq.wavelet = acq.wavelet[:, :401]
    m = (dev(p.vp), dev(p.vs), dev(p.rho))
    ns = acq.ns
    tv = lambda x: dev(np.repeat(np.asarray(x)[None], ns, 0))
    obs = efwi.Plan(acq, exec="batched")
    d_obs = obs.forward(tv(p.true_vp), tv(p.true_vs), tv(p.true_rho)).clone()
    obs.close()
    outs = []
    for S in (0, 200):
        plan = efwi.Plan(acq, exec="batched", ckpt_interval=20, stored_steps=S)
        assert plan.info()["stored_steps"] == S
        outs.append([t.clone() for t in plan.gradient(*m, d_obs, return_data=True)])
        plan.sync_status()
        plan.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_guided_wave_full_size_auto_schedule_equals_sqrt(efwi):
    """The bench's workload and launch configuration at full size (1000x300, 32 shots,
    4000 steps, ckpt_interval = auto, which keeps the final steps that fit the device):
    the gradient equals the sqrt(nt) schedule's bit for bit, and the schedule keeps
    most of the steps (the rest of HBM holds their velocities)."""
    p = rounded(W.guided_wave_1000x300())
    acq = p.acq
    m = (dev(p.vp), dev(p.vs), dev(p.rho))
    ns = acq.ns
    tv = lambda x: dev(np.repeat(np.asarray(x)[None], ns, 0))
    outs, infos = [], []
    d_obs = None
    for ck in (0, "auto"):
        plan = efwi.Plan(acq, exec="batched", ckpt_interval=ck)
        if d_obs is None:
            d_obs = plan.forward(tv(p.true_vp), tv(p.true_vs), tv(p.true_rho)).clone()
        outs.append([t.clone() for t in plan.gradient(*m, d_obs, return_data=True)])
        infos.append(plan.info())
        plan.sync_status()
        plan.close()
        torch.cuda.empty_cache()
    assert infos[0]["stored_steps"] == 0
    K = infos[1]["ckpt_interval"]
    assert K < acq.nt and infos[1]["stored_steps"] >= acq.nt // 2
    assert (acq.nt - infos[1]["stored_steps"]) % K == 0
    for a, b in zip(*outs):
        assert torch.equal(a, b)
