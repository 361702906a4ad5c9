"""Reduced-precision forward-velocity snapshots (FP16 / BF16) on the GPU.

The adjoint's imaging condition (eq. 6) cross-correlates the adjoint wavefield
with the forward velocities v^{n+1/2} of every step, which the gradient keeps
either for every step (full storage) or for one checkpoint segment at a time.
With snap_store = fp16 / bf16 they are kept as RNE(v 2^k), s 2^k in
[2^14, 2^15) with s = max |v| of the step, field and shot; the time stepping,
the data and the misfit stay FP32 and do not change.

The gradient errors against the FP64 oracle are printed and bounded by
SNAP_BOUND, stated in the design notes next to the measured values.
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
# gradient rel-L2 against the oracle with reduced-precision snapshots: the unit roundoff
# u of the storage format (every stored element errs by <= u |x|; the imaging's strain
# rates are finite differences of the stored velocities, which cancel part of their
# magnitude: 0.2-0.55 u measured)
SNAP_BOUND = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


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


CASES = {
    "tiny_strain": lambda: W.tiny(nx=40, nz=30, ns=3, nt=80, npml=6),
    "tiny_windows": lambda: W.tiny(nx=48, nz=26, ns=3, nt=60, npml=4, win=[[0, 30], [9, 37], [20, 28]]),
    "tiny_force": lambda: W.with_forces(W.tiny(nx=41, nz=30, ns=3, nt=70, npml=5,
                                               win=[[0, 34], [5, 36], [11, 30]])),
    "random_layered_128": W.random_layered_128,
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    p = rounded(CASES[request.param]())
    d_obs = observed(p)
    return request.param, p, d_obs, E.gradient(p.acq, p.vp, p.vs, p.rho, d_obs), E.forward(p.acq, p.vp, p.vs,
                                                                                         p.rho)


@pytest.mark.parametrize("store", ["fp16", "bf16"])
@pytest.mark.parametrize("schedule", ["full", "sqrt"])
def test_snapshot_gradient_against_oracle(efwi, case, store, schedule):
    name, p, d_obs, (phi_o, gvp_o, gvs_o, grho_o), d_o = case
    K = p.acq.nt if schedule == "full" else 0
    plan = efwi.Plan(p.acq, exec="batched", ckpt_interval=K, snap_store=store)
    info = plan.info()
    assert info["snap_store"] == {"fp16": 1, "bf16": 2}[store]
    assert (info["ckpt_interval"] >= p.acq.nt) == (schedule == "full")
    phi, gvp, gvs, grho, d = plan.gradient(dev(p.vp), dev(p.vs), dev(p.rho), dev(d_obs), return_data=True)
    plan.sync_status()
    errs = {"d": rel_l2(d.cpu().numpy(), d_o), "phi": abs(phi.item() - phi_o) / phi_o}
    for k, g, go in (("g_vp", gvp, gvp_o), ("g_vs", gvs, gvs_o), ("g_rho", grho, grho_o)):
        errs[k] = rel_l2(g.cpu().numpy(), go)
    print(f"{name}, {store} snapshots, {schedule} storage, errors vs FP64 oracle: "
          + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert errs["d"] <= TOL and errs["phi"] <= TOL        # the forward pass is FP32 as before
    for k in ("g_vp", "g_vs", "g_rho"):
        assert 0 < errs[k] <= SNAP_BOUND[store], k
    plan.close()


@pytest.mark.parametrize("store", ["fp16", "bf16"])
def test_snapshot_schedules_agree(efwi, store):
    """With FP32 checkpoints the recompute reproduces the forward pass bit for bit,
    so every schedule stores the same snapshots: the gradients differ only by the
    grouping of the Kahan-folded segment sums."""
    p = rounded(W.tiny(nx=40, nz=30, ns=2, nt=90, npml=6))
    d_obs = observed(p)
    args = (dev(p.vp), dev(p.vs), dev(p.rho), dev(d_obs))
    outs = []
    for K in (p.acq.nt, 0, 7, 1):
        plan = efwi.Plan(p.acq, exec="batched", ckpt_interval=K, snap_store=store)
        outs.append([t.clone() for t in plan.gradient(*args)])
        plan.close()
    for o in outs[1:]:
        assert torch.equal(outs[0][0], o[0])
        for a, b in zip(outs[0][1:], o[1:]):
            assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) <= 1e-6


SHAPES = [(32, 8), (32, 16), (64, 8)]
# every forward variant compiled with the snapshot work (the others are not candidates then)
VARIANTS = [("loads", s) for s in SHAPES] + [(k, (32, 16)) for k in ("tma", "tma_pairs", "tma_staged")] + \
    [("tma_pairs:split", (32, 16)), ("tma_staged:split", (32, 16)), ("tma_pairs", (32, 8))]


@pytest.mark.parametrize("store", ["fp16", "bf16"])
def test_snapshot_forward_variants_are_bitwise_identical(efwi, store, monkeypatch):
    """Every forward variant writes the same 2-byte snapshots with the same scales
    (uneven windows, ragged tiles): the gradients are bit for bit the same."""
    p = rounded(W.tiny(nx=70, nz=41, ns=3, nt=40, npml=5, win=[[0, 45], [13, 57], [30, 40]]))
    d_obs = observed(p)
    args = (dev(p.vp), dev(p.vs), dev(p.rho), dev(d_obs))
    ref = None
    monkeypatch.setenv("EFWI_ADJ_PERSIST", "0")
    for stencil, (tx, tz) in VARIANTS:
        stencil, _, layout = stencil.partition(":")
        if layout == "split":
            monkeypatch.setenv("EFWI_TMA_VEC", "3")
        else:
            monkeypatch.delenv("EFWI_TMA_VEC", raising=False)
        plan = efwi.Plan(p.acq, exec="batched", tile=(tx, tz), stencil=stencil, adj_tile=(32, 16),
                         adj_stencil="loads", ckpt_interval=p.acq.nt, snap_store=store)
        info = plan.info()
        assert (info["tile_x"], info["tile_z"]) == (tx, tz)
        assert info["stencil"] == {"loads": 1, "tma": 2, "tma_pairs": 3, "tma_staged": 4}[stencil]
        out = [t.clone() for t in plan.gradient(*args, return_data=True)]
        plan.sync_status()
        plan.close()
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref, out):
                assert torch.equal(a, b), (stencil, layout, tx, tz)


@pytest.mark.parametrize("store", ["fp16", "bf16"])
@pytest.mark.parametrize("ckpt", ["full", "segments"])
def test_snapshot_adjoint_variants_are_bitwise_identical(efwi, store, ckpt, monkeypatch):
    """The scaled-stress adjoint reads the 2-byte snapshots with per-thread loads or
    through TMA copies (one cell or a cell pair per thread), every step stored or
    recomputed per segment: the gradients are bit for bit the same."""
    p = rounded(W.tiny(nx=70, nz=41, ns=3, nt=40, npml=5, win=[[0, 45], [13, 57], [30, 40]]))
    d_obs = observed(p)
    args = (dev(p.vp), dev(p.vs), dev(p.rho), dev(d_obs))
    ref = None
    K = p.acq.nt if ckpt == "full" else 7
    for adj_stencil, vec in (("loads", None), ("tma", "1"), ("tma", "2"), ("tma", "3")):
        if vec:
            monkeypatch.setenv("EFWI_ADJ_VEC", vec)
        plan = efwi.Plan(p.acq, exec="batched", tile=(32, 16), stencil="tma_pairs", adj_tile=(32, 16),
                         adj_stencil=adj_stencil, ckpt_interval=K, snap_store=store)
        info = plan.info()
        assert info["adj_form"] == 2 and info["adj_stencil"] == {"loads": 1, "tma": 2}[adj_stencil]
        assert info["adj_layout"] == (int(vec) if vec else 0)
        out = [t.clone() for t in plan.gradient(*args, return_data=True)]
        plan.sync_status()
        plan.close()
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref, out):
                assert torch.equal(a, b), (adj_stencil, vec)


def test_auto_schedule_and_replays(efwi):
    """ckpt_interval="auto" stores every step of a small problem; repeated calls
    (graph replays) are bitwise identical; the plan reports what it chose."""
    p = rounded(W.tiny(nx=40, nz=30, ns=2, nt=50, npml=6))
    d_obs = observed(p)
    args = (dev(p.vp), dev(p.vs), dev(p.rho), dev(d_obs))
    plan = efwi.Plan(p.acq, exec="batched", ckpt_interval="auto", snap_store="fp16")
    info = plan.info()
    assert info["ckpt_interval"] == p.acq.nt and info["n_ckpt"] == 1 and info["snap_store"] == 1
    a = [t.clone() for t in plan.gradient(*args)]
    b = [t.clone() for t in plan.gradient(*args)]
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    plan.close()


def test_snapshot_rejections(efwi):
    p = rounded(W.tiny(nx=24, nz=20, ns=1, nt=10, npml=3))
    with pytest.raises(efwi.EfwiError):
        efwi.Plan(p.acq, exec="plain", snap_store="fp16")
    with pytest.raises(efwi.EfwiError):
        efwi.Plan(p.acq, exec="batched", snap_store="fp16", overlap="on")


def test_guided_wave_full_storage_fp16_matches_fp32_sampled(efwi):
    """1000x300 grid, 32 shots, 400 steps: FP16 snapshots of every step against FP32
    snapshots on the same grid (same data and misfit; gradient close)."""
    p = rounded(W.guided_wave_1000x300())
    acq = copy.deepcopy(p.acq)
    acq.nt = 400
    acq.wavelet = acq.wavelet[:, :401]
    m = (dev(p.vp), dev(p.vs), dev(p.rho))
    ns = acq.ns
    obs = efwi.Plan(acq, exec="batched")
    tv = lambda x: dev(np.repeat(np.asarray(x)[None], ns, 0))
    d_obs = obs.forward(tv(p.true_vp), tv(p.true_vs), tv(p.true_rho))
    outs = {}
    for store, K in (("fp32", 0), ("fp16", acq.nt), ("bf16", acq.nt)):
        plan = efwi.Plan(acq, exec="batched", ckpt_interval=K, snap_store=store)
        outs[store] = [t.clone() for t in plan.gradient(*m, d_obs, return_data=True)]
        plan.sync_status()
        plan.close()
    obs.close()
    for store in ("fp16", "bf16"):
        assert torch.equal(outs[store][4], outs["fp32"][4])       # data
        assert outs[store][0].item() == outs["fp32"][0].item()    # misfit
        errs = [rel_l2(outs[store][k].cpu().numpy(), outs["fp32"][k].cpu().numpy()) for k in (1, 2, 3)]
        print(f"guided wave 1000x300x32, 400 steps, {store} vs FP32 snapshots: {errs}")
        assert max(errs) <= SNAP_BOUND[store]
