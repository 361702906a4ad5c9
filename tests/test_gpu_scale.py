"""Full-size GPU cases: the uneven-window (3000x800, 96 shots), differentiation
(2000x600, 64 shots) and full-iteration (4000x1200, shot group of the 128)
configurations, run through the C ABI at their full grids, shot counts and
step counts.

The FP64 oracle cannot run these sizes, so each test compares what it can
compute one by one (the data of one shot over its first steps, on a window of
that shot that waves do not leave in that time, where the crop changes
nothing) and checks properties that hold at any size: the misfit equals
1/2 |d - d_obs|^2 of the returned data, the gradient of a component vanishes
outside its shot's window, reduced-precision checkpoints change neither the
data nor (beyond their error bound) the gradient, full snapshot storage and
sqrt(nt) checkpointing give identical results."""
import dataclasses
import time

import numpy as np
import pytest
import torch

import workloads as W
from common import rel_l2, rounded
from oracle import elastic as E

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def efwi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_14130_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.float32))).cuda()


def true_model(p):
    ns = p.acq.ns
    return [dev(np.broadcast_to(np.asarray(m, np.float32)[None], (ns,) + np.shape(m)))
            for m in (p.true_vp, p.true_vs, p.true_rho)]


def early_oracle_check(p, d_gpu, shot, x0, w, nsteps, own_window=False):
    """Data of shot `shot` (d_gpu: device [ntr, nt]) over its first nsteps against
    the oracle on the window [x0, x0 + w); unless that window is the shot's own
    (the GPU ran it on the same domain), asserts that the waves stay inside it
    meanwhile.  The compared traces must carry signal."""
    o = rounded(W.oracle_window(p, shot, x0, w))
    a = o.acq
    if not own_window:
        sx = a.src_xz[0, 0] / a.dx
        dist = min(sx - x0, x0 + w - 1 - sx) * a.dx
        vmax = float(np.max(o.vp[0]))
        assert vmax * nsteps * a.dt < 0.9 * dist, "window too narrow for the compared steps"
    short = dataclasses.replace(a, nt=nsteps, wavelet=np.asarray(a.wavelet)[:, :nsteps + 1])
    ref = E.forward(short, o.vp, o.vs, o.rho)
    idx = torch.as_tensor(np.asarray(o.meta["traces"]), device=d_gpu.device)
    got = d_gpu[idx, :nsteps].double().cpu().numpy()
    assert np.abs(ref).max() > 0 and ref.shape[0] >= 20
    err = rel_l2(got, ref)
    assert err <= TOL, err
    return err


def misfit_of(d, d_obs):
    r = d.double() - d_obs.double()
    return 0.5 * float(torch.sum(r * r))


def grad_outside_windows_is_zero(acq, gs):
    for s, (x0, w) in enumerate(acq.windows()):
        for g in gs:
            gs_ = g[s]
            assert torch.all(gs_[:, :x0] == 0) and torch.all(gs_[:, x0 + w:] == 0)
            assert torch.isfinite(gs_).all() and float(gs_.abs().max()) > 0


def test_uneven_windows_3000x800_full(efwi):
    """96 shots on windows 600-1800 cells wide, nt=4000, one persistent launch per
    step: FP32 and scaled-FP16 checkpoints; the narrowest shot's first 500 steps
    against the oracle on the same window."""
    p = W.uneven_windows_3000x800()
    acq = p.acq
    acq.wavelet = np.asarray(acq.wavelet, np.float32).astype(np.float64)
    m = [dev(v) for v in (p.vp, p.vs, p.rho)]
    out = {}
    for store in ("fp32", "fp16"):
        plan = efwi.Plan(acq, exec="batched", ckpt_store=store)
        if store == "fp32":
            d_obs = plan.forward(*true_model(p)).clone()
        t0 = time.perf_counter()
        phi, gvp, gvs, grho, d = plan.gradient(*m, d_obs, return_data=True)
        torch.cuda.synchronize()
        print(f"\n3000x800 x96 {store}: {time.perf_counter() - t0:.2f} s per gradient, "
              f"workspace {plan.info()['workspace_bytes'] / 1e9:.1f} GB")
        plan.sync_status()
        out[store] = (float(phi.item()), gvp.clone(), gvs.clone(), grho.clone(), d.clone())
        del gvp, gvs, grho, d
        plan.close()
    phi, gvp, gvs, grho, d = out["fp32"]
    assert phi == pytest.approx(misfit_of(d, d_obs), rel=1e-9)
    grad_outside_windows_is_zero(acq, (gvp, gvs, grho))
    assert torch.equal(out["fp16"][4], d)                 # data do not depend on the store
    for a, b in zip(out["fp16"][1:4], (gvp, gvs, grho)):
        assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 2e-3
    win = acq.windows()
    s = int(np.argmin(win[:, 1]))
    early_oracle_check(p, d, s, int(win[s, 0]), int(win[s, 1]), 500, own_window=True)


def test_differentiation_2000x600_full(efwi):
    """64 shots, nt=6000: sqrt(nt) checkpointing against full snapshot storage on a
    3-shot group (bitwise-identical data, misfit and gradients; workspace and
    time reported), then the 64-shot gradient with a sampled oracle check."""
    p = W.differentiation_2000x600()
    acq = p.acq
    acq.wavelet = np.asarray(acq.wavelet, np.float32).astype(np.float64)
    g3 = W.shot_subset(p, [30, 31, 32])
    m3 = [dev(v) for v in (g3.vp, g3.vs, g3.rho)]
    res = {}
    for name, K in (("sqrt", 0), ("full", acq.nt)):
        plan = efwi.Plan(g3.acq, exec="batched", ckpt_interval=K)
        d_obs3 = plan.forward(*true_model(g3)).clone()
        plan.gradient(*m3, d_obs3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = [t.clone() for t in plan.gradient(*m3, d_obs3, return_data=True)]
        torch.cuda.synchronize()
        info = plan.info()
        print(f"\n2000x600 x3 {name}: ckpt interval {info['ckpt_interval']}, "
              f"{time.perf_counter() - t0:.2f} s per gradient, workspace {info['workspace_bytes'] / 1e9:.1f} GB")
        res[name] = (out, info["workspace_bytes"])
        plan.sync_status()
        plan.close()
    # the data and the misfit come from the same forward pass; the gradients differ only
    # in the rounding of the imaging sums (sqrt(nt): FP32 partials per segment, Kahan-folded;
    # full storage: one segment)
    assert torch.equal(res["sqrt"][0][0], res["full"][0][0]) and torch.equal(res["sqrt"][0][4], res["full"][0][4])
    for a, b in zip(res["sqrt"][0][1:4], res["full"][0][1:4]):
        assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 1e-5
    assert res["full"][1] > 10 * res["sqrt"][1]

    m = [dev(v) for v in (p.vp, p.vs, p.rho)]
    plan = efwi.Plan(acq, exec="batched")
    d_obs = plan.forward(*true_model(p)).clone()
    t0 = time.perf_counter()
    phi, gvp, gvs, grho, d = plan.gradient(*m, d_obs, return_data=True)
    torch.cuda.synchronize()
    print(f"2000x600 x64 sqrt: {time.perf_counter() - t0:.2f} s per gradient, "
          f"workspace {plan.info()['workspace_bytes'] / 1e9:.1f} GB")
    plan.sync_status()
    plan.close()
    assert float(phi.item()) == pytest.approx(misfit_of(d, d_obs), rel=1e-9)
    for g in (gvp, gvs, grho):
        assert torch.isfinite(g).all() and float(g.abs().max()) > 0
    # the 3-shot group is a slice of the 64-shot batch: same shots, same results
    for a, b in zip(res["sqrt"][0][1:4], (gvp, gvs, grho)):
        assert torch.equal(a, b[30:33])
    s, x0, w = 32, 700, 600
    early_oracle_check(p, d, s, x0, w, 500)


def test_full_iteration_4000x1200_group(efwi):
    """One shot group (8 of the 128 sources, next to the fibre centre) of the
    4000x1200 full-iteration workload, nt=8000, FP16 checkpoints: observed data
    from the true model and the error-free sources, modelled with the seeded
    source errors.  Data-term gradient (sampled oracle check of one shot), the
    consistency-term gradient of all 128 components evaluated with the group's
    plan (sampled pixels against the oracle, phi_reg = 1/2 <g_reg, m~>), and an
    l-BFGS update at the group's full vector length (3 x 8 x 4.8 M) against the
    oracle's two-loop recursion."""
    from oracle import extension as X
    from oracle import lbfgs as L
    from paper_2305_14130_gb300.optim import LBFGS
    p = W.full_iteration_4000x1200()
    g = W.shot_subset(p, range(60, 68))
    g.acq.wavelet = np.asarray(g.acq.wavelet, np.float32).astype(np.float64)
    true_acq = dataclasses.replace(g.acq, mt=g.meta["true_mt"],
                                   wavelet=np.asarray(g.meta["true_wavelet"], np.float32).astype(np.float64))
    plan_true = efwi.Plan(true_acq, exec="batched", ckpt_store="fp16")
    d_obs = plan_true.forward(*true_model(g)).clone()
    plan_true.close()
    plan = efwi.Plan(g.acq, exec="batched", ckpt_store="fp16")
    m = [dev(v) for v in (g.vp, g.vs, g.rho)]
    t0 = time.perf_counter()
    phi, gvp, gvs, grho, d = plan.gradient(*m, d_obs, return_data=True)
    torch.cuda.synchronize()
    print(f"\n4000x1200 x8 fp16: {time.perf_counter() - t0:.2f} s per gradient, "
          f"workspace {plan.info()['workspace_bytes'] / 1e9:.1f} GB")
    phi0 = float(phi.item())
    assert phi0 == pytest.approx(misfit_of(d, d_obs), rel=1e-9) and phi0 > 0
    for gg in (gvp, gvs, grho):
        assert torch.isfinite(gg).all() and float(gg.abs().max()) > 0
    early_oracle_check(g, d, 4, 1700, 600, 500)
    del d

    # consistency term of all 128 components of the extended problem (1 % seeded noise per
    # component), evaluated with this group's plan on the full grid
    nsall, nz, nx = p.acq.ns, p.acq.nz, p.acq.nx
    gen = torch.Generator(device="cuda").manual_seed(5)
    base = dev(p.vp[0])
    mall = base[None] * (1 + 0.01 * torch.randn((nsall, nz, nx), device="cuda", generator=gen))
    b, bp, sink = efwi.zoi_weights(nsall, nx, nz, p.acq.dx, p.acq.dz, p.zoi)
    eta = 1e-3
    phi_r, g_r = plan.regularization_grad(mall, b, bp, sink, eta)
    phi_r = float(phi_r.item())
    half_dot = 0.5 * float(torch.sum(g_r.double() * mall.double()))
    assert phi_r > 0 and half_dot == pytest.approx(phi_r, rel=1e-4)
    rng = np.random.default_rng(5)
    src = np.rint(p.acq.src_xz / p.acq.dx).astype(int)
    pix = [(int(src[s, 1]) + dz, int(src[s, 0]) + dx) for s in range(0, nsall, 9) for dz in (-3, 0, 2)
           for dx in (-5, 0, 7)]
    pix += [(int(v), int(u)) for v, u in zip(rng.integers(0, nz, 40), rng.integers(0, nx, 40))]
    jj, ii = (torch.as_tensor(a, device="cuda") for a in np.array(pix).T)
    sub = lambda t, dt=np.float64: t[:, jj, ii].cpu().numpy().astype(dt)[:, None, :]
    _, g_ref = X.regularization(sub(mall), sub(b), sub(bp), sub(sink, np.uint8), eta)
    assert rel_l2(sub(g_r)[:, 0, :], g_ref[:, 0, :]) <= TOL
    del mall, b, bp, sink, g_r

    # l-BFGS update at the full vector length: a short steepest-descent step of the
    # data term (largest model change 0.05 m/s), the pair it gives, the new direction
    x = torch.cat([t.reshape(-1) for t in m])
    g0 = torch.cat([t.reshape(-1) for t in (gvp, gvs, grho)])
    del gvp, gvs, grho
    opt = LBFGS(x.numel(), m=5)
    d0 = opt.direction(g0)
    assert torch.equal(d0, -g0)
    a = 0.05 / float(d0.abs().max())
    x1 = x + a * d0
    shape = (3, g.acq.ns, nz, nx)
    xv = x1.view(shape)
    g1 = torch.empty_like(x)
    gv = g1.view(shape)
    phi1, *_ = plan.gradient(xv[0], xv[1], xv[2], d_obs, out=(gv[0], gv[1], gv[2]))
    phi1 = float(phi1.item())
    assert phi1 < phi0
    s_, y_ = x1 - x, g1 - g0
    accepted = opt.push(s_, y_)
    d1 = opt.direction(g1)
    assert float(torch.dot(g1.double(), d1.double())) < 0
    S = s_.double().cpu().numpy()[None] if accepted else np.zeros((0, x.numel()))
    Y = y_.double().cpu().numpy()[None] if accepted else np.zeros((0, x.numel()))
    ref = -L.two_loop(g1.double().cpu().numpy(), S, Y)
    assert rel_l2(d1.cpu().numpy(), ref) <= 1e-5
    print(f"l-BFGS at n = {x.numel()}: pair {'stored' if accepted else 'rejected'}, "
          f"phi {phi0:.6e} -> {phi1:.6e}")
    opt.close()
    plan.sync_status()
    plan.close()
