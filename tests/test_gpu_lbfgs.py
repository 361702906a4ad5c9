"""GPU tests of the device l-BFGS (C-ABI efwi_lbfgs_*) against the optimizer
oracle: two-loop directions, whole iterations (line-search steps, objective
values, iterates) on a quadratic, and an inversion of a tiny extended-FWI
problem through the library's own gradient and regularization."""
import numpy as np
import pytest
import torch

import workloads as W
from common import rel_l2, rounded
from oracle import extension as X
from oracle import lbfgs as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def efwi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_14130_gb300 as m
    return m


def _spd_pairs(n, k, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 5.0, n)
    S = rng.standard_normal((k, n)).astype(np.float32)
    Y = (S * a + 0.01 * rng.standard_normal((k, n))).astype(np.float32)
    return S, Y


@pytest.mark.parametrize("n,k", [(1, 0), (7, 2), (300_001, 5), (300_001, 8)])
def test_direction_matches_two_loop(efwi, n, k):
    """k pairs pushed into a handle keeping m = 5: the direction uses the
    newest min(k, 5); FP32 vectors, FP64 inner products."""
    from paper_2305_14130_gb300.optim import LBFGS
    S, Y = _spd_pairs(n, k, 3)
    g = np.random.default_rng(4).standard_normal(n).astype(np.float32)
    opt = LBFGS(n, m=5)
    for s, y in zip(S, Y):
        assert opt.push(torch.tensor(s, device="cuda"), torch.tensor(y, device="cuda"))
    d = opt.direction(torch.tensor(g, device="cuda")).cpu().numpy()
    ref = -L.two_loop(g.astype(np.float64), S[-5:].astype(np.float64), Y[-5:].astype(np.float64))
    if k == 0:
        assert np.array_equal(d, -g)
    else:
        assert rel_l2(d, ref) <= 1e-5
    opt.close()


def test_rejected_pair_keeps_the_history(efwi):
    from paper_2305_14130_gb300.optim import LBFGS
    n = 1000
    S, Y = _spd_pairs(n, 5, 5)
    g = torch.tensor(np.random.default_rng(6).standard_normal(n).astype(np.float32), device="cuda")
    opt = LBFGS(n, m=5)
    for s, y in zip(S, Y):
        opt.push(torch.tensor(s, device="cuda"), torch.tensor(y, device="cuda"))
    d0 = opt.direction(g).clone()
    s = torch.tensor(S[0], device="cuda")
    assert not opt.push(s, -s)              # s^T y < 0: not stored, nothing overwritten
    assert torch.equal(opt.direction(g), d0)
    opt.close()


def _quadratic(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 50.0, n).astype(np.float32)
    c = rng.standard_normal(n).astype(np.float32)
    return a, c


def test_iterations_match_oracle_on_a_quadratic(efwi):
    """phi(x) = 1/2 sum a_i (x_i - c_i)^2 + 1 evaluated on the device (FP64 sum);
    eight iterations: accepted steps, objective values and iterates agree with
    the FP64 oracle running the same algorithm."""
    from paper_2305_14130_gb300.optim import LBFGS
    n = 200_003
    a, c = _quadratic(n, 7)
    at, ct = torch.tensor(a, device="cuda"), torch.tensor(c, device="cuda")

    def obj(x, g):
        r = x - ct
        g.copy_(at * r)
        return 0.5 * float(torch.sum(at.double() * r.double() * r.double())) + 1.0

    def f(x):
        r = x - c.astype(np.float64)
        return 0.5 * float(np.sum(a * r * r)) + 1.0, a * r

    iters = 8
    ref = L.lbfgs(f, np.zeros(n), iters=iters, m=5)
    opt = LBFGS(n, m=5)
    x = torch.zeros(n, device="cuda")
    g = torch.empty(n, device="cuda")
    phi = obj(x, g)
    for k in range(iters):
        phi, info = opt.iterate(x, phi, g, obj)
        assert not info["ls_failed"]
        assert info["alpha"] == pytest.approx(ref[k]["alpha"], rel=1e-4)
        assert phi == pytest.approx(ref[k]["phi"], rel=1e-5)
        assert info["rate"] == pytest.approx(ref[k]["rate"], rel=1e-3, abs=1e-7)
        assert info["evals"] == ref[k]["evals"]
    assert rel_l2(x.cpu().numpy(), ref[-1]["x"]) <= 1e-4
    opt.close()


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_search_backs_off_from_non_finite_trials(efwi, bad):
    """phi(x) = (x_0 - 1)^2 + 1 + 1/2 |x_1..|^2, not finite for x_0 >= 3 (as an unstable
    simulation gives); the first trial moves x by 8 along d = -g and lands there.
    The device iteration takes the oracle's trial points and accepted step."""
    from paper_2305_14130_gb300.optim import LBFGS
    n = 5
    trials = []

    def obj(x, g):
        xv = x.double().cpu().numpy()
        trials.append(float(xv[0]))
        if xv[0] >= 3.0:
            g.fill_(bad)
            return bad
        gv = xv.copy()
        gv[0] = 2.0 * (xv[0] - 1.0)
        g.copy_(torch.tensor(gv, dtype=torch.float32))
        return float((xv[0] - 1.0) ** 2 + 1.0 + 0.5 * np.sum(xv[1:] ** 2))

    ref_trials = []

    def f(x):
        ref_trials.append(float(x[0]))
        if x[0] >= 3.0:
            return bad, np.full(n, bad)
        gv = x.copy()
        gv[0] = 2.0 * (x[0] - 1.0)
        return float((x[0] - 1.0) ** 2 + 1.0 + 0.5 * np.sum(x[1:] ** 2)), gv

    x0 = np.zeros(n)
    phi0, g0 = f(x0)
    d = -g0
    a_ref, phi_ref, _, evals_ref = L.wolfe_search(f, x0, phi0, g0, d, 8.0 / np.linalg.norm(d))
    opt = LBFGS(n, m=5)
    opt.set_step0(8.0)
    x = torch.zeros(n, device="cuda")
    g = torch.empty(n, device="cuda")
    phi = obj(x, g)
    phi, info = opt.iterate(x, phi, g, obj)
    assert not info["ls_failed"] and info["evals"] == evals_ref
    assert trials[1:] == pytest.approx(ref_trials[1:], rel=1e-6)
    assert trials[1] >= 3.0 and phi == pytest.approx(phi_ref, rel=1e-6)
    assert info["alpha"] == pytest.approx(a_ref, rel=1e-6)
    opt.close()


def test_run_stops_on_the_eq13_rate(efwi):
    from paper_2305_14130_gb300.optim import LBFGS
    n = 4096
    a, c = _quadratic(n, 8)
    at, ct = torch.tensor(a, device="cuda"), torch.tensor(c, device="cuda")

    def obj(x, g):
        r = x - ct
        g.copy_(at * r)
        return 0.5 * float(torch.sum(at.double() * r.double() * r.double())) + 1.0

    opt = LBFGS(n, m=5)
    x = torch.zeros(n, device="cuda")
    g, info = opt.run(x, obj, max_iter=200, min_rate=1e-3)
    assert info["stop"] in ("rate", "no_step")
    assert info["iters"] < 200
    if info["stop"] == "rate":
        assert 0 <= info["rate"] < 1e-3
    assert info["phi"] == pytest.approx(obj(x, torch.empty_like(x)), rel=1e-6)
    assert info["phi"] < 1.0 + 1e-2 * (obj(torch.zeros_like(x), torch.empty_like(x)) - 1.0)
    opt.close()


def test_objective_errors_propagate(efwi):
    from paper_2305_14130_gb300.optim import LBFGS
    opt = LBFGS(16)
    x = torch.zeros(16, device="cuda")
    g = torch.ones(16, device="cuda")

    def bad(x, g):
        raise RuntimeError("objective failed")
    with pytest.raises(RuntimeError, match="objective failed"):
        opt.iterate(x, 1.0, g, bad)
    opt.close()


def test_extended_fwi_inversion_decreases_the_objective(efwi):
    """A few l-BFGS iterations of the extended objective (eq. 8) on a tiny
    problem, through plan.gradient and plan.regularization_grad: the objective
    decreases every iteration and each rate is eq. 13 of consecutive values."""
    from paper_2305_14130_gb300.optim import LBFGS, extended_fwi_objective
    p = rounded(W.tiny(nx=40, nz=30, ns=3, nt=60, npml=6))
    acq = p.acq
    plan = efwi.Plan(acq, exec="batched")
    dev = lambda v, dt=np.float32: torch.tensor(np.asarray(v, dt), device="cuda")
    true = [np.broadcast_to(v, p.vp.shape).copy() for v in (p.true_vp, p.true_vs, p.true_rho)]
    d_obs = plan.forward(*[dev(v) for v in true]).clone()
    bo, bpo, sinko = X.zoi_weights(p.zoi, acq.nx, acq.nz, acq.dx, acq.dz)
    obj = extended_fwi_objective(plan, d_obs, dev(bo), dev(bpo), dev(sinko, np.uint8), (1e-3, 1e-3, 1e-3))
    x = torch.cat([dev(v).reshape(-1) for v in (p.vp, p.vs, p.rho)])
    g = torch.empty_like(x)
    opt = LBFGS(x.numel(), m=5)
    phi = obj(x, g)
    phis = [phi]
    for _ in range(4):
        phi, info = opt.iterate(x, phi, g, obj)
        if info["ls_failed"]:
            break
        assert phi < phis[-1]
        assert info["rate"] == pytest.approx((phis[-1] - phi) / phis[-1], rel=1e-12)
        phis.append(phi)
    assert len(phis) >= 3
    opt.close()
    plan.close()


@pytest.mark.parametrize("n,k", [(7, 0), (300_001, 0), (300_001, 5)])
def test_direction_with_diagonal_guess_matches_two_loop(efwi, n, k):
    """H_0 = gamma D (D without pairs) set through efwi_lbfgs_set_h0."""
    from paper_2305_14130_gb300.optim import LBFGS
    S, Y = _spd_pairs(n, k, 21)
    D = np.random.default_rng(22).uniform(0.05, 4.0, n).astype(np.float32)
    g = np.random.default_rng(23).standard_normal(n).astype(np.float32)
    opt = LBFGS(n, m=5)
    opt.set_h0(torch.tensor(D, device="cuda"))
    for s, y in zip(S, Y):
        assert opt.push(torch.tensor(s, device="cuda"), torch.tensor(y, device="cuda"))
    d = opt.direction(torch.tensor(g, device="cuda")).cpu().numpy()
    ref = -L.two_loop(g.astype(np.float64), S.astype(np.float64), Y.astype(np.float64), D.astype(np.float64))
    assert rel_l2(d, ref) <= (1e-7 if k == 0 else 1e-5)
    opt.set_h0(None)                          # back to gamma I (pairs forgotten): d = -g
    assert np.array_equal(opt.direction(torch.tensor(g, device="cuda")).cpu().numpy(), -g)
    opt.close()


def test_iterations_with_diagonal_guess_match_oracle(efwi):
    """The quadratic of the test above with D = 1/a (its exact inverse Hessian,
    the role the inverse pseudo-Hessian plays for the wave-equation problem):
    steps, objective values and evaluation counts agree with the oracle."""
    from paper_2305_14130_gb300.optim import LBFGS
    n = 200_003
    a, c = _quadratic(n, 9)
    D = (1.0 / a).astype(np.float32)
    at, ct = torch.tensor(a, device="cuda"), torch.tensor(c, device="cuda")

    def obj(x, g):
        r = x - ct
        g.copy_(at * r)
        return 0.5 * float(torch.sum(at.double() * r.double() * r.double())) + 1.0

    def f(x):
        r = x - c.astype(np.float64)
        return 0.5 * float(np.sum(a * r * r)) + 1.0, a * r

    iters = 2                                 # a doubling search along the Newton direction, then the exact step
    ref = L.lbfgs(f, np.zeros(n), iters=iters, m=5, D=D.astype(np.float64))
    opt = LBFGS(n, m=5)
    opt.set_h0(torch.tensor(D, device="cuda"))
    x = torch.zeros(n, device="cuda")
    g = torch.empty(n, device="cuda")
    phi = obj(x, g)
    for k in range(iters):
        if ref[k]["alpha"] is None:
            break
        phi, info = opt.iterate(x, phi, g, obj)
        assert not info["ls_failed"]
        assert info["alpha"] == pytest.approx(ref[k]["alpha"], rel=1e-4)
        assert phi == pytest.approx(ref[k]["phi"], rel=1e-5)
        assert info["evals"] == ref[k]["evals"]
    opt.close()


def test_pseudo_hessian_preconditioned_inversion_decreases_the_objective(efwi):
    """The paper's first comparison method on a tiny problem: l-BFGS with the
    clipped, scaled inverse pseudo-Hessian as initial inverse Hessian, on the
    extended objective (eq. 8); every iteration lowers it, eq. 13 rates."""
    from paper_2305_14130_gb300.optim import LBFGS, extended_fwi_objective, pseudo_hessian_h0
    p = rounded(W.tiny(nx=40, nz=30, ns=3, nt=60, npml=6))
    acq = p.acq
    plan = efwi.Plan(acq, exec="batched")
    dev = lambda v, dt=np.float32: torch.tensor(np.asarray(v, dt), device="cuda")
    true = [np.broadcast_to(v, p.vp.shape).copy() for v in (p.true_vp, p.true_vs, p.true_rho)]
    d_obs = plan.forward(*[dev(v) for v in true]).clone()
    bo, bpo, sinko = X.zoi_weights(p.zoi, acq.nx, acq.nz, acq.dx, acq.dz)
    obj = extended_fwi_objective(plan, d_obs, dev(bo), dev(bpo), dev(sinko, np.uint8), (1e-3, 1e-3, 1e-3))
    x = torch.cat([dev(v).reshape(-1) for v in (p.vp, p.vs, p.rho)])
    D = pseudo_hessian_h0(plan, x, eps=0.05)
    assert D.shape == x.shape and float(D.min()) >= 0.05 * (1 - 1e-6) and float(D.max()) == 1.0
    g = torch.empty_like(x)
    opt = LBFGS(x.numel(), m=5)
    opt.set_h0(D)
    phi = obj(x, g)
    phis = [phi]
    for _ in range(4):
        phi, info = opt.iterate(x, phi, g, obj)
        if info["ls_failed"]:
            break
        assert phi < phis[-1]
        assert info["rate"] == pytest.approx((phis[-1] - phi) / phis[-1], rel=1e-12)
        phis.append(phi)
    assert len(phis) >= 3
    opt.close()
    plan.close()


def test_history_saved_and_restored_bit_for_bit(efwi):
    """Resuming an inversion: the history saved by state() (the newest m pairs,
    oldest first) and restored into a new handle with the same diagonal H_0 gives
    bit-identical directions; an empty history restores to steepest descent."""
    from paper_2305_14130_gb300.optim import LBFGS
    n = 100_003
    S, Y = _spd_pairs(n, 7, 31)
    D = torch.tensor(np.random.default_rng(32).uniform(0.2, 3.0, n).astype(np.float32), device="cuda")
    g = torch.tensor(np.random.default_rng(33).standard_normal(n).astype(np.float32), device="cuda")
    opt = LBFGS(n, m=5)
    opt.set_h0(D)
    for s, y in zip(S, Y):
        assert opt.push(torch.tensor(s, device="cuda"), torch.tensor(y, device="cuda"))
    d0 = opt.direction(g).clone()
    Ss, Ys = opt.state()
    assert Ss.shape == (5, n)
    assert np.array_equal(Ss.cpu().numpy(), S[-5:]) and np.array_equal(Ys.cpu().numpy(), Y[-5:])
    opt2 = LBFGS(n, m=5)
    opt2.set_h0(D)
    opt2.load_state(Ss, Ys)
    assert torch.equal(opt2.direction(g), d0)
    opt3 = LBFGS(n, m=5)
    opt3.load_state(*LBFGS(n, m=5).state())
    assert torch.equal(opt3.direction(g), -g)
    for o in (opt, opt2, opt3):
        o.close()
