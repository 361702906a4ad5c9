"""Pins of the oracle's adjoint and gradient (eq. 6) to the forward map (no GPU).

* dot-product tests <L x, y> = <x, L^T y> to 1e-12 for the whole step map
  (all wavefields, CPML memory variables, DAS accumulators) and for the
  wavelet -> data map, in both DAS modes, for particle-velocity receivers and
  with a cropped window;
* central finite differences of the misfit against <g, dm> for Vp, Vs and
  rho separately;
* zero residual gives an exactly zero gradient.
"""
import numpy as np
import pytest

import workloads as W
from oracle import elastic as E


def _random_state(sh, rng):
    st = sh.zero_state()
    for k in ("vx", "vz", "sxx", "szz", "sxz"):
        st[k] = rng.standard_normal(st[k].shape)
    for k in range(8):
        st["psi"][k] = rng.standard_normal(st["psi"][k].shape)
    st["U"] = rng.standard_normal(st["U"].shape)
    return st


def _inner(a, b):
    s = sum(float(np.sum(a[k] * b[k])) for k in ("vx", "vz", "sxx", "szz", "sxz", "U"))
    return s + sum(float(np.sum(a["psi"][k] * b["psi"][k])) for k in range(8))


@pytest.mark.parametrize("mode", [W.STRAIN, W.STRAIN_RATE, W.VELOCITY])
@pytest.mark.parametrize("win", [None, [[3, 16], [5, 17]]])
def test_dot_product_state_map(mode, win):
    p = W.tiny(das_mode=mode, win=win)
    rng = np.random.default_rng(1)
    for s in range(p.acq.ns):
        sh = E.Shot(p.acq, s, p.vp[s], p.vs[s], p.rho[s])
        sh.wav = np.zeros_like(sh.wav)
        x0 = _random_state(sh, rng)
        d = sh.forward(x0)[0]
        y = rng.standard_normal(d.shape)
        _, adj, _ = sh.adjoint(y, st0=x0)
        lhs, rhs = float(np.sum(d * y)), _inner(x0, adj)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("mode,force", [(W.STRAIN, False), (W.STRAIN_RATE, False), (W.VELOCITY, False),
                                        (W.STRAIN, True)])
def test_dot_product_wavelet_map(mode, force):
    p = W.tiny(das_mode=mode)
    if force:
        p = W.with_forces(p)
    rng = np.random.default_rng(2)
    sh = E.Shot(p.acq, 1, p.vp[1], p.vs[1], p.rho[1])
    w = rng.standard_normal(sh.wav.shape)
    sh.wav = w
    d = sh.forward()[0]
    y = rng.standard_normal(d.shape)
    _, _, gw = sh.adjoint(y)
    lhs, rhs = float(np.sum(d * y)), float(np.sum(w * gw))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _fd_check(p, d_obs, rel_h=1e-6, tol=1e-6, seed=5):
    acq = p.acq
    phi, gvp, gvs, grho = E.gradient(acq, p.vp, p.vs, p.rho, d_obs)
    rng = np.random.default_rng(seed)
    for k, g in enumerate((gvp, gvs, grho)):
        ms = [p.vp, p.vs, p.rho]
        dm = rng.standard_normal(ms[k].shape)
        h = rel_h * np.abs(ms[k]).max()
        mp = list(ms); mp[k] = ms[k] + h * dm
        mm = list(ms); mm[k] = ms[k] - h * dm
        fd = (E.misfit(E.forward(acq, *mp), d_obs) - E.misfit(E.forward(acq, *mm), d_obs)) / (2 * h)
        an = float(np.sum(g * dm))
        assert abs(fd - an) <= tol * abs(an), (k, fd, an)


@pytest.mark.parametrize("mode", [W.STRAIN, W.STRAIN_RATE, W.VELOCITY])
def test_gradient_finite_difference_tiny(mode):
    p = W.tiny(das_mode=mode, win=[[0, 24], [2, 20]])
    ns = p.acq.ns
    d_obs = E.forward(p.acq, *(np.repeat(m[None], ns, 0) for m in (p.true_vp, p.true_vs, p.true_rho)))
    _fd_check(p, d_obs)


def test_gradient_finite_difference_force_sources():
    """Vector-force sources: the injected term dt b F w delta_h depends on the
    buoyancy, so the b part of the gradient carries an extra term."""
    p = W.with_forces(W.tiny(win=[[0, 24], [2, 20]]))
    ns = p.acq.ns
    d_obs = E.forward(p.acq, *(np.repeat(m[None], ns, 0) for m in (p.true_vp, p.true_vs, p.true_rho)))
    _fd_check(p, d_obs)


def test_gradient_finite_difference_128():
    """128x128 dx=2 m random-layered model, 4 shots, nt=600 (FP64 FD check).

    One random direction perturbs Vp, Vs and rho together (each parameter is
    checked on its own by the tiny-grid test above).
    """
    p = W.random_layered_128()
    acq, ns = p.acq, p.acq.ns
    d_obs = E.forward(acq, *(np.repeat(m[None], ns, 0) for m in (p.true_vp, p.true_vs, p.true_rho)))
    phi, *g = E.gradient(acq, p.vp, p.vs, p.rho, d_obs)
    rng = np.random.default_rng(7)
    ms = [p.vp, p.vs, p.rho]
    dm = [rng.standard_normal(m.shape) * np.abs(m).max() for m in ms]
    h = 1e-6
    fp = E.misfit(E.forward(acq, *(m + h * d for m, d in zip(ms, dm))), d_obs)
    fm = E.misfit(E.forward(acq, *(m - h * d for m, d in zip(ms, dm))), d_obs)
    fd = (fp - fm) / (2 * h)
    an = sum(float(np.sum(gk * d)) for gk, d in zip(g, dm))
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_zero_residual_gives_zero_gradient():
    p = W.tiny()
    d = E.forward(p.acq, p.vp, p.vs, p.rho)
    phi, gvp, gvs, grho = E.gradient(p.acq, p.vp, p.vs, p.rho, d)
    assert phi == 0.0
    assert not gvp.any() and not gvs.any() and not grho.any()


def test_gradient_zero_outside_window():
    p = W.tiny(win=[[4, 12], [9, 14]])
    rng = np.random.default_rng(4)
    d_obs = rng.standard_normal((p.acq.ntr, p.acq.nt)) * 1e-9
    _, gvp, gvs, grho = E.gradient(p.acq, p.vp, p.vs, p.rho, d_obs)
    for s, (x0, w) in enumerate(p.acq.windows()):
        for g in (gvp, gvs, grho):
            assert not g[s, :, :x0].any() and not g[s, :, x0 + w:].any()
            assert g[s, :, x0:x0 + w].any()


def test_summed_component_gradients_are_the_conventional_gradient():
    """With every component equal to one model m (conventional FWI, eq. 6), the
    extended objective's data term (eq. 8) is the conventional misfit of m, so
    sum_s g_s must be its gradient: checked by central finite differences of the
    conventional misfit along a perturbation of m shared by all shots, per
    parameter (windows make the shots see different parts of m)."""
    p = W.tiny(nx=26, nz=20, ns=3, nt=40, win=[[0, 26], [3, 18], [8, 16]])
    acq = p.acq
    ns = acq.ns
    d_obs = E.forward(acq, *(np.repeat(m[None], ns, 0) for m in (p.true_vp, p.true_vs, p.true_rho)))
    m0 = [np.asarray(v, np.float64) for v in (p.true_vp * 1.01, p.true_vs * 0.99, p.true_rho * 1.02)]
    ext = lambda ms: [np.repeat(m[None], ns, 0) for m in ms]
    _, *g = E.gradient(acq, *ext(m0), d_obs)
    rng = np.random.default_rng(11)
    for k in range(3):
        dm = rng.standard_normal(m0[k].shape)
        h = 1e-6 * np.abs(m0[k]).max()
        mp = list(m0); mp[k] = m0[k] + h * dm
        mm = list(m0); mm[k] = m0[k] - h * dm
        fd = (E.misfit(E.forward(acq, *ext(mp)), d_obs) - E.misfit(E.forward(acq, *ext(mm)), d_obs)) / (2 * h)
        an = float(np.sum(g[k].sum(axis=0) * dm))
        assert abs(fd - an) <= 1e-6 * abs(an), (k, fd, an)
