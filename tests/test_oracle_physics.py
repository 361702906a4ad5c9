"""Pins of the oracle's forward propagator to physics (no GPU).

* closed-form 2D Green's function of an explosion (eq. 2, moment tensor),
  for particle velocity and for the DAS gauge strain (eq. 3);
* second-order convergence when dx and dt halve;
* force/velocity reciprocity;
* CPML reflections against a 3x larger domain;
* exact linearity in the moment tensor and the source time function;
* DAS strain is the running time integral of DAS strain rate.
"""
import numpy as np

import workloads as W
from oracle import elastic as E
from greens2d import explosion_ux, explosion_vx


def _homog_acq(n, dx, dt, nt, src, f0, vp=3000.0, vs=1732.0, rho=2000.0, ch=None, gauge=10.0,
               mt=(1e6, 1e6, 0.0), das_mode=W.STRAIN):
    m = lambda v: np.full((n, n), v)
    if ch is None:
        chx, cht, ptr = np.zeros((0, 2)), np.zeros((0, 2)), np.array([0, 0], np.int32)
    else:
        chx, cht, ptr = np.asarray(ch[0], float), np.asarray(ch[1], float), np.array([0, len(ch[0])], np.int32)
    acq = W.Acquisition(nx=n, nz=n, dx=dx, dz=dx, nt=nt, dt=dt, src_xz=np.array([src], float),
                        mt=np.array([mt], float), wavelet=W.ricker(f0, nt, dt)[None], tr_ptr=ptr,
                        ch_xz=chx, ch_t=cht, gauge=gauge, ref_vp=m(vp), ref_vs=m(vs), ref_rho=m(rho),
                        pml_f0=f0, das_mode=das_mode)
    return acq, m(vp), m(vs), m(rho)


def _greens_errors(dx, dt, T, f0, L, recx, gauge=10.0):
    n = int(round(L / dx))
    nt = int(round(T / dt))
    xs = zs = (n // 2) * dx
    geo = (xs + recx + 0.5 * dx, zs)                       # exactly on the vx grid
    ch = ([[xs + recx, zs]], [[1.0, 0.0]])
    acq, vp, vs, rho = _homog_acq(n, dx, dt, nt, (xs, zs), f0, ch=ch, gauge=gauge)
    d, g, _ = E.Shot(acq, 0, vp, vs, rho, geophones=[geo]).forward()
    tv = (np.arange(nt) + 0.5) * dt                         # v lives at t_{n+1/2}
    ana_v = explosion_vx(tv, geo[0] - xs, 0.0, 1e6, 2000.0, 3000.0, f0, 1.5 / f0)
    td = (np.arange(nt) + 1.0) * dt                         # DAS sample n is u at t_{n+1}
    up = explosion_ux(td, recx + gauge / 2, 0.0, 1e6, 2000.0, 3000.0, f0, 1.5 / f0)
    um = explosion_ux(td, recx - gauge / 2, 0.0, 1e6, 2000.0, 3000.0, f0, 1.5 / f0)
    ana_d = (up - um) / gauge
    ev = np.linalg.norm(g[0, 0] - ana_v) / np.linalg.norm(ana_v)
    ed = np.linalg.norm(d[0] - ana_d) / np.linalg.norm(ana_d)
    return ev, ed


def test_greens_function_explosion():
    """15 points per shortest wavelength: velocity and DAS strain within 1.5 % of the closed form."""
    ev, ed = _greens_errors(2.0, 2.5e-4, 0.13, 40.0, 400.0, 150.0)
    assert ev < 1.5e-2, ev
    assert ed < 1.5e-2, ed


def test_greens_function_second_order_convergence():
    """Halving dx and dt cuts the error about 4x (2nd order in time dominates)."""
    e1 = _greens_errors(2.0, 2.5e-4, 0.09, 50.0, 240.0, 80.0)[0]
    e2 = _greens_errors(1.0, 1.25e-4, 0.09, 50.0, 240.0, 80.0)[0]
    assert 3.0 < e1 / e2 < 5.0, (e1, e2)


def test_reciprocity_force_velocity():
    """v_z at B from f_x at A equals v_x at A from f_z at B (heterogeneous medium, CPML on)."""
    rng = np.random.default_rng(3)
    n, dx, dt, nt, f0 = 60, 2.0, 2e-4, 300, 40.0
    vp = 3000 + 300 * rng.random((n, n)); vs = vp / 1.8; rho = 2000 + 200 * rng.random((n, n))
    A = (22 * dx + 0.5 * dx, 30 * dx)
    B = (38 * dx, 33 * dx + 0.5 * dx)

    def run(src, force, rec, comp):
        acq = W.Acquisition(nx=n, nz=n, dx=dx, dz=dx, nt=nt, dt=dt, src_xz=np.array([src]),
                            mt=np.zeros((1, 3)), wavelet=W.ricker(f0, nt, dt)[None],
                            tr_ptr=np.array([0, 0], np.int32), ch_xz=np.zeros((0, 2)), ch_t=np.zeros((0, 2)),
                            gauge=1.0, ref_vp=vp, ref_vs=vs, ref_rho=rho, pml_f0=f0)
        return E.Shot(acq, 0, vp, vs, rho, force=force, geophones=[rec]).forward()[1][0, comp]

    g1 = run(A, (1.0, 0.0), B, 1)
    g2 = run(B, (0.0, 1.0), A, 0)
    assert np.abs(g1).max() > 0
    assert np.linalg.norm(g1 - g2) / np.linalg.norm(g1) < 1e-12


def test_cpml_reflections_small():
    """A 40-cell domain with CPML matches a 3x larger domain to 1e-3 in amplitude."""
    dx, dt, f0, nt = 2.0, 2e-4, 40.0, 500

    def run(n, off):
        src = (off * dx + 20 * dx, off * dx + 20 * dx)
        rec = (off * dx + 30 * dx + 0.5 * dx, off * dx + 20 * dx)
        acq, vp, vs, rho = _homog_acq(n, dx, dt, nt, src, f0)
        return E.Shot(acq, 0, vp, vs, rho, geophones=[rec]).forward()[1][0, 0]

    small, big = run(41, 0), run(123, 41)
    assert np.linalg.norm(small - big) / np.linalg.norm(big) < 1e-3


def test_linearity_in_moment_tensor_and_wavelet():
    p = W.tiny(ns=1, nt=30)
    acq = p.acq
    d0 = E.forward(acq, p.vp, p.vs, p.rho)
    acq2 = W.Acquisition(**{**acq.__dict__, "mt": 2.5 * acq.mt})
    d2 = E.forward(acq2, p.vp, p.vs, p.rho)
    assert np.allclose(d2, 2.5 * d0, rtol=1e-13, atol=1e-13 * np.abs(d0).max())
    rng = np.random.default_rng(0)
    w1, w2 = rng.standard_normal(acq.wavelet.shape), rng.standard_normal(acq.wavelet.shape)
    da = E.forward(W.Acquisition(**{**acq.__dict__, "wavelet": w1}), p.vp, p.vs, p.rho)
    db = E.forward(W.Acquisition(**{**acq.__dict__, "wavelet": w2}), p.vp, p.vs, p.rho)
    dab = E.forward(W.Acquisition(**{**acq.__dict__, "wavelet": w1 + w2}), p.vp, p.vs, p.rho)
    assert np.allclose(dab, da + db, rtol=0, atol=1e-12 * np.abs(dab).max())


def test_das_strain_is_integral_of_strain_rate():
    p = W.tiny(ns=1, nt=30, das_mode=W.STRAIN)
    d_strain = E.forward(p.acq, p.vp, p.vs, p.rho)
    pr = W.tiny(ns=1, nt=30, das_mode=W.STRAIN_RATE)
    d_rate = E.forward(pr.acq, pr.vp, pr.vs, pr.rho)
    assert np.allclose(d_strain, np.cumsum(d_rate, axis=1) * p.acq.dt, rtol=1e-12,
                       atol=1e-12 * np.abs(d_strain).max())


def test_velocity_receivers_equal_geophone_recordings():
    """2-C particle-velocity traces (VELOCITY mode, t = (1, 0) and (0, 1) at each
    channel point) equal the oracle's separate geophone recording of (vx, vz)
    at the same points, the path the Green's-function test pins."""
    p = W.two_component(W.tiny(ns=1, nt=40))
    acq = p.acq
    pts = acq.ch_xz[::2]
    d, g, _ = E.Shot(acq, 0, p.vp[0], p.vs[0], p.rho[0], geophones=pts).forward()
    assert np.abs(g).max() > 0
    assert np.allclose(d[0::2], g[:, 0], rtol=0, atol=1e-15 * np.abs(g).max())
    assert np.allclose(d[1::2], g[:, 1], rtol=0, atol=1e-15 * np.abs(g).max())


def test_explosion_is_mirror_symmetric():
    """Homogeneous medium, explosion on the centre node: v_x is odd about the source."""
    n, dx, dt, nt, f0 = 41, 2.0, 2e-4, 120, 60.0
    c = 20 * dx
    acq, vp, vs, rho = _homog_acq(n, dx, dt, nt, (c, c), f0)
    right = (c + 6 * dx + 0.5 * dx, c)
    left = (c - 6 * dx - 0.5 * dx, c)
    g = E.Shot(acq, 0, vp, vs, rho, geophones=[right, left]).forward()[1]
    assert np.abs(g[0, 0]).max() > 0
    assert np.allclose(g[0, 0], -g[1, 0], rtol=0, atol=1e-12 * np.abs(g[0, 0]).max())
