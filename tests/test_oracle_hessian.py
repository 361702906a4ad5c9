"""Pins of the oracle's pseudo-Hessian (the paper's illumination-compensation
comparison method: zero-lag auto-correlation of the absolute particle
velocity, summed over shots, clipped and scaled).  No GPU.

* H at a pixel equals the sum over shots and time samples of the squared
  2-C receiver traces recorded at that node by the oracle's geophone path
  (itself pinned to the closed-form Green's function), so a wrong staggered
  neighbour, a dropped 1/2 or a missing component fails;
* exact quadratic scaling with the source amplitude and additivity over shots;
* zero outside every shot's window;
* the clipped, scaled inverse: values in [eps, 1], 1 where H <= eps max H,
  eps at the maximum, non-increasing in H, ones for a vanishing H.
"""
import copy

import numpy as np

import workloads as W
from oracle import elastic as E
from oracle import hessian as PH

WIN = [[0, 20], [6, 21]]


def _problem():
    return W.tiny(nx=30, nz=18, ns=2, nt=50, npml=4, win=WIN)


def test_equals_squared_receiver_traces():
    p = _problem()
    acq = p.acq
    H = PH.pseudo_hessian(acq, p.vp, p.vs, p.rho)
    pix = [(3, 4), (9, 7), (10, 12), (15, 9), (22, 5), (26, 14), (19, 16)]
    ref = np.zeros(len(pix))
    for s, (x0, w) in enumerate(WIN):
        inside = [k for k, (i, j) in enumerate(pix) if x0 <= i < x0 + w]
        pts = [(pix[k][0] * acq.dx, pix[k][1] * acq.dz) for k in inside]
        _, geo, _ = E.Shot(acq, s, p.vp[s], p.vs[s], p.rho[s], geophones=pts).forward()
        for q, k in enumerate(inside):
            ref[k] += float(np.sum(geo[q, 0] ** 2) + np.sum(geo[q, 1] ** 2))
    got = np.array([H[j, i] for i, j in pix])
    assert np.all(ref > 0)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def test_amplitude_squared_and_shot_additivity():
    p = _problem()
    acq = p.acq
    H = PH.pseudo_hessian(acq, p.vp, p.vs, p.rho)
    parts = [PH.pseudo_hessian(acq, p.vp, p.vs, p.rho, shots=[s]) for s in range(acq.ns)]
    np.testing.assert_allclose(H, parts[0] + parts[1], rtol=1e-13, atol=0)
    a2 = copy.deepcopy(acq)
    a2.wavelet = 2.0 * np.asarray(acq.wavelet)
    H2 = PH.pseudo_hessian(a2, p.vp, p.vs, p.rho)
    np.testing.assert_allclose(H2, 4.0 * H, rtol=1e-12, atol=0)


def test_zero_outside_windows():
    p = W.tiny(nx=30, nz=18, ns=2, nt=30, npml=4, win=[[2, 10], [15, 11]])
    H = PH.pseudo_hessian(p.acq, p.vp, p.vs, p.rho)
    outside = np.ones(30, bool)
    outside[2:12] = outside[15:26] = False
    assert np.all(H[:, outside] == 0.0)
    assert np.all(H[:, ~outside] > 0.0)


def test_clipped_scaled_inverse():
    rng = np.random.default_rng(3)
    H = rng.random((7, 9)) ** 4 * 5.0
    eps = 0.05
    P = PH.inverse_pseudo_hessian(H, eps)
    c = eps * H.max()
    assert np.all((P >= eps - 1e-15) & (P <= 1.0))
    assert np.all(P[H <= c] == 1.0)
    assert P.flat[np.argmax(H)] == eps
    order = np.argsort(H, axis=None)
    assert np.all(np.diff(P.flat[order]) <= 0.0)
    np.testing.assert_allclose(P[H > c], c / H[H > c], rtol=1e-15)
    assert np.all(PH.inverse_pseudo_hessian(np.zeros((3, 4)), eps) == 1.0)
