"""FP64 oracle for the model extension along sources: zone-of-influence weights,
the footprint operator W, the weighted collapse S_w and the consistency term
1/2 eta^2 ||(I - S^T S_w) W m~||^2 of the extended misfit with its gradient.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The operators are built per pixel as small dense Ns x Ns matrices straight from
their definitions and applied with a plain matrix product:

* eq. 10  b = (cos^n(pi r / 2) - log nu) / (1 - log nu), 0 <= r <= 1
  (natural log).  Outer taper: r = Euclidean distance outside the active
  x-span / taper width, clamped to [0, 1].  Sinkhole: Mahalanobis distance
  d_M = sqrt((x-x_s)^2/a_x^2 + (z-z_s)^2/a_z^2), r = clamp(1 - d_M, 0, 1),
  inside the sinkhole iff d_M < 1.  The two weights combine by min().
* eq. 11  inside the sinkhole of s:  (W m)_s = b_s m_s
          + (1 - b_s) / sum_{i != s} b_i * sum_{i != s} b_i m_i,
  elsewhere (W m)_s = m_s.  With one source the sum is empty and W = I.
* eq. 12  S_w m~ = sum_s b'_s m_s / sum_s b'_s, b'_s = 1 inside the sinkhole
  of s and b_s outside.  S^T copies a physical model to every component.
* eq. 8   phi_reg = 1/2 eta^2 ||(I - S^T S_w) W m~||^2, applied to each
          parameter field (Vp, Vs, rho) with its own eta.
"""
from __future__ import annotations

import numpy as np


def zoi_profile(r, n, nu):
    """eq. 10 weight for a normalised distance r in [0, 1]."""
    r = np.clip(np.asarray(r, np.float64), 0.0, 1.0)
    ln = np.log(nu)
    return (np.cos(0.5 * np.pi * r) ** n - ln) / (1.0 - ln)


def zoi_weights(zoi, nx, nz, dx, dz):
    """b, b' and the sinkhole flag for every source: arrays [Ns, nz, nx]."""
    ns = zoi.sink_xz.shape[0]
    x = (np.arange(nx) * dx)[None, :]
    z = (np.arange(nz) * dz)[:, None]
    b = np.zeros((ns, nz, nx)); bp = np.zeros((ns, nz, nx)); sink = np.zeros((ns, nz, nx), np.uint8)
    for s in range(ns):
        xa, xb = zoi.active_x[s]
        dist = np.maximum(np.maximum(xa - x, x - xb), 0.0) + 0.0 * z
        r_out = np.minimum(dist / zoi.taper[s], 1.0)
        dm = np.sqrt(((x - zoi.sink_xz[s, 0]) / zoi.sink_ax[s]) ** 2 + ((z - zoi.sink_xz[s, 1]) / zoi.sink_az[s]) ** 2)
        inside = dm < 1.0
        r_sink = np.clip(1.0 - dm, 0.0, 1.0)
        b[s] = np.minimum(zoi_profile(r_out, zoi.n, zoi.nu), zoi_profile(r_sink, zoi.n, zoi.nu))
        bp[s] = np.where(inside, 1.0, b[s])
        sink[s] = inside
    return b, bp, sink


def w_matrices(b, sink):
    """Per-pixel W (eq. 11): b, sink are [Ns, npix]; returns [npix, Ns, Ns]."""
    ns, npix = b.shape
    W = np.zeros((npix, ns, ns))
    for s in range(ns):
        W[:, s, s] = 1.0
    if ns == 1:
        return W
    for s in range(ns):
        others = [i for i in range(ns) if i != s]
        denom = b[others].sum(axis=0)
        ins = sink[s].astype(bool)
        W[ins, s, s] = b[s, ins]
        for i in others:
            W[ins, s, i] = (1.0 - b[s, ins]) * b[i, ins] / denom[ins]
    return W


def sw_rows(bp):
    """Per-pixel S_w row (eq. 12): bp is [Ns, npix]; returns omega [npix, Ns]."""
    return (bp / bp.sum(axis=0, keepdims=True)).T


def consistency_operator(b, bp, sink):
    """A = (I - S^T S_w) W per pixel: [npix, Ns, Ns]."""
    W = w_matrices(b, sink)
    om = sw_rows(bp)
    ns = b.shape[0]
    Pm = np.eye(ns)[None] - np.ones((1, ns, 1)) * om[:, None, :]
    return Pm @ W


def regularization(m, b, bp, sink, eta, chunk=4096):
    """phi_reg = 1/2 eta^2 ||A m~||^2 and its gradient eta^2 A^T A m~ (eq. 8, second term).

    m, b, bp, sink: [Ns, nz, nx].  Returns (phi_reg, grad [Ns, nz, nx]).
    """
    ns = m.shape[0]
    shp = m.shape
    mf = np.asarray(m, np.float64).reshape(ns, -1)
    bf = np.asarray(b, np.float64).reshape(ns, -1)
    bpf = np.asarray(bp, np.float64).reshape(ns, -1)
    sf = np.asarray(sink).reshape(ns, -1)
    g = np.zeros_like(mf)
    phi = 0.0
    for p0 in range(0, mf.shape[1], chunk):
        sl = slice(p0, p0 + chunk)
        A = consistency_operator(bf[:, sl], bpf[:, sl], sf[:, sl])
        r = np.einsum("pij,jp->pi", A, mf[:, sl])
        phi += 0.5 * eta ** 2 * float(np.sum(r * r))
        g[:, sl] = eta ** 2 * np.einsum("pji,pj->ip", A, r)
    return phi, g.reshape(shp)


def collapse(m, b, bp, sink, chunk=4096):
    """Final physical model m^ = S_w W m~ (eq. 9): [Ns, nz, nx] -> [nz, nx].

    Applied to the per-source gradients g~ it gives the preconditioned gradient
    S_w W g~ of eq. 15.  Pixels are independent; they are processed in chunks.
    """
    ns = m.shape[0]
    mf = np.asarray(m, np.float64).reshape(ns, -1)
    bf = np.asarray(b, np.float64).reshape(ns, -1)
    bpf = np.asarray(bp, np.float64).reshape(ns, -1)
    sf = np.asarray(sink).reshape(ns, -1)
    out = np.zeros(mf.shape[1])
    for p0 in range(0, mf.shape[1], chunk):
        sl = slice(p0, p0 + chunk)
        W = w_matrices(bf[:, sl], sf[:, sl])
        om = sw_rows(bpf[:, sl])
        y = np.einsum("pij,jp->pi", W, mf[:, sl])
        out[sl] = np.einsum("pi,pi->p", om, y)
    return out.reshape(m.shape[1:])
