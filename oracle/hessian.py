"""FP64 oracle of the pseudo-Hessian preconditioner, the paper's first
comparison method (illumination compensation): a diagonal operator built by
auto-correlating the absolute particle velocity wavefields in time at zero
lag, summing over shots, clipping and scaling; the l-BFGS solver receives it
as its initial inverse-Hessian guess (pseudo-Hessian = diagonal of the
approximate Hessian, preconditioning paragraph and comparison section).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Readings where the paper gives no formula (also listed in the design notes)
---------------------------------------------------------------------------
* |v|^2 at a pixel (node (i, j)) uses the particle velocity sampled at the
  node the way a 2-C receiver samples it: the mean of the two staggered
  neighbours of each component, vx at (i -+ 1/2, j) and vz at (i, j -+ 1/2).
* The zero-lag auto-correlation is the sum over the time levels t_{n+1/2},
  n = 0..nt-1, of |v|^2 (no dt factor).
* H(x) = sum_s sum_n |v_s(x, t_{n+1/2})|^2; shot s runs in its own component
  m_s of the extended model and contributes only inside its window.
* Clipping and scaling: P(x) = c / max(H(x), c) with c = eps * max_x H, so
  P is 1 where H <= c (clipped) and eps where H is largest; P = 1 everywhere
  when H vanishes.  P multiplies the gradient (it scales the update down near
  the sources, where H is large).
"""
from __future__ import annotations

import numpy as np

from .elastic import Shot


def node_speed2(sh, vx, vz):
    """|v|^2 on the physical nodes of shot sh's window, [nz, w]."""
    P, nz, w = sh.P, sh.acq.nz, sh.w
    vxn = 0.5 * (vx[P:P + nz, P - 1:P + w - 1] + vx[P:P + nz, P:P + w])
    vzn = 0.5 * (vz[P - 1:P + nz - 1, P:P + w] + vz[P:P + nz, P:P + w])
    return vxn * vxn + vzn * vzn


def pseudo_hessian(acq, vp, vs, rho, shots=None):
    """H [nz, nx]: zero-lag auto-correlation of |v|, summed over the shots."""
    H = np.zeros((acq.nz, acq.nx))
    win = acq.windows()
    for s in (range(acq.ns) if shots is None else shots):
        sh = Shot(acq, s, vp[s], vs[s], rho[s])
        x0, w = (int(v) for v in win[s])
        st = sh.zero_state()
        for n in range(acq.nt):
            st, _, _ = sh.step(st, n)
            H[:, x0:x0 + w] += node_speed2(sh, st["vx"], st["vz"])
    return H


def inverse_pseudo_hessian(H, eps):
    """Clipped and scaled inverse P = c / max(H, c), c = eps max(H); ones if H == 0."""
    H = np.asarray(H, np.float64)
    hmax = float(H.max()) if H.size else 0.0
    if not hmax > 0.0:
        return np.ones_like(H)
    c = eps * hmax
    return c / np.maximum(H, c)
