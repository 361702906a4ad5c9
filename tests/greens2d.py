"""Closed-form 2D homogeneous elastic response to an explosive point source.

Used only by tests to pin the oracle's propagator to the physics.  For an
isotropic moment tensor M = M0 I the body force -M grad(delta) w(t) (eq. 2,
third case) is a gradient, so the displacement is u = grad(phi) with

    phi_tt - alpha^2 lap(phi) = -(M0 / rho) delta(x) w(t).

The 2D Green's function of the scalar wave equation is
G(r, t) = H(t - r/c) / (2 pi c sqrt(c^2 t^2 - r^2)); substituting
tau = (r/c) cosh(theta) removes its singularity:

    (G * f)(t) = 1/(2 pi c^2) int_0^{acosh(c t / r)} f(t - (r/c) cosh(theta)) dtheta,

and d/dr (G * f) = -1/(2 pi c^3) int_0^{...} cosh(theta) f'(t - (r/c) cosh(theta)) dtheta
(the boundary term vanishes because the delayed Ricker is ~0 at t = 0).
Hence  u_x = -(M0/rho) (x/r) d/dr (G * w),  v_x = -(M0/rho) (x/r) d/dr (G * w').
"""
import numpy as np


def ricker_derivs(t, f0, t0):
    """w, w', w'' of the Ricker wavelet (1 - 2u^2) exp(-u^2), u = pi f0 (t - t0)."""
    a = np.pi * f0
    u = a * (t - t0)
    e = np.exp(-u * u)
    w = (1 - 2 * u * u) * e
    w1 = a * (-6 * u + 4 * u ** 3) * e
    w2 = a * a * (-6 + 24 * u * u - 8 * u ** 4) * e
    return w, w1, w2


def _dr_conv(t, r, c, fprime, nquad=4000):
    """d/dr (G * f)(t) with f' given as a callable, for an array of times t."""
    out = np.zeros_like(t)
    for k, tk in enumerate(t):
        if c * tk <= r:
            continue
        th_max = np.arccosh(c * tk / r)
        th = np.linspace(0.0, th_max, nquad)
        y = np.cosh(th) * fprime(tk - (r / c) * np.cosh(th))
        out[k] = -np.trapezoid(y, th) / (2 * np.pi * c ** 3)
    return out


def explosion_ux(t, x, z, M0, rho, vp, f0, t0):
    """Displacement u_x at offset (x, z) from the source (source at the origin)."""
    r = np.hypot(x, z)
    d = _dr_conv(t, r, vp, lambda s: ricker_derivs(s, f0, t0)[1])
    return -(M0 / rho) * (x / r) * d


def explosion_vx(t, x, z, M0, rho, vp, f0, t0):
    """Particle velocity v_x at offset (x, z) from the source."""
    r = np.hypot(x, z)
    d = _dr_conv(t, r, vp, lambda s: ricker_derivs(s, f0, t0)[2])
    return -(M0 / rho) * (x / r) * d
