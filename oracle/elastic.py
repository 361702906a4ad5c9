"""FP64 oracle: 2D isotropic elastic velocity-stress modelling, DAS sampling,
L2 misfit and the exact discrete adjoint-state gradient, one shot at a time.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Plain numpy, float64,
whole-array operations; no tiling, fusion or reordering.

What it follows
---------------
* Wave equation A(m) u_s = f_s (eq. 1) with m = (Vp, Vs, rho); the paper fixes
  no scheme, so it is written as the velocity-stress system on a Virieux
  staggered grid, 4th order in space (c1 = 9/8, c2 = -1/24) and 2nd order
  (leapfrog) in time, with a convolutional PML (Komatitsch & Martin 2007,
  kappa = 1, quadratic damping, alpha = pi f0 (1 - r)).
* Moment-tensor point source -M grad(delta) w(t) (eq. 2, third case): since
  -M grad(delta) w = div(-M delta w), the stresses are driven by -M delta w;
  per step sigma^{n+1} -= M (w_{n+1} - w_n) delta_h, delta_h = bilinear
  weight / (dx dz).  A vector-force source F delta w (eq. 2, second case)
  enters the velocity sub-step: v^{n+1/2} += dt b F w(t_n) delta_h on the
  staggered v grids; it replaces the moment tensor of its shot.
* Sampling operator K_r (eq. 3) as DAS gauge-averaged axial strain
  t.(u(p+) - u(p-))/L with u the running time integral of the particle
  velocity at the gauge ends (or strain rate with v instead of u), or as a
  particle-velocity receiver (the synthetic section's 2-C acquisition):
  trace value t.v(p) at the channel point p, one trace per component t.
* Misfit phi = 1/2 sum_s sum_r ||d_{s,r} - d_obs||^2 (eq. 4; first term of
  eq. 8 with the model m_s specific to shot s).
* Gradient g_s = J_s^T (d_s - d_obs_s) (eq. 6) by the adjoint-state method:
  every sub-step of the discrete forward map is transposed literally
  (derivative operators by explicit scatter), run backwards in time, and the
  zero-lag products of adjoint and forward quantities give the derivatives
  with respect to lambda, mu, mu_xz, b_x, b_z, which the chain rule maps to
  (Vp, Vs, rho) on the physical grid.

Readings where the paper is silent (also listed in the design notes)
--------------------------------------------------------------------
* The physical nx x nz grid is padded by P = npml + 1 cells on every side.
  The padding holds a frozen reference model (edge-replicated), so only the
  physical cells are inversion variables.  The CPML damping is zero on the
  first padding node (index positions P-1 .. N-P) and ramps over the outer
  npml cells, so no staggered position whose material depends on a physical
  node carries PML memory.
* Ghost values outside the padded grid are zero, so the staggered derivative
  operators are exact transposes of each other up to sign.
* Staggering (row j = z, column i = x): sxx, szz, lambda, mu at (i, j);
  vx, b_x at (i+1/2, j); vz, b_z at (i, j+1/2); sxz, mu_xz at (i+1/2, j+1/2).
  mu_xz is the harmonic mean of the 4 surrounding mu, b_x/b_z the arithmetic
  mean of 1/rho of the 2 surrounding nodes (last row/column repeated).
* Time levels: sigma at t_n = n dt, v at t_{n+1/2}; one step n maps
  (v^{n-1/2}, sigma^n) -> (v^{n+1/2}, sigma^{n+1}); sample n of the data is
  taken after the velocity update of step n (n = 0..nt-1).
"""
from __future__ import annotations

import numpy as np

C1 = 9.0 / 8.0
C2 = -1.0 / 24.0
STRAIN, STRAIN_RATE, VELOCITY = 0, 1, 2


# ---------------------------------------------------------------------------
# 4th-order staggered derivatives with zero ghosts, and their literal transposes
# ---------------------------------------------------------------------------

def _gx(f):
    return np.pad(f, ((0, 0), (2, 2)))


def dxp(f, h):
    """d/dx from integer to half positions: out[:, i] lives at x-index i+1/2."""
    g = _gx(f)
    return (C1 * (g[:, 3:-1] - g[:, 2:-2]) + C2 * (g[:, 4:] - g[:, 1:-3])) / h


def dxm(f, h):
    """d/dx from half to integer positions: input f[:, i] lives at i+1/2, out at i."""
    g = _gx(f)
    return (C1 * (g[:, 2:-2] - g[:, 1:-3]) + C2 * (g[:, 3:-1] - g[:, 0:-4])) / h


def dxp_T(y, h):
    """Transpose of dxp, as a scatter of each output's stencil back onto its inputs."""
    g = np.zeros((y.shape[0], y.shape[1] + 4))
    g[:, 3:-1] += C1 * y
    g[:, 2:-2] -= C1 * y
    g[:, 4:] += C2 * y
    g[:, 1:-3] -= C2 * y
    return g[:, 2:-2] / h


def dxm_T(y, h):
    """Transpose of dxm, as a scatter."""
    g = np.zeros((y.shape[0], y.shape[1] + 4))
    g[:, 2:-2] += C1 * y
    g[:, 1:-3] -= C1 * y
    g[:, 3:-1] += C2 * y
    g[:, 0:-4] -= C2 * y
    return g[:, 2:-2] / h


def dzp(f, h):
    return dxp(f.T, h).T


def dzm(f, h):
    return dxm(f.T, h).T


def dzp_T(y, h):
    return dxp_T(y.T, h).T


def dzm_T(y, h):
    return dxm_T(y.T, h).T


# ---------------------------------------------------------------------------
# Materials, CPML profiles, point weights
# ---------------------------------------------------------------------------

def materials(vp, vs, rho):
    """lambda, mu at nodes; mu_xz (harmonic, 4 nodes); b_x, b_z (arithmetic 1/rho, 2 nodes)."""
    lam = rho * (vp ** 2 - 2.0 * vs ** 2)
    mu = rho * vs ** 2
    me = np.pad(mu, ((0, 1), (0, 1)), mode="edge")
    re = np.pad(rho, ((0, 1), (0, 1)), mode="edge")
    m00, m01, m10, m11 = me[:-1, :-1], me[:-1, 1:], me[1:, :-1], me[1:, 1:]
    zero = (m00 == 0) | (m01 == 0) | (m10 == 0) | (m11 == 0)
    with np.errstate(divide="ignore"):
        muxz = np.where(zero, 0.0, 4.0 / (1.0 / m00 + 1.0 / m01 + 1.0 / m10 + 1.0 / m11))
    bx = 0.5 * (1.0 / re[:-1, :-1] + 1.0 / re[:-1, 1:])
    bz = 0.5 * (1.0 / re[:-1, :-1] + 1.0 / re[1:, :-1])
    return lam, mu, muxz, bx, bz


def cpml_profile(N, P, h, npml, R, vmax, f0, dt, half):
    """CPML coefficients (a, b) along one axis of N padded cells.

    psi <- b psi + a d(.)  with  b = exp(-(d + alpha) dt),
    a = d (b - 1) / (d + alpha);  d(r) = d0 r^2, d0 = -3 vmax ln(R) / (2 L),
    alpha = pi f0 (1 - r), r = distance into the layer / L, L = npml h.
    """
    pos = np.arange(N, dtype=np.float64) + (0.5 if half else 0.0)
    dist = np.maximum(np.maximum((P - 1) - pos, pos - (N - P)), 0.0)
    L = npml * h
    r = np.minimum(dist * h / L, 1.0)
    d0 = -3.0 * vmax * np.log(R) / (2.0 * L)
    d = d0 * r ** 2
    alpha = np.pi * f0 * (1.0 - r)
    b = np.exp(-(d + alpha) * dt)
    a = np.where(d > 0, d * (b - 1.0) / np.where(d > 0, d + alpha, 1.0), 0.0)
    return a, b


def bilinear(fi, fj):
    """4 (j, i, weight) corners of a fractional padded index (fi along x, fj along z)."""
    i0, j0 = int(np.floor(fi)), int(np.floor(fj))
    ti, tj = fi - i0, fj - j0
    return [(j0, i0, (1 - ti) * (1 - tj)), (j0, i0 + 1, ti * (1 - tj)),
            (j0 + 1, i0, (1 - ti) * tj), (j0 + 1, i0 + 1, ti * tj)]


# ---------------------------------------------------------------------------
# One shot
# ---------------------------------------------------------------------------

class Shot:
    """Forward and adjoint time stepping of shot s with its own model m_s.

    vp, vs, rho: [nz, nx] physical model (the extended component of shot s).
    force: optional (fx, fz) replacing the moment tensor by a vector force
    (default: acq.force[s] when the acquisition has forces).
    geophones: optional [k, 2] points where (vx, vz) are also recorded.
    """

    def __init__(self, acq, s, vp, vs, rho, force=None, geophones=None):
        self.acq, self.s = acq, s
        P = acq.npml + 1
        x0, w = (int(v) for v in acq.windows()[s])
        self.P, self.x0, self.w = P, x0, w
        nz = acq.nz
        self.NX, self.NZ = w + 2 * P, nz + 2 * P
        self.dx, self.dz, self.dt = acq.dx, acq.dz, acq.dt

        def padded(phys, ref):
            out = np.pad(np.asarray(ref, np.float64)[:, x0:x0 + w], P, mode="edge")
            out[P:P + nz, P:P + w] = np.asarray(phys, np.float64)[:, x0:x0 + w]
            return out

        self.vp = padded(vp, acq.ref_vp)
        self.vs = padded(vs, acq.ref_vs)
        self.rho = padded(rho, acq.ref_rho)
        self.lam, self.mu, self.muxz, self.bx, self.bz = materials(self.vp, self.vs, self.rho)

        vmax, f0 = acq.vmax(), acq.pml_f0
        prof = lambda N, h, half: cpml_profile(N, P, h, acq.npml, acq.pml_R, vmax, f0, acq.dt, half)
        ax_i, bx_i = prof(self.NX, acq.dx, False)
        ax_h, bx_h = prof(self.NX, acq.dx, True)
        az_i, bz_i = prof(self.NZ, acq.dz, False)
        az_h, bz_h = prof(self.NZ, acq.dz, True)
        X = lambda v: v[None, :]
        Z = lambda v: v[:, None]
        # (a, b) for psi_1..psi_8, in the order used by the sub-steps
        self.pml = [(X(ax_h), X(bx_h)), (Z(az_i), Z(bz_i)), (X(ax_i), X(bx_i)), (Z(az_h), Z(bz_h)),
                    (X(ax_i), X(bx_i)), (Z(az_i), Z(bz_i)), (Z(az_h), Z(bz_h)), (X(ax_h), X(bx_h))]

        # source
        sx, sz = acq.src_xz[s]
        self.wav = np.asarray(acq.wavelet[s], np.float64)
        if force is None and getattr(acq, "force", None) is not None:
            force = np.asarray(acq.force[s], np.float64)
        self.force = force
        self.inj_node = self._weights(sx, sz, 0.0, 0.0)
        self.inj_xz = self._weights(sx, sz, 0.5, 0.5)
        self.inj_vx = self._weights(sx, sz, 0.5, 0.0)
        self.inj_vz = self._weights(sx, sz, 0.0, 0.5)
        self.M = np.asarray(acq.mt[s], np.float64)

        # DAS gauges of this shot: per trace, endpoints p+ and p-, components x and z
        a, b = int(acq.tr_ptr[s]), int(acq.tr_ptr[s + 1])
        self.ntr = b - a
        self.ch_t = np.asarray(acq.ch_t[a:b], np.float64)
        self.gauge = float(acq.gauge)
        # per trace c and component k (0: vx at p+, 1: vz at p+, 2: vx at p-, 3: vz at p-),
        # the 4 bilinear corners (row, column, weight) on that component's grid
        self.das_j = np.zeros((self.ntr, 4, 4), np.int64)
        self.das_i = np.zeros((self.ntr, 4, 4), np.int64)
        self.das_wt = np.zeros((self.ntr, 4, 4))
        for c in range(self.ntr):
            cx, cz = acq.ch_xz[a + c]
            tx, tz = self.ch_t[c]
            if acq.das_mode == VELOCITY:            # one point; the "p-" samples get zero weight
                pp = pm = (cx, cz)
            else:
                pp = (cx + 0.5 * self.gauge * tx, cz + 0.5 * self.gauge * tz)
                pm = (cx - 0.5 * self.gauge * tx, cz - 0.5 * self.gauge * tz)
            for k, (pt, ox, oz) in enumerate(((pp, 0.5, 0.0), (pp, 0.0, 0.5), (pm, 0.5, 0.0), (pm, 0.0, 0.5))):
                for q, (j, i, wt) in enumerate(self._weights(pt[0], pt[1], ox, oz)):
                    self.das_j[c, k, q], self.das_i[c, k, q], self.das_wt[c, k, q] = j, i, wt
        self.geo = []
        if geophones is not None:
            for gx, gz in np.asarray(geophones, np.float64):
                self.geo.append((self._weights(gx, gz, 0.5, 0.0), self._weights(gx, gz, 0.0, 0.5)))

    def _weights(self, x, z, ox, oz):
        acq = self.acq
        if not (0.0 <= x / acq.dx - self.x0 <= self.w - 1 and 0.0 <= z / acq.dz <= acq.nz - 1):
            raise ValueError(f"point ({x}, {z}) outside the physical window of shot {self.s}")
        fi = x / acq.dx - self.x0 + self.P - ox
        fj = z / acq.dz + self.P - oz
        return bilinear(fi, fj)

    # -- state -------------------------------------------------------------
    def zero_state(self):
        z = lambda: np.zeros((self.NZ, self.NX))
        return {"vx": z(), "vz": z(), "sxx": z(), "szz": z(), "sxz": z(),
                "psi": [z() for _ in range(8)], "U": np.zeros((self.ntr, 4))}

    @staticmethod
    def copy_state(st):
        return {k: ([a.copy() for a in v] if isinstance(v, list) else v.copy()) for k, v in st.items()}

    @staticmethod
    def _sample(f, wl):
        return sum(wt * f[j, i] for j, i, wt in wl)

    @staticmethod
    def _spread(f, wl, val):
        for j, i, wt in wl:
            f[j, i] += wt * val

    # -- forward sub-steps ---------------------------------------------------
    def _velocity(self, st, n):
        """v^{n+1/2} = v^{n-1/2} + dt b (D sigma^n + psi); returns new v, psi_1..4 and the increments."""
        dx, dz, dt = self.dx, self.dz, self.dt
        e = [dxp(st["sxx"], dx), dzm(st["sxz"], dz), dxm(st["sxz"], dx), dzp(st["szz"], dz)]
        psi = [self.pml[k][1] * st["psi"][k] + self.pml[k][0] * e[k] for k in range(4)]
        acc_x = e[0] + psi[0] + e[1] + psi[1]
        acc_z = e[2] + psi[2] + e[3] + psi[3]
        vx = st["vx"] + dt * self.bx * acc_x
        vz = st["vz"] + dt * self.bz * acc_z
        if self.force is not None:
            wn = self.wav[n] / (self.dx * self.dz)
            vx = vx.copy(); vz = vz.copy()
            bxs = [(j, i, wt * dt * self.bx[j, i]) for j, i, wt in self.inj_vx]
            bzs = [(j, i, wt * dt * self.bz[j, i]) for j, i, wt in self.inj_vz]
            self._spread(vx, bxs, self.force[0] * wn)
            self._spread(vz, bzs, self.force[1] * wn)
        return vx, vz, psi, acc_x, acc_z

    def _strain_rates(self, vx, vz, psi_in):
        dx, dz = self.dx, self.dz
        f = [dxm(vx, dx), dzm(vz, dz), dzp(vx, dz), dxp(vz, dx)]
        psi = [self.pml[4 + k][1] * psi_in[4 + k] + self.pml[4 + k][0] * f[k] for k in range(4)]
        Ex = f[0] + psi[0]
        Ez = f[1] + psi[1]
        Exz = f[2] + psi[2] + f[3] + psi[3]
        return Ex, Ez, Exz, psi

    def _das(self, U, vx, vz):
        """Update the running displacements U and return sample d^n of every trace."""
        dt, L = self.dt, self.gauge
        j, i, wt = self.das_j, self.das_i, self.das_wt
        vals = np.empty((self.ntr, 4))
        for k, f in enumerate((vx, vz, vx, vz)):
            vals[:, k] = np.sum(wt[:, k] * f[j[:, k], i[:, k]], axis=1)
        tx, tz = self.ch_t[:, 0], self.ch_t[:, 1]
        if self.acq.das_mode == STRAIN:
            U += dt * vals
            return (tx * (U[:, 0] - U[:, 2]) + tz * (U[:, 1] - U[:, 3])) / L
        if self.acq.das_mode == VELOCITY:
            return tx * vals[:, 0] + tz * vals[:, 1]
        return (tx * (vals[:, 0] - vals[:, 2]) + tz * (vals[:, 1] - vals[:, 3])) / L

    def step(self, st, n):
        """Advance the state x^n -> x^{n+1}; returns (new state, d^n, geophone samples)."""
        dt = self.dt
        vx, vz, psi_v, _, _ = self._velocity(st, n)
        U = st["U"].copy()
        d = self._das(U, vx, vz)
        geo = [(self._sample(vx, gx), self._sample(vz, gz)) for gx, gz in self.geo]
        Ex, Ez, Exz, psi_s = self._strain_rates(vx, vz, st["psi"])
        sxx = st["sxx"] + dt * (self.lam * (Ex + Ez) + 2.0 * self.mu * Ex)
        szz = st["szz"] + dt * (self.lam * (Ex + Ez) + 2.0 * self.mu * Ez)
        sxz = st["sxz"] + dt * self.muxz * Exz
        if self.force is None:
            dw = (self.wav[n + 1] - self.wav[n]) / (self.dx * self.dz)
            self._spread(sxx, self.inj_node, -self.M[0] * dw)
            self._spread(szz, self.inj_node, -self.M[1] * dw)
            self._spread(sxz, self.inj_xz, -self.M[2] * dw)
        new = {"vx": vx, "vz": vz, "sxx": sxx, "szz": szz, "sxz": sxz, "psi": psi_v + psi_s, "U": U}
        return new, d, geo

    # -- runs ------------------------------------------------------------------
    def forward(self, st0=None, keep_every=0):
        """Run nt steps. Returns data [ntr, nt], geophone data [k, 2, nt], checkpoints {n: x^n}."""
        nt = self.acq.nt
        st = self.zero_state() if st0 is None else self.copy_state(st0)
        d = np.zeros((self.ntr, nt))
        geo = np.zeros((len(self.geo), 2, nt))
        ck = {}
        for n in range(nt):
            if keep_every and n % keep_every == 0:
                ck[n] = self.copy_state(st)
            st, d[:, n], g = self.step(st, n)
            if self.geo:
                geo[:, :, n] = np.array(g)
        return d, geo, ck

    def zero_adjoint(self):
        return self.zero_state()

    def adjoint_step(self, adj, st, n, r_n, G, gw):
        """Transpose of step n (x^n -> x^{n+1}) applied to the adjoint state, in place.

        adj: adjoint of x^{n+1} on entry, of x^n on exit.  st: forward state x^n.
        r_n: residual sample n of every trace.  G: dict of zero-lag sums for
        lam, mu, muxz, bx, bz.  gw: gradient with respect to the wavelet.
        """
        dt, dx, dz = self.dt, self.dx, self.dz
        # forward intermediates of step n, recomputed from x^n
        vx, vz, _, acc_x, acc_z = self._velocity(st, n)
        Ex, Ez, Exz, _ = self._strain_rates(vx, vz, st["psi"])

        sxx_h, szz_h, sxz_h = adj["sxx"], adj["szz"], adj["sxz"]
        # source term: sigma^{n+1} -= M (w_{n+1} - w_n) delta_h
        if self.force is None:
            proj = (self.M[0] * self._sample(sxx_h, self.inj_node) + self.M[1] * self._sample(szz_h, self.inj_node)
                    + self.M[2] * self._sample(sxz_h, self.inj_xz)) / (dx * dz)
            gw[n + 1] -= proj
            gw[n] += proj

        # stress sub-step transposed
        Exh = dt * ((self.lam + 2.0 * self.mu) * sxx_h + self.lam * szz_h)
        Ezh = dt * (self.lam * sxx_h + (self.lam + 2.0 * self.mu) * szz_h)
        Exzh = dt * self.muxz * sxz_h
        G["lam"] += dt * (sxx_h + szz_h) * (Ex + Ez)
        G["mu"] += 2.0 * dt * (sxx_h * Ex + szz_h * Ez)
        G["muxz"] += dt * sxz_h * Exz
        fh = []
        for k, Eh in zip(range(4, 8), (Exh, Ezh, Exzh, Exzh)):
            a, b = self.pml[k]
            Psi = adj["psi"][k] + Eh
            fh.append(Eh + a * Psi)
            adj["psi"][k] = b * Psi
        adj["vx"] = adj["vx"] + dxm_T(fh[0], dx) + dzp_T(fh[2], dz)
        adj["vz"] = adj["vz"] + dzm_T(fh[1], dz) + dxp_T(fh[3], dx)

        # DAS sampling transposed
        if self.ntr:
            tx, tz = self.ch_t[:, 0], self.ch_t[:, 1]
            if self.acq.das_mode == VELOCITY:
                rc = np.asarray(r_n, np.float64)
                dd = np.stack([tx * rc, tz * rc, 0 * rc, 0 * rc], axis=1)
            else:
                rc = np.asarray(r_n, np.float64) / self.gauge
                dd = np.stack([tx * rc, tz * rc, -tx * rc, -tz * rc], axis=1)   # d d^n / d (U or v samples)
            if self.acq.das_mode == STRAIN:
                adj["U"] += dd
                val = dt * adj["U"]
            else:
                val = dd
            for k, name in enumerate(("vx", "vz", "vx", "vz")):
                np.add.at(adj[name], (self.das_j[:, k].ravel(), self.das_i[:, k].ravel()),
                          (self.das_wt[:, k] * val[:, k:k + 1]).ravel())

        # velocity sub-step transposed
        vx_h, vz_h = adj["vx"], adj["vz"]
        if self.force is not None:
            wn = 1.0 / (dx * dz)
            gw[n] += self.force[0] * wn * sum(wt * dt * self.bx[j, i] * vx_h[j, i] for j, i, wt in self.inj_vx)
            gw[n] += self.force[1] * wn * sum(wt * dt * self.bz[j, i] * vz_h[j, i] for j, i, wt in self.inj_vz)
        G["bx"] += vx_h * dt * acc_x
        G["bz"] += vz_h * dt * acc_z
        if self.force is not None:          # the force term dt b F w_n delta_h depends on b too
            wn = self.wav[n] / (dx * dz)
            for j, i, wt in self.inj_vx:
                G["bx"][j, i] += vx_h[j, i] * dt * self.force[0] * wn * wt
            for j, i, wt in self.inj_vz:
                G["bz"][j, i] += vz_h[j, i] * dt * self.force[1] * wn * wt
        qx = dt * self.bx * vx_h
        qz = dt * self.bz * vz_h
        eh = []
        for k, q in zip(range(4), (qx, qx, qz, qz)):
            a, b = self.pml[k]
            Psi = adj["psi"][k] + q
            eh.append(q + a * Psi)
            adj["psi"][k] = b * Psi
        adj["sxx"] = sxx_h + dxp_T(eh[0], dx)
        adj["sxz"] = sxz_h + dzm_T(eh[1], dz) + dxm_T(eh[2], dx)
        adj["szz"] = szz_h + dzp_T(eh[3], dz)

    def adjoint(self, residual, st0=None, block=None):
        """Backpropagate residual [ntr, nt] through all steps.

        Forward states are kept every ``block`` steps and recomputed inside each
        block (a deterministic recompute: identical to storing every state).
        Returns (G dict on the padded grid, adjoint of x^0, wavelet gradient).
        """
        nt = self.acq.nt
        if block is None:
            block = max(1, int(np.ceil(np.sqrt(nt))))
        _, _, ck = self.forward(st0, keep_every=block)
        shape = (self.NZ, self.NX)
        G = {k: np.zeros(shape) for k in ("lam", "mu", "muxz", "bx", "bz")}
        gw = np.zeros(nt + 1)
        adj = self.zero_adjoint()
        starts = sorted(ck)
        for b0 in reversed(starts):
            b1 = min(b0 + block, nt)
            states = [ck[b0]]
            for n in range(b0, b1 - 1):
                states.append(self.step(states[-1], n)[0])
            for n in range(b1 - 1, b0 - 1, -1):
                self.adjoint_step(adj, states[n - b0], n, residual[:, n], G, gw)
        return G, adj, gw

    def chain_rule(self, G):
        """Map zero-lag sums for (lambda, mu, mu_xz, b_x, b_z) to (Vp, Vs, rho) on the physical window.

        lambda = rho (Vp^2 - 2 Vs^2), mu = rho Vs^2; d mu_xz / d mu_k = mu_xz^2 / (4 mu_k^2);
        d b / d rho_k = -1 / (2 rho_k^2) for each of the two nodes a buoyancy point averages.
        """
        P, NX, NZ = self.P, self.NX, self.NZ
        vp, vs, rho, mu = self.vp, self.vs, self.rho, self.mu
        dlam = G["lam"].copy()
        dmu = G["mu"].copy()
        drho = np.zeros((NZ, NX))
        t = G["muxz"] * self.muxz ** 2 / 4.0
        gbx, gbz = G["bx"], G["bz"]
        for j in range(1, NZ - 1):
            for i in range(1, NX - 1):
                dmu[j, i] += (t[j, i] + t[j, i - 1] + t[j - 1, i] + t[j - 1, i - 1]) / mu[j, i] ** 2
                drho[j, i] = -0.5 / rho[j, i] ** 2 * (gbx[j, i] + gbx[j, i - 1] + gbz[j, i] + gbz[j - 1, i])
        g_vp = dlam * 2.0 * rho * vp
        g_vs = 2.0 * rho * vs * (dmu - 2.0 * dlam)
        g_rho = dlam * (vp ** 2 - 2.0 * vs ** 2) + dmu * vs ** 2 + drho
        sl = (slice(P, P + self.acq.nz), slice(P, P + self.w))
        return g_vp[sl], g_vs[sl], g_rho[sl]


# ---------------------------------------------------------------------------
# Whole-problem entry points (all shots, extended model)
# ---------------------------------------------------------------------------

def _split(acq, d):
    return [d[acq.tr_ptr[s]:acq.tr_ptr[s + 1]] for s in range(acq.ns)]


def forward(acq, vp, vs, rho, shots=None):
    """Modelled DAS data d[Ntr, nt] of the extended model (vp, vs, rho: [Ns, nz, nx]).

    Shot s uses its own component m_s (first term of eq. 8).
    """
    d = np.zeros((acq.ntr, acq.nt))
    for s in (range(acq.ns) if shots is None else shots):
        a, b = acq.tr_ptr[s], acq.tr_ptr[s + 1]
        d[a:b] = Shot(acq, s, vp[s], vs[s], rho[s]).forward()[0]
    return d


def misfit(d, d_obs):
    """phi = 1/2 sum (d - d_obs)^2 over every shot, trace and sample (eq. 4)."""
    r = np.asarray(d, np.float64) - np.asarray(d_obs, np.float64)
    return 0.5 * float(np.sum(r * r))


def gradient(acq, vp, vs, rho, d_obs, shots=None, block=None):
    """phi_data and the per-component gradients g_s (eq. 6 applied to each m_s).

    Returns (phi, g_vp, g_vs, g_rho) with g_* of shape [Ns, nz, nx]; cells outside
    a shot's window get zero.
    """
    g = [np.zeros((acq.ns, acq.nz, acq.nx)) for _ in range(3)]
    phi = 0.0
    win = acq.windows()
    for s in (range(acq.ns) if shots is None else shots):
        a, b = acq.tr_ptr[s], acq.tr_ptr[s + 1]
        sh = Shot(acq, s, vp[s], vs[s], rho[s])
        d = sh.forward()[0]
        r = d - np.asarray(d_obs[a:b], np.float64)
        phi += 0.5 * float(np.sum(r * r))
        G, _, _ = sh.adjoint(r, block=block)
        x0, w = win[s]
        for k, gk in enumerate(sh.chain_rule(G)):
            g[k][s, :, x0:x0 + w] = gk
    return phi, g[0], g[1], g[2]
