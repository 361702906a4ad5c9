"""Seeded synthetic inputs for the source-extended elastic FWI hot path.

This module only *describes* problems: grids, layered elastic models, source
positions, moment tensors, source time functions (Ricker), DAS fibre geometry,
per-shot windows and zone-of-influence parameters.  It holds none of the
method's arithmetic (no wave propagation, no misfit, no gradient, no
regularization); both the FP64 oracle (``oracle/``) and the CUDA library
(``paper_2305_14130_gb300``) consume what it returns.

The paper's own synthetic geometry and field data are not available, so the
workloads below stand in for them with the paper's shapes: a low-velocity
waveguide layer, sources inside the layer on a horizontal well, a DAS fibre
with 1 m channel spacing and a 10 m gauge on a parallel well (Synthetic
examples section, Table 1; field-data section).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

STRAIN = 0        # gauge-averaged axial strain (running displacement)
STRAIN_RATE = 1   # gauge-averaged axial strain rate (velocity)
VELOCITY = 2      # particle-velocity receiver: one trace per component t, value t.v(p)


@dataclass
class Acquisition:
    """Plain container for one shot-batched problem (SI units, metres/seconds).

    Positions are metres in the physical grid frame: node (ix, iz) sits at
    (ix*dx, iz*dz).  Arrays are float64 unless noted.
    """
    nx: int
    nz: int
    dx: float
    dz: float
    nt: int
    dt: float
    src_xz: np.ndarray            # [Ns, 2]
    mt: np.ndarray                # [Ns, 3]  (Mxx, Mzz, Mxz)
    wavelet: np.ndarray           # [Ns, nt+1] source time function at t_n = n*dt
    tr_ptr: np.ndarray            # [Ns+1] int32, traces of shot s: tr_ptr[s]..tr_ptr[s+1]-1
    ch_xz: np.ndarray             # [Ntr, 2] gauge centres
    ch_t: np.ndarray              # [Ntr, 2] unit tangents
    gauge: float                  # gauge length L (m)
    ref_vp: np.ndarray            # [nz, nx] frozen reference model (absorbing-layer material)
    ref_vs: np.ndarray
    ref_rho: np.ndarray
    win: Optional[np.ndarray] = None  # [Ns, 2] int32 (x0, width) in cells; None = full grid
    das_mode: int = STRAIN
    npml: int = 20
    pml_R: float = 1e-3
    pml_vmax: float = 0.0         # 0 -> max of reference Vp
    pml_f0: float = 0.0           # dominant frequency used for the CPML alpha profile
    force: Optional[np.ndarray] = None  # [Ns, 2] vector force (Fx, Fz); replaces the moment tensor

    @property
    def ns(self) -> int:
        return int(self.src_xz.shape[0])

    @property
    def ntr(self) -> int:
        return int(self.ch_xz.shape[0])

    def windows(self) -> np.ndarray:
        if self.win is None:
            w = np.zeros((self.ns, 2), np.int32)
            w[:, 1] = self.nx
            return w
        return np.asarray(self.win, np.int32)

    def vmax(self) -> float:
        return float(self.pml_vmax) if self.pml_vmax > 0 else float(self.ref_vp.max())


@dataclass
class ZOI:
    """Zone-of-influence parameters per shot (eq. 10 of the paper).

    active_x: [Ns, 2] x-span (m) where the outer weight is 1; taper: [Ns]
    outer taper width (m); sink_xz: [Ns, 2] sinkhole centres (m);
    sink_ax, sink_az: [Ns] ellipse semi-axes (m); n: stiffness exponent;
    nu: height parameter in (0, 1).
    """
    active_x: np.ndarray
    taper: np.ndarray
    sink_xz: np.ndarray
    sink_ax: np.ndarray
    sink_az: np.ndarray
    n: float = 2.0
    nu: float = 0.99


@dataclass
class Problem:
    name: str
    acq: Acquisition
    vp: np.ndarray      # [Ns, nz, nx] extended starting model (float64)
    vs: np.ndarray
    rho: np.ndarray
    true_vp: Optional[np.ndarray] = None   # [nz, nx] model that generates observed data
    true_vs: Optional[np.ndarray] = None
    true_rho: Optional[np.ndarray] = None
    zoi: Optional[ZOI] = None
    eta: tuple = (1.0, 1.0, 1.0)
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# Source time function and moment tensors (inputs to the method)
# ----------------------------------------------------------------------------

def ricker(f0: float, nt: int, dt: float, shift: float = 0.0, t0: Optional[float] = None) -> np.ndarray:
    """Ricker wavelet sampled at t_n = n*dt, n = 0..nt (nt+1 samples).

    w(t) = (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0 - shift,
    t0 = 1.5/f0 by default (|w(0)| ~ 1e-8).
    """
    if t0 is None:
        t0 = 1.5 / f0
    t = np.arange(nt + 1, dtype=np.float64) * dt
    tau = t - t0 - shift
    a = (np.pi * f0 * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def rotate_mt(mxx: float, mzz: float, mxz: float, theta: float) -> tuple:
    """R M R^T for a 2x2 symmetric moment tensor and a rotation by theta (rad)."""
    c, s = np.cos(theta), np.sin(theta)
    R = np.array([[c, -s], [s, c]])
    M = np.array([[mxx, mxz], [mxz, mzz]])
    Mr = R @ M @ R.T
    return float(Mr[0, 0]), float(Mr[1, 1]), float(Mr[0, 1])


# ----------------------------------------------------------------------------
# Models
# ----------------------------------------------------------------------------

def smooth_random_field(shape, corr_cells: float, seed: int, amp: float) -> np.ndarray:
    """Gaussian-smoothed white noise, scaled to max |.| = amp (seeded)."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    f = gaussian_filter(rng.standard_normal(shape), corr_cells, mode="reflect")
    return amp * f / np.abs(f).max()


def waveguide_model(nx, nz, dz, top=(4500.0, 2600.0, 2500.0), layer=(3600.0, 2000.0, 2350.0),
                    z_top=135.0, thickness=30.0, pert=0.03, corr_m=20.0, dx=1.0, seeds=(1, 2)):
    """Low-velocity shale layer between two faster layers plus a +-3 % random field."""
    z = np.arange(nz) * dz
    inside = (z >= z_top) & (z < z_top + thickness)
    vp = np.where(inside, layer[0], top[0])[:, None] * np.ones((1, nx))
    vs = np.where(inside, layer[1], top[1])[:, None] * np.ones((1, nx))
    rho = np.where(inside, layer[2], top[2])[:, None] * np.ones((1, nx))
    if pert > 0:
        corr = corr_m / dx
        vp = vp * (1.0 + smooth_random_field((nz, nx), corr, seeds[0], pert))
        vs = vs * (1.0 + smooth_random_field((nz, nx), corr, seeds[1], pert))
    return vp, vs, rho


def random_layered_model(nx, nz, seed=0, vp_range=(3000.0, 5000.0), rho_range=(2000.0, 2600.0),
                         nlayers_range=(4, 8)):
    rng = np.random.default_rng(seed)
    nl = int(rng.integers(nlayers_range[0], nlayers_range[1] + 1))
    cuts = np.sort(rng.choice(np.arange(4, nz - 4), nl - 1, replace=False))
    bounds = np.concatenate([[0], cuts, [nz]])
    vp = np.empty((nz, nx)); rho = np.empty((nz, nx))
    for k in range(nl):
        vp[bounds[k]:bounds[k + 1]] = rng.uniform(*vp_range)
        rho[bounds[k]:bounds[k + 1]] = rng.uniform(*rho_range)
    vs = vp / 1.8
    return vp, vs, rho


def gaussian_bump(nx, nz, ic, jc, hx, hz):
    i = np.arange(nx)[None, :]
    j = np.arange(nz)[:, None]
    return np.exp(-((i - ic) / hx) ** 2 - ((j - jc) / hz) ** 2)


def extend(m: np.ndarray, ns: int) -> np.ndarray:
    return np.repeat(np.asarray(m, np.float64)[None], ns, axis=0).copy()


def extend_view(m: np.ndarray, ns: int) -> np.ndarray:
    """[ns, nz, nx] read-only view of one model (no copy): the starting extended
    model of the large workloads, where a copy per component would take GBs."""
    m = np.asarray(m, np.float64)
    return np.broadcast_to(m[None], (ns,) + m.shape)


def horizontal_fibre(x_first, n, spacing, z):
    ch = np.stack([x_first + spacing * np.arange(n), np.full(n, float(z))], axis=1)
    t = np.tile(np.array([[1.0, 0.0]]), (n, 1))
    return ch, t


def same_traces_per_shot(ns, ch, t):
    ntr = ch.shape[0]
    tr_ptr = (np.arange(ns + 1) * ntr).astype(np.int32)
    return tr_ptr, np.tile(ch, (ns, 1)), np.tile(t, (ns, 1))


def default_zoi(acq: Acquisition, taper_m: float, sink_ax: float, sink_az: float, n=2.0, nu=0.99) -> ZOI:
    ns = acq.ns
    act = np.zeros((ns, 2))
    for s in range(ns):
        a, b = acq.tr_ptr[s], acq.tr_ptr[s + 1]
        xs = np.concatenate([acq.ch_xz[a:b, 0], [acq.src_xz[s, 0]]])
        act[s] = (xs.min(), xs.max())
    return ZOI(active_x=act, taper=np.full(ns, taper_m), sink_xz=acq.src_xz.copy(),
               sink_ax=np.full(ns, sink_ax), sink_az=np.full(ns, sink_az), n=n, nu=nu)


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

def single_shot_200x100() -> Problem:
    """Single explosive shot, 200x100 grid, dx=2 m, two layers, nt=1000, dt=0.2 ms.

    Source at grid (100, 50), 100 Hz Ricker; 80 horizontal DAS channels at grid
    row 60 (z=120 m), 1 m spacing, 8 m gauge.  Observed data come from the same
    model with a +5 % Vs Gaussian anomaly of 20x10 cells (centre seeded, rng 0).
    """
    nx, nz, dx = 200, 100, 2.0
    nt, dt, f0 = 1000, 2e-4, 100.0
    top = np.array([4000.0, 2300.0, 2500.0])
    vp = np.full((nz, nx), top[0]); vs = np.full((nz, nx), top[1]); rho = np.full((nz, nx), top[2])
    vp[75:] *= 1.1; vs[75:] *= 1.1; rho[75:] *= 1.1
    rng = np.random.default_rng(0)
    ic = rng.uniform(80, 120); jc = rng.uniform(52, 58)
    tvs = vs * (1.0 + 0.05 * gaussian_bump(nx, nz, ic, jc, 10.0, 5.0))
    ch, t = horizontal_fibre(160.0, 80, 1.0, 60 * dx)
    tr_ptr, chs, ts = same_traces_per_shot(1, ch, t)
    acq = Acquisition(nx=nx, nz=nz, dx=dx, dz=dx, nt=nt, dt=dt,
                      src_xz=np.array([[100 * dx, 50 * dx]]), mt=np.array([[1e6, 1e6, 0.0]]),
                      wavelet=ricker(f0, nt, dt)[None], tr_ptr=tr_ptr, ch_xz=chs, ch_t=ts,
                      gauge=8.0, ref_vp=vp, ref_vs=vs, ref_rho=rho, pml_f0=f0)
    return Problem("single_shot_200x100", acq, extend(vp, 1), extend(vs, 1), extend(rho, 1),
                   true_vp=vp.copy(), true_vs=tvs, true_rho=rho.copy(),
                   meta={"anomaly_centre": (ic, jc)})


def guided_wave_1000x300(ns: int = 32, nt: int = 4000, nch: int = 500) -> Problem:
    """Guided-wave extended FWI: 1000x300 grid, dx=1 m, 30 m shale waveguide.

    Vp/Vs/rho 3600/2000/2350 inside 4500/2600/2500 with +-3 % smoothed random
    perturbations (corr. 20 m, seeds 1 and 2); 32 diagonal moment-tensor sources
    (M33/M11 = 0.75) at z=150 m, x = 252 + 16k m; 150 Hz Ricker; 500 DAS
    channels at z=190 m (1 m spacing, 10 m gauge); nt=4000, dt=0.1 ms.
    Observed data: a +4 % Vp / +6 % Vs Gaussian anomaly in the layer.
    """
    nx, nz, dx = 1000, 300, 1.0
    dt, f0 = 1e-4, 150.0
    vp, vs, rho = waveguide_model(nx, nz, dx, dx=dx)
    xs = 252.0 + 16.0 * np.arange(ns) * (32 / ns)
    src = np.stack([xs, np.full(ns, 150.0)], axis=1)
    mt = np.tile(np.array([[1e6, 0.75e6, 0.0]]), (ns, 1))
    ch, t = horizontal_fibre(250.0, nch, 1.0 * (500 / nch), 190.0)
    tr_ptr, chs, ts = same_traces_per_shot(ns, ch, t)
    wav = np.tile(ricker(f0, nt, dt)[None], (ns, 1))
    bump = gaussian_bump(nx, nz, 520, 150, 40, 10)
    acq = Acquisition(nx=nx, nz=nz, dx=dx, dz=dx, nt=nt, dt=dt, src_xz=src, mt=mt, wavelet=wav,
                      tr_ptr=tr_ptr, ch_xz=chs, ch_t=ts, gauge=10.0,
                      ref_vp=vp, ref_vs=vs, ref_rho=rho, pml_f0=f0)
    zoi = default_zoi(acq, taper_m=50.0, sink_ax=12.0, sink_az=6.0)
    return Problem("guided_wave_1000x300", acq, extend(vp, ns), extend(vs, ns), extend(rho, ns),
                   true_vp=vp * (1 + 0.04 * bump), true_vs=vs * (1 + 0.06 * bump), true_rho=rho.copy(),
                   zoi=zoi, eta=(1e-3, 1e-3, 1e-3))


def random_layered_128(ns: int = 4, nt: int = 600) -> Problem:
    """128x128 dx=2 m random-layered model (seed 0), 4 shots, nt=600, dt=0.2 ms."""
    nx = nz = 128
    dx, dt, f0 = 2.0, 2e-4, 50.0
    vp, vs, rho = random_layered_model(nx, nz, seed=0)
    xs = np.linspace(40.0, 216.0, ns)
    src = np.stack([xs, np.full(ns, 120.0)], axis=1)
    mt = np.tile(np.array([[1e6, 0.75e6, 2e5]]), (ns, 1))
    ch, t = horizontal_fibre(30.0, 100, 2.0, 170.0)
    tr_ptr, chs, ts = same_traces_per_shot(ns, ch, t)
    wav = np.tile(ricker(f0, nt, dt)[None], (ns, 1))
    acq = Acquisition(nx=nx, nz=nz, dx=dx, dz=dx, nt=nt, dt=dt, src_xz=src, mt=mt, wavelet=wav,
                      tr_ptr=tr_ptr, ch_xz=chs, ch_t=ts, gauge=10.0,
                      ref_vp=vp, ref_vs=vs, ref_rho=rho, pml_f0=f0)
    bump = gaussian_bump(nx, nz, 64, 64, 12, 8)
    return Problem("random_layered_128", acq, extend(vp, ns), extend(vs, ns), extend(rho, ns),
                   true_vp=vp * (1 + 0.03 * bump), true_vs=vs * (1 + 0.05 * bump), true_rho=rho * (1 + 0.02 * bump),
                   zoi=default_zoi(acq, taper_m=40.0, sink_ax=16.0, sink_az=10.0))


def uneven_windows(nx: int, nz: int, dx: float, dt: float, ns: int, nt: int, wmin: int, wmax: int, z_top: float,
                   z_src: float, z_fib: float, seed: int = 0, name: str = "uneven_windows") -> Problem:
    """Waveguide with every shot on its own cropped window of uneven width.

    Window widths uniform in [wmin, wmax] cells (seeded), each centred on its
    shot (clipped to the grid); channels are the fibre channels inside the
    window.  150 Hz Ricker.
    """
    f0 = 150.0
    vp, vs, rho = waveguide_model(nx, nz, dx, z_top=z_top, thickness=30.0, dx=dx)
    rng = np.random.default_rng(seed)
    widths = rng.integers(wmin, wmax + 1, ns)
    xs = np.linspace(0.2 * nx * dx, 0.8 * nx * dx, ns)
    src = np.stack([xs, np.full(ns, z_src)], axis=1)
    mt = np.tile(np.array([[1e6, 0.75e6, 0.0]]), (ns, 1))
    fib, ft = horizontal_fibre(dx * 2, int((nx - 4) * dx), 1.0, z_fib)
    win = np.zeros((ns, 2), np.int32)
    chs, tts, ptr = [], [], [0]
    for s in range(ns):
        c = int(round(xs[s] / dx))
        x0 = int(np.clip(c - widths[s] // 2, 0, nx - widths[s]))
        win[s] = (x0, widths[s])
        lo, hi = (x0 + 8) * dx, (x0 + widths[s] - 9) * dx
        keep = (fib[:, 0] - 5.0 >= lo) & (fib[:, 0] + 5.0 <= hi)
        chs.append(fib[keep]); tts.append(ft[keep]); ptr.append(ptr[-1] + int(keep.sum()))
    wav = np.tile(ricker(f0, nt, dt)[None], (ns, 1))
    acq = Acquisition(nx=nx, nz=nz, dx=dx, dz=dx, nt=nt, dt=dt, src_xz=src, mt=mt, wavelet=wav,
                      tr_ptr=np.array(ptr, np.int32), ch_xz=np.concatenate(chs), ch_t=np.concatenate(tts),
                      gauge=10.0, ref_vp=vp, ref_vs=vs, ref_rho=rho, win=win, pml_f0=f0)
    bump = gaussian_bump(nx, nz, nx // 2, int(round((z_top + 15.0) / dx)), nx // 20 + 2, 8)
    return Problem(name, acq, extend_view(vp, ns), extend_view(vs, ns), extend_view(rho, ns),
                   true_vp=vp * (1 + 0.04 * bump), true_vs=vs * (1 + 0.06 * bump), true_rho=rho.copy())


def uneven_windows_3000x800(ns: int = 96, nt: int = 4000, seed: int = 0) -> Problem:
    """3000x800 dx=0.75 m waveguide, 96 shots each on its own cropped window.

    Window widths uniform in [600, 1800] cells (seeded); layer at 270-300 m,
    sources at 300 m, fibre at 340 m; dt = 0.075 ms.
    """
    return uneven_windows(3000, 800, 0.75, 7.5e-5, ns, nt, 600, 1800, z_top=270.0, z_src=300.0, z_fib=340.0, seed=seed,
                          name="uneven_windows_3000x800")


def uneven_windows_subset_256x128(ns: int = 6, nt: int = 500, seed: int = 0) -> Problem:
    """256x128 parity subset of the uneven-window configuration: same dx, layer
    thickness, source-fibre offset (40 m) and width distribution scaled to the
    grid (widths uniform in [51, 153] cells); layer at 33-63 m, sources at 48 m,
    fibre at 88 m."""
    return uneven_windows(256, 128, 0.75, 7.5e-5, ns, nt, 51, 153, z_top=33.0, z_src=48.0, z_fib=88.0, seed=seed,
                          name="uneven_windows_subset_256x128")


def tiny(nx=24, nz=20, ns=2, nt=40, dx=5.0, dt=5e-4, npml=4, das_mode=STRAIN, win=None, seed=0,
         heterogeneous=True, nch=6) -> Problem:
    """A few-hundred-cell problem for oracle self-tests (FD gradients, dot tests)."""
    rng = np.random.default_rng(seed)
    vp = 3000.0 + (400.0 * rng.random((nz, nx)) if heterogeneous else 0.0)
    vs = vp / 1.8
    rho = 2200.0 + (200.0 * rng.random((nz, nx)) if heterogeneous else 0.0)
    vp = np.broadcast_to(vp, (nz, nx)).astype(np.float64)
    vs = np.broadcast_to(vs, (nz, nx)).astype(np.float64)
    rho = np.broadcast_to(rho, (nz, nx)).astype(np.float64)
    xs = np.linspace(0.3 * nx * dx, 0.6 * nx * dx, ns) + 0.37 * dx
    src = np.stack([xs, np.full(ns, 0.45 * nz * dx + 0.21 * dx)], axis=1)
    mt = np.stack([np.full(ns, 1e6), np.full(ns, 0.75e6), np.full(ns, 3e5)], axis=1)
    ch = np.stack([np.linspace(0.25 * nx * dx, 0.7 * nx * dx, nch), np.full(nch, 0.7 * nz * dx + 0.3 * dx)], axis=1)
    ang = np.linspace(0.0, 0.8, nch)
    t = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    if win is None:
        tr_ptr, chs, ts = same_traces_per_shot(ns, ch, t)
    else:
        # keep, per shot, the channels whose gauge ends lie inside its window
        chs, ts, ptr = [], [], [0]
        for s in range(ns):
            x0, w = win[s]
            ends = np.concatenate([ch - 0.5 * 2.5 * dx * t, ch + 0.5 * 2.5 * dx * t])[:, 0] / dx
            ok = np.all(((ends >= x0) & (ends <= x0 + w - 1)).reshape(2, -1), axis=0)
            chs.append(ch[ok]); ts.append(t[ok]); ptr.append(ptr[-1] + int(ok.sum()))
        tr_ptr, chs, ts = np.array(ptr, np.int32), np.concatenate(chs), np.concatenate(ts)
    f0 = 0.08 / dt
    wav = np.stack([ricker(f0, nt, dt, shift=0.1 * s / f0) for s in range(ns)])
    acq = Acquisition(nx=nx, nz=nz, dx=dx, dz=dx, nt=nt, dt=dt, src_xz=src, mt=mt, wavelet=wav,
                      tr_ptr=tr_ptr, ch_xz=chs, ch_t=ts, gauge=2.5 * dx, ref_vp=vp.copy(),
                      ref_vs=vs.copy(), ref_rho=rho.copy(), das_mode=das_mode, npml=npml, pml_f0=f0,
                      win=win)
    rng2 = np.random.default_rng(seed + 100)
    ext_vp = extend(vp, ns) * (1 + 0.02 * rng2.standard_normal((ns, nz, nx)))
    ext_vs = extend(vs, ns) * (1 + 0.02 * rng2.standard_normal((ns, nz, nx)))
    ext_rho = extend(rho, ns) * (1 + 0.02 * rng2.standard_normal((ns, nz, nx)))
    return Problem("tiny", acq, ext_vp, ext_vs, ext_rho, true_vp=vp, true_vs=vs, true_rho=rho,
                   zoi=default_zoi(acq, taper_m=3 * dx, sink_ax=3 * dx, sink_az=2 * dx))


def with_forces(p: Problem, angle_deg: float = 30.0, amplitude: float = 1e6) -> Problem:
    """The same problem driven by vector-force sources (eq. 2, second case) at the
    source positions instead of moment tensors: F_s of the given amplitude, its
    direction rotated by angle_deg * s from vertical."""
    a = p.acq
    ang = np.deg2rad(angle_deg) * np.arange(a.ns)
    f = amplitude * np.stack([np.sin(ang), np.cos(ang)], axis=1)
    return replace(p, acq=replace(a, force=f))


def two_component(p: Problem) -> Problem:
    """The same problem recorded by 2-C particle-velocity receivers at the
    channel positions instead of DAS gauges: every channel becomes two traces,
    horizontal (t = (1, 0)) then vertical (t = (0, 1))."""
    a = p.acq
    ptr, xz, t = [0], [], []
    for s in range(a.ns):
        lo, hi = int(a.tr_ptr[s]), int(a.tr_ptr[s + 1])
        for c in range(lo, hi):
            xz += [a.ch_xz[c], a.ch_xz[c]]
            t += [(1.0, 0.0), (0.0, 1.0)]
        ptr.append(ptr[-1] + 2 * (hi - lo))
    acq = replace(a, tr_ptr=np.array(ptr, np.int32), ch_xz=np.array(xz, np.float64).reshape(-1, 2),
                  ch_t=np.array(t, np.float64).reshape(-1, 2), das_mode=VELOCITY)
    return replace(p, acq=acq)


def with_windows(p: Problem, win) -> Problem:
    return replace(p, acq=replace(p.acq, win=np.asarray(win, np.int32)))


def seeded_data(shape, seed, scale=1.0):
    """Seeded synthetic 'observed' traces for parity cases that need any d_obs."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(shape)


def differentiation_2000x600(ns: int = 64, nt: int = 6000, nch: int = 500) -> Problem:
    """Differentiation-path workload at scale: 2000x600 grid, dx=1 m, the
    random-layered model (seed 0, Vp 3000-5000 m/s, Vs = Vp/1.8, 4-8 layers),
    64 moment-tensor sources at z=300 m spread over x = 200-1800 m, 500 DAS
    channels at z=340 m (1 m spacing, 10 m gauge, centred), 150 Hz Ricker,
    nt=6000, dt=0.1 ms.  Observed data: a +3 % Vp / +5 % Vs / +2 % rho Gaussian
    anomaly between the source line and the fibre."""
    nx, nz, dx = 2000, 600, 1.0
    dt, f0 = 1e-4, 150.0
    vp, vs, rho = random_layered_model(nx, nz, seed=0)
    xs = np.linspace(200.0, 1800.0, ns) + 0.37
    src = np.stack([xs, np.full(ns, 300.0)], axis=1)
    mt = np.tile(np.array([[1e6, 0.75e6, 2e5]]), (ns, 1))
    ch, t = horizontal_fibre(1000.0 - nch / 2, nch, 1.0, 340.0)
    tr_ptr, chs, ts = same_traces_per_shot(ns, ch, t)
    wav = np.tile(ricker(f0, nt, dt)[None], (ns, 1))
    acq = Acquisition(nx=nx, nz=nz, dx=dx, dz=dx, nt=nt, dt=dt, src_xz=src, mt=mt, wavelet=wav,
                      tr_ptr=tr_ptr, ch_xz=chs, ch_t=ts, gauge=10.0,
                      ref_vp=vp, ref_vs=vs, ref_rho=rho, pml_f0=f0)
    bump = gaussian_bump(nx, nz, 1000, 320, 60, 12)
    return Problem("differentiation_2000x600", acq, extend_view(vp, ns), extend_view(vs, ns), extend_view(rho, ns),
                   true_vp=vp * (1 + 0.03 * bump), true_vs=vs * (1 + 0.05 * bump), true_rho=rho * (1 + 0.02 * bump),
                   zoi=default_zoi(acq, taper_m=50.0, sink_ax=12.0, sink_az=6.0), eta=(1e-3, 1e-3, 1e-3))


def full_iteration_4000x1200(ns: int = 128, nt: int = 8000, nch: int = 1500, seed: int = 0) -> Problem:
    """Full extended-FWI iteration at scale: 4000x1200 grid, dx=0.5 m, the
    waveguide (30 m shale layer at 285-315 m, +-3 % random fields with a 20 m
    correlation length), 128 perforation-like moment-tensor sources on a
    horizontal well in the layer (z=300 m, x = 200-1800 m), 1500 DAS channels at
    z=340 m (0.5 m spacing, 10 m gauge, centred), 150 Hz Ricker, nt=8000,
    dt=0.05 ms.

    The acquisition carries the modelled sources, with seeded source errors
    (rng(seed)): amplitude x U(0.9, 1.1), time shift U(-0.2, 0.2) ms and a
    mechanism rotation U(-15, 15) degrees (R M R^T).  The error-free sources
    that generate the observed data are in meta["true_mt"] and
    meta["true_wavelet"]; the observed data also see a +4 % Vp / +6 % Vs
    Gaussian anomaly in the layer.
    """
    nx, nz, dx = 4000, 1200, 0.5
    dt, f0 = 5e-5, 150.0
    vp, vs, rho = waveguide_model(nx, nz, dx, z_top=285.0, thickness=30.0, dx=dx)
    xs = np.linspace(200.0, 1800.0, ns) + 0.13
    src = np.stack([xs, np.full(ns, 300.0)], axis=1)
    mt_true = np.tile(np.array([[1e6, 0.75e6, 0.0]]), (ns, 1))
    wav_true = np.tile(ricker(f0, nt, dt)[None], (ns, 1))
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.9, 1.1, ns)
    shift = rng.uniform(-2e-4, 2e-4, ns)
    theta = np.deg2rad(rng.uniform(-15.0, 15.0, ns))
    mt = np.array([rotate_mt(*(amp[s] * mt_true[s]), theta[s]) for s in range(ns)])
    wav = np.stack([ricker(f0, nt, dt, shift=shift[s]) for s in range(ns)])
    ch, t = horizontal_fibre(1000.0 - 0.25 * nch, nch, 0.5, 340.0)
    tr_ptr, chs, ts = same_traces_per_shot(ns, ch, t)
    acq = Acquisition(nx=nx, nz=nz, dx=dx, dz=dx, nt=nt, dt=dt, src_xz=src, mt=mt, wavelet=wav,
                      tr_ptr=tr_ptr, ch_xz=chs, ch_t=ts, gauge=10.0,
                      ref_vp=vp, ref_vs=vs, ref_rho=rho, pml_f0=f0)
    bump = gaussian_bump(nx, nz, 2000, 600, 80, 20)
    return Problem("full_iteration_4000x1200", acq, extend_view(vp, ns), extend_view(vs, ns), extend_view(rho, ns),
                   true_vp=vp * (1 + 0.04 * bump), true_vs=vs * (1 + 0.06 * bump), true_rho=rho.copy(),
                   zoi=default_zoi(acq, taper_m=50.0, sink_ax=12.0, sink_az=6.0), eta=(1e-3, 1e-3, 1e-3),
                   meta={"true_mt": mt_true, "true_wavelet": wav_true, "amplitude": amp, "shift_s": shift,
                         "rotation_rad": theta})


def shot_subset(p: Problem, shots) -> Problem:
    """The problem restricted to the given shots (their traces, windows and
    extended-model components)."""
    a = p.acq
    shots = [int(s) for s in shots]
    ptr, idx = [0], []
    for s in shots:
        lo, hi = int(a.tr_ptr[s]), int(a.tr_ptr[s + 1])
        idx.extend(range(lo, hi))
        ptr.append(ptr[-1] + hi - lo)
    idx = np.asarray(idx, np.int64)
    sel = lambda v: None if v is None else np.asarray(v)[shots]
    acq = replace(a, src_xz=a.src_xz[shots], mt=a.mt[shots], wavelet=np.asarray(a.wavelet)[shots],
                  tr_ptr=np.asarray(ptr, np.int32), ch_xz=a.ch_xz[idx].reshape(-1, 2), ch_t=a.ch_t[idx].reshape(-1, 2),
                  win=sel(a.win), force=sel(a.force))
    meta = dict(p.meta)
    meta["shots"] = shots
    meta["traces"] = idx
    for k in ("true_mt", "true_wavelet"):
        if k in meta:
            meta[k] = np.asarray(meta[k])[shots]
    zoi = None
    if p.zoi is not None:
        z = p.zoi
        zoi = replace(z, active_x=z.active_x[shots], taper=z.taper[shots], sink_xz=z.sink_xz[shots],
                      sink_ax=z.sink_ax[shots], sink_az=z.sink_az[shots])
    return replace(p, acq=acq, vp=p.vp[shots], vs=p.vs[shots], rho=p.rho[shots], zoi=zoi, meta=meta)


def oracle_window(p: Problem, shot: int, x0: int, w: int) -> Problem:
    """One shot of p on the cropped window [x0, x0 + w) of its grid, keeping
    only the traces whose gauge ends lie inside it: an early-time stand-in for
    the full grid (identical until waves reach the window's edge)."""
    q = shot_subset(p, [shot])
    a = q.acq
    half = 0.5 * a.gauge * a.ch_t
    ends = np.concatenate([a.ch_xz - half, a.ch_xz + half])[:, 0] / a.dx
    ok = np.all(((ends >= x0 + 1) & (ends <= x0 + w - 2)).reshape(2, -1), axis=0)
    idx = np.nonzero(ok)[0]
    acq = replace(a, tr_ptr=np.array([0, len(idx)], np.int32), ch_xz=a.ch_xz[idx], ch_t=a.ch_t[idx],
                  win=np.array([[x0, w]], np.int32))
    meta = dict(q.meta)
    meta["traces"] = np.asarray(q.meta["traces"])[idx]
    return replace(q, acq=acq, meta=meta)
