"""Pins of the oracle's model-extension operators (eqs. 8-12), no GPU.

* eq. 10 end values and monotonicity, sinkhole membership;
* rows of W sum to one (eq. 11 text); W = I outside every sinkhole;
* (I - S^T S_w) annihilates a constant extension, so phi_reg(1 (x) m) = 0;
* one source: phi_reg = 0;
* no sinkholes: phi_reg is the closed-form weighted variance;
* hand-computed one-pixel examples (tests/golden/reg_one_pixel.txt);
* the gradient matches central differences (phi_reg is quadratic) and the
  dense operator assembled over all pixels of a 31-sample 1D model with 3
  sources (the setting of Figure 2).
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import extension as X

GOLD = os.path.join(os.path.dirname(__file__), "golden", "reg_one_pixel.txt")


def _golden():
    vals = {}
    with open(GOLD) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = np.array([float(t) for t in v.split()])
    return vals


def test_zoi_profile_end_values_and_monotone():
    for n, nu in ((2.0, 0.99), (4.0, 0.5), (1.0, 0.1)):
        assert X.zoi_profile(0.0, n, nu) == pytest.approx(1.0, abs=1e-15)
        ln = np.log(nu)
        assert X.zoi_profile(1.0, n, nu) == pytest.approx(-ln / (1 - ln), rel=1e-14)
        r = np.linspace(0, 1, 101)
        assert np.all(np.diff(X.zoi_profile(r, n, nu)) <= 0)
    assert X.zoi_profile(1.0, 2.0, 0.99) == pytest.approx(0.00995, rel=1e-3)


def test_zoi_weights_geometry():
    zoi = W.ZOI(active_x=np.array([[20.0, 80.0]]), taper=np.array([10.0]), sink_xz=np.array([[50.0, 20.0]]),
                sink_ax=np.array([8.0]), sink_az=np.array([4.0]), n=2.0, nu=0.5)
    b, bp, sink = X.zoi_weights(zoi, 101, 41, 1.0, 1.0)
    floor = -np.log(0.5) / (1 - np.log(0.5))
    assert b[0, 20, 50] == pytest.approx(floor)          # at the source: r = 1
    assert sink[0, 20, 50] == 1 and bp[0, 20, 50] == 1.0
    assert b[0, 20, 30] == pytest.approx(1.0)            # active span, outside the sinkhole
    assert b[0, 20, 100] == pytest.approx(floor)         # beyond the taper
    assert b[0, 20, 85] == pytest.approx(X.zoi_profile(0.5, 2.0, 0.5))  # halfway through the taper
    assert sink[0, 20, 58] == 0 and sink[0, 20, 57] == 1  # semi-axis 8 m along x
    assert sink[0, 24, 50] == 0 and sink[0, 23, 50] == 1  # semi-axis 4 m along z
    assert np.all(bp[0][sink[0] == 0] == b[0][sink[0] == 0])


def _fig2_setup():
    """1D model with 31 samples and 3 sources (the setting of Figure 2)."""
    zoi = W.ZOI(active_x=np.array([[0.0, 30.0]] * 3), taper=np.full(3, 5.0),
                sink_xz=np.array([[5.0, 0.0], [15.0, 0.0], [25.0, 0.0]]), sink_ax=np.full(3, 4.0),
                sink_az=np.full(3, 1.0), n=2.0, nu=0.9)
    return X.zoi_weights(zoi, 31, 1, 1.0, 1.0)


def test_w_rows_sum_to_one_and_identity_outside_sinkholes():
    b, bp, sink = _fig2_setup()
    Wm = X.w_matrices(b.reshape(3, -1), sink.reshape(3, -1))
    assert np.allclose(Wm.sum(axis=2), 1.0, atol=1e-15)
    outside = ~sink.reshape(3, -1).any(axis=0)
    assert outside.any()
    assert np.all(Wm[outside] == np.eye(3))
    # inside sinkhole s at its source location, the diagonal is the floor weight
    for s, x in enumerate((5, 15, 25)):
        assert Wm[x, s, s] == pytest.approx(b[s, 0, x])


def test_constant_extension_is_in_the_null_space():
    rng = np.random.default_rng(0)
    b, bp, sink = _fig2_setup()
    m = np.repeat(rng.standard_normal((1, 1, 31)), 3, axis=0)
    phi, g = X.regularization(m, b, bp, sink, eta=3.0)
    assert phi < 1e-28 and np.abs(g).max() < 1e-13


def test_single_source_has_no_regularization():
    rng = np.random.default_rng(1)
    b = rng.random((1, 5, 7)) * 0.9 + 0.05
    sink = (rng.random((1, 5, 7)) > 0.5).astype(np.uint8)
    bp = np.where(sink == 1, 1.0, b)
    phi, g = X.regularization(rng.standard_normal((1, 5, 7)), b, bp, sink, eta=2.0)
    assert phi == 0.0 and not g.any()


def test_no_sinkholes_is_weighted_variance():
    rng = np.random.default_rng(2)
    ns = 4
    b = rng.random((ns, 6, 5)) * 0.9 + 0.1
    m = rng.standard_normal((ns, 6, 5))
    eta = 0.7
    phi, _ = X.regularization(m, b, b, np.zeros_like(b, np.uint8), eta)
    mean = (b * m).sum(0) / b.sum(0)
    assert phi == pytest.approx(0.5 * eta ** 2 * np.sum((m - mean) ** 2), rel=1e-13)


@pytest.mark.parametrize("case", ["A", "B"])
def test_hand_computed_pixel(case):
    gold = _golden()
    b = gold[f"{case}.b"][:, None, None]
    sink = gold[f"{case}.sink"].astype(np.uint8)[:, None, None]
    bp = np.where(sink == 1, 1.0, b)
    m = gold[f"{case}.m"][:, None, None]
    eta = 1.3
    phi, g = X.regularization(m, b, bp, sink, eta)
    assert phi == pytest.approx(gold[f"{case}.phi_over_eta2"][0] * eta ** 2, rel=1e-13)
    assert np.allclose(g[:, 0, 0], gold[f"{case}.grad_over_eta2"] * eta ** 2, rtol=1e-13, atol=1e-15)


def _dense_operator(b, bp, sink):
    """(I - S^T S_w) W assembled as one (Ns*npix) x (Ns*npix) matrix, entry by entry."""
    ns, npix = b.shape
    N = ns * npix
    Wd = np.zeros((N, N)); Pd = np.zeros((N, N))
    idx = lambda s, p: s * npix + p
    for p in range(npix):
        for s in range(ns):
            if sink[s, p] and ns > 1:
                tot = sum(b[i, p] for i in range(ns) if i != s)
                Wd[idx(s, p), idx(s, p)] = b[s, p]
                for i in range(ns):
                    if i != s:
                        Wd[idx(s, p), idx(i, p)] = (1 - b[s, p]) * b[i, p] / tot
            else:
                Wd[idx(s, p), idx(s, p)] = 1.0
        tot = sum(bp[i, p] for i in range(ns))
        for s in range(ns):
            Pd[idx(s, p), idx(s, p)] += 1.0
            for i in range(ns):
                Pd[idx(s, p), idx(i, p)] -= bp[i, p] / tot
    return Pd @ Wd


def test_gradient_against_dense_operator_and_fd():
    rng = np.random.default_rng(3)
    b, bp, sink = _fig2_setup()
    m = rng.standard_normal((3, 1, 31))
    eta = 1.7
    phi, g = X.regularization(m, b, bp, sink, eta)
    A = _dense_operator(b.reshape(3, -1), bp.reshape(3, -1), sink.reshape(3, -1))
    x = m.reshape(-1)
    assert phi == pytest.approx(0.5 * eta ** 2 * float(x @ A.T @ A @ x), rel=1e-12)
    assert np.allclose(g.reshape(-1), eta ** 2 * A.T @ (A @ x), rtol=1e-12, atol=1e-14)
    dm = rng.standard_normal(m.shape)
    h = 1e-3
    fd = (X.regularization(m + h * dm, b, bp, sink, eta)[0] - X.regularization(m - h * dm, b, bp, sink, eta)[0]) / (2 * h)
    assert fd == pytest.approx(float(np.sum(g * dm)), rel=1e-9)


def test_collapse_of_constant_extension_is_identity():
    rng = np.random.default_rng(4)
    b, bp, sink = _fig2_setup()
    m = rng.standard_normal((1, 1, 31))
    assert np.allclose(X.collapse(np.repeat(m, 3, axis=0), b, bp, sink), m[0], atol=1e-14)


def test_collapse_hand_computed_pixel():
    """One pixel, three sources, inside the sinkhole of source 0 only:
    (W m)_0 = b_0 m_0 + (1 - b_0)(b_1 m_1 + b_2 m_2)/(b_1 + b_2) = 0.5 + 0.5 * 2.2 = 1.6,
    (W m)_1 = 2, (W m)_2 = 3 (eq. 11); b' = (1, b_1, b_2) (eq. 12), so
    S_w W m = (1.6 + 0.8 * 2 + 0.2 * 3) / 2 = 1.9 (eq. 9)."""
    b = np.array([0.5, 0.8, 0.2]).reshape(3, 1, 1)
    bp = np.array([1.0, 0.8, 0.2]).reshape(3, 1, 1)
    sink = np.array([1, 0, 0], np.uint8).reshape(3, 1, 1)
    m = np.array([1.0, 2.0, 3.0]).reshape(3, 1, 1)
    assert X.collapse(m, b, bp, sink)[0, 0] == pytest.approx(1.9, abs=1e-15)


def test_collapse_single_source_and_no_sinkholes():
    """Ns = 1: W = I and S_w = 1, so the collapse returns the component itself;
    without sinkholes W = I and the collapse is the b'-weighted mean."""
    rng = np.random.default_rng(5)
    m = rng.standard_normal((1, 4, 7))
    b = rng.uniform(0.1, 1, (1, 4, 7))
    assert np.array_equal(X.collapse(m, b, b, np.ones((1, 4, 7), np.uint8)), m[0])
    m = rng.standard_normal((3, 4, 7))
    b = rng.uniform(0.1, 1, (3, 4, 7))
    ref = (b * m).sum(0) / b.sum(0)
    assert np.allclose(X.collapse(m, b, b, np.zeros((3, 4, 7), np.uint8)), ref, rtol=1e-14, atol=1e-14)


def test_collapse_chunks_do_not_change_the_result():
    rng = np.random.default_rng(6)
    b, bp, sink = _fig2_setup()
    m = rng.standard_normal((3, 1, 31))
    assert np.array_equal(X.collapse(m, b, bp, sink, chunk=7), X.collapse(m, b, bp, sink))
