"""Pins of the optimizer oracle (l-BFGS, strong-Wolfe line search, eq. 13) to
facts independent of its code: the dense BFGS inverse-Hessian formula, the
secant equation, closed-form line minimisers of quadratics, the Wolfe
conditions themselves, and finite termination on convex quadratics."""
import numpy as np
import pytest

from oracle import lbfgs as L


def _pairs(n, k, seed):
    """k pairs with y = A s for an SPD A (so s^T y > 0), rows oldest first."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(rng.uniform(0.5, 5.0, n)) @ Q.T
    S = rng.standard_normal((k, n))
    return S, S @ A.T, A


@pytest.mark.parametrize("k", [0, 1, 3, 5])
def test_two_loop_equals_dense_bfgs_matrix(k):
    S, Y, _ = _pairs(12, k, 1)
    g = np.random.default_rng(2).standard_normal(12)
    H = L.bfgs_inverse_hessian(S, Y)
    assert np.allclose(L.two_loop(g, S, Y), H @ g, rtol=1e-12, atol=1e-12)


def test_dense_matrix_satisfies_secant_equation_and_symmetry():
    S, Y, _ = _pairs(9, 4, 3)
    H = L.bfgs_inverse_hessian(S, Y)
    assert np.allclose(H @ Y[-1], S[-1], rtol=1e-12, atol=1e-12)
    assert np.allclose(H, H.T, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(H) > 0)


def test_n_pairs_of_a_quadratic_reproduce_its_inverse_hessian():
    """n A-conjugate pairs y_i = A s_i of a quadratic: BFGS keeps H y_j = s_j
    for every earlier pair (hereditary property), so after the n-th update
    H = A^{-1} exactly, whatever H_0."""
    n = 6
    rng = np.random.default_rng(4)
    A = np.diag(rng.uniform(1.0, 3.0, n))
    S = np.eye(n)                       # A-conjugate for a diagonal A
    Y = S @ A.T
    H = L.bfgs_inverse_hessian(S, Y)
    assert np.allclose(H, np.linalg.inv(A), rtol=1e-12, atol=1e-12)


def test_zoom_hits_the_minimiser_of_a_one_dimensional_quadratic():
    """phi(a) = phi0 + phi'(0) a + c a^2 / 2 (here a* = 1/4): a first step
    a0 = 0.3 just beyond the minimiser has phi'(a0) > 0 and, with c2 = 0.1,
    fails the curvature condition; the quadratic interpolating the bracket
    ends is phi itself, so the first zoom trial is a* = -phi'(0)/c exactly
    (inside the inner 80 % of [0, 0.3])."""
    c, x0 = 4.0, np.array([3.0])

    def f(x):
        return 0.5 * c * float(x @ x), c * x

    phi0, g0 = f(x0)
    d = -g0
    a, phi, g, evals = L.wolfe_search(f, x0, phi0, g0, d, a0=0.3, c2=0.1)
    assert a == pytest.approx(1.0 / c, rel=1e-14)
    assert evals == 2
    assert abs(phi) < 1e-25


@pytest.mark.parametrize("fun", ["quadratic", "rosenbrock"])
def test_accepted_step_satisfies_the_strong_wolfe_conditions(fun):
    rng = np.random.default_rng(5)
    if fun == "quadratic":
        A = np.diag(rng.uniform(0.1, 10.0, 8))

        def f(x):
            return 0.5 * float(x @ A @ x), A @ x
        x0 = rng.standard_normal(8)
    else:
        def f(x):
            phi = float(np.sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2))
            g = np.zeros_like(x)
            g[:-1] = -400.0 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2.0 * (1 - x[:-1])
            g[1:] += 200.0 * (x[1:] - x[:-1] ** 2)
            return phi, g
        x0 = np.full(6, -1.2)
    c1, c2 = 1e-4, 0.9
    for a0 in (1e-3, 1.0, 50.0):
        phi0, g0 = f(x0)
        d = -g0
        a, phi, g, _ = L.wolfe_search(f, x0, phi0, g0, d, a0, c1, c2, max_ls=40)
        assert a is not None
        assert phi <= phi0 + c1 * a * (g0 @ d) + 1e-12 * abs(phi0)
        assert abs(g @ d) <= -c2 * (g0 @ d)


def test_lbfgs_minimises_a_convex_quadratic_and_reports_eq13_rates():
    rng = np.random.default_rng(6)
    n = 20
    a = rng.uniform(0.5, 20.0, n)
    c = rng.standard_normal(n)

    def f(x):
        r = x - c
        return 0.5 * float(np.sum(a * r * r)) + 1.0, a * r

    it = L.lbfgs(f, np.zeros(n), iters=60, m=5)
    assert np.linalg.norm(it[-1]["x"] - c) < 1e-6
    it = [r for r in it if r["rate"] is not None]     # a last failed search (at the minimum) moves nothing
    phis = [f(np.zeros(n))[0]] + [r["phi"] for r in it]
    for k, r in enumerate(it):
        assert r["rate"] == pytest.approx((phis[k] - phis[k + 1]) / phis[k], rel=1e-15)
        assert r["phi"] <= phis[k]


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_search_backs_off_from_non_finite_trials(bad):
    """phi(x) = (x - 1)^2 + 1 is defined only for x < 3 (beyond, a value that is not
    finite, as an unstable simulation gives).  From x = 0 along d = 1 with first trial
    a = 8 the search must bisect back into [0, 3) and return a strong-Wolfe step
    there: phi(a) <= phi0 + c1 a phi'(0) and |phi'(a)| <= c2 |phi'(0)|."""
    calls = []

    def f(x):
        calls.append(float(x[0]))
        if x[0] >= 3.0:
            return bad, np.array([bad])
        return float((x[0] - 1.0) ** 2 + 1.0), np.array([2.0 * (x[0] - 1.0)])
    x0 = np.zeros(1)
    phi0, g0 = f(x0)
    d = np.ones(1)
    c1, c2 = 1e-4, 0.9
    a, phi, g, evals = L.wolfe_search(f, x0, phi0, g0, d, 8.0, c1, c2, max_ls=20)
    assert a is not None and 0 < a < 3.0
    assert phi <= phi0 + c1 * a * (g0 @ d)
    assert abs(g @ d) <= -c2 * (g0 @ d)
    # 8 and 4 are not finite: the bracket [0, 8] is halved twice; at 2 the sufficient
    # decrease fails (phi(2) = phi(0)), and the quadratic through phi(0), phi'(0), phi(2)
    # has its minimum at 1, the exact minimiser
    assert calls[1:] == [8.0, 4.0, 2.0, 1.0] and evals == 4 and a == 1.0


def test_bracketing_extrapolates_by_the_secant_of_the_slope():
    """phi(x) = (x - 50)^2 from x = 0 along d = 1, first trial 1: phi'(0) = -100 and
    phi'(1) = -98, whose secant vanishes at 50, clipped to 10 x the step; at 10 the
    secant through (1, -98), (10, -80) vanishes at 50 (within [20, 100]): the exact
    minimiser, where phi' = 0 meets the curvature condition (c2 = 0.1, so that 10,
    with |phi'| = 80, does not)."""
    calls = []

    def f(x):
        calls.append(float(x[0]))
        return float((x[0] - 50.0) ** 2), np.array([2.0 * (x[0] - 50.0)])
    x0 = np.zeros(1)
    phi0, g0 = f(x0)
    a, phi, g, evals = L.wolfe_search(f, x0, phi0, g0, np.ones(1), 1.0, c2=0.1)
    assert calls[1:] == [1.0, 10.0, 50.0] and evals == 3 and a == 50.0 and phi == 0.0


def test_failed_search_keeps_the_point():
    """A direction of ascent never satisfies the sufficient decrease."""
    def f(x):
        return float(x @ x), 2 * x
    x0 = np.array([1.0, -2.0])
    phi0, g0 = f(x0)
    a, phi, g, evals = L.wolfe_search(f, x0, phi0, g0, g0, 1.0, max_ls=5)
    assert a is None and evals == 5


# --- diagonal initial inverse Hessian (the pseudo-Hessian preconditioner) ----------

@pytest.mark.parametrize("k", [0, 1, 3, 5])
def test_two_loop_with_diagonal_equals_dense_bfgs_matrix(k):
    """The recursion with H_0 = gamma D equals the dense update from H_0 = gamma D
    (gamma = s^T y / y^T D y of the newest pair; D itself without pairs)."""
    S, Y, _ = _pairs(10, k, 11)
    D = np.random.default_rng(12).uniform(0.1, 3.0, 10)
    g = np.random.default_rng(13).standard_normal(10)
    H = L.bfgs_inverse_hessian(S, Y, D)
    assert np.allclose(L.two_loop(g, S, Y, D), H @ g, rtol=1e-12, atol=1e-12)
    if k == 0:
        assert np.allclose(H, np.diag(D), rtol=0, atol=0)


def test_constant_diagonal_is_the_identity_guess():
    """D = c 1 changes nothing once a pair is stored (gamma absorbs c)."""
    S, Y, _ = _pairs(8, 3, 14)
    g = np.random.default_rng(15).standard_normal(8)
    assert np.allclose(L.two_loop(g, S, Y, np.full(8, 7.5)), L.two_loop(g, S, Y), rtol=1e-13, atol=1e-13)


def test_diagonal_guess_keeps_secant_equation_and_hereditary_property():
    S, Y, _ = _pairs(9, 4, 16)
    D = np.random.default_rng(17).uniform(0.2, 2.0, 9)
    H = L.bfgs_inverse_hessian(S, Y, D)
    assert np.allclose(H @ Y[-1], S[-1], rtol=1e-12, atol=1e-12)
    assert np.allclose(H, H.T, atol=1e-12) and np.all(np.linalg.eigvalsh(H) > 0)
    n = 6
    A = np.diag(np.random.default_rng(18).uniform(1.0, 3.0, n))
    Hn = L.bfgs_inverse_hessian(np.eye(n), A, np.random.default_rng(19).uniform(0.1, 5.0, n))
    assert np.allclose(Hn, np.linalg.inv(A), rtol=1e-12, atol=1e-12)


def test_exact_diagonal_preconditioner_points_at_the_minimiser():
    """phi = 1/2 (x - c)^T A (x - c) with A diagonal and D = A^{-1}: the first
    direction is c - x0 exactly, the first trial step 1/||d|| along it."""
    rng = np.random.default_rng(20)
    a = rng.uniform(0.5, 40.0, 30)
    c = rng.standard_normal(30)

    def f(x):
        return 0.5 * float(np.sum(a * (x - c) ** 2)), a * (x - c)

    x0 = np.zeros(30)
    _, g0 = f(x0)
    assert np.allclose(-L.two_loop(g0, [], [], 1.0 / a), c - x0, rtol=1e-14, atol=0)
    out = L.lbfgs(f, x0, iters=1, D=1.0 / a)
    # along the Newton direction phi(t) = (1 - t)^2 phi(x0): the first trial t0 = 1/||c||
    # (here in [0.1, 1]) meets both strong Wolfe conditions and is accepted as it is
    t0 = 1.0 / np.linalg.norm(c)
    assert 0.1 < t0 < 1.0
    assert out[0]["alpha"] == pytest.approx(t0, rel=1e-14) and out[0]["evals"] == 1
    assert out[0]["phi"] == pytest.approx((1.0 - t0) ** 2 * f(x0)[0], rel=1e-12)
