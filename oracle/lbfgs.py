"""FP64 oracle of the optimizer: l-BFGS with a strong-Wolfe line search and the
convergence rate of eq. 13 (the paper inverts with l-BFGS, a step length
satisfying the Wolfe conditions, and stops when the rate drops below 0.1 %).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``bfgs_inverse_hessian``: the inverse-Hessian approximation by its
  definition, dense: H_0 = gamma I with gamma = s^T y / y^T y of the newest
  pair, then for every stored pair, oldest first,
  H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T, rho = 1 / y^T s
  (Nocedal & Wright, eq. 6.17 and 7.20).  With a positive diagonal D as the
  initial guess (the paper hands l-BFGS an approximate inverse pseudo-Hessian
  as its initial inverse Hessian), H_0 = gamma D with gamma = s^T y / y^T D y,
  and H_0 = D without pairs.
* ``two_loop``: the same product H g by the two-loop recursion (Nocedal &
  Wright, Alg. 7.4), for vectors too long for a dense matrix.
* ``wolfe_search``: Nocedal & Wright Alg. 3.5 (bracketing: while the trial
  meets sufficient decrease and phi' < 0, the next, longer trial is the zero
  of the secant of phi' through the last two points, kept within 2 to 10 times
  the current step, or twice the step when phi' did not increase; the
  algorithm leaves the choice in (a_i, a_max) open) and Alg. 3.6 (zoom); the
  zoom trial is the minimiser of the quadratic
  through phi(lo), phi'(lo), phi(hi), replaced by the bracket midpoint when it
  falls outside the inner 80 % of the bracket or the quadratic is not convex.
  A trial without a finite objective or slope (outside the algorithm, which
  assumes a smooth objective: a step that makes the modelling unstable) is
  read as failing sufficient decrease, phi = +inf, so the zoom bisects
  towards the shorter end of the bracket.
* ``lbfgs``: the iteration: d = -H g (restart from -H_0 g if d is not a
  descent direction), first step 1/||d|| without stored pairs else 1, store the pair
  only when s^T y > 0, keep the newest m pairs, rate_{k+1} = (Phi_k -
  Phi_{k+1}) / Phi_k (eq. 13).
"""
from __future__ import annotations

import numpy as np


def bfgs_inverse_hessian(S, Y, D=None, n=None):
    """Dense H from the pairs (rows of S and Y, oldest first); D: optional
    positive diagonal of the initial guess."""
    S = np.asarray(S, np.float64)
    Y = np.asarray(Y, np.float64)
    n = S.shape[1] if S.ndim == 2 else (len(D) if D is not None else n)
    D0 = np.eye(n) if D is None else np.diag(np.asarray(D, np.float64))
    if S.shape[0] == 0:
        return D0
    H = (S[-1] @ Y[-1]) / (Y[-1] @ D0 @ Y[-1]) * D0
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


def two_loop(g, S, Y, D=None):
    """H g by the two-loop recursion (pairs as rows, oldest first); D: optional
    positive diagonal of the initial guess H_0."""
    S = np.asarray(S, np.float64)
    Y = np.asarray(Y, np.float64)
    q = np.array(g, np.float64)
    Dv = np.ones_like(q) if D is None else np.asarray(D, np.float64)
    k = S.shape[0]
    if k == 0:
        return Dv * q
    rho = [1.0 / (Y[i] @ S[i]) for i in range(k)]
    alpha = [0.0] * k
    for i in range(k - 1, -1, -1):
        alpha[i] = rho[i] * (S[i] @ q)
        q = q - alpha[i] * Y[i]
    r = (S[-1] @ Y[-1]) / (Y[-1] @ (Dv * Y[-1])) * (Dv * q)
    for i in range(k):
        beta = rho[i] * (Y[i] @ r)
        r = r + (alpha[i] - beta) * S[i]
    return r


def _interp(lo, hi):
    """Zoom trial between lo = (a, phi, dphi) and hi = (a, phi, dphi)."""
    w = hi[0] - lo[0]
    den = 2.0 * (hi[1] - lo[1] - lo[2] * w)
    a = lo[0] - lo[2] * w * w / den if den > 0 else lo[0] + 0.5 * w
    lower = min(lo[0], hi[0]) + 0.1 * abs(w)
    upper = max(lo[0], hi[0]) - 0.1 * abs(w)
    if not (lower <= a <= upper):
        a = lo[0] + 0.5 * w
    return a


def _extrapolate(prev, t):
    """Next bracketing trial after t = (a, phi, dphi), which met sufficient decrease
    with phi'(a) < 0 (the minimum lies further): the zero of the secant of phi'
    through prev and t when phi' increased (exact for a quadratic), kept within
    [2 a, 10 a]; 2 a otherwise."""
    a = t[0]
    if t[2] > prev[2]:
        sec = a - t[2] * (a - prev[0]) / (t[2] - prev[2])
        return min(max(sec, 2.0 * a), 10.0 * a)
    return 2.0 * a


def wolfe_search(f, x, phi0, g0, d, a0, c1=1e-4, c2=0.9, max_ls=20):
    """Step a with phi(a) <= phi0 + c1 a phi'(0) and |phi'(a)| <= -c2 phi'(0).

    f(x) -> (phi, g).  Returns (a, phi, g, evals) or (None, None, None, evals).
    """
    dphi0 = float(g0 @ d)
    evals = 0

    def ev(a):
        nonlocal evals
        evals += 1
        phi, g = f(x + a * d)
        phi, dphi = float(phi), float(g @ d)
        if not (np.isfinite(phi) and np.isfinite(dphi)):
            phi = np.inf             # no finite value: the step is too long (fails sufficient decrease)
        return (a, phi, dphi), g

    def armijo_fails(t):
        return t[1] > phi0 + c1 * t[0] * dphi0

    def curvature(t):
        return abs(t[2]) <= -c2 * dphi0

    def zoom(lo, hi):
        while evals < max_ls:
            t, g = ev(_interp(lo, hi))
            if armijo_fails(t) or t[1] >= lo[1]:
                hi = t
            else:
                if curvature(t):
                    return t, g
                if t[2] * (hi[0] - lo[0]) >= 0:
                    hi = lo
                lo = t
        return None, None

    prev = (0.0, float(phi0), dphi0)
    a = a0
    i = 1
    while evals < max_ls:
        t, g = ev(a)
        if armijo_fails(t) or (i > 1 and t[1] >= prev[1]):
            t, g = zoom(prev, t)
            break
        if curvature(t):
            break
        if t[2] >= 0:
            t, g = zoom(t, prev)
            break
        a = _extrapolate(prev, t)
        prev = t
        i += 1
    else:
        t = None
    if t is None:
        return None, None, None, evals
    return t[0], t[1], g, evals


def lbfgs(f, x0, iters, m=5, c1=1e-4, c2=0.9, max_ls=20, D=None):
    """Iterates of l-BFGS from x0: list of dicts (x, phi, alpha, rate, evals).
    D: optional positive diagonal initial inverse Hessian."""
    x = np.array(x0, np.float64)
    phi, g = f(x)
    S, Y = [], []
    out = []
    for _ in range(iters):
        d = -two_loop(g, S, Y, D)
        if not (g @ d < 0):
            S, Y = [], []
            d = -two_loop(g, S, Y, D)
        a0 = min(1.0, 1.0 / np.sqrt(d @ d)) if not S else 1.0
        a, phi1, g1, evals = wolfe_search(f, x, phi, g, d, a0, c1, c2, max_ls)
        if a is None:
            out.append({"x": x.copy(), "phi": phi, "alpha": None, "rate": None, "evals": evals})
            break
        x1 = x + a * d
        s, y = x1 - x, g1 - g
        if s @ y > 0 and y @ y > 0:
            S.append(s)
            Y.append(y)
            S, Y = S[-m:], Y[-m:]
        rate = (phi - phi1) / phi
        x, phi, g = x1, phi1, g1
        out.append({"x": x.copy(), "phi": phi, "alpha": a, "rate": rate, "evals": evals})
    return out
