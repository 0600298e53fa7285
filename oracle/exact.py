"""numpy part of the FP64 oracle.  Test infrastructure.

* ``brute_force_cqk``: enumerate every assignment of the variables to
  {lower bound, upper bound, free} (3^n of them), solve the linear equation
  b'x = r for lambda on the free set, keep the KKT-consistent assignment.  The
  problem is strictly convex (Sec. 1), so the KKT point is the unique minimiser.
  For n <= 12.
* ``kkt_residuals``: how far (x, lambda) is from x = x(lambda), b'x = r.
* ``project_simplex`` / ``project_l1``: the simplex projection by the sort-based
  closed form, and the l1-ball projection by Lemma 3.2 (x = y inside the ball,
  else sgn(y) * P_simplex(|y|), sgn(0) = 0 as in the notation of Sec. 1).
* ``grad_*``: the implicit-function derivative of the solution map (the paper
  has no backward pass; the derivation is stated in the docstrings).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import reference as _ref


def brute_force_cqk(a, b, d, l, u, r):
    """Unique minimiser of (CQK) by active-set enumeration.  Returns (lam, x), or
    None if no assignment is KKT-consistent (infeasible r).

    Every assignment s in {0: at l, 1: at u, 2: free}^n is tried (vectorised
    over assignments).  For a free set F with q = sum_F b_i^2/d_i > 0,
    lambda = (r - sum_L b l - sum_U b u - sum_F b a/d)/q; the assignment is
    consistent when the free t_i = (a_i + lambda b_i)/d_i lie in [l_i, u_i], and
    t_i <= l_i on L, t_i >= u_i on U."""
    a, b, d, l, u = (np.asarray(v, dtype=np.float64) for v in (a, b, d, l, u))
    n = a.shape[0]
    S = np.array(list(itertools.product((0, 1, 2), repeat=n)), dtype=np.int8).reshape(-1, n)
    L, U, F = S == 0, S == 1, S == 2
    ok = ~np.any((L & np.isinf(l)) | (U & np.isinf(u)), axis=1)
    lf = np.where(np.isinf(l), 0.0, l)
    uf = np.where(np.isinf(u), 0.0, u)
    fixed = (L * (b * lf)).sum(axis=1) + (U * (b * uf)).sum(axis=1)
    q = (F * (b * b / d)).sum(axis=1)
    s0 = (F * (b * a / d)).sum(axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        lam = np.where(q > 0, (r - fixed - s0) / np.where(q > 0, q, 1.0), 0.0)
    t = (a[None, :] + lam[:, None] * b[None, :]) / d[None, :]
    tol = 1e-12 * (1 + np.abs(t))
    with np.errstate(invalid="ignore"):
        bad_f = F & ((t < l - tol) | (t > u + tol))
        bad_l = L & (t > l + tol)
        bad_u = U & (t < u - tol)
    consistent = ok & ~np.any(bad_f | bad_l | bad_u, axis=1)
    # with q == 0 (no free variable) lambda is not determined by the equation;
    # such an assignment only counts if b'x = r holds with every variable at a bound
    consistent &= (q > 0) | (np.abs(fixed - r) <= 1e-12 * (abs(r) + 1))
    rows = np.nonzero(consistent & (q > 0))[0]
    if rows.size == 0:
        rows = np.nonzero(consistent)[0]
        if rows.size == 0:
            return None
    k = rows[0]
    x = np.where(L[k], l, np.where(U[k], u, t[k]))
    return float(lam[k]), x


def kkt_residuals(x, lam, a, b, d, l, u, r):
    """(max_i |x_i - x_i(lam)|, |b'x - r| / sum|b_i x_i|)."""
    xl = _ref.x_of_lambda(lam, a, b, d, l, u)
    bx = np.asarray(b) * np.asarray(x)
    feas = abs(float(np.sum(bx, dtype=np.longdouble)) - r) / max(float(np.sum(np.abs(bx))), 1e-300)
    return float(np.max(np.abs(np.asarray(x) - xl))), feas


def project_simplex(y, r=1.0):
    """Projection onto {x >= 0, sum x = r} (eq. (proj_Delta)).  Returns (lam*, x*)."""
    return _ref.project_simplex_sort(y, r)


def project_l1(y, r=1.0):
    """Projection onto {sum |x_i| <= r} by Lemma 3.2.  Returns (lam*, x*, inside).

    Inside the ball x = y and lam* = 0; otherwise lam* <= 0 solves the dual of
    (proj_Delta) for |y| and x_i = sgn(y_i) max{0, |y_i| + lam*}."""
    y = np.asarray(y, dtype=np.float64)
    if float(np.sum(np.abs(y), dtype=np.longdouble)) <= r:
        return 0.0, y.copy(), True
    lam, p = _ref.project_simplex_sort(np.abs(y), r)
    return lam, np.sign(y) * p, False


def lambda0_simplex_formula(y, r):
    """eq. (CQKlambda0) for the simplex data (b = d = 1, a = y): (r - sum y)/n."""
    y = np.asarray(y, dtype=np.float64)
    return float((r - np.sum(y, dtype=np.longdouble)) / y.shape[0])


def grad_cqk(x, lam, a, b, d, l, u, g):
    """Gradient of g'x*(a, b, d, r, l, u) at the solution (x = x*, lam = lam*).

    Sets: F = {l < x < u} (free), L = non-free with (a + lam b)/d <= l, U = the
    rest.  On F, x_i = (a_i + lam b_i)/d_i; off F x_i is the bound; and
    sum_i b_i x_i = r.  Differentiating and eliminating d lam gives, with
    Q = sum_F b_i^2/d_i and mu = (sum_F b_i g_i/d_i)/Q:
      da_i = (g_i - mu b_i)/d_i on F, 0 off F
      dd_i = -x_i da_i
      db_i = lam da_i - mu x_i          (the second term for every i)
      dl_i = g_i - mu b_i on L, 0 elsewhere
      du_i = g_i - mu b_i on U, 0 elsewhere
      dr   = mu
    When F is empty (Q = 0) the map is not differentiable in r; mu = 0 is used
    and ``nondiff`` is set.
    Returns dict(a, b, d, l, u, r, mu, Q, nondiff, free)."""
    x, a, b, d, l, u, g = (np.asarray(v, dtype=np.float64) for v in (x, a, b, d, l, u, g))
    F = (x > l) & (x < u)
    t = (a + lam * b) / d
    L = (~F) & (t <= l)
    U = (~F) & (~L)
    Q = float(np.sum(b[F] ** 2 / d[F], dtype=np.longdouble))
    nondiff = not (Q > 0)
    mu = float(np.sum(b[F] * g[F] / d[F], dtype=np.longdouble)) / Q if not nondiff else 0.0
    ga = np.where(F, (g - mu * b) / d, 0.0)
    gd = -x * ga
    gb = lam * ga - mu * x
    gl = np.where(L, g - mu * b, 0.0)
    gu = np.where(U, g - mu * b, 0.0)
    return dict(a=ga, b=gb, d=gd, l=gl, u=gu, r=mu, mu=mu, Q=Q, nondiff=nondiff, free=F)


def grad_simplex(x, g):
    """Gradient of g'P_simplex(y, r) in y and r: with F = {x > 0},
    dy_i = g_i - mean_F(g) on F, 0 off F; dr = mean_F(g) (the general formula
    with b = d = 1, l = 0, u = +inf)."""
    x, g = np.asarray(x, dtype=np.float64), np.asarray(g, dtype=np.float64)
    F = x > 0
    mu = float(np.mean(g[F])) if np.any(F) else 0.0
    return dict(y=np.where(F, g - mu, 0.0), r=mu, mu=mu, free=F)


def grad_l1(y, x, g, inside):
    """Gradient of g'P_l1ball(y, r): identity inside the ball (dr = 0); outside,
    with s = sgn(y), F = {x != 0}, mu = mean_F(s g): dy_i = g_i - s_i mu on F,
    0 off F; dr = mu."""
    y, x, g = (np.asarray(v, dtype=np.float64) for v in (y, x, g))
    if inside:
        return dict(y=g.copy(), r=0.0, mu=0.0, free=np.ones_like(y, dtype=bool))
    s = np.sign(y)
    F = x != 0
    mu = float(np.mean((s * g)[F])) if np.any(F) else 0.0
    return dict(y=np.where(F, g - s * mu, 0.0), r=mu, mu=mu, free=F)
