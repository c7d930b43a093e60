"""Per-stage box QP of the control-limited backward pass (oracle).

Sec. IV-2: with u_min <= u_t <= u_max the stagewise control update comes from
a box-constrained QP solved as in control-limited DDP (Tassa, Mansard, Todorov
2014):

    min_d  1/2 d' H d + g' d     s.t.  lo <= d <= hi,

with H = Q_uu, g = Q_u, lo = u_min - u_bar, hi = u_max - u_bar.  The method
is projected Newton (Bertsekas 1982): at the current point, dimensions at a
bound whose gradient points out of the box are clamped; a Newton step is taken
on the remaining (free) dimensions; the step is projected back onto the box
and backtracked until an Armijo condition holds.

Readings (the paper gives no parameters):
  start       d = clamp(0)
  clamped     Bertsekas' epsilon-active set: a dimension within
              eps_i = EPS_REL (1 + hi_i - lo_i) of a bound whose gradient points
              out of the box, (d_i <= lo_i + eps_i and grad_i > 0) or
              (d_i >= hi_i - eps_i and grad_i < 0); it is set onto that bound
              and the gradient re-evaluated there.  With an exact comparison
              instead, a control a rounding error inside its bound counts as
              interior: the Newton step on every dimension, projected, is then
              no descent direction, the line search fails and the QP returns
              d = 0 with every dimension free, so the result would jump with
              rounding-level changes of its inputs.
  stop        no free dimension, or the free set equals the one of the previous
              iteration after a full (step 1) Newton step that the projection
              did not cut (then d is the minimiser on that face and the clamped
              signs were re-checked at it), or 20 iterations
  Armijo      phi(d_new) - phi(d) <= 0.1 * grad' (d_new - d), step *= 0.6,
              at most 30 trials (no trial accepted: stop at d)
  result      d (= k_t), the final free set, and the Cholesky factor of
              H restricted to it (used for K_t and by the adjoint pass).
A non-positive pivot in the Cholesky factor is reported as failure.
"""
from __future__ import annotations

import numpy as np

MAX_IT = 20
MAX_LS = 30
ARMIJO = 0.1
STEP_DEC = 0.6
EPS_REL = 1e-6


def cholesky(H):
    """Plain Cholesky H = L L' (lower); returns None on a non-positive pivot."""
    n = H.shape[0]
    L = np.zeros_like(H, dtype=float)
    for j in range(n):
        s = H[j, j] - np.dot(L[j, :j], L[j, :j])
        if not (s > 0.0):
            return None
        L[j, j] = np.sqrt(s)
        for i in range(j + 1, n):
            L[i, j] = (H[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    return L


def chol_solve(L, b):
    """Solve (L L') y = b by forward then backward substitution."""
    n = L.shape[0]
    z = np.zeros(n)
    for i in range(n):
        z[i] = (b[i] - np.dot(L[i, :i], z[:i])) / L[i, i]
    y = np.zeros(n)
    for i in reversed(range(n)):
        y[i] = (z[i] - np.dot(L[i + 1:, i], y[i + 1:])) / L[i, i]
    return y


def solve(H, g, lo, hi, stats=None):
    """Projected-Newton box QP.  Returns (d, free[bool], L, ok).

    ``stats`` (a dict, optional) receives the margins behind the clamped /
    free decisions of every iteration (degeneracy bookkeeping, reading R11):
    'grad', the smallest |grad_i| / (1 + max|g|) of a dimension inside the
    epsilon band of a bound (its sign decides), and 'band', the smallest
    distance of a dimension to the edge of that band, / (1 + hi_i - lo_i)."""
    n = g.shape[0]
    d = np.clip(np.zeros(n), lo, hi)
    free_prev = None
    last_full = False
    L = None
    free_fact = np.zeros(n, dtype=bool)
    eps = EPS_REL * (1.0 + (hi - lo))
    gscale = 1.0 + np.max(np.abs(g))
    for _ in range(MAX_IT):
        grad = g + H @ d
        if stats is not None:
            near = (d <= lo + eps) | (d >= hi - eps)
            if near.any():
                stats["grad"] = min(stats.get("grad", np.inf), float(np.min(np.abs(grad[near]))) / gscale)
            edge = np.minimum(np.abs(d - (lo + eps)), np.abs((hi - eps) - d)) / (1.0 + (hi - lo))
            stats["band"] = min(stats.get("band", np.inf), float(np.min(edge)))
        at_lo = (d <= lo + eps) & (grad > 0)
        at_hi = (d >= hi - eps) & (grad < 0)
        d = np.where(at_lo, lo, np.where(at_hi, hi, d))
        grad = g + H @ d
        clamped = at_lo | at_hi
        free = ~clamped
        if not free.any():
            return d, free, None, True
        if last_full and free_prev is not None and np.array_equal(free, free_prev):
            return d, free, L, True
        fi = np.flatnonzero(free)
        L = cholesky(H[np.ix_(fi, fi)])
        if L is None:
            return d, free, None, False
        free_fact = free
        ci = np.flatnonzero(clamped)
        rhs = -(g[fi] + H[np.ix_(fi, ci)] @ d[ci])
        d_newton = chol_solve(L, rhs)
        direction = np.zeros(n)
        direction[fi] = d_newton - d[fi]
        phi0 = g @ d + 0.5 * d @ H @ d
        step = 1.0
        accepted = False
        for _ls in range(MAX_LS):
            trial = d + step * direction
            dn = np.clip(trial, lo, hi)
            phin = g @ dn + 0.5 * dn @ H @ dn
            if phin - phi0 <= ARMIJO * (grad @ (dn - d)):
                accepted = True
                break
            step *= STEP_DEC
        if not accepted:
            return d, free_fact, L, True
        last_full = (step == 1.0) and bool(np.all((trial >= lo) & (trial <= hi)))
        free_prev = free
        d = dn
    return d, free_fact, L, True


def enumerate_kkt(H, g, lo, hi, tol=1e-9):
    """Brute force: try all 3^n active sets (each dim free / at lo / at hi) and
    return the points satisfying the KKT conditions of the box QP.  Used only by
    the pins; for a positive definite H exactly one point qualifies."""
    n = g.shape[0]
    sols = []
    for code in range(3 ** n):
        state = []
        c = code
        for _ in range(n):
            state.append(c % 3)
            c //= 3
        state = np.array(state)
        d = np.zeros(n)
        d[state == 1] = lo[state == 1]
        d[state == 2] = hi[state == 2]
        fi = np.flatnonzero(state == 0)
        if fi.size:
            oi = np.flatnonzero(state != 0)
            d[fi] = np.linalg.solve(H[np.ix_(fi, fi)], -(g[fi] + H[np.ix_(fi, oi)] @ d[oi]))
        if np.any(d < lo - tol) or np.any(d > hi + tol):
            continue
        grad = g + H @ d
        ok = True
        for i in range(n):
            if state[i] == 1 and grad[i] < -tol:
                ok = False
            if state[i] == 2 and grad[i] > tol:
                ok = False
        if ok:
            sols.append(d)
    return sols
