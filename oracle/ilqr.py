"""Box-constrained iLQR forward solve of Eq. (3) (oracle, FP64, one instance).

    min_{x, u}  sum_{t=0}^{N-1} 1/2 z_t' C_t z_t + c_t' z_t,   z_t = [x_t; u_t]
    s.t.        x_{t+1} = f(x_t, u_t),  x_0 = x_init,  u_lo <= u_t <= u_hi

with the diagonal surrogate of Eq. (2): C_t = diag(Q_t, R) and
c_t = [-Q_t * x_ref_t; -R * u_ref], or with general C_t (symmetric positive
semidefinite) and c_t when the problem carries them.  The iteration is Algorithm 2's inner
loop (Rollout -> {LQ, FBP, FFP, Converged?}) with the three stages of
Sec. IV: 1) rollout and linearization, 2) Riccati backward pass with the box
QP (Tassa et al. 2014), 3) forward pass with the line search over
alpha in {1, 0.5, 0.25, 0.1}.

Readings where the paper is silent, by number (R1, R4-R6; the others are stated where they apply):
  R1 cost   stage costs on (x_t, u_t) for t = 0..N-1, no terminal cost; the
            rollout produces x_1..x_{N-1}.  The value reported and compared
            is the centred form sum 1/2 (x-x_ref)'Q(x-x_ref) + 1/2 (u-u_ref)'R(u-u_ref),
            which differs from Eq. (3)'s objective by the constant
            1/2 (x_ref'Q x_ref + u_ref'R u_ref) per stage.
  R4 line search  every alpha is rolled out; alpha* = argmin J(alpha), ties to
            the earlier (larger) alpha, and -- as Sec. IV-3 states -- the best
            candidate becomes the next nominal.  Only when no candidate has a
            finite cost is the nominal kept (status STALLED).  J(alpha) - J is
            evaluated as the sum of the stage-wise cost changes (cost_change),
            an exact identity for the quadratic cost that does not lose small
            differences to the rounding of J's total.
  R5 converged    max_t |u^k_t - u^{k-1}_t|_inf < tol after an accepted step;
            at most max_iter iterations; every executed iteration is counted.
  R6 start  U^0 = clamp(u_ref) (or clamp(u_init) when given).
  Forward pass    u_hat_t = clamp(u_bar_t + alpha k_t + K_t (x_hat_t - x_bar_t)).
  Value update    Tassa's form V_x = Q_x + K'Q_uu k + K'Q_u + Q_ux'k,
                  V_xx = Q_xx + K'Q_uu K + K'Q_ux + Q_ux'K (symmetrised),
                  with K = -Q_uu,ff^-1 Q_ux,f on free rows and 0 on clamped rows.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import boxqp

CONVERGED, STALLED, MAX_ITER, NONFINITE, NONPD = 0, 1, 2, 3, 4   # STALLED: no finite candidate
ALPHAS = (1.0, 0.5, 0.25, 0.1)
MATERIAL_DU = 1e-4   # control change [N] below which a decision is immaterial


@dataclasses.dataclass
class Problem:
    """One MPC instance (arrays in float64)."""
    x0: np.ndarray          # [nx]
    Q: np.ndarray           # [Nq, nx]; Nq = 1 shares one diagonal over the stages
    x_ref: np.ndarray       # [N, nx]
    R: np.ndarray           # [nu]
    u_ref: np.ndarray       # [nu]
    u_lo: np.ndarray        # [nu]
    u_hi: np.ndarray        # [nu]
    n: int                  # horizon actually solved (<= N)
    u_init: np.ndarray | None = None   # [N, nu] warm start
    # General stage cost of Eq. (2), 1/2 z' C_t z + c_t' z with z = [x; u]:
    # when C is given it replaces the diagonal surrogate (Q, x_ref, R, u_ref)
    # in the cost; Nc = 1 shares one (C, c) over the stages.
    C: np.ndarray | None = None        # [Nc, nz, nz], symmetric positive semidefinite
    c: np.ndarray | None = None        # [Nc, nz]

    def Qt(self, t):
        return self.Q[t] if self.Q.shape[0] > 1 else self.Q[0]

    @property
    def general(self):
        return self.C is not None

    def Ct(self, t):
        """C_t of Eq. (2): the general matrix, or diag(Q_t, R)."""
        if self.general:
            return self.C[t] if self.C.shape[0] > 1 else self.C[0]
        return np.diag(np.concatenate([self.Qt(t), self.R]))

    def ct(self, t):
        """c_t of Eq. (2): the general vector, or [-Q_t x_ref_t; -R u_ref]."""
        if self.general:
            return self.c[t] if self.c.shape[0] > 1 else self.c[0]
        return np.concatenate([-self.Qt(t) * self.x_ref[t], -self.R * self.u_ref])


def problem_from_batch(batch: dict, i: int) -> Problem:
    hz = batch.get("horizon")
    N = batch["x_ref"].shape[1]
    n = int(hz[i]) if hz is not None else N
    ui = batch.get("u_init")
    Cb, cb = batch.get("C"), batch.get("c")
    return Problem(x0=np.asarray(batch["x0"][i], float), Q=np.asarray(batch["Q"][i], float),
                   x_ref=np.asarray(batch["x_ref"][i], float), R=np.asarray(batch["R"][i], float),
                   u_ref=np.asarray(batch["u_ref"][i], float), u_lo=np.asarray(batch["u_lo"][i], float),
                   u_hi=np.asarray(batch["u_hi"][i], float), n=n,
                   u_init=None if ui is None else np.asarray(ui[i], float),
                   C=None if Cb is None else np.asarray(Cb[i], float),
                   c=None if cb is None else np.asarray(cb[i], float))


def total_cost(prob: Problem, X, U):
    """Centred form of Eq. (3)'s objective over stages 0..n-1 (reading R1);
    with a general cost, Eq. (3)'s objective itself."""
    J = 0.0
    if prob.general:
        for t in range(prob.n):
            z = np.concatenate([X[t], U[t]])
            J += 0.5 * (z @ prob.Ct(t) @ z) + prob.ct(t) @ z
        return J
    for t in range(prob.n):
        dx = X[t] - prob.x_ref[t]
        du = U[t] - prob.u_ref
        J += 0.5 * (dx @ (prob.Qt(t) * dx)) + 0.5 * (du @ (prob.R * du))
    return J


def cost_change(prob: Problem, X, U, Xa, Ua, with_scale=False):
    """J(Xa, Ua) - J(X, U) summed stage by stage from the differences,
    d' C (z - z_ref + d/2) with d = z_a - z: the exact change of the quadratic
    cost, evaluated without cancelling against the size of J (reading R4).
    With ``with_scale`` also the sum of the terms' magnitudes, the size a
    rounding error of the sum is relative to."""
    dJ = 0.0
    scale = 0.0
    if prob.general:
        # d' (C (z + d/2) + c): the same identity for a general C
        for t in range(prob.n):
            z = np.concatenate([X[t], U[t]])
            d = np.concatenate([Xa[t] - X[t], Ua[t] - U[t]])
            tz = d * (prob.Ct(t) @ (z + 0.5 * d) + prob.ct(t))
            dJ += tz.sum()
            scale += np.abs(tz).sum()
        return (dJ, scale) if with_scale else dJ
    for t in range(prob.n):
        dx = Xa[t] - X[t]
        du = Ua[t] - U[t]
        tx = dx * (prob.Qt(t) * ((X[t] - prob.x_ref[t]) + 0.5 * dx))
        tu = du * (prob.R * ((U[t] - prob.u_ref) + 0.5 * du))
        dJ += tx.sum() + tu.sum()
        scale += np.abs(tx).sum() + np.abs(tu).sum()
    return (dJ, scale) if with_scale else dJ


@dataclasses.dataclass
class BackwardResult:
    ok: bool
    K: list      # [n] of (nu, nx)
    k: list      # [n] of (nu,)
    free: list   # [n] of bool (nu,)
    L: list      # [n] Cholesky factor of Q_uu restricted to the free set (or None)
    Quu: list
    Qux: list
    margin: float  # smallest |grad_i| over bound-decided dimensions (degeneracy)
    band: float = np.inf   # smallest distance of a control to the edge of the QP's epsilon band


def backward_pass(prob: Problem, X, U, F, free_override=None, qp_perturb=None) -> BackwardResult:
    """Sec. IV-2: Riccati recursion with the per-stage box QP, t = n-1 .. 0.

    Q_t = C_t + F_t' V_{t+1} F_t,  q_t = (C_t z_t + c_t) + F_t' v_{t+1}
    (V_n = 0, v_n = 0; stage n-1 has no dynamics term).  ``free_override``
    (a free mask per stage) replaces the box QP's free sets in K_t, the
    factor and the value update: the LQR of a given active set.
    ``qp_perturb`` (test instrument, None in the method) maps each stage's
    (Q_uu, q_u) to the pair the box QP gets, to measure how sensitive a step
    is to errors of its inputs (reading R11)."""
    n, nx, nu = prob.n, X.shape[1], U.shape[1]
    V = np.zeros((nx, nx))
    v = np.zeros(nx)
    Ks, ks, frees, Ls, Quus, Quxs = [None] * n, [None] * n, [None] * n, [None] * n, [None] * n, [None] * n
    margin = np.inf
    band = np.inf
    for t in reversed(range(n)):
        if prob.general:
            Ct = prob.Ct(t)
            ct = Ct @ np.concatenate([X[t], U[t]]) + prob.ct(t)
        else:
            Ct = np.diag(np.concatenate([prob.Qt(t), prob.R]))
            ct = np.concatenate([prob.Qt(t) * (X[t] - prob.x_ref[t]), prob.R * (U[t] - prob.u_ref)])
        if t < n - 1:
            Ft = F[t]
            Qm = Ct + Ft.T @ V @ Ft
            qv = ct + Ft.T @ v
        else:
            Qm = Ct
            qv = ct
        Qxx, Qxu = Qm[:nx, :nx], Qm[:nx, nx:]
        Qux, Quu = Qm[nx:, :nx], Qm[nx:, nx:]
        qx, qu = qv[:nx], qv[nx:]
        lo = prob.u_lo - U[t]
        hi = prob.u_hi - U[t]
        qs = {}
        if qp_perturb is not None:
            Quu, qu = qp_perturb(Quu, qu)
        k, free, L, ok = boxqp.solve(Quu, qu, lo, hi, stats=qs)
        margin = min(margin, qs.get("grad", np.inf))
        band = min(band, qs.get("band", np.inf))
        if not ok:
            return BackwardResult(False, Ks, ks, frees, Ls, Quus, Quxs, margin, band)
        if free_override is not None:
            free = np.asarray(free_override[t], dtype=bool)
            fi0 = np.flatnonzero(free)
            L = boxqp.cholesky(Quu[np.ix_(fi0, fi0)]) if fi0.size else None
        grad = qu + Quu @ k
        atb = (k <= lo) | (k >= hi)
        if atb.any():
            rel = np.abs(grad[atb]) / (1.0 + np.max(np.abs(qu)))
            margin = min(margin, float(np.min(rel)))
        K = np.zeros((nu, nx))
        fi = np.flatnonzero(free)
        for j in range(nx):
            if fi.size:
                K[fi, j] = -boxqp.chol_solve(L, Qux[fi, j])
        V = Qxx + K.T @ Quu @ K + K.T @ Qux + Qux.T @ K
        V = 0.5 * (V + V.T)
        v = qx + K.T @ Quu @ k + K.T @ qu + Qux.T @ k
        Ks[t], ks[t], frees[t], Ls[t], Quus[t], Quxs[t] = K, k, free, L, Quu, Qux
    return BackwardResult(True, Ks, ks, frees, Ls, Quus, Quxs, margin, band)


def forward_pass(model, prob: Problem, X, U, bp: BackwardResult, alpha):
    """Sec. IV-3: affine feedback update and rollout for one alpha."""
    n = prob.n
    Xn = np.zeros_like(X)
    Un = np.zeros_like(U)
    xh = prob.x0.copy()
    for t in range(n):
        Xn[t] = xh
        uh = U[t] + alpha * bp.k[t] + bp.K[t] @ (xh - X[t])
        Un[t] = np.clip(uh, prob.u_lo, prob.u_hi)
        if t < n - 1:
            xh = model.step(xh, Un[t])
    return Xn, Un


@dataclasses.dataclass
class Solution:
    X: np.ndarray        # [N, nx] (zeros past the horizon)
    U: np.ndarray        # [N, nu]
    J: float
    iters: int
    status: int
    F: list              # final linearization at (X, U) (A6)
    bp: BackwardResult   # final factorization at (X, U) (A6)
    ls_margin: float     # smallest relative gap behind a material alpha decision
    qp_margin: float     # smallest |grad| behind a clamped/free decision
    alpha_hist: list
    ls_margin_any: float = np.inf   # the same over every alpha decision, material or not
    du_hist: list = dataclasses.field(default_factory=list)   # max_t |u^k_t - u^(k-1)_t| of every step (R5)
    qp_band: float = np.inf   # smallest distance of a control to the edge of a QP's epsilon band


def linearize(model, prob: Problem, X, U):
    """Sec. IV-1: F_t = [A_t B_t] at the nominal, t = 0..n-2."""
    return [model.jacobian(X[t], U[t]) for t in range(prob.n - 1)]


def solve(model, prob: Problem, max_iter=10, tol=1e-6, alphas=ALPHAS, qp_perturb=None) -> Solution:
    """Algorithm 2's inner loop for one instance, then the factorization at the
    returned iterate that the backward pass differentiates (Sec. IV).
    ``qp_perturb``: see backward_pass (test instrument)."""
    n = prob.n
    N = prob.x_ref.shape[0]
    nx, nu = prob.x0.shape[0], prob.u_ref.shape[0]
    U = np.zeros((N, nu))
    u0 = prob.u_init[:n] if prob.u_init is not None else np.tile(prob.u_ref, (n, 1))
    U[:n] = np.clip(u0, prob.u_lo, prob.u_hi)
    X = np.zeros((N, nx))
    X[:n] = model.rollout(prob.x0, U[:n])
    J = total_cost(prob, X, U)
    status, iters = MAX_ITER, 0
    ls_margin, qp_margin, ls_margin_any, qp_band = np.inf, np.inf, np.inf, np.inf
    hist, du_hist = [], []
    if not np.isfinite(J):
        return Solution(X, U, J, 0, NONFINITE, [], None, ls_margin, qp_margin, hist, ls_margin_any)
    for it in range(max_iter):
        iters = it + 1
        F = linearize(model, prob, X, U)
        bp = backward_pass(prob, X, U, F, qp_perturb=qp_perturb)
        if not bp.ok:
            status = NONPD
            break
        qp_margin = min(qp_margin, bp.margin)
        qp_band = min(qp_band, bp.band)
        cands = []
        scale = 1e-300
        for a in alphas:
            Xa, Ua = forward_pass(model, prob, X, U, bp, a)
            dJa, sc = cost_change(prob, X, U, Xa, Ua, with_scale=True)
            cands.append((dJa if np.isfinite(dJa) else np.inf, Xa, Ua))
            if np.isfinite(sc):
                scale = max(scale, sc)
        Js = np.array([c[0] for c in cands])      # J(alpha) - J for every alpha
        best = int(np.argmin(Js))          # first minimum: the larger alpha on ties
        # Degeneracy bookkeeping (reading R11): the gap behind each decision
        # whose alternatives differ materially in the controls, relative to the
        # magnitude of the terms the cost changes are summed from.
        Ub = cands[best][2]
        for i, c in enumerate(cands):
            if i == best or not np.isfinite(c[0]):
                continue
            diff = np.max(np.abs(c[2][:n] - Ub[:n]))
            if diff > 0:
                ls_margin_any = min(ls_margin_any, abs(c[0] - Js[best]) / scale)
            if diff > MATERIAL_DU:
                ls_margin = min(ls_margin, abs(c[0] - Js[best]) / scale)
        du = float(np.max(np.abs(Ub[:n] - U[:n])))
        if not np.isfinite(Js[best]):
            status = STALLED
            hist.append(None)
            break
        hist.append(alphas[best])
        du_hist.append(du)
        J = J + Js[best]
        X, U = cands[best][1], cands[best][2]
        if du < tol:
            status = CONVERGED
            break
    F = linearize(model, prob, X, U)
    bp = backward_pass(prob, X, U, F)
    return Solution(X, U, total_cost(prob, X, U), iters, status, F, bp, ls_margin, qp_margin, hist, ls_margin_any,
                    du_hist, qp_band)


def at_iterate(model, prob: Problem, U, free_override=None) -> Solution:
    """The record of a given control sequence U (clamped to the bounds): its
    rollout, its cost, and the linearization and factorization at it that the
    backward pass differentiates (the final step of ``solve``), optionally
    with given free sets."""
    n, N = prob.n, prob.x_ref.shape[0]
    Uc = np.zeros((N, prob.u_ref.shape[0]))
    Uc[:n] = np.clip(U[:n], prob.u_lo, prob.u_hi)
    X = np.zeros((N, prob.x0.shape[0]))
    X[:n] = model.rollout(prob.x0, Uc[:n])
    F = linearize(model, prob, X, Uc)
    bp = backward_pass(prob, X, Uc, F, free_override)
    return Solution(X, Uc, total_cost(prob, X, Uc), 0, MAX_ITER, F, bp, np.inf, np.inf, [])


def solve_batch(model, batch: dict, idx=None, max_iter=None, tol=None):
    """Solve instances ``idx`` of a workload dict one by one."""
    B = batch["x0"].shape[0]
    idx = range(B) if idx is None else idx
    mi = batch.get("max_iter", 10) if max_iter is None else max_iter
    tl = batch.get("tol", 1e-6) if tol is None else tol
    return [solve(model, problem_from_batch(batch, i), mi, tl) for i in idx]
