"""Backward pass of the differentiable MPC layer (oracle, FP64, one instance).

Sec. IV: gradients of an external loss L with respect to (C_t, c_t) and
x_init come from implicit differentiation of the KKT conditions at the
solution (Amos et al. 2018), so they do not depend on the iteration count.
At the returned iterate tau* = (x*, u*) the problem is replaced by its LQR:
the same C_t, dynamics linearised to x_{t+1} = F_t tau_t + f_t, and the final
box-QP active set frozen (clamped controls held at their bounds).  Writing
that LQR's KKT system as K w = -h(theta), every gradient follows from one
solve with the loss gradient as right-hand side:

    d_tau = solution of the same LQR with linear term g_t = dL/dtau_t,
            x_init = 0, f_t = 0 and the clamped controls held at 0

    dL/dc_t       = d_tau_t
    dL/dC_t       = 1/2 (d_tau_t tau*_t' + tau*_t d_tau_t')
    dL/dx_init    = lambda_0 of that LQR = v_hat_0 (its value gradient at x=0)

With the diagonal surrogate C_t = diag(Q_t, R), c_t = [-Q_t x_ref_t; -R u_ref]:

    dL/dQ_t,i     = d_x,t,i (x*_t,i - x_ref,t,i)      (summed over t when Q is shared)
    dL/dx_ref,t   = -Q_t * d_x,t
    dL/dR_j       = sum_t d_u,t,j (u*_t,j - u_ref,j)
    dL/du_ref     = -R * sum_t d_u,t

``adjoint`` solves the LQR with the Riccati factorization of the final
backward pass (its K_t, free sets and Cholesky factors), ``dense_kkt_adjoint``
assembles and solves the whole KKT matrix by LU as an independent check, and
``frozen_lqr_solve`` is the primal LQR whose finite differences pin both.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import boxqp


@dataclasses.dataclass
class Gradients:
    dQ: np.ndarray      # like prob.Q
    dx_ref: np.ndarray  # [N, nx]
    dx0: np.ndarray     # [nx]
    dR: np.ndarray      # [nu]
    du_ref: np.ndarray  # [nu]
    dX: np.ndarray      # [N, nx]  d_tau (state part)
    dU: np.ndarray      # [N, nu]  d_tau (control part)
    dC: np.ndarray | None = None   # like prob.C: dL/dC_t (summed over t when C is shared)
    dc: np.ndarray | None = None   # like prob.c: dL/dc_t


def _assemble(prob, sol, dX, dU, dx0):
    n, N = prob.n, prob.x_ref.shape[0]
    nx, nu = dX.shape[1], dU.shape[1]
    dQ = np.zeros_like(prob.Q)
    dxr = np.zeros((N, nx))
    for t in range(n):
        e = sol.X[t] - prob.x_ref[t]
        if prob.Q.shape[0] > 1:
            dQ[t] = dX[t] * e
        else:
            dQ[0] += dX[t] * e
        dxr[t] = -prob.Qt(t) * dX[t]
    dR = np.zeros(nu)
    du_ref = np.zeros(nu)
    for t in range(n):
        dR += dU[t] * (sol.U[t] - prob.u_ref)
        du_ref += -prob.R * dU[t]
    # the general form: dL/dc_t = d_tau_t, dL/dC_t = 1/2 (d_tau_t tau*_t' + tau*_t d_tau_t')
    # (shaped like prob.C and prob.c; for the surrogate, C like Q and c per stage)
    nz = nx + nu
    NC = prob.C.shape[0] if prob.general else prob.Q.shape[0]
    Nc = prob.c.shape[0] if prob.general else N
    dC = np.zeros((NC, nz, nz))
    dc = np.zeros((Nc, nz))
    for t in range(n):
        d = np.concatenate([dX[t], dU[t]])
        z = np.concatenate([sol.X[t], sol.U[t]])
        dC[t if NC > 1 else 0] += 0.5 * (np.outer(d, z) + np.outer(z, d))
        dc[t if Nc > 1 else 0] += d
    return Gradients(dQ, dxr, dx0, dR, du_ref, dX, dU, dC, dc)


def adjoint(prob, sol, grad_x, grad_u) -> Gradients:
    """A8: backward affine sweep + forward sweep of the adjoint LQR reusing
    the final factorization (K_t, free set, Cholesky of Q_uu,ff)."""
    n, N = prob.n, prob.x_ref.shape[0]
    nx, nu = prob.x0.shape[0], prob.u_ref.shape[0]
    bp, F = sol.bp, sol.F
    vh = np.zeros(nx)
    khat = [None] * n
    for t in reversed(range(n)):
        g = np.concatenate([grad_x[t], grad_u[t]])
        qh = g + (F[t].T @ vh if t < n - 1 else 0.0)
        qhx, qhu = qh[:nx], qh[nx:]
        kh = np.zeros(nu)
        fi = np.flatnonzero(bp.free[t])
        if fi.size:
            kh[fi] = -boxqp.chol_solve(bp.L[t], qhu[fi])
        K, Quu, Qux = bp.K[t], bp.Quu[t], bp.Qux[t]
        vh = qhx + K.T @ Quu @ kh + K.T @ qhu + Qux.T @ kh
        khat[t] = kh
    dX = np.zeros((N, nx))
    dU = np.zeros((N, nu))
    dx = np.zeros(nx)
    for t in range(n):
        du = bp.K[t] @ dx + khat[t]
        dX[t], dU[t] = dx, du
        if t < n - 1:
            dx = F[t] @ np.concatenate([dx, du])
    return _assemble(prob, sol, dX, dU, vh)


def _kkt_matrix(prob, sol):
    """KKT matrix [[H, E'], [E, 0]] of the frozen LQR and the row bookkeeping."""
    n = prob.n
    nx, nu = prob.x0.shape[0], prob.u_ref.shape[0]
    nz = nx + nu
    H = np.zeros((n * nz, n * nz))
    for t in range(n):
        H[t * nz:(t + 1) * nz, t * nz:(t + 1) * nz] = prob.Ct(t)
    rows = []
    # x_0 = x_init
    for i in range(nx):
        r = np.zeros(n * nz)
        r[i] = 1.0
        rows.append(r)
    # x_{t+1} - F_t tau_t = f_t
    for t in range(n - 1):
        for i in range(nx):
            r = np.zeros(n * nz)
            r[(t + 1) * nz + i] = 1.0
            r[t * nz:(t + 1) * nz] -= sol.F[t][i]
            rows.append(r)
    # clamped controls fixed
    clamped = []
    for t in range(n):
        for j in range(nu):
            if not sol.bp.free[t][j]:
                r = np.zeros(n * nz)
                r[t * nz + nx + j] = 1.0
                rows.append(r)
                clamped.append((t, j))
    E = np.array(rows)
    m = E.shape[0]
    Kkt = np.zeros((n * nz + m, n * nz + m))
    Kkt[:n * nz, :n * nz] = H
    Kkt[:n * nz, n * nz:] = E.T
    Kkt[n * nz:, :n * nz] = E
    return Kkt, n * nz, clamped


def dense_kkt_adjoint(prob, sol, grad_x, grad_u) -> Gradients:
    """Independent check of ``adjoint``: assemble the frozen LQR's KKT matrix
    and solve [[H, E'], [E, 0]] [d_tau; nu] = [-g; 0] by LU (numpy.linalg.solve);
    dL/dx_init = -nu on the x_0 = x_init rows."""
    n, N = prob.n, prob.x_ref.shape[0]
    nx, nu = prob.x0.shape[0], prob.u_ref.shape[0]
    nz = nx + nu
    Kkt, nv, _ = _kkt_matrix(prob, sol)
    rhs = np.zeros(Kkt.shape[0])
    for t in range(n):
        rhs[t * nz:t * nz + nx] = -grad_x[t]
        rhs[t * nz + nx:(t + 1) * nz] = -grad_u[t]
    w = np.linalg.solve(Kkt, rhs)
    dX = np.zeros((N, nx))
    dU = np.zeros((N, nu))
    for t in range(n):
        dX[t] = w[t * nz:t * nz + nx]
        dU[t] = w[t * nz + nx:(t + 1) * nz]
    dx0 = -w[nv:nv + nx]
    return _assemble(prob, sol, dX, dU, dx0)


def frozen_lqr_solve(prob, sol, model, Q=None, x_ref=None, x0=None, R=None, u_ref=None, C=None, c=None):
    """Primal solution of the frozen LQR at tau* for perturbed cost / initial
    state: dynamics x_{t+1} = F_t tau_t + f_t with f_t = f(tau*_t) - F_t tau*_t,
    clamped controls held at u*.  Returns (X, U).  Finite differences of
    g . tau through this map pin the adjoint gradients."""
    n, N = prob.n, prob.x_ref.shape[0]
    nx, nu = prob.x0.shape[0], prob.u_ref.shape[0]
    nz = nx + nu
    Q = prob.Q if Q is None else Q
    x_ref = prob.x_ref if x_ref is None else x_ref
    x0 = prob.x0 if x0 is None else x0
    R = prob.R if R is None else R
    u_ref = prob.u_ref if u_ref is None else u_ref
    C = prob.C if C is None else C
    c = prob.c if c is None else c
    p2 = dataclasses.replace(prob, Q=Q, x_ref=x_ref, x0=x0, R=R, u_ref=u_ref, C=C, c=c)
    Kkt, nv, clamped = _kkt_matrix(p2, sol)
    rhs = np.zeros(Kkt.shape[0])
    for t in range(n):
        rhs[t * nz:(t + 1) * nz] = -p2.ct(t)
    r = nv
    rhs[r:r + nx] = x0
    r += nx
    for t in range(n - 1):
        zt = np.concatenate([sol.X[t], sol.U[t]])
        ft = model.step(sol.X[t], sol.U[t]) - sol.F[t] @ zt
        rhs[r:r + nx] = ft
        r += nx
    for (t, j) in clamped:
        rhs[r] = sol.U[t][j]
        r += 1
    w = np.linalg.solve(Kkt, rhs)
    X = np.zeros((N, nx))
    U = np.zeros((N, nu))
    for t in range(n):
        X[t] = w[t * nz:t * nz + nx]
        U[t] = w[t * nz + nx:(t + 1) * nz]
    return X, U
