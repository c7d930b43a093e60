"""Pins of the oracle's general stage cost, Eq. (2): 1/2 z' C_t z + c_t' z with a
symmetric positive semidefinite C_t (cross terms between states and controls
included), and of its gradients dL/dC_t, dL/dc_t.

Independent references: the normal equations of whole linear-quadratic
problems, the dense KKT solve, central finite differences, and the diagonal
surrogate of the same cost.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import adjoint, ilqr
from oracle.model import LinearModel, Quadrotor

QUAD = Quadrotor(W.DEFAULT_MODEL)


def _surrogate_as_general(prob):
    """The same problem with C_t = diag(Q_t, R) and c_t = [-Q_t x_ref_t; -R u_ref]
    given explicitly (C shared when Q is, c per stage)."""
    N = prob.x_ref.shape[0]
    C = np.stack([np.diag(np.concatenate([q, prob.R])) for q in prob.Q])
    c = np.stack([np.concatenate([-prob.Qt(t) * prob.x_ref[t], -prob.R * prob.u_ref]) for t in range(N)])
    return dataclasses.replace(prob, C=C, c=c)


@pytest.mark.parametrize("seed,cfg", [(0, "hover"), (2, "track")])
def test_diagonal_C_reproduces_the_surrogate(seed, cfg):
    """With C_t = diag(Q_t, R) the general path solves the same problem:
    same controls and states, a cost lower by the constant
    sum_t 1/2 (x_ref' Q x_ref + u_ref' R u_ref), and dL/dQ_t,i equal to
    dL/dC_t,ii - x_ref_t,i dL/dc_t,i (chain rule through both)."""
    b = W.hover_targets(4, 8, seed=seed) if cfg == "hover" else W.race_track(4, 8, seed=seed)
    prob = ilqr.problem_from_batch(b, seed % 4)
    gen = _surrogate_as_general(prob)
    s0 = ilqr.solve(QUAD, prob, max_iter=30, tol=1e-10)
    s1 = ilqr.solve(QUAD, gen, max_iter=30, tol=1e-10)
    assert s0.status == s1.status == ilqr.CONVERGED
    np.testing.assert_allclose(s1.U, s0.U, atol=1e-8)
    np.testing.assert_allclose(s1.X, s0.X, atol=1e-8)
    const = sum(0.5 * (prob.x_ref[t] @ (prob.Qt(t) * prob.x_ref[t]) + prob.u_ref @ (prob.R * prob.u_ref))
                for t in range(prob.n))
    J0, J1 = ilqr.total_cost(prob, s0.X, s0.U), ilqr.total_cost(gen, s1.X, s1.U)
    assert abs((J1 + const) - J0) <= 1e-9 * max(1.0, const)
    rng = np.random.default_rng(seed)
    gx, gu = rng.normal(size=prob.x_ref.shape), rng.normal(size=(prob.x_ref.shape[0], 4))
    g0 = adjoint.adjoint(prob, s0, gx, gu)
    g1 = adjoint.adjoint(gen, s1, gx, gu)
    dQ = np.diagonal(g1.dC[0])[:13] - sum(prob.x_ref[t] * g1.dc[t][:13] for t in range(prob.n))
    np.testing.assert_allclose(dQ, g0.dQ[0], rtol=1e-7, atol=1e-9 * max(1.0, np.max(np.abs(g0.dQ))))
    np.testing.assert_allclose(g1.dx0, g0.dx0, rtol=1e-7, atol=1e-10)


def _general_lq(rng, nx=4, nu=2, N=6, bound=1e6):
    """Linear dynamics and a dense cost: C_t = M_t' M_t + 0.1 I (state-control
    cross terms included), c_t ~ N(0, 1), per stage."""
    nz = nx + nu
    A = rng.normal(scale=0.4, size=(nx, nx)) + 0.8 * np.eye(nx)
    A /= max(1.0, np.max(np.abs(np.linalg.eigvals(A))) / 0.95)
    B = rng.normal(size=(nx, nu))
    f0 = rng.normal(scale=0.1, size=nx)
    M = rng.normal(size=(N, nz, nz))
    C = np.einsum("tki,tkj->tij", M, M) + 0.1 * np.eye(nz)
    c = rng.normal(size=(N, nz))
    prob = ilqr.Problem(x0=rng.normal(size=nx), Q=np.ones((1, nx)), x_ref=np.zeros((N, nx)),
                        R=np.ones(nu), u_ref=rng.normal(scale=0.2, size=nu), u_lo=np.full(nu, -bound),
                        u_hi=np.full(nu, bound), n=N, C=C, c=c)
    return LinearModel(A, B, f0), prob


def _normal_equations_controls(model, prob):
    """Whole-horizon reduced problem: z_t = G_t U + h_t is affine in the
    stacked controls U, so the cost is 1/2 U' H U + g' U + const with
    H = sum_t G_t' C_t G_t and g = sum_t G_t' (C_t h_t + c_t); U* = -H^-1 g."""
    N, nx, nu = prob.n, model.nx, model.nu
    Gx, hx = np.zeros((nx, N * nu)), prob.x0.copy()
    H = np.zeros((N * nu, N * nu))
    g = np.zeros(N * nu)
    for t in range(N):
        Gu = np.zeros((nu, N * nu))
        Gu[:, t * nu:(t + 1) * nu] = np.eye(nu)
        G = np.vstack([Gx, Gu])
        h = np.concatenate([hx, np.zeros(nu)])
        H += G.T @ prob.Ct(t) @ G
        g += G.T @ (prob.Ct(t) @ h + prob.ct(t))
        Gx = model.A @ Gx + model.B @ Gu
        hx = model.A @ hx + model.f0
    return np.linalg.solve(H, -g).reshape(N, nu)


@pytest.mark.parametrize("seed", range(4))
def test_general_lq_one_iteration_is_exact(seed):
    """Linear dynamics, dense C_t, inactive bounds: the first iteration at
    alpha = 1 lands on the solution of the normal equations, and the adjoint
    sweep equals the dense KKT solve."""
    rng = np.random.default_rng(300 + seed)
    model, prob = _general_lq(rng)
    sol = ilqr.solve(model, prob, max_iter=1, tol=0.0)
    U_exact = _normal_equations_controls(model, prob)
    np.testing.assert_allclose(sol.U, U_exact, atol=1e-9 * max(1.0, np.max(np.abs(U_exact))))
    assert sol.alpha_hist[0] == 1.0
    sol = ilqr.solve(model, prob, max_iter=5, tol=1e-12)
    gx, gu = rng.normal(size=(prob.n, model.nx)), rng.normal(size=(prob.n, model.nu))
    a = adjoint.adjoint(prob, sol, gx, gu)
    d = adjoint.dense_kkt_adjoint(prob, sol, gx, gu)
    for name in ("dX", "dU", "dx0", "dC", "dc"):
        va, vd = getattr(a, name), getattr(d, name)
        np.testing.assert_allclose(va, vd, rtol=1e-9, atol=1e-10 * max(1.0, np.max(np.abs(vd))))


def _general_quad(seed, N=8):
    """Quadrotor instance with a dense shared C = diag(Q, R) + 0.05 M'M
    (state-control cross terms) and c_t = -C z_ref,t per stage."""
    b = W.hover_targets(4, N, seed=seed)
    base = ilqr.problem_from_batch(b, seed % 4)
    rng = np.random.default_rng(50 + seed)
    M = rng.normal(size=(17, 17))
    C = np.diag(np.concatenate([base.Q[0], base.R])) + 0.05 * (M.T @ M) / 17
    c = np.stack([-C @ np.concatenate([base.x_ref[t], base.u_ref]) for t in range(N)])
    prob = dataclasses.replace(base, C=C[None], c=c)
    sol = ilqr.solve(QUAD, prob, max_iter=40, tol=1e-10)
    return prob, sol


@pytest.mark.parametrize("seed", [1, 2])
def test_general_adjoint_matches_finite_differences_of_frozen_lqr(seed):
    """Central differences of L = g . tau through the frozen LQR with respect
    to c_t (every entry) and to symmetric perturbations of the shared C
    (C_ij and C_ji together: dL = dL/dC_ij + dL/dC_ji)."""
    prob, sol = _general_quad(seed)
    assert sol.status == ilqr.CONVERGED
    rng = np.random.default_rng(seed + 11)
    N = prob.x_ref.shape[0]
    gx, gu = rng.normal(size=(N, 13)), rng.normal(size=(N, 4))
    gr = adjoint.adjoint(prob, sol, gx, gu)
    d = adjoint.dense_kkt_adjoint(prob, sol, gx, gu)
    np.testing.assert_allclose(gr.dC, d.dC, rtol=1e-9, atol=1e-10 * np.max(np.abs(d.dC)))

    def L(**kw):
        X, U = adjoint.frozen_lqr_solve(prob, sol, QUAD, **kw)
        return np.sum(gx * X) + np.sum(gu * U)

    eps = 1e-4
    num_c = np.zeros_like(prob.c)
    for idx in np.ndindex(prob.c.shape):
        p, m = prob.c.copy(), prob.c.copy()
        p[idx] += eps
        m[idx] -= eps
        num_c[idx] = (L(c=p) - L(c=m)) / (2 * eps)
    assert np.linalg.norm(num_c - gr.dc) / np.linalg.norm(num_c) < 1e-6
    pairs = [(i, i) for i in (0, 4, 9, 14)] + [(int(i), int(j)) for i, j in rng.integers(0, 17, size=(12, 2)) if i != j]
    for i, j in pairs:
        E = np.zeros((17, 17))
        E[i, j] = E[j, i] = 1.0
        h = eps * min(1.0, max(abs(prob.C[0, i, j]), 1e-2))     # relative for small entries (R = 0.01)
        num = (L(C=prob.C + h * E[None]) - L(C=prob.C - h * E[None])) / (2 * h)
        ana = gr.dC[0, i, j] if i == j else gr.dC[0, i, j] + gr.dC[0, j, i]
        assert abs(num - ana) <= 1e-6 * max(1.0, abs(num)), (i, j, num, ana)


@pytest.mark.parametrize("seed", range(2))
def test_general_adjoint_matches_fd_of_whole_solver_linear_dynamics(seed):
    """Linear dynamics and a dense cost with bounds partly active: finite
    differences of the whole iLQR solve agree with dL/dc_t and dL/dC_t."""
    rng = np.random.default_rng(400 + seed)
    model, prob = _general_lq(rng, bound=0.5)
    sol = ilqr.solve(model, prob, max_iter=60, tol=1e-13)
    assert sol.status in (ilqr.CONVERGED, ilqr.STALLED)
    gx, gu = rng.normal(size=(prob.n, model.nx)), rng.normal(size=(prob.n, model.nu))
    gr = adjoint.adjoint(prob, sol, gx, gu)

    def L(p):
        s = ilqr.solve(model, p, max_iter=60, tol=1e-13)
        return np.sum(gx * s.X) + np.sum(gu * s.U)

    eps = 1e-6
    num_c = np.zeros_like(prob.c)
    for idx in np.ndindex(prob.c.shape):
        p, m = prob.c.copy(), prob.c.copy()
        p[idx] += eps
        m[idx] -= eps
        num_c[idx] = (L(dataclasses.replace(prob, c=p)) - L(dataclasses.replace(prob, c=m))) / (2 * eps)
    assert np.linalg.norm(num_c - gr.dc) / np.linalg.norm(num_c) < 1e-5
    for t, i, j in ((0, 0, 0), (2, 1, 4), (5, 3, 5), (3, 5, 5)):
        E = np.zeros_like(prob.C)
        E[t, i, j] = E[t, j, i] = 1.0
        num = (L(dataclasses.replace(prob, C=prob.C + eps * E)) -
               L(dataclasses.replace(prob, C=prob.C - eps * E))) / (2 * eps)
        ana = gr.dC[t, i, j] if i == j else gr.dC[t, i, j] + gr.dC[t, j, i]
        assert abs(num - ana) <= 1e-5 * max(1.0, abs(num)), (t, i, j, num, ana)


@pytest.mark.parametrize("general", [False, True])
def test_stagewise_cost_change_is_the_difference_of_costs(general):
    """Reading R4: the line search compares candidates by the stage-wise cost
    change d'(C (z + d/2) + c); for the quadratic cost it equals
    J(z + d) - J(z) exactly (up to rounding), for the diagonal and the
    general form, and its scale bounds the terms."""
    rng = np.random.default_rng(21)
    b = W.hover_targets(2, 7, seed=22)
    prob = ilqr.problem_from_batch(b, 1)
    if general:
        M = rng.normal(size=(7, 17, 17))
        C = np.einsum("tki,tkj->tij", M, M) / 17 + np.diag(np.concatenate([prob.Q[0], prob.R]))
        prob = dataclasses.replace(prob, C=C, c=rng.normal(size=(7, 17)))
    X, U = rng.normal(size=(7, 13)), rng.normal(size=(7, 4)) + 2.0
    Xa, Ua = X + 0.1 * rng.normal(size=X.shape), U + 0.1 * rng.normal(size=U.shape)
    dJ, scale = ilqr.cost_change(prob, X, U, Xa, Ua, with_scale=True)
    ref = ilqr.total_cost(prob, Xa, Ua) - ilqr.total_cost(prob, X, U)
    assert abs(dJ - ref) <= 1e-12 * max(1.0, abs(ilqr.total_cost(prob, X, U)))
    assert scale >= abs(dJ)
