"""Pins of the oracle's box QP, iLQR forward solve and adjoint backward pass.

Independent references: brute-force active-set enumeration, scipy's bounded
least squares, dense KKT solves of whole linear-quadratic problems (LU), and
central finite differences.
"""
import dataclasses

import numpy as np
import pytest
from scipy.optimize import lsq_linear

import workloads as W
from oracle import boxqp, ilqr, adjoint
from oracle.model import Quadrotor, LinearModel

QUAD = Quadrotor(W.DEFAULT_MODEL)


# ------------------------------------------------------------------ box QP ------

@pytest.mark.parametrize("seed", range(40))
def test_boxqp_matches_enumeration(seed):
    """The unique KKT point of a strictly convex 4-d box QP, found by trying
    all 3^4 = 81 active sets, equals the projected-Newton result."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(4, 4))
    H = A @ A.T + 0.05 * np.eye(4)
    g = rng.normal(scale=3.0, size=4)
    lo = -rng.uniform(0.0, 1.0, 4)
    hi = rng.uniform(0.0, 1.0, 4)
    if seed % 5 == 0:
        lo[0] = 0.0          # a control sitting exactly on its bound
    d, free, L, ok = boxqp.solve(H, g, lo, hi)
    assert ok
    sols = boxqp.enumerate_kkt(H, g, lo, hi)
    assert len(sols) >= 1
    np.testing.assert_allclose(d, sols[0], atol=1e-10)
    # the factor belongs to H restricted to the returned free set
    fi = np.flatnonzero(free)
    if fi.size:
        np.testing.assert_allclose(L @ L.T, H[np.ix_(fi, fi)], atol=1e-12)
    # every clamped dimension sits on a bound with its gradient pointing out
    grad = g + H @ d
    for i in np.flatnonzero(~free):
        assert (d[i] == lo[i] and grad[i] > 0) or (d[i] == hi[i] and grad[i] < 0)


# Stage 0 of a race-track instance's fourth iteration: two rotors at their
# 0 N bound (u = [2.2387, 0, 0, 1.0517] N), the rotor pairs nearly collinear in H.
NEAR_H = np.array([[8.29442083, -8.24721083, 1.51574164, -1.65046398],
                   [-8.24721083, 8.68940243, -1.57066555, 1.50579661],
                   [1.51574164, -1.57066555, 8.408479, -8.05725247],
                   [-1.65046398, 1.50579661, -8.05725247, 8.1897023]])
NEAR_G = np.array([-2.17662926, 3.60192572, 2.73650408, -1.44773018])
NEAR_U = np.array([2.23866527, 0.0, 0.0, 1.05174372])


@pytest.mark.parametrize("shift", [0.0, 1e-12, -1e-12, 3e-7])
def test_boxqp_near_bound_controls_match_enumeration(shift):
    """Controls a rounding error (or a fraction of the epsilon-active width)
    inside their bound, with the gradient pointing out of the box: the QP
    clamps them (Bertsekas' epsilon-active set) and returns the unique KKT
    point, the same for every shift, instead of a result that jumps with
    the rounding of its inputs."""
    u = NEAR_U.copy()
    u[1] += abs(shift)
    u[2] += abs(shift)
    lo, hi = -u, 8.5 - u
    d, free, L, ok = boxqp.solve(NEAR_H, NEAR_G, lo, hi)
    assert ok
    sols = boxqp.enumerate_kkt(NEAR_H, NEAR_G, lo, hi)
    assert len(sols) == 1
    np.testing.assert_allclose(d, sols[0], atol=1e-9)
    np.testing.assert_array_equal(free, [True, False, False, True])
    # the clamped controls sit exactly on their bound
    assert d[1] == lo[1] and d[2] == lo[2]


@pytest.mark.parametrize("seed", range(20))
def test_boxqp_epsilon_active_matches_enumeration(seed):
    """Random strictly convex QPs whose start lies within the epsilon-active
    width of a bound in some dimensions: the result is the enumerated KKT
    point of the same QP to within that width."""
    rng = np.random.default_rng(100 + seed)
    A = rng.normal(size=(4, 4))
    H = A @ A.T + 0.05 * np.eye(4)
    g = rng.normal(scale=3.0, size=4)
    lo = -rng.uniform(0.0, 1.0, 4)
    hi = rng.uniform(0.0, 1.0, 4)
    near = rng.integers(0, 4)
    if seed % 2:
        lo[near] = -0.5 * boxqp.EPS_REL * (1.0 + hi[near] - lo[near]) * rng.uniform()
    else:
        hi[near] = 0.5 * boxqp.EPS_REL * (1.0 + hi[near] - lo[near]) * rng.uniform()
    d, free, L, ok = boxqp.solve(H, g, lo, hi)
    assert ok
    sols = boxqp.enumerate_kkt(H, g, lo, hi)
    assert len(sols) >= 1
    np.testing.assert_allclose(d, sols[0], atol=1e-5)


def test_boxqp_interior_is_newton_step():
    H = np.diag([2.0, 3.0, 4.0, 5.0])
    g = np.array([0.1, -0.2, 0.3, -0.4])
    d, free, L, ok = boxqp.solve(H, g, -np.ones(4), np.ones(4))
    np.testing.assert_allclose(d, -g / np.diag(H), atol=1e-15)
    assert free.all()


def test_boxqp_reports_non_pd():
    H = np.diag([1.0, -1.0, 1.0, 1.0])
    d, free, L, ok = boxqp.solve(H, np.ones(4), -np.ones(4), np.ones(4))
    assert not ok


# ------------------------------------------------------- linear-quadratic pins ----

def _lq_instance(rng, nx=4, nu=2, N=6, bound=1e6):
    A = rng.normal(scale=0.4, size=(nx, nx)) + 0.8 * np.eye(nx)
    A /= max(1.0, np.max(np.abs(np.linalg.eigvals(A))) / 0.95)
    B = rng.normal(size=(nx, nu))
    f0 = rng.normal(scale=0.1, size=nx)
    prob = ilqr.Problem(x0=rng.normal(size=nx), Q=rng.uniform(0.1, 10, size=(N, nx)),
                        x_ref=rng.normal(size=(N, nx)), R=rng.uniform(0.05, 1.0, nu),
                        u_ref=rng.normal(scale=0.2, size=nu), u_lo=np.full(nu, -bound),
                        u_hi=np.full(nu, bound), n=N)
    return LinearModel(A, B, f0), prob


def _dense_lq_controls(model, prob):
    """Whole-horizon reduced least squares: x = Phi x0 + Gamma U + const, cost
    1/2 |sqrt(Q)(x - x_ref)|^2 + 1/2 |sqrt(R)(u - u_ref)|^2, solved by scipy's
    bounded linear least squares (exact for these convex problems)."""
    N, nx, nu = prob.n, model.nx, model.nu
    # affine map from U (flattened) to each x_t
    Gam = [np.zeros((nx, N * nu))]
    c = [prob.x0.copy()]
    for t in range(N - 1):
        G = model.A @ Gam[t]
        G[:, t * nu:(t + 1) * nu] += model.B
        Gam.append(G)
        c.append(model.A @ c[t] + model.f0)
    rows, rhs = [], []
    for t in range(N):
        sq = np.sqrt(prob.Qt(t))
        rows.append(sq[:, None] * Gam[t])
        rhs.append(sq * (prob.x_ref[t] - c[t]))
        E = np.zeros((nu, N * nu))
        E[:, t * nu:(t + 1) * nu] = np.diag(np.sqrt(prob.R))
        rows.append(E)
        rhs.append(np.sqrt(prob.R) * prob.u_ref)
    Mx = np.vstack(rows)
    b = np.concatenate(rhs)
    lo = np.tile(prob.u_lo, N)
    hi = np.tile(prob.u_hi, N)
    res = lsq_linear(Mx, b, bounds=(lo, hi), method="bvls", tol=1e-14, lsmr_tol=None)
    return res.x.reshape(N, nu)


@pytest.mark.parametrize("seed", range(6))
def test_lq_one_iteration_is_exact_lqr(seed):
    """Linear dynamics, quadratic cost, inactive bounds: the first iteration at
    alpha = 1 lands on the exact LQR optimum (the dense least-squares
    solution); J(alpha) is a quadratic in alpha with its minimum at 1."""
    rng = np.random.default_rng(seed)
    model, prob = _lq_instance(rng)
    sol = ilqr.solve(model, prob, max_iter=1, tol=0.0)
    U_exact = _dense_lq_controls(model, prob)
    np.testing.assert_allclose(sol.U, U_exact, atol=1e-9)
    assert sol.alpha_hist[0] == 1.0
    # J along the line search is quadratic in alpha with minimum at alpha = 1
    X0 = model.rollout(prob.x0, np.tile(prob.u_ref, (prob.n, 1)))
    U0 = np.tile(prob.u_ref, (prob.n, 1))
    bp = ilqr.backward_pass(prob, X0, U0, ilqr.linearize(model, prob, X0, U0))
    Js = []
    alphas = np.linspace(0, 2, 9)
    for a in alphas:
        Xa, Ua = ilqr.forward_pass(model, prob, X0, U0, bp, a)
        Js.append(ilqr.total_cost(prob, Xa, Ua))
    coef = np.polyfit(alphas, Js, 2)
    assert abs(-coef[1] / (2 * coef[0]) - 1.0) < 1e-9
    np.testing.assert_allclose(np.polyval(coef, alphas), Js, rtol=1e-10)
    # the second iteration makes no further change: converged
    sol2 = ilqr.solve(model, prob, max_iter=5, tol=1e-9)
    assert sol2.status in (ilqr.CONVERGED, ilqr.STALLED)
    assert sol2.iters == 2


@pytest.mark.parametrize("seed", range(6))
def test_box_lq_converges_to_bounded_least_squares(seed):
    """Linear dynamics with active bounds: converged box-DDP equals the global
    optimum of the convex box-constrained QP (scipy BVLS)."""
    rng = np.random.default_rng(50 + seed)
    model, prob = _lq_instance(rng, bound=0.3)
    sol = ilqr.solve(model, prob, max_iter=60, tol=1e-12)
    assert sol.status in (ilqr.CONVERGED, ilqr.STALLED)
    U_exact = _dense_lq_controls(model, prob)
    assert np.sum(np.isclose(np.abs(U_exact), 0.3)) > 0      # bounds do bind
    np.testing.assert_allclose(sol.U, U_exact, atol=1e-7)


def test_box_lq_tiny_matches_active_set_enumeration():
    """N * nu = 8: enumerate all 3^8 assignments of (free, lower, upper) to
    every control, solve each equality-constrained QP, keep the KKT point."""
    rng = np.random.default_rng(11)
    model, prob = _lq_instance(rng, nx=2, nu=2, N=4, bound=0.25)
    N, nx, nu = prob.n, 2, 2
    # reduced quadratic in U: 1/2 U'HU + g'U
    Gam = [np.zeros((nx, N * nu))]
    c = [prob.x0.copy()]
    for t in range(N - 1):
        G = model.A @ Gam[t]
        G[:, t * nu:(t + 1) * nu] += model.B
        Gam.append(G)
        c.append(model.A @ c[t] + model.f0)
    H = np.zeros((N * nu, N * nu))
    g = np.zeros(N * nu)
    for t in range(N):
        Qd = np.diag(prob.Qt(t))
        H += Gam[t].T @ Qd @ Gam[t]
        g += Gam[t].T @ Qd @ (c[t] - prob.x_ref[t])
        H[t * nu:(t + 1) * nu, t * nu:(t + 1) * nu] += np.diag(prob.R)
        g[t * nu:(t + 1) * nu] -= prob.R * prob.u_ref
    lo = np.tile(prob.u_lo, N)
    hi = np.tile(prob.u_hi, N)
    sols = boxqp.enumerate_kkt(H, g, lo, hi)
    assert len(sols) == 1
    sol = ilqr.solve(model, prob, max_iter=60, tol=1e-13)
    np.testing.assert_allclose(sol.U[:N].ravel(), sols[0], atol=1e-8)


def test_hover_fixed_point_of_solver():
    """x0 = x_ref = hover and u_ref = m g / 4: the start is optimal, cost 0,
    the first step is zero (CONVERGED after one iteration), and dL/dQ = 0
    because x* = x_ref."""
    N = 10
    x0 = np.zeros(13)
    x0[0:3] = [0.5, -0.2, 2.0]
    x0[3] = 1.0
    prob = ilqr.Problem(x0=x0, Q=np.full((1, 13), 3.0), x_ref=np.tile(x0, (N, 1)),
                        R=np.full(4, 0.01), u_ref=np.full(4, W.DEFAULT_MODEL.hover_thrust),
                        u_lo=np.zeros(4), u_hi=np.full(4, 8.5), n=N)
    sol = ilqr.solve(QUAD, prob, max_iter=10, tol=1e-6)
    np.testing.assert_allclose(sol.U, W.DEFAULT_MODEL.hover_thrust, atol=1e-12)
    assert abs(sol.J) < 1e-20
    assert sol.status == ilqr.CONVERGED and sol.iters == 1
    gx = np.zeros((N, 13))
    gu = np.zeros((N, 4))
    gu[0] = 1.0
    gr = adjoint.adjoint(prob, sol, gx, gu)
    np.testing.assert_allclose(gr.dQ, 0.0, atol=1e-14)


# ----------------------------------------------------------------- adjoint ----

def _quad_solution(seed, N=8, cfg="hover"):
    b = W.hover_targets(4, N, seed=seed) if cfg == "hover" else W.race_track(4, N, seed=seed)
    prob = ilqr.problem_from_batch(b, seed % 4)
    sol = ilqr.solve(QUAD, prob, max_iter=30, tol=1e-10)
    return prob, sol


@pytest.mark.parametrize("seed,cfg", [(0, "hover"), (1, "hover"), (2, "track"), (3, "track")])
def test_adjoint_matches_dense_kkt(seed, cfg):
    """The Riccati adjoint sweep equals the LU solve of the whole frozen-LQR
    KKT system, for d_tau and every gradient block."""
    prob, sol = _quad_solution(seed, cfg=cfg)
    rng = np.random.default_rng(seed)
    gx = rng.normal(size=prob.x_ref.shape)
    gu = rng.normal(size=(prob.x_ref.shape[0], 4))
    a = adjoint.adjoint(prob, sol, gx, gu)
    d = adjoint.dense_kkt_adjoint(prob, sol, gx, gu)
    for name in ("dX", "dU", "dQ", "dx_ref", "dx0", "dR", "du_ref"):
        va, vd = getattr(a, name), getattr(d, name)
        np.testing.assert_allclose(va, vd, rtol=1e-9, atol=1e-10 * max(1.0, np.max(np.abs(vd))))


@pytest.mark.parametrize("seed,cfg", [(0, "hover"), (2, "track")])
def test_converged_solution_is_its_own_frozen_lqr(seed, cfg):
    """At a converged iterate the frozen LQR (same cost, dynamics linearised
    at tau*, clamped controls held) is solved by tau* itself."""
    prob, sol = _quad_solution(seed, cfg=cfg)
    assert sol.status in (ilqr.CONVERGED, ilqr.STALLED)
    X, U = adjoint.frozen_lqr_solve(prob, sol, QUAD)
    np.testing.assert_allclose(U, sol.U, atol=1e-6)
    np.testing.assert_allclose(X, sol.X, atol=1e-6)


@pytest.mark.parametrize("seed,cfg", [(0, "hover"), (3, "track")])
def test_adjoint_matches_finite_differences_of_frozen_lqr(seed, cfg):
    """Central differences (eps = 1e-4) of L = g . tau through the frozen LQR
    solve with respect to Q, x_ref, x0, R and u_ref."""
    prob, sol = _quad_solution(seed, cfg=cfg)
    rng = np.random.default_rng(seed + 7)
    N = prob.x_ref.shape[0]
    gx = rng.normal(size=(N, 13))
    gu = rng.normal(size=(N, 4))
    gr = adjoint.adjoint(prob, sol, gx, gu)

    def L(**kw):
        X, U = adjoint.frozen_lqr_solve(prob, sol, QUAD, **kw)
        return np.sum(gx * X) + np.sum(gu * U)

    def fd(name, base):
        out = np.zeros_like(base)
        for idx in np.ndindex(base.shape):
            # eps = 1e-4, relative for parameters far below 1 (R = 0.01)
            eps = 1e-4 * min(1.0, max(abs(base[idx]), 1e-2))
            p, m = base.copy(), base.copy()
            p[idx] += eps
            m[idx] -= eps
            out[idx] = (L(**{name: p}) - L(**{name: m})) / (2 * eps)
        return out

    for name, base, ana in (("Q", prob.Q, gr.dQ), ("x_ref", prob.x_ref, gr.dx_ref),
                            ("x0", prob.x0, gr.dx0), ("R", prob.R, gr.dR),
                            ("u_ref", prob.u_ref, gr.du_ref)):
        num = fd(name, base)
        scale = max(1e-9, np.linalg.norm(num))
        assert np.linalg.norm(num - ana) / scale < 1e-6, name


@pytest.mark.parametrize("seed", range(3))
def test_adjoint_matches_fd_of_whole_solver_linear_dynamics(seed):
    """Linear dynamics (one iteration is exact, bounds partly active): finite
    differences of the whole iLQR solve agree with the adjoint gradients."""
    rng = np.random.default_rng(200 + seed)
    model, prob = _lq_instance(rng, bound=0.6 if seed else 1e6)
    sol = ilqr.solve(model, prob, max_iter=60, tol=1e-13)
    N = prob.n
    gx = rng.normal(size=(N, model.nx))
    gu = rng.normal(size=(N, model.nu))
    gr = adjoint.adjoint(prob, sol, gx, gu)

    def L(p):
        s = ilqr.solve(model, p, max_iter=60, tol=1e-13)
        return np.sum(gx * s.X) + np.sum(gu * s.U)

    eps = 1e-5
    for name, ana in (("x0", gr.dx0), ("x_ref", gr.dx_ref), ("Q", gr.dQ)):
        base = getattr(prob, name)
        num = np.zeros_like(base)
        for idx in np.ndindex(base.shape):
            p, m = base.copy(), base.copy()
            p[idx] += eps
            m[idx] -= eps
            num[idx] = (L(dataclasses.replace(prob, **{name: p})) -
                        L(dataclasses.replace(prob, **{name: m}))) / (2 * eps)
        assert np.linalg.norm(num - ana) / max(1e-9, np.linalg.norm(num)) < 1e-5, name


def test_quadrotor_whole_solver_fd_gap_is_small():
    """Reading R10: on the nonlinear model the adjoint differentiates the LQR
    at tau* (Gauss-Newton, no second derivatives of f), so finite differences of
    the whole solver differ by that neglected term.  The gap is reported, and
    only bounded loosely here."""
    prob, sol = _quad_solution(1)
    N = prob.x_ref.shape[0]
    gu = np.zeros((N, 4))
    gu[0] = 1.0
    gx = np.zeros((N, 13))
    gr = adjoint.adjoint(prob, sol, gx, gu)

    def L(p):
        s = ilqr.solve(QUAD, p, max_iter=40, tol=1e-12)
        return np.sum(s.U[0])

    eps = 1e-5
    num = np.zeros(13)
    for i in range(13):
        p, m = prob.x0.copy(), prob.x0.copy()
        p[i] += eps
        m[i] -= eps
        num[i] = (L(dataclasses.replace(prob, x0=p)) - L(dataclasses.replace(prob, x0=m))) / (2 * eps)
    gap = np.linalg.norm(num - gr.dx0) / np.linalg.norm(num)
    cos = np.dot(num, gr.dx0) / (np.linalg.norm(num) * np.linalg.norm(gr.dx0))
    print(f"whole-solver FD gap (R10) = {gap:.3f}, cosine = {cos:.4f}")
    # a sign or index slip would give gap ~ 1-2 and cosine <= 0
    assert gap < 0.5 and cos > 0.9
