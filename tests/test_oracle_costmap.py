"""Pins of the oracle's actor cost map (Sec. V-A: MLP, 2 x 512 ReLU, sigmoid
output scaled to the weight bounds) and of its composition with the MPC
adjoint.  References: closed forms of the sigmoid output, central finite
differences, and the frozen-LQR solve of the MPC oracle."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import adjoint, costmap, ilqr
from oracle.model import Quadrotor

QUAD = Quadrotor(W.DEFAULT_MODEL)


def test_output_is_the_scaled_sigmoid_and_bounded():
    """With the output layer's weights zero, Q = q_lo + (q_hi - q_lo) sigmoid(b3)
    for every input; for any input every weight lies in (q_lo, q_hi)."""
    N = 4
    params = costmap.init_params(26, N * 13, seed=1)
    params[4] = np.zeros_like(params[4])
    params[5] = np.linspace(-3, 3, N * 13)
    o = np.random.default_rng(2).normal(size=(5, 26)) * 10
    Q, _ = costmap.forward(params, o, N)
    expect = 0.1 + 9.9 / (1.0 + np.exp(-np.linspace(-3, 3, N * 13)))
    np.testing.assert_allclose(Q, np.broadcast_to(expect.reshape(N, 13), Q.shape), rtol=1e-14)
    params = costmap.init_params(26, N * 13, seed=3)
    Q, _ = costmap.forward(params, o, N)
    assert np.all(Q > costmap.Q_LO) and np.all(Q < costmap.Q_HI)
    # far out the sigmoid saturates to its bounds in floating point, never past them
    Q, _ = costmap.forward(params, o * 1e4, N)
    assert np.all(Q >= costmap.Q_LO) and np.all(Q <= costmap.Q_HI)


@pytest.mark.parametrize("seed", range(2))
def test_backward_matches_finite_differences(seed):
    """L = sum(G * Q): dL/dW_l, dL/db_l and dL/do against central differences
    on sampled entries of every layer (small width, so no ReLU kink is crossed)."""
    rng = np.random.default_rng(seed)
    N, B = 3, 4
    params = costmap.init_params(26, N * 13, seed=seed, hidden=16)
    o = rng.normal(size=(B, 26))
    G = rng.normal(size=(B, N, 13))
    Q, cache = costmap.forward(params, o, N)
    grads, do = costmap.backward(params, cache, G)

    def L(ps, oo):
        return float(np.sum(G * costmap.forward(ps, oo, N)[0]))

    eps = 1e-6
    for l, P in enumerate(params):
        for idx in [tuple(rng.integers(0, s) for s in P.shape) for _ in range(6)]:
            pp = [p.copy() for p in params]
            pm = [p.copy() for p in params]
            pp[l][idx] += eps
            pm[l][idx] -= eps
            num = (L(pp, o) - L(pm, o)) / (2 * eps)
            assert abs(num - grads[l][idx]) <= 1e-6 * max(1.0, abs(num)), (l, idx)
    for idx in [(0, 3), (2, 17), (3, 25)]:
        op, om = o.copy(), o.copy()
        op[idx] += eps
        om[idx] -= eps
        num = (L(params, op) - L(params, om)) / (2 * eps)
        assert abs(num - do[idx]) <= 1e-6 * max(1.0, abs(num)), idx


def test_cost_map_composed_with_the_mpc_adjoint():
    """Observation -> per-stage Q -> MPC (frozen at its solution): the chain
    rule dL/dW = costmap.backward(adjoint dL/dQ) against central differences
    of L = g . tau through the frozen-LQR solve, for sampled weights."""
    B, N = 2, 6
    b = W.hover_targets(B, N, seed=4)
    params = costmap.init_params(26, N * 13, seed=5, hidden=16)
    o = costmap.observation(b["x0"], b["x_ref"])
    Q, cache = costmap.forward(params, o, N)
    rng = np.random.default_rng(6)
    gx, gu = rng.normal(size=(B, N, 13)), rng.normal(size=(B, N, 4))
    dQ = np.zeros_like(Q)
    probs, sols = [], []
    for i in range(B):
        pr = dataclasses.replace(ilqr.problem_from_batch(b, i), Q=Q[i])
        so = ilqr.solve(QUAD, pr, max_iter=30, tol=1e-10)
        assert so.status == ilqr.CONVERGED
        dQ[i] = adjoint.adjoint(pr, so, gx[i], gu[i]).dQ
        probs.append(pr)
        sols.append(so)
    grads, _ = costmap.backward(params, cache, dQ)

    def L(ps):
        Qp, _ = costmap.forward(ps, o, N)
        tot = 0.0
        for i in range(B):
            X, U = adjoint.frozen_lqr_solve(probs[i], sols[i], QUAD, Q=Qp[i])
            tot += np.sum(gx[i] * X) + np.sum(gu[i] * U)
        return tot

    eps = 1e-6
    for l in (0, 2, 4, 5):
        P = params[l]
        for idx in [tuple(rng.integers(0, s) for s in P.shape) for _ in range(4)]:
            pp = [p.copy() for p in params]
            pm = [p.copy() for p in params]
            pp[l][idx] += eps
            pm[l][idx] -= eps
            num = (L(pp) - L(pm)) / (2 * eps)
            assert abs(num - grads[l][idx]) <= 1e-5 * max(1e-3, abs(num)), (l, idx, num, grads[l][idx])
