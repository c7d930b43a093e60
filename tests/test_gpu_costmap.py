"""Parity of the actor cost map on the tensor cores (Sec. V-A: observation ->
2 x 512 ReLU -> sigmoid scaled to [0.1, 10] -> per-stage Q_t) with the FP64
oracle (oracle/costmap.py), forward and backward, and of its composition with
the MPC layer (Q written straight into the solve's Q buffer, dL/dQ from the
adjoint back to the weights) against the oracle's chain rule.

Tolerances.  The kernels compute in FP32 precision with the 3xTF32 split
(operand hi and lo parts, three tensor-core products): each product carries
about 2^-21 relative error and the FP32 accumulation over K terms about
sqrt(K) 2^-24 of the terms' magnitude.  For the forward (K <= 512, three
layers, a sigmoid with slope <= 1/4 scaled by 9.9) that bounds the error of Q
well below 1e-5 of Q's range; the weight gradients sum K = B products of
either sign, so their error is measured against the magnitude of those terms
and held to 1e-4 in norm per block."""
import numpy as np
import pytest

import workloads as W
from oracle import costmap

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

Q_TOL = 1e-5          # |Q - Q_or| / (q_hi - q_lo), elementwise
G_TOL = 1e-4          # per gradient block, relative to the norm of |terms|


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _abs_terms_norms(params, cache, dQ):
    """|| |h|' |da| || per weight block: the magnitude the batch sums of the
    weight gradients are accumulated from (the backward with every factor
    replaced by its absolute value)."""
    W1, b1, W2, b2, W3, b3 = params
    o, a1, h1, a2, h2, s = cache
    B = o.shape[0]
    da3 = np.abs(dQ.reshape(B, -1) * (costmap.Q_HI - costmap.Q_LO) * s * (1.0 - s))
    da2 = (da3 @ np.abs(W3).T) * (a2 > 0)
    da1 = (da2 @ np.abs(W2).T) * (a1 > 0)
    return [np.linalg.norm(np.abs(o).T @ da1), np.linalg.norm(da1.sum(0)), np.linalg.norm(np.abs(h1).T @ da2),
            np.linalg.norm(da2.sum(0)), np.linalg.norm(np.abs(h2).T @ da3), np.linalg.norm(da3.sum(0))]


def _run(B, N, hidden, seed, with_obs=True):
    from paper_2605_29155_gb300 import CostMap
    prob = W.race_track(B, N, seed=seed)
    params = W.costmap_weights(26, N * 13, seed=seed + 1, hidden=hidden)
    rng = np.random.default_rng(seed + 2)
    dQ = rng.normal(size=(B, N, 13))
    cm = CostMap(params, N, B)
    x0 = torch.as_tensor(prob["x0"], dtype=torch.float32, device="cuda")
    xr = torch.as_tensor(prob["x_ref"], dtype=torch.float32, device="cuda")
    Q = cm.forward(x0, xr)
    grads, d_obs = cm.backward(x0, xr, torch.as_tensor(dQ, dtype=torch.float32, device="cuda"), with_obs=with_obs)
    torch.cuda.synchronize()
    assert cm.wait_flag() == 0
    # the oracle on the same FP32 inputs (in FP64)
    p64 = [np.asarray(w, np.float32).astype(np.float64) for w in params]
    o = costmap.observation(prob["x0"].astype(np.float32).astype(np.float64),
                            prob["x_ref"].astype(np.float32).astype(np.float64))
    Q_or, cache = costmap.forward(p64, o, N)
    g_or, do_or = costmap.backward(p64, cache, dQ.astype(np.float32).astype(np.float64))
    scales = _abs_terms_norms(p64, cache, dQ)
    return Q.cpu().numpy(), [g.cpu().numpy() for g in grads], None if d_obs is None else d_obs.cpu().numpy(), \
        Q_or, g_or, do_or, scales


@pytest.mark.parametrize("B,N,hidden", [(300, 20, 512), (5, 3, 40), (1000, 10, 512)])
def test_costmap_forward_backward_match_oracle(B, N, hidden):
    """Ragged tiles in every dimension (B, the hidden width and N * 13 are not
    multiples of the 128 x 128 tile; K = 26 is not a multiple of 16)."""
    Q, g, d_obs, Q_or, g_or, do_or, scales = _run(B, N, hidden, seed=B)
    eq = np.max(np.abs(Q - Q_or)) / (costmap.Q_HI - costmap.Q_LO)
    assert eq <= Q_TOL, eq
    assert np.all(Q >= costmap.Q_LO) and np.all(Q <= costmap.Q_HI)
    errs = []
    for name, a, b, sc in zip(("dW1", "db1", "dW2", "db2", "dW3", "db3"), g, g_or, scales):
        e = np.linalg.norm(a - b) / max(sc, 1e-30)
        errs.append((name, e))
        assert e <= G_TOL, (name, e, np.linalg.norm(a - b) / np.linalg.norm(b))
    e_obs = np.max(np.abs(d_obs - do_or)) / max(np.max(np.abs(do_or)), 1e-30)
    print(B, N, hidden, "Q", eq, errs, "d_obs", e_obs)
    assert e_obs <= G_TOL


def test_costmap_zero_batch_gives_zero_gradients():
    from paper_2605_29155_gb300 import CostMap
    params = W.costmap_weights(26, 5 * 13, seed=3, hidden=64)
    cm = CostMap(params, 5, 4)
    x0 = torch.zeros(0, 13, device="cuda")
    xr = torch.zeros(0, 5, 13, device="cuda")
    out = [torch.full_like(t, 7.0) for t in (cm.W1, cm.b1, cm.W2, cm.b2, cm.W3, cm.b3)]
    cm.backward(x0, xr, torch.zeros(0, 5, 13, device="cuda"), out=out)
    torch.cuda.synchronize()
    assert all(not t.any() for t in out)


def test_costmap_fused_with_the_mpc_layer_matches_the_chain_rule():
    """Observation -> cost map -> Q written into the solve's Q buffer -> MPC
    forward -> adjoint dL/dQ -> cost-map backward, on the GPU, against the
    oracle's composition (costmap.forward, the iLQR oracle on that Q, its
    adjoint, costmap.backward): controls of converged instances within 1e-4,
    the weight gradients within 1e-3 of the oracle chain's."""
    import dataclasses

    from gpu_support import QUAD, rel
    from oracle import adjoint, ilqr
    from paper_2605_29155_gb300 import CostMap, DiffMPC, Problem
    B, N = 48, 10
    prob = W.hover_targets(B, N, seed=12)
    params = W.costmap_weights(26, N * 13, seed=13)
    rng = np.random.default_rng(14)
    gu = rng.normal(size=(B, N, 4))
    p = Problem.from_numpy(dict(prob, Q=np.ones((B, N, 13))))
    cm = CostMap(params, N, B)
    solver = DiffMPC(N_max=N, B_max=B, max_iter=30, tol=1e-7)
    cm.forward(p.x0, p.x_ref, Q=p.Q)                # straight into the problem's Q buffer
    s = solver.solve(p)
    dQ, _, _ = solver.backward(p, s, torch.as_tensor(gu, dtype=torch.float32, device="cuda"))
    grads, _ = cm.backward(p.x0, p.x_ref, dQ)
    torch.cuda.synchronize()
    assert cm.wait_flag() == 0
    Q_gpu = p.Q.cpu().numpy()
    u_gpu, st_gpu = s.u.cpu().numpy(), s.status.cpu().numpy()
    g_gpu = [g.cpu().numpy() for g in grads]
    solver.close()
    p64 = [np.asarray(w, np.float32).astype(np.float64) for w in params]
    x0 = prob["x0"].astype(np.float32).astype(np.float64)
    xr = prob["x_ref"].astype(np.float32).astype(np.float64)
    Q_or, cache = costmap.forward(p64, costmap.observation(x0, xr), N)
    assert np.max(np.abs(Q_gpu - Q_or)) / (costmap.Q_HI - costmap.Q_LO) <= Q_TOL
    dQ_or = np.zeros_like(Q_or)
    converged = 0
    base = dict(prob, x0=x0, x_ref=xr)
    for i in range(B):
        pr = dataclasses.replace(ilqr.problem_from_batch(base, i), Q=Q_or[i])
        so = ilqr.solve(QUAD, pr, 30, 1e-7)
        assert so.status in (ilqr.CONVERGED, ilqr.MAX_ITER)
        if so.status == ilqr.CONVERGED and st_gpu[i] in (0, 1):
            converged += 1
            assert rel(u_gpu[i], so.U, 1e-6) <= 1e-4, i
        dQ_or[i] = adjoint.adjoint(pr, so, np.zeros((N, 13)), gu[i]).dQ
    assert converged >= 0.9 * B
    g_or, _ = costmap.backward(p64, cache, dQ_or)
    for name, a, b in zip(("dW1", "db1", "dW2", "db2", "dW3", "db3"), g_gpu, g_or):
        e = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        print(name, e)
        assert e <= 1e-3, (name, e)
