"""Actor cost map of CA-AC-MPC (oracle, FP64): observation -> stage-cost weights.

Test infrastructure only: the tests and bench.py's CPU legs may use this
module; the product path never does.

Sec. V-A: the actor predicts the stage-cost coefficients with a neural cost
map, an MLP with two hidden layers of 512 ReLU units and a sigmoid output
layer that bounds and scales the coefficients (Sec. III: the actor maps the
observation to the quadratic cost parameters of each stage).

Readings where the paper defers to the AC-MPC codebase (not printed):
  observation  o = [x_init; x_ref,0] (26 values): the state and the first
               reference point of the instance.
  output       the diagonal weights Q_t of every stage, Q = q_lo + (q_hi - q_lo)
               sigmoid(a), with [q_lo, q_hi] = [0.1, 10] (the range of the
               synthetic workloads), an [N, 13] block per instance.
  weights      layer l: y = W_l' h + b_l, W_l of shape [n_in, n_out]; the
               initialisation (uniform +-1/sqrt(n_in), seeded) stands in for
               trained weights.

forward() returns Q and a cache; backward() maps dL/dQ (the MPC adjoint's
gradient) to dL/dW_l, dL/db_l and dL/do by the chain rule through the layers.
"""
from __future__ import annotations

import numpy as np
from scipy.special import expit

HIDDEN = 512
Q_LO, Q_HI = 0.1, 10.0
NX = 13


def init_params(n_in: int, n_out: int, seed: int = 0, hidden: int = HIDDEN):
    """Weights (W1, b1, W2, b2, W3, b3) of the in -> hidden -> hidden -> out map."""
    rng = np.random.default_rng(seed)
    sizes = [(n_in, hidden), (hidden, hidden), (hidden, n_out)]
    params = []
    for a, b in sizes:
        lim = 1.0 / np.sqrt(a)
        params.append(rng.uniform(-lim, lim, size=(a, b)))
        params.append(rng.uniform(-lim, lim, size=b))
    return params


def observation(x0: np.ndarray, x_ref: np.ndarray) -> np.ndarray:
    """o = [x_init; x_ref,0] per instance: [B, 26]."""
    return np.concatenate([x0, x_ref[:, 0]], axis=1)


def sigmoid(a):
    """1 / (1 + exp(-a)), without overflow for large |a| (scipy's expit)."""
    return expit(a)


def forward(params, o: np.ndarray, N: int):
    """Q [B, N, 13] from observations o [B, n_in], with the cache for backward."""
    W1, b1, W2, b2, W3, b3 = params
    a1 = o @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    a3 = h2 @ W3 + b3
    s = sigmoid(a3)
    Q = (Q_LO + (Q_HI - Q_LO) * s).reshape(o.shape[0], N, NX)
    return Q, (o, a1, h1, a2, h2, s)


def backward(params, cache, dQ: np.ndarray):
    """dL/dQ [B, N, 13] -> (dW1, db1, dW2, db2, dW3, db3), dL/do."""
    W1, b1, W2, b2, W3, b3 = params
    o, a1, h1, a2, h2, s = cache
    B = o.shape[0]
    da3 = dQ.reshape(B, -1) * (Q_HI - Q_LO) * s * (1.0 - s)     # d sigmoid = s (1 - s)
    dW3 = h2.T @ da3
    db3 = da3.sum(axis=0)
    dh2 = da3 @ W3.T
    da2 = dh2 * (a2 > 0)
    dW2 = h1.T @ da2
    db2 = da2.sum(axis=0)
    dh1 = da2 @ W2.T
    da1 = dh1 * (a1 > 0)
    dW1 = o.T @ da1
    db1 = da1.sum(axis=0)
    do = da1 @ W1.T
    return [dW1, db1, dW2, db2, dW3, db3], do
