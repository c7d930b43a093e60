"""Seeded synthetic inputs for the batched quadrotor MPC layer.

This module is shared by the FP64 oracle, the CUDA path, the tests and the
benchmark.  It only draws random numbers and lays out arrays: it holds none of
the method's arithmetic (no dynamics, no cost, no solver step).

The paper evaluates on a reconstructed drone-racing track and on hover
stabilisation at random targets (Sec. V, Sec. V-A); neither dataset is
available, so these generators stand in for them with the shapes and value
ranges stated below.  Every array is float64 (the GPU path casts to its own
working precision); every function takes an explicit seed.

Problem layout (instance-major, row-major, one row per MPC instance):
  x0     [B, 13]      initial state x_init of Eq. (3): p(3), q(4, w first), v(3), w(3)
  Q      [B, Nq, 13]  diagonal state weights, Nq = 1 (shared over stages) or N
  x_ref  [B, N, 13]   state reference per stage
  R      [B, 4]       diagonal control weights
  u_ref  [B, 4]       control reference
  u_lo   [B, 4]       lower thrust bound  (u_min of Eq. (3))
  u_hi   [B, 4]       upper thrust bound  (u_max of Eq. (3))
  horizon [B] int32 or None (None: every instance uses the full N)
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NX = 13
NU = 4


@dataclasses.dataclass(frozen=True)
class ModelParams:
    """Quadrotor constants (the paper states none; these are the workload's)."""
    mass: float = 0.75
    inertia: tuple = (2.5e-3, 2.1e-3, 4.3e-3)
    arm: float = 0.15
    kappa: float = 0.016          # yaw-moment-to-thrust ratio [m]
    gravity: float = 9.81
    dt: float = 0.02
    u_min: float = 0.0
    u_max: float = 8.5

    @property
    def hover_thrust(self) -> float:
        return self.mass * self.gravity / 4.0


DEFAULT_MODEL = ModelParams()
HOVER_POSITION = np.array([0.0, 0.0, 2.0])


def _random_attitudes(rng: np.random.Generator, B: int, sigma: float) -> np.ndarray:
    """Unit quaternions exp(r/2) for rotation vectors r ~ N(0, sigma^2 I)."""
    r = rng.normal(0.0, sigma, size=(B, 3))
    ang = np.linalg.norm(r, axis=1)
    half = 0.5 * ang
    s = np.where(ang > 1e-12, np.sin(half) / np.maximum(ang, 1e-300), 0.5)
    q = np.empty((B, 4))
    q[:, 0] = np.cos(half)
    q[:, 1:] = r * s[:, None]
    return q


def _base_problem(rng, B, N, Nq, model, u_hi_spread=0.0):
    mp = model
    Q = rng.uniform(0.1, 10.0, size=(B, Nq, NX))
    R = np.full((B, NU), 0.01)
    u_ref = np.full((B, NU), mp.hover_thrust)
    u_lo = np.full((B, NU), mp.u_min)
    if u_hi_spread > 0:
        u_hi = np.repeat(mp.u_max * rng.uniform(1.0 - u_hi_spread, 1.0 + u_hi_spread,
                                                size=(B, 1)), NU, axis=1)
    else:
        u_hi = np.full((B, NU), mp.u_max)
    return Q, R, u_ref, u_lo, u_hi


def hover_targets(B: int, N: int, seed: int = 0, Nq: int = 1, model: ModelParams = DEFAULT_MODEL,
                  per_stage_jitter: float = 0.0, horizons=None, u_hi_spread: float = 0.0) -> dict:
    """Hover stabilisation at random targets (the setting of Sec. V-A).

    x_ref: hover +- N(0, 0.5) m in position, identity attitude, zero velocity
    and rate (constant over the stages unless ``per_stage_jitter`` > 0).
    x0: hover +- N(0, 0.3) m in position, attitude exp(N(0, 0.2) rad).
    Q diag ~ U(0.1, 10), R = 0.01 I, u_ref = m g / 4, u in [0, 8.5] N.
    """
    rng = np.random.default_rng(seed)
    Q, R, u_ref, u_lo, u_hi = _base_problem(rng, B, N, Nq, model, u_hi_spread)
    target = HOVER_POSITION + rng.normal(0.0, 0.5, size=(B, 3))
    x_ref = np.zeros((B, N, NX))
    x_ref[:, :, 0:3] = target[:, None, :]
    if per_stage_jitter > 0:
        x_ref[:, :, 0:3] += rng.normal(0.0, per_stage_jitter, size=(B, N, 3))
    x_ref[:, :, 3] = 1.0
    x0 = np.zeros((B, NX))
    x0[:, 0:3] = HOVER_POSITION + rng.normal(0.0, 0.3, size=(B, 3))
    x0[:, 3:7] = _random_attitudes(rng, B, 0.2)
    return dict(x0=x0, Q=Q, x_ref=x_ref, R=R, u_ref=u_ref, u_lo=u_lo, u_hi=u_hi,
                horizon=horizons)


def _track(rng):
    """Closed synthetic race track: 7 gates on an ellipse with 15 m x 7.5 m
    semi-axes (30 m span) at heights U(1.5, 3.5) m."""
    n_gates = 7
    heights = rng.uniform(1.5, 3.5, size=n_gates)
    return 15.0, 7.5, heights


def _track_point(a, b, heights, theta):
    n = heights.shape[0]
    s = (theta % (2 * math.pi)) / (2 * math.pi) * n
    i0 = np.floor(s).astype(np.int64) % n
    i1 = (i0 + 1) % n
    w = s - np.floor(s)
    h = (1 - w) * heights[i0] + w * heights[i1]
    dh = (heights[i1] - heights[i0]) * n / (2 * math.pi)
    p = np.stack([a * np.cos(theta), b * np.sin(theta), h], axis=-1)
    d = np.stack([-a * np.sin(theta), b * np.cos(theta), dh], axis=-1)
    return p, d


def race_track(B: int, N: int, seed: int = 0, model: ModelParams = DEFAULT_MODEL,
               Nq: int = 1, horizons=None, u_hi_spread: float = 0.0) -> dict:
    """Drone-racing-shaped batch (stand-in for the reconstructed track of Sec. V).

    Each instance starts at a uniform arc position of the track, flying along
    the tangent at U(0, 20) m/s with attitude exp(N(0, 0.2) rad) and a
    position offset N(0, 0.3) m; its reference x_ref_t is the track point
    reached after t*dt seconds at that speed, with tangent velocity, identity
    attitude and zero rate.
    """
    rng = np.random.default_rng(seed)
    a, b, heights = _track(rng)
    Q, R, u_ref, u_lo, u_hi = _base_problem(rng, B, N, Nq, model, u_hi_spread)
    theta0 = rng.uniform(0.0, 2 * math.pi, size=B)
    speed = rng.uniform(0.0, 20.0, size=B)
    p0, d0 = _track_point(a, b, heights, theta0)
    dn0 = np.linalg.norm(d0, axis=-1)
    x0 = np.zeros((B, NX))
    x0[:, 0:3] = p0 + rng.normal(0.0, 0.3, size=(B, 3))
    x0[:, 3:7] = _random_attitudes(rng, B, 0.2)
    x0[:, 7:10] = d0 / dn0[:, None] * speed[:, None]
    t = np.arange(N) * model.dt
    theta = theta0[:, None] + speed[:, None] * t[None, :] / dn0[:, None]
    p, d = _track_point(a, b, heights, theta)
    x_ref = np.zeros((B, N, NX))
    x_ref[:, :, 0:3] = p
    x_ref[:, :, 3] = 1.0
    x_ref[:, :, 7:10] = d / np.linalg.norm(d, axis=-1, keepdims=True) * speed[:, None, None]
    return dict(x0=x0, Q=Q, x_ref=x_ref, R=R, u_ref=u_ref, u_lo=u_lo, u_hi=u_hi,
                horizon=horizons)


def uneven_horizons(B: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=B).astype(np.int32)


# --- the five workloads of the scope table ------------------------------------------

def cfg_tiny(seed: int = 0) -> dict:
    """B=8, N=10, shared Q; <=10 iterations; loss = sum of first controls."""
    p = hover_targets(8, 10, seed=seed)
    p.update(max_iter=10, tol=1e-6)
    return p


def cfg_train(seed: int = 0, B: int = 1024) -> dict:
    """B=1024, N=20; <=8 iterations, tol 1e-6; loss = w . u_0, w ~ N(0, 1) (seed 1)."""
    p = hover_targets(B, 20, seed=seed)
    p.update(max_iter=8, tol=1e-6)
    return p


def cfg_track(seed: int = 0, B: int = 4096, N: int = 20) -> dict:
    """B=4096, N=20 race-track batch; <=8 iterations, tol 1e-6."""
    p = race_track(B, N, seed=seed)
    p.update(max_iter=8, tol=1e-6)
    return p


def cfg_uneven(seed: int = 0, B: int = 2048) -> dict:
    """B=2048, horizons U{5..40}, u_hi = 8.5 * U(0.8, 1.2); <=12 iterations, tol 1e-6."""
    hz = uneven_horizons(B, 5, 40, seed + 1000)
    p = race_track(B, 40, seed=seed, horizons=hz, u_hi_spread=0.2)
    p.update(max_iter=12, tol=1e-6)
    return p


def cfg_mem(seed: int = 0, B: int = 8192) -> dict:
    """B=8192, N=30, per-stage Q and x_ref (30 x 26 cost parameters per instance)."""
    p = hover_targets(B, 30, seed=seed, Nq=30, per_stage_jitter=0.1)
    p.update(max_iter=8, tol=1e-6)
    return p


def loss_weights_u0(B: int, N: int, seed: int = 1) -> np.ndarray:
    """grad_u for the loss L = sum_i w_i . u_{i,0} with w ~ N(0, 1): shape [B, N, 4]."""
    rng = np.random.default_rng(seed)
    g = np.zeros((B, N, NU))
    g[:, 0, :] = rng.normal(0.0, 1.0, size=(B, NU))
    return g


def loss_sum_first_controls(B: int, N: int) -> np.ndarray:
    """grad_u for L = sum of the first controls: ones at t = 0."""
    g = np.zeros((B, N, NU))
    g[:, 0, :] = 1.0
    return g


def subset(prob: dict, idx) -> dict:
    """Instances ``idx`` of a problem dict (arrays sliced on the batch axis)."""
    out = {}
    for k, v in prob.items():
        if isinstance(v, np.ndarray) and v.ndim >= 1 and k not in ():
            out[k] = v[idx]
        else:
            out[k] = v
    return out


def costmap_weights(n_in: int, n_out: int, seed: int = 0, hidden: int = 512):
    """Random-init weights (W1, b1, W2, b2, W3, b3) of the actor's cost map,
    n_in -> hidden -> hidden -> n_out, W_l of shape [n_in_l, n_out_l], every
    entry uniform in +-1/sqrt(n_in_l) (seeded): the stand-in for trained
    weights of that architecture."""
    rng = np.random.default_rng(seed)
    out = []
    for a, b in ((n_in, hidden), (hidden, hidden), (hidden, n_out)):
        lim = 1.0 / np.sqrt(a)
        out.append(rng.uniform(-lim, lim, size=(a, b)))
        out.append(rng.uniform(-lim, lim, size=b))
    return out
