"""Pins of the oracle's quadrotor model (RK4 map and analytic Jacobians).

Each check compares against something other than the model code itself:
complex-step and central-difference derivatives, closed-form trajectories,
scipy's rotation library, and the rotor cross products of the stated layout.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import workloads as W
from oracle.model import Quadrotor, NX, NU

MP = W.DEFAULT_MODEL
M = Quadrotor(MP)


def _random_state(rng, omega_scale=2.0, speed=3.0):
    x = np.zeros(NX)
    x[0:3] = rng.normal(0, 1, 3)
    q = rng.normal(0, 1, 4)
    x[3:7] = q / np.linalg.norm(q) * rng.uniform(0.9, 1.1)   # not exactly unit on purpose
    x[7:10] = rng.normal(0, speed, 3)
    x[10:13] = rng.normal(0, omega_scale, 3)
    return x


@pytest.mark.parametrize("seed", range(5))
def test_continuous_jacobian_complex_step(seed):
    rng = np.random.default_rng(seed)
    x = _random_state(rng)
    u = rng.uniform(0, 8.5, 4)
    A, B = M.jac_cont(x, u)
    h = 1e-30
    for j in range(NX):
        e = np.zeros(NX, complex)
        e[j] = 1j * h
        col = np.imag(M.f_cont(x + e, u.astype(complex))) / h
        np.testing.assert_allclose(A[:, j], col, rtol=1e-13, atol=1e-13)
    for j in range(NU):
        e = np.zeros(NU, complex)
        e[j] = 1j * h
        col = np.imag(M.f_cont(x.astype(complex), u + e)) / h
        np.testing.assert_allclose(B[:, j], col, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_rk4_jacobian_complex_step_and_fd(seed):
    rng = np.random.default_rng(100 + seed)
    x = _random_state(rng)
    u = rng.uniform(0, 8.5, 4)
    F = M.jacobian(x, u)
    assert F.shape == (NX, NX + NU)
    h = 1e-30
    z = np.concatenate([x, u]).astype(complex)
    for j in range(NX + NU):
        zz = z.copy()
        zz[j] += 1j * h
        col = np.imag(M.step(zz[:NX], zz[NX:])) / h
        np.testing.assert_allclose(F[:, j], col, rtol=1e-12, atol=1e-14)
    # central differences, eps = 1e-6: truncation ~eps^2
    eps = 1e-6
    zr = np.concatenate([x, u])
    for j in range(NX + NU):
        zp, zm = zr.copy(), zr.copy()
        zp[j] += eps
        zm[j] -= eps
        col = (M.step(zp[:NX], zp[NX:]) - M.step(zm[:NX], zm[NX:])) / (2 * eps)
        np.testing.assert_allclose(F[:, j], col, rtol=1e-6, atol=1e-8)


def test_free_fall_closed_form():
    """u = 0, level attitude, no rotation: constant acceleration -g e3; RK4 is
    exact on polynomials of degree <= 4, so the closed form holds to rounding."""
    x = np.zeros(NX)
    x[0:3] = [1.0, -2.0, 3.0]
    x[3] = 1.0
    x[7:10] = [0.5, -0.25, 2.0]
    U = np.zeros((41, 4))
    X = M.rollout(x, U)
    t = np.arange(41) * MP.dt
    p = x[0:3][None, :] + x[7:10][None, :] * t[:, None]
    p[:, 2] -= 0.5 * MP.gravity * t ** 2
    np.testing.assert_allclose(X[:, 0:3], p, atol=1e-12)
    np.testing.assert_allclose(X[:, 9], 2.0 - MP.gravity * t, atol=1e-12)
    np.testing.assert_allclose(X[:, 3:7], np.tile([1, 0, 0, 0], (41, 1)), atol=0)


def test_hover_is_a_fixed_point():
    x = np.zeros(NX)
    x[0:3] = [0.3, 0.2, 2.0]
    x[3] = 1.0
    u = np.full(4, MP.mass * MP.gravity / 4)
    np.testing.assert_allclose(M.f_cont(x, u), 0.0, atol=1e-14)
    np.testing.assert_allclose(M.step(x, u), x, atol=1e-14)


def test_thrust_direction_matches_rotation_library():
    """v' = (sum u / m) * third column of the body-to-world rotation - g e3
    (scipy Rotation, scalar-last quaternion convention)."""
    rng = np.random.default_rng(7)
    for _ in range(10):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        x = np.zeros(NX)
        x[3:7] = q
        u = rng.uniform(0, 8.5, 4)
        Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        vdot = u.sum() / MP.mass * Rm[:, 2] - np.array([0, 0, MP.gravity])
        np.testing.assert_allclose(M.f_cont(x, u)[7:10], vdot, atol=1e-12)


def test_torque_from_rotor_cross_products():
    """At zero body rate, w' = J^-1 tau with tau = sum_i r_i x (0,0,u_i)
    + kappa s_i u_i e3 for the X layout FR, RL, FL, RR with spins (+,+,-,-)."""
    d = MP.arm / np.sqrt(2)
    pos = np.array([[d, -d, 0], [-d, d, 0], [d, d, 0], [-d, -d, 0]])
    spin = np.array([1, 1, -1, -1])
    rng = np.random.default_rng(3)
    for _ in range(5):
        u = rng.uniform(0, 8.5, 4)
        tau = sum(np.cross(pos[i], [0, 0, u[i]]) for i in range(4))
        tau = tau + np.array([0, 0, MP.kappa * np.dot(spin, u)])
        x = np.zeros(NX)
        x[3] = 1.0
        np.testing.assert_allclose(M.f_cont(x, u)[10:13], tau / np.array(MP.inertia), rtol=1e-13, atol=1e-12)


def test_quaternion_principal_axis_closed_form():
    """Equal thrusts (no torque) and a rate about the principal z axis keep w
    constant, so q' = Omega q is linear: RK4 gives exactly P(h Omega)^n q0 with
    P the degree-4 Taylor polynomial, and q(t) = q0 (x) exp(w t / 2) up to the
    RK4 local error (h |w| / 2)^5 / 120 per step."""
    wz = 3.0
    x = np.zeros(NX)
    q0 = np.array([0.9, 0.1, -0.3, 0.2])
    q0 /= np.linalg.norm(q0)
    x[3:7] = q0
    x[12] = wz
    n = 40
    X = M.rollout(x, np.full((n + 1, 4), 2.0))
    h = MP.dt
    Om = 0.5 * np.array([[0, 0, 0, -wz], [0, 0, wz, 0], [0, -wz, 0, 0], [wz, 0, 0, 0]])
    Z = h * Om
    P = np.eye(4) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    q = q0.copy()
    for k in range(1, n + 1):
        q = P @ q
        np.testing.assert_allclose(X[k, 3:7], q, atol=1e-14)
    # against the exact rotation: body-frame rotation about z composes on the right
    Rq0 = Rotation.from_quat([q0[1], q0[2], q0[3], q0[0]])
    theta = h * wz / 2
    bound = 1.5 * n * theta ** 5 / 120 + 1e-14
    for k in (10, 20, 40):
        Rt = Rq0 * Rotation.from_rotvec([0, 0, wz * k * h])
        qe = Rt.as_quat()
        qe = np.array([qe[3], qe[0], qe[1], qe[2]])
        if np.dot(qe, X[k, 3:7]) < 0:
            qe = -qe
        assert np.max(np.abs(X[k, 3:7] - qe)) <= bound


@pytest.mark.parametrize("seed", range(4))
def test_quaternion_norm_drift_bound(seed):
    """|w| <= 5 rad/s: the raw RK4 quaternion keeps |q| = 1 to within the RK4
    local error, n (h|w|/2)^5 / 120 over n steps (no renormalisation, reading
    R3).  A sign slip in q' breaks its skew symmetry and drifts at O(h)."""
    rng = np.random.default_rng(seed)
    x = np.zeros(NX)
    q = rng.normal(size=4)
    x[3:7] = q / np.linalg.norm(q)
    w = rng.normal(size=3)
    x[10:13] = 5.0 * w / np.linalg.norm(w)
    U = np.full((41, 4), 1.8)
    X = M.rollout(x, U)
    norms = np.linalg.norm(X[:, 3:7], axis=1)
    wmax = np.max(np.linalg.norm(X[:, 10:13], axis=1))
    assert wmax < 6.0
    bound = 40 * (MP.dt * wmax / 2) ** 5 / 120
    assert np.max(np.abs(norms - 1)) < bound
