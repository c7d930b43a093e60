"""Quadrotor model for the oracle: continuous dynamics, RK4 map, Jacobians.

The paper uses a nonlinear state-transition map x_{t+1} = f(x_t, u_t)
(Sec. III-A, Eq. (1)) and analytic Jacobians A_t = df/dx, B_t = df/du of it
(Sec. IV-1) but never writes the model down.  The model here is the workload's
(13 states, 4 rotor thrusts); the choices the paper leaves open are readings:

  state   x = [p (3), q (4, Hamilton, scalar first), v (3), w (3, body rates)]
  p'      = v
  q'      = 1/2 q (x) [0, w]
  v'      = (sum u / m) R(q) e3 - g e3, with R(q) e3 written as the homogeneous
            quadratic form [2(xz + wy), 2(yz - wx), w^2 - x^2 - y^2 + z^2]
  w'      = J^-1 (tau - w x J w),  tau = sum_i r_i x (0, 0, u_i) + kappa s_i u_i e3
  rotors  X layout at distance l/sqrt(2) on each axis, order FR, RL, FL, RR,
          spin signs s = (+1, +1, -1, -1)
  f       one classic RK4 step of length dt with u held constant; the
          quaternion is integrated as 4 raw components (no renormalisation).

Everything here accepts complex arrays so that complex-step derivatives can
check the hand-written Jacobians.
"""
from __future__ import annotations

import numpy as np

NX, NU = 13, 4


class Quadrotor:
    """Quadrotor dynamics with parameters taken from a ``workloads.ModelParams``."""

    def __init__(self, params):
        self.p = params
        self.m = float(params.mass)
        self.J = np.array(params.inertia, dtype=float)
        self.g = float(params.gravity)
        self.dt = float(params.dt)
        d = params.arm / np.sqrt(2.0)
        # rotor positions (body x, y) for FR, RL, FL, RR and spin signs
        self.rotor_xy = np.array([[d, -d], [-d, d], [d, d], [-d, -d]])
        self.spin = np.array([1.0, 1.0, -1.0, -1.0])
        self.kappa = float(params.kappa)
        self.nx, self.nu = NX, NU

    # -- torque map ------------------------------------------------------------
    def torque_matrix(self) -> np.ndarray:
        """M (3x4) with tau = M u: tau_x = sum y_i u_i, tau_y = -sum x_i u_i,
        tau_z = kappa sum s_i u_i."""
        M = np.zeros((3, 4))
        M[0] = self.rotor_xy[:, 1]
        M[1] = -self.rotor_xy[:, 0]
        M[2] = self.kappa * self.spin
        return M

    # -- continuous model --------------------------------------------------------
    def f_cont(self, x, u):
        dt_ = np.result_type(x, u, float)
        x = np.asarray(x, dtype=dt_)
        u = np.asarray(u, dtype=dt_)
        qw, qx, qy, qz = x[3], x[4], x[5], x[6]
        wx, wy, wz = x[10], x[11], x[12]
        T = u[0] + u[1] + u[2] + u[3]
        out = np.zeros(NX, dtype=dt_)
        out[0:3] = x[7:10]
        # q (x) [0, w] = (-qv.w, qw w + qv x w), times 1/2
        out[3] = 0.5 * (-qx * wx - qy * wy - qz * wz)
        out[4] = 0.5 * (qw * wx + qy * wz - qz * wy)
        out[5] = 0.5 * (qw * wy + qz * wx - qx * wz)
        out[6] = 0.5 * (qw * wz + qx * wy - qy * wx)
        r3 = np.array([2 * (qx * qz + qw * qy), 2 * (qy * qz - qw * qx),
                       qw * qw - qx * qx - qy * qy + qz * qz], dtype=dt_)
        out[7:10] = (T / self.m) * r3
        out[9] = out[9] - self.g
        w = x[10:13]
        Jw = self.J * w
        wxJw = np.array([w[1] * Jw[2] - w[2] * Jw[1],
                         w[2] * Jw[0] - w[0] * Jw[2],
                         w[0] * Jw[1] - w[1] * Jw[0]], dtype=dt_)
        tau = self.torque_matrix() @ u
        out[10:13] = (tau - wxJw) / self.J
        return out

    def jac_cont(self, x, u):
        """Analytic (Ac, Bc) = (df_c/dx, df_c/du) of the continuous model, dense."""
        x = np.asarray(x, dtype=float)
        u = np.asarray(u, dtype=float)
        qw, qx, qy, qz = x[3:7]
        wx, wy, wz = x[10:13]
        T = u.sum()
        Jx, Jy, Jz = self.J
        A = np.zeros((NX, NX))
        A[0:3, 7:10] = np.eye(3)
        A[3:7, 3:7] = 0.5 * np.array([[0.0, -wx, -wy, -wz],
                                      [wx, 0.0, wz, -wy],
                                      [wy, -wz, 0.0, wx],
                                      [wz, wy, -wx, 0.0]])
        A[3:7, 10:13] = 0.5 * np.array([[-qx, -qy, -qz],
                                        [qw, -qz, qy],
                                        [qz, qw, -qx],
                                        [-qy, qx, qw]])
        dr3 = np.array([[2 * qy, 2 * qz, 2 * qw, 2 * qx],
                        [-2 * qx, -2 * qw, 2 * qz, 2 * qy],
                        [2 * qw, -2 * qx, -2 * qy, 2 * qz]])
        A[7:10, 3:7] = (T / self.m) * dr3
        # d(w x Jw)/dw
        G = np.array([[0.0, (Jz - Jy) * wz, (Jz - Jy) * wy],
                      [(Jx - Jz) * wz, 0.0, (Jx - Jz) * wx],
                      [(Jy - Jx) * wy, (Jy - Jx) * wx, 0.0]])
        A[10:13, 10:13] = -G / self.J[:, None]
        B = np.zeros((NX, NU))
        r3 = np.array([2 * (qx * qz + qw * qy), 2 * (qy * qz - qw * qx),
                       qw * qw - qx * qx - qy * qy + qz * qz])
        B[7:10, :] = (r3 / self.m)[:, None]
        B[10:13, :] = self.torque_matrix() / self.J[:, None]
        return A, B

    # -- discrete map (RK4) -------------------------------------------------------
    def step(self, x, u):
        """x_{t+1} = f(x_t, u_t): one RK4 step of length dt, u constant."""
        h = self.dt
        k1 = self.f_cont(x, u)
        k2 = self.f_cont(x + 0.5 * h * k1, u)
        k3 = self.f_cont(x + 0.5 * h * k2, u)
        k4 = self.f_cont(x + h * k3, u)
        return x + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)

    def jacobian(self, x, u):
        """F_t = [A_t B_t] = d f / d(x, u) (13 x 17) by the chain rule through
        the four RK4 stages (Sec. IV-1 analytic derivatives)."""
        h = self.dt
        x = np.asarray(x, dtype=float)
        E = np.hstack([np.eye(NX), np.zeros((NX, NU))])
        k1 = self.f_cont(x, u)
        x2 = x + 0.5 * h * k1
        k2 = self.f_cont(x2, u)
        x3 = x + 0.5 * h * k2
        k3 = self.f_cont(x3, u)
        x4 = x + h * k3
        D = []
        prev = None
        for xs, c in ((x, 0.0), (x2, 0.5 * h), (x3, 0.5 * h), (x4, h)):
            A, B = self.jac_cont(xs, u)
            arg = E if prev is None else E + c * prev
            Dk = A @ arg + np.hstack([np.zeros((NX, NX)), B])
            D.append(Dk)
            prev = Dk
        return E + (h / 6.0) * (D[0] + 2.0 * D[1] + 2.0 * D[2] + D[3])

    def rollout(self, x0, U):
        """States x_0..x_{N-1} for controls u_0..u_{N-1} (x_N is not used)."""
        N = U.shape[0]
        X = np.zeros((N, NX), dtype=np.result_type(x0, U, float))
        X[0] = x0
        for t in range(N - 1):
            X[t + 1] = self.step(X[t], U[t])
        return X


class LinearModel:
    """x_{t+1} = A x + B u + f0: linear dynamics for the LQ pins of the solver."""

    def __init__(self, A, B, f0=None):
        self.A = np.asarray(A, dtype=float)
        self.B = np.asarray(B, dtype=float)
        self.nx, self.nu = self.B.shape
        self.f0 = np.zeros(self.nx) if f0 is None else np.asarray(f0, dtype=float)

    def step(self, x, u):
        return self.A @ x + self.B @ u + self.f0

    def jacobian(self, x, u):
        return np.hstack([self.A, self.B])

    def rollout(self, x0, U):
        N = U.shape[0]
        X = np.zeros((N, self.nx), dtype=np.result_type(x0, U, float))
        X[0] = x0
        for t in range(N - 1):
            X[t + 1] = self.step(X[t], U[t])
        return X
