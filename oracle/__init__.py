"""FP64 CPU oracle for the batched differentiable MPC layer.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2605_29155_gb300``) never imports, links or runs it, and
this package imports nothing from the product path: the two share only the
seeded input generators in ``workloads``.

Plain, slow, one-instance-at-a-time NumPy in float64 (complex128 where a
complex-step check drives it).  Each function cites the passage it follows:

  model.py   quadrotor dynamics f(x, u) as RK4 of the continuous model and its
             analytic Jacobians [A_t B_t] (Sec. IV-1)
  boxqp.py   per-stage box QP, projected Newton (Sec. IV-2, Tassa et al. 2014)
  ilqr.py    box-constrained iLQR forward solve of Eq. (3): rollout,
             linearization, Riccati backward pass with the box QP, line search
             over alpha in {1, 0.5, 0.25, 0.1} (Sec. IV-1..3, Algorithm 2)
  adjoint.py implicit KKT differentiation of the solution (Sec. IV: gradients
             w.r.t. (C_t, c_t) and x_init at the converged solution), as an
             adjoint LQR sweep, plus an independent dense-KKT solve used only to
             cross-check it.
  costmap.py the actor's cost map (Sec. V-A: MLP with two 512-unit ReLU
             layers and a sigmoid output), observation -> per-stage Q, with
             its backward from dL/dQ.

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: complex-step and finite differences, closed-form trajectories, exact
LQR on linear-quadratic instances, brute-force active-set enumeration and
dense KKT solves.
"""
from . import model, boxqp, ilqr, adjoint, costmap  # noqa: F401
