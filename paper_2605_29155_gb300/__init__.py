"""GB300-native batched differentiable MPC layer (box-constrained iLQR forward,
adjoint LQR backward) behind the C ABI of include/camp.h.

The compute path is libcamp.so (CUDA, sm_103a); importing the package fails
loudly when it has not been built.
"""
from . import camp  # noqa: F401  (raises ImportError without libcamp.so)
from .costmap import CostMap  # noqa: F401
from .layer import DiffMPC, DiffMPCFunction, Problem, Solution, diff_mpc  # noqa: F401
