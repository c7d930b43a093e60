"""Thin ctypes binding of ``include/camp.h`` (same names, argument marshalling only).

Every function here forwards to ``libcamp.so``; nothing computes on the host.
Importing this module raises ImportError when the library has not been built:
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_size_t, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcamp.so")

MPC_OK, MPC_ERR_ARG, MPC_ERR_SHAPE, MPC_ERR_CUDA, MPC_ERR_TIMEOUT, MPC_ERR_STATE = 0, -1, -2, -3, -4, -5
MPC_F32, MPC_F64 = 0, 1
MPC_STORE_ALL, MPC_RECOMPUTE, MPC_STORE_AUTO = 0, 1, 2
MPC_EXEC_PERSISTENT, MPC_EXEC_PLAIN, MPC_EXEC_SCAN, MPC_EXEC_AUTO = 0, 1, 2, 3
MPC_ST_CONVERGED, MPC_ST_STALLED, MPC_ST_MAX_ITER, MPC_ST_NONFINITE, MPC_ST_NONPD = 0, 1, 2, 3, 4

EXPORTED = ("mpc_config_default", "mpc_create", "mpc_destroy", "mpc_tape_bytes", "mpc_solve_fwd",
            "mpc_solve_bwd", "mpc_autotune", "mpc_exec_form", "mpc_launch_shape", "mpc_launch_count", "mpc_strerror",
            "mpc_status_str", "mpc_solve_fwd_noalloc", "mpc_solve_bwd_general", "mpc_fp32_fma_probe",
            "mpc_costmap_workspace_bytes", "mpc_costmap_forward", "mpc_costmap_backward")
MPC_NOALLOC_B_MAX, MPC_NOALLOC_N_MAX = 256, 40


class mpc_config(ctypes.Structure):
    _fields_ = [("nx", c_int), ("nu", c_int), ("N_max", c_int), ("B_max", c_int), ("dtype", c_int),
                ("dt", c_double), ("mass", c_double), ("inertia", c_double * 3), ("arm", c_double),
                ("kappa_yaw", c_double), ("gravity", c_double), ("max_iter", c_int), ("tol", c_double),
                ("n_alpha", c_int), ("alpha", c_double * 4), ("store_mode", c_int), ("exec_mode", c_int),
                ("tpi", c_int), ("ipb", c_int), ("tape_budget", c_size_t)]


class mpc_problem(ctypes.Structure):
    _fields_ = [("B", c_int), ("N", c_int), ("horizon", c_void_p), ("x0", c_void_p), ("Q", c_void_p),
                ("Nq", c_int), ("x_ref", c_void_p), ("R", c_void_p), ("u_ref", c_void_p), ("u_lo", c_void_p),
                ("u_hi", c_void_p), ("u_init", c_void_p), ("C", c_void_p), ("NC", c_int), ("c", c_void_p),
                ("Nc", c_int)]


class mpc_solution(ctypes.Structure):
    _fields_ = [("u", c_void_p), ("x", c_void_p), ("cost", c_void_p), ("iters", c_void_p),
                ("status", c_void_p), ("tape", c_void_p), ("tape_bytes", c_size_t)]


class mpc_costmap(ctypes.Structure):
    _fields_ = [("n_in", c_int), ("hidden", c_int), ("n_out", c_int), ("W1", c_void_p), ("b1", c_void_p),
                ("W2", c_void_p), ("b2", c_void_p), ("W3", c_void_p), ("b3", c_void_p), ("q_lo", ctypes.c_float),
                ("q_hi", ctypes.c_float)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcamp.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    lib.mpc_config_default.argtypes = [POINTER(mpc_config)]
    lib.mpc_config_default.restype = None
    lib.mpc_create.argtypes = [POINTER(mpc_config), POINTER(c_void_p)]
    lib.mpc_create.restype = c_int
    lib.mpc_destroy.argtypes = [c_void_p]
    lib.mpc_destroy.restype = c_int
    lib.mpc_tape_bytes.argtypes = [c_void_p, c_int, c_int]
    lib.mpc_tape_bytes.restype = c_size_t
    lib.mpc_solve_fwd.argtypes = [c_void_p, POINTER(mpc_problem), POINTER(mpc_solution), c_void_p]
    lib.mpc_solve_fwd.restype = c_int
    lib.mpc_solve_bwd.argtypes = [c_void_p, POINTER(mpc_problem), POINTER(mpc_solution), c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p]
    lib.mpc_solve_bwd.restype = c_int
    lib.mpc_solve_bwd_general.argtypes = [c_void_p, POINTER(mpc_problem), POINTER(mpc_solution), c_void_p,
                                          c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.mpc_solve_bwd_general.restype = c_int
    lib.mpc_autotune.argtypes = [c_void_p, POINTER(mpc_problem), POINTER(mpc_solution), c_void_p, POINTER(c_int)]
    lib.mpc_autotune.restype = c_int
    lib.mpc_exec_form.argtypes = [c_void_p, POINTER(c_int)]
    lib.mpc_exec_form.restype = c_int
    lib.mpc_launch_shape.argtypes = [c_void_p, c_int, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_int)]
    lib.mpc_launch_shape.restype = c_int
    lib.mpc_launch_count.argtypes = [c_void_p, c_int, POINTER(c_int), POINTER(c_int)]
    lib.mpc_launch_count.restype = c_int
    lib.mpc_strerror.argtypes = [c_int]
    lib.mpc_strerror.restype = ctypes.c_char_p
    lib.mpc_status_str.argtypes = [c_int]
    lib.mpc_status_str.restype = ctypes.c_char_p
    lib.mpc_solve_fwd_noalloc.argtypes = [POINTER(mpc_config), POINTER(mpc_problem), POINTER(mpc_solution), c_void_p]
    lib.mpc_solve_fwd_noalloc.restype = c_int
    lib.mpc_fp32_fma_probe.argtypes = [c_int, c_void_p, c_void_p, POINTER(c_double)]
    lib.mpc_fp32_fma_probe.restype = c_int
    lib.mpc_costmap_workspace_bytes.argtypes = [c_int, c_int, c_int]
    lib.mpc_costmap_workspace_bytes.restype = c_size_t
    lib.mpc_costmap_forward.argtypes = [POINTER(mpc_costmap), c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p]
    lib.mpc_costmap_forward.restype = c_int
    lib.mpc_costmap_backward.argtypes = [POINTER(mpc_costmap), c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.mpc_costmap_backward.restype = c_int
    return lib


_lib = _load()


class CampError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {mpc_strerror(code)} ({code})")
        self.code = code


def check(code, where=""):
    if code != MPC_OK:
        raise CampError(code, where)
    return code


def mpc_config_default() -> mpc_config:
    cfg = mpc_config()
    _lib.mpc_config_default(byref(cfg))
    return cfg


def mpc_create(cfg: mpc_config):
    """Returns (code, handle)."""
    h = c_void_p()
    code = _lib.mpc_create(byref(cfg), byref(h))
    return code, h


def mpc_destroy(h) -> int:
    return _lib.mpc_destroy(h)


def mpc_tape_bytes(h, B: int, N: int) -> int:
    return _lib.mpc_tape_bytes(h, B, N)


def mpc_solve_fwd(h, prob: mpc_problem, sol: mpc_solution, stream: int) -> int:
    return _lib.mpc_solve_fwd(h, byref(prob), byref(sol), c_void_p(stream))


def mpc_solve_bwd(h, prob: mpc_problem, sol: mpc_solution, grad_u: int, grad_x: int, dQ: int, dx_ref: int,
                  dx0: int, stream: int) -> int:
    return _lib.mpc_solve_bwd(h, byref(prob), byref(sol), c_void_p(grad_u), c_void_p(grad_x or None),
                              c_void_p(dQ), c_void_p(dx_ref), c_void_p(dx0), c_void_p(stream))


def mpc_solve_bwd_general(h, prob: mpc_problem, sol: mpc_solution, grad_u: int, grad_x: int, dC: int, dc: int,
                          dx0: int, stream: int) -> int:
    return _lib.mpc_solve_bwd_general(h, byref(prob), byref(sol), c_void_p(grad_u), c_void_p(grad_x or None),
                                      c_void_p(dC), c_void_p(dc), c_void_p(dx0), c_void_p(stream))


def mpc_autotune(h, prob: mpc_problem, sol: mpc_solution, stream: int):
    """Returns (code, ipb)."""
    ipb = c_int(0)
    code = _lib.mpc_autotune(h, byref(prob), byref(sol), c_void_p(stream), byref(ipb))
    return code, ipb.value


def mpc_exec_form(h):
    """Returns (code, exec form)."""
    e = c_int(0)
    code = _lib.mpc_exec_form(h, byref(e))
    return code, e.value


def mpc_launch_shape(h, B: int, N: int):
    """Returns (code, tpi, ipb, grid)."""
    a, b, c = c_int(), c_int(), c_int()
    code = _lib.mpc_launch_shape(h, B, N, byref(a), byref(b), byref(c))
    return code, a.value, b.value, c.value


def mpc_launch_count(h, has_horizon: bool):
    """Returns (code, fwd launches, bwd launches)."""
    f, b = c_int(), c_int()
    code = _lib.mpc_launch_count(h, 1 if has_horizon else 0, byref(f), byref(b))
    return code, f.value, b.value


def mpc_solve_fwd_noalloc(cfg: mpc_config, prob: mpc_problem, sol: mpc_solution, stream: int) -> int:
    return _lib.mpc_solve_fwd_noalloc(byref(cfg), byref(prob), byref(sol), c_void_p(stream))


def mpc_fp32_fma_probe(trips: int, sink: int, stream: int):
    """Returns (code, flops enqueued)."""
    fl = c_double(0.0)
    code = _lib.mpc_fp32_fma_probe(trips, c_void_p(sink), c_void_p(stream), byref(fl))
    return code, fl.value


def mpc_costmap_workspace_bytes(B: int, hidden: int, n_out: int) -> int:
    return _lib.mpc_costmap_workspace_bytes(B, hidden, n_out)


def mpc_costmap_forward(net: mpc_costmap, B: int, N: int, x0: int, x_ref: int, Q: int, ws: int, stream: int) -> int:
    return _lib.mpc_costmap_forward(byref(net), B, N, c_void_p(x0), c_void_p(x_ref), c_void_p(Q), c_void_p(ws),
                                    c_void_p(stream))


def mpc_costmap_backward(net: mpc_costmap, B: int, N: int, x0: int, x_ref: int, dQ: int, ws: int, dW1: int, db1: int,
                         dW2: int, db2: int, dW3: int, db3: int, d_obs: int, stream: int) -> int:
    return _lib.mpc_costmap_backward(byref(net), B, N, c_void_p(x0), c_void_p(x_ref), c_void_p(dQ), c_void_p(ws),
                                     c_void_p(dW1), c_void_p(db1), c_void_p(dW2), c_void_p(db2), c_void_p(dW3),
                                     c_void_p(db3), c_void_p(d_obs or None), c_void_p(stream))


def mpc_strerror(code: int) -> str:
    return _lib.mpc_strerror(code).decode()


def mpc_status_str(status: int) -> str:
    return _lib.mpc_status_str(status).decode()
