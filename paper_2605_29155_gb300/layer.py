"""Torch-facing differentiable MPC layer over the C ABI.

PyTorch supplies device memory and streams only: every step of the forward
and backward solve runs in libcamp.so's kernels.  ``DiffMPCFunction`` is one
module-level ``torch.autograd.Function`` (never a per-call subclass), its
forward needs no autograd graph, and its backward is the adjoint LQR solve of
the library (implicit KKT differentiation at the returned solution, Sec. IV).
"""
from __future__ import annotations

import dataclasses

import torch

from . import camp

_DTYPES = {torch.float32: camp.MPC_F32, torch.float64: camp.MPC_F64}


@dataclasses.dataclass
class Problem:
    """Device tensors of one batched problem (layout of include/camp.h)."""
    x0: torch.Tensor        # [B, 13]
    Q: torch.Tensor         # [B, Nq, 13]
    x_ref: torch.Tensor     # [B, N, 13]
    R: torch.Tensor         # [B, 4]
    u_ref: torch.Tensor     # [B, 4]
    u_lo: torch.Tensor      # [B, 4]
    u_hi: torch.Tensor      # [B, 4]
    horizon: torch.Tensor | None = None   # [B] int32
    u_init: torch.Tensor | None = None    # [B, N, 4]
    # general stage cost of Eq. (2) in place of the diagonal one (Q, x_ref, R
    # unused; u_ref still gives the start U^0)
    C: torch.Tensor | None = None         # [B, NC, 17, 17], NC in {1, N}
    c: torch.Tensor | None = None         # [B, Nc, 17], Nc in {1, N}

    @property
    def B(self):
        return self.x0.shape[0]

    @property
    def N(self):
        return self.x_ref.shape[1]

    @staticmethod
    def from_numpy(d: dict, device="cuda", dtype=torch.float32) -> "Problem":
        def t(a):
            return torch.as_tensor(a, dtype=dtype, device=device).contiguous()
        hz = d.get("horizon")
        ui = d.get("u_init")
        Cg, cg = d.get("C"), d.get("c")
        return Problem(x0=t(d["x0"]), Q=t(d["Q"]), x_ref=t(d["x_ref"]), R=t(d["R"]), u_ref=t(d["u_ref"]),
                       u_lo=t(d["u_lo"]), u_hi=t(d["u_hi"]),
                       horizon=None if hz is None else torch.as_tensor(hz, dtype=torch.int32, device=device).contiguous(),
                       u_init=None if ui is None else t(ui), C=None if Cg is None else t(Cg),
                       c=None if cg is None else t(cg))


@dataclasses.dataclass
class Solution:
    u: torch.Tensor         # [B, N, 4]
    x: torch.Tensor         # [B, N, 13]
    cost: torch.Tensor      # [B]
    iters: torch.Tensor     # [B] int32
    status: torch.Tensor    # [B] int32
    tape: torch.Tensor | None


def _ptr(t):
    return 0 if t is None else t.data_ptr()


class DiffMPC:
    """A library handle plus the buffers of one (B, N) problem shape.

    ``solve`` / ``backward`` enqueue on the current torch stream and return at
    once; outputs are preallocated per shape so repeated calls (and CUDA graph
    replays) reuse the same memory.
    """

    def __init__(self, N_max=40, B_max=8192, dtype=torch.float32, max_iter=8, tol=1e-6,
                 store_mode="store_all", exec_mode="persistent", ipb=0, model=None, alphas=None,
                 device=None, tpi=0, tape_budget=0):
        if not torch.cuda.is_available():
            raise RuntimeError("DiffMPC needs a CUDA device (libcamp.so has no CPU path)")
        self.device = torch.device(device or "cuda")
        self.dtype = dtype
        cfg = camp.mpc_config_default()
        cfg.N_max, cfg.B_max, cfg.dtype = int(N_max), int(B_max), _DTYPES[dtype]
        cfg.max_iter, cfg.tol = int(max_iter), float(tol)
        modes = {"store_all": camp.MPC_STORE_ALL, "recompute": camp.MPC_RECOMPUTE, "auto": camp.MPC_STORE_AUTO}
        if store_mode not in modes:
            raise ValueError(f"store_mode must be one of {sorted(modes)}")
        cfg.store_mode = modes[store_mode]
        modes = {"persistent": camp.MPC_EXEC_PERSISTENT, "plain": camp.MPC_EXEC_PLAIN, "scan": camp.MPC_EXEC_SCAN,
                 "auto": camp.MPC_EXEC_AUTO}
        if exec_mode not in modes:
            raise ValueError(f"exec_mode must be one of {sorted(modes)}")
        cfg.exec_mode = modes[exec_mode]
        cfg.ipb = int(ipb)
        cfg.tpi = int(tpi)
        cfg.tape_budget = int(tape_budget)
        if model is not None:
            cfg.dt, cfg.mass, cfg.arm, cfg.kappa_yaw, cfg.gravity = model.dt, model.mass, model.arm, model.kappa, model.gravity
            for i in range(3):
                cfg.inertia[i] = model.inertia[i]
        if alphas is not None:
            cfg.n_alpha = len(alphas)
            for i, a in enumerate(alphas):
                cfg.alpha[i] = a
        self.cfg = cfg
        with torch.cuda.device(self.device):
            code, self.h = camp.mpc_create(cfg)
        camp.check(code, "mpc_create")
        self._bufs = {}

    def close(self):
        if getattr(self, "h", None):
            camp.mpc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- marshalling ----------------------------------------------------------------
    def _cproblem(self, p: Problem):
        names = ("x0", "Q", "x_ref", "R", "u_ref", "u_lo", "u_hi") + (("C", "c") if p.C is not None else ())
        for name in names:
            t = getattr(p, name)
            if t is None or t.dtype != self.dtype or not t.is_contiguous() or t.device.type != "cuda":
                raise ValueError(f"{name} must be a contiguous {self.dtype} CUDA tensor")
        if p.C is not None and (p.C.dim() != 4 or p.C.shape[2:] != (17, 17) or p.c.dim() != 3 or p.c.shape[2] != 17):
            raise ValueError("C must be [B, NC, 17, 17] and c [B, Nc, 17]")
        return camp.mpc_problem(B=p.B, N=p.N, horizon=_ptr(p.horizon), x0=_ptr(p.x0), Q=_ptr(p.Q),
                                Nq=p.Q.shape[1], x_ref=_ptr(p.x_ref), R=_ptr(p.R), u_ref=_ptr(p.u_ref),
                                u_lo=_ptr(p.u_lo), u_hi=_ptr(p.u_hi), u_init=_ptr(p.u_init),
                                C=_ptr(p.C), NC=0 if p.C is None else p.C.shape[1],
                                c=_ptr(p.c), Nc=0 if p.c is None else p.c.shape[1])

    def alloc_solution(self, B, N) -> Solution:
        dev, dt = self.device, self.dtype
        tb = camp.mpc_tape_bytes(self.h, B, N)
        tape = torch.empty(max(tb // torch.tensor([], dtype=dt).element_size(), 1), dtype=dt, device=dev) if tb else None
        return Solution(u=torch.empty(B, N, 4, dtype=dt, device=dev), x=torch.empty(B, N, 13, dtype=dt, device=dev),
                        cost=torch.empty(B, dtype=dt, device=dev), iters=torch.empty(B, dtype=torch.int32, device=dev),
                        status=torch.empty(B, dtype=torch.int32, device=dev), tape=tape)

    @staticmethod
    def _csolution(s: Solution):
        return camp.mpc_solution(u=_ptr(s.u), x=_ptr(s.x), cost=_ptr(s.cost), iters=_ptr(s.iters),
                                 status=_ptr(s.status), tape=_ptr(s.tape),
                                 tape_bytes=0 if s.tape is None else s.tape.numel() * s.tape.element_size())

    # -- solves ---------------------------------------------------------------------
    def solve(self, p: Problem, out: Solution | None = None) -> Solution:
        s = out if out is not None else self.alloc_solution(p.B, p.N)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        camp.check(camp.mpc_solve_fwd(self.h, self._cproblem(p), self._csolution(s), stream), "mpc_solve_fwd")
        return s

    def backward(self, p: Problem, s: Solution, grad_u, grad_x=None, out=None):
        B, N = p.B, p.N
        if out is None:
            out = (torch.empty_like(p.Q), torch.empty_like(p.x_ref), torch.empty_like(p.x0))
        dQ, dxr, dx0 = out
        gu = grad_u.contiguous()
        gx = None if grad_x is None else grad_x.contiguous()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        camp.check(camp.mpc_solve_bwd(self.h, self._cproblem(p), self._csolution(s), gu.data_ptr(), _ptr(gx),
                                      dQ.data_ptr(), dxr.data_ptr(), dx0.data_ptr(), stream), "mpc_solve_bwd")
        return dQ, dxr, dx0

    def backward_general(self, p: Problem, s: Solution, grad_u, grad_x=None, out=None):
        """Gradients of a general-cost problem: (dL/dC, dL/dc, dL/dx0)."""
        if out is None:
            out = (torch.empty_like(p.C), torch.empty_like(p.c), torch.empty_like(p.x0))
        dC, dc, dx0 = out
        gu = grad_u.contiguous()
        gx = None if grad_x is None else grad_x.contiguous()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        camp.check(camp.mpc_solve_bwd_general(self.h, self._cproblem(p), self._csolution(s), gu.data_ptr(), _ptr(gx),
                                              dC.data_ptr(), dc.data_ptr(), dx0.data_ptr(), stream),
                   "mpc_solve_bwd_general")
        return dC, dc, dx0

    def autotune(self, p: Problem, s: Solution | None = None) -> int:
        s = s if s is not None else self.alloc_solution(p.B, p.N)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        code, ipb = camp.mpc_autotune(self.h, self._cproblem(p), self._csolution(s), stream)
        camp.check(code, "mpc_autotune")
        return ipb

    @property
    def exec_form(self) -> str:
        """The launch form solves use: "persistent", "plain" or "scan" (under
        exec_mode "auto", the one autotune measured faster)."""
        code, e = camp.mpc_exec_form(self.h)
        camp.check(code, "mpc_exec_form")
        return {camp.MPC_EXEC_PERSISTENT: "persistent", camp.MPC_EXEC_PLAIN: "plain", camp.MPC_EXEC_SCAN: "scan"}[e]

    def launch_shape(self, B, N):
        code, tpi, ipb, grid = camp.mpc_launch_shape(self.h, B, N)
        camp.check(code, "mpc_launch_shape")
        return tpi, ipb, grid

    def launch_count(self, has_horizon=False):
        code, f, b = camp.mpc_launch_count(self.h, has_horizon)
        camp.check(code, "mpc_launch_count")
        return f, b


class DiffMPCFunction(torch.autograd.Function):
    """u*, x* = MPC(x0, Q, x_ref; R, u_ref, u_lo, u_hi) with gradients w.r.t.
    x0, Q and x_ref from the library's adjoint solve.

    Every tensor the backward needs goes through ctx.save_for_backward, never
    a plain ctx attribute: an output kept on ctx would form a reference cycle
    (output -> grad_fn -> ctx -> output) that holds device memory until the
    garbage collector happens to run."""

    @staticmethod
    def forward(ctx, solver: DiffMPC, x0, Q, x_ref, R, u_ref, u_lo, u_hi, horizon=None):
        p = Problem(x0=x0.detach().contiguous(), Q=Q.detach().contiguous(), x_ref=x_ref.detach().contiguous(),
                    R=R.detach().contiguous(), u_ref=u_ref.detach().contiguous(), u_lo=u_lo.detach().contiguous(),
                    u_hi=u_hi.detach().contiguous(), horizon=horizon)
        s = solver.solve(p)
        ctx.solver = solver
        ctx.has_horizon = horizon is not None
        ctx.has_tape = s.tape is not None
        none = torch.empty(0, device=x0.device)
        ctx.save_for_backward(p.x0, p.Q, p.x_ref, p.R, p.u_ref, p.u_lo, p.u_hi,
                              horizon if horizon is not None else none, s.u, s.x, s.cost, s.iters, s.status,
                              s.tape if s.tape is not None else none)
        ctx.mark_non_differentiable(s.cost, s.iters, s.status)
        return s.u, s.x, s.cost, s.iters, s.status

    @staticmethod
    def backward(ctx, grad_u, grad_x, *_):
        x0, Q, x_ref, R, u_ref, u_lo, u_hi, hz, u, x, cost, iters, status, tape = ctx.saved_tensors
        p = Problem(x0=x0, Q=Q, x_ref=x_ref, R=R, u_ref=u_ref, u_lo=u_lo, u_hi=u_hi,
                    horizon=hz if ctx.has_horizon else None)
        s = Solution(u=u, x=x, cost=cost, iters=iters, status=status, tape=tape if ctx.has_tape else None)
        if grad_u is None:
            grad_u = torch.zeros_like(u)
        dQ, dxr, dx0 = ctx.solver.backward(p, s, grad_u, grad_x)
        return None, dx0, dQ, dxr, None, None, None, None, None


def diff_mpc(solver: DiffMPC, x0, Q, x_ref, R, u_ref, u_lo, u_hi, horizon=None):
    """Functional form: returns (u*, x*, cost, iters, status)."""
    return DiffMPCFunction.apply(solver, x0, Q, x_ref, R, u_ref, u_lo, u_hi, horizon)
