"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and the
FP64 oracle on the same seeded inputs, and compare them instance by instance.

Tolerances (FP32 path vs FP64 oracle, per instance):
  controls   |u - u_or|_2 / max(|u_or|_2, 1e-6)            <= 1e-4
  cost       |J - J_or| / max(|J_or|, 1e-12)                 <= 1e-5
  gradients  |g - g_or|_2 / max(|g_or|_2, 1e-9) per block   <= 1e-3, where for
             a Q shared over the stages the denominator is at least 0.1 x the
             size of the per-stage terms its gradient sums (dq_term_scale)
Instances the oracle solves to convergence are compared with its solution.
Instances still iterating at max_iter follow a path that rounding-level
decisions steer (reading R12), so for them the returned iterate is checked
instead: x* against the FP64 rollout of u*, the cost at (x*, u*), and the
gradients against the oracle's adjoint at that same iterate.

The FP64 path runs the same kernels in double: with every decision the same
(early iterations, tol = 0) it agrees to 1e-8; run to convergence, the last
accepted step (smaller than tol by definition) may go either way, so controls
agree to about tol.
"""
from __future__ import annotations

import functools

import numpy as np

import workloads as W
from oracle import adjoint, ilqr
from oracle.model import Quadrotor

QUAD = Quadrotor(W.DEFAULT_MODEL)

U_TOL32, J_TOL32, G_TOL32 = 1e-4, 1e-5, 1e-3
U_TOL64, J_TOL64, G_TOL64 = 1e-8, 1e-10, 1e-7       # identical decisions (early iterations)
U_TOL64C, J_TOL64C, G_TOL64C = 1e-6, 1e-9, 1e-5     # to convergence: last step < tol may differ
# decisions the FP32 path cannot resolve: relative cost-change gaps / gradient margins
LS_MARGIN32, QP_MARGIN32 = 1e-5, 1e-5
# alpha decisions FP64 cannot resolve (any size of step)
TIE64 = 1e-9


# Tape layout (opaque to callers, read here only to compare free sets): per
# group of 32 instances and per stage, 210 rows of 32 values -- the computed
# columns of F_t (143), K_t (52), the masked factor (14), the free mask (1).
TAPE_REC, TAPE_MASK_ROW = 210, 209


def tape_rows(tape, B, N, row):
    """Row `row` of every instance's tape record, as a [B, N] tensor."""
    G = (B + 31) // 32
    return tape[: G * N * TAPE_REC * 32].view(G, N, TAPE_REC, 32)[:, :, row, :].permute(0, 2, 1).reshape(G * 32, N)[:B]


def tape_records(tape, B, N):
    """Every instance's tape records as a [B, N, 210] tensor."""
    G = (B + 31) // 32
    return tape[: G * N * TAPE_REC * 32].view(G, N, TAPE_REC, 32).permute(0, 3, 1, 2).reshape(G * 32, N, TAPE_REC)[:B]


def run_gpu(prob, dtype, max_iter, tol, grad_u=None, grad_x=None, store_mode="store_all",
            exec_mode="persistent", ipb=0, N_max=None, B_max=None, solver=None, tpi=0):
    import torch
    from paper_2605_29155_gb300 import DiffMPC, Problem

    B, N = prob["x0"].shape[0], prob["x_ref"].shape[1]
    own = solver is None
    if own:
        solver = DiffMPC(N_max=N_max or N, B_max=B_max or max(B, 1), dtype=dtype, max_iter=max_iter, tol=tol,
                         store_mode=store_mode, exec_mode=exec_mode, ipb=ipb, tpi=tpi)
    p = Problem.from_numpy(prob, dtype=dtype)
    s = solver.solve(p)
    out = dict(u=s.u, x=s.x, cost=s.cost, iters=s.iters, status=s.status)
    if s.tape is not None:
        out["masks"] = tape_rows(s.tape, B, N, TAPE_MASK_ROW).to(torch.int32)
    if grad_u is not None:
        gu = torch.as_tensor(grad_u, dtype=dtype, device="cuda")
        gx = None if grad_x is None else torch.as_tensor(grad_x, dtype=dtype, device="cuda")
        dQ, dxr, dx0 = solver.backward(p, s, gu, gx)
        out.update(dQ=dQ, dx_ref=dxr, dx0=dx0)
    torch.cuda.synchronize()
    res = {k: v.detach().cpu().numpy() for k, v in out.items()}
    if own:
        solver.close()
    return res


def oracle_solve(prob, idx, max_iter, tol, grad_u=None, grad_x=None):
    out = []
    N = prob["x_ref"].shape[1]
    for i in idx:
        pr = ilqr.problem_from_batch(prob, i)
        so = ilqr.solve(QUAD, pr, max_iter, tol)
        gr = None
        if grad_u is not None and so.status in (ilqr.CONVERGED, ilqr.STALLED, ilqr.MAX_ITER):
            gx = np.zeros((N, 13)) if grad_x is None else grad_x[i]
            gr = adjoint.adjoint(pr, so, gx, grad_u[i])
        out.append((pr, so, gr))
    return out


def rel(a, b, floor):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), floor))


def compare(gpu, orc, idx, u_tol, j_tol, g_tol, counts="exact", skip_degenerate=False, skip_ties=0.0):
    """Per-instance comparison; returns a report dict and a list of failures.

    counts: "exact"  status and iteration count identical;
            "final"  CONVERGED and STALLED (both normal ends) count as equal and
                     the counts may differ by one: the last accepted step of a
                     converging solve is below tol and can fall either way;
            None     not compared."""
    fails, report = [], dict(max_u=0.0, max_J=0.0, max_g=0.0, excluded=0, compared=0)
    for k, i in enumerate(idx):
        pr, so, gr = orc[k]
        if skip_degenerate and (so.ls_margin < LS_MARGIN32 or so.qp_margin < QP_MARGIN32):
            report["excluded"] += 1
            continue
        if skip_ties and so.ls_margin_any < skip_ties:
            report["excluded"] += 1
            continue
        report["compared"] += 1
        gs, gi = int(gpu["status"][i]), int(gpu["iters"][i])
        if counts == "exact" and (gs != so.status or gi != so.iters):
            fails.append((i, "status/iters", (gs, gi), (so.status, so.iters)))
            continue
        if counts == "final":
            cls = lambda st: 0 if st in (0, 1) else st
            if cls(gs) != cls(so.status) or abs(gi - so.iters) > 1:
                fails.append((i, "status/iters", (gs, gi), (so.status, so.iters)))
                continue
        eu = rel(gpu["u"][i], so.U, 1e-6)
        ex = rel(gpu["x"][i], so.X, 1e-6)
        ej = abs(float(gpu["cost"][i]) - so.J) / max(abs(so.J), 1e-12)
        report["max_u"] = max(report["max_u"], eu, ex)
        report["max_J"] = max(report["max_J"], ej)
        if eu > u_tol or ex > u_tol:
            fails.append((i, "u/x", eu, ex))
        if ej > j_tol:
            fails.append((i, "cost", ej))
        if gr is not None and "dQ" in gpu:
            for name, ref in (("dQ", gr.dQ), ("dx_ref", gr.dx_ref), ("dx0", gr.dx0)):
                eg = rel(gpu[name][i], ref, 1e-9)
                report["max_g"] = max(report["max_g"], eg)
                if eg > g_tol:
                    fails.append((i, name, eg))
    return report, fails


@functools.lru_cache(maxsize=None)
def cached_problem(name, B, N, seed=0, horizons=False):
    if name == "hover":
        return W.hover_targets(B, N, seed=seed,
                               horizons=W.uneven_horizons(B, 1, N, seed + 5) if horizons else None)
    if name == "track":
        return W.race_track(B, N, seed=seed,
                            horizons=W.uneven_horizons(B, 1, N, seed + 5) if horizons else None)
    if name == "mem":
        return W.hover_targets(B, N, seed=seed, Nq=N, per_stage_jitter=0.1)
    if name == "uneven":
        return W.race_track(B, N, seed=seed, horizons=W.uneven_horizons(B, 5, N, seed + 1000), u_hi_spread=0.2)
    raise KeyError(name)


def _mask_bits(m):
    return np.array([(int(m) >> a) & 1 for a in range(4)], dtype=bool)


def _degenerate(prob_i, so_bp, U, t, a, du=1e-4, rel_grad=1e-4):
    """A free/clamped decision FP32 cannot be expected to reproduce: the
    control lies within du of a bound, or its gradient at the bound is tiny."""
    lo, hi = prob_i.u_lo[a], prob_i.u_hi[a]
    if min(abs(U[t][a] - lo), abs(hi - U[t][a])) < du:
        return True
    return so_bp.margin < rel_grad


def compare32(gpu, prob, orc, idx, grad_u, grad_x=None):
    """FP32 gate: instances the oracle converges, and instances whose returned
    iterate is the oracle's (the same path), against the oracle's solution;
    the rest at their own returned iterate.  Gradients are compared with the oracle's
    adjoint on the GPU's own final free sets (tape masks); a free set that
    differs from the oracle's must differ only at degenerate controls.
    Returns (report, failures)."""
    N = prob["x_ref"].shape[1]
    rep = dict(converged=0, same_iterate=0, at_iterate=0, mask_differs=0, max_u=0.0, max_J=0.0, max_g=0.0,
               max_roll=0.0)
    fails = []
    for k, i in enumerate(idx):
        pr, so, gr = orc[k]
        gx = np.zeros((N, 13)) if grad_x is None else grad_x[i]
        eu = rel(gpu["u"][i], so.U, 1e-6)
        ex = rel(gpu["x"][i], so.X, 1e-6)
        if so.status == ilqr.CONVERGED or (eu <= U_TOL32 and ex <= U_TOL32):
            # same solution (or the same iterate of the same path)
            rep["converged" if so.status == ilqr.CONVERGED else "same_iterate"] += 1
            ref, ref_gr = so, gr
            rep["max_u"] = max(rep["max_u"], eu, ex)
            if eu > U_TOL32 or ex > U_TOL32:
                fails.append((i, "u/x", eu, ex))
        else:
            rep["at_iterate"] += 1
            ref = ilqr.at_iterate(QUAD, pr, gpu["u"][i].astype(float))
            er = rel(gpu["x"][i], ref.X, 1e-6)
            rep["max_roll"] = max(rep["max_roll"], er)
            if er > U_TOL32:
                fails.append((i, "rollout", er))
            ref_gr = adjoint.adjoint(pr, ref, gx, grad_u[i]) if grad_u is not None else None
        ej = abs(float(gpu["cost"][i]) - ref.J) / max(abs(ref.J), 1e-12)
        rep["max_J"] = max(rep["max_J"], ej)
        if ej > J_TOL32:
            fails.append((i, "cost", ej))
        if ref_gr is None or "dQ" not in gpu:
            continue
        if "masks" in gpu:
            gm = [_mask_bits(gpu["masks"][i][t]) for t in range(pr.n)]
            diff = [(t, a) for t in range(pr.n) for a in range(4) if gm[t][a] != ref.bp.free[t][a]]
            if diff:
                rep["mask_differs"] += 1
                if not all(_degenerate(pr, ref.bp, ref.U, t, a) for t, a in diff):
                    fails.append((i, "free set", diff[:4]))
                    continue
                ref2 = ilqr.at_iterate(QUAD, pr, ref.U, free_override=gm)
                ref2.X = ref.X
                ref_gr = adjoint.adjoint(pr, ref2, gx, grad_u[i])
        for name, r in (("dQ", ref_gr.dQ), ("dx_ref", ref_gr.dx_ref), ("dx0", ref_gr.dx0)):
            floor = 1e-9
            if name == "dQ" and pr.Q.shape[0] == 1:
                floor = max(floor, 0.1 * dq_term_scale(pr, ref, ref_gr))
            eg = rel(gpu[name][i], r, floor)
            rep["max_g"] = max(rep["max_g"], eg)
            if eg > G_TOL32:
                fails.append((i, name, eg))
    return rep, fails


def dq_term_scale(pr, sol, gr):
    """|| sum_t |d_x,t * (x*_t - x_ref,t)| ||: the size of the terms a shared
    Q's gradient sums over the stages.  Those terms can cancel (the sum can be
    ~60x smaller than their magnitudes), and a rounding error of the sum is
    relative to them, not to the sum."""
    terms = np.array([gr.dX[t] * (sol.X[t] - pr.x_ref[t]) for t in range(pr.n)])
    return float(np.linalg.norm(np.abs(terms).sum(0)))
