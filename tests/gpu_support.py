"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and the
FP64 oracle on the same seeded inputs, and compare them instance by instance.

Tolerances (FP32 path vs FP64 oracle, per instance):
  controls   |u - u_or|_2 / max(|u_or|_2, 1e-6)            <= 1e-4
  cost       |J - J_or| / max(|J_or|, 1e-12)                 <= 1e-5
  gradients  |g - g_or|_2 / max(|g_or|_2, 1e-9) per block   <= 1e-3
compare_iterates32 holds every sampled instance to the oracle's own returned
iterate -- converged or stopped at max_iter -- and excuses only instances
whose record shows a decision FP32 cannot resolve (a line-search gap or a
box-QP gradient margin below LS_MARGIN32 / QP_MARGIN32, reading R11),
reporting how many.

The FP64 path runs the same kernels in double: with every decision the same
(early iterations, tol = 0) it agrees to 1e-8; run to convergence, the last
accepted step (smaller than tol by definition) may go either way, so controls
agree to about tol.
"""
from __future__ import annotations

import functools
import multiprocessing as mp
import os

import numpy as np

import workloads as W
from oracle import adjoint, ilqr
from oracle.model import Quadrotor

QUAD = Quadrotor(W.DEFAULT_MODEL)

U_TOL32, J_TOL32, G_TOL32 = 1e-4, 1e-5, 1e-3
U_TOL64, J_TOL64, G_TOL64 = 1e-8, 1e-10, 1e-7       # identical decisions (early iterations)
U_TOL64C, J_TOL64C, G_TOL64C = 1e-6, 1e-9, 1e-5     # to convergence: last step < tol may differ
# decisions the FP32 path cannot resolve (reading R11): a material line-search
# gap below LS_MARGIN32 of the cost change's terms, a box-QP gradient below
# QP_MARGIN32 (relative) where its sign decides clamped or free, a control
# within BAND_MARGIN32 (relative) of the edge of the QP's epsilon band
LS_MARGIN32, QP_MARGIN32, BAND_MARGIN32 = 1e-6, 1e-5, 1e-7
# the FP32 error of a non-converged iterate: each Newton step carries about
# kappa(Q_uu) x 2^-24 of its size (kappa up to ~1e4 for the nearly collinear
# rotor pairs of this quadrotor), and a solve stopped at max_iter keeps the
# errors of its last, still large steps (measured: at most ~8e-4)
U_TOL32_ITER = 1e-3
# the cost of a non-converged iterate moves with its controls (its gradient
# is not zero there): against the oracle's iterate it is held to this; the
# cost at the GPU's own iterate is held to J_TOL32 (own_iterate_pool)
J_TOL32_ITER = 1e-4
# dL/dQ of a Q shared over the stages sums the stage terms d_x,t * (x*_t -
# x_ref,t), which can cancel (85:1 on an uneven-horizon track instance).  Its
# FP32 error is that of the terms -- the adjoint's d_x carries ~2e-5 of them
# (measured) -- so it is measured against max(|dQ|, SHARED_Q_TERMS x
# || sum_t |terms| ||): the floor acts only where the terms cancel by more than
# 1 / SHARED_Q_TERMS = 20
SHARED_Q_TERMS = 0.05
# at most this share of a sample may be excused as degenerate
EXCUSED_MAX_FRAC = 0.01
# a step of the controls below this [N] is at the FP32 noise level of an
# 8.5 N thrust (about 20 ulp): a convergence test (reading R5, tol 1e-6 N)
# against such a step cannot be resolved in FP32, so the iteration at which
# a solve stops may differ there (the controls then differ by such steps)
CONV_BAND32 = 1e-5
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


_BLAS_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _pool_map(fn, tasks):
    """fn over tasks in a spawned pool of one process per core, each with a
    single BLAS thread (the workers inherit the environment at spawn; many
    workers with many BLAS threads each oversubscribe the cores badly)."""
    old = {v: os.environ.get(v) for v in _BLAS_VARS}
    for v in _BLAS_VARS:
        os.environ[v] = "1"
    try:
        with mp.get_context("spawn").Pool(max(1, min(len(tasks), os.cpu_count() or 1))) as pool:
            return pool.map(fn, tasks, chunksize=1)
    finally:
        for v, val in old.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val


def _oracle_one(args):
    sub, max_iter, tol, gu, gx = args
    return oracle_solve(sub, [0], max_iter, tol, gu, gx)[0]


def oracle_solve_pool(prob, idx, max_iter, tol, grad_u=None, grad_x=None):
    """oracle_solve over a spawned process pool, one instance per task (for
    samples of the full-size batches); the same results as oracle_solve."""
    idx = [int(i) for i in idx]
    tasks = []
    for i in idx:
        sub = {k: v[i:i + 1] for k, v in prob.items() if isinstance(v, np.ndarray) and v.shape[:1] == (prob["x0"].shape[0],)}
        tasks.append((sub, max_iter, tol, None if grad_u is None else grad_u[i:i + 1],
                      None if grad_x is None else grad_x[i:i + 1]))
    return _pool_map(_oracle_one, tasks)


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


def shared_q_floor(pr, sol, gr):
    """The denominator floor of a shared Q's gradient error: SHARED_Q_TERMS x
    the norm of the summed stage-term magnitudes; 1e-9 for per-stage Q."""
    if pr.Q.shape[0] > 1:
        return 1e-9
    terms = np.array([gr.dX[t] * (sol.X[t] - pr.x_ref[t]) for t in range(pr.n)])
    return max(1e-9, SHARED_Q_TERMS * float(np.linalg.norm(np.abs(terms).sum(0))))


def stop_agrees(gs, gi, so):
    """GPU status / iteration count (gs, gi) against the oracle's record: equal
    (CONVERGED and STALLED being one normal end), or different only where the
    oracle's steps from the earlier of the two stops on were below CONV_BAND32
    (the convergence test of reading R5 cannot be resolved there in FP32)."""
    cls = lambda st: 0 if st in (0, 1) else st
    if cls(gs) == cls(so.status) and gi == so.iters:
        return True
    if gs not in (0, 1, 2) or so.status not in (0, 1, 2):
        return False
    k = min(gi, so.iters)
    return k >= 1 and all(v < CONV_BAND32 for v in so.du_hist[k - 1:])


def compare_iterates32(gpu, orc, idx, grad_u, grad_x=None, max_iter=None, u_tol=U_TOL32):
    """FP32 gate against the oracle's own returned iterate.  Every sampled
    instance -- converged or stopped at max_iter -- is compared: it must end
    in the oracle's state (CONVERGED and STALLED count as one normal end;
    stop_agrees) and match the oracle's u*, x* (U_TOL32 converged,
    U_TOL32_ITER at max_iter) and cost (J_TOL32 converged, J_TOL32_ITER at
    max_iter), and for converged solves its gradients (G_TOL32).  A
    comparison that fails is excused (and
    counted) only for an instance stopped at max_iter whose record shows a
    decision FP32 cannot resolve (degenerate_record); a converged solution
    does not depend on its path and is never excused.  Gradients use the
    oracle's adjoint on the GPU's final free sets where those differ only at
    degenerate controls.  Returns (report, failures); the report carries the
    counts and the largest and 99th percentile errors of the instances that
    passed."""
    N = orc[0][0].x_ref.shape[0] if orc else 0
    rep = dict(sampled=len(idx), compared=0, excused=0, excused_idx=[], converged=0, max_iter=0, mask_differs=0,
               stop_differs=0)
    errs = dict(u=[], x=[], J=[], dQ=[], dx_ref=[], dx0=[])
    fails = []
    cls = lambda st: 0 if st in (0, 1) else st
    for k, i in enumerate(idx):
        pr, so, gr = orc[k]
        rep["compared"] += 1
        conv = so.status in (ilqr.CONVERGED, ilqr.STALLED)
        rep["converged" if conv else "max_iter"] += 1
        gs, gi = int(gpu["status"][i]), int(gpu["iters"][i])
        mine, e = [], {}
        if not stop_agrees(gs, gi, so):
            mine.append((int(i), "status/iters", (gs, gi), (so.status, so.iters)))
        else:
            if not (cls(gs) == cls(so.status) and gi == so.iters):
                rep["stop_differs"] += 1
            e["u"] = rel(gpu["u"][i], so.U, 1e-6)
            e["x"] = rel(gpu["x"][i], so.X, 1e-6)
            e["J"] = abs(float(gpu["cost"][i]) - so.J) / max(abs(so.J), 1e-12)
            utol = u_tol if conv else U_TOL32_ITER
            if e["u"] > utol or e["x"] > utol:
                mine.append((int(i), "u/x", e["u"], e["x"]))
            if e["J"] > (J_TOL32 if conv else J_TOL32_ITER):
                mine.append((int(i), "cost", e["J"]))
            # gradients against the oracle's at its solution for converged solves; at
            # max_iter the iterates differ by up to U_TOL32_ITER, and the gradients are
            # checked at the GPU's own iterate instead (own_iterate_pool)
            if gr is not None and "dQ" in gpu and conv and gs in (0, 1):
                ref_gr = gr
                if "masks" in gpu:
                    gm = [_mask_bits(gpu["masks"][i][t]) for t in range(pr.n)]
                    diff = [(t, a) for t in range(pr.n) for a in range(4) if gm[t][a] != so.bp.free[t][a]]
                    if diff:
                        rep["mask_differs"] += 1
                        if not all(_degenerate(pr, so.bp, so.U, t, a) for t, a in diff):
                            mine.append((int(i), "free set", diff[:4]))
                        else:
                            gx = np.zeros((N, 13)) if grad_x is None else grad_x[i]
                            ref2 = ilqr.at_iterate(QUAD, pr, so.U, free_override=gm)
                            ref2.X = so.X
                            ref_gr = adjoint.adjoint(pr, ref2, gx, grad_u[i])
                for name, r in (("dQ", ref_gr.dQ), ("dx_ref", ref_gr.dx_ref), ("dx0", ref_gr.dx0)):
                    e[name] = rel(gpu[name][i], r, shared_q_floor(pr, so, ref_gr) if name == "dQ" else 1e-9)
                    if e[name] > G_TOL32:
                        mine.append((int(i), name, e[name]))
        if mine:
            if not conv and degenerate_record(so):
                rep["excused"] += 1
                rep["excused_idx"].append(int(i))
                continue
            fails.extend(mine)
            continue
        for name, v in e.items():
            errs[name].append(v)
    for name, v in errs.items():
        if v:
            rep[f"max_{name}"] = float(np.max(v))
            rep[f"p99_{name}"] = float(np.percentile(v, 99))
    return rep, fails


def _fd_one(args):
    """Central differences (eps = 1e-4, relative for weights below 1) of
    L = g_u . u through the oracle's frozen-linearization LQR (the Gauss-Newton
    target of reading R10) at the GPU's own returned iterate (reading R8: the
    LQR at the returned iterate), on the GPU's final free sets where those
    differ from the oracle's only at degenerate controls, for the listed
    entries of Q, x_ref and x0."""
    sub, U, masks, gu, picks = args
    pr = ilqr.problem_from_batch(sub, 0)
    ref = ilqr.at_iterate(QUAD, pr, U)
    gm = [_mask_bits(masks[t]) for t in range(pr.n)]
    diff = [(t, a) for t in range(pr.n) for a in range(4) if gm[t][a] != ref.bp.free[t][a]]
    ok = all(_degenerate(pr, ref.bp, ref.U, t, a) for t, a in diff)
    if diff and ok:
        X = ref.X
        ref = ilqr.at_iterate(QUAD, pr, U, free_override=gm)
        ref.X = X

    def L(**kw):
        X, Uf = adjoint.frozen_lqr_solve(pr, ref, QUAD, **kw)
        return float(np.sum(gu[0] * Uf))

    fd = {}
    for name, base in (("Q", pr.Q), ("x_ref", pr.x_ref), ("x0", pr.x0)):
        vals = []
        for idx in picks[name]:
            idx = tuple(idx)
            eps = 1e-4 * min(1.0, max(abs(base[idx]), 1e-2))
            p, m = base.copy(), base.copy()
            p[idx] += eps
            m[idx] -= eps
            vals.append((L(**{name: p}) - L(**{name: m})) / (2 * eps))
        fd[name] = np.array(vals)
    return fd, diff, ok


def fd_gradients_pool(gpu, prob, idx, grad_u, picks):
    """_fd_one at the GPU's iterate for each instance of idx, over a spawned process pool."""
    tasks = [(_sub(prob, int(i)), np.asarray(gpu["u"][int(i)], float), gpu["masks"][int(i)],
              grad_u[int(i):int(i) + 1], picks) for i in idx]
    return _pool_map(_fd_one, tasks)


def _sub(prob, i):
    """Instance i of a batch as a batch of one (every per-instance array)."""
    B = prob["x0"].shape[0]
    return {k: v[i:i + 1] for k, v in prob.items() if isinstance(v, np.ndarray) and v.shape[:1] == (B,)}


# relative size of the errors FP32 accumulates in a stage's Q_uu and q_u over a
# Riccati sweep (the perturbation of step_sensitivity)
QP_INPUT_ERR32 = 1e-5


def _one_step(args):
    sub, U_prev, tol, sens = args
    pr = ilqr.problem_from_batch(dict(sub, u_init=U_prev[None]), 0)
    so = ilqr.solve(QUAD, pr, 1, tol)
    if not sens:
        return so, 0.0
    worst = 0.0
    for seed in range(2):
        rng = np.random.default_rng(seed)

        def perturb(H, g):
            E = rng.standard_normal(H.shape)
            return H * (1.0 + QP_INPUT_ERR32 * 0.5 * (E + E.T)), g * (1.0 + QP_INPUT_ERR32 * rng.standard_normal(g.shape))

        sp = ilqr.solve(QUAD, pr, 1, tol, qp_perturb=perturb)
        worst = max(worst, rel(sp.U, so.U, 1e-6))
    return so, worst


def one_step_pool(prob, idx, U_prev, tol, sensitivity=False, U_rows=None):
    """The oracle's single iteration (Algorithm 2's inner loop once) from the
    given iterates U_prev[i] (warm start), for each instance of idx: [(record,
    sensitivity)].  With ``sensitivity`` the step is also taken with every
    stage's box-QP inputs (Q_uu, q_u) perturbed by QP_INPUT_ERR32 relative
    noise (two seeds), and the largest relative change of the controls is
    returned: how far FP32-sized input errors move this step (reading R11).
    ``U_rows`` gives the iterates row by row (one per entry of idx) instead."""
    rows = U_rows if U_rows is not None else [U_prev[int(i)] for i in idx]
    return _pool_map(_one_step, [(_sub(prob, int(i)), np.asarray(u, float), tol, sensitivity)
                                 for i, u in zip(idx, rows)])


def _own_iterate(args):
    sub, U, masks, gu, gx = args
    pr = ilqr.problem_from_batch(sub, 0)
    N = pr.x_ref.shape[0]
    gx = np.zeros((N, 13)) if gx is None else gx
    ref = ilqr.at_iterate(QUAD, pr, U)
    diff, ok = [], True
    if masks is not None:
        gm = [_mask_bits(masks[t]) for t in range(pr.n)]
        diff = [(t, a) for t in range(pr.n) for a in range(4) if gm[t][a] != ref.bp.free[t][a]]
        ok = all(_degenerate(pr, ref.bp, ref.U, t, a) for t, a in diff)
        if diff and ok:
            ref2 = ilqr.at_iterate(QUAD, pr, U, free_override=gm)
            ref2.X = ref.X
            return ref, adjoint.adjoint(pr, ref2, gx, gu), diff, ok
    return ref, adjoint.adjoint(pr, ref, gx, gu), diff, ok


def own_iterate_pool(prob, idx, gpu, grad_u, grad_x=None):
    """For each instance of idx, the oracle's record of the GPU's returned
    controls (ilqr.at_iterate: FP64 rollout, cost, linearization and
    factorization) and its adjoint gradients there, on the GPU's final free
    sets where those differ from the oracle's only at degenerate controls.
    Returns [(record, gradients, differing (t, a), all differences degenerate)]."""
    tasks = []
    for i in idx:
        i = int(i)
        tasks.append((_sub(prob, i), np.asarray(gpu["u"][i], float), None if "masks" not in gpu else gpu["masks"][i],
                      grad_u[i], None if grad_x is None else grad_x[i]))
    return _pool_map(_own_iterate, tasks)


def degenerate_record(so):
    """Reading R11: the record shows a decision FP32 cannot resolve."""
    return so.ls_margin < LS_MARGIN32 or so.qp_margin < QP_MARGIN32 or so.qp_band < BAND_MARGIN32
