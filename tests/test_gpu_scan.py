"""Parity of the stage-parallel Riccati phase (exec_mode "scan": the
associative-scan LQR of the related work in Sec. II with the box QPs' free
sets guessed, then the stages the guess got wrong by the sequential
recursion) with the FP64 oracle's sequential recursion of Sec. IV-2, and
with the library's own sequential phase.

Every stage's box QP is the one the sequential recursion solves, from the same
V_{t+1}, v_{t+1} up to rounding, so the iterates are the oracle's: in FP64 to
rounding while every decision is clear-cut (the same gates as the sequential
path's FP64 tests); in FP32 within the product path's gates.  The scan's FP32
costate carries about 1e-4 of its size in rounding (the composed transition
parts); the kernel's costate pass reruns the recursion's vector part
sequentially, so the converged controls meet the sequential path's U_TOL32.
With store-all the forward's final factorization (the tape) is the sequential
recursion on the whole block; the backward is the library's, and the gradients are
held to the sequential path's gates."""
import numpy as np
import pytest

from gpu_support import (EXCUSED_MAX_FRAC, G_TOL32, G_TOL64, G_TOL64C, J_TOL64, J_TOL64C, TIE64, U_TOL32, U_TOL64,
                         U_TOL64C, cached_problem, compare, compare_iterates32, oracle_solve, oracle_solve_pool, rel,
                         run_gpu)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _grads(B, N, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(B, N, 4)), rng.normal(size=(B, N, 13)) * 0.1


@pytest.mark.parametrize("name,B,N,horizons", [("hover", 8, 10, False), ("track", 37, 20, True),
                                               ("uneven", 33, 40, False), ("mem", 9, 30, False)])
def test_scan_fp64_early_iterations_identical_to_oracle(name, B, N, horizons):
    """Three iterations with tol = 0 in double: values agree with the oracle's
    to rounding (ragged horizons, shared and per-stage Q, guesses that miss
    where saturations move)."""
    prob = cached_problem(name, B, N, 0, horizons)
    gu, gx = _grads(B, N, 1)
    gpu = run_gpu(prob, torch.float64, 3, 0.0, gu, gx, N_max=40, exec_mode="scan")
    idx = list(range(B))
    orc = oracle_solve(prob, idx, 3, 0.0, gu, gx)
    report, fails = compare(gpu, orc, idx, U_TOL64, J_TOL64, G_TOL64, skip_ties=TIE64)
    print(name, report)
    assert report["compared"] >= 0.8 * B
    assert not fails, (fails[:5], report)


@pytest.mark.parametrize("name,B,N,horizons,mi", [("hover", 8, 10, False, 10), ("track", 37, 20, True, 8),
                                                  ("uneven", 33, 40, False, 12)])
def test_scan_fp64_to_convergence_matches_oracle(name, B, N, horizons, mi):
    prob = cached_problem(name, B, N, 0, horizons)
    gu, gx = _grads(B, N, 1)
    gpu = run_gpu(prob, torch.float64, mi, 1e-6, gu, gx, N_max=40, exec_mode="scan")
    idx = list(range(B))
    orc = oracle_solve(prob, idx, mi, 1e-6, gu, gx)
    report, fails = compare(gpu, orc, idx, U_TOL64C, J_TOL64C, G_TOL64C, counts="final")
    print(name, report)
    assert not fails, (fails[:5], report)


@pytest.mark.parametrize("B,N", [(1, 50), (5, 2), (6, 50), (3, 64)])
def test_scan_latency_horizons_match_oracle(B, N):
    """The horizons of the solver-latency setting (hover, exactly five
    iterations with tol = 0), handles sized to N, and the longest horizon the
    library takes: FP64 to rounding; FP32 within 1e-3 of the oracle's
    controls (the sequential path's bound for this setting)."""
    prob = cached_problem("hover", B, N, 7)
    gu, gx = _grads(B, N, 3)
    idx = list(range(B))
    orc = oracle_solve(prob, idx, 5, 0.0, gu, gx)
    gpu = run_gpu(prob, torch.float64, 5, 0.0, gu, gx, exec_mode="scan")
    report, fails = compare(gpu, orc, idx, U_TOL64, J_TOL64, G_TOL64, skip_ties=TIE64)
    print("fp64", B, N, report)
    assert report["compared"] >= B - 1
    assert not fails, (fails[:5], report)
    gpu32 = run_gpu(prob, torch.float32, 5, 0.0, gu, gx, exec_mode="scan")
    assert np.all(np.isfinite(gpu32["u"])) and np.all(gpu32["iters"] == 5)
    for i in range(B):
        u_or = orc[i][1].U
        e = np.linalg.norm(gpu32["u"][i] - u_or) / max(np.linalg.norm(u_or), 1e-6)
        print("fp32", i, e)
        assert e <= 1e-3


@pytest.mark.parametrize("name,B,N,horizons,mi", [("hover", 64, 20, False, 20), ("track", 64, 20, True, 20),
                                                  ("hover", 24, 50, False, 20)])
def test_scan_fp32_matches_oracle(name, B, N, horizons, mi):
    """FP32: every instance against the oracle's own returned iterate with the
    product path's gates, converged controls within U_TOL32 (only
    recorded-degenerate decisions of solves stopped at max_iter excused)."""
    prob = cached_problem(name, B, N, 0, horizons)
    gu, gx = _grads(B, N, 2)
    gpu = run_gpu(prob, torch.float32, mi, 1e-6, gu, gx, N_max=max(N, 40), exec_mode="scan")
    idx = list(range(B))
    orc = oracle_solve_pool(prob, idx, mi, 1e-6, gu, gx)
    report, fails = compare_iterates32(gpu, orc, idx, gu, gx)
    print(name, N, report, fails[:5])
    assert report["excused"] <= max(1, EXCUSED_MAX_FRAC * B)
    assert not fails, (fails[:5], report)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_scan_agrees_with_the_sequential_phase(dtype):
    """The same solves through the sequential plain form and the scan form:
    same statuses and iteration counts, controls of the solves that both
    converged within rounding of each other (FP64 the identical-decision gate
    U_TOL64; FP32 U_TOL32)."""
    dt = getattr(torch, dtype)
    prob = cached_problem("track", 48, 20, 4, True)
    a = run_gpu(prob, dt, 20, 1e-6, exec_mode="plain", ipb=1)
    b = run_gpu(prob, dt, 20, 1e-6, exec_mode="scan")
    conv = (a["status"] == 0) & (b["status"] == 0)
    assert conv.sum() >= 0.5 * len(conv)
    if dtype == "float64":
        assert np.array_equal(a["status"], b["status"]) and np.array_equal(a["iters"], b["iters"])
    err = max(rel(a["u"][i], b["u"][i], 1e-6) for i in np.flatnonzero(conv))
    print(dtype, err)
    assert err <= (U_TOL64 if dtype == "float64" else U_TOL32)


def test_scan_general_cost_keeps_the_sequential_phase():
    """A general cost in the scan form runs the sequential Riccati phase:
    the result equals the plain form's."""
    import workloads as W
    B, N = 16, 10
    prob = W.hover_targets(B, N, seed=3)
    diag = np.concatenate([prob["Q"][:, 0], prob["R"]], axis=1)
    C = np.einsum("bi,ij->bij", diag, np.eye(17))[:, None]
    zr = np.concatenate([prob["x_ref"], np.repeat(prob["u_ref"][:, None], N, axis=1)], axis=2)
    c = -np.einsum("bkij,btj->bti", C, zr)
    gp = dict(prob, C=C, c=c)
    a = run_gpu(gp, torch.float64, 8, 1e-6, exec_mode="plain", ipb=1)
    b = run_gpu(gp, torch.float64, 8, 1e-6, exec_mode="scan")
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["iters"], b["iters"])


def test_scan_edge_cases():
    """Horizon one (no dynamics: u* = clamp(u_ref)), every control pinned
    (u_lo = u_hi: no free control, no gains), a non-finite input flagged and
    isolated, and an empty batch, in the scan form."""
    rng = np.random.default_rng(9)
    gu = rng.normal(size=(16, 10, 4))
    prob = dict(cached_problem("hover", 16, 10, 5))
    prob["horizon"] = np.ones(16, dtype=np.int32)
    prob["u_ref"] = prob["u_ref"] + np.linspace(-3, 8, 16)[:, None]
    g = run_gpu(prob, torch.float64, 8, 1e-6, gu, exec_mode="scan")
    np.testing.assert_allclose(g["u"][:, 0], np.clip(prob["u_ref"], 0, 8.5), atol=1e-12)
    assert np.all(g["u"][:, 1:] == 0) and np.all(g["x"][:, 1:] == 0)
    prob2 = dict(cached_problem("hover", 16, 10, 6))
    prob2["u_lo"] = prob2["u_hi"] = np.full((16, 4), 3.0)
    g2 = run_gpu(prob2, torch.float32, 8, 1e-6, gu, exec_mode="scan")
    assert np.all(g2["u"] == 3.0) and np.all(np.isin(g2["status"], [0, 1]))
    ref = run_gpu(prob2, torch.float32, 8, 1e-6, gu, exec_mode="plain", ipb=1)
    assert np.array_equal(g2["status"], ref["status"]) and np.array_equal(g2["iters"], ref["iters"])
    prob3 = dict(cached_problem("hover", 12, 10, 7))
    prob3["x0"] = prob3["x0"].copy()
    prob3["x0"][3, 0] = np.nan
    prob3["Q"] = prob3["Q"].copy()
    prob3["Q"][5, 0, 2] = np.inf
    g3 = run_gpu(prob3, torch.float32, 8, 1e-6, gu[:12], exec_mode="scan")
    assert g3["status"][3] == 3 and g3["status"][5] == 3
    ok = [i for i in range(12) if i not in (3, 5)]
    assert np.isfinite(g3["u"][ok]).all() and np.all(np.isin(g3["status"][ok], [0, 1, 2]))
    from paper_2605_29155_gb300 import DiffMPC, Problem, camp
    solver = DiffMPC(N_max=10, B_max=4, exec_mode="scan")
    p = Problem.from_numpy({k: (v[:0] if isinstance(v, np.ndarray) else v)
                            for k, v in cached_problem("hover", 4, 10, 1).items()})
    out = solver.alloc_solution(0, 10)
    code = camp.mpc_solve_fwd(solver.h, solver._cproblem(p), solver._csolution(out),
                              torch.cuda.current_stream().cuda_stream)
    assert code == camp.MPC_OK
    solver.close()


def test_scan_graph_replay_and_recompute():
    """The scan form's forward and backward captured in one CUDA graph replay
    bit-identically to the eager calls.  In the scan form the store-all tape
    comes from a final stage-parallel factorization and the recompute backward
    re-factors sequentially: the forward outputs are the same bit for bit, the
    gradients the same within the FP32 gradient gate."""
    from paper_2605_29155_gb300 import DiffMPC, Problem
    B, N = 12, 30
    prob = cached_problem("hover", B, N, 8)
    gu, gx = _grads(B, N, 8)
    solver = DiffMPC(N_max=N, B_max=B, exec_mode="scan", max_iter=6, tol=0.0)
    p = Problem.from_numpy(prob)
    gu_t = torch.as_tensor(gu, dtype=torch.float32, device="cuda")
    s = solver.alloc_solution(B, N)
    grads = (torch.empty_like(p.Q), torch.empty_like(p.x_ref), torch.empty_like(p.x0))
    solver.solve(p, s)
    solver.backward(p, s, gu_t, out=grads)
    torch.cuda.synchronize()
    eager = [t.clone() for t in (s.u, s.cost, s.iters, *grads)]
    for t in (s.u, s.cost, *grads):
        t.zero_()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            solver.solve(p, s)
            solver.backward(p, s, gu_t, out=grads)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, (s.u, s.cost, s.iters, *grads)):
        assert torch.equal(a, b)
    solver.close()
    a = run_gpu(prob, torch.float32, 6, 0.0, gu, gx, exec_mode="scan", store_mode="store_all")
    b = run_gpu(prob, torch.float32, 6, 0.0, gu, gx, exec_mode="scan", store_mode="recompute")
    for k in ("u", "x", "cost", "iters", "status"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    for k in ("dQ", "dx_ref", "dx0"):
        for i in range(B):
            e = rel(a[k][i], b[k][i], 1e-9)
            assert e <= G_TOL32, (k, i, e)
