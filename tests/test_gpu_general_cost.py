"""Parity of the general stage cost of Eq. (2) -- dense C_t (state-control
cross terms included) and c_t -- on the CUDA path (through the C ABI) with the
FP64 oracle, and its gradients dL/dC_t, dL/dc_t, dL/dx0."""
import numpy as np
import pytest

import workloads as W
from gpu_support import G_TOL64C, J_TOL64C, QUAD, TIE64
from oracle import adjoint, ilqr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def general_problem(B, N, seed, NC, Nc, cfg="hover"):
    """A seeded batch with C = diag(Q, R) + 0.05 M'M / 17 (M ~ N(0, 1), 17 x 17)
    and c_t = -C z_ref,t, z_ref,t = [x_ref_t; u_ref]: the hover or track
    targets with cross terms.  NC, Nc in {1, N}."""
    b = W.hover_targets(B, N, seed=seed) if cfg == "hover" else W.race_track(B, N, seed=seed)
    rng = np.random.default_rng(seed + 100)
    C = np.zeros((B, NC, 17, 17))
    c = np.zeros((B, Nc, 17))
    for i in range(B):
        for k in range(NC):
            M = rng.normal(size=(17, 17))
            C[i, k] = np.diag(np.concatenate([b["Q"][i, 0], b["R"][i]])) + 0.05 * (M.T @ M) / 17
        for k in range(Nc):
            Ck = C[i, k if NC > 1 else 0]
            c[i, k] = -Ck @ np.concatenate([b["x_ref"][i, k], b["u_ref"][i]])
    return dict(b, C=C, c=c)


def run_general(prob, dtype, max_iter, tol, gu, gx=None, store_mode="store_all", tpi=0, exec_mode="persistent",
                ipb=0):
    from paper_2605_29155_gb300 import DiffMPC, Problem
    B, N = prob["x0"].shape[0], prob["x_ref"].shape[1]
    solver = DiffMPC(N_max=N, B_max=B, dtype=dtype, max_iter=max_iter, tol=tol, store_mode=store_mode, tpi=tpi,
                     exec_mode=exec_mode, ipb=ipb)
    p = Problem.from_numpy(prob, dtype=dtype)
    s = solver.solve(p)
    g_u = torch.as_tensor(gu, dtype=dtype, device="cuda")
    g_x = None if gx is None else torch.as_tensor(gx, dtype=dtype, device="cuda")
    dC, dc, dx0 = solver.backward_general(p, s, g_u, g_x)
    torch.cuda.synchronize()
    out = dict(u=s.u, x=s.x, cost=s.cost, iters=s.iters, status=s.status, dC=dC, dc=dc, dx0=dx0)
    res = {k: v.detach().cpu().numpy() for k, v in out.items()}
    solver.close()
    return res


def oracle_general(prob, idx, max_iter, tol, gu, gx=None):
    out = []
    N = prob["x_ref"].shape[1]
    for i in idx:
        pr = ilqr.problem_from_batch(prob, i)
        so = ilqr.solve(QUAD, pr, max_iter, tol)
        gr = adjoint.adjoint(pr, so, np.zeros((N, 13)) if gx is None else gx[i], gu[i])
        out.append((pr, so, gr))
    return out


def rel(a, b, floor):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), floor))


def _grads(B, N, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(B, N, 4)), rng.normal(size=(B, N, 13)) * 0.1


@pytest.mark.parametrize("NC,Nc,cfg,tpi", [(1, 10, "hover", 4), (10, 1, "hover", 4), (10, 10, "track", 4),
                                            (1, 10, "track", 8)])
def test_fp64_general_cost_identical_to_oracle(NC, Nc, cfg, tpi):
    """Same kernels in double, three iterations with tol = 0 (every decision
    clear-cut): controls, cost and dL/dC, dL/dc, dL/dx0 agree to rounding,
    with C shared or per stage and c shared or per stage."""
    B, N = 8, 10
    prob = general_problem(B, N, 3, NC, Nc, cfg)
    gu, gx = _grads(B, N, 5)
    g = run_general(prob, torch.float64, 3, 0.0, gu, gx, tpi=tpi)
    orc = oracle_general(prob, range(B), 3, 0.0, gu, gx)
    compared = 0
    for i, (pr, so, gr) in enumerate(orc):
        if so.ls_margin < TIE64:
            continue
        compared += 1
        assert g["status"][i] == so.status and g["iters"][i] == so.iters, i
        assert rel(g["u"][i], so.U, 1e-6) < 1e-8, i
        assert abs(g["cost"][i] - ilqr.total_cost(pr, so.X, so.U)) <= 1e-10 * max(1.0, abs(g["cost"][i])), i
        for name, a, b_ in (("dC", g["dC"][i], gr.dC), ("dc", g["dc"][i], gr.dc), ("dx0", g["dx0"][i], gr.dx0)):
            assert rel(a, b_, 1e-9) < 1e-7, (i, name, rel(a, b_, 1e-9))
    assert compared >= B - 1
    # dL/dC is symmetric, as the oracle's
    assert np.allclose(g["dC"], np.swapaxes(g["dC"], -1, -2), rtol=0, atol=0)


@pytest.mark.parametrize("cfg", ["hover", "track"])
def test_fp32_general_cost_matches_oracle(cfg):
    """The product path: FP32 against the FP64 oracle on converged instances,
    controls within 1e-4 and each gradient block within 1e-3 (relative), and
    the cost within 1e-5 of the size of its terms, sum_t |1/2 z'C z| + |c'z|.
    The general cost is not centred: with c_t = -C z_ref it equals
    1/2 (z - z_ref)' C (z - z_ref) - 1/2 z_ref' C z_ref, and on hover
    instances the two parts nearly cancel (J = 0.010 against terms of 5.0 on
    instance 25), so an FP32 sum can resolve J only relative to its terms
    (measured: <= 1e-7 of them).  The plain relative error is reported."""
    B, N = 32, 20
    prob = general_problem(B, N, 7, 1, N, cfg)
    gu, _ = _grads(B, N, 8)
    g = run_general(prob, torch.float32, 30, 1e-6, gu, tpi=8 if cfg == "track" else 4)
    orc = oracle_general(prob, range(B), 30, 1e-6, gu)
    compared, bad, worst = 0, [], {}
    for i, (pr, so, gr) in enumerate(orc):
        if so.status != ilqr.CONVERGED or g["status"][i] not in (0, 1):
            continue
        compared += 1
        J = ilqr.total_cost(pr, so.X, so.U)
        zs = [np.concatenate([so.X[t], so.U[t]]) for t in range(pr.n)]
        scale = sum(abs(0.5 * z @ pr.Ct(t) @ z) + abs(pr.ct(t) @ z) for t, z in enumerate(zs))
        errs = dict(u=rel(g["u"][i], so.U, 1e-6), J=abs(g["cost"][i] - J) / max(abs(J), 1e-12),
                    J_terms=abs(g["cost"][i] - J) / max(scale, 1e-12),
                    dC=rel(g["dC"][i], gr.dC, 1e-9), dc=rel(g["dc"][i], gr.dc, 1e-9), dx0=rel(g["dx0"][i], gr.dx0, 1e-9))
        for k_, v in errs.items():
            worst[k_] = max(worst.get(k_, 0.0), v)
        if errs["u"] > 1e-4 or errs["J_terms"] > 1e-5 or max(errs["dC"], errs["dc"], errs["dx0"]) > 1e-3:
            bad.append((i, errs))
    print(cfg, "compared", compared, "worst", worst, "bad", bad[:3])
    assert compared >= 0.75 * B
    assert not bad, bad[:3]


def test_diagonal_C_through_the_general_path_matches_the_diagonal_path():
    """C_t = diag(Q_t, R), c_t = [-Q_t x_ref_t; -R u_ref] given explicitly: the
    same controls as the diagonal form, a cost lower by the dropped constant,
    and dL/dQ_i = dL/dC_ii - sum_t x_ref,t,i dL/dc_t,i.  FP64 to convergence:
    the two forms round the cost gradient differently, so the last step (below
    tol) may differ, as between any two converged FP64 runs."""
    from gpu_support import run_gpu
    B, N = 6, 10
    b = W.hover_targets(B, N, seed=9)
    C = np.zeros((B, 1, 17, 17))
    c = np.zeros((B, N, 17))
    for i in range(B):
        C[i, 0] = np.diag(np.concatenate([b["Q"][i, 0], b["R"][i]]))
        for t in range(N):
            c[i, t] = np.concatenate([-b["Q"][i, 0] * b["x_ref"][i, t], -b["R"][i] * b["u_ref"][i]])
    gu, _ = _grads(B, N, 10)
    d = run_gpu(b, torch.float64, 10, 1e-9, gu)
    g = run_general(dict(b, C=C, c=c), torch.float64, 10, 1e-9, gu)
    np.testing.assert_allclose(g["u"], d["u"], rtol=0, atol=1e-8)
    const = 0.5 * (np.einsum("bi,bti,bti->b", b["Q"][:, 0], b["x_ref"], b["x_ref"]) +
                   N * np.einsum("bi,bi,bi->b", b["R"], b["u_ref"], b["u_ref"]))
    np.testing.assert_allclose(g["cost"] + const, d["cost"], rtol=J_TOL64C, atol=1e-12)
    dQ = np.diagonal(g["dC"][:, 0], axis1=-2, axis2=-1)[:, :13] - np.einsum("bti,bti->bi", b["x_ref"], g["dc"][:, :, :13])
    for a, b_ in ((dQ, d["dQ"][:, 0]), (g["dx0"], d["dx0"])):
        for i in range(B):
            assert rel(a[i], b_[i], 1e-9) < G_TOL64C, i


@pytest.mark.parametrize("NC,Nc", [(1, 1), (1, "N"), ("N", 1), ("N", "N")])
@pytest.mark.parametrize("exec_mode", ["persistent", "plain"])
def test_general_cost_uneven_horizons_both_launch_forms(NC, Nc, exec_mode):
    """Per-instance horizons with the general cost, C and c each shared or per
    stage, in the persistent form (longest-horizon-first work queue) and the
    plain form: FP64, three iterations with tol = 0, against the oracle to
    rounding -- controls, cost, dL/dC, dL/dc, dL/dx0 -- and exact zeros in
    every output and per-stage gradient past each instance's horizon."""
    B, N = 12, 10
    NC = N if NC == "N" else NC
    Nc = N if Nc == "N" else Nc
    prob = general_problem(B, N, 17, NC, Nc, "track")
    prob["horizon"] = W.uneven_horizons(B, 1, N, 18)
    gu, gx = _grads(B, N, 19)
    g = run_general(prob, torch.float64, 3, 0.0, gu, gx, exec_mode=exec_mode, tpi=4, ipb=5)
    orc = oracle_general(prob, range(B), 3, 0.0, gu, gx)
    compared = 0
    for i, (pr, so, gr) in enumerate(orc):
        n = pr.n
        assert not g["u"][i, n:].any() and not g["x"][i, n:].any(), i
        if NC > 1:
            assert not g["dC"][i, n:].any(), i
        if Nc > 1:
            assert not g["dc"][i, n:].any(), i
        if so.ls_margin < TIE64:
            continue
        compared += 1
        assert g["status"][i] == so.status and g["iters"][i] == so.iters, i
        # same decisions; FP64 rounding in another arithmetic order, amplified by the
        # conditioning of short-horizon instances with cross terms, reaches ~2e-8 here
        assert rel(g["u"][i], so.U, 1e-6) < 1e-7, (i, rel(g["u"][i], so.U, 1e-6))
        assert abs(g["cost"][i] - ilqr.total_cost(pr, so.X, so.U)) <= 1e-10 * max(1.0, abs(g["cost"][i])), i
        for name, a, b_ in (("dC", g["dC"][i], gr.dC), ("dc", g["dc"][i], gr.dc), ("dx0", g["dx0"][i], gr.dx0)):
            assert rel(a, b_, 1e-9) < 1e-6, (i, name, rel(a, b_, 1e-9))
    assert compared >= B - 1


def test_general_plain_form_is_bit_identical_to_persistent():
    """FP32, uneven horizons, per-stage C and c: the plain form (one launch
    per phase) gives the persistent form's bits."""
    B, N = 40, 12
    prob = general_problem(B, N, 23, N, N, "track")
    prob["horizon"] = W.uneven_horizons(B, 1, N, 24)
    gu, gx = _grads(B, N, 25)
    a = run_general(prob, torch.float32, 8, 1e-6, gu, gx, exec_mode="persistent", tpi=4, ipb=8)
    b = run_general(prob, torch.float32, 8, 1e-6, gu, gx, exec_mode="plain", tpi=4, ipb=5)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_general_recompute_backward_is_bit_identical_to_store_all():
    B, N = 40, 12
    prob = general_problem(B, N, 11, N, N, "track")
    gu, gx = _grads(B, N, 12)
    a = run_general(prob, torch.float32, 8, 1e-6, gu, gx, store_mode="store_all")
    r = run_general(prob, torch.float32, 8, 1e-6, gu, gx, store_mode="recompute")
    for k in ("u", "dC", "dc", "dx0"):
        assert np.array_equal(a[k], r[k]), k


def test_general_cost_api_errors():
    """Validation of the general-cost fields: c is required with C, NC and Nc
    must be 1 or N, each backward entry point refuses the other cost form, and
    the allocation-free forward takes only the diagonal form."""
    from paper_2605_29155_gb300 import DiffMPC, Problem, camp
    B, N = 4, 10
    prob = general_problem(B, N, 13, 1, N)
    p = Problem.from_numpy(prob)
    s = DiffMPC(N_max=N, B_max=B)
    sol = s.alloc_solution(B, N)
    st = torch.cuda.current_stream().cuda_stream
    cs = s._csolution(sol)
    cp = s._cproblem(p)
    cp.c = None
    assert camp.mpc_solve_fwd(s.h, cp, cs, st) == camp.MPC_ERR_ARG
    cp = s._cproblem(p)
    cp.NC = 3
    assert camp.mpc_solve_fwd(s.h, cp, cs, st) == camp.MPC_ERR_SHAPE
    cp = s._cproblem(p)
    cp.Nc = 0
    assert camp.mpc_solve_fwd(s.h, cp, cs, st) == camp.MPC_ERR_SHAPE
    # Q and x_ref are not needed with a general cost
    cp = s._cproblem(p)
    cp.Q = None
    cp.x_ref = None
    assert camp.mpc_solve_fwd(s.h, cp, cs, st) == camp.MPC_OK
    g = torch.zeros(B, N, 4, device="cuda")
    dC, dc, dx0 = torch.empty_like(p.C), torch.empty_like(p.c), torch.empty_like(p.x0)
    dQ, dxr = torch.empty_like(p.Q), torch.empty_like(p.x_ref)
    assert camp.mpc_solve_bwd(s.h, s._cproblem(p), cs, g.data_ptr(), 0, dQ.data_ptr(), dxr.data_ptr(),
                              dx0.data_ptr(), st) == camp.MPC_ERR_STATE
    pd = Problem.from_numpy({k: v for k, v in prob.items() if k not in ("C", "c")})
    assert camp.mpc_solve_bwd_general(s.h, s._cproblem(pd), cs, g.data_ptr(), 0, dC.data_ptr(), dc.data_ptr(),
                                      dx0.data_ptr(), st) == camp.MPC_ERR_STATE
    assert camp.mpc_solve_fwd_noalloc(s.cfg, s._cproblem(p), cs, st) == camp.MPC_ERR_ARG
    torch.cuda.synchronize()
    s.close()
