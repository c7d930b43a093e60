"""mpc_solve_fwd_noalloc: the forward solve for callers that cannot allocate
device memory while running (its scratch is a fixed device array inside the
library).  Checked through the C ABI against mpc_solve_fwd on two calls in a
row, the second on a different problem shape, so that state the shared array
keeps from the first call cannot leak into the second."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U_TOL32, J_TOL32 = 1e-4, 1e-5     # the FP32 tolerances of the parity tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_29155_gb300 import camp
    return camp


def _solve_both(lib, prob, max_iter=8):
    from paper_2605_29155_gb300 import DiffMPC, Problem
    B, N = prob["x0"].shape[0], prob["x_ref"].shape[1]
    ref = DiffMPC(N_max=N, B_max=B, max_iter=max_iter, tol=1e-6)
    p = Problem.from_numpy(prob)
    s_ref = ref.solve(p)
    cfg = lib.mpc_config_default()
    cfg.max_iter, cfg.tol = max_iter, 1e-6
    s_na = ref.alloc_solution(B, N)
    for t in (s_na.u, s_na.x, s_na.cost, s_na.tape):
        t.fill_(float("nan"))
    code = lib.mpc_solve_fwd_noalloc(cfg, ref._cproblem(p), ref._csolution(s_na),
                                     torch.cuda.current_stream().cuda_stream)
    assert code == lib.MPC_OK, lib.mpc_strerror(code)
    torch.cuda.synchronize()
    out = {k: (getattr(s_ref, k).cpu().numpy(), getattr(s_na, k).cpu().numpy())
           for k in ("u", "x", "cost", "iters", "status", "tape")}
    hz = prob.get("horizon")
    out["n"] = np.full(B, N) if hz is None else np.clip(hz, 1, N)
    out["shape"] = (B, N)
    ref.close()
    return out


def _check(out):
    u_ref, u_na = out["u"]
    err = np.linalg.norm(u_na - u_ref, axis=(1, 2)) / np.maximum(np.linalg.norm(u_ref, axis=(1, 2)), 1e-6)
    assert err.max() <= U_TOL32
    c_ref, c_na = out["cost"]
    assert np.max(np.abs(c_na - c_ref) / np.maximum(np.abs(c_ref), 1e-12)) <= J_TOL32
    np.testing.assert_array_equal(out["status"][0], out["status"][1])
    np.testing.assert_array_equal(out["iters"][0], out["iters"][1])
    x_ref, x_na = out["x"]
    assert np.isfinite(x_na).all()
    assert np.max(np.abs(x_na - x_ref)) <= U_TOL32 * max(1.0, np.abs(x_ref).max())
    # the tape holds one record per stage inside each instance's horizon
    B, N = out["shape"]
    G = (B + 31) // 32
    t_ref, t_na = (t[: G * N * 210 * 32].reshape(G, N, 210, 32).transpose(0, 3, 1, 2).reshape(G * 32, N, 210)[:B]
                   for t in out["tape"])
    for i in range(B):
        n = out["n"][i]
        assert np.isfinite(t_na[i, :n]).all()
        assert np.max(np.abs(t_na[i, :n] - t_ref[i, :n])) <= 1e-3 * max(1.0, np.abs(t_ref[i, :n]).max())


def test_noalloc_matches_handle_solve_twice_in_a_row(lib):
    first = W.race_track(200, 20, seed=21)
    _check(_solve_both(lib, first))
    second = W.race_track(64, 40, seed=22, horizons=W.uneven_horizons(64, 5, 40, 23), u_hi_spread=0.2)
    _check(_solve_both(lib, second, max_iter=12))


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    cfg = lib.mpc_config_default()
    big = lib.mpc_problem(B=lib.MPC_NOALLOC_B_MAX + 1, N=20, Nq=1)
    assert lib.mpc_solve_fwd_noalloc(cfg, big, lib.mpc_solution(), 0) == lib.MPC_ERR_SHAPE
    long_ = lib.mpc_problem(B=8, N=lib.MPC_NOALLOC_N_MAX + 1, Nq=1)
    assert lib.mpc_solve_fwd_noalloc(cfg, long_, lib.mpc_solution(), 0) == lib.MPC_ERR_SHAPE
    cfg.dtype = lib.MPC_F64
    assert lib.mpc_solve_fwd_noalloc(cfg, lib.mpc_problem(B=8, N=20, Nq=1), lib.mpc_solution(), 0) == lib.MPC_ERR_ARG
