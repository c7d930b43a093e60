"""mpc_solve_fwd_noalloc: the forward solve for callers that cannot allocate
device memory while running (its scratch is a fixed device array inside the
library).  Checked through the C ABI against mpc_solve_fwd on two calls in a
row, the second on a different problem shape, so that state the shared array
keeps from the first call cannot leak into the second."""
import os
import subprocess
import sys

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


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import workloads as W
from paper_2605_29155_gb300 import camp
prob = W.hover_targets(16, 10, seed=31)
B, N = 16, 10
dev = torch.device("cuda", 0)
torch.cuda.set_device(dev)
t = {k: torch.as_tensor(prob[k], dtype=torch.float32, device=dev).contiguous()
     for k in ("x0", "Q", "x_ref", "R", "u_ref", "u_lo", "u_hi")}
out = dict(u=torch.full((B, N, 4), float("nan"), device=dev), x=torch.full((B, N, 13), float("nan"), device=dev),
           cost=torch.full((B,), float("nan"), device=dev), iters=torch.zeros(B, dtype=torch.int32, device=dev),
           status=torch.full((B,), -7, dtype=torch.int32, device=dev),
           tape=torch.empty((B + 31) // 32 * 32 * N * 210, device=dev))
cfg = camp.mpc_config_default()
cfg.max_iter, cfg.tol = 20, 1e-6
cp = camp.mpc_problem(B=B, N=N, x0=t["x0"].data_ptr(), Q=t["Q"].data_ptr(), Nq=t["Q"].shape[1],
                      x_ref=t["x_ref"].data_ptr(), R=t["R"].data_ptr(), u_ref=t["u_ref"].data_ptr(),
                      u_lo=t["u_lo"].data_ptr(), u_hi=t["u_hi"].data_ptr())
cs = camp.mpc_solution(u=out["u"].data_ptr(), x=out["x"].data_ptr(), cost=out["cost"].data_ptr(),
                       iters=out["iters"].data_ptr(), status=out["status"].data_ptr(), tape=out["tape"].data_ptr(),
                       tape_bytes=out["tape"].numel() * 4)
code = camp.mpc_solve_fwd_noalloc(cfg, cp, cs, torch.cuda.current_stream().cuda_stream)
assert code == camp.MPC_OK, camp.mpc_strerror(code)
torch.cuda.synchronize()
res = {k + "_na": v.cpu().numpy() for k, v in out.items() if k != "tape"}
# a handle solve on the same inputs, only after the allocation-free call
from paper_2605_29155_gb300 import DiffMPC, Problem
ref = DiffMPC(N_max=N, B_max=B, max_iter=20, tol=1e-6)
s = ref.solve(Problem.from_numpy(prob))
torch.cuda.synchronize()
res.update({k + "_h": getattr(s, k).cpu().numpy() for k in ("u", "x", "cost", "iters", "status")})
ref.close()
np.savez(sys.argv[2], **res)
"""


def test_noalloc_in_a_fresh_process_without_any_handle(lib, tmp_path):
    """The entry point's own use: a process that never creates a handle (so
    nothing but this call prepares the kernels) solves a hover batch; its
    result is checked against the FP64 oracle and against a handle solve made
    afterwards in the same process."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = tmp_path / "fresh.npz"
    r = subprocess.run([sys.executable, "-c", _FRESH, root, str(out)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    d = np.load(out)
    np.testing.assert_array_equal(d["status_na"], d["status_h"])
    np.testing.assert_array_equal(d["iters_na"], d["iters_h"])
    for k in ("u", "x", "cost"):
        a, b = d[k + "_na"], d[k + "_h"]
        assert np.isfinite(a).all()
        assert np.max(np.abs(a - b)) <= U_TOL32 * max(1.0, np.abs(b).max()), k
    from gpu_support import oracle_solve
    prob = W.hover_targets(16, 10, seed=31)
    orc = oracle_solve(prob, range(16), 20, 1e-6)
    compared = 0
    for i, (_, so, _) in enumerate(orc):
        if so.status != 0:
            continue
        compared += 1
        err = np.linalg.norm(d["u_na"][i] - so.U) / max(np.linalg.norm(so.U), 1e-6)
        assert err <= U_TOL32, (i, err)
        assert abs(float(d["cost_na"][i]) - so.J) <= J_TOL32 * max(abs(so.J), 1e-12), i
    assert compared >= 12
