"""The boundary's configuration on the GPU: the launch-shape autotuner, the
automatic choice of launch form, and the automatic choice between storing
the tape and recomputing it."""
import numpy as np
import pytest

from gpu_support import cached_problem, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _solve(solver, prob):
    from paper_2605_29155_gb300 import Problem
    p = Problem.from_numpy(prob)
    s = solver.solve(p)
    torch.cuda.synchronize()
    return {k: getattr(s, k).cpu().numpy() for k in ("u", "x", "cost", "iters", "status")}


def test_autotune_picks_a_valid_shape_and_solves_as_the_pinned_shape():
    """mpc_autotune times the launch shapes on the problem and keeps the
    fastest; a solve at the chosen shape is bit-identical to a solve on a
    handle pinned to that shape."""
    from paper_2605_29155_gb300 import DiffMPC, Problem
    prob = cached_problem("track", 300, 20, 4, True)
    B, N = 300, 20
    tuned = DiffMPC(N_max=N, B_max=B, max_iter=8, tol=1e-6)
    p = Problem.from_numpy(prob)
    ipb = tuned.autotune(p)
    tpi, ipb2, grid = tuned.launch_shape(B, N)
    assert tpi in (4, 8) and 1 <= ipb <= 32 and ipb == ipb2
    assert 1 <= grid <= -(-B // ipb)
    a = _solve(tuned, prob)
    tuned.close()
    pinned = DiffMPC(N_max=N, B_max=B, max_iter=8, tol=1e-6, tpi=tpi, ipb=ipb)
    assert pinned.launch_shape(B, N) == (tpi, ipb, grid)
    b = _solve(pinned, prob)
    pinned.close()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("name,B,N", [("hover", 2, 40), ("track", 8, 20)])
def test_auto_form_keeps_the_faster_form_and_solves_as_it(name, B, N):
    """exec_mode "auto": persistent until autotune has run; autotune times the
    persistent shapes and the stage-parallel form on the problem and keeps the
    faster; a solve then equals one on a handle fixed to that form (and, for
    the persistent form, that shape) bit for bit."""
    from paper_2605_29155_gb300 import DiffMPC, Problem
    prob = cached_problem(name, B, N, 4)
    p = Problem.from_numpy(prob)
    auto = DiffMPC(N_max=N, B_max=B, max_iter=8, tol=1e-6, exec_mode="auto")
    assert auto.exec_form == "persistent"
    auto.autotune(p)
    form = auto.exec_form
    tpi, ipb, _ = auto.launch_shape(B, N)
    print(name, B, N, "auto keeps", form, "tpi", tpi, "ipb", ipb)
    assert form in ("persistent", "scan")
    a = _solve(auto, prob)
    auto.close()
    if form == "scan":
        fixed = DiffMPC(N_max=N, B_max=B, max_iter=8, tol=1e-6, exec_mode="scan", tpi=tpi)
    else:
        fixed = DiffMPC(N_max=N, B_max=B, max_iter=8, tol=1e-6, tpi=tpi, ipb=ipb)
    b = _solve(fixed, prob)
    fixed.close()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_store_auto_stores_within_its_budget_and_recomputes_beyond_it():
    """MPC_STORE_AUTO keeps the tape for a shape whose tape fits the budget
    and recomputes for one whose tape does not; both give the same bits as
    the fixed modes (store-all and recompute are bit-identical)."""
    from paper_2605_29155_gb300 import DiffMPC
    prob = cached_problem("mem", 40, 30, 2)
    B, N = 40, 30
    rng = np.random.default_rng(4)
    gu, gx = rng.normal(size=(B, N, 4)), rng.normal(size=(B, N, 13)) * 0.1
    tape = (B + 31) // 32 * 32 * N * 210 * 4
    ref = run_gpu(prob, torch.float32, 8, 1e-6, gu, gx, store_mode="store_all")
    roomy = DiffMPC(N_max=N, B_max=B, max_iter=8, tol=1e-6, store_mode="auto")
    assert roomy.alloc_solution(B, N).tape is not None and roomy.alloc_solution(B, N).tape.numel() * 4 >= tape
    a = run_gpu(prob, torch.float32, 8, 1e-6, gu, gx, solver=roomy)
    roomy.close()
    tight = DiffMPC(N_max=N, B_max=B, max_iter=8, tol=1e-6, store_mode="auto", tape_budget=tape - 1)
    assert tight.alloc_solution(B, N).tape is None
    assert tight.alloc_solution(B, 10).tape is not None        # a shorter horizon's tape fits
    b = run_gpu(prob, torch.float32, 8, 1e-6, gu, gx, solver=tight)
    tight.close()
    assert "masks" in a and "masks" not in b
    for k in ref:
        np.testing.assert_array_equal(a[k], ref[k], err_msg=k)
        if k != "masks":
            np.testing.assert_array_equal(b[k], ref[k], err_msg=k)
