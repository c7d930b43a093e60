"""The training-step batch (hover targets, B = 1024, N = 20, FP32, <= 8
iterations, tol 1e-6, loss L = w . u_0 with w ~ N(0, 1)): the GPU's dL/dQ,
dL/dx_ref and dL/dx0 from the adjoint solve against central finite
differences (eps = 1e-4) of the FP64 oracle's frozen-linearization LQR (the
Gauss-Newton target, reading R10) at the GPU's returned iterate (reading R8)
on 32 instances drawn with seed 2."""
import numpy as np
import pytest

import workloads as W
from gpu_support import G_TOL32, fd_gradients_pool, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_train_batch_gradients_match_central_differences():
    prob = W.cfg_train()
    B, N = prob["x0"].shape[0], prob["x_ref"].shape[1]
    gu = W.loss_weights_u0(B, N, seed=1)
    gpu = run_gpu(prob, torch.float32, prob["max_iter"], prob["tol"], gu, None, N_max=N, B_max=B)
    idx = np.random.default_rng(2).choice(B, 32, replace=False)
    # every entry of Q (shared over the stages), x_ref and x0: each block's
    # relative error is the norm-wise one of reading R12
    picks = dict(Q=[(0, i) for i in range(13)], x0=[(i,) for i in range(13)],
                 x_ref=[(t, i) for t in range(N) for i in range(13)])
    res = fd_gradients_pool(gpu, prob, idx, gu, picks)
    worst, bad = {}, []
    for i, (fd, diff, ok) in zip(idx, res):
        if not ok:
            bad.append((int(i), "free set", diff[:4]))
            continue
        for name, key in (("Q", "dQ"), ("x_ref", "dx_ref"), ("x0", "dx0")):
            g = np.array([gpu[key][i][tuple(p)] for p in picks[name]])
            e = np.linalg.norm(g - fd[name]) / max(np.linalg.norm(fd[name]), 1e-9)
            worst[name] = max(worst.get(name, 0.0), e)
            if e > G_TOL32:
                bad.append((int(i), name, e))
    print("worst relative error against central differences", worst)
    assert not bad, bad[:5]
