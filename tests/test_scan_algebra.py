"""The algebra of the stage-parallel Riccati form (the associative-scan LQR of
the related work cited in Sec. II, with the box QP's clamped controls folded
into the elements), restated in FP64 NumPy and pinned against the oracle's
sequential recursion of Sec. IV-2.  CPU only: this checks the method the
scan kernel implements, independently of any GPU.

A stage with free set f and clamped offsets d_c is the element
    A = A_t,  b = B_c d_c - B_f R_f^-1 r_f,  C = B_f R_f^-1 B_f',  eta = -q_t,  J = Q_t
(value function V(x) = 1/2 x'Jx - eta'x; the last stage has A = B = 0), and an
earlier element i combines with a later j through M = (I + C_i J_j)^-1:
    A = A_j M A_i,  b = A_j M (b_i + C_i eta_j) + b_j,  C = A_j M C_i A_j' + C_j,
    eta = A_i' M' (eta_j - J_j b_i) + eta_i,  J = A_i' M' J_j A_i + J_i."""
import numpy as np
import pytest

import workloads as W
from oracle import ilqr
from oracle.model import Quadrotor

QUAD = Quadrotor(W.DEFAULT_MODEL)
NX, NU = 13, 4


def element(F, prob, X, U, t, free, dc):
    n = prob.n
    A = F[t][:, :NX] if t < n - 1 else np.zeros((NX, NX))
    B = F[t][:, NX:] if t < n - 1 else np.zeros((NX, NU))
    q = prob.Qt(t) * (X[t] - prob.x_ref[t])
    r = prob.R * (U[t] - prob.u_ref)
    f = np.asarray(free, bool)
    Bf, Bc = B[:, f], B[:, ~f]
    C = Bf @ np.diag(1.0 / prob.R[f]) @ Bf.T
    b = Bc @ dc[~f] - Bf @ (r[f] / prob.R[f])
    return [A, b, C, -q, np.diag(prob.Qt(t))]


def combine(ei, ej):
    Ai, bi, Ci, ni, Ji = ei
    Aj, bj, Cj, nj, Jj = ej
    M = np.linalg.inv(np.eye(NX) + Ci @ Jj)
    return [Aj @ M @ Ai, Aj @ M @ (bi + Ci @ nj) + bj, Aj @ M @ Ci @ Aj.T + Cj,
            Ai.T @ M.T @ (nj - Jj @ bi) + ni, Ai.T @ M.T @ Jj @ Ai + Ji]


def suffixes_chunked(els, chunks):
    """S_t = e_t (x) ... (x) e_{n-1} in the kernel's grouping: fold each chunk
    from the back, combine the chunk totals, then each stage's partial with the
    suffix of the chunks after it."""
    n = len(els)
    ch = -(-n // chunks)
    bounds = [(w * ch, min(n, w * ch + ch)) for w in range(chunks) if w * ch < n]
    part = [None] * n
    for t0, t1 in bounds:
        acc = els[t1 - 1]
        part[t1 - 1] = acc
        for t in range(t1 - 2, t0 - 1, -1):
            acc = combine(els[t], acc)
            part[t] = acc
    totals = [part[t0] for t0, _ in bounds]
    after = [None] * len(bounds)
    for w in range(len(bounds) - 2, -1, -1):
        after[w] = totals[w + 1] if after[w + 1] is None else combine(totals[w + 1], after[w + 1])
    S = [None] * n
    for w, (t0, t1) in enumerate(bounds):
        for t in range(t0, t1):
            S[t] = part[t] if after[w] is None else combine(part[t], after[w])
    return S


def _rand_element(rng):
    def psd():
        G = rng.normal(size=(NX, 5))
        return G @ G.T * 0.1
    return [np.eye(NX) + 0.1 * rng.normal(size=(NX, NX)), rng.normal(size=NX), psd(), rng.normal(size=NX), psd()]


def test_combine_is_associative():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b, c = (_rand_element(rng) for _ in range(3))
        left = combine(combine(a, b), c)
        right = combine(a, combine(b, c))
        for x, y in zip(left, right):
            assert np.max(np.abs(x - y)) <= 1e-10 * (1 + np.max(np.abs(y)))


@pytest.mark.parametrize("name,N,iters", [("hover", 20, 0), ("hover", 50, 2), ("track", 20, 3)])
@pytest.mark.parametrize("chunks", [1, 8])
def test_suffix_scan_reproduces_the_sequential_gains(name, N, iters, chunks):
    """For the oracle's own free sets and clamped offsets (d_c = k_t on clamped
    controls), V_{t+1}, v_{t+1} from the suffixes give every stage's Q_uu,
    q_u, Q_ux, and from them the oracle's k_t and K_t (FP64, 1e-9)."""
    batch = W.hover_targets(4, N, seed=3) if name == "hover" else W.race_track(4, N, seed=3)
    clamped = 0
    for i in range(4):
        pr = ilqr.problem_from_batch(batch, i)
        if iters:
            so = ilqr.solve(QUAD, pr, iters, 0.0)
            X, U = so.X, so.U
        else:
            U = np.zeros((N, NU))
            U[:pr.n] = np.clip(np.tile(pr.u_ref, (pr.n, 1)), pr.u_lo, pr.u_hi)
            X = np.zeros((N, NX))
            X[:pr.n] = QUAD.rollout(pr.x0, U[:pr.n])
        F = ilqr.linearize(QUAD, pr, X, U)
        bp = ilqr.backward_pass(pr, X, U, F)
        assert bp.ok
        n = pr.n
        els = [element(F, pr, X, U, t, bp.free[t], np.where(bp.free[t], 0.0, bp.k[t])) for t in range(n)]
        S = suffixes_chunked(els, chunks)
        for t in range(n - 1):
            V, v = S[t + 1][4], -S[t + 1][3]
            A, B = F[t][:, :NX], F[t][:, NX:]
            Quu = np.diag(pr.R) + B.T @ V @ B
            qu = pr.R * (U[t] - pr.u_ref) + B.T @ v
            Qux = B.T @ V @ A
            f = np.asarray(bp.free[t], bool)
            clamped += int((~f).sum())
            k = bp.k[t].copy()
            K = np.zeros((NU, NX))
            if f.any():
                k[f] = np.linalg.solve(Quu[np.ix_(f, f)], -(qu[f] + Quu[np.ix_(f, ~f)] @ k[~f]))
                K[f] = -np.linalg.solve(Quu[np.ix_(f, f)], Qux[f])
            sk = 1.0 + np.max(np.abs(bp.k[t]))
            sK = 1.0 + np.max(np.abs(bp.K[t]))
            assert np.max(np.abs(k - bp.k[t])) <= 1e-9 * sk, (i, t)
            assert np.max(np.abs(K - bp.K[t])) <= 1e-9 * sK, (i, t)
    print(name, N, iters, chunks, "clamped controls", clamped)
    assert clamped > 0          # the clamped offsets' part of b is exercised


def test_single_stage_step_in_woodbury_form():
    """A single stage's C = G G' (G = B_f R_f^-1/2) has rank <= 4: e_t (x) (J,
    eta) through S = I + G'J G (4 x 4) equals the general combine."""
    rng = np.random.default_rng(1)
    for _ in range(10):
        A = np.eye(NX) + 0.05 * rng.normal(size=(NX, NX))
        B = rng.normal(size=(NX, NU)) * 0.1
        R = rng.uniform(0.01, 1.0, NU)
        free = rng.random(NU) > 0.3
        G = np.where(free[None, :], B / np.sqrt(R)[None, :], 0.0)
        b = rng.normal(size=NX)
        eta_t, Qd = rng.normal(size=NX), rng.uniform(0.1, 10, NX)
        Gj = rng.normal(size=(NX, NX))
        J = Gj @ Gj.T
        eta = rng.normal(size=NX)
        ei = [A, b, G @ G.T, eta_t, np.diag(Qd)]
        ref = combine(ei, [np.zeros((NX, NX)), np.zeros(NX), np.zeros((NX, NX)), eta, J])
        S = np.eye(NU) + G.T @ J @ G
        JG = J @ G
        Wm = J - JG @ np.linalg.solve(S, JG.T)
        y = eta - J @ b
        z = y - JG @ np.linalg.solve(S, G.T @ y)
        Jn = A.T @ Wm @ A + np.diag(Qd)
        en = A.T @ z + eta_t
        assert np.max(np.abs(Jn - ref[4])) <= 1e-10 * np.max(np.abs(ref[4]))
        assert np.max(np.abs(en - ref[3])) <= 1e-10 * (1 + np.max(np.abs(ref[3])))


def costate_pass(F, pr, X, U, free, k_clamped, Quu, Qux):
    """The scan kernel's costate pass in FP64: with each stage's free set,
    clamped offsets, Q_uu and Q_ux given, the vector part of the sequential
    recursion from the last stage back,
        g = r_t + B_t' v_{t+1},  k_f = -Q_uu,ff^-1 (g_f + Q_uu,fc k_c),
        v_t = q_t + A_t' v_{t+1} + Q_ux' k
    (the value update's K_t'(Q_uu k + g) is zero: Q_uu k + g vanishes on the
    free set, K_t on the clamped one).  Returns every stage's k."""
    n = pr.n
    v = np.zeros(NX)
    ks = [None] * n
    for t in range(n - 1, -1, -1):
        A = F[t][:, :NX] if t < n - 1 else np.zeros((NX, NX))
        B = F[t][:, NX:] if t < n - 1 else np.zeros((NX, NU))
        q = pr.Qt(t) * (X[t] - pr.x_ref[t])
        g = pr.R * (U[t] - pr.u_ref) + B.T @ v
        f = np.asarray(free[t], bool)
        k = np.where(f, 0.0, k_clamped[t])
        if f.any():
            k[f] = -np.linalg.solve(Quu[t][np.ix_(f, f)], g[f] + Quu[t][np.ix_(f, ~f)] @ k[~f])
        v = q + A.T @ v + Qux[t].T @ k
        ks[t] = k
    return ks


@pytest.mark.parametrize("name,N,iters", [("hover", 50, 2), ("track", 20, 3)])
def test_costate_pass_reproduces_the_sequential_feedforward(name, N, iters):
    """Given the oracle's free sets, clamped offsets, Q_uu and Q_ux, the
    costate pass gives the oracle's k_t at every stage (FP64, 1e-9)."""
    batch = W.hover_targets(4, N, seed=5) if name == "hover" else W.race_track(4, N, seed=5)
    clamped = 0
    for i in range(4):
        pr = ilqr.problem_from_batch(batch, i)
        so = ilqr.solve(QUAD, pr, iters, 0.0)
        F = ilqr.linearize(QUAD, pr, so.X, so.U)
        bp = ilqr.backward_pass(pr, so.X, so.U, F)
        assert bp.ok
        ks = costate_pass(F, pr, so.X, so.U, bp.free, bp.k, bp.Quu, bp.Qux)
        scale = 1.0 + max(np.max(np.abs(k)) for k in bp.k)
        for t in range(pr.n):
            assert np.max(np.abs(ks[t] - bp.k[t])) <= 1e-9 * scale, (i, t)
            clamped += int((~np.asarray(bp.free[t], bool)).sum())
    assert clamped > 0 or name == "hover"


def test_costate_pass_is_insensitive_to_the_scan_matrices_at_convergence():
    """Q_uu and Q_ux come from the scan's V and carry its rounding.  At a
    converged iterate they multiply a vanishing k, so relative noise of 1e-5
    on them moves the costate pass's k by at most 1e-8 of the controls' scale,
    and by at least 100 times less than the same noise on the transitions
    A_t, B_t, which carry the costate (the pass keeps the sequential
    recursion's precision where the controls are decided)."""
    batch = W.hover_targets(4, 50, seed=6)
    rng = np.random.default_rng(7)
    for i in range(4):
        pr = ilqr.problem_from_batch(batch, i)
        so = ilqr.solve(QUAD, pr, 20, 1e-9)
        F = ilqr.linearize(QUAD, pr, so.X, so.U)
        bp = ilqr.backward_pass(pr, so.X, so.U, F)
        noisy = lambda M: [m * (1 + 1e-5 * rng.standard_normal(m.shape)) for m in M]
        k0 = costate_pass(F, pr, so.X, so.U, bp.free, bp.k, bp.Quu, bp.Qux)
        k1 = costate_pass(F, pr, so.X, so.U, bp.free, bp.k, noisy(bp.Quu), noisy(bp.Qux))
        # the controls' scale: a 1e-5 error of the costate would move k by
        # about 1e-5 of |Q_uu^-1 B'v|, which is of the order of the controls
        scale = 1.0 + np.max(np.abs(so.U))
        d = max(np.max(np.abs(a - b)) for a, b in zip(k0, k1))
        # the same noise on the transitions, which carry the costate
        Fn = [f * (1 + 1e-5 * rng.standard_normal(f.shape)) for f in F]
        k2 = costate_pass(Fn, pr, so.X, so.U, bp.free, bp.k, bp.Quu, bp.Qux)
        dv = max(np.max(np.abs(a - b)) for a, b in zip(k0, k2))
        print(i, so.status, so.iters, d / scale, dv / scale)
        assert d <= 1e-8 * scale, (i, d)
        assert dv >= 100 * d, (i, d, dv)
