// camp_scan.cu -- the Riccati recursion of Sec. IV-2 in parallel over the
// stages: the associative-scan LQR of the related work cited in Sec. II, made
// to carry the per-stage box QP.  One block serves one instance; the other
// phases of the plain launch form (rollout, line search, output) are the
// k_mpc phases run with one instance per block.
//
// The scan.  With each stage's free set f_t and clamped offsets d_c fixed,
// stage t of the LQR in the deviations (dx, du) -- cost 1/2 dx'Q_t dx + q_t'dx
// + 1/2 du'R du + r_t'du, dynamics dx' = A_t dx + B_t du -- is the element
//   A_e = A_t,  b_e = B_c d_c - B_f R_f^-1 r_f,  C_e = B_f R_f^-1 B_f',
//   eta_e = -q_t,  J_e = Q_t
// (Saerkkae and Garcia-Fernandez's conditional value-function elements, in the
// convention V(x) = 1/2 x'Jx - eta'x; the last stage has A = B = 0).  Elements
// combine associatively, an earlier stage i before a later suffix j, as
//   M  = (I + C_i J_j)^-1
//   A  = A_j M A_i,            b   = A_j M (b_i + C_i eta_j) + b_j,
//   C  = A_j (M C_i) A_j' + C_j,   eta = A_i' M' (eta_j - J_j b_i) + eta_i,
//   J  = A_i' (J_j M) A_i + J_i,
// and the suffix S_t = e_t (x) ... (x) e_{n-1} holds the value function of
// stage t: V_t = J(S_t), v_t = -eta(S_t).  M C_i and J_j M are symmetric
// ((C_i^-1 + J_j)^-1 and (J_j^-1 + C_i)^-1) and are symmetrized, as are C and
// J.  In FP32, composing the elements' transition parts (A, b, C) still costs
// the costate about two digits against the sequential recursion; a costate
// pass (refine_costate) then reruns the recursion's vector part sequentially,
// so that k_t, the step the line search takes, carries the sequential form's
// rounding.
//
// The free sets.  The box QP makes the recursion depend on free-set decisions.
// The scan therefore takes every stage's free set and clamped offsets as a
// guess (the previous iteration's, all free at the first), scans, and solves
// every stage's box QP from the scanned V_{t+1}, v_{t+1} in parallel.  Let c be
// the latest stage whose free set or clamped offsets differ from the guess.
// Stages after c saw exact values, so their results are final, and stage c's
// QP saw an exact V_{c+1}, so its result is final too.  The stages c-1 .. 0
// then run the sequential recursion on the whole block: each box QP from the
// exact V_{t+1} (on one lane, while the other warps form V A), then V_t, v_t.  When the guess was right
// (c < 0) the whole recursion took one scan; at worst it took a scan plus the
// sequential recursion.  Either way every stage's QP is the one the
// sequential recursion solves (same V_{t+1} up to rounding), so k_t, K_t and
// the free sets are the sequential method's.  A non-positive pivot at a final
// stage ends the solve as in the sequential recursion (status NONPD).  The
// final factorization at the returned iterate (the tape the backward replays)
// runs the sequential recursion for every stage: the gradients then carry the
// sequential form's FP32 rounding.
//
// The scan on SW warps: chunk w holds ch = ceil(n / SW) consecutive stages.
// (A) Each warp folds its chunk into one element from the back, (B) the
// chunks' totals are suffix-scanned in log2(SW) levels of general combines,
// and (C) each warp sweeps J and eta back through its chunk from the suffix of
// the chunks after it.  A single stage's C = G G' has rank <= 4, so (A) and
// (C) use the Woodbury form with a 4 x 4 factor instead of a 13 x 13 inverse.
#include "camp_device.cuh"
#include "camp_internal.h"

namespace camp {

constexpr int SW = 8;                  // warps per block
// the stages' box QPs run with one lane per stage on warps 0 and 1
static_assert(MAX_N <= 64, "the stage-parallel Riccati phase takes at most 64 stages");
constexpr int M13 = NX * NX;
// element layout: A (13 x 13), b, C (13 x 13), eta, J (13 x 13)
constexpr int E_A = 0, E_B = M13, E_C = M13 + NX, E_N = 2 * M13 + NX, E_J = 2 * M13 + 2 * NX,
              ELEM = 3 * M13 + 2 * NX;
constexpr int SV = M13 + NX;           // J and eta of a stage's suffix
// Per-stage record of the scan: QP data and results.
//   H (4 x 4), g, q (13), r (4), k, masked factor (NL), free mask, ok,
//   the guessed clamped offsets and free mask, the clamped sides (bit a: at the
//   upper bound) of the last result (the next iteration's guess), diag(Q_t),
//   Q_ux (4 x 13, row-major)
constexpr int G_H = 0, G_G = 16, G_Q = 20, G_R = 33, G_K = 37, G_L = 41, G_M = 55, G_OK = 56, G_DC = 57,
              G_AM = 61, G_SIDE = 62, G_QD = 64, G_QU = 80, GREC = 136;
constexpr int FREC = NX * NZ;          // F_t = [A_t B_t], row-major 13 x 17
constexpr int FSTR = 224;              // F_t's stride: 16-byte aligned records
// A stage's factors for the single-stage steps: A_t, G = B_f R_f^-1/2 (13 x 4),
// b_t, eta_t = -q_t, diag Q_t
constexpr int SF_A = 0, SF_G = M13, SF_B = M13 + 52, SF_E = M13 + 52 + NX, SF_Q = M13 + 52 + 2 * NX,
              SF_SIZE = M13 + 52 + 3 * NX;

// Elements of one position's workspace for horizons up to N.
__host__ __device__ constexpr size_t scan_pos_elems(int N) {
    // F and G first, their records 16-byte aligned; the total a multiple of 4
    return ((size_t)N * (FSTR + GREC + SV + SF_SIZE) + (size_t)2 * SW * ELEM + 3) / 4 * 4;
}
size_t scan_ws_elems(size_t slots, int N) { return slots * scan_pos_elems(N); }

template <typename T> struct ScanWs {
    T *F, *Sv, *G, *SF, *Uc;
};
template <typename T> __device__ __forceinline__ ScanWs<T> scan_ws(T* base, int pos, int N) {
    T* p = base + (size_t)pos * scan_pos_elems(N);
    ScanWs<T> w;
    w.F = p; p += (size_t)N * FSTR;
    w.G = p; p += (size_t)N * GREC;
    w.Sv = p; p += (size_t)N * SV;
    w.SF = p; p += (size_t)N * SF_SIZE;
    w.Uc = p;
    return w;
}

// ------------------------------------------------ warp-level 13 x 13 algebra
// O = X Y (+ Ad), X or Y transposed as TX / TY, row strides ldx, ldy, ldo.
// Lane l computes the entries l + 32 k (k < 6) side by side, so their
// 13-term sums interleave.  O may not alias X or Y.  The caller syncs the warp.
template <bool TX, bool TY, typename T>
__device__ __forceinline__ void wmm(const T* X, int ldx, const T* Y, int ldy, T* O, int ldo, const T* Ad, int lane) {
    constexpr int SL = (M13 + 31) / 32;
    int r[SL], c[SL];
    T s[SL];
#pragma unroll
    for (int k = 0; k < SL; ++k) {
        const int e0 = lane + 32 * k, e = e0 < M13 ? e0 : M13 - 1;
        r[k] = e / NX;
        c[k] = e - NX * r[k];
        s[k] = Ad ? Ad[r[k] * NX + c[k]] : T(0);
    }
#pragma unroll
    for (int kk = 0; kk < NX; ++kk)
#pragma unroll
        for (int k = 0; k < SL; ++k)
            s[k] += (TX ? X[kk * ldx + r[k]] : X[r[k] * ldx + kk]) * (TY ? Y[c[k] * ldy + kk] : Y[kk * ldy + c[k]]);
#pragma unroll
    for (int k = 0; k < SL; ++k)
        if (lane + 32 * k < M13) O[r[k] * ldo + c[k]] = s[k];
}

// O <- (O + O') / 2 (row stride NX).
template <typename T> __device__ __forceinline__ void wsym(T* O, int lane) {
    for (int e = lane; e < M13; e += 32) {
        const int r = e / NX, c = e - NX * r;
        if (r < c) {
            const T m = T(0.5) * (O[r * NX + c] + O[c * NX + r]);
            O[r * NX + c] = m;
            O[c * NX + r] = m;
        }
    }
}

// Gauss-Jordan with partial pivoting on G = [Z | I] (13 x 26, row stride 26):
// leaves Z^-1 in the right half.  Returns false on a zero pivot.  `col` is 13
// entries of scratch.  Lane l owns the entries l + 32 k (k < 11) throughout.
template <typename T> __device__ bool wgj(T* G, T* col, int lane) {
    constexpr int LD = 2 * NX, NE = NX * LD, SL = (NE + 31) / 32;
    int ii[SL], cc[SL];
#pragma unroll
    for (int k = 0; k < SL; ++k) {
        const int e0 = lane + 32 * k, e = e0 < NE ? e0 : NE - 1;
        ii[k] = e / LD;
        cc[k] = e - LD * ii[k];
    }
    bool ok = true;
    for (int p = 0; p < NX; ++p) {
        T v = (lane >= p && lane < NX) ? fabs(G[lane * LD + p]) : T(-1);
        int idx = lane;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const T v2 = __shfl_xor_sync(FULL, v, o);
            const int i2 = __shfl_xor_sync(FULL, idx, o);
            if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
        }
        ok = ok && v > T(0);
        if (idx != p && lane < LD) {
            const T a = G[p * LD + lane];
            G[p * LD + lane] = G[idx * LD + lane];
            G[idx * LD + lane] = a;
        }
        __syncwarp();
        if (lane < NX) col[lane] = G[lane * LD + p];
        __syncwarp();
        const T ip = T(1) / col[p];
        T gp[SL], fi[SL], gv[SL];
#pragma unroll
        for (int k = 0; k < SL; ++k) {
            gp[k] = G[p * LD + cc[k]] * ip;
            fi[k] = col[ii[k]];
            gv[k] = G[ii[k] * LD + cc[k]];
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < SL; ++k)
            if (lane + 32 * k < NE) G[ii[k] * LD + cc[k]] = ii[k] == p ? gp[k] : gv[k] - fi[k] * gp[k];
        __syncwarp();
    }
    return ok;
}

// Work area of one warp (entries): two operand elements, the result, the
// Gauss-Jordan block and four 13 x 13 temporaries, 13 of pivot scratch.
constexpr int WA_I = 0, WA_J = ELEM, WA_O = 2 * ELEM, WA_G = 3 * ELEM, WA_T = 3 * ELEM + 2 * M13,
              WA_COL = WA_T + 4 * M13, WA_SIZE = WA_COL + 16;
// Work area of a sequential stage (inside the warp's area): S_{t+1}'s J and
// eta on entry, S_t's on exit (the place the scan's Riccati steps use too);
// F_t (two buffers of 224); temporaries.
constexpr int SQ_J = WA_J + E_J, SQ_N = WA_J + E_N, SQ_F = WA_I, SQ_P = WA_T, SQ_X = WA_T + M13,
              SQ_U = WA_T + 2 * M13, SQ_K = SQ_U + 64, SQ_H = SQ_U + 128, SQ_V = WA_O;

// out = ei (x) ej (the earlier element first).  full: every part of the
// result; else only J and eta (into out + E_J, out + E_N).  All in this warp's
// shared memory; out may not alias the operands.  Returns false when
// I + C_i J_j is singular.
template <typename T>
__device__ bool wcombine(const T* ei, const T* ej, T* out, T* wa, bool full, int lane) {
    constexpr int LD = 2 * NX;
    T* G = wa + WA_G;
    T* T0 = wa + WA_T;
    T* T1 = T0 + M13;
    T* T2 = T1 + M13;
    T* T3 = T2 + M13;
    // G = [I + C_i J_j | I]
    wmm<false, false>(ei + E_C, NX, ej + E_J, NX, G, LD, (const T*)nullptr, lane);
    __syncwarp();
    for (int e = lane; e < M13; e += 32) {
        const int r = e / NX, c = e - NX * r;
        if (r == c) G[r * LD + c] += T(1);
        G[r * LD + NX + c] = r == c ? T(1) : T(0);
    }
    __syncwarp();
    const bool ok = wgj(G, wa + WA_COL, lane);
    const T* Mi = G + NX;                                   // M = (I + C_i J_j)^-1, row stride LD
    // T0 = sym(J_j M)
    wmm<false, false>(ej + E_J, NX, Mi, LD, T0, NX, (const T*)nullptr, lane);
    __syncwarp();
    wsym(T0, lane);
    // eta: y = eta_j - J_j b_i (T3[0..12]), then z = M' y (T3[16..28])
    if (lane < NX) {
        T s = ej[E_N + lane];
#pragma unroll
        for (int k = 0; k < NX; ++k) s -= ej[E_J + lane * NX + k] * ei[E_B + k];
        T3[lane] = s;
    }
    __syncwarp();
    // T1 = A_i' T0
    wmm<true, false>(ei + E_A, NX, T0, NX, T1, NX, (const T*)nullptr, lane);
    if (lane < NX) {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) s += Mi[k * LD + lane] * T3[k];
        T3[16 + lane] = s;
    }
    __syncwarp();
    // J = sym(T1 A_i) + J_i;  eta = A_i' z + eta_i
    wmm<false, false>(T1, NX, ei + E_A, NX, out + E_J, NX, ei + E_J, lane);
    if (lane < NX) {
        T s = ei[E_N + lane];
#pragma unroll
        for (int k = 0; k < NX; ++k) s += ei[E_A + k * NX + lane] * T3[16 + k];
        out[E_N + lane] = s;
    }
    __syncwarp();
    wsym(out + E_J, lane);
    if (!full) {
        __syncwarp();
        return ok;
    }
    // T0 = A_j M,  T1 = sym(M C_i)
    wmm<false, false>(ej + E_A, NX, Mi, LD, T0, NX, (const T*)nullptr, lane);
    wmm<false, false>(Mi, LD, ei + E_C, NX, T1, NX, (const T*)nullptr, lane);
    // y = b_i + C_i eta_j (T3[0..12])
    if (lane < NX) {
        T s = ei[E_B + lane];
#pragma unroll
        for (int k = 0; k < NX; ++k) s += ei[E_C + lane * NX + k] * ej[E_N + k];
        T3[lane] = s;
    }
    __syncwarp();
    wsym(T1, lane);
    // A = T0 A_i;  b = T0 y + b_j
    wmm<false, false>(T0, NX, ei + E_A, NX, out + E_A, NX, (const T*)nullptr, lane);
    if (lane < NX) {
        T s = ej[E_B + lane];
#pragma unroll
        for (int k = 0; k < NX; ++k) s += T0[lane * NX + k] * T3[k];
        out[E_B + lane] = s;
    }
    __syncwarp();
    // C = sym(A_j T1 A_j') + C_j
    wmm<false, false>(ej + E_A, NX, T1, NX, T2, NX, (const T*)nullptr, lane);
    __syncwarp();
    wmm<false, true>(T2, NX, ej + E_A, NX, out + E_C, NX, ej + E_C, lane);
    __syncwarp();
    wsym(out + E_C, lane);
    __syncwarp();
    return ok;
}

// Copies of ELEM entries (or a part) between global and shared memory by a warp.
template <typename T> __device__ __forceinline__ void wcopy(T* dst, const T* src, int n, int lane) {
    for (int e = lane; e < n; e += 32) dst[e] = src[e];
}

// -------------------------------------------------- scan, QPs and gains ---
// Shared state of a block.
template <typename T> struct ScanShared {
    T R[NU], uref[NU], ulo[NU], uhi[NU];
    int cw[2];          // per QP warp: the latest changed stage
    int fail;
};

// ------------------------------------------- single-stage (rank-4) steps --
// A single stage's element has C_t = G G' with G = B_f R_f^-1/2 (13 x 4, zero
// columns for clamped controls), so combining it in front of a suffix needs
// only the 4 x 4 matrix S = I + G'J G (Woodbury):
//   M = (I + G G'J)^-1 = I - G S^-1 G'J,   J M = J - (J G) S^-1 (J G)',
//   M C_t = G S^-1 G',   M' y = y - J G S^-1 G'y.
// A step reads stage t's factors (the SF_* layout) from a warp's shared memory
// and keeps these temporaries there (ST_SIZE entries):
constexpr int ST_JG = 0, ST_S = 52, ST_Y = 68, ST_Z = 84, ST_W4 = 136, ST_ZV = 144, ST_W = 160, ST_T1 = ST_W + M13,
              ST_AG = ST_T1 + M13, ST_X = ST_AG + 52, ST_AM = ST_X + 52, ST_BN = ST_AM + M13, ST_SIZE = ST_BN + 16;
// the regions of a warp's area the steps use stay inside it
static_assert(WA_O + ST_SIZE <= WA_SIZE, "step temporaries");
static_assert(264 + SF_SIZE <= ELEM, "double-buffered stage factors");
static_assert(FSTR + FREC <= ELEM, "double-buffered F_t of the sequential tail");
static_assert(FSTR >= FREC && FSTR % 4 == 0 && GREC % 4 == 0, "F and G records start on 16 bytes");
static_assert(SQ_H + 20 <= WA_COL, "sequential-stage temporaries");

// Every stage's factors for the guessed free sets and clamped offsets into
// SF (one job per stage and row).
template <typename T> __device__ void stage_factors_all(const ScanWs<T>& W, const ScanShared<T>& sh, int n) {
    for (int job = threadIdx.x; job < n * NX; job += blockDim.x) {
        const int t = job / NX, i = job - NX * t;
        const T* F = W.F + (size_t)t * FSTR + i * NZ;
        const T* G = W.G + (size_t)t * GREC;
        T* sf = W.SF + (size_t)t * SF_SIZE;
        // every load first (one round trip), then the arithmetic
        T f[NZ], r[NU], dc[NU];
#pragma unroll
        for (int k = 0; k < NZ; ++k) f[k] = F[k];
#pragma unroll
        for (int a = 0; a < NU; ++a) { r[a] = G[G_R + a]; dc[a] = G[G_DC + a]; }
        const int fm = (int)G[G_AM];
        const T q = G[G_Q + i], qd = G[G_QD + i];
#pragma unroll
        for (int k = 0; k < NX; ++k) sf[SF_A + i * NX + k] = f[k];
        T bi = T(0);
#pragma unroll
        for (int a = 0; a < NU; ++a) {
            const T Bia = f[NX + a];
            const bool fr = (fm >> a) & 1;
            sf[SF_G + i * NU + a] = fr ? Bia / sqrt(sh.R[a]) : T(0);
            bi += fr ? -(Bia / sh.R[a]) * r[a] : Bia * dc[a];
        }
        sf[SF_B + i] = bi;
        sf[SF_E + i] = -q;
        sf[SF_Q + i] = qd;
    }
}

// Asynchronous copy of n entries by a warp (cp.async; committed as one group).
template <typename T> __device__ __forceinline__ void wprefetch(T* dst, const T* src, int n, int lane) {
    for (int e = lane; e < n; e += 32) cp_async(dst + e, src + e);
    cp_async_commit();
}
__device__ __forceinline__ void wwait() {
    cp_async_wait_all();
    __syncwarp();
}

// The common part of a step in front of the suffix (J, eta): J G, S = I + G'J G
// (factored in every lane), y = eta - J b, Z = S^-1 (J G)', w = S^-1 G'y,
// W = J - (J G) Z, z = y - (J G) w.
template <typename T>
__device__ void lr_common(const T* J, const T* eta, const T* sf, T* tp, int lane, T (&Ls)[NL]) {
    for (int e = lane; e < NX * NU; e += 32) {
        const int i = e / NU, a = e - NU * i;
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) s += J[i * NX + k] * sf[SF_G + k * NU + a];
        tp[ST_JG + e] = s;
    }
    __syncwarp();
    if (lane < 16) {
        const int a = lane >> 2, c = lane & 3;
        T s = a == c ? T(1) : T(0);
#pragma unroll
        for (int i = 0; i < NX; ++i) s += sf[SF_G + i * NU + a] * tp[ST_JG + i * NU + c];
        tp[ST_S + lane] = s;
    } else if (lane < 16 + NX) {
        const int i = lane - 16;
        T s = eta[i];
#pragma unroll
        for (int k = 0; k < NX; ++k) s -= J[i * NX + k] * sf[SF_B + k];
        tp[ST_Y + i] = s;
    }
    __syncwarp();
    T S[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) S[a][c] = tp[ST_S + a * 4 + c];
    chol_masked(S, 15, Ls);                             // S = I + G'JG is positive definite
    if (lane < NX) {
        T rhs[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) rhs[a] = tp[ST_JG + lane * NU + a];
        chol_solve4(Ls, rhs, y);
#pragma unroll
        for (int a = 0; a < 4; ++a) tp[ST_Z + a * NX + lane] = y[a];
    } else if (lane == NX) {
        T rhs[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            T s = T(0);
#pragma unroll
            for (int i = 0; i < NX; ++i) s += sf[SF_G + i * NU + a] * tp[ST_Y + i];
            rhs[a] = s;
        }
        chol_solve4(Ls, rhs, y);
#pragma unroll
        for (int a = 0; a < 4; ++a) tp[ST_W4 + a] = y[a];
    }
    __syncwarp();
    for (int e = lane; e < M13; e += 32) {
        const int i = e / NX, k = e - NX * i;
        T s = J[e];
#pragma unroll
        for (int a = 0; a < NU; ++a) s -= tp[ST_JG + i * NU + a] * tp[ST_Z + a * NX + k];
        tp[ST_W + e] = s;
    }
    if (lane < NX) {
        T s = tp[ST_Y + lane];
#pragma unroll
        for (int a = 0; a < NU; ++a) s -= tp[ST_JG + lane * NU + a] * tp[ST_W4 + a];
        tp[ST_ZV + lane] = s;
    }
    __syncwarp();
}

// J = A'W A + Q_t (symmetrized), eta = A'z + eta_t from lr_common's W, z.
template <typename T> __device__ void lr_half_tail(T* J, T* eta, const T* sf, T* tp, int lane) {
    wmm<false, false>(tp + ST_W, NX, sf + SF_A, NX, tp + ST_T1, NX, (const T*)nullptr, lane);
    __syncwarp();
    wmm<true, false>(sf + SF_A, NX, tp + ST_T1, NX, J, NX, (const T*)nullptr, lane);
    if (lane < NX) {
        T s = sf[SF_E + lane];
#pragma unroll
        for (int k = 0; k < NX; ++k) s += sf[SF_A + k * NX + lane] * tp[ST_ZV + k];
        eta[lane] = s;
    }
    __syncwarp();
    if (lane < NX) J[lane * NX + lane] += sf[SF_Q + lane];
    __syncwarp();
    wsym(J, lane);
    __syncwarp();
}

// (J, eta) <- e_t (x) (J, eta): the Riccati step of stage t for its free set.
template <typename T> __device__ void lr_half(T* J, T* eta, const T* sf, T* tp, int lane) {
    T Ls[NL];
    lr_common(J, eta, sf, tp, lane, Ls);
    lr_half_tail(J, eta, sf, tp, lane);
}

// R <- e_t (x) R for a whole element R (A, b, C, eta, J) in shared memory:
//   A_R M = A_R - (A_R G) Z,  A = (A_R M) A_t,  b = (A_R M)(b_t + G G'eta_R) + b_R,
//   C = (A_R G) S^-1 (A_R G)' + C_R,  J, eta as in lr_half.
template <typename T> __device__ void lr_full(T* Rl, const T* sf, T* tp, int lane) {
    T* RA = Rl + E_A;
    T* Rb = Rl + E_B;
    T* RC = Rl + E_C;
    T Ls[NL];
    lr_common(Rl + E_J, Rl + E_N, sf, tp, lane, Ls);
    // A_R G (13 x 4)
    for (int e = lane; e < NX * NU; e += 32) {
        const int i = e / NU, a = e - NU * i;
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) s += RA[i * NX + k] * sf[SF_G + k * NU + a];
        tp[ST_AG + e] = s;
    }
    // G'eta_R (4) into BN[12..15]
    if (lane >= 16 && lane < 20) {
        const int a = lane - 16;
        T s = T(0);
#pragma unroll
        for (int i = 0; i < NX; ++i) s += sf[SF_G + i * NU + a] * Rl[E_N + i];
        tp[ST_BN + 12 + a] = s;
    }
    __syncwarp();
    // X = S^-1 (A_R G)' (4 x 13);  A_R M
    if (lane < NX) {
        T rhs[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) rhs[a] = tp[ST_AG + lane * NU + a];
        chol_solve4(Ls, rhs, y);
#pragma unroll
        for (int a = 0; a < 4; ++a) tp[ST_X + a * NX + lane] = y[a];
    }
    for (int e = lane; e < M13; e += 32) {
        const int i = e / NX, k = e - NX * i;
        T s = RA[e];
#pragma unroll
        for (int a = 0; a < NU; ++a) s -= tp[ST_AG + i * NU + a] * tp[ST_Z + a * NX + k];
        tp[ST_AM + e] = s;
    }
    __syncwarp();
    // b_t + G G'eta_R into Y (y is no longer needed)
    if (lane < NX) {
        T s = sf[SF_B + lane];
#pragma unroll
        for (int a = 0; a < NU; ++a) s += sf[SF_G + lane * NU + a] * tp[ST_BN + 12 + a];
        tp[ST_Y + lane] = s;
    }
    __syncwarp();
    if (lane < NX) {
        T s = Rb[lane];
#pragma unroll
        for (int k = 0; k < NX; ++k) s += tp[ST_AM + lane * NX + k] * tp[ST_Y + k];
        tp[ST_BN + lane] = s;
    }
    // C = C_R + (A_R G) X
    for (int e = lane; e < M13; e += 32) {
        const int i = e / NX, k = e - NX * i;
        T s = RC[e];
#pragma unroll
        for (int a = 0; a < NU; ++a) s += tp[ST_AG + i * NU + a] * tp[ST_X + a * NX + k];
        RC[e] = s;
    }
    __syncwarp();
    wsym(RC, lane);
    wmm<false, false>(tp + ST_AM, NX, sf + SF_A, NX, RA, NX, (const T*)nullptr, lane);
    if (lane < NX) Rb[lane] = tp[ST_BN + lane];
    __syncwarp();
    lr_half_tail(Rl + E_J, Rl + E_N, sf, tp, lane);
}

// The suffixes S_t of every stage t < n (J and eta into Sv) for the guessed
// free sets.  Barriers inside: every thread of the block calls it.  Sets *bad
// when some I + C J of the chunk-level combines was singular.
template <typename T>
__device__ void scan_suffixes(const ScanWs<T>& W, const ScanShared<T>& sh, T* wa, int n, int* bad) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = (n + SW - 1) / SW;
    const int last = (n - 1) / ch;
    const int t0 = w * ch, t1 = min(n, t0 + ch) - 1;
    T* tp = wa + WA_O;
    bool ok = true;
    // A: each chunk's total e_t0 (x) ... (x) e_t1, folded from the back with
    // the single-stage steps
    if (w <= last) {
        T* Rl = wa + WA_J;
        T* sb[2] = {wa + WA_I, wa + WA_I + 264};     // double-buffered stage factors
        wprefetch(sb[0], W.SF + (size_t)t1 * SF_SIZE, SF_SIZE, lane);
        wwait();
        if (t1 - 1 >= t0) wprefetch(sb[1], W.SF + (size_t)(t1 - 1) * SF_SIZE, SF_SIZE, lane);
        const T* sf = sb[0];
        for (int e = lane; e < M13; e += 32) {
            const int i = e / NX, k = e - NX * i;
            T c = T(0);
#pragma unroll
            for (int a = 0; a < NU; ++a) c += sf[SF_G + i * NU + a] * sf[SF_G + k * NU + a];
            Rl[E_A + e] = sf[SF_A + e];
            Rl[E_C + e] = c;
            Rl[E_J + e] = i == k ? sf[SF_Q + i] : T(0);
        }
        if (lane < NX) {
            Rl[E_B + lane] = sf[SF_B + lane];
            Rl[E_N + lane] = sf[SF_E + lane];
        }
        __syncwarp();
        for (int t = t1 - 1, k = 1; t >= t0; --t, k ^= 1) {
            wwait();
            if (t - 1 >= t0) wprefetch(sb[k ^ 1], W.SF + (size_t)(t - 1) * SF_SIZE, SF_SIZE, lane);
            lr_full(Rl, sb[k], tp, lane);
        }
        wcopy(W.Uc + (size_t)w * ELEM, Rl, ELEM, lane);
    }
    __syncthreads();
    // B: suffix scan of the chunk totals over the chunks (log2 levels; the
    // last level's results are used only for J and eta)
    int cur = 0;
    for (int d = 1; d <= last; d <<= 1) {
        const bool full = 2 * d <= last;
        if (w <= last) {
            T* dst = W.Uc + ((size_t)(cur ^ 1) * SW + w) * ELEM;
            const T* src = W.Uc + ((size_t)cur * SW + w) * ELEM;
            if (w + d <= last) {
                wcopy(wa + WA_I, src, ELEM, lane);
                wcopy(wa + WA_J, W.Uc + ((size_t)cur * SW + w + d) * ELEM, ELEM, lane);
                __syncwarp();
                ok = wcombine(wa + WA_I, wa + WA_J, wa + WA_O, wa, full, lane) && ok;
                wcopy(dst, wa + WA_O, ELEM, lane);
            } else {
                wcopy(dst, src, ELEM, lane);
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    // C: the Riccati steps through each chunk from the suffix of the chunks
    // after it (zero after the last)
    if (w <= last) {
        T* J = wa + SQ_J;
        T* eta = wa + SQ_N;
        const T* U = W.Uc + ((size_t)cur * SW + w + 1) * ELEM;
        for (int e = lane; e < SV; e += 32) {
            const bool e_j = e < M13;
            const T v = w < last ? (e_j ? U[E_J + e] : U[E_N + e - M13]) : T(0);
            if (e_j) J[e] = v;
            else eta[e - M13] = v;
        }
        __syncwarp();
        T* sb[2] = {wa + WA_I, wa + WA_I + 264};
        wprefetch(sb[0], W.SF + (size_t)t1 * SF_SIZE, SF_SIZE, lane);
        for (int t = t1, k = 0; t >= t0; --t, k ^= 1) {
            wwait();
            if (t - 1 >= t0) wprefetch(sb[k ^ 1], W.SF + (size_t)(t - 1) * SF_SIZE, SF_SIZE, lane);
            lr_half(J, eta, sb[k], tp, lane);
            T* sv = W.Sv + (size_t)t * SV;
            wcopy(sv, J, M13, lane);
            wcopy(sv + M13, eta, NX, lane);
        }
    }
    if (!ok && lane == 0) atomicOr(bad, 1);
    __syncthreads();
}

// Column a of stage t's QP data: H[a'][a] = R_a d_a'a + B_a'' V_{t+1} B_a for
// a' <= a, and g_a = r_a + B_a' v_{t+1} (V_n = 0, v_n = 0).
template <typename T>
__device__ __forceinline__ void qp_column(const ScanWs<T>& W, const ScanShared<T>& sh, int t, int a, int n) {
    const T* F = W.F + (size_t)t * FSTR;
    T* G = W.G + (size_t)t * GREC;
    T vb[NX];
    T ga = G[G_R + a];
    if (t + 1 < n) {
        const T* V = W.Sv + (size_t)(t + 1) * SV;
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < NX; ++k) s += V[i * NX + k] * F[k * NZ + NX + a];
            vb[i] = s;
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) ga -= F[i * NZ + NX + a] * V[M13 + i];     // v = -eta
    } else {
#pragma unroll
        for (int i = 0; i < NX; ++i) vb[i] = T(0);
    }
    for (int a2 = 0; a2 <= a; ++a2) {
        T s = a2 == a ? sh.R[a] : T(0);
#pragma unroll
        for (int i = 0; i < NX; ++i) s += F[i * NZ + NX + a2] * vb[i];
        G[G_H + a2 * NU + a] = s;
    }
    G[G_G + a] = ga;
}

// The QP data of every stage t < n (one job per stage and control column).
template <typename T> __device__ void qp_inputs(const ScanWs<T>& W, const ScanShared<T>& sh, int n) {
    for (int job = threadIdx.x; job < n * NU; job += blockDim.x) qp_column(W, sh, job / NU, job % NU, n);
}

// The box QP of stage t for the lanes with `on` (warp-collective): solves from
// H (upper triangle, Hs[a * 4 + c] for a <= c), g and the bounds, writes k,
// the factor, the free mask, ok, the clamped sides and the new guess to the
// stage's record, returns them in d, Lf, mask, and returns whether the free
// set or the clamped offsets differ from the old guess.
template <typename T>
__device__ bool qp_stage(const Params<T>& P, const ScanWs<T>& W, const ScanShared<T>& sh, int pos, int t, bool on,
                         const T* Hs, const T* gs, T (&d)[4], T (&Lf)[NL], int& mask, bool& ok) {
    const int tt = on ? t : 0;
    T* G = W.G + (size_t)tt * GREC;
    const T* sr = P.stg + srow(P, pos, tt, 0);
    T H[4][4], g[4], lo[4], hi[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int c = 0; c < 4; ++c) H[a][c] = on ? (a <= c ? Hs[a * NU + c] : Hs[c * NU + a]) : T(a == c);
        g[a] = on ? gs[a] : T(0);
        const T ub = on ? sr[(R_U + a) * GW] : T(0);
        lo[a] = sh.ulo[a] - ub;
        hi[a] = sh.uhi[a] - ub;
    }
    mask = 0;
    ok = box_qp(on, H, g, lo, hi, d, Lf, mask);
    if (!on) return false;
    const int am = (int)G[G_AM];
    bool changed = mask != am;
    int side = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const bool cl = !((mask >> a) & 1);
        changed = changed || (cl && d[a] != G[G_DC + a]);
        side |= (cl && d[a] == hi[a]) ? (1 << a) : 0;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        G[G_K + a] = d[a];
        G[G_DC + a] = ((mask >> a) & 1) ? T(0) : d[a];
    }
#pragma unroll
    for (int i = 0; i < NL; ++i) G[G_L + i] = Lf[i];
    G[G_M] = (T)mask;
    G[G_AM] = (T)mask;
    G[G_SIDE] = (T)side;
    G[G_OK] = ok ? T(1) : T(0);
    return changed;
}

// The box QPs of every stage t < n on warps 0 and 1 (lane = stage) against
// the guesses; records in sh.cw the latest stage whose result changed.
template <typename T>
__device__ void stage_qps(const Params<T>& P, const ScanWs<T>& W, ScanShared<T>& sh, int pos, int n) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= 2) return;
    int latest = -1;
    if (w * 32 < n) {
        const int t = w * 32 + lane;
        const T* G = W.G + (size_t)(t < n ? t : 0) * GREC;
        T d[4], Lf[NL];
        int mask;
        bool ok;
        latest = qp_stage(P, W, sh, pos, t, t < n, G + G_H, G + G_G, d, Lf, mask, ok) ? t : -1;
    }
    latest = __reduce_max_sync(FULL, latest + 1) - 1;
    if (lane == 0) sh.cw[w] = latest;
}


// One stage of the sequential recursion (Tassa's value update, as the oracle
// and the sequential phase take it), on the whole block (every thread calls
// it; it returns the same value in all):
//   Q_xx = Q_t + A'V A,  Q_ux = B'V A,  Q_uu = R + B'V B,  q = q_t + A'v,
//   q_u = r_t + B'v  (V, v of stage t+1, in shared memory),
//   the box QP (unless `have_qp`: the stored result is final),
//   K = -Q_uu,ff^-1 Q_ux,f (zero rows for clamped controls),
//   V_t = Q_xx + Q_ux'K (symmetrized),  v_t = q + K'(Q_uu k + q_u) + Q_ux'k,
// V_t and eta_t = -v_t into shared memory and Sv[t].  The box QP runs on one
// lane of warp 0 while the other warps form V A; the products are spread over
// the block's threads, one output each, in the order of the warp-level
// products (the same rounding).  Returns false on a non-positive pivot.
template <typename T>
__device__ bool seq_stage(const Params<T>& P, const ScanWs<T>& W, const ScanShared<T>& sh, T* wa, int pos, int t,
                          int n, bool have_qp, int tid, T* Fs, int* s_ok) {
    T* Js = wa + SQ_J;
    T* es = wa + SQ_N;
    T* P1 = wa + SQ_P;
    T* Qx = wa + SQ_X;
    T* Qu = wa + SQ_U;
    T* Kt = wa + SQ_K;
    T* Hg = wa + SQ_H;                  // H (16, upper used), g (4)
    T* G = W.G + (size_t)t * GREC;
    const int warp = tid >> 5, lane = tid & 31;
    if (!have_qp) {
        // V B into P1 (13 x 4), then H and g
        if (tid < NX * NU) {
            const int i = tid / NU, a = tid - NU * i;
            T s = T(0);
#pragma unroll
            for (int k = 0; k < NX; ++k) s += Js[i * NX + k] * Fs[k * NZ + NX + a];
            P1[tid] = s;
        }
        __syncthreads();
        if (tid < 16) {
            const int a2 = tid >> 2, a = tid & 3;
            T s = a2 == a ? sh.R[a] : T(0);
#pragma unroll
            for (int i = 0; i < NX; ++i) s += Fs[i * NZ + NX + a2] * P1[i * NU + a];
            Hg[tid] = s;
        } else if (tid < 20) {
            const int a = tid - 16;
            T s = G[G_R + a];
#pragma unroll
            for (int i = 0; i < NX; ++i) s -= Fs[i * NZ + NX + a] * es[i];
            Hg[tid] = s;
        }
        __syncthreads();
    }
    // warp 0: the box QP (or its stored result); lanes 0..12 keep d and the
    // factor for K_t and v_t
    T d[4], Lf[NL];
    int mask = 0;
    if (warp == 0) {
        bool ok;
        if (have_qp) {
            if (lane < 16) Hg[lane] = G[G_H + lane];
            else if (lane < 20) Hg[lane] = G[G_G + lane - 16];
#pragma unroll
            for (int a = 0; a < 4; ++a) d[a] = G[G_K + a];
#pragma unroll
            for (int i = 0; i < NL; ++i) Lf[i] = G[G_L + i];
            mask = (int)G[G_M];
            ok = G[G_OK] != T(0);
        } else {
            qp_stage(P, W, sh, pos, t, lane == 0, Hg, Hg + 16, d, Lf, mask, ok);
            if (lane < 20) G[lane < 16 ? G_H + lane : G_G + lane - 16] = Hg[lane];     // for the costate pass
            mask = __shfl_sync(FULL, mask, 0);
            ok = __shfl_sync(FULL, ok ? 1 : 0, 0) != 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) d[a] = __shfl_sync(FULL, d[a], 0);
#pragma unroll
            for (int i = 0; i < NL; ++i) Lf[i] = __shfl_sync(FULL, Lf[i], 0);
        }
        if (lane == 0) *s_ok = ok ? 1 : 0;
    } else if (tid - 32 < M13) {
        // P1 = V A
        const int e = tid - 32, r = e / NX, c = e - NX * r;
        T s = T(0);
#pragma unroll
        for (int kk = 0; kk < NX; ++kk) s += Js[r * NX + kk] * Fs[kk * NZ + c];
        P1[e] = s;
    }
    __syncthreads();
    // Qx = A' P1 (13 x 13), Qu = B' P1 (4 x 13)
    if (tid < M13) {
        const int r = tid / NX, c = tid - NX * r;
        T s = T(0);
#pragma unroll
        for (int kk = 0; kk < NX; ++kk) s += Fs[kk * NZ + r] * P1[kk * NX + c];
        Qx[tid] = s;
    } else if (tid < M13 + NU * NX) {
        const int e = tid - M13, a = e / NX, c = e - NX * a;
        T s = T(0);
#pragma unroll
        for (int i = 0; i < NX; ++i) s += Fs[i * NZ + NX + a] * P1[i * NX + c];
        Qu[e] = s;
    }
    __syncthreads();
    // column `tid` of K_t, and v_t's entry `tid` (lanes 0..12 of warp 0)
    T vt = T(0);
    if (tid < NX) {
        Qx[tid * NX + tid] += G[G_QD + tid];
        T rhs[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) rhs[a] = ((mask >> a) & 1) ? Qu[a * NX + tid] : T(0);
        chol_solve4(Lf, rhs, y);
        T kc[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            kc[a] = ((mask >> a) & 1) ? -y[a] : T(0);
            Kt[a * NX + tid] = kc[a];
        }
        T w[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            T s = Hg[16 + a];
#pragma unroll
            for (int c = 0; c < 4; ++c) s += (a <= c ? Hg[a * NU + c] : Hg[c * NU + a]) * d[c];
            w[a] = s;
        }
        T s = G[G_Q + tid];
#pragma unroll
        for (int k = 0; k < NX; ++k) s -= Fs[k * NZ + tid] * es[k];
#pragma unroll
        for (int a = 0; a < NU; ++a) s += kc[a] * w[a] + Qu[a * NX + tid] * d[a];
        vt = s;
    }
    __syncthreads();
    // V_t = Qx + Qu'K, symmetrized (the mean of the two computed entries), in
    // place of V_{t+1} and into Sv[t]; eta_t = -v_t
    T* so = W.Sv + (size_t)t * SV;
    if (tid < M13) {
        const int r = tid / NX, c = tid - NX * r;
        if (r <= c) {
            T s1 = Qx[tid], s2 = Qx[c * NX + r];
#pragma unroll
            for (int a = 0; a < NU; ++a) {
                s1 += Qu[a * NX + r] * Kt[a * NX + c];
                s2 += Qu[a * NX + c] * Kt[a * NX + r];
            }
            const T m = r == c ? s1 : T(0.5) * (s1 + s2);
            Js[r * NX + c] = m;
            Js[c * NX + r] = m;
            so[r * NX + c] = m;
            so[c * NX + r] = m;
        }
    }
    if (tid < NX) {
        es[tid] = -vt;
        so[M13 + tid] = -vt;
    }
    __syncthreads();
    return *s_ok != 0;
}

// K_t = -Q_uu,ff^-1 Q_ux,f (zero rows for clamped controls), Q_ux = B_t'
// V_{t+1} A_t, and k_t into the stage records (one job per stage and state
// column).
template <typename T>
__device__ void write_gains(const Params<T>& P, const ScanWs<T>& W, int pos, int n, int b, bool tape) {
    for (int job = threadIdx.x; job < n * NX; job += blockDim.x) {
        const int t = job / NX, c = job - NX * t;
        const T* F = W.F + (size_t)t * FSTR;
        const T* G = W.G + (size_t)t * GREC;
        T* grow = P.stg + srow(P, pos, t, 0);
        T qc[NU] = {T(0), T(0), T(0), T(0)};
        if (t + 1 < n) {
            const T* V = W.Sv + (size_t)(t + 1) * SV;
            T va[NX];
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                T s = T(0);
#pragma unroll
                for (int k = 0; k < NX; ++k) s += V[i * NX + k] * F[k * NZ + c];
                va[i] = s;
            }
#pragma unroll
            for (int a = 0; a < NU; ++a) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < NX; ++i) s += F[i * NZ + NX + a] * va[i];
                qc[a] = s;
            }
        }
        if (!tape) {
#pragma unroll
            for (int a = 0; a < NU; ++a) W.G[(size_t)t * GREC + G_QU + a * NX + c] = qc[a];
        }
        const int mask = (int)G[G_M];
        T Lf[NL], rhs[4], y[4];
#pragma unroll
        for (int i = 0; i < NL; ++i) Lf[i] = G[G_L + i];
#pragma unroll
        for (int a = 0; a < 4; ++a) rhs[a] = ((mask >> a) & 1) ? qc[a] : T(0);
        chol_solve4(Lf, rhs, y);
        if (tape) {
            // the tape record of stage t: computed column c of F_t (c < 11),
            // column c of K_t, and with c == 0 the masked factor and the mask
#pragma unroll
            for (int a = 0; a < NU; ++a) P.tape[trow(P, b, t, T_K + a * NX + c)] = ((mask >> a) & 1) ? -y[a] : T(0);
            if (c < NGC) {
#pragma unroll
                for (int i = 0; i < NX; ++i) P.tape[trow(P, b, t, T_F + c * NX + i)] = F[i * NZ + gcol(c)];
            }
            if (c == 0) {
#pragma unroll
                for (int i = 0; i < NL; ++i) P.tape[trow(P, b, t, T_L + i)] = Lf[i];
                P.tape[trow(P, b, t, T_M)] = (T)mask;
            }
            continue;
        }
#pragma unroll
        for (int a = 0; a < NU; ++a) grow[(R_K + a * NX + c) * GW] = ((mask >> a) & 1) ? -y[a] : T(0);
        if (c == 0) {
#pragma unroll
            for (int a = 0; a < NU; ++a) grow[(R_KK + a) * GW] = G[G_K + a];
        }
    }
}

// The costate in the sequential recursion's precision.  The scan's v_t comes
// out of composed transition parts (A, b, C), whose FP32 rounding reaches the
// costate, and a converged solve's controls are the zero of that gradient.
// With every stage's free set, factor, Q_uu and Q_ux as the phase found them,
// the vector part of the recursion runs again on one warp, from the last stage
// back:
//   g = r_t + B_t' v_{t+1},   k_f = -Q_uu,ff^-1 (g_f + Q_uu,fc k_c)  (k_c: the
//   clamped offsets),   v_t = q_t + A_t' v_{t+1} + Q_ux' k,
// and k_t is rewritten in the stage records.  (The value update's K_t'(Q_uu k
// + g) vanishes: Q_uu k + g is zero on the free set and K_t on the clamped
// one.)  Q_uu and Q_ux come from the scan's V, but they multiply k, which is
// small near convergence, so their rounding barely reaches v_t.  Matrix-vector
// work only: v_{t+1} stays in lanes 0..12 and is broadcast by shuffles; each
// stage's F_t and record are copied into a ring in shared memory (the whole
// block's area, free by now) RC_RING - 1 stages ahead.
constexpr int RC_F = 0, RC_G = FSTR, RC_SIZE = RC_G + GREC, RC_RING = 8;
static_assert(RC_SIZE % 4 == 0, "ring slots start on 16 bytes");

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
static_assert(RC_RING * RC_SIZE <= SW * WA_SIZE, "the costate pass's ring fits the block's shared memory");

// One stage's data of the costate pass, in the registers of each lane.
template <typename T> struct RcStage {
    T fc[NX];          // the lane's column of F_t
    T base;            // q_t (lanes 0..12) or r_t (lanes 16..19) of that column
    T qr[NU];          // Q_ux's column `lane`
    T dc[NU];          // the clamped offsets
    T H[NU][NU];       // Q_uu
    T Lf[NL];          // its factor on the free set
    int mask;          // the free set
};

template <typename T>
__device__ __forceinline__ void rc_load(const T* S, int cc, int bidx, int li, RcStage<T>& d) {
    const T* G = S + RC_G;
#pragma unroll
    for (int i = 0; i < NX; ++i) d.fc[i] = S[RC_F + i * NZ + cc];
    d.base = bidx < 0 ? T(0) : G[bidx];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
        d.qr[a] = G[G_QU + a * NX + li];
        d.dc[a] = G[G_DC + a];
#pragma unroll
        for (int c = a; c < NU; ++c) d.H[a][c] = d.H[c][a] = G[G_H + a * NU + c];
    }
#pragma unroll
    for (int i = 0; i < NL; ++i) d.Lf[i] = G[G_L + i];
    d.mask = (int)G[G_M];
}

template <typename T>
__device__ void refine_costate(const Params<T>& P, const ScanWs<T>& W, T* ring, int pos, int n, int lane) {
    // 16-byte copies: the records and the ring's slots start on 16 bytes
    constexpr int V = 16 / sizeof(T);
    auto fetch = [&](int t, T* d) {
        for (int e = lane * V; e < FSTR; e += 32 * V) cp_async16(d + RC_F + e, W.F + (size_t)t * FSTR + e);
        for (int e = lane * V; e < GREC; e += 32 * V) cp_async16(d + RC_G + e, W.G + (size_t)t * GREC + e);
        cp_async_commit();
    };
    // one commit group per stage (empty ones past stage 0): stage n-1-x in
    // group x and slot x % RC_RING
    for (int x = 0; x < RC_RING - 1; ++x) {
        if (n - 1 - x >= 0) fetch(n - 1 - x, ring + x * RC_SIZE);
        else cp_async_commit();
    }
    // the column of F_t this lane takes: A_t's column `lane` (lanes 0..12, for
    // A_t' v) or B_t's column lane - 16 (lanes 16..19, for g), and the record
    // entry that goes with it (q_t or r_t)
    const int col = lane < NX ? lane : (lane >= 16 && lane < 16 + NU ? NX + lane - 16 : -1);
    const int cc = col < 0 ? 0 : col;
    const int bidx = col < 0 ? -1 : (col < NX ? G_Q + col : G_R + col - NX);
    const int li = lane < NX ? lane : 0;
    // k_t's entry `lane` in the stage records, stage n-1 first
    T* kst = P.stg + srow(P, pos, n - 1, 0) + (size_t)(R_KK + (lane < NU ? lane : 0)) * GW;
    asm volatile("cp.async.wait_group %0;\n" ::"n"(RC_RING - 2) : "memory");
    __syncwarp();
    T vr = T(0);                                        // v_{t+1}, component `lane`
    // stage t from `cur`, with stage t-1's data loaded into `nxt` meanwhile
    auto step = [&](int t, int x, const RcStage<T>& cur, RcStage<T>& nxt) {
        __syncwarp();                                   // every lane is done with the slot refilled below
        const int ahead = t - (RC_RING - 1);
        if (ahead >= 0) fetch(ahead, ring + ((x + RC_RING - 1) % RC_RING) * RC_SIZE);
        else cp_async_commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(RC_RING - 2) : "memory");
        __syncwarp();
        if (t > 0) rc_load(ring + ((x + 1) % RC_RING) * RC_SIZE, cc, bidx, li, nxt);
        // q_t + A_t' v (lanes 0..12) and g = r_t + B_t' v (lanes 16..19)
        T s0 = cur.base, s1 = T(0);
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            const T vi = __shfl_sync(FULL, vr, i);
            if (i & 1) s1 += cur.fc[i] * vi;
            else s0 += cur.fc[i] * vi;
        }
        const T sf = s0 + s1;
        T g[NU];
#pragma unroll
        for (int a = 0; a < NU; ++a) g[a] = __shfl_sync(FULL, sf, 16 + a);
        // k on the free set (every lane, the same values)
        const int mask = cur.mask;
        T kk[NU], rhs[NU], y[NU];
#pragma unroll
        for (int a = 0; a < NU; ++a) kk[a] = ((mask >> a) & 1) ? T(0) : cur.dc[a];
#pragma unroll
        for (int a = 0; a < NU; ++a) {
            T r = T(0);
#pragma unroll
            for (int c = 0; c < NU; ++c) r += ((mask >> c) & 1) ? T(0) : cur.H[a][c] * kk[c];
            rhs[a] = ((mask >> a) & 1) ? r + g[a] : T(0);
        }
        chol_solve4(cur.Lf, rhs, y);
#pragma unroll
        for (int a = 0; a < NU; ++a) kk[a] = ((mask >> a) & 1) ? -y[a] : kk[a];
        T v = sf;
#pragma unroll
        for (int a = 0; a < NU; ++a) v += cur.qr[a] * kk[a];
        vr = lane < NX ? v : T(0);
        if (lane < NU) *kst = lane == 0 ? kk[0] : (lane == 1 ? kk[1] : (lane == 2 ? kk[2] : kk[3]));
        kst -= (size_t)SREC * GW;
    };
    // two stages a trip, the two register sets swapping roles
    RcStage<T> ra, rb;
    rc_load(ring, cc, bidx, li, ra);
    for (int t = n - 1, x = 0; t >= 0; t -= 2, x += 2) {
        step(t, x, ra, rb);
        if (t == 0) break;
        step(t - 1, x + 1, rb, ra);
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------- kernel --
// The Riccati phase of one iteration (A2 + A3) for the instance at position
// blockIdx.x, in the plain launch form with one instance per block: reads the
// nominal and cost rows from the stage records, writes K_t, k_t there, counts
// the iteration and sets NONPD on a non-positive pivot -- what k_mpc's Riccati
// phase does for an instance, with the stages in parallel.
template <typename T>
__global__ void __launch_bounds__(SW * 32, 1) k_scan_ric(const __grid_constant__ Params<T> P, int final_fac) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* wa = reinterpret_cast<T*>(smem_raw) + (size_t)(threadIdx.x >> 5) * WA_SIZE;
    __shared__ ScanShared<T> sh;
    __shared__ int s_bad, s_ok;
    const int pos = blockIdx.x;
    if (pos >= P.B) return;
    const int b = P.order ? P.order[pos] : pos;
    int n = P.horizon ? P.horizon[b] : P.N;
    n = n < 1 ? 1 : (n > P.N ? P.N : n);
    // an iteration's Riccati phase runs for a running instance and counts the
    // iteration; the final factorization (into the tape) runs for a finished
    // one, after the iterations
    const int st0 = P.status[b];                            // the same in every thread
    if (final_fac ? !(st0 == ST_CONVERGED || st0 == ST_STALLED || st0 == ST_MAX_ITER) : st0 != ST_RUNNING) return;
    const int done = P.iters[b];                            // iterations before this phase
    const int iters = final_fac ? done : done + 1;
    const ScanWs<T> W = scan_ws(P.scan, pos, P.N_ws);
    const int tid = threadIdx.x;
    if (tid < 4 * NU) {
        const int q = tid >> 2, a = tid & 3;
        const T* src = q == 0 ? P.R : (q == 1 ? P.uref : (q == 2 ? P.ulo : P.uhi));
        T* dst = q == 0 ? sh.R : (q == 1 ? sh.uref : (q == 2 ? sh.ulo : sh.uhi));
        dst[a] = src[(size_t)b * NU + a];
    }
    if (tid == 0) { s_bad = 0; sh.fail = 0; }
    __syncthreads();
    // the cost expansion at the nominal (x as hi + lo) and the first guesses
    for (int t = tid; t < n; t += blockDim.x) {
        const T* sr = P.stg + srow(P, pos, t, 0);
        T* G = W.G + (size_t)t * GREC;
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            const T q = sr[(R_Q + i) * GW];
            G[G_QD + i] = q;
            G[G_Q + i] = q * ((sr[(R_X + i) * GW] - sr[(R_XR + i) * GW]) + sr[(R_XL + i) * GW]);
        }
        const int pm = done >= 1 ? (int)G[G_M] : 15;
        const int ps = done >= 1 ? (int)G[G_SIDE] : 0;
#pragma unroll
        for (int a = 0; a < NU; ++a) {
            const T u = sr[(R_U + a) * GW];
            G[G_R + a] = sh.R[a] * (u - sh.uref[a]);
            const bool cl = !((pm >> a) & 1);
            G[G_DC + a] = cl ? (((ps >> a) & 1) ? sh.uhi[a] - u : sh.ulo[a] - u) : T(0);
        }
        G[G_AM] = (T)pm;
        if (t == n - 1) {
            for (int e = 0; e < FREC; ++e) W.F[(size_t)t * FSTR + e] = T(0);
        }
    }
    // A2: F_t = [A_t B_t] at the nominal x (hi part), t < n - 1: the computed
    // columns by forward tangents, the constant ones (position, velocity) exact
    const T hv = hv_coef(P.mdl);
    for (int job = tid; job < (n - 1) * (NGC + 1); job += blockDim.x) {
        const int t = job / (NGC + 1), jj = job - (NGC + 1) * t;
        T* F = W.F + (size_t)t * FSTR;
        if (jj == NGC) {
#pragma unroll
            for (int i = 0; i < NX; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    F[i * NZ + j] = i == j ? T(1) : T(0);
                    F[i * NZ + 7 + j] = (i == 7 + j) ? T(1) : (i == j ? hv : T(0));
                }
            continue;
        }
        const T* sr = P.stg + srow(P, pos, t, 0);
        T x[NX], u[NU], col[1][NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) x[i] = sr[(R_X + i) * GW];
#pragma unroll
        for (int a = 0; a < NU; ++a) u[a] = sr[(R_U + a) * GW];
        const int jc[1] = {gcol(jj)};
        tangent_columns<T, 1>(P.mdl, x, u, jc, col);
#pragma unroll
        for (int i = 0; i < NX; ++i) F[i * NZ + jc[0]] = col[0][i];
    }
    __syncthreads();
    // A3 of an iteration: one scan pass with the guessed free sets, then the
    // stages the guess got wrong by the sequential recursion.  The final
    // factorization takes the sequential recursion for every stage: the tape's
    // V_t and K_t then carry the sequential form's rounding, not that of the
    // composed transition parts
    int c = n - 1;
    if (!final_fac) {
        stage_factors_all(W, sh, n);
        __syncthreads();
        scan_suffixes(W, sh, wa, n, &s_bad);
        qp_inputs(W, sh, n);
        __syncthreads();
        stage_qps(P, W, sh, pos, n);
        __syncthreads();
        c = max(sh.cw[0], sh.cw[1]);
        // stages after c saw exact values and stage c an exact V_{c+1}: their
        // QPs are final, and a failed one at them ends the solve
        if (tid < n && tid >= c && W.G[(size_t)tid * GREC + G_OK] == T(0)) atomicOr(&sh.fail, 1);
        __syncthreads();
    }
    // (I + C J is singular only for non-finite data: C and J are positive
    // semidefinite, so its eigenvalues are at least 1)
    bool fail = sh.fail != 0 || s_bad != 0;
    if (!fail && c >= 0) {
        // the sequential stages on the whole block, in warp 0's work area
        T* wa0 = reinterpret_cast<T*>(smem_raw);
        // S_{c+1}'s J and eta (zero past the last stage)
        for (int e = tid; e < SV; e += blockDim.x) {
            const T v = c + 1 < n ? W.Sv[(size_t)(c + 1) * SV + e] : T(0);
            wa0[e < M13 ? SQ_J + e : SQ_N + e - M13] = v;
        }
        // F_t double-buffered: warp 0 copies the next stage's during this one
        T* fb[2] = {wa0 + SQ_F, wa0 + SQ_F + FSTR};
        if (tid < 32) wprefetch(fb[0], W.F + (size_t)c * FSTR, FREC, tid);
        bool ok = true;
        for (int t = c, k = 0; t >= 0 && ok; --t, k ^= 1) {
            if (tid < 32) cp_async_wait_all();
            __syncthreads();
            if (tid < 32 && t > 0) wprefetch(fb[k ^ 1], W.F + (size_t)(t - 1) * FSTR, FREC, tid);
            ok = seq_stage(P, W, sh, wa0, pos, t, n, t == c && !final_fac, tid, fb[k], &s_ok);
        }
        if (tid < 32) cp_async_wait_all();
        if (!ok && tid == 0) sh.fail = 1;
        __syncthreads();
        fail = sh.fail != 0;
    }
    if (!fail) write_gains(P, W, pos, n, b, final_fac != 0);
    if (!fail && !final_fac) {
        __syncthreads();
        if ((tid >> 5) == 0) refine_costate(P, W, reinterpret_cast<T*>(smem_raw), pos, n, tid & 31);
    }
    if (tid == 0) {
        P.iters[b] = iters;
        if (fail) P.status[b] = ST_NONPD;
    }
}

template <typename T> cudaError_t prepare_scan() {
    return cudaFuncSetAttribute(k_scan_ric<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((size_t)SW * WA_SIZE * sizeof(T)));
}

template <typename T> cudaError_t launch_scan_ric(const Params<T>& P, cudaStream_t st, int final_fac) {
    k_scan_ric<T><<<P.B, SW * 32, (size_t)SW * WA_SIZE * sizeof(T), st>>>(P, final_fac);
    return cudaGetLastError();
}

template cudaError_t prepare_scan<float>();
template cudaError_t prepare_scan<double>();
template cudaError_t launch_scan_ric<float>(const Params<float>&, cudaStream_t, int);
template cudaError_t launch_scan_ric<double>(const Params<double>&, cudaStream_t, int);

}  // namespace camp
