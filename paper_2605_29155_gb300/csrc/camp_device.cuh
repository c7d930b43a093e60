// camp_device.cuh -- per-instance device code of the batched differentiable MPC
// layer (box-constrained iLQR forward, adjoint LQR backward), templated on the
// working precision T (float on the product path, double for logic checks).
//
// Mapping: one warp (32 lanes) owns one MPC instance at a time.  The warp's
// matrices live in a per-warp shared-memory record (WarpSmem); every matrix
// product of the Riccati recursion is split over the lanes by output entry;
// the per-stage box QP runs on lane 0; the line search rolls out each alpha on
// its own lane.  Per-instance trajectories, gains and Jacobians that outlive a
// phase live in a global scratch "slot" owned by the warp (L2-resident).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace camp {

constexpr int NX = 13, NU = 4, NZ = 17;
constexpr int NF = NX * NZ;            // entries of F_t = [A_t B_t], stored column-major
constexpr int TAPE_STRIDE = 288;       // tape record per stage (elements)
constexpr int TAPE_F = 0, TAPE_K = 221, TAPE_L = 273, TAPE_MASK = 283;
constexpr int KREC = 56;               // K_t (52, row-major) + k_t (4)
constexpr int SP_STRIDE = 32;          // RK4 stage points per stage: 4 x (q, w, pad)
constexpr int CREC = 30;               // line-search candidate per stage: x hi (13), x lo (13), u (4)
constexpr int NTRI_Q = NZ * (NZ + 1) / 2;   // 153 upper-triangle entries of Q_t
constexpr int NTRI_V = NX * (NX + 1) / 2;   // 91 upper-triangle entries of V_t
constexpr int QP_MAX_IT = 20, QP_MAX_LS = 30;
constexpr unsigned FULL = 0xffffffffu;

enum { ST_CONVERGED = 0, ST_STALLED = 1, ST_MAX_ITER = 2, ST_NONFINITE = 3, ST_NONPD = 4,
       ST_RUNNING = -1 };

template <typename T> struct Model {
    T h, inv_m, g;
    T Jx, Jy, Jz, iJx, iJy, iJz;
    T M[3][4];                          // torque map tau = M u
};

template <typename T> struct Params {
    Model<T> mdl;
    int B, N, Nq, max_iter, n_alpha, store_all, N_ws;
    T tol;
    T alpha[4];
    const int* horizon;
    const int* order;                   // LPT order of instances (or NULL)
    const T *x0, *Q, *xref, *R, *uref, *ulo, *uhi, *uinit;
    T *u, *x, *cost;
    int *iters, *status;
    T* tape;
    T *wsF, *wsK, *wsCand, *wsSP, *wsKh, *wsXlo;
    int* queue;
};

template <typename T> struct AdjArgs {
    const T *gu, *gx;
    T *dQ, *dxref, *dx0;
    int recompute;
};

// Per-warp shared-memory record.
template <typename T> struct WarpSmem {
    T V[NX * NX];      // value Hessian V_{t+1} (full symmetric storage)
    T v[NX];           // value gradient v_{t+1}
    T F[NF];           // F_t column-major: F[j*13 + i] = dx+_i / dz_j
    T W[NF];           // V_{t+1} F_t, column-major
    T Qm[NZ * NZ];     // Q_t (row-major, full)
    T q[NZ];           // q_t
    T c[NZ];           // C_t z_t + c_t at the nominal
    T Cd[NZ];          // diag C_t
    T K[NU * NX];      // K_t row-major
    T k[NU];           // k_t
    T L[10];           // Cholesky of Q_uu on the free set (packed lower, masked)
    T x0[NX];
    T R[NU], uref[NU], ulo[NU], uhi[NU];
    T Jc[4];
    T vh[NX];          // adjoint value gradient
    T qh[NZ];          // adjoint q-hat
    T dx[NX];          // adjoint forward-sweep state
    T du[NU];
    T dQacc[NX];
    int mask;
    int ok;
};

template <typename T> __device__ __forceinline__ T clampT(T v, T lo, T hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

template <typename T> __device__ __forceinline__ bool finiteT(T v) { return isfinite(v); }

// ------------------------------------------------------------------ model ----
// Continuous quadrotor model x' = f_c(x, u):
//   p' = v;  q' = 1/2 q (x) [0, w];  v' = (sum u / m) R(q) e3 - g e3;
//   w' = J^-1 (M u - w x J w).
template <typename T>
__device__ __forceinline__ void f_cont(const Model<T>& m, const T* x, const T* u, T* d) {
    const T qw = x[3], qx = x[4], qy = x[5], qz = x[6];
    const T wx = x[10], wy = x[11], wz = x[12];
    const T th = u[0] + u[1] + u[2] + u[3];
    d[0] = x[7]; d[1] = x[8]; d[2] = x[9];
    d[3] = T(0.5) * (-qx * wx - qy * wy - qz * wz);
    d[4] = T(0.5) * (qw * wx + qy * wz - qz * wy);
    d[5] = T(0.5) * (qw * wy + qz * wx - qx * wz);
    d[6] = T(0.5) * (qw * wz + qx * wy - qy * wx);
    const T a = th * m.inv_m;
    d[7] = a * (T(2) * (qx * qz + qw * qy));
    d[8] = a * (T(2) * (qy * qz - qw * qx));
    d[9] = a * (qw * qw - qx * qx - qy * qy + qz * qz) - m.g;
    const T tx = m.M[0][0] * u[0] + m.M[0][1] * u[1] + m.M[0][2] * u[2] + m.M[0][3] * u[3];
    const T ty = m.M[1][0] * u[0] + m.M[1][1] * u[1] + m.M[1][2] * u[2] + m.M[1][3] * u[3];
    const T tz = m.M[2][0] * u[0] + m.M[2][1] * u[1] + m.M[2][2] * u[2] + m.M[2][3] * u[3];
    const T jwx = m.Jx * wx, jwy = m.Jy * wy, jwz = m.Jz * wz;
    d[10] = (tx - (wy * jwz - wz * jwy)) * m.iJx;
    d[11] = (ty - (wz * jwx - wx * jwz)) * m.iJy;
    d[12] = (tz - (wx * jwy - wy * jwx)) * m.iJz;
}

// One classic RK4 step of length h with u held constant (in place).
template <typename T>
__device__ __forceinline__ void rk4_step(const Model<T>& m, T* x, const T* u) {
    T k[NX], acc[NX], xs[NX];
    const T hh = T(0.5) * m.h;
    f_cont(m, x, u, k);
#pragma unroll
    for (int i = 0; i < NX; ++i) { acc[i] = k[i]; xs[i] = x[i] + hh * k[i]; }
    f_cont(m, xs, u, k);
#pragma unroll
    for (int i = 0; i < NX; ++i) { acc[i] = acc[i] + T(2) * k[i]; xs[i] = x[i] + hh * k[i]; }
    f_cont(m, xs, u, k);
#pragma unroll
    for (int i = 0; i < NX; ++i) { acc[i] = acc[i] + T(2) * k[i]; xs[i] = x[i] + m.h * k[i]; }
    f_cont(m, xs, u, k);
    const T h6 = m.h / T(6);
#pragma unroll
    for (int i = 0; i < NX; ++i) x[i] = x[i] + h6 * (acc[i] + k[i]);
}

// (hi, lo) += d: the rounding error of hi + d is carried in lo (2Sum, then a
// fast renormalisation), so a trajectory accumulated over many steps keeps the
// increments' precision instead of the state's.
template <typename T>
__device__ __forceinline__ void acc2(T& hi, T& lo, T d) {
    const T s = hi + d;
    const T bb = s - hi;
    const T err = (hi - (s - bb)) + (d - bb);
    const T l = lo + err;
    hi = s + l;
    lo = l - (hi - s);
}

// RK4 step whose state is the unevaluated sum hi + lo: the four stages are
// evaluated at hi in working precision, the increment h/6 (k1+2k2+2k3+k4) is
// added with acc2.
template <typename T>
__device__ __forceinline__ void rk4_step2(const Model<T>& m, T* xh, T* xl, const T* u) {
    T k[NX], acc[NX], xs[NX];
    const T hh = T(0.5) * m.h;
    f_cont(m, xh, u, k);
#pragma unroll
    for (int i = 0; i < NX; ++i) { acc[i] = k[i]; xs[i] = xh[i] + hh * k[i]; }
    f_cont(m, xs, u, k);
#pragma unroll
    for (int i = 0; i < NX; ++i) { acc[i] = acc[i] + T(2) * k[i]; xs[i] = xh[i] + hh * k[i]; }
    f_cont(m, xs, u, k);
#pragma unroll
    for (int i = 0; i < NX; ++i) { acc[i] = acc[i] + T(2) * k[i]; xs[i] = xh[i] + m.h * k[i]; }
    f_cont(m, xs, u, k);
    const T h6 = m.h / T(6);
#pragma unroll
    for (int i = 0; i < NX; ++i) acc2(xh[i], xl[i], h6 * (acc[i] + k[i]));
}

// RK4 stage points of one step: for s = 1..4 the (q, w) of xi_s (xi_1 = x,
// xi_2 = x + h/2 k1, xi_3 = x + h/2 k2, xi_4 = x + h k3) and the thrust.
template <typename T>
__device__ __forceinline__ void rk4_stage_points(const Model<T>& m, const T* x, const T* u, T* sp) {
    T k[NX], xs[NX];
    const T hh = T(0.5) * m.h;
#pragma unroll
    for (int i = 0; i < NX; ++i) xs[i] = x[i];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
#pragma unroll
        for (int i = 0; i < 4; ++i) sp[s * 8 + i] = xs[3 + i];
#pragma unroll
        for (int i = 0; i < 3; ++i) sp[s * 8 + 4 + i] = xs[10 + i];
        if (s < 3) {
            f_cont(m, xs, u, k);
            const T c = (s < 2) ? hh : m.h;
#pragma unroll
            for (int i = 0; i < NX; ++i) xs[i] = x[i] + c * k[i];
        }
    }
    sp[7] = u[0] + u[1] + u[2] + u[3];
}

// Jacobian-vector product of f_c at a stage point (q, w given in sp8, thrust th):
// out = A_c dx + B_c du.
template <typename T>
__device__ __forceinline__ void jvp_cont(const Model<T>& m, const T* sp8, T th, const T* dx, const T* du,
                                         T* out) {
    const T qw = sp8[0], qx = sp8[1], qy = sp8[2], qz = sp8[3];
    const T wx = sp8[4], wy = sp8[5], wz = sp8[6];
    const T dqw = dx[3], dqx = dx[4], dqy = dx[5], dqz = dx[6];
    const T dwx = dx[10], dwy = dx[11], dwz = dx[12];
    out[0] = dx[7]; out[1] = dx[8]; out[2] = dx[9];
    out[3] = T(0.5) * (-wx * dqx - wy * dqy - wz * dqz) + T(0.5) * (-qx * dwx - qy * dwy - qz * dwz);
    out[4] = T(0.5) * (wx * dqw + wz * dqy - wy * dqz) + T(0.5) * (qw * dwx - qz * dwy + qy * dwz);
    out[5] = T(0.5) * (wy * dqw - wz * dqx + wx * dqz) + T(0.5) * (qz * dwx + qw * dwy - qx * dwz);
    out[6] = T(0.5) * (wz * dqw + wy * dqx - wx * dqy) + T(0.5) * (-qy * dwx + qx * dwy + qw * dwz);
    const T a = th * m.inv_m;
    const T dth = du[0] + du[1] + du[2] + du[3];
    const T b = dth * m.inv_m;
    out[7] = a * (T(2) * qy * dqw + T(2) * qz * dqx + T(2) * qw * dqy + T(2) * qx * dqz)
           + b * (T(2) * (qx * qz + qw * qy));
    out[8] = a * (-T(2) * qx * dqw - T(2) * qw * dqx + T(2) * qz * dqy + T(2) * qy * dqz)
           + b * (T(2) * (qy * qz - qw * qx));
    out[9] = a * (T(2) * qw * dqw - T(2) * qx * dqx - T(2) * qy * dqy + T(2) * qz * dqz)
           + b * (qw * qw - qx * qx - qy * qy + qz * qz);
    const T gx = (m.Jz - m.Jy) * (wz * dwy + wy * dwz);
    const T gy = (m.Jx - m.Jz) * (wz * dwx + wx * dwz);
    const T gz = (m.Jy - m.Jx) * (wy * dwx + wx * dwy);
    const T tx = m.M[0][0] * du[0] + m.M[0][1] * du[1] + m.M[0][2] * du[2] + m.M[0][3] * du[3];
    const T ty = m.M[1][0] * du[0] + m.M[1][1] * du[1] + m.M[1][2] * du[2] + m.M[1][3] * du[3];
    const T tz = m.M[2][0] * du[0] + m.M[2][1] * du[1] + m.M[2][2] * du[2] + m.M[2][3] * du[3];
    out[10] = (tx - gx) * m.iJx;
    out[11] = (ty - gy) * m.iJy;
    out[12] = (tz - gz) * m.iJz;
}

// Column j of F_t = d RK4 / d(x, u): forward tangent through the four stages,
// d_s = J_c(xi_s) [dx + c_s d_{s-1}; du],  col = dx + h/6 (d1 + 2 d2 + 2 d3 + d4).
template <typename T>
__device__ __forceinline__ void tangent_column(const Model<T>& m, const T* sp, int j, T* col) {
    T dx[NX], du[NU], arg[NX], d[NX], acc[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) dx[i] = (i == j) ? T(1) : T(0);
#pragma unroll
    for (int a = 0; a < NU; ++a) du[a] = (NX + a == j) ? T(1) : T(0);
    const T th = sp[7];
    const T hh = T(0.5) * m.h;
    jvp_cont(m, sp + 0, th, dx, du, d);
#pragma unroll
    for (int i = 0; i < NX; ++i) { acc[i] = d[i]; arg[i] = dx[i] + hh * d[i]; }
    jvp_cont(m, sp + 8, th, arg, du, d);
#pragma unroll
    for (int i = 0; i < NX; ++i) { acc[i] = acc[i] + T(2) * d[i]; arg[i] = dx[i] + hh * d[i]; }
    jvp_cont(m, sp + 16, th, arg, du, d);
#pragma unroll
    for (int i = 0; i < NX; ++i) { acc[i] = acc[i] + T(2) * d[i]; arg[i] = dx[i] + m.h * d[i]; }
    jvp_cont(m, sp + 24, th, arg, du, d);
    const T h6 = m.h / T(6);
#pragma unroll
    for (int i = 0; i < NX; ++i) col[i] = dx[i] + h6 * (acc[i] + d[i]);
}

// ------------------------------------------------------------- box QP ------
// Packed lower-triangular index of a 4x4 factor.
__device__ __forceinline__ int lidx(int i, int j) { return i * (i + 1) / 2 + j; }

// Cholesky of H with the rows/columns outside `mask` replaced by the identity:
// the free block is factored exactly, clamped dimensions decouple.
template <typename T>
__device__ __forceinline__ bool chol_masked(const T (&H)[4][4], int mask, T (&L)[10]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool fj = (mask >> j) & 1;
        if (!fj) {
            L[lidx(j, j)] = T(1);
#pragma unroll
            for (int i = j + 1; i < 4; ++i) L[lidx(i, j)] = T(0);
            continue;
        }
        T s = H[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[lidx(j, k)] * L[lidx(j, k)];
        if (!(s > T(0))) return false;
        const T ljj = sqrt(s);
        L[lidx(j, j)] = ljj;
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            if ((mask >> i) & 1) {
                T t = H[i][j];
#pragma unroll
                for (int k = 0; k < j; ++k) t -= L[lidx(i, k)] * L[lidx(j, k)];
                L[lidx(i, j)] = t / ljj;
            } else {
                L[lidx(i, j)] = T(0);
            }
        }
    }
    return true;
}

// Solve (L L') y = b with a masked factor (b must be 0 on clamped dimensions).
template <typename T>
__device__ __forceinline__ void chol_solve4(const T* L, const T (&b)[4], T (&y)[4]) {
    T z[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        T s = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L[lidx(i, k)] * z[k];
        z[i] = s / L[lidx(i, i)];
    }
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        T s = z[i];
#pragma unroll
        for (int k = i + 1; k < 4; ++k) s -= L[lidx(k, i)] * y[k];
        y[i] = s / L[lidx(i, i)];
    }
}

template <typename T>
__device__ __forceinline__ T qp_value(const T (&H)[4][4], const T (&g)[4], const T (&d)[4]) {
    T lin = T(0), quad = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        lin += g[i] * d[i];
        T r = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) r += H[i][k] * d[k];
        quad += d[i] * r;
    }
    return lin + T(0.5) * quad;
}

// Projected-Newton box QP (Tassa et al. 2014, Bertsekas 1982):
//   min 1/2 d'Hd + g'd  s.t. lo <= d <= hi,  start d = clamp(0).
// Clamped set: at a bound with the gradient pointing out of the box.  Newton
// step on the free set, projected onto the box, Armijo backtracking (0.1, x0.6).
// Stops with no free dimension, or when the free set repeats after a full step
// the projection did not cut, or after QP_MAX_IT iterations.  Returns false on
// a non-positive pivot.  `L` and `mask` describe the last factored free set.
template <typename T>
__device__ bool box_qp(const T (&H)[4][4], const T (&g)[4], const T (&lo)[4], const T (&hi)[4],
                       T (&d)[4], T (&L)[10], int& mask_out) {
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = clampT(T(0), lo[i], hi[i]);
    int free_prev = -1, mask_fact = 0;
    bool last_full = false;
#pragma unroll
    for (int i = 0; i < 10; ++i) L[i] = T(0);
    L[0] = L[2] = L[5] = L[9] = T(1);
    for (int it = 0; it < QP_MAX_IT; ++it) {
        T grad[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            T s = g[i];
#pragma unroll
            for (int k = 0; k < 4; ++k) s += H[i][k] * d[k];
            grad[i] = s;
        }
        int fm = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool cl = (d[i] <= lo[i] && grad[i] > T(0)) || (d[i] >= hi[i] && grad[i] < T(0));
            if (!cl) fm |= 1 << i;
        }
        if (fm == 0) {
#pragma unroll
            for (int i = 0; i < 10; ++i) L[i] = T(0);
            L[0] = L[2] = L[5] = L[9] = T(1);
            mask_out = 0;
            return true;
        }
        if (last_full && fm == free_prev) { mask_out = fm; return true; }
        if (!chol_masked(H, fm, L)) { mask_out = fm; return false; }
        mask_fact = fm;
        T rhs[4], dn[4], dir[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if ((fm >> i) & 1) {
                T s = g[i];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (!((fm >> k) & 1)) s += H[i][k] * d[k];
                rhs[i] = -s;
            } else {
                rhs[i] = T(0);
            }
        }
        chol_solve4(L, rhs, dn);
#pragma unroll
        for (int i = 0; i < 4; ++i) dir[i] = ((fm >> i) & 1) ? dn[i] - d[i] : T(0);
        const T phi0 = qp_value(H, g, d);
        T step = T(1);
        bool acc = false;
        T trial[4], dnew[4];
        for (int ls = 0; ls < QP_MAX_LS; ++ls) {
#pragma unroll
            for (int i = 0; i < 4; ++i) { trial[i] = d[i] + step * dir[i]; dnew[i] = clampT(trial[i], lo[i], hi[i]); }
            const T phin = qp_value(H, g, dnew);
            T gd = T(0);
#pragma unroll
            for (int i = 0; i < 4; ++i) gd += grad[i] * (dnew[i] - d[i]);
            if (phin - phi0 <= T(0.1) * gd) { acc = true; break; }
            step *= T(0.6);
        }
        if (!acc) { mask_out = mask_fact; return true; }
        bool inside = true;
#pragma unroll
        for (int i = 0; i < 4; ++i) inside = inside && (trial[i] >= lo[i]) && (trial[i] <= hi[i]);
        last_full = (step == T(1)) && inside;
        free_prev = fm;
#pragma unroll
        for (int i = 0; i < 4; ++i) d[i] = dnew[i];
    }
    mask_out = mask_fact;
    return true;
}

// ------------------------------------------------------------ helpers -------
template <typename T> struct Inst {
    int b, n, slot;
    const T* Qb;      // Q rows of this instance
    const T* xrefb;
    T* ub;            // nominal / output u  [N][4]
    T* xb;            // nominal / output x  [N][13]
    T* F;             // slot scratch: F_t   [N_ws][221]
    T* Kr;            // slot scratch: K_t,k_t [N_ws][56]
    T* cand;          // slot scratch: candidates [4][N_ws][17]
    T* sp;            // slot scratch: stage points [N_ws][32]
    T* kh;            // slot scratch: adjoint k-hat [N_ws][4]
    T* xlo;           // slot scratch: low part of the nominal state [N_ws][13]
};

template <typename T>
__device__ __forceinline__ Inst<T> make_inst(const Params<T>& P, int b, int slot) {
    Inst<T> I;
    I.b = b;
    int n = P.horizon ? P.horizon[b] : P.N;
    n = n < 1 ? 1 : (n > P.N ? P.N : n);
    I.n = n;
    I.slot = slot;
    I.Qb = P.Q + (size_t)b * P.Nq * NX;
    I.xrefb = P.xref + (size_t)b * P.N * NX;
    I.ub = P.u + (size_t)b * P.N * NU;
    I.xb = P.x + (size_t)b * P.N * NX;
    const size_t s = (size_t)slot;
    I.F = P.wsF + s * P.N_ws * NF;
    I.Kr = P.wsK + s * P.N_ws * KREC;
    I.cand = P.wsCand + s * 4 * P.N_ws * CREC;
    I.sp = P.wsSP + s * P.N_ws * SP_STRIDE;
    I.kh = P.wsKh + s * P.N_ws * NU;
    I.xlo = P.wsXlo + s * P.N_ws * NX;
    return I;
}

template <typename T>
__device__ __forceinline__ const T* Qrow(const Params<T>& P, const Inst<T>& I, int t) {
    return I.Qb + (P.Nq > 1 ? t : 0) * NX;
}

template <typename T>
__device__ __forceinline__ void load_instance(const Params<T>& P, const Inst<T>& I, WarpSmem<T>& S, int lane) {
    if (lane < NX) S.x0[lane] = P.x0[(size_t)I.b * NX + lane];
    if (lane < NU) {
        S.R[lane] = P.R[I.b * NU + lane];
        S.uref[lane] = P.uref[I.b * NU + lane];
        S.ulo[lane] = P.ulo[I.b * NU + lane];
        S.uhi[lane] = P.uhi[I.b * NU + lane];
    }
    __syncwarp();
}

// --------------------------------------------------------- A1 rollout -------
// U^0 = clamp(u_init or u_ref), X^0 by RK4 from x_init (lane 0), J^0.  States
// are carried as hi + lo (rk4_step2); hi is the output x, lo stays in the slot.
// Stages past the horizon are zero-filled.  Returns J^0 on every lane.
template <typename T>
__device__ T initial_rollout(const Params<T>& P, const Inst<T>& I, const WarpSmem<T>& S, int lane) {
    const int n = I.n;
    for (int e = n * NU + lane; e < P.N * NU; e += 32) I.ub[e] = T(0);
    for (int e = n * NX + lane; e < P.N * NX; e += 32) I.xb[e] = T(0);
    T J = T(0);
    if (lane == 0) {
        T xh[NX], xl[NX], us[NU];
#pragma unroll
        for (int i = 0; i < NX; ++i) { xh[i] = S.x0[i]; xl[i] = T(0); }
        for (int t = 0; t < n; ++t) {
#pragma unroll
            for (int a = 0; a < NU; ++a) {
                const T u0 = P.uinit ? P.uinit[((size_t)I.b * P.N + t) * NU + a] : S.uref[a];
                us[a] = clampT(u0, S.ulo[a], S.uhi[a]);
                I.ub[t * NU + a] = us[a];
            }
            const T* Qt = Qrow(P, I, t);
            const T* xr = I.xrefb + t * NX;
            T sx = T(0), su = T(0);
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                I.xb[t * NX + i] = xh[i];
                I.xlo[t * NX + i] = xl[i];
                const T e = (xh[i] - xr[i]) + xl[i];
                sx += e * (Qt[i] * e);
            }
#pragma unroll
            for (int a = 0; a < NU; ++a) { const T e = us[a] - S.uref[a]; su += e * (S.R[a] * e); }
            J += T(0.5) * sx + T(0.5) * su;
            if (t < n - 1) rk4_step2(P.mdl, xh, xl, us);
        }
    }
    __syncwarp();
    return __shfl_sync(FULL, J, 0);
}

// ------------------------------------------------------ A2 linearization ----
// F_t = [A_t B_t] at the nominal for t = 0..n-2 into Fdst ([t][221], column-major):
// lanes first take one stage each for the RK4 stage points, then one
// (stage, column) tangent each.
template <typename T>
__device__ void linearize(const Params<T>& P, const Inst<T>& I, T* Fdst, int lane) {
    const int ns = I.n - 1;
    for (int t = lane; t < ns; t += 32) {
        T xs[NX], us[NU], sp[SP_STRIDE];
#pragma unroll
        for (int i = 0; i < NX; ++i) xs[i] = I.xb[t * NX + i];
#pragma unroll
        for (int a = 0; a < NU; ++a) us[a] = I.ub[t * NU + a];
        rk4_stage_points(P.mdl, xs, us, sp);
#pragma unroll
        for (int i = 0; i < SP_STRIDE; ++i) I.sp[t * SP_STRIDE + i] = sp[i];
    }
    __syncwarp();
    for (int w = lane; w < ns * NZ; w += 32) {
        const int t = w / NZ, j = w - t * NZ;
        T sp[SP_STRIDE], col[NX];
#pragma unroll
        for (int i = 0; i < SP_STRIDE; ++i) sp[i] = I.sp[t * SP_STRIDE + i];
        tangent_column(P.mdl, sp, j, col);
        T* dst = Fdst + (size_t)t * NF + j * NX;
#pragma unroll
        for (int i = 0; i < NX; ++i) dst[i] = col[i];
    }
    __syncwarp();
}

// ---------------------------------------------- A3 Riccati with box QP ------
// Sec. IV-2, t = n-1 .. 0 with V_n = 0, v_n = 0:
//   Q_t = C_t + F_t' V_{t+1} F_t,   q_t = (C_t z_t + c_t) + F_t' v_{t+1}
//   k_t, free set <- box QP(Q_uu, q_u, u_lo - u_t, u_hi - u_t)
//   K_t = -Q_uu,ff^-1 Q_ux,f on free rows, 0 on clamped rows
//   V_t = Q_xx + Q_xu K_t,   v_t = q_x + Q_xu k_t
// K_t, k_t go to the slot scratch.  Options:
//   use_lo   cost gradient at the hi + lo nominal (iterations); otherwise at
//            x* as returned (the factorization the backward differentiates)
//   tape     also store F_t, K_t, the masked factor and the free mask
//   replay   skip the recursion and read F_t, K_t, factor and mask from the tape
//   adj      after each stage, the adjoint backward step (Sec. IV implicit
//            differentiation) on that stage's factorization:
//              qh = g_t + F_t' vh_{t+1};  kh_t = -(Q_uu,ff)^-1 qh_u,f;  vh_t = qh_x + K_t' qh_u
template <typename T> struct RicOpts {
    T* tape;
    const AdjArgs<T>* adj;
    bool replay;
    bool use_lo;
};

template <typename T>
__device__ bool riccati(const Params<T>& P, const Inst<T>& I, WarpSmem<T>& S, int lane,
                        const int* triQ, const int* triV, const RicOpts<T> o) {
    const int n = I.n;
    for (int e = lane; e < NX * NX; e += 32) S.V[e] = T(0);
    if (lane < NX) { S.v[lane] = T(0); S.vh[lane] = T(0); }
    __syncwarp();
    for (int t = n - 1; t >= 0; --t) {
        const bool dyn = (t < n - 1);
        if (o.replay) {
            const T* rec = P.tape + ((size_t)I.b * P.N + t) * TAPE_STRIDE;
            for (int e = lane; e < TAPE_MASK; e += 32) {
                const T val = rec[e];
                if (e < TAPE_K) S.F[e] = val;
                else if (e < TAPE_L) S.K[e - TAPE_K] = val;
                else S.L[e - TAPE_L] = val;
            }
            if (lane == 0) S.mask = (int)rec[TAPE_MASK];
            __syncwarp();
        } else {
            const T* Qt = Qrow(P, I, t);
            if (lane < NZ) {
                T cd, e;
                if (lane < NX) {
                    cd = Qt[lane];
                    e = I.xb[t * NX + lane] - I.xrefb[t * NX + lane];
                    if (o.use_lo) e += I.xlo[t * NX + lane];
                } else {
                    const int a = lane - NX;
                    cd = S.R[a];
                    e = I.ub[t * NU + a] - S.uref[a];
                }
                S.Cd[lane] = cd;
                S.c[lane] = cd * e;
            }
            if (dyn) {
                const T* Ft = I.F + (size_t)t * NF;
                for (int e = lane; e < NF; e += 32) S.F[e] = Ft[e];
            }
            __syncwarp();
            if (dyn) {
                // W = V F (column-major)
                for (int e = lane; e < NF; e += 32) {
                    const int j = e / NX, i = e - j * NX;
                    T s = T(0);
#pragma unroll
                    for (int k = 0; k < NX; ++k) s += S.V[i * NX + k] * S.F[j * NX + k];
                    S.W[e] = s;
                }
                __syncwarp();
                // Q = C + F' W (upper triangle, mirrored), q = c + F' v
                for (int p = lane; p < NTRI_Q + NZ; p += 32) {
                    if (p < NTRI_Q) {
                        const int ab = triQ[p], a = ab >> 8, bb = ab & 0xff;
                        T s = (a == bb) ? S.Cd[a] : T(0);
#pragma unroll
                        for (int k = 0; k < NX; ++k) s += S.F[a * NX + k] * S.W[bb * NX + k];
                        S.Qm[a * NZ + bb] = s;
                        S.Qm[bb * NZ + a] = s;
                    } else {
                        const int a = p - NTRI_Q;
                        T s = S.c[a];
#pragma unroll
                        for (int k = 0; k < NX; ++k) s += S.F[a * NX + k] * S.v[k];
                        S.q[a] = s;
                    }
                }
            } else {
                for (int e = lane; e < NZ * NZ; e += 32) {
                    const int a = e / NZ, bb = e - a * NZ;
                    S.Qm[e] = (a == bb) ? S.Cd[a] : T(0);
                }
                if (lane < NZ) S.q[lane] = S.c[lane];
            }
            __syncwarp();
            if (lane == 0) {
                T H[4][4], g[4], lo[4], hi[4], d[4], L[10];
                int mask = 0;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) H[a][bb] = S.Qm[(NX + a) * NZ + NX + bb];
                    g[a] = S.q[NX + a];
                    const T ub = I.ub[t * NU + a];
                    lo[a] = S.ulo[a] - ub;
                    hi[a] = S.uhi[a] - ub;
                }
                const bool ok = box_qp(H, g, lo, hi, d, L, mask);
#pragma unroll
                for (int a = 0; a < 4; ++a) S.k[a] = d[a];
#pragma unroll
                for (int i = 0; i < 10; ++i) S.L[i] = L[i];
                S.mask = mask;
                S.ok = ok ? 1 : 0;
            }
            __syncwarp();
            if (!S.ok) return false;
            const int mask = S.mask;
            // K_t columns
            if (lane < NX) {
                T rhs[4], y[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) rhs[a] = ((mask >> a) & 1) ? S.Qm[(NX + a) * NZ + lane] : T(0);
                chol_solve4(S.L, rhs, y);
#pragma unroll
                for (int a = 0; a < 4; ++a) S.K[a * NX + lane] = ((mask >> a) & 1) ? -y[a] : T(0);
            }
            __syncwarp();
            // V_t, v_t
            for (int p = lane; p < NTRI_V + NX; p += 32) {
                if (p < NTRI_V) {
                    const int ij = triV[p], i = ij >> 8, j = ij & 0xff;
                    T s = S.Qm[i * NZ + j];
#pragma unroll
                    for (int a = 0; a < NU; ++a) s += S.Qm[i * NZ + NX + a] * S.K[a * NX + j];
                    S.V[i * NX + j] = s;
                    S.V[j * NX + i] = s;
                } else {
                    const int i = p - NTRI_V;
                    T s = S.q[i];
#pragma unroll
                    for (int a = 0; a < NU; ++a) s += S.Qm[i * NZ + NX + a] * S.k[a];
                    S.v[i] = s;
                }
            }
            // gains to the slot scratch (and tape)
            T* kr = I.Kr + (size_t)t * KREC;
            for (int e = lane; e < KREC; e += 32) kr[e] = (e < NU * NX) ? S.K[e] : S.k[e - NU * NX];
            if (o.tape) {
                T* rec = o.tape + ((size_t)I.b * P.N + t) * TAPE_STRIDE;
                for (int e = lane; e < TAPE_STRIDE; e += 32) {
                    T val;
                    if (e < TAPE_K) val = dyn ? S.F[e] : T(0);
                    else if (e < TAPE_L) val = S.K[e - TAPE_K];
                    else if (e < TAPE_MASK) val = S.L[e - TAPE_L];
                    else if (e == TAPE_MASK) val = T(mask);
                    else val = T(0);
                    rec[e] = val;
                }
            }
        }
        if (o.adj) {
            const AdjArgs<T>* adj = o.adj;
            __syncwarp();
            if (lane < NZ) {
                T g;
                if (lane < NX) g = adj->gx ? adj->gx[((size_t)I.b * P.N + t) * NX + lane] : T(0);
                else g = adj->gu[((size_t)I.b * P.N + t) * NU + lane - NX];
                if (dyn) {
#pragma unroll
                    for (int k = 0; k < NX; ++k) g += S.F[lane * NX + k] * S.vh[k];
                }
                S.qh[lane] = g;
            }
            __syncwarp();
            const int mask = S.mask;
            if (lane < NX) {
                T s = S.qh[lane];
#pragma unroll
                for (int a = 0; a < NU; ++a) s += S.K[a * NX + lane] * S.qh[NX + a];
                S.vh[lane] = s;
            } else if (lane == 16) {
                T rhs[4], y[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) rhs[a] = ((mask >> a) & 1) ? S.qh[NX + a] : T(0);
                chol_solve4(S.L, rhs, y);
#pragma unroll
                for (int a = 0; a < 4; ++a) I.kh[t * NU + a] = ((mask >> a) & 1) ? -y[a] : T(0);
            }
        }
        __syncwarp();
    }
    return true;
}

// ------------------------------------------------- A4 line search ----------
// Sec. IV-3: every alpha rolled out on its own lane,
//   u_hat_t = clamp(u_t + alpha k_t + K_t (x_hat_t - x_t)),  x_hat_{t+1} = RK4.
// The candidates are compared through their cost change with respect to the
// nominal, accumulated stage by stage from the differences themselves,
//   dJ_t = (x_hat - x)' Q (x - x_ref + (x_hat - x)/2) + (u_hat - u)' R (u - u_ref + (u_hat - u)/2),
// which equals J(alpha) - J exactly for the quadratic cost but does not cancel
// against J's magnitude; with the hi + lo states it resolves differences far
// below the working precision of J.  alpha* = first argmin, and the best
// candidate becomes the next nominal (Sec. IV-3).  Returns 0 (step taken: du,
// J updated) or 1 (no candidate with a finite cost: nominal kept).
template <typename T>
__device__ int line_search(const Params<T>& P, const Inst<T>& I, WarpSmem<T>& S, int lane, T& Jnom, T& du_out) {
    const int n = I.n;
    if (lane < P.n_alpha) {
        const T alpha = P.alpha[lane];
        T xh[NX], xl[NX], uh[NU];
#pragma unroll
        for (int i = 0; i < NX; ++i) { xh[i] = S.x0[i]; xl[i] = T(0); }
        T dJ = T(0), dJl = T(0);
        T* cd = I.cand + (size_t)lane * P.N_ws * CREC;
        for (int t = 0; t < n; ++t) {
            const T* kr = I.Kr + (size_t)t * KREC;
            const T* Qt = Qrow(P, I, t);
            const T* xr = I.xrefb + t * NX;
            T dxv[NX];
#pragma unroll
            for (int i = 0; i < NX; ++i) dxv[i] = (xh[i] - I.xb[t * NX + i]) + (xl[i] - I.xlo[t * NX + i]);
            T sx = T(0), su = T(0);
#pragma unroll
            for (int a = 0; a < NU; ++a) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < NX; ++i) s += kr[a * NX + i] * dxv[i];
                const T ub = I.ub[t * NU + a];
                const T un = ub + alpha * kr[NU * NX + a] + s;
                uh[a] = clampT(un, S.ulo[a], S.uhi[a]);
                const T d = uh[a] - ub;
                su += d * (S.R[a] * ((ub - S.uref[a]) + T(0.5) * d));
            }
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                const T eb = (I.xb[t * NX + i] - xr[i]) + I.xlo[t * NX + i];
                sx += dxv[i] * (Qt[i] * (eb + T(0.5) * dxv[i]));
            }
            acc2(dJ, dJl, sx + su);
#pragma unroll
            for (int i = 0; i < NX; ++i) { cd[t * CREC + i] = xh[i]; cd[t * CREC + NX + i] = xl[i]; }
#pragma unroll
            for (int a = 0; a < NU; ++a) cd[t * CREC + 2 * NX + a] = uh[a];
            if (t < n - 1) rk4_step2(P.mdl, xh, xl, uh);
        }
        dJ = dJ + dJl;
        S.Jc[lane] = finiteT(dJ) ? dJ : T(INFINITY);
    }
    __syncwarp();
    int best = 0;
    T Jb = S.Jc[0];
    for (int c = 1; c < P.n_alpha; ++c)
        if (S.Jc[c] < Jb) { Jb = S.Jc[c]; best = c; }
    if (!finiteT(Jb)) return 1;
    const T* cd = I.cand + (size_t)best * P.N_ws * CREC;
    T dmax = T(0);
    for (int e = lane; e < n * CREC; e += 32) {
        const int t = e / CREC, j = e - t * CREC;
        const T val = cd[e];
        if (j < NX) {
            I.xb[t * NX + j] = val;
        } else if (j < 2 * NX) {
            I.xlo[t * NX + j - NX] = val;
        } else {
            T* up = I.ub + t * NU + (j - 2 * NX);
            const T d = fabs(val - *up);
            dmax = d > dmax ? d : dmax;
            *up = val;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T other = __shfl_xor_sync(FULL, dmax, o);
        dmax = other > dmax ? other : dmax;
    }
    __syncwarp();
    Jnom = Jnom + Jb;
    du_out = dmax;
    return 0;
}

// ---------------------------------------------- A8 adjoint forward sweep ----
// dx_0 = 0; du_t = K_t dx_t + kh_t; dx_{t+1} = F_t [dx_t; du_t]; with
// d_tau_t = [dx_t; du_t]:  dQ_t = dx_t * (x*_t - x_ref,t),  dx_ref,t = -Q_t * dx_t,
// dx0 = vh_0 (value gradient of the adjoint LQR).  Fsrc / Ksrc: per-stage F_t
// and K_t with strides fs / ks (tape records or slot scratch).
template <typename T>
__device__ void adjoint_forward(const Params<T>& P, const Inst<T>& I, WarpSmem<T>& S, int lane,
                                const T* Fsrc, size_t fs, const T* Ksrc, size_t ks, const AdjArgs<T>& A) {
    const int n = I.n;
    const size_t b = I.b;
    if (lane < NX) { S.dx[lane] = T(0); S.dQacc[lane] = T(0); A.dx0[b * NX + lane] = S.vh[lane]; }
    __syncwarp();
    for (int t = 0; t < n; ++t) {
        const T* Kt = Ksrc + (size_t)t * ks;
        if (lane < NU) {
            T s = I.kh[t * NU + lane];
#pragma unroll
            for (int i = 0; i < NX; ++i) s += Kt[lane * NX + i] * S.dx[i];
            S.du[lane] = s;
        }
        if (lane >= 16 && lane < 16 + NX) {
            const int i = lane - 16;
            const T* Qt = Qrow(P, I, t);
            const T dxi = S.dx[i];
            const T e = I.xb[t * NX + i] - I.xrefb[t * NX + i];
            if (P.Nq > 1) A.dQ[(b * P.Nq + t) * NX + i] = dxi * e;
            else S.dQacc[i] += dxi * e;
            A.dxref[(b * P.N + t) * NX + i] = -Qt[i] * dxi;
        }
        __syncwarp();
        if (t < n - 1) {
            const T* Ft = Fsrc + (size_t)t * fs;
            T s = T(0);
            if (lane < NX) {
#pragma unroll
                for (int k = 0; k < NX; ++k) s += Ft[k * NX + lane] * S.dx[k];
#pragma unroll
                for (int a = 0; a < NU; ++a) s += Ft[(NX + a) * NX + lane] * S.du[a];
            }
            __syncwarp();
            if (lane < NX) S.dx[lane] = s;
            __syncwarp();
        }
    }
    // zero the stages past the horizon, write the shared-Q sum
    for (int e = n * NX + lane; e < P.N * NX; e += 32) A.dxref[b * P.N * NX + e] = T(0);
    if (P.Nq > 1) {
        for (int e = n * NX + lane; e < P.Nq * NX; e += 32) A.dQ[b * P.Nq * NX + e] = T(0);
    } else if (lane < NX) {
        A.dQ[b * NX + lane] = S.dQacc[lane];
    }
    __syncwarp();
}

}  // namespace camp
