// camp_device.cuh -- per-instance device code of the batched differentiable MPC
// layer (box-constrained iLQR forward, adjoint LQR backward), templated on the
// working precision T (float on the product path, double for logic checks).
//
// Mapping: a group of TPI lanes (8, 16 or 32) owns one MPC instance; a warp
// runs 32 / TPI instances in lockstep.  Each instance's matrices live in its
// shared-memory record (WarpSmem); every matrix product of the Riccati
// recursion is split over the group's lanes by output entry; the per-stage box
// QP runs on one lane; the line search rolls out each alpha on its own lane.
// Per-instance trajectories, gains and Jacobians that outlive a phase live in
// a global scratch "slot" owned by the group (L2-resident).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace camp {

constexpr int NX = 13, NU = 4, NZ = 17;
constexpr int NF = NX * NZ;            // entries of F_t = [A_t B_t], stored column-major
constexpr int NFC = 11 * NX;           // scratch copy of F_t: only its 11 computed columns
constexpr int LD = 16;                 // row / column stride of V_t and F_t in shared memory (128-bit aligned)
constexpr int TAPE_STRIDE = 288;       // tape record per stage (elements)
constexpr int TAPE_F = 0, TAPE_K = 221, TAPE_L = 273, TAPE_MASK = 287;
constexpr int NL = 14;                 // factor: packed lower 4x4 (10) + reciprocal diagonal (4)
constexpr int KREC = 56;               // K_t (52, row-major) + k_t (4)
constexpr int SP_STRIDE = 32;          // RK4 stage points per stage: 4 x (q, w, pad)
constexpr int CREC = 30;               // line-search candidate per stage: x hi (13), x lo (13), u (4)
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

// Per-instance shared-memory record.
template <typename T> struct alignas(16) WarpSmem {
    T V[NX * LD];      // value Hessian V_{t+1}: V[i*LD + j] (full symmetric storage)
    T F[2][NZ * LD];   // F_t column-major, F[t & 1][j*LD + i] = dx+_i / dz_j (double buffered)
    T Qxu[NX * NU];    // x-u block of Q_t again, Qxu[i*4 + a] = Q[i][13 + a]
    T v[LD];           // value gradient v_{t+1} (13 used)
    T stg[2][112];     // a stage's inputs, prefetched (double buffered): K_t, k_t (56), then
                       // x_t, x lo_t, u_t, Q_t, x_ref,t (SIN entries)
    T Qm[NZ * NZ];     // Q_t (row-major, full)
    T q[NZ];           // q_t
    T c[NZ];           // C_t z_t + c_t at the nominal
    T Cd[NZ];          // diag C_t
    T K[NU * NX];      // K_t row-major
    T k[NU];           // k_t
    T L[NL];           // Cholesky of Q_uu on the free set (packed lower, masked) + 1/diag
    T x0[NX];
    T R[NU], uref[NU], ulo[NU], uhi[NU];
    T ut[NU];          // the nominal u_t of the current Riccati stage
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

// 13 (or 4) consecutive entries of a 16-byte aligned shared-memory row, read
// with 128-bit loads.
__device__ __forceinline__ void ld13(const float* p, float (&o)[NX]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 u = reinterpret_cast<const float4*>(p)[k];
        o[4 * k] = u.x; o[4 * k + 1] = u.y; o[4 * k + 2] = u.z; o[4 * k + 3] = u.w;
    }
    o[12] = p[12];
}
__device__ __forceinline__ void ld13(const double* p, double (&o)[NX]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double2 u = reinterpret_cast<const double2*>(p)[k];
        o[2 * k] = u.x; o[2 * k + 1] = u.y;
    }
    o[12] = p[12];
}
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
    const float4 u = *reinterpret_cast<const float4*>(p);
    o[0] = u.x; o[1] = u.y; o[2] = u.z; o[3] = u.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
    const double2 u = reinterpret_cast<const double2*>(p)[0], w = reinterpret_cast<const double2*>(p)[1];
    o[0] = u.x; o[1] = u.y; o[2] = w.x; o[3] = w.y;
}

// Asynchronous global -> shared copies (cp.async): the data lands in shared
// memory without passing through registers; a lane waits for its own copies
// with cp_async_wait_all, and a warp barrier after that makes every lane's
// copies visible to the group.
template <typename T> __device__ __forceinline__ void cp_async(T* dst, const T* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
// 16 bytes; both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

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

// One classic RK4 step of length h with u held constant, on a state carried
// as the unevaluated sum hi + lo: the four stages are evaluated at hi in
// working precision, the increment h/6 (k1 + 2k2 + 2k3 + k4) is added with acc2.
template <typename T>
__device__ __forceinline__ void rk4_step2(const Model<T>& m, T* xh, T* xl, const T* u) {
    T k[NX], acc[NX], xs[NX];
    const T hh = T(0.5) * m.h;
#pragma unroll
    for (int i = 0; i < NX; ++i) xs[i] = xh[i];
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        f_cont(m, xs, u, k);
        const T w = (st == 0 || st == 3) ? T(1) : T(2);
        const T c = (st < 2) ? hh : m.h;
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            acc[i] = (st == 0) ? k[i] : acc[i] + w * k[i];
            xs[i] = xh[i] + c * k[i];
        }
    }
    const T h6 = m.h / T(6);
#pragma unroll
    for (int i = 0; i < NX; ++i) acc2(xh[i], xl[i], h6 * acc[i]);
}

// RK4 stage points of one step: for s = 1..4 the (q, w) of xi_s (xi_1 = x,
// xi_2 = x + h/2 k1, xi_3 = x + h/2 k2, xi_4 = x + h k3) and the thrust.
template <typename T>
__device__ __forceinline__ void rk4_stage_points(const Model<T>& m, const T* x, const T* u, T* __restrict__ sp) {
    T k[NX], xs[NX];
    const T hh = T(0.5) * m.h;
#pragma unroll
    for (int i = 0; i < NX; ++i) xs[i] = x[i];
#pragma unroll
    for (int st = 0; st < 4; ++st) {
#pragma unroll
        for (int i = 0; i < 4; ++i) sp[st * 8 + i] = xs[3 + i];
#pragma unroll
        for (int i = 0; i < 3; ++i) sp[st * 8 + 4 + i] = xs[10 + i];
        if (st < 3) {
            f_cont(m, xs, u, k);
            const T c = (st < 2) ? hh : m.h;
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

// The 6 columns of F_t for p and v are constant: position enters nothing
// (F[:, p_i] = e_{p_i}) and velocity only the position (F[:, v_i] = e_{v_i} +
// h e_{p_i}, h written as (h/6) * 6 as the RK4 combination forms it).  The
// other 11 columns (q, w, u) are computed; GCOL maps 0..10 to them.
__device__ __forceinline__ int gcol(int jj) { return jj < 4 ? 3 + jj : 6 + jj; }
__device__ __forceinline__ int tcol(int jj) { return jj < 3 ? jj : jj + 4; }
constexpr int NGC = 11, NTC = 6;
template <typename T> __device__ __forceinline__ T hv_coef(const Model<T>& m) { return (m.h / T(6)) * T(6); }

// Column j of F_t = d RK4 / d(x, u): forward tangent through the four stages,
// d_s = J_c(xi_s) [dx + c_s d_{s-1}; du],  col = dx + h/6 (d1 + 2 d2 + 2 d3 + d4).
template <typename T>
__device__ __forceinline__ void tangent_column(const Model<T>& m, const T* __restrict__ sp, int j, T* col) {
    T dx[NX], du[NU], arg[NX], d[NX], acc[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) { dx[i] = (i == j) ? T(1) : T(0); arg[i] = dx[i]; }
#pragma unroll
    for (int a = 0; a < NU; ++a) du[a] = (NX + a == j) ? T(1) : T(0);
    const T th = sp[7];
    const T hh = T(0.5) * m.h;
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        jvp_cont(m, sp + 8 * st, th, arg, du, d);
        const T w = (st == 0 || st == 3) ? T(1) : T(2);
        const T c = (st < 2) ? hh : m.h;
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            acc[i] = (st == 0) ? d[i] : acc[i] + w * d[i];
            arg[i] = dx[i] + c * d[i];
        }
    }
    const T h6 = m.h / T(6);
#pragma unroll
    for (int i = 0; i < NX; ++i) col[i] = dx[i] + h6 * acc[i];
}

// ------------------------------------------------------------- box QP ------
// Packed lower-triangular index of a 4x4 factor.
__device__ __forceinline__ int lidx(int i, int j) { return i * (i + 1) / 2 + j; }

// Pivot of the Cholesky factor: l = sqrt(s) and 1 / l.  In FP32 from the
// hardware reciprocal square root refined by one Newton step (about 1 ulp, as
// accurate as the correctly rounded pair for the gradients, and a much shorter
// serial chain in the box QP); in FP64 correctly rounded.
__device__ __forceinline__ void pivot(float s, float& l, float& il) {
    il = rsqrtf(s);
    il = il * (1.5f - 0.5f * s * il * il);
    l = s * il;
}
__device__ __forceinline__ void pivot(double s, double& l, double& il) {
    l = sqrt(s);
    il = 1.0 / l;
}

// Cholesky of H with the rows/columns outside `mask` replaced by the identity:
// the free block is factored exactly, clamped dimensions decouple.  L[10 + j]
// holds 1 / L_jj so that the solves multiply instead of divide.
template <typename T>
__device__ __forceinline__ bool chol_masked(const T (&H)[4][4], int mask, T (&L)[NL]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool fj = (mask >> j) & 1;
        if (!fj) {
            L[lidx(j, j)] = T(1);
            L[10 + j] = T(1);
#pragma unroll
            for (int i = j + 1; i < 4; ++i) L[lidx(i, j)] = T(0);
            continue;
        }
        T s = H[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[lidx(j, k)] * L[lidx(j, k)];
        if (!(s > T(0))) return false;
        T ljj, ij;
        pivot(s, ljj, ij);
        L[lidx(j, j)] = ljj;
        L[10 + j] = ij;
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            if ((mask >> i) & 1) {
                T t = H[i][j];
#pragma unroll
                for (int k = 0; k < j; ++k) t -= L[lidx(i, k)] * L[lidx(j, k)];
                L[lidx(i, j)] = t * ij;
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
        z[i] = s * L[10 + i];
    }
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        T s = z[i];
#pragma unroll
        for (int k = i + 1; k < 4; ++k) s -= L[lidx(k, i)] * y[k];
        y[i] = s * L[10 + i];
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
                       T (&d)[4], T (&L)[NL], int& mask_out) {
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = clampT(T(0), lo[i], hi[i]);
    int free_prev = -1, mask_fact = 0;
    bool last_full = false;
#pragma unroll
    for (int i = 0; i < NL; ++i) L[i] = T(0);
    L[0] = L[2] = L[5] = L[9] = L[10] = L[11] = L[12] = L[13] = T(1);
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
            for (int i = 0; i < NL; ++i) L[i] = T(0);
            L[0] = L[2] = L[5] = L[9] = L[10] = L[11] = L[12] = L[13] = T(1);
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
        bool inside = true, strict = true;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            inside = inside && (trial[i] >= lo[i]) && (trial[i] <= hi[i]);
            strict = strict && (trial[i] > lo[i]) && (trial[i] < hi[i]);
        }
        last_full = (step == T(1)) && inside;
        free_prev = fm;
#pragma unroll
        for (int i = 0; i < 4; ++i) d[i] = dnew[i];
        // A full step strictly inside the box with every dimension free: no
        // dimension sits on a bound at the new point, so the next iteration
        // would find the same (full) free set and stop here.
        if (last_full && strict && fm == 15) { mask_out = fm; return true; }
    }
    mask_out = mask_fact;
    return true;
}

// ------------------------------------------------------------ lanes --------
// An instance is owned by a group of TPI consecutive lanes of a warp; a warp
// holds PACK = 32 / TPI instances and runs them in lockstep.  Every loop that
// contains a warp barrier runs a warp-uniform number of times (the largest
// horizon in the pack); each group does its own instance's share under a
// per-group predicate.  Per-instance arithmetic is the same for every TPI:
// each output entry is produced by one lane, in the same order of operations.
template <int TPI> struct Lanes {
    static constexpr int PACK = 32 / TPI;
    int lane, g, l;
    __device__ __forceinline__ Lanes() {
        lane = threadIdx.x & 31;
        g = lane / TPI;
        l = lane - g * TPI;
    }
    __device__ __forceinline__ int src(int sub) const { return g * TPI + sub; }
};

__device__ __forceinline__ void wsync() { __syncwarp(); }

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int w = __shfl_xor_sync(FULL, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// ------------------------------------------------------------ helpers -------
template <typename T> struct Inst {
    int b, n, slot;
    const T* Qb;      // Q rows of this instance
    const T* xrefb;
    T* ub;            // nominal / output u  [N][4]
    T* xb;            // nominal / output x  [N][13]
    T* F;             // slot scratch: computed columns of F_t [N_ws][11][13]
    T* Kr;            // slot scratch: K_t,k_t [N_ws][56]
    T* cand;          // slot scratch: candidates [4][N_ws][30]
    T* sp;            // slot scratch: stage points [N_ws][32]
    T* kh;            // slot scratch: adjoint k-hat [N_ws][4]
    T* xlo;           // slot scratch: low part of the nominal state [N_ws][13]
};

// Instance b in scratch slot `slot`; `valid` false gives an empty instance
// (n = 0) whose pointers are never dereferenced.
template <typename T>
__device__ __forceinline__ Inst<T> make_inst(const Params<T>& P, int b, int slot, bool valid) {
    Inst<T> I;
    I.b = b;
    int n = P.horizon ? P.horizon[b] : P.N;
    n = n < 1 ? 1 : (n > P.N ? P.N : n);
    I.n = valid ? n : 0;
    I.slot = slot;
    I.Qb = P.Q + (size_t)b * P.Nq * NX;
    I.xrefb = P.xref + (size_t)b * P.N * NX;
    I.ub = P.u + (size_t)b * P.N * NU;
    I.xb = P.x + (size_t)b * P.N * NX;
    const size_t s = (size_t)slot;
    I.F = P.wsF + s * P.N_ws * NFC;
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

// A stage's nominal and cost inputs as staged in shared memory (after K_t, k_t
// in the line search's record): x_t, x lo_t, u_t, Q_t, x_ref,t.
constexpr int SI_X = 0, SI_XL = NX, SI_U = 2 * NX, SI_Q = 2 * NX + NU, SI_R = 3 * NX + NU, SIN = 4 * NX + NU;

template <typename T>
__device__ __forceinline__ const T* stage_input_src(const Params<T>& P, const Inst<T>& I, int t, int e) {
    if (e < SI_XL) return I.xb + t * NX + e;
    if (e < SI_U) return I.xlo + t * NX + e - SI_XL;
    if (e < SI_Q) return I.ub + t * NU + e - SI_U;
    if (e < SI_R) return Qrow(P, I, t) + e - SI_Q;
    return I.xrefb + t * NX + e - SI_R;
}

// Starts the asynchronous copy of stage t's inputs to dst[0..SIN).
template <typename T, int TPI>
__device__ __forceinline__ void stage_inputs_async(const Params<T>& P, const Inst<T>& I, const Lanes<TPI>& L, int t,
                                                   T* dst) {
    constexpr int R = (SIN + TPI - 1) / TPI;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = L.l + r * TPI;
        if (e < SIN) cp_async(dst + e, stage_input_src(P, I, t, e));
    }
}

template <typename T, int TPI>
__device__ __forceinline__ void load_instance(const Params<T>& P, const Inst<T>& I, WarpSmem<T>& S,
                                              const Lanes<TPI>& L, bool act) {
    if (act) {
        for (int e = L.l; e < NX; e += TPI) S.x0[e] = P.x0[(size_t)I.b * NX + e];
        for (int e = L.l; e < 4 * NU; e += TPI) {
            const int w = e >> 2, a = e & 3;
            const T* src = w == 0 ? P.R : (w == 1 ? P.uref : (w == 2 ? P.ulo : P.uhi));
            T* dst = w == 0 ? S.R : (w == 1 ? S.uref : (w == 2 ? S.ulo : S.uhi));
            dst[a] = src[I.b * NU + a];
        }
    }
    wsync();
}

// --------------------------------------------------------- A1 rollout -------
// U^0 = clamp(u_init or u_ref), X^0 by RK4 from x_init (one lane), J^0.  States
// are carried as hi + lo (rk4_step2); hi is the output x, lo stays in the slot.
// Stages past the horizon are zero-filled.  Returns J^0 on every lane of the group.
template <typename T, int TPI>
__device__ T initial_rollout(const Params<T>& P, const Inst<T>& I, const WarpSmem<T>& S, const Lanes<TPI>& L,
                             bool act) {
    T J = T(0);
    if (act) {
        const int n = I.n;
        for (int e = n * NU + L.l; e < P.N * NU; e += TPI) I.ub[e] = T(0);
        for (int e = n * NX + L.l; e < P.N * NX; e += TPI) I.xb[e] = T(0);
        if (L.l == 0) {
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
    }
    wsync();
    return __shfl_sync(FULL, J, L.src(0));
}

// ------------------------------------------------------ A2 linearization ----
// F_t = [A_t B_t] at the nominal for t = 0..n-2 into the slot (its 11
// computed columns, [t][11][13]): the group's lanes
// first take one stage each for the RK4 stage points, then one
// (stage, column) tangent each.
template <typename T, int TPI>
__device__ void linearize(const Params<T>& P, const Inst<T>& I, const Lanes<TPI>& L, bool act) {
    const int ns = act ? I.n - 1 : 0;
    for (int t = L.l; t < ns; t += TPI) {
        T xs[NX], us[NU];
#pragma unroll
        for (int i = 0; i < NX; ++i) xs[i] = I.xb[t * NX + i];
#pragma unroll
        for (int a = 0; a < NU; ++a) us[a] = I.ub[t * NU + a];
        rk4_stage_points(P.mdl, xs, us, I.sp + t * SP_STRIDE);
    }
    wsync();
    for (int w = L.l; w < ns * NGC; w += TPI) {
        const int t = w / NGC, jj = w - t * NGC;
        T col[NX];
        tangent_column(P.mdl, I.sp + t * SP_STRIDE, gcol(jj), col);
        T* dst = I.F + (size_t)t * NFC + jj * NX;
#pragma unroll
        for (int i = 0; i < NX; ++i) dst[i] = col[i];
    }
    wsync();
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
// Returns false (for the group) when a free block of Q_uu is not positive
// definite; the group's remaining stages are then skipped.
template <typename T> struct RicOpts {
    T* tape;
    const AdjArgs<T>* adj;
    bool replay;
    bool use_lo;
};

template <typename T, int TPI>
__device__ bool riccati(const Params<T>& P, const Inst<T>& I, WarpSmem<T>& S, const Lanes<TPI>& L,
                        const RicOpts<T> o, bool act) {
    const int n = act ? I.n : 0;
    const int nmax = warp_max(n);
    for (int e = L.l; e < NX * LD; e += TPI) S.V[e] = T(0);
    for (int e = L.l; e < NX; e += TPI) { S.v[e] = T(0); S.vh[e] = T(0); }
    if (L.l == 0) S.ok = 1;
    const T hv = hv_coef(P.mdl);
    // The six constant columns of F_t (p and v: identity, plus hv on the p
    // rows of the v columns) are the same at every stage: both buffers.
    for (int e = L.l; e < NTC * NX; e += TPI) {
        const int jj = e / NX, i = e - jj * NX, j = tcol(jj);
        const T val = (i == j) ? T(1) : ((j >= 7 && i == j - 7) ? hv : T(0));
        S.F[0][j * LD + i] = val;
        S.F[1][j * LD + i] = val;
    }
    bool alive = true;
    // Software pipeline: while stage t computes, stage t - 1's F_t columns and
    // cost inputs are copied asynchronously into the other buffers.
    auto prefetch = [&](int tt) {
        if (tt < 0 || tt >= n || o.replay) return;
        if (tt < n - 1) {
            const T* Ft = I.F + (size_t)tt * NFC;
            T* Fd = S.F[tt & 1];
            constexpr int FR = (NFC + TPI - 1) / TPI;
#pragma unroll
            for (int r = 0; r < FR; ++r) {
                const int e = L.l + r * TPI;
                if (e < NFC) {
                    const int jj = e / NX;
                    cp_async(Fd + gcol(jj) * LD + e - jj * NX, Ft + e);
                }
            }
        }
        stage_inputs_async(P, I, L, tt, S.stg[tt & 1] + KREC);
        cp_async_commit();
    };
    prefetch(n - 1);
    for (int t = nmax - 1; t >= 0; --t) {
        const bool on = alive && t < n;
        const bool dyn = on && t < n - 1;
        bool go = on;
        T* Fc = S.F[t & 1];
        if (o.replay) {
            wsync();
            if (on) {
                const T* rec = P.tape + ((size_t)I.b * P.N + t) * TAPE_STRIDE;
                for (int e = L.l; e < TAPE_MASK; e += TPI) {
                    const T val = rec[e];
                    if (e < TAPE_K) {
                        const int j = e / NX;
                        Fc[j * LD + e - j * NX] = val;
                    } else if (e < TAPE_L) {
                        S.K[e - TAPE_K] = val;
                    } else {
                        S.L[e - TAPE_L] = val;
                    }
                }
                if (L.l == 0) S.mask = (int)rec[TAPE_MASK];
            }
            wsync();
        } else {
            cp_async_wait_all();
            wsync();
            if (on) {
                const T* si = S.stg[t & 1] + KREC;
                for (int a = L.l; a < NZ; a += TPI) {
                    if (a < NX) {
                        const T qa = si[SI_Q + a], ea = si[SI_X + a] - si[SI_R + a];
                        S.Cd[a] = qa;
                        S.c[a] = qa * (o.use_lo ? ea + si[SI_XL + a] : ea);
                    } else {
                        const T cd = S.R[a - NX], ua = si[SI_U + a - NX];
                        S.Cd[a] = cd;
                        S.c[a] = cd * (ua - S.uref[a - NX]);
                        S.ut[a - NX] = ua;
                    }
                }
                prefetch(t - 1);
            }
            wsync();
            if (dyn) {
                // Column products.  Item c < NGC is the computed column gcol(c),
                // item c >= NGC the constant column tcol(c - NGC) (the costly
                // items first, so that no lane takes two of them while others
                // idle); its lane forms
                //   W[:, j] = V F[:, j]            (in registers)
                //   Q[r, j] = C_rj + F[:, r]' W[:, j] for every row r (rows of the
                //             constant columns take one or two entries of W[:, j])
                //   q[j]    = c_j + F[:, j]' v
                // and, for a computed column, mirrors its entries in the constant
                // rows into Q[j, r], so the upper triangle of Q is complete; the
                // lanes of the u columns also fill Qxu.
                for (int c = L.l; c < NZ; c += TPI) {
                    const bool cc = c >= NGC;
                    const int j = cc ? tcol(c - NGC) : gcol(c);
                    T w[NX];
                    T qj;
                    if (cc) {
#pragma unroll
                        for (int i = 0; i < NX; ++i)
                            w[i] = (j < 3) ? S.V[i * LD + j] : S.V[i * LD + j] + hv * S.V[i * LD + j - 7];
                        qj = S.c[j] + ((j < 3) ? S.v[j] : S.v[j] + hv * S.v[j - 7]);
                    } else {
                        T f[NX];
                        ld13(Fc + j * LD, f);
#pragma unroll
                        for (int i = 0; i < NX; ++i) {
                            T vr[NX];
                            ld13(S.V + i * LD, vr);
                            T s = T(0);
#pragma unroll
                            for (int k = 0; k < NX; ++k) s += vr[k] * f[k];
                            w[i] = s;
                        }
                        T vv[NX];
                        ld13(S.v, vv);
                        T s = S.c[j];
#pragma unroll
                        for (int k = 0; k < NX; ++k) s += f[k] * vv[k];
                        qj = s;
                    }
                    S.q[j] = qj;
#pragma unroll
                    for (int r = 0; r < NZ; ++r) {
                        const bool rc = r < 3 || (r >= 7 && r < 10);
                        if (cc && !rc) continue;          // filled by the computed column's mirror
                        T s = (r == j) ? S.Cd[j] : T(0);
                        if (r < 3) {
                            s += w[r];
                        } else if (r >= 7 && r < 10) {
                            s += w[r] + hv * w[r - 7];
                        } else {
                            T fr[NX];
                            ld13(Fc + r * LD, fr);
#pragma unroll
                            for (int k = 0; k < NX; ++k) s += fr[k] * w[k];
                        }
                        S.Qm[r * NZ + j] = s;
                        if (!cc && rc) S.Qm[j * NZ + r] = s;
                        if (!cc && r < NX && j >= NX) S.Qxu[r * NU + j - NX] = s;
                    }
                }
            } else if (on) {
                for (int e = L.l; e < NZ * NZ; e += TPI) {
                    const int a = e / NZ, bb = e - a * NZ;
                    S.Qm[e] = (a == bb) ? S.Cd[a] : T(0);
                }
                for (int e = L.l; e < NX * NU; e += TPI) S.Qxu[e] = T(0);
                for (int a = L.l; a < NZ; a += TPI) S.q[a] = S.c[a];
            }
            wsync();
            if (on && L.l == 0) {
                T H[4][4], g[4], lo[4], hi[4], d[4], Lf[NL];
                int mask = 0;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb)
                        H[a][bb] = a <= bb ? S.Qm[(NX + a) * NZ + NX + bb] : S.Qm[(NX + bb) * NZ + NX + a];
                    g[a] = S.q[NX + a];
                    const T ub = S.ut[a];
                    lo[a] = S.ulo[a] - ub;
                    hi[a] = S.uhi[a] - ub;
                }
                const bool ok = box_qp(H, g, lo, hi, d, Lf, mask);
#pragma unroll
                for (int a = 0; a < 4; ++a) S.k[a] = d[a];
#pragma unroll
                for (int i = 0; i < NL; ++i) S.L[i] = Lf[i];
                S.mask = mask;
                S.ok = ok ? 1 : 0;
            }
            wsync();
            if (on && !S.ok) alive = false;
            go = on && alive;
            const int mask = S.mask;
            if (go) {
                // Column c of K_t (to shared memory and the slot scratch), then,
                // from it in registers, the upper part of column c of
                //   V_t = Q_xx + Q_xu K_t   (mirrored: V_t is stored in full)
                // and v_t[c] = q_x[c] + Q_xu[c, :] k_t.
                T* kr = I.Kr + (size_t)t * KREC;
                for (int c = L.l; c < NX; c += TPI) {
                    T qc[4], rhs[4], y[4], kc[4];
                    ld4(S.Qxu + c * NU, qc);
#pragma unroll
                    for (int a = 0; a < 4; ++a) rhs[a] = ((mask >> a) & 1) ? qc[a] : T(0);
                    chol_solve4(S.L, rhs, y);
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        kc[a] = ((mask >> a) & 1) ? -y[a] : T(0);
                        S.K[a * NX + c] = kc[a];
                        kr[a * NX + c] = kc[a];
                    }
#pragma unroll
                    for (int i = 0; i < NX; ++i) {
                        if (i > c) break;
                        T qi[4];
                        ld4(S.Qxu + i * NU, qi);
                        T s = S.Qm[i * NZ + c];
#pragma unroll
                        for (int a = 0; a < NU; ++a) s += qi[a] * kc[a];
                        S.V[i * LD + c] = s;
                        S.V[c * LD + i] = s;
                    }
                    T s = S.q[c];
#pragma unroll
                    for (int a = 0; a < NU; ++a) s += qc[a] * S.k[a];
                    S.v[c] = s;
                }
                if (L.l == 0) {
#pragma unroll
                    for (int a = 0; a < NU; ++a) kr[NU * NX + a] = S.k[a];
                }
            }
            if (o.tape) {
                wsync();
                if (go) {
                    T* rec = o.tape + ((size_t)I.b * P.N + t) * TAPE_STRIDE;
                    for (int e = L.l; e < TAPE_STRIDE; e += TPI) {
                        T val;
                        if (e < TAPE_K) {
                            const int j = e / NX;
                            val = dyn ? Fc[j * LD + e - j * NX] : T(0);
                        } else if (e < TAPE_L) {
                            val = S.K[e - TAPE_K];
                        } else if (e < TAPE_MASK) {
                            val = S.L[e - TAPE_L];
                        } else {
                            val = T(mask);
                        }
                        rec[e] = val;
                    }
                }
            }
        }
        if (o.adj) {
            const AdjArgs<T>* adj = o.adj;
            wsync();
            if (go) {
                for (int a = L.l; a < NZ; a += TPI) {
                    T g;
                    if (a < NX) g = adj->gx ? adj->gx[((size_t)I.b * P.N + t) * NX + a] : T(0);
                    else g = adj->gu[((size_t)I.b * P.N + t) * NU + a - NX];
                    if (dyn) {
#pragma unroll
                        for (int k = 0; k < NX; ++k) g += Fc[a * LD + k] * S.vh[k];
                    }
                    S.qh[a] = g;
                }
            }
            wsync();
            if (go) {
                const int mask = S.mask;
                for (int i = L.l; i < NX; i += TPI) {
                    T s = S.qh[i];
#pragma unroll
                    for (int a = 0; a < NU; ++a) s += S.K[a * NX + i] * S.qh[NX + a];
                    S.vh[i] = s;
                }
                if (L.l == TPI - 1) {
                    T rhs[4], y[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) rhs[a] = ((mask >> a) & 1) ? S.qh[NX + a] : T(0);
                    chol_solve4(S.L, rhs, y);
#pragma unroll
                    for (int a = 0; a < 4; ++a) I.kh[t * NU + a] = ((mask >> a) & 1) ? -y[a] : T(0);
                }
            }
        }
        wsync();
    }
    return alive;
}

// ------------------------------------------------- A4 line search ----------
// Sec. IV-3: each alpha rolled out on its own lane of the group,
//   u_hat_t = clamp(u_t + alpha k_t + K_t (x_hat_t - x_t)),  x_hat_{t+1} = RK4.
// The candidates are compared through their cost change with respect to the
// nominal, accumulated stage by stage from the differences themselves,
//   dJ_t = (x_hat - x)' Q (x - x_ref + (x_hat - x)/2) + (u_hat - u)' R (u - u_ref + (u_hat - u)/2),
// which equals J(alpha) - J exactly for the quadratic cost but does not cancel
// against J's magnitude; with the hi + lo states it resolves differences far
// below the working precision of J.  alpha* = first argmin, and the best
// candidate becomes the next nominal (Sec. IV-3).  Each stage's gains, nominal
// and cost rows are copied into shared memory by all lanes of the group
// (asynchronous copies) one stage ahead.  Returns 0 (step taken: du, J
// updated) or 1 (no candidate with a finite cost: nominal kept).
// Stage t's staged record: K_t, k_t (KREC), then the stage inputs (SIN).
template <typename T, int TPI>
__device__ int line_search(const Params<T>& P, const Inst<T>& I, WarpSmem<T>& S, const Lanes<TPI>& L, bool act,
                           T& Jnom, T& du_out) {
    static_assert(TPI >= 4, "line search needs 4 candidate lanes");
    const int n = act ? I.n : 0;
    const int nmax = warp_max(n);
    auto issue = [&](int tt) {
        if (tt >= n) return;
        T* dst = S.stg[tt & 1];
        const T* kr = I.Kr + (size_t)tt * KREC;
        constexpr int PER = 16 / sizeof(T), NCH = KREC / PER;
        for (int e = L.l; e < NCH; e += TPI) cp_async16(dst + e * PER, kr + e * PER);
        stage_inputs_async(P, I, L, tt, dst + KREC);
        cp_async_commit();
    };
    issue(0);
    cp_async_wait_all();
    wsync();
    const bool cl = act && L.l < P.n_alpha;
    const T alpha = cl ? P.alpha[L.l] : T(0);
    T xh[NX], xl[NX], uh[NU];
#pragma unroll
    for (int i = 0; i < NX; ++i) { xh[i] = act ? S.x0[i] : T(0); xl[i] = T(0); }
    T dJ = T(0), dJl = T(0);
    T* cd = I.cand + (size_t)(L.l & 3) * P.N_ws * CREC;
    for (int t = 0; t < nmax; ++t) {
        issue(t + 1);
        if (cl && t < n) {
            const T* sb = S.stg[t & 1];
            const T* kr = sb;
            const T* xbt = sb + KREC + SI_X;
            const T* xlt = sb + KREC + SI_XL;
            const T* ubt = sb + KREC + SI_U;
            const T* Qt = sb + KREC + SI_Q;
            const T* xr = sb + KREC + SI_R;
            T dxv[NX];
#pragma unroll
            for (int i = 0; i < NX; ++i) dxv[i] = (xh[i] - xbt[i]) + (xl[i] - xlt[i]);
            T sx = T(0), su = T(0);
#pragma unroll
            for (int a = 0; a < NU; ++a) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < NX; ++i) s += kr[a * NX + i] * dxv[i];
                const T ub = ubt[a];
                const T un = ub + alpha * kr[NU * NX + a] + s;
                uh[a] = clampT(un, S.ulo[a], S.uhi[a]);
                const T d = uh[a] - ub;
                su += d * (S.R[a] * ((ub - S.uref[a]) + T(0.5) * d));
            }
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                const T eb = (xbt[i] - xr[i]) + xlt[i];
                sx += dxv[i] * (Qt[i] * (eb + T(0.5) * dxv[i]));
            }
            acc2(dJ, dJl, sx + su);
#pragma unroll
            for (int i = 0; i < NX; ++i) { cd[t * CREC + i] = xh[i]; cd[t * CREC + NX + i] = xl[i]; }
#pragma unroll
            for (int a = 0; a < NU; ++a) cd[t * CREC + 2 * NX + a] = uh[a];
            if (t < n - 1) rk4_step2(P.mdl, xh, xl, uh);
        }
        cp_async_wait_all();
        wsync();
    }
    if (cl) {
        dJ = dJ + dJl;
        S.Jc[L.l] = finiteT(dJ) ? dJ : T(INFINITY);
    }
    wsync();
    int r = 0;
    T dmax = T(0), Jb = T(0);
    if (act) {
        int best = 0;
        Jb = S.Jc[0];
        for (int c = 1; c < P.n_alpha; ++c)
            if (S.Jc[c] < Jb) { Jb = S.Jc[c]; best = c; }
        if (!finiteT(Jb)) {
            r = 1;
        } else {
            const T* cb = I.cand + (size_t)best * P.N_ws * CREC;
            for (int e = L.l; e < n * CREC; e += TPI) {
                const int t = e / CREC, j = e - t * CREC;
                const T val = cb[e];
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
        }
    }
#pragma unroll
    for (int o = TPI / 2; o > 0; o >>= 1) {
        const T other = __shfl_xor_sync(FULL, dmax, o);
        dmax = other > dmax ? other : dmax;
    }
    wsync();
    if (act && r == 0) {
        Jnom = Jnom + Jb;
        du_out = dmax;
    }
    return r;
}

// ---------------------------------------------- A8 adjoint forward sweep ----
// dx_0 = 0; du_t = K_t dx_t + kh_t; dx_{t+1} = F_t [dx_t; du_t]; with
// d_tau_t = [dx_t; du_t]:  dQ_t = dx_t * (x*_t - x_ref,t),  dx_ref,t = -Q_t * dx_t,
// dx0 = vh_0 (value gradient of the adjoint LQR).  Fsrc / Ksrc: per-stage F_t
// and K_t with strides fs / ks: tape records (full F_t) or slot scratch (its
// 11 computed columns, fcompact).
template <typename T, int TPI>
__device__ void adjoint_forward(const Params<T>& P, const Inst<T>& I, WarpSmem<T>& S, const Lanes<TPI>& L,
                                bool act, const T* Fsrc, size_t fs, bool fcompact, const T* Ksrc, size_t ks,
                                const AdjArgs<T>& A) {
    const int n = act ? I.n : 0;
    const int nmax = warp_max(n);
    const size_t b = I.b;
    constexpr int RX = (NX + TPI - 1) / TPI;
    if (act) {
        for (int i = L.l; i < NX; i += TPI) { S.dx[i] = T(0); S.dQacc[i] = T(0); A.dx0[b * NX + i] = S.vh[i]; }
    }
    wsync();
    for (int t = 0; t < nmax; ++t) {
        const bool on = t < n;
        if (on) {
            const T* Kt = Ksrc + (size_t)t * ks;
            for (int a = L.l; a < NU; a += TPI) {
                T s = I.kh[t * NU + a];
#pragma unroll
                for (int i = 0; i < NX; ++i) s += Kt[a * NX + i] * S.dx[i];
                S.du[a] = s;
            }
            const T* Qt = Qrow(P, I, t);
            for (int i = L.l; i < NX; i += TPI) {
                const T dxi = S.dx[i];
                const T e = I.xb[t * NX + i] - I.xrefb[t * NX + i];
                if (P.Nq > 1) A.dQ[(b * P.Nq + t) * NX + i] = dxi * e;
                else S.dQacc[i] += dxi * e;
                A.dxref[(b * P.N + t) * NX + i] = -Qt[i] * dxi;
            }
        }
        wsync();
        T snew[RX];
        if (on && t < n - 1) {
            // dx_{t+1} = F_t [dx_t; du_t]: the 11 computed columns, then the
            // constant p and v columns
            const T* Ft = Fsrc + (size_t)t * fs;
#pragma unroll
            for (int r = 0; r < RX; ++r) {
                const int i = L.l + r * TPI;
                if (i < NX) {
                    T s = T(0);
#pragma unroll
                    for (int jj = 0; jj < NGC; ++jj) {
                        const int j = gcol(jj);
                        s += Ft[(fcompact ? jj : j) * NX + i] * (j < NX ? S.dx[j] : S.du[j - NX]);
                    }
                    if (i < 3) s += S.dx[i] + hv_coef(P.mdl) * S.dx[i + 7];
                    else if (i >= 7 && i < 10) s += S.dx[i];
                    snew[r] = s;
                }
            }
        }
        wsync();
        if (on && t < n - 1) {
#pragma unroll
            for (int r = 0; r < RX; ++r) {
                const int i = L.l + r * TPI;
                if (i < NX) S.dx[i] = snew[r];
            }
        }
        wsync();
    }
    if (act) {
        // zero the stages past the horizon, write the shared-Q sum
        for (int e = n * NX + L.l; e < P.N * NX; e += TPI) A.dxref[b * P.N * NX + e] = T(0);
        if (P.Nq > 1) {
            for (int e = n * NX + L.l; e < P.Nq * NX; e += TPI) A.dQ[b * P.Nq * NX + e] = T(0);
        } else {
            for (int i = L.l; i < NX; i += TPI) A.dQ[b * NX + i] = S.dQacc[i];
        }
    }
    wsync();
}

template <typename T, int TPI>
__device__ void zero_grads(const Params<T>& P, const AdjArgs<T>& A, int b, const Lanes<TPI>& L, bool act) {
    if (act) {
        for (int e = L.l; e < P.Nq * NX; e += TPI) A.dQ[(size_t)b * P.Nq * NX + e] = T(0);
        for (int e = L.l; e < P.N * NX; e += TPI) A.dxref[(size_t)b * P.N * NX + e] = T(0);
        for (int i = L.l; i < NX; i += TPI) A.dx0[(size_t)b * NX + i] = T(0);
    }
    wsync();
}

}  // namespace camp
