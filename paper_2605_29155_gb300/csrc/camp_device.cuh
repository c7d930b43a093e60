// camp_device.cuh -- device code of the batched differentiable MPC layer
// (box-constrained iLQR forward, adjoint LQR backward), templated on the
// working precision T (float on the product path, double for logic checks).
//
// Mapping: a block of NW warps serves a pack of up to 32 instances, one
// instance per lane: lane l of every warp works on instance l of the pack, and
// the warps split each instance's work between them.  The serial parts of the
// method (the per-stage box QP, each line-search rollout, the adjoint forward
// sweep) thus run 32 instances per warp instruction, and the parallel parts
// (the 11 computed columns of the RK4 Jacobian, the 13x13 / 17x17 Riccati
// products, the gain columns) are divided between the warps.  Per-instance
// matrices live in shared memory as [row][lane] arrays (conflict-free: lane l
// reads word l of a row); per-instance trajectories, gains and line-search
// candidates live in a global scratch laid out by groups of 32 positions
// ([group][stage][row][32]), so every warp access to them is one or two
// 128-byte lines.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace camp {

constexpr int NX = 13, NU = 4, NZ = 17;
constexpr int NGC = 11, NTC = 6;       // computed / constant columns of F_t = [A_t B_t]
constexpr int NFC = NGC * NX;          // entries of the computed columns
constexpr int NV = NX * (NX + 1) / 2;  // packed upper triangle of V (13 x 13)
constexpr int NQ = NZ * (NZ + 1) / 2;  // packed upper triangle of Q (17 x 17)
constexpr int NL = 14;                 // masked Cholesky factor of Q_uu: packed lower 4x4 (10) + 1/diag (4)
constexpr int GW = 32;                 // positions per group of the global scratch and tape layouts
constexpr int QP_MAX_IT = 20, QP_MAX_LS = 30;
constexpr unsigned FULL = 0xffffffffu;

// Per-stage record of the global scratch (rows of GW positions):
// nominal x (hi, lo), u, the cost rows Q_t, x_ref,t, then the gains K_t, k_t.
constexpr int R_X = 0, R_XL = 13, R_U = 26, R_Q = 30, R_XR = 43, CST = 56, R_K = 56, R_KK = 108, SREC = 112;
constexpr int CREC = 30;               // line-search candidate per stage: x hi, x lo, u
// Tape record per stage (rows of GW instances): computed columns of F_t,
// K_t (row-major), masked factor, free mask.
constexpr int T_F = 0, T_K = 143, T_L = 195, T_M = 209, TREC = 210;

enum { ST_CONVERGED = 0, ST_STALLED = 1, ST_MAX_ITER = 2, ST_NONFINITE = 3, ST_NONPD = 4,
       ST_RUNNING = -1 };

template <typename T> struct Model {
    T h, inv_m, g;
    T Jx, Jy, Jz, iJx, iJy, iJz;
    T M[3][4];                          // torque map tau = M u
    T TJ[3][4];                         // J^-1 M: body-rate rows of B_c
    T gyr[3];                           // (Jz - Jy)/Jx, (Jx - Jz)/Jy, (Jy - Jx)/Jz
};

// The quadrotor constants in the working precision.  X layout, rotors FR, RL,
// FL, RR at (+-d, +-d) with d = arm / sqrt(2), spins (+1, +1, -1, -1):
// tau_x = sum y_i u_i, tau_y = -sum x_i u_i, tau_z = kappa sum s_i u_i.
template <typename T>
inline void fill_model(Model<T>& m, double dt, double mass, const double* inertia, double arm, double kappa,
                       double gravity) {
    m.h = (T)dt;
    m.inv_m = (T)(1.0 / mass);
    m.g = (T)gravity;
    m.Jx = (T)inertia[0];
    m.Jy = (T)inertia[1];
    m.Jz = (T)inertia[2];
    m.iJx = (T)(1.0 / inertia[0]);
    m.iJy = (T)(1.0 / inertia[1]);
    m.iJz = (T)(1.0 / inertia[2]);
    const double d = arm / sqrt(2.0);
    const double rx[4] = {d, -d, d, -d}, ry[4] = {-d, d, d, -d}, sp[4] = {1, 1, -1, -1};
    for (int i = 0; i < 4; ++i) {
        const double Mi[3] = {ry[i], -rx[i], kappa * sp[i]};
        for (int r = 0; r < 3; ++r) {
            m.M[r][i] = (T)Mi[r];
            m.TJ[r][i] = (T)(Mi[r] / inertia[r]);
        }
    }
    m.gyr[0] = (T)((inertia[2] - inertia[1]) / inertia[0]);
    m.gyr[1] = (T)((inertia[0] - inertia[2]) / inertia[1]);
    m.gyr[2] = (T)((inertia[1] - inertia[0]) / inertia[2]);
}

template <typename T> struct Params {
    Model<T> mdl;
    int B, N, Nq, max_iter, n_alpha, store_all, N_ws, ipb;
    T tol;
    T alpha[4];
    const int* horizon;
    const int* order;                   // processing order of the instances (or NULL)
    const T *x0, *Q, *xref, *R, *uref, *ulo, *uhi, *uinit;
    const T *Cg, *cg;                   // general cost of Eq. (2): C [B, NC, 17, 17], c [B, Nc, 17] (or NULL)
    int NC, Nc;
    T *u, *x, *cost;
    int *iters, *status;
    T* tape;
    T *stg, *cand, *kh;                 // global scratch, by position in the processing order
    T* scan;                            // workspace of the stage-parallel Riccati (or NULL)
    int* queue;
};

template <typename T> struct AdjArgs {
    const T *gu, *gx;
    T *dQ, *dxref, *dx0;
    T *dC, *dc;                         // general cost: dL/dC [B, NC, 17, 17], dL/dc [B, Nc, 17]
    int recompute;
};

// The general stage cost of instance b at stage t: C_t (17 x 17, row-major,
// symmetric) and c_t, shared over the stages when NC (Nc) is 1.
template <typename T>
__device__ __forceinline__ const T* Cmat(const Params<T>& P, int b, int t) {
    return P.Cg + ((size_t)b * P.NC + (P.NC > 1 ? t : 0)) * (NZ * NZ);
}
template <typename T>
__device__ __forceinline__ const T* cvec(const Params<T>& P, int b, int t) {
    return P.cg + ((size_t)b * P.Nc + (P.Nc > 1 ? t : 0)) * NZ;
}

// Packed upper-triangular indices (row <= column) of V (13 x 13) and Q (17 x 17).
__host__ __device__ constexpr int vidx(int i, int j) {
    return i <= j ? i * NX - i * (i - 1) / 2 + (j - i) : j * NX - j * (j - 1) / 2 + (i - j);
}
__host__ __device__ constexpr int qidx(int i, int j) {
    return i <= j ? i * NZ - i * (i - 1) / 2 + (j - i) : j * NZ - j * (j - 1) / 2 + (i - j);
}

// The 6 columns of F_t for p and v are constant: position enters nothing
// (F[:, p_i] = e_{p_i}) and velocity only the position (F[:, v_i] = e_{v_i} +
// h e_{p_i}, h written as (h/6) * 6 as the RK4 combination forms it).  The
// other 11 columns (q, w, u) are computed; gcol maps 0..10 to them.
__host__ __device__ constexpr int gcol(int jj) { return jj < 4 ? 3 + jj : 6 + jj; }

// ------------------------------------------------------- shared memory ----
// Lanes per pack in shared memory: 32 in FP32; 16 in FP64 (whose records are
// twice as large), plus one spare column that the idle lanes 16..31 of an
// FP64 warp read and write instead of a live instance's.
template <typename T> struct SL {
    static constexpr int W = sizeof(T) == 4 ? 32 : 16;
    static constexpr int A = sizeof(T) == 4 ? 32 : 17;
};

template <typename T> struct RicSmem {
    static constexpr int A = SL<T>::A;
    T F[2][NFC][A];        // computed columns of F_s, F[s & 1][jj * 13 + i]
    T Q[2][NQ][A];         // P_s = C_s + F_s' Q_xx,s+1 F_s, completed in place to Q_s (packed upper)
    T q[2][NZ][A];         // q_s
    T M[NX * NU][A];       // M_t = Q_xu,t L_t^-T (row-major): V_t = Q_xx,t - M_t M_t'
    T N[NZ * NU][A];       // N_s = F_s' M_s+1 (row-major)
    T v[NX][A];            // v_t = q_x,t + Q_xu,t k_t
    T cst[3][CST][A];      // nominal and cost rows of stages s (by s mod 3)
};
template <typename T> struct LsSmem {
    static constexpr int A = SL<T>::A;
    T stg[2][SREC][A];     // a stage's nominal, cost and gain rows (double buffered)
};
template <typename T> struct TapeSmem {
    static constexpr int A = SL<T>::A;
    T rec[2][TREC][A];     // a stage's tape record (double buffered)
};
template <typename T> struct alignas(16) BlockSmem {
    static constexpr int A = SL<T>::A;
    T K[NU * NX][A];       // K_t, row-major
    T k[NU][A];
    T L[NL][A];
    T x0[NX][A];
    T R[NU][A], uref[NU][A], ulo[NU][A], uhi[NU][A];
    T Jc[4][A];            // line search: cost change of each candidate
    T dmax[4][A];          // line search: max |u_hat - u| of each candidate
    T vh[NX][A];           // adjoint value gradient
    T qh[NZ][A];           // adjoint q-hat
    T wa[NZ][A];           // adjoint F_t' vh_{t+1}, formed one stage ahead
    int mask[A];
    int ok[A];
    union {
        RicSmem<T> r;
        LsSmem<T> s;
        TapeSmem<T> tp;
    } u;
};

// General cost with one C shared over the stages (NC = 1): the pack's C is
// staged once into shared memory right after BlockSmem, as [entry][lane] rows
// like the other per-instance matrices (kernels of the general cost are
// launched with this region added to their dynamic shared memory).
template <typename T> constexpr size_t gen_smem_bytes() { return sizeof(T) * (NZ * NZ) * SL<T>::A; }
template <typename T>
__device__ __forceinline__ T* cshared(const BlockSmem<T>& S) {
    return reinterpret_cast<T*>(reinterpret_cast<char*>(const_cast<BlockSmem<T>*>(&S)) + sizeof(BlockSmem<T>));
}

// Entry e = i * 17 + k of an instance's C_t: from the shared-memory copy when
// C is shared over the stages, else from the caller's array (through L1).
template <typename T> struct CView {
    const T* p;
    int stride;
    __device__ __forceinline__ T operator()(int e) const { return p[(size_t)e * stride]; }
};

template <typename T> __device__ __forceinline__ T clampT(T v, T lo, T hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}
template <typename T> __device__ __forceinline__ bool finiteT(T v) { return isfinite(v); }

// Asynchronous 4- or 8-byte global -> shared copies (cp.async): a thread waits
// for its own copies with cp_async_wait_all; a barrier after that makes them
// visible to the block.
template <typename T> __device__ __forceinline__ void cp_async(T* dst, const T* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Drops the L2 lines of `bytes` of dead scratch at p (128-byte aligned)
// without writing them back to HBM; their contents become undefined.  The
// block's threads split the lines; the caller makes sure that no thread still
// reads them and that no other block's data shares them.
__device__ __forceinline__ void l2_discard(void* p, size_t bytes) {
    char* c = (char*)p;
    for (size_t o = (size_t)threadIdx.x * 128; o < bytes; o += (size_t)blockDim.x * 128)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(c + o) : "memory");
}
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
// xi_2 = x + h/2 k1, xi_3 = x + h/2 k2, xi_4 = x + h k3) in sp[8 s .. 8 s + 6],
// and the total thrust in sp[7].
template <typename T>
__device__ __forceinline__ void rk4_stage_points(const Model<T>& m, const T* x, const T* u, T* sp) {
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

// Coefficients of the continuous Jacobian J_c = [A_c B_c] at one RK4 stage
// point (q, w, total thrust th), so that J_c [dx; du] costs about one
// multiply-add per nonzero entry and the coefficients are shared by every
// direction pushed through the same stage point.
template <typename T> struct JcCoef {
    T hq[4], hw[3];                     // quaternion rows: 1/2 q, 1/2 w
    T c7[4], c8[4], c9[4];              // velocity rows, d/dq of (th/m) R(q) e3
    T r7, r8, r9;                       // velocity rows, R(q) e3 / m per unit of total thrust
    T g10y, g10z, g11x, g11z, g12x, g12y;   // body-rate rows, gyroscopic terms
};

template <typename T>
__device__ __forceinline__ void jc_coef(const Model<T>& m, const T* sp8, T th, JcCoef<T>& c) {
    const T qw = sp8[0], qx = sp8[1], qy = sp8[2], qz = sp8[3];
    const T wx = sp8[4], wy = sp8[5], wz = sp8[6];
    c.hq[0] = T(0.5) * qw; c.hq[1] = T(0.5) * qx; c.hq[2] = T(0.5) * qy; c.hq[3] = T(0.5) * qz;
    c.hw[0] = T(0.5) * wx; c.hw[1] = T(0.5) * wy; c.hw[2] = T(0.5) * wz;
    const T a2 = T(2) * (th * m.inv_m);
    c.c7[0] = a2 * qy;  c.c7[1] = a2 * qz;  c.c7[2] = a2 * qw;  c.c7[3] = a2 * qx;
    c.c8[0] = -a2 * qx; c.c8[1] = -a2 * qw; c.c8[2] = a2 * qz;  c.c8[3] = a2 * qy;
    c.c9[0] = a2 * qw;  c.c9[1] = -a2 * qx; c.c9[2] = -a2 * qy; c.c9[3] = a2 * qz;
    c.r7 = (T(2) * (qx * qz + qw * qy)) * m.inv_m;
    c.r8 = (T(2) * (qy * qz - qw * qx)) * m.inv_m;
    c.r9 = (qw * qw - qx * qx - qy * qy + qz * qz) * m.inv_m;
    c.g10y = -m.gyr[0] * wz; c.g10z = -m.gyr[0] * wy;
    c.g11x = -m.gyr[1] * wz; c.g11z = -m.gyr[1] * wx;
    c.g12x = -m.gyr[2] * wy; c.g12y = -m.gyr[2] * wx;
}

// out = J_c [dx; du] with the precomputed coefficients.
template <typename T>
__device__ __forceinline__ void jc_apply(const Model<T>& m, const JcCoef<T>& c, const T* dx, const T* du, T* out) {
    const T dqw = dx[3], dqx = dx[4], dqy = dx[5], dqz = dx[6];
    const T dwx = dx[10], dwy = dx[11], dwz = dx[12];
    out[0] = dx[7]; out[1] = dx[8]; out[2] = dx[9];
    out[3] = -c.hw[0] * dqx - c.hw[1] * dqy - c.hw[2] * dqz - c.hq[1] * dwx - c.hq[2] * dwy - c.hq[3] * dwz;
    out[4] = c.hw[0] * dqw + c.hw[2] * dqy - c.hw[1] * dqz + c.hq[0] * dwx - c.hq[3] * dwy + c.hq[2] * dwz;
    out[5] = c.hw[1] * dqw - c.hw[2] * dqx + c.hw[0] * dqz + c.hq[3] * dwx + c.hq[0] * dwy - c.hq[1] * dwz;
    out[6] = c.hw[2] * dqw + c.hw[1] * dqx - c.hw[0] * dqy - c.hq[2] * dwx + c.hq[1] * dwy + c.hq[0] * dwz;
    const T dth = du[0] + du[1] + du[2] + du[3];
    out[7] = c.c7[0] * dqw + c.c7[1] * dqx + c.c7[2] * dqy + c.c7[3] * dqz + c.r7 * dth;
    out[8] = c.c8[0] * dqw + c.c8[1] * dqx + c.c8[2] * dqy + c.c8[3] * dqz + c.r8 * dth;
    out[9] = c.c9[0] * dqw + c.c9[1] * dqx + c.c9[2] * dqy + c.c9[3] * dqz + c.r9 * dth;
    out[10] = m.TJ[0][0] * du[0] + m.TJ[0][1] * du[1] + m.TJ[0][2] * du[2] + m.TJ[0][3] * du[3]
            + c.g10y * dwy + c.g10z * dwz;
    out[11] = m.TJ[1][0] * du[0] + m.TJ[1][1] * du[1] + m.TJ[1][2] * du[2] + m.TJ[1][3] * du[3]
            + c.g11x * dwx + c.g11z * dwz;
    out[12] = m.TJ[2][0] * du[0] + m.TJ[2][1] * du[1] + m.TJ[2][2] * du[2] + m.TJ[2][3] * du[3]
            + c.g12x * dwx + c.g12y * dwy;
}

// Directional derivative of the RK4 step, F_t [dx; du], by a forward tangent
// through the four stages: d_s = J_c(xi_s) [dx + c_s d_{s-1}; du],
// out = dx + h/6 (d1 + 2 d2 + 2 d3 + d4).  With a unit direction it is one
// column of F_t.
template <typename T>
__device__ __forceinline__ void rk4_tangent(const Model<T>& m, const T* sp, const T* dx, const T* du, T* out) {
    T arg[NX], d[NX], acc[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) arg[i] = dx[i];
    const T th = sp[7];
    const T hh = T(0.5) * m.h;
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        JcCoef<T> jc;
        jc_coef(m, sp + 8 * st, th, jc);
        jc_apply(m, jc, arg, du, d);
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
    for (int i = 0; i < NX; ++i) out[i] = dx[i] + h6 * acc[i];
}

// Columns j[0..NC) of F_t = d RK4 / d(x, u) at (x, u) together: unit
// directions pushed through the four RK4 stages side by side,
//   d_s = J_c(xi_s) [e_j + c_s d_{s-1}; e_u],  col = e_j + h/6 (d1 + 2 d2 + 2 d3 + d4),
// with the stage points xi_1 = x, xi_{s+1} = x + c_{s+1} f_c(xi_s, u) formed
// on the way.  One loop trip per stage keeps the code small; each stage's
// Jacobian coefficients are formed once for all NC columns, whose chains
// interleave.  j = -1 gives an unused column.
template <typename T, int NC>
__device__ __forceinline__ void tangent_columns(const Model<T>& m, const T (&x)[NX], const T (&u)[NU],
                                                const int (&j)[NC], T (&col)[NC][NX]) {
    T xi[NX], arg[NC][NX], acc[NC][NX], du[NC][NU];
#pragma unroll
    for (int i = 0; i < NX; ++i) xi[i] = x[i];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { arg[k][i] = (i == j[k]) ? T(1) : T(0); acc[k][i] = T(0); }
#pragma unroll
        for (int a = 0; a < NU; ++a) du[k][a] = (NX + a == j[k]) ? T(1) : T(0);
    }
    const T th = u[0] + u[1] + u[2] + u[3];
    const T hh = T(0.5) * m.h;
#pragma unroll 1
    for (int st = 0; st < 4; ++st) {
        JcCoef<T> c;
        const T sp8[8] = {xi[3], xi[4], xi[5], xi[6], xi[10], xi[11], xi[12], th};
        jc_coef(m, sp8, th, c);
        const T w = (st == 0 || st == 3) ? T(1) : T(2);
        const T cs = (st < 2) ? hh : m.h;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            T d[NX];
            jc_apply(m, c, arg[k], du[k], d);
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                acc[k][i] = (st == 0) ? d[i] : acc[k][i] + w * d[i];
                arg[k][i] = ((i == j[k]) ? T(1) : T(0)) + cs * d[i];
            }
        }
        if (st < 3) {
            T kf[NX];
            f_cont(m, xi, u, kf);
#pragma unroll
            for (int i = 0; i < NX; ++i) xi[i] = x[i] + cs * kf[i];
        }
    }
    const T h6 = m.h / T(6);
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
        for (int i = 0; i < NX; ++i) col[k][i] = ((i == j[k]) ? T(1) : T(0)) + h6 * acc[k][i];
}

template <typename T> __device__ __forceinline__ T hv_coef(const Model<T>& m) { return (m.h / T(6)) * T(6); }

// ------------------------------------------------------------- box QP ------
// Packed lower-triangular index of a 4x4 factor.
__host__ __device__ constexpr int lidx(int i, int j) { return i * (i + 1) / 2 + j; }

// Pivot of the Cholesky factor: l = sqrt(s) and 1 / l.  In FP32 from the
// hardware reciprocal square root (a few ulp; the factor's error stays orders
// of magnitude below the FP32 path's tolerances, and the box QP's serial chain
// is the critical path of a Riccati stage); in FP64 correctly rounded.
__device__ __forceinline__ void pivot(float s, float& l, float& il) {
    il = rsqrtf(s);
    l = s * il;
}
__device__ __forceinline__ void pivot(double s, double& l, double& il) {
    l = sqrt(s);
    il = 1.0 / l;
}

// Cholesky of H with the rows/columns outside `mask` replaced by the identity:
// the free block is factored exactly, clamped dimensions decouple.  L[10 + j]
// holds 1 / L_jj so that the solves multiply instead of divide.  Straight-line
// code (selects, no branches), so the lanes of a warp -- different instances
// with different free sets -- never diverge here.  Returns false when a free
// pivot is not positive (the factor is then meaningless).
template <typename T>
__device__ __forceinline__ bool chol_masked(const T (&H)[4][4], int mask, T (&L)[NL]) {
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool fj = (mask >> j) & 1;
        T s = H[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[lidx(j, k)] * L[lidx(j, k)];
        const bool pos = s > T(0);
        ok = ok && (pos || !fj);
        T ljj, ij;
        pivot(fj && pos ? s : T(1), ljj, ij);
        L[lidx(j, j)] = fj ? ljj : T(1);
        L[10 + j] = fj ? ij : T(1);
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            T t = H[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[lidx(i, k)] * L[lidx(j, k)];
            L[lidx(i, j)] = (fj && ((mask >> i) & 1)) ? t * ij : T(0);
        }
    }
    return ok;
}

// Solve (L L') y = b with a masked factor (b must be 0 on clamped dimensions).
template <typename T>
__device__ __forceinline__ void chol_solve4(const T (&L)[NL], const T (&b)[4], T (&y)[4]) {
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

template <typename T> __device__ __forceinline__ void identity_factor(T (&L)[NL]) {
#pragma unroll
    for (int i = 0; i < NL; ++i) L[i] = T(0);
    L[0] = L[2] = L[5] = L[9] = L[10] = L[11] = L[12] = L[13] = T(1);
}

// Projected-Newton box QP (Tassa et al. 2014, Bertsekas 1982):
//   min 1/2 d'Hd + g'd  s.t. lo <= d <= hi,  start d = clamp(0).
// Clamped set: Bertsekas' epsilon-active set -- within eps_i = 1e-6 (1 + hi_i
// - lo_i) of a bound with the gradient pointing out of the box; such a
// dimension is set onto the bound and the gradient re-evaluated there (an
// exact comparison would let a rounding error decide whether a control on its
// bound is free, and with it the whole step).  Newton step on the free set,
// projected onto the box, Armijo backtracking (0.1, x0.6).
// Stops with no free dimension, or when the free set repeats after a full step
// the projection did not cut, or after QP_MAX_IT iterations.  Returns false on
// a non-positive pivot.  `L` and `mask` describe the last factored free set.
//
// Called by all 32 lanes of a warp (one instance each; `on` false for lanes
// without a problem).  Every lane runs the same straight-line iteration and
// keeps or discards its result by selects; the loop ends when every lane has
// stopped, and only the rare backtracking beyond the full step branches.
template <typename T>
__device__ bool box_qp(bool on, const T (&H)[4][4], const T (&g)[4], const T (&lo)[4], const T (&hi)[4],
                       T (&d)[4], T (&L)[NL], int& mask_out) {
    T eps[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        d[i] = clampT(T(0), lo[i], hi[i]);
        eps[i] = T(1e-6) * (T(1) + (hi[i] - lo[i]));
    }
    int free_prev = -1, mask_fact = 0;
    bool last_full = false, done = !on, ok = true;
    identity_factor(L);
    mask_out = 0;
    for (int it = 0; it < QP_MAX_IT; ++it) {
        if (__all_sync(FULL, done)) break;
        T grad[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            T s = g[i];
#pragma unroll
            for (int k = 0; k < 4; ++k) s += H[i][k] * d[k];
            grad[i] = s;
        }
        int fm = 0;
        bool moved = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool al = d[i] <= lo[i] + eps[i] && grad[i] > T(0);
            const bool ah = d[i] >= hi[i] - eps[i] && grad[i] < T(0);
            const T dc = al ? lo[i] : (ah ? hi[i] : d[i]);
            moved = moved || (!done && dc != d[i]);
            d[i] = done ? d[i] : dc;
            fm |= (al || ah) ? 0 : (1 << i);
        }
        if (__any_sync(FULL, moved)) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                T s = g[i];
#pragma unroll
                for (int k = 0; k < 4; ++k) s += H[i][k] * d[k];
                grad[i] = s;
            }
        }
        const bool none_free = fm == 0;
        const bool repeat = last_full && fm == free_prev;
        if (__all_sync(FULL, done || none_free || repeat)) {
            // Every lane stops in this trip without a new factor (typically
            // the trip that confirms a free set): the outcomes the full trip
            // below would select, without its factorization and line search.
            if (!done) {
                if (none_free) identity_factor(L);
                mask_out = none_free ? 0 : fm;
            }
            done = true;
            break;
        }
        T Ln[NL];
        const bool pd = chol_masked(H, fm, Ln);
        T rhs[4], dn[4], dir[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            T s = g[i];
#pragma unroll
            for (int k = 0; k < 4; ++k) s = ((fm >> k) & 1) ? s : s + H[i][k] * d[k];
            rhs[i] = ((fm >> i) & 1) ? -s : T(0);
        }
        chol_solve4(Ln, rhs, dn);
#pragma unroll
        for (int i = 0; i < 4; ++i) dir[i] = ((fm >> i) & 1) ? dn[i] - d[i] : T(0);
        const T phi0 = qp_value(H, g, d);
        T step = T(1), trial[4], dnew[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) { trial[i] = d[i] + dir[i]; dnew[i] = clampT(trial[i], lo[i], hi[i]); }
        T gd = T(0);
#pragma unroll
        for (int i = 0; i < 4; ++i) gd += grad[i] * (dnew[i] - d[i]);
        bool acc = qp_value(H, g, dnew) - phi0 <= T(0.1) * gd;
        const bool live = !done && !none_free && !repeat && pd;
        // Backtracking beyond the full step: the trial steps 0.6^k are tried
        // four at a time (side by side), and the first that satisfies the
        // Armijo condition is taken -- the same step, in the same order, as
        // trying them one by one.
        if (__any_sync(FULL, live && !acc)) {
            for (int ls0 = 1; ls0 < QP_MAX_LS; ls0 += 4) {
                if (!__any_sync(FULL, live && !acc)) break;
                T st[4], tr[4][4], dn4[4][4];
                bool ac[4];
                T s = step;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    s *= T(0.6);
                    st[k] = s;
                    T gd2 = T(0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        tr[k][i] = d[i] + s * dir[i];
                        dn4[k][i] = clampT(tr[k][i], lo[i], hi[i]);
                        gd2 += grad[i] * (dn4[k][i] - d[i]);
                    }
                    ac[k] = ls0 + k < QP_MAX_LS && qp_value(H, g, dn4[k]) - phi0 <= T(0.1) * gd2;
                }
                if (live && !acc) {
                    int kk = 4;
#pragma unroll
                    for (int k = 3; k >= 0; --k) kk = ac[k] ? k : kk;
                    const int kt = kk < 4 ? kk : 3;     // the last trial when none passed
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (k == kt) {
                            step = st[k];
#pragma unroll
                            for (int i = 0; i < 4; ++i) { trial[i] = tr[k][i]; dnew[i] = dn4[k][i]; }
                        }
                    }
                    acc = kk < 4;
                }
            }
        }
        bool inside = true, strict = true;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            inside = inside && (trial[i] >= lo[i]) && (trial[i] <= hi[i]);
            strict = strict && (trial[i] > lo[i]) && (trial[i] < hi[i]);
        }
        // outcome of this iteration for a lane still running, by selects:
        //   nothing free -> stop with the identity factor and mask 0;
        //   the free set repeats after a full step -> stop (last factor kept);
        //   otherwise the new factor is kept, and a non-positive pivot stops
        //   (not ok), a failed line search stops, an accepted step moves d and
        //   stops when it is a full step strictly inside with all free
        const bool run = !done;
        const bool fac = run && !none_free && !repeat;
        const bool step_ok = fac && pd && acc;
        const bool full = (step == T(1)) && inside;
        const bool stop_new = step_ok && full && strict && fm == 15;
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const T idv = (i == 0 || i == 2 || i == 5 || i == 9 || i >= 10) ? T(1) : T(0);
            L[i] = (run && none_free) ? idv : (fac ? Ln[i] : L[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) d[i] = step_ok ? dnew[i] : d[i];
        mask_fact = fac ? fm : mask_fact;
        last_full = step_ok ? full : last_full;
        free_prev = step_ok ? fm : free_prev;
        if (run) {
            if (none_free) mask_out = 0;
            else if (repeat || !pd || !acc || stop_new) mask_out = fm;
        }
        ok = ok && !(fac && !pd);
        done = done || none_free || repeat || (fac && (!pd || !acc)) || stop_new;
    }
    if (!done) mask_out = mask_fact;
    return ok;
}


// ------------------------------------------------------------ work split ----
// Which warp does what, for NW = 4 or 8 warps per block.  Computed columns
// are numbered jj = 0..10 (gcol(jj) is the column of F_t / Q_t).  While warp 0
// solves stage t's box QPs, warps 1..NW-1 form P_{t-1} and the tangent
// columns of F_{t-2}:
//   pcol(w, s)   the computed columns j of P_{t-1} warp w forms (its column
//                of W = Q_xx F and the entries of P in rows of columns <= j);
//                column jj costs about 169 + 13 jj multiply-adds
//   CONST_W      the warp that forms the block of the constant p, v rows/columns
//   tcol(w, s)   the tangent columns warp w computes
// Warp 0 takes neither.  The steps after the QP split their columns / rows
// round-robin over all NW warps.
// The tables, by warp.  Warp 0 solves the box QPs and takes neither; with 8
// warps per block warp 4, which shares warp 0's scheduler, takes none either,
// so that the QPs -- the critical path of a stage -- issue unhindered.
__constant__ int c_pcol4[4][4] = {{-1, -1, -1, -1}, {10, 7, 4, 1}, {9, 6, 3, 0}, {8, 5, 2, -1}};
__constant__ int c_tcol4[4][4] = {{-1, -1, -1, -1}, {0, 1, 2, 3}, {4, 5, 6, 7}, {8, 9, 10, -1}};
__constant__ int c_pcol8[8][2] = {{-1, -1}, {10, 0}, {9, 1}, {8, 2}, {-1, -1}, {7, 3}, {6, 4}, {5, -1}};
__constant__ int c_tcol8[8][2] = {{-1, -1}, {0, 1}, {2, 3}, {4, 5}, {-1, -1}, {6, 7}, {8, 9}, {10, -1}};

template <int NW> struct Split;
template <> struct Split<4> {
    static constexpr int NP = 4, NT = 4, CONST_W = 3;
    __device__ static int pcol(int w, int s) { return c_pcol4[w][s]; }
    __device__ static int tcol(int w, int s) { return c_tcol4[w][s]; }
};
template <> struct Split<8> {
    static constexpr int NP = 2, NT = 2, CONST_W = 7;
    __device__ static int pcol(int w, int s) { return c_pcol8[w][s]; }
    __device__ static int tcol(int w, int s) { return c_tcol8[w][s]; }
};

// ------------------------------------------------------------ lanes --------
// The calling thread's place: warp w of NW, lane l = instance l of the pack,
// its shared-memory column sl (l, or the spare column for an FP64 lane past
// the pack), its position pos in the processing order (scratch index) and
// instance b.
struct Lane {
    int w, l, sl, pos, b;
    bool valid;
};

template <typename T>
__device__ __forceinline__ CView<T> cview(const Params<T>& P, const BlockSmem<T>& S, const Lane& L, int t) {
    if (P.NC == 1) return CView<T>{cshared(S) + L.sl, SL<T>::A};
    return CView<T>{Cmat(P, L.b, t), 1};
}

// Scratch row e of stage t for position pos ([group][stage][row][GW]).
template <typename T>
__device__ __forceinline__ size_t srow(const Params<T>& P, int pos, int t, int e) {
    return (((size_t)(pos / GW) * P.N_ws + t) * SREC + e) * GW + (pos % GW);
}
template <typename T>
__device__ __forceinline__ size_t crow(const Params<T>& P, int c, int pos, int t, int e) {
    const size_t groups = ((size_t)P.B + GW - 1) / GW;
    return ((((size_t)c * groups + pos / GW) * P.N_ws + t) * CREC + e) * GW + (pos % GW);
}
template <typename T>
__device__ __forceinline__ size_t khrow(const Params<T>& P, int pos, int t, int a) {
    return (((size_t)(pos / GW) * P.N_ws + t) * NU + a) * GW + (pos % GW);
}
// Tape row e of stage t for instance b ([group of GW instances][stage][row][GW]).
template <typename T>
__device__ __forceinline__ size_t trow(const Params<T>& P, int b, int t, int e) {
    return (((size_t)(b / GW) * P.N + t) * TREC + e) * GW + (b % GW);
}

template <typename T>
__device__ __forceinline__ const T* Qrow(const Params<T>& P, int b, int t) {
    return P.Q + ((size_t)b * P.Nq + (P.Nq > 1 ? t : 0)) * NX;
}

// The pack's per-instance constants into shared memory (rows split by warp);
// with a general cost shared over the stages, also C.
template <typename T, int NW, bool GEN>
__device__ void load_constants(const Params<T>& P, BlockSmem<T>& S, const Lane& L) {
    if constexpr (GEN) {
        if (L.valid && P.NC == 1) {
            T* Cs = cshared(S);
            const T* Cg = P.Cg + (size_t)L.b * (NZ * NZ);
            for (int e = L.w; e < NZ * NZ; e += NW) Cs[e * SL<T>::A + L.sl] = Cg[e];
        }
    }
    if (L.valid) {
        for (int e = L.w; e < NX + 4 * NU; e += NW) {
            if (e < NX) {
                S.x0[e][L.sl] = P.x0[(size_t)L.b * NX + e];
            } else {
                const int r = e - NX, q = r >> 2, a = r & 3;
                const T* src = q == 0 ? P.R : (q == 1 ? P.uref : (q == 2 ? P.ulo : P.uhi));
                T(*dst)[SL<T>::A] = q == 0 ? S.R : (q == 1 ? S.uref : (q == 2 ? S.ulo : S.uhi));
                dst[a][L.sl] = src[(size_t)L.b * NU + a];
            }
        }
    }
}

// The cost rows Q_t, x_ref,t of every stage t < n into the scratch records
// (stages split by warp).  With `nominal` also x*, u* from the solution
// outputs as the nominal (x lo = 0): the backward's re-factorization point.
template <typename T, int NW, bool GEN>
__device__ void load_stage_rows(const Params<T>& P, const Lane& L, int n, bool nominal) {
    if (!L.valid) return;
    for (int t = L.w; t < n; t += NW) {
        T* dr = P.stg + srow(P, L.pos, t, 0);
        T buf[2 * NX];
        if constexpr (GEN) {
            // the diagonal cost rows are not used with a general cost: they
            // hold c_t instead (rows R_Q .. R_Q + 16), the rest zeros
            const T* cv = cvec(P, L.b, t);
#pragma unroll
            for (int i = 0; i < 2 * NX; ++i) buf[i] = i < NZ ? cv[i] : T(0);
        } else {
            const T* q = Qrow(P, L.b, t);
            const T* xr = P.xref + ((size_t)L.b * P.N + t) * NX;
#pragma unroll
            for (int i = 0; i < NX; ++i) { buf[i] = q[i]; buf[NX + i] = xr[i]; }
        }
        if (nominal) {
            const T* xs = P.x + ((size_t)L.b * P.N + t) * NX;
            const T* us = P.u + ((size_t)L.b * P.N + t) * NU;
            T nb[NX + NU];
#pragma unroll
            for (int i = 0; i < NX; ++i) nb[i] = xs[i];
#pragma unroll
            for (int a = 0; a < NU; ++a) nb[NX + a] = us[a];
#pragma unroll
            for (int i = 0; i < NX; ++i) { dr[(R_X + i) * GW] = nb[i]; dr[(R_XL + i) * GW] = T(0); }
#pragma unroll
            for (int a = 0; a < NU; ++a) dr[(R_U + a) * GW] = nb[NX + a];
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) { dr[(R_Q + i) * GW] = buf[i]; dr[(R_XR + i) * GW] = buf[NX + i]; }
    }
}

// --------------------------------------------------------- A1 rollout -------
// U^0 = clamp(u_init or u_ref), X^0 by RK4 from x_init, J^0 (warp 0; the
// state is carried as hi + lo).  Writes the nominal records; returns J^0 in
// S.Jc[0] for the block (after the caller's barrier).
template <typename T, int NW, bool GEN>
__device__ void initial_rollout(const Params<T>& P, BlockSmem<T>& S, const Lane& L, int n) {
    if (L.w != 0) return;
    T J = T(0);
    if (n > 0) {
        const int sl = L.sl;
        T xh[NX], xl[NX], us[NU], R[NU], ur[NU], lo[NU], hi[NU];
#pragma unroll
        for (int i = 0; i < NX; ++i) { xh[i] = S.x0[i][sl]; xl[i] = T(0); }
#pragma unroll
        for (int a = 0; a < NU; ++a) {
            R[a] = S.R[a][sl]; ur[a] = S.uref[a][sl]; lo[a] = S.ulo[a][sl]; hi[a] = S.uhi[a][sl];
        }
        for (int t = 0; t < n; ++t) {
            T* sr = P.stg + srow(P, L.pos, t, 0);
            T qv[NX], xr[NX], u0[NU];
#pragma unroll
            for (int i = 0; i < NX; ++i) { qv[i] = sr[(R_Q + i) * GW]; xr[i] = sr[(R_XR + i) * GW]; }
#pragma unroll
            for (int a = 0; a < NU; ++a) u0[a] = P.uinit ? P.uinit[((size_t)L.b * P.N + t) * NU + a] : ur[a];
            T sx = T(0), su = T(0);
#pragma unroll
            for (int a = 0; a < NU; ++a) {
                us[a] = clampT(u0[a], lo[a], hi[a]);
                sr[(R_U + a) * GW] = us[a];
                const T e = us[a] - ur[a];
                su += e * (R[a] * e);
            }
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                sr[(R_X + i) * GW] = xh[i];
                sr[(R_XL + i) * GW] = xl[i];
                const T e = (xh[i] - xr[i]) + xl[i];
                sx += e * (qv[i] * e);
            }
            if constexpr (GEN) {
                // 1/2 z' C z + c' z = sum_i z_i (1/2 (C z)_i + c_i)
                const CView<T> Cm = cview(P, S, L, t);
                T cv[NZ];
#pragma unroll
                for (int i = 0; i < NZ; ++i) cv[i] = sr[(R_Q + i) * GW];
                T z[NZ];
#pragma unroll
                for (int i = 0; i < NX; ++i) z[i] = xh[i] + xl[i];
#pragma unroll
                for (int a = 0; a < NU; ++a) z[NX + a] = us[a];
                T sz = T(0);
#pragma unroll
                for (int i = 0; i < NZ; ++i) {
                    T cz = T(0);
#pragma unroll
                    for (int k = 0; k < NZ; ++k) cz += Cm(i * NZ + k) * z[k];
                    sz += z[i] * (T(0.5) * cz + cv[i]);
                }
                J += sz;
            } else {
                J += T(0.5) * sx + T(0.5) * su;
            }
            if (t < n - 1) rk4_step2(P.mdl, xh, xl, us);
        }
    }
    S.Jc[0][L.sl] = J;
}

// ---------------------------------------------- A3 Riccati with box QP ------
// Sec. IV-2, t = n-1 .. 0 with V_n = 0, v_n = 0:
//   Q_t = C_t + F_t' V_{t+1} F_t,   q_t = (C_t z_t + c_t) + F_t' v_{t+1}
//   k_t, free set <- box QP(Q_uu, q_u, u_lo - u_t, u_hi - u_t)
//   K_t = -Q_uu,ff^-1 Q_ux,f on free rows, 0 on clamped rows
//   V_t = Q_xx + Q_xu K_t,   v_t = q_x + Q_xu k_t
// with the linearization of Sec. IV-1 fused in (the tangent columns of F_s
// are formed in the sweep, never stored outside shared memory).
//
// Pipelining.  With L_t the Cholesky factor of the free block of Q_uu,t and
// M_t = Q_xu,t L_t^-T (zero columns for clamped controls), Q_xu K_t = -M_t M_t',
// so V_t = Q_xx,t - M_t M_t' and
//   Q_{t-1} = P_{t-1} - N_{t-1} N_{t-1}',  P_{t-1} = C_{t-1} + F_{t-1}' Q_xx,t F_{t-1},
//   N_{t-1} = F_{t-1}' M_t,  q_{t-1} = c_{t-1} + F_{t-1}' v_t.
// P_{t-1} does not depend on stage t's box QP, so it is formed while warp 0
// solves the QPs; after them only the short steps M_t, K_t, v_t, then
// N_{t-1}, q_{t-1} remain before stage t-1's QP can start.  Stage t runs as
//   phase 1  warp 0: Q_uu,t = P_uu - N_u N_u', box QP (k_t, free set, factor);
//            warps 1..NW-1: P_{t-1} (from Q_xx,t = P_xx - N_x N_x' formed on
//            load) and the tangent columns of F_{t-2};
//   phase 2  columns of M_t, K_t and v_t, with Q_xu,t = P_xu - N_x N_u' formed
//            on load (gains to the scratch for the line search);
//   phase 3  rows of N_{t-1} and q_{t-1}; on request the tape rows;
// separated by block barriers, plus the adjoint step on request.  Quantities
// of stages past an instance's horizon are exact zeros, so that its last
// stage starts from V = 0, v = 0 (Q = C, q = c).
// Options:
//   use_lo   cost gradient at the hi + lo nominal (iterations); otherwise at
//            x* as returned (the factorization the backward differentiates)
//   tape     also store F_t, K_t, the masked factor and the free mask
//   adj      the adjoint backward step after each stage
//   replay   no recursion: each stage's F_t, K_t, factor and free mask come
//            from the tape (copied to shared memory one stage ahead) for the
//            adjoint step
// Every sweep of the method -- iterations, final factorization, backward
// re-factorization, tape replay -- runs through this one function from one
// call site, so the same arithmetic gives the same bits in every mode.
// Returns false for an instance whose free block of Q_uu is not positive
// definite; its remaining stages are skipped.
template <typename T> struct RicOpts {
    T* tape;
    const AdjArgs<T>* adj;
    bool use_lo;
    bool replay;
};

// Writes the tangent columns of F_s this warp owns, or zeros when s is the
// instance's last stage (no dynamics: with F = 0 and V_{s+1} = 0 the stage
// reduces to Q = C, q = c).
template <typename T, int NW>
__device__ __forceinline__ void tangent_step(const Params<T>& P, BlockSmem<T>& S, const Lane& L, int s, int n,
                                             bool on) {
    constexpr int A = SL<T>::A;
    if (s < 0) return;
    const bool dyn = on && s < n - 1;
    const bool last = on && s == n - 1;
    T* Fd = &S.u.r.F[s & 1][0][L.sl];
    constexpr int NT = Split<NW>::NT;
    int jj[NT], jc[NT];
    bool any = false;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        jj[k] = Split<NW>::tcol(L.w, k);
        jc[k] = jj[k] < 0 ? -1 : gcol(jj[k]);
        any = any || jj[k] >= 0;
    }
    if (!any) return;
    if (dyn) {
        const T* cs = &S.u.r.cst[s % 3][0][L.sl];
        T xs[NX], us[NU];
#pragma unroll
        for (int i = 0; i < NX; ++i) xs[i] = cs[(R_X + i) * A];
#pragma unroll
        for (int a = 0; a < NU; ++a) us[a] = cs[(R_U + a) * A];
        T col[NT][NX];
        tangent_columns<T, NT>(P.mdl, xs, us, jc, col);
#pragma unroll
        for (int k = 0; k < NT; ++k) {
            if (jj[k] < 0) continue;
#pragma unroll
            for (int i = 0; i < NX; ++i) Fd[(jj[k] * NX + i) * A] = col[k][i];
        }
    } else if (last) {
#pragma unroll
        for (int k = 0; k < NT; ++k) {
            if (jj[k] < 0) continue;
#pragma unroll
            for (int i = 0; i < NX; ++i) Fd[(jj[k] * NX + i) * A] = T(0);
        }
    }
}

// Cost row j of stage s: C_jj and (C z + c)_j at the nominal z (x as hi + lo
// with use_lo).  GEN: the general C_s, c_s of Eq. (2) (read from the input).
template <typename T, bool GEN>
__device__ __forceinline__ void cost_row(const Params<T>& P, const BlockSmem<T>& S, const T* cs, const Lane& L,
                                         int s, int j, bool use_lo, T& Cd, T& c) {
    constexpr int A = SL<T>::A;
    const int sl = L.sl;
    if constexpr (GEN) {
        const CView<T> Cm = cview(P, S, L, s);
        T acc = cs[(R_Q + j) * A];
#pragma unroll
        for (int k = 0; k < NX; ++k)
            acc += Cm(j * NZ + k) * (use_lo ? cs[(R_X + k) * A] + cs[(R_XL + k) * A] : cs[(R_X + k) * A]);
#pragma unroll
        for (int a = 0; a < NU; ++a) acc += Cm(j * NZ + NX + a) * cs[(R_U + a) * A];
        Cd = Cm(j * NZ + j);
        c = acc;
        return;
    }
    if (j < NX) {
        const T q = cs[(R_Q + j) * A];
        const T e = cs[(R_X + j) * A] - cs[(R_XR + j) * A];
        Cd = q;
        c = q * (use_lo ? e + cs[(R_XL + j) * A] : e);
    } else {
        const int a = j - NX;
        Cd = S.R[a][sl];
        c = Cd * (cs[(R_U + a) * A] - S.uref[a][sl]);
    }
}

template <typename T>
__device__ __forceinline__ T dot13(const T (&a)[NX], const T (&b)[NX]) {
    T s0 = a[0] * b[0], s1 = a[1] * b[1], s2 = a[2] * b[2];
#pragma unroll
    for (int k = 3; k < NX; k += 3) {
        s0 += a[k] * b[k];
        if (k + 1 < NX) s1 += a[k + 1] * b[k + 1];
        if (k + 2 < NX) s2 += a[k + 2] * b[k + 2];
    }
    return (s0 + s1) + s2;
}

// Phase 1, warps 1..NW-1: P_s = C_s + F_s' Q_xx,s+1 F_s (all 153 entries)
// into Q[s & 1]; exact zeros for an instance whose stage s is past its
// horizon.  Q_xx,s+1 = P_xx,s+1 - N_x,s+1 N_x,s+1' is formed in registers as
// it is loaded (every warp forms its own copy; nothing waits for a shared
// one); one loop trip per computed column j of this
// warp forms W[:, j] = Q_xx f_j (the reduction index outermost), the diagonal
// entry, the entries in the rows of the constant columns (p_a takes W[p_a],
// v_a takes W[v_a] + hv W[p_a]) and F[:, r]' W[:, j] in the rows of the
// computed columns r < j, two rows per trip.
// GEN: the general C_s of Eq. (2) enters every entry of P_s, not only the
// diagonal.
template <typename T, int NW, bool GEN>
__device__ __forceinline__ void form_p(const Params<T>& P, BlockSmem<T>& S, const Lane& L, int s, bool ons) {
    constexpr int A = SL<T>::A;
    constexpr int NP = Split<NW>::NP;
    const int sl = L.sl;
    const T hv = hv_coef(P.mdl);
    const T* cs = &S.u.r.cst[s % 3][0][sl];
    const T* Fb = &S.u.r.F[s & 1][0][sl];
    const T* Qn = &S.u.r.Q[(s + 1) & 1][0][sl];
    const T* Nb = &S.u.r.N[0][sl];
    T* Ps = &S.u.r.Q[s & 1][0][sl];
    CView<T> Cm{nullptr, 0};
    if constexpr (GEN) Cm = cview(P, S, L, s);
    const bool cw = L.w == Split<NW>::CONST_W;
    if (Split<NW>::pcol(L.w, 0) < 0 && !cw) return;
    T V[NV], nx[NX][NU];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
        for (int a = 0; a < NU; ++a) nx[i][a] = Nb[(i * NU + a) * A];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
        for (int k = i; k < NX; ++k) {
            T v = Qn[qidx(i, k) * A];
#pragma unroll
            for (int a = 0; a < NU; ++a) v -= nx[i][a] * nx[k][a];
            V[vidx(i, k)] = v;
        }
    if (cw) {
        // the block of the constant rows/columns p_a = a, v_a = 7 + a:
        //   P[p_a][p_b] = V[p_a][p_b] (+ C),  P[p_a][v_b] = V[p_a][v_b] + hv V[p_a][p_b],
        //   P[v_a][v_b] = (V[v_a][v_b] + hv V[v_a][p_b]) + hv (V[p_a][v_b] + hv V[p_a][p_b]) (+ C)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            T Cp, cp, Cv, cv;
            cost_row<T, GEN>(P, S, cs, L, s, b, false, Cp, cp);
            cost_row<T, GEN>(P, S, cs, L, s, 7 + b, false, Cv, cv);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const T Vpp = V[vidx(a, b)];
                const T Wpv = V[vidx(a, 7 + b)] + hv * Vpp;
                Ps[qidx(a, 7 + b) * A] = ons ? (GEN ? Cm(a * NZ + 7 + b) + Wpv : Wpv) : T(0);
                if (a <= b) {
                    Ps[qidx(a, b) * A] = ons ? (GEN ? Cm(a * NZ + b) + Vpp : (a == b ? Cp + Vpp : Vpp)) : T(0);
                    const T v2 = (V[vidx(7 + a, 7 + b)] + hv * V[vidx(7 + a, b)]) + hv * Wpv;
                    Ps[qidx(7 + a, 7 + b) * A] =
                        ons ? (GEN ? Cm((7 + a) * NZ + 7 + b) + v2 : (a == b ? Cv + v2 : v2)) : T(0);
                }
            }
        }
    }
#pragma unroll 1
    for (int k = 0; k < NP; ++k) {
        const int jj = Split<NW>::pcol(L.w, k);
        if (jj < 0) break;
        const int j = gcol(jj);
        T f[NX], W[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) { f[i] = Fb[(jj * NX + i) * A]; W[i] = T(0); }
        T Cd, cj;
        cost_row<T, GEN>(P, S, cs, L, s, j, false, Cd, cj);
#pragma unroll
        for (int kk = 0; kk < NX; ++kk)
#pragma unroll
            for (int i = 0; i < NX; ++i) W[i] += V[vidx(i, kk)] * f[kk];
        Ps[qidx(j, j) * A] = ons ? Cd + dot13(f, W) : T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Ps[qidx(a, j) * A] = ons ? (GEN ? Cm(a * NZ + j) + W[a] : W[a]) : T(0);
            const T wv = W[7 + a] + hv * W[a];
            Ps[qidx(7 + a, j) * A] = ons ? (GEN ? Cm((7 + a) * NZ + j) + wv : wv) : T(0);
        }
#pragma unroll 1
        for (int r = 0; r < jj; r += 2) {
            const int r1 = r + 1 < jj ? r + 1 : r;
            T f0[NX], f1[NX];
#pragma unroll
            for (int i = 0; i < NX; ++i) { f0[i] = Fb[(r * NX + i) * A]; f1[i] = Fb[(r1 * NX + i) * A]; }
            const T a0 = dot13(f0, W), a1 = dot13(f1, W);
            Ps[qidx(gcol(r), j) * A] = ons ? (GEN ? Cm(gcol(r) * NZ + j) + a0 : a0) : T(0);
            if (r1 != r) Ps[qidx(gcol(r1), j) * A] = ons ? (GEN ? Cm(gcol(r1) * NZ + j) + a1 : a1) : T(0);
        }
    }
}

// --------------------------------------------- A8 adjoint backward step ----
// One stage of the adjoint LQR's backward sweep (Sec. IV implicit
// differentiation, Amos et al. 2018) on the stage's frozen factorization:
//   qh_t = g_t + F_t' vh_{t+1};  kh_t = -(Q_uu,ff)^-1 qh_u,f (0 on clamped rows);
//   vh_t = qh_x + K_t' qh_u,
// with F_t' vh_{t+1} formed one stage ahead (S.wa; zero at the last stage).
// Kp, Lp point at row 0 of the stage's K_t and masked factor in shared
// memory, Fp at row 0 of F_{t-1}'s computed columns (for S.wa of the next
// stage).  Three barrier-separated steps; the copies of the caller's prefetch
// are waited for before the last.
template <typename T, int NW>
__device__ __forceinline__ void adjoint_step(const Params<T>& P, BlockSmem<T>& S, const Lane& L, int t, int n,
                                             bool go, const AdjArgs<T>& A, const T* Kp, const T* Lp, int mask,
                                             const T* Fp) {
    constexpr int SA = SL<T>::A;
    const int sl = L.sl;
    const T hv = hv_coef(P.mdl);
    if (go) {
        const size_t gxo = ((size_t)L.b * P.N + t) * NX, guo = ((size_t)L.b * P.N + t) * NU;
        for (int j = L.w; j < NZ; j += NW) {
            const T g = j < NX ? (A.gx ? A.gx[gxo + j] : T(0)) : A.gu[guo + j - NX];
            S.qh[j][sl] = g + (t < n - 1 ? S.wa[j][sl] : T(0));
        }
    }
    __syncthreads();
    if (go) {
        T qu[NU];
#pragma unroll
        for (int a = 0; a < NU; ++a) qu[a] = S.qh[NX + a][sl];
        if (L.w == 0) {
            T Lf[NL], rhs[4], y[4];
#pragma unroll
            for (int i = 0; i < NL; ++i) Lf[i] = Lp[i * SA];
#pragma unroll
            for (int a = 0; a < 4; ++a) rhs[a] = ((mask >> a) & 1) ? qu[a] : T(0);
            chol_solve4(Lf, rhs, y);
#pragma unroll
            for (int a = 0; a < 4; ++a) P.kh[khrow(P, L.pos, t, a)] = ((mask >> a) & 1) ? -y[a] : T(0);
        }
        for (int i = L.w; i < NX; i += NW) {
            T s = S.qh[i][sl];
#pragma unroll
            for (int a = 0; a < NU; ++a) s += Kp[(a * NX + i) * SA] * qu[a];
            S.vh[i][sl] = s;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // F_{t-1}' vh_t for the next stage
    if (go && t > 0) {
        T vh[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) vh[i] = S.vh[i][sl];
        for (int j = L.w; j < NZ; j += NW) {
            T s;
            if (j < 3) {
                s = vh[j];
            } else if (j >= 7 && j < 10) {
                s = vh[j] + hv * vh[j - 7];
            } else {
                const int jj = j < 7 ? j - 3 : j - 6;
                T f[NX];
#pragma unroll
                for (int i = 0; i < NX; ++i) f[i] = Fp[(jj * NX + i) * SA];
                s = dot13(f, vh);
            }
            S.wa[j][sl] = s;
        }
    }
    __syncthreads();
}

template <typename T, int NW, bool GEN>
__device__ bool riccati(const Params<T>& P, BlockSmem<T>& S, const Lane& L, int n, const RicOpts<T>& o) {
    constexpr int A = SL<T>::A;
    const int sl = L.sl;
    const T hv = hv_coef(P.mdl);
    const int nmax = __reduce_max_sync(FULL, n);
    // The factorization the backward differentiates forms V_t = Q_xx + Q_xu K_t
    // explicitly after the box QP and P_{t-1} = C + F' V_t F from it (N = 0),
    // which keeps the subtraction of the controlled directions in the 13 x 13
    // value Hessian, where FP32 resolves it best; the iterations use the
    // pipelined form above.
    const bool vform = !o.use_lo;
    bool alive = true;
    // copies of stage tt's nominal and cost rows into cst[tt % 3], and of its
    // tape record into rec[tt & 1] (rows split by warp)
    auto stage_copy = [&](int tt) {
        if (tt >= 0 && tt < n) {
            T* dst = &S.u.r.cst[tt % 3][0][sl];
            const T* src = P.stg + srow(P, L.pos, tt, 0);
            for (int e = L.w; e < CST; e += NW) cp_async(dst + e * A, src + e * GW);
        }
        cp_async_commit();
    };
    auto rec_copy = [&](int tt) {
        if (tt >= 0 && tt < n) {
            T* dst = &S.u.tp.rec[tt & 1][0][sl];
            const T* src = P.tape + trow(P, L.b, tt, 0);
            for (int e = L.w; e < TREC; e += NW) cp_async(dst + e * A, src + e * GW);
        }
        cp_async_commit();
    };
    // replay starts at the last stage; the recursion one stage later, at a
    // stage past every horizon (t = nmax), where everything is zero
    const int t0 = o.replay ? nmax - 1 : nmax;
    if (o.replay) {
        rec_copy(nmax - 1);
        cp_async_wait_all();
        __syncthreads();
    } else {
        for (int e = L.w; e < NQ; e += NW) S.u.r.Q[nmax & 1][e][sl] = T(0);
        for (int e = L.w; e < NZ * NU; e += NW) S.u.r.N[e][sl] = T(0);
        stage_copy(nmax - 1);
        stage_copy(nmax - 2);
        cp_async_wait_all();
        __syncthreads();
        tangent_step<T, NW>(P, S, L, nmax - 1, n, n > 0);
        __syncthreads();
    }
    for (int t = t0; t >= 0; --t) {
        const bool on = alive && t < n;
        // the stage's factorization for the adjoint step: replayed or just formed
        const T *Kp, *Lp, *Fp;
        int amask;
        bool ago;
        if (o.replay) {
            rec_copy(t - 1);
            const T* R = &S.u.tp.rec[t & 1][0][sl];
            Kp = R + T_K * A;
            Lp = R + T_L * A;
            Fp = &S.u.tp.rec[(t + 1) & 1][0][sl] + T_F * A;      // the record of stage t-1
            amask = on ? (int)R[T_M * A] : 0;
            ago = on;
        } else {
            // ---- phase 1
            if (L.w == 0) {
                const T* cs = &S.u.r.cst[t % 3][0][sl];
                const T* Pt = &S.u.r.Q[t & 1][0][sl];
                T H[4][4], g[4], lo[4], hi[4], d[4], Lf[NL], nu[NU][NU];
                int mask = 0;
#pragma unroll
                for (int a = 0; a < NU; ++a)
#pragma unroll
                    for (int b = 0; b < NU; ++b) nu[a][b] = S.u.r.N[(NX + a) * NU + b][sl];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
#pragma unroll
                    for (int b = a; b < 4; ++b) {
                        T s = Pt[qidx(NX + a, NX + b) * A];
#pragma unroll
                        for (int k = 0; k < NU; ++k) s -= nu[a][k] * nu[b][k];
                        H[a][b] = s;
                        H[b][a] = s;
                    }
                    g[a] = S.u.r.q[t & 1][NX + a][sl];
                    const T ub = t < n ? cs[(R_U + a) * A] : T(0);
                    lo[a] = S.ulo[a][sl] - ub;
                    hi[a] = S.uhi[a][sl] - ub;
                }
                const bool ok = box_qp(on, H, g, lo, hi, d, Lf, mask);
                if (on) {
#pragma unroll
                    for (int a = 0; a < 4; ++a) S.k[a][sl] = d[a];
#pragma unroll
                    for (int i = 0; i < NL; ++i) S.L[i][sl] = Lf[i];
                    S.mask[sl] = mask;
                    S.ok[sl] = ok ? 1 : 0;
                }
            } else {
                if (t >= 1 && !vform) form_p<T, NW, GEN>(P, S, L, t - 1, alive && t - 1 < n);
                tangent_step<T, NW>(P, S, L, t - 2, n, alive && n > 0);
            }
            __syncthreads();
            if (on && !S.ok[sl]) alive = false;
            const bool go = on && alive;
            // ---- phase 2: columns c of M_t (forward solves), K_t (back
            // solves) and v_t
            stage_copy(t - 3);
            {
                T Lf[NL], kk[NU];
                const int mask = go ? S.mask[sl] : 0;
#pragma unroll
                for (int i = 0; i < NL; ++i) Lf[i] = S.L[i][sl];
#pragma unroll
                for (int a = 0; a < NU; ++a) kk[a] = S.k[a][sl];
                const T* Qt = &S.u.r.Q[t & 1][0][sl];
                const T* Nb = &S.u.r.N[0][sl];
                T nu[NU][NU];
#pragma unroll
                for (int a = 0; a < NU; ++a)
#pragma unroll
                    for (int b = 0; b < NU; ++b) nu[a][b] = Nb[((NX + a) * NU + b) * A];
                T* grow = go ? P.stg + srow(P, L.pos, t, 0) : nullptr;
#pragma unroll 1
                for (int c0 = L.w; c0 < NX; c0 += 2 * NW) {
                    // two columns c = c0, c0 + NW side by side
                    int cc[2];
                    T qc[2][NU], z[2][NU], y[2][NU], vq[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int c = c0 + h * NW;
                        cc[h] = c < NX ? c : -1;
                        const int cl = c < NX ? c : 0;
                        T nc[NU];
#pragma unroll
                        for (int b = 0; b < NU; ++b) nc[b] = Nb[(cl * NU + b) * A];
#pragma unroll
                        for (int a = 0; a < NU; ++a) {
                            T s = Qt[qidx(cl, NX + a) * A];
#pragma unroll
                            for (int b = 0; b < NU; ++b) s -= nc[b] * nu[a][b];
                            qc[h][a] = s;
                        }
                        vq[h] = S.u.r.q[t & 1][cl][sl];
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        // forward solve L z = qc on the free set (masked factor: clamped rows give 0)
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            T s = ((mask >> i) & 1) ? qc[h][i] : T(0);
#pragma unroll
                            for (int k = 0; k < i; ++k) s -= Lf[lidx(i, k)] * z[h][k];
                            z[h][i] = s * Lf[10 + i];
                        }
                        // back solve L' y = z
#pragma unroll
                        for (int i = 3; i >= 0; --i) {
                            T s = z[h][i];
#pragma unroll
                            for (int k = i + 1; k < 4; ++k) s -= Lf[lidx(k, i)] * y[h][k];
                            y[h][i] = s * Lf[10 + i];
                        }
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int c = cc[h];
                        if (c < 0) continue;
                        T vc = vq[h];
#pragma unroll
                        for (int a = 0; a < NU; ++a) {
                            vc += qc[h][a] * kk[a];
                            const T kc = ((mask >> a) & 1) ? -y[h][a] : T(0);
                            S.u.r.M[c * NU + a][sl] = go ? z[h][a] : T(0);
                            S.K[a * NX + c][sl] = go ? kc : T(0);
                            if (go) grow[(R_K + a * NX + c) * GW] = kc;
                        }
                        S.u.r.v[c][sl] = go ? vc : T(0);
                    }
                }
                if (L.w == 0 && go) {
#pragma unroll
                    for (int a = 0; a < NU; ++a) grow[(R_KK + a) * GW] = kk[a];
                }
            }
            __syncthreads();
            if (vform) {
                // V_t = Q_xx,t + Q_xu,t K_t in place of Q_xx,t (columns c
                // round-robin; in this form N_t = 0, so Q_t = P_t), then
                // P_{t-1} = C + F' V_t F
                T* Qt = &S.u.r.Q[t & 1][0][sl];
#pragma unroll 1
                for (int c = L.w; c < NX; c += NW) {
                    T kc[NU];
#pragma unroll
                    for (int a = 0; a < NU; ++a) kc[a] = S.K[a * NX + c][sl];
#pragma unroll 1
                    for (int i = 0; i <= c; ++i) {
                        T s = Qt[qidx(i, c) * A];
#pragma unroll
                        for (int a = 0; a < NU; ++a) s += Qt[qidx(i, NX + a) * A] * kc[a];
                        Qt[qidx(i, c) * A] = s;
                    }
                }
                __syncthreads();
                if (t >= 1 && L.w >= 1) form_p<T, NW, GEN>(P, S, L, t - 1, alive && t - 1 < n);
            }
            // ---- phase 3: rows j of N_{t-1} = F_{t-1}' M_t (zero in the V form) and q_{t-1} = c_{t-1} + F_{t-1}' v_t
            if (t >= 1) {
                const int s = t - 1;
                const bool ons = alive && s < n;
                const T* cs = &S.u.r.cst[s % 3][0][sl];
                const T* Fb = &S.u.r.F[s & 1][0][sl];
                T Mr[NX][NU], vv[NX];
#pragma unroll
                for (int i = 0; i < NX; ++i) {
                    vv[i] = S.u.r.v[i][sl];
#pragma unroll
                    for (int a = 0; a < NU; ++a) Mr[i][a] = vform ? T(0) : S.u.r.M[i * NU + a][sl];
                }
#pragma unroll 1
                for (int j = L.w; j < NZ; j += NW) {
                    T Cd, c;
                    cost_row<T, GEN>(P, S, cs, L, s, j, o.use_lo, Cd, c);
                    T nj[NU], qj;
                    if (j < 3 || (j >= 7 && j < 10)) {
                        const int p = j < 3 ? j : j - 7;
                        const bool vel = j >= 7;
#pragma unroll
                        for (int a = 0; a < NU; ++a) {
                            const T mj = S.u.r.M[j * NU + a][sl];
                            const T m = vel ? mj + hv * S.u.r.M[p * NU + a][sl] : mj;
                            nj[a] = vform ? T(0) : m;
                        }
                        qj = c + (vel ? S.u.r.v[j][sl] + hv * S.u.r.v[p][sl] : S.u.r.v[j][sl]);
                    } else {
                        const int jj = j < 7 ? j - 3 : j - 6;
                        T f[NX];
#pragma unroll
                        for (int i = 0; i < NX; ++i) f[i] = Fb[(jj * NX + i) * A];
#pragma unroll
                        for (int a = 0; a < NU; ++a) {
                            T mc[NX];
#pragma unroll
                            for (int i = 0; i < NX; ++i) mc[i] = Mr[i][a];
                            nj[a] = dot13(f, mc);
                        }
                        qj = c + dot13(f, vv);
                        if (o.tape && ons) {
#pragma unroll
                            for (int i = 0; i < NX; ++i) o.tape[trow(P, L.b, s, T_F + jj * NX + i)] = f[i];
                        }
                    }
#pragma unroll
                    for (int a = 0; a < NU; ++a) S.u.r.N[j * NU + a][sl] = ons ? nj[a] : T(0);
                    S.u.r.q[s & 1][j][sl] = ons ? qj : T(0);
                }
            }
            if (o.tape && go) {
                const int mask = S.mask[sl];
                for (int e = T_K + L.w; e < TREC; e += NW) {
                    T val;
                    if (e < T_L) val = S.K[e - T_K][sl];
                    else if (e < T_M) val = S.L[e - T_L][sl];
                    else val = T(mask);
                    o.tape[trow(P, L.b, t, e)] = val;
                }
            }
            cp_async_wait_all();
            __syncthreads();
            Kp = &S.K[0][sl];
            Lp = &S.L[0][sl];
            Fp = &S.u.r.F[(t + 1) & 1][0][sl];                       // F_{t-1}
            amask = go ? S.mask[sl] : 0;
            ago = go;
        }
        if (o.adj) adjoint_step<T, NW>(P, S, L, t, n, ago, *o.adj, Kp, Lp, amask, Fp);
    }
    return alive;
}

// ------------------------------------------------- A4 line search ----------
// Sec. IV-3: warp c rolls out candidate alpha_c for every instance of the pack,
//   u_hat_t = clamp(u_t + alpha k_t + K_t (x_hat_t - x_t)),  x_hat_{t+1} = RK4.
// The candidates are compared through their cost change with respect to the
// nominal, accumulated stage by stage from the differences themselves,
//   dJ_t = (x_hat - x)' Q (x - x_ref + (x_hat - x)/2) + (u_hat - u)' R (u - u_ref + (u_hat - u)/2),
// which equals J(alpha) - J exactly for the quadratic cost but does not cancel
// against J's magnitude; with the hi + lo states it resolves differences far
// below the working precision of J.  alpha* = first argmin, and the best
// candidate becomes the next nominal (Sec. IV-3).  Each stage's gains,
// nominal and cost rows are copied into shared memory by all warps one stage
// ahead.  Returns 0 (step taken: du, J updated) or 1 (no candidate with a
// finite cost: nominal kept).
template <typename T, int NW, bool GEN>
__device__ int line_search(const Params<T>& P, BlockSmem<T>& S, const Lane& L, int n, T& Jnom, T& du_out) {
    constexpr int A = SL<T>::A;
    const int sl = L.sl;
    const int nmax = __reduce_max_sync(FULL, n);
    const bool cl = n > 0 && L.w < P.n_alpha;
    const T alpha = L.w == 0 ? P.alpha[0] : (L.w == 1 ? P.alpha[1] : (L.w == 2 ? P.alpha[2] : P.alpha[3]));
    auto issue = [&](int tt) {
        if (tt < n) {
            T* dst = &S.u.s.stg[tt & 1][0][sl];
            const T* src = P.stg + srow(P, L.pos, tt, 0);
            for (int e = L.w; e < SREC; e += NW) cp_async(dst + e * A, src + e * GW);
        }
        cp_async_commit();
    };
    issue(0);
    cp_async_wait_all();
    __syncthreads();
    T xh[NX], xl[NX], R[NU], ur[NU], ulo[NU], uhi[NU];
#pragma unroll
    for (int i = 0; i < NX; ++i) { xh[i] = S.x0[i][sl]; xl[i] = T(0); }
#pragma unroll
    for (int a = 0; a < NU; ++a) {
        R[a] = S.R[a][sl]; ur[a] = S.uref[a][sl]; ulo[a] = S.ulo[a][sl]; uhi[a] = S.uhi[a][sl];
    }
    T dJ = T(0), dJl = T(0), dmx = T(0);
    const int c = L.w & 3;
    for (int t = 0; t < nmax; ++t) {
        issue(t + 1);
        if (cl && t < n) {
            const T* sb = &S.u.s.stg[t & 1][0][sl];
            T dxv[NX], uh[NU];
#pragma unroll
            for (int i = 0; i < NX; ++i) dxv[i] = (xh[i] - sb[(R_X + i) * A]) + (xl[i] - sb[(R_XL + i) * A]);
            T sx = T(0), su = T(0);
#pragma unroll
            for (int a = 0; a < NU; ++a) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < NX; ++i) s += sb[(R_K + a * NX + i) * A] * dxv[i];
                const T ub = sb[(R_U + a) * A];
                const T un = ub + alpha * sb[(R_KK + a) * A] + s;
                uh[a] = clampT(un, ulo[a], uhi[a]);
                const T d = uh[a] - ub;
                su += d * (R[a] * ((ub - ur[a]) + T(0.5) * d));
                const T ad = fabs(d);
                dmx = ad > dmx ? ad : dmx;
            }
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                const T eb = (sb[(R_X + i) * A] - sb[(R_XR + i) * A]) + sb[(R_XL + i) * A];
                sx += dxv[i] * (sb[(R_Q + i) * A] * (eb + T(0.5) * dxv[i]));
            }
            if constexpr (GEN) {
                // d' (C (z + d/2) + c) with the general C_t, c_t
                const CView<T> Cm = cview(P, S, L, t);
                T zh[NZ], dz[NZ];
#pragma unroll
                for (int i = 0; i < NX; ++i) {
                    dz[i] = dxv[i];
                    zh[i] = (sb[(R_X + i) * A] + sb[(R_XL + i) * A]) + T(0.5) * dxv[i];
                }
#pragma unroll
                for (int a = 0; a < NU; ++a) {
                    const T ub = sb[(R_U + a) * A];
                    dz[NX + a] = uh[a] - ub;
                    zh[NX + a] = ub + T(0.5) * dz[NX + a];
                }
                T sg = T(0);
#pragma unroll
                for (int i = 0; i < NZ; ++i) {
                    T r = sb[(R_Q + i) * A];
#pragma unroll
                    for (int k = 0; k < NZ; ++k) r += Cm(i * NZ + k) * zh[k];
                    sg += dz[i] * r;
                }
                acc2(dJ, dJl, sg);
            } else {
                acc2(dJ, dJl, sx + su);
            }
            T* cr = P.cand + crow(P, c, L.pos, t, 0);
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                cr[i * GW] = xh[i];
                cr[(NX + i) * GW] = xl[i];
            }
#pragma unroll
            for (int a = 0; a < NU; ++a) cr[(2 * NX + a) * GW] = uh[a];
            if (t < n - 1) rk4_step2(P.mdl, xh, xl, uh);
        }
        cp_async_wait_all();
        __syncthreads();
    }
    if (cl) {
        dJ = dJ + dJl;
        S.Jc[L.w][sl] = finiteT(dJ) ? dJ : T(INFINITY);
        S.dmax[L.w][sl] = dmx;
    }
    __syncthreads();
    int r = 0;
    if (n > 0) {
        int best = 0;
        T Jb = S.Jc[0][sl];
        for (int k = 1; k < P.n_alpha; ++k)
            if (S.Jc[k][sl] < Jb) { Jb = S.Jc[k][sl]; best = k; }
        if (!finiteT(Jb)) {
            r = 1;
        } else {
            // the best candidate becomes the nominal: all of a stage's loads, then its stores
            for (int t = L.w; t < n; t += NW) {
                const T* cr = P.cand + crow(P, best, L.pos, t, 0);
                T* dr = P.stg + srow(P, L.pos, t, R_X);
                T buf[CREC];
#pragma unroll
                for (int e = 0; e < CREC; ++e) buf[e] = cr[e * GW];
#pragma unroll
                for (int e = 0; e < CREC; ++e) dr[e * GW] = buf[e];
            }
            Jnom = Jnom + Jb;
            du_out = S.dmax[best][sl];
        }
    }
    __syncthreads();
    // The candidates are dead until the next line search writes them again:
    // when the pack owns whole groups of the scratch layout, their lines leave
    // L2 without a write-back.
    const int base = L.pos - L.l;
    if (P.ipb == GW && base % GW == 0) {
        for (int c2 = 0; c2 < P.n_alpha; ++c2)
            l2_discard(P.cand + crow(P, c2, base, 0, 0), (size_t)nmax * CREC * GW * sizeof(T));
    }
    return r;
}

// ---------------------------------------------- A8 adjoint forward sweep ----
// dx_0 = 0; du_t = K_t dx_t + kh_t; dx_{t+1} = F_t [dx_t; du_t], formed as the
// directional derivative of the RK4 step at (x*_t, u*_t) (one forward tangent
// instead of 17 columns); with d_tau_t = [dx_t; du_t]:
//   dQ_t = dx_t * (x*_t - x_ref,t),  dx_ref,t = -Q_t * dx_t,  dx0 = vh_0.
// Warp 0, one instance per lane.  K_t comes from the tape (store-all) or the
// gain records the re-factorization wrote (recompute).  x*_t - x_ref,t is
// formed from the state as the forward carried it, hi + lo, re-rolled here
// from x_init and u* (the returned x* is its rounding): a tracking error much
// smaller than the state keeps its digits.
template <typename T, int NW, bool GEN>
__device__ void adjoint_forward(const Params<T>& P, const BlockSmem<T>& S, const Lane& L, int n,
                                const AdjArgs<T>& A) {
    if (L.w != 0 || n <= 0) return;
    const size_t b = L.b;
    // the sums over the stages of a shared Q (c) are carried as hi + lo
    // (acc2): their terms can cancel to a sum far smaller than themselves
    T dx[NX], dq[NX], dql[NX], dcs[NZ], dcl[NZ], xh[NX], xl[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        dx[i] = T(0); dq[i] = T(0); dql[i] = T(0); A.dx0[b * NX + i] = S.vh[i][L.sl];
        xh[i] = S.x0[i][L.sl]; xl[i] = T(0);
    }
#pragma unroll
    for (int i = 0; i < NZ; ++i) { dcs[i] = T(0); dcl[i] = T(0); }
    for (int t = 0; t < n; ++t) {
        // the stage's operands first
        const T* kr = A.recompute ? P.stg + srow(P, L.pos, t, R_K) : P.tape + trow(P, L.b, t, T_K);
        const T* xs = P.x + (b * P.N + t) * NX;
        T K[NU * NX], kh[NU], xv[NX], xrv[NX], qv[NX], us[NU];
#pragma unroll
        for (int e = 0; e < NU * NX; ++e) K[e] = kr[e * GW];
#pragma unroll
        for (int a = 0; a < NU; ++a) {
            kh[a] = P.kh[khrow(P, L.pos, t, a)];
            us[a] = P.u[(b * P.N + t) * NU + a];
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) xv[i] = xs[i];
        if constexpr (!GEN) {
            const T* xr = P.xref + (b * P.N + t) * NX;
            const T* Qt = Qrow(P, L.b, t);
#pragma unroll
            for (int i = 0; i < NX; ++i) { xrv[i] = xr[i]; qv[i] = Qt[i]; }
        }
        T du[NU];
#pragma unroll
        for (int a = 0; a < NU; ++a) {
            T s = kh[a];
#pragma unroll
            for (int i = 0; i < NX; ++i) s += K[a * NX + i] * dx[i];
            du[a] = s;
        }
        if constexpr (GEN) {
            // dL/dc_t = d_tau_t, dL/dC_t = 1/2 (d_tau_t z*_t' + z*_t d_tau_t')
            T d[NZ], z[NZ];
#pragma unroll
            for (int i = 0; i < NX; ++i) { d[i] = dx[i]; z[i] = xv[i]; }
#pragma unroll
            for (int a = 0; a < NU; ++a) { d[NX + a] = du[a]; z[NX + a] = us[a]; }
            if (P.Nc > 1) {
#pragma unroll
                for (int i = 0; i < NZ; ++i) A.dc[(b * P.Nc + t) * NZ + i] = d[i];
            } else {
#pragma unroll
                for (int i = 0; i < NZ; ++i) acc2(dcs[i], dcl[i], d[i]);
            }
            // d_tau_t and z*_t into the (free) candidate scratch, by position:
            // all warps form dL/dC from them afterwards (assemble_dC)
#pragma unroll
            for (int i = 0; i < NZ; ++i) {
                P.cand[crow(P, 0, L.pos, t, i)] = d[i];
                P.cand[crow(P, 1, L.pos, t, i)] = z[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                const T e = (xh[i] - xrv[i]) + xl[i];
                if (P.Nq > 1) A.dQ[(b * P.Nq + t) * NX + i] = dx[i] * e;
                else acc2(dq[i], dql[i], dx[i] * e);
                A.dxref[(b * P.N + t) * NX + i] = -qv[i] * dx[i];
            }
        }
        if (t < n - 1) {
            T sp[32], nx[NX];
            rk4_stage_points(P.mdl, xv, us, sp);
            rk4_tangent(P.mdl, sp, dx, du, nx);
#pragma unroll
            for (int i = 0; i < NX; ++i) dx[i] = nx[i];
            if constexpr (!GEN) rk4_step2(P.mdl, xh, xl, us);
        }
    }
    if constexpr (GEN) {
        if (P.Nc > 1) {
            for (int e = n * NZ; e < P.Nc * NZ; ++e) A.dc[b * P.Nc * NZ + e] = T(0);
        } else {
#pragma unroll
            for (int i = 0; i < NZ; ++i) A.dc[b * NZ + i] = dcs[i] + dcl[i];
        }
    } else {
        for (int e = n * NX; e < P.N * NX; ++e) A.dxref[b * P.N * NX + e] = T(0);
        if (P.Nq > 1) {
            for (int e = n * NX; e < P.Nq * NX; ++e) A.dQ[b * P.Nq * NX + e] = T(0);
        } else {
#pragma unroll
            for (int i = 0; i < NX; ++i) A.dQ[b * NX + i] = dq[i] + dql[i];
        }
    }
}

// General cost: dL/dC_t = 1/2 (d_tau_t z*_t' + z*_t d_tau_t') from the stage
// vectors adjoint_forward left in the candidate scratch (after a block
// barrier), summed over the stages when C is shared.  The 153 upper entries
// are split over the NW warps and mirrored, so dL/dC is exactly symmetric;
// stages past the horizon get zeros.
template <typename T, int NW>
__device__ void assemble_dC(const Params<T>& P, const AdjArgs<T>& A, const Lane& L, int n) {
    if (!L.valid || n <= 0) return;
    const size_t b = L.b;
    for (int e = L.w; e < NZ * (NZ + 1) / 2; e += NW) {
        int i = 0, r = e;
        while (r >= NZ - i) { r -= NZ - i; ++i; }
        const int k = i + r;
        T acc = T(0), accl = T(0);     // hi + lo sum over the stages of a shared C
        for (int t = 0; t < P.N; ++t) {
            T v = T(0);
            if (t < n) {
                const T di = P.cand[crow(P, 0, L.pos, t, i)], dk = P.cand[crow(P, 0, L.pos, t, k)];
                const T zi = P.cand[crow(P, 1, L.pos, t, i)], zk = P.cand[crow(P, 1, L.pos, t, k)];
                v = T(0.5) * (di * zk + zi * dk);
            }
            if (P.NC > 1) {
                T* dCt = A.dC + (b * P.NC + t) * (NZ * NZ);
                dCt[i * NZ + k] = v;
                dCt[k * NZ + i] = v;
            } else {
                acc2(acc, accl, v);
            }
        }
        if (P.NC == 1) {
            const T tot = acc + accl;
            A.dC[b * NZ * NZ + i * NZ + k] = tot;
            A.dC[b * NZ * NZ + k * NZ + i] = tot;
        }
    }
}

template <typename T, int NW, bool GEN>
__device__ void zero_grads(const Params<T>& P, const AdjArgs<T>& A, const Lane& L, bool act) {
    if (!act) return;
    const size_t b = L.b;
    if constexpr (GEN) {
        for (int e = L.w; e < P.NC * NZ * NZ; e += NW) A.dC[b * P.NC * NZ * NZ + e] = T(0);
        for (int e = L.w; e < P.Nc * NZ; e += NW) A.dc[b * P.Nc * NZ + e] = T(0);
    } else {
        for (int e = L.w; e < P.Nq * NX; e += NW) A.dQ[b * P.Nq * NX + e] = T(0);
        for (int e = L.w; e < P.N * NX; e += NW) A.dxref[b * P.N * NX + e] = T(0);
    }
    for (int i = L.w; i < NX; i += NW) A.dx0[b * NX + i] = T(0);
}

// A7: the cost of the diagonal form (reading R1's centred sum, all terms
// non-negative) at the returned iterate, evaluated afresh from the nominal
// records with the state as hi + lo.  The running J^0 + sum of accepted cost
// changes carries rounding relative to J^0, which a solve can lower by orders
// of magnitude; this sum's rounding is relative to the returned cost.  Warp 0.
template <typename T>
__device__ T final_cost(const Params<T>& P, const BlockSmem<T>& S, const Lane& L, int n) {
    T J = T(0);
    for (int t = 0; t < n; ++t) {
        const T* sr = P.stg + srow(P, L.pos, t, 0);
        T sx = T(0), su = T(0);
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            const T e = (sr[(R_X + i) * GW] - sr[(R_XR + i) * GW]) + sr[(R_XL + i) * GW];
            sx += e * (sr[(R_Q + i) * GW] * e);
        }
#pragma unroll
        for (int a = 0; a < NU; ++a) {
            const T e = sr[(R_U + a) * GW] - S.uref[a][L.sl];
            su += e * (S.R[a][L.sl] * e);
        }
        J += T(0.5) * sx + T(0.5) * su;
    }
    return J;
}

// A7: the nominal trajectory into the caller's u*, x* (zero past the horizon).
template <typename T, int NW>
__device__ void write_solution(const Params<T>& P, const Lane& L, int n) {
    if (!L.valid) return;
    const size_t b = L.b;
    for (int t = L.w; t < P.N; t += NW) {
        T* xo = P.x + (b * P.N + t) * NX;
        T* uo = P.u + (b * P.N + t) * NU;
        T buf[NX + NU];
#pragma unroll
        for (int e = 0; e < NX + NU; ++e) buf[e] = T(0);
        if (t < n) {
            const T* sr = P.stg + srow(P, L.pos, t, 0);
#pragma unroll
            for (int i = 0; i < NX; ++i) buf[i] = sr[(R_X + i) * GW];
#pragma unroll
            for (int a = 0; a < NU; ++a) buf[NX + a] = sr[(R_U + a) * GW];
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) xo[i] = buf[i];
#pragma unroll
        for (int a = 0; a < NU; ++a) uo[a] = buf[NX + a];
    }
}

}  // namespace camp
