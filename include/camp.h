/*
 * camp.h -- C ABI of the batched differentiable MPC layer for GB300 (sm_103a).
 *
 * The layer solves, for each of B independent instances, the box-constrained
 * optimal-control problem of Eq. (3) (Sec. IV):
 *
 *     min_{x,u}  sum_{t=0}^{N-1} 1/2 z_t' C_t z_t + c_t' z_t,   z_t = [x_t; u_t]
 *     s.t.       x_{t+1} = f(x_t, u_t),  x_0 = x_init,  u_lo <= u_t <= u_hi
 *
 * with the diagonal quadratic surrogate of Eq. (2): C_t = diag(Q_t, R) and
 * c_t = [-Q_t * x_ref_t ; -R * u_ref].  f is one RK4 step (length dt) of a
 * 13-state quadrotor (p, q = (w, x, y, z), v, body rate) driven by 4 rotor
 * thrusts.  The forward solve is the control-limited iLQR of Sec. IV
 * (rollout + analytic linearization, Riccati backward pass with a per-stage
 * box QP, forward pass with a line search over alpha); the backward solve is
 * the implicit KKT differentiation of Sec. IV (Amos et al. 2018), done as one
 * adjoint LQR sweep at the returned solution with its active set frozen.
 *
 * Conventions for every entry point:
 *   - Array pointers are DEVICE pointers on the handle's device, row-major,
 *     instance-major (the layout of a contiguous torch tensor), in the
 *     handle's dtype (float for MPC_F32, double for MPC_F64), int32 for the
 *     int arrays.  Pointers must be aligned to their element size.
 *   - The caller owns every input, output and tape buffer.  The handle owns a
 *     scratch workspace sized in mpc_create; no solve call allocates, copies
 *     to or from the host, or synchronises, so the calls can be captured in a
 *     CUDA graph (mpc_autotune excepted).
 *   - Return codes are synchronous results of host-side validation and of the
 *     kernel launch itself (MPC_OK or a negative MPC_ERR_*); nothing aborts or
 *     throws across the ABI.  Numeric outcomes are asynchronous, per instance,
 *     in status[] (MPC_ST_*).
 *   - A handle is not thread-safe and its workspace is shared by all its
 *     calls: use one handle per stream.
 */
#ifndef CAMP_H
#define CAMP_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define MPC_OK            0
#define MPC_ERR_ARG      (-1)   /* NULL handle/pointer or a value out of range      */
#define MPC_ERR_SHAPE    (-2)   /* B, N, Nq beyond the handle's capacity or invalid */
#define MPC_ERR_CUDA     (-3)   /* a CUDA call failed (allocation, launch)          */
#define MPC_ERR_TIMEOUT  (-4)   /* reserved: a bounded device wait gave up          */
#define MPC_ERR_STATE    (-5)   /* call not valid in the handle's configuration     */

/* dtypes */
#define MPC_F32 0
#define MPC_F64 1

/* what the forward keeps for the backward (Sec. IV: differentiate at the solution) */
#define MPC_STORE_ALL   0      /* tape holds F_t, K_t, chol(Q_uu,ff), free set per stage */
#define MPC_RECOMPUTE   1      /* no tape: the backward re-linearises and re-factors    */
#define MPC_STORE_AUTO  2      /* per (B, N): store the tape when it fits the config's  */
                               /* tape_budget, else recompute                          */

/* how the forward iterations are launched */
#define MPC_EXEC_PERSISTENT 0  /* one persistent launch, work queue over instances      */
#define MPC_EXEC_PLAIN      1  /* three launches per iteration (Sec. IV's structure)     */
#define MPC_EXEC_SCAN       2  /* the plain form with one instance per block and the     */
                               /* Riccati recursion of Sec. IV-2 in parallel over the   */
                               /* stages: the associative-scan LQR of the related work  */
                               /* in Sec. II on the box QPs' free sets of the previous  */
                               /* iteration, then the stages whose QP disagrees solved  */
                               /* sequentially (same K_t, k_t as the sequential         */
                               /* recursion up to rounding).  For small batches and     */
                               /* long horizons.  The general cost keeps the sequential */
                               /* Riccati phase.  Needs R > 0 (the elements use R^-1).  */
                               /* mpc_create allocates about                            */
                               /* (N_max * 0.8k + 8.5k) * sizeof(dtype) bytes more per  */
                               /* instance of B_max.                                    */
#define MPC_EXEC_AUTO       3  /* persistent or scan, whichever mpc_autotune measures     */
                               /* faster on the caller's problem (persistent until it   */
                               /* has run; mpc_exec_form tells which).  Which one wins  */
                               /* depends on the problem, not only its shape: a few     */
                               /* instances whose saturations settle early favour the   */
                               /* scan.  Allocates the scan workspace.                  */

/* per-instance status written by mpc_solve_fwd */
#define MPC_ST_CONVERGED  0    /* max_t |u^k_t - u^(k-1)_t|_inf < tol after a step      */
#define MPC_ST_STALLED    1    /* no alpha gave a finite cost: the nominal is returned  */
#define MPC_ST_MAX_ITER   2    /* max_iter iterations executed                          */
#define MPC_ST_NONFINITE  3    /* an input or the initial cost was not finite           */
#define MPC_ST_NONPD      4    /* a free block of Q_uu had a non-positive pivot         */

typedef struct mpc_handle mpc_handle;   /* opaque, owned by the library */

typedef struct mpc_config {
    int    nx, nu;          /* must be 13 and 4                                        */
    int    N_max;           /* largest horizon any call will use, 1..64                */
    int    B_max;           /* largest batch any call will use, >= 1                   */
    int    dtype;           /* MPC_F32 or MPC_F64                                      */
    double dt;              /* RK4 step [s]                                            */
    double mass;            /* [kg]                                                    */
    double inertia[3];      /* diagonal body inertia [kg m^2]                          */
    double arm;             /* rotor distance from the centre [m] (X layout)           */
    double kappa_yaw;       /* yaw moment per newton of thrust [m]                     */
    double gravity;         /* [m/s^2]                                                 */
    int    max_iter;        /* iLQR iterations K (Algorithm 2), 0..1000                */
    double tol;             /* convergence threshold on max |du| [N]                   */
    int    n_alpha;         /* number of line-search coefficients, 1..4                */
    double alpha[4];        /* coefficients in (0, 1], default {1, .5, .25, .1}        */
    int    store_mode;      /* MPC_STORE_ALL, MPC_RECOMPUTE or MPC_STORE_AUTO          */
    int    exec_mode;       /* MPC_EXEC_PERSISTENT, _PLAIN, _SCAN or _AUTO             */
    int    tpi;             /* threads per instance = warps per block: 0 (4 until      */
                            /* mpc_autotune picks), 4 or 8                              */
    int    ipb;             /* instances per block (one per lane): 0 (auto) or 1..32,  */
                            /* 1..16 in MPC_F64                                         */
    size_t tape_budget;     /* MPC_STORE_AUTO: largest tape [bytes] a (B, N) shape may  */
                            /* store; 0 = a quarter of the device memory free at       */
                            /* mpc_create                                               */
} mpc_config;

typedef struct mpc_problem {
    int         B, N;       /* batch and horizon (buffer stride); 0 <= B <= B_max       */
    const int  *horizon;    /* [B] per-instance horizon, clamped to [1, N]; NULL = N   */
    const void *x0;         /* [B, 13]  x_init                                         */
    const void *Q;          /* [B, Nq, 13] diagonal state weights (>= 0)               */
    int         Nq;         /* 1 (one Q for every stage) or N (one per stage)          */
    const void *x_ref;      /* [B, N, 13]                                              */
    const void *R;          /* [B, 4]   diagonal control weights (> 0)                 */
    const void *u_ref;      /* [B, 4]                                                  */
    const void *u_lo;       /* [B, 4]   u_min                                          */
    const void *u_hi;       /* [B, 4]   u_max (>= u_lo)                                */
    const void *u_init;     /* [B, N, 4] warm start, or NULL for clamp(u_ref)          */
    /* General stage cost of Eq. (2), 1/2 z_t' C_t z_t + c_t' z_t with z_t = [x_t; u_t],
     * in place of the diagonal form: NULL C selects the diagonal form (Q, Nq, x_ref,
     * R and u_ref as above).  With C given, Q, Nq and x_ref are not read (may be
     * NULL), R is not used, u_ref only gives the start U^0, and the cost reported
     * is Eq. (3)'s objective itself. */
    const void *C;          /* [B, NC, 17, 17] symmetric positive semidefinite C_t     */
    int         NC;         /* 1 (one C for every stage) or N                          */
    const void *c;          /* [B, Nc, 17] c_t (required with C)                       */
    int         Nc;         /* 1 or N                                                  */
} mpc_problem;

typedef struct mpc_solution {
    void   *u;              /* [B, N, 4]  u* (zero past each horizon); u*_0 is the action */
    void   *x;              /* [B, N, 13] x* (x*_0 = x_init; zero past each horizon)    */
    void   *cost;           /* [B] sum_t 1/2|x-x_ref|_Q^2 + 1/2|u-u_ref|_R^2 at (x*,u*)  */
                            /* (general cost: sum_t 1/2 z'C z + c'z)                  */
    int    *iters;          /* [B] iterations executed                                 */
    int    *status;         /* [B] MPC_ST_*                                             */
    void   *tape;           /* >= mpc_tape_bytes(B, N) bytes, 256-aligned (none if 0)   */
    size_t  tape_bytes;
} mpc_solution;

/* Fill *cfg with the quadrotor workload's defaults (m = 0.75 kg, J =
 * diag(2.5e-3, 2.1e-3, 4.3e-3), arm 0.15 m, kappa 0.016 m, g = 9.81, dt = 0.02,
 * max_iter 8, tol 1e-6, alpha = {1, .5, .25, .1} (Sec. IV-3), N_max 40,
 * B_max 8192, MPC_F32, MPC_STORE_ALL, MPC_EXEC_PERSISTENT, tpi = ipb = 0). */
void mpc_config_default(mpc_config *cfg);

/* Validate *cfg, allocate the workspace on the current device and return a
 * handle in *out.  Errors: MPC_ERR_ARG (NULL or out-of-range field),
 * MPC_ERR_CUDA (no device / allocation failed). */
int mpc_create(const mpc_config *cfg, mpc_handle **out);

/* Free the workspace and the handle (NULL is accepted).  The caller must make
 * sure no call on it is still running on the GPU. */
int mpc_destroy(mpc_handle *h);

/* Bytes of tape mpc_solve_fwd writes for a (B, N) problem: ceil(B/32)*32*N*210
 * elements of the handle's dtype in MPC_STORE_ALL mode (per stage and instance:
 * the 11 computed columns of F_t, K_t, the masked factor of Q_uu,ff and the free
 * mask), 0 in MPC_RECOMPUTE mode (or for a NULL handle).  In MPC_STORE_AUTO mode
 * the same size when it is at most the handle's budget (mpc_config.tape_budget,
 * by default a quarter of the device memory free at mpc_create), else 0: solves
 * of that shape then recompute.  This is how a caller learns which way a shape
 * goes. */
size_t mpc_tape_bytes(const mpc_handle *h, int B, int N);

/* Forward solve (Eq. (3) by box-constrained iLQR, Algorithm 2's inner loop):
 * writes u, x, cost, iters, status and, when mpc_tape_bytes(B, N) > 0, the tape with
 * the linearization and factorization at the returned iterate.  Enqueued on
 * `stream`; returns before the GPU finishes.  Errors: MPC_ERR_ARG (NULL
 * pointer, bad Nq, tape too small), MPC_ERR_SHAPE (B > B_max, N outside
 * 1..N_max), MPC_ERR_CUDA (launch failed).  B = 0 returns MPC_OK at once. */
int mpc_solve_fwd(mpc_handle *h, const mpc_problem *p, mpc_solution *s, cudaStream_t stream);

/* Backward solve (Sec. IV implicit KKT differentiation as an adjoint LQR):
 * given dL/du* (grad_u [B, N, 4]) and optionally dL/dx* (grad_x [B, N, 13],
 * NULL = 0), writes dL/dQ (dQ [B, Nq, 13]), dL/dx_ref (dx_ref [B, N, 13]) and
 * dL/dx_init (dx0 [B, 13]).  `p` and `s` must be the ones of the matching
 * mpc_solve_fwd, unchanged since.  Instances with status NONFINITE or NONPD get
 * zero gradients.  Same error codes as mpc_solve_fwd. */
int mpc_solve_bwd(mpc_handle *h, const mpc_problem *p, const mpc_solution *s,
                  const void *grad_u, const void *grad_x,
                  void *dQ, void *dx_ref, void *dx0, cudaStream_t stream);

/* Backward solve for a problem with the general cost (p->C non-NULL): as
 * mpc_solve_bwd, but writes dL/dC (dC [B, NC, 17, 17], symmetric:
 * 1/2 (d_tau z*' + z* d_tau') per stage, summed over the stages when NC = 1),
 * dL/dc (dc [B, Nc, 17]: d_tau per stage, summed when Nc = 1) and dL/dx_init
 * (dx0 [B, 13]).  MPC_ERR_STATE for a problem with the diagonal form (and
 * mpc_solve_bwd returns MPC_ERR_STATE for one with the general form). */
int mpc_solve_bwd_general(mpc_handle *h, const mpc_problem *p, const mpc_solution *s,
                          const void *grad_u, const void *grad_x,
                          void *dC, void *dc, void *dx0, cudaStream_t stream);

/* Time the persistent forward for each launch shape (threads per instance x
 * instances per block; a nonzero tpi or ipb in the config pins that value) on
 * this problem (overwriting *s), keep the fastest in the handle and report its
 * ipb in *ipb_out (may be NULL; mpc_launch_shape gives the whole shape).
 * Under MPC_EXEC_AUTO it then times the stage-parallel form (MPC_EXEC_SCAN) at
 * the best warp count and keeps whichever form was faster.  MPC_ERR_STATE for
 * the plain and scan forms.  Synchronises `stream`; not capturable. */
int mpc_autotune(mpc_handle *h, const mpc_problem *p, mpc_solution *s,
                 cudaStream_t stream, int *ipb_out);

/* The launch form the handle's solves use (MPC_EXEC_PERSISTENT, _PLAIN or
 * _SCAN): the config's, or under MPC_EXEC_AUTO the one mpc_autotune chose
 * (persistent before it has run).  MPC_ERR_ARG for NULL arguments. */
int mpc_exec_form(const mpc_handle *h, int *exec);

/* Launch shape the next persistent forward on (B, N) will use: threads per
 * instance, instances per block, blocks.  Any out pointer may be NULL. */
int mpc_launch_shape(const mpc_handle *h, int B, int N, int *tpi, int *ipb, int *grid);

/* Number of kernel launches one mpc_solve_fwd / mpc_solve_bwd on (B, N, with or
 * without per-instance horizons) enqueues in the handle's configuration (in
 * MPC_STORE_AUTO mode: for the (B_max, N_max) shape). */
int mpc_launch_count(const mpc_handle *h, int has_horizon, int *fwd, int *bwd);

/* Forward solve that allocates nothing.  The paper has no counterpart: this is
 * for callers that cannot allocate device memory while they run (a real-time
 * control loop that must not allocate after start-up, a plug-in whose host
 * application owns every device allocation).  Same problem, outputs and
 * per-instance statuses as mpc_solve_fwd in the persistent form, without a
 * handle: the scratch is one statically allocated device array (9.7 MB,
 * held on every device the library runs on until the process exits).
 *   cfg    as for mpc_create, dtype must be MPC_F32 (exec_mode, tpi, ipb,
 *          N_max and B_max are ignored); MPC_STORE_ALL writes the tape.
 *   p, s   device pointers as for mpc_solve_fwd; B <= MPC_NOALLOC_B_MAX and
 *          N <= MPC_NOALLOC_N_MAX, else MPC_ERR_SHAPE.
 * The first call on a device looks the array up and sets the kernels' shared-
 * memory limit with that device current; make it before any stream capture.
 * No handle (mpc_create) is needed before it.  The looked-up address is cached
 * per device for the life of the process and is invalid after cudaDeviceReset.
 * All calls share the array: calls whose GPU work overlaps race on it and must
 * not be issued.  Errors as for mpc_solve_fwd. */
#define MPC_NOALLOC_B_MAX 256
#define MPC_NOALLOC_N_MAX 40
int mpc_solve_fwd_noalloc(const mpc_config *cfg, const mpc_problem *p, mpc_solution *s, cudaStream_t stream);

/* Measurement support (the paper has no counterpart): the FP32 multiply-add
 * throughput of this GPU, the denominator of the forward solve's roofline.
 * Enqueues on `stream` one launch of 2 blocks of 1024 threads per SM, each
 * thread running 8 independent chains of `trips` x 16 fused multiply-adds, and
 * returns in *flops (may be NULL) the flops it executes (2 per multiply-add);
 * the caller times it (CUDA events) and divides.  `sink` is a device float
 * the kernel practically never writes.  Errors: MPC_ERR_ARG (trips < 1, NULL
 * sink), MPC_ERR_CUDA. */
int mpc_fp32_fma_probe(int trips, float *sink, cudaStream_t stream, double *flops);

/* Static text for a return code (mpc_strerror) or an MPC_ST_* status (mpc_status_str). */
const char *mpc_strerror(int code);
const char *mpc_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* CAMP_H */
