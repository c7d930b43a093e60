// camp_api.cu -- the C ABI (include/camp.h): validation, workspace, launch shapes.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "camp.h"
#include "camp_device.cuh"
#include "camp_internal.h"

using namespace camp;

struct mpc_handle {
    mpc_config cfg;
    int device;
    int num_sms;
    int slots;              // scratch positions (= B_max)
    void* ws;               // one allocation holding every scratch region
    size_t ws_bytes;
    void *stg, *cand, *kh;  // per-stage records, line-search candidates, adjoint k-hat
    void* scan;             // stage-parallel Riccati workspace (MPC_EXEC_SCAN and MPC_EXEC_AUTO)
    int exec;               // the launch form solves use: the config's, or under MPC_EXEC_AUTO
                            // the one mpc_autotune measured faster (persistent until then)
    int* queue;             // [2] work-queue tickets (forward, backward)
    int* order;             // [B_max] longest-horizon-first order
    int tpi;                // threads per instance (warps per block): 4 or 8
    int ipb;                // instances per block, 0 = as many as fill one block per SM
    size_t tape_budget;     // MPC_STORE_AUTO: largest tape (bytes) a shape may store
};

static size_t elem_size(int dtype) { return dtype == MPC_F64 ? sizeof(double) : sizeof(float); }
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

extern "C" void mpc_config_default(mpc_config* c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->nx = 13;
    c->nu = 4;
    c->N_max = 40;
    c->B_max = 8192;
    c->dtype = MPC_F32;
    c->dt = 0.02;
    c->mass = 0.75;
    c->inertia[0] = 2.5e-3;
    c->inertia[1] = 2.1e-3;
    c->inertia[2] = 4.3e-3;
    c->arm = 0.15;
    c->kappa_yaw = 0.016;
    c->gravity = 9.81;
    c->max_iter = 8;
    c->tol = 1e-6;
    c->n_alpha = 4;
    c->alpha[0] = 1.0;
    c->alpha[1] = 0.5;
    c->alpha[2] = 0.25;
    c->alpha[3] = 0.1;
    c->store_mode = MPC_STORE_ALL;
    c->exec_mode = MPC_EXEC_PERSISTENT;
    c->tpi = 0;
    c->ipb = 0;
}

static int validate_config(const mpc_config* c) {
    if (!c) return MPC_ERR_ARG;
    if (c->nx != NX || c->nu != NU) return MPC_ERR_ARG;
    if (c->N_max < 1 || c->N_max > MAX_N) return MPC_ERR_ARG;
    if (c->B_max < 1 || c->B_max > (1 << 24)) return MPC_ERR_ARG;
    if (c->dtype != MPC_F32 && c->dtype != MPC_F64) return MPC_ERR_ARG;
    if (!finite_pos(c->dt) || !finite_pos(c->mass)) return MPC_ERR_ARG;
    for (int i = 0; i < 3; ++i)
        if (!finite_pos(c->inertia[i])) return MPC_ERR_ARG;
    if (!isfinite(c->arm) || c->arm < 0 || !isfinite(c->kappa_yaw) || !isfinite(c->gravity)) return MPC_ERR_ARG;
    if (c->max_iter < 0 || c->max_iter > 1000) return MPC_ERR_ARG;
    if (!isfinite(c->tol) || c->tol < 0) return MPC_ERR_ARG;
    if (c->n_alpha < 1 || c->n_alpha > 4) return MPC_ERR_ARG;
    for (int i = 0; i < c->n_alpha; ++i)
        if (!(c->alpha[i] > 0.0 && c->alpha[i] <= 1.0)) return MPC_ERR_ARG;
    if (c->store_mode != MPC_STORE_ALL && c->store_mode != MPC_RECOMPUTE && c->store_mode != MPC_STORE_AUTO)
        return MPC_ERR_ARG;
    if (c->exec_mode != MPC_EXEC_PERSISTENT && c->exec_mode != MPC_EXEC_PLAIN && c->exec_mode != MPC_EXEC_SCAN &&
        c->exec_mode != MPC_EXEC_AUTO)
        return MPC_ERR_ARG;
    if (c->tpi != 0 && c->tpi != 4 && c->tpi != 8) return MPC_ERR_ARG;
    if (c->ipb < 0 || c->ipb > (c->dtype == MPC_F64 ? 16 : 32)) return MPC_ERR_ARG;
    return MPC_OK;
}

extern "C" int mpc_create(const mpc_config* cfg, mpc_handle** out) {
    if (!out) return MPC_ERR_ARG;
    *out = nullptr;
    const int v = validate_config(cfg);
    if (v != MPC_OK) return v;
    mpc_handle* h = (mpc_handle*)calloc(1, sizeof(mpc_handle));
    if (!h) return MPC_ERR_CUDA;
    h->cfg = *cfg;
    h->tpi = cfg->tpi ? cfg->tpi : 4;
    h->ipb = cfg->ipb;
    if (cudaGetDevice(&h->device) != cudaSuccess) { free(h); return MPC_ERR_CUDA; }
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        free(h);
        return MPC_ERR_CUDA;
    }
    cudaError_t pe = cfg->dtype == MPC_F64 ? prepare_kernels<double>() : prepare_kernels<float>();
    const bool with_scan = cfg->exec_mode == MPC_EXEC_SCAN || cfg->exec_mode == MPC_EXEC_AUTO;
    h->exec = cfg->exec_mode == MPC_EXEC_AUTO ? MPC_EXEC_PERSISTENT : cfg->exec_mode;
    if (pe == cudaSuccess && with_scan)
        pe = cfg->dtype == MPC_F64 ? prepare_scan<double>() : prepare_scan<float>();
    if (pe != cudaSuccess) { free(h); return MPC_ERR_CUDA; }
    if (cfg->store_mode == MPC_STORE_AUTO) {
        // the tape budget: the config's, or a quarter of the device memory free at creation
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { free(h); return MPC_ERR_CUDA; }
        h->tape_budget = cfg->tape_budget ? cfg->tape_budget : free_b / 4;
    }
    h->slots = cfg->B_max;
    const size_t es = elem_size(cfg->dtype);
    const size_t S = (size_t)h->slots;
    const int Nw = cfg->N_max;
    const size_t bS = align256(stg_elems(S, Nw) * es);
    const size_t bC = align256(cand_elems(S, Nw) * es);
    const size_t bH = align256(kh_elems(S, Nw) * es);
    const size_t bQ = align256(2 * sizeof(int));
    const size_t bO = align256((size_t)cfg->B_max * sizeof(int));
    const size_t bP = with_scan ? align256(scan_ws_elems(S, Nw) * es) : 0;
    h->ws_bytes = bS + bC + bH + bQ + bO + bP;
    if (cudaMalloc(&h->ws, h->ws_bytes) != cudaSuccess) { free(h); return MPC_ERR_CUDA; }
    // All-ones bytes are NaN in float and double: a read of scratch that no
    // phase wrote surfaces as a NaN result instead of stale data.
    if (cudaMemset(h->ws, 0xff, h->ws_bytes) != cudaSuccess) { cudaFree(h->ws); free(h); return MPC_ERR_CUDA; }
    char* p = (char*)h->ws;
    h->stg = p; p += bS;
    h->cand = p; p += bC;
    h->kh = p; p += bH;
    h->queue = (int*)p; p += bQ;
    h->order = (int*)p; p += bO;
    h->scan = bP ? p : nullptr;
    *out = h;
    return MPC_OK;
}

extern "C" int mpc_destroy(mpc_handle* h) {
    if (!h) return MPC_OK;
    if (h->ws) cudaFree(h->ws);
    free(h);
    return MPC_OK;
}

// Whether solves of shape (B, N) keep the tape: always in MPC_STORE_ALL, never
// in MPC_RECOMPUTE, and in MPC_STORE_AUTO when the tape fits the budget.
static bool stores_tape(const mpc_handle* h, int B, int N) {
    if (h->cfg.store_mode == MPC_STORE_ALL) return true;
    if (h->cfg.store_mode == MPC_RECOMPUTE) return false;
    return tape_elems(B > 0 ? B : 0, N > 0 ? N : 0) * elem_size(h->cfg.dtype) <= h->tape_budget;
}

extern "C" size_t mpc_tape_bytes(const mpc_handle* h, int B, int N) {
    if (!h || B <= 0 || N <= 0 || !stores_tape(h, B, N)) return 0;
    return tape_elems(B, N) * elem_size(h->cfg.dtype);
}

// Instances per block for a batch of B: the handle's fixed value, or as many
// as spread the batch over one block per SM.
static int ipb_cap(const mpc_handle* h) { return h->cfg.dtype == MPC_F64 ? 16 : 32; }

static int ipb_for(const mpc_handle* h, int B) {
    if (h->ipb) return h->ipb;
    const int per_sm = (B + h->num_sms - 1) / h->num_sms;
    const int cap = ipb_cap(h);
    return per_sm < 1 ? 1 : (per_sm > cap ? cap : per_sm);
}

static int grid_for(const mpc_handle* h, int B, int ipb) {
    const int bps = h->cfg.dtype == MPC_F64 ? persistent_blocks_per_sm<double>(h->tpi)
                                            : persistent_blocks_per_sm<float>(h->tpi);
    long long g = (long long)(bps > 0 ? bps : 1) * h->num_sms;
    const long long need = (B + ipb - 1) / ipb;
    if (g > need) g = need;
    return (int)(g > 0 ? g : 1);
}

static int check_problem(const mpc_handle* h, const mpc_problem* p) {
    if (!h || !p) return MPC_ERR_ARG;
    if (p->B < 0 || p->B > h->cfg.B_max) return MPC_ERR_SHAPE;
    if (p->N < 1 || p->N > h->cfg.N_max) return MPC_ERR_SHAPE;
    if (p->C) {
        // general cost: C and c with their own sharing; Q and x_ref unused
        if (!p->c) return MPC_ERR_ARG;
        if ((p->NC != 1 && p->NC != p->N) || (p->Nc != 1 && p->Nc != p->N)) return MPC_ERR_SHAPE;
    } else if (p->Nq != 1 && p->Nq != p->N) {
        return MPC_ERR_SHAPE;
    }
    if (p->B == 0) return MPC_OK;
    if (!p->x0 || !p->R || !p->u_ref || !p->u_lo || !p->u_hi) return MPC_ERR_ARG;
    if (!p->C && (!p->Q || !p->x_ref)) return MPC_ERR_ARG;
    return MPC_OK;
}

template <typename T>
static Params<T> make_params(const mpc_handle* h, const mpc_problem* p, const mpc_solution* s, int ipb) {
    Params<T> P;
    memset(&P, 0, sizeof(P));
    const mpc_config& c = h->cfg;
    fill_model(P.mdl, c.dt, c.mass, c.inertia, c.arm, c.kappa_yaw, c.gravity);
    P.B = p->B;
    P.N = p->N;
    P.Nq = p->Nq;
    P.max_iter = h->cfg.max_iter;
    P.n_alpha = h->cfg.n_alpha;
    P.store_all = stores_tape(h, p->B, p->N) ? 1 : 0;
    P.N_ws = h->cfg.N_max;
    P.ipb = ipb;
    P.tol = (T)h->cfg.tol;
    for (int i = 0; i < 4; ++i) P.alpha[i] = (T)h->cfg.alpha[i];
    P.horizon = p->horizon;
    P.order = nullptr;
    P.x0 = (const T*)p->x0;
    P.Q = (const T*)p->Q;
    P.xref = (const T*)p->x_ref;
    P.R = (const T*)p->R;
    P.uref = (const T*)p->u_ref;
    P.ulo = (const T*)p->u_lo;
    P.uhi = (const T*)p->u_hi;
    P.uinit = (const T*)p->u_init;
    P.Cg = (const T*)p->C;
    P.cg = (const T*)p->c;
    P.NC = p->C ? p->NC : 1;
    P.Nc = p->C ? p->Nc : 1;
    P.u = (T*)s->u;
    P.x = (T*)s->x;
    P.cost = (T*)s->cost;
    P.iters = s->iters;
    P.status = s->status;
    P.tape = (T*)s->tape;
    P.stg = (T*)h->stg;
    P.cand = (T*)h->cand;
    P.kh = (T*)h->kh;
    P.scan = (T*)h->scan;
    P.queue = h->queue;
    return P;
}

extern "C" int mpc_solve_fwd(mpc_handle* h, const mpc_problem* p, mpc_solution* s, cudaStream_t stream) {
    int r = check_problem(h, p);
    if (r != MPC_OK) return r;
    if (!s) return MPC_ERR_ARG;
    if (p->B == 0) return MPC_OK;
    if (!s->u || !s->x || !s->cost || !s->iters || !s->status) return MPC_ERR_ARG;
    if (stores_tape(h, p->B, p->N)) {
        if (!s->tape || s->tape_bytes < mpc_tape_bytes(h, p->B, p->N)) return MPC_ERR_ARG;
    }
    cudaError_t e;
    const int ipb = ipb_for(h, p->B);
    const int grid = grid_for(h, p->B, ipb);
    if (h->cfg.dtype == MPC_F64) {
        const Params<double> P = make_params<double>(h, p, s, ipb);
        e = launch_forward<double>(P, h->exec, h->tpi, grid, h->order, stream);
    } else {
        const Params<float> P = make_params<float>(h, p, s, ipb);
        e = launch_forward<float>(P, h->exec, h->tpi, grid, h->order, stream);
    }
    return e == cudaSuccess ? MPC_OK : MPC_ERR_CUDA;
}

extern "C" int mpc_solve_bwd(mpc_handle* h, const mpc_problem* p, const mpc_solution* s, const void* grad_u,
                             const void* grad_x, void* dQ, void* dx_ref, void* dx0, cudaStream_t stream) {
    int r = check_problem(h, p);
    if (r != MPC_OK) return r;
    if (!s) return MPC_ERR_ARG;
    if (p->B == 0) return MPC_OK;
    if (p->C) return MPC_ERR_STATE;     // a general cost has mpc_solve_bwd_general
    if (!s->u || !s->x || !s->status || !grad_u || !dQ || !dx_ref || !dx0) return MPC_ERR_ARG;
    const int recompute = stores_tape(h, p->B, p->N) ? 0 : 1;
    if (!recompute && (!s->tape || s->tape_bytes < mpc_tape_bytes(h, p->B, p->N))) return MPC_ERR_ARG;
    cudaError_t e;
    const int ipb = ipb_for(h, p->B);
    const int grid = grid_for(h, p->B, ipb);
    if (h->cfg.dtype == MPC_F64) {
        const Params<double> P = make_params<double>(h, p, s, ipb);
        AdjArgs<double> A{(const double*)grad_u, (const double*)grad_x, (double*)dQ, (double*)dx_ref,
                          (double*)dx0, nullptr, nullptr, recompute};
        e = launch_backward<double>(P, A, h->tpi, grid, h->order, stream);
    } else {
        const Params<float> P = make_params<float>(h, p, s, ipb);
        AdjArgs<float> A{(const float*)grad_u, (const float*)grad_x, (float*)dQ, (float*)dx_ref, (float*)dx0,
                         nullptr, nullptr, recompute};
        e = launch_backward<float>(P, A, h->tpi, grid, h->order, stream);
    }
    return e == cudaSuccess ? MPC_OK : MPC_ERR_CUDA;
}

extern "C" int mpc_solve_bwd_general(mpc_handle* h, const mpc_problem* p, const mpc_solution* s,
                                     const void* grad_u, const void* grad_x, void* dC, void* dc, void* dx0,
                                     cudaStream_t stream) {
    int r = check_problem(h, p);
    if (r != MPC_OK) return r;
    if (!s) return MPC_ERR_ARG;
    if (!p->C) return MPC_ERR_STATE;    // the diagonal form has mpc_solve_bwd
    if (p->B == 0) return MPC_OK;
    if (!s->u || !s->x || !s->status || !grad_u || !dC || !dc || !dx0) return MPC_ERR_ARG;
    const int recompute = stores_tape(h, p->B, p->N) ? 0 : 1;
    if (!recompute && (!s->tape || s->tape_bytes < mpc_tape_bytes(h, p->B, p->N))) return MPC_ERR_ARG;
    cudaError_t e;
    const int ipb = ipb_for(h, p->B);
    const int grid = grid_for(h, p->B, ipb);
    if (h->cfg.dtype == MPC_F64) {
        const Params<double> P = make_params<double>(h, p, s, ipb);
        AdjArgs<double> A{(const double*)grad_u, (const double*)grad_x, nullptr, nullptr, (double*)dx0,
                          (double*)dC, (double*)dc, recompute};
        e = launch_backward<double>(P, A, h->tpi, grid, h->order, stream);
    } else {
        const Params<float> P = make_params<float>(h, p, s, ipb);
        AdjArgs<float> A{(const float*)grad_u, (const float*)grad_x, nullptr, nullptr, (float*)dx0, (float*)dC,
                         (float*)dc, recompute};
        e = launch_backward<float>(P, A, h->tpi, grid, h->order, stream);
    }
    return e == cudaSuccess ? MPC_OK : MPC_ERR_CUDA;
}

extern "C" int mpc_autotune(mpc_handle* h, const mpc_problem* p, mpc_solution* s, cudaStream_t stream,
                            int* ipb_out) {
    int r = check_problem(h, p);
    if (r != MPC_OK) return r;
    const bool auto_form = h->cfg.exec_mode == MPC_EXEC_AUTO;
    if (h->cfg.exec_mode != MPC_EXEC_PERSISTENT && !auto_form) return MPC_ERR_STATE;
    if (p->B == 0) { if (ipb_out) *ipb_out = ipb_for(h, 0); return MPC_OK; }
    const int keep_tpi = h->tpi, keep_ipb = h->ipb, keep_exec = h->exec;
    h->exec = MPC_EXEC_PERSISTENT;
    // candidate instances per block: one, two, three or four blocks' worth per
    // SM, and full packs (fewer blocks than SMs when the batch is small)
    int cands[5], nc = 0;
    for (int k = 0; k <= 4; ++k) {
        int v = k == 0 ? ipb_cap(h) : (p->B + k * h->num_sms - 1) / (k * h->num_sms);
        v = v < 1 ? 1 : (v > ipb_cap(h) ? ipb_cap(h) : v);
        bool dup = false;
        for (int i = 0; i < nc; ++i) dup = dup || cands[i] == v;
        if (!dup) cands[nc++] = v;
    }
    const int tpis[2] = {4, 8};
    float best_ms = 3.0e38f;
    int best_tpi = keep_tpi, best_ipb = keep_ipb;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MPC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return MPC_ERR_CUDA; }
    for (int ti = 0; ti < 2 && r == MPC_OK; ++ti) {
        if (h->cfg.tpi && h->cfg.tpi != tpis[ti]) continue;
        for (int ci = 0; ci < nc && r == MPC_OK; ++ci) {
            const int ipb = h->cfg.ipb ? h->cfg.ipb : cands[ci];
            if (h->cfg.ipb && ci > 0) break;
            h->tpi = tpis[ti];
            h->ipb = ipb;
            if ((r = mpc_solve_fwd(h, p, s, stream)) != MPC_OK) break;          // warm-up
            cudaEventRecord(e0, stream);
            for (int rep = 0; rep < 3 && r == MPC_OK; ++rep) r = mpc_solve_fwd(h, p, s, stream);
            cudaEventRecord(e1, stream);
            if (r != MPC_OK || cudaEventSynchronize(e1) != cudaSuccess) { r = MPC_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) { best_ms = ms; best_tpi = tpis[ti]; best_ipb = ipb; }
        }
    }
    // MPC_EXEC_AUTO: the stage-parallel form at the best warp count, against
    // the best persistent shape
    int best_exec = MPC_EXEC_PERSISTENT;
    if (auto_form && r == MPC_OK) {
        h->tpi = best_tpi;
        h->exec = MPC_EXEC_SCAN;
        if ((r = mpc_solve_fwd(h, p, s, stream)) == MPC_OK) {
            cudaEventRecord(e0, stream);
            for (int rep = 0; rep < 3 && r == MPC_OK; ++rep) r = mpc_solve_fwd(h, p, s, stream);
            cudaEventRecord(e1, stream);
            if (r != MPC_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                r = MPC_ERR_CUDA;
            } else {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) best_exec = MPC_EXEC_SCAN;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->tpi = r == MPC_OK ? best_tpi : keep_tpi;
    h->ipb = r == MPC_OK ? best_ipb : keep_ipb;
    h->exec = r == MPC_OK ? best_exec : keep_exec;
    if (ipb_out) *ipb_out = ipb_for(h, p->B);
    return r;
}

extern "C" int mpc_exec_form(const mpc_handle* h, int* exec) {
    if (!h || !exec) return MPC_ERR_ARG;
    *exec = h->exec;
    return MPC_OK;
}

extern "C" int mpc_launch_shape(const mpc_handle* h, int B, int N, int* tpi, int* ipb, int* grid) {
    if (!h || B < 0 || N < 1 || N > h->cfg.N_max) return MPC_ERR_ARG;
    const int i = ipb_for(h, B);
    if (tpi) *tpi = h->tpi;
    if (ipb) *ipb = i;
    if (grid) *grid = B > 0 ? grid_for(h, B, i) : 0;
    return MPC_OK;
}

extern "C" int mpc_launch_count(const mpc_handle* h, int has_horizon, int* fwd, int* bwd) {
    if (!h) return MPC_ERR_ARG;
    const int hz = has_horizon ? 1 : 0;
    if (fwd) {
        if (h->exec == MPC_EXEC_PERSISTENT) *fwd = 1 + hz;
        else *fwd = hz + 2 + 2 * h->cfg.max_iter + (stores_tape(h, h->cfg.B_max, h->cfg.N_max) ? 1 : 0);
    }
    if (bwd) *bwd = 1 + hz;
    return MPC_OK;
}

extern "C" const char* mpc_strerror(int code) {
    switch (code) {
        case MPC_OK: return "ok";
        case MPC_ERR_ARG: return "invalid argument";
        case MPC_ERR_SHAPE: return "shape outside the handle's capacity";
        case MPC_ERR_CUDA: return "CUDA call failed";
        case MPC_ERR_TIMEOUT: return "bounded device wait timed out";
        case MPC_ERR_STATE: return "not valid in this configuration";
        default: return "unknown error";
    }
}

extern "C" const char* mpc_status_str(int st) {
    switch (st) {
        case MPC_ST_CONVERGED: return "converged";
        case MPC_ST_STALLED: return "stalled";
        case MPC_ST_MAX_ITER: return "max_iter";
        case MPC_ST_NONFINITE: return "nonfinite";
        case MPC_ST_NONPD: return "nonpd";
        default: return "unknown";
    }
}
