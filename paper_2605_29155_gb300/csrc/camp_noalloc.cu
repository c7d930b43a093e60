// camp_noalloc.cu -- mpc_solve_fwd_noalloc: the persistent FP32 forward solve
// with its scratch in a fixed, statically allocated device array instead of a
// handle's cudaMalloc'd workspace.
//
// For callers that may not allocate device memory once they are running: a
// real-time control loop that must not allocate after start-up, a plug-in whose
// host application owns every device allocation, or code that runs where an
// allocation would break a memory budget or a stream-ordered allocator.  They
// pass inputs and outputs; this entry point allocates nothing (no cudaMalloc,
// cudaFree or allocating library call).
//
// Limits: FP32, B <= MPC_NOALLOC_B_MAX, N <= MPC_NOALLOC_N_MAX.  The scratch
// array lives in every process that loads the library, on every device it
// runs on, until the process exits.
//
// Set-up: the first call on a device looks up the array's device address
// (cudaGetSymbolAddress) and raises the kernels' shared-memory limit
// (cudaFuncSetAttribute) with that device current; make that first call before
// any stream capture.  The address is cached per device for the life of the
// process: after cudaDeviceReset (or any teardown of the device's primary
// context) it is stale, and this entry point must not be called again.
// Every call shares the one array and leaves its contents behind: the
// work-queue counter is cleared on the stream at the start of each call, and
// every other scratch entry is written before it is read.  Calls
// whose GPU work overlaps (different streams, or different host threads
// without ordering) race on the array and must not be issued.
#include <math.h>
#include <mutex>
#include <string.h>

#include "camp.h"
#include "camp_device.cuh"
#include "camp_internal.h"

using namespace camp;

namespace {

constexpr int NA_TPI = 4;                                   // the handle's default threads per instance
constexpr size_t NA_SLOTS = MPC_NOALLOC_B_MAX;

constexpr size_t a256(size_t floats) { return (floats + 63) & ~(size_t)63; }   // 64 floats = 256 bytes
constexpr size_t NA_GROUPS = (NA_SLOTS + 31) / 32;
constexpr size_t OFF_S = 0;                                                          // per-stage records
constexpr size_t OFF_C = OFF_S + a256(NA_GROUPS * 32 * MPC_NOALLOC_N_MAX * SREC);    // line-search candidates
constexpr size_t OFF_H = OFF_C + a256(4 * NA_GROUPS * 32 * MPC_NOALLOC_N_MAX * CREC);
constexpr size_t OFF_Q = OFF_H + a256(NA_GROUPS * 32 * MPC_NOALLOC_N_MAX * NU);      // 2 ints: work-queue tickets
constexpr size_t OFF_O = OFF_Q + 64;                                                 // order: MPC_NOALLOC_B_MAX ints
constexpr size_t NA_FLOATS = OFF_O + a256(MPC_NOALLOC_B_MAX);

}  // namespace

// The scratch array (2,416,960 floats, 9.7 MB).  In host code this name is only a host-side
// stand-in: kernels get the device address looked up below.
static __device__ __align__(256) float g_noalloc_scratch[NA_FLOATS];

namespace {

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_setup_mutex;
float* g_scratch_dev[NA_MAX_DEVICES] = {};
int g_num_sms[NA_MAX_DEVICES] = {};

// Once per device, with that device current: the array's device address, the
// SM count, and the kernels' shared-memory limit.  The FP32 kernels need far
// more dynamic shared memory than the default 48 KB; mpc_create raises that
// limit too, but a caller of this entry point may never create a handle.
// cudaFuncSetAttribute allocates nothing.
int setup_device(int dev, float** scratch, int* sms) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return MPC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MPC_ERR_CUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            return MPC_ERR_CUDA;
        if (prepare_kernels<float>() != cudaSuccess) return MPC_ERR_CUDA;
        g_num_sms[dev] = n;
        g_scratch_dev[dev] = (float*)p;
    }
    *scratch = g_scratch_dev[dev];
    *sms = g_num_sms[dev];
    return MPC_OK;
}

bool pos(double v) { return isfinite(v) && v > 0.0; }

// The configuration rules of mpc_create, restricted to this entry point's dtype.
int check_config(const mpc_config* c) {
    if (!c) return MPC_ERR_ARG;
    if (c->nx != NX || c->nu != NU || c->dtype != MPC_F32) return MPC_ERR_ARG;
    if (!pos(c->dt) || !pos(c->mass) || !pos(c->inertia[0]) || !pos(c->inertia[1]) || !pos(c->inertia[2]))
        return MPC_ERR_ARG;
    if (!isfinite(c->arm) || c->arm < 0 || !isfinite(c->kappa_yaw) || !isfinite(c->gravity)) return MPC_ERR_ARG;
    if (c->max_iter < 0 || c->max_iter > 1000 || !isfinite(c->tol) || c->tol < 0) return MPC_ERR_ARG;
    if (c->n_alpha < 1 || c->n_alpha > 4) return MPC_ERR_ARG;
    for (int i = 0; i < c->n_alpha; ++i)
        if (!(c->alpha[i] > 0.0 && c->alpha[i] <= 1.0)) return MPC_ERR_ARG;
    if (c->store_mode != MPC_STORE_ALL && c->store_mode != MPC_RECOMPUTE) return MPC_ERR_ARG;
    return MPC_OK;
}

}  // namespace

extern "C" int mpc_solve_fwd_noalloc(const mpc_config* cfg, const mpc_problem* p, mpc_solution* s,
                                     cudaStream_t stream) {
    int r = check_config(cfg);
    if (r != MPC_OK) return r;
    if (!p || !s) return MPC_ERR_ARG;
    if (p->C) return MPC_ERR_ARG;       // the diagonal cost form only
    if (p->B < 0 || p->B > MPC_NOALLOC_B_MAX) return MPC_ERR_SHAPE;
    if (p->N < 1 || p->N > MPC_NOALLOC_N_MAX) return MPC_ERR_SHAPE;
    if (p->Nq != 1 && p->Nq != p->N) return MPC_ERR_SHAPE;
    if (p->B == 0) return MPC_OK;
    if (!p->x0 || !p->Q || !p->x_ref || !p->R || !p->u_ref || !p->u_lo || !p->u_hi) return MPC_ERR_ARG;
    if (!s->u || !s->x || !s->cost || !s->iters || !s->status) return MPC_ERR_ARG;
    const bool store_all = cfg->store_mode == MPC_STORE_ALL;
    if (store_all && (!s->tape || s->tape_bytes < tape_elems(p->B, p->N) * sizeof(float)))
        return MPC_ERR_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MPC_ERR_CUDA;
    float* ws = nullptr;
    int sms = 0;
    if ((r = setup_device(dev, &ws, &sms)) != MPC_OK) return r;

    Params<float> P;
    memset(&P, 0, sizeof(P));
    fill_model(P.mdl, cfg->dt, cfg->mass, cfg->inertia, cfg->arm, cfg->kappa_yaw, cfg->gravity);
    P.B = p->B;
    P.N = p->N;
    P.Nq = p->Nq;
    P.max_iter = cfg->max_iter;
    P.n_alpha = cfg->n_alpha;
    P.store_all = store_all ? 1 : 0;
    P.N_ws = MPC_NOALLOC_N_MAX;
    P.tol = (float)cfg->tol;
    for (int i = 0; i < 4; ++i) P.alpha[i] = (float)cfg->alpha[i];
    P.horizon = p->horizon;
    P.x0 = (const float*)p->x0;
    P.Q = (const float*)p->Q;
    P.xref = (const float*)p->x_ref;
    P.R = (const float*)p->R;
    P.uref = (const float*)p->u_ref;
    P.ulo = (const float*)p->u_lo;
    P.uhi = (const float*)p->u_hi;
    P.uinit = (const float*)p->u_init;
    P.u = (float*)s->u;
    P.x = (float*)s->x;
    P.cost = (float*)s->cost;
    P.iters = s->iters;
    P.status = s->status;
    P.tape = store_all ? (float*)s->tape : nullptr;
    P.stg = ws + OFF_S;
    P.cand = ws + OFF_C;
    P.kh = ws + OFF_H;
    P.queue = (int*)(ws + OFF_Q);
    int* order = (int*)(ws + OFF_O);

    // one block of up to 32 instances per SM
    int ipb = (p->B + sms - 1) / sms;
    ipb = ipb < 1 ? 1 : (ipb > 32 ? 32 : ipb);
    P.ipb = ipb;
    int bps = persistent_blocks_per_sm<float>(NA_TPI);
    long long grid = (long long)(bps > 0 ? bps : 1) * sms;
    const long long need = (p->B + ipb - 1) / ipb;
    if (grid > need) grid = need;
    const cudaError_t e = launch_forward<float>(P, MPC_EXEC_PERSISTENT, NA_TPI, (int)grid, order, stream);
    return e == cudaSuccess ? MPC_OK : MPC_ERR_CUDA;
}
