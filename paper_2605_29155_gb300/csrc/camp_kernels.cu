// camp_kernels.cu -- the kernel and launch sequences of the batched MPC layer.
//
// One kernel template, k_mpc<T, TPI>, runs every phase of the method through a
// phase machine over a pack of 32 / TPI instances (a group of TPI lanes per
// instance, the pack in lockstep).  Every phase has exactly one call site, so
// every launch form executes the same machine code for it and gives
// bit-identical results.
//
// Forward (Sec. IV, Algorithm 2's inner loop):
//   persistent form (one launch): each warp pulls packs of instances from an
//     atomic work queue (longest horizon first when horizons differ) and runs
//     their whole solves -- rollout, then per iteration linearization,
//     Riccati + box QP, line search, convergence test -- and the final
//     factorization at the returned iterates, with no host round trip.  An
//     instance that converges stops updating while the rest of its pack
//     iterates.
//   plain form: Sec. IV's structure, three launches per iteration
//     (rollout + linearization, Riccati backward pass with bounds, forward
//     pass + line search) over all instances, the per-instance convergence
//     mask kept in status[].
// Backward (Sec. IV implicit differentiation): one persistent launch of the
//   adjoint LQR, replaying the tape or re-linearizing and re-factoring.
#include "camp_device.cuh"
#include "camp_internal.h"

namespace camp {

enum Phase {
    PH_INIT = 0,    // A1 rollout
    PH_LIN = 1,     // A2 linearization (iteration)
    PH_RIC = 2,     // A3 Riccati + box QP (iteration)
    PH_LS = 3,      // A4 line search + A5 convergence
    PH_FLIN = 4,    // A6 linearization at the returned iterate
    PH_FRIC = 5,    // A6 factorization -> tape
    PH_BLIN = 6,    // backward, recompute: linearization at x*
    PH_BRIC = 7,    // backward, recompute: factorization + adjoint backward sweep
    PH_BTAPE = 8,   // backward, store-all: adjoint backward sweep from the tape
    PH_BFWD = 9,    // A8 adjoint forward sweep + gradient assembly
    PH_BZERO = 10,  // backward of a failed instance: zero gradients
    PH_END = 11,    // write the forward's per-instance results
    PH_DONE = 12
};
constexpr int MODE_FWD = -1, MODE_BWD = -2;

__device__ __forceinline__ bool finished_ok(int st) {
    return st == ST_CONVERGED || st == ST_STALLED || st == ST_MAX_ITER;
}

// Whether a plain-form launch of phase `ph` applies to an instance in state `st`.
__device__ __forceinline__ bool plain_applies(int ph, int st) {
    if (ph == PH_INIT) return true;
    if (ph == PH_LIN || ph == PH_RIC || ph == PH_LS) return st == ST_RUNNING;
    return finished_ok(st);
}

__device__ __forceinline__ bool warp_any(bool v) { return __any_sync(FULL, v) != 0; }

// mode >= 0: plain form, run phase `mode` once for the pack = global warp index.
// mode == MODE_FWD / MODE_BWD: persistent forward / backward over the work queue.
// `last`: the plain line-search launch of the final iteration.
template <typename T, int TPI>
__global__ void __launch_bounds__(256, 2) k_mpc(Params<T> P, AdjArgs<T> A, int mode, int last) {
    constexpr int PACK = 32 / TPI;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Lanes<TPI> L;
    const int wib = threadIdx.x >> 5;
    WarpSmem<T>& S = reinterpret_cast<WarpSmem<T>*>(smem_raw)[wib * PACK + L.g];
    const int wglob = blockIdx.x * (blockDim.x >> 5) + wib;
    const bool plain = mode >= 0;
    bool first = true;
    for (;;) {
        int base;
        if (plain) {
            if (!first) break;
            first = false;
            base = wglob * PACK;
            if (base >= P.B) break;
        } else {
            int tk = 0;
            if (L.lane == 0) tk = atomicAdd(P.queue + (mode == MODE_BWD ? 1 : 0), PACK);
            base = __shfl_sync(FULL, tk, 0);
            if (base >= P.B) break;
        }
        const int idx = base + L.g;
        const bool valid = idx < P.B;
        const int b = valid ? (P.order ? P.order[idx] : idx) : 0;
        const Inst<T> I = make_inst(P, b, plain ? (valid ? b : 0) : wglob * PACK + L.g, valid);

        // per-instance state (uniform within the group)
        int status = ST_RUNNING, iters = 0;
        T J = T(0);
        bool ok_bwd = false;
        int ph;
        if (plain) {
            ph = mode;
            if (valid && ph != PH_INIT) {
                status = P.status[b];
                iters = P.iters[b];
                J = P.cost[b];
            }
        } else if (mode == MODE_FWD) {
            ph = PH_INIT;
        } else {
            status = valid ? P.status[b] : ST_NONFINITE;
            ok_bwd = valid && finished_ok(status);
            ph = warp_any(ok_bwd) ? (A.recompute ? PH_BLIN : PH_BTAPE) : PH_BZERO;
        }
        const bool applies = plain ? (valid && plain_applies(mode, status)) : valid;
        load_instance(P, I, S, L, applies);
        const int after_fwd = P.store_all ? PH_FLIN : PH_END;
        while (ph != PH_DONE) {
            int next = PH_DONE;
            if (ph == PH_INIT) {
                const bool act = applies;
                J = initial_rollout(P, I, S, L, act);
                if (act) {
                    if (!finiteT(J)) status = ST_NONFINITE;
                    else if (P.max_iter == 0) status = ST_MAX_ITER;
                }
                next = warp_any(act && status == ST_RUNNING) ? PH_LIN : after_fwd;
            } else if (ph == PH_LIN || ph == PH_FLIN || ph == PH_BLIN) {
                const bool act = ph == PH_LIN ? (applies && status == ST_RUNNING)
                                : (ph == PH_FLIN ? (applies && finished_ok(status)) : ok_bwd);
                if (ph == PH_LIN && act) ++iters;
                linearize(P, I, L, act);
                next = ph + 1;
            } else if (ph == PH_RIC || ph == PH_FRIC || ph == PH_BRIC || ph == PH_BTAPE) {
                const bool act = ph == PH_RIC ? (applies && status == ST_RUNNING)
                                : (ph == PH_FRIC ? (applies && finished_ok(status)) : ok_bwd);
                RicOpts<T> o;
                o.tape = ph == PH_FRIC ? P.tape : (T*)nullptr;
                o.adj = (ph == PH_BRIC || ph == PH_BTAPE) ? &A : (const AdjArgs<T>*)nullptr;
                o.replay = ph == PH_BTAPE;
                o.use_lo = ph == PH_RIC;
                const bool ok = riccati(P, I, S, L, o, act);
                if (ph == PH_RIC) {
                    if (act && !ok) status = ST_NONPD;
                    next = warp_any(act && ok) ? PH_LS : after_fwd;
                } else if (ph == PH_FRIC) {
                    if (act && !ok) status = ST_NONPD;
                    next = PH_END;
                } else {
                    ok_bwd = ok_bwd && ok;
                    next = PH_BFWD;
                }
            } else if (ph == PH_LS) {
                const bool act = applies && status == ST_RUNNING;
                T du = T(0);
                const int r = line_search(P, I, S, L, act, J, du);
                if (act) {
                    if (r) status = ST_STALLED;
                    else if (du < P.tol) status = ST_CONVERGED;
                    else if (plain ? (last != 0) : (iters >= P.max_iter)) status = ST_MAX_ITER;
                }
                next = warp_any(act && status == ST_RUNNING) ? PH_LIN : after_fwd;
            } else if (ph == PH_BFWD) {
                const T* tb = A.recompute ? (const T*)nullptr : P.tape + (size_t)I.b * P.N * TAPE_STRIDE;
                const T* Fs = A.recompute ? (const T*)I.F : tb + TAPE_F;
                const T* Ks = A.recompute ? (const T*)I.Kr : tb + TAPE_K;
                const size_t fs = A.recompute ? (size_t)NFC : (size_t)TAPE_STRIDE;
                const size_t ks = A.recompute ? (size_t)KREC : (size_t)TAPE_STRIDE;
                adjoint_forward(P, I, S, L, ok_bwd, Fs, fs, A.recompute != 0, Ks, ks, A);
                next = PH_BZERO;
            } else if (ph == PH_BZERO) {
                zero_grads(P, A, b, L, valid && !ok_bwd);
                next = PH_DONE;
            } else if (ph == PH_END) {
                next = PH_DONE;
            }
            if (plain) break;
            ph = next;
        }
        if (mode != MODE_BWD && applies && L.l == 0) {
            P.cost[b] = J;
            P.iters[b] = iters;
            P.status[b] = status;
        }
        __syncwarp();
    }
}

// Longest-horizon-first order for the work queue (counting sort, one block).
__global__ void k_lpt_order(const int* horizon, int B, int N, int* order) {
    __shared__ int cnt[MAX_N + 2];
    for (int i = threadIdx.x; i < MAX_N + 2; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        int h = horizon[b];
        h = h < 1 ? 1 : (h > N ? N : h);
        atomicAdd(&cnt[h], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int h = N; h >= 1; --h) { const int c = cnt[h]; cnt[h] = run; run += c; }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        int h = horizon[b];
        h = h < 1 ? 1 : (h > N ? N : h);
        order[atomicAdd(&cnt[h], 1)] = b;
    }
}

// ------------------------------------------------------------ host side ----
template <typename T> size_t warp_smem_bytes() { return sizeof(WarpSmem<T>); }

template <typename T> static const void* kernel_for(int tpi) {
    if (tpi == 8) return (const void*)k_mpc<T, 8>;
    if (tpi == 16) return (const void*)k_mpc<T, 16>;
    return (const void*)k_mpc<T, 32>;
}

// Allow the largest dynamic shared memory a block may need (32 instances),
// capped by the device's opt-in limit less the kernel's static tables.
template <typename T> cudaError_t prepare_kernels() {
    int dev = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    for (int tpi = 8; tpi <= 32; tpi *= 2) {
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, kernel_for<T>(tpi)))) return e;
        size_t want = (size_t)(256 / tpi) * sizeof(WarpSmem<T>);
        const size_t cap = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        if (want > cap) want = cap;
        if ((e = cudaFuncSetAttribute(kernel_for<T>(tpi), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want)))
            return e;
    }
    return cudaSuccess;
}

template <typename T> int persistent_blocks_per_sm(int tpi, int ipb) {
    int nb = 0;
    const size_t smem = (size_t)ipb * sizeof(WarpSmem<T>);
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_for<T>(tpi), tpi * ipb, smem);
    return e == cudaSuccess ? nb : 0;
}

template <typename T>
static void launch_tpi(int tpi, int grid, int threads, size_t smem, cudaStream_t st, const Params<T>& P,
                       const AdjArgs<T>& A, int mode, int last) {
    if (tpi == 8) k_mpc<T, 8><<<grid, threads, smem, st>>>(P, A, mode, last);
    else if (tpi == 16) k_mpc<T, 16><<<grid, threads, smem, st>>>(P, A, mode, last);
    else k_mpc<T, 32><<<grid, threads, smem, st>>>(P, A, mode, last);
}

template <typename T>
cudaError_t launch_forward(const Params<T>& Pin, int exec_mode, int tpi, int ipb, int grid, int* order_ws,
                           cudaStream_t st) {
    Params<T> P = Pin;
    AdjArgs<T> A{};
    const size_t smem = (size_t)ipb * sizeof(WarpSmem<T>);
    const int threads = tpi * ipb;
    cudaError_t e;
    P.order = nullptr;
    if (exec_mode == 0) {
        if ((e = cudaMemsetAsync(P.queue, 0, sizeof(int), st))) return e;
        if (P.horizon) {
            k_lpt_order<<<1, 1024, 0, st>>>(P.horizon, P.B, P.N, order_ws);
            P.order = order_ws;
        }
        launch_tpi<T>(tpi, grid, threads, smem, st, P, A, MODE_FWD, 0);
        return cudaGetLastError();
    }
    const int blocks = (P.B + ipb - 1) / ipb;
    launch_tpi<T>(tpi, blocks, threads, smem, st, P, A, PH_INIT, 0);
    for (int it = 0; it < P.max_iter; ++it) {
        launch_tpi<T>(tpi, blocks, threads, smem, st, P, A, PH_LIN, 0);
        launch_tpi<T>(tpi, blocks, threads, smem, st, P, A, PH_RIC, 0);
        launch_tpi<T>(tpi, blocks, threads, smem, st, P, A, PH_LS, it == P.max_iter - 1);
    }
    if (P.store_all) {
        launch_tpi<T>(tpi, blocks, threads, smem, st, P, A, PH_FLIN, 0);
        launch_tpi<T>(tpi, blocks, threads, smem, st, P, A, PH_FRIC, 0);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backward(const Params<T>& Pin, const AdjArgs<T>& A, int tpi, int ipb, int grid, int* order_ws,
                            cudaStream_t st) {
    Params<T> P = Pin;
    const size_t smem = (size_t)ipb * sizeof(WarpSmem<T>);
    cudaError_t e;
    if ((e = cudaMemsetAsync(P.queue + 1, 0, sizeof(int), st))) return e;
    P.order = nullptr;
    if (P.horizon) {
        k_lpt_order<<<1, 1024, 0, st>>>(P.horizon, P.B, P.N, order_ws);
        P.order = order_ws;
    }
    launch_tpi<T>(tpi, grid, tpi * ipb, smem, st, P, A, MODE_BWD, 0);
    return cudaGetLastError();
}

#define CAMP_INSTANTIATE(T)                                                                              \
    template size_t warp_smem_bytes<T>();                                                                \
    template cudaError_t prepare_kernels<T>();                                                           \
    template int persistent_blocks_per_sm<T>(int, int);                                                  \
    template cudaError_t launch_forward<T>(const Params<T>&, int, int, int, int, int*, cudaStream_t);    \
    template cudaError_t launch_backward<T>(const Params<T>&, const AdjArgs<T>&, int, int, int, int*, cudaStream_t);

CAMP_INSTANTIATE(float)
CAMP_INSTANTIATE(double)

}  // namespace camp
