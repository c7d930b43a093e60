// camp_kernels.cu -- the kernel and launch sequences of the batched MPC layer.
//
// One kernel template, k_mpc<T, NW, GEN>, runs every phase of the method through a
// phase machine over a pack of up to 32 instances (16 in FP64; one instance
// per lane, NW warps per block splitting each instance's work).  Every phase has exactly
// one call site, so every launch form executes the same machine code for it
// and gives bit-identical results.  GEN selects the stage cost: the diagonal
// form of Eq. (2) (Q, x_ref, R, u_ref) or a general C_t, c_t.
//
// Forward (Sec. IV, Algorithm 2's inner loop):
//   persistent form (one launch): each block pulls packs of instances from an
//     atomic work queue (longest horizon first when horizons differ) and runs
//     their whole solves -- rollout, then per iteration the Riccati backward
//     pass with the linearization fused in and the line search, the
//     convergence test -- and the final factorization at the returned
//     iterates, with no host round trip.  An instance that converges stops
//     updating while the rest of its pack iterates.
//   plain form: one launch per phase over all instances (rollout; per
//     iteration linearization + Riccati backward pass with bounds, forward
//     pass + line search; final factorization; output), the per-instance
//     convergence mask kept in status[].
// Backward (Sec. IV implicit differentiation): one persistent launch of the
//   adjoint LQR, replaying the tape or re-linearizing and re-factoring.
#include "camp_device.cuh"
#include "camp_internal.h"

namespace camp {

enum Phase {
    PH_INIT = 0,    // A1 rollout
    PH_RIC = 1,     // A2 + A3 linearization, Riccati + box QP (iteration)
    PH_LS = 2,      // A4 line search + A5 convergence
    PH_FRIC = 3,    // A6 linearization + factorization at the returned iterate -> tape
    PH_END = 4,     // A7 write the solution
    PH_BPREP = 5,   // backward: which instances have a solution to differentiate
    PH_BSWEEP = 6,  // A8 adjoint backward sweep (re-factorization or tape replay)
    PH_BFWD = 7,    // A8 adjoint forward sweep + gradients (zeros for failed instances)
    PH_DONE = 8
};
constexpr int MODE_FWD = -1, MODE_BWD = -2;

__device__ __forceinline__ bool finished_ok(int st) {
    return st == ST_CONVERGED || st == ST_STALLED || st == ST_MAX_ITER;
}

// Whether a plain-form launch of phase `ph` applies to an instance in state `st`.
__device__ __forceinline__ bool plain_applies(int ph, int st) {
    if (ph == PH_INIT || ph == PH_END) return true;
    if (ph == PH_RIC || ph == PH_LS) return st == ST_RUNNING;
    return finished_ok(st);
}

// Every warp holds the same per-lane state (lane l of every warp is instance l),
// so a warp vote gives the block's decision without a barrier.
__device__ __forceinline__ bool pack_any(bool v) { return __any_sync(FULL, v) != 0; }

// mode >= 0: plain form, run phase `mode` once for pack blockIdx.x.
// mode == MODE_FWD / MODE_BWD: persistent forward / backward over the work queue.
// `last`: the plain line-search launch of the final iteration.
template <typename T, int NW, bool GEN>
__global__ void __launch_bounds__(NW * 32, 8 / NW) k_mpc(const __grid_constant__ Params<T> P,
                                                          const __grid_constant__ AdjArgs<T> A, int mode, int last) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BlockSmem<T>& S = *reinterpret_cast<BlockSmem<T>*>(smem_raw);
    __shared__ int s_base;
    Lane L;
    L.w = threadIdx.x >> 5;
    L.l = threadIdx.x & 31;
    const bool plain = mode >= 0;
    for (int round = 0;; ++round) {
        int base;
        if (plain) {
            if (round > 0) break;
            base = blockIdx.x * P.ipb;
        } else {
            if (threadIdx.x == 0) s_base = atomicAdd(P.queue + (mode == MODE_BWD ? 1 : 0), P.ipb);
            __syncthreads();
            base = s_base;
        }
        if (base >= P.B) break;
        L.pos = base + L.l;
        L.valid = L.l < P.ipb && L.l < SL<T>::W && L.pos < P.B;
        L.sl = L.l < SL<T>::W ? L.l : SL<T>::W;
        L.b = L.valid ? (P.order ? P.order[L.pos] : L.pos) : 0;
        int nh = P.horizon ? P.horizon[L.b] : P.N;
        nh = nh < 1 ? 1 : (nh > P.N ? P.N : nh);
        const int n = L.valid ? nh : 0;
        load_constants<T, NW, GEN>(P, S, L);

        // per-instance state, the same in every warp
        int status = ST_RUNNING, iters = 0;
        T J = T(0);
        bool okb = false;                  // backward: the instance has a solution to differentiate
        int ph = plain ? mode : (mode == MODE_BWD ? PH_BPREP : PH_INIT);
        if (plain && L.valid && ph != PH_INIT) {
            status = P.status[L.b];
            iters = P.iters[L.b];
            J = P.cost[L.b];
        }
        const bool applies = plain ? (L.valid && plain_applies(mode, status)) : L.valid;
        __syncthreads();
        const int after_fwd = P.store_all ? PH_FRIC : PH_END;
        while (ph != PH_DONE) {
            int next = PH_DONE;
            if (ph == PH_INIT) {
                const bool act = applies;
                load_stage_rows<T, NW, GEN>(P, L, act ? n : 0, false);
                __syncthreads();
                initial_rollout<T, NW, GEN>(P, S, L, act ? n : 0);
                __syncthreads();
                J = S.Jc[0][L.sl];
                if (act) {
                    if (!finiteT(J)) status = ST_NONFINITE;
                    else if (P.max_iter == 0) status = ST_MAX_ITER;
                }
                next = pack_any(act && status == ST_RUNNING) ? PH_RIC : after_fwd;
                __syncthreads();
            } else if (ph == PH_RIC || ph == PH_FRIC || ph == PH_BSWEEP) {
                // every Riccati sweep of the method, from this one call site
                bool act;
                RicOpts<T> o{nullptr, nullptr, false, false};
                if (ph == PH_RIC) {
                    act = applies && status == ST_RUNNING;
                    if (act) ++iters;
                    o.use_lo = true;
                } else if (ph == PH_FRIC) {
                    act = applies && finished_ok(status);
                    o.tape = P.tape;
                } else {
                    act = okb;
                    o.adj = &A;
                    o.replay = !A.recompute;
                }
                const bool ok = riccati<T, NW, GEN>(P, S, L, act ? n : 0, o);
                if (ph == PH_RIC) {
                    if (act && !ok) status = ST_NONPD;
                    next = pack_any(act && ok) ? PH_LS : after_fwd;
                } else if (ph == PH_FRIC) {
                    if (act && !ok) status = ST_NONPD;
                    next = PH_END;
                } else {
                    okb = okb && ok;
                    next = PH_BFWD;
                }
                __syncthreads();
            } else if (ph == PH_LS) {
                const bool act = applies && status == ST_RUNNING;
                T du = T(0);
                const int r = line_search<T, NW, GEN>(P, S, L, act ? n : 0, J, du);
                if (act) {
                    if (r) status = ST_STALLED;
                    else if (du < P.tol) status = ST_CONVERGED;
                    else if (plain ? (last != 0) : (iters >= P.max_iter)) status = ST_MAX_ITER;
                }
                next = pack_any(act && status == ST_RUNNING) ? PH_RIC : after_fwd;
            } else if (ph == PH_END) {
                if constexpr (!GEN) {
                    if (L.w == 0 && applies && finiteT(J)) J = final_cost<T>(P, S, L, n);
                }
                write_solution<T, NW>(P, L, applies ? n : 0);
                next = PH_DONE;
            } else if (ph == PH_BPREP) {
                const int st = L.valid ? P.status[L.b] : ST_NONFINITE;
                okb = L.valid && finished_ok(st);
                next = PH_BFWD;
                if (pack_any(okb)) {
                    if (A.recompute) load_stage_rows<T, NW, GEN>(P, L, okb ? n : 0, true);
                    next = PH_BSWEEP;
                }
                __syncthreads();
            } else if (ph == PH_BFWD) {
                adjoint_forward<T, NW, GEN>(P, S, L, okb ? n : 0, A);
                if constexpr (GEN) {
                    __syncthreads();
                    assemble_dC<T, NW>(P, A, L, okb ? n : 0);
                }
                zero_grads<T, NW, GEN>(P, A, L, L.valid && !okb);
                next = PH_DONE;
            }
            if (plain) break;
            ph = next;
        }
        if (mode != MODE_BWD && applies && L.w == 0) {
            P.cost[L.b] = J;
            P.iters[L.b] = iters;
            P.status[L.b] = status;
        }
        __syncthreads();
        // After A7 the pack's stage records are dead (the backward writes its
        // own): when the pack owns whole groups, their lines leave L2 without
        // a write-back.
        if ((mode == MODE_FWD || mode == PH_END) && P.ipb == GW && base % GW == 0) {
            const int nmax = __reduce_max_sync(FULL, n);
            l2_discard(P.stg + srow(P, base, 0, 0), (size_t)nmax * SREC * GW * sizeof(T));
        }
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
template <typename T> size_t block_smem_bytes() { return sizeof(BlockSmem<T>); }

// Dynamic shared memory of a block: BlockSmem, plus the shared C of the
// general cost behind it for those kernels.
template <typename T> static size_t smem_for(bool gen) {
    return sizeof(BlockSmem<T>) + (gen ? gen_smem_bytes<T>() : 0);
}

// The kernel for nw warps per block, with the diagonal cost (gen false) or the
// general cost of Eq. (2).
template <typename T> static const void* kernel_for(int nw, bool gen = false) {
    if (gen) return nw == 8 ? (const void*)k_mpc<T, 8, true> : (const void*)k_mpc<T, 4, true>;
    return nw == 8 ? (const void*)k_mpc<T, 8, false> : (const void*)k_mpc<T, 4, false>;
}

template <typename T> cudaError_t prepare_kernels() {
    cudaError_t e;
    for (int g = 0; g < 2; ++g)
        for (int nw = 4; nw <= 8; nw *= 2) {
            if ((e = cudaFuncSetAttribute(kernel_for<T>(nw, g == 1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_for<T>(g == 1))))
                return e;
        }
    return cudaSuccess;
}

template <typename T> int persistent_blocks_per_sm(int nw) {
    int nb = 1 << 30;
    for (int g = 0; g < 2; ++g) {
        int k = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, kernel_for<T>(nw, g == 1), nw * 32,
                                                          smem_for<T>(g == 1)) != cudaSuccess)
            return 0;
        nb = k < nb ? k : nb;
    }
    return nb;
}

template <typename T>
static void launch_nw(int nw, int grid, cudaStream_t st, const Params<T>& P, const AdjArgs<T>& A, int mode,
                      int last) {
    const size_t smem = smem_for<T>(P.Cg != nullptr);
    if (P.Cg) {
        if (nw == 8) k_mpc<T, 8, true><<<grid, 256, smem, st>>>(P, A, mode, last);
        else k_mpc<T, 4, true><<<grid, 128, smem, st>>>(P, A, mode, last);
    } else {
        if (nw == 8) k_mpc<T, 8, false><<<grid, 256, smem, st>>>(P, A, mode, last);
        else k_mpc<T, 4, false><<<grid, 128, smem, st>>>(P, A, mode, last);
    }
}

template <typename T>
cudaError_t launch_forward(const Params<T>& Pin, int exec_mode, int nw, int grid, int* order_ws, cudaStream_t st) {
    Params<T> P = Pin;
    AdjArgs<T> A{};
    cudaError_t e;
    P.order = nullptr;
    if (P.horizon) {
        k_lpt_order<<<1, 1024, 0, st>>>(P.horizon, P.B, P.N, order_ws);
        P.order = order_ws;
    }
    if (exec_mode == 0) {
        if ((e = cudaMemsetAsync(P.queue, 0, sizeof(int), st))) return e;
        launch_nw<T>(nw, grid, st, P, A, MODE_FWD, 0);
        return cudaGetLastError();
    }
    // exec_mode 2: the plain form with one instance per block and, for the
    // diagonal cost, the stage-parallel Riccati phase (camp_scan.cu)
    const bool scan = exec_mode == 2;
    if (scan) P.ipb = 1;
    const int blocks = (P.B + P.ipb - 1) / P.ipb;
    launch_nw<T>(nw, blocks, st, P, A, PH_INIT, 0);
    for (int it = 0; it < P.max_iter; ++it) {
        if (scan && !P.Cg) {
            if ((e = launch_scan_ric<T>(P, st, 0))) return e;
        } else {
            launch_nw<T>(nw, blocks, st, P, A, PH_RIC, 0);
        }
        launch_nw<T>(nw, blocks, st, P, A, PH_LS, it == P.max_iter - 1);
    }
    if (P.store_all) {
        if (scan && !P.Cg) {
            if ((e = launch_scan_ric<T>(P, st, 1))) return e;
        } else {
            launch_nw<T>(nw, blocks, st, P, A, PH_FRIC, 0);
        }
    }
    launch_nw<T>(nw, blocks, st, P, A, PH_END, 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backward(const Params<T>& Pin, const AdjArgs<T>& A, int nw, int grid, int* order_ws,
                            cudaStream_t st) {
    Params<T> P = Pin;
    cudaError_t e;
    if ((e = cudaMemsetAsync(P.queue + 1, 0, sizeof(int), st))) return e;
    P.order = nullptr;
    if (P.horizon) {
        k_lpt_order<<<1, 1024, 0, st>>>(P.horizon, P.B, P.N, order_ws);
        P.order = order_ws;
    }
    launch_nw<T>(nw, grid, st, P, A, MODE_BWD, 0);
    return cudaGetLastError();
}

#define CAMP_INSTANTIATE(T)                                                                              \
    template size_t block_smem_bytes<T>();                                                               \
    template cudaError_t prepare_kernels<T>();                                                           \
    template int persistent_blocks_per_sm<T>(int);                                                       \
    template cudaError_t launch_forward<T>(const Params<T>&, int, int, int, int*, cudaStream_t);         \
    template cudaError_t launch_backward<T>(const Params<T>&, const AdjArgs<T>&, int, int, int*, cudaStream_t);

CAMP_INSTANTIATE(float)
CAMP_INSTANTIATE(double)

}  // namespace camp
