// camp_kernels.cu -- kernels and launch sequences of the batched MPC layer.
//
// Forward (Sec. IV, Algorithm 2's inner loop):
//   persistent form: one launch; each warp pulls instances from an atomic work
//     queue (longest horizon first when horizons differ) and runs the whole
//     iLQR solve of that instance -- rollout, then per iteration linearization,
//     Riccati + box QP, line search, convergence test -- and the final
//     factorization at the returned iterate, with no host round trip.
//   plain form: Sec. IV's structure, three launches per iteration
//     (rollout + linearization, Riccati backward pass with bounds, forward
//     pass + line search) over all instances, with per-instance convergence
//     masks in status[]; it shares every device function with the persistent
//     form and gives bit-identical results.
// Backward (Sec. IV implicit differentiation): one persistent launch of the
//   adjoint LQR sweep, from the tape or with the linearization recomputed.
#include "camp_device.cuh"
#include "camp_internal.h"

namespace camp {

__device__ void init_tables(int* triQ, int* triV) {
    for (int p = threadIdx.x; p < NTRI_Q; p += blockDim.x) {
        int a = 0, r = p;
        while (r >= NZ - a) { r -= NZ - a; ++a; }
        triQ[p] = (a << 8) | (a + r);
    }
    for (int p = threadIdx.x; p < NTRI_V; p += blockDim.x) {
        int a = 0, r = p;
        while (r >= NX - a) { r -= NX - a; ++a; }
        triV[p] = (a << 8) | (a + r);
    }
}

template <typename T>
__device__ void solve_one(const Params<T>& P, int b, int slot, WarpSmem<T>& S, int lane,
                          const int* triQ, const int* triV) {
    const Inst<T> I = make_inst(P, b, slot);
    load_instance(P, I, S, lane);
    T J = initial_rollout(P, I, S, lane);
    int status = ST_MAX_ITER, iters = 0;
    if (!finiteT(J)) {
        status = ST_NONFINITE;
    } else {
        for (int it = 0; it < P.max_iter; ++it) {
            iters = it + 1;
            linearize(P, I, I.F, lane);
            if (!riccati(P, I, S, lane, triQ, triV, I.F, (T*)nullptr, (const AdjArgs<T>*)nullptr)) {
                status = ST_NONPD;
                break;
            }
            T du = T(0);
            if (line_search(P, I, S, lane, J, du)) { status = ST_STALLED; break; }
            if (du < P.tol) { status = ST_CONVERGED; break; }
        }
        if (P.store_all && status != ST_NONPD) {
            linearize(P, I, I.F, lane);
            if (!riccati(P, I, S, lane, triQ, triV, I.F, P.tape, (const AdjArgs<T>*)nullptr)) status = ST_NONPD;
        }
    }
    if (lane == 0) { P.cost[b] = J; P.iters[b] = iters; P.status[b] = status; }
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ WarpSmem<T>& warp_smem(unsigned char* raw) {
    return reinterpret_cast<WarpSmem<T>*>(raw)[threadIdx.x >> 5];
}

// ---------------------------------------------------------------- forward ---
template <typename T>
__global__ void __launch_bounds__(256) k_fused(Params<T> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int triQ[NTRI_Q], triV[NTRI_V];
    init_tables(triQ, triV);
    __syncthreads();
    WarpSmem<T>& S = warp_smem<T>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(P.queue, 1);
        idx = __shfl_sync(FULL, idx, 0);
        if (idx >= P.B) break;
        const int b = P.order ? P.order[idx] : idx;
        solve_one(P, b, slot, S, lane, triQ, triV);
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

// plain form: one warp per instance, instance index = slot
template <typename T>
__global__ void __launch_bounds__(256) k_plain_init(Params<T> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem<T>& S = warp_smem<T>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= P.B) return;
    const Inst<T> I = make_inst(P, b, b);
    load_instance(P, I, S, lane);
    const T J = initial_rollout(P, I, S, lane);
    if (lane == 0) {
        P.cost[b] = J;
        P.iters[b] = 0;
        P.status[b] = finiteT(J) ? (P.max_iter > 0 ? ST_RUNNING : ST_MAX_ITER) : ST_NONFINITE;
    }
}

__device__ __forceinline__ bool plain_active(int st, int final_pass) {
    return final_pass ? (st == ST_CONVERGED || st == ST_STALLED || st == ST_MAX_ITER) : (st == ST_RUNNING);
}

template <typename T>
__global__ void __launch_bounds__(256) k_plain_lin(Params<T> P, int final_pass) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= P.B) return;
    const int st = P.status[b];
    if (!plain_active(st, final_pass)) return;
    const Inst<T> I = make_inst(P, b, b);
    if (!final_pass && lane == 0) P.iters[b] += 1;
    linearize(P, I, I.F, lane);
}

template <typename T>
__global__ void __launch_bounds__(256) k_plain_ric(Params<T> P, int final_pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int triQ[NTRI_Q], triV[NTRI_V];
    init_tables(triQ, triV);
    __syncthreads();
    WarpSmem<T>& S = warp_smem<T>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= P.B) return;
    const int st = P.status[b];
    if (!plain_active(st, final_pass)) return;
    const Inst<T> I = make_inst(P, b, b);
    load_instance(P, I, S, lane);
    const bool ok = riccati(P, I, S, lane, triQ, triV, I.F, final_pass ? P.tape : (T*)nullptr,
                            (const AdjArgs<T>*)nullptr);
    if (!ok && lane == 0) P.status[b] = ST_NONPD;
}

template <typename T>
__global__ void __launch_bounds__(256) k_plain_ls(Params<T> P, int last) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem<T>& S = warp_smem<T>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= P.B) return;
    if (P.status[b] != ST_RUNNING) return;
    const Inst<T> I = make_inst(P, b, b);
    load_instance(P, I, S, lane);
    T J = P.cost[b];
    T du = T(0);
    const int r = line_search(P, I, S, lane, J, du);
    if (lane == 0) {
        int st = ST_RUNNING;
        if (r) st = ST_STALLED;
        else if (du < P.tol) st = ST_CONVERGED;
        else if (last) st = ST_MAX_ITER;
        P.cost[b] = J;
        P.status[b] = st;
    }
}

// --------------------------------------------------------------- backward ---
template <typename T>
__device__ void adjoint_backward_tape(const Params<T>& P, const Inst<T>& I, WarpSmem<T>& S, int lane,
                                      const AdjArgs<T>& A) {
    const int n = I.n;
    if (lane < NX) S.vh[lane] = T(0);
    __syncwarp();
    for (int t = n - 1; t >= 0; --t) {
        const T* rec = P.tape + ((size_t)I.b * P.N + t) * TAPE_STRIDE;
        if (lane < NZ) {
            T g;
            if (lane < NX) g = A.gx ? A.gx[((size_t)I.b * P.N + t) * NX + lane] : T(0);
            else g = A.gu[((size_t)I.b * P.N + t) * NU + lane - NX];
            if (t < n - 1) {
#pragma unroll
                for (int k = 0; k < NX; ++k) g += rec[TAPE_F + lane * NX + k] * S.vh[k];
            }
            S.qh[lane] = g;
        }
        __syncwarp();
        if (lane < NX) {
            T s = S.qh[lane];
#pragma unroll
            for (int a = 0; a < NU; ++a) s += rec[TAPE_K + a * NX + lane] * S.qh[NX + a];
            S.vh[lane] = s;
        } else if (lane == 16) {
            const int mask = (int)rec[TAPE_MASK];
            T L[10], rhs[4], y[4];
#pragma unroll
            for (int i = 0; i < 10; ++i) L[i] = rec[TAPE_L + i];
#pragma unroll
            for (int a = 0; a < 4; ++a) rhs[a] = ((mask >> a) & 1) ? S.qh[NX + a] : T(0);
            chol_solve4(L, rhs, y);
#pragma unroll
            for (int a = 0; a < 4; ++a) I.kh[t * NU + a] = ((mask >> a) & 1) ? -y[a] : T(0);
        }
        __syncwarp();
    }
}

template <typename T>
__device__ void zero_grads(const Params<T>& P, const AdjArgs<T>& A, int b, int lane) {
    for (int e = lane; e < P.Nq * NX; e += 32) A.dQ[(size_t)b * P.Nq * NX + e] = T(0);
    for (int e = lane; e < P.N * NX; e += 32) A.dxref[(size_t)b * P.N * NX + e] = T(0);
    if (lane < NX) A.dx0[(size_t)b * NX + lane] = T(0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_adjoint(Params<T> P, AdjArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int triQ[NTRI_Q], triV[NTRI_V];
    init_tables(triQ, triV);
    __syncthreads();
    WarpSmem<T>& S = warp_smem<T>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(P.queue + 1, 1);
        idx = __shfl_sync(FULL, idx, 0);
        if (idx >= P.B) break;
        const int b = P.order ? P.order[idx] : idx;
        const int st = P.status[b];
        if (!(st == ST_CONVERGED || st == ST_STALLED || st == ST_MAX_ITER)) {
            zero_grads(P, A, b, lane);
            __syncwarp();
            continue;
        }
        const Inst<T> I = make_inst(P, b, slot);
        load_instance(P, I, S, lane);
        if (A.recompute) {
            linearize(P, I, I.F, lane);
            if (!riccati(P, I, S, lane, triQ, triV, I.F, (T*)nullptr, &A)) {
                zero_grads(P, A, b, lane);
                __syncwarp();
                continue;
            }
            adjoint_forward(P, I, S, lane, I.F, (size_t)NF, I.Kr, (size_t)KREC, A);
        } else {
            adjoint_backward_tape(P, I, S, lane, A);
            const T* tb = P.tape + (size_t)I.b * P.N * TAPE_STRIDE;
            adjoint_forward(P, I, S, lane, tb + TAPE_F, (size_t)TAPE_STRIDE, tb + TAPE_K, (size_t)TAPE_STRIDE, A);
        }
    }
}

// ------------------------------------------------------------ host side ----
template <typename T> size_t warp_smem_bytes() { return sizeof(WarpSmem<T>); }

template <typename T> cudaError_t prepare_kernels() {
    const int maxb = (int)(8 * sizeof(WarpSmem<T>));
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
    if ((e = cudaFuncSetAttribute(k_plain_init<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
    if ((e = cudaFuncSetAttribute(k_plain_ric<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
    if ((e = cudaFuncSetAttribute(k_plain_ls<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
    if ((e = cudaFuncSetAttribute(k_adjoint<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
    return cudaSuccess;
}

template <typename T> int persistent_blocks_per_sm(int ipb, int which) {
    int nb = 0;
    const size_t smem = (size_t)ipb * sizeof(WarpSmem<T>);
    cudaError_t e = which == 0
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fused<T>, 32 * ipb, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adjoint<T>, 32 * ipb, smem);
    return e == cudaSuccess ? nb : 0;
}

template <typename T>
cudaError_t launch_forward(const Params<T>& Pin, int exec_mode, int ipb, int grid, int* order_ws,
                           cudaStream_t st) {
    Params<T> P = Pin;
    const size_t smem = (size_t)ipb * sizeof(WarpSmem<T>);
    const int threads = 32 * ipb;
    cudaError_t e;
    if (exec_mode == 0) {
        if ((e = cudaMemsetAsync(P.queue, 0, 2 * sizeof(int), st))) return e;
        P.order = nullptr;
        if (P.horizon) {
            k_lpt_order<<<1, 1024, 0, st>>>(P.horizon, P.B, P.N, order_ws);
            P.order = order_ws;
        }
        k_fused<T><<<grid, threads, smem, st>>>(P);
        return cudaGetLastError();
    }
    P.order = nullptr;
    const int blocks = (P.B + ipb - 1) / ipb;
    k_plain_init<T><<<blocks, threads, smem, st>>>(P);
    for (int it = 0; it < P.max_iter; ++it) {
        k_plain_lin<T><<<blocks, threads, 0, st>>>(P, 0);
        k_plain_ric<T><<<blocks, threads, smem, st>>>(P, 0);
        k_plain_ls<T><<<blocks, threads, smem, st>>>(P, it == P.max_iter - 1);
    }
    if (P.store_all) {
        k_plain_lin<T><<<blocks, threads, 0, st>>>(P, 1);
        k_plain_ric<T><<<blocks, threads, smem, st>>>(P, 1);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backward(const Params<T>& Pin, const AdjArgs<T>& A, int ipb, int grid, int* order_ws,
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
    k_adjoint<T><<<grid, 32 * ipb, smem, st>>>(P, A);
    return cudaGetLastError();
}

#define CAMP_INSTANTIATE(T)                                                                              \
    template size_t warp_smem_bytes<T>();                                                                \
    template cudaError_t prepare_kernels<T>();                                                           \
    template int persistent_blocks_per_sm<T>(int, int);                                                  \
    template cudaError_t launch_forward<T>(const Params<T>&, int, int, int, int*, cudaStream_t);         \
    template cudaError_t launch_backward<T>(const Params<T>&, const AdjArgs<T>&, int, int, int*, cudaStream_t);

CAMP_INSTANTIATE(float)
CAMP_INSTANTIATE(double)

}  // namespace camp
