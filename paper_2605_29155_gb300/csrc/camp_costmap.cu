// camp_costmap.cu -- the actor's cost map (Sec. V-A, Sec. III-C) on the
// tensor cores: an MLP with two hidden layers of 512 ReLU units and a sigmoid
// output scaled to the cost weights' bounds, observation -> per-stage Q_t, and
// its backward from dL/dQ (the MPC adjoint's gradient) to the weights.
//
// Every layer is one dense contraction, run by one kernel: C = A B' on 5th
// generation tensor cores (tcgen05.mma, kind::tf32, one 128 x 128 FP32
// accumulator tile in tensor memory per CTA), with the layer's bias and
// activation fused into the epilogue that reads the accumulator back
// (tcgen05.ld).  FP32 accuracy comes from the 3xTF32 split (Ootomo & Yokota,
// "Recovering single precision accuracy from Tensor Cores while surpassing the
// FP32 theoretical peak performance", 2022): each operand x is split into
// x_hi = tf32(x) and x_lo = tf32(x - x_hi), and A B' = A_hi B_hi' + A_hi B_lo'
// + A_lo B_hi' to within FP32 rounding.
//
// Operands are staged in shared memory by the CTA's threads in the canonical
// K-major layout without swizzle (8-row x 16-byte core matrices), through
// accessors that also assemble the observation [x_init; x_ref,0], append the
// row of ones whose product gives a bias gradient, and form dL/da3 =
// dL/dQ (q_hi - q_lo) s (1 - s) on the fly.  Two stages of K = 16 alternate:
// while the tensor core works on one, the threads split the next stage's
// elements (read into registers a trip earlier) into the other, once an
// mbarrier signalled by tcgen05.commit tells that it is free, and send out the
// reads of the stage after.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "camp.h"
#include "camp_costmap.h"

namespace cmap {

constexpr int TM = 128;             // rows of an accumulator tile (M of one MMA)
constexpr int TN = 128;             // columns (N of one MMA), = TMEM columns
constexpr int TK = 16;              // K of one pipeline stage: two MMA k-steps of 8
constexpr int THREADS = 256;        // 8 warps: warp w reads TMEM lanes 32 (w % 4) .., columns 64 (w / 4) ..
constexpr int TILE_FLOATS = TM * TK;                // one operand tile (TM == TN)
constexpr int STAGE_FLOATS = 4 * TILE_FLOATS;       // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM_BYTES = 2 * STAGE_FLOATS * 4 + 64;
constexpr long long WAIT_LIMIT = 1ll << 24;         // bounded mbarrier waits
constexpr int SPLIT_MIN_K = 1024;                   // contractions this long are split over K ...
constexpr int SPLIT_MAX = 32;                       // ... into at most this many parts
constexpr int SPLIT_CHUNK = 128;                    // of at least this K each

// Operand kinds: how element (r, k) of A (r = m) or B (r = n) is read.
enum Kind {
    K_PLAIN = 0,      // p[r s0 + k s1], r < rows, k < K
    K_ONES_ROW = 1,   // as K_PLAIN for r < rows; r == rows gives 1 (bias-gradient row)
    K_OBS = 2,        // the observation: o(b, j) = j < 13 ? x0[b, j] : x_ref[b, 0, j - 13], with
                      // (b, j) = (r, k) (s0 = 0) or (k, r) (s0 = 1); r == rows gives 1 when ones
    K_DA3 = 3         // dL/da3 = dQ (q_hi - q_lo) s (1 - s), dQ = p, s = p2, at p[r s0 + k s1]
};

struct Operand {
    const float* p;
    const float* p2;
    long long s0, s1;
    int rows;         // valid rows (r >= rows reads 0, except a ones row)
    int kind;
    int ones;         // K_OBS: add the ones row at r == rows
    int ld2;          // K_OBS: x_ref row stride (N * 13)
};

enum Epi {
    E_STORE = 0,      // C[m, n] = acc
    E_BIAS_RELU = 1,  // C[m, n] = max(acc + bias[n], 0)
    E_SIGQ = 2,       // s = sigmoid(acc + bias[n]); C2[m, n] = s; C[m, n] = q_lo + (q_hi - q_lo) s
    E_MASK = 3,       // C[m, n] = acc * (H[m, n] > 0), H = C2
    E_SPLIT = 4       // m < M - 1: C[m, n] = acc; m == M - 1: C2[n] = acc (weight and bias gradients)
};

struct Gemm {
    Operand A, B;
    int M, N, K;
    int epi;
    const float* bias;
    float* C;
    long long ldc;
    float* C2;
    long long ldc2;
    float q_lo, q_hi;
    int* err;
    int kper;           // split-K: K per part (a multiple of TK); 0 = no split
    float* part;        // split-K: [parts, M, N] partial accumulators
};

__device__ __forceinline__ float load_op(const Operand& o, int r, int k, int K, float q_span) {
    if (k >= K) return 0.f;
    if (o.kind == K_OBS) {
        int b = o.s0 ? k : r, j = o.s0 ? r : k;
        if (r == o.rows) return o.ones ? 1.f : 0.f;
        if (r > o.rows) return 0.f;
        return j < 13 ? o.p[(long long)b * 13 + j] : o.p2[(long long)b * o.ld2 + (j - 13)];
    }
    if (r >= o.rows) return (o.kind == K_ONES_ROW && r == o.rows) ? 1.f : 0.f;
    const long long i = (long long)r * o.s0 + (long long)k * o.s1;
    if (o.kind == K_DA3) {
        const float s = o.p2[i];
        return o.p[i] * q_span * s * (1.f - s);
    }
    return o.p[i];
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Float offset of element (r, k) of a [128 x TK] tile in the canonical K-major
// layout without swizzle: core matrices of 8 rows x 4 floats (128 contiguous
// bytes), the TK / 4 cores of an 8-row group side by side.
__device__ __forceinline__ int core_off(int r, int k) { return ((r >> 3) * (TK / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }

// Shared-memory matrix descriptor of tcgen05: start address, leading-dimension
// byte offset (between the core matrices adjacent in K), stride-dimension byte
// offset (between the 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of tcgen05.mma kind::tf32: FP32 accumulator, TF32
// A and B, both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void put_split(float* hi, float* lo, int off, float x) {
    const uint32_t h = to_tf32(x);
    hi[off] = __uint_as_float(h);
    lo[off] = __uint_as_float(to_tf32(x - __uint_as_float(h)));
}

// One K = TK stage of A (rows r0..r0+127) or B, in two steps so that the
// global reads of the next stage overlap the tensor core's work on this one:
// gather_tile reads the thread's EPT elements into registers, scatter_tile
// splits them into hi / lo TF32 tiles in shared memory.  The thread-to-element
// map depends on which dimension the operand is contiguous in:
//   k (k-fast): four consecutive k of one row per group, one vector load where
//     16-byte aligned and in bounds, and one 16-byte store per tile (the four
//     are adjacent in a core matrix; a quarter-warp fills one core matrix);
//   r (r-fast): each warp store covers one whole 8 x 4 core matrix (lane l at
//     row l % 8, k l / 8), so the 32 stores hit 32 banks; its reads are 32-byte
//     runs of 8 rows at four k.
// The observation and ragged or misaligned edges take the scalar path.
constexpr int EPT = TM * TK / THREADS;              // elements per thread and tile
constexpr int GROUPS = EPT / 4;                     // k-fast: groups of four

__device__ __forceinline__ bool k_fast(const Operand& o) { return o.kind == K_OBS ? o.s0 == 0 : o.s1 == 1; }

// k-fast group g: (r, k .. k + 3), a row of one core matrix.  Each
// quarter-warp writes one whole core matrix (rows 8 rb .. 8 rb + 7 at k-block
// lane / 8: 128 contiguous bytes), and a warp reads 8 rows x 16 k.
__device__ __forceinline__ void kf_pos(int g, int& r, int& k) {
    const int lane = threadIdx.x & 31, rb = (threadIdx.x >> 5) * GROUPS + g;
    r = rb * 8 + (lane & 7);
    k = (lane >> 3) * 4;
}
// r-fast element q: core matrix cm = (threadIdx.x / 32) * EPT + q, at row
// 8 (cm / (TK / 4)) + lane % 8 and k 4 (cm % (TK / 4)) + lane / 8
__device__ __forceinline__ void rf_pos(int q, int& r, int& k) {
    const int lane = threadIdx.x & 31, cm = (threadIdx.x >> 5) * EPT + q;
    r = (cm / (TK / 4)) * 8 + (lane & 7);
    k = (cm % (TK / 4)) * 4 + (lane >> 3);
}

__device__ __forceinline__ void gather_tile(const Operand& o, int r0, int k0, int K, float q_span, float (&v)[EPT]) {
    if (!k_fast(o)) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            int r, k;
            rf_pos(q, r, k);
            v[q] = load_op(o, r0 + r, k0 + k, K, q_span);
        }
        return;
    }
#pragma unroll
    for (int g = 0; g < GROUPS; ++g) {
        int r, k;
        kf_pos(g, r, k);
        const int rr = r0 + r, kk = k0 + k;
        bool vec = o.kind != K_OBS && kk + 3 < K && rr < o.rows;
        const long long i0 = (long long)rr * o.s0 + (long long)kk * o.s1;
        vec = vec && ((((size_t)(o.p + i0)) & 15) == 0) && (o.kind != K_DA3 || ((((size_t)(o.p2 + i0)) & 15) == 0));
        if (vec) {
            float4 x = *reinterpret_cast<const float4*>(o.p + i0);
            if (o.kind == K_DA3) {
                const float4 sv = *reinterpret_cast<const float4*>(o.p2 + i0);
                x.x *= q_span * sv.x * (1.f - sv.x);
                x.y *= q_span * sv.y * (1.f - sv.y);
                x.z *= q_span * sv.z * (1.f - sv.z);
                x.w *= q_span * sv.w * (1.f - sv.w);
            }
            v[4 * g + 0] = x.x;
            v[4 * g + 1] = x.y;
            v[4 * g + 2] = x.z;
            v[4 * g + 3] = x.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) v[4 * g + j] = load_op(o, rr, kk + j, K, q_span);
        }
    }
}

__device__ __forceinline__ void scatter_tile(const Operand& o, const float (&v)[EPT], float* hi, float* lo) {
    if (!k_fast(o)) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            int r, k;
            rf_pos(q, r, k);
            put_split(hi, lo, core_off(r, k), v[q]);
        }
        return;
    }
#pragma unroll
    for (int g = 0; g < GROUPS; ++g) {
        int r, k;
        kf_pos(g, r, k);
        float4 h, l;
        float* hp = &h.x;
        float* lp = &l.x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t t = to_tf32(v[4 * g + j]);
            hp[j] = __uint_as_float(t);
            lp[j] = __uint_as_float(to_tf32(v[4 * g + j] - __uint_as_float(t)));
        }
        const int off = core_off(r, k);                 // k % 4 == 0: 16-byte aligned
        *reinterpret_cast<float4*>(hi + off) = h;
        *reinterpret_cast<float4*>(lo + off) = l;
    }
}

__global__ void __launch_bounds__(THREADS, 1) k_gemm_3xtf32(const __grid_constant__ Gemm g) {
    extern __shared__ __align__(1024) float sm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const float q_span = g.q_hi - g.q_lo;
    // this CTA's range of K: all of it, or part blockIdx.z of a split
    const int kbeg = g.kper ? blockIdx.z * g.kper : 0;
    const int kend = g.kper ? min(g.K, kbeg + g.kper) : g.K;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    const int nk = (kend - kbeg + TK - 1) / TK;
    auto stage = [&](int s) { return sm + s * STAGE_FLOATS; };
    float va[EPT], vb[EPT];                         // the next stage's elements, read ahead
    auto gather = [&](int c) {
        gather_tile(g.A, m0, kbeg + c * TK, kend, q_span, va);
        gather_tile(g.B, n0, kbeg + c * TK, kend, q_span, vb);
    };
    auto scatter = [&](int c) {
        float* st = stage(c & 1);
        scatter_tile(g.A, va, st, st + TILE_FLOATS);
        scatter_tile(g.B, vb, st + 2 * TILE_FLOATS, st + 3 * TILE_FLOATS);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };
    gather(0);
    scatter(0);
    if (nk > 1) gather(1);
    __syncthreads();
    bool ok = true;
    int issued = -1;                    // the last chunk whose MMAs were committed
    for (int c = 0; c < nk; ++c) {
        issued = c;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float* st = stage(c & 1);
            const uint32_t a_hi = smem_u32(st), a_lo = smem_u32(st + TILE_FLOATS);
            const uint32_t b_hi = smem_u32(st + 2 * TILE_FLOATS), b_lo = smem_u32(st + 3 * TILE_FLOATS);
#pragma unroll
            for (int j = 0; j < TK / 8; ++j) {
                const uint32_t off = j * 256;            // two 16-byte K cores per k-step of 8
                const uint32_t lbo = 128, sbo = (TK / 4) * 128;
                const uint32_t first = (c == 0 && j == 0) ? 0u : 1u;
                mma_tf32(tmem, smem_desc(a_lo + off, lbo, sbo), smem_desc(b_hi + off, lbo, sbo), first);
                mma_tf32(tmem, smem_desc(a_hi + off, lbo, sbo), smem_desc(b_lo + off, lbo, sbo), 1u);
                mma_tf32(tmem, smem_desc(a_hi + off, lbo, sbo), smem_desc(b_hi + off, lbo, sbo), 1u);
            }
            mma_commit(smem_u32(&mbar[c & 1]));
        }
        if (c + 1 < nk) {
            // chunk c + 1's elements were read during the previous trip; its
            // stage (c + 1) & 1 was last read by the MMAs of chunk c - 1.  The
            // reads of chunk c + 2 then go out for the next trip.
            if (c >= 1 && !mbar_wait(smem_u32(&mbar[(c - 1) & 1]), ((c - 1) >> 1) & 1)) ok = false;
            if (!__syncthreads_and(ok)) { ok = false; break; }
            scatter(c + 1);
            if (c + 2 < nk) gather(c + 2);
            __syncthreads();
        }
    }
    // the last issued chunk's commit covers every MMA issued before it; this
    // (bounded) wait also runs after a failure, before the memory is freed
    if (issued >= 0 && !mbar_wait(smem_u32(&mbar[issued & 1]), (issued >> 1) & 1)) ok = false;
    if (!__syncthreads_and(ok)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // warp w reads the accumulator rows of its TMEM lane quarter, in the
        // columns of its half
        const int quarter = warp & 3, half = warp >> 2;
        const int m = m0 + quarter * 32 + (tid & 31);
#pragma unroll 1
        for (int cb = half * (TN / 2); cb < (half + 1) * (TN / 2); cb += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cb, v);
            if (m >= g.M) continue;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = n0 + cb + i;
                if (n >= g.N) continue;
                const float a = v[i];
                if (g.kper) {
                    // a part of a split contraction: the raw partial sum
                    g.part[((long long)blockIdx.z * g.M + m) * g.N + n] = a;
                    continue;
                }
                const long long ci = (long long)m * g.ldc + n;
                switch (g.epi) {
                    case E_BIAS_RELU: g.C[ci] = fmaxf(a + g.bias[n], 0.f); break;
                    case E_SIGQ: {
                        const float s = 1.f / (1.f + expf(-(a + g.bias[n])));
                        g.C2[(long long)m * g.ldc2 + n] = s;
                        g.C[ci] = g.q_lo + (g.q_hi - g.q_lo) * s;
                        break;
                    }
                    case E_MASK: g.C[ci] = g.C2[(long long)m * g.ldc2 + n] > 0.f ? a : 0.f; break;
                    case E_SPLIT:
                        if (m < g.M - 1) g.C[ci] = a;
                        else g.C2[n] = a;
                        break;
                    default: g.C[ci] = a; break;
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(g.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
    }
}

// The parts of a split contraction summed in a fixed order (deterministic),
// then the store of E_STORE / E_SPLIT.
__global__ void k_splitk_reduce(const __grid_constant__ Gemm g, int parts) {
    const long long total = (long long)g.M * g.N;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(idx / g.N), n = (int)(idx % g.N);
        float a = 0.f;
        for (int z = 0; z < parts; ++z) a += g.part[((long long)z * g.M + m) * g.N + n];
        if (g.epi == E_SPLIT && m == g.M - 1) g.C2[n] = a;
        else g.C[(long long)m * g.ldc + n] = a;
    }
}

// Parts of a split over K for a contraction of length K (1 = no split).
int split_parts(int K) {
    if (K < SPLIT_MIN_K) return 1;
    int p = (K + SPLIT_CHUNK - 1) / SPLIT_CHUNK;
    return p < SPLIT_MAX ? p : SPLIT_MAX;
}

cudaError_t launch(const Gemm& gin, cudaStream_t st) {
    Gemm g = gin;
    static int prepared[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !prepared[dev]) {
        e = cudaFuncSetAttribute(k_gemm_3xtf32, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        prepared[dev] = 1;
    }
    const int parts = g.part && (g.epi == E_STORE || g.epi == E_SPLIT) ? split_parts(g.K) : 1;
    g.kper = 0;
    if (parts > 1) {
        const int per = (g.K + parts - 1) / parts;
        g.kper = (per + TK - 1) / TK * TK;
    }
    const int nz = g.kper ? (g.K + g.kper - 1) / g.kper : 1;
    const dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, nz);
    k_gemm_3xtf32<<<grid, THREADS, SMEM_BYTES, st>>>(g);
    if (nz > 1) {
        const long long total = (long long)g.M * g.N;
        const int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
        k_splitk_reduce<<<blocks, 256, 0, st>>>(g, nz);
    }
    return cudaGetLastError();
}

Operand plain(const float* p, long long s0, long long s1, int rows, int kind = K_PLAIN) {
    Operand o{};
    o.p = p;
    o.s0 = s0;
    o.s1 = s1;
    o.rows = rows;
    o.kind = kind;
    return o;
}

// Workspace layout: the error flag (an int in the first 256 bytes), then the
// floats h1 [B, H], h2 [B, H], s [B, n_out], da2 [B, H], da1 [B, H], and the
// partial sums of the split weight-gradient contractions [SPLIT_MAX, H + 1,
// max(H, n_out)].
struct Ws {
    float *h1, *h2, *s, *da2, *da1, *part;
    int* err;
};
size_t part_floats(int H, int n_out) { return (size_t)SPLIT_MAX * (H + 1) * (H > n_out ? H : n_out); }
Ws carve(void* ws, int B, int H, int n_out) {
    float* f = (float*)((char*)ws + 256);
    const size_t bh = ((size_t)B * H + 63) & ~(size_t)63, bo = ((size_t)B * n_out + 63) & ~(size_t)63;
    Ws w;
    w.err = (int*)ws;
    w.h1 = f;
    w.h2 = w.h1 + bh;
    w.s = w.h2 + bh;
    w.da2 = w.s + bo;
    w.da1 = w.da2 + bh;
    w.part = w.da1 + bh;
    return w;
}

int check_net(const mpc_costmap* net, int B, int N) {
    if (!net || !net->W1 || !net->b1 || !net->W2 || !net->b2 || !net->W3 || !net->b3) return MPC_ERR_ARG;
    if (net->n_in != 26 || net->hidden < 1 || net->n_out != N * 13) return MPC_ERR_SHAPE;
    if (B < 0 || N < 1) return MPC_ERR_SHAPE;
    if (!(net->q_hi > net->q_lo)) return MPC_ERR_ARG;
    return MPC_OK;
}

}  // namespace cmap

using namespace cmap;

extern "C" size_t mpc_costmap_workspace_bytes(int B, int hidden, int n_out) {
    if (B < 0 || hidden < 1 || n_out < 1) return 0;
    const size_t bh = ((size_t)B * hidden + 63) & ~(size_t)63, bo = ((size_t)B * n_out + 63) & ~(size_t)63;
    return (4 * bh + bo + part_floats(hidden, n_out)) * sizeof(float) + 256;
}

extern "C" int mpc_costmap_forward(const mpc_costmap* net, int B, int N, const float* x0, const float* x_ref,
                                   float* Q, void* ws, cudaStream_t stream) {
    int r = check_net(net, B, N);
    if (r != MPC_OK) return r;
    if (B == 0) return MPC_OK;
    if (!x0 || !x_ref || !Q || !ws) return MPC_ERR_ARG;
    const int H = net->hidden, n_out = net->n_out;
    Ws w = carve(ws, B, H, n_out);
    if (cudaMemsetAsync(w.err, 0, sizeof(int), stream) != cudaSuccess) return MPC_ERR_CUDA;
    Gemm g{};
    g.err = w.err;
    g.q_lo = net->q_lo;
    g.q_hi = net->q_hi;
    // h1 = relu(o W1 + b1): A(m, k) = o(m, k), B(n, k) = W1[k, n]
    g.A = Operand{x0, x_ref, 0, 0, B, K_OBS, 0, N * 13};
    g.B = plain(net->W1, 1, H, H);
    g.M = B; g.N = H; g.K = 26;
    g.epi = E_BIAS_RELU; g.bias = net->b1; g.C = w.h1; g.ldc = H;
    if (launch(g, stream) != cudaSuccess) return MPC_ERR_CUDA;
    // h2 = relu(h1 W2 + b2)
    g.A = plain(w.h1, H, 1, B);
    g.B = plain(net->W2, 1, H, H);
    g.K = H; g.bias = net->b2; g.C = w.h2;
    if (launch(g, stream) != cudaSuccess) return MPC_ERR_CUDA;
    // Q = q_lo + (q_hi - q_lo) sigmoid(h2 W3 + b3), written as [B, N, 13]; s kept for the backward
    g.A = plain(w.h2, H, 1, B);
    g.B = plain(net->W3, 1, n_out, n_out);
    g.N = n_out; g.epi = E_SIGQ; g.bias = net->b3; g.C = Q; g.ldc = n_out; g.C2 = w.s; g.ldc2 = n_out;
    if (launch(g, stream) != cudaSuccess) return MPC_ERR_CUDA;
    return MPC_OK;
}

extern "C" int mpc_costmap_backward(const mpc_costmap* net, int B, int N, const float* x0, const float* x_ref,
                                    const float* dQ, void* ws, float* dW1, float* db1, float* dW2, float* db2,
                                    float* dW3, float* db3, float* d_obs, cudaStream_t stream) {
    int r = check_net(net, B, N);
    if (r != MPC_OK) return r;
    if (!dW1 || !db1 || !dW2 || !db2 || !dW3 || !db3) return MPC_ERR_ARG;
    const int H = net->hidden, n_out = net->n_out;
    if (B == 0) {
        // no samples: every gradient is zero
        const size_t z[6] = {(size_t)26 * H, (size_t)H, (size_t)H * H, (size_t)H, (size_t)H * n_out, (size_t)n_out};
        float* p[6] = {dW1, db1, dW2, db2, dW3, db3};
        for (int i = 0; i < 6; ++i)
            if (cudaMemsetAsync(p[i], 0, z[i] * sizeof(float), stream) != cudaSuccess) return MPC_ERR_CUDA;
        return MPC_OK;
    }
    if (!x0 || !x_ref || !dQ || !ws) return MPC_ERR_ARG;
    Ws w = carve(ws, B, H, n_out);
    Gemm g{};
    g.err = w.err;
    g.q_lo = net->q_lo;
    g.q_hi = net->q_hi;
    // [dW3; db3] = [h2 | 1]' da3, da3 = dQ (q_hi - q_lo) s (1 - s): A(m, k) = h2[k, m], B(n, k) = da3[k, n]
    g.A = plain(w.h2, 1, H, H, K_ONES_ROW);
    g.B = Operand{dQ, w.s, 1, n_out, n_out, K_DA3, 0, 0};
    g.M = H + 1; g.N = n_out; g.K = B;
    g.epi = E_SPLIT; g.C = dW3; g.ldc = n_out; g.C2 = db3; g.part = w.part;
    if (launch(g, stream) != cudaSuccess) return MPC_ERR_CUDA;
    // da2 = (da3 W3') * (h2 > 0): A(m, k) = da3[m, k], B(n, k) = W3[n, k]
    g.A = Operand{dQ, w.s, n_out, 1, B, K_DA3, 0, 0};
    g.B = plain(net->W3, n_out, 1, H);
    g.M = B; g.N = H; g.K = n_out;
    g.epi = E_MASK; g.C = w.da2; g.ldc = H; g.C2 = w.h2; g.ldc2 = H; g.part = nullptr;
    if (launch(g, stream) != cudaSuccess) return MPC_ERR_CUDA;
    // [dW2; db2] = [h1 | 1]' da2
    g.A = plain(w.h1, 1, H, H, K_ONES_ROW);
    g.B = plain(w.da2, 1, H, H);
    g.M = H + 1; g.N = H; g.K = B;
    g.epi = E_SPLIT; g.C = dW2; g.ldc = H; g.C2 = db2; g.part = w.part;
    if (launch(g, stream) != cudaSuccess) return MPC_ERR_CUDA;
    // da1 = (da2 W2') * (h1 > 0)
    g.A = plain(w.da2, H, 1, B);
    g.B = plain(net->W2, H, 1, H);
    g.M = B; g.N = H; g.K = H;
    g.epi = E_MASK; g.C = w.da1; g.ldc = H; g.C2 = w.h1; g.ldc2 = H; g.part = nullptr;
    if (launch(g, stream) != cudaSuccess) return MPC_ERR_CUDA;
    // [dW1; db1] = [o | 1]' da1: A(m, k) = o(k, m)
    g.A = Operand{x0, x_ref, 1, 0, 26, K_OBS, 1, N * 13};
    g.B = plain(w.da1, 1, H, H);
    g.M = 27; g.N = H; g.K = B;
    g.epi = E_SPLIT; g.C = dW1; g.ldc = H; g.C2 = db1; g.part = w.part;
    if (launch(g, stream) != cudaSuccess) return MPC_ERR_CUDA;
    if (d_obs) {
        // dL/do = da1 W1': A(m, k) = da1[m, k], B(n, k) = W1[n, k]
        g.A = plain(w.da1, H, 1, B);
        g.B = plain(net->W1, H, 1, 26);
        g.M = B; g.N = 26; g.K = H;
        g.epi = E_STORE; g.C = d_obs; g.ldc = 26; g.part = nullptr;
        if (launch(g, stream) != cudaSuccess) return MPC_ERR_CUDA;
    }
    return MPC_OK;
}
