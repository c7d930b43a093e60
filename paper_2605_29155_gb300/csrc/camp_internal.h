// camp_internal.h -- declarations shared by the kernel and the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace camp {

constexpr int MAX_N = 64;           // largest horizon the library accepts

template <typename T> struct Params;
template <typename T> struct AdjArgs;

// Shared memory of one block; kernel attributes; resident blocks per SM for
// NW warps per block.
template <typename T> size_t block_smem_bytes();
template <typename T> cudaError_t prepare_kernels();
template <typename T> int persistent_blocks_per_sm(int nw);
template <typename T>
cudaError_t launch_forward(const Params<T>& P, int exec_mode, int nw, int grid, int* order_ws, cudaStream_t st);
// The stage-parallel Riccati phase (camp_scan.cu): kernel attributes, one
// launch over P.B instances (one per block), workspace size and dynamic shared
// memory.
template <typename T> cudaError_t prepare_scan();
template <typename T> cudaError_t launch_scan_ric(const Params<T>& P, cudaStream_t st, int final_fac);
size_t scan_ws_elems(size_t slots, int N);
template <typename T>
cudaError_t launch_backward(const Params<T>& P, const AdjArgs<T>& A, int nw, int grid, int* order_ws,
                            cudaStream_t st);

// A launch shape: tpi threads per instance (one lane in each of tpi warps:
// 4 or 8) and ipb instances per block (1..32, one per lane).
inline bool shape_ok(int tpi, int ipb) { return (tpi == 4 || tpi == 8) && ipb >= 1 && ipb <= 32; }

// Scratch sizes (elements) for `slots` positions and horizons up to N_ws.
inline size_t groups_of(size_t slots) { return (slots + 31) / 32; }
inline size_t stg_elems(size_t slots, int N_ws) { return groups_of(slots) * 32 * (size_t)N_ws * 112; }
inline size_t cand_elems(size_t slots, int N_ws) { return 4 * groups_of(slots) * 32 * (size_t)N_ws * 30; }
inline size_t kh_elems(size_t slots, int N_ws) { return groups_of(slots) * 32 * (size_t)N_ws * 4; }
// Tape elements for (B, N): one 210-row record per stage per group of 32 instances.
inline size_t tape_elems(int B, int N) { return groups_of((size_t)B) * 32 * (size_t)N * 210; }

}  // namespace camp
