// camp_internal.h -- declarations shared by the kernel and the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace camp {

constexpr int MAX_N = 64;           // largest horizon the library accepts

template <typename T> struct Params;
template <typename T> struct AdjArgs;

// Per-instance shared-memory record size; kernel attributes; occupancy of the
// kernel for a (threads per instance, instances per block) shape.
template <typename T> size_t warp_smem_bytes();
template <typename T> cudaError_t prepare_kernels();
template <typename T> int persistent_blocks_per_sm(int tpi, int ipb);
template <typename T>
cudaError_t launch_forward(const Params<T>& P, int exec_mode, int tpi, int ipb, int grid, int* order_ws,
                           cudaStream_t st);
template <typename T>
cudaError_t launch_backward(const Params<T>& P, const AdjArgs<T>& A, int tpi, int ipb, int grid, int* order_ws,
                            cudaStream_t st);

// A launch shape is valid when tpi is 8, 16 or 32 and a block (tpi * ipb
// threads) is 1 to 8 whole warps.
inline bool shape_ok(int tpi, int ipb) {
    return (tpi == 8 || tpi == 16 || tpi == 32) && ipb >= 1 && tpi * ipb >= 32 && tpi * ipb <= 256 &&
           (tpi * ipb) % 32 == 0;
}

}  // namespace camp
