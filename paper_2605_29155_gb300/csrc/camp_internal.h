// camp_internal.h -- declarations shared by the kernel and the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace camp {

constexpr int MAX_N = 64;           // largest horizon the library accepts

template <typename T> struct Params;
template <typename T> struct AdjArgs;

template <typename T> size_t warp_smem_bytes();
template <typename T> cudaError_t prepare_kernels();
// which: 0 = persistent forward, 1 = adjoint
template <typename T> int persistent_blocks_per_sm(int ipb, int which);
template <typename T>
cudaError_t launch_forward(const Params<T>& P, int exec_mode, int ipb, int grid, int* order_ws, cudaStream_t st);
template <typename T>
cudaError_t launch_backward(const Params<T>& P, const AdjArgs<T>& A, int ipb, int grid, int* order_ws,
                            cudaStream_t st);

}  // namespace camp
