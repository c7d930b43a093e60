// camp_peak.cu -- FP32 FMA throughput probe (mpc_fp32_fma_probe): the measured
// denominator of the forward solve's roofline, whose arithmetic is plain FP32
// multiply-adds on the CUDA cores.
//
// Every thread runs 8 independent multiply-add chains, a = a * m + c with m
// and c kernel arguments (nothing folds at compile time), 16 steps per loop
// trip.  The chains converge to c / (1 - m) for 0 < m < 1, so the values stay
// finite.  Their sum decides a store that practically never happens, which
// keeps every chain live without an output array.
#include "camp.h"

namespace {

constexpr int PEAK_THREADS = 1024;
constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_UNROLL = 16;

__global__ void __launch_bounds__(PEAK_THREADS, 2) k_ffma_peak(float* sink, float m, float c, int trips) {
    float a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
    if (s == -1.2345f) sink[0] = s;
}

}  // namespace

extern "C" int mpc_fp32_fma_probe(int trips, float* sink, cudaStream_t stream, double* flops) {
    if (trips < 1 || !sink) return MPC_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MPC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return MPC_ERR_CUDA;
    const int grid = 2 * sms;
    k_ffma_peak<<<grid, PEAK_THREADS, 0, stream>>>(sink, 0.999999f, 1e-6f, trips);
    if (flops) *flops = 2.0 * grid * PEAK_THREADS * (double)PEAK_CHAINS * PEAK_UNROLL * trips;
    return cudaGetLastError() == cudaSuccess ? MPC_OK : MPC_ERR_CUDA;
}
