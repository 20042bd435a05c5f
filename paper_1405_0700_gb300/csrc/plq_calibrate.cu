// Roofline calibration: the FMA throughput of the CUDA cores in FP64 and FP32.
//
// The hopping operator does 1320 flop per site; in FP64 on this GPU that
// arithmetic, not HBM, can be the bound.  This kernel measures the sustained
// FMA rate with independent dependency chains per thread (enough in flight to
// fill the pipes), so the FP64 roofline is quoted against a measured number.
#include <chrono>

#include "plq_internal.cuh"

namespace plq {
namespace {

template <class T, int CHAINS>
__global__ void fma_chain_kernel(T *out, int iters, T a, T b) {
    T v[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) v[c] = fma(v[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += v[c];
    if (s == (T)12345.678) out[blockIdx.x] = s;  // keeps the chains live; never true in practice
}

template <class T>
plq_status measure(int device, double *flops) {
    PLQ_CUDA(cudaSetDevice(device));
    int sms = 0;
    PLQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int block = 256, grid = sms * 8, iters = 4096;
    constexpr int CHAINS = 8;
    T *out = nullptr;
    PLQ_CUDA(cudaMalloc(&out, sizeof(T) * grid));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_chain_kernel<T, CHAINS><<<grid, block>>>(out, 64, (T)0.999, (T)1e-4);  // warm
    cudaEventRecord(e0);
    fma_chain_kernel<T, CHAINS><<<grid, block>>>(out, iters, (T)0.999, (T)1e-4);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_error(e, "fma_chain_kernel");
    *flops = 2.0 * CHAINS * (double)iters * grid * block / (ms * 1e-3);
    return PLQ_OK;
}

}  // namespace
}  // namespace plq

extern "C" plq_status plq_measure_fma_rate(int device, int prec, double *flops_per_second) {
    if (!flops_per_second) return plq::set_error(PLQ_ERR_ARG, "null output");
    if (prec == PLQ_F64) return plq::measure<double>(device, flops_per_second);
    if (prec == PLQ_F32) return plq::measure<float>(device, flops_per_second);
    return plq::set_error(PLQ_ERR_ARG, "prec must be PLQ_F64 or PLQ_F32");
}
