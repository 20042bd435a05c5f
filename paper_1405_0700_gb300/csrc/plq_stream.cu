// Link x spinor streaming micro-benchmark (the paper's prefetch experiment,
// Sec. 2.2 and its Fig. of sequential / random / pointer-array access).
//
// psi(i) = U(i) phi(i): one SU(3) matrix times the four colour vectors of a
// spinor, per site, over n sites stored site by site (array of structures,
// as in the paper's CPU code; FP32: 24 floats of phi, 18 of U, 24 of psi).
//   mode 0  sequential:            site i handles record i
//   mode 1  random, index array:   site i handles record x[i]
//   mode 2  random, pointer array: site i follows precomputed pointers
//                                  psi'(i), U'(i), phi'(i) to the records
// It measures what the access pattern costs on this GPU (coalesced streaming
// vs gathered records) as a calibration of the operator's bandwidth figures.
#include "plq_fields.cuh"

namespace plq {
namespace {

template <class T>
__device__ __forceinline__ void link_spinor(const T *U, const T *phi, T *psi) {
    cx<T> u[3][3], v[4][3];
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k / 3][k % 3] = {U[2 * k], U[2 * k + 1]};
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k / 3][k % 3] = {phi[2 * k], phi[2 * k + 1]};
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<T> z{0, 0};
#pragma unroll
            for (int b = 0; b < 3; ++b) z = cfma(u[a][b], v[s][b], z);
            psi[2 * (3 * s + a)] = z.re;
            psi[2 * (3 * s + a) + 1] = z.im;
        }
}

template <class T>
__global__ void stream_kernel(int mode, long long n, const T *U, const T *phi, T *psi, const int *x,
                              const void *const *ptrs) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (mode == 2) {
            T *po = static_cast<T *>(const_cast<void *>(ptrs[i]));
            const T *pu = static_cast<const T *>(ptrs[n + i]);
            const T *pp = static_cast<const T *>(ptrs[2 * n + i]);
            link_spinor(pu, pp, po);
        } else {
            const long long j = mode == 1 ? (long long)x[i] : i;
            if (j < 0 || j >= n) continue;  // out-of-range index entries are skipped
            link_spinor(U + 18 * j, phi + 24 * j, psi + 24 * j);
        }
    }
}

}  // namespace
}  // namespace plq

using namespace plq;

extern "C" plq_status plq_link_spinor_stream(int mode, long long nsites, const void *U, const void *phi, void *psi,
                                             const int *index, const void *const *pointers, int prec,
                                             void *stream) {
    if (mode < 0 || mode > 2) return set_error(PLQ_ERR_ARG, "mode must be 0, 1 or 2");
    if (nsites <= 0) return set_error(PLQ_ERR_ARG, "nsites must be positive");
    if (!U || !phi || !psi) return set_error(PLQ_ERR_ARG, "null field");
    if (mode == 1 && !index) return set_error(PLQ_ERR_ARG, "mode 1 needs the index array");
    if (mode == 2 && !pointers) return set_error(PLQ_ERR_ARG, "mode 2 needs the pointer arrays");
    if (prec != PLQ_F64 && prec != PLQ_F32) return set_error(PLQ_ERR_ARG, "prec must be PLQ_F64 or PLQ_F32");
    int dev = 0, sms = 0;
    PLQ_CUDA(cudaGetDevice(&dev));
    PLQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int block = 256;
    const long long want = (nsites + block - 1) / block;
    const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == PLQ_F64)
        stream_kernel<double><<<grid, block, 0, s>>>(mode, nsites, static_cast<const double *>(U),
                                                     static_cast<const double *>(phi), static_cast<double *>(psi),
                                                     index, pointers);
    else
        stream_kernel<float><<<grid, block, 0, s>>>(mode, nsites, static_cast<const float *>(U),
                                                    static_cast<const float *>(phi), static_cast<float *>(psi), index,
                                                    pointers);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}
