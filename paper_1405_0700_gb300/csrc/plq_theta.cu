// Two-pass hopping operator through the auxiliary fields of Eq. (2).
//
// Pass 1 (one thread per INPUT site y): for every direction mu
//   theta+_mu(y) = upper half of (1 - gamma_mu) phi(y)
//   theta-_mu(y) = U_mu(y)^dagger * upper half of (1 + gamma_mu) phi(y)
// (only the upper two spin components are stored: the lower two follow from
// them, the remark after Eq. (2)).
// Pass 2 (one thread per OUTPUT site x): psi(x) = sum_mu [U_mu(x) theta+_mu(x + mu)
// + theta-_mu(x - mu)], with the lower spin components rebuilt on the fly.
//
// This is the schedule the paper's distributed code uses to overlap the
// exchange of theta on the boundary with bulk computation (Sec. 2.2).  On one
// GPU there is nothing to exchange and it moves twice the bytes of the fused
// gather kernel (theta makes a round trip through memory); it is kept as the
// comm-ready structure and as a measured comparison.
#include "plq_hop_impl.cuh"

namespace plq {
namespace {

// theta layout: 8 blocks (2*mu + {0: theta+, 1: theta-}) of 6 complex per
// input site, stored as the first 6 complex components of a spinor-shaped
// half field block (FP64: 6 planes of double2; FP32: 3 planes of float4).
template <int P>
struct Half;
template <>
struct Half<PLQ_F64> {
    __device__ static void store(void *base, size_t Vh, int i, const cx<double> h[6]) {
        double2 *p = static_cast<double2 *>(base) + i;
#pragma unroll
        for (int k = 0; k < 6; ++k) __stcg(p + k * Vh, make_double2(h[k].re, h[k].im));
    }
    __device__ static void load(const void *base, size_t Vh, int i, cx<double> h[6]) {
        const double2 *p = static_cast<const double2 *>(base) + i;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            double2 t = __ldcg(p + k * Vh);
            h[k] = {t.x, t.y};
        }
    }
    static constexpr size_t bytes = 96;
};
template <>
struct Half<PLQ_F32> {
    __device__ static void store(void *base, size_t Vh, int i, const cx<float> h[6]) {
        float4 *p = static_cast<float4 *>(base) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            __stcg(p + k * Vh, make_float4(h[2 * k].re, h[2 * k].im, h[2 * k + 1].re, h[2 * k + 1].im));
    }
    __device__ static void load(const void *base, size_t Vh, int i, cx<float> h[6]) {
        const float4 *p = static_cast<const float4 *>(base) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 t = __ldcg(p + k * Vh);
            h[2 * k] = {t.x, t.y};
            h[2 * k + 1] = {t.z, t.w};
        }
    }
    static constexpr size_t bytes = 48;
};

template <int P, int R, int MU>
__device__ __forceinline__ void theta_dir(const HopArgs &a, int in_par, int y, const cx<RealOf<P>> phi[12],
                                          char *theta, size_t blk) {
    using T = RealOf<P>;
    const int Vh = a.lat.Vh;
    cx<T> h[6];
    project<MU, -1>(phi, h);
    Half<P>::store(theta + (2 * MU) * blk, Vh, y, h);
    project<MU, +1>(phi, h);
    cx<T> u[3][3];
    Link<P, R>::load(static_cast<const char *>(a.gauge) + (size_t)(in_par * 4 + MU) * a.gblock, Vh, y, u);
    cx<T> uh[6];
    su3_dag_mul(u, h, uh);
    Half<P>::store(theta + (2 * MU + 1) * blk, Vh, y, uh);
}

template <int P, int R>
__global__ void __launch_bounds__(128) theta_kernel(const HopArgs a, char *theta, size_t blk) {
    using T = RealOf<P>;
    const int in_par = 1 - a.out_parity;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < a.lat.Vh; y += gridDim.x * blockDim.x) {
        cx<T> phi[12];
        Spinor<P>::load(a.in, (size_t)a.lat.Vh, (size_t)y, phi);
        theta_dir<P, R, 0>(a, in_par, y, phi, theta, blk);
        theta_dir<P, R, 1>(a, in_par, y, phi, theta, blk);
        theta_dir<P, R, 2>(a, in_par, y, phi, theta, blk);
        theta_dir<P, R, 3>(a, in_par, y, phi, theta, blk);
    }
}

template <int P, int R, int MU>
__device__ __forceinline__ void gather_dir(const HopArgs &a, const SiteGeom &g, int i, const char *theta, size_t blk,
                                           cx<RealOf<P>> acc[12]) {
    using T = RealOf<P>;
    const Lattice &L = a.lat;
    const int st = lex_stride(L, MU);
    const int cm = g.c[MU], Lm = L.L[MU];
    {  // U_mu(x) theta+_mu(x + mu)
        const int j = ((cm == Lm - 1) ? g.lex - (Lm - 1) * st : g.lex + st) >> 1;
        cx<T> h[6];
        Half<P>::load(theta + (2 * MU) * blk, L.Vh, j, h);
        if (MU == 0 && cm == Lm - 1 && L.t_bc < 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = {-h[k].re, -h[k].im};
        }
        cx<T> u[3][3];
        Link<P, R>::load(static_cast<const char *>(a.gauge) + (size_t)(a.out_parity * 4 + MU) * a.gblock, L.Vh, i, u);
        cx<T> uh[6];
        su3_mul(u, h, uh);
        reconstruct<MU, -1>(acc, uh);
    }
    {  // theta-_mu(x - mu)
        const int j = ((cm == 0) ? g.lex + (Lm - 1) * st : g.lex - st) >> 1;
        cx<T> h[6];
        Half<P>::load(theta + (2 * MU + 1) * blk, L.Vh, j, h);
        if (MU == 0 && cm == 0 && L.t_bc < 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = {-h[k].re, -h[k].im};
        }
        reconstruct<MU, +1>(acc, h);
    }
}

template <int P, int R>
__global__ void __launch_bounds__(128) gather_kernel(const HopArgs a, const char *theta, size_t blk) {
    using T = RealOf<P>;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.lat.Vh; i += gridDim.x * blockDim.x) {
        const SiteGeom g = site_geom(a.lat, a.out_parity, i);
        cx<T> acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {T(0), T(0)};
        gather_dir<P, R, 0>(a, g, i, theta, blk, acc);
        gather_dir<P, R, 1>(a, g, i, theta, blk, acc);
        gather_dir<P, R, 2>(a, g, i, theta, blk, acc);
        gather_dir<P, R, 3>(a, g, i, theta, blk, acc);
        Spinor<P>::store(a.out, (size_t)a.lat.Vh, (size_t)i, acc);
    }
}

template <int P, int R>
plq_status launch_theta(const HopArgs &a, char *theta, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int block = 128;
    const long long want = ((long long)a.lat.Vh + block - 1) / block;
    const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    const size_t blk = Half<P>::bytes * (size_t)a.lat.Vh;
    theta_kernel<P, R><<<grid, block, 0, s>>>(a, theta, blk);
    PLQ_CUDA(cudaGetLastError());
    gather_kernel<P, R><<<grid, block, 0, s>>>(a, theta, blk);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

}  // namespace
}  // namespace plq

using namespace plq;

extern "C" size_t plq_theta_bytes(const plq_ctx *c, int prec) {
    if (!c || (prec != PLQ_F64 && prec != PLQ_F32)) return 0;
    return 8 * (prec == PLQ_F64 ? 96 : 48) * (size_t)c->lat.Vh;
}

extern "C" plq_status plq_hopping_eo_theta(plq_ctx *c, int out_parity, void *out, const void *in, void *theta,
                                           int prec, void *stream) {
    if (!c) return set_error(PLQ_ERR_ARG, "null context");
    auto aligned = [](const void *p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (!aligned(out) || !aligned(in) || !aligned(theta)) return set_error(PLQ_ERR_ARG, "null or misaligned pointer");
    if (out == in) return set_error(PLQ_ERR_ARG, "in and out must not overlap");
    if (out_parity != 0 && out_parity != 1) return set_error(PLQ_ERR_ARG, "out_parity must be 0 or 1");
    if (prec != PLQ_F64 && prec != PLQ_F32) return set_error(PLQ_ERR_ARG, "the theta schedule supports FP64 and FP32");
    if (!c->gauge[prec].ptr) return set_error(PLQ_ERR_STATE, "no gauge field uploaded for precision %d", prec);
    PLQ_CUDA(cudaSetDevice(c->device));
    HopArgs a;
    a.in = in;
    a.out = out;
    a.gauge = c->gauge[prec].ptr;
    a.gblock = c->gauge[prec].block;
    a.out_parity = out_parity;
    a.lat = c->lat;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *th = static_cast<char *>(theta);
    const bool r12 = c->gauge[prec].reals == 12;
    if (prec == PLQ_F64) return r12 ? launch_theta<PLQ_F64, 12>(a, th, s) : launch_theta<PLQ_F64, 18>(a, th, s);
    return r12 ? launch_theta<PLQ_F32, 12>(a, th, s) : launch_theta<PLQ_F32, 18>(a, th, s);
}
