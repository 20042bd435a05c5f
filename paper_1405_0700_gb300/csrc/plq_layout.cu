// Layout kernels: canonical AoS FP64 fields <-> packed even-odd SoA fields.
#include "plq_fields.cuh"

namespace plq {

namespace {

int grid_for(long long work, int block, int per_sm = 8) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (work + block - 1) / block;
    long long cap = (long long)sms * per_sm;
    return (int)(want < cap ? want : cap);
}

// Canonical fields of nrhs right-hand sides stored back to back (each V sites
// x 12 complex, lexicographic) <-> packed full field (even half, odd half;
// element (plane k, site i, rhs r) at (k*Vh + i)*nrhs + r).
template <int P>
__global__ void pack_spinor_kernel(Lattice L, int nrhs, char *out, const double *in, size_t half_bytes) {
    using T = RealOf<P>;
    const long long per_par = (long long)L.Vh * nrhs;
    const long long total = 2 * per_par;
    const size_t V = 2 * (size_t)L.Vh;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int par = (int)(idx / per_par);
        const long long e = idx - par * per_par;
        const int i = (int)(e / nrhs);
        const int r = (int)(e - (long long)i * nrhs);
        const SiteGeom g = site_geom(L, par, i);
        const double2 *src = reinterpret_cast<const double2 *>(in) + ((size_t)r * V + (size_t)g.lex) * 12;
        cx<T> v[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 z = src[k];
            v[k] = {(T)z.x, (T)z.y};
        }
        Spinor<P>::store(out + par * half_bytes, (size_t)per_par, (size_t)e, v);
    }
}

template <int P>
__global__ void unpack_spinor_kernel(Lattice L, int nrhs, double *out, const char *in, size_t half_bytes) {
    using T = RealOf<P>;
    const long long per_par = (long long)L.Vh * nrhs;
    const long long total = 2 * per_par;
    const size_t V = 2 * (size_t)L.Vh;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int par = (int)(idx / per_par);
        const long long e = idx - par * per_par;
        const int i = (int)(e / nrhs);
        const int r = (int)(e - (long long)i * nrhs);
        const SiteGeom g = site_geom(L, par, i);
        cx<T> v[12];
        Spinor<P>::load(in + par * half_bytes, (size_t)per_par, (size_t)e, v);
        double2 *dst = reinterpret_cast<double2 *>(out) + ((size_t)r * V + (size_t)g.lex) * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = make_double2((double)v[k].re, (double)v[k].im);
    }
}

// Writes the packed form of one link (9 complex, row-major) at site i of a
// (parity, mu) block, for storage precision P and R reals.
template <int P, int R>
__device__ void store_link(char *blk, int Vh, int i, const double2 u[9]);

template <>
__device__ void store_link<PLQ_F64, 18>(char *blk, int Vh, int i, const double2 u[9]) {
    double2 *p = reinterpret_cast<double2 *>(blk) + i;
    for (int k = 0; k < 9; ++k) p[(size_t)k * Vh] = u[k];
}
template <>
__device__ void store_link<PLQ_F64, 12>(char *blk, int Vh, int i, const double2 u[9]) {
    double2 *p = reinterpret_cast<double2 *>(blk) + i;
    for (int k = 0; k < 6; ++k) p[(size_t)k * Vh] = u[k];
}
template <>
__device__ void store_link<PLQ_F32, 18>(char *blk, int Vh, int i, const double2 u[9]) {
    float4 *p = reinterpret_cast<float4 *>(blk) + i;
    for (int k = 0; k < 4; ++k)
        p[(size_t)k * Vh] = make_float4((float)u[2 * k].x, (float)u[2 * k].y, (float)u[2 * k + 1].x, (float)u[2 * k + 1].y);
    float2 *q = reinterpret_cast<float2 *>(reinterpret_cast<float4 *>(blk) + 4 * (size_t)Vh) + i;
    *q = make_float2((float)u[8].x, (float)u[8].y);
}
template <>
__device__ void store_link<PLQ_F32, 12>(char *blk, int Vh, int i, const double2 u[9]) {
    float4 *p = reinterpret_cast<float4 *>(blk) + i;
    for (int k = 0; k < 3; ++k)
        p[(size_t)k * Vh] = make_float4((float)u[2 * k].x, (float)u[2 * k].y, (float)u[2 * k + 1].x, (float)u[2 * k + 1].y);
}
template <>
__device__ void store_link<PLQ_F16, 18>(char *blk, int Vh, int i, const double2 u[9]) {
    uint4 *p = reinterpret_cast<uint4 *>(blk) + i;
    for (int k = 0; k < 2; ++k) {
        uint4 t;
        t.x = f2h((float)u[4 * k].x, (float)u[4 * k].y);
        t.y = f2h((float)u[4 * k + 1].x, (float)u[4 * k + 1].y);
        t.z = f2h((float)u[4 * k + 2].x, (float)u[4 * k + 2].y);
        t.w = f2h((float)u[4 * k + 3].x, (float)u[4 * k + 3].y);
        p[(size_t)k * Vh] = t;
    }
    unsigned *q = reinterpret_cast<unsigned *>(reinterpret_cast<uint4 *>(blk) + 2 * (size_t)Vh) + i;
    *q = f2h((float)u[8].x, (float)u[8].y);
}
template <>
__device__ void store_link<PLQ_F16, 12>(char *blk, int Vh, int i, const double2 u[9]) {
    uint4 *p = reinterpret_cast<uint4 *>(blk) + i;
    uint4 t;
    t.x = f2h((float)u[0].x, (float)u[0].y);
    t.y = f2h((float)u[1].x, (float)u[1].y);
    t.z = f2h((float)u[2].x, (float)u[2].y);
    t.w = f2h((float)u[3].x, (float)u[3].y);
    *p = t;
    uint2 *q = reinterpret_cast<uint2 *>(reinterpret_cast<uint4 *>(blk) + (size_t)Vh) + i;
    *q = make_uint2(f2h((float)u[4].x, (float)u[4].y), f2h((float)u[5].x, (float)u[5].y));
}

__device__ double2 dmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// max deviation of u from SU(3): |u u^dagger - 1| and |row2 - conj(row0 x row1)|
__device__ double su3_defect(const double2 u[9]) {
    double d = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double re = 0, im = 0;
            for (int c = 0; c < 3; ++c) {  // u[a][c] * conj(u[b][c])
                re += u[3 * a + c].x * u[3 * b + c].x + u[3 * a + c].y * u[3 * b + c].y;
                im += u[3 * a + c].y * u[3 * b + c].x - u[3 * a + c].x * u[3 * b + c].y;
            }
            d = fmax(d, fabs(re - (a == b ? 1.0 : 0.0)));
            d = fmax(d, fabs(im));
        }
    for (int c = 0; c < 3; ++c) {
        const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        double2 x = dmul(u[c1], u[3 + c2]), y = dmul(u[c2], u[3 + c1]);
        double2 r = make_double2(x.x - y.x, -(x.y - y.y));  // conj(row0 x row1)_c
        d = fmax(d, fabs(r.x - u[6 + c].x));
        d = fmax(d, fabs(r.y - u[6 + c].y));
    }
    return d;
}

template <int P, int R>
__global__ void pack_gauge_kernel(Lattice L, char *out, const double *in, size_t block, unsigned *bad) {
    const long long total = 2LL * L.Vh;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int par = (int)(idx / L.Vh);
        const int i = (int)(idx - (long long)par * L.Vh);
        const SiteGeom g = site_geom(L, par, i);
        const double2 *src = reinterpret_cast<const double2 *>(in) + (size_t)g.lex * 36;
        for (int mu = 0; mu < 4; ++mu) {
            double2 u[9];
            for (int k = 0; k < 9; ++k) u[k] = src[9 * mu + k];
            if (R == 12 && su3_defect(u) > 1e-12) atomicOr(bad, 1u);
            store_link<P, R>(out + (size_t)(par * 4 + mu) * block, L.Vh, i, u);
        }
    }
}

}  // namespace

plq_status launch_pack_spinor(const Lattice &L, void *out, const double *in, int prec, int nrhs, cudaStream_t s) {
    const size_t half = spinor_site_bytes(prec) * L.Vh * nrhs;
    const int block = 256, grid = grid_for(2LL * L.Vh * nrhs, block);
    char *o = static_cast<char *>(out);
    if (prec == PLQ_F64) pack_spinor_kernel<PLQ_F64><<<grid, block, 0, s>>>(L, nrhs, o, in, half);
    else if (prec == PLQ_F32) pack_spinor_kernel<PLQ_F32><<<grid, block, 0, s>>>(L, nrhs, o, in, half);
    else pack_spinor_kernel<PLQ_F16><<<grid, block, 0, s>>>(L, nrhs, o, in, half);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status launch_unpack_spinor(const Lattice &L, double *out, const void *in, int prec, int nrhs, cudaStream_t s) {
    const size_t half = spinor_site_bytes(prec) * L.Vh * nrhs;
    const int block = 256, grid = grid_for(2LL * L.Vh * nrhs, block);
    const char *i = static_cast<const char *>(in);
    if (prec == PLQ_F64) unpack_spinor_kernel<PLQ_F64><<<grid, block, 0, s>>>(L, nrhs, out, i, half);
    else if (prec == PLQ_F32) unpack_spinor_kernel<PLQ_F32><<<grid, block, 0, s>>>(L, nrhs, out, i, half);
    else unpack_spinor_kernel<PLQ_F16><<<grid, block, 0, s>>>(L, nrhs, out, i, half);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status launch_pack_gauge(const Lattice &L, void *out, const double *in, int prec, int reals, size_t block,
                             unsigned *bad, cudaStream_t s) {
    const int tb = 128, grid = grid_for(2LL * L.Vh, tb);
    char *o = static_cast<char *>(out);
    if (prec == PLQ_F64) {
        if (reals == 12) pack_gauge_kernel<PLQ_F64, 12><<<grid, tb, 0, s>>>(L, o, in, block, bad);
        else pack_gauge_kernel<PLQ_F64, 18><<<grid, tb, 0, s>>>(L, o, in, block, bad);
    } else if (prec == PLQ_F32) {
        if (reals == 12) pack_gauge_kernel<PLQ_F32, 12><<<grid, tb, 0, s>>>(L, o, in, block, bad);
        else pack_gauge_kernel<PLQ_F32, 18><<<grid, tb, 0, s>>>(L, o, in, block, bad);
    } else {
        if (reals == 12) pack_gauge_kernel<PLQ_F16, 12><<<grid, tb, 0, s>>>(L, o, in, block, bad);
        else pack_gauge_kernel<PLQ_F16, 18><<<grid, tb, 0, s>>>(L, o, in, block, bad);
    }
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

}  // namespace plq
