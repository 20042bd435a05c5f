// Device-side access to packed fields: complex arithmetic, spinor and link
// loads/stores in FP64, FP32 and FP16 storage, and block reductions.
#pragma once

#include "plq_internal.cuh"

namespace plq {

template <class R>
struct cx {
    R re, im;
};

template <class R>
__device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
__device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R>
__device__ __forceinline__ cx<R> cscale(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <class R>
__device__ __forceinline__ cx<R> cconj(cx<R> a) { return {a.re, -a.im}; }

// a*b + c
template <class R>
__device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> c) {
    c.re = fma(a.re, b.re, c.re);
    c.re = fma(-a.im, b.im, c.re);
    c.im = fma(a.re, b.im, c.im);
    c.im = fma(a.im, b.re, c.im);
    return c;
}
// conj(a)*b + c
template <class R>
__device__ __forceinline__ cx<R> cfma_conj(cx<R> a, cx<R> b, cx<R> c) {
    c.re = fma(a.re, b.re, c.re);
    c.re = fma(a.im, b.im, c.re);
    c.im = fma(a.re, b.im, c.im);
    c.im = fma(-a.im, b.re, c.im);
    return c;
}

// z * i^K for K = 0..3 (+1, +i, -1, -i): no multiplications.
template <int K, class R>
__device__ __forceinline__ cx<R> mul_ipow(cx<R> z) {
    if constexpr ((K & 3) == 0) return z;
    else if constexpr ((K & 3) == 1) return {-z.im, z.re};
    else if constexpr ((K & 3) == 2) return {-z.re, -z.im};
    else return {z.im, -z.re};
}

// ---------------------------------------------------------------- loads
// Read-only, L1-cacheable (neighbour spinors are reused by up to 8 sites).
__device__ __forceinline__ float4 ld_nc(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ double2 ld_nc(const double2 *p) { return __ldg(p); }
__device__ __forceinline__ uint4 ld_nc(const uint4 *p) { return __ldg(p); }
__device__ __forceinline__ float ld_nc(const float *p) { return __ldg(p); }
// Streaming (evict-first): links are read exactly once per half-apply.
__device__ __forceinline__ float4 ld_stream(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ float2 ld_stream(const float2 *p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_stream(const double2 *p) { return __ldcs(p); }
__device__ __forceinline__ uint4 ld_stream(const uint4 *p) { return __ldcs(p); }
__device__ __forceinline__ uint2 ld_stream(const uint2 *p) { return __ldcs(p); }
__device__ __forceinline__ unsigned ld_stream(const unsigned *p) { return __ldcs(p); }

template <int P>
struct Real_;
template <>
struct Real_<PLQ_F64> {
    using T = double;
};
template <>
struct Real_<PLQ_F32> {
    using T = float;
};
template <>
struct Real_<PLQ_F16> {
    using T = float;
};
template <int P>
using RealOf = typename Real_<P>::T;

__device__ __forceinline__ float2 h2f(unsigned u) {
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}
__device__ __forceinline__ unsigned f2h(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned *>(&h);
}

// Packed half field: 12 complex components per site and rhs.
// `stride` = Vh * nrhs (elements of one plane); `e` = site * nrhs + rhs.
template <int P>
struct Spinor;

template <>
struct Spinor<PLQ_F64> {
    __device__ static void load(const void *base, size_t stride, size_t e, cx<double> v[12]) {
        const double2 *p = static_cast<const double2 *>(base) + e;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 t = ld_nc(p + k * stride);
            v[k] = {t.x, t.y};
        }
    }
    __device__ static void store(void *base, size_t stride, size_t e, const cx<double> v[12]) {
        double2 *p = static_cast<double2 *>(base) + e;
#pragma unroll
        for (int k = 0; k < 12; ++k) __stcs(p + k * stride, make_double2(v[k].re, v[k].im));
    }
};

template <>
struct Spinor<PLQ_F32> {
    __device__ static void load(const void *base, size_t stride, size_t e, cx<float> v[12]) {
        const float4 *p = static_cast<const float4 *>(base) + e;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 t = ld_nc(p + k * stride);
            v[2 * k] = {t.x, t.y};
            v[2 * k + 1] = {t.z, t.w};
        }
    }
    __device__ static void store(void *base, size_t stride, size_t e, const cx<float> v[12]) {
        float4 *p = static_cast<float4 *>(base) + e;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            __stcs(p + k * stride, make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im));
    }
};

template <>
struct Spinor<PLQ_F16> {
    // 3 planes of uint4 (8 halves), then stride floats of norms.
    __device__ static void load(const void *base, size_t stride, size_t e, cx<float> v[12]) {
        const uint4 *p = static_cast<const uint4 *>(base) + e;
        const float *nrm = reinterpret_cast<const float *>(static_cast<const uint4 *>(base) + 3 * stride);
        const float n = ld_nc(nrm + e);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 t = ld_nc(p + k * stride);
            float2 a = h2f(t.x), b = h2f(t.y), c = h2f(t.z), d = h2f(t.w);
            v[4 * k + 0] = {a.x * n, a.y * n};
            v[4 * k + 1] = {b.x * n, b.y * n};
            v[4 * k + 2] = {c.x * n, c.y * n};
            v[4 * k + 3] = {d.x * n, d.y * n};
        }
    }
    // The stored (normalised) components and the site norm separately: the
    // hopping kernel projects first and scales the 6 projected components
    // instead of the 12 loaded ones.
    __device__ static float load_unscaled(const void *base, size_t stride, size_t e, cx<float> v[12]) {
        const uint4 *p = static_cast<const uint4 *>(base) + e;
        const float *nrm = reinterpret_cast<const float *>(static_cast<const uint4 *>(base) + 3 * stride);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 t = ld_nc(p + k * stride);
            float2 a = h2f(t.x), b = h2f(t.y), c = h2f(t.z), d = h2f(t.w);
            v[4 * k + 0] = {a.x, a.y};
            v[4 * k + 1] = {b.x, b.y};
            v[4 * k + 2] = {c.x, c.y};
            v[4 * k + 3] = {d.x, d.y};
        }
        return ld_nc(nrm + e);
    }
    __device__ static void store(void *base, size_t stride, size_t e, const cx<float> v[12]) {
        uint4 *p = static_cast<uint4 *>(base) + e;
        float *nrm = reinterpret_cast<float *>(static_cast<uint4 *>(base) + 3 * stride);
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].re), fabsf(v[k].im)));
        // A site whose largest component is below the smallest normal float
        // (2^-126) is stored as zero: 1/m would overflow to infinity.  Such
        // sites occur at the edge of the support of the early Krylov vectors
        // of a point source, many orders of magnitude below the field's norm.
        constexpr float kMinNormal = 1.17549435e-38f;
        if (!(m >= kMinNormal)) m = 0.f;
        const float inv = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 t;
            t.x = f2h(v[4 * k + 0].re * inv, v[4 * k + 0].im * inv);
            t.y = f2h(v[4 * k + 1].re * inv, v[4 * k + 1].im * inv);
            t.z = f2h(v[4 * k + 2].re * inv, v[4 * k + 2].im * inv);
            t.w = f2h(v[4 * k + 3].re * inv, v[4 * k + 3].im * inv);
            __stcs(p + k * stride, t);
        }
        __stcs(nrm + e, m);
    }
};

// ---------------------------------------------------------------- links
// One (parity, mu) block of Vh links.  Complex element (row, col) = row*3 + col.
template <int P, int R>
struct Link;

template <class T>
__device__ __forceinline__ void reconstruct_row2(cx<T> u[3][3]) {
    // row2 = conj(row0 x row1): the third row of an SU(3) matrix.
    u[2][0] = cconj(csub(cfma(u[0][1], u[1][2], cx<T>{0, 0}), cfma(u[0][2], u[1][1], cx<T>{0, 0})));
    u[2][1] = cconj(csub(cfma(u[0][2], u[1][0], cx<T>{0, 0}), cfma(u[0][0], u[1][2], cx<T>{0, 0})));
    u[2][2] = cconj(csub(cfma(u[0][0], u[1][1], cx<T>{0, 0}), cfma(u[0][1], u[1][0], cx<T>{0, 0})));
}

template <int R>
struct Link<PLQ_F64, R> {
    __device__ static void load(const void *blk, int Vh, int i, cx<double> u[3][3]) {
        const double2 *p = static_cast<const double2 *>(blk) + i;
        constexpr int n = R / 2;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            double2 t = ld_stream(p + (size_t)k * Vh);
            u[k / 3][k % 3] = {t.x, t.y};
        }
        if constexpr (R == 12) reconstruct_row2(u);
    }
};

template <>
struct Link<PLQ_F32, 18> {
    __device__ static void load(const void *blk, int Vh, int i, cx<float> u[3][3]) {
        const float4 *p = static_cast<const float4 *>(blk) + i;
        cx<float> c[9];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 t = ld_stream(p + (size_t)k * Vh);
            c[2 * k] = {t.x, t.y};
            c[2 * k + 1] = {t.z, t.w};
        }
        float2 t = ld_stream(reinterpret_cast<const float2 *>(static_cast<const float4 *>(blk) + 4 * (size_t)Vh) + i);
        c[8] = {t.x, t.y};
#pragma unroll
        for (int k = 0; k < 9; ++k) u[k / 3][k % 3] = c[k];
    }
};

template <>
struct Link<PLQ_F32, 12> {
    __device__ static void load(const void *blk, int Vh, int i, cx<float> u[3][3]) {
        const float4 *p = static_cast<const float4 *>(blk) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 t = ld_stream(p + (size_t)k * Vh);
            u[(2 * k) / 3][(2 * k) % 3] = {t.x, t.y};
            u[(2 * k + 1) / 3][(2 * k + 1) % 3] = {t.z, t.w};
        }
        reconstruct_row2(u);
    }
};

template <>
struct Link<PLQ_F16, 18> {
    // 2 planes of uint4 (complex 0..3, 4..7) + 1 plane of half2 (complex 8)
    __device__ static void load(const void *blk, int Vh, int i, cx<float> u[3][3]) {
        const uint4 *p = static_cast<const uint4 *>(blk) + i;
        cx<float> c[9];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            uint4 t = ld_stream(p + (size_t)k * Vh);
            float2 a = h2f(t.x), b = h2f(t.y), d = h2f(t.z), e = h2f(t.w);
            c[4 * k] = {a.x, a.y};
            c[4 * k + 1] = {b.x, b.y};
            c[4 * k + 2] = {d.x, d.y};
            c[4 * k + 3] = {e.x, e.y};
        }
        float2 t = h2f(ld_stream(reinterpret_cast<const unsigned *>(static_cast<const uint4 *>(blk) + 2 * (size_t)Vh) + i));
        c[8] = {t.x, t.y};
#pragma unroll
        for (int k = 0; k < 9; ++k) u[k / 3][k % 3] = c[k];
    }
};

template <>
struct Link<PLQ_F16, 12> {
    // 1 plane of uint4 (complex 0..3) + 1 plane of uint2 (complex 4, 5)
    __device__ static void load(const void *blk, int Vh, int i, cx<float> u[3][3]) {
        const uint4 *p = static_cast<const uint4 *>(blk) + i;
        uint4 t = ld_stream(p);
        uint2 q = ld_stream(reinterpret_cast<const uint2 *>(static_cast<const uint4 *>(blk) + (size_t)Vh) + i);
        float2 a = h2f(t.x), b = h2f(t.y), d = h2f(t.z), e = h2f(t.w), f = h2f(q.x), g = h2f(q.y);
        u[0][0] = {a.x, a.y};
        u[0][1] = {b.x, b.y};
        u[0][2] = {d.x, d.y};
        u[1][0] = {e.x, e.y};
        u[1][1] = {f.x, f.y};
        u[1][2] = {g.x, g.y};
        reconstruct_row2(u);
    }
};

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Finalize step of one right-hand side's reduction: update its solver
// scalars in device memory from the grid totals tot[0..NV).
__device__ __forceinline__ void finalize_one(int fin, SolverState *st, const double *tot) {
    // A frozen right-hand side contributed nothing to this reduction: its
    // scalars must not change.
    if (st->stop) return;
    switch (fin) {
    case FIN_CG_ALPHA:
        st->pAp = tot[0];
        st->alpha = st->rho / tot[0];
        if (!isfinite(st->alpha)) { st->flags |= FLAG_NAN; st->stop = 1; }
        if (st->hist && st->iter < st->hist_cap) st->hist[3 * st->iter] = st->alpha;
        break;
    case FIN_CG_BETA:
        st->rho_new = tot[0];
        st->beta = tot[0] / st->rho;
        st->rho = tot[0];
        if (st->hist && st->iter < st->hist_cap) {
            st->hist[3 * st->iter + 1] = st->beta;
            st->hist[3 * st->iter + 2] = tot[0];
        }
        st->iter += 1;
        if (!isfinite(tot[0])) { st->flags |= FLAG_NAN; st->stop = 1; }
        else if (tot[0] <= st->stop_r2 || st->iter >= st->maxit) st->stop = 1;
        break;
    case FIN_BICG_ALPHA: {
        st->rv = make_double2(tot[0], tot[1]);
        const double m = fabs(tot[0]) + fabs(tot[1]);
        if (!(m > st->tiny)) { st->flags |= (isfinite(m) ? FLAG_BREAKDOWN : FLAG_NAN); st->stop = 1; break; }
        st->c_alpha = cdiv(st->c_rho, st->rv);
        break;
    }
    case FIN_BICG_OMEGA:
        st->ts = make_double2(tot[0], tot[1]);
        st->tt = tot[2];
        if (!(tot[2] > 0.0) || !finite2(st->ts)) {
            st->flags |= (isfinite(tot[2]) && finite2(st->ts) ? FLAG_BREAKDOWN : FLAG_NAN);
            st->stop = 1;
            break;
        }
        st->c_omega = make_double2(tot[0] / tot[2], tot[1] / tot[2]);
        if (fabs(st->c_omega.x) + fabs(st->c_omega.y) == 0.0) { st->flags |= FLAG_BREAKDOWN; st->stop = 1; }
        break;
    case FIN_BICG_RHO: {
        const double2 rn = make_double2(tot[0], tot[1]);
        st->r2 = tot[2];
        st->iter += 1;
        if (!finite2(rn) || !isfinite(tot[2])) { st->flags |= FLAG_NAN; st->stop = 1; break; }
        if (tot[2] <= st->stop_r2 || st->iter >= st->maxit) { st->stop = 1; st->c_rho_new = rn; break; }
        if (!(fabs(rn.x) + fabs(rn.y) > 0.0)) { st->flags |= FLAG_BREAKDOWN; st->stop = 1; break; }
        st->c_beta = cmul(cdiv(rn, st->c_rho), cdiv(st->c_alpha, st->c_omega));
        st->c_rho = rn;
        st->c_rho_new = rn;
        break;
    }
    default:
        break;
    }
}

// Per-thread FP64 accumulator of NV sums for the RT right-hand sides a thread
// always handles: those of its right-hand-side column c (c*RT .. c*RT+RT-1).
// Kernels arrange their threads so that the column is fixed for the whole
// kernel: c = (linear thread index) mod ncols, with ncols = n / RT columns
// (2-D blocks of (n/RT) x sites, or 1-D blocks whose size is a multiple of n
// walking the elements with a stride that is too).  Contributions computed in
// the working precision (one site's 12 components) are added in FP64, and the
// combination over threads, warps and blocks below runs in a fixed order, so
// the sums are reproducible bit for bit for a given launch configuration.
template <int NV, int RT = 1>
struct RedAcc {
    double v[NV][RT];
    __device__ __forceinline__ void add(int k, int t, double x) { v[k][t] += x; }
};

// Linear thread index and thread count of a (possibly 2-D) block.
__device__ __forceinline__ int ltid() { return threadIdx.y * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int lsize() { return blockDim.x * blockDim.y; }

template <int NV, int RT>
__device__ __forceinline__ void red_init(RedAcc<NV, RT> &acc) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int t = 0; t < RT; ++t) acc.v[k][t] = 0.0;
}

// Sum over the lanes of a warp that may be partial (the block's thread count
// need not be a multiple of 32); lane 0 gets the total.
template <class V>
__device__ __forceinline__ V warp_sum(V x, int lane, int active) {
    const unsigned mask = active >= 32 ? 0xffffffffu : ((1u << active) - 1u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const V y = __shfl_down_sync(mask, x, o);
        if (lane + o < active) x += y;
    }
    return x;
}

// Combine the accumulators of the whole grid (ncols right-hand-side columns
// of RT right-hand sides each): within a warp the lanes of each column are
// folded onto its first lanes, row after row; the warps of a block then add
// their column sums into shared slots one warp after the other; each block
// writes its partial sums to red.partials, and the last block to finish
// (ticket counter) adds them in block order, stores the totals in
// red.sums[k*n + r] and applies the finalize step to red.st[r].  Every thread
// of every block must call it.
template <int NV, int RT>
__device__ void grid_reduce(const Reduce &red, const RedAcc<NV, RT> &acc, int ncols) {
    __shared__ double slot[kPartialSlots];
    __shared__ double tots[kPartialSlots];
    __shared__ bool last;
    const int tid = ltid(), lane = tid & 31, warp = tid >> 5, nthr = lsize(), nw = (nthr + 31) >> 5;
    const int active = min(32, nthr - warp * 32);  // lanes present in this thread's warp
    const int n = ncols * RT, slots = NV * n;
    double *mine = red.partials + (size_t)blockIdx.x * kPartialSlots;
    for (int t = tid; t < slots; t += nthr) slot[t] = 0.0;
    double w[NV][RT];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int t = 0; t < RT; ++t) w[k][t] = acc.v[k][t];
    if (ncols == 1) {
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
            for (int t = 0; t < RT; ++t) w[k][t] = warp_sum(w[k][t], lane, active);
    } else {
        const unsigned mask = active >= 32 ? 0xffffffffu : ((1u << active) - 1u);
        for (int o = ncols; o < 32; o += ncols) {
#pragma unroll
            for (int k = 0; k < NV; ++k)
#pragma unroll
                for (int t = 0; t < RT; ++t) {
                    const double y = __shfl_down_sync(mask, w[k][t], o);
                    if (lane < ncols && lane + o < active) w[k][t] += y;
                }
        }
    }
    __syncthreads();
    const int lead = min(ncols, active);  // lanes holding their warp's column sums
    for (int ww = 0; ww < nw; ++ww) {
        if (warp == ww && lane < lead) {
            const int c = tid % ncols;
#pragma unroll
            for (int k = 0; k < NV; ++k)
#pragma unroll
                for (int t = 0; t < RT; ++t) slot[k * n + c * RT + t] += w[k][t];
        }
        __syncthreads();
    }
    for (int t = tid; t < slots; t += nthr) mine[t] = slot[t];
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(red.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    // The last block sums every slot over the blocks in a fixed order.  With at
    // least twice as many full warps as slots, g = (full warps) / slots warps
    // share a slot: warp q of the slot's group takes blocks q*32 + lane,
    // q*32 + lane + g*32, ... (four loads in flight per lane), then the group's
    // warp sums are added in warp order.  Otherwise each warp takes whole slots,
    // a partial last warp striding by its `active` lanes, so that every block is
    // still visited.
    const double *part = red.partials;
    auto strided_sum = [&](int t, int first, int step) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int b = first;
        for (; b + 3 * step < (int)gridDim.x; b += 4 * step) {
            s0 += __ldcg(part + (size_t)b * kPartialSlots + t);
            s1 += __ldcg(part + (size_t)(b + step) * kPartialSlots + t);
            s2 += __ldcg(part + (size_t)(b + 2 * step) * kPartialSlots + t);
            s3 += __ldcg(part + (size_t)(b + 3 * step) * kPartialSlots + t);
        }
        for (; b < (int)gridDim.x; b += step) s0 += __ldcg(part + (size_t)b * kPartialSlots + t);
        return (s0 + s1) + (s2 + s3);
    };
    const int nfull = nthr >> 5;
    const int g = nfull >= 2 * slots ? nfull / slots : 1;
    if (g > 1) {
        const int t = warp / g, q = warp % g;
        if (warp < slots * g) {  // full warps only: slots * g <= nfull
            double s = strided_sum(t, q * 32 + lane, g * 32);
            s = warp_sum(s, lane, active);
            if (lane == 0) slot[t * g + q] = s;  // slot[] is free again
        }
        __syncthreads();
        if (tid < slots) {
            double s = 0.0;
            for (int k = 0; k < g; ++k) s += slot[tid * g + k];
            tots[tid] = s;
        }
    } else {
        for (int t = warp; t < slots; t += nw) {
            double s = strided_sum(t, lane, active);
            s = warp_sum(s, lane, active);
            if (lane == 0) tots[t] = s;
        }
    }
    __syncthreads();
    if (tid < n) {
        const int r = tid;
        double tr[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            tr[k] = tots[k * n + r];
            red.sums[k * n + r] = tr[k];
        }
        if (red.st) finalize_one(red.fin, red.st + r, tr);
    }
    if (tid == 0) *red.ticket = 0u;
}

// ---------------------------------------------------------------- geometry
// Coordinates of checkerboard site i of parity `par` (x = 2*(i mod Lx/2) + offset).
struct SiteGeom {
    int c[4];     // t, x, y, z
    int lex;      // lexicographic index
};

__device__ __forceinline__ SiteGeom site_geom(const Lattice &L, int par, int i) {
    SiteGeom g;
    unsigned xh, y, z;
    unsigned r = fd_divmod((unsigned)i, L.div_xh, &xh);
    r = fd_divmod(r, L.div_y, &y);
    const int t = (int)fd_divmod(r, L.div_z, &z);
    const int x = 2 * (int)xh + ((par + (int)y + (int)z + t) & 1);
    g.c[0] = t;
    g.c[1] = x;
    g.c[2] = (int)y;
    g.c[3] = (int)z;
    g.lex = ((t * L.L[3] + (int)z) * L.L[2] + (int)y) * L.L[1] + x;
    return g;
}

}  // namespace plq
