// Fused vector kernels of the Krylov solvers.
//
// Every kernel handles whole (site, right-hand side) elements -- 12 complex
// components -- per thread so that the FP16 storage format (per-site norm) is
// encoded and decoded in one place, loops over elements with a grid-stride
// loop on a grid sized to the resident blocks of all SMs, and fuses its
// axpy-type updates with the reductions the solver needs next.  Coefficients
// come from the device-side SolverState of each right-hand side, so no kernel
// waits for the host.
#include "plq_fields.cuh"

namespace plq {

namespace {

constexpr int kBlock = 256;

// Threads per block of the reducing kernels for n interleaved right-hand
// sides: a multiple of n, so that with the grid-stride element loop every
// thread keeps one right-hand side (element e belongs to e mod n) and the
// reduction can combine its FP64 partial sums in a fixed order.
int red_block(int n) { return n > 1 ? n * (kBlock / n) : kBlock; }

int grid_for(long long work, bool reduce, int block = kBlock) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (work + block - 1) / block;
    long long cap = (long long)sms * 8;
    if (reduce && cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

__device__ __forceinline__ int rhs_of(long long e, int n) { return n == 1 ? 0 : (int)(e % n); }

#define ELEM_LOOP(N)                                                                       \
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)(N); \
         e += (long long)gridDim.x * blockDim.x)

template <class A, class B>
__device__ __forceinline__ void convert(const cx<A> in[12], cx<B> out[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = {(B)in[k].re, (B)in[k].im};
}

template <int PD, int PS>
__global__ void copy_convert_kernel(long long N, void *dst, const void *src) {
    ELEM_LOOP(N) {
        cx<RealOf<PS>> a[12];
        Spinor<PS>::load(src, N, e, a);
        cx<RealOf<PD>> b[12];
        convert(a, b);
        Spinor<PD>::store(dst, N, e, b);
    }
}

template <int P>
__global__ void zero_kernel(long long N, void *dst) {
    ELEM_LOOP(N) {
        cx<RealOf<P>> a[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) a[k] = {0, 0};
        Spinor<P>::store(dst, N, e, a);
    }
}

// gamma5 = diag(1, 1, -1, -1): negate spin components 2 and 3
template <int P>
__global__ void gamma5_kernel(long long N, void *dst, const void *src) {
    ELEM_LOOP(N) {
        cx<RealOf<P>> a[12];
        Spinor<P>::load(src, N, e, a);
#pragma unroll
        for (int k = 6; k < 12; ++k) a[k] = {-a[k].re, -a[k].im};
        Spinor<P>::store(dst, N, e, a);
    }
}

template <int P>
__global__ void norm2_kernel(long long N, int n, const void *v, Reduce red) {
    using T = RealOf<P>;
    RedAcc<1> acc;
    red_init(acc);
    ELEM_LOOP(N) {
        cx<T> a[12];
        Spinor<P>::load(v, N, e, a);
        T s = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) s += a[k].re * a[k].re + a[k].im * a[k].im;
        acc.add(0, 0, s);
    }
    grid_reduce(red, acc, n);
}

// <a, b> (re, im) and |b|^2
template <int P>
__global__ void dot_norm_kernel(long long N, int n, const void *av, const void *bv, Reduce red) {
    using T = RealOf<P>;
    RedAcc<3> acc;
    red_init(acc);
    ELEM_LOOP(N) {
        cx<T> a[12], b[12];
        Spinor<P>::load(av, N, e, a);
        Spinor<P>::load(bv, N, e, b);
        T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            s0 += a[k].re * b[k].re + a[k].im * b[k].im;
            s1 += a[k].re * b[k].im - a[k].im * b[k].re;
            s2 += b[k].re * b[k].re + b[k].im * b[k].im;
        }
        acc.add(0, 0, s0);
        acc.add(1, 0, s1);
        acc.add(2, 0, s2);
    }
    grid_reduce(red, acc, n);
}

// x += alpha p ; r -= alpha q ; rho_new = |r|^2   (x may be stored at higher precision PX)
template <int P, int PX>
__global__ void cg_update_kernel(long long N, int n, void *x, void *r, const void *p, const void *q, Reduce red,
                                 const SolverState *st) {
    using T = RealOf<P>;
    using TX = RealOf<PX>;
    RedAcc<1> acc;
    red_init(acc);
    ELEM_LOOP(N) {
        const int rr = rhs_of(e, n);
        if (st[rr].stop) continue;
        const T alpha = (T)st[rr].alpha;
        cx<T> pv[12], qv[12], rv[12];
        cx<TX> xv[12];
        Spinor<P>::load(p, N, e, pv);
        Spinor<P>::load(q, N, e, qv);
        Spinor<P>::load(r, N, e, rv);
        Spinor<PX>::load(x, N, e, xv);
        T s = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            xv[k].re = fma((TX)alpha, (TX)pv[k].re, xv[k].re);
            xv[k].im = fma((TX)alpha, (TX)pv[k].im, xv[k].im);
            rv[k].re = fma(-alpha, qv[k].re, rv[k].re);
            rv[k].im = fma(-alpha, qv[k].im, rv[k].im);
            s += rv[k].re * rv[k].re + rv[k].im * rv[k].im;
        }
        Spinor<PX>::store(x, N, e, xv);
        Spinor<P>::store(r, N, e, rv);
        acc.add(0, 0, s);
    }
    grid_reduce(red, acc, n);
}

// p = r + beta p
template <int P>
__global__ void cg_direction_kernel(long long N, int n, void *p, const void *r, const SolverState *st) {
    using T = RealOf<P>;
    ELEM_LOOP(N) {
        const int rr = rhs_of(e, n);
        if (st[rr].stop) continue;
        const T beta = (T)st[rr].beta;
        cx<T> pv[12], rv[12];
        Spinor<P>::load(p, N, e, pv);
        Spinor<P>::load(r, N, e, rv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            pv[k].re = fma(beta, pv[k].re, rv[k].re);
            pv[k].im = fma(beta, pv[k].im, rv[k].im);
        }
        Spinor<P>::store(p, N, e, pv);
    }
}

// dst64 += src
template <int PS>
__global__ void accumulate_kernel(long long N, void *dst, const void *src) {
    ELEM_LOOP(N) {
        cx<RealOf<PS>> a[12];
        cx<double> d[12];
        Spinor<PS>::load(src, N, e, a);
        Spinor<PLQ_F64>::load(dst, N, e, d);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            d[k].re += (double)a[k].re;
            d[k].im += (double)a[k].im;
        }
        Spinor<PLQ_F64>::store(dst, N, e, d);
    }
}

// Per right-hand-side power-of-two scales of the mixed-precision solves.
struct RhsScale {
    double f[PLQ_MAX_RHS];
};

// f[r] by selects (run-time indexing would copy the array to local memory)
__device__ __forceinline__ double scale_of(const RhsScale &S, long long e, int n) {
    if (n == 1) return S.f[0];
    const int r = (int)(e % n);
    double v = S.f[0];
#pragma unroll
    for (int q = 1; q < PLQ_MAX_RHS; ++q) v = r == q ? S.f[q] : v;
    return v;
}

// dst (FP64, n interleaved right-hand sides) *= f[rhs]
__global__ void scale64_kernel(long long N, int n, double2 *v, RhsScale S) {
    ELEM_LOOP(N) {
        const double f = scale_of(S, e, n);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 a = v[(size_t)k * N + e];
            v[(size_t)k * N + e] = make_double2(f * a.x, f * a.y);
        }
    }
}

// dst (FP64) += f[rhs] * src
template <int PS>
__global__ void accumulate_scaled_kernel(long long N, int n, void *dst, const void *src, RhsScale S) {
    ELEM_LOOP(N) {
        const double f = scale_of(S, e, n);
        cx<RealOf<PS>> a[12];
        cx<double> d[12];
        Spinor<PS>::load(src, N, e, a);
        Spinor<PLQ_F64>::load(dst, N, e, d);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            d[k].re = fma(f, (double)a[k].re, d[k].re);
            d[k].im = fma(f, (double)a[k].im, d[k].im);
        }
        Spinor<PLQ_F64>::store(dst, N, e, d);
    }
}

// dst = scale (1 + i nu gamma5) src
template <int P>
__global__ void twist_kernel(long long N, void *dst, const void *src, double nu, double scale) {
    using T = RealOf<P>;
    ELEM_LOOP(N) {
        cx<T> v[12];
        Spinor<P>::load(src, N, e, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const T g = (T)(k < 6 ? nu : -nu);
            v[k] = {(T)scale * (v[k].re - g * v[k].im), (T)scale * (v[k].im + g * v[k].re)};
        }
        Spinor<P>::store(dst, N, e, v);
    }
}

// y = x + a y  (FP64)
__global__ void xpay64_kernel(long long N, const void *x, double a, void *y) {
    ELEM_LOOP(N) {
        cx<double> xv[12], yv[12];
        Spinor<PLQ_F64>::load(x, N, e, xv);
        Spinor<PLQ_F64>::load(y, N, e, yv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            yv[k].re = fma(a, yv[k].re, xv[k].re);
            yv[k].im = fma(a, yv[k].im, xv[k].im);
        }
        Spinor<PLQ_F64>::store(y, N, e, yv);
    }
}

template <class T>
__device__ __forceinline__ cx<T> cmulc(double2 c, cx<T> z) {
    const T a = (T)c.x, b = (T)c.y;
    return {a * z.re - b * z.im, a * z.im + b * z.re};
}

// p = r + beta (p - omega v)
template <int P>
__global__ void bicg_p_kernel(long long N, int n, void *p, const void *r, const void *v, const SolverState *st) {
    using T = RealOf<P>;
    ELEM_LOOP(N) {
        const int rr = rhs_of(e, n);
        if (st[rr].stop) continue;
        const double2 beta = st[rr].c_beta, omega = st[rr].c_omega;
        cx<T> pv[12], rv[12], vv[12];
        Spinor<P>::load(p, N, e, pv);
        Spinor<P>::load(r, N, e, rv);
        Spinor<P>::load(v, N, e, vv);
#pragma unroll
        for (int k = 0; k < 12; ++k) pv[k] = cadd(rv[k], cmulc(beta, csub(pv[k], cmulc(omega, vv[k]))));
        Spinor<P>::store(p, N, e, pv);
    }
}

// s = r - alpha v
template <int P>
__global__ void bicg_s_kernel(long long N, int n, void *s, const void *r, const void *v, const SolverState *st) {
    using T = RealOf<P>;
    ELEM_LOOP(N) {
        const int rr = rhs_of(e, n);
        if (st[rr].stop) continue;
        const double2 alpha = st[rr].c_alpha;
        cx<T> rv[12], vv[12];
        Spinor<P>::load(r, N, e, rv);
        Spinor<P>::load(v, N, e, vv);
#pragma unroll
        for (int k = 0; k < 12; ++k) rv[k] = csub(rv[k], cmulc(alpha, vv[k]));
        Spinor<P>::store(s, N, e, rv);
    }
}

// x += alpha p + omega s ; r = s - omega t ; <rhat, r>, |r|^2
template <int P, int PX>
__global__ void bicg_update_kernel(long long N, int n, void *x, void *r, const void *p, const void *s,
                                   const void *t, const void *rhat, Reduce red, const SolverState *st) {
    using T = RealOf<P>;
    using TX = RealOf<PX>;
    RedAcc<3> acc;
    red_init(acc);
    ELEM_LOOP(N) {
        const int rr = rhs_of(e, n);
        if (st[rr].stop) continue;
        const double2 alpha = st[rr].c_alpha, omega = st[rr].c_omega;
        cx<T> pv[12], sv[12], tv[12], hv[12];
        cx<TX> xv[12];
        Spinor<P>::load(p, N, e, pv);
        Spinor<P>::load(s, N, e, sv);
        Spinor<P>::load(t, N, e, tv);
        Spinor<P>::load(rhat, N, e, hv);
        Spinor<PX>::load(x, N, e, xv);
        T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            cx<T> dx = cadd(cmulc(alpha, pv[k]), cmulc(omega, sv[k]));
            xv[k] = {xv[k].re + (TX)dx.re, xv[k].im + (TX)dx.im};
            cx<T> rn = csub(sv[k], cmulc(omega, tv[k]));
            sv[k] = rn;
            s0 += hv[k].re * rn.re + hv[k].im * rn.im;
            s1 += hv[k].re * rn.im - hv[k].im * rn.re;
            s2 += rn.re * rn.re + rn.im * rn.im;
        }
        Spinor<PX>::store(x, N, e, xv);
        Spinor<P>::store(r, N, e, sv);
        acc.add(0, 0, s0);
        acc.add(1, 0, s1);
        acc.add(2, 0, s2);
    }
    grid_reduce(red, acc, n);
}

}  // namespace

#define DISPATCH_PB(prec, BLK, KERNEL, ...)                                                \
    do {                                                                                   \
        if ((prec) == PLQ_F64) KERNEL<PLQ_F64><<<grid, (BLK), 0, s>>>(__VA_ARGS__);        \
        else if ((prec) == PLQ_F32) KERNEL<PLQ_F32><<<grid, (BLK), 0, s>>>(__VA_ARGS__);   \
        else KERNEL<PLQ_F16><<<grid, (BLK), 0, s>>>(__VA_ARGS__);                          \
    } while (0)

#define DISPATCH_P(prec, KERNEL, ...)                                                      \
    do {                                                                                   \
        if ((prec) == PLQ_F64) KERNEL<PLQ_F64><<<grid, kBlock, 0, s>>>(__VA_ARGS__);       \
        else if ((prec) == PLQ_F32) KERNEL<PLQ_F32><<<grid, kBlock, 0, s>>>(__VA_ARGS__);  \
        else KERNEL<PLQ_F16><<<grid, kBlock, 0, s>>>(__VA_ARGS__);                         \
    } while (0)

plq_status blas_copy_convert(long long N, void *dst, int pd, const void *src, int ps, cudaStream_t s) {
    const int grid = grid_for(N, false);
#define CC(A, B) \
    if (pd == A && ps == B) copy_convert_kernel<A, B><<<grid, kBlock, 0, s>>>(N, dst, src)
    CC(PLQ_F64, PLQ_F64); else CC(PLQ_F64, PLQ_F32); else CC(PLQ_F64, PLQ_F16);
    else CC(PLQ_F32, PLQ_F64); else CC(PLQ_F32, PLQ_F32); else CC(PLQ_F32, PLQ_F16);
    else CC(PLQ_F16, PLQ_F64); else CC(PLQ_F16, PLQ_F32); else CC(PLQ_F16, PLQ_F16);
#undef CC
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_zero(long long N, void *dst, int prec, cudaStream_t s) {
    const int grid = grid_for(N, false);
    DISPATCH_P(prec, zero_kernel, N, dst);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_gamma5(long long N, void *dst, const void *src, int prec, cudaStream_t s) {
    const int grid = grid_for(N, false);
    DISPATCH_P(prec, gamma5_kernel, N, dst, src);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_norm2(long long N, int n, const void *v, int prec, const Reduce &red, cudaStream_t s) {
    const int blk = red_block(n);
    const int grid = grid_for(N, true, blk);
    DISPATCH_PB(prec, blk, norm2_kernel, N, n, v, red);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_dot_norm(long long N, int n, const void *a, const void *b, int prec, const Reduce &red,
                         cudaStream_t s) {
    const int blk = red_block(n);
    const int grid = grid_for(N, true, blk);
    DISPATCH_PB(prec, blk, dot_norm_kernel, N, n, a, b, red);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_cg_update(long long N, int n, void *x, void *r, const void *p, const void *q, int prec,
                          const Reduce &red, const SolverState *st, cudaStream_t s) {
    const int blk = red_block(n);
    const int grid = grid_for(N, true, blk);
    // the solution accumulator is FP64 for FP64 solves and FP32 otherwise
    if (prec == PLQ_F64) cg_update_kernel<PLQ_F64, PLQ_F64><<<grid, blk, 0, s>>>(N, n, x, r, p, q, red, st);
    else if (prec == PLQ_F32) cg_update_kernel<PLQ_F32, PLQ_F32><<<grid, blk, 0, s>>>(N, n, x, r, p, q, red, st);
    else cg_update_kernel<PLQ_F16, PLQ_F32><<<grid, blk, 0, s>>>(N, n, x, r, p, q, red, st);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_cg_direction(long long N, int n, void *p, const void *r, int prec, const SolverState *st,
                             cudaStream_t s) {
    const int grid = grid_for(N, false);
    DISPATCH_P(prec, cg_direction_kernel, N, n, p, r, st);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_accumulate(long long N, void *dst64, const void *src, int ps, cudaStream_t s) {
    const int grid = grid_for(N, false);
    DISPATCH_P(ps, accumulate_kernel, N, dst64, src);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_scale64(long long N, int n, void *v, const double *f, cudaStream_t s) {
    RhsScale S{};
    for (int r = 0; r < n && r < PLQ_MAX_RHS; ++r) S.f[r] = f[r];
    scale64_kernel<<<grid_for(N, false), kBlock, 0, s>>>(N, n, static_cast<double2 *>(v), S);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_accumulate_scaled(long long N, int n, void *dst64, const void *src, int ps, const double *f,
                                  cudaStream_t s) {
    RhsScale S{};
    for (int r = 0; r < n && r < PLQ_MAX_RHS; ++r) S.f[r] = f[r];
    const int grid = grid_for(N, false);
    DISPATCH_P(ps, accumulate_scaled_kernel, N, n, dst64, src, S);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_twist(long long N, void *dst, const void *src, int prec, double nu, double scale, cudaStream_t s) {
    const int grid = grid_for(N, false);
    DISPATCH_P(prec, twist_kernel, N, dst, src, nu, scale);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_xpay64(long long N, const void *x, double a, void *y, cudaStream_t s) {
    const int grid = grid_for(N, false);
    xpay64_kernel<<<grid, kBlock, 0, s>>>(N, x, a, y);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_bicg_p(long long N, int n, void *p, const void *r, const void *v, int prec, const SolverState *st,
                       cudaStream_t s) {
    const int grid = grid_for(N, false);
    DISPATCH_P(prec, bicg_p_kernel, N, n, p, r, v, st);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_bicg_s(long long N, int n, void *sv, const void *r, const void *v, int prec, const SolverState *st,
                       cudaStream_t s) {
    const int grid = grid_for(N, false);
    DISPATCH_P(prec, bicg_s_kernel, N, n, sv, r, v, st);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_bicg_update(long long N, int n, void *x, void *r, const void *p, const void *sv, const void *t,
                            const void *rhat, int prec, const Reduce &red, const SolverState *st, cudaStream_t s) {
    const int blk = red_block(n);
    const int grid = grid_for(N, true, blk);
    if (prec == PLQ_F64)
        bicg_update_kernel<PLQ_F64, PLQ_F64><<<grid, blk, 0, s>>>(N, n, x, r, p, sv, t, rhat, red, st);
    else if (prec == PLQ_F32)
        bicg_update_kernel<PLQ_F32, PLQ_F32><<<grid, blk, 0, s>>>(N, n, x, r, p, sv, t, rhat, red, st);
    else
        bicg_update_kernel<PLQ_F16, PLQ_F32><<<grid, blk, 0, s>>>(N, n, x, r, p, sv, t, rhat, red, st);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

}  // namespace plq
