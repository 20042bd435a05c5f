// Fused vector kernels of the Krylov solvers.
//
// Every kernel handles whole sites (12 complex components) per thread so that
// the FP16 storage format (per-site norm) is encoded and decoded in one
// place, loops over sites with a grid-stride loop on a grid sized to the
// resident blocks of all SMs, and fuses its axpy-type updates with the
// reductions the solver needs next.  Coefficients come from the device-side
// SolverState, so no kernel waits for the host.
#include "plq_fields.cuh"

namespace plq {

namespace {

constexpr int kBlock = 256;

int grid_for(long long work, bool reduce) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (work + kBlock - 1) / kBlock;
    long long cap = (long long)sms * 8;
    if (reduce && cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

#define SITE_LOOP(Vh)                                                                       \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)(Vh); \
         i += (long long)gridDim.x * blockDim.x)

template <class A, class B>
__device__ __forceinline__ void convert(const cx<A> in[12], cx<B> out[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = {(B)in[k].re, (B)in[k].im};
}

template <int PD, int PS>
__global__ void copy_convert_kernel(int Vh, void *dst, const void *src) {
    SITE_LOOP(Vh) {
        cx<RealOf<PS>> a[12];
        Spinor<PS>::load(src, Vh, i, a);
        cx<RealOf<PD>> b[12];
        convert(a, b);
        Spinor<PD>::store(dst, Vh, i, b);
    }
}

template <int P>
__global__ void zero_kernel(int Vh, void *dst) {
    SITE_LOOP(Vh) {
        cx<RealOf<P>> a[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) a[k] = {0, 0};
        Spinor<P>::store(dst, Vh, i, a);
    }
}

// gamma5 = diag(1, 1, -1, -1): negate spin components 2 and 3
template <int P>
__global__ void gamma5_kernel(int Vh, void *dst, const void *src) {
    SITE_LOOP(Vh) {
        cx<RealOf<P>> a[12];
        Spinor<P>::load(src, Vh, i, a);
#pragma unroll
        for (int k = 6; k < 12; ++k) a[k] = {-a[k].re, -a[k].im};
        Spinor<P>::store(dst, Vh, i, a);
    }
}

template <int P>
__global__ void norm2_kernel(int Vh, const void *v, Reduce red) {
    using T = RealOf<P>;
    T acc[1] = {0};
    SITE_LOOP(Vh) {
        cx<T> a[12];
        Spinor<P>::load(v, Vh, i, a);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[0] += a[k].re * a[k].re + a[k].im * a[k].im;
    }
    double tot[1];
    if (grid_reduce<1, T>(red, acc, tot)) finalize(red, tot, 1);
}

// <a, b> (re, im) and |b|^2
template <int P>
__global__ void dot_norm_kernel(int Vh, const void *av, const void *bv, Reduce red) {
    using T = RealOf<P>;
    T acc[3] = {0, 0, 0};
    SITE_LOOP(Vh) {
        cx<T> a[12], b[12];
        Spinor<P>::load(av, Vh, i, a);
        Spinor<P>::load(bv, Vh, i, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            acc[0] += a[k].re * b[k].re + a[k].im * b[k].im;
            acc[1] += a[k].re * b[k].im - a[k].im * b[k].re;
            acc[2] += b[k].re * b[k].re + b[k].im * b[k].im;
        }
    }
    double tot[3];
    if (grid_reduce<3, T>(red, acc, tot)) finalize(red, tot, 3);
}

// x += alpha p ; r -= alpha q ; rho_new = |r|^2   (x may be stored at higher precision PX)
template <int P, int PX>
__global__ void cg_update_kernel(int Vh, void *x, void *r, const void *p, const void *q, Reduce red,
                                 const SolverState *st) {
    using T = RealOf<P>;
    using TX = RealOf<PX>;
    if (st->stop) return;
    const T alpha = (T)st->alpha;
    T acc[1] = {0};
    SITE_LOOP(Vh) {
        cx<T> pv[12], qv[12], rv[12];
        cx<TX> xv[12];
        Spinor<P>::load(p, Vh, i, pv);
        Spinor<P>::load(q, Vh, i, qv);
        Spinor<P>::load(r, Vh, i, rv);
        Spinor<PX>::load(x, Vh, i, xv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            xv[k].re = fma((TX)alpha, (TX)pv[k].re, xv[k].re);
            xv[k].im = fma((TX)alpha, (TX)pv[k].im, xv[k].im);
            rv[k].re = fma(-alpha, qv[k].re, rv[k].re);
            rv[k].im = fma(-alpha, qv[k].im, rv[k].im);
            acc[0] += rv[k].re * rv[k].re + rv[k].im * rv[k].im;
        }
        Spinor<PX>::store(x, Vh, i, xv);
        Spinor<P>::store(r, Vh, i, rv);
    }
    double tot[1];
    if (grid_reduce<1, T>(red, acc, tot)) finalize(red, tot, 1);
}

// p = r + beta p
template <int P>
__global__ void cg_direction_kernel(int Vh, void *p, const void *r, const SolverState *st) {
    using T = RealOf<P>;
    if (st->stop) return;
    const T beta = (T)st->beta;
    SITE_LOOP(Vh) {
        cx<T> pv[12], rv[12];
        Spinor<P>::load(p, Vh, i, pv);
        Spinor<P>::load(r, Vh, i, rv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            pv[k].re = fma(beta, pv[k].re, rv[k].re);
            pv[k].im = fma(beta, pv[k].im, rv[k].im);
        }
        Spinor<P>::store(p, Vh, i, pv);
    }
}

// dst64 += src
template <int PS>
__global__ void accumulate_kernel(int Vh, void *dst, const void *src) {
    SITE_LOOP(Vh) {
        cx<RealOf<PS>> a[12];
        cx<double> d[12];
        Spinor<PS>::load(src, Vh, i, a);
        Spinor<PLQ_F64>::load(dst, Vh, i, d);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            d[k].re += (double)a[k].re;
            d[k].im += (double)a[k].im;
        }
        Spinor<PLQ_F64>::store(dst, Vh, i, d);
    }
}

// y = x + a y  (FP64)
__global__ void xpay64_kernel(int Vh, const void *x, double a, void *y) {
    SITE_LOOP(Vh) {
        cx<double> xv[12], yv[12];
        Spinor<PLQ_F64>::load(x, Vh, i, xv);
        Spinor<PLQ_F64>::load(y, Vh, i, yv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            yv[k].re = fma(a, yv[k].re, xv[k].re);
            yv[k].im = fma(a, yv[k].im, xv[k].im);
        }
        Spinor<PLQ_F64>::store(y, Vh, i, yv);
    }
}

template <class T>
__device__ __forceinline__ cx<T> cmulc(double2 c, cx<T> z) {
    const T a = (T)c.x, b = (T)c.y;
    return {a * z.re - b * z.im, a * z.im + b * z.re};
}

// p = r + beta (p - omega v)
template <int P>
__global__ void bicg_p_kernel(int Vh, void *p, const void *r, const void *v, const SolverState *st) {
    using T = RealOf<P>;
    if (st->stop) return;
    const double2 beta = st->c_beta, omega = st->c_omega;
    SITE_LOOP(Vh) {
        cx<T> pv[12], rv[12], vv[12];
        Spinor<P>::load(p, Vh, i, pv);
        Spinor<P>::load(r, Vh, i, rv);
        Spinor<P>::load(v, Vh, i, vv);
#pragma unroll
        for (int k = 0; k < 12; ++k) pv[k] = cadd(rv[k], cmulc(beta, csub(pv[k], cmulc(omega, vv[k]))));
        Spinor<P>::store(p, Vh, i, pv);
    }
}

// s = r - alpha v
template <int P>
__global__ void bicg_s_kernel(int Vh, void *s, const void *r, const void *v, const SolverState *st) {
    using T = RealOf<P>;
    if (st->stop) return;
    const double2 alpha = st->c_alpha;
    SITE_LOOP(Vh) {
        cx<T> rv[12], vv[12];
        Spinor<P>::load(r, Vh, i, rv);
        Spinor<P>::load(v, Vh, i, vv);
#pragma unroll
        for (int k = 0; k < 12; ++k) rv[k] = csub(rv[k], cmulc(alpha, vv[k]));
        Spinor<P>::store(s, Vh, i, rv);
    }
}

// x += alpha p + omega s ; r = s - omega t ; <rhat, r>, |r|^2
template <int P, int PX>
__global__ void bicg_update_kernel(int Vh, void *x, void *r, const void *p, const void *s, const void *t,
                                   const void *rhat, Reduce red, const SolverState *st) {
    using T = RealOf<P>;
    using TX = RealOf<PX>;
    if (st->stop) return;
    const double2 alpha = st->c_alpha, omega = st->c_omega;
    T acc[3] = {0, 0, 0};
    SITE_LOOP(Vh) {
        cx<T> pv[12], sv[12], tv[12], hv[12];
        cx<TX> xv[12];
        Spinor<P>::load(p, Vh, i, pv);
        Spinor<P>::load(s, Vh, i, sv);
        Spinor<P>::load(t, Vh, i, tv);
        Spinor<P>::load(rhat, Vh, i, hv);
        Spinor<PX>::load(x, Vh, i, xv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            cx<T> dx = cadd(cmulc(alpha, pv[k]), cmulc(omega, sv[k]));
            xv[k] = {xv[k].re + (TX)dx.re, xv[k].im + (TX)dx.im};
            cx<T> rn = csub(sv[k], cmulc(omega, tv[k]));
            sv[k] = rn;
            acc[0] += hv[k].re * rn.re + hv[k].im * rn.im;
            acc[1] += hv[k].re * rn.im - hv[k].im * rn.re;
            acc[2] += rn.re * rn.re + rn.im * rn.im;
        }
        Spinor<PX>::store(x, Vh, i, xv);
        Spinor<P>::store(r, Vh, i, sv);
    }
    double tot[3];
    if (grid_reduce<3, T>(red, acc, tot)) finalize(red, tot, 3);
}

}  // namespace

#define DISPATCH_P(prec, KERNEL, ...)                                                 \
    do {                                                                              \
        if ((prec) == PLQ_F64) KERNEL<PLQ_F64><<<grid, kBlock, 0, s>>>(__VA_ARGS__);  \
        else if ((prec) == PLQ_F32) KERNEL<PLQ_F32><<<grid, kBlock, 0, s>>>(__VA_ARGS__); \
        else KERNEL<PLQ_F16><<<grid, kBlock, 0, s>>>(__VA_ARGS__);                    \
    } while (0)

plq_status blas_copy_convert(int Vh, void *dst, int pd, const void *src, int ps, cudaStream_t s) {
    const int grid = grid_for(Vh, false);
#define CC(A, B) \
    if (pd == A && ps == B) copy_convert_kernel<A, B><<<grid, kBlock, 0, s>>>(Vh, dst, src)
    CC(PLQ_F64, PLQ_F64); else CC(PLQ_F64, PLQ_F32); else CC(PLQ_F64, PLQ_F16);
    else CC(PLQ_F32, PLQ_F64); else CC(PLQ_F32, PLQ_F32); else CC(PLQ_F32, PLQ_F16);
    else CC(PLQ_F16, PLQ_F64); else CC(PLQ_F16, PLQ_F32); else CC(PLQ_F16, PLQ_F16);
#undef CC
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_zero(int Vh, void *dst, int prec, cudaStream_t s) {
    const int grid = grid_for(Vh, false);
    DISPATCH_P(prec, zero_kernel, Vh, dst);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_gamma5(int Vh, void *dst, const void *src, int prec, cudaStream_t s) {
    const int grid = grid_for(Vh, false);
    DISPATCH_P(prec, gamma5_kernel, Vh, dst, src);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_norm2(int Vh, const void *v, int prec, const Reduce &red, cudaStream_t s) {
    const int grid = grid_for(Vh, true);
    DISPATCH_P(prec, norm2_kernel, Vh, v, red);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_dot_norm(int Vh, const void *a, const void *b, int prec, const Reduce &red, cudaStream_t s) {
    const int grid = grid_for(Vh, true);
    DISPATCH_P(prec, dot_norm_kernel, Vh, a, b, red);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_cg_update(int Vh, void *x, void *r, const void *p, const void *q, int prec, const Reduce &red,
                          const SolverState *st, cudaStream_t s) {
    const int grid = grid_for(Vh, true);
    // the solution accumulator is FP64 for FP64 solves and FP32 otherwise
    if (prec == PLQ_F64) cg_update_kernel<PLQ_F64, PLQ_F64><<<grid, kBlock, 0, s>>>(Vh, x, r, p, q, red, st);
    else if (prec == PLQ_F32) cg_update_kernel<PLQ_F32, PLQ_F32><<<grid, kBlock, 0, s>>>(Vh, x, r, p, q, red, st);
    else cg_update_kernel<PLQ_F16, PLQ_F32><<<grid, kBlock, 0, s>>>(Vh, x, r, p, q, red, st);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_cg_direction(int Vh, void *p, const void *r, int prec, const SolverState *st, cudaStream_t s) {
    const int grid = grid_for(Vh, false);
    DISPATCH_P(prec, cg_direction_kernel, Vh, p, r, st);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_accumulate(int Vh, void *dst64, const void *src, int ps, cudaStream_t s) {
    const int grid = grid_for(Vh, false);
    DISPATCH_P(ps, accumulate_kernel, Vh, dst64, src);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_xpay64(int Vh, const void *x, double a, void *y, cudaStream_t s) {
    const int grid = grid_for(Vh, false);
    xpay64_kernel<<<grid, kBlock, 0, s>>>(Vh, x, a, y);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_bicg_p(int Vh, void *p, const void *r, const void *v, int prec, const SolverState *st,
                       cudaStream_t s) {
    const int grid = grid_for(Vh, false);
    DISPATCH_P(prec, bicg_p_kernel, Vh, p, r, v, st);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_bicg_s(int Vh, void *sv, const void *r, const void *v, int prec, const SolverState *st,
                       cudaStream_t s) {
    const int grid = grid_for(Vh, false);
    DISPATCH_P(prec, bicg_s_kernel, Vh, sv, r, v, st);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status blas_bicg_update(int Vh, void *x, void *r, const void *p, const void *sv, const void *t,
                            const void *rhat, int prec, const Reduce &red, const SolverState *st, cudaStream_t s) {
    const int grid = grid_for(Vh, true);
    if (prec == PLQ_F64)
        bicg_update_kernel<PLQ_F64, PLQ_F64><<<grid, kBlock, 0, s>>>(Vh, x, r, p, sv, t, rhat, red, st);
    else if (prec == PLQ_F32)
        bicg_update_kernel<PLQ_F32, PLQ_F32><<<grid, kBlock, 0, s>>>(Vh, x, r, p, sv, t, rhat, red, st);
    else
        bicg_update_kernel<PLQ_F16, PLQ_F32><<<grid, kBlock, 0, s>>>(Vh, x, r, p, sv, t, rhat, red, st);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

}  // namespace plq
