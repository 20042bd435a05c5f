// Persistent batched CG: many independent even-odd solves (different lattices,
// kappas and iteration counts) in one cooperative kernel launch, captured in a
// CUDA graph.
//
// Every system runs its own state machine (setup, FP64 true residual, inner
// CG iterations at the inner precision, FP64 reliable update, final x_o).
// The kernel advances all systems in lockstep phases separated by grid-wide
// barriers; in each phase every active system contributes its sites to one
// concatenated work range that all blocks share, so a converged (retired)
// system simply stops contributing and its share of the GPU goes to the
// others.  Each phase reduces at most one number per system (a norm); the
// totals are combined with atomics and every block then applies the same
// deterministic state update from them, so no block waits for another to
// publish scalars.  The barrier spins with a time limit: on expiry it records
// PLQ_ERR_TIMEOUT in a status word and all blocks leave the kernel.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "plq_hop_impl.cuh"

namespace plq {
namespace {

constexpr int kMaxSys = 64;

struct BatchSystem {
    Lattice lat;
    double kappa, tol, delta;
    int maxit, use_x0;
    const void *g64;  // FP64 18-real gauge copy
    size_t gb64;
    const void *gL;   // inner-precision gauge copy
    size_t gbL;
    const void *be, *bo;
    void *xe, *xo;
    int inner_scaled;  // 1: scale the inner iteration (FP32 / FP16 inner precision)
    void *bhat, *s64, *to64;           // FP64 half fields (to64: odd)
    void *rL, *pL, *qL, *mpL, *toL;    // inner half fields (toL: odd)
    void *xL;                          // inner solution accumulator (FP32 or FP64)
};

struct BatchResult {
    int iterations, n_reliable, flags, done;
    double true_rel_schur;  // ||bhat - Mhat x_e|| / ||b|| at the last check
};

enum Mode {
    M_SETUP0 = 0,  // |b|^2, x_e = 0
    M_SETUP1,      // bhat = b_e + kappa H_eo b_o
    M_RES1,        // to = H_oe x_e                            (FP64)
    M_RES2,        // s = bhat - x_e + kappa^2 H_eo to, |s|^2   (FP64; s also kept as sL)
    M_RES3,        // toL = D_oe sL                            (inner, dagger)
    M_RES4,        // rL = sL - kappa^2 D_eo toL, |rL|^2       (inner, dagger)
    M_RES5,        // xL = 0, p = rL (+ beta p)
    M_IT1,         // to = H_oe p
    M_IT2,         // mp = p - kappa^2 H_eo to, |mp|^2 -> alpha
    M_IT3,         // to = D_oe mp
    M_IT4,         // q = mp - kappa^2 D_eo to
    M_IT5,         // x += alpha p, r -= alpha q, |r|^2 -> beta
    M_IT6,         // p = r + beta p
    M_ACC,         // x_e += xL (FP64)
    M_FIN1,        // x_o = b_o + kappa H_oe x_e
    M_ZERO,        // zero source: x_o = 0
    M_DONE
};

enum { BF_NAN = 1, BF_NOT_CONVERGED = 2 };

struct SysRun {
    int mode, iter, nrel, first, flags, reduces;
    double b2, s2, r2, rho, alpha, beta, last_rho, stop_r2, target2, sigma;
    double sc;  // power of two applied where the residual enters the inner precision
};

struct BatchArgs {
    const BatchSystem *sys;
    BatchResult *res;
    int nsys;
    double *acc;          // 3 x kMaxSys rotating accumulators
    unsigned *bar_count;  // barrier
    unsigned *bar_gen;
    int *status;          // 0 ok, PLQ_ERR_TIMEOUT
    long long spin_limit; // clock cycles a barrier may wait
    long long max_phases;
};

// Grid-wide barrier with a bounded wait.  Returns false if any block gave up.
__device__ bool grid_sync(const BatchArgs &a) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned *gen = a.bar_gen;
        volatile int *status = a.status;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(a.bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            *a.bar_count = 0u;
            __threadfence();
            atomicAdd(a.bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (*status != 0) break;
                if (clock64() - t0 > a.spin_limit) {
                    atomicCAS(a.status, 0, (int)PLQ_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok = (*status == 0);
    }
    __syncthreads();
    return ok != 0;
}

template <int P>
__device__ __forceinline__ void ld(const void *f, int Vh, int i, cx<RealOf<P>> v[12]) {
    Spinor<P>::load(f, (size_t)Vh, (size_t)i, v);
}
template <int P>
__device__ __forceinline__ void st(void *f, int Vh, int i, const cx<RealOf<P>> v[12]) {
    Spinor<P>::store(f, (size_t)Vh, (size_t)i, v);
}

// z * i^k for a run-time k (0..3)
template <class T>
__device__ __forceinline__ cx<T> mul_ipow_rt(cx<T> z, int k) {
    const bool sw = k & 1, neg_re = k == 1 || k == 2, neg_im = k >= 2;
    cx<T> w = {sw ? z.im : z.re, sw ? z.re : z.im};
    if (neg_re) w.re = -w.re;
    if (neg_im) w.im = -w.im;
    return w;
}

// Direction d = 2 mu + back of one output site with every direction-dependent
// choice taken at run time.  The persistent kernel inlines a hopping site for
// each of its phases; for the FP64 phases one copy of the direction body
// (instead of eight unrolled copies per phase) keeps its code and register
// demand down.  Projection table as in plq_hop_impl.cuh: spin pair (2, 3) for
// mu = 0, 3 and (3, 2) for mu = 1, 2, phases i^k0, i^k1 of (1 - gamma_mu),
// k + 2 for (1 + gamma_mu); DAG swaps the two projectors.
template <int P, int R>
__device__ __forceinline__ void hop_dir_rt(const Lattice &L, const char *g, size_t gb, int par, bool dag,
                                           const void *in, const SiteGeom &geo, int i, int d,
                                           cx<RealOf<P>> acc[12]) {
    using T = RealOf<P>;
    const int mu = d >> 1;
    const bool back = d & 1;
    const int st = lex_stride(L, mu);
    const int cm = mu == 0 ? geo.c[0] : mu == 1 ? geo.c[1] : mu == 2 ? geo.c[2] : geo.c[3];
    const int Lm = mu == 0 ? L.L[0] : mu == 1 ? L.L[1] : mu == 2 ? L.L[2] : L.L[3];
    int j;
    bool flip;
    if (!back) {
        j = ((cm == Lm - 1) ? geo.lex - (Lm - 1) * st : geo.lex + st) >> 1;
        flip = mu == 0 && cm == Lm - 1 && L.t_bc < 0;
    } else {
        j = ((cm == 0) ? geo.lex + (Lm - 1) * st : geo.lex - st) >> 1;
        flip = mu == 0 && cm == 0 && L.t_bc < 0;
    }
    const int lpar = back ? 1 - par : par;
    cx<T> u[3][3];
    Link<P, R>::load(g + (size_t)(lpar * 4 + mu) * gb, L.Vh, back ? j : i, u);
    if (back) {  // U^dagger
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int y = x; y < 3; ++y) {
                const cx<T> p = u[x][y], q = u[y][x];
                u[x][y] = {q.re, -q.im};
                u[y][x] = {p.re, -p.im};
            }
    }
    const bool p2 = mu == 0 || mu == 3;
    const int kb0 = mu == 1 || mu == 3 ? 1 : 0;
    const int kb1 = mu == 0 ? 0 : mu == 1 ? 1 : mu == 2 ? 2 : 3;
    const int add = (back != dag) ? 2 : 0;
    const int k0 = (kb0 + add) & 3, k1 = (kb1 + add) & 3;
    cx<T> phi[12], h[6], uh[6];
    T sc = load_for_projection<P>(in, (size_t)L.Vh, (size_t)j, phi);
    if (flip) sc = -sc;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<T> a0 = p2 ? phi[6 + c] : phi[9 + c], a1 = p2 ? phi[9 + c] : phi[6 + c];
        h[c] = cadd(phi[c], mul_ipow_rt(a0, k0));
        h[3 + c] = cadd(phi[3 + c], mul_ipow_rt(a1, k1));
    }
    if (P == PLQ_F16 || flip) {
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = {sc * h[k].re, sc * h[k].im};
    }
    su3_mul(u, h, uh);
    const int j0 = (4 - k0) & 3, j1 = (4 - k1) & 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = cadd(acc[c], uh[c]);
        acc[3 + c] = cadd(acc[3 + c], uh[3 + c]);
        const cx<T> l0 = mul_ipow_rt(uh[c], j0), l1 = mul_ipow_rt(uh[3 + c], j1);
        acc[6 + c] = cadd(acc[6 + c], p2 ? l0 : l1);
        acc[9 + c] = cadd(acc[9 + c], p2 ? l1 : l0);
    }
}

template <int P, int R>
__device__ void hop_site(const Lattice &lat, const void *g, size_t gb, int par, bool dag, const void *in, int i,
                         cx<RealOf<P>> acc[12]) {
    const SiteGeom geo = site_geom(lat, par, i);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {RealOf<P>(0), RealOf<P>(0)};
    if constexpr (P != PLQ_F64) {  // memory-bound phases: unrolled, loads hoisted across directions
        HopArgs a;
        a.in = in;
        a.gauge = g;
        a.gblock = gb;
        a.out_parity = par;
        a.nrhs = 1;
        a.lat = lat;
        if (dag) {
            hop_dir<P, R, 0, true, false>(a, geo, i, 0, acc);
            hop_dir<P, R, 1, true, false>(a, geo, i, 0, acc);
            hop_dir<P, R, 2, true, false>(a, geo, i, 0, acc);
            hop_dir<P, R, 3, true, false>(a, geo, i, 0, acc);
        } else {
            hop_dir<P, R, 0, false, false>(a, geo, i, 0, acc);
            hop_dir<P, R, 1, false, false>(a, geo, i, 0, acc);
            hop_dir<P, R, 2, false, false>(a, geo, i, 0, acc);
            hop_dir<P, R, 3, false, false>(a, geo, i, 0, acc);
        }
    } else {
        // FP64 phases (bound by the FP64 pipe): one run-time loop over the directions
#pragma unroll 1
        for (int d = 0; d < 8; ++d)
            hop_dir_rt<P, R>(lat, static_cast<const char *>(g), gb, par, dag, in, geo, i, d, acc);
    }
}

template <class T>
__device__ __forceinline__ T norm12(const cx<T> v[12]) {
    T s = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) s += v[k].re * v[k].re + v[k].im * v[k].im;
    return s;
}

// One site of the phase `mode` of system B; returns its contribution to the
// phase's reduction (0 when the phase reduces nothing).
template <int PL, int RL>
__device__ double run_site(int mode, const BatchSystem &B, const SysRun &R, int i) {
    using T = RealOf<PL>;
    constexpr int PX = PL == PLQ_F64 ? PLQ_F64 : PLQ_F32;
    const int Vh = B.lat.Vh;
    const double kk = B.kappa * B.kappa;
    switch (mode) {
    case M_SETUP0: {
        cx<double> u[12], v[12];
        ld<PLQ_F64>(B.be, Vh, i, u);
        ld<PLQ_F64>(B.bo, Vh, i, v);
        if (!B.use_x0) {
            cx<double> z[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) z[k] = {0.0, 0.0};
            st<PLQ_F64>(B.xe, Vh, i, z);
        }
        return norm12(u) + norm12(v);
    }
    case M_SETUP1: {
        cx<double> acc[12], b[12];
        hop_site<PLQ_F64, 18>(B.lat, B.g64, B.gb64, 0, false, B.bo, i, acc);
        ld<PLQ_F64>(B.be, Vh, i, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {fma(B.kappa, acc[k].re, b[k].re), fma(B.kappa, acc[k].im, b[k].im)};
        st<PLQ_F64>(B.bhat, Vh, i, acc);
        return 0.0;
    }
    case M_RES1:
    case M_FIN1: {
        cx<double> acc[12];
        hop_site<PLQ_F64, 18>(B.lat, B.g64, B.gb64, 1, false, B.xe, i, acc);
        if (mode == M_FIN1) {
            cx<double> b[12];
            ld<PLQ_F64>(B.bo, Vh, i, b);
#pragma unroll
            for (int k = 0; k < 12; ++k)
                acc[k] = {fma(B.kappa, acc[k].re, b[k].re), fma(B.kappa, acc[k].im, b[k].im)};
            st<PLQ_F64>(B.xo, Vh, i, acc);
        } else {
            st<PLQ_F64>(B.to64, Vh, i, acc);
        }
        return 0.0;
    }
    case M_RES2: {
        cx<double> acc[12], bh[12], x[12];
        hop_site<PLQ_F64, 18>(B.lat, B.g64, B.gb64, 0, false, B.to64, i, acc);
        ld<PLQ_F64>(B.bhat, Vh, i, bh);
        ld<PLQ_F64>(B.xe, Vh, i, x);
        cx<T> sl[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            acc[k] = {fma(kk, acc[k].re, bh[k].re - x[k].re), fma(kk, acc[k].im, bh[k].im - x[k].im)};
            sl[k] = {(T)(R.sc * acc[k].re), (T)(R.sc * acc[k].im)};
        }
        st<PLQ_F64>(B.s64, Vh, i, acc);
        st<PL>(B.mpL, Vh, i, sl);  // mpL is free until the inner iteration starts
        return norm12(acc);
    }
    // r = Mhat^dagger s, the residual of the normal equations, only restarts the
    // inner iteration: it is formed at the inner precision (s itself is FP64)
    case M_RES3: {
        cx<T> acc[12];
        hop_site<PL, RL>(B.lat, B.gL, B.gbL, 1, true, B.mpL, i, acc);
        st<PL>(B.toL, Vh, i, acc);
        return 0.0;
    }
    case M_RES4: {
        cx<T> acc[12], sl[12];
        hop_site<PL, RL>(B.lat, B.gL, B.gbL, 0, true, B.toL, i, acc);
        ld<PL>(B.mpL, Vh, i, sl);
        const T a = (T)(-kk);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {fma(a, acc[k].re, sl[k].re), fma(a, acc[k].im, sl[k].im)};
        st<PL>(B.rL, Vh, i, acc);
        return (double)norm12(acc);
    }
    case M_RES5: {
        cx<T> rl[12], p[12];
        cx<RealOf<PX>> z[12];
        ld<PL>(B.rL, Vh, i, rl);
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = {0, 0};
        st<PX>(B.xL, Vh, i, z);
        if (R.first) {
            st<PL>(B.pL, Vh, i, rl);
        } else {
            ld<PL>(B.pL, Vh, i, p);
            const T beta = (T)R.beta;
#pragma unroll
            for (int k = 0; k < 12; ++k) p[k] = {fma(beta, p[k].re, rl[k].re), fma(beta, p[k].im, rl[k].im)};
            st<PL>(B.pL, Vh, i, p);
        }
        return 0.0;
    }
    case M_IT1:
    case M_IT3: {
        cx<T> acc[12];
        hop_site<PL, RL>(B.lat, B.gL, B.gbL, 1, mode == M_IT3, mode == M_IT1 ? B.pL : B.mpL, i, acc);
        st<PL>(B.toL, Vh, i, acc);
        return 0.0;
    }
    case M_IT2:
    case M_IT4: {
        cx<T> acc[12], x[12];
        hop_site<PL, RL>(B.lat, B.gL, B.gbL, 0, mode == M_IT4, B.toL, i, acc);
        ld<PL>(mode == M_IT2 ? B.pL : B.mpL, Vh, i, x);
        const T a = (T)(-kk);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {fma(a, acc[k].re, x[k].re), fma(a, acc[k].im, x[k].im)};
        st<PL>(mode == M_IT2 ? B.mpL : B.qL, Vh, i, acc);
        return mode == M_IT2 ? (double)norm12(acc) : 0.0;
    }
    case M_IT5: {
        cx<T> p[12], q[12], r[12];
        cx<RealOf<PX>> x[12];
        ld<PL>(B.pL, Vh, i, p);
        ld<PL>(B.qL, Vh, i, q);
        ld<PL>(B.rL, Vh, i, r);
        ld<PX>(B.xL, Vh, i, x);
        const T al = (T)R.alpha;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            x[k] = {fma((RealOf<PX>)al, (RealOf<PX>)p[k].re, x[k].re), fma((RealOf<PX>)al, (RealOf<PX>)p[k].im, x[k].im)};
            r[k] = {fma(-al, q[k].re, r[k].re), fma(-al, q[k].im, r[k].im)};
        }
        st<PX>(B.xL, Vh, i, x);
        st<PL>(B.rL, Vh, i, r);
        return (double)norm12(r);
    }
    case M_IT6: {
        cx<T> p[12], r[12];
        ld<PL>(B.pL, Vh, i, p);
        ld<PL>(B.rL, Vh, i, r);
        const T be = (T)R.beta;
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k] = {fma(be, p[k].re, r[k].re), fma(be, p[k].im, r[k].im)};
        st<PL>(B.pL, Vh, i, p);
        return 0.0;
    }
    case M_ACC: {
        cx<double> x[12];
        cx<RealOf<PX>> xl[12];
        ld<PLQ_F64>(B.xe, Vh, i, x);
        ld<PX>(B.xL, Vh, i, xl);
        const double isc = 1.0 / R.sc;  // exact: R.sc is a power of two
#pragma unroll
        for (int k = 0; k < 12; ++k)
            x[k] = {fma(isc, (double)xl[k].re, x[k].re), fma(isc, (double)xl[k].im, x[k].im)};
        st<PLQ_F64>(B.xe, Vh, i, x);
        return 0.0;
    }
    case M_ZERO: {
        cx<double> z[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = {0.0, 0.0};
        st<PLQ_F64>(B.xo, Vh, i, z);
        st<PLQ_F64>(B.xe, Vh, i, z);
        return 0.0;
    }
    default:
        return 0.0;
    }
}

__device__ __forceinline__ bool reduces(int mode) {
    return mode == M_SETUP0 || mode == M_RES2 || mode == M_RES4 || mode == M_IT2 || mode == M_IT5;
}

// Deterministic state update after a phase, applied identically by every
// block from the reduced total `v`.
__device__ void advance(SysRun &R, const BatchSystem &B, double v) {
    switch (R.mode) {
    case M_SETUP0:
        R.b2 = v;
        if (!isfinite(v)) { R.flags |= BF_NAN; R.mode = M_DONE; }
        else R.mode = (v == 0.0) ? M_ZERO : M_SETUP1;
        // inner quantities carry 2^-(exponent of |b|), so that sources of any
        // magnitude sit in the inner precision's exponent range
        if (isfinite(v) && v > 0.0 && B.inner_scaled) R.sc = ldexp(1.0, -ilogb(sqrt(v)));
        break;
    case M_SETUP1: R.mode = M_RES1; break;
    case M_RES1: R.mode = M_RES2; break;
    case M_RES2:
        R.s2 = v;
        if (!isfinite(v)) { R.flags |= BF_NAN; R.mode = M_FIN1; }
        else if (v <= B.tol * B.tol * R.b2) R.mode = M_FIN1;
        else if (R.iter >= B.maxit) { R.flags |= BF_NOT_CONVERGED; R.mode = M_FIN1; }
        else R.mode = M_RES3;
        break;
    case M_RES3: R.mode = M_RES4; break;
    case M_RES4: {
        R.r2 = v;
        const double ratio = sqrt(v / R.s2);
        const double t = R.sigma * ratio * B.tol * sqrt(R.b2);
        R.target2 = t * t;
        R.stop_r2 = fmax(B.delta * B.delta * v, R.target2);
        R.beta = R.first ? 0.0 : v / R.last_rho;
        R.rho = v;
        R.mode = M_RES5;
        break;
    }
    case M_RES5: R.first = 0; R.mode = M_IT1; break;
    case M_IT1: R.mode = M_IT2; break;
    case M_IT2:
        R.alpha = R.rho / v;
        if (!isfinite(R.alpha)) { R.flags |= BF_NAN; R.mode = M_FIN1; }
        else R.mode = M_IT3;
        break;
    case M_IT3: R.mode = M_IT4; break;
    case M_IT4: R.mode = M_IT5; break;
    case M_IT5: {
        const double rho_old = R.rho;
        R.beta = v / rho_old;
        R.rho = v;
        R.iter += 1;
        if (!isfinite(v)) { R.flags |= BF_NAN; R.mode = M_FIN1; break; }
        if (v <= R.stop_r2 || R.iter >= B.maxit) {
            R.last_rho = rho_old;  // |r|^2 of the iteration before the trigger
            if (v <= R.target2 * 1.0000001) R.sigma *= 0.25;
            R.mode = M_ACC;
        } else {
            R.mode = M_IT6;
        }
        break;
    }
    case M_IT6: R.mode = M_IT1; break;
    case M_ACC: R.nrel += 1; R.mode = M_RES1; break;
    case M_FIN1: R.mode = M_DONE; break;
    case M_ZERO: R.mode = M_DONE; break;
    default: break;
    }
}

// 4 blocks of 128 threads per SM (<= 128 registers): measured on the 16-solve
// batch, 0.117 s against 0.18 s with 2 blocks and 0.14 s with 3
template <int PL, int RL>
__global__ void __launch_bounds__(128, 4) batched_cg_kernel(BatchArgs a) {
    __shared__ SysRun run[kMaxSys];
    __shared__ long long prefix[kMaxSys + 1];
    __shared__ double bsum[kMaxSys];
    const int ns = a.nsys;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        SysRun R;
        R.mode = M_SETUP0;
        R.iter = R.nrel = R.flags = R.reduces = 0;
        R.first = 1;
        R.b2 = R.s2 = R.r2 = R.rho = R.alpha = R.beta = R.last_rho = R.stop_r2 = R.target2 = 0.0;
        R.sigma = 0.5;
        R.sc = 1.0;
        run[s] = R;
    }
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long phase = 0; phase < a.max_phases; ++phase) {
        double *acc_now = a.acc + (phase % 3) * kMaxSys;
        double *acc_next = a.acc + ((phase + 1) % 3) * kMaxSys;
        // work ranges of the active systems
        if (threadIdx.x == 0) {
            long long off = 0;
            for (int s = 0; s < ns; ++s) {
                prefix[s] = off;
                if (run[s].mode != M_DONE) off += a.sys[s].lat.Vh;
            }
            prefix[ns] = off;
        }
        for (int s = threadIdx.x; s < ns; s += blockDim.x) bsum[s] = 0.0;
        if (blockIdx.x == 0)
            for (int s = threadIdx.x; s < kMaxSys; s += blockDim.x) acc_next[s] = 0.0;
        __syncthreads();
        const long long total = prefix[ns];
        if (total == 0) break;  // every system retired
        for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += stride) {
            int s = 0;
            while (g >= prefix[s + 1]) ++s;
            const int i = (int)(g - prefix[s]);
            const double v = run_site<PL, RL>(run[s].mode, a.sys[s], run[s], i);
            if (reduces(run[s].mode)) {
                // warp-level sum when the whole warp works on one system
                const unsigned m = __activemask();
                const int s0 = __shfl_sync(m, s, __ffs(m) - 1);
                if (__all_sync(m, s == s0) && m == 0xffffffffu) {
                    double w = v;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(m, w, o);
                    if ((threadIdx.x & 31) == 0) atomicAdd(&bsum[s], w);
                } else {
                    atomicAdd(&bsum[s], v);
                }
            }
        }
        __syncthreads();
        for (int s = threadIdx.x; s < ns; s += blockDim.x)
            if (run[s].mode != M_DONE && reduces(run[s].mode) && bsum[s] != 0.0) atomicAdd(&acc_now[s], bsum[s]);
        if (!grid_sync(a)) return;
        // identical state update in every block
        for (int s = threadIdx.x; s < ns; s += blockDim.x) {
            if (run[s].mode == M_DONE) continue;
            const double v = reduces(run[s].mode) ? __ldcg(&acc_now[s]) : 0.0;
            advance(run[s], a.sys[s], v);
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        for (int s = threadIdx.x; s < ns; s += blockDim.x) {
            BatchResult r;
            r.iterations = run[s].iter;
            r.n_reliable = run[s].nrel;
            r.flags = run[s].flags;
            r.done = run[s].mode == M_DONE;
            r.true_rel_schur = run[s].b2 > 0 ? sqrt(run[s].s2 / run[s].b2) : 0.0;
            a.res[s] = r;
        }
    }
}

template <int PL, int RL>
plq_status launch_batched(const BatchArgs &args, cudaStream_t s, int *grid_out, int *block_out, bool *captured) {
    auto kern = batched_cg_kernel<PL, RL>;
    const int block = 128;
    int nb = 0, dev = 0, sms = 0;
    PLQ_CUDA(cudaGetDevice(&dev));
    PLQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PLQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, block, 0));
    if (nb < 1) return set_error(PLQ_ERR_CUDA, "batched CG kernel does not fit on an SM");
    const int grid = nb * sms;  // every block co-resident: required by the grid barrier
    *grid_out = grid;
    *block_out = block;
    BatchArgs a = args;
    void *params[] = {&a};
    // one cooperative launch, captured in a CUDA graph when the runtime allows it
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    *captured = false;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        cudaError_t e = cudaLaunchCooperativeKernel((void *)kern, dim3(grid), dim3(block), params, 0, s);
        cudaError_t e2 = cudaStreamEndCapture(s, &graph);
        if (e == cudaSuccess && e2 == cudaSuccess && graph &&
            cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
            *captured = true;
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();  // clear a refused capture; the direct launch below reports real errors
    }
    if (*captured) {
        cudaError_t e = cudaGraphLaunch(exec, s);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch(batched CG)");
    } else {
        PLQ_CUDA(cudaLaunchCooperativeKernel((void *)kern, dim3(grid), dim3(block), params, 0, s));
    }
    return PLQ_OK;
}

}  // namespace

}  // namespace plq

using namespace plq;

extern "C" plq_status plq_cg_solve_batched(plq_ctx **ctxs, int n, void **x, const void **b, const double *kappa,
                                           const plq_solver_params *params, plq_solve_info *infos,
                                           plq_batch_info *binfo, void *stream) {
    if (infos && n > 0 && n <= kMaxSys) std::memset(infos, 0, sizeof(plq_solve_info) * n);
    if (binfo) std::memset(binfo, 0, sizeof(*binfo));
    if (!ctxs || !x || !b || !kappa) return set_error(PLQ_ERR_ARG, "null argument");
    if (n < 1 || n > kMaxSys) return set_error(PLQ_ERR_ARG, "n must be in 1..%d", kMaxSys);
    const double tol = (params && params->tol > 0) ? params->tol : 1e-10;
    const int maxit = (params && params->maxit > 0) ? params->maxit : 20000;
    const int inner = params ? params->inner_prec : PLQ_F64;
    const double delta = inner == PLQ_F64 ? 0.0
                                           : ((params && params->delta > 0) ? params->delta
                                                                            : (inner == PLQ_F16 ? 1e-2 : 1e-3));
    const int use_x0 = params ? params->use_x0 : 0;
    if (!valid_prec(inner)) return set_error(PLQ_ERR_ARG, "bad inner precision %d", inner);
    const int device = ctxs[0] ? ctxs[0]->device : -1;
    int reals = 0;
    for (int k = 0; k < n; ++k) {
        plq_ctx *c = ctxs[k];
        if (!c) return set_error(PLQ_ERR_ARG, "null context %d", k);
        if (c->device != device) return set_error(PLQ_ERR_ARG, "all systems must be on one device");
        if (!x[k] || !b[k] || (reinterpret_cast<uintptr_t>(x[k]) & 15) || (reinterpret_cast<uintptr_t>(b[k]) & 15))
            return set_error(PLQ_ERR_ARG, "null or misaligned field of system %d", k);
        if (!std::isfinite(kappa[k])) return set_error(PLQ_ERR_ARG, "kappa of system %d not finite", k);
        if (!c->gauge[PLQ_F64].ptr || c->gauge[PLQ_F64].reals != 18)
            return set_error(PLQ_ERR_STATE, "system %d: the batched solver needs an 18-real FP64 gauge copy", k);
        if (!c->gauge[inner].ptr) return set_error(PLQ_ERR_STATE, "system %d: no gauge copy for inner precision", k);
        if (k == 0) reals = c->gauge[inner].reals;
        else if (c->gauge[inner].reals != reals)
            return set_error(PLQ_ERR_ARG, "all systems need the same inner link format");
    }
    if (inner == PLQ_F64 && reals != 18) return set_error(PLQ_ERR_ARG, "FP64 inner solves need 18-real links");
    PLQ_CUDA(cudaSetDevice(device));

    // per-system workspace in each context
    const int PX = inner == PLQ_F64 ? PLQ_F64 : PLQ_F32;
    std::vector<BatchSystem> sys(n);
    for (int k = 0; k < n; ++k) {
        plq_ctx *c = ctxs[k];
        const size_t Vh = c->lat.Vh;
        const size_t h64 = spinor_site_bytes(PLQ_F64) * Vh, hL = spinor_site_bytes(inner) * Vh,
                     hX = spinor_site_bytes(PX) * Vh;
        PLQ_TRY(ensure_work(c, 3 * h64 + 5 * hL + hX + 4096));
        char *w = static_cast<char *>(c->work);
        BatchSystem &B = sys[k];
        B.lat = c->lat;
        B.kappa = kappa[k];
        B.tol = tol;
        B.delta = delta;
        B.maxit = maxit;
        B.use_x0 = use_x0;
        B.g64 = c->gauge[PLQ_F64].ptr;
        B.gb64 = c->gauge[PLQ_F64].block;
        B.gL = c->gauge[inner].ptr;
        B.gbL = c->gauge[inner].block;
        B.inner_scaled = inner != PLQ_F64;
        B.be = b[k];
        B.bo = static_cast<const char *>(b[k]) + h64;
        B.xe = x[k];
        B.xo = static_cast<char *>(x[k]) + h64;
        B.bhat = w;
        B.s64 = w + h64;
        B.to64 = w + 2 * h64;
        char *wl = w + 3 * h64;
        B.rL = wl;
        B.pL = wl + hL;
        B.qL = wl + 2 * hL;
        B.mpL = wl + 3 * hL;
        B.toL = wl + 4 * hL;
        B.xL = wl + 5 * hL;
    }
    // small batch scratch: descriptors, results, accumulators, barrier words
    const size_t bytes_sys = sizeof(BatchSystem) * n, bytes_res = sizeof(BatchResult) * n;
    const size_t bytes = bytes_sys + bytes_res + sizeof(double) * 3 * kMaxSys + 64;
    char *scratch = nullptr;
    PLQ_CUDA(cudaMalloc(&scratch, bytes));
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t s = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    plq_status stt = PLQ_OK;
    std::vector<BatchResult> res(n);
    int grid = 0, block = 0;
    bool captured = false;
    double secs = 0.0;
    do {
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&ev1);
        if (e == cudaSuccess) e = cudaEventRecord(ev0, user);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev0, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(scratch, sys.data(), bytes_sys, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(scratch + bytes_sys, 0, bytes - bytes_sys, s);
        if (e != cudaSuccess) {
            stt = cuda_error(e, "batched solver setup");
            break;
        }
        BatchArgs a;
        a.sys = reinterpret_cast<const BatchSystem *>(scratch);
        a.res = reinterpret_cast<BatchResult *>(scratch + bytes_sys);
        a.nsys = n;
        a.acc = reinterpret_cast<double *>(scratch + bytes_sys + bytes_res);
        char *words = scratch + bytes_sys + bytes_res + sizeof(double) * 3 * kMaxSys;
        a.bar_count = reinterpret_cast<unsigned *>(words);
        a.bar_gen = reinterpret_cast<unsigned *>(words + 16);
        a.status = reinterpret_cast<int *>(words + 32);
        {
            int khz = 0;  // SM clock in kHz (clock64 counts SM cycles)
            cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
            const double lim = (params && params->wait_limit_s > 0) ? params->wait_limit_s : 5.0;
            const double cyc = lim * (khz > 0 ? khz : 2000000) * 1e3;
            a.spin_limit = cyc < 1.0 ? 1LL : cyc > 1e15 ? (long long)1e15 : (long long)cyc;
        }
        a.max_phases = 16LL * (maxit + 64) + 4096;
        auto t0 = std::chrono::steady_clock::now();
        if (inner == PLQ_F64) stt = launch_batched<PLQ_F64, 18>(a, s, &grid, &block, &captured);
        else if (inner == PLQ_F32 && reals == 18) stt = launch_batched<PLQ_F32, 18>(a, s, &grid, &block, &captured);
        else if (inner == PLQ_F32) stt = launch_batched<PLQ_F32, 12>(a, s, &grid, &block, &captured);
        else stt = launch_batched<PLQ_F16, 12>(a, s, &grid, &block, &captured);
        if (stt != PLQ_OK) break;
        if (inner == PLQ_F16 && reals != 12) {
            stt = set_error(PLQ_ERR_ARG, "FP16 inner solves use 12-real links");
            break;
        }
        int status_word = 0;
        e = cudaMemcpyAsync(res.data(), a.res, bytes_res, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&status_word, a.status, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (e != cudaSuccess) {
            stt = cuda_error(e, "batched CG kernel");
            break;
        }
        if (status_word != 0) {
            stt = set_error(PLQ_ERR_TIMEOUT, "batched CG: a grid barrier exceeded its wait limit");
            break;
        }
    } while (0);
    // true residual of every system with the FP64 operator (independent of the kernel's bookkeeping)
    int status = stt;
    for (int k = 0; k < n && stt == PLQ_OK; ++k) {
        double r2 = 0, b2 = 0;
        plq_status e = wilson_residual64(ctxs[k], kappa[k], x[k], b[k], &r2, &b2, s);
        if (e != PLQ_OK) {
            status = e;
            break;
        }
        const double rel = b2 > 0 ? std::sqrt(r2 / b2) : 0.0;
        int st_k = PLQ_OK;
        if (res[k].flags & BF_NAN) st_k = PLQ_ERR_NAN;
        else if ((res[k].flags & BF_NOT_CONVERGED) || !res[k].done || !(rel <= tol)) st_k = PLQ_ERR_NOT_CONVERGED;
        if (infos) {
            infos[k].status = st_k;
            infos[k].iterations = res[k].iterations;
            infos[k].n_reliable = res[k].n_reliable;
            infos[k].true_rel_residual = rel;
            infos[k].seconds = secs;
            infos[k].hop_applications = 4.0 * res[k].iterations + 4.0 * (res[k].n_reliable + 1) + 2;
        }
        if (st_k != PLQ_OK && status == PLQ_OK)
            status = set_error(st_k, "system %d: %s (residual %.3e after %d iterations)", k,
                               st_k == PLQ_ERR_NAN ? "NaN" : "not converged", rel, res[k].iterations);
    }
    if (binfo) {
        binfo->grid = grid;
        binfo->block = block;
        binfo->graph_captured = captured ? 1 : 0;
        binfo->seconds = secs;
        binfo->launches = (stt == PLQ_OK) ? 1 : 0;
    }
    if (s) {
        cudaEventRecord(ev1, s);
        cudaStreamWaitEvent(user, ev1, 0);
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaFree(scratch);
    return status;
}
