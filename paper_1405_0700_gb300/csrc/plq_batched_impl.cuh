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
//
// This header holds the kernel and its launcher; each inner precision and link
// format is instantiated in its own translation unit (plq_batched_*.cu) and
// the host entry points live in plq_batched.cu.
#pragma once

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "plq_hop_impl.cuh"

namespace plq {
namespace batch {

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
    M_RES0,        // x_e = 0: s = bhat, |s|^2 (no operator; s also kept as sL)
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
    M_FIN1,        // x_o = b_o + kappa H_oe x_e (H_oe x_e of the last check, kept in to)
    M_ZERO,        // zero source: x_o = 0
    M_DONE
};

enum { BF_NAN = 1, BF_NOT_CONVERGED = 2 };

struct SysRun {
    int mode, iter, nrel, first, flags, reduces;
    int toe;    // to64 holds H_oe x_e of the current x_e
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
__device__ inline bool grid_sync(const BatchArgs &a) {
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
    case M_RES0: {  // M_RES1/M_RES2 at x_e = 0 give s = bhat exactly
        cx<double> bh[12];
        cx<T> sl[12];
        ld<PLQ_F64>(B.bhat, Vh, i, bh);
#pragma unroll
        for (int k = 0; k < 12; ++k) sl[k] = {(T)(R.sc * bh[k].re), (T)(R.sc * bh[k].im)};
        st<PLQ_F64>(B.s64, Vh, i, bh);
        st<PL>(B.mpL, Vh, i, sl);  // mpL is free until the inner iteration starts
        return norm12(bh);
    }
    case M_RES1: {
        cx<double> acc[12];
        hop_site<PLQ_F64, 18>(B.lat, B.g64, B.gb64, 1, false, B.xe, i, acc);
        st<PLQ_F64>(B.to64, Vh, i, acc);
        return 0.0;
    }
    case M_FIN1: {
        // H_oe x_e of the final x_e was stored by its residual check (M_RES1),
        // so x_o takes the same FP64 values without a second application; after
        // a check at x_e = 0 (M_RES0) it is zero
        cx<double> acc[12], b[12];
        if (R.toe) {
            ld<PLQ_F64>(B.to64, Vh, i, acc);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = {0.0, 0.0};
        }
        ld<PLQ_F64>(B.bo, Vh, i, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {fma(B.kappa, acc[k].re, b[k].re), fma(B.kappa, acc[k].im, b[k].im)};
        st<PLQ_F64>(B.xo, Vh, i, acc);
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
    return mode == M_SETUP0 || mode == M_RES0 || mode == M_RES2 || mode == M_RES4 || mode == M_IT2 ||
           mode == M_IT5;
}

// Deterministic state update after a phase, applied identically by every
// block from the reduced total `v`.
__device__ inline void advance(SysRun &R, const BatchSystem &B, double v) {
    switch (R.mode) {
    case M_SETUP0:
        R.b2 = v;
        if (!isfinite(v)) { R.flags |= BF_NAN; R.mode = M_DONE; }
        else R.mode = (v == 0.0) ? M_ZERO : M_SETUP1;
        // inner quantities carry 2^-(exponent of |b|), so that sources of any
        // magnitude sit in the inner precision's exponent range
        if (isfinite(v) && v > 0.0 && B.inner_scaled) R.sc = ldexp(1.0, -ilogb(sqrt(v)));
        break;
    case M_SETUP1: R.mode = B.use_x0 ? M_RES1 : M_RES0; break;
    case M_RES1:
        R.toe = 1;
        R.mode = M_RES2;
        break;
    case M_RES0:
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

// BLOCK threads per block with the register budget of MINB resident blocks
// per SM: 512 threads per SM at <= 128 registers for blocks of 64, 128 and
// 256 threads, 384 threads at <= 168 registers (fewer spills) for blocks of
// 192; the tuner picks among them and among the number of blocks launched.
template <int PL, int RL, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) batched_cg_kernel(BatchArgs a) {
    __shared__ SysRun run[kMaxSys];
    __shared__ long long prefix[kMaxSys + 1];
    __shared__ double bsum[kMaxSys];
    const int ns = a.nsys;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        SysRun R;
        R.mode = M_SETUP0;
        R.iter = R.nrel = R.flags = R.reduces = R.toe = 0;
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
            s = PLQ_GUARD(a.status, s, ns);
            const int i = PLQ_GUARD(a.status, (int)(g - prefix[s]), a.sys[s].lat.Vh);
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


// Launch shapes of the persistent kernel the tuner chooses from (threads per
// block, blocks per SM its register budget is set for).
struct Shape {
    int block, minb;
};
constexpr Shape kShapes[] = {{128, 4}, {64, 8}, {256, 2}, {192, 2}};
constexpr int kNumShapes = 4;

struct LaunchOut {
    int grid = 0, block = 0, bps = 0;
    bool captured = false, reused = false;
};

// One cooperative launch of the persistent kernel with shape (BLOCK, MINB)
// and bps resident blocks per SM (<= 0 or above what fits: all that fit),
// captured in a CUDA graph.  The instantiated graph is kept in `cache` and
// replayed by the next call whose key matches: the kernel's arguments point
// into the cache's persistent descriptor scratch, which every call rewrites
// before the launch, so a replay solves the new systems.
template <int PL, int RL, int BLOCK, int MINB>
plq_status launch_shape(const BatchArgs &args, int shape, int bps_req, cudaStream_t s, Ctx::BatchCache &cache,
                        LaunchOut *out) {
    auto kern = batched_cg_kernel<PL, RL, BLOCK, MINB>;
    int nb = 0, dev = 0, sms = 0;
    PLQ_CUDA(cudaGetDevice(&dev));
    PLQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PLQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BLOCK, 0));
    if (nb < 1) return set_error(PLQ_ERR_CUDA, "batched CG kernel does not fit on an SM");
    const int bps = (bps_req > 0 && bps_req < nb) ? bps_req : nb;
    const int grid = bps * sms;  // every block co-resident: required by the grid barrier
    out->grid = grid;
    out->block = BLOCK;
    out->bps = bps;
    BatchArgs a = args;
    const unsigned long long key[6] = {
        (unsigned long long)shape | ((unsigned long long)PL << 8) | ((unsigned long long)RL << 16) | (1ull << 40),
        (unsigned long long)grid, (unsigned long long)reinterpret_cast<uintptr_t>(args.sys),
        (unsigned long long)args.nsys, (unsigned long long)args.spin_limit, (unsigned long long)args.max_phases};
    static_assert(sizeof(key) == sizeof(cache.key), "graph key size");
    if (cache.exec && std::memcmp(cache.key, key, sizeof(key)) == 0) {
        out->captured = out->reused = true;
        const cudaError_t e = cudaGraphLaunch(cache.exec, s);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch(batched CG)");
        return PLQ_OK;
    }
    if (cache.exec) {
        cudaGraphExecDestroy(cache.exec);
        cache.exec = nullptr;
    }
    void *params[] = {&a};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const cudaError_t e = cudaLaunchCooperativeKernel((void *)kern, dim3(grid), dim3(BLOCK), params, 0, s);
        const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
        if (e == cudaSuccess && e2 == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
            out->captured = true;
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();  // clear a refused capture; the direct launch below reports real errors
    }
    if (out->captured) {
        const cudaError_t e = cudaGraphLaunch(exec, s);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            return cuda_error(e, "cudaGraphLaunch(batched CG)");
        }
        cache.exec = exec;
        std::memcpy(cache.key, key, sizeof(key));
    } else {
        PLQ_CUDA(cudaLaunchCooperativeKernel((void *)kern, dim3(grid), dim3(BLOCK), params, 0, s));
    }
    return PLQ_OK;
}

template <int PL, int RL>
plq_status launch_batched(const BatchArgs &args, int shape, int bps, cudaStream_t s, Ctx::BatchCache &cache,
                          LaunchOut *out) {
    switch (shape) {
    case 1: return launch_shape<PL, RL, kShapes[1].block, kShapes[1].minb>(args, 1, bps, s, cache, out);
    case 2: return launch_shape<PL, RL, kShapes[2].block, kShapes[2].minb>(args, 2, bps, s, cache, out);
    case 3: return launch_shape<PL, RL, kShapes[3].block, kShapes[3].minb>(args, 3, bps, s, cache, out);
    default: return launch_shape<PL, RL, kShapes[0].block, kShapes[0].minb>(args, 0, bps, s, cache, out);
    }
}

// One translation unit per inner precision and link format.
plq_status launch_f64_18(const BatchArgs &a, int shape, int bps, cudaStream_t s, Ctx::BatchCache &c, LaunchOut *o);
plq_status launch_f32_18(const BatchArgs &a, int shape, int bps, cudaStream_t s, Ctx::BatchCache &c, LaunchOut *o);
plq_status launch_f32_12(const BatchArgs &a, int shape, int bps, cudaStream_t s, Ctx::BatchCache &c, LaunchOut *o);
plq_status launch_f16_12(const BatchArgs &a, int shape, int bps, cudaStream_t s, Ctx::BatchCache &c, LaunchOut *o);

}  // namespace batch
}  // namespace plq
