// Site-fused hopping kernel (Eq. (1) through the half spinors of Eq. (2)).
//
// One thread computes one output site (and one right-hand side).  For each of
// the 8 neighbours y = x +- mu it
//   1. loads phi(y) and projects it to the upper two spin components h of
//      (1 -/+ gamma_mu) phi(y)  (the half-spinor remark after Eq. (2)),
//   2. applies the time boundary sign if the hop crosses t = T-1 <-> 0,
//   3. multiplies h by U_mu(x) (forward) or U_mu(x - mu)^dagger (backward),
//   4. accumulates U h into the upper spin components and the fixed
//      +-1 / +-i recombination of it into the lower ones.
// The gather form computes U_mu(x - mu)^dagger (1 + gamma_mu) phi(x - mu) at
// the destination, which equals theta-_mu(x - mu) of Eq. (2).
//
// Projection table.  With gamma_mu = [[0, A], [A^dagger, 0]] (chiral basis),
// the upper part of (1 - gamma_mu) phi is h_k = phi_k + c_k phi_{p_k}
// (k = 0, 1) and its lower part is phi_{p_k} component = conj(c_k) h_k:
//   mu = 0: p = (2, 3), c = (+1, +1)
//   mu = 1: p = (3, 2), c = (+i, +i)
//   mu = 2: p = (3, 2), c = (+1, -1)
//   mu = 3: p = (2, 3), c = (+i, -i)
// (1 + gamma_mu) flips the sign of c.  c is stored as a power of i.
#pragma once

#include <atomic>

#include "plq_fields.cuh"

namespace plq {

// v = scale * (1 + i nu gamma5) v with gamma5 = diag(1, 1, -1, -1) in spin
template <class T>
__device__ __forceinline__ void twist12(cx<T> v[12], T nu, T scale) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const T g = k < 6 ? nu : -nu;
        v[k] = {scale * (v[k].re - g * v[k].im), scale * (v[k].im + g * v[k].re)};
    }
}

template <int MU>
struct Proj;
template <>
struct Proj<0> {
    static constexpr int p0 = 2, p1 = 3, k0 = 0, k1 = 0;
};
template <>
struct Proj<1> {
    static constexpr int p0 = 3, p1 = 2, k0 = 1, k1 = 1;
};
template <>
struct Proj<2> {
    static constexpr int p0 = 3, p1 = 2, k0 = 0, k1 = 2;
};
template <>
struct Proj<3> {
    static constexpr int p0 = 2, p1 = 3, k0 = 1, k1 = 3;
};

// Upper two spin components of (1 + S*gamma_mu) phi, S = -1 or +1.
template <int MU, int S, class T>
__device__ __forceinline__ void project(const cx<T> phi[12], cx<T> h[6]) {
    using Q = Proj<MU>;
    constexpr int k0 = Q::k0 + (S > 0 ? 2 : 0), k1 = Q::k1 + (S > 0 ? 2 : 0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        h[c] = cadd(phi[c], mul_ipow<k0>(phi[3 * Q::p0 + c]));
        h[3 + c] = cadd(phi[3 + c], mul_ipow<k1>(phi[3 * Q::p1 + c]));
    }
}

// acc += full spinor rebuilt from the colour-rotated upper components uh.
template <int MU, int S, class T>
__device__ __forceinline__ void reconstruct(cx<T> acc[12], const cx<T> uh[6]) {
    using Q = Proj<MU>;
    constexpr int k0 = Q::k0 + (S > 0 ? 2 : 0), k1 = Q::k1 + (S > 0 ? 2 : 0);
    // conj(i^k) = i^(4-k)
    constexpr int j0 = (4 - (k0 & 3)) & 3, j1 = (4 - (k1 & 3)) & 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = cadd(acc[c], uh[c]);
        acc[3 + c] = cadd(acc[3 + c], uh[3 + c]);
        acc[3 * Q::p0 + c] = cadd(acc[3 * Q::p0 + c], mul_ipow<j0>(uh[c]));
        acc[3 * Q::p1 + c] = cadd(acc[3 * Q::p1 + c], mul_ipow<j1>(uh[3 + c]));
    }
}

// uh = U h (two spin components)
template <class T>
__device__ __forceinline__ void su3_mul(const cx<T> u[3][3], const cx<T> h[6], cx<T> uh[6]) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<T> z{0, 0};
#pragma unroll
            for (int b = 0; b < 3; ++b) z = cfma(u[a][b], h[3 * s + b], z);
            uh[3 * s + a] = z;
        }
}

// uh = U^dagger h
template <class T>
__device__ __forceinline__ void su3_dag_mul(const cx<T> u[3][3], const cx<T> h[6], cx<T> uh[6]) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<T> z{0, 0};
#pragma unroll
            for (int b = 0; b < 3; ++b) z = cfma_conj(u[b][a], h[3 * s + b], z);
            uh[3 * s + a] = z;
        }
}

// ---------------------------------------------------------------- packed FP32
// sm_100 and later issue two FP32 additions, multiplications or FMAs per
// instruction on a register pair (__fadd2_rn, __fmul2_rn, __ffma2_rn).  A
// complex number {re, im} is such a pair: the pair form of the projection,
// SU(3) product and reconstruction below is used where it measured faster
// (see packed_pairs()).
__device__ __forceinline__ float2 f2of(cx<float> z) { return make_float2(z.re, z.im); }
__device__ __forceinline__ cx<float> cxof(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// a + i^K b on pairs: K even in one packed instruction, K odd in two scalar ones
template <int K>
__device__ __forceinline__ float2 add_ipow2(float2 a, float2 b) {
    if constexpr ((K & 3) == 0) return add2(a, b);
    else if constexpr ((K & 3) == 2) return fma2(b, make_float2(-1.f, -1.f), a);
    else if constexpr ((K & 3) == 1) return make_float2(a.x - b.y, a.y + b.x);
    else return make_float2(a.x + b.y, a.y - b.x);
}

// Upper two spin components of (1 + S gamma_mu) phi as pairs.
template <int MU, int S>
__device__ __forceinline__ void project2(const cx<float> phi[12], float2 h[6]) {
    using Q = Proj<MU>;
    constexpr int k0 = Q::k0 + (S > 0 ? 2 : 0), k1 = Q::k1 + (S > 0 ? 2 : 0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        h[c] = add_ipow2<k0>(f2of(phi[c]), f2of(phi[3 * Q::p0 + c]));
        h[3 + c] = add_ipow2<k1>(f2of(phi[3 + c]), f2of(phi[3 * Q::p1 + c]));
    }
}

// acc += the full spinor rebuilt from the colour-rotated upper components uh.
template <int MU, int S>
__device__ __forceinline__ void reconstruct2(cx<float> acc[12], const float2 uh[6]) {
    using Q = Proj<MU>;
    constexpr int k0 = Q::k0 + (S > 0 ? 2 : 0), k1 = Q::k1 + (S > 0 ? 2 : 0);
    constexpr int j0 = (4 - (k0 & 3)) & 3, j1 = (4 - (k1 & 3)) & 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = cxof(add2(f2of(acc[c]), uh[c]));
        acc[3 + c] = cxof(add2(f2of(acc[3 + c]), uh[3 + c]));
        acc[3 * Q::p0 + c] = cxof(add_ipow2<j0>(f2of(acc[3 * Q::p0 + c]), uh[c]));
        acc[3 * Q::p1 + c] = cxof(add_ipow2<j1>(f2of(acc[3 * Q::p1 + c]), uh[3 + c]));
    }
}

// uh = U h (BACK = false) or U^dagger h (BACK = true) for both spin components
// with the link's natural pairs u = {re, im} and broadcast spinor pairs:
// zA = sum_b {h.re, h.re} * u, zB = sum_b {h.im, h.im} * u; then
// U h = {zA.re - zB.im, zA.im + zB.re} and U^dagger h = {zA.re + zB.im, zB.re - zA.im}.
template <bool BACK>
__device__ __forceinline__ void su3_apply_pairs(const cx<float> u[3][3], const float2 h[6], float2 uh[6]) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        float2 hr[3], hi[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            hr[b] = make_float2(h[3 * s + b].x, h[3 * s + b].x);
            hi[b] = make_float2(h[3 * s + b].y, h[3 * s + b].y);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float2 zA = mul2(hr[0], f2of(BACK ? u[0][a] : u[a][0]));
            zA = fma2(hr[1], f2of(BACK ? u[1][a] : u[a][1]), zA);
            zA = fma2(hr[2], f2of(BACK ? u[2][a] : u[a][2]), zA);
            float2 zB = mul2(hi[0], f2of(BACK ? u[0][a] : u[a][0]));
            zB = fma2(hi[1], f2of(BACK ? u[1][a] : u[a][1]), zB);
            zB = fma2(hi[2], f2of(BACK ? u[2][a] : u[a][2]), zB);
            uh[3 * s + a] = BACK ? make_float2(zA.x + zB.y, zB.x - zA.y) : make_float2(zA.x - zB.y, zA.y + zB.x);
        }
    }
}

// a + i^K b on half2 complex numbers (K odd: the swapped pair times (-1, +1)
// or (+1, -1))
template <int K>
__device__ __forceinline__ __half2 hadd_ipow(__half2 a, __half2 b) {
    if constexpr ((K & 3) == 0) return __hadd2(a, b);
    else if constexpr ((K & 3) == 2) return __hsub2(a, b);
    else if constexpr ((K & 3) == 1) return __hfma2(__lowhigh2highlow(b), __floats2half2_rn(-1.f, 1.f), a);
    else return __hfma2(__lowhigh2highlow(b), __floats2half2_rn(1.f, -1.f), a);
}

// FP16 storage: load the neighbour's 12 stored (normalised) complex
// components, project them to the upper two spin components of
// (1 + S gamma_mu) phi in half2 arithmetic (the stored values lie in [-1, 1],
// their sums in [-2, 2]), and convert only the 6 projected ones; returns the
// site norm.
template <int MU, int S>
__device__ __forceinline__ float project_f16(const void *base, size_t stride, size_t e, float2 h[6]) {
    using Q = Proj<MU>;
    constexpr int k0 = Q::k0 + (S > 0 ? 2 : 0), k1 = Q::k1 + (S > 0 ? 2 : 0);
    const uint4 *p = static_cast<const uint4 *>(base) + e;
    const float *nrm = reinterpret_cast<const float *>(static_cast<const uint4 *>(base) + 3 * stride);
    unsigned w[12];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint4 t = ld_nc(p + k * stride);
        w[4 * k] = t.x;
        w[4 * k + 1] = t.y;
        w[4 * k + 2] = t.z;
        w[4 * k + 3] = t.w;
    }
    const float n = ld_nc(nrm + e);
    auto hv = [&](int c) { return *reinterpret_cast<const __half2 *>(&w[c]); };
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        h[c] = __half22float2(hadd_ipow<k0>(hv(c), hv(3 * Q::p0 + c)));
        h[3 + c] = __half22float2(hadd_ipow<k1>(hv(3 + c), hv(3 * Q::p1 + c)));
    }
    return n;
}

__device__ __forceinline__ int lex_stride(const Lattice &L, int mu) {
    // strides of t, x, y, z in the lexicographic index
    return mu == 0 ? L.L[1] * L.L[2] * L.L[3] : mu == 1 ? 1 : mu == 2 ? L.L[1] : L.L[1] * L.L[2];
}

// Neighbour spinor for the projection: FP16 storage returns the normalised
// components and the site norm (applied to the 6 projected components, not
// the 12 loaded ones); the other formats return scale 1.
template <int P>
__device__ __forceinline__ RealOf<P> load_for_projection(const void *base, size_t stride, size_t e,
                                                        cx<RealOf<P>> phi[12]) {
    if constexpr (P == PLQ_F16) {
        return Spinor<PLQ_F16>::load_unscaled(base, stride, e, phi);
    } else {
        Spinor<P>::load(base, stride, e, phi);
        return RealOf<P>(1);
    }
}

// Which single-right-hand-side formats use the packed pair arithmetic above:
// measured on the 32^3 x 64 half-application, it speeds up FP16 storage with
// 12-real links (80.2 -> 77.1 us; the kernel is bound by instruction issue)
// and slows down the others (FP32 18-real 121.6 -> 127.9 us, FP32 12-real
// 97.1 -> 98.6 us, FP16 18-real 76.7 -> 90.0 us), which keep the scalar form.
template <int P, int R>
constexpr bool packed_pairs() {
    return P == PLQ_F16 && R == 12;
}

// One neighbour's contribution: project phi(y) with (1 + S gamma_mu), apply
// the time-boundary sign and the FP16 site norm, multiply by U (BACK = false)
// or U^dagger (BACK = true), rebuild and accumulate.  Formats with
// packed_pairs() use the pair arithmetic (FP16 storage projects in half2
// first).
template <int P, int R, int MU, int S, bool BACK>
__device__ __forceinline__ void hop_one(const void *in, size_t stride, size_t e, bool flip,
                                        const cx<RealOf<P>> u[3][3], cx<RealOf<P>> acc[12]) {
    using T = RealOf<P>;
    if constexpr (!packed_pairs<P, R>()) {
        cx<T> phi[12], h[6], uh[6];
        T sc = load_for_projection<P>(in, stride, e, phi);
        project<MU, S>(phi, h);
        if (MU == 0 && flip) sc = -sc;
        if (P == PLQ_F16 || (MU == 0 && flip)) {
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = {sc * h[k].re, sc * h[k].im};
        }
        if constexpr (BACK) su3_dag_mul(u, h, uh);
        else su3_mul(u, h, uh);
        reconstruct<MU, S>(acc, uh);
    } else {
        float2 h[6], uh[6];
        float sc = 1.f;
        if constexpr (P == PLQ_F16) {
            sc = project_f16<MU, S>(in, stride, e, h);
        } else {
            cx<float> phi[12];
            Spinor<P>::load(in, stride, e, phi);
            project2<MU, S>(phi, h);
        }
        if (MU == 0 && flip) sc = -sc;
        if (P == PLQ_F16 || (MU == 0 && flip)) {
            const float2 sc2 = make_float2(sc, sc);
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = mul2(h[k], sc2);
        }
        su3_apply_pairs<BACK>(u, h, uh);
        reconstruct2<MU, S>(acc, uh);
    }
}

// Contribution of direction MU (forward and backward) to the accumulators of
// RT right-hand sides r0 .. r0+RT-1 of output site i.  Each link is loaded once
// and applied to all RT neighbour spinors.
// DAG: gamma5 H gamma5 = H^dagger, i.e. the projectors (1 -/+ gamma) swapped.
template <int P, int R, int MU, bool DAG, bool TBL, int RT>
__device__ __forceinline__ void hop_dir(const HopArgs &a, const SiteGeom &g, int i, int r0,
                                        cx<RealOf<P>> (&acc)[RT][12]) {
    using T = RealOf<P>;
    const Lattice &L = a.lat;
    const int n = a.nrhs;
    const size_t stride = (size_t)L.Vh * n;
    const int st = lex_stride(L, MU);
    const int cm = g.c[MU];
    const int Lm = L.L[MU];
    const char *gbase = static_cast<const char *>(a.gauge);
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF*gamma
    constexpr int SB = -SF;

    // forward neighbour x + mu
    {
        int j;
        bool flip;
        if constexpr (TBL) {
            const int v = __ldg(a.nbr + (size_t)(2 * MU) * L.Vh + i);
            j = v & 0x7fffffff;
            flip = v < 0;
        } else {
            const int yl = (cm == Lm - 1) ? g.lex - (Lm - 1) * st : g.lex + st;
            j = yl >> 1;
            flip = MU == 0 && cm == Lm - 1 && L.t_bc < 0;
        }
        j = PLQ_GUARD(a.kstatus, j, L.Vh);
        cx<T> u[3][3];
        Link<P, R>::load(gbase + (size_t)(a.out_parity * 4 + MU) * a.gblock, L.Vh, i, u);
#pragma unroll
        for (int t = 0; t < RT; ++t) hop_one<P, R, MU, SF, false>(a.in, stride, (size_t)j * n + r0 + t, flip, u, acc[t]);
    }
    // backward neighbour x - mu
    {
        int j;
        bool flip;
        if constexpr (TBL) {
            const int v = __ldg(a.nbr + (size_t)(2 * MU + 1) * L.Vh + i);
            j = v & 0x7fffffff;
            flip = v < 0;
        } else {
            const int yl = (cm == 0) ? g.lex + (Lm - 1) * st : g.lex - st;
            j = yl >> 1;
            flip = MU == 0 && cm == 0 && L.t_bc < 0;
        }
        j = PLQ_GUARD(a.kstatus, j, L.Vh);
        cx<T> u[3][3];
        Link<P, R>::load(gbase + (size_t)((1 - a.out_parity) * 4 + MU) * a.gblock, L.Vh, j, u);
#pragma unroll
        for (int t = 0; t < RT; ++t) hop_one<P, R, MU, SB, true>(a.in, stride, (size_t)j * n + r0 + t, flip, u, acc[t]);
    }
}

// Single right-hand-side form (used by the batched persistent kernel).
template <int P, int R, int MU, bool DAG, bool TBL>
__device__ __forceinline__ void hop_dir(const HopArgs &a, const SiteGeom &g, int i, int rr, cx<RealOf<P>> acc[12]) {
    cx<RealOf<P>>(&a1)[1][12] = *reinterpret_cast<cx<RealOf<P>>(*)[1][12]>(acc);
    hop_dir<P, R, MU, DAG, TBL, 1>(a, g, i, rr, a1);
}

// Threads are arranged as (n / RT right-hand-side tiles) x (sites): the
// threads of one site are adjacent and share its link loads through L1, and
// each thread applies every link it loads to RT right-hand sides.
template <int P, int R, int EPI, bool DAG, bool TBL, int RT>
__device__ __forceinline__ void hop_body(const HopArgs &a) {
    using T = RealOf<P>;
    const int n = a.nrhs;
    const long long total = (long long)a.lat.Vh * n;
    const size_t stride = (size_t)total;
    constexpr int NV = EPI == EPI_XPAY_NORM ? 1 : EPI == EPI_XPAY_DOTW ? 2 : EPI == EPI_XPAY_TS ? 3 : 0;
    RedAcc<(NV > 0 ? NV : 1), RT> racc;
    red_init(racc);

    const int r0 = threadIdx.x * RT;
    const int i_end = a.site_end < 0 ? a.lat.Vh : a.site_end;
    const int plane = a.lat.L[2] * (a.lat.L[1] >> 1);  // checkerboard sites of one (t, z) plane
    const int zc = a.zc;
    for (int li = a.site_begin + blockIdx.x * blockDim.y + threadIdx.y; li < i_end; li += gridDim.x * blockDim.y) {
        int i = li;
        if (zc > 0) {  // z-chunk order: (chunk, t, z in chunk, y, x)
            const int per_chunk = a.lat.L[0] * zc * plane;
            const int c = li / per_chunk;
            int rem = li - c * per_chunk;
            const int t = rem / (zc * plane);
            rem -= t * zc * plane;
            const int zi = rem / plane;
            const int w = rem - zi * plane;
            i = (t * a.lat.L[3] + c * zc + zi) * plane + w;
        }
        i = PLQ_GUARD(a.kstatus, i, a.lat.Vh);
        bool all_frozen = a.st != nullptr;
#pragma unroll
        for (int t = 0; t < RT; ++t) all_frozen = all_frozen && a.st[r0 + t].stop;
        if (all_frozen) continue;  // frozen right-hand sides
        SiteGeom g{};
        if constexpr (!TBL) g = site_geom(a.lat, a.out_parity, i);
        cx<T> acc[RT][12];
#pragma unroll
        for (int t = 0; t < RT; ++t)
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[t][k] = {T(0), T(0)};
        hop_dir<P, R, 0, DAG, TBL, RT>(a, g, i, r0, acc);
        hop_dir<P, R, 1, DAG, TBL, RT>(a, g, i, r0, acc);
        hop_dir<P, R, 2, DAG, TBL, RT>(a, g, i, r0, acc);
        hop_dir<P, R, 3, DAG, TBL, RT>(a, g, i, r0, acc);

#pragma unroll
        for (int t = 0; t < RT; ++t) {
            const int rr = r0 + t;
            if (RT > 1 && a.st != nullptr && a.st[rr].stop) continue;
            const long long idx = PLQ_GUARD(a.kstatus, (long long)i * n + rr, (long long)stride);
            if (a.nu_h != 0.0 || a.scale_h != 1.0) twist12(acc[t], (T)a.nu_h, (T)a.scale_h);
            if constexpr (EPI != EPI_PLAIN) {
                cx<T> xv[12];
                Spinor<P>::load(a.x, stride, (size_t)idx, xv);
                if (a.nu_x != 0.0) twist12(xv, (T)a.nu_x, T(1));
                const T s = (T)a.a;
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    acc[t][k].re = fma(s, acc[t][k].re, xv[k].re);
                    acc[t][k].im = fma(s, acc[t][k].im, xv[k].im);
                }
                if constexpr (EPI == EPI_XPAY_NORM) {
                    T s0 = 0;
#pragma unroll
                    for (int k = 0; k < 12; ++k) s0 += acc[t][k].re * acc[t][k].re + acc[t][k].im * acc[t][k].im;
                    racc.add(0, t, s0);
                } else if constexpr (EPI == EPI_XPAY_DOTW) {
                    cx<T> wv[12];
                    Spinor<P>::load(a.w, stride, (size_t)idx, wv);
                    T s0 = 0, s1 = 0;
#pragma unroll
                    for (int k = 0; k < 12; ++k) {  // <w, out> = sum conj(w) out
                        s0 += wv[k].re * acc[t][k].re + wv[k].im * acc[t][k].im;
                        s1 += wv[k].re * acc[t][k].im - wv[k].im * acc[t][k].re;
                    }
                    racc.add(0, t, s0);
                    racc.add(1, t, s1);
                } else if constexpr (EPI == EPI_XPAY_TS) {
                    T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
                    for (int k = 0; k < 12; ++k) {  // <out, x> and |out|^2
                        s0 += acc[t][k].re * xv[k].re + acc[t][k].im * xv[k].im;
                        s1 += acc[t][k].re * xv[k].im - acc[t][k].im * xv[k].re;
                        s2 += acc[t][k].re * acc[t][k].re + acc[t][k].im * acc[t][k].im;
                    }
                    racc.add(0, t, s0);
                    racc.add(1, t, s1);
                    racc.add(2, t, s2);
                }
            }
            Spinor<P>::store(a.out, stride, (size_t)idx, acc[t]);
        }
    }
    if constexpr (NV > 0) grid_reduce(a.red, racc, blockDim.x);
}

// Register budget of the one-RHS kernels (0: the compiler's choice under a
// 256-thread launch bound).  Left alone the compiler hoists the loads of
// several directions and takes ~140 registers (FP32, 18-real links), which
// leaves 3 blocks of 128 threads per SM; a cap trades part of that hoisting
// for resident warps, i.e. more bytes in flight per SM.  The values are the
// fastest of a sweep (64..112) on the 32^3x64 half-application: 80 for FP32
// with 18-real links, 72 for the other FP32/FP16 formats, 96 for the
// epilogue kernels of the solvers.  FP64 is bound by its arithmetic and
// runs uncapped, as do the neighbour-table variants (~72 registers anyway)
// and the RHS-tiled kernels, whose tiles live in registers.
template <int P, int R, int EPI, bool TBL, int RT>
constexpr int hop_reg_cap() {
    if (RT != 1 || TBL || P == PLQ_F64) return 0;
    if (EPI != EPI_PLAIN) return 96;
    return (P == PLQ_F32 && R == 18) ? 80 : 72;
}

template <int P, int R, int EPI, bool DAG, bool TBL, int RT = 1>
__global__ void __launch_bounds__(256) hop_kernel(const HopArgs a) {
    hop_body<P, R, EPI, DAG, TBL, RT>(a);
}

template <int P, int R, int EPI, bool DAG, bool TBL, int RT, int NREG>
__global__ void __maxnreg__(NREG) hop_kernel_capped(const HopArgs a) {
    hop_body<P, R, EPI, DAG, TBL, RT>(a);
}

// Multi-RHS variant with the links staged in shared memory.  A block owns
// blockDim.y sites; its threads first load the 8 links of each of those sites
// once (rebuilding row 2 of 12-real links once) together with the neighbour
// indices, then every (site, RHS-tile) thread reads its links from shared
// memory, where the n/RT threads of a site get them as broadcasts.  This
// removes the per-RHS link requests that make the L1 the bottleneck of the
// plain multi-RHS kernel.
constexpr int kMaxSitesPerBlock = 32;

// Asynchronous global -> shared copies (cp.async; completion is tracked per
// thread in commit groups, so a thread that copies into and reads from its own
// slots needs no block barrier).  The 16-byte form bypasses L1.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most `pending` of this thread's groups are still in flight
__device__ __forceinline__ void cp_async_wait(int pending) {
    if (pending <= 0) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    else if (pending == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else asm volatile("cp.async.wait_group 2;\n" ::: "memory");
}

// 16-byte planes of one spinor element in storage format P: 6 (FP32: two
// complex numbers each), 3 (FP16: four each, plus a float site norm)
template <int P>
constexpr int spinor_planes() {
    return P == PLQ_F16 ? 3 : 6;
}

// Shared memory of the multi-RHS kernel for `sites` sites and `threads`
// threads: links and neighbour indices, then NB per-thread slots of one
// neighbour spinor (16-byte planes, then the FP16 norms).
template <int P, int NB>
__host__ __device__ constexpr size_t mrhs_smem_bytes(int sites, int threads) {
    return (((size_t)sites * 8 * (9 * sizeof(cx<RealOf<P>>) + sizeof(int)) + 15) & ~(size_t)15) +
           (size_t)NB * threads * (16 * spinor_planes<P>() + (P == PLQ_F16 ? sizeof(float) : 0));
}

// NB = 0: each thread loads its neighbour spinors straight into registers.
// NB = 2 or 3 (one right-hand side per thread): the spinors of the next NB - 1
// directions are already on their way into the thread's shared-memory slots
// while it computes the current direction.  The loads of this kernel mostly
// miss L1 and wait on L2; with 80 registers a thread can hold only one
// direction's spinor, so the copies into shared memory are what lets a thread
// keep more than one direction's loads in flight.
template <int P, int R, int EPI, bool DAG, int RT, int NB>
__global__ void __maxnreg__(RT == 1 ? 80 : 168) hop_mrhs_kernel(const HopArgs a) {
    static_assert(NB == 0 || (RT == 1 && NB >= 2 && NB <= 3), "spinor slots need one RHS per thread");
    using T = RealOf<P>;
    constexpr int NP = spinor_planes<P>();
    // dynamic shared memory sized for this block's sites (the rest of the SM's
    // 256 KB stays L1 for the neighbour spinors): links, then neighbour indices
    extern __shared__ __align__(16) unsigned char mrhs_smem[];
    cx<T>(*sU)[8][9] = reinterpret_cast<cx<T>(*)[8][9]>(mrhs_smem);
    int(*sJ)[8] = reinterpret_cast<int(*)[8]>(mrhs_smem + (size_t)blockDim.y * 8 * 9 * sizeof(cx<T>));
    uint4 *sP = reinterpret_cast<uint4 *>(mrhs_smem + mrhs_smem_bytes<P, 0>(blockDim.y, 0));
    float *sN = reinterpret_cast<float *>(sP + (size_t)NB * NP * blockDim.x * blockDim.y);
    const int n = a.nrhs;
    const size_t stride = (size_t)a.lat.Vh * n;
    constexpr int NV = EPI == EPI_XPAY_NORM ? 1 : 0;
    RedAcc<1, RT> racc;
    red_init(racc);
    const Lattice &L = a.lat;
    const char *gbase = static_cast<const char *>(a.gauge);
    const int S = blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
    const int r0 = threadIdx.x * RT;
    const int plane = L.L[2] * (L.L[1] >> 1);
    const int zc = a.zc;
    const int nblk = (L.Vh + S - 1) / S;
    if (a.st != nullptr) {
        // every right-hand side frozen (a solver's iterations past convergence):
        // nothing to stage or compute; the reduction still counts this block
        bool all_stopped = true;
        for (int r = 0; r < n; ++r) all_stopped = all_stopped && a.st[r].stop;
        if (all_stopped) {
            if constexpr (NV > 0) grid_reduce(a.red, racc, blockDim.x);
            return;
        }
    }
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        __syncthreads();  // the previous site block is done with the shared links
        // stage: (site, direction) pairs
        for (int q = tid; q < S * 8; q += nthr) {
            const int k = q >> 3, d = q & 7, mu = d >> 1, back = d & 1;
            const int li = blk * S + k;
            if (li >= L.Vh) continue;
            int i = li;
            if (zc > 0) {
                const int per_chunk = L.L[0] * zc * plane;
                const int c = li / per_chunk;
                int rem = li - c * per_chunk;
                const int t = rem / (zc * plane);
                rem -= t * zc * plane;
                const int zi = rem / plane;
                i = (t * L.L[3] + c * zc + zi) * plane + (rem - zi * plane);
            }
            i = PLQ_GUARD(a.kstatus, i, L.Vh);
            const SiteGeom g = site_geom(L, a.out_parity, i);
            const int st = mu == 0 ? L.L[1] * L.L[2] * L.L[3] : mu == 1 ? 1 : mu == 2 ? L.L[1] : L.L[1] * L.L[2];
            const int cm = g.c[mu], Lm = L.L[mu];
            int j;
            bool flip;
            if (!back) {
                j = ((cm == Lm - 1) ? g.lex - (Lm - 1) * st : g.lex + st) >> 1;
                flip = mu == 0 && cm == Lm - 1 && L.t_bc < 0;
            } else {
                j = ((cm == 0) ? g.lex + (Lm - 1) * st : g.lex - st) >> 1;
                flip = mu == 0 && cm == 0 && L.t_bc < 0;
            }
            j = PLQ_GUARD(a.kstatus, j, L.Vh);
            cx<T> u[3][3];
            Link<P, R>::load(gbase + (size_t)((back ? 1 - a.out_parity : a.out_parity) * 4 + mu) * a.gblock, L.Vh,
                             back ? j : i, u);
            // the time-boundary sign goes into the staged link (row 2 of a 12-real
            // link is already rebuilt here), so the consumers never apply it
            const T sg = flip ? T(-1) : T(1);
#pragma unroll
            for (int e = 0; e < 9; ++e) sU[k][d][e] = {sg * u[e / 3][e % 3].re, sg * u[e / 3][e % 3].im};
            sJ[k][d] = j;
        }
        __syncthreads();
        const int k = threadIdx.y;
        const int li = blk * S + k;
        if (li >= L.Vh) continue;
        int i = li;
        if (zc > 0) {
            const int per_chunk = L.L[0] * zc * plane;
            const int c = li / per_chunk;
            int rem = li - c * per_chunk;
            const int t = rem / (zc * plane);
            rem -= t * zc * plane;
            const int zi = rem / plane;
            i = (t * L.L[3] + c * zc + zi) * plane + (rem - zi * plane);
        }
        bool all_frozen = a.st != nullptr;
#pragma unroll
        for (int t = 0; t < RT; ++t) all_frozen = all_frozen && a.st[r0 + t].stop;
        if (all_frozen) continue;
        // copy the neighbour spinor of direction d into slot b of this thread
        auto issue = [&](int d, int b) {
            const size_t e = (size_t)PLQ_GUARD(a.kstatus, sJ[k][d], L.Vh) * n + r0;
            const uint4 *src = static_cast<const uint4 *>(a.in) + e;
#pragma unroll
            for (int q = 0; q < NP; ++q) cp_async16(&sP[(size_t)(b * NP + q) * nthr + tid], src + q * stride);
            if constexpr (P == PLQ_F16)
                cp_async4(&sN[b * nthr + tid],
                          reinterpret_cast<const float *>(static_cast<const uint4 *>(a.in) + NP * stride) + e);
            cp_async_commit();
        };
        if constexpr (NB > 0) {
#pragma unroll
            for (int d = 0; d < NB - 1; ++d) issue(d, d);
        }
        cx<T> acc[RT][12];
#pragma unroll
        for (int t = 0; t < RT; ++t)
#pragma unroll
            for (int e = 0; e < 12; ++e) acc[t][e] = {T(0), T(0)};
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int j = PLQ_GUARD(a.kstatus, sJ[k][d], L.Vh);
            const int mu = d >> 1;
            if constexpr (NB > 0) {
                (void)j;
                // slot (d + NB - 1) % NB was read in the previous direction, whose
                // arithmetic has consumed the values
                if (d + NB - 1 < 8) issue(d + NB - 1, (d + NB - 1) % NB);
                cp_async_wait(d + NB - 1 < 8 ? NB - 1 : 7 - d);
            }
#pragma unroll
            for (int t = 0; t < RT; ++t) {
                cx<T> phi[12];
                T sc;
                if constexpr (NB > 0) {
                    const int b = d % NB;
                    if constexpr (P == PLQ_F16) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const uint4 v = sP[(size_t)(b * NP + q) * nthr + tid];
                            const float2 x0 = h2f(v.x), x1 = h2f(v.y), x2 = h2f(v.z), x3 = h2f(v.w);
                            phi[4 * q + 0] = {x0.x, x0.y};
                            phi[4 * q + 1] = {x1.x, x1.y};
                            phi[4 * q + 2] = {x2.x, x2.y};
                            phi[4 * q + 3] = {x3.x, x3.y};
                        }
                        sc = sN[b * nthr + tid];
                    } else {
#pragma unroll
                        for (int q = 0; q < 6; ++q) {
                            const float4 v = reinterpret_cast<const float4 *>(sP)[(size_t)(b * NP + q) * nthr + tid];
                            phi[2 * q] = {v.x, v.y};
                            phi[2 * q + 1] = {v.z, v.w};
                        }
                        sc = T(1);
                    }
                } else {
                    sc = load_for_projection<P>(a.in, stride, (size_t)j * n + r0 + t, phi);
                }
                cx<T> hh[6], uh[6];
                // project, scale, multiply by U (forward) or U^dagger (backward), rebuild
#define PLQ_DIR(MU)                                                                        \
    if (mu == MU) {                                                                        \
        constexpr int SF = DAG ? +1 : -1;                                                  \
        if ((d & 1) == 0) project<MU, SF>(phi, hh);                                        \
        else project<MU, -SF>(phi, hh);                                                    \
    }
                PLQ_DIR(0) PLQ_DIR(1) PLQ_DIR(2) PLQ_DIR(3)
#undef PLQ_DIR
                if constexpr (P == PLQ_F16) {  // the site norm of the FP16 storage
#pragma unroll
                    for (int e = 0; e < 6; ++e) hh[e] = {sc * hh[e].re, sc * hh[e].im};
                }
                const cx<T>(*su)[9] = &sU[k][d];
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        cx<T> z{0, 0};
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            if ((d & 1) == 0) z = cfma((*su)[3 * r + c], hh[3 * s + c], z);
                            else z = cfma_conj((*su)[3 * c + r], hh[3 * s + c], z);
                        }
                        uh[3 * s + r] = z;
                    }
#define PLQ_REC(MU)                                                                        \
    if (mu == MU) {                                                                        \
        constexpr int SF = DAG ? +1 : -1;                                                  \
        if ((d & 1) == 0) reconstruct<MU, SF>(acc[t], uh);                                 \
        else reconstruct<MU, -SF>(acc[t], uh);                                             \
    }
                PLQ_REC(0) PLQ_REC(1) PLQ_REC(2) PLQ_REC(3)
#undef PLQ_REC
            }
        }
#pragma unroll
        for (int t = 0; t < RT; ++t) {
            const int rr = r0 + t;
            if (a.st != nullptr && a.st[rr].stop) continue;
            const long long idx = PLQ_GUARD(a.kstatus, (long long)i * n + rr, (long long)stride);
            if (a.nu_h != 0.0 || a.scale_h != 1.0) twist12(acc[t], (T)a.nu_h, (T)a.scale_h);
            if constexpr (EPI != EPI_PLAIN) {
                cx<T> xv[12];
                Spinor<P>::load(a.x, stride, (size_t)idx, xv);
                if (a.nu_x != 0.0) twist12(xv, (T)a.nu_x, T(1));
                const T s = (T)a.a;
#pragma unroll
                for (int e = 0; e < 12; ++e) {
                    acc[t][e].re = fma(s, acc[t][e].re, xv[e].re);
                    acc[t][e].im = fma(s, acc[t][e].im, xv[e].im);
                }
                if constexpr (EPI == EPI_XPAY_NORM) {
                    T s0 = 0;
#pragma unroll
                    for (int e = 0; e < 12; ++e) s0 += acc[t][e].re * acc[t][e].re + acc[t][e].im * acc[t][e].im;
                    racc.add(0, t, s0);
                }
            }
            Spinor<P>::store(a.out, stride, (size_t)idx, acc[t]);
        }
    }
    if constexpr (NV > 0) grid_reduce(a.red, racc, blockDim.x);
}

template <int P, int R, int EPI, bool DAG, int RT, int NB>
plq_status launch_mrhs_t(const HopArgs &a, cudaStream_t s, int block) {
    if (a.block > 0) block = a.block;
    if (block <= 0 || block > 1024) block = 128;
    const int n = a.nrhs;
    const int tiles = n / RT;
    int spb = block / tiles > 0 ? block / tiles : 1;
    if (spb > kMaxSitesPerBlock) spb = kMaxSitesPerBlock;
    for (int q = spb; q >= 1; --q)
        if ((q * tiles) % 32 == 0) {
            spb = q;
            break;
        }
    const int threads = tiles * spb;
    const size_t smem = mrhs_smem_bytes<P, NB>(spb, threads);
    // occupancy per (sites per block, threads per site), filled on first use
    static std::atomic<int> per_sm[kMaxSitesPerBlock + 1][PLQ_MAX_RHS + 1];
    auto kern = hop_mrhs_kernel<P, R, EPI, DAG, RT, NB>;
    if (per_sm[spb][tiles].load(std::memory_order_relaxed) == 0) {
        int nb = 0;
        cudaError_t e = cudaSuccess;
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncAttributes fa{};
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
        if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(hop_mrhs)");
        if (threads > fa.maxThreadsPerBlock) nb = 0;
        per_sm[spb][tiles].store(nb > 0 ? nb : -1, std::memory_order_relaxed);
    }
    const int fit = per_sm[spb][tiles].load(std::memory_order_relaxed);
    if (fit < 0) return set_error(PLQ_ERR_ARG, "a block of %d threads does not fit the multi-RHS kernel", threads);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = ((long long)a.lat.Vh + spb - 1) / spb;
    long long cap = a.spt > 0 ? (want + a.spt - 1) / a.spt : (long long)fit * sms;
    if (EPI >= EPI_XPAY_NORM && cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
    const int grid = (int)(want < cap ? want : cap);
    if (grid <= 0) return PLQ_OK;
    kern<<<grid, dim3(tiles, spb), smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "hop_mrhs_kernel launch");
    return PLQ_OK;
}

template <int P, int R, int RT, int NB>
plq_status dispatch_mrhs(const HopArgs &a, int epi, cudaStream_t s, int block) {
    switch (epi) {
    case EPI_PLAIN:
        return a.dagger ? launch_mrhs_t<P, R, EPI_PLAIN, true, RT, NB>(a, s, block)
                        : launch_mrhs_t<P, R, EPI_PLAIN, false, RT, NB>(a, s, block);
    case EPI_XPAY:
        return a.dagger ? launch_mrhs_t<P, R, EPI_XPAY, true, RT, NB>(a, s, block)
                        : launch_mrhs_t<P, R, EPI_XPAY, false, RT, NB>(a, s, block);
    default:
        return a.dagger ? launch_mrhs_t<P, R, EPI_XPAY_NORM, true, RT, NB>(a, s, block)
                        : launch_mrhs_t<P, R, EPI_XPAY_NORM, false, RT, NB>(a, s, block);
    }
}

// Launch helper: grid = min(work blocks, resident blocks on all SMs).
template <int P, int R, int EPI, bool DAG, bool TBL = false, int RT = 1>
plq_status launch_hop_t(const HopArgs &a, cudaStream_t s, int block) {
    if (a.block > 0) block = a.block;
    if (block <= 0 || block > 1024) block = 128;
    const int n = a.nrhs;
    const int tiles = n / RT;  // threads per site
    // sites per block: as many as fit in `block` threads, rounded so that the
    // block is a whole number of warps when that is possible
    int spb = block / tiles > 0 ? block / tiles : 1;
    for (int q = spb; q >= 1; --q)
        if ((q * tiles) % 32 == 0) {
            spb = q;
            break;
        }
    const int threads = tiles * spb;
    // resident blocks per SM for each block size, filled on first use (-1:
    // the block does not fit this kernel's registers or launch bound)
    static std::atomic<int> per_sm[1025];
    constexpr int nreg = hop_reg_cap<P, R, EPI, TBL, RT>();
    auto kern = [] {
        if constexpr (nreg > 0) return hop_kernel_capped<P, R, EPI, DAG, TBL, RT, (nreg > 0 ? nreg : 255)>;
        else return hop_kernel<P, R, EPI, DAG, TBL, RT>;
    }();
    if (per_sm[threads].load(std::memory_order_relaxed) == 0) {
        int nb = 0;
        // the occupancy query does not apply the kernel's launch bound: the
        // attribute's thread limit covers both it and the registers
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, kern);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, 0);
        if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(hop)");
        if (threads > fa.maxThreadsPerBlock) nb = 0;
        per_sm[threads].store(nb > 0 ? nb : -1, std::memory_order_relaxed);
    }
    const int fit = per_sm[threads].load(std::memory_order_relaxed);
    if (fit < 0) return set_error(PLQ_ERR_ARG, "a block of %d threads does not fit the hopping kernel", threads);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int i_end = a.site_end < 0 ? a.lat.Vh : a.site_end;
    const long long want = ((long long)(i_end - a.site_begin) + spb - 1) / spb;
    long long cap = a.spt > 0 ? (want + a.spt - 1) / a.spt : (long long)fit * sms;
    if (EPI >= EPI_XPAY_NORM && cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
    const int grid = (int)(want < cap ? want : cap);
    if (grid <= 0) return PLQ_OK;
    const dim3 bdim(tiles, spb);
    kern<<<grid, bdim, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "hop_kernel launch");
    return PLQ_OK;
}

template <int P, int R, int RT>
plq_status dispatch_tiled(const HopArgs &a, int epi, cudaStream_t s, int block) {
    switch (epi) {
    case EPI_PLAIN:
        return a.dagger ? launch_hop_t<P, R, EPI_PLAIN, true, false, RT>(a, s, block)
                        : launch_hop_t<P, R, EPI_PLAIN, false, false, RT>(a, s, block);
    case EPI_XPAY:
        return a.dagger ? launch_hop_t<P, R, EPI_XPAY, true, false, RT>(a, s, block)
                        : launch_hop_t<P, R, EPI_XPAY, false, false, RT>(a, s, block);
    default:
        return a.dagger ? launch_hop_t<P, R, EPI_XPAY_NORM, true, false, RT>(a, s, block)
                        : launch_hop_t<P, R, EPI_XPAY_NORM, false, false, RT>(a, s, block);
    }
}

}  // namespace plq

#include "plq_hop_rows.cuh"

namespace plq {

template <int P, int R>
plq_status dispatch_hop(const HopArgs &a, int epi, cudaStream_t s, int block) {
    // Right-hand-side tiles (RT > 1) exist for the FP32-arithmetic storage
    // formats and the epilogues of operator applications and CG; the
    // neighbour-table variants for the plain and xpay epilogues; the
    // row-streamed kernel for whole-lattice applications with those epilogues.
    if constexpr (P != PLQ_F64) {
        if (a.smem_links == 4 && a.site_begin == 0 && a.site_end < 0 && epi <= EPI_XPAY_NORM)
            return dispatch_rows<P, R>(a, epi, s);
        if (a.smem_links && a.nrhs > 1 && a.site_begin == 0 && a.site_end < 0 && epi <= EPI_XPAY_NORM) {
            if (a.rhs_tile == 2 && a.nrhs % 2 == 0) return dispatch_mrhs<P, R, 2, 0>(a, epi, s, block);
            if (a.smem_links == 2) return dispatch_mrhs<P, R, 1, 2>(a, epi, s, block);
            if (a.smem_links == 3) return dispatch_mrhs<P, R, 1, 3>(a, epi, s, block);
            return dispatch_mrhs<P, R, 1, 0>(a, epi, s, block);
        }
        if (a.rhs_tile > 1 && a.nrhs % a.rhs_tile == 0 && epi <= EPI_XPAY_NORM) {
            if (a.rhs_tile == 2) return dispatch_tiled<P, R, 2>(a, epi, s, block);
            if (a.rhs_tile == 4) return dispatch_tiled<P, R, 4>(a, epi, s, block);
        }
    }
    const bool tbl = a.nbr != nullptr;
    switch (epi) {
    case EPI_PLAIN:
        if (tbl)
            return a.dagger ? launch_hop_t<P, R, EPI_PLAIN, true, true>(a, s, block)
                            : launch_hop_t<P, R, EPI_PLAIN, false, true>(a, s, block);
        return a.dagger ? launch_hop_t<P, R, EPI_PLAIN, true>(a, s, block) : launch_hop_t<P, R, EPI_PLAIN, false>(a, s, block);
    case EPI_XPAY:
        if (tbl)
            return a.dagger ? launch_hop_t<P, R, EPI_XPAY, true, true>(a, s, block)
                            : launch_hop_t<P, R, EPI_XPAY, false, true>(a, s, block);
        return a.dagger ? launch_hop_t<P, R, EPI_XPAY, true>(a, s, block) : launch_hop_t<P, R, EPI_XPAY, false>(a, s, block);
    case EPI_XPAY_NORM:
        if (tbl)
            return a.dagger ? launch_hop_t<P, R, EPI_XPAY_NORM, true, true>(a, s, block)
                            : launch_hop_t<P, R, EPI_XPAY_NORM, false, true>(a, s, block);
        return a.dagger ? launch_hop_t<P, R, EPI_XPAY_NORM, true>(a, s, block)
                        : launch_hop_t<P, R, EPI_XPAY_NORM, false>(a, s, block);
    case EPI_XPAY_DOTW:
        return launch_hop_t<P, R, EPI_XPAY_DOTW, false>(a, s, block);
    case EPI_XPAY_TS:
        return launch_hop_t<P, R, EPI_XPAY_TS, false>(a, s, block);
    default:
        return set_error(PLQ_ERR_ARG, "bad epilogue %d", epi);
    }
}

}  // namespace plq
