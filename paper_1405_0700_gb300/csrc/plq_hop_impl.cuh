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

#include "plq_fields.cuh"

namespace plq {

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

__device__ __forceinline__ int lex_stride(const Lattice &L, int mu) {
    // strides of t, x, y, z in the lexicographic index
    return mu == 0 ? L.L[1] * L.L[2] * L.L[3] : mu == 1 ? 1 : mu == 2 ? L.L[1] : L.L[1] * L.L[2];
}

// Contribution of direction MU (forward and backward) to acc.
// DAG: gamma5 H gamma5 = H^dagger, i.e. the projectors (1 -/+ gamma) swapped.
template <int P, int R, int MU, bool DAG, bool TBL>
__device__ __forceinline__ void hop_dir(const HopArgs &a, const SiteGeom &g, int i, int rr, cx<RealOf<P>> acc[12]) {
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
        cx<T> phi[12];
        Spinor<P>::load(a.in, stride, (size_t)j * n + rr, phi);
        cx<T> h[6];
        project<MU, SF>(phi, h);
        if (MU == 0 && flip) {
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = {-h[k].re, -h[k].im};
        }
        cx<T> u[3][3];
        Link<P, R>::load(gbase + (size_t)(a.out_parity * 4 + MU) * a.gblock, L.Vh, i, u);
        cx<T> uh[6];
        su3_mul(u, h, uh);
        reconstruct<MU, SF>(acc, uh);
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
        cx<T> phi[12];
        Spinor<P>::load(a.in, stride, (size_t)j * n + rr, phi);
        cx<T> h[6];
        project<MU, SB>(phi, h);
        if (MU == 0 && flip) {
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = {-h[k].re, -h[k].im};
        }
        cx<T> u[3][3];
        Link<P, R>::load(gbase + (size_t)((1 - a.out_parity) * 4 + MU) * a.gblock, L.Vh, j, u);
        cx<T> uh[6];
        su3_dag_mul(u, h, uh);
        reconstruct<MU, SB>(acc, uh);
    }
}

template <int P, int R, int EPI, bool DAG, bool TBL>
__global__ void __launch_bounds__(256) hop_kernel(const HopArgs a) {
    using T = RealOf<P>;
    const int n = a.nrhs;
    const long long total = (long long)a.lat.Vh * n;
    const size_t stride = (size_t)total;
    constexpr int NV = EPI == EPI_XPAY_NORM ? 1 : EPI == EPI_XPAY_DOTW ? 2 : EPI == EPI_XPAY_TS ? 3 : 0;
    RedAcc<(NV > 0 ? NV : 1), T> racc;
    if constexpr (NV > 0) red_init(racc, n);

    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = n == 1 ? (int)idx : (int)(idx / n);
        const int rr = (int)(idx - (long long)i * n);
        if (a.st != nullptr && a.st[rr].stop) continue;  // frozen right-hand side
        SiteGeom g{};
        if constexpr (!TBL) g = site_geom(a.lat, a.out_parity, i);
        cx<T> acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {T(0), T(0)};
        hop_dir<P, R, 0, DAG, TBL>(a, g, i, rr, acc);
        hop_dir<P, R, 1, DAG, TBL>(a, g, i, rr, acc);
        hop_dir<P, R, 2, DAG, TBL>(a, g, i, rr, acc);
        hop_dir<P, R, 3, DAG, TBL>(a, g, i, rr, acc);

        if constexpr (EPI != EPI_PLAIN) {
            cx<T> xv[12];
            Spinor<P>::load(a.x, stride, (size_t)idx, xv);
            const T s = (T)a.a;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                acc[k].re = fma(s, acc[k].re, xv[k].re);
                acc[k].im = fma(s, acc[k].im, xv[k].im);
            }
            if constexpr (EPI == EPI_XPAY_NORM) {
                T s0 = 0;
#pragma unroll
                for (int k = 0; k < 12; ++k) s0 += acc[k].re * acc[k].re + acc[k].im * acc[k].im;
                racc.add(0, rr, s0);
            } else if constexpr (EPI == EPI_XPAY_DOTW) {
                cx<T> wv[12];
                Spinor<P>::load(a.w, stride, (size_t)idx, wv);
                T s0 = 0, s1 = 0;
#pragma unroll
                for (int k = 0; k < 12; ++k) {  // <w, out> = sum conj(w) out
                    s0 += wv[k].re * acc[k].re + wv[k].im * acc[k].im;
                    s1 += wv[k].re * acc[k].im - wv[k].im * acc[k].re;
                }
                racc.add(0, rr, s0);
                racc.add(1, rr, s1);
            } else if constexpr (EPI == EPI_XPAY_TS) {
                T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
                for (int k = 0; k < 12; ++k) {  // <out, x> and |out|^2
                    s0 += acc[k].re * xv[k].re + acc[k].im * xv[k].im;
                    s1 += acc[k].re * xv[k].im - acc[k].im * xv[k].re;
                    s2 += acc[k].re * acc[k].re + acc[k].im * acc[k].im;
                }
                racc.add(0, rr, s0);
                racc.add(1, rr, s1);
                racc.add(2, rr, s2);
            }
        }
        Spinor<P>::store(a.out, stride, (size_t)idx, acc);
    }
    if constexpr (NV > 0) grid_reduce(a.red, racc);
}

// Launch helper: grid = min(work blocks, resident blocks on all SMs).
template <int P, int R, int EPI, bool DAG, bool TBL = false>
plq_status launch_hop_t(const HopArgs &a, cudaStream_t s, int block) {
    if (a.block > 0) block = a.block;
    static int per_sm[1025] = {0};
    auto kern = hop_kernel<P, R, EPI, DAG, TBL>;
    if (block <= 0 || block > 1024) block = 128;
    if (per_sm[block] == 0) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, block, 0);
        if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(hop)");
        per_sm[block] = nb > 0 ? nb : 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long total = (long long)a.lat.Vh * a.nrhs;
    long long want = (total + block - 1) / block;
    long long cap = (long long)per_sm[block] * sms;
    if (EPI >= EPI_XPAY_NORM && cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
    const int grid = (int)(want < cap ? want : cap);
    if (grid <= 0) return PLQ_OK;
    kern<<<grid, block, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "hop_kernel launch");
    return PLQ_OK;
}

template <int P, int R>
plq_status dispatch_hop(const HopArgs &a, int epi, cudaStream_t s, int block) {
    // The neighbour-table variants exist for the plain and xpay epilogues
    // (operator applications); the reducing epilogues compute indices inline.
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
