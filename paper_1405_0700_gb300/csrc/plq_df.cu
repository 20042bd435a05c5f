// FP64-accuracy hopping operator in float-float arithmetic (storage PLQ_DF64).
//
// Storage.  A PLQ_DF64 half field of n right-hand sides is the FP32 half
// field of the high parts followed by the FP32 half field of the low parts
// (6 + 6 planes of float4, 192 B per site and right-hand side -- the bytes of
// FP64).  A PLQ_DF64 gauge block (parity, mu) is the FP32 18-real block of the
// high parts followed by that of the low parts (144 B per link).  Packing
// splits every double d exactly into hi = rn(d), lo = rn(d - hi).
//
// Operator.  The same Eq. (1) as every other precision, through the half
// spinors of Eq. (2): projection and reconstruction with float-float
// additions whose low parts are renormalised once per site; each SU(3) x
// half-spinor row as one sum of six products whose high parts are added by
// TwoSum and whose rounding errors and low-order terms are gathered in one
// float (renormalised once per row).
//
// Used by the mixed-precision solvers for the reliable-update residual
// s = bhat - Mhat x (two half-applications), where the FP64 operator would
// otherwise dominate the solve time on this GPU.
#include <atomic>

#include "plq_df.cuh"
#include "plq_hop_impl.cuh"

namespace plq {
namespace {

struct DfArgs {
    const void *in = nullptr;
    void *out = nullptr;
    const void *x = nullptr;   // xpay source (PLQ_DF64 layout) or null
    const void *gauge = nullptr;
    size_t gblock = 0;
    int out_parity = 0;
    int nrhs = 1;
    Lattice lat;
    double a = 0.0;            // out = x + a * (H in)
    double nu_h = 0.0;         // H in -> scale_h * (1 + i nu_h gamma5) H in
    double scale_h = 1.0;
};

// half field: high parts (FP32 layout), then low parts
struct DfSpinor {
    __device__ static void load(const void *base, size_t stride, size_t e, cx<df> v[12]) {
        const float4 *ph = static_cast<const float4 *>(base) + e;
        const float4 *pl = ph + 6 * stride;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 h = ld_nc(ph + k * stride), l = ld_nc(pl + k * stride);
            v[2 * k] = {{h.x, l.x}, {h.y, l.y}};
            v[2 * k + 1] = {{h.z, l.z}, {h.w, l.w}};
        }
    }
    __device__ static void store(void *base, size_t stride, size_t e, const cx<df> v[12]) {
        float4 *ph = static_cast<float4 *>(base) + e;
        float4 *pl = ph + 6 * stride;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            __stcs(ph + k * stride, make_float4(v[2 * k].re.hi, v[2 * k].im.hi, v[2 * k + 1].re.hi, v[2 * k + 1].im.hi));
            __stcs(pl + k * stride, make_float4(v[2 * k].re.lo, v[2 * k].im.lo, v[2 * k + 1].re.lo, v[2 * k + 1].im.lo));
        }
    }
};

__device__ __forceinline__ void load_link_df(const char *blk, int Vh, int i, cx<df> u[3][3]) {
    cx<float> h[3][3], l[3][3];
    Link<PLQ_F32, 18>::load(blk, Vh, i, h);
    Link<PLQ_F32, 18>::load(blk + (size_t)72 * Vh, Vh, i, l);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) u[a][b] = {{h[a][b].re, l[a][b].re}, {h[a][b].im, l[a][b].im}};
}

// uh = U h (DAG = false) or U^dagger h (DAG = true), two spin components
template <bool DAG>
__device__ __forceinline__ void su3_mul_df(const cx<df> u[3][3], const cx<df> h[6], cx<df> uh[6]) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dacc re, im;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const cx<df> m = DAG ? u[b][a] : u[a][b];
                const cx<df> v = h[3 * s + b];
                // U:        re = m.re v.re - m.im v.im,  im = m.re v.im + m.im v.re
                // U^dagger: re = m.re v.re + m.im v.im,  im = m.re v.im - m.im v.re
                const df mi = DAG ? -m.im : m.im;
                if (b == 0) {
                    re = dacc_prod(m.re, v.re);
                    im = dacc_prod(m.re, v.im);
                } else {
                    dacc_fma(re, m.re, v.re);
                    dacc_fma(im, m.re, v.im);
                }
                dacc_fma(re, -mi, v.im);
                dacc_fma(im, mi, v.re);
            }
            uh[3 * s + a] = {dacc_value(re), dacc_value(im)};
        }
}

// z * i^k for a run-time k (0..3): selects and sign flips only
__device__ __forceinline__ cx<df> mul_ipow_rt(cx<df> z, int k) {
    const bool sw = k & 1, neg_re = k == 1 || k == 2, neg_im = k >= 2;
    cx<df> w = {sw ? z.im : z.re, sw ? z.re : z.im};
    if (neg_re) w.re = -w.re;
    if (neg_im) w.im = -w.im;
    return w;
}

// Direction d = 2 mu + back, with everything that depends on it taken at run
// time: the float-float body is long, and one copy of it executed eight times
// per site keeps the kernel inside the instruction cache (eight unrolled
// copies do not fit, and the warps then stall on instruction fetch).
// Projection table of the chiral basis as in plq_hop_impl.cuh: spin pair
// (p0, p1) = (2, 3) for mu = 0, 3 and (3, 2) for mu = 1, 2; phases i^k0, i^k1
// of (1 - gamma_mu), with k + 2 for (1 + gamma_mu).
__device__ __forceinline__ void hop_dir_df(const DfArgs &a, const SiteGeom &g, int i, int r, int d, cx<df> acc[12]) {
    const Lattice &L = a.lat;
    const int n = a.nrhs;
    const size_t stride = (size_t)L.Vh * n;
    const int mu = d >> 1;
    const bool back = d & 1;
    const int st = lex_stride(L, mu);
    // selects, not run-time indexing (which would put the arrays in local memory)
    const int cm = mu == 0 ? g.c[0] : mu == 1 ? g.c[1] : mu == 2 ? g.c[2] : g.c[3];
    const int Lm = mu == 0 ? L.L[0] : mu == 1 ? L.L[1] : mu == 2 ? L.L[2] : L.L[3];
    int j;
    bool flip;
    if (!back) {
        j = ((cm == Lm - 1) ? g.lex - (Lm - 1) * st : g.lex + st) >> 1;
        flip = mu == 0 && cm == Lm - 1 && L.t_bc < 0;
    } else {
        j = ((cm == 0) ? g.lex + (Lm - 1) * st : g.lex - st) >> 1;
        flip = mu == 0 && cm == 0 && L.t_bc < 0;
    }
    const char *gbase = static_cast<const char *>(a.gauge);
    const int lpar = back ? 1 - a.out_parity : a.out_parity;
    cx<df> u[3][3];
    load_link_df(gbase + (size_t)(lpar * 4 + mu) * a.gblock, L.Vh, back ? j : i, u);
    if (back) {  // U^dagger
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int y = x; y < 3; ++y) {
                const cx<df> p = u[x][y], q = u[y][x];
                u[x][y] = {q.re, -q.im};
                u[y][x] = {p.re, -p.im};
            }
    }
    const bool p2 = mu == 0 || mu == 3;  // p0 = 2 (else 3)
    const int kb0 = mu == 1 || mu == 3 ? 1 : 0;
    const int kb1 = mu == 0 ? 0 : mu == 1 ? 1 : mu == 2 ? 2 : 3;
    const int k0 = (kb0 + (back ? 2 : 0)) & 3, k1 = (kb1 + (back ? 2 : 0)) & 3;
    cx<df> phi[12], h[6], uh[6];
    DfSpinor::load(a.in, stride, (size_t)j * n + r, phi);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<df> a0 = p2 ? phi[6 + c] : phi[9 + c], a1 = p2 ? phi[9 + c] : phi[6 + c];
        const cx<df> b0 = mul_ipow_rt(a0, k0), b1 = mul_ipow_rt(a1, k1);
        h[c] = {add_lazy(phi[c].re, b0.re), add_lazy(phi[c].im, b0.im)};
        h[3 + c] = {add_lazy(phi[3 + c].re, b1.re), add_lazy(phi[3 + c].im, b1.im)};
    }
    if (flip) {
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = {-h[k].re, -h[k].im};
    }
    su3_mul_df<false>(u, h, uh);
    // lower spins: component p_k gets conj(i^k) = i^(4 - k) times upper component k
    const int j0 = (4 - k0) & 3, j1 = (4 - k1) & 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        auto acc_add = [](cx<df> &a, cx<df> v) { a = {add_lazy(a.re, v.re), add_lazy(a.im, v.im)}; };
        acc_add(acc[c], uh[c]);
        acc_add(acc[3 + c], uh[3 + c]);
        const cx<df> l0 = mul_ipow_rt(uh[c], j0), l1 = mul_ipow_rt(uh[3 + c], j1);
        acc_add(acc[6 + c], p2 ? l0 : l1);
        acc_add(acc[9 + c], p2 ? l1 : l0);
    }
}

// one thread per (output site, right-hand side)
// (168 registers, no spills; capping them at 112 or 128 made it slower)
template <bool XPAY>
__global__ void __launch_bounds__(128) hop_df_kernel(const DfArgs a) {
    const int n = a.nrhs;
    const long long total = (long long)a.lat.Vh * n;
    const size_t stride = (size_t)total;
    const bool twist = a.nu_h != 0.0 || a.scale_h != 1.0;
    const df nu = df_from_double(a.nu_h), sc = df_from_double(a.scale_h), aa = df_from_double(a.a);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), r = (int)(e - (long long)i * n);
        const SiteGeom g = site_geom(a.lat, a.out_parity, i);
        cx<df> acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 1
        for (int d = 0; d < 8; ++d) hop_dir_df(a, g, i, r, d, acc);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {renorm(acc[k].re), renorm(acc[k].im)};
        if (twist) {  // scale * (1 + i g nu) acc, g = +1 (upper spins) / -1 (lower)
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const df gn = k < 6 ? nu : -nu;
                const cx<df> v = acc[k];
                acc[k] = {sc * (v.re - gn * v.im), sc * (v.im + gn * v.re)};
            }
        }
        if constexpr (XPAY) {
            cx<df> xv[12];
            DfSpinor::load(a.x, stride, (size_t)e, xv);
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = {xv[k].re + aa * acc[k].re, xv[k].im + aa * acc[k].im};
        }
        DfSpinor::store(a.out, stride, (size_t)e, acc);
    }
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

template <bool XPAY>
plq_status launch_df(const DfArgs &a, cudaStream_t s) {
    static std::atomic<int> per_sm{0};  // occupancy, filled on first use
    const int block = 128;
    if (per_sm.load(std::memory_order_relaxed) == 0) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, hop_df_kernel<XPAY>, block, 0);
        if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(hop_df)");
        per_sm.store(nb > 0 ? nb : 1, std::memory_order_relaxed);
    }
    const long long total = (long long)a.lat.Vh * a.nrhs;
    const long long want = (total + block - 1) / block, cap = (long long)per_sm.load(std::memory_order_relaxed) * sm_count();
    const int grid = (int)(want < cap ? want : cap);
    if (grid <= 0) return PLQ_OK;
    hop_df_kernel<XPAY><<<grid, block, 0, s>>>(a);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

// FP64 half field (12 planes of double2) <-> PLQ_DF64 half field, N elements
// (site * n + rhs); right-hand side r is scaled by 2^sh[r] on the way in and
// by 2^-sh[r] on the way out.
struct Shifts {
    int sh[PLQ_MAX_RHS];
};

// sh[r] by selects (run-time indexing would copy the array to local memory)
__device__ __forceinline__ int shift_of(const Shifts &S, long long e, int n) {
    if (n == 1) return S.sh[0];
    const int r = (int)(e % n);
    int v = S.sh[0];
#pragma unroll
    for (int q = 1; q < PLQ_MAX_RHS; ++q) v = r == q ? S.sh[q] : v;
    return v;
}

__global__ void split_kernel(long long N, int n, Shifts S, float4 *out, const double2 *in) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int es = shift_of(S, e, n);
        const double sc = __longlong_as_double((long long)(es + 1023) << 52);  // 2^es
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 a = in[(size_t)(2 * k) * N + e], b = in[(size_t)(2 * k + 1) * N + e];
            const df ar = df_from_double_bits(a.x, es, sc), ai = df_from_double_bits(a.y, es, sc),
                     br = df_from_double_bits(b.x, es, sc), bi = df_from_double_bits(b.y, es, sc);
            out[(size_t)k * N + e] = make_float4(ar.hi, ai.hi, br.hi, bi.hi);
            out[(size_t)(6 + k) * N + e] = make_float4(ar.lo, ai.lo, br.lo, bi.lo);
        }
    }
}

__global__ void join_kernel(long long N, int n, Shifts S, double2 *out, const float4 *in) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int es = -shift_of(S, e, n);
        const double sc = __longlong_as_double((long long)(es + 1023) << 52);  // 2^es
        // float -> double conversions are exact; one FP64 add and multiply each
        auto join = [sc](float h, float l) { return ((double)h + (double)l) * sc; };
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 h = in[(size_t)k * N + e], l = in[(size_t)(6 + k) * N + e];
            out[(size_t)(2 * k) * N + e] = make_double2(join(h.x, l.x), join(h.y, l.y));
            out[(size_t)(2 * k + 1) * N + e] = make_double2(join(h.z, l.z), join(h.w, l.w));
        }
    }
}

// canonical AoS FP64 (nrhs fields back to back) <-> packed full PLQ_DF64 field
__global__ void pack_df_kernel(Lattice L, int nrhs, char *out, const double *in, size_t half_bytes) {
    const long long per_par = (long long)L.Vh * nrhs, total = 2 * per_par;
    const size_t V = 2 * (size_t)L.Vh;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int par = (int)(idx / per_par);
        const long long e = idx - par * per_par;
        const int i = (int)(e / nrhs), r = (int)(e - (long long)i * nrhs);
        const SiteGeom g = site_geom(L, par, i);
        const double2 *src = reinterpret_cast<const double2 *>(in) + ((size_t)r * V + (size_t)g.lex) * 12;
        cx<df> v[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 z = src[k];
            v[k] = {df_from_double(z.x), df_from_double(z.y)};
        }
        DfSpinor::store(out + par * half_bytes, (size_t)per_par, (size_t)e, v);
    }
}

__global__ void unpack_df_kernel(Lattice L, int nrhs, double *out, const char *in, size_t half_bytes) {
    const long long per_par = (long long)L.Vh * nrhs, total = 2 * per_par;
    const size_t V = 2 * (size_t)L.Vh;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int par = (int)(idx / per_par);
        const long long e = idx - par * per_par;
        const int i = (int)(e / nrhs), r = (int)(e - (long long)i * nrhs);
        const SiteGeom g = site_geom(L, par, i);
        cx<df> v[12];
        DfSpinor::load(in + par * half_bytes, (size_t)per_par, (size_t)e, v);
        double2 *dst = reinterpret_cast<double2 *>(out) + ((size_t)r * V + (size_t)g.lex) * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = make_double2(df_to_double(v[k].re), df_to_double(v[k].im));
    }
}

// canonical AoS FP64 links -> 8 PLQ_DF64 blocks (high FP32-18 block, then low)
__global__ void pack_gauge_df_kernel(Lattice L, char *out, const double *in, size_t block) {
    const long long total = 2LL * L.Vh;
    const size_t Vh = (size_t)L.Vh;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int par = (int)(idx / L.Vh);
        const int i = (int)(idx - (long long)par * L.Vh);
        const SiteGeom g = site_geom(L, par, i);
        const double2 *src = reinterpret_cast<const double2 *>(in) + (size_t)g.lex * 36;
        for (int mu = 0; mu < 4; ++mu) {
            df re[9], im[9];
            for (int k = 0; k < 9; ++k) {
                const double2 z = src[9 * mu + k];
                re[k] = df_from_double(z.x);
                im[k] = df_from_double(z.y);
            }
            char *blk = out + (size_t)(par * 4 + mu) * block;
            for (int part = 0; part < 2; ++part) {
                float4 *p = reinterpret_cast<float4 *>(blk + part * 72 * Vh) + i;
                auto pick = [&](const df &d) { return part ? d.lo : d.hi; };
                for (int k = 0; k < 4; ++k)
                    p[k * Vh] = make_float4(pick(re[2 * k]), pick(im[2 * k]), pick(re[2 * k + 1]), pick(im[2 * k + 1]));
                float2 *q = reinterpret_cast<float2 *>(reinterpret_cast<float4 *>(blk + part * 72 * Vh) + 4 * Vh) + i;
                *q = make_float2(pick(re[8]), pick(im[8]));
            }
        }
    }
}

int grid_of(long long work, int block) {
    const long long want = (work + block - 1) / block, cap = (long long)sm_count() * 8;
    return (int)(want < cap ? want : cap);
}

}  // namespace

size_t df_site_bytes() { return 192; }

plq_status df_gauge_upload(plq_ctx *c, const double *U, int is_device, int link_reals, cudaStream_t s) {
    if (link_reals != 18) return set_error(PLQ_ERR_ARG, "PLQ_DF64 links are stored with 18 reals");
    const size_t V = 2 * (size_t)c->lat.Vh;
    const size_t canon = V * 72 * sizeof(double);
    const double *src = U;
    double *tmp = nullptr;
    if (!is_device) {
        PLQ_CUDA(cudaMalloc(&tmp, canon));
        cudaError_t e = cudaMemcpyAsync(tmp, U, canon, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_error(e, "gauge H2D copy");
        }
        src = tmp;
    }
    GaugeCopy &g = c->gauge_df;
    const size_t block = (size_t)144 * c->lat.Vh;
    plq_status st = PLQ_OK;
    if (!g.ptr) {
        cudaError_t e = cudaMalloc(&g.ptr, block * 8);
        if (e != cudaSuccess) {
            g.ptr = nullptr;
            st = cuda_error(e, "gauge allocation");
        }
    }
    if (st == PLQ_OK) {
        pack_gauge_df_kernel<<<grid_of(2LL * c->lat.Vh, 128), 128, 0, s>>>(c->lat, static_cast<char *>(g.ptr), src,
                                                                          block);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "gauge pack");
    }
    if (tmp) cudaFree(tmp);
    if (st != PLQ_OK) return st;
    g.reals = 18;
    g.block = block;
    return PLQ_OK;
}

plq_status df_pack_spinor(const Lattice &L, void *out, const double *in, int nrhs, cudaStream_t s) {
    const size_t half = df_site_bytes() * L.Vh * nrhs;
    pack_df_kernel<<<grid_of(2LL * L.Vh * nrhs, 256), 256, 0, s>>>(L, nrhs, static_cast<char *>(out), in, half);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status df_unpack_spinor(const Lattice &L, double *out, const void *in, int nrhs, cudaStream_t s) {
    const size_t half = df_site_bytes() * L.Vh * nrhs;
    unpack_df_kernel<<<grid_of(2LL * L.Vh * nrhs, 256), 256, 0, s>>>(L, nrhs, out, static_cast<const char *>(in),
                                                                      half);
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status df_split(long long N, int n, const int *shifts, void *out, const void *in, cudaStream_t s) {
    Shifts S{};
    for (int r = 0; r < n && r < PLQ_MAX_RHS; ++r) S.sh[r] = shifts ? shifts[r] : 0;
    split_kernel<<<grid_of(N, 256), 256, 0, s>>>(N, n, S, static_cast<float4 *>(out), static_cast<const double2 *>(in));
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status df_join(long long N, int n, const int *shifts, void *out, const void *in, cudaStream_t s) {
    Shifts S{};
    for (int r = 0; r < n && r < PLQ_MAX_RHS; ++r) S.sh[r] = shifts ? shifts[r] : 0;
    join_kernel<<<grid_of(N, 256), 256, 0, s>>>(N, n, S, static_cast<double2 *>(out), static_cast<const float4 *>(in));
    PLQ_CUDA(cudaGetLastError());
    return PLQ_OK;
}

plq_status df_hop(const plq_ctx *c, int out_parity, void *out, const void *in, const void *x, double a, double nu_h,
                  double scale_h, int nrhs, cudaStream_t s) {
    if (!c->gauge_df.ptr) return set_error(PLQ_ERR_STATE, "no PLQ_DF64 gauge copy (call plq_gauge_upload with PLQ_DF64)");
    DfArgs d;
    d.in = in;
    d.out = out;
    d.x = x;
    d.gauge = c->gauge_df.ptr;
    d.gblock = c->gauge_df.block;
    d.out_parity = out_parity;
    d.nrhs = nrhs;
    d.lat = c->lat;
    d.a = a;
    d.nu_h = nu_h;
    d.scale_h = scale_h;
    return x ? launch_df<true>(d, s) : launch_df<false>(d, s);
}

}  // namespace plq
