// Incremental EigCG (Sec. 3 of the paper: the deflation solver it added to
// tmLQCD; algorithm of Stathopoulos and Orginos, SIAM J. Sci. Comput. 32
// (2010) 439) on the even-odd normal equations A x_e = Mhat^dag bhat,
// A = Mhat^dag Mhat, in FP64.
//
// eigCG(nev, m): CG whose normalised residuals v_j = r_j / |r_j| (the Lanczos
// vectors of A) are kept in a search space V with the tridiagonal
//   T[j, j] = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T[j, j+1] = -sqrt(beta_j)/alpha_j
// built from the CG coefficients.  When V holds m vectors it is restarted
// with 2 nev Ritz vectors (the nev lowest of T and of its leading (m-1) block,
// orthonormalised, Rayleigh-Ritz on that space); at convergence the nev
// lowest Ritz vectors are added to a growing orthonormal deflation basis U
// with H = U^H A U.  Every solve starts from the Galerkin guess
// x0 = U H^{-1} U^H rhs ("init-CG").
//
// GPU mapping: the CG iterations are the fused kernels of the other solvers,
// captured in CUDA graphs; each iteration also copies r_{j+1} into its slot
// of V, and the device records alpha_j, beta_j, |r_{j+1}|^2, so the host
// builds T without stopping the GPU.  Restarts and Ritz extraction are a
// small dense eigenproblem on the host (Jacobi, at most m = 64) and one
// linear-combination kernel over V on the device; Gram-Schmidt and the
// projections onto U are multi-vector dot / axpy kernels.
//
// Precision.  The CG iterations, H = U^H A U, the Galerkin start and every
// residual are FP64.  The search space V (Lanczos vectors, restarts, Ritz
// vectors) and the Gram-Schmidt orthogonalisation of new basis vectors work
// on FP32 copies: they only shape the deflation subspace, whose Galerkin
// projection is exact for whatever vectors U holds (H is computed for those
// vectors), while in FP64 these dense multi-vector sweeps are bound by this
// GPU's FP64 FMA rate (~1/60 of FP32) and dominate the accumulation phase.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "plq_solver_common.cuh"

struct plq_eigcg {
    plq_ctx *ctx = nullptr;
    int nev = 10, m = 60, max_vectors = 300;
    int nvec = 0;                        // vectors in U
    double2 *U = nullptr;                // max_vectors slots (FP64)
    float2 *U32 = nullptr;               // the same vectors in FP32 (Gram-Schmidt)
    float2 *V = nullptr, *V2 = nullptr;  // m + 1 FP32 slots each (double buffer for restarts)
    double2 *work = nullptr;             // 4 slots: Aw, w, odd and even temporaries
    float2 *work32 = nullptr;            // 1 slot: w in FP32
    double *hist = nullptr;              // device history of CG coefficients
    int hist_cap = 0;
    double *coef = nullptr;              // device coefficient matrix (lincomb)
    std::vector<std::complex<double>> H; // U^H A U, row-major nvec x nvec (max_vectors^2)
    size_t slot = 0;                     // complex elements per slot: 12 * Vh
};

namespace plq {
namespace {

constexpr int kMaxM = 64;
constexpr int kDotChunk = 16;

// ---------------------------------------------------------------- host dense algebra
// Cyclic Jacobi eigendecomposition of a real symmetric n x n matrix A
// (row-major, destroyed).  w ascending, Z columns (row-major Z[i*n + j] =
// component i of eigenvector j).
void jacobi_eigh(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &Z) {
    Z.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double a = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += a;
                if (i != j) off += a;
            }
        if (off <= 1e-30 * (tot > 0 ? tot : 1.0)) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double zkp = Z[(size_t)k * n + p], zkq = Z[(size_t)k * n + q];
                    Z[(size_t)k * n + p] = c * zkp - s * zkq;
                    Z[(size_t)k * n + q] = s * zkp + c * zkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
    std::vector<double> Zs((size_t)n * n);
    w.resize(n);
    for (int j = 0; j < n; ++j) {
        w[j] = A[(size_t)idx[j] * n + idx[j]];
        for (int i = 0; i < n; ++i) Zs[(size_t)i * n + j] = Z[(size_t)i * n + idx[j]];
    }
    Z.swap(Zs);
}

// Orthonormalise the k columns of the m x k row-major matrix M (modified
// Gram-Schmidt, two passes).
void orthonormalize_columns(int m, int k, std::vector<double> &M) {
    for (int pass = 0; pass < 2; ++pass)
        for (int j = 0; j < k; ++j) {
            for (int i = 0; i < j; ++i) {
                double d = 0.0;
                for (int r = 0; r < m; ++r) d += M[(size_t)r * k + i] * M[(size_t)r * k + j];
                for (int r = 0; r < m; ++r) M[(size_t)r * k + j] -= d * M[(size_t)r * k + i];
            }
            double nrm = 0.0;
            for (int r = 0; r < m; ++r) nrm += M[(size_t)r * k + j] * M[(size_t)r * k + j];
            nrm = std::sqrt(nrm);
            for (int r = 0; r < m; ++r) M[(size_t)r * k + j] = nrm > 0 ? M[(size_t)r * k + j] / nrm : 0.0;
        }
}

// Solve H y = g for Hermitian positive definite H (n x n row-major) by Cholesky.
bool chol_solve(int n, const std::vector<std::complex<double>> &Hm, int ld, std::vector<std::complex<double>> &y) {
    using C = std::complex<double>;
    std::vector<C> L((size_t)n * n, C(0, 0));
    for (int j = 0; j < n; ++j) {
        double d = std::real(Hm[(size_t)j * ld + j]);
        for (int k = 0; k < j; ++k) d -= std::norm(L[(size_t)j * n + k]);
        if (!(d > 0)) return false;
        const double ljj = std::sqrt(d);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            C s = Hm[(size_t)i * ld + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * std::conj(L[(size_t)j * n + k]);
            L[(size_t)i * n + j] = s / ljj;
        }
    }
    for (int i = 0; i < n; ++i) {  // L z = g
        C s = y[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
        y[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // L^H y = z
        C s = y[i];
        for (int k = i + 1; k < n; ++k) s -= std::conj(L[(size_t)k * n + i]) * y[k];
        y[i] = s / std::real(L[(size_t)i * n + i]);
    }
    return true;
}

// ---------------------------------------------------------------- device kernels
int grid_of(long long work, bool reduce) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (work + 255) / 256, cap = (long long)sms * 8;
    if (reduce && cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

// out_l = sum_i C[i*k + l] * in_i  for l < k (real coefficients; FP32 slots `stride` apart)
__global__ void lincomb32_kernel(long long N, const float2 *in, size_t stride, int m, const float *C, int k,
                                 float2 *out, size_t out_stride) {
    __shared__ float Cs[kMaxM * 24];
    for (int t = threadIdx.x; t < m * k; t += blockDim.x) Cs[t] = C[t];
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        float2 acc[24];
#pragma unroll
        for (int l = 0; l < 24; ++l) acc[l] = make_float2(0.f, 0.f);
        for (int i = 0; i < m; ++i) {
            const float2 v = __ldg(in + i * stride + e);
#pragma unroll
            for (int l = 0; l < 24; ++l)
                if (l < k) {
                    acc[l].x = fmaf(Cs[i * k + l], v.x, acc[l].x);
                    acc[l].y = fmaf(Cs[i * k + l], v.y, acc[l].y);
                }
        }
#pragma unroll
        for (int l = 0; l < 24; ++l)
            if (l < k) out[l * out_stride + e] = acc[l];
    }
}

// out = f * in in FP32 (f a power of two that brings the field into the FP32
// exponent range)
__global__ void to32_kernel(long long N, float2 *out, const double2 *in, double f) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const double2 a = in[e];
        out[e] = make_float2((float)(f * a.x), (float)(f * a.y));
    }
}

__global__ void to64_kernel(long long N, double2 *out, const float2 *in) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const float2 a = in[e];
        out[e] = make_double2((double)a.x, (double)a.y);
    }
}

// out = base + sum_i c_i in_i over FP32 slots (complex coefficients; base may alias out)
__global__ void zlincomb32_kernel(long long N, const float2 *in, size_t stride, int m, const double2 *c,
                                  const float2 *base, float2 *out) {
    __shared__ float2 cs[kDotChunk];
    for (int t = threadIdx.x; t < m; t += blockDim.x) cs[t] = make_float2((float)c[t].x, (float)c[t].y);
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        float2 a = base ? base[e] : make_float2(0.f, 0.f);
        for (int i = 0; i < m; ++i) {
            const float2 v = __ldg(in + i * stride + e), w = cs[i];
            a.x = fmaf(w.x, v.x, fmaf(-w.y, v.y, a.x));
            a.y = fmaf(w.x, v.y, fmaf(w.y, v.x, a.y));
        }
        out[e] = a;
    }
}

// d_i = <u_i, w> for i < cnt (<= kDotChunk), FP32 slots; per-thread FP32 partial
// sums (a handful of elements each), FP64 across threads and blocks
__global__ void multidot32_kernel(long long N, const float2 *U, size_t stride, int cnt, const float2 *w, Reduce red) {
    RedAcc<2 * kDotChunk> acc;
    red_init(acc);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const float2 b = w[e];
        for (int i = 0; i < cnt; ++i) {
            const float2 a = __ldg(U + i * stride + e);
            acc.v[2 * i][0] += a.x * b.x + a.y * b.y;
            acc.v[2 * i + 1][0] += a.x * b.y - a.y * b.x;
        }
    }
    grid_reduce(red, acc, 1);
}

__global__ void scale32_kernel(long long N, float2 *v, float s) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const float2 a = v[e];
        v[e] = make_float2(s * a.x, s * a.y);
    }
}

// out = base + sum_i c_i in_i (complex coefficients; base may alias out)
__global__ void zlincomb_kernel(long long N, const double2 *in, size_t stride, int m, const double2 *c,
                                const double2 *base, double2 *out) {
    __shared__ double2 cs[kDotChunk];
    for (int t = threadIdx.x; t < m; t += blockDim.x) cs[t] = c[t];
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        double2 a = base ? base[e] : make_double2(0.0, 0.0);
        for (int i = 0; i < m; ++i) {
            const double2 v = __ldg(in + i * stride + e), w = cs[i];
            a.x = fma(w.x, v.x, fma(-w.y, v.y, a.x));
            a.y = fma(w.x, v.y, fma(w.y, v.x, a.y));
        }
        out[e] = a;
    }
}

// d_i = <u_i, w> for i < cnt (<= kDotChunk)
__global__ void multidot_kernel(long long N, const double2 *U, size_t stride, int cnt, const double2 *w, Reduce red) {
    RedAcc<2 * kDotChunk> acc;
    red_init(acc);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const double2 b = w[e];
        for (int i = 0; i < cnt; ++i) {
            const double2 a = __ldg(U + i * stride + e);
            acc.v[2 * i][0] += a.x * b.x + a.y * b.y;
            acc.v[2 * i + 1][0] += a.x * b.y - a.y * b.x;
        }
    }
    grid_reduce(red, acc, 1);
}

struct Eig {
    plq_eigcg *E;
    Solve S;
    long long N;  // complex elements of a half field
};

plq_status dots(Eig &G, const double2 *Ubase, int cnt, const double2 *w, std::vector<std::complex<double>> &d) {
    d.assign(cnt, {0, 0});
    for (int c0 = 0; c0 < cnt; c0 += kDotChunk) {
        const int c = std::min(kDotChunk, cnt - c0);
        Reduce r = reduce_of(G.S.c, FIN_NONE);
        r.st = nullptr;
        multidot_kernel<<<grid_of(G.N, true), 256, 0, G.S.s>>>(G.N, Ubase + c0 * G.E->slot, G.E->slot, c, w, r);
        PLQ_CUDA(cudaGetLastError());
        double buf[2 * kDotChunk];
        PLQ_TRY(read_sums(G.S, buf, 2 * c));
        for (int i = 0; i < c; ++i) d[c0 + i] = {buf[2 * i], buf[2 * i + 1]};
    }
    return PLQ_OK;
}

// out = base + sum_i c_i U_i, in chunks
plq_status zcomb(Eig &G, const double2 *Ubase, const std::vector<std::complex<double>> &c, const double2 *base,
                 double2 *out) {
    const int cnt = (int)c.size();
    if (cnt == 0) {
        if (base != out) PLQ_CUDA(cudaMemcpyAsync(out, base, G.N * sizeof(double2), cudaMemcpyDeviceToDevice, G.S.s));
        return PLQ_OK;
    }
    double2 *cdev = reinterpret_cast<double2 *>(G.E->coef);
    for (int c0 = 0; c0 < cnt; c0 += kDotChunk) {
        const int k = std::min(kDotChunk, cnt - c0);
        PLQ_CUDA(cudaMemcpyAsync(cdev, c.data() + c0, k * sizeof(double2), cudaMemcpyHostToDevice, G.S.s));
        zlincomb_kernel<<<grid_of(G.N, false), 256, 0, G.S.s>>>(G.N, Ubase + c0 * G.E->slot, G.E->slot, k, cdev,
                                                                c0 == 0 ? base : out, out);
        PLQ_CUDA(cudaGetLastError());
        PLQ_CUDA(cudaStreamSynchronize(G.S.s));  // cdev is reused by the next chunk
    }
    return PLQ_OK;
}

plq_status dots32(Eig &G, const float2 *Ubase, int cnt, const float2 *w, std::vector<std::complex<double>> &d) {
    d.assign(cnt, {0, 0});
    for (int c0 = 0; c0 < cnt; c0 += kDotChunk) {
        const int c = std::min(kDotChunk, cnt - c0);
        Reduce r = reduce_of(G.S.c, FIN_NONE);
        r.st = nullptr;
        multidot32_kernel<<<grid_of(G.N, true), 256, 0, G.S.s>>>(G.N, Ubase + c0 * G.E->slot, G.E->slot, c, w, r);
        PLQ_CUDA(cudaGetLastError());
        double buf[2 * kDotChunk];
        PLQ_TRY(read_sums(G.S, buf, 2 * c));
        for (int i = 0; i < c; ++i) d[c0 + i] = {buf[2 * i], buf[2 * i + 1]};
    }
    return PLQ_OK;
}

// w += sum_i c_i U32_i, in chunks (FP32)
plq_status zcomb32(Eig &G, const float2 *Ubase, const std::vector<std::complex<double>> &c, float2 *w) {
    const int cnt = (int)c.size();
    double2 *cdev = reinterpret_cast<double2 *>(G.E->coef);
    for (int c0 = 0; c0 < cnt; c0 += kDotChunk) {
        const int k = std::min(kDotChunk, cnt - c0);
        PLQ_CUDA(cudaMemcpyAsync(cdev, c.data() + c0, k * sizeof(double2), cudaMemcpyHostToDevice, G.S.s));
        zlincomb32_kernel<<<grid_of(G.N, false), 256, 0, G.S.s>>>(G.N, Ubase + c0 * G.E->slot, G.E->slot, k, cdev,
                                                                  w, w);
        PLQ_CUDA(cudaGetLastError());
        PLQ_CUDA(cudaStreamSynchronize(G.S.s));  // cdev is reused by the next chunk
    }
    return PLQ_OK;
}

// out_l = sum_i C[i*k + l] in_i over FP32 slots (real, k <= 24, m <= kMaxM)
plq_status rcomb(Eig &G, const float2 *in, int m, const std::vector<double> &C, int k, float2 *out) {
    std::vector<float> Cf(C.begin(), C.begin() + (size_t)m * k);
    float *cdev = reinterpret_cast<float *>(G.E->coef);
    PLQ_CUDA(cudaMemcpyAsync(cdev, Cf.data(), sizeof(float) * m * k, cudaMemcpyHostToDevice, G.S.s));
    lincomb32_kernel<<<grid_of(G.N, false), 256, 0, G.S.s>>>(G.N, in, G.E->slot, m, cdev, k, out, G.E->slot);
    PLQ_CUDA(cudaGetLastError());
    PLQ_CUDA(cudaStreamSynchronize(G.S.s));
    return PLQ_OK;
}

// y = A v with A = Mhat^dag Mhat (FP64); tmp_o: odd half field, tmp_e: even
plq_status apply_A(Eig &G, double2 *y, const double2 *v, void *tmp_o, void *tmp_e) {
    const double kk = G.S.kappa * G.S.kappa;
    PLQ_TRY(hop(G.S, PLQ_F64, 1, tmp_o, v, EPI_PLAIN, 0, nullptr, 0.0));
    PLQ_TRY(hop(G.S, PLQ_F64, 0, tmp_e, tmp_o, EPI_XPAY, 0, v, -kk));
    PLQ_TRY(hop(G.S, PLQ_F64, 1, tmp_o, tmp_e, EPI_PLAIN, 1, nullptr, 0.0));
    return hop(G.S, PLQ_F64, 0, y, tmp_o, EPI_XPAY, 1, tmp_e, -kk);
}

// Add the vectors w (FP32, in the slots of `src`, count cnt) to the deflation
// basis: classical Gram-Schmidt twice against U in FP32, normalisation, then
// the new row and column of H = U^H A U in FP64 for the FP64 copy of w.
plq_status add_to_basis(Eig &G, const float2 *src, int cnt, void *tmp_o, void *tmp_e) {
    plq_eigcg *E = G.E;
    double2 *Aw = E->work, *w = E->work + E->slot;
    float2 *w32 = E->work32;
    for (int q = 0; q < cnt && E->nvec < E->max_vectors; ++q) {
        PLQ_CUDA(cudaMemcpyAsync(w32, src + q * E->slot, G.N * sizeof(float2), cudaMemcpyDeviceToDevice, G.S.s));
        std::vector<std::complex<double>> d;
        for (int pass = 0; pass < 2 && E->nvec > 0; ++pass) {  // classical Gram-Schmidt, twice
            PLQ_TRY(dots32(G, E->U32, E->nvec, w32, d));
            for (auto &z : d) z = -z;
            PLQ_TRY(zcomb32(G, E->U32, d, w32));
        }
        std::vector<std::complex<double>> nn;
        PLQ_TRY(dots32(G, w32, 1, w32, nn));
        const double n2 = std::real(nn[0]);
        if (!(n2 > 1e-20)) continue;  // linearly dependent: skip
        scale32_kernel<<<grid_of(G.N, false), 256, 0, G.S.s>>>(G.N, w32, (float)(1.0 / std::sqrt(n2)));
        PLQ_CUDA(cudaGetLastError());
        to64_kernel<<<grid_of(G.N, false), 256, 0, G.S.s>>>(G.N, w, w32);
        PLQ_CUDA(cudaGetLastError());
        PLQ_TRY(apply_A(G, Aw, w, tmp_o, tmp_e));
        std::vector<std::complex<double>> col;
        PLQ_TRY(dots(G, E->U, E->nvec, Aw, col));
        std::vector<std::complex<double>> self;
        PLQ_TRY(dots(G, w, 1, Aw, self));
        const int k = E->nvec, ld = E->max_vectors;
        for (int i = 0; i < k; ++i) {
            E->H[(size_t)i * ld + k] = col[i];
            E->H[(size_t)k * ld + i] = std::conj(col[i]);
        }
        E->H[(size_t)k * ld + k] = std::real(self[0]);
        PLQ_CUDA(cudaMemcpyAsync(E->U + k * E->slot, w, G.N * sizeof(double2), cudaMemcpyDeviceToDevice, G.S.s));
        PLQ_CUDA(cudaMemcpyAsync(E->U32 + k * E->slot, w32, G.N * sizeof(float2), cudaMemcpyDeviceToDevice, G.S.s));
        E->nvec += 1;
    }
    PLQ_CUDA(cudaStreamSynchronize(G.S.s));
    return PLQ_OK;
}

}  // namespace
}  // namespace plq

using namespace plq;

extern "C" plq_status plq_eigcg_create(plq_ctx *ctx, int nev, int m, int max_vectors, plq_eigcg **out) {
    if (!ctx || !out) return set_error(PLQ_ERR_ARG, "null argument");
    *out = nullptr;
    if (nev < 1 || m < 2 * nev + 2 || m > kMaxM || 2 * nev > 24)
        return set_error(PLQ_ERR_ARG, "need 1 <= nev, 2*nev <= 24 and 2*nev + 2 <= m <= %d", kMaxM);
    if (max_vectors < nev) return set_error(PLQ_ERR_ARG, "max_vectors must be >= nev");
    PLQ_CUDA(cudaSetDevice(ctx->device));
    plq_eigcg *E = new plq_eigcg();
    E->ctx = ctx;
    E->nev = nev;
    E->m = m;
    E->max_vectors = max_vectors;
    E->slot = 12 * (size_t)ctx->lat.Vh;
    const size_t sb = E->slot * sizeof(double2), sb32 = E->slot * sizeof(float2);
    E->hist_cap = 1 << 16;
    cudaError_t e = cudaMalloc(&E->U, sb * max_vectors);
    if (e == cudaSuccess) e = cudaMalloc(&E->U32, sb32 * max_vectors);
    if (e == cudaSuccess) e = cudaMalloc(&E->V, sb32 * (m + 1));
    if (e == cudaSuccess) e = cudaMalloc(&E->V2, sb32 * (m + 1));
    if (e == cudaSuccess) e = cudaMalloc(&E->work, sb * 4);
    if (e == cudaSuccess) e = cudaMalloc(&E->work32, sb32);
    if (e == cudaSuccess) e = cudaMalloc(&E->hist, sizeof(double) * 3 * E->hist_cap);
    if (e == cudaSuccess) e = cudaMalloc(&E->coef, sizeof(double) * kMaxM * 24 * 2);
    if (e != cudaSuccess) {
        plq_status st = cuda_error(e, "EigCG allocation (U holds max_vectors half fields)");
        plq_eigcg_destroy(E);
        return st;
    }
    E->H.assign((size_t)max_vectors * max_vectors, {0, 0});
    *out = E;
    return PLQ_OK;
}

extern "C" plq_status plq_eigcg_destroy(plq_eigcg *E) {
    if (!E) return PLQ_OK;
    cudaSetDevice(E->ctx->device);
    cudaDeviceSynchronize();
    for (void *p : {(void *)E->U, (void *)E->U32, (void *)E->V, (void *)E->V2, (void *)E->work, (void *)E->work32,
                    (void *)E->hist, (void *)E->coef})
        if (p) cudaFree(p);
    delete E;
    return PLQ_OK;
}

extern "C" int plq_eigcg_vectors(const plq_eigcg *E) { return E ? E->nvec : 0; }

extern "C" int plq_eigcg_projected_matrix(const plq_eigcg *E, double *H, int ld) {
    if (!E) {
        set_error(PLQ_ERR_ARG, "null eigcg handle");
        return -1;
    }
    const int k = E->nvec;
    if (!H) return k;
    if (ld < k) {
        set_error(PLQ_ERR_ARG, "leading dimension %d below the %d basis vectors", ld, k);
        return -1;
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            const std::complex<double> h = E->H[(size_t)i * E->max_vectors + j];
            H[2 * ((size_t)i * ld + j)] = h.real();
            H[2 * ((size_t)i * ld + j) + 1] = h.imag();
        }
    return k;
}

extern "C" plq_status plq_eigcg_solve(plq_eigcg *E, void *x, const void *b, double kappa,
                                      const plq_solver_params *params, int accumulate, plq_solve_info *info,
                                      void *stream) {
    if (info) std::memset(info, 0, sizeof(*info));
    if (!E) return set_error(PLQ_ERR_ARG, "null EigCG handle");
    plq_ctx *c = E->ctx;
    if (!x || !b || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(b) & 15))
        return set_error(PLQ_ERR_ARG, "null or misaligned field pointer");
    if (!c->gauge[PLQ_F64].ptr) return set_error(PLQ_ERR_STATE, "EigCG needs the FP64 gauge copy");
    const double tol = (params && params->tol > 0) ? params->tol : 1e-8;
    const int maxit = (params && params->maxit > 0) ? params->maxit : 20000;
    PLQ_CUDA(cudaSetDevice(c->device));
    Eig G;
    G.E = E;
    G.S.c = c;
    G.S.Vh = c->lat.Vh;
    G.S.n = 1;
    G.S.N = G.S.Vh;
    G.S.kappa = kappa;
    G.S.P = G.S.PX = PLQ_F64;
    G.N = (long long)E->slot;
    const size_t h64 = spinor_site_bytes(PLQ_F64) * (size_t)G.S.Vh;
    PLQ_TRY(ensure_work(c, 6 * h64 + 4096));
    char *w = static_cast<char *>(c->work);
    void *bhat = w, *rhs = w + h64, *r = w + 2 * h64, *p = w + 3 * h64, *q = w + 4 * h64, *mp = w + 5 * h64;
    void *to = E->work + 2 * E->slot;  // odd temporary (also used by apply_A)
    void *te = E->work + 3 * E->slot;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t s = nullptr;
    PLQ_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    G.S.s = s;
    cudaEvent_t ev = nullptr;
    cudaEventCreate(&ev);
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(s, ev, 0);
    auto wall0 = std::chrono::steady_clock::now();
    const char *be = static_cast<const char *>(b), *bo = be + h64;
    char *xe = static_cast<char *>(x), *xo = xe + h64;
    plq_status st = PLQ_OK, result = PLQ_OK;
    int iters = 0;
    double true_rel = 0.0;
    const double kk = kappa * kappa;
    do {
        // rhs = Mhat^dag bhat, bhat = b_e + kappa H_eo b_o
        if ((st = hop(G.S, PLQ_F64, 0, bhat, bo, EPI_XPAY, 0, be, kappa)) != PLQ_OK) break;
        if ((st = hop(G.S, PLQ_F64, 1, to, bhat, EPI_PLAIN, 1, nullptr, 0.0)) != PLQ_OK) break;
        if ((st = hop(G.S, PLQ_F64, 0, rhs, to, EPI_XPAY, 1, bhat, -kk)) != PLQ_OK) break;
        double rhs2 = 0;
        if ((st = norm2_64(G.S, rhs, &rhs2)) != PLQ_OK) break;
        // init-CG: x0 = U H^{-1} U^H rhs
        if (E->nvec > 0) {
            std::vector<std::complex<double>> y;
            if ((st = dots(G, E->U, E->nvec, static_cast<const double2 *>(rhs), y)) != PLQ_OK) break;
            if (!chol_solve(E->nvec, E->H, E->max_vectors, y)) {
                st = set_error(PLQ_ERR_STATE, "deflation matrix U^H A U is not positive definite");
                break;
            }
            if ((st = zcomb(G, E->U, y, nullptr, static_cast<double2 *>(static_cast<void *>(xe)))) != PLQ_OK) break;
        } else if ((st = blas_zero(G.S.N, xe, PLQ_F64, s)) != PLQ_OK) {
            break;
        }
        // r = rhs - A x0, p = r
        if ((st = apply_A(G, static_cast<double2 *>(q), static_cast<const double2 *>(static_cast<void *>(xe)), to, te)) !=
            PLQ_OK)
            break;
        if ((st = blas_copy_convert(G.S.N, r, PLQ_F64, q, PLQ_F64, s)) != PLQ_OK) break;
        if ((st = blas_xpay64(G.S.N, rhs, -1.0, r, s)) != PLQ_OK) break;
        if ((st = blas_copy_convert(G.S.N, p, PLQ_F64, r, PLQ_F64, s)) != PLQ_OK) break;
        double rho0 = 0;
        if ((st = norm2_64(G.S, r, &rho0)) != PLQ_OK) break;
        const bool eig = accumulate && E->nvec < E->max_vectors;
        // the raw residuals r_j go into the FP32 search space scaled by 2^-(exponent
        // of |r_0|) (and their norms in nrm with them), whatever the source magnitude
        const double vscale = rho0 > 0.0 && std::isfinite(rho0) ? std::ldexp(1.0, -std::ilogb(std::sqrt(rho0))) : 1.0;
        const int m = E->m, nev = E->nev, k2 = 2 * nev;
        // search space bookkeeping (host): raw vectors in V, their norms, T
        std::vector<double> T((size_t)(m + 1) * (m + 1), 0.0), nrm(m + 1, 1.0);
        int vs = 1;  // V slot 0 holds r_0 (raw)
        if (eig) {
            to32_kernel<<<grid_of(G.N, false), 256, 0, s>>>(G.N, E->V, static_cast<const double2 *>(r), vscale);
            PLQ_CUDA(cudaGetLastError());
            nrm[0] = vscale * std::sqrt(rho0);
        }
        double alpha_prev = 0, beta_prev = 0;
        bool have_prev = false;
        SolverState init;
        std::memset(&init, 0, sizeof init);
        init.rho = rho0;
        init.stop_r2 = tol * tol * rhs2;
        init.maxit = maxit;
        init.hist = E->hist;
        init.hist_cap = E->hist_cap;
        std::vector<SolverState> cur(1);
        bool converged = rho0 <= init.stop_r2;
        int ritz_k = 0;  // complete vectors in V at the end
        while (!converged && iters < maxit && st == PLQ_OK) {
            init.iter = iters;
            std::vector<SolverState> sv(1, init);
            if ((st = put_states(G.S, sv)) != PLQ_OK) break;
            const int L = eig ? (m - vs + 1) : 16;
            float2 *Vb = E->V;
            auto body = [&](int i) -> plq_status {
                PLQ_TRY(hop(G.S, PLQ_F64, 1, to, p, EPI_PLAIN, 0, nullptr, 0.0, FIN_NONE, nullptr, true));
                PLQ_TRY(hop(G.S, PLQ_F64, 0, mp, to, EPI_XPAY_NORM, 0, p, -kk, FIN_CG_ALPHA, nullptr, true));
                PLQ_TRY(hop(G.S, PLQ_F64, 1, to, mp, EPI_PLAIN, 1, nullptr, 0.0, FIN_NONE, nullptr, true));
                PLQ_TRY(hop(G.S, PLQ_F64, 0, q, to, EPI_XPAY, 1, mp, -kk, FIN_NONE, nullptr, true));
                Reduce rb = reduce_of(c, FIN_CG_BETA);
                PLQ_TRY(blas_cg_update(G.S.N, 1, xe, r, p, q, PLQ_F64, rb, c->state, s));
                if (eig) {  // raw r_{j+1} into its (FP32) slot of the search space
                    to32_kernel<<<grid_of(G.N, false), 256, 0, s>>>(G.N, Vb + (size_t)(vs + i) * E->slot,
                                                                    static_cast<const double2 *>(r), vscale);
                    PLQ_CUDA(cudaGetLastError());
                }
                return blas_cg_direction(G.S.N, 1, p, r, PLQ_F64, c->state, s);
            };
            // one graph of exactly L iterations (the ones that fill V)
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            PLQ_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            for (int i = 0; i < L && st == PLQ_OK; ++i) st = body(i);
            cudaError_t ce = cudaStreamEndCapture(s, &graph);
            if (st != PLQ_OK) {
                if (graph) cudaGraphDestroy(graph);
                break;
            }
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, s);
            if (exec) cudaGraphExecDestroy(exec);
            if (ce != cudaSuccess) {
                st = cuda_error(ce, "EigCG iteration graph");
                break;
            }
            if ((st = get_states(G.S, cur)) != PLQ_OK) break;
            const int done = cur[0].iter - iters;
            if (cur[0].flags & FLAG_NAN) {
                result = set_error(PLQ_ERR_NAN, "NaN in EigCG");
                break;
            }
            std::vector<double> h(3 * (size_t)done);
            if (done > 0)
                PLQ_CUDA(cudaMemcpy(h.data(), E->hist + 3 * (size_t)iters, sizeof(double) * 3 * done,
                                    cudaMemcpyDeviceToHost));
            converged = cur[0].rho <= init.stop_r2;
            if (eig) {
                for (int t = 0; t < done; ++t) {
                    const double al = h[3 * t], be2 = h[3 * t + 1], rn = h[3 * t + 2];
                    const int sl = vs - 1 + t;
                    T[(size_t)sl * (m + 1) + sl] = 1.0 / al + (have_prev ? beta_prev / alpha_prev : 0.0);
                    const double off = -std::sqrt(be2) / al;
                    if (sl + 1 <= m) {
                        T[(size_t)sl * (m + 1) + sl + 1] = off;
                        T[(size_t)(sl + 1) * (m + 1) + sl] = off;
                        nrm[sl + 1] = vscale * std::sqrt(rn);
                    }
                    alpha_prev = al;
                    beta_prev = be2;
                    have_prev = true;
                }
                ritz_k = vs - 1 + done;  // complete vectors
                if (!converged && ritz_k == m && iters + done < maxit) {
                    // restart with 2 nev Ritz vectors
                    std::vector<double> Tm((size_t)m * m);
                    for (int i2 = 0; i2 < m; ++i2)
                        for (int j2 = 0; j2 < m; ++j2) Tm[(size_t)i2 * m + j2] = T[(size_t)i2 * (m + 1) + j2];
                    std::vector<double> wv, Y, w2, Y2;
                    jacobi_eigh(m, Tm, wv, Y);
                    std::vector<double> Tm1((size_t)(m - 1) * (m - 1));
                    for (int i2 = 0; i2 < m - 1; ++i2)
                        for (int j2 = 0; j2 < m - 1; ++j2) Tm1[(size_t)i2 * (m - 1) + j2] = Tm[(size_t)i2 * m + j2];
                    jacobi_eigh(m - 1, Tm1, w2, Y2);
                    std::vector<double> Qm((size_t)m * k2, 0.0);
                    for (int i2 = 0; i2 < m; ++i2)
                        for (int l = 0; l < nev; ++l) {
                            Qm[(size_t)i2 * k2 + l] = Y[(size_t)i2 * m + l];
                            Qm[(size_t)i2 * k2 + nev + l] = i2 < m - 1 ? Y2[(size_t)i2 * (m - 1) + l] : 0.0;
                        }
                    orthonormalize_columns(m, k2, Qm);
                    std::vector<double> Hq((size_t)k2 * k2, 0.0), TQ((size_t)m * k2, 0.0);
                    for (int i2 = 0; i2 < m; ++i2)
                        for (int l = 0; l < k2; ++l) {
                            double sacc = 0;
                            for (int j2 = 0; j2 < m; ++j2) sacc += Tm[(size_t)i2 * m + j2] * Qm[(size_t)j2 * k2 + l];
                            TQ[(size_t)i2 * k2 + l] = sacc;
                        }
                    for (int a2 = 0; a2 < k2; ++a2)
                        for (int b2 = 0; b2 < k2; ++b2) {
                            double sacc = 0;
                            for (int i2 = 0; i2 < m; ++i2) sacc += Qm[(size_t)i2 * k2 + a2] * TQ[(size_t)i2 * k2 + b2];
                            Hq[(size_t)a2 * k2 + b2] = sacc;
                        }
                    std::vector<double> Mv, Z;
                    jacobi_eigh(k2, Hq, Mv, Z);
                    std::vector<double> QZ((size_t)m * k2, 0.0), C((size_t)m * k2);
                    for (int i2 = 0; i2 < m; ++i2)
                        for (int l = 0; l < k2; ++l) {
                            double sacc = 0;
                            for (int j2 = 0; j2 < k2; ++j2) sacc += Qm[(size_t)i2 * k2 + j2] * Z[(size_t)j2 * k2 + l];
                            QZ[(size_t)i2 * k2 + l] = sacc;
                            C[(size_t)i2 * k2 + l] = sacc / nrm[i2];  // raw slots -> normalised V
                        }
                    if ((st = rcomb(G, E->V, m, C, k2, E->V2)) != PLQ_OK) break;
                    PLQ_CUDA(cudaMemcpyAsync(E->V2 + (size_t)k2 * E->slot, E->V + (size_t)m * E->slot,
                                             G.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
                    std::swap(E->V, E->V2);
                    const double tlast = -std::sqrt(beta_prev) / alpha_prev;
                    std::fill(T.begin(), T.end(), 0.0);
                    for (int l = 0; l < k2; ++l) {
                        T[(size_t)l * (m + 1) + l] = Mv[l];
                        const double cpl = tlast * QZ[(size_t)(m - 1) * k2 + l];
                        T[(size_t)k2 * (m + 1) + l] = cpl;
                        T[(size_t)l * (m + 1) + k2] = cpl;
                        nrm[l] = 1.0;
                    }
                    nrm[k2] = nrm[m];
                    vs = k2 + 1;
                } else {
                    vs = ritz_k + 1;
                }
            }
            iters += done;
            init.rho = cur[0].rho;  // the next batch continues the recurrence
            if (done == 0) break;
        }
        if (st != PLQ_OK || result != PLQ_OK) break;
        // Ritz vectors of the final space -> deflation basis
        if (eig && ritz_k >= nev) {
            const int K = std::min(ritz_k, m);
            std::vector<double> TK((size_t)K * K);
            for (int i2 = 0; i2 < K; ++i2)
                for (int j2 = 0; j2 < K; ++j2) TK[(size_t)i2 * K + j2] = T[(size_t)i2 * (m + 1) + j2];
            std::vector<double> wv, Y;
            jacobi_eigh(K, TK, wv, Y);
            std::vector<double> C((size_t)K * nev);
            for (int i2 = 0; i2 < K; ++i2)
                for (int l = 0; l < nev; ++l) C[(size_t)i2 * nev + l] = Y[(size_t)i2 * K + l] / nrm[i2];
            if ((st = rcomb(G, E->V, K, C, nev, E->V2)) != PLQ_OK) break;
            if ((st = add_to_basis(G, E->V2, nev, to, te)) != PLQ_OK) break;
        }
        // x_o and the true residual with the FP64 operator
        if ((st = hop(G.S, PLQ_F64, 1, xo, xe, EPI_XPAY, 0, bo, kappa)) != PLQ_OK) break;
        double r2 = 0, b2 = 0;
        if ((st = wilson_residual64(c, kappa, x, b, &r2, &b2, s)) != PLQ_OK) break;
        true_rel = b2 > 0 ? std::sqrt(r2 / b2) : 0.0;
        if (!converged) result = set_error(PLQ_ERR_NOT_CONVERGED, "EigCG: no convergence in %d iterations", iters);
    } while (0);
    cudaEventRecord(ev, s);
    cudaStreamWaitEvent(user, ev, 0);
    cudaStreamSynchronize(s);
    cudaEventDestroy(ev);
    cudaStreamDestroy(s);
    const int status = st != PLQ_OK ? st : result;
    if (info) {
        info->status = status;
        info->iterations = iters;
        info->n_reliable = E->nvec;  // deflation vectors now held
        info->true_rel_residual = true_rel;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - wall0).count();
        info->hop_applications = 4.0 * iters;
    }
    return status;
}
