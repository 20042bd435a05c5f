// Krylov solvers on the even-odd preconditioned Wilson operator.
//
// The paper's library provides "a few efficient linear solvers" without naming
// them; this file implements
//   * CG on the normal equations Mhat^dag Mhat x_e = Mhat^dag bhat, and
//   * BiCGstab (van der Vorst) on Mhat x_e = bhat,
// with Mhat = 1 - kappa^2 H_eo H_oe, bhat = b_e + kappa H_eo b_o and
// x_o = b_o + kappa H_oe x_e, for one or several (n <= 12) right-hand sides
// solved together: every operator application of the batch loads each link
// once for all of them (the multi-RHS hopping kernel), while each right-hand
// side keeps its own Krylov scalars and convergence state.
//
// Precision.  The Krylov iteration runs at the inner precision (FP64, or FP32
// / FP16 storage with FP32 arithmetic).  An FP64 outer loop owns the solution
// x_e and the true residual s = bhat - Mhat x_e: whenever the inner residual
// of every active right-hand side has fallen by `delta` (or reached its
// estimated target) the inner solution is added to x_e in FP64, s is
// recomputed with the FP64 operator and the iteration continues from it.  For
// CG the search direction p is kept across these reliable updates (Clark et
// al., "Solving lattice QCD systems of equations using mixed precision solvers
// on GPUs", 2010); BiCGstab restarts from the recomputed residual (defect
// correction).  Convergence is declared only on the FP64 true residual:
// ||b - M x|| / ||b|| = ||s|| / ||b|| <= tol.
//
// Each inner iteration is a fixed sequence of kernels that read their
// coefficients from device-resident SolverStates and update them in the last
// block of each fused reduction; a batch of `check_every` iterations is
// captured once into a CUDA graph and replayed, and the host only polls the
// states between batches.  Once a right-hand side's stop flag is set
// (triggered, converged, maxit, NaN or breakdown) every later kernel skips its
// elements, so its x and r stay consistent.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "plq_solver_common.cuh"

namespace plq {
namespace {

struct Params {
    double tol;
    int maxit;
    int inner;
    double delta;
    int use_x0;
    int k;
    double mu;
    int residual;  // PLQ_F64 or PLQ_DF64 arithmetic of the reliable-update residuals
};

plq_status parse(const plq_solver_params *p, Params *o) {
    o->tol = (p && p->tol > 0) ? p->tol : 1e-10;
    o->maxit = (p && p->maxit > 0) ? p->maxit : 20000;
    o->inner = p ? p->inner_prec : PLQ_F64;
    // Default reliable-update trigger: FP64 work is expensive on this GPU, so
    // the inner solve runs as far as its precision allows between updates.
    // Measured on 24^3 x 48 (and 32^3 x 64 with 12 point sources): FP32 inner
    // iterations keep the FP64 iteration count for any trigger down to 1e-5,
    // and below 3e-4 the updates are set by the tolerance alone (3 instead of
    // 4 at 1e-3); FP16 storage needs 1e-2 (1e-3 already costs iterations).
    const int inner = p ? p->inner_prec : PLQ_F64;
    o->delta = (p && p->delta > 0) ? p->delta : (inner == PLQ_F16 ? 1e-2 : 1e-4);
    o->use_x0 = p ? p->use_x0 : 0;
    o->k = (p && p->check_every > 0) ? p->check_every : 16;
    o->mu = p ? p->mu : 0.0;
    if (!std::isfinite(o->mu)) return set_error(PLQ_ERR_ARG, "twisted mass mu not finite");
    if (!valid_prec(o->inner)) return set_error(PLQ_ERR_ARG, "bad inner precision %d", o->inner);
    if (o->delta >= 1.0) return set_error(PLQ_ERR_ARG, "delta must be < 1");
    if (o->k > 256) o->k = 256;
    o->residual = p ? p->residual_prec : PLQ_F64;
    if (o->residual != PLQ_F64 && o->residual != PLQ_DF64)
        return set_error(PLQ_ERR_ARG, "residual_prec must be PLQ_F64 or PLQ_DF64");
    return PLQ_OK;
}

// s = bhat - Mhat x_e (FP64); per right-hand side |s|^2
plq_status true_residual(Solve &S, void *s64, void *tmp_o64, const void *bhat, const void *xe, double *s2) {
    PLQ_TRY(hop(S, PLQ_F64, 1, tmp_o64, xe, EPI_PLAIN, 0, nullptr, 0.0, FIN_NONE, nullptr, false, tw_first(S, false)));
    if (S.nu != 0.0) PLQ_TRY(blas_twist(S.N, s64, xe, PLQ_F64, S.nu, 1.0, S.s));  // s = A x_e
    else PLQ_TRY(blas_copy_convert(S.N, s64, PLQ_F64, xe, PLQ_F64, S.s));
    PLQ_TRY(blas_xpay64(S.N, bhat, -1.0, s64, S.s));  // s = bhat - A x_e
    PLQ_TRY(hop(S, PLQ_F64, 0, s64, tmp_o64, EPI_XPAY_NORM, 0, s64, S.kappa * S.kappa));
    return read_sums(S, s2, S.n);
}

// The same residual with both half-applications in float-float arithmetic
// (PLQ_DF64): x_e and bhat - A x_e are split into float-float fields (dfe,
// even), the odd intermediate lives in dfo; s is joined back into FP64 for
// the norm and the restart.  A x_e and bhat - A x_e stay FP64.  sh[r] scales
// right-hand side r by a power of two (the inverse of its source norm) so
// that the float-float fields sit in the FP32 exponent range whatever the
// magnitude of the source; the operator is linear, the join undoes it.
plq_status true_residual_df(Solve &S, const int *sh, void *s64, void *dfo, void *dfe, const void *bhat, const void *xe,
                            double *s2) {
    const Tw t1 = tw_first(S, false);
    PLQ_TRY(df_split(S.N, S.n, sh, dfe, xe, S.s));
    PLQ_TRY(df_hop(S.c, 1, dfo, dfe, nullptr, 0.0, t1.nu_h, t1.scale_h, S.n, S.s));
    if (S.nu != 0.0) PLQ_TRY(blas_twist(S.N, s64, xe, PLQ_F64, S.nu, 1.0, S.s));
    else PLQ_TRY(blas_copy_convert(S.N, s64, PLQ_F64, xe, PLQ_F64, S.s));
    PLQ_TRY(blas_xpay64(S.N, bhat, -1.0, s64, S.s));
    PLQ_TRY(df_split(S.N, S.n, sh, dfe, s64, S.s));
    PLQ_TRY(df_hop(S.c, 0, dfe, dfo, dfe, S.kappa * S.kappa, 0.0, 1.0, S.n, S.s));
    PLQ_TRY(df_join(S.N, S.n, sh, s64, dfe, S.s));
    S.hops += 2;
    return norm2_64(S, s64, s2);
}

// zero right-hand side r of an FP64 half field of N elements (n interleaved)
__global__ void zero_rhs_kernel(long long N, int n, int r, double2 *f) {
    for (long long e = r + (long long)n * (blockIdx.x * (long long)blockDim.x + threadIdx.x); e < N;
         e += (long long)n * gridDim.x * blockDim.x)
        for (int k = 0; k < 12; ++k) f[k * N + e] = make_double2(0.0, 0.0);
}

enum { SOLVER_CG = 0, SOLVER_BICGSTAB = 1 };

plq_status solve_impl(plq_ctx *c, void *x, const void *b, double kappa, int n, const plq_solver_params *pp,
                      plq_solve_info *infos, void *stream, int method) {
    if (infos && n > 0 && n <= PLQ_MAX_RHS) std::memset(infos, 0, sizeof(plq_solve_info) * n);
    if (!c) return set_error(PLQ_ERR_ARG, "null context");
    if (n < 1 || n > PLQ_MAX_RHS) return set_error(PLQ_ERR_ARG, "nrhs must be in 1..%d", PLQ_MAX_RHS);
    if (!x || !b || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(b) & 15))
        return set_error(PLQ_ERR_ARG, "null or misaligned field pointer");
    if (x == b) return set_error(PLQ_ERR_ARG, "x and b must not overlap");
    if (!std::isfinite(kappa)) return set_error(PLQ_ERR_ARG, "kappa not finite");
    Params P;
    PLQ_TRY(parse(pp, &P));
    // BiCGstab restarts from each recomputed residual (defect correction), so a
    // longer inner cycle costs it iterations: with FP32 inner iterations it keeps
    // 1e-3 (24^3 x 48: 20 iterations at 1e-3, 22 at 1e-4)
    if (method == SOLVER_BICGSTAB && P.inner == PLQ_F32 && !(pp && pp->delta > 0)) P.delta = 1e-3;
    if (!c->gauge[PLQ_F64].ptr) return set_error(PLQ_ERR_STATE, "solvers need the FP64 gauge copy");
    if (!c->gauge[P.inner].ptr) return set_error(PLQ_ERR_STATE, "no gauge copy for inner precision %d", P.inner);
    const bool df_res = P.residual == PLQ_DF64 && P.inner != PLQ_F64;
    if (df_res && !c->gauge_df.ptr)
        return set_error(PLQ_ERR_STATE, "residual_prec = PLQ_DF64 needs the PLQ_DF64 gauge copy");
    PLQ_CUDA(cudaSetDevice(c->device));

    Solve S;
    S.c = c;
    S.Vh = c->lat.Vh;
    S.n = n;
    S.N = (long long)S.Vh * n;
    S.kappa = kappa;
    S.P = P.inner;
    S.PX = P.inner == PLQ_F64 ? PLQ_F64 : PLQ_F32;
    S.nu = 2.0 * kappa * P.mu;
    const size_t h64 = spinor_site_bytes(PLQ_F64) * (size_t)S.N;
    const size_t hL = spinor_site_bytes(S.P) * (size_t)S.N;
    const size_t hX = spinor_site_bytes(S.PX) * (size_t)S.N;
    const int nL = method == SOLVER_CG ? 5 : 7;
    const size_t need = 5 * h64 + nL * hL + hX + 4096;
    PLQ_TRY(ensure_work(c, need));
    char *w = static_cast<char *>(c->work);
    void *bhat = w, *s64 = w + h64, *r64 = w + 2 * h64, *tmp_o64 = w + 3 * h64, *t64 = w + 4 * h64;
    char *wl = w + 5 * h64;
    void *L[7];
    for (int i = 0; i < nL; ++i) L[i] = wl + i * hL;
    void *xL = wl + nL * hL;
    // key of the inner-iteration graph (see Ctx::SolveGraph)
    unsigned long long gkey[10] = {};
    {
        double kk = kappa, nu = S.nu;
        gkey[0] = (unsigned long long)method;
        gkey[1] = (unsigned long long)S.P | ((unsigned long long)S.PX << 8) | ((unsigned long long)n << 16);
        gkey[2] = (unsigned long long)S.N;
        std::memcpy(&gkey[3], &kk, sizeof(double));
        std::memcpy(&gkey[4], &nu, sizeof(double));
        gkey[5] = (unsigned long long)P.k;
        gkey[6] = (unsigned long long)reinterpret_cast<uintptr_t>(c->work);
        gkey[7] = (unsigned long long)c->tune_version;
        gkey[8] = 1;  // marks a valid key
        // the captured launches hold the inner gauge copy's address and format
        gkey[9] = (unsigned long long)reinterpret_cast<uintptr_t>(c->gauge[S.P].ptr) ^
                  ((unsigned long long)c->gauge[S.P].reals << 56);
    }

    // internal stream ordered after the caller's stream
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t s = nullptr;
    PLQ_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    S.s = s;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    auto cleanup = [&]() {
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (s) cudaStreamDestroy(s);
    };
    cudaError_t ce = cudaEventCreate(&ev0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&ev1);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev0, user);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, ev0, 0);
    if (ce != cudaSuccess) {
        cleanup();
        return cuda_error(ce, "solver stream setup");
    }
    auto wall0 = std::chrono::steady_clock::now();

    const char *be = static_cast<const char *>(b), *bo = be + h64;
    char *xe = static_cast<char *>(x), *xo = xe + h64;
    plq_status st = PLQ_OK;
    std::vector<double> n_e(n), n_o(n), bnorm2(n), bnorm(n), s2(n), r2(n), true_rel(n, 0.0);
    std::vector<double> sigma(n, 0.5), last_rho(n, 0.0), best(n, INFINITY), target2(n, 0.0);
    std::vector<int> iters(n, 0), n_rel(n, 0), stall(n, 0), done(n, 0), result(n, PLQ_OK);
    std::vector<std::string> msg(n);
    std::vector<SolverState> init(n), fin(n);
    bool first = true;

    do {
        if ((st = norm2_64(S, be, n_e.data())) != PLQ_OK) break;
        if ((st = norm2_64(S, bo, n_o.data())) != PLQ_OK) break;
        if (!P.use_x0 && (st = blas_zero(S.N, xe, PLQ_F64, s)) != PLQ_OK) break;
        for (int r = 0; r < n; ++r) {
            bnorm2[r] = n_e[r] + n_o[r];
            bnorm[r] = std::sqrt(bnorm2[r]);
            if (!std::isfinite(bnorm2[r])) {
                done[r] = 1;
                result[r] = PLQ_ERR_NAN;
                msg[r] = "source contains NaN or Inf";
            } else if (bnorm2[r] == 0.0) {
                // zero source: x = 0 exactly
                done[r] = 1;
                zero_rhs_kernel<<<256, 256, 0, s>>>(S.N, n, r, static_cast<double2 *>(static_cast<void *>(xe)));
                if (method == SOLVER_BICGSTAB) {
                    result[r] = PLQ_ERR_BREAKDOWN;
                    msg[r] = "BiCGstab breakdown: rho = <rhat, r0> = 0 (zero source)";
                }
            }
        }
        // Right-hand side r is scaled by 2^-(exponent of |b_r|) wherever it enters a
        // narrower format -- the float-float fields and the inner (FP32/FP16)
        // iteration -- so that sources of any magnitude sit in their exponent
        // range (an FP32 residual of a 1e-45 source would flush to zero).  The
        // scale is fixed for the whole solve, so the kept direction p and the
        // inner scalars stay consistent across reliable updates.
        std::vector<int> dfsh(n, 0);
        std::vector<double> isc(n, 1.0), sc(n, 1.0);
        for (int r = 0; r < n; ++r)
            if (bnorm[r] > 0.0 && std::isfinite(bnorm[r])) {
                dfsh[r] = -std::ilogb(bnorm[r]);
                if (S.P != PLQ_F64) {
                    sc[r] = std::ldexp(1.0, dfsh[r]);
                    isc[r] = std::ldexp(1.0, -dfsh[r]);
                }
            }
        // bhat = b_e + kappa H_eo A^{-1} b_o (A = 1 for Wilson)
        const void *bsrc = bo;
        if (S.nu != 0.0) {  // (r64 is free until the iteration starts)
            if ((st = blas_twist(S.N, r64, bo, PLQ_F64, -S.nu, 1.0 / (1.0 + S.nu * S.nu), s)) != PLQ_OK) break;
            bsrc = r64;
        }
        if (df_res) {  // in float-float: t64 / tmp_o64 hold the split fields
            if ((st = df_split(S.N, n, dfsh.data(), tmp_o64, bsrc, s)) != PLQ_OK) break;
            if ((st = df_split(S.N, n, dfsh.data(), t64, be, s)) != PLQ_OK) break;
            if ((st = df_hop(c, 0, t64, tmp_o64, t64, kappa, 0.0, 1.0, n, s)) != PLQ_OK) break;
            if ((st = df_join(S.N, n, dfsh.data(), bhat, t64, s)) != PLQ_OK) break;
            S.hops += 1;
        } else if ((st = hop(S, PLQ_F64, 0, bhat, bsrc, EPI_XPAY, 0, be, kappa)) != PLQ_OK) {
            break;
        }

        const double delta = S.P == PLQ_F64 ? 0.0 : P.delta;
        // tmp_o64 holds H_oe x_e of the current x_e (an FP64 residual check of the
        // Wilson operator left it there); the final x_o and full residual reuse it
        bool have_toe = false;
        for (;;) {
            if (first && !P.use_x0) {
                // x_e = 0: s = bhat exactly, without applying the operator
                have_toe = false;
                st = blas_copy_convert(S.N, s64, PLQ_F64, bhat, PLQ_F64, s);
                if (st == PLQ_OK) st = norm2_64(S, s64, s2.data());
            } else {
                // (t64 is free until the final check; it holds the float-float fields)
                st = df_res ? true_residual_df(S, dfsh.data(), s64, tmp_o64, t64, bhat, xe, s2.data())
                            : true_residual(S, s64, tmp_o64, bhat, xe, s2.data());
                have_toe = !df_res && S.nu == 0.0;
            }
            if (st != PLQ_OK) break;
            bool all_done = true;
            for (int r = 0; r < n; ++r) {
                if (done[r]) continue;
                if (!std::isfinite(s2[r])) {
                    done[r] = 1;
                    result[r] = PLQ_ERR_NAN;
                    msg[r] = "NaN in the FP64 residual";
                    continue;
                }
                true_rel[r] = std::sqrt(s2[r]) / bnorm[r];
                if (true_rel[r] <= P.tol) {
                    done[r] = 1;
                    continue;
                }
                if (iters[r] >= P.maxit) {
                    done[r] = 1;
                    result[r] = PLQ_ERR_NOT_CONVERGED;
                    msg[r] = "no convergence within maxit";
                    continue;
                }
                if (s2[r] < 0.99 * best[r]) {
                    best[r] = s2[r];
                    stall[r] = 0;
                } else if (++stall[r] >= 20) {
                    done[r] = 1;
                    result[r] = PLQ_ERR_NOT_CONVERGED;
                    msg[r] = "residual stalled";
                    continue;
                }
                all_done = false;
            }
            if (all_done) break;
            for (int r = 0; r < n; ++r) {
                std::memset(&init[r], 0, sizeof(SolverState));
                init[r].iter = iters[r];
                init[r].maxit = P.maxit;
                init[r].stop = done[r];
            }
            if (method == SOLVER_CG) {
                // r = Mhat^dag s, the residual of the normal equations.  s is the
                // FP64 true residual; r only restarts the inner iteration, so with
                // a low-precision inner solve it is formed at that precision (two
                // inner-precision half-applies instead of two FP64 ones).
                void *rL = L[0], *pL = L[1], *qL = L[2], *mpL = L[3], *toL = L[4];
                if (S.P == PLQ_F64) {
                    if ((st = hop(S, PLQ_F64, 1, tmp_o64, s64, EPI_PLAIN, 1, nullptr, 0.0, FIN_NONE, nullptr, false,
                                  tw_first(S, true))) != PLQ_OK)
                        break;
                    if ((st = hop(S, PLQ_F64, 0, r64, tmp_o64, EPI_XPAY_NORM, 1, s64, -kappa * kappa, FIN_NONE,
                                  nullptr, false, tw_second(S, true))) != PLQ_OK)
                        break;
                    if ((st = blas_copy_convert(S.N, rL, S.P, r64, PLQ_F64, s)) != PLQ_OK) break;
                } else {
                    void *sL = mpL;  // free until the inner iteration starts
                    if ((st = blas_scale64(S.N, n, s64, sc.data(), s)) != PLQ_OK) break;
                    if ((st = blas_copy_convert(S.N, sL, S.P, s64, PLQ_F64, s)) != PLQ_OK) break;
                    if ((st = hop(S, S.P, 1, toL, sL, EPI_PLAIN, 1, nullptr, 0.0, FIN_NONE, nullptr, false,
                                  tw_first(S, true))) != PLQ_OK)
                        break;
                    if ((st = hop(S, S.P, 0, rL, toL, EPI_XPAY_NORM, 1, sL, -kappa * kappa, FIN_NONE, nullptr, false,
                                  tw_second(S, true))) != PLQ_OK)
                        break;
                }
                if ((st = read_sums(S, r2.data(), n)) != PLQ_OK) break;
                if ((st = blas_zero(S.N, xL, S.PX, s)) != PLQ_OK) break;
                for (int r = 0; r < n; ++r) {
                    if (done[r]) continue;
                    const double ratio = std::sqrt(r2[r] / s2[r]);
                    target2[r] = std::pow(sigma[r] * ratio * P.tol * bnorm[r], 2);
                    init[r].rho = r2[r];
                    // Reliable update: the direction survives and the iteration goes on
                    // as if the recursive residual had been replaced by the true one:
                    // p = r_true + beta p, beta = |r_true|^2 / rho_k with rho_k the
                    // |r|^2 of the iteration before the one that triggered.
                    init[r].beta = first ? 0.0 : r2[r] / last_rho[r];
                    init[r].stop_r2 = std::fmax(delta * delta * r2[r], target2[r]);
                }
                if ((st = put_states(S, init)) != PLQ_OK) break;
                if (first) st = blas_copy_convert(S.N, pL, S.P, rL, S.P, s);
                else st = blas_cg_direction(S.N, n, pL, rL, S.P, c->state, s);
                if (st != PLQ_OK) break;
                const double kk = kappa * kappa;
                const int PI = S.P;
                auto body = [&]() -> plq_status {
                    PLQ_TRY(hop(S, PI, 1, toL, pL, EPI_PLAIN, 0, nullptr, 0.0, FIN_NONE, nullptr, true, tw_first(S, false)));
                    PLQ_TRY(hop(S, PI, 0, mpL, toL, EPI_XPAY_NORM, 0, pL, -kk, FIN_CG_ALPHA, nullptr, true,
                                tw_second(S, false)));
                    PLQ_TRY(hop(S, PI, 1, toL, mpL, EPI_PLAIN, 1, nullptr, 0.0, FIN_NONE, nullptr, true, tw_first(S, true)));
                    PLQ_TRY(hop(S, PI, 0, qL, toL, EPI_XPAY, 1, mpL, -kk, FIN_NONE, nullptr, true, tw_second(S, true)));
                    Reduce rb = reduce_of(c, FIN_CG_BETA);
                    PLQ_TRY(blas_cg_update(S.N, n, xL, rL, pL, qL, PI, rb, c->state, s));
                    return blas_cg_direction(S.N, n, pL, rL, PI, c->state, s);
                };
                if ((st = run_batches(S, P.k, body, fin, &c->solve_graph[method], gkey)) != PLQ_OK) break;
            } else {
                void *rL = L[0], *rhL = L[1], *pL = L[2], *vL = L[3], *sL = L[4], *tL = L[5], *toL = L[6];
                if ((st = blas_scale64(S.N, n, s64, sc.data(), s)) != PLQ_OK) break;
                if ((st = blas_copy_convert(S.N, rL, S.P, s64, PLQ_F64, s)) != PLQ_OK) break;
                if ((st = blas_copy_convert(S.N, rhL, S.P, rL, S.P, s)) != PLQ_OK) break;
                if ((st = blas_copy_convert(S.N, pL, S.P, rL, S.P, s)) != PLQ_OK) break;
                if ((st = blas_zero(S.N, xL, S.PX, s)) != PLQ_OK) break;
                for (int r = 0; r < n; ++r) {
                    if (done[r]) continue;
                    // (inner quantities carry the factor sc[r])
                    target2[r] = std::pow(sigma[r] * P.tol * bnorm[r] * sc[r], 2);
                    init[r].c_rho = make_double2(s2[r] * sc[r] * sc[r], 0.0);
                    init[r].stop_r2 = std::fmax(delta * delta * s2[r] * sc[r] * sc[r], target2[r]);
                    init[r].tiny = 1e-300;
                }
                if ((st = put_states(S, init)) != PLQ_OK) break;
                const double kk = kappa * kappa;
                const int PI = S.P;
                auto body = [&]() -> plq_status {
                    PLQ_TRY(hop(S, PI, 1, toL, pL, EPI_PLAIN, 0, nullptr, 0.0, FIN_NONE, nullptr, true, tw_first(S, false)));
                    PLQ_TRY(hop(S, PI, 0, vL, toL, EPI_XPAY_DOTW, 0, pL, -kk, FIN_BICG_ALPHA, rhL, true,
                                tw_second(S, false)));
                    PLQ_TRY(blas_bicg_s(S.N, n, sL, rL, vL, PI, c->state, s));
                    PLQ_TRY(hop(S, PI, 1, toL, sL, EPI_PLAIN, 0, nullptr, 0.0, FIN_NONE, nullptr, true, tw_first(S, false)));
                    PLQ_TRY(hop(S, PI, 0, tL, toL, EPI_XPAY_TS, 0, sL, -kk, FIN_BICG_OMEGA, nullptr, true,
                                tw_second(S, false)));
                    Reduce rb = reduce_of(c, FIN_BICG_RHO);
                    PLQ_TRY(blas_bicg_update(S.N, n, xL, rL, pL, sL, tL, rhL, PI, rb, c->state, s));
                    return blas_bicg_p(S.N, n, pL, rL, vL, PI, c->state, s);
                };
                if ((st = run_batches(S, P.k, body, fin, &c->solve_graph[method], gkey)) != PLQ_OK) break;
            }
            for (int r = 0; r < n; ++r) {
                if (done[r]) continue;
                const int progressed = fin[r].iter - iters[r];
                iters[r] = fin[r].iter;
                if (fin[r].flags & FLAG_NAN) {
                    done[r] = 1;
                    result[r] = PLQ_ERR_NAN;
                    msg[r] = "NaN or Inf in the inner iteration";
                } else if ((fin[r].flags & FLAG_BREAKDOWN) && progressed == 0) {
                    done[r] = 1;
                    result[r] = PLQ_ERR_BREAKDOWN;
                    msg[r] = "Krylov breakdown (rho or omega vanished)";
                }
                ++n_rel[r];
                // the inner target was reached but the FP64 check may still fail:
                // tighten the estimate for the next round
                const double fr = method == SOLVER_CG ? fin[r].rho : fin[r].r2;
                if (fr <= target2[r] * 1.0000001) sigma[r] *= 0.25;
                // FIN_CG_BETA left rho = rho_{k+1} and beta = rho_{k+1} / rho_k
                last_rho[r] = fin[r].beta > 0.0 ? fin[r].rho / fin[r].beta : fin[r].rho;
            }
            // reliable update: x_e += x_inner (FP64); frozen right-hand sides add zero
            if ((st = blas_accumulate_scaled(S.N, n, xe, xL, S.PX, isc.data(), s)) != PLQ_OK) break;
            first = false;
        }
        if (st != PLQ_OK) break;
        // x_o = A^{-1} (b_o + kappa H_oe x_e)
        if (df_res) {
            if ((st = df_split(S.N, n, dfsh.data(), t64, xe, s)) != PLQ_OK) break;
            if ((st = df_split(S.N, n, dfsh.data(), tmp_o64, bo, s)) != PLQ_OK) break;
            if ((st = df_hop(c, 1, tmp_o64, t64, tmp_o64, kappa, 0.0, 1.0, n, s)) != PLQ_OK) break;
            if ((st = df_join(S.N, n, dfsh.data(), xo, tmp_o64, s)) != PLQ_OK) break;
            S.hops += 1;
        } else if (have_toe) {
            // the same FP64 values as the operator's xpay epilogue: fma(kappa, H_oe x_e, b_o)
            if ((st = blas_copy_convert(S.N, xo, PLQ_F64, tmp_o64, PLQ_F64, s)) != PLQ_OK) break;
            if ((st = blas_xpay64(S.N, bo, kappa, xo, s)) != PLQ_OK) break;
        } else if ((st = hop(S, PLQ_F64, 1, xo, xe, EPI_XPAY, 0, bo, kappa)) != PLQ_OK) {
            break;
        }
        if (S.nu != 0.0 && (st = blas_twist(S.N, xo, xo, PLQ_F64, -S.nu, 1.0 / (1.0 + S.nu * S.nu), s)) != PLQ_OK)
            break;
        // full true residual ||b - M x|| with the FP64 operator, both parities
        std::vector<double> re(n), ro(n);
        if ((st = hop(S, PLQ_F64, 0, t64, xo, EPI_XPAY, 0, xe, -kappa, FIN_NONE, nullptr, false, tw_diag(S))) != PLQ_OK)
            break;
        if ((st = blas_xpay64(S.N, be, -1.0, t64, s)) != PLQ_OK) break;
        if ((st = norm2_64(S, t64, re.data())) != PLQ_OK) break;
        if (have_toe) {  // (M x)_o = x_o - kappa H_oe x_e, H_oe x_e still in tmp_o64
            if ((st = blas_xpay64(S.N, xo, -kappa, tmp_o64, s)) != PLQ_OK) break;
        } else if ((st = hop(S, PLQ_F64, 1, tmp_o64, xe, EPI_XPAY, 0, xo, -kappa, FIN_NONE, nullptr, false,
                             tw_diag(S))) != PLQ_OK) {
            break;
        }
        if ((st = blas_xpay64(S.N, bo, -1.0, tmp_o64, s)) != PLQ_OK) break;
        if ((st = norm2_64(S, tmp_o64, ro.data())) != PLQ_OK) break;
        for (int r = 0; r < n; ++r) {
            if (bnorm2[r] == 0.0 || !std::isfinite(bnorm2[r])) continue;
            true_rel[r] = std::sqrt((re[r] + ro[r]) / bnorm2[r]);
            if (!(true_rel[r] <= P.tol) && result[r] == PLQ_OK) {
                result[r] = PLQ_ERR_NOT_CONVERGED;
                msg[r] = "final residual above tol";
            }
        }
    } while (0);

    cudaError_t e1 = cudaEventRecord(ev1, s);
    if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(user, ev1, 0);
    if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(s);
    auto wall1 = std::chrono::steady_clock::now();
    cleanup();
    if (st == PLQ_OK && e1 != cudaSuccess) st = cuda_error(e1, "solver completion");
    int status = st;
    if (status == PLQ_OK) {
        for (int r = 0; r < n; ++r)
            if (result[r] != PLQ_OK) {
                status = set_error(result[r], "rhs %d: %s (residual %.3e after %d iterations)", r, msg[r].c_str(),
                                   true_rel[r], iters[r]);
                break;
            }
    }
    if (infos) {
        const double secs = std::chrono::duration<double>(wall1 - wall0).count();
        for (int r = 0; r < n; ++r) {
            infos[r].status = st != PLQ_OK ? st : result[r];
            infos[r].iterations = iters[r];
            infos[r].n_reliable = n_rel[r];
            infos[r].true_rel_residual = true_rel[r];
            infos[r].seconds = secs;
            infos[r].hop_applications = S.hops + 4.0 * iters[r];
        }
    }
    return status;
}

}  // namespace

// ||b - M x||^2 and ||b||^2 of full FP64 fields with the FP64 operator (uses
// the context's workspace; synchronises the stream).
plq_status wilson_residual64(plq_ctx *c, double kappa, const void *x, const void *b, double *r2, double *b2,
                             cudaStream_t s) {
    Solve S;
    S.c = c;
    S.s = s;
    S.Vh = c->lat.Vh;
    S.n = 1;
    S.N = S.Vh;
    S.kappa = kappa;
    const size_t h64 = spinor_site_bytes(PLQ_F64) * (size_t)S.Vh;
    PLQ_TRY(ensure_work(c, 2 * h64));
    char *te = static_cast<char *>(c->work), *to = te + h64;
    const char *xe = static_cast<const char *>(x), *xo = xe + h64;
    const char *be = static_cast<const char *>(b), *bo = be + h64;
    double re = 0, ro = 0, ne = 0, no = 0;
    PLQ_TRY(hop(S, PLQ_F64, 0, te, xo, EPI_XPAY, 0, xe, -kappa));
    PLQ_TRY(blas_xpay64(S.N, be, -1.0, te, s));
    PLQ_TRY(norm2_64(S, te, &re));
    PLQ_TRY(hop(S, PLQ_F64, 1, to, xe, EPI_XPAY, 0, xo, -kappa));
    PLQ_TRY(blas_xpay64(S.N, bo, -1.0, to, s));
    PLQ_TRY(norm2_64(S, to, &ro));
    PLQ_TRY(norm2_64(S, be, &ne));
    PLQ_TRY(norm2_64(S, bo, &no));
    *r2 = re + ro;
    *b2 = ne + no;
    return PLQ_OK;
}

}  // namespace plq

extern "C" {

plq_status plq_cg_solve(plq_ctx *ctx, void *x, const void *b, double kappa, const plq_solver_params *params,
                        plq_solve_info *info, void *stream) {
    return plq::solve_impl(ctx, x, b, kappa, 1, params, info, stream, plq::SOLVER_CG);
}

plq_status plq_bicgstab_solve(plq_ctx *ctx, void *x, const void *b, double kappa, const plq_solver_params *params,
                              plq_solve_info *info, void *stream) {
    return plq::solve_impl(ctx, x, b, kappa, 1, params, info, stream, plq::SOLVER_BICGSTAB);
}

plq_status plq_cg_solve_multi(plq_ctx *ctx, void *x, const void *b, double kappa, int nrhs,
                              const plq_solver_params *params, plq_solve_info *infos, void *stream) {
    return plq::solve_impl(ctx, x, b, kappa, nrhs, params, infos, stream, plq::SOLVER_CG);
}

plq_status plq_bicgstab_solve_multi(plq_ctx *ctx, void *x, const void *b, double kappa, int nrhs,
                                    const plq_solver_params *params, plq_solve_info *infos, void *stream) {
    return plq::solve_impl(ctx, x, b, kappa, nrhs, params, infos, stream, plq::SOLVER_BICGSTAB);
}

}  // extern "C"
