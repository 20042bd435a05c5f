// Krylov solvers on the even-odd preconditioned Wilson operator.
//
// The paper's library provides "a few efficient linear solvers" without naming
// them; this file implements
//   * CG on the normal equations Mhat^dag Mhat x_e = Mhat^dag bhat, and
//   * BiCGstab (van der Vorst) on Mhat x_e = bhat,
// with Mhat = 1 - kappa^2 H_eo H_oe, bhat = b_e + kappa H_eo b_o and
// x_o = b_o + kappa H_oe x_e.
//
// Precision.  The Krylov iteration runs at the inner precision (FP64, or FP32
// / FP16 storage with FP32 arithmetic).  An FP64 outer loop owns the solution
// x_e and the true residual s = bhat - Mhat x_e: whenever the inner residual
// has fallen by `delta` (or reached the estimated target) the inner
// solution is added to x_e in FP64, s is recomputed with the FP64 operator and
// the iteration continues from it.  For CG the search direction p is kept
// across these reliable updates (Clark et al., "Solving lattice QCD systems of
// equations using mixed precision solvers on GPUs", 2010); BiCGstab restarts
// from the recomputed residual (defect correction).  Convergence is declared
// only on the FP64 true residual: ||b - M x|| / ||b|| = ||s|| / ||b|| <= tol.
//
// Each inner iteration is a fixed sequence of kernels that read their
// coefficients from a device-resident SolverState and update it in the last
// block of each fused reduction; a batch of `check_every` iterations is
// captured once into a CUDA graph and replayed, and the host only polls the
// state between batches.  Once the state's stop flag is set (converged,
// triggered, maxit, NaN or breakdown) the remaining kernels of the batch
// return immediately, so x and r stay consistent.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "plq_internal.cuh"

namespace plq {
namespace {

struct Solve {
    plq_ctx *c;
    cudaStream_t s;  // internal capture-capable stream
    int Vh;
    double kappa;
    int P;   // inner storage precision
    int PX;  // inner solution accumulator precision
    double hops = 0;
};

Reduce reduce_of(plq_ctx *c, int fin) {
    Reduce r;
    r.partials = c->partials;
    r.ticket = c->ticket;
    r.sums = c->sums;
    r.st = c->state;
    r.fin = fin;
    return r;
}

plq_status hop(Solve &S, int prec, int out_par, void *out, const void *in, int epi, int dagger, const void *x,
               double a, int fin = FIN_NONE, const void *w = nullptr, bool freeze = false) {
    plq_ctx *c = S.c;
    HopArgs h;
    h.in = in;
    h.out = out;
    h.x = x;
    h.w = w;
    h.a = a;
    h.gauge = c->gauge[prec].ptr;
    h.gblock = c->gauge[prec].block;
    h.out_parity = out_par;
    h.dagger = dagger;
    h.lat = c->lat;
    h.red = reduce_of(c, fin);
    if (epi < EPI_XPAY_NORM) h.red.st = nullptr;
    h.st = freeze ? c->state : nullptr;
    apply_tune(c, prec, 1, h);
    S.hops += 1;
    return launch_hop(h, prec, c->gauge[prec].reals, epi, S.s);
}

plq_status read_sums(Solve &S, double *out, int n) {
    PLQ_CUDA(cudaMemcpyAsync(S.c->sums_host, S.c->sums, sizeof(double) * n, cudaMemcpyDeviceToHost, S.s));
    PLQ_CUDA(cudaStreamSynchronize(S.s));
    for (int k = 0; k < n; ++k) out[k] = S.c->sums_host[k];
    return PLQ_OK;
}

plq_status norm2_64(Solve &S, const void *v, double *out) {
    Reduce r = reduce_of(S.c, FIN_NONE);
    r.st = nullptr;
    PLQ_TRY(blas_norm2(S.Vh, v, PLQ_F64, r, S.s));
    return read_sums(S, out, 1);
}

plq_status put_state(Solve &S, const SolverState &st) {
    *S.c->state_host = st;
    PLQ_CUDA(cudaMemcpyAsync(S.c->state, S.c->state_host, sizeof(SolverState), cudaMemcpyHostToDevice, S.s));
    PLQ_CUDA(cudaStreamSynchronize(S.s));
    return PLQ_OK;
}

plq_status get_state(Solve &S, SolverState *st) {
    PLQ_CUDA(cudaMemcpyAsync(S.c->state_host, S.c->state, sizeof(SolverState), cudaMemcpyDeviceToHost, S.s));
    PLQ_CUDA(cudaStreamSynchronize(S.s));
    *st = *S.c->state_host;
    return PLQ_OK;
}

// Run `body` (one inner iteration) as graph-captured batches of `k` until the
// device state says stop.  `iters_out` gets the state's final iteration count.
template <class Body>
plq_status run_batches(Solve &S, int k, Body body, SolverState *final_state) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    PLQ_CUDA(cudaStreamBeginCapture(S.s, cudaStreamCaptureModeThreadLocal));
    plq_status st = PLQ_OK;
    const double hops0 = S.hops;
    for (int i = 0; i < k && st == PLQ_OK; ++i) st = body();
    cudaError_t e = cudaStreamEndCapture(S.s, &graph);
    if (st != PLQ_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    const double hops_per_iter = (S.hops - hops0) / k;
    S.hops = hops0;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
    SolverState cur;
    std::memset(&cur, 0, sizeof cur);
    int last_iter = -1, idle = 0;
    for (;;) {
        e = cudaGraphLaunch(exec, S.s);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            return cuda_error(e, "cudaGraphLaunch");
        }
        st = get_state(S, &cur);
        if (st != PLQ_OK) break;
        if (cur.stop) break;
        // every batch runs at least one iteration unless the state froze it;
        // a state that neither advances nor stops is a logic error, not a hang
        idle = (cur.iter == last_iter) ? idle + 1 : 0;
        last_iter = cur.iter;
        if (idle >= 2) {
            st = set_error(PLQ_ERR_STATE, "inner iteration made no progress");
            break;
        }
    }
    cudaGraphExecDestroy(exec);
    *final_state = cur;
    return st;
}

struct Params {
    double tol;
    int maxit;
    int inner;
    double delta;
    int use_x0;
    int k;
};

plq_status parse(const plq_solver_params *p, Params *o) {
    o->tol = (p && p->tol > 0) ? p->tol : 1e-10;
    o->maxit = (p && p->maxit > 0) ? p->maxit : 20000;
    o->inner = p ? p->inner_prec : PLQ_F64;
    o->delta = (p && p->delta > 0) ? p->delta : 0.1;
    o->use_x0 = p ? p->use_x0 : 0;
    o->k = (p && p->check_every > 0) ? p->check_every : 16;
    if (!valid_prec(o->inner)) return set_error(PLQ_ERR_ARG, "bad inner precision %d", o->inner);
    if (o->delta >= 1.0) return set_error(PLQ_ERR_ARG, "delta must be < 1");
    if (o->k > 256) o->k = 256;
    return PLQ_OK;
}

// s = bhat - Mhat x_e (FP64); returns ||s||^2
plq_status true_residual(Solve &S, void *s64, void *tmp_o64, const void *bhat, const void *xe, double *s2) {
    PLQ_TRY(hop(S, PLQ_F64, 1, tmp_o64, xe, EPI_PLAIN, 0, nullptr, 0.0));
    PLQ_TRY(blas_copy_convert(S.Vh, s64, PLQ_F64, xe, PLQ_F64, S.s));
    PLQ_TRY(blas_xpay64(S.Vh, bhat, -1.0, s64, S.s));  // s = bhat - x_e
    PLQ_TRY(hop(S, PLQ_F64, 0, s64, tmp_o64, EPI_XPAY_NORM, 0, s64, S.kappa * S.kappa));
    return read_sums(S, s2, 1);
}

enum { SOLVER_CG = 0, SOLVER_BICGSTAB = 1 };

plq_status solve_impl(plq_ctx *c, void *x, const void *b, double kappa, const plq_solver_params *pp,
                      plq_solve_info *info, void *stream, int method) {
    if (info) std::memset(info, 0, sizeof(*info));
    if (!c) return set_error(PLQ_ERR_ARG, "null context");
    if (!x || !b || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(b) & 15))
        return set_error(PLQ_ERR_ARG, "null or misaligned field pointer");
    if (x == b) return set_error(PLQ_ERR_ARG, "x and b must not overlap");
    if (!std::isfinite(kappa)) return set_error(PLQ_ERR_ARG, "kappa not finite");
    Params P;
    PLQ_TRY(parse(pp, &P));
    if (!c->gauge[PLQ_F64].ptr) return set_error(PLQ_ERR_STATE, "solvers need the FP64 gauge copy");
    if (!c->gauge[P.inner].ptr)
        return set_error(PLQ_ERR_STATE, "no gauge copy for inner precision %d", P.inner);
    PLQ_CUDA(cudaSetDevice(c->device));

    Solve S;
    S.c = c;
    S.Vh = c->lat.Vh;
    S.kappa = kappa;
    S.P = P.inner;
    S.PX = P.inner == PLQ_F64 ? PLQ_F64 : PLQ_F32;
    const size_t h64 = spinor_site_bytes(PLQ_F64) * S.Vh;
    const size_t hL = spinor_site_bytes(S.P) * S.Vh;
    const size_t hX = spinor_site_bytes(S.PX) * S.Vh;
    const int nL = method == SOLVER_CG ? 5 : 7;
    const size_t need = 5 * h64 + nL * hL + hX + 4096;
    PLQ_TRY(ensure_work(c, need));
    char *w = static_cast<char *>(c->work);
    void *bhat = w, *s64 = w + h64, *r64 = w + 2 * h64, *tmp_o64 = w + 3 * h64, *t64 = w + 4 * h64;
    char *wl = w + 5 * h64;
    void *L[7];
    for (int i = 0; i < nL; ++i) L[i] = wl + i * hL;
    void *xL = wl + nL * hL;

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
    double n_e = 0, n_o = 0;
    int iters = 0, n_rel = 0;
    int result = PLQ_OK;
    double true_rel = 0.0;

    do {
        if ((st = norm2_64(S, be, &n_e)) != PLQ_OK) break;
        if ((st = norm2_64(S, bo, &n_o)) != PLQ_OK) break;
        const double bnorm2 = n_e + n_o;
        if (!std::isfinite(bnorm2)) {
            result = set_error(PLQ_ERR_NAN, "source contains NaN or Inf");
            break;
        }
        if (bnorm2 == 0.0) {
            st = blas_zero(S.Vh, xe, PLQ_F64, s);
            if (st == PLQ_OK) st = blas_zero(S.Vh, xo, PLQ_F64, s);
            if (method == SOLVER_BICGSTAB && st == PLQ_OK)
                result = set_error(PLQ_ERR_BREAKDOWN, "BiCGstab breakdown: rho = <rhat, r0> = 0 (zero source)");
            break;
        }
        const double bnorm = std::sqrt(bnorm2);
        // bhat = b_e + kappa H_eo b_o
        if ((st = hop(S, PLQ_F64, 0, bhat, bo, EPI_XPAY, 0, be, kappa)) != PLQ_OK) break;
        if (!P.use_x0 && (st = blas_zero(S.Vh, xe, PLQ_F64, s)) != PLQ_OK) break;

        const double delta = S.P == PLQ_F64 ? 0.0 : P.delta;
        double sigma = 0.5;  // safety factor on the estimated inner target
        double last_rho = 0.0;  // |r|^2 of the second-to-last iteration of the last inner CG run
        double best = INFINITY;
        int stall = 0;
        bool first = true;
        for (;;) {
            double s2 = 0;
            if ((st = true_residual(S, s64, tmp_o64, bhat, xe, &s2)) != PLQ_OK) break;
            if (!std::isfinite(s2)) {
                result = set_error(PLQ_ERR_NAN, "NaN in the FP64 residual");
                break;
            }
            true_rel = std::sqrt(s2) / bnorm;
            if (true_rel <= P.tol) break;
            if (iters >= P.maxit) {
                result = set_error(PLQ_ERR_NOT_CONVERGED, "no convergence in %d iterations (residual %.3e)",
                                   iters, true_rel);
                break;
            }
            if (s2 < 0.99 * best) {
                best = s2;
                stall = 0;
            } else if (++stall >= 20) {
                result = set_error(PLQ_ERR_NOT_CONVERGED, "residual stalled at %.3e", true_rel);
                break;
            }
            SolverState init;
            std::memset(&init, 0, sizeof init);
            init.iter = iters;
            init.maxit = P.maxit;
            init.tiny = 0.0;
            double target2 = 0.0;
            int start_iter = iters;
            SolverState fin;
            if (method == SOLVER_CG) {
                // r = Mhat^dag s, the residual of the normal equations
                if ((st = hop(S, PLQ_F64, 1, tmp_o64, s64, EPI_PLAIN, 1, nullptr, 0.0)) != PLQ_OK) break;
                if ((st = hop(S, PLQ_F64, 0, r64, tmp_o64, EPI_XPAY_NORM, 1, s64, -kappa * kappa)) != PLQ_OK) break;
                double r2 = 0;
                if ((st = read_sums(S, &r2, 1)) != PLQ_OK) break;
                const double ratio = std::sqrt(r2 / s2);
                void *rL = L[0], *pL = L[1], *qL = L[2], *mpL = L[3], *toL = L[4];
                if ((st = blas_copy_convert(S.Vh, rL, S.P, r64, PLQ_F64, s)) != PLQ_OK) break;
                if ((st = blas_zero(S.Vh, xL, S.PX, s)) != PLQ_OK) break;
                target2 = std::pow(sigma * ratio * P.tol * bnorm, 2);
                init.rho = r2;
                // Reliable update: the direction survives and the iteration goes on
                // as if the recursive residual had been replaced by the true one:
                // p = r_true + beta p, beta = |r_true|^2 / rho_k with rho_k the
                // |r|^2 of the iteration before the one that triggered.
                init.beta = first ? 0.0 : r2 / last_rho;
                init.stop_r2 = std::fmax(delta * delta * r2, target2);
                if ((st = put_state(S, init)) != PLQ_OK) break;
                if (first) st = blas_copy_convert(S.Vh, pL, S.P, rL, S.P, s);
                else st = blas_cg_direction(S.Vh, pL, rL, S.P, c->state, s);
                if (st != PLQ_OK) break;
                const double kk = kappa * kappa;
                const int PI = S.P;
                auto body = [&]() -> plq_status {
                    PLQ_TRY(hop(S, PI, 1, toL, pL, EPI_PLAIN, 0, nullptr, 0.0, FIN_NONE, nullptr, true));
                    PLQ_TRY(hop(S, PI, 0, mpL, toL, EPI_XPAY_NORM, 0, pL, -kk, FIN_CG_ALPHA, nullptr, true));
                    PLQ_TRY(hop(S, PI, 1, toL, mpL, EPI_PLAIN, 1, nullptr, 0.0, FIN_NONE, nullptr, true));
                    PLQ_TRY(hop(S, PI, 0, qL, toL, EPI_XPAY, 1, mpL, -kk, FIN_NONE, nullptr, true));
                    Reduce rb = reduce_of(c, FIN_CG_BETA);
                    PLQ_TRY(blas_cg_update(S.Vh, xL, rL, pL, qL, PI, rb, c->state, s));
                    return blas_cg_direction(S.Vh, pL, rL, PI, c->state, s);
                };
                if ((st = run_batches(S, P.k, body, &fin)) != PLQ_OK) break;
            } else {
                void *rL = L[0], *rhL = L[1], *pL = L[2], *vL = L[3], *sL = L[4], *tL = L[5], *toL = L[6];
                if ((st = blas_copy_convert(S.Vh, rL, S.P, s64, PLQ_F64, s)) != PLQ_OK) break;
                if ((st = blas_copy_convert(S.Vh, rhL, S.P, rL, S.P, s)) != PLQ_OK) break;
                if ((st = blas_copy_convert(S.Vh, pL, S.P, rL, S.P, s)) != PLQ_OK) break;
                if ((st = blas_zero(S.Vh, xL, S.PX, s)) != PLQ_OK) break;
                target2 = std::pow(sigma * P.tol * bnorm, 2);
                init.c_rho = make_double2(s2, 0.0);
                init.stop_r2 = std::fmax(delta * delta * s2, target2);
                init.tiny = 1e-300;
                if ((st = put_state(S, init)) != PLQ_OK) break;
                const double kk = kappa * kappa;
                const int PI = S.P;
                auto body = [&]() -> plq_status {
                    PLQ_TRY(hop(S, PI, 1, toL, pL, EPI_PLAIN, 0, nullptr, 0.0, FIN_NONE, nullptr, true));
                    PLQ_TRY(hop(S, PI, 0, vL, toL, EPI_XPAY_DOTW, 0, pL, -kk, FIN_BICG_ALPHA, rhL, true));
                    PLQ_TRY(blas_bicg_s(S.Vh, sL, rL, vL, PI, c->state, s));
                    PLQ_TRY(hop(S, PI, 1, toL, sL, EPI_PLAIN, 0, nullptr, 0.0, FIN_NONE, nullptr, true));
                    PLQ_TRY(hop(S, PI, 0, tL, toL, EPI_XPAY_TS, 0, sL, -kk, FIN_BICG_OMEGA, nullptr, true));
                    Reduce rb = reduce_of(c, FIN_BICG_RHO);
                    PLQ_TRY(blas_bicg_update(S.Vh, xL, rL, pL, sL, tL, rhL, PI, rb, c->state, s));
                    return blas_bicg_p(S.Vh, pL, rL, vL, PI, c->state, s);
                };
                if ((st = run_batches(S, P.k, body, &fin)) != PLQ_OK) break;
            }
            const int done = fin.iter - start_iter;
            S.hops += 4.0 * done;
            iters = fin.iter;
            if (fin.flags & FLAG_NAN) {
                result = set_error(PLQ_ERR_NAN, "NaN or Inf in the inner iteration");
                break;
            }
            if ((fin.flags & FLAG_BREAKDOWN) && done == 0) {
                result = set_error(PLQ_ERR_BREAKDOWN, "Krylov breakdown (rho or omega vanished)");
                break;
            }
            // reliable update: x_e += x_inner (FP64)
            if ((st = blas_accumulate(S.Vh, xe, xL, S.PX, s)) != PLQ_OK) break;
            ++n_rel;
            first = false;
            // the inner target was reached but the FP64 check may still fail:
            // tighten the estimate for the next round
            const double fr = method == SOLVER_CG ? fin.rho : fin.r2;
            // FIN_CG_BETA left rho = rho_{k+1} and beta = rho_{k+1} / rho_k
            last_rho = fin.beta > 0.0 ? fin.rho / fin.beta : fin.rho;
            if (fr <= target2 * 1.0000001) sigma *= 0.25;
        }
        if (st != PLQ_OK || result != PLQ_OK) break;
        // x_o = b_o + kappa H_oe x_e
        if ((st = hop(S, PLQ_F64, 1, xo, xe, EPI_XPAY, 0, bo, kappa)) != PLQ_OK) break;
        // full true residual ||b - M x|| with the FP64 operator, both parities
        double re = 0, ro = 0;
        if ((st = hop(S, PLQ_F64, 0, t64, xo, EPI_XPAY, 0, xe, -kappa)) != PLQ_OK) break;
        if ((st = blas_xpay64(S.Vh, be, -1.0, t64, s)) != PLQ_OK) break;
        if ((st = norm2_64(S, t64, &re)) != PLQ_OK) break;
        if ((st = hop(S, PLQ_F64, 1, tmp_o64, xe, EPI_XPAY, 0, xo, -kappa)) != PLQ_OK) break;
        if ((st = blas_xpay64(S.Vh, bo, -1.0, tmp_o64, s)) != PLQ_OK) break;
        if ((st = norm2_64(S, tmp_o64, &ro)) != PLQ_OK) break;
        true_rel = std::sqrt((re + ro) / bnorm2);
        if (!(true_rel <= P.tol) && result == PLQ_OK)
            result = set_error(PLQ_ERR_NOT_CONVERGED, "final residual %.3e above tol %.3e", true_rel, P.tol);
    } while (0);

    cudaError_t e1 = cudaEventRecord(ev1, s);
    if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(user, ev1, 0);
    if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(s);
    auto wall1 = std::chrono::steady_clock::now();
    cleanup();
    if (st == PLQ_OK && e1 != cudaSuccess) st = cuda_error(e1, "solver completion");
    const int status = st != PLQ_OK ? st : result;
    if (info) {
        info->status = status;
        info->iterations = iters;
        info->n_reliable = n_rel;
        info->true_rel_residual = true_rel;
        info->seconds = std::chrono::duration<double>(wall1 - wall0).count();
        info->hop_applications = S.hops;
    }
    return status;
}

}  // namespace
}  // namespace plq

extern "C" {

plq_status plq_cg_solve(plq_ctx *ctx, void *x, const void *b, double kappa, const plq_solver_params *params,
                        plq_solve_info *info, void *stream) {
    return plq::solve_impl(ctx, x, b, kappa, params, info, stream, plq::SOLVER_CG);
}

plq_status plq_bicgstab_solve(plq_ctx *ctx, void *x, const void *b, double kappa, const plq_solver_params *params,
                              plq_solve_info *info, void *stream) {
    return plq::solve_impl(ctx, x, b, kappa, params, info, stream, plq::SOLVER_BICGSTAB);
}

}  // extern "C"
