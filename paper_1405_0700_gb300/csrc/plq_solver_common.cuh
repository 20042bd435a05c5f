// Host-side helpers shared by the solver translation units: the launch of
// one hopping half-application inside a solve, reductions read back to the
// host, device solver states and graph-captured batches of iterations.
#pragma once

#include <cstring>
#include <vector>

#include "plq_fields.cuh"

namespace plq {
namespace {

struct Solve {
    plq_ctx *c;
    cudaStream_t s;  // internal capture-capable stream
    int Vh;
    int n;           // right-hand sides
    long long N;     // elements of a half field: Vh * n
    double kappa;
    int P;   // inner storage precision
    int PX;  // inner solution accumulator precision
    double nu = 0.0;  // twisted mass: nu = 2 kappa mu (0 = Wilson)
    double hops = 0;
};

// Twisted-mass terms of one hopping launch (all zero / one for Wilson).
struct Tw {
    double nu_x = 0.0, nu_h = 0.0, scale_h = 1.0;
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
               double a, int fin = FIN_NONE, const void *w = nullptr, bool freeze = false, Tw tw = Tw()) {
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
    h.nrhs = S.n;
    h.lat = c->lat;
    h.red = reduce_of(c, fin);
    if (fin == FIN_NONE) h.red.st = nullptr;
    h.st = freeze ? c->state : nullptr;
    h.nu_x = tw.nu_x;
    h.nu_h = tw.nu_h;
    h.scale_h = tw.scale_h;
    apply_tune(c, prec, S.n, h);
    S.hops += 1;
    return launch_hop(h, prec, c->gauge[prec].reals, epi, S.s);
}

// The two half-applications of Mhat (dagger: Mhat^dagger = gamma5 Mhat(-mu) gamma5):
//   Mhat v = A v - kappa^2 H_eo A^{-1} H_oe v,  A = 1 + i nu gamma5.
Tw tw_first(const Solve &S, bool dag) {  // A^{-1} (or A(-mu)^{-1}) on H_oe v
    Tw t;
    t.nu_h = dag ? S.nu : -S.nu;
    t.scale_h = 1.0 / (1.0 + S.nu * S.nu);
    return t;
}
Tw tw_second(const Solve &S, bool dag) {  // A (or A(-mu)) on the source
    Tw t;
    t.nu_x = dag ? -S.nu : S.nu;
    return t;
}
Tw tw_diag(const Solve &S) {  // A on the xpay source of a full M application
    Tw t;
    t.nu_x = S.nu;
    return t;
}

plq_status read_sums(Solve &S, double *out, int count) {
    PLQ_CUDA(cudaMemcpyAsync(S.c->sums_host, S.c->sums, sizeof(double) * count, cudaMemcpyDeviceToHost, S.s));
    PLQ_CUDA(cudaStreamSynchronize(S.s));
    for (int k = 0; k < count; ++k) out[k] = S.c->sums_host[k];
    return PLQ_OK;
}

// per right-hand side |v|^2 of an FP64 half field
plq_status norm2_64(Solve &S, const void *v, double *out) {
    Reduce r = reduce_of(S.c, FIN_NONE);
    r.st = nullptr;
    PLQ_TRY(blas_norm2(S.N, S.n, v, PLQ_F64, r, S.s));
    return read_sums(S, out, S.n);
}

plq_status put_states(Solve &S, const std::vector<SolverState> &st) {
    std::memcpy(S.c->state_host, st.data(), sizeof(SolverState) * S.n);
    PLQ_CUDA(cudaMemcpyAsync(S.c->state, S.c->state_host, sizeof(SolverState) * S.n, cudaMemcpyHostToDevice, S.s));
    PLQ_CUDA(cudaStreamSynchronize(S.s));
    return PLQ_OK;
}

plq_status get_states(Solve &S, std::vector<SolverState> &st) {
    PLQ_CUDA(cudaMemcpyAsync(S.c->state_host, S.c->state, sizeof(SolverState) * S.n, cudaMemcpyDeviceToHost, S.s));
    PLQ_CUDA(cudaStreamSynchronize(S.s));
    std::memcpy(st.data(), S.c->state_host, sizeof(SolverState) * S.n);
    return PLQ_OK;
}

// Run `body` (one inner iteration) as graph-captured batches of `k` until the
// device state of every right-hand side says stop.  With a cache, the
// instantiated graph is kept and reused while the key matches (the body's
// launches depend only on what the key records).
template <class Body>
plq_status run_batches(Solve &S, int k, Body body, std::vector<SolverState> &cur, Ctx::SolveGraph *cache = nullptr,
                       const unsigned long long *key = nullptr) {
    cudaGraphExec_t exec = nullptr;
    plq_status st = PLQ_OK;
    cudaError_t e = cudaSuccess;
    if (cache && cache->exec && std::memcmp(cache->key, key, sizeof(cache->key)) == 0) {
        exec = cache->exec;
    } else {
        cudaGraph_t graph = nullptr;
        PLQ_CUDA(cudaStreamBeginCapture(S.s, cudaStreamCaptureModeThreadLocal));
        const double hops0 = S.hops;
        for (int i = 0; i < k && st == PLQ_OK; ++i) st = body();
        e = cudaStreamEndCapture(S.s, &graph);
        S.hops = hops0;
        if (st != PLQ_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
        if (cache) {
            if (cache->exec) cudaGraphExecDestroy(cache->exec);
            cache->exec = exec;
            std::memcpy(cache->key, key, sizeof(cache->key));
        }
    }
    long long last_sum = -1;
    int idle = 0;
    for (;;) {
        e = cudaGraphLaunch(exec, S.s);
        if (e != cudaSuccess) {
            st = cuda_error(e, "cudaGraphLaunch");
            break;
        }
        st = get_states(S, cur);
        if (st != PLQ_OK) break;
        bool all = true;
        long long sum = 0;
        for (int r = 0; r < S.n; ++r) {
            all = all && cur[r].stop;
            sum += cur[r].iter;
        }
        if (all) break;
        // every batch advances some right-hand side unless all are frozen; a
        // state that neither advances nor stops is a logic error, not a hang
        idle = (sum == last_sum) ? idle + 1 : 0;
        last_sum = sum;
        if (idle >= 2) {
            st = set_error(PLQ_ERR_STATE, "inner iteration made no progress");
            break;
        }
    }
    if (!cache) cudaGraphExecDestroy(exec);
    return st;
}

}  // namespace
}  // namespace plq
