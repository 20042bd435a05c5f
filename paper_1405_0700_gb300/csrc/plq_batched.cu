// Persistent batched CG: the host entry points (descriptor tables, the
// persistent scratch, stream and graph kept in the first context, the FP64
// verification of every returned solution, and the launch-shape tuner).  The
// kernel and its launcher are in plq_batched_impl.cuh, instantiated per inner
// format in plq_batched_*.cu.
#include <cstdio>
#include <cstdlib>
#include <string>

#include "plq_batched_impl.cuh"

using namespace plq;
using namespace plq::batch;

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
                                                                            : (inner == PLQ_F16 ? 1e-2 : 1e-4));
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
    // small batch scratch: descriptors, results, accumulators, barrier words;
    // kept in the first context with its stream and instantiated graph
    Ctx::BatchCache &bc = ctxs[0]->batch;
    const size_t bytes_sys = sizeof(BatchSystem) * n, bytes_res = sizeof(BatchResult) * n;
    const size_t bytes = bytes_sys + bytes_res + sizeof(double) * 3 * kMaxSys + 64;
    if (bc.bytes < bytes) {
        if (bc.exec) {
            cudaGraphExecDestroy(bc.exec);
            bc.exec = nullptr;
        }
        if (bc.scratch) cudaFree(bc.scratch);
        bc.scratch = nullptr;
        bc.bytes = 0;
        PLQ_CUDA(cudaMalloc(&bc.scratch, bytes));
        bc.bytes = bytes;
    }
    if (!bc.stream) PLQ_CUDA(cudaStreamCreateWithFlags(&bc.stream, cudaStreamNonBlocking));
    char *scratch = static_cast<char *>(bc.scratch);
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t s = bc.stream;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    plq_status stt = PLQ_OK;
    std::vector<BatchResult> res(n);
    LaunchOut lo;
    double secs = 0.0;
    do {
        cudaError_t e = cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev1, cudaEventDisableTiming);
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
        if (inner == PLQ_F16 && reals != 12) {
            stt = set_error(PLQ_ERR_ARG, "FP16 inner solves use 12-real links");
            break;
        }
        auto t0 = std::chrono::steady_clock::now();
        if (inner == PLQ_F64) stt = launch_f64_18(a, bc.shape, bc.blocks_per_sm, s, bc, &lo);
        else if (inner == PLQ_F32 && reals == 18) stt = launch_f32_18(a, bc.shape, bc.blocks_per_sm, s, bc, &lo);
        else if (inner == PLQ_F32) stt = launch_f32_12(a, bc.shape, bc.blocks_per_sm, s, bc, &lo);
        else stt = launch_f16_12(a, bc.shape, bc.blocks_per_sm, s, bc, &lo);
        if (stt != PLQ_OK) break;
        int status_word = 0;
        e = cudaMemcpyAsync(res.data(), a.res, bytes_res, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&status_word, a.status, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (e != cudaSuccess) {
            stt = cuda_error(e, "batched CG kernel");
            break;
        }
        if (status_word == PLQ_ERR_BOUNDS) {
            stt = set_error(PLQ_ERR_BOUNDS, "batched CG: a device bounds guard found an index out of range");
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
            // inner: 4 per iteration, 2 per reliable update; FP64: bhat, 2 per residual
            // check after the first (the first is free at x_e = 0), 2 for the check above
            infos[k].hop_applications =
                4.0 * res[k].iterations + 4.0 * res[k].n_reliable + (use_x0 ? 5.0 : 3.0);
        }
        if (st_k != PLQ_OK && status == PLQ_OK)
            status = set_error(st_k, "system %d: %s (residual %.3e after %d iterations)", k,
                               st_k == PLQ_ERR_NAN ? "NaN" : "not converged", rel, res[k].iterations);
    }
    if (binfo) {
        binfo->grid = lo.grid;
        binfo->block = lo.block;
        binfo->graph_captured = lo.captured ? 1 : 0;
        binfo->seconds = secs;
        binfo->launches = (stt == PLQ_OK) ? 1 : 0;
        binfo->blocks_per_sm = lo.bps;
        binfo->graph_reused = lo.reused ? 1 : 0;
    }
    if (ev1 && cudaEventRecord(ev1, s) == cudaSuccess) cudaStreamWaitEvent(user, ev1, 0);
    cudaStreamSynchronize(s);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    return status;
}

namespace {

int shape_of_block(int block) {
    for (int k = 0; k < kNumShapes; ++k)
        if (kShapes[k].block == block) return k;
    return -1;
}

// "GPU|batched|inner|links|n|lattice,lattice,..." (lattices in batch order)
std::string batch_key(plq_ctx **ctxs, int n, int inner) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, ctxs[0]->device);
    std::string k = prop.name;
    for (char &ch : k)
        if (ch == ' ') ch = '_';
    char buf[96];
    snprintf(buf, sizeof buf, "|batched|%d|%d|%d|", inner, ctxs[0]->gauge[inner].reals, n);
    k += buf;
    for (int i = 0; i < n; ++i) {
        snprintf(buf, sizeof buf, "%s%dx%dx%dx%d", i ? "," : "", ctxs[i]->lat.L[1], ctxs[i]->lat.L[2],
                 ctxs[i]->lat.L[3], ctxs[i]->lat.L[0]);
        k += buf;
    }
    return k;
}

bool batch_cache_lookup(const char *path, const std::string &key, int *block, int *bps, double *secs) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    std::vector<char> line(8192);
    bool found = false;
    while (fgets(line.data(), (int)line.size(), f)) {
        std::vector<char> k(line.size());
        int bl = 0, bp = 0;
        double sc = 0;
        if (sscanf(line.data(), "%8191s %d %d %lf", k.data(), &bl, &bp, &sc) == 4 && key == k.data() &&
            shape_of_block(bl) >= 0 && bp >= 0 && bp <= 64) {
            *block = bl;
            *bps = bp;
            *secs = sc;
            found = true;  // last entry wins
        }
    }
    fclose(f);
    return found;
}

}  // namespace

extern "C" plq_status plq_set_batched_launch(plq_ctx *ctx, int block, int blocks_per_sm) {
    if (!ctx) return set_error(PLQ_ERR_ARG, "null context");
    const int shape = block == 0 ? 0 : shape_of_block(block);
    if (shape < 0) return set_error(PLQ_ERR_ARG, "batched CG block must be 0, 64, 128, 192 or 256 (got %d)", block);
    if (blocks_per_sm < 0 || blocks_per_sm > 64) return set_error(PLQ_ERR_ARG, "blocks_per_sm must be in 0..64");
    ctx->batch.shape = shape;
    ctx->batch.blocks_per_sm = blocks_per_sm;
    ctx->batch.tuned = 1;
    return PLQ_OK;
}

extern "C" plq_status plq_autotune_batched(plq_ctx **ctxs, int n, void **x, const void **b, const double *kappa,
                                           const plq_solver_params *params, const char *cache_path,
                                           plq_batch_info *best_info) {
    if (best_info) std::memset(best_info, 0, sizeof(*best_info));
    if (!ctxs || n < 1 || n > kMaxSys || !ctxs[0]) return set_error(PLQ_ERR_ARG, "bad batch");
    const int inner = params ? params->inner_prec : PLQ_F64;
    if (!valid_prec(inner)) return set_error(PLQ_ERR_ARG, "bad inner precision %d", inner);
    if (!ctxs[0]->gauge[inner].ptr) return set_error(PLQ_ERR_STATE, "no gauge copy for the inner precision");
    const char *path = cache_path ? cache_path : getenv("PLQ_TUNE_CACHE");
    const std::string key = batch_key(ctxs, n, inner);
    Ctx::BatchCache &bc = ctxs[0]->batch;
    int blk = 0, bps = 0;
    double secs = 0;
    if (path && batch_cache_lookup(path, key, &blk, &bps, &secs)) {
        bc.shape = shape_of_block(blk);
        bc.blocks_per_sm = bps;
        bc.tuned = 1;
        if (best_info) {
            best_info->block = blk;
            best_info->blocks_per_sm = bps;
            best_info->seconds = secs;
        }
        return PLQ_OK;
    }
    // every shape with all resident blocks and with one block per SM fewer;
    // each candidate solves the batch twice (the first call captures its
    // graph) and is timed on the second
    double best = 1e300;
    int best_shape = 0, best_bps = 0;
    plq_batch_info bestbi{};
    for (int sh = 0; sh < kNumShapes; ++sh) {
        int full = 0;
        for (int pass = 0; pass < 2; ++pass) {
            const int want = pass == 0 ? 0 : full - 1;
            if (pass == 1 && want < 1) break;
            bc.shape = sh;
            bc.blocks_per_sm = want;
            plq_batch_info bi{};
            plq_status st = plq_cg_solve_batched(ctxs, n, x, b, kappa, params, nullptr, &bi, nullptr);
            if (st == PLQ_OK) st = plq_cg_solve_batched(ctxs, n, x, b, kappa, params, nullptr, &bi, nullptr);
            if (st != PLQ_OK) return st;
            if (pass == 0) full = bi.blocks_per_sm;
            if (bi.seconds < best) {
                best = bi.seconds;
                best_shape = sh;
                best_bps = want == 0 ? 0 : bi.blocks_per_sm;
                bestbi = bi;
            }
        }
    }
    bc.shape = best_shape;
    bc.blocks_per_sm = best_bps;
    bc.tuned = 1;
    if (best_info) *best_info = bestbi;
    if (path) {
        FILE *f = fopen(path, "a");
        if (f) {
            fprintf(f, "%s %d %d %.6f\n", key.c_str(), kShapes[best_shape].block, best_bps, best);
            fclose(f);
        }
    }
    return PLQ_OK;
}
