// C ABI of libplq: context, errors, gauge upload, layout conversion and the
// operator entry points (hopping, Wilson, Schur).  Solvers live in
// plq_solvers.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "plq_internal.cuh"

namespace plq {

static thread_local char g_err[512] = "";

plq_status set_error(plq_status code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

plq_status cuda_error(cudaError_t e, const char *what) {
    return set_error(e == cudaErrorMemoryAllocation ? PLQ_ERR_NOMEM : PLQ_ERR_CUDA, "%s: %s (%s)", what,
                     cudaGetErrorString(e), cudaGetErrorName(e));
}

plq_status launch_hop_f64_18(const HopArgs &a, int epi, cudaStream_t s, int block);
plq_status launch_hop_f64_12(const HopArgs &a, int epi, cudaStream_t s, int block);
plq_status launch_hop_f32_18(const HopArgs &a, int epi, cudaStream_t s, int block);
plq_status launch_hop_f32_12(const HopArgs &a, int epi, cudaStream_t s, int block);
plq_status launch_hop_f16_18(const HopArgs &a, int epi, cudaStream_t s, int block);
plq_status launch_hop_f16_12(const HopArgs &a, int epi, cudaStream_t s, int block);

int hop_default_block(int prec) { return prec == PLQ_F64 ? 128 : 128; }

plq_status launch_hop(const HopArgs &a, int prec, int reals, int epi, cudaStream_t s) {
    const int block = a.block > 0 ? a.block : hop_default_block(prec);
    const bool r12 = reals == 12;
    switch (prec) {
    case PLQ_F64: return r12 ? launch_hop_f64_12(a, epi, s, block) : launch_hop_f64_18(a, epi, s, block);
    case PLQ_F32: return r12 ? launch_hop_f32_12(a, epi, s, block) : launch_hop_f32_18(a, epi, s, block);
    case PLQ_F16: return r12 ? launch_hop_f16_12(a, epi, s, block) : launch_hop_f16_18(a, epi, s, block);
    default: return set_error(PLQ_ERR_ARG, "bad precision %d", prec);
    }
}

plq_status ensure_work(Ctx *c, size_t bytes) {
    if (c->work_bytes >= bytes) return PLQ_OK;
    if (c->work) {
        cudaFree(c->work);
        c->work = nullptr;
        c->work_bytes = 0;
    }
    PLQ_CUDA(cudaMalloc(&c->work, bytes));
    c->work_bytes = bytes;
    return PLQ_OK;
}

plq_status ensure_pipeline(Ctx *c) {
    if (c->copy_in) return PLQ_OK;
    PLQ_CUDA(cudaStreamCreateWithFlags(&c->copy_in, cudaStreamNonBlocking));
    PLQ_CUDA(cudaStreamCreateWithFlags(&c->copy_out, cudaStreamNonBlocking));
    PLQ_CUDA(cudaStreamCreateWithFlags(&c->compute, cudaStreamNonBlocking));
    for (auto &e : c->ev) PLQ_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return PLQ_OK;
}

plq_status ensure_stage(Ctx *c, size_t bytes) {
    if (c->stage_bytes >= bytes) return PLQ_OK;
    if (c->stage) {
        cudaFree(c->stage);
        c->stage = nullptr;
        c->stage_bytes = 0;
    }
    PLQ_CUDA(cudaMalloc(&c->stage, bytes));
    c->stage_bytes = bytes;
    return PLQ_OK;
}

}  // namespace plq

using namespace plq;

namespace {

bool aligned16(const void *p) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

plq_status check_ctx(const plq_ctx *ctx) {
    if (!ctx) return set_error(PLQ_ERR_ARG, "null context");
    return PLQ_OK;
}

plq_status use_device(const plq_ctx *ctx) {
    PLQ_CUDA(cudaSetDevice(ctx->device));
    return PLQ_OK;
}

plq_status need_gauge(const plq_ctx *ctx, int prec) {
    if (!valid_prec(prec)) return set_error(PLQ_ERR_ARG, "bad precision %d", prec);
    if (!ctx->gauge[prec].ptr)
        return set_error(PLQ_ERR_STATE, "no gauge field uploaded for precision %d (call plq_gauge_upload)", prec);
    return PLQ_OK;
}

HopArgs hop_args(const plq_ctx *ctx, int prec, int out_parity, void *out, const void *in, int nrhs = 1) {
    HopArgs a;
    a.nrhs = nrhs;
    a.in = in;
    a.out = out;
    a.gauge = ctx->gauge[prec].ptr;
    a.gblock = ctx->gauge[prec].block;
    a.out_parity = out_parity;
    a.lat = ctx->lat;
    apply_tune(ctx, prec, nrhs, a);
    return a;
}

}  // namespace

extern "C" {

const char *plq_last_error(void) { return g_err; }

int plq_version(void) { return 1 * 10000 + 0 * 100 + 0; }

plq_status plq_init(plq_ctx **out, const int dims[4], int t_bc, int device) {
    g_err[0] = 0;
    if (!out || !dims) return set_error(PLQ_ERR_ARG, "null argument");
    *out = nullptr;
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || (dims[mu] & 1))
            return set_error(PLQ_ERR_ARG, "dims[%d] = %d: every extent must be even and >= 2", mu, dims[mu]);
        V *= dims[mu];
    }
    if (V > (1LL << 30)) return set_error(PLQ_ERR_ARG, "volume %lld above 2^30 sites", V);
    if (t_bc != 1 && t_bc != -1) return set_error(PLQ_ERR_ARG, "t_bc must be +1 or -1 (got %d)", t_bc);
    int ndev = 0;
    PLQ_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return set_error(PLQ_ERR_ARG, "device %d of %d", device, ndev);
    PLQ_CUDA(cudaSetDevice(device));
    plq_ctx *c = new (std::nothrow) plq_ctx();
    if (!c) return set_error(PLQ_ERR_NOMEM, "host allocation");
    c->lat = make_lattice(dims, t_bc);
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaMalloc(&c->partials, sizeof(double) * kPartialSlots * kMaxReduceBlocks);
    if (e == cudaSuccess) e = cudaMalloc(&c->kstatus, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(c->kstatus, 0, sizeof(int) * 4);
    {
        int khz = 0;  // SM clock in kHz: kernel waits count clock64() cycles
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
        c->spin_limit = (long long)(5.0 * (khz > 0 ? khz : 2000000) * 1e3);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->ticket, sizeof(unsigned) * 16);
    if (e == cudaSuccess) e = cudaMalloc(&c->sums, sizeof(double) * kPartialSlots);
    if (e == cudaSuccess) e = cudaMalloc(&c->state, sizeof(SolverState) * PLQ_MAX_RHS);
    if (e == cudaSuccess) e = cudaMallocHost(&c->sums_host, sizeof(double) * kPartialSlots);
    if (e == cudaSuccess) e = cudaMallocHost(&c->state_host, sizeof(SolverState) * PLQ_MAX_RHS);
    if (e == cudaSuccess) e = cudaMemset(c->ticket, 0, sizeof(unsigned) * 16);
    if (e == cudaSuccess) e = cudaMemset(c->state, 0, sizeof(SolverState) * PLQ_MAX_RHS);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        plq_status st = cuda_error(e, "plq_init allocation");
        plq_finalize(c);
        return st;
    }
    *out = c;
    return PLQ_OK;
}

plq_status plq_finalize(plq_ctx *c) {
    if (!c) return PLQ_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto &g : c->gauge)
        if (g.ptr) cudaFree(g.ptr);
    if (c->gauge_df.ptr) cudaFree(c->gauge_df.ptr);
    for (auto &g : c->solve_graph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->host_graph.exec) cudaGraphExecDestroy(c->host_graph.exec);
    for (auto &t : c->nbr)
        if (t) cudaFree(t);
    if (c->partials) cudaFree(c->partials);
    if (c->kstatus) cudaFree(c->kstatus);
    if (c->ticket) cudaFree(c->ticket);
    if (c->sums) cudaFree(c->sums);
    if (c->state) cudaFree(c->state);
    if (c->sums_host) cudaFreeHost(c->sums_host);
    if (c->state_host) cudaFreeHost(c->state_host);
    if (c->work) cudaFree(c->work);
    if (c->stage) cudaFree(c->stage);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->copy_in) cudaStreamDestroy(c->copy_in);
    if (c->copy_out) cudaStreamDestroy(c->copy_out);
    if (c->compute) cudaStreamDestroy(c->compute);
    if (c->batch.exec) cudaGraphExecDestroy(c->batch.exec);
    if (c->batch.scratch) cudaFree(c->batch.scratch);
    if (c->batch.stream) cudaStreamDestroy(c->batch.stream);
    delete c;
    return PLQ_OK;
}

long plq_half_volume(const plq_ctx *c) { return c ? (long)c->lat.Vh : 0; }

plq_status plq_set_wait_limit(plq_ctx *c, double seconds) {
    PLQ_TRY(check_ctx(c));
    if (!(seconds > 0.0) || !std::isfinite(seconds)) return set_error(PLQ_ERR_ARG, "wait limit must be > 0 s");
    int khz = 0;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->device);
    const double cyc = seconds * (khz > 0 ? khz : 2000000) * 1e3;
    c->spin_limit = cyc < 1.0 ? 1LL : cyc > 1e15 ? (long long)1e15 : (long long)cyc;
    return PLQ_OK;
}

plq_status plq_device_status(plq_ctx *c, int clear) {
    PLQ_TRY(check_ctx(c));
    PLQ_TRY(use_device(c));
    int v = 0;
    PLQ_CUDA(cudaMemcpy(&v, c->kstatus, sizeof(int), cudaMemcpyDeviceToHost));
    if (clear && v != 0) PLQ_CUDA(cudaMemset(c->kstatus, 0, sizeof(int)));
    if (v != 0) return set_error(v, "a kernel of this context gave up a bounded wait (status %d)", v);
    return PLQ_OK;
}

size_t plq_field_bytes(const plq_ctx *c, int prec, int nrhs) {
    if (c && prec == PLQ_DF64 && nrhs >= 1 && nrhs <= PLQ_MAX_RHS) return df_site_bytes() * (size_t)c->lat.Vh * nrhs;
    if (!c || !valid_prec(prec) || nrhs < 1 || nrhs > PLQ_MAX_RHS) return 0;
    return spinor_site_bytes(prec) * (size_t)c->lat.Vh * (size_t)nrhs;
}

plq_status plq_gauge_upload(plq_ctx *c, const double *U, int is_device, int link_reals, int prec, void *stream) {
    PLQ_TRY(check_ctx(c));
    if (!U) return set_error(PLQ_ERR_ARG, "null gauge field");
    if (link_reals != 18 && link_reals != 12) return set_error(PLQ_ERR_ARG, "link_reals must be 18 or 12");
    if (!valid_prec(prec) && prec != PLQ_DF64) return set_error(PLQ_ERR_ARG, "bad precision %d", prec);
    if (is_device && !aligned16(U)) return set_error(PLQ_ERR_ARG, "gauge pointer not 16-byte aligned");
    PLQ_TRY(use_device(c));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == PLQ_DF64) return df_gauge_upload(c, U, is_device, link_reals, s);
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
    GaugeCopy &g = c->gauge[prec];
    const size_t block = link_site_bytes(prec, link_reals) * c->lat.Vh;
    if (g.ptr && (g.block != block)) {
        cudaStreamSynchronize(s);
        cudaFree(g.ptr);
        g.ptr = nullptr;
    }
    plq_status st = PLQ_OK;
    if (!g.ptr) {
        cudaError_t e = cudaMalloc(&g.ptr, block * 8);
        if (e != cudaSuccess) {
            st = cuda_error(e, "gauge allocation");
            g.ptr = nullptr;
        }
    }
    unsigned *bad = c->ticket + 8;
    if (st == PLQ_OK) {
        cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) st = cuda_error(e, "memset");
    }
    if (st == PLQ_OK) st = launch_pack_gauge(c->lat, g.ptr, src, prec, link_reals, block, bad, s);
    unsigned bad_h = 0;
    if (st == PLQ_OK) {
        cudaError_t e = cudaMemcpyAsync(&bad_h, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "gauge pack");
    }
    if (tmp) cudaFree(tmp);
    if (st != PLQ_OK) return st;
    if (bad_h) {
        cudaFree(g.ptr);
        g = GaugeCopy();
        return set_error(PLQ_ERR_ARG, "link_reals = 12 needs SU(3) links (deviation above 1e-12)");
    }
    g.reals = link_reals;
    g.block = block;
    return PLQ_OK;
}

plq_status plq_pack_spinor(plq_ctx *c, void *out, const double *in, int prec, int nrhs, void *stream) {
    PLQ_TRY(check_ctx(c));
    if (!aligned16(out) || !aligned16(in)) return set_error(PLQ_ERR_ARG, "null or misaligned field pointer");
    if (!valid_prec(prec) && prec != PLQ_DF64) return set_error(PLQ_ERR_ARG, "bad precision %d", prec);
    if (nrhs < 1 || nrhs > PLQ_MAX_RHS) return set_error(PLQ_ERR_ARG, "nrhs must be in 1..%d", PLQ_MAX_RHS);
    PLQ_TRY(use_device(c));
    if (prec == PLQ_DF64) return df_pack_spinor(c->lat, out, in, nrhs, static_cast<cudaStream_t>(stream));
    return launch_pack_spinor(c->lat, out, in, prec, nrhs, static_cast<cudaStream_t>(stream));
}

plq_status plq_unpack_spinor(plq_ctx *c, double *out, const void *in, int prec, int nrhs, void *stream) {
    PLQ_TRY(check_ctx(c));
    if (!aligned16(out) || !aligned16(in)) return set_error(PLQ_ERR_ARG, "null or misaligned field pointer");
    if (!valid_prec(prec) && prec != PLQ_DF64) return set_error(PLQ_ERR_ARG, "bad precision %d", prec);
    if (nrhs < 1 || nrhs > PLQ_MAX_RHS) return set_error(PLQ_ERR_ARG, "nrhs must be in 1..%d", PLQ_MAX_RHS);
    PLQ_TRY(use_device(c));
    if (prec == PLQ_DF64) return df_unpack_spinor(c->lat, out, in, nrhs, static_cast<cudaStream_t>(stream));
    return launch_unpack_spinor(c->lat, out, in, prec, nrhs, static_cast<cudaStream_t>(stream));
}

plq_status plq_hopping_eo(plq_ctx *c, int out_parity, void *out, const void *in, int prec, int nrhs, void *stream) {
    PLQ_TRY(check_ctx(c));
    if (!aligned16(out) || !aligned16(in)) return set_error(PLQ_ERR_ARG, "null or misaligned field pointer");
    if (out == in) return set_error(PLQ_ERR_ARG, "in and out must not overlap");
    if (out_parity != 0 && out_parity != 1) return set_error(PLQ_ERR_ARG, "out_parity must be 0 or 1");
    if (nrhs < 1 || nrhs > PLQ_MAX_RHS) return set_error(PLQ_ERR_ARG, "nrhs must be in 1..%d", PLQ_MAX_RHS);
    if (prec == PLQ_DF64) {
        PLQ_TRY(use_device(c));
        return df_hop(c, out_parity, out, in, nullptr, 0.0, 0.0, 1.0, nrhs, static_cast<cudaStream_t>(stream));
    }
    PLQ_TRY(need_gauge(c, prec));
    PLQ_TRY(use_device(c));
    HopArgs a = hop_args(c, prec, out_parity, out, in, nrhs);
    return launch_hop(a, prec, c->gauge[prec].reals, EPI_PLAIN, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {

constexpr int kMaxHostSlabs = 64;

// Time-slice boundaries bound[0..K] (bound[0] = 0, bound[K] = T) of the host
// pipeline's slabs: ramps of 1, 1, 2, 4, ... slices (each below T/8) at both
// ends, slabs of T/8 slices between them; returns K.
int host_slab_bounds(int T, int *bound) {
    const int m = T / 8 > 1 ? T / 8 : 1;
    int ramp[16], nr = 0, rs = 0;
    for (int v = 1; nr < 16;) {
        if (v >= m || 2 * (rs + v) > T) break;
        ramp[nr++] = v;
        rs += v;
        if (nr >= 2) v *= 2;
    }
    int sizes[kMaxHostSlabs], K = 0;
    for (int q = 0; q < nr; ++q) sizes[K++] = ramp[q];
    int mid = T - 2 * rs;
    while (mid > 0 && K < kMaxHostSlabs - nr) {
        const int v = mid < m ? mid : m;
        sizes[K++] = v;
        mid -= v;
    }
    if (mid > 0) sizes[K - 1] += mid;  // unreachable for T <= 8 * kMaxHostSlabs / 2
    for (int q = nr - 1; q >= 0; --q) sizes[K++] = ramp[q];
    bound[0] = 0;
    for (int k = 0; k < K; ++k) bound[k + 1] = bound[k] + sizes[k];
    return K;
}

// Enqueue the host pipeline of plq_hopping_eo_host.  `origin` is the stream
// the copies in start from and that ends ordered after the last copy out.
plq_status enqueue_host_pipeline(plq_ctx *c, int out_parity, char *hout, const char *hin, int prec, int nrhs,
                                 cudaStream_t origin) {
    const size_t bytes = plq_field_bytes(c, prec, nrhs);
    char *din = static_cast<char *>(c->stage), *dout = din + bytes;
    // Pipeline over time slabs, the overlap of Sec. 2.2 applied to the host
    // link: input slabs stream in on one copy engine, the output sites whose
    // neighbours (t - 1, t, t + 1) have all arrived are computed, and finished
    // output slabs stream back on the other engine while later slabs compute.
    const int T = c->lat.L[0];
    const int slab = c->lat.Vh / T;  // checkerboard sites per time slice
    // Slab sizes: each copy costs ~6 us on top of its bytes, while the first
    // output waits for three input slabs and the last copy out follows the
    // last compute.  So the slabs grow 1, 1, 2, 4, ... time slices up to T/8
    // and shrink the same way at the end: short fill and drain, few copies.
    // 32^3x64 FP32 (100 MB each way): 0.813 ms, against 0.829 ms with 16
    // equal slabs; the link moves the same bytes in 0.60 ms as one copy in
    // each direction.
    int bound[kMaxHostSlabs + 1];
    const int K = host_slab_bounds(T, bound);
    const size_t n = (size_t)nrhs, VhN = (size_t)c->lat.Vh * n;
    const int nplanes = prec == PLQ_F64 ? 12 : prec == PLQ_F32 ? 6 : 3;
    auto chunk_t0 = [&](int k) { return bound[k]; };
    auto copy_chunk = [&](char *dst, const char *src, int k, cudaMemcpyKind kind, cudaStream_t s) -> cudaError_t {
        const size_t e0 = (size_t)chunk_t0(k) * slab * n, e1 = (size_t)chunk_t0(k + 1) * slab * n;
        cudaError_t e = cudaMemcpy2DAsync(dst + e0 * 16, VhN * 16, src + e0 * 16, VhN * 16, (e1 - e0) * 16, nplanes,
                                          kind, s);
        if (e == cudaSuccess && prec == PLQ_F16)  // per-site norms
            e = cudaMemcpyAsync(dst + 48 * VhN + e0 * 4, src + 48 * VhN + e0 * 4, (e1 - e0) * 4, kind, s);
        return e;
    };
    cudaEvent_t *ev_in = c->ev, *ev_done = c->ev + 64, *ev_start = c->ev + 128;
    PLQ_CUDA(cudaEventRecord(ev_start[0], origin));
    PLQ_CUDA(cudaStreamWaitEvent(c->compute, ev_start[0], 0));
    PLQ_CUDA(cudaStreamWaitEvent(c->copy_out, ev_start[0], 0));
    // input order: the last slab first (slab 0 needs it through the periodic time direction)
    for (int q = 0; q < K; ++q) {
        const int k = (q + K - 1) % K;
        PLQ_CUDA(copy_chunk(din, hin, k, cudaMemcpyHostToDevice, origin));
        PLQ_CUDA(cudaEventRecord(ev_in[k], origin));
    }
    for (int k = 0; k < K; ++k) {
        // slabs k - 1 and k arrived before slab k + 1 (copy order), except
        // at the start, where K - 1, 0 and 1 are needed
        if (k == 0) {
            PLQ_CUDA(cudaStreamWaitEvent(c->compute, ev_in[K - 1], 0));
            PLQ_CUDA(cudaStreamWaitEvent(c->compute, ev_in[0], 0));
        }
        PLQ_CUDA(cudaStreamWaitEvent(c->compute, ev_in[(k + 1) % K], 0));
        HopArgs a = hop_args(c, prec, out_parity, dout, din, nrhs);
        a.site_begin = chunk_t0(k) * slab;
        a.site_end = chunk_t0(k + 1) * slab;
        a.zc = 0;  // site ranges are in checkerboard order
        PLQ_TRY(launch_hop(a, prec, c->gauge[prec].reals, EPI_PLAIN, c->compute));
        PLQ_CUDA(cudaEventRecord(ev_done[k], c->compute));
        PLQ_CUDA(cudaStreamWaitEvent(c->copy_out, ev_done[k], 0));
        PLQ_CUDA(copy_chunk(hout, dout, k, cudaMemcpyDeviceToHost, c->copy_out));
    }
    PLQ_CUDA(cudaEventRecord(ev_start[1], c->copy_out));
    PLQ_CUDA(cudaStreamWaitEvent(origin, ev_start[1], 0));
    return PLQ_OK;
}

}  // namespace

extern "C" {

int plq_host_slabs(int T, int *bounds) {
    if (T < 2 || (T & 1) || !bounds) return 0;
    int b[kMaxHostSlabs + 1];
    const int K = host_slab_bounds(T, b);
    for (int k = 0; k <= K; ++k) bounds[k] = b[k];
    return K;
}

plq_status plq_hopping_eo_host(plq_ctx *c, int out_parity, void *out_host, const void *in_host, int prec, int nrhs,
                               void *stream) {
    PLQ_TRY(check_ctx(c));
    if (!out_host || !in_host) return set_error(PLQ_ERR_ARG, "null host pointer");
    if (out_parity != 0 && out_parity != 1) return set_error(PLQ_ERR_ARG, "out_parity must be 0 or 1");
    if (nrhs < 1 || nrhs > PLQ_MAX_RHS) return set_error(PLQ_ERR_ARG, "nrhs must be in 1..%d", PLQ_MAX_RHS);
    PLQ_TRY(need_gauge(c, prec));
    PLQ_TRY(use_device(c));
    const size_t bytes = plq_field_bytes(c, prec, nrhs);
    PLQ_TRY(ensure_stage(c, 2 * bytes));
    PLQ_TRY(ensure_pipeline(c));
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    const char *hin = static_cast<const char *>(in_host);
    char *hout = static_cast<char *>(out_host);
    // The ~150 copies, launches and event operations of the pipeline are
    // captured once into a CUDA graph and replayed while the buffers and the
    // launch configuration stay the same (pageable host memory, which graphs
    // cannot copy from asynchronously, takes the direct path).
    cudaPointerAttributes pa{}, pb{};
    const bool pinned = cudaPointerGetAttributes(&pa, hin) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
                        cudaPointerGetAttributes(&pb, hout) == cudaSuccess && pb.type == cudaMemoryTypeHost;
    cudaGetLastError();  // a pageable pointer may leave an error from the attribute query
    // (the captured launches hold the gauge copy's address: a re-upload in another
    // link format reallocates it)
    unsigned long long key[8] = {reinterpret_cast<uintptr_t>(hin),
                                 reinterpret_cast<uintptr_t>(hout),
                                 (unsigned long long)prec | ((unsigned long long)nrhs << 8) |
                                     ((unsigned long long)out_parity << 16) |
                                     ((unsigned long long)c->gauge[prec].reals << 24),
                                 reinterpret_cast<uintptr_t>(c->stage),
                                 (unsigned long long)c->tune_version,
                                 reinterpret_cast<uintptr_t>(c->gauge[prec].ptr),
                                 (unsigned long long)c->gauge[prec].block,
                                 1ull};
    Ctx::HostGraph &hg = c->host_graph;
    if (pinned && !(hg.exec && std::memcmp(hg.key, key, sizeof(key)) == 0)) {
        if (hg.exec) {
            cudaGraphExecDestroy(hg.exec);
            hg.exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        PLQ_CUDA(cudaStreamBeginCapture(c->copy_in, cudaStreamCaptureModeThreadLocal));
        plq_status st = enqueue_host_pipeline(c, out_parity, hout, hin, prec, nrhs, c->copy_in);
        cudaError_t e = cudaStreamEndCapture(c->copy_in, &graph);
        if (st == PLQ_OK && e == cudaSuccess) e = cudaGraphInstantiate(&hg.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (st != PLQ_OK) return st;
        if (e != cudaSuccess) {
            hg.exec = nullptr;
            return cuda_error(e, "host pipeline graph");
        }
        std::memcpy(hg.key, key, sizeof(key));
    }
    cudaEvent_t *ev_start = c->ev + 128;
    PLQ_CUDA(cudaEventRecord(ev_start[2], user));
    PLQ_CUDA(cudaStreamWaitEvent(c->copy_in, ev_start[2], 0));
    if (pinned) PLQ_CUDA(cudaGraphLaunch(hg.exec, c->copy_in));
    else PLQ_TRY(enqueue_host_pipeline(c, out_parity, hout, hin, prec, nrhs, c->copy_in));
    PLQ_CUDA(cudaEventRecord(ev_start[3], c->copy_in));
    PLQ_CUDA(cudaStreamWaitEvent(user, ev_start[3], 0));
    PLQ_CUDA(cudaStreamSynchronize(user));
    return PLQ_OK;
}

plq_status plq_wilson_apply(plq_ctx *c, void *out, const void *in, double kappa, int prec, void *stream) {
    PLQ_TRY(check_ctx(c));
    if (!aligned16(out) || !aligned16(in)) return set_error(PLQ_ERR_ARG, "null or misaligned field pointer");
    if (out == in) return set_error(PLQ_ERR_ARG, "in and out must not overlap");
    PLQ_TRY(need_gauge(c, prec));
    PLQ_TRY(use_device(c));
    const size_t half = plq_field_bytes(c, prec, 1);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const char *ie = static_cast<const char *>(in), *io = ie + half;
    char *oe = static_cast<char *>(out), *oo = oe + half;
    // out_e = in_e - kappa H_eo in_o ; out_o = in_o - kappa H_oe in_e
    HopArgs a = hop_args(c, prec, 0, oe, io);
    a.x = ie;
    a.a = -kappa;
    PLQ_TRY(launch_hop(a, prec, c->gauge[prec].reals, EPI_XPAY, s));
    HopArgs b = hop_args(c, prec, 1, oo, ie);
    b.x = io;
    b.a = -kappa;
    return launch_hop(b, prec, c->gauge[prec].reals, EPI_XPAY, s);
}

plq_status plq_twisted_apply(plq_ctx *c, void *out, const void *in, double kappa, double mu, int prec,
                             void *stream) {
    PLQ_TRY(check_ctx(c));
    if (!aligned16(out) || !aligned16(in)) return set_error(PLQ_ERR_ARG, "null or misaligned field pointer");
    if (out == in) return set_error(PLQ_ERR_ARG, "in and out must not overlap");
    PLQ_TRY(need_gauge(c, prec));
    PLQ_TRY(use_device(c));
    const size_t half = plq_field_bytes(c, prec, 1);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const char *ie = static_cast<const char *>(in), *io = ie + half;
    char *oe = static_cast<char *>(out), *oo = oe + half;
    // out_p = (1 + 2 i kappa mu gamma5) in_p - kappa H_{p,1-p} in_{1-p}
    HopArgs a = hop_args(c, prec, 0, oe, io);
    a.x = ie;
    a.a = -kappa;
    a.nu_x = 2.0 * kappa * mu;
    PLQ_TRY(launch_hop(a, prec, c->gauge[prec].reals, EPI_XPAY, s));
    HopArgs b = hop_args(c, prec, 1, oo, ie);
    b.x = io;
    b.a = -kappa;
    b.nu_x = 2.0 * kappa * mu;
    return launch_hop(b, prec, c->gauge[prec].reals, EPI_XPAY, s);
}

plq_status plq_schur_apply(plq_ctx *c, void *out, const void *in, void *tmp, double kappa, int dagger, int prec,
                           void *stream) {
    PLQ_TRY(check_ctx(c));
    if (!aligned16(out) || !aligned16(in) || !aligned16(tmp))
        return set_error(PLQ_ERR_ARG, "null or misaligned field pointer");
    if (out == in || tmp == in || tmp == out) return set_error(PLQ_ERR_ARG, "in, out and tmp must be distinct");
    PLQ_TRY(need_gauge(c, prec));
    PLQ_TRY(use_device(c));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HopArgs a = hop_args(c, prec, 1, tmp, in);
    a.dagger = dagger ? 1 : 0;
    PLQ_TRY(launch_hop(a, prec, c->gauge[prec].reals, EPI_PLAIN, s));
    HopArgs b = hop_args(c, prec, 0, out, tmp);
    b.dagger = dagger ? 1 : 0;
    b.x = in;
    b.a = -kappa * kappa;
    return launch_hop(b, prec, c->gauge[prec].reals, EPI_XPAY, s);
}

}  // extern "C"
