// Autotuner of the hopping kernel's launch: threads per block and the
// neighbour-index mode (inline coordinate arithmetic, or the precomputed
// neighbour table that plays the role of the pointer arrays of Sec. 2.2).
// Results are kept per (precision, nrhs) in the context and, optionally, in a
// text cache keyed by GPU name, lattice, precision, link format and nrhs.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "plq_fields.cuh"

namespace plq {
namespace {

__global__ void build_nbr_kernel(Lattice L, int par, int *tab) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.Vh; i += gridDim.x * blockDim.x) {
        const SiteGeom g = site_geom(L, par, i);
        for (int mu = 0; mu < 4; ++mu) {
            const int st = mu == 0 ? L.L[1] * L.L[2] * L.L[3] : mu == 1 ? 1 : mu == 2 ? L.L[1] : L.L[1] * L.L[2];
            const int c = g.c[mu], Lm = L.L[mu];
            const int fl = (c == Lm - 1) ? g.lex - (Lm - 1) * st : g.lex + st;
            const int bl = (c == 0) ? g.lex + (Lm - 1) * st : g.lex - st;
            const bool ff = mu == 0 && c == Lm - 1 && L.t_bc < 0;
            const bool fb = mu == 0 && c == 0 && L.t_bc < 0;
            tab[(size_t)(2 * mu) * L.Vh + i] = (fl >> 1) | (ff ? (int)0x80000000u : 0);
            tab[(size_t)(2 * mu + 1) * L.Vh + i] = (bl >> 1) | (fb ? (int)0x80000000u : 0);
        }
    }
}

const char *prec_name(int p) { return p == PLQ_F64 ? "f64" : p == PLQ_F32 ? "f32" : "f16"; }

std::string tune_key(const Ctx *c, int prec, int nrhs) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, c->device);
    char buf[512];
    snprintf(buf, sizeof buf, "%s|%dx%dx%dx%d|%s|%d|%d", prop.name, c->lat.L[1], c->lat.L[2], c->lat.L[3],
             c->lat.L[0], prec_name(prec), c->gauge[prec].reals, nrhs);
    for (char *p = buf; *p; ++p)
        if (*p == ' ') *p = '_';
    return buf;
}

bool cache_lookup(const char *path, const std::string &key, TuneEntry *e) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        char k[600];
        int block = 0, mode = 0, tile = 1, zc = 0, sm = 0, spt = 0;
        float us = 0;
        // key block index_mode rhs_tile z_chunk smem_links us [sites_per_thread]
        const int got = sscanf(line, "%599s %d %d %d %d %d %f %d", k, &block, &mode, &tile, &zc, &sm, &us, &spt);
        const bool valid = (block == 0 || (block >= 32 && block <= 1024 && block % 32 == 0)) && (mode == 0 || mode == 1) &&
                           (tile == 1 || tile == 2 || tile == 4) && zc >= 0 && sm >= 0 && sm <= 4 && spt >= 0 &&
                           spt <= 64 && !(sm >= 2 && tile != 1) && !(sm == 1 && tile == 4);
        if (got >= 7 && key == k && valid) {
            e->block = block;
            e->index_mode = mode;
            e->rhs_tile = tile;
            e->zc = zc;
            e->smem_links = sm;
            e->spt = spt;
            e->us = us;
            found = true;  // last entry wins
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const TuneEntry &e) {
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %.3f %d\n", key.c_str(), e.block, e.index_mode, e.rhs_tile, e.zc, e.smem_links,
            e.us, e.spt);
    fclose(f);
}

}  // namespace

plq_status ensure_nbr_tables(Ctx *c) {
    if (c->nbr[0] && c->nbr[1]) return PLQ_OK;
    for (int p = 0; p < 2; ++p) {
        if (c->nbr[p]) continue;
        PLQ_CUDA(cudaMalloc(&c->nbr[p], sizeof(int) * 8 * (size_t)c->lat.Vh));
        build_nbr_kernel<<<(c->lat.Vh + 255) / 256, 256>>>(c->lat, p, c->nbr[p]);
        PLQ_CUDA(cudaGetLastError());
    }
    PLQ_CUDA(cudaDeviceSynchronize());
    return PLQ_OK;
}

void apply_tune(const Ctx *c, int prec, int nrhs, HopArgs &a) {
    if (nrhs < 1 || nrhs > PLQ_MAX_RHS || !valid_prec(prec)) return;
    const TuneEntry &e = c->tune[prec][nrhs];
    if (e.block > 0) a.block = e.block;
    a.nbr = (e.index_mode == 1) ? c->nbr[a.out_parity] : nullptr;
    a.rhs_tile = (e.rhs_tile > 1 && nrhs % e.rhs_tile == 0) ? e.rhs_tile : 1;
    a.zc = (e.zc > 0 && c->lat.L[3] % e.zc == 0) ? e.zc : 0;
    a.smem_links = (nrhs > 1 || e.smem_links == 4) ? e.smem_links : 0;
    a.spt = e.spt;
    a.kstatus = c->kstatus;
    if (c->spin_limit > 0) a.spin_limit = c->spin_limit;
}

}  // namespace plq

using namespace plq;

extern "C" plq_status plq_autotune(plq_ctx *c, int prec, int nrhs, const char *cache_path, plq_tune_result *res) {
    if (!c) return set_error(PLQ_ERR_ARG, "null context");
    if (!valid_prec(prec)) return set_error(PLQ_ERR_ARG, "bad precision %d", prec);
    if (nrhs < 1 || nrhs > PLQ_MAX_RHS) return set_error(PLQ_ERR_ARG, "nrhs must be in 1..%d", PLQ_MAX_RHS);
    if (!c->gauge[prec].ptr) return set_error(PLQ_ERR_STATE, "autotune needs the gauge copy of precision %d", prec);
    PLQ_CUDA(cudaSetDevice(c->device));
    if (res) std::memset(res, 0, sizeof(*res));
    const char *path = cache_path ? cache_path : getenv("PLQ_TUNE_CACHE");
    const std::string key = tune_key(c, prec, nrhs);
    TuneEntry best;
    if (path && cache_lookup(path, key, &best)) {
        if (best.index_mode == 1) PLQ_TRY(ensure_nbr_tables(c));
        c->tune[prec][nrhs] = best;
        ++c->tune_version;
        if (res) {
            res->block = best.block;
            res->index_mode = best.index_mode;
            res->rhs_tile = best.rhs_tile;
            res->z_chunk = best.zc;
            res->smem_links = best.smem_links;
            res->sites_per_thread = best.spt;
            res->us_per_launch = best.us;
            res->from_cache = 1;
        }
        return PLQ_OK;
    }
    PLQ_TRY(ensure_nbr_tables(c));
    const size_t bytes = spinor_site_bytes(prec) * (size_t)c->lat.Vh * nrhs;
    void *in = nullptr, *out = nullptr;
    PLQ_CUDA(cudaMalloc(&in, bytes));
    cudaError_t e = cudaMalloc(&out, bytes);
    if (e != cudaSuccess) {
        cudaFree(in);
        return cuda_error(e, "autotune buffers");
    }
    cudaMemset(in, 0, bytes);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // block sizes a kernel cannot launch (registers x threads above the SM's
    // register file, or above its launch bound) are skipped
    static const int blocks[] = {64, 96, 128, 192, 256, 512, 1024};
    plq_status st = PLQ_OK;
    best.us = 1e30f;
    int tried = 0;
    const int reps = 10;
    // candidates: index mode x block size, plus right-hand-side tiles for nrhs > 1
    struct Cand {
        int mode, tile, zc, smem;
    };
    Cand cands[32];
    int nc = 0;
    const int Lz = c->lat.L[3];
    int zcs[3] = {0, 0, 0}, nz = 1;
    for (int z : {8, 4})
        if (z < Lz && Lz % z == 0) zcs[nz++] = z;
    for (int zi = 0; zi < nz; ++zi) {
        const int z = zcs[zi];
        cands[nc++] = {0, 1, z, 0};
        if (z == 0) cands[nc++] = {1, 1, 0, 0};
        if (prec != PLQ_F64 && nrhs % 2 == 0) cands[nc++] = {0, 2, z, 0};
        if (prec != PLQ_F64 && nrhs % 4 == 0) cands[nc++] = {0, 4, z, 0};
        if (prec != PLQ_F64 && nrhs > 1) cands[nc++] = {0, 1, z, 1};
        // neighbour spinors copied ahead into shared memory: wins for FP16 storage
        // on large lattices (site order chunks did not add to it)
        if (prec != PLQ_F64 && nrhs > 1 && z == 0) cands[nc++] = {0, 1, z, 2};
        if (prec != PLQ_F64 && nrhs > 1 && z == 0) cands[nc++] = {0, 1, z, 3};
        if (prec != PLQ_F64 && nrhs > 1 && nrhs % 2 == 0) cands[nc++] = {0, 2, z, 1};
    }
    // time one configuration; PLQ_ERR_ARG from the first launch means that
    // the block does not fit the kernel (us stays negative)
    auto time_cfg = [&](const TuneEntry &t, float *us_out) -> plq_status {
        HopArgs a;
        a.in = in;
        a.out = out;
        a.gauge = c->gauge[prec].ptr;
        a.gblock = c->gauge[prec].block;
        a.out_parity = 0;
        a.nrhs = nrhs;
        a.lat = c->lat;
        a.block = t.block;
        a.nbr = t.index_mode ? c->nbr[0] : nullptr;
        a.rhs_tile = t.rhs_tile;
        a.zc = t.zc;
        a.smem_links = t.smem_links;
        a.spt = t.spt;
        a.kstatus = c->kstatus;
        a.spin_limit = c->spin_limit;
        *us_out = -1.f;
        plq_status r = launch_hop(a, prec, c->gauge[prec].reals, EPI_PLAIN, s);
        if (r == PLQ_ERR_ARG) return PLQ_OK;
        if (r == PLQ_OK) r = launch_hop(a, prec, c->gauge[prec].reals, EPI_PLAIN, s);
        cudaEventRecord(e0, s);
        for (int q = 0; q < reps && r == PLQ_OK; ++q) r = launch_hop(a, prec, c->gauge[prec].reals, EPI_PLAIN, s);
        cudaEventRecord(e1, s);
        if (r != PLQ_OK) return r;
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) return cuda_error(ce, "autotune timing");
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        *us_out = ms * 1000.f / reps;
        ++tried;
        return PLQ_OK;
    };
    for (int ci = 0; ci < nc && st == PLQ_OK; ++ci) {
        for (int b : blocks) {
            TuneEntry t;
            t.block = b;
            t.index_mode = cands[ci].mode;
            t.rhs_tile = cands[ci].tile;
            t.zc = cands[ci].zc;
            t.smem_links = cands[ci].smem;
            float us = -1.f;
            st = time_cfg(t, &us);
            if (st != PLQ_OK) break;
            if (us >= 0.f && us < best.us) {
                t.us = us;
                best = t;
            }
        }
    }
    // sites per thread: a grid sized for k sites (site blocks) per thread
    // against the one-wave grid of the sweep above
    for (int k : {1, 2, 4, 8}) {
        if (st != PLQ_OK) break;
        TuneEntry t = best;
        t.spt = k;
        float us = -1.f;
        st = time_cfg(t, &us);
        if (st == PLQ_OK && us >= 0.f && us < best.us) {
            t.us = us;
            best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(in);
    cudaFree(out);
    if (st != PLQ_OK) return st;
    c->tune[prec][nrhs] = best;
    ++c->tune_version;
    if (path) cache_store(path, key, best);
    if (res) {
        res->block = best.block;
        res->index_mode = best.index_mode;
        res->rhs_tile = best.rhs_tile;
        res->z_chunk = best.zc;
        res->smem_links = best.smem_links;
        res->sites_per_thread = best.spt;
        res->us_per_launch = best.us;
        res->from_cache = 0;
        res->candidates = tried;
    }
    return PLQ_OK;
}

extern "C" plq_status plq_set_launch(plq_ctx *c, int prec, int nrhs, int block, int index_mode, int rhs_tile,
                                     int z_chunk, int smem_links, int sites_per_thread) {
    if (!c) return set_error(PLQ_ERR_ARG, "null context");
    if (!valid_prec(prec)) return set_error(PLQ_ERR_ARG, "bad precision %d", prec);
    if (nrhs < 1 || nrhs > PLQ_MAX_RHS) return set_error(PLQ_ERR_ARG, "nrhs must be in 1..%d", PLQ_MAX_RHS);
    if (block != 0 && (block < 32 || block > 1024 || (block % 32)))
        return set_error(PLQ_ERR_ARG, "block must be 0 or a multiple of 32 in 32..1024");
    if (sites_per_thread < 0 || sites_per_thread > 64)
        return set_error(PLQ_ERR_ARG, "sites_per_thread must be in 0..64");
    if (index_mode != 0 && index_mode != 1) return set_error(PLQ_ERR_ARG, "index_mode must be 0 or 1");
    if (rhs_tile != 1 && rhs_tile != 2 && rhs_tile != 4) return set_error(PLQ_ERR_ARG, "rhs_tile must be 1, 2 or 4");
    if (nrhs % rhs_tile) return set_error(PLQ_ERR_ARG, "rhs_tile must divide nrhs");
    if (z_chunk < 0 || (z_chunk > 0 && c->lat.L[3] % z_chunk))
        return set_error(PLQ_ERR_ARG, "z_chunk must be 0 or divide Lz");
    if (smem_links < 0 || smem_links > 4) return set_error(PLQ_ERR_ARG, "smem_links must be 0, 1, 2, 3 or 4");
    if (smem_links >= 2 && rhs_tile != 1) return set_error(PLQ_ERR_ARG, "smem_links 2, 3 and 4 need rhs_tile 1");
    if (smem_links == 4 && prec == PLQ_F64) return set_error(PLQ_ERR_ARG, "smem_links 4 needs FP32 or FP16 storage");
    if (smem_links == 1 && rhs_tile == 4) return set_error(PLQ_ERR_ARG, "smem_links 1 needs rhs_tile 1 or 2");
    PLQ_CUDA(cudaSetDevice(c->device));
    if (index_mode == 1) PLQ_TRY(ensure_nbr_tables(c));
    c->tune[prec][nrhs].block = block;
    c->tune[prec][nrhs].index_mode = index_mode;
    c->tune[prec][nrhs].rhs_tile = rhs_tile;
    c->tune[prec][nrhs].zc = z_chunk;
    c->tune[prec][nrhs].smem_links = smem_links;
    c->tune[prec][nrhs].spt = sites_per_thread;
    ++c->tune_version;
    return PLQ_OK;
}
