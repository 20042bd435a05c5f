// Internal declarations of libplq: context, packed-field access, kernel
// parameter blocks and the launchers shared between translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "plq.h"
#include "plq_fastdiv.h"

namespace plq {

// ---------------------------------------------------------------- errors
plq_status set_error(plq_status code, const char *fmt, ...);
plq_status cuda_error(cudaError_t e, const char *what);

#define PLQ_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t e__ = (call);                                        \
        if (e__ != cudaSuccess) return ::plq::cuda_error(e__, #call);    \
    } while (0)

#define PLQ_TRY(call)                                                    \
    do {                                                                 \
        plq_status s__ = (call);                                         \
        if (s__ != PLQ_OK) return s__;                                   \
    } while (0)

// ---------------------------------------------------------------- lattice
struct Lattice {
    int L[4];   // {T, Lx, Ly, Lz}
    int Vh;     // sites per parity
    int t_bc;   // -1 antiperiodic, +1 periodic in time
    // multiply-shift divisors by Lx/2, Ly and Lz (site coordinates from a
    // checkerboard index without hardware integer division)
    FastDiv div_xh, div_y, div_z;
};

// Fill the extents, Vh and the divisors of a lattice.
inline Lattice make_lattice(const int dims[4], int t_bc) {
    Lattice L{};
    for (int mu = 0; mu < 4; ++mu) L.L[mu] = dims[mu];
    L.Vh = (int)((long long)dims[0] * dims[1] * dims[2] * dims[3] / 2);
    L.t_bc = t_bc;
    L.div_xh = make_fastdiv((uint32_t)(dims[1] / 2));
    L.div_y = make_fastdiv((uint32_t)dims[2]);
    L.div_z = make_fastdiv((uint32_t)dims[3]);
    return L;
}

inline bool valid_prec(int p) { return p == PLQ_F64 || p == PLQ_F32 || p == PLQ_F16; }

// Device bounds guards of the debug build (compiled with -DPLQ_DEBUG): an
// index outside [0, n) is recorded as PLQ_ERR_BOUNDS in the status word (when
// the kernel has one) and replaced by 0, so the access stays inside the
// buffer and nothing faults.  In the normal build a guard is the index itself.
#ifdef PLQ_DEBUG
__device__ __forceinline__ long long plq_guard(int *status, long long v, long long n) {
    if (v < 0 || v >= n) {
        if (status) atomicCAS(status, 0, (int)PLQ_ERR_BOUNDS);
        return 0;
    }
    return v;
}
#define PLQ_GUARD(status, v, n) ((decltype((v) + 0))::plq::plq_guard((status), (long long)(v), (long long)(n)))
#else
#define PLQ_GUARD(status, v, n) (v)
#endif

// bytes per site and right-hand side of a packed half field
inline size_t spinor_site_bytes(int prec) { return prec == PLQ_F64 ? 192 : prec == PLQ_F32 ? 96 : 52; }

// bytes per site of one (parity, mu) block of packed links
inline size_t link_site_bytes(int prec, int reals) {
    const size_t per_real = prec == PLQ_F64 ? 8 : prec == PLQ_F32 ? 4 : 2;
    return per_real * (size_t)reals;
}

struct GaugeCopy {
    void *ptr = nullptr;
    int reals = 0;       // 18 or 12; 0 = absent
    size_t block = 0;    // bytes of one (parity, mu) block
};

// Device-resident scalars of a Krylov solve.  Kernels read their
// coefficients from here and the last block of each reduction writes them,
// so an iteration needs no host round trip (and can be graph-captured).
struct SolverState {
    double rho;       // <r, r> (CG) of the previous iteration
    double rho_new;   // <r, r> just computed
    double alpha, beta;
    double pAp;       // ||Mhat p||^2 = <p, Mhat^dag Mhat p>
    double stop_r2;   // freeze once rho_new <= stop_r2
    double2 c_rho, c_rho_new, c_alpha, c_omega, c_beta;  // BiCGstab (complex)
    double2 rv;       // <rhat, v>
    double2 ts;       // <t, s>
    double tt;        // <t, t>
    double r2;        // ||r||^2 (BiCGstab)
    double tiny;      // breakdown threshold scale
    int stop;         // 1: converged / triggered; kernels of the iteration return early
    int iter;         // iterations completed
    int flags;        // bit 0 NaN, bit 1 breakdown
    int maxit;        // stop once iter reaches this
    // Optional per-iteration record of the CG coefficients (EigCG builds its
    // Lanczos matrix from them): hist[3*j + {0, 1, 2}] = alpha_j, beta_j,
    // |r_{j+1}|^2 for iteration j < hist_cap.
    double *hist;
    int hist_cap;
    int pad2;
};

enum { FLAG_NAN = 1, FLAG_BREAKDOWN = 2 };

// Reduction of up to 4 doubles per block, combined by the last block to
// finish (ticket counter), which then applies a finalize step `fin`.
enum Finalize {
    FIN_NONE = 0,       // just leave the sums in sums[]
    FIN_CG_ALPHA,       // pAp = s0; alpha = rho / pAp
    FIN_CG_BETA,        // rho_new = s0; beta = rho_new / rho; rho = rho_new; iter++; stop test
    FIN_BICG_ALPHA,     // rv = (s0, s1); alpha = rho_new / rv
    FIN_BICG_OMEGA,     // ts = (s0, s1); tt = s2; omega = ts / tt
    FIN_BICG_RHO,       // rho_new = (s0, s1); r2 = s2; beta; iter++; stop test
};

struct Reduce {
    double *partials = nullptr;   // kPartialSlots doubles per block
    unsigned *ticket = nullptr;   // zero on entry, left zero on exit
    double *sums = nullptr;       // grid totals: sums[k * nrhs + r]
    SolverState *st = nullptr;    // per right-hand side targets of the finalize step (array of nrhs)
    int fin = FIN_NONE;
};

constexpr int kMaxReduceBlocks = 4096;
constexpr int kPartialSlots = 64;  // >= 4 values x PLQ_MAX_RHS right-hand sides

struct TuneEntry {
    int block = 0;       // 0 = default
    int index_mode = 0;  // 0 inline coordinates, 1 neighbour table
    int rhs_tile = 1;    // right-hand sides per thread
    int zc = 0;          // z-chunk site order (0 = natural)
    int smem_links = 0;  // multi-RHS links staged in shared memory
    int spt = 0;         // sites per thread: 0 = one wave of resident blocks
    float us = 0.f;
};

struct Ctx {
    Lattice lat{};
    TuneEntry tune[3][PLQ_MAX_RHS + 1];
    int *nbr[2] = {nullptr, nullptr};  // neighbour tables per output parity (built on demand)
    int device = 0;
    int *kstatus = nullptr;          // device word: PLQ_ERR_TIMEOUT once a bounded kernel wait gave up
    long long spin_limit = 0;        // clock cycles a kernel wait may take (about 5 s by default)
    GaugeCopy gauge[3];
    GaugeCopy gauge_df;  // PLQ_DF64 links (float-float, 18 reals)
    // reduction scratch
    double *partials = nullptr;         // kPartialSlots * kMaxReduceBlocks
    unsigned *ticket = nullptr;
    double *sums = nullptr;             // kPartialSlots
    double *sums_host = nullptr;        // pinned mirror of sums
    SolverState *state = nullptr;       // PLQ_MAX_RHS solver states
    SolverState *state_host = nullptr;  // pinned mirror
    // solver workspace (allocated on first use, grown as needed)
    void *work = nullptr;
    size_t work_bytes = 0;
    // staging for the host entry points
    void *stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t copy_in = nullptr, copy_out = nullptr, compute = nullptr;  // host-path pipeline
    cudaEvent_t ev[3 * 64] = {};
    int num_sms = 0;
    // Instantiated inner-iteration graph of the last CG / BiCGstab solve, reused
    // by the next reliable-update cycle and the next solve with the same key
    // (method, precisions, sizes, kappa, mu, batch length, workspace address,
    // launch configuration version, inner gauge copy address and format).
    struct SolveGraph {
        cudaGraphExec_t exec = nullptr;
        unsigned long long key[10] = {};
    } solve_graph[2];
    unsigned tune_version = 0;  // bumped whenever a launch configuration changes
    // Instantiated pipeline of plq_hopping_eo_host for the last (host buffers,
    // precision, nrhs, parity, staging area, launch version) it ran with.
    struct HostGraph {
        cudaGraphExec_t exec = nullptr;
        unsigned long long key[8] = {};
    } host_graph;
    // The persistent batched CG solves launched with this context first in
    // their list: descriptor and barrier scratch, internal stream, the
    // instantiated graph of the last launch (replayed while its key matches)
    // and the launch shape chosen by plq_autotune_batched / plq_set_batched_launch.
    struct BatchCache {
        void *scratch = nullptr;
        size_t bytes = 0;
        cudaStream_t stream = nullptr;
        cudaGraphExec_t exec = nullptr;
        unsigned long long key[6] = {};
        int shape = 0;          // index into the kernel's launch shapes
        int blocks_per_sm = 0;  // 0: as many as fit
        int tuned = 0;          // 1 once a shape was chosen by timing or by hand
    } batch;
};

plq_status ensure_work(Ctx *c, size_t bytes);
plq_status ensure_nbr_tables(Ctx *c);
// ||b - M x||^2 and ||b||^2 of packed full FP64 fields (Wilson operator, FP64;
// uses the context's workspace and synchronises the stream)
plq_status wilson_residual64(struct plq_ctx *c, double kappa, const void *x, const void *b, double *r2, double *b2,
                             cudaStream_t s);
plq_status ensure_stage(Ctx *c, size_t bytes);
plq_status ensure_pipeline(Ctx *c);

// ---------------------------------------------------------------- hopping
enum Epilogue {
    EPI_PLAIN = 0,   // out = H in
    EPI_XPAY = 1,    // out = x + a * H in
    EPI_XPAY_NORM = 2,  // ... and sum |out|^2
    EPI_XPAY_DOTW = 3,  // ... and sum <w, out> (complex)
    EPI_XPAY_TS = 4,    // ... and sum <out, x> (complex), |out|^2
};

struct HopArgs {
    const void *in = nullptr;
    void *out = nullptr;
    const void *x = nullptr;   // epilogue source (same parity as out)
    const void *w = nullptr;   // epilogue dot partner
    const void *gauge = nullptr;
    size_t gblock = 0;         // bytes of one (parity, mu) gauge block
    double a = 0.0;
    int out_parity = 0;
    int nrhs = 1;
    int dagger = 0;
    Lattice lat{};
    Reduce red{};
    const SolverState *st = nullptr;  // per-rhs states: elements whose st[rhs].stop is set are skipped
    // Neighbour table of the output parity (the pointer-array addressing of
    // Sec. 2.2): entry (2*mu + back)*Vh + i holds the checkerboard index of the
    // neighbour, with bit 31 set when the hop crosses the time boundary.  NULL:
    // neighbours are computed from the coordinates.
    const int *nbr = nullptr;
    int block = 0;  // threads per block; 0 = default
    int rhs_tile = 1;  // right-hand sides per thread (1, 2 or 4; must divide nrhs)
    // Site order: 0 = checkerboard order (t slowest).  zc > 0 walks the lattice
    // in z-chunks of zc planes (t runs inside a chunk), which shrinks the span
    // of input data reused through the time direction to zc/Lz of a time
    // slab per slice -- what keeps multi-RHS neighbour reuse inside L2.
    int zc = 0;
    // Twisted-mass epilogue terms (0 = plain Wilson): the hopping result is
    // replaced by scale_h * (1 + i nu_h gamma5) H in, and the xpay source x by
    // (1 + i nu_x gamma5) x.
    double nu_x = 0.0, nu_h = 0.0, scale_h = 1.0;
    int site_begin = 0;   // output sites [site_begin, site_end) of the parity;
    int site_end = -1;    // -1: up to Vh
    int smem_links = 0;   // multi-RHS: stage each block's links in shared memory
    // Grid size: 0 = as many blocks as are resident on the GPU at once (each
    // thread walks its share of the sites); k > 0 = enough blocks for k sites
    // (site blocks of the multi-RHS kernel) per thread.
    int spt = 0;
    // Bounded waits of the row-streamed kernel: a wait gives up after
    // spin_limit clock cycles and records PLQ_ERR_TIMEOUT in *kstatus.
    long long spin_limit = 1LL << 40;
    int *kstatus = nullptr;
};

// Launch the hopping kernel for (prec, link reals, epilogue).  block = 0 picks
// the tuned default.
plq_status launch_hop(const HopArgs &a, int prec, int reals, int epi, cudaStream_t s);

int hop_default_block(int prec);

// Fill block / neighbour table of `a` from the context's tuned choice.
void apply_tune(const Ctx *c, int prec, int nrhs, HopArgs &a);

// ---------------------------------------------------------------- layouts
plq_status launch_pack_spinor(const Lattice &lat, void *out, const double *in, int prec, int nrhs, cudaStream_t s);

// ---------------------------------------------------------------- PLQ_DF64 (plq_df.cu)
size_t df_site_bytes();
plq_status df_gauge_upload(struct plq_ctx *c, const double *U, int is_device, int link_reals, cudaStream_t s);
plq_status df_pack_spinor(const Lattice &L, void *out, const double *in, int nrhs, cudaStream_t s);
plq_status df_unpack_spinor(const Lattice &L, double *out, const void *in, int nrhs, cudaStream_t s);
// FP64 half field of N = Vh * n elements <-> PLQ_DF64 half field; right-hand
// side r is scaled by 2^shifts[r] into the float-float field and back
// (shifts may be null: no scaling)
plq_status df_split(long long N, int n, const int *shifts, void *out, const void *in, cudaStream_t s);
plq_status df_join(long long N, int n, const int *shifts, void *out, const void *in, cudaStream_t s);
// out = scale_h (1 + i nu_h gamma5) H in, or with x: out = x + a * that (all PLQ_DF64)
plq_status df_hop(const struct plq_ctx *c, int out_parity, void *out, const void *in, const void *x, double a,
                  double nu_h, double scale_h, int nrhs, cudaStream_t s);
plq_status launch_unpack_spinor(const Lattice &lat, double *out, const void *in, int prec, int nrhs, cudaStream_t s);
plq_status launch_pack_gauge(const Lattice &lat, void *out, const double *in, int prec, int reals, size_t block,
                             unsigned *bad, cudaStream_t s);

// ---------------------------------------------------------------- blas
// Vectors are packed half fields of N = Vh * n elements (n right-hand sides
// interleaved); element e belongs to right-hand side e % n.  Kernels that take
// `st` skip elements whose st[rhs].stop is set and read their coefficients
// from st[rhs]; reductions produce sums[k * n + rhs].
plq_status blas_copy_convert(long long N, void *dst, int pdst, const void *src, int psrc, cudaStream_t s);
plq_status blas_zero(long long N, void *dst, int prec, cudaStream_t s);
plq_status blas_gamma5(long long N, void *dst, const void *src, int prec, cudaStream_t s);
plq_status blas_norm2(long long N, int n, const void *v, int prec, const Reduce &red, cudaStream_t s);
plq_status blas_dot_norm(long long N, int n, const void *a, const void *b, int prec, const Reduce &red,
                         cudaStream_t s);
// x += alpha p; r -= alpha q; rho_new = |r|^2
plq_status blas_cg_update(long long N, int n, void *x, void *r, const void *p, const void *q, int prec,
                          const Reduce &red, const SolverState *st, cudaStream_t s);
// p = r + beta p
plq_status blas_cg_direction(long long N, int n, void *p, const void *r, int prec, const SolverState *st,
                             cudaStream_t s);
// dst(F64) += convert(src)
plq_status blas_accumulate(long long N, void *dst64, const void *src, int psrc, cudaStream_t s);
// v (FP64, n interleaved right-hand sides) *= f[r];  dst64 += f[r] * src
plq_status blas_scale64(long long N, int n, void *v, const double *f, cudaStream_t s);
plq_status blas_accumulate_scaled(long long N, int n, void *dst64, const void *src, int psrc, const double *f,
                                  cudaStream_t s);
// dst = scale * (1 + i nu gamma5) src (same precision, may alias)
plq_status blas_twist(long long N, void *dst, const void *src, int prec, double nu, double scale, cudaStream_t s);
// y = x + a * y (FP64, host scalar)
plq_status blas_xpay64(long long N, const void *x, double a, void *y, cudaStream_t s);
// BiCGstab: p = r + beta (p - omega v); s = r - alpha v; x += alpha p + omega s, r = s - omega t, <rhat, r>, |r|^2
plq_status blas_bicg_p(long long N, int n, void *p, const void *r, const void *v, int prec, const SolverState *st,
                       cudaStream_t s);
plq_status blas_bicg_s(long long N, int n, void *sv, const void *r, const void *v, int prec, const SolverState *st,
                       cudaStream_t s);
plq_status blas_bicg_update(long long N, int n, void *x, void *r, const void *p, const void *sv, const void *t,
                            const void *rhat, int prec, const Reduce &red, const SolverState *st, cudaStream_t s);

}  // namespace plq

struct plq_ctx : public plq::Ctx {};
