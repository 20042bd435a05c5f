/*
 * plq.h -- C ABI of the GB300 Wilson-Dirac library (libplq.so).
 *
 * The library implements the hot path of "PLQCD library for Lattice QCD on
 * multi-core machines" (Abdel-Rehim et al., LATTICE 2013): the hopping part of
 * the Wilson-Dirac operator, Eq. (1),
 *
 *   psi(x) = sum_mu [ U_mu(x) (1 - gamma_mu) phi(x + mu)
 *                     + U_mu(x - mu)^dagger (1 + gamma_mu) phi(x - mu) ],
 *
 * evaluated through the two-component half spinors of Eq. (2) and the remark
 * after it (only the upper two spin components of theta+- are computed), and
 * the linear solvers that call it.  Every operation runs in CUDA kernels on
 * one GPU; no call falls back to the CPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * dims[4] = {T, Lx, Ly, Lz}: mu = 0 is time, mu = 1, 2, 3 are x, y, z.  Every
 *   extent must be even and >= 2.  V = T*Lx*Ly*Lz sites, Vh = V/2 per parity.
 * Parity of a site = (t + x + y + z) mod 2; parity 0 is "even".
 * Lexicographic site index: s = ((t*Lz + z)*Ly + y)*Lx + x.  The checkerboard
 *   index of a site inside its parity is s/2 (integer division; x is fastest
 *   and Lx is even, so this is a bijection per parity).
 * Boundary conditions: periodic in x, y, z; a hop that crosses between
 *   t = T-1 and t = 0 is multiplied by t_bc (-1 = antiperiodic, +1 periodic).
 *   The sign is applied inside the kernels, never folded into stored links.
 * gamma basis (chiral, the DD-HMC documentation the paper cites after
 *   Eq. (2)): gamma_mu = [[0, A_mu], [A_mu^dagger, 0]], A_0 = -1,
 *   A_k = -i sigma_k, gamma_5 = diag(1, 1, -1, -1).
 * Wilson operator M = 1 - kappa*H (H exactly as Eq. (1); free-field critical
 *   kappa = 1/8).  Even-odd Schur complement Mhat = 1 - kappa^2 H_eo H_oe.
 *
 * Canonical (user) layouts, interleaved (re, im) FP64:
 *   spinor  phi[s][spin 0..3][colour 0..2]            24 doubles per site
 *   gauge   U[s][mu 0..3][row 0..2][col 0..2]         72 doubles per site
 *
 * Internal ("packed") layouts, device memory, structure of arrays:
 *   A half field holds the Vh sites of one parity for nrhs right-hand sides.
 *   Its components are grouped in 16-byte planes; plane k of site i and
 *   right-hand side r is element ((k*Vh + i)*nrhs + r).  Complex component
 *   c = spin*3 + colour.
 *     PLQ_F64: 12 planes of (re, im) double           192 B per site and rhs
 *     PLQ_F32:  6 planes of (re0, im0, re1, im1) float  96 B per site and rhs
 *     PLQ_F16:  3 planes of 8 IEEE binary16 values (4 complex), followed by a
 *               float plane of per-site norms n = max |real or imaginary
 *               component|; stored halves are component / n    52 B per site
 *     PLQ_DF64: the PLQ_F32 half field of the high parts followed by the
 *               PLQ_F32 half field of the low parts of every real,
 *               value = hi + lo (float-float)               192 B per site
 *   A full field is the even half followed by the odd half.
 *   plq_field_bytes() gives the byte size of one half field.
 *
 * Memory ownership: fields passed to the entry points are caller-owned device
 * buffers (for example PyTorch tensors) unless a parameter says otherwise.
 * Every device pointer must be 16-byte aligned.  The library owns its packed
 * copies of the gauge field and its solver workspace, released by
 * plq_finalize.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Operator calls are asynchronous on that stream.  Solver calls
 * synchronise it before they return because they fill plq_solve_info.
 *
 * Threads: entry points may be called from any host thread.  Calls that use
 * the same context (its gauge copies, workspace, tuning table and solver
 * graphs) must not overlap; different contexts may be used concurrently.
 *
 * Errors: every function returns PLQ_OK (0) or an error code; the matching
 * message is available from plq_last_error() in the calling thread.  No entry
 * point traps on the device, asserts, or throws across the ABI.  Invalid
 * arguments (NULL or misaligned pointers, bad precision, bad parity, nrhs out
 * of range) return PLQ_ERR_ARG and launch nothing.
 */
#ifndef PLQ_H
#define PLQ_H

#include <stddef.h>

#if defined(__GNUC__)
#define PLQ_API __attribute__((visibility("default")))
#else
#define PLQ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int plq_status;

enum {
    PLQ_OK = 0,
    PLQ_ERR_ARG = 1,           /* invalid argument; nothing was launched          */
    PLQ_ERR_CUDA = 2,          /* a CUDA runtime call failed                       */
    PLQ_ERR_NOMEM = 3,         /* device or pinned allocation failed               */
    PLQ_ERR_NOT_CONVERGED = 4, /* solver hit maxit before reaching tol             */
    PLQ_ERR_BREAKDOWN = 5,     /* Krylov breakdown (rho or omega vanished)         */
    PLQ_ERR_NAN = 6,           /* a NaN or Inf appeared in a solver scalar         */
    PLQ_ERR_TIMEOUT = 7,       /* a device-side wait ran out of its spin limit     */
    PLQ_ERR_STATE = 8,         /* call out of order (e.g. no gauge field uploaded) */
    PLQ_ERR_BOUNDS = 9         /* debug build (PLQ_DEBUG): a device bounds guard found an
                                  index out of range (recorded, access redirected)  */
};

/* Storage precisions of packed fields.  PLQ_F32 and PLQ_F16 compute in FP32;
 * PLQ_F64 computes in FP64.  PLQ_DF64 stores every real as an unevaluated sum
 * of two floats (hi = rn(d), lo = rn(d - hi): about 48 significant bits, the
 * exponent range of FP32) and computes in float-float arithmetic built from
 * the error-free TwoSum and FMA-based TwoProduct; it gives FP64-level
 * accuracy (relative error ~1e-14) at FP32 instruction rates.  PLQ_DF64 is
 * accepted by plq_field_bytes, plq_gauge_upload (18 reals), plq_pack_spinor,
 * plq_unpack_spinor and plq_hopping_eo, and as residual_prec of the solvers;
 * every other entry point returns PLQ_ERR_ARG for it. */
enum { PLQ_F64 = 0, PLQ_F32 = 1, PLQ_F16 = 2, PLQ_DF64 = 3 };

/* Maximum number of right-hand sides of the multi-RHS operator (one link load
 * serves all of them; 12 = the spin x colour columns of a point source). */
#define PLQ_MAX_RHS 12

typedef struct plq_ctx plq_ctx;

/* Solver parameters.  Fields left zero take the documented default. */
typedef struct {
    double tol;        /* target true relative residual ||b - M x|| / ||b||, default 1e-10 */
    int maxit;         /* cap on inner Krylov iterations (all restarts), default 20000     */
    int inner_prec;    /* PLQ_F64 (plain FP64 solve), PLQ_F32 or PLQ_F16 inner precision   */
    double delta;      /* reliable-update trigger: the FP64 residual is recomputed when the
                          inner residual fell by this factor since the last update;
                          default 1e-4 for FP32 (1e-3 for BiCGstab), 1e-2 for FP16 inner
                          solves (ignored when inner_prec == PLQ_F64)                       */
    int use_x0;        /* 1: x holds an initial guess on entry (resume); 0: start from 0   */
    int check_every;   /* inner iterations per host convergence poll, default 16           */
    double mu;         /* twisted mass: solve M_tm = 1 - kappa H + 2 i kappa mu gamma5
                          (0: the Wilson operator M)                                        */
    int residual_prec; /* arithmetic of the FP64-accuracy steps of a mixed-precision solve
                          (bhat, the reliable-update residuals s = bhat - Mhat x and the
                          odd solution x_o): PLQ_F64 (default) or PLQ_DF64 (needs the
                          PLQ_DF64 gauge copy).  The residual of the returned x is always
                          computed in FP64.  Used by plq_cg_solve(_multi) and
                          plq_bicgstab_solve(_multi); other solvers ignore it.               */
    double wait_limit_s; /* plq_cg_solve_batched: longest a block of the persistent kernel
                            may wait at a grid barrier before the solve gives up with
                            PLQ_ERR_TIMEOUT (0: about 5 s)                                   */
} plq_solver_params;

/* Per-solve report. */
typedef struct {
    int status;               /* same value the call returns                             */
    int iterations;           /* inner Krylov iterations performed                       */
    int n_reliable;           /* FP64 residual recomputations (reliable updates)         */
    double true_rel_residual; /* ||b - M x|| / ||b|| of the returned x, computed in FP64 */
    double seconds;           /* wall time of the solve on the stream                    */
    double hop_applications;  /* half-lattice hopping applications launched              */
} plq_solve_info;

/* Message of the last error in this thread ("" if none).  The pointer stays
 * valid until the next failing call in the same thread.
 * Defined by: paper silent (error reporting of this library). */
PLQ_API const char *plq_last_error(void);

/* Library version, major*10000 + minor*100 + patch.
 * Defined by: paper silent. */
PLQ_API int plq_version(void);

/* Create a context for a lattice on CUDA device `device` (made current for
 * the calling thread).  dims as described above; t_bc is -1 (antiperiodic
 * time, the default physics) or +1.  Returns PLQ_ERR_ARG for odd or < 2
 * extents, volumes above 2^30 sites, or |t_bc| != 1.  *ctx receives the
 * handle; release it with plq_finalize.
 * Defined by: Sec. 2, Eq. (1) (a four-dimensional lattice, directions
 * mu = 0..3, nearest-neighbour hops).  Paper silent on which mu is time, on
 * the boundary conditions and on the even-odd split; the readings taken are
 * those stated at the top of this header. */
PLQ_API plq_status plq_init(plq_ctx **ctx, const int dims[4], int t_bc, int device);

/* Free every device and host resource of the context.  NULL is accepted.
 * Defined by: paper silent (resource management of this library). */
PLQ_API plq_status plq_finalize(plq_ctx *ctx);

/* Defined by: paper silent (failure detection of this library's kernels).
 *
 * Longest time a wait inside a kernel of this context may take (the
 * row-streamed hopping kernel waits for its shared-memory copies) before it
 * gives up: the kernel then records PLQ_ERR_TIMEOUT in the context's device
 * status word, leaves its output incomplete and returns (default about 5 s).
 * Host only; takes effect for the launches that follow. */
PLQ_API plq_status plq_set_wait_limit(plq_ctx *ctx, double seconds);

/* Defined by: paper silent (failure detection of this library's kernels).
 *
 * Reads the context's device status word (synchronising the device): PLQ_OK,
 * or the error a kernel recorded (PLQ_ERR_TIMEOUT: a bounded wait gave up;
 * PLQ_ERR_BOUNDS: in a library built with PLQ_DEBUG, a device bounds guard
 * found an out-of-range index), which is then also the return value.
 * clear != 0 resets the word. */
PLQ_API plq_status plq_device_status(plq_ctx *ctx, int clear);

/* Number of sites of one parity, Vh.
 * Defined by: paper silent (the even-odd split is a reading: sites of one
 * parity only hop to sites of the other, Eq. (1)). */
PLQ_API long plq_half_volume(const plq_ctx *ctx);

/* Bytes of one packed half field of precision `prec` holding `nrhs`
 * right-hand sides (0 on bad arguments).
 * Defined by: paper silent on storage (Sec. 4 only mentions data-ordering
 * strategies); the layouts are those described at the top of this header. */
PLQ_API size_t plq_field_bytes(const plq_ctx *ctx, int prec, int nrhs);

/* Pack the gauge field into the library-owned copy of precision `prec`
 * (Eq. (1): U_mu(x) is the link from x to x + mu).
 *   U          canonical FP64 gauge field (72 doubles per site), host memory
 *              if is_device == 0 (copied synchronously), device memory if 1.
 *   link_reals 18 (full 3x3) or 12 (rows 0 and 1; row 2 is rebuilt in the
 *              kernels as conj(row0 x row1), valid for SU(3) links only).
 *   prec       PLQ_F64, PLQ_F32 or PLQ_F16 storage of the copy.
 * Each precision has its own copy; uploading again replaces it.  Solvers need
 * the PLQ_F64 copy and the copy of their inner precision.  For link_reals ==
 * 12 every link is checked to be special unitary to 1e-12 (max abs deviation
 * of U U^dagger from 1 and of row 2 from conj(row0 x row1)); PLQ_ERR_ARG if
 * not.  Synchronises `stream`. */
PLQ_API plq_status plq_gauge_upload(plq_ctx *ctx, const double *U, int is_device, int link_reals, int prec, void *stream);

/* Canonical FP64 spinor fields -> packed full field of precision `prec`.
 *   in   device, `nrhs` canonical fields back to back (nrhs * V * 24 doubles)
 *   out  device, 2 * plq_field_bytes(prec, nrhs) bytes: the even half field
 *        then the odd half field, right-hand sides interleaved as described
 *        above.
 * Conversion to FP32 / FP16 rounds to nearest; FP16 stores component/norm.
 * Defined by: the spinor phi(x) of Eq. (1) (4 spin x 3 colour complex
 * components per site); paper silent on layouts and reduced precisions. */
PLQ_API plq_status plq_pack_spinor(plq_ctx *ctx, void *out, const double *in, int prec, int nrhs, void *stream);

/* Packed full field of precision `prec` -> `nrhs` canonical FP64 fields.
 * Defined by: the inverse of plq_pack_spinor (paper silent on layouts). */
PLQ_API plq_status plq_unpack_spinor(plq_ctx *ctx, double *out, const void *in, int prec, int nrhs, void *stream);

/* Half-lattice hopping operator (Eq. (1) restricted to one output parity):
 *   out = H_{p,1-p} in,  p = out_parity (0: out even, in odd; 1: out odd, in even)
 * `in` and `out` are packed half fields of precision `prec` with `nrhs`
 * right-hand sides (1..PLQ_MAX_RHS); with nrhs > 1 every link is loaded once
 * for all right-hand sides.  Needs the gauge copy of precision `prec`.
 * `in` and `out` must not overlap. */
PLQ_API plq_status plq_hopping_eo(plq_ctx *ctx, int out_parity, void *out, const void *in, int prec, int nrhs, void *stream);

/* Same operation on HOST buffers (packed layout, pinned or pageable): the
 * input half field is copied to the device, the operator applied and the
 * result copied back, pipelined over time slabs (plq_host_slabs) so that
 * copies in, compute and copies out overlap -- the communication/computation
 * overlap of Sec. 2.2 applied to the host link; the stream is synchronised
 * before return.  Uses a library-owned device staging area. */
PLQ_API plq_status plq_hopping_eo_host(plq_ctx *ctx, int out_parity, void *out_host, const void *in_host, int prec, int nrhs,
                               void *stream);

/* Time slabs of the plq_hopping_eo_host pipeline (Sec. 2.2: the lattice split
 * so that transfers of one part overlap computation on another) for time
 * extent T (even, >= 2):
 * writes the slab boundaries bounds[0] = 0 < bounds[1] < ... < bounds[K] = T
 * (caller-owned, room for 65 ints) and returns K <= 64, or 0 on bad arguments.
 * Slabs grow 1, 1, 2, 4, ... time slices (each below T/8) from both ends with
 * slabs of T/8 slices between them.  Host only; no device work. */
PLQ_API int plq_host_slabs(int T, int *bounds);

/* Wilson operator on the full lattice: out = M in = in - kappa * H in.
 * `in` and `out` are packed full fields (even half then odd half) of
 * precision `prec`, nrhs = 1; they must not overlap.
 * Defined by: H is Eq. (1) of Sec. 2 (the hopping part of the Wilson-Dirac
 * operator); the normalisation M = 1 - kappa H (hopping parameter kappa, no
 * factor 1/2 in the projectors) is a reading, the paper being silent on it. */
PLQ_API plq_status plq_wilson_apply(plq_ctx *ctx, void *out, const void *in, double kappa, int prec, void *stream);

/* Twisted-mass Wilson operator (the fermions of the paper's Sec. 3 EigCG
 * solves; the operator itself is the standard twisted-mass formulation the
 * paper cites): out = M_tm in = in - kappa H in + 2 i kappa mu gamma5 in, on
 * packed full fields of precision `prec`.  mu = 0 gives plq_wilson_apply.
 * The solvers handle M_tm when plq_solver_params.mu != 0, with the Schur
 * complement Mhat_tm = A - kappa^2 H_eo A^{-1} H_oe, A = 1 + 2 i kappa mu
 * gamma5, and Mhat_tm(mu)^dagger = gamma5 Mhat_tm(-mu) gamma5. */
PLQ_API plq_status plq_twisted_apply(plq_ctx *ctx, void *out, const void *in, double kappa, double mu, int prec,
                                     void *stream);

/* Even-odd Schur operator on even half fields: out = Mhat in =
 * in - kappa^2 H_eo H_oe in (dagger != 0: Mhat^dagger = gamma5 Mhat gamma5).
 * `tmp` is a caller-owned odd half field of the same precision.
 * Defined by: two half-lattice applications of Eq. (1) (Sec. 2); the even-odd
 * preconditioning itself is a reading (paper silent). */
PLQ_API plq_status plq_schur_apply(plq_ctx *ctx, void *out, const void *in, void *tmp, double kappa, int dagger, int prec,
                           void *stream);

/* Defined by: Sec. 4 states that the library holds "a few associated
 * solvers" for the Wilson-Dirac operator of Eq. (1) without naming them
 * (paper silent on the algorithms); CG on the even-odd normal equations and
 * BiCGstab are the readings taken, mixed precision with reliable updates
 * follows Clark et al. (2010).
 *
 * Solve M x = b by conjugate gradients on the even-odd preconditioned normal
 * equations Mhat^dagger Mhat x_e = Mhat^dagger bhat, bhat = b_e + kappa H_eo b_o,
 * then x_o = b_o + kappa H_oe x_e.  x and b are packed full FP64 fields.
 * inner_prec PLQ_F32/PLQ_F16 runs the Krylov iteration at that precision with
 * FP64 reliable updates (residual recomputation and solution accumulation in
 * FP64).  Converged when ||b - M x|| / ||b|| <= tol, verified in FP64 before
 * return.  Returns PLQ_ERR_NOT_CONVERGED at maxit (x holds the last iterate). */
PLQ_API plq_status plq_cg_solve(plq_ctx *ctx, void *x, const void *b, double kappa, const plq_solver_params *params,
                        plq_solve_info *info, void *stream);

/* Same system solved by BiCGstab on Mhat x_e = bhat (no normal equations).
 * Returns PLQ_ERR_BREAKDOWN when rho or omega vanish.
 * Defined by: paper silent on the algorithm (see plq_cg_solve); BiCGstab of
 * van der Vorst (1992). */
PLQ_API plq_status plq_bicgstab_solve(plq_ctx *ctx, void *x, const void *b, double kappa, const plq_solver_params *params,
                              plq_solve_info *info, void *stream);

/* Defined by: the solvers above (paper silent on the algorithms) with the
 * operator applied to several vectors per link load, Sec. 2.3's one SU(3)
 * matrix times two vectors widened to up to 12.
 *
 * Several right-hand sides at once: x and b are packed full FP64 fields
 * holding `nrhs` (1..PLQ_MAX_RHS) interleaved right-hand sides (as produced
 * by plq_pack_spinor with that nrhs); `infos` points to nrhs reports.  Every
 * operator application of the solve loads each link once for all of them
 * (the multi-RHS hopping kernel); each right-hand side keeps its own Krylov
 * scalars, stops on its own true residual and is frozen (its elements
 * skipped) once converged.  Reliable updates are taken for the whole batch
 * when every active right-hand side has reached its trigger.  The return
 * value is PLQ_OK if every right-hand side converged, else the status of the
 * first that did not (its message names it). */
PLQ_API plq_status plq_cg_solve_multi(plq_ctx *ctx, void *x, const void *b, double kappa, int nrhs,
                                      const plq_solver_params *params, plq_solve_info *infos, void *stream);
PLQ_API plq_status plq_bicgstab_solve_multi(plq_ctx *ctx, void *x, const void *b, double kappa, int nrhs,
                                            const plq_solver_params *params, plq_solve_info *infos, void *stream);

/* Incremental EigCG: the deflation solver of the paper's Sec. 3 (Stathopoulos
 * and Orginos' eigCG; the paper's runs use nev = 10, m = 60, 30 right-hand
 * sides for 300 vectors, FP64, relative tolerance 1e-8).  A handle holds a
 * growing orthonormal basis U of approximate low eigenvectors of A =
 * Mhat^dag Mhat (even-odd normal equations) and H = U^H A U.
 *   plq_eigcg_create: nev Ritz vectors per accumulating solve, search space m
 *     (2*nev + 2 <= m <= 64, 2*nev <= 24), room for max_vectors basis vectors
 *     (device memory: max_vectors + 4 FP64 half fields and max_vectors +
 *     2*(m+1) + 1 FP32 ones).
 *   plq_eigcg_solve: solves M x = b (packed full FP64 fields).  The Krylov
 *     solve on the normal equations starts from the Galerkin guess
 *     x0 = U H^{-1} U^H rhs; with accumulate != 0 (and room left in U) it is
 *     eigCG and its nev lowest Ritz vectors are added to U afterwards,
 *     otherwise plain CG.  Stops when the normal-equation residual falls to
 *     params->tol (default 1e-8) relative to its right-hand side; info reports
 *     the true residual ||b - M x|| / ||b|| and, in n_reliable, the number of
 *     basis vectors now held.  The CG iterations, H, the Galerkin guess and
 *     all residuals are FP64; the search space (Lanczos vectors, restarts,
 *     Ritz vectors) and the Gram-Schmidt of new basis vectors use FP32 copies
 *     (they shape the subspace only; H is computed for the vectors stored).
 *     Wilson operator (mu = 0).
 *   plq_eigcg_vectors: basis vectors held. */
typedef struct plq_eigcg plq_eigcg;
PLQ_API plq_status plq_eigcg_create(plq_ctx *ctx, int nev, int m, int max_vectors, plq_eigcg **out);
PLQ_API plq_status plq_eigcg_destroy(plq_eigcg *eig);
PLQ_API int plq_eigcg_vectors(const plq_eigcg *eig);
/* The projected matrix H = U^H A U of the deflation basis (Sec. 3: the
 * Rayleigh-Ritz matrix whose eigenvalues approximate the lowest eigenvalues
 * of A): with k = plq_eigcg_vectors(eig) basis vectors, writes H[i][j] as
 * (re, im) doubles at H[2*(i*ld + j)] for i, j < k (host memory, caller-owned,
 * ld >= k) and returns k; with H == NULL only returns k.  -1 on a NULL handle
 * or ld < k.  Host copy only; no device work. */
PLQ_API int plq_eigcg_projected_matrix(const plq_eigcg *eig, double *H, int ld);
PLQ_API plq_status plq_eigcg_solve(plq_eigcg *eig, void *x, const void *b, double kappa,
                                   const plq_solver_params *params, int accumulate, plq_solve_info *info,
                                   void *stream);

/* Launch report of plq_cg_solve_batched. */
typedef struct {
    int grid;            /* blocks of the persistent kernel (all co-resident)  */
    int block;           /* threads per block                                  */
    int graph_captured;  /* 1 if the launch ran as a captured CUDA graph       */
    int launches;        /* kernel launches of the solve (1 on success)        */
    double seconds;      /* time of the persistent kernel                      */
    int blocks_per_sm;   /* resident blocks per SM launched                     */
    int graph_reused;    /* 1 if the instantiated graph of an earlier call with
                            the same launch was replayed                        */
} plq_batch_info;

/* Defined by: paper silent (the CG of plq_cg_solve, whose algorithm the
 * paper does not name, applied to many independent systems at once).
 *
 * The descriptor scratch, the internal stream and the instantiated CUDA graph
 * of the launch are kept in ctxs[0] (freed by its plq_finalize): a later call
 * with ctxs[0] first and the same launch shape, number of systems and
 * parameters replays that graph (plq_batch_info.graph_reused) after
 * rewriting the descriptors, so it may solve other systems, sources or
 * kappas.  The launch shape (threads per block, resident blocks per SM) is
 * the one set on ctxs[0] by plq_set_batched_launch or plq_autotune_batched,
 * else 128 threads and all blocks that fit.
 *
 * Batched CG: n (1..64) independent systems M_k x_k = b_k -- different
 * lattices (one context each, same device), kappas and iteration counts --
 * solved by ONE persistent cooperative kernel launch, captured in a CUDA
 * graph.  Each system runs the algorithm of plq_cg_solve (even-odd normal
 * equations, inner precision params->inner_prec with FP64 reliable updates)
 * as its own state machine; all systems advance in lockstep phases separated
 * by grid-wide barriers, and the sites of every still-active system form one
 * shared work range, so converged systems retire and their blocks move to the
 * others.  Barriers wait with a time limit (params->wait_limit_s, default
 * about 5 s) and report PLQ_ERR_TIMEOUT instead of hanging: every block
 * leaves the kernel and the context stays usable.  Each context needs an 18-real FP64
 * gauge copy and a copy of the inner precision (the same link format for all
 * systems; FP16 inner solves use 12-real links).  x[k], b[k]: packed full
 * FP64 fields of context k.  infos (n entries) and binfo may be NULL.  After
 * the kernel every system's true residual is recomputed with the FP64
 * operator; the call returns PLQ_OK only if all are <= tol. */
PLQ_API plq_status plq_cg_solve_batched(plq_ctx **ctxs, int n, void **x, const void **b, const double *kappa,
                                        const plq_solver_params *params, plq_solve_info *infos,
                                        plq_batch_info *binfo, void *stream);

/* Defined by: paper silent (launch parameters of plq_cg_solve_batched).
 *
 * Launch shape of the persistent batched kernel for batches whose first
 * context is `ctx`: block = threads per block, 64, 128, 192 or 256 (0: 128),
 * compiled with the register budget of 512 resident threads per SM (192:
 * 384 threads, 168 registers), and blocks_per_sm = resident blocks per SM to
 * launch (0: as many as fit; values above that are clamped). */
PLQ_API plq_status plq_set_batched_launch(plq_ctx *ctx, int block, int blocks_per_sm);

/* Defined by: paper silent (tuner of plq_cg_solve_batched's launch).
 *
 * Times plq_cg_solve_batched on the given systems (same arguments; x is
 * overwritten by the solves) for every block size of plq_set_batched_launch
 * with all resident blocks per SM and with one fewer, each solved twice and
 * timed on the second call (which replays the captured graph), and keeps the
 * fastest kernel time in ctxs[0].  cache_path (NULL: the PLQ_TUNE_CACHE
 * environment variable, if set) names the text file of plq_autotune: a line
 * keyed by GPU name, inner precision, link format, number of systems and
 * their lattices skips the timing; a miss appends the result.  best (may be
 * NULL) receives the launch report of the chosen shape (from the cache:
 * block, blocks_per_sm and seconds only).  Synchronises the device. */
PLQ_API plq_status plq_autotune_batched(plq_ctx **ctxs, int n, void **x, const void **b, const double *kappa,
                                        const plq_solver_params *params, const char *cache_path,
                                        plq_batch_info *best);

/* Allocation-free Schur operator.  No counterpart in the paper: this is a
 * service to callers that cannot allocate device memory at the moment they
 * apply the operator -- applications that hand all device memory to their
 * own pool or allocator and forbid anyone else from calling cudaMalloc,
 * real-time or latency-critical loops that must not take the allocator's
 * locks or wait for it, and callers that run under a fixed device-memory
 * budget agreed at start-up.  It computes the same result as plq_schur_apply
 * (out = Mhat in, or Mhat^dagger in when dagger != 0), in the same launch
 * configuration (plq_autotune / plq_set_launch), but keeps the odd-parity
 * intermediate H_oe in in a fixed device array of PLQ_NOALLOC_SCRATCH_BYTES
 * bytes compiled into the library, so the call itself allocates nothing: no
 * cudaMalloc, cudaFree or allocating library routine.  (The context, its
 * gauge copy and the in/out fields are set up beforehand, as for every other
 * call.)
 *   in, out   caller-owned even half fields of precision `prec`, distinct.
 *   Limits    PLQ_ERR_ARG when one odd half field of `prec` is larger than
 *             PLQ_NOALLOC_SCRATCH_BYTES (8 MiB: Vh up to 43,690 sites in FP64,
 *             87,381 in FP32, 161,319 in FP16).
 * The array exists once per GPU that loads the library and stays allocated
 * until the process exits.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current) and caches
 * it; make that first call before any stream capture.  A cudaDeviceReset
 * destroys the module instance the cached address points into, together with
 * every context created before it; the next call after a reset sees that the
 * cached address no longer belongs to the device and looks it up again.
 * Every call on a device shares the one array: calls whose kernels overlap
 * on the GPU (different streams, or different contexts on the same device)
 * race on it and must be serialised by the caller.  The array keeps the last
 * call's contents; each call overwrites all of the part it reads before
 * reading it. */
#define PLQ_NOALLOC_SCRATCH_BYTES (8u << 20)
PLQ_API plq_status plq_schur_apply_noalloc(plq_ctx *ctx, void *out, const void *in, double kappa, int dagger,
                                           int prec, void *stream);

/* Result of plq_autotune. */
typedef struct {
    int block;            /* threads per block chosen                                      */
    int index_mode;       /* 0: neighbours from coordinates; 1: precomputed neighbour table */
    int rhs_tile;         /* right-hand sides per thread (each loaded link serves all)     */
    int z_chunk;          /* site order: 0 = time slowest; z > 0 = z-chunks of z planes    */
    int smem_links;       /* nrhs > 1: 0 none; 1 links of a block of sites staged in shared
                             memory; 2 / 3 the same plus the neighbour spinors of the next
                             1 / 2 directions copied ahead into per-thread shared slots;
                             any nrhs (FP32/FP16): 4 row-streamed kernel, whole rows of
                             neighbour spinors copied into a ring of shared-memory slots
                             by bulk (TMA) copies, sites_per_thread then being the number
                             of slots (0: as many as fit); set by plq_set_launch only
                             (the tuner does not time it: slower on GB300)             */
    double us_per_launch; /* measured time of one half-lattice application                 */
    int from_cache;       /* 1 if the choice came from the cache file                      */
    int candidates;       /* configurations timed                                          */
    int sites_per_thread; /* grid size: 0 one wave of resident blocks, each thread walking
                             its share of the sites; k > 0 enough blocks for k sites (site
                             blocks, with smem_links) per thread                           */
} plq_tune_result;

/* Autotuner of the hopping kernel's launch for precision `prec` and `nrhs`
 * right-hand sides: times every threads-per-block value in {64, 96, 128, 192,
 * 256, 512, 1024} that the kernel can launch (registers x threads within the
 * SM's register file and the kernel's launch bound) with neighbour indices computed inline from the coordinates and read
 * from a precomputed per-site table (the pointer-array addressing the paper
 * describes for out-of-order site access, Sec. 2.2), and for nrhs > 1 (FP32
 * and FP16 storage) with 2 or 4 right-hand sides per thread (register tiles
 * that reuse each loaded link, Sec. 2.3's one-matrix-two-vectors idea
 * widened), with the links of a block of sites staged once in shared memory
 * (nrhs > 1; with or without the neighbour spinors of the next directions
 * copied ahead asynchronously, the GPU counterpart of the paper's software
 * prefetch, Sec. 2.2), and with the sites walked in z-chunks of 8 or 4 planes (time
 * inside a chunk, which keeps the data reused through the time direction
 * within L2 for large multi-RHS fields), then the fastest of these with 1, 2,
 * 4 or 8 sites per thread against its one-wave grid, and keeps the fastest in
 * the context for every later operator and solver call of that precision.
 * cache_path (NULL: the PLQ_TUNE_CACHE environment variable, if set) names a
 * text file keyed by GPU name, lattice, precision, link format and nrhs: a
 * hit skips the timing, a miss appends the new result.  Needs the gauge copy
 * of `prec`; allocates two temporary half fields; synchronises the device.
 * `res` may be NULL. */
PLQ_API plq_status plq_autotune(plq_ctx *ctx, int prec, int nrhs, const char *cache_path, plq_tune_result *res);

/* Defined by: the launch parameters that plq_autotune sweeps (index mode:
 * the pointer arrays of Sec. 2.2; right-hand-side tiles: Sec. 2.3).
 *
 * Set the hopping launch of (prec, nrhs) by hand: block = threads per block
 * (0 = library default, else a multiple of 32 up to 1024; a block the kernel
 * cannot launch makes the operator calls return PLQ_ERR_ARG), index_mode 0 or 1,
 * rhs_tile 1, 2 or 4 (dividing nrhs), z_chunk 0 or a divisor of Lz and
 * smem_links 0..4 (1..3: nrhs > 1, FP32/FP16; 4: FP32/FP16, needs nrhs x Lx/2
 * <= 512 and, for FP16 storage, site-norm runs of 16-byte multiples, else the
 * operator calls return PLQ_ERR_ARG; with 1, rhs_tile 1 or 2; with 2, 3 or 4,
 * rhs_tile 1) and sites_per_thread 0..64, as above. */
PLQ_API plq_status plq_set_launch(plq_ctx *ctx, int prec, int nrhs, int block, int index_mode, int rhs_tile,
                                  int z_chunk, int smem_links, int sites_per_thread);

/* Two-pass schedule of the hopping operator through the auxiliary fields of
 * Eq. (2): pass 1 computes, at every input site y, theta+_mu(y) = (1 -
 * gamma_mu) phi(y) and theta-_mu(y) = U_mu(y)^dagger (1 + gamma_mu) phi(y)
 * (upper two spin components only, the remark after Eq. (2)); pass 2
 * gathers psi(x) = sum_mu [U_mu(x) theta+_mu(x + mu) + theta-_mu(x - mu)].
 * This is the order of operations the paper's distributed code uses to
 * overlap the boundary exchange of theta with bulk work (Sec. 2.2); on one
 * GPU it is a comparison point for the fused plq_hopping_eo (same result,
 * twice the memory traffic).  `theta` is a caller-owned device buffer of
 * plq_theta_bytes(ctx, prec) bytes.  FP64 and FP32 only; nrhs = 1. */
PLQ_API size_t plq_theta_bytes(const plq_ctx *ctx, int prec);
PLQ_API plq_status plq_hopping_eo_theta(plq_ctx *ctx, int out_parity, void *out, const void *in, void *theta,
                                        int prec, void *stream);

/* Link x spinor streaming micro-benchmark (the paper's prefetch / access
 * pattern experiment, Sec. 2.2): psi(i) = U(i) phi(i) -- one SU(3) matrix on
 * the four colour vectors of a spinor -- for nsites records stored site by
 * site (18 reals of U, 24 of phi and psi; prec PLQ_F64 or PLQ_F32).
 *   mode 0: sequential, record i;
 *   mode 1: random through the device index array `index` (record index[i];
 *           entries outside [0, nsites) are skipped);
 *   mode 2: random through precomputed device pointer arrays `pointers`
 *           (3*nsites entries: psi'(i), then U'(i), then phi'(i)), which the
 *           caller must fill with addresses of valid records.
 * Asynchronous on `stream`; the caller times it. */
PLQ_API plq_status plq_link_spinor_stream(int mode, long long nsites, const void *U, const void *phi, void *psi,
                                          const int *index, const void *const *pointers, int prec, void *stream);

/* Roofline calibration (a measurement helper; paper silent, it has no
 * counterpart):
 * the sustained FMA throughput of the CUDA cores of `device` in FP64
 * (prec = PLQ_F64) or FP32 (PLQ_F32), in flop/s (an FMA counts 2), measured
 * with independent FMA chains in every thread of a full-GPU grid.  Allocates
 * a small scratch buffer and synchronises the device. */
PLQ_API plq_status plq_measure_fma_rate(int device, int prec, double *flops_per_second);

#ifdef __cplusplus
}
#endif

#endif /* PLQ_H */
