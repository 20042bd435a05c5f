/*
 * Plain FP64 C oracle of the Wilson-Dirac hopping operator.
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
 * baseline leg load this library.  It shares no code with the CUDA path.
 *
 * It evaluates Eq. (1) of "PLQCD library for Lattice QCD on multi-core
 * machines" (Sec. 2) site by site, with full 4x4 projectors (1 -/+ gamma_mu):
 *
 *   psi(x) = sum_mu [ U_mu(x) (1 - gamma_mu) phi(x + mu)
 *                     + U_mu(x - mu)^dagger (1 + gamma_mu) phi(x - mu) ]
 *
 * The outer loop over lattice sites is an OpenMP "for" construct, the
 * threading model of Sec. 2.1.  There is no blocking, no half-spinor trick and
 * no precomputed neighbour table: a reader can check each line against Eq. (1).
 *
 * Conventions (identical to the NumPy oracle, stated independently here):
 *   dims = {T, Lx, Ly, Lz}; mu = 0 is time, mu = 1, 2, 3 are x, y, z.
 *   lexicographic site s = ((t*Lz + z)*Ly + y)*Lx + x.
 *   phi[s][spin][colour] and U[s][mu][row][col] are interleaved (re, im) doubles.
 *   Space is periodic; a hop that crosses between t = T-1 and t = 0 is
 *   multiplied by t_bc (-1 for antiperiodic time).
 *   gamma basis: chiral, gamma_mu = [[0, A_mu], [A_mu^dagger, 0]],
 *   A_0 = -1, A_k = -i sigma_k (the DD-HMC documentation cited after Eq. (2)).
 */
#include <complex.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static cplx gamma_mat[4][4][4];
static int gamma_ready = 0;

static void init_gamma(void)
{
    if (gamma_ready) return;
    memset(gamma_mat, 0, sizeof(gamma_mat));
    /* gamma_0 */
    gamma_mat[0][0][2] = -1; gamma_mat[0][1][3] = -1;
    gamma_mat[0][2][0] = -1; gamma_mat[0][3][1] = -1;
    /* gamma_1 */
    gamma_mat[1][0][3] = -I; gamma_mat[1][1][2] = -I;
    gamma_mat[1][2][1] = I;  gamma_mat[1][3][0] = I;
    /* gamma_2 */
    gamma_mat[2][0][3] = -1; gamma_mat[2][1][2] = 1;
    gamma_mat[2][2][1] = 1;  gamma_mat[2][3][0] = -1;
    /* gamma_3 */
    gamma_mat[3][0][2] = -I; gamma_mat[3][1][3] = I;
    gamma_mat[3][2][0] = I;  gamma_mat[3][3][1] = -I;
    gamma_ready = 1;
}

static long lex_index(const int L[4], const int c[4])
{
    /* L and c in mu order: {T, Lx, Ly, Lz} and {t, x, y, z} */
    return (((long)c[0] * L[3] + c[3]) * L[2] + c[2]) * L[1] + c[1];
}

static void coords_of(const int L[4], long s, int c[4])
{
    c[1] = (int)(s % L[1]); s /= L[1];
    c[2] = (int)(s % L[2]); s /= L[2];
    c[3] = (int)(s % L[3]); s /= L[3];
    c[0] = (int)s;
}

/* out[spin][colour] = psi(x) of Eq. (1) at lexicographic site s. */
static void hopping_site(const int L[4], int t_bc, const cplx *U, const cplx *phi, long s, cplx out[4][3])
{
    int c[4], n[4];
    cplx proj[4][3];
    coords_of(L, s, c);
    for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a) out[sp][a] = 0;

    for (int mu = 0; mu < 4; ++mu) {
        /* forward term: U_mu(x) (1 - gamma_mu) phi(x + mu) */
        memcpy(n, c, sizeof(n));
        n[mu] = (c[mu] + 1) % L[mu];
        double sign = (mu == 0 && c[0] == L[0] - 1) ? (double)t_bc : 1.0;
        long y = lex_index(L, n);
        const cplx *py = phi + 12 * y;
        for (int sp = 0; sp < 4; ++sp)
            for (int b = 0; b < 3; ++b) {
                cplx v = 0;
                for (int tp = 0; tp < 4; ++tp) {
                    cplx p = (sp == tp ? 1.0 : 0.0) - gamma_mat[mu][sp][tp];
                    v += p * py[3 * tp + b];
                }
                proj[sp][b] = v;
            }
        const cplx *Ux = U + 36 * s + 9 * mu;
        for (int sp = 0; sp < 4; ++sp)
            for (int a = 0; a < 3; ++a) {
                cplx acc = 0;
                for (int b = 0; b < 3; ++b) acc += Ux[3 * a + b] * proj[sp][b];
                out[sp][a] += sign * acc;
            }

        /* backward term: U_mu(x - mu)^dagger (1 + gamma_mu) phi(x - mu) */
        memcpy(n, c, sizeof(n));
        n[mu] = (c[mu] - 1 + L[mu]) % L[mu];
        sign = (mu == 0 && c[0] == 0) ? (double)t_bc : 1.0;
        y = lex_index(L, n);
        py = phi + 12 * y;
        for (int sp = 0; sp < 4; ++sp)
            for (int b = 0; b < 3; ++b) {
                cplx v = 0;
                for (int tp = 0; tp < 4; ++tp) {
                    cplx p = (sp == tp ? 1.0 : 0.0) + gamma_mat[mu][sp][tp];
                    v += p * py[3 * tp + b];
                }
                proj[sp][b] = v;
            }
        const cplx *Uy = U + 36 * y + 9 * mu;
        for (int sp = 0; sp < 4; ++sp)
            for (int a = 0; a < 3; ++a) {
                cplx acc = 0;
                for (int b = 0; b < 3; ++b) acc += conj(Uy[3 * b + a]) * proj[sp][b];
                out[sp][a] += sign * acc;
            }
    }
}

static int set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* Number of OpenMP threads the oracle uses when nthreads <= 0. */
int plq_oracle_threads(int nthreads) { return set_threads(nthreads); }

/* psi = H phi over the whole lattice (Eq. (1)). */
void plq_oracle_hopping(const int dims[4], int t_bc, const double *U, const double *phi, double *psi, int nthreads)
{
    init_gamma();
    set_threads(nthreads);
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    const cplx *u = (const cplx *)U;
    const cplx *p = (const cplx *)phi;
    cplx *o = (cplx *)psi;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; ++s) {
        cplx out[4][3];
        hopping_site(dims, t_bc, u, p, s, out);
        memcpy(o + 12 * s, out, sizeof(out));
    }
}

/* psi = M phi = phi - kappa H phi over the whole lattice. */
void plq_oracle_wilson(const int dims[4], int t_bc, double kappa, const double *U, const double *phi, double *psi,
                       int nthreads)
{
    init_gamma();
    set_threads(nthreads);
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    const cplx *u = (const cplx *)U;
    const cplx *p = (const cplx *)phi;
    cplx *o = (cplx *)psi;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; ++s) {
        cplx out[4][3];
        hopping_site(dims, t_bc, u, p, s, out);
        for (int k = 0; k < 12; ++k) o[12 * s + k] = p[12 * s + k] - kappa * (&out[0][0])[k];
    }
}

/* out[i] = (H phi)(sites[i]) for a list of lexicographic sites. */
void plq_oracle_hopping_sites(const int dims[4], int t_bc, const double *U, const double *phi, const long *sites,
                              long nsites, double *out, int nthreads)
{
    init_gamma();
    set_threads(nthreads);
    const cplx *u = (const cplx *)U;
    const cplx *p = (const cplx *)phi;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < nsites; ++i) {
        cplx r[4][3];
        hopping_site(dims, t_bc, u, p, sites[i], r);
        memcpy(o + 12 * i, r, sizeof(r));
    }
}
