"""FP64 NumPy oracle for the Wilson-Dirac hopping operator and its solvers.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline leg may import this module.  It shares no code with the CUDA path and
the CUDA path never calls it.

What it computes (paper: "PLQCD library for Lattice QCD on multi-core
machines", Sec. 2):

* ``hopping``: the hopping part of the lattice Dirac operator, Eq. (1),
      psi(x) = sum_mu [ U_mu(x) (1 - gamma_mu) phi(x + mu)
                        + U_mu(x - mu)^dagger (1 + gamma_mu) phi(x - mu) ],
  written out literally with full 4x4 gamma matrices and whole-lattice shifts.
* ``hopping_theta``: the same operator through the auxiliary fields of Eq. (2),
  theta+_mu(x) = (1 - gamma_mu) phi(x) and theta-_mu(x) = U_mu(x)^dagger
  (1 + gamma_mu) phi(x), psi(x) = sum_mu [U_mu(x) theta+_mu(x + mu) +
  theta-_mu(x - mu)].  Used to pin Eq. (1) against Eq. (2).
* ``link_spinor_product``: psi(i) = U(i) phi(i), the kernel of the paper's
  prefetch experiment (Sec. 2.2).
* The Wilson operator M = 1 - kappa*H, its even-odd Schur complement
  Mhat = 1 - kappa^2 H_eo H_oe, and textbook CG (on Mhat^dagger Mhat) and
  BiCGstab (on Mhat) solvers.  The paper names no solver and no normalisation;
  the readings used here are:

  - gamma basis: the chiral basis of the DD-HMC code documentation that the
    paper cites for the half-spinor trick (Sec. 2, after Eq. (2)):
    gamma_mu = [[0, A_mu], [A_mu^dagger, 0]] with A_0 = -1 and
    A_k = -i sigma_k, so gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 =
    diag(1, 1, -1, -1);
  - mu = 0 is time; space is periodic, time antiperiodic: a hop that crosses
    between t = T-1 and t = 0 picks up the factor ``t_bc`` (-1);
  - H is taken exactly as Eq. (1) (projectors without a factor 1/2), so the
    free-field critical kappa is 1/8;
  - even sites have (t + x + y + z) even.

Fields use the canonical layout of the ``synthetic`` module: spinors
``(T, Lz, Ly, Lx, 4, 3)`` and links ``(T, Lz, Ly, Lx, 4, 3, 3)``, complex128.
Even-odd fields are full-lattice arrays that are zero on the other parity.
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------
# Dirac matrices (chiral basis of the DD-HMC documentation)
# --------------------------------------------------------------------------
_i = 1j
GAMMA = np.array(
    [
        [[0, 0, -1, 0], [0, 0, 0, -1], [-1, 0, 0, 0], [0, -1, 0, 0]],
        [[0, 0, 0, -_i], [0, 0, -_i, 0], [0, _i, 0, 0], [_i, 0, 0, 0]],
        [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
        [[0, 0, -_i, 0], [0, 0, 0, _i], [_i, 0, 0, 0], [0, -_i, 0, 0]],
    ],
    dtype=np.complex128,
)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ONE4 = np.eye(4, dtype=np.complex128)

# array axis of direction mu in a (T, Lz, Ly, Lx, ...) field
_AXIS = (0, 3, 2, 1)


def axis_of(mu):
    return _AXIS[mu]


def parity(shape4):
    """(t + x + y + z) mod 2 on a lattice of array shape (T, Lz, Ly, Lx)."""
    T, Lz, Ly, Lx = shape4
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return (t + x + y + z) % 2


def shift_fermion(f, mu, step, t_bc):
    """f(x + step*mu) for a fermion field: periodic in space, ``t_bc`` in time.

    A site whose neighbour lies across the time boundary (t = T-1 going
    forward, t = 0 going backward) receives the neighbour times ``t_bc``.
    """
    out = np.roll(f, -step, axis=_AXIS[mu])
    if mu == 0 and t_bc != 1:
        T = f.shape[0]
        edge = T - 1 if step > 0 else 0
        out[edge] = out[edge] * t_bc
    return out


def shift_gauge(U_mu, mu, step):
    """U_mu(x + step*mu) for one link direction: the gauge field is periodic."""
    return np.roll(U_mu, -step, axis=_AXIS[mu])


def _spin_colour(P, V, f):
    """Apply spin matrix P (4x4) and per-site colour matrix V (3x3) to f."""
    return np.einsum("...ab,st,...tb->...sa", V, P, f, optimize=True)


def hopping(U, phi, t_bc=-1):
    """Eq. (1): the hopping operator with full 4x4 projectors (1 -/+ gamma_mu)."""
    psi = np.zeros_like(phi)
    for mu in range(4):
        U_mu = U[..., mu, :, :]
        # forward: U_mu(x) (1 - gamma_mu) phi(x + mu)
        psi += _spin_colour(ONE4 - GAMMA[mu], U_mu, shift_fermion(phi, mu, +1, t_bc))
        # backward: U_mu(x - mu)^dagger (1 + gamma_mu) phi(x - mu)
        U_back_dag = np.conj(np.swapaxes(shift_gauge(U_mu, mu, -1), -1, -2))
        psi += _spin_colour(ONE4 + GAMMA[mu], U_back_dag, shift_fermion(phi, mu, -1, t_bc))
    return psi


def theta_fields(U, phi, mu):
    """Auxiliary fields of Eq. (2) at every site: theta+_mu(x) and theta-_mu(x)."""
    U_mu = U[..., mu, :, :]
    eye3 = np.broadcast_to(np.eye(3, dtype=np.complex128), U_mu.shape)
    theta_p = _spin_colour(ONE4 - GAMMA[mu], eye3, phi)
    theta_m = _spin_colour(ONE4 + GAMMA[mu], np.conj(np.swapaxes(U_mu, -1, -2)), phi)
    return theta_p, theta_m


def hopping_theta(U, phi, t_bc=-1):
    """Eq. (2): psi(x) = sum_mu [U_mu(x) theta+_mu(x + mu) + theta-_mu(x - mu)]."""
    psi = np.zeros_like(phi)
    eye4 = ONE4
    for mu in range(4):
        theta_p, theta_m = theta_fields(U, phi, mu)
        psi += _spin_colour(eye4, U[..., mu, :, :], shift_fermion(theta_p, mu, +1, t_bc))
        psi += shift_fermion(theta_m, mu, -1, t_bc)
    return psi


# --------------------------------------------------------------------------
# Wilson operator, even-odd decomposition
# --------------------------------------------------------------------------
def wilson(U, phi, kappa, t_bc=-1):
    """M phi = phi - kappa * H phi."""
    return phi - kappa * hopping(U, phi, t_bc)


def gamma5(phi):
    return np.einsum("st,...tc->...sc", GAMMA5, phi)


def restrict(phi, par):
    """Keep the sites of parity ``par`` (0 even, 1 odd); zero the others."""
    mask = parity(phi.shape[:4]) == par
    return phi * mask[..., None, None]


def hop_eo(U, phi, out_parity, t_bc=-1):
    """H restricted to output parity ``out_parity`` and input parity 1-out_parity.

    ``hop_eo(U, v, 0)`` is H_eo v_o and ``hop_eo(U, v, 1)`` is H_oe v_e.
    """
    return restrict(hopping(U, restrict(phi, 1 - out_parity), t_bc), out_parity)


def schur(U, v_e, kappa, t_bc=-1):
    """Mhat v_e = v_e - kappa^2 H_eo H_oe v_e on even sites."""
    v_e = restrict(v_e, 0)
    return v_e - kappa * kappa * hop_eo(U, hop_eo(U, v_e, 1, t_bc), 0, t_bc)


def schur_dag(U, v_e, kappa, t_bc=-1):
    """Mhat^dagger = gamma5 Mhat gamma5 (gamma5 H gamma5 = H^dagger)."""
    return gamma5(schur(U, gamma5(v_e), kappa, t_bc))


def schur_rhs(U, b, kappa, t_bc=-1):
    """bhat_e = b_e + kappa H_eo b_o."""
    return restrict(b, 0) + kappa * hop_eo(U, b, 0, t_bc)


def reconstruct_odd(U, x_e, b, kappa, t_bc=-1):
    """x_o = b_o + kappa H_oe x_e."""
    return restrict(b, 1) + kappa * hop_eo(U, x_e, 1, t_bc)


def inner(a, b):
    """<a, b> = sum conj(a) b."""
    return np.vdot(a.ravel(), b.ravel())


def norm(a):
    return float(np.sqrt(np.real(inner(a, a))))


# --------------------------------------------------------------------------
# Twisted-mass Wilson operator (Sec. 3: the tmLQCD solves use twisted-mass fermions)
# --------------------------------------------------------------------------
# The paper does not print the operator; the reading is the standard one of
# the twisted-mass formulation it cites (Frezzotti et al.): in the hopping
# normalisation M_tm = 1 - kappa H + 2 i kappa mu gamma5.
def twisted(U, phi, kappa, mu, t_bc=-1):
    """M_tm phi = phi - kappa H phi + 2 i kappa mu gamma5 phi."""
    return wilson(U, phi, kappa, t_bc) + 2j * kappa * mu * gamma5(phi)


def twist_diag(phi, kappa, mu, inverse=False):
    """The site-diagonal part A = 1 + 2 i kappa mu gamma5 (or its inverse)."""
    nu = 2 * kappa * mu
    if inverse:
        return (phi - 1j * nu * gamma5(phi)) / (1 + nu * nu)
    return phi + 1j * nu * gamma5(phi)


def schur_tm(U, v_e, kappa, mu, t_bc=-1):
    """Mhat_tm v_e = A v_e - kappa^2 H_eo A^{-1} H_oe v_e (A = 1 + 2 i kappa mu gamma5)."""
    v_e = restrict(v_e, 0)
    inner = twist_diag(hop_eo(U, v_e, 1, t_bc), kappa, mu, inverse=True)
    return twist_diag(v_e, kappa, mu) - kappa * kappa * hop_eo(U, inner, 0, t_bc)


def schur_tm_rhs(U, b, kappa, mu, t_bc=-1):
    """bhat_e = b_e + kappa H_eo A^{-1} b_o."""
    return restrict(b, 0) + kappa * hop_eo(U, twist_diag(restrict(b, 1), kappa, mu, inverse=True), 0, t_bc)


def reconstruct_odd_tm(U, x_e, b, kappa, mu, t_bc=-1):
    """x_o = A^{-1} (b_o + kappa H_oe x_e)."""
    return twist_diag(restrict(b, 1) + kappa * hop_eo(U, x_e, 1, t_bc), kappa, mu, inverse=True)


def solve_cg_eo_tm(U, b, kappa, mu, tol=1e-10, maxit=20000, t_bc=-1, check_every=10):
    """M_tm x = b by CG on Mhat_tm^dag Mhat_tm, with Mhat_tm(mu)^dag = gamma5 Mhat_tm(-mu) gamma5."""
    bhat = schur_tm_rhs(U, b, kappa, mu, t_bc)
    bnorm = norm(b)
    Mh = lambda v: schur_tm(U, v, kappa, mu, t_bc)
    Mhd = lambda v: gamma5(schur_tm(U, gamma5(v), kappa, -mu, t_bc))
    state = {"n": 0}

    def check(x, rnorm):
        state["n"] += 1
        if state["n"] % check_every:
            return False
        return norm(bhat - Mh(x)) <= tol * bnorm

    x_e, it, hist = cg(lambda v: Mhd(Mh(v)), Mhd(bhat), None, 0.0, maxit, check)
    x = restrict(x_e, 0) + reconstruct_odd_tm(U, x_e, b, kappa, mu, t_bc)
    rel = norm(b - twisted(U, x, kappa, mu, t_bc)) / bnorm
    return SolveResult(x, it, "ok" if rel <= tol else "not_converged", rel, hist)


# --------------------------------------------------------------------------
# Solvers
# --------------------------------------------------------------------------
class SolveResult:
    def __init__(self, x, iterations, status, true_rel_residual, history):
        self.x = x
        self.iterations = iterations
        self.status = status
        self.true_rel_residual = true_rel_residual
        self.history = history


def cg(apply_A, rhs, x0=None, tol=1e-12, maxit=10000, check=None):
    """Hestenes-Stiefel conjugate gradients for a Hermitian positive A.

    r = rhs - A x, p = r, rho = <r, r>; each step q = A p,
    alpha = rho / <p, q>, x += alpha p, r -= alpha q, beta = rho'/rho,
    p = r + beta p.  Stops when ``check(x, rnorm)`` returns True (if given)
    or when ||r|| <= tol * ||rhs||.
    """
    x = np.zeros_like(rhs) if x0 is None else x0.copy()
    r = rhs - apply_A(x) if x0 is not None else rhs.copy()
    p = r.copy()
    rho = np.real(inner(r, r))
    bnorm = norm(rhs)
    history = [np.sqrt(rho)]
    for it in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rho / np.real(inner(p, q))
        x = x + alpha * p
        r = r - alpha * q
        rho_new = np.real(inner(r, r))
        history.append(np.sqrt(rho_new))
        done = check(x, np.sqrt(rho_new)) if check is not None else np.sqrt(rho_new) <= tol * bnorm
        if done:
            return x, it, history
        p = r + (rho_new / rho) * p
        rho = rho_new
    return x, maxit, history


def solve_cg_eo(U, b, kappa, tol=1e-10, maxit=20000, t_bc=-1, check_every=10):
    """Solve M x = b by CG on the even-odd normal equations Mhat^dag Mhat x_e = Mhat^dag bhat.

    Converged when the true residual ||bhat - Mhat x_e|| <= tol * ||b||, which
    equals ||b - M x|| / ||b|| once x_o = b_o + kappa H_oe x_e.
    """
    bhat = schur_rhs(U, b, kappa, t_bc)
    bnorm = norm(b)
    A = lambda v: schur_dag(U, schur(U, v, kappa, t_bc), kappa, t_bc)
    rhs = schur_dag(U, bhat, kappa, t_bc)
    state = {"n": 0}

    def check(x, rnorm):
        state["n"] += 1
        if state["n"] % check_every:
            return False
        return norm(bhat - schur(U, x, kappa, t_bc)) <= tol * bnorm

    x_e, it, hist = cg(A, rhs, None, 0.0, maxit, check)
    x = restrict(x_e, 0) + reconstruct_odd(U, x_e, b, kappa, t_bc)
    rel = norm(b - wilson(U, x, kappa, t_bc)) / bnorm
    return SolveResult(x, it, "ok" if rel <= tol else "not_converged", rel, hist)


class Breakdown(RuntimeError):
    pass


def bicgstab(apply_M, rhs, x0=None, tol=1e-12, maxit=10000, check=None, breakdown=1e-300):
    """BiCGstab (van der Vorst, 1992) for a general nonsingular M.

    r0 = rhs - M x, rhat = r0, rho = alpha = omega = 1, v = p = 0; each step
    rho' = <rhat, r>, beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v),
    v = M p, alpha = rho' / <rhat, v>, s = r - alpha v, t = M s,
    omega = <t, s> / <t, t>, x += alpha p + omega s, r = s - omega t.
    """
    x = np.zeros_like(rhs) if x0 is None else x0.copy()
    r = rhs - apply_M(x) if x0 is not None else rhs.copy()
    rhat = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(rhs)
    p = np.zeros_like(rhs)
    scale = norm(rhs) ** 2
    history = [norm(r)]
    for it in range(1, maxit + 1):
        rho_new = inner(rhat, r)
        if abs(rho_new) <= breakdown * scale:
            raise Breakdown("rho")
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply_M(p)
        alpha = rho_new / inner(rhat, v)
        s = r - alpha * v
        t = apply_M(s)
        tt = np.real(inner(t, t))
        if tt == 0.0:
            x = x + alpha * p
            return x, it, history
        omega = inner(t, s) / tt
        if abs(omega) <= breakdown:
            raise Breakdown("omega")
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        history.append(norm(r))
        done = check(x, history[-1]) if check is not None else history[-1] <= tol * np.sqrt(scale)
        if done:
            return x, it, history
    return x, maxit, history


def solve_bicgstab_eo(U, b, kappa, tol=1e-10, maxit=20000, t_bc=-1):
    """Solve M x = b by BiCGstab on Mhat x_e = bhat, then reconstruct x_o."""
    bhat = schur_rhs(U, b, kappa, t_bc)
    bnorm = norm(b)
    M = lambda v: schur(U, v, kappa, t_bc)

    def check(x, rnorm):
        if rnorm > tol * bnorm:
            return False
        return norm(bhat - M(x)) <= tol * bnorm

    x_e, it, hist = bicgstab(M, bhat, None, 0.0, maxit, check)
    x = restrict(x_e, 0) + reconstruct_odd(U, x_e, b, kappa, t_bc)
    rel = norm(b - wilson(U, x, kappa, t_bc)) / bnorm
    return SolveResult(x, it, "ok" if rel <= tol else "not_converged", rel, hist)


# --------------------------------------------------------------------------
# Dense forms (small lattices only)
# --------------------------------------------------------------------------
def dense(apply, shape):
    """Dense matrix of a linear map on spinor fields, column by column."""
    n = int(np.prod(shape))
    D = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        D[:, j] = apply(e.reshape(shape)).ravel()
        e[j] = 0.0
    return D


def brute_force_hopping_dense(U, t_bc=-1):
    """Dense H assembled block by block with explicit site loops (Eq. (1)).

    Row block of site x, column block of its neighbour y; inside a block the
    index is spin*3 + colour.  Built from coordinates and explicit neighbour
    arithmetic, independent of ``hopping``.
    """
    T, Lz, Ly, Lx = U.shape[:4]
    L = (T, Lx, Ly, Lz)
    n = T * Lz * Ly * Lx

    def lex(c):  # c = (t, x, y, z)
        t, x, y, z = c
        return ((t * Lz + z) * Ly + y) * Lx + x

    D = np.zeros((12 * n, 12 * n), dtype=np.complex128)
    for t in range(T):
        for z in range(Lz):
            for y in range(Ly):
                for x in range(Lx):
                    c = [t, x, y, z]
                    s = lex(c)
                    for mu in range(4):
                        fwd = list(c)
                        fwd[mu] = (c[mu] + 1) % L[mu]
                        sign_f = t_bc if (mu == 0 and c[0] == T - 1) else 1
                        bwd = list(c)
                        bwd[mu] = (c[mu] - 1) % L[mu]
                        sign_b = t_bc if (mu == 0 and c[0] == 0) else 1
                        Ux = U[t, z, y, x, mu]
                        tb, xb, yb, zb = bwd
                        Ub = U[tb, zb, yb, xb, mu]
                        jf, jb = lex(fwd), lex(bwd)
                        D[12 * s:12 * s + 12, 12 * jf:12 * jf + 12] += sign_f * np.kron(ONE4 - GAMMA[mu], Ux)
                        D[12 * s:12 * s + 12, 12 * jb:12 * jb + 12] += sign_b * np.kron(ONE4 + GAMMA[mu], Ub.conj().T)
    return D


# --------------------------------------------------------------------------
# The link x spinor kernel of the prefetch experiment (Sec. 2.2)
# --------------------------------------------------------------------------
def link_spinor_product(U, phi):
    """psi(i) = U(i) phi(i) for records i = 0 .. n-1: the kernel that the paper
    isolates to measure prefetching and addressing (Sec. 2.2, overlap of
    communication with computation: sequential access, access through an index
    array x[i] and through a pointer array).  The access order decides only which
    record a loop step reaches; each record's result is its own SU(3) matrix
    applied to the colour vector of each of its four spin components.

    U: (n, 3, 3) complex, phi: (n, 4, 3) complex; returns (n, 4, 3).  Written as a
    loop over the 4 spin components of a per-record matrix-vector product."""
    U = np.asarray(U, dtype=np.complex128)
    phi = np.asarray(phi, dtype=np.complex128)
    out = np.empty_like(phi)
    for s in range(4):
        out[:, s, :] = np.matmul(U, phi[:, s, :, None])[:, :, 0]
    return out
