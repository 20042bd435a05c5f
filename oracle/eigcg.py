"""FP64 NumPy oracle of incremental EigCG (deflation for many right-hand sides).

TEST INFRASTRUCTURE (see the package header): only tests and the benchmark's
CPU legs use it; it shares no code with the CUDA path.

The paper (Sec. 3) adds EigCG (Stathopoulos and Orginos, SIAM J. Sci. Comput.
32 (2010) 439) to tmLQCD and runs it with nev = 10 eigenvectors per
right-hand side, a search space of m = 60 and 30 right-hand sides (300
vectors), in double precision to a relative tolerance of 1e-8.  The algorithm
as published, for a Hermitian positive definite A:

eigCG(nev, m) is CG in which the normalised residuals v_j = r_j / |r_j| --
the Lanczos vectors of A -- are kept in a search space V with the Lanczos
tridiagonal matrix T built from the CG coefficients:
    T[j, j]   = 1/alpha_j + beta_{j-1}/alpha_{j-1}
    T[j, j+1] = T[j+1, j] = -sqrt(beta_j)/alpha_j
(the sign of the off-diagonal follows from r_{j+1} = r_j - alpha_j A p_j).
When V holds m vectors it is restarted with 2*nev Ritz vectors: the nev
lowest eigenvectors Y of T and the nev lowest of its leading (m-1)x(m-1) block
(padded with a zero row) are orthonormalised into Q (m x 2nev); the Ritz pairs
(Z, M) of H = Q^T T Q give V <- V Q Z and T <- diag(M); the next Lanczos vector
couples to the restarted basis through t * (Q Z)[m-1, :], t being the
off-diagonal entry it would have had.  At convergence the nev lowest Ritz
vectors of the space are returned.

Incremental eigCG accumulates those vectors over the first right-hand sides in
an orthonormal basis U with H = U^H A U, and starts every solve from the
Galerkin projection x0 = U H^{-1} U^H b ("init-CG"); the right-hand sides after
the accumulation phase run plain CG from that x0.
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def eigcg(apply_A, b, x0, nev, m, tol, maxit=100000, return_space=False):
    """eigCG(nev, m) on A x = b from x0.  Returns (x, iterations, ritz_vectors, ritz_values)
    (and the final search space V and its matrix T when ``return_space``).

    Converged when |r| <= tol * |b| (the recursive residual, as in plain CG).
    """
    x = x0.copy()
    r = b - apply_A(x)
    p = r.copy()
    rho = np.real(_dot(r, r))
    bnorm = np.sqrt(np.real(_dot(b, b)))
    n_shape = b.shape
    V = np.zeros((m + 1,) + n_shape, dtype=np.complex128)
    T = np.zeros((m + 1, m + 1))
    vs = 0
    V[0] = r / np.sqrt(rho)
    vs = 1
    alpha_prev = beta_prev = None
    it = 0
    complete = False  # True when the last vector of V has its diagonal entry
    while it < maxit:
        Ap = apply_A(p)
        alpha = rho / np.real(_dot(p, Ap))
        T[vs - 1, vs - 1] = 1.0 / alpha + (beta_prev / alpha_prev if alpha_prev is not None else 0.0)
        x = x + alpha * p
        r = r - alpha * Ap
        rho_new = np.real(_dot(r, r))
        beta = rho_new / rho
        p = r + beta * p
        it += 1
        t = -np.sqrt(beta) / alpha
        if np.sqrt(rho_new) <= tol * bnorm:
            rho = rho_new
            complete = True
            break
        if vs == m:
            Tm = T[:m, :m]
            w, Y = np.linalg.eigh(Tm)
            Y = Y[:, :nev]
            w2, Y2 = np.linalg.eigh(Tm[: m - 1, : m - 1])
            Yold = np.vstack([Y2[:, :nev], np.zeros((1, nev))])
            Q, _ = np.linalg.qr(np.hstack([Y, Yold]))
            H = Q.T @ Tm @ Q
            M, Z = np.linalg.eigh(H)
            QZ = Q @ Z
            k = QZ.shape[1]
            V[:k] = np.tensordot(QZ.T, V[:m], axes=(1, 0))
            T[:, :] = 0.0
            T[:k, :k] = np.diag(M)
            c = t * QZ[m - 1, :]
            T[k, :k] = c
            T[:k, k] = c
            vs = k
        else:
            T[vs, vs - 1] = T[vs - 1, vs] = t
        V[vs] = r / np.sqrt(rho_new)
        vs += 1
        alpha_prev, beta_prev = alpha, beta
        rho = rho_new
    # Ritz vectors of the final space
    k = vs if complete else vs - 1
    w, Y = np.linalg.eigh(T[:k, :k])
    ritz = np.tensordot(Y[:, :nev].T, V[:k], axes=(1, 0))
    if return_space:
        return x, it, ritz, w[:nev], V[:k].copy(), T[:k, :k].copy()
    return x, it, ritz, w[:nev]


class IncrementalEigCG:
    """Incremental eigCG: accumulate nev Ritz vectors per solve over the first
    `n_accumulate` right-hand sides; every solve starts from x0 = U H^{-1} U^H b."""

    def __init__(self, apply_A, nev=10, m=60, n_accumulate=30, tol=1e-8):
        self.A = apply_A
        self.nev, self.m, self.n_acc, self.tol = nev, m, n_accumulate, tol
        self.U = []          # orthonormal basis vectors
        self.H = np.zeros((0, 0), dtype=np.complex128)
        self.solved = 0

    def init_guess(self, b):
        if not self.U:
            return np.zeros_like(b)
        Ub = np.array([_dot(u, b) for u in self.U])
        y = np.linalg.solve(self.H, Ub)
        return np.tensordot(y, np.array(self.U), axes=(0, 0))

    def _add(self, vectors):
        for v in vectors:
            w = v.copy()
            for _ in range(2):  # classical Gram-Schmidt, twice
                for u in self.U:
                    w = w - _dot(u, w) * u
            nrm = np.sqrt(np.real(_dot(w, w)))
            if nrm < 1e-10:
                continue
            w = w / nrm
            Aw = self.A(w)
            col = np.array([_dot(u, Aw) for u in self.U])
            k = len(self.U)
            Hn = np.zeros((k + 1, k + 1), dtype=np.complex128)
            Hn[:k, :k] = self.H
            Hn[:k, k] = col
            Hn[k, :k] = np.conj(col)
            Hn[k, k] = np.real(_dot(w, Aw))
            self.H = Hn
            self.U.append(w)

    def solve(self, b):
        x0 = self.init_guess(b)
        if self.solved < self.n_acc:
            x, it, ritz, _ = eigcg(self.A, b, x0, self.nev, self.m, self.tol)
            self._add(list(ritz))
        else:
            x, it = cg_plain(self.A, b, x0, self.tol)
        self.solved += 1
        return x, it


def cg_plain(apply_A, b, x0, tol, maxit=100000):
    """Textbook CG from x0 until |r| <= tol |b|."""
    x = x0.copy()
    r = b - apply_A(x)
    p = r.copy()
    rho = np.real(_dot(r, r))
    bnorm = np.sqrt(np.real(_dot(b, b)))
    for it in range(1, maxit + 1):
        if np.sqrt(rho) <= tol * bnorm:
            return x, it - 1
        Ap = apply_A(p)
        alpha = rho / np.real(_dot(p, Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        rho_new = np.real(_dot(r, r))
        p = r + (rho_new / rho) * p
        rho = rho_new
    return x, maxit
