"""Pins of the EigCG oracle (no GPU): Ritz pairs against dense eigenpairs,
deflation against its definition, and the paper's printed parameters."""
import numpy as np
import pytest

import synthetic as S
from oracle import eigcg as E
from oracle import wilson as W


def paper_parameters():
    vals = {}
    for line in open(__file__.replace("test_oracle_eigcg.py", "golden/eigcg_paper_parameters.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


@pytest.fixture(scope="module")
def system():
    dims = (4, 2, 2, 4)  # 64 sites, 32 even: A is 384 x 384
    kappa = 0.124
    U = S.gauge_field(dims, 0.3, 71)
    par = W.parity(S.lattice_shape(dims))
    shape = S.lattice_shape(dims) + (4, 3)
    A = lambda v: W.schur_dag(U, W.schur(U, v, kappa), kappa)
    even = np.repeat(par.ravel() == 0, 12)
    Ad = W.dense(A, shape)[np.ix_(even, even)]
    return U, kappa, shape, A, even, Ad


def test_paper_parameters_fixture():
    p = paper_parameters()
    assert (p["nev"], p["m"], p["rhs_accumulated"], p["vectors"]) == (10, 60, 30, 300)
    assert p["nev"] * p["rhs_accumulated"] == p["vectors"]
    assert p["tol"] == 1e-8


def test_eigcg_solves_and_ritz_values_bound_the_spectrum(system):
    U, kappa, shape, A, even, Ad = system
    b = W.restrict(S.gaussian_spinor((4, 2, 2, 4), 72), 0)
    x, it, ritz, theta = E.eigcg(A, b, np.zeros_like(b), nev=4, m=16, tol=1e-10)
    assert np.linalg.norm(A(x) - b) <= 1e-9 * np.linalg.norm(b)
    lam = np.linalg.eigvalsh(Ad)
    # Rayleigh-Ritz: the k-th Ritz value is >= the k-th eigenvalue (Cauchy interlacing) ...
    assert np.all(theta >= lam[:4] * (1 - 1e-10))
    # ... every Ritz pair has an eigenvalue within its residual norm (Hermitian
    # Bauer-Fike), and the lowest one has converged onto the smallest eigenvalue
    for k in range(4):
        v = ritz[k]
        res = np.linalg.norm(A(v) - theta[k] * v) / np.linalg.norm(v)
        assert np.min(np.abs(lam - theta[k])) <= res * (1 + 1e-8) + 1e-14
    assert abs(theta[0] - lam[0]) < 1e-2 * lam[0]


@pytest.mark.parametrize("m,nev", [(400, 4), (16, 4), (12, 3)])
def test_tridiagonal_is_the_projected_operator(system, m, nev):
    # The T built from the CG coefficients (and restarted) is V^H A V of the kept
    # search space: checks the Lanczos/CG relation, its signs and the restart.
    U, kappa, shape, A, even, Ad = system
    b = W.restrict(S.gaussian_spinor((4, 2, 2, 4), 76), 0)
    _, it, _, _, V, T = E.eigcg(A, b, np.zeros_like(b), nev=nev, m=m, tol=1e-10, return_space=True)
    k = min(T.shape[0], 14)  # the early basis vectors keep their orthogonality best
    Vm = np.array([v.reshape(-1)[even] for v in V[:k]]).T
    H = Vm.conj().T @ Ad @ Vm
    assert np.max(np.abs(H - T[:k, :k])) < 1e-8 * np.abs(Ad).max()


def test_eigcg_ritz_vectors_are_orthonormal(system):
    U, kappa, shape, A, even, Ad = system
    b = W.restrict(S.gaussian_spinor((4, 2, 2, 4), 73), 0)
    _, _, ritz, _ = E.eigcg(A, b, np.zeros_like(b), nev=4, m=12, tol=1e-10)
    G = np.array([[np.vdot(a, c) for c in ritz] for a in ritz])
    assert np.max(np.abs(G - np.eye(len(ritz)))) < 1e-8


def test_without_restart_matches_plain_cg(system):
    # with m larger than the iteration count eigCG is exactly CG
    U, kappa, shape, A, even, Ad = system
    b = W.restrict(S.gaussian_spinor((4, 2, 2, 4), 74), 0)
    x1, it1, _, _ = E.eigcg(A, b, np.zeros_like(b), nev=2, m=500, tol=1e-9)
    x2, it2 = E.cg_plain(A, b, np.zeros_like(b), 1e-9)
    assert it1 == it2 and np.allclose(x1, x2, atol=1e-12 * np.abs(x2).max())


def test_init_cg_with_exact_eigenvectors(system):
    # Galerkin start on the lowest exact eigenvectors removes those modes from the error
    U, kappa, shape, A, even, Ad = system
    lam, vecs = np.linalg.eigh(Ad)
    inc = E.IncrementalEigCG(A, nev=4, m=12, n_accumulate=0, tol=1e-9)
    for k in range(6):
        v = np.zeros(shape, complex)
        v.reshape(-1)[even] = vecs[:, k]
        inc._add([v])
    b = W.restrict(S.gaussian_spinor((4, 2, 2, 4), 75), 0)
    x0 = inc.init_guess(b)
    e0 = np.linalg.solve(Ad, b.reshape(-1)[even]) - x0.reshape(-1)[even]
    assert np.max(np.abs(vecs[:, :6].conj().T @ e0)) < 1e-10 * np.abs(e0).max()
    _, it_defl = E.cg_plain(A, b, x0, 1e-9)
    _, it_plain = E.cg_plain(A, b, np.zeros_like(b), 1e-9)
    assert it_defl < it_plain


def test_incremental_eigcg_reduces_iterations(system):
    U, kappa, shape, A, even, Ad = system
    inc = E.IncrementalEigCG(A, nev=3, m=12, n_accumulate=4, tol=1e-9)
    its = []
    for s in range(6):
        b = W.restrict(S.gaussian_spinor((4, 2, 2, 4), 80 + s), 0)
        x, it = inc.solve(b)
        assert np.linalg.norm(A(x) - b) <= 2e-9 * np.linalg.norm(b)
        its.append(it)
    assert len(inc.U) >= 8
    assert its[-1] < its[0]
