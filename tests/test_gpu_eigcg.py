"""Incremental EigCG on the GPU (Sec. 3 of the paper) against the oracle."""
import numpy as np
import pytest

import synthetic as S
from oracle import c_oracle as C
from oracle import eigcg as E
from oracle import wilson as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1405_0700_gb300 import F64, Context  # noqa: E402
from paper_1405_0700_gb300.plq import EigCG  # noqa: E402


def lowest_eigenvalues(apply_A, dims, k):
    """The k lowest eigenvalues of A = Mhat^dag Mhat on the even sites (Lanczos on the
    oracle's operator, independent of any eigCG code)."""
    from scipy.sparse.linalg import LinearOperator, eigsh

    shape = S.lattice_shape(dims) + (4, 3)
    even = W.parity(S.lattice_shape(dims)) == 0
    n = int(even.sum()) * 12

    def mv(v):
        full = np.zeros(shape, dtype=np.complex128)
        full[even] = v.reshape(-1, 4, 3)
        return apply_A(full)[even].ravel()

    op = LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    return np.sort(eigsh(op, k=k, which="SA", tol=1e-12, ncv=120, return_eigenvectors=False))


def test_eigcg_matches_oracle_and_deflates():
    """A smooth field near the critical kappa (isolated low modes), incremental EigCG as
    in Sec. 3 (nev vectors accumulated per solve).  For every solve: the normal-equation
    residual of the returned x_e is within the requested tolerance; x_e agrees with the
    exact solution (the oracle's CG run to 1e-14) and with the oracle's incremental eigCG
    within the bound |x - x'| <= (|r| + |r'|) / lambda_min that those residuals imply; the
    odd half agrees with x_o = b_o + kappa H_oe x_e of the exact solution.  At the end, the
    eigenvalues of the accumulated basis' H = U^H A U (Ritz values) lie above the true
    lowest eigenvalues (Cauchy interlacing) and agree with the oracle's to 1e-6, and the
    deflated solves need fewer iterations."""
    dims = (16, 4, 4, 4)
    kappa, tol, nev = 0.1255, 1e-10, 8
    U = S.gauge_field(dims, 0.05, 91)
    A = lambda v: W.schur_dag(U, W.schur(U, v, kappa), kappa)
    lam = lowest_eigenvalues(A, dims, 10)
    inc = E.IncrementalEigCG(A, nev=nev, m=24, n_accumulate=6, tol=tol)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        eig = EigCG(ctx, nev=nev, m=24, max_vectors=48)
        its, vecs = [], []
        for k in range(8):
            b = S.gaussian_spinor(dims, 300 + k)
            bd = ctx.to_device(b, F64)
            x = ctx.empty_full(F64)
            info = eig.solve(x, bd, kappa, tol=tol, accumulate=k < 6)
            xs = ctx.to_host(x, F64)
            its.append(info.iterations)
            vecs.append(eig.vectors)
            rhs = W.schur_dag(U, W.schur_rhs(U, b, kappa), kappa)
            xe = W.restrict(xs, 0)
            r_g = W.norm(rhs - A(xe))
            assert r_g <= 2 * tol * W.norm(rhs), (k, r_g / W.norm(rhs))
            x_star, _ = E.cg_plain(A, rhs, np.zeros_like(rhs), 1e-14)
            r_star = W.norm(rhs - A(x_star))
            assert W.norm(xe - x_star) <= 1.01 * (r_g + r_star) / lam[0], k
            x_o, _ = inc.solve(rhs)
            r_o = W.norm(rhs - A(x_o))
            assert W.norm(xe - x_o) <= 1.01 * (r_g + r_o) / lam[0], k
            # odd half: |H_oe| <= 8 for SU(3) links, so its error is at most 8 kappa times that of x_e
            odd_star = W.reconstruct_odd(U, x_star, b, kappa)
            assert W.norm(W.restrict(xs, 1) - odd_star) <= 1.01 * 8 * kappa * (r_g + r_star) / lam[0], k
            res = np.linalg.norm(b - C.wilson(U, xs, kappa)) / np.linalg.norm(b)
            assert abs(info.true_rel_residual - res) < 1e-12
        Hg = eig.projected_matrix()
        eig.close()
    assert vecs[0] == nev and vecs[5] == 6 * nev and vecs[7] == 6 * nev
    assert Hg.shape == (6 * nev, 6 * nev) and np.allclose(Hg, Hg.conj().T, atol=1e-14)
    theta_g = np.linalg.eigvalsh(Hg)[:nev]
    theta_o = np.linalg.eigvalsh(inc.H)[:nev]
    # The library orthonormalises its basis in FP32 (|U^H U - 1| ~ 1e-7), so the eigenvalues
    # of its H are Rayleigh-Ritz values only up to a relative perturbation of that size:
    # Cauchy interlacing (theta_k >= lambda_k) is asserted with a 1e-6 relative allowance.
    rel_o = (theta_g - theta_o) / theta_o
    rel_l = (theta_g - lam[:nev]) / lam[:nev]
    assert np.all(rel_l >= -1e-6), (rel_l, theta_g, lam[:nev])
    assert np.max(np.abs(rel_o)) <= 1e-6, (rel_o, theta_g, theta_o)
    assert np.max(rel_l) <= 1e-6, (rel_l, theta_g, lam[:nev])
    assert its[-1] <= 0.8 * its[0], its


def test_first_solve_matches_oracle_cg_iterations():
    # with an empty basis eigCG is CG: the iteration count must match the oracle's
    dims = (8, 4, 4, 4)
    kappa = 0.122
    U, b = S.gauge_and_spinor(dims, 0.3, 92)
    A = lambda v: W.schur_dag(U, W.schur(U, v, kappa), kappa)
    rhs = W.schur_dag(U, W.schur_rhs(U, b, kappa), kappa)
    _, it_oracle, _, _ = E.eigcg(A, rhs, np.zeros_like(rhs), nev=4, m=20, tol=1e-9)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        eig = EigCG(ctx, nev=4, m=20, max_vectors=8)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        info = eig.solve(x, bd, kappa, tol=1e-9)
        eig.close()
    assert abs(info.iterations - it_oracle) <= 2, (info.iterations, it_oracle)


def test_eigcg_rejects_bad_parameters():
    from paper_1405_0700_gb300 import PLQError

    with Context((4, 4, 4, 4)) as ctx:
        with pytest.raises(PLQError):
            EigCG(ctx, nev=10, m=12)  # m < 2 nev + 2


def test_eigcg_accumulates_for_tiny_sources():
    # the FP32 search space is scaled by a power of two: a source of norm ~1e-40
    # still yields the nev new basis vectors per accumulating solve
    dims = (16, 4, 4, 4)
    kappa = 0.1255
    U = S.gauge_field(dims, 0.05, 91)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        eig = EigCG(ctx, nev=8, m=24, max_vectors=24)
        for k in range(3):
            b = S.gaussian_spinor(dims, 400 + k) * 1e-40
            bd = ctx.to_device(b, F64)
            x = ctx.empty_full(F64)
            info = eig.solve(x, bd, kappa, tol=1e-10, accumulate=True)
            xs = ctx.to_host(x, F64)
            res = np.linalg.norm(b - C.wilson(U, xs, kappa)) / np.linalg.norm(b)
            assert res < 1e-7, (k, res)
        assert eig.vectors == 24
        eig.close()
