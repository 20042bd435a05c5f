"""Oracle solvers against dense linear algebra (no GPU)."""
import numpy as np
import pytest

import synthetic as S
from oracle import wilson as W


@pytest.fixture(scope="module")
def system():
    dims = (4, 4, 4, 4)
    U, b = S.gauge_and_spinor(dims, 0.3, 1)
    kappa = 0.12
    shape = S.lattice_shape(dims) + (4, 3)
    M = W.dense(lambda v: W.wilson(U, v, kappa), shape)
    x_ref = np.linalg.solve(M, b.ravel()).reshape(shape)
    return U, b, kappa, x_ref


def test_cg_eo_matches_dense_solve(system):
    U, b, kappa, x_ref = system
    res = W.solve_cg_eo(U, b, kappa, tol=1e-10)
    assert res.status == "ok" and res.true_rel_residual <= 1e-10
    assert np.linalg.norm(res.x - x_ref) / np.linalg.norm(x_ref) < 1e-8


def test_bicgstab_eo_matches_dense_solve(system):
    U, b, kappa, x_ref = system
    res = W.solve_bicgstab_eo(U, b, kappa, tol=1e-10)
    assert res.status == "ok" and res.true_rel_residual <= 1e-10
    assert np.linalg.norm(res.x - x_ref) / np.linalg.norm(x_ref) < 1e-8


def test_cg_error_a_norm_decreases():
    # CG minimises the A-norm of the error over growing Krylov spaces: it never increases.
    dims = (2, 2, 2, 4)
    U, b = S.gauge_and_spinor(dims, 0.3, 2)
    kappa = 0.12
    A = lambda v: W.schur_dag(U, W.schur(U, v, kappa), kappa)
    rhs = W.schur_dag(U, W.schur_rhs(U, b, kappa), kappa)
    shape = b.shape
    Ad = W.dense(A, shape)
    par = np.repeat(W.parity(shape[:4]).ravel(), 12) == 0
    Ae = Ad[np.ix_(par, par)]
    x_star = np.zeros(b.size, complex)
    x_star[par] = np.linalg.solve(Ae, rhs.ravel()[par])
    errs = []

    def check(x, rn):
        e = x.ravel() - x_star
        errs.append(np.real(np.vdot(e, Ad @ e)))
        return rn < 1e-12

    W.cg(A, rhs, None, 0.0, 500, check)
    assert len(errs) > 5
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) + 1e-28 for i in range(len(errs) - 1))


def test_bicgstab_zero_source_breaks_down():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.3, 3)
    with pytest.raises(W.Breakdown):
        W.bicgstab(lambda v: W.schur(U, v, 0.1), np.zeros(S.lattice_shape(dims) + (4, 3), complex), None, 1e-10, 10)
