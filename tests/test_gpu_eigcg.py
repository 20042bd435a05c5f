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


def test_eigcg_matches_oracle_and_deflates():
    """A smooth field near the critical kappa (isolated low modes): incremental
    EigCG accumulates nev vectors per solve and the later solves need fewer
    iterations; every iteration count follows the oracle's."""
    dims = (16, 4, 4, 4)
    kappa = 0.1255
    U = S.gauge_field(dims, 0.05, 91)
    A = lambda v: W.schur_dag(U, W.schur(U, v, kappa), kappa)
    inc = E.IncrementalEigCG(A, nev=8, m=24, n_accumulate=6, tol=1e-10)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        eig = EigCG(ctx, nev=8, m=24, max_vectors=48)
        its, its_oracle, vecs = [], [], []
        for k in range(8):
            b = S.gaussian_spinor(dims, 300 + k)
            bd = ctx.to_device(b, F64)
            x = ctx.empty_full(F64)
            info = eig.solve(x, bd, kappa, tol=1e-10, accumulate=k < 6)
            xs = ctx.to_host(x, F64)
            res = np.linalg.norm(b - C.wilson(U, xs, kappa)) / np.linalg.norm(b)
            assert res < 1e-7, (k, res)
            assert abs(info.true_rel_residual - res) < 1e-10
            its.append(info.iterations)
            vecs.append(eig.vectors)
            rhs = W.schur_dag(U, W.schur_rhs(U, b, kappa), kappa)
            _, it_o = inc.solve(rhs)
            its_oracle.append(it_o)
        eig.close()
    assert vecs[0] == 8 and vecs[5] == 48 and vecs[7] == 48
    assert its[-1] <= 0.8 * its[0], its
    for g, o in zip(its, its_oracle):
        assert abs(g - o) <= 3, (its, its_oracle)


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
