"""Twisted-mass operator and solvers on the GPU against the oracle."""
import numpy as np
import pytest

import synthetic as S
from oracle import wilson as W
from gpuhelp import TOL, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1405_0700_gb300 import F16, F32, F64, Context  # noqa: E402


@pytest.mark.parametrize("prec", [F64, F32, F16])
def test_twisted_apply(prec):
    dims = (10, 4, 6, 8)
    U, phi = S.gauge_and_spinor(dims, 0.3, 3)
    kappa, mu = 0.12, 0.05
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18 if prec != F16 else 12, prec)
        inp = ctx.to_device(phi, prec)
        out = ctx.empty_full(prec)
        ctx.twisted_apply(out, inp, kappa, mu, prec)
        got = ctx.to_host(out, prec)
    assert rel(got, W.twisted(U, phi, kappa, mu)) <= TOL[prec]


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
@pytest.mark.parametrize("inner", [F64, F32])
def test_twisted_solve(method, inner):
    dims = (8, 8, 8, 8)
    U, b = S.gauge_and_spinor(dims, 0.3, 4)
    kappa, mu = 0.124, 0.01
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        if inner != F64:
            ctx.gauge_upload(U, 12, inner)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        fn = ctx.cg_solve if method == "cg" else ctx.bicgstab_solve
        info = fn(x, bd, kappa, inner_prec=inner, mu=mu)
        xs = ctx.to_host(x, F64)
    res = np.linalg.norm(b - W.twisted(U, xs, kappa, mu)) / np.linalg.norm(b)
    assert res <= 1e-10, (res, info.as_dict())
    assert abs(info.true_rel_residual - res) < 1e-11
