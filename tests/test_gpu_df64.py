"""PLQ_DF64: FP64 storage in float-float (hi + lo) form, float-float arithmetic.

The operator is checked against the FP64 oracle at the FP64 tolerance; the
solvers that use it for their reliable-update residuals against the oracle's
true residual of the returned x."""
import numpy as np
import pytest

import synthetic as S
from oracle import c_oracle as C
from oracle import wilson as W

from gpuhelp import TOL, gpu_hopping_full, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1405_0700_gb300 import DF64, F16, F32, F64, Context, PLQError  # noqa: E402
from paper_1405_0700_gb300 import plq  # noqa: E402


def test_pack_unpack_keeps_48_bits():
    dims = (4, 4, 2, 6)
    phi = S.gaussian_spinor(dims, 3)
    phi[0, 0, 0, 0] *= 1e-20  # small entries keep their relative precision too
    with Context(dims) as ctx:
        back = ctx.to_host(ctx.to_device(phi, DF64), DF64)
    for part in (np.real, np.imag):  # each real keeps 48 bits: |error| <= 2^-49 |value| (2^-47 allowed)
        assert np.all(np.abs(part(back) - part(phi)) <= 2.0 ** -47 * np.abs(part(phi)))
    assert rel(back, phi) < 1e-14


@pytest.mark.parametrize("dims,t_bc", [((8, 4, 4, 4), -1), ((6, 4, 2, 8), -1), ((4, 6, 4, 2), 1), ((2, 2, 2, 2), -1)])
def test_hopping_matches_oracle(dims, t_bc):
    U, phi = S.gauge_and_spinor(dims, 0.3, 11)
    with Context(dims, t_bc=t_bc) as ctx:
        ctx.gauge_upload(U, 18, DF64)
        got = gpu_hopping_full(ctx, phi, DF64)
    ref = W.hopping(U, phi, t_bc=t_bc)
    err = rel(got, ref)
    assert err <= TOL[DF64], err
    # the float-float result is far more accurate than FP32 arithmetic could be
    assert err < 1e-13


def test_hopping_agrees_with_fp64_kernel():
    dims = (8, 8, 4, 4)
    U, phi = S.gauge_and_spinor(dims, 0.3, 12)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, DF64)
        ctx.gauge_upload(U, 18, F64)
        a = gpu_hopping_full(ctx, phi, DF64)
        b = gpu_hopping_full(ctx, phi, F64)
    assert rel(a, b) < 1e-13


@pytest.mark.parametrize("nrhs", [2, 5, 12])
def test_multi_rhs(nrhs):
    dims = (6, 4, 2, 4)
    U = S.gauge_field(dims, 0.3, 6)
    phis = np.stack([S.gaussian_spinor(dims, 100 + r) for r in range(nrhs)])
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, DF64)
        got = gpu_hopping_full(ctx, phis, DF64, nrhs).reshape(phis.shape)
    for r in range(nrhs):
        assert rel(got[r], W.hopping(U, phis[r])) <= TOL[DF64], r


def test_full_size_32c64_sampled_sites():
    dims = (64, 32, 32, 32)
    U, phi = S.gauge_and_spinor(dims, 0.2, 2)
    V = S.volume(dims)
    rng = np.random.default_rng(0)
    sites = np.concatenate([[0, 1, V - 1, V // 2], rng.integers(0, V, 2000)])
    ref = C.hopping_sites(U, phi, sites)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, DF64)
        got = gpu_hopping_full(ctx, phi, DF64).reshape(V, 4, 3)[sites]
    assert rel(got, ref) <= TOL[DF64]


def test_argument_errors():
    dims = (4, 4, 4, 4)
    U, phi = S.gauge_and_spinor(dims, 0.3, 1)
    with Context(dims) as ctx:
        with pytest.raises(PLQError):
            ctx.gauge_upload(U, 12, DF64)  # float-float links are stored with 18 reals
        inp = ctx.to_device(phi, DF64)
        e_in, o_in = ctx.halves(inp, DF64)
        out = ctx.empty_half(DF64)
        with pytest.raises(PLQError) as ei:
            ctx.hopping_eo(0, out, o_in, DF64)  # no float-float gauge copy yet
        assert ei.value.status == plq.PLQ_ERR_STATE
        ctx.gauge_upload(U, 18, DF64)
        full = ctx.empty_full(DF64)
        with pytest.raises(PLQError) as ei:
            ctx.wilson_apply(full, inp, 0.1, DF64)  # only the hopping operator takes PLQ_DF64
        assert ei.value.status == plq.PLQ_ERR_ARG
        # residual_prec = DF64 without the float-float gauge copy is refused before any work
        ctx2 = Context(dims)
        try:
            ctx2.gauge_upload(U, 18, F64)
            ctx2.gauge_upload(U, 12, F32)
            b = ctx2.to_device(phi, F64)
            x = ctx2.empty_full(F64)
            with pytest.raises(PLQError) as ei:
                ctx2.cg_solve(x, b, 0.12, inner_prec=F32, residual_prec=DF64)
            assert ei.value.status == plq.PLQ_ERR_STATE
            with pytest.raises(PLQError) as ei:
                ctx2.cg_solve(x, b, 0.12, inner_prec=F32, residual_prec=F16)
            assert ei.value.status == plq.PLQ_ERR_ARG
        finally:
            ctx2.close()


def solve(method, dims, eps, seed, kappa, inner, residual_prec, mu=0.0, nrhs=1, sources=None):
    U, b = S.gauge_and_spinor(dims, eps, seed)
    if sources is not None:
        b = np.stack(sources)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        ctx.gauge_upload(U, 12, inner)
        ctx.gauge_upload(U, 18, DF64)
        bd = ctx.to_device(b, F64, nrhs)
        x = ctx.empty_full(F64, nrhs)
        if nrhs == 1:
            fn = ctx.cg_solve if method == "cg" else ctx.bicgstab_solve
            info = fn(x, bd, kappa, inner_prec=inner, residual_prec=residual_prec, mu=mu)
        else:
            fn = ctx.cg_solve_multi if method == "cg" else ctx.bicgstab_solve_multi
            info = fn(x, bd, kappa, nrhs, inner_prec=inner, residual_prec=residual_prec)
        xs = ctx.to_host(x, F64, nrhs)
    return U, b, xs, info


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
@pytest.mark.parametrize("inner", [F32, F16])
def test_solvers_with_float_float_residuals(method, inner):
    kappa = 0.12
    U, b, x, info = solve(method, (8, 8, 8, 8), 0.3, 1, kappa, inner, DF64)
    res = float(np.linalg.norm(b - C.wilson(U, x, kappa)) / np.linalg.norm(b))
    assert res <= 1e-10, (res, info.as_dict())
    assert abs(info.true_rel_residual - res) < 1e-11
    assert info.n_reliable >= 2
    # the same solve with FP64 residuals reaches the same solution
    _, _, x64, info64 = solve(method, (8, 8, 8, 8), 0.3, 1, kappa, inner, F64)
    assert rel(x, x64) < 1e-8
    assert abs(info.iterations - info64.iterations) <= max(3, info64.iterations // 10)


def test_twisted_cg_with_float_float_residuals():
    kappa, mu = 0.125, 0.05
    U, b, x, info = solve("cg", (8, 4, 4, 8), 0.3, 2, kappa, F32, DF64, mu=mu)
    res = float(np.linalg.norm(b - W.twisted(U, x, kappa, mu)) / np.linalg.norm(b))
    assert res <= 1e-10, (res, info.as_dict())


def test_multi_rhs_point_sources_with_float_float_residuals():
    dims = (16, 8, 8, 8)
    kappa = 0.121
    srcs = [S.point_source(dims, s, c) for s in range(4) for c in range(3)]
    U, b, x, infos = solve("cg", dims, 0.25, 4, kappa, F32, DF64, nrhs=12, sources=srcs)
    x = x.reshape((12,) + b.shape[1:])
    for r in range(12):
        res = float(np.linalg.norm(b[r] - C.wilson(U, x[r], kappa)) / np.linalg.norm(b[r]))
        assert res <= 1e-10, (r, res, infos[r].as_dict())


@pytest.mark.parametrize("scale", [1e-45, 1e-30, 1e30])
@pytest.mark.parametrize("residual_prec", [F64, DF64])
@pytest.mark.parametrize("method", ["cg", "bicgstab"])
def test_mixed_solves_for_any_source_magnitude(scale, residual_prec, method):
    """The inner (FP32) iteration and the float-float fields see each right-hand
    side scaled by a power of two, so sources far outside the FP32 exponent range
    solve as well as O(1) ones."""
    dims = (8, 4, 4, 8)
    kappa = 0.12
    U, b = S.gauge_and_spinor(dims, 0.3, 8)
    b = b * scale
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        ctx.gauge_upload(U, 12, F32)
        ctx.gauge_upload(U, 18, DF64)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        fn = ctx.cg_solve if method == "cg" else ctx.bicgstab_solve
        info = fn(x, bd, kappa, inner_prec=F32, residual_prec=residual_prec)
        xs = ctx.to_host(x, F64)
    res = float(np.linalg.norm(b - C.wilson(U, xs, kappa)) / np.linalg.norm(b))
    assert res <= 1e-10, (scale, res, info.as_dict())
    assert abs(info.true_rel_residual - res) < 1e-11
