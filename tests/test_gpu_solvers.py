"""GPU solvers: the true FP64 residual of each returned x, computed by the oracle."""
import numpy as np
import pytest

import synthetic as S
from oracle import c_oracle as C
from oracle import wilson as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1405_0700_gb300 import F16, F32, F64, Context, PLQError  # noqa: E402
from paper_1405_0700_gb300 import plq  # noqa: E402


def oracle_residual(U, b, x, kappa):
    return float(np.linalg.norm(b - C.wilson(U, x, kappa)) / np.linalg.norm(b))


def run(method, dims, eps, seed, kappa, inner, tol=1e-10, **kw):
    U, b = S.gauge_and_spinor(dims, eps, seed)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        if inner != F64:
            ctx.gauge_upload(U, 12, inner)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        fn = ctx.cg_solve if method == "cg" else ctx.bicgstab_solve
        info = fn(x, bd, kappa, tol=tol, inner_prec=inner, **kw)
        xs = ctx.to_host(x, F64)
    return U, b, xs, info


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
@pytest.mark.parametrize("inner", [F64, F32, F16])
def test_solve_8c8_reaches_true_residual(method, inner):
    U, b, x, info = run(method, (8, 8, 8, 8), 0.3, 1, 0.12, inner)
    res = oracle_residual(U, b, x, 0.12)
    assert res <= 1e-10, (res, info.as_dict())
    assert abs(info.true_rel_residual - res) < 1e-11
    if inner != F64:
        assert info.n_reliable >= 2


def test_cg_matches_dense_solution():
    dims = (4, 4, 4, 4)
    U, b = S.gauge_and_spinor(dims, 0.3, 1)
    kappa = 0.12
    shape = b.shape
    M = W.dense(lambda v: W.wilson(U, v, kappa), shape)
    x_ref = np.linalg.solve(M, b.ravel()).reshape(shape)
    for method in ("cg", "bicgstab"):
        _, _, x, _ = run(method, dims, 0.3, 1, kappa, F32)
        assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-8


def test_cg_and_bicgstab_agree_anisotropic():
    dims = (10, 4, 6, 8)
    _, _, x1, _ = run("cg", dims, 0.3, 3, 0.115, F32)
    _, _, x2, _ = run("bicgstab", dims, 0.3, 3, 0.115, F32)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-8


def test_resume_from_x0():
    dims = (8, 4, 4, 4)
    U, b = S.gauge_and_spinor(dims, 0.3, 4)
    kappa = 0.12
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        info1 = ctx.cg_solve(x, bd, kappa, tol=1e-5)
        info2 = ctx.cg_solve(x, bd, kappa, tol=1e-10, use_x0=True)
        xs = ctx.to_host(x, F64)
    assert oracle_residual(U, b, xs, kappa) <= 1e-10
    fresh = run("cg", dims, 0.3, 4, kappa, F64)[3]
    assert info2.iterations < fresh.iterations


def test_checkpoint_and_resume_in_a_new_context(tmp_path):
    """A solve stopped by its iteration cap writes x to a .npy checkpoint; a new context
    loads it (bit for bit) and resumes from it with use_x0 to the true residual 1e-10."""
    dims = (8, 4, 4, 4)
    U, b = S.gauge_and_spinor(dims, 0.3, 4)
    kappa = 0.12
    path = str(tmp_path / "x.npy")
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        info1 = ctx.cg_solve(x, bd, kappa, tol=1e-10, maxit=10, raise_on_error=False)
        assert info1.status == plq.PLQ_ERR_NOT_CONVERGED
        ctx.save_field(path, x, F64)
        saved = ctx.to_host(x, F64)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        bd = ctx.to_device(b, F64)
        x = ctx.load_field(path, F64)
        assert np.array_equal(ctx.to_host(x, F64), saved)
        ctx.cg_solve(x, bd, kappa, tol=1e-10, use_x0=True)
        xs = ctx.to_host(x, F64)
    assert oracle_residual(U, b, xs, kappa) <= 1e-10


def test_maxit_returns_not_converged():
    with pytest.raises(PLQError) as e:
        run("cg", (8, 4, 4, 4), 0.3, 5, 0.12, F64, maxit=5)
    assert e.value.status == plq.PLQ_ERR_NOT_CONVERGED
    assert e.value.info.iterations <= 5 + 16


def test_nan_source_returns_nan_status():
    dims = (4, 4, 4, 4)
    U, b = S.gauge_and_spinor(dims, 0.3, 6)
    b[1, 2, 3, 0, 1, 2] = np.nan
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        with pytest.raises(PLQError) as e:
            ctx.cg_solve(x, bd, 0.12)
        assert e.value.status == plq.PLQ_ERR_NAN


def test_zero_source():
    dims = (4, 4, 4, 4)
    U = S.gauge_field(dims, 0.3, 7)
    b = np.zeros(S.lattice_shape(dims) + (4, 3), complex)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        info = ctx.cg_solve(x, bd, 0.12)
        assert info.status == plq.PLQ_OK and info.iterations == 0
        assert not torch.any(x.view(torch.float64) != 0)
        with pytest.raises(PLQError) as e:
            ctx.bicgstab_solve(x, bd, 0.12)
        assert e.value.status == plq.PLQ_ERR_BREAKDOWN


def test_missing_inner_gauge_copy():
    dims = (4, 4, 4, 4)
    U, b = S.gauge_and_spinor(dims, 0.3, 8)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        with pytest.raises(PLQError) as e:
            ctx.cg_solve(x, bd, 0.12, inner_prec=F16)
        assert e.value.status == plq.PLQ_ERR_STATE


def run_multi(method, dims, eps, seed, kappa, inner, sources, tile=1, sm=0, **kw):
    U = S.gauge_field(dims, eps, seed)
    n = len(sources)
    b = np.stack(sources)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        if inner != F64:
            ctx.gauge_upload(U, 12, inner)
            ctx.set_launch(inner, n, 0, 0, tile, 0, sm)
        bd = ctx.to_device(b, F64, n)
        x = ctx.empty_full(F64, n)
        fn = ctx.cg_solve_multi if method == "cg" else ctx.bicgstab_solve_multi
        infos = fn(x, bd, kappa, n, inner_prec=inner, **kw)
        xs = ctx.to_host(x, F64, n).reshape((n,) + b.shape[1:])
    return U, b, xs, infos


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
@pytest.mark.parametrize("inner", [F64, F32, F16])
def test_multi_rhs_point_sources(method, inner):
    """The 12 spin x colour columns of a point-source propagator, solved together
    (on a 8^3 x 16 lattice; the 48^3 x 96 version is the propagator benchmark)."""
    # the spin x colour columns of a point-source propagator, solved together
    dims = (16, 8, 8, 8)
    kappa = 0.121
    srcs = [S.point_source(dims, s, c) for s in range(4) for c in range(3)]
    U, b, x, infos = run_multi(method, dims, 0.25, 4, kappa, inner, srcs)
    for r in range(12):
        res = oracle_residual(U, b[r], x[r], kappa)
        assert res <= 1e-10, (r, res, infos[r].as_dict())
        assert abs(infos[r].true_rel_residual - res) < 1e-11


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
def test_fp16_inner_point_source_long_lattice(method):
    """A point source on a 192 x 2^3 lattice: the support of the early Krylov vectors
    grows along t with values falling by ~2 kappa per site, so before it wraps around
    its edge passes through FP32's subnormal range; the FP16 inner iterations must store
    those sites (as zero) without producing infinities or NaNs."""
    dims = (192, 2, 2, 2)
    kappa = 0.115
    srcs = [S.point_source(dims, 0, c) for c in range(3)]
    U, b, x, infos = run_multi(method, dims, 0.25, 22, kappa, F16, srcs)
    for r in range(3):
        res = oracle_residual(U, b[r], x[r], kappa)
        assert res <= 1e-10, (r, res, infos[r].as_dict())


@pytest.mark.parametrize("tile,sm", [(2, 0), (4, 0), (1, 1), (2, 1), (1, 2), (1, 3), (1, 4)])
def test_multi_rhs_cg_with_rhs_tiles(tile, sm):
    dims = (8, 4, 4, 8)
    kappa = 0.12
    srcs = [S.point_source(dims, s, c) for s in range(4) for c in range(3)]
    U, b, x, infos = run_multi("cg", dims, 0.3, 9, kappa, F32, srcs, tile=tile, sm=sm)
    for r in range(12):
        assert oracle_residual(U, b[r], x[r], kappa) <= 1e-10


def test_multi_rhs_matches_single_solves():
    dims = (8, 4, 4, 4)
    kappa = 0.12
    srcs = [S.gaussian_spinor(dims, 40 + r) for r in range(3)]
    U, b, x, infos = run_multi("cg", dims, 0.3, 7, kappa, F32, srcs)
    for r in range(3):
        assert oracle_residual(U, b[r], x[r], kappa) <= 1e-10
    # each right-hand side's solution is the single solve of that source
    U1 = S.gauge_field(dims, 0.3, 7)
    with Context(dims) as ctx:
        ctx.gauge_upload(U1, 18, F64)
        ctx.gauge_upload(U1, 12, F32)
        for r in range(3):
            bd = ctx.to_device(srcs[r], F64)
            xd = ctx.empty_full(F64)
            ctx.cg_solve(xd, bd, kappa, inner_prec=F32)
            x1 = ctx.to_host(xd, F64)
            assert np.linalg.norm(x1 - x[r]) / np.linalg.norm(x1) < 1e-8


def test_multi_rhs_zero_and_nonzero_sources():
    dims = (8, 4, 4, 4)
    kappa = 0.12
    srcs = [S.gaussian_spinor(dims, 50), np.zeros(S.lattice_shape(dims) + (4, 3), complex),
            S.gaussian_spinor(dims, 51)]
    U, b, x, infos = run_multi("cg", dims, 0.3, 8, kappa, F32, srcs)
    assert np.all(x[1] == 0) and infos[1].iterations == 0
    for r in (0, 2):
        assert oracle_residual(U, b[r], x[r], kappa) <= 1e-10


def test_batched_uneven_systems_one_launch():
    """Several lattices, kappas and seeds solved by one persistent launch; each
    solution checked with the oracle's operator."""
    from paper_1405_0700_gb300 import plq as P

    specs = S.batch_solve_specs(n=5, sizes=((8, 4, 4, 4), (16, 8, 8, 8), (10, 4, 6, 8)))
    ctxs, xs, bs, Us, srcs = [], [], [], [], []
    for sp in specs:
        U, b = S.gauge_and_spinor(sp["dims"], sp["eps"], sp["seed"])
        ctx = Context(sp["dims"])
        ctx.gauge_upload(U, 18, F64)
        ctx.gauge_upload(U, 12, F32)
        ctxs.append(ctx)
        bs.append(ctx.to_device(b, F64))
        xs.append(ctx.empty_full(F64))
        Us.append(U)
        srcs.append(b)
    infos, binfo = P.cg_solve_batched(ctxs, xs, bs, [sp["kappa"] for sp in specs], inner_prec=F32)
    assert binfo["launches"] == 1
    for k, sp in enumerate(specs):
        x = ctxs[k].to_host(xs[k], F64)
        res = oracle_residual(Us[k], srcs[k], x, sp["kappa"])
        assert res <= 1e-10, (k, res, infos[k].as_dict())
        assert abs(infos[k].true_rel_residual - res) < 1e-11
    # uneven iteration counts: the systems really were independent
    assert len({i.iterations for i in infos}) > 1
    for c in ctxs:
        c.close()


def test_batched_sources_of_any_magnitude():
    """Systems whose sources lie far outside the FP32 exponent range, in one
    persistent launch with an FP32 inner iteration (each system's inner
    quantities are scaled by a power of two)."""
    from paper_1405_0700_gb300 import plq as P

    dims = (8, 4, 4, 4)
    ctxs, xs, bs, Us, srcs = [], [], [], [], []
    for k, scale in enumerate((1e-45, 1.0, 1e30)):
        U, b = S.gauge_and_spinor(dims, 0.3, 70 + k)
        b = b * scale
        ctx = Context(dims)
        ctx.gauge_upload(U, 18, F64)
        ctx.gauge_upload(U, 12, F32)
        ctxs.append(ctx)
        bs.append(ctx.to_device(b, F64))
        xs.append(ctx.empty_full(F64))
        Us.append(U)
        srcs.append(b)
    infos, _ = P.cg_solve_batched(ctxs, xs, bs, [0.12] * 3, inner_prec=F32)
    for k in range(3):
        res = oracle_residual(Us[k], srcs[k], ctxs[k].to_host(xs[k], F64), 0.12)
        assert res <= 1e-10, (k, res, infos[k].as_dict())
    for c in ctxs:
        c.close()


def test_batched_resume_from_a_given_x():
    """use_x0 in the persistent launch: the first residual check then applies the
    operator to the given x_e (not the x_e = 0 shortcut), and the final x_o comes
    from the H_oe x_e of the last check.  Resuming from a converged x returns it
    after one check and no iteration; resuming from a perturbed x converges again.
    Each x is checked with the oracle's operator."""
    from paper_1405_0700_gb300 import plq as P

    specs = S.batch_solve_specs(n=3, sizes=((8, 4, 4, 4), (16, 8, 8, 8)))
    ctxs, xs, bs, Us, srcs = [], [], [], [], []
    for sp in specs:
        U, b = S.gauge_and_spinor(sp["dims"], sp["eps"], sp["seed"])
        ctx = Context(sp["dims"])
        ctx.gauge_upload(U, 18, F64)
        ctx.gauge_upload(U, 12, F32)
        ctxs.append(ctx)
        bs.append(ctx.to_device(b, F64))
        xs.append(ctx.empty_full(F64))
        Us.append(U)
        srcs.append(b)
    kappas = [sp["kappa"] for sp in specs]
    P.cg_solve_batched(ctxs, xs, bs, kappas, inner_prec=F32)
    infos, _ = P.cg_solve_batched(ctxs, xs, bs, kappas, inner_prec=F32, use_x0=True)
    for k in range(len(specs)):
        assert infos[k].iterations == 0, infos[k].as_dict()
        res = oracle_residual(Us[k], srcs[k], ctxs[k].to_host(xs[k], F64), kappas[k])
        assert res <= 1e-10, (k, res)
        assert abs(infos[k].true_rel_residual - res) < 1e-11
    # perturb every x (both parities) and resume
    for k, sp in enumerate(specs):
        noise = S.gaussian_spinor(sp["dims"], 900 + k) * 1e-3
        xs[k] = ctxs[k].to_device(ctxs[k].to_host(xs[k], F64) + noise, F64)
    infos, _ = P.cg_solve_batched(ctxs, xs, bs, kappas, inner_prec=F32, use_x0=True)
    for k in range(len(specs)):
        assert infos[k].iterations > 0
        res = oracle_residual(Us[k], srcs[k], ctxs[k].to_host(xs[k], F64), kappas[k])
        assert res <= 1e-10, (k, res, infos[k].as_dict())
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("inner", [F64, F16])
def test_batched_inner_precisions(inner):
    from paper_1405_0700_gb300 import plq as P

    dims = (8, 4, 4, 4)
    U, b = S.gauge_and_spinor(dims, 0.3, 61)
    ctx = Context(dims)
    ctx.gauge_upload(U, 18, F64)
    if inner == F16:
        ctx.gauge_upload(U, 12, F16)
    bd = ctx.to_device(b, F64)
    x = ctx.empty_full(F64)
    infos, binfo = P.cg_solve_batched([ctx], [x], [bd], [0.12], inner_prec=inner)
    assert oracle_residual(U, b, ctx.to_host(x, F64), 0.12) <= 1e-10
    ctx.close()


def test_batched_zero_source_and_maxit():
    from paper_1405_0700_gb300 import plq as P

    dims = (8, 4, 4, 4)
    U, b = S.gauge_and_spinor(dims, 0.3, 62)
    ctx = Context(dims)
    ctx.gauge_upload(U, 18, F64)
    ctx.gauge_upload(U, 12, F32)
    zero = ctx.to_device(np.zeros_like(b), F64)
    x = ctx.empty_full(F64)
    infos, _ = P.cg_solve_batched([ctx], [x], [zero], [0.12], inner_prec=F32)
    assert not torch.any(x.view(torch.float64) != 0)
    bd = ctx.to_device(b, F64)
    with pytest.raises(PLQError) as e:
        P.cg_solve_batched([ctx], [x], [bd], [0.12], inner_prec=F32, maxit=3)
    assert e.value.status == plq.PLQ_ERR_NOT_CONVERGED
    ctx.close()


def test_batched_barrier_wait_limit_reports_timeout():
    """A grid-barrier wait limit of one clock cycle: the first block to wait at a
    barrier gives up, every block leaves the persistent kernel (the others see the
    status word at their next barrier), the call returns PLQ_ERR_TIMEOUT, and the
    same contexts then solve normally."""
    from paper_1405_0700_gb300 import plq as P

    dims = (8, 4, 4, 8)
    U, b = S.gauge_and_spinor(dims, 0.3, 63)
    ctx = Context(dims)
    ctx.gauge_upload(U, 18, F64)
    ctx.gauge_upload(U, 12, F32)
    bd = ctx.to_device(b, F64)
    x = ctx.empty_full(F64)
    with pytest.raises(PLQError) as e:
        P.cg_solve_batched([ctx], [x], [bd], [0.12], inner_prec=F32, wait_limit_s=1e-12)
    assert e.value.status == plq.PLQ_ERR_TIMEOUT
    torch.cuda.synchronize()
    infos, binfo = P.cg_solve_batched([ctx], [x], [bd], [0.12], inner_prec=F32)
    assert binfo["launches"] == 1
    assert oracle_residual(U, b, ctx.to_host(x, F64), 0.12) <= 1e-10
    ctx.close()


def test_solver_graph_follows_gauge_and_launch_changes():
    """The instantiated inner-iteration graph is reused between solves; a new gauge
    field, another link format (a reallocated copy), another kappa or another launch
    configuration must each give the correct solution of the new system."""
    dims = (8, 4, 4, 8)
    U1, b = S.gauge_and_spinor(dims, 0.3, 81)
    U2 = S.gauge_field(dims, 0.3, 82)
    with Context(dims) as ctx:
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        steps = [(U1, 12, 0.12, None), (U1, 12, 0.12, None), (U2, 12, 0.12, None), (U2, 18, 0.12, None),
                 (U2, 18, 0.115, None), (U2, 18, 0.115, 64)]
        for U, reals, kappa, block in steps:
            ctx.gauge_upload(U, 18, F64)
            ctx.gauge_upload(U, reals, F32)
            if block:
                ctx.set_launch(F32, 1, block, 0, 1, 0, 0)
            ctx.cg_solve(x, bd, kappa, inner_prec=F32)
            res = oracle_residual(U, b, ctx.to_host(x, F64), kappa)
            assert res <= 1e-10, (reals, kappa, block, res)


@pytest.mark.parametrize("method,inner,tile,sm", [("cg", F32, 1, 0), ("cg", F16, 1, 1), ("cg", F32, 2, 0),
                                                  ("bicgstab", F32, 1, 0), ("cg", F64, 1, 0)])
def test_solves_are_bitwise_reproducible(method, inner, tile, sm):
    """Every reduction of the solvers (fused operator epilogues and vector kernels) adds
    FP64 partial sums in a fixed order, so two identical multi-right-hand-side solves in
    the same launch configuration return bit-identical iteration counts, residuals and
    solutions; the residuals also pass the oracle's check."""
    dims = (16, 8, 8, 8)
    kappa = 0.12
    n = 6
    U = S.gauge_field(dims, 0.3, 13)
    srcs = np.stack([S.gaussian_spinor(dims, 60 + r) for r in range(n)])
    runs = []
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        if inner != F64:
            ctx.gauge_upload(U, 12, inner)
            ctx.set_launch(inner, n, 0, 0, 1 if n % tile else tile, 0, sm)
        bd = ctx.to_device(srcs, F64, n)
        fn = ctx.cg_solve_multi if method == "cg" else ctx.bicgstab_solve_multi
        for _ in range(2):
            x = ctx.empty_full(F64, n)
            x.zero_()
            infos = fn(x, bd, kappa, n, inner_prec=inner)
            runs.append((ctx.to_host(x, F64, n), [(i.iterations, i.n_reliable, i.true_rel_residual) for i in infos]))
    (x0, i0), (x1, i1) = runs
    assert i0 == i1
    assert np.array_equal(x0.view(np.float64), x1.view(np.float64))
    xs = x0.reshape((n,) + srcs.shape[1:])
    for r in range(n):
        assert oracle_residual(U, srcs[r], xs[r], kappa) <= 1e-10


def _batch(n=4, seed_shift=0):
    specs = S.batch_solve_specs(n=n, sizes=((8, 4, 4, 4), (16, 8, 8, 8), (10, 4, 6, 8)))
    ctxs, xs, bs, Us, srcs = [], [], [], [], []
    for sp in specs:
        U = S.gauge_field(sp["dims"], sp["eps"], sp["seed"])
        ctx = Context(sp["dims"])
        ctx.gauge_upload(U, 18, F64)
        ctx.gauge_upload(U, 12, F32)
        ctxs.append(ctx)
        xs.append(ctx.empty_full(F64))
        Us.append(U)
    return specs, ctxs, xs, Us


def _check_batch(specs, ctxs, xs, Us, srcs, infos):
    for k, sp in enumerate(specs):
        x = ctxs[k].to_host(xs[k], F64)
        res = oracle_residual(Us[k], srcs[k], x, sp["kappa"])
        assert res <= 1e-10, (k, res, infos[k].as_dict())


def test_batched_graph_is_reused_for_new_sources():
    """The second persistent launch with the same first context and shape replays the
    instantiated graph: with the same sources it returns bit-identical solutions, with
    new sources and kappas it solves the new systems (the descriptors are rewritten
    before every launch)."""
    from paper_1405_0700_gb300 import plq as P

    specs, ctxs, xs, Us = _batch()
    kappas = [sp["kappa"] for sp in specs]
    srcs = [S.gaussian_spinor(sp["dims"], 700 + k) for k, sp in enumerate(specs)]
    bs = [c.to_device(b, F64) for c, b in zip(ctxs, srcs)]
    infos, b1 = P.cg_solve_batched(ctxs, xs, bs, kappas, inner_prec=F32)
    first = [c.to_host(x, F64) for c, x in zip(ctxs, xs)]
    _check_batch(specs, ctxs, xs, Us, srcs, infos)
    infos2, b2 = P.cg_solve_batched(ctxs, xs, bs, kappas, inner_prec=F32)
    assert b1["graph_captured"] == 1 and b2["graph_reused"] == 1 and b1["grid"] == b2["grid"]
    for c, x, f in zip(ctxs, xs, first):
        assert np.array_equal(c.to_host(x, F64), f)
    assert [i.iterations for i in infos2] == [i.iterations for i in infos]
    srcs3 = [S.gaussian_spinor(sp["dims"], 800 + k) for k, sp in enumerate(specs)]
    bs3 = [c.to_device(b, F64) for c, b in zip(ctxs, srcs3)]
    kappas3 = [k * 0.98 for k in kappas]
    specs3 = [dict(sp, kappa=k) for sp, k in zip(specs, kappas3)]
    infos3, b3 = P.cg_solve_batched(ctxs, xs, bs3, kappas3, inner_prec=F32)
    assert b3["graph_reused"] == 1
    _check_batch(specs3, ctxs, xs, Us, srcs3, infos3)
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("block,bps", [(64, 0), (128, 2), (192, 0), (256, 1)])
def test_batched_launch_shapes(block, bps):
    """Every launch shape of the persistent kernel (threads per block and resident blocks
    per SM) solves the batch; the report names the shape used."""
    from paper_1405_0700_gb300 import plq as P

    specs, ctxs, xs, Us = _batch()
    srcs = [S.gaussian_spinor(sp["dims"], 900 + k) for k, sp in enumerate(specs)]
    bs = [c.to_device(b, F64) for c, b in zip(ctxs, srcs)]
    P.set_batched_launch(ctxs[0], block, bps)
    infos, bi = P.cg_solve_batched(ctxs, xs, bs, [sp["kappa"] for sp in specs], inner_prec=F32)
    assert bi["block"] == block and (bps == 0 or bi["blocks_per_sm"] == bps)
    _check_batch(specs, ctxs, xs, Us, srcs, infos)
    with pytest.raises(PLQError):
        P.set_batched_launch(ctxs[0], 100, 0)
    for c in ctxs:
        c.close()


def test_batched_autotune_and_cache(tmp_path):
    """The launch-shape tuner times the shapes on the batch, keeps the fastest in the
    first context and writes it to the cache file, which a second tuning call reads
    back without timing; solves with the chosen shape stay correct."""
    from paper_1405_0700_gb300 import plq as P

    specs, ctxs, xs, Us = _batch()
    kappas = [sp["kappa"] for sp in specs]
    srcs = [S.gaussian_spinor(sp["dims"], 1000 + k) for k, sp in enumerate(specs)]
    bs = [c.to_device(b, F64) for c, b in zip(ctxs, srcs)]
    path = str(tmp_path / "tune.txt")
    best = P.autotune_batched(ctxs, xs, bs, kappas, inner_prec=F32, cache_path=path)
    assert best["block"] in (64, 128, 192, 256) and best["seconds"] > 0
    line = open(path).read().strip().split()
    assert len(line) == 4 and int(line[1]) == best["block"]
    again = P.autotune_batched(ctxs, xs, bs, kappas, inner_prec=F32, cache_path=path)
    assert again["block"] == best["block"] and again["grid"] == 0  # from the cache: nothing ran
    infos, bi = P.cg_solve_batched(ctxs, xs, bs, kappas, inner_prec=F32)
    assert bi["block"] == best["block"]
    _check_batch(specs, ctxs, xs, Us, srcs, infos)
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("sm", [0, 1, 4])
@pytest.mark.parametrize("n", [12, 5])
def test_multi_rhs_identical_sources_iterate_alike(sm, n):
    """n copies of one source solved together must each take the iterations of the single
    solve: every right-hand side's reductions (operator epilogues and vector kernels, whose
    blocks for n = 12 or 5 end in a partial warp) must see all of its elements."""
    dims = (16, 8, 8, 8)
    kappa = 0.12
    U, b = S.gauge_and_spinor(dims, 0.3, 21)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        ctx.gauge_upload(U, 12, F32)
        bd1 = ctx.to_device(b, F64)
        x1 = ctx.empty_full(F64)
        single = ctx.cg_solve(x1, bd1, kappa, inner_prec=F32)
        ctx.set_launch(F32, n, 0, 0, 1, 0, sm)
        bd = ctx.to_device(np.stack([b] * n), F64, n)
        x = ctx.empty_full(F64, n)
        infos = ctx.cg_solve_multi(x, bd, kappa, n, inner_prec=F32)
        xs = ctx.to_host(x, F64, n).reshape((n,) + b.shape)
    its = [i.iterations for i in infos]
    assert max(its) - min(its) <= 1 and abs(its[0] - single.iterations) <= 1, (its, single.iterations)
    for r in range(n):
        assert oracle_residual(U, b, xs[r], kappa) <= 1e-10
