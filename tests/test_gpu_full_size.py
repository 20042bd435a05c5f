"""The benchmark workloads at their full sizes, in the launch configurations the
benchmark uses (autotuned), checked against the oracle on sampled outputs or on
the true residual it computes."""
import numpy as np
import pytest

import synthetic as S
from oracle import c_oracle as C

from gpuhelp import TOL, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1405_0700_gb300 import DF64, F16, F32, F64, Context  # noqa: E402
from paper_1405_0700_gb300 import plq as P  # noqa: E402


def test_multi_rhs_48c96_twelve_rhs_sampled_sites():
    """48^3 x 96 with 12 right-hand sides (the propagator workload's operator), in the
    tuner's launch.  RHS r is (r + 1) * phi, so every RHS has its own expected value and
    a mix-up between right-hand sides shows; sites are checked one by one against the
    C oracle's Eq. (1)."""
    dims = (96, 48, 48, 48)
    n = 12
    U = S.gauge_field(dims, 0.25, 4)
    phi = S.gaussian_spinor(dims, 41)
    V = S.volume(dims)
    rng = np.random.default_rng(5)
    sites = np.concatenate([[0, 1, V - 1, V // 2 - 1, V // 2], rng.integers(0, V, 1500)])
    ref = C.hopping_sites(U, phi, sites)
    with Context(dims) as ctx:
        for prec, reals in ((F32, 18), (F32, 12), (F16, 12)):
            ctx.gauge_upload(U, reals, prec)
            tuned = ctx.autotune(prec, n)
            one = torch.from_numpy(np.ascontiguousarray(phi).view(np.float64).ravel()).cuda()
            canon = torch.cat([one * (r + 1) for r in range(n)])
            del one
            full = ctx.empty_full(prec, n)
            ctx.pack_spinor(full, canon, prec, n)
            del canon
            e_in, o_in = ctx.halves(full, prec, n)
            out = ctx.empty_full(prec, n)
            e_out, o_out = ctx.halves(out, prec, n)
            ctx.hopping_eo(0, e_out, o_in, prec, n)
            ctx.hopping_eo(1, o_out, e_in, prec, n)
            del full
            back = torch.empty(n * V * 24, dtype=torch.float64, device="cuda")
            ctx.unpack_spinor(back, out, prec, n)
            del out
            got = back.view(n, V, 12, 2)[:, torch.from_numpy(sites).cuda()].cpu().numpy()
            del back
            got = (got[..., 0] + 1j * got[..., 1]).reshape(n, len(sites), 4, 3)
            for r in range(n):
                assert rel(got[r], (r + 1) * ref) <= TOL[prec], (prec, reals, tuned, r, rel(got[r], (r + 1) * ref))
            torch.cuda.empty_cache()


def test_propagator_48c96_point_sources_sampled_residual():
    """The propagator workload's solve (48^3 x 96, eps 0.25, seed 4, kappa 0.121, point
    sources, FP32 inner iterations with 12-real links, FP64 residual checks, true
    residual 1e-10) for two of its spin x colour columns, solved together.  The returned
    x is checked with the C oracle's Eq. (1) on sampled sites, the source site and its
    eight neighbours among them: at every site |b - M x| must stay below the global bound
    1e-10 |b| (a full FP64 CPU solve at this size would take hours)."""
    dims = (96, 48, 48, 48)
    n, kappa = 2, 0.121
    cols = (0, 7)  # spin 0 colour 0, spin 2 colour 1
    U = S.gauge_field(dims, 0.25, 4)
    V = S.volume(dims)
    T, Lx, Ly, Lz = dims
    # the origin, its 8 neighbours (lexicographic site = ((t Lz + z) Ly + y) Lx + x) and random sites
    near = [0, 1, Lx - 1, Lx, (Ly - 1) * Lx, Lx * Ly, (Lz - 1) * Lx * Ly, Lx * Ly * Lz, (T - 1) * Lx * Ly * Lz]
    rng = np.random.default_rng(8)
    sites = np.concatenate([near, rng.integers(0, V, 1200)]).astype(np.int64)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        ctx.gauge_upload(U, 12, F32)
        ctx.autotune(F32, n)
        b = torch.zeros(n * V * 24, dtype=torch.float64, device="cuda")
        for r, c in enumerate(cols):
            b[r * V * 24 + 2 * c] = 1.0
        bd = ctx.empty_full(F64, n)
        ctx.pack_spinor(bd, b, F64, n)
        del b
        x = ctx.empty_full(F64, n)
        infos = ctx.cg_solve_multi(x, bd, kappa, n, tol=1e-10, inner_prec=F32, maxit=3000)
        del bd
        back = torch.empty(n * V * 24, dtype=torch.float64, device="cuda")
        ctx.unpack_spinor(back, x, F64, n)
        del x
        for r, c in enumerate(cols):
            assert infos[r].true_rel_residual <= 1e-10, infos[r].as_dict()
            xr = back[r * V * 24:(r + 1) * V * 24].cpu().numpy().view(np.complex128).reshape(T, Lz, Ly, Lx, 4, 3)
            mx = xr.reshape(V, 4, 3)[sites] - kappa * C.hopping_sites(U, xr, sites)
            bs = np.zeros((len(sites), 4, 3), dtype=np.complex128)
            bs[0, c // 3, c % 3] = 1.0  # sites[0] is the origin
            res = np.abs(bs - mx).max()
            assert res <= 1e-10, (r, c, res)
            # the solution is not trivially small where the source sits
            assert np.abs(xr[0, 0, 0, 0, c // 3, c % 3]) > 0.5
        torch.cuda.empty_cache()


@pytest.mark.parametrize("inner,residual_prec", [(F32, F64), (F16, DF64)])
def test_mixed_cg_24c48_benchmark_configuration(inner, residual_prec):
    """The solver workload (24^3 x 48, eps 0.3, seed 3, kappa 0.120, true residual 1e-10),
    the returned x checked with the C oracle's Wilson operator."""
    dims = (48, 24, 24, 24)
    kappa = 0.120
    U, b = S.gauge_and_spinor(dims, 0.3, 3)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        ctx.gauge_upload(U, 12, inner)
        ctx.gauge_upload(U, 18, DF64)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        info = ctx.cg_solve(x, bd, kappa, tol=1e-10, inner_prec=inner, residual_prec=residual_prec)
        xs = ctx.to_host(x, F64)
    res = float(np.linalg.norm(b - C.wilson(U, xs, kappa)) / np.linalg.norm(b))
    assert res <= 1e-10, (res, info.as_dict())
    assert abs(info.true_rel_residual - res) < 1e-11


def test_batched_benchmark_lattice_sizes():
    """One system of each lattice of the batch workload (8^3x16, 16^3x32, 24^3x48) with
    its seed and kappa, in one persistent launch; each x checked with the C oracle."""
    specs = S.batch_solve_specs(n=3)
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
        xk = ctxs[k].to_host(xs[k], F64)
        res = float(np.linalg.norm(srcs[k] - C.wilson(Us[k], xk, sp["kappa"])) / np.linalg.norm(srcs[k]))
        assert res <= 1e-10, (sp["dims"], res, infos[k].as_dict())
    for c in ctxs:
        c.close()


def test_batched_sixteen_uneven_systems():
    """The whole batch workload: 16 systems (lattices cycling 8^3x16 / 16^3x32 / 24^3x48,
    per-system seeds and kappas in [0.110, 0.124]) in one persistent launch of the mixed
    FP32-inner CG; every returned x is checked with the C oracle's Wilson operator."""
    specs = S.batch_solve_specs(n=16)
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
    iters = set()
    for k, sp in enumerate(specs):
        xk = ctxs[k].to_host(xs[k], F64)
        res = float(np.linalg.norm(srcs[k] - C.wilson(Us[k], xk, sp["kappa"])) / np.linalg.norm(srcs[k]))
        assert res <= 1e-10, (k, sp["dims"], res, infos[k].as_dict())
        assert abs(infos[k].true_rel_residual - res) < 1e-11, (k, infos[k].true_rel_residual, res)
        iters.add(infos[k].iterations)
    assert len(iters) > 1  # uneven systems: the batch really retires systems at different times
    for c in ctxs:
        c.close()
