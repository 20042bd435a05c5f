"""GPU hopping operator against the FP64 oracle (Eq. (1)), through the C ABI."""
import numpy as np
import pytest

import synthetic as S
from oracle import c_oracle as C
from oracle import wilson as W
from gpuhelp import TOL, gpu_hopping_full, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1405_0700_gb300 import F16, F32, F64, Context, PLQError  # noqa: E402
from paper_1405_0700_gb300 import plq  # noqa: E402

LATTICES = [
    (2, 2, 2, 2),      # x + mu = x - mu: forward and backward hops hit the same site
    (4, 4, 4, 4),
    (8, 8, 8, 8),      # the 8^4 small-lattice workload
    (8, 4, 4, 4),      # 4^3 x 8
    (10, 4, 6, 8),     # anisotropic: catches axis mix-ups
    (6, 2, 4, 2),      # Vh = 48: a ragged single block
    (14, 6, 2, 10),    # Vh = 840: several blocks and a ragged tail
]
FORMATS = [(F64, 18), (F64, 12), (F32, 18), (F32, 12), (F16, 18), (F16, 12)]


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("prec,reals", FORMATS)
def test_hopping_matches_oracle(dims, prec, reals):
    U, phi = S.gauge_and_spinor(dims, 0.3, 1)
    ref = W.hopping(U, phi)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, reals, prec)
        got = gpu_hopping_full(ctx, phi, prec)
    assert rel(got, ref) <= TOL[prec], (dims, prec, reals, rel(got, ref))


@pytest.mark.parametrize("prec", [F64, F32])
def test_periodic_time_boundary(prec):
    dims = (4, 4, 2, 6)
    U, phi = S.gauge_and_spinor(dims, 0.3, 2)
    ref = W.hopping(U, phi, t_bc=+1)
    with Context(dims, t_bc=+1) as ctx:
        ctx.gauge_upload(U, 18, prec)
        got = gpu_hopping_full(ctx, phi, prec)
    assert rel(got, ref) <= TOL[prec]


def test_free_field_plane_wave():
    # U = 1: H e^{ipx} u = [sum 2cos p - 2i gamma sin p] e^{ipx} u (closed form, independent of the oracle).
    dims = (8, 4, 6, 4)
    T, Lx, Ly, Lz = dims
    shape = S.lattice_shape(dims)
    U = np.broadcast_to(np.eye(3, dtype=complex), shape + (4, 3, 3)).copy()
    p = np.array([3 * np.pi / T, 2 * np.pi / Lx, 4 * np.pi / Ly, 6 * np.pi / Lz])
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    phase = np.exp(1j * (p[0] * t + p[1] * x + p[2] * y + p[3] * z))
    u = np.random.default_rng(3).standard_normal((4, 3)) + 0j
    phi = phase[..., None, None] * u
    K = sum(2 * np.cos(p[m]) * np.eye(4) - 2j * np.sin(p[m]) * W.GAMMA[m] for m in range(4))
    expect = phase[..., None, None] * (K @ u)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 12, F64)
        got = gpu_hopping_full(ctx, phi, F64)
    assert rel(got, expect) < 1e-13


@pytest.mark.parametrize("prec", [F64, F32, F16])
def test_wilson_apply(prec):
    dims = (8, 4, 4, 4)
    U, phi = S.gauge_and_spinor(dims, 0.3, 4)
    kappa = 0.12
    ref = W.wilson(U, phi, kappa)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, prec)
        inp = ctx.to_device(phi, prec)
        out = ctx.empty_full(prec)
        ctx.wilson_apply(out, inp, kappa, prec)
        got = ctx.to_host(out, prec)
    assert rel(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [F64, F32])
@pytest.mark.parametrize("dagger", [False, True])
def test_schur_apply(prec, dagger):
    dims = (4, 4, 6, 2)
    U, phi = S.gauge_and_spinor(dims, 0.3, 5)
    kappa = 0.13
    v = W.restrict(phi, 0)
    ref = (W.schur_dag if dagger else W.schur)(U, v, kappa)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, prec)
        full = ctx.to_device(v, prec)
        e_in, _ = ctx.halves(full, prec)
        out = ctx.empty_full(prec)
        out.zero_()
        e_out, _ = ctx.halves(out, prec)
        tmp = ctx.empty_half(prec)
        ctx.schur_apply(e_out, e_in, tmp, kappa, prec, dagger=dagger)
        got = ctx.to_host(out, prec)
    assert rel(got, ref) <= TOL[prec]


@pytest.mark.parametrize("nrhs", [1, 2, 5, 12])
@pytest.mark.parametrize("prec,reals", [(F64, 18), (F32, 18), (F32, 12), (F16, 12)])
def test_multi_rhs(nrhs, prec, reals):
    dims = (6, 4, 2, 4)
    U = S.gauge_field(dims, 0.3, 6)
    phis = np.stack([S.gaussian_spinor(dims, 100 + r) for r in range(nrhs)])
    with Context(dims) as ctx:
        ctx.gauge_upload(U, reals, prec)
        got = gpu_hopping_full(ctx, phis if nrhs > 1 else phis[0], prec, nrhs)
    got = got.reshape((nrhs,) + phis.shape[1:])
    for r in range(nrhs):
        assert rel(got[r], W.hopping(U, phis[r])) <= TOL[prec], r


@pytest.mark.parametrize("tile,zc,sm", [(2, 0, 0), (4, 0, 0), (1, 2, 0), (2, 4, 0), (1, 0, 1), (2, 4, 1),
                                        (1, 0, 2), (1, 4, 3)])
@pytest.mark.parametrize("prec,reals", [(F32, 18), (F32, 12), (F16, 12), (F16, 18)])
def test_multi_rhs_tiles(tile, zc, sm, prec, reals):
    # each thread applies every link it loads to `tile` right-hand sides; zc walks the
    # sites in z-chunks; two applications in a row
    dims = (6, 4, 2, 8)
    nrhs = 12
    U = S.gauge_field(dims, 0.3, 16)
    phis = np.stack([S.gaussian_spinor(dims, 200 + r) for r in range(nrhs)])
    with Context(dims) as ctx:
        ctx.gauge_upload(U, reals, prec)
        ctx.set_launch(prec, nrhs, 96, 0, tile, zc, sm)
        for _ in range(2):
            got = gpu_hopping_full(ctx, phis, prec, nrhs).reshape(phis.shape)
            for r in range(nrhs):
                assert rel(got[r], W.hopping(U, phis[r])) <= TOL[prec], r


@pytest.mark.parametrize("sm", [1, 2, 3])
@pytest.mark.parametrize("prec,reals", [(F32, 18), (F16, 12)])
@pytest.mark.parametrize("nrhs,block", [(5, 96), (2, 256), (3, 64)])
def test_multi_rhs_shared_staging_ragged(sm, prec, reals, nrhs, block):
    """Shared-memory link staging, with and without the neighbour spinors copied ahead
    (1 or 2 directions), for right-hand-side counts whose sites per block do not divide
    the half volume (a ragged last block) and blocks that are not whole warps."""
    dims = (6, 4, 2, 6)
    U = S.gauge_field(dims, 0.3, 17)
    phis = np.stack([S.gaussian_spinor(dims, 300 + r) for r in range(nrhs)])
    with Context(dims) as ctx:
        ctx.gauge_upload(U, reals, prec)
        ctx.set_launch(prec, nrhs, block, 0, 1, 0, sm)
        got = gpu_hopping_full(ctx, phis, prec, nrhs).reshape(phis.shape)
    for r in range(nrhs):
        assert rel(got[r], W.hopping(U, phis[r])) <= TOL[prec], r


def test_set_launch_rejects_bad_staging():
    dims = (4, 4, 2, 4)
    with Context(dims) as ctx:
        for sm, tile in ((5, 1), (-1, 1), (2, 2), (3, 4), (1, 4), (4, 2)):
            with pytest.raises(PLQError) as e:
                ctx.set_launch(F32, 4, 64, 0, tile, 0, sm)
            assert e.value.status == plq.PLQ_ERR_ARG


@pytest.mark.parametrize("prec,reals,nrhs", [(F32, 18, 1), (F16, 12, 1), (F32, 12, 3), (F64, 18, 2)])
def test_host_entry_point_matches_device(prec, reals, nrhs):
    """plq_hopping_eo_host (time-slab pipeline; captured as a graph for pinned buffers
    and replayed while they stay the same) equals plq_hopping_eo bit for bit, for
    pinned and pageable host buffers, repeated calls and a change of buffers."""
    dims = (16, 4, 4, 6)
    U = S.gauge_field(dims, 0.3, 7)
    phis = np.stack([S.gaussian_spinor(dims, 70 + r) for r in range(nrhs)])
    with Context(dims) as ctx:
        ctx.gauge_upload(U, reals, prec)
        full = ctx.to_device(phis if nrhs > 1 else phis[0], prec, nrhs)
        e_in, o_in = ctx.halves(full, prec, nrhs)
        dev_out = ctx.empty_half(prec, nrhs)
        for parity, src in ((0, o_in), (1, e_in)):
            ctx.hopping_eo(parity, dev_out, src, prec, nrhs)
            expect = dev_out.cpu()
            for pinned in (True, False):
                host_in = src.cpu()
                host_out = torch.zeros_like(host_in)
                if pinned:
                    host_in, host_out = host_in.pin_memory(), host_out.pin_memory()
                for _ in range(2):  # the second call replays the captured pipeline
                    host_out.zero_()
                    ctx.hopping_eo_host(parity, host_out, host_in, prec, nrhs)
                    torch.cuda.synchronize()
                    assert torch.equal(host_out, expect), (parity, pinned)


def test_errors_are_reported_not_faulted():
    dims = (4, 4, 4, 4)
    with Context(dims) as ctx:
        buf = ctx.empty_half(F32)
        buf2 = ctx.empty_half(F32)
        with pytest.raises(PLQError) as e:
            ctx.hopping_eo(0, buf, buf2, F32)  # no gauge uploaded
        assert e.value.status == plq.PLQ_ERR_STATE
        U = S.gauge_field(dims, 0.3, 1)
        ctx.gauge_upload(U, 18, F32)
        with pytest.raises(PLQError) as e:
            ctx.hopping_eo(2, buf, buf2, F32)
        assert e.value.status == plq.PLQ_ERR_ARG
        with pytest.raises(PLQError) as e:
            ctx.hopping_eo(0, buf, buf, F32)
        assert e.value.status == plq.PLQ_ERR_ARG
        with pytest.raises(PLQError) as e:
            ctx.hopping_eo(0, buf[1:], buf2, F32)  # misaligned
        assert e.value.status == plq.PLQ_ERR_ARG
        with pytest.raises(PLQError) as e:
            ctx.hopping_eo(0, buf, buf2, F32, nrhs=13)
        assert e.value.status == plq.PLQ_ERR_ARG
        # 12-real storage needs SU(3) links
        bad = U.copy()
        bad[0, 0, 0, 0, 1] *= 1.5
        with pytest.raises(PLQError) as e:
            ctx.gauge_upload(bad, 12, F32)
        assert e.value.status == plq.PLQ_ERR_ARG
        torch.cuda.synchronize()


def test_full_size_32c64_sampled_sites():
    """32^3 x 64 (the benchmark workload) in the benchmark's launch configuration,
    checked at sampled output sites computed one by one by the C oracle."""
    dims = (64, 32, 32, 32)
    U, phi = S.gauge_and_spinor(dims, 0.2, 2)
    V = S.volume(dims)
    rng = np.random.default_rng(0)
    sites = np.concatenate([[0, 1, V - 1, V // 2], rng.integers(0, V, 2000)])
    ref = C.hopping_sites(U, phi, sites)
    with Context(dims) as ctx:
        for prec, reals in [(F32, 18), (F32, 12), (F16, 12), (F64, 18)]:
            ctx.gauge_upload(U, reals, prec)
            got = gpu_hopping_full(ctx, phi, prec).reshape(V, 4, 3)[sites]
            assert rel(got, ref) <= TOL[prec], (prec, reals, rel(got, ref))


@pytest.mark.parametrize("prec", [F64, F32, F16])
def test_neighbour_table_mode_matches_oracle(prec):
    # index mode 1: neighbours read from the precomputed table (pointer arrays of Sec. 2.2)
    dims = (10, 4, 6, 8)
    U, phi = S.gauge_and_spinor(dims, 0.3, 9)
    kappa = 0.12
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 12 if prec == F16 else 18, prec)
        ctx.set_launch(prec, 1, 64, 1, 1, 2)
        got = gpu_hopping_full(ctx, phi, prec)
        inp = ctx.to_device(phi, prec)
        out = ctx.empty_full(prec)
        ctx.wilson_apply(out, inp, kappa, prec)
        gotw = ctx.to_host(out, prec)
    assert rel(got, W.hopping(U, phi)) <= TOL[prec]
    assert rel(gotw, W.wilson(U, phi, kappa)) <= TOL[prec]


def test_autotune_and_cache(tmp_path):
    dims = (16, 8, 8, 8)
    U, phi = S.gauge_and_spinor(dims, 0.3, 10)
    cache = str(tmp_path / "tune.txt")
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F32)
        r = ctx.autotune(F32, 1, cache_path=cache)
        assert r["from_cache"] == 0 and r["candidates"] >= 10
        assert r["block"] in (64, 96, 128, 192, 256, 512) and r["sites_per_thread"] in (0, 1, 2, 4, 8)
        got = gpu_hopping_full(ctx, phi, F32)  # runs with the tuned launch
        assert rel(got, W.hopping(U, phi)) <= TOL[F32]
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F32)
        r2 = ctx.autotune(F32, 1, cache_path=cache)
        assert r2["from_cache"] == 1
        for k in ("block", "index_mode", "rhs_tile", "z_chunk", "smem_links", "sites_per_thread"):
            assert r2[k] == r[k], k
    assert open(cache).read().count("\n") == 1


def test_autotune_cache_ignores_invalid_lines(tmp_path):
    """A cache line with an out-of-range field is skipped (the tuner times instead);
    a line in the older seven-field form reads as one wave of resident blocks."""
    dims = (8, 4, 4, 4)
    U = S.gauge_field(dims, 0.3, 11)
    cache = tmp_path / "tune.txt"
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F32)
        r = ctx.autotune(F32, 1, cache_path=str(cache))
    key = cache.read_text().split()[0]
    cache.write_text(f"{key} 100 0 1 0 0 1.0\n")  # block 100: not a multiple of 32
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F32)
        assert ctx.autotune(F32, 1, cache_path=str(cache))["from_cache"] == 0
    cache.write_text(f"{key} 64 0 1 0 0 1.0\n")
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F32)
        r3 = ctx.autotune(F32, 1, cache_path=str(cache))
        assert r3["from_cache"] == 1 and r3["block"] == 64 and r3["sites_per_thread"] == 0


@pytest.mark.parametrize("prec,reals,nrhs,block,sm,spt", [
    (F32, 18, 1, 512, 0, 0), (F32, 18, 1, 512, 0, 1), (F32, 12, 1, 128, 0, 4), (F16, 12, 1, 64, 0, 8),
    (F64, 18, 1, 128, 0, 2), (F32, 18, 12, 96, 1, 2), (F16, 12, 5, 512, 3, 1), (F32, 12, 4, 256, 0, 3)])
def test_block_sizes_and_sites_per_thread(prec, reals, nrhs, block, sm, spt):
    """Blocks above 256 threads (where the kernel's registers allow) and grids sized for
    k sites per thread, including grids that leave a ragged last block."""
    dims = (6, 4, 4, 6)
    U = S.gauge_field(dims, 0.3, 18)
    phis = np.stack([S.gaussian_spinor(dims, 400 + r) for r in range(nrhs)])
    with Context(dims) as ctx:
        ctx.gauge_upload(U, reals, prec)
        ctx.set_launch(prec, nrhs, block, 0, 1, 0, sm, spt)
        got = gpu_hopping_full(ctx, phis if nrhs > 1 else phis[0], prec, nrhs).reshape(phis.shape)
    for r in range(nrhs):
        assert rel(got[r], W.hopping(U, phis[r])) <= TOL[prec], r


def test_block_that_does_not_fit_is_an_argument_error():
    """1024 threads x 80 registers exceed the SM's register file: the operator call
    returns PLQ_ERR_ARG (nothing launched) and the context keeps working."""
    dims = (4, 4, 4, 4)
    U, phi = S.gauge_and_spinor(dims, 0.3, 19)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F32)
        ctx.set_launch(F32, 1, 1024, 0, 1, 0, 0, 0)
        with pytest.raises(PLQError) as e:
            gpu_hopping_full(ctx, phi, F32)
        assert e.value.status == plq.PLQ_ERR_ARG
        ctx.set_launch(F32, 1, 0, 0, 1, 0, 0, 0)
        assert rel(gpu_hopping_full(ctx, phi, F32), W.hopping(U, phi)) <= TOL[F32]


@pytest.mark.parametrize("T", [2, 6, 24, 40, 96])
def test_host_entry_point_slab_schedules(T):
    """Time extents whose slab schedules differ (one slice per slab; ramps of 1, 1, 2
    ... slices at both ends with T/8 slices between, and a remainder slab): the host
    pipeline equals plq_hopping_eo bit for bit on both parities."""
    dims = (T, 4, 2, 2)
    U = S.gauge_field(dims, 0.3, 20)
    phi = S.gaussian_spinor(dims, 21)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F32)
        full = ctx.to_device(phi, F32)
        e_in, o_in = ctx.halves(full, F32)
        dev_out = ctx.empty_half(F32)
        for parity, src in ((0, o_in), (1, e_in)):
            ctx.hopping_eo(parity, dev_out, src, F32)
            host_in = src.cpu().pin_memory()
            host_out = torch.zeros_like(host_in).pin_memory()
            ctx.hopping_eo_host(parity, host_out, host_in, F32)
            torch.cuda.synchronize()
            assert torch.equal(host_out, dev_out.cpu()), parity


def test_fp16_storage_of_values_down_to_the_subnormal_range():
    """Sites whose largest component spans 1 .. 1e-44: FP16 storage keeps every site
    with a normal-range maximum to half-precision accuracy, stores sites below 2^-126 as
    zero (no infinities or NaNs), and the operator on such a field stays within the
    FP16 tolerance."""
    dims = (8, 4, 4, 4)
    U = S.gauge_field(dims, 0.3, 23)
    phi = S.gaussian_spinor(dims, 24)
    scale = np.power(10.0, -(np.arange(S.volume(dims)) % 46))  # 1, 0.1, ..., 1e-45 per site
    phi = phi * scale.reshape(S.lattice_shape(dims) + (1, 1))
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 12, F16)
        back = ctx.to_host(ctx.to_device(phi, F16), F16)
        got = gpu_hopping_full(ctx, phi, F16)
    assert np.all(np.isfinite(back)) and np.all(np.isfinite(got))
    site_max = np.abs(phi).max(axis=(-2, -1))
    big = site_max >= 2.0 ** -126
    err = np.abs(back - phi).max(axis=(-2, -1))
    assert np.all(err[big] <= 1e-3 * site_max[big])
    assert np.all(back[~big] == 0)
    assert rel(got, W.hopping(U, phi)) <= TOL[F16]


def test_host_entry_point_follows_gauge_format_change():
    dims = (8, 4, 4, 4)
    U, phi = S.gauge_and_spinor(dims, 0.3, 12)
    with Context(dims) as ctx:
        host_in = host_out = None
        for reals in (18, 12, 18):
            ctx.gauge_upload(U, reals, F32)
            full = ctx.to_device(phi, F32)
            e_in, o_in = ctx.halves(full, F32)
            dev_out = ctx.empty_half(F32)
            ctx.hopping_eo(0, dev_out, o_in, F32)
            if host_in is None:
                host_in = o_in.cpu().pin_memory()
                host_out = torch.empty_like(host_in).pin_memory()
            ctx.hopping_eo_host(0, host_out, host_in, F32)
            torch.cuda.synchronize()
            assert torch.equal(host_out, dev_out.cpu()), reals


ROW_LATTICES = [(8, 8, 8, 8), (10, 4, 6, 8), (6, 16, 2, 4), (4, 8, 2, 6)]


def rows_fit(dims, prec, reals, nrhs):
    """The row-streamed kernel's conditions: n x Lx/2 threads <= 512 and, for FP16
    storage, a run of site norms that is a multiple of 16 bytes."""
    lxh = dims[1] // 2
    if nrhs * lxh > 512:
        return False
    return not (prec == F16 and (lxh * nrhs) % 4)


@pytest.mark.parametrize("dims", ROW_LATTICES)
@pytest.mark.parametrize("prec,reals", [(F32, 18), (F32, 12), (F16, 12), (F16, 18)])
@pytest.mark.parametrize("nrhs,slots", [(1, 0), (4, 3), (12, 0), (3, 2)])
def test_row_streamed_kernel(dims, prec, reals, nrhs, slots):
    """The row-streamed kernel (whole neighbour rows and their links copied into a ring of
    shared-memory slots by bulk copies) against the oracle, for several slot counts and
    right-hand-side counts; where the rows cannot be copied in 16-byte runs the launch is
    an argument error."""
    U = S.gauge_field(dims, 0.3, 18)
    phis = np.stack([S.gaussian_spinor(dims, 400 + r) for r in range(nrhs)])
    with Context(dims) as ctx:
        ctx.gauge_upload(U, reals, prec)
        ctx.set_launch(prec, nrhs, 0, 0, 1, 0, 4, slots)
        if not rows_fit(dims, prec, reals, nrhs):
            with pytest.raises(PLQError) as e:
                gpu_hopping_full(ctx, phis if nrhs > 1 else phis[0], prec, nrhs)
            assert e.value.status == plq.PLQ_ERR_ARG
            return
        got = gpu_hopping_full(ctx, phis if nrhs > 1 else phis[0], prec, nrhs).reshape(phis.shape)
        assert ctx.device_status() == plq.PLQ_OK
    for r in range(nrhs):
        assert rel(got[r], W.hopping(U, phis[r])) <= TOL[prec], (r, rel(got[r], W.hopping(U, phis[r])))


@pytest.mark.parametrize("prec,reals", [(F32, 18), (F16, 12)])
def test_row_streamed_wilson_and_twisted_epilogues(prec, reals):
    """The operator epilogues (Wilson M = 1 - kappa H, twisted mass) in the row-streamed
    launch, against the oracle."""
    dims = (8, 8, 4, 4)
    U, phi = S.gauge_and_spinor(dims, 0.3, 19)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, reals, prec)
        ctx.set_launch(prec, 1, 0, 0, 1, 0, 4, 0)
        full = ctx.to_device(phi, prec)
        out = ctx.empty_full(prec)
        ctx.wilson_apply(out, full, 0.12, prec)
        assert rel(ctx.to_host(out, prec), W.wilson(U, phi, 0.12)) <= TOL[prec]
        ctx.twisted_apply(out, full, 0.12, 0.05, prec)
        assert rel(ctx.to_host(out, prec), W.twisted(U, phi, 0.12, 0.05)) <= TOL[prec]


def test_row_streamed_wait_limit_reports_timeout():
    """Every wait of the row-streamed kernel is bounded: with a limit of one clock cycle
    its first wait for a shared-memory copy gives up, the kernel records PLQ_ERR_TIMEOUT
    in the context's status word and returns (no fault, no hang); with the default limit
    restored the same context computes the right result.  The block has 6 warps (12
    right-hand sides x 16 sites), so warps other than the one issuing the copies reach
    their first wait while the copies are in flight."""
    dims = (4, 32, 8, 4)
    n = 12
    U = S.gauge_field(dims, 0.3, 20)
    phis = np.stack([S.gaussian_spinor(dims, 500 + r) for r in range(n)])
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F32)
        ctx.set_launch(F32, n, 0, 0, 1, 0, 4, 3)
        ctx.set_wait_limit(1e-12)
        gpu_hopping_full(ctx, phis, F32, n)
        assert ctx.device_status(clear=True) == plq.PLQ_ERR_TIMEOUT
        assert ctx.device_status() == plq.PLQ_OK
        ctx.set_wait_limit(5.0)
        got = gpu_hopping_full(ctx, phis, F32, n).reshape(phis.shape)
        assert ctx.device_status() == plq.PLQ_OK
    for r in range(n):
        assert rel(got[r], W.hopping(U, phis[r])) <= TOL[F32]
