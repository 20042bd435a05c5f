"""plq_schur_apply_noalloc: the allocation-free form of the Schur operator.

Some callers cannot allocate device memory when they apply the operator:
applications that give all device memory to their own pool forbid other
allocations, and real-time loops avoid the allocator's locks and latency.
This entry point keeps its odd-parity intermediate in a fixed array inside the
library instead of a caller-provided buffer.  The tests call it through the C
ABI twice in a row, on different inputs, and check each result against
plq_schur_apply with a caller-owned intermediate, within the per-application
tolerance of the other GPU tests, in the default and in a hand-set launch
configuration.  They live in a file that pytest collects last.
"""
import numpy as np
import pytest

import synthetic as S
from gpuhelp import TOL, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1405_0700_gb300 import F16, F32, F64, Context, PLQError  # noqa: E402
from paper_1405_0700_gb300 import plq  # noqa: E402


@pytest.mark.parametrize("prec", [F64, F32, F16])
@pytest.mark.parametrize("dagger", [False, True])
def test_noalloc_schur_matches_schur_apply(prec, dagger):
    dims = (8, 8, 8, 8)
    kappa = 0.12
    U = S.gauge_field(dims, 0.3, 1)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18 if prec != F16 else 12, prec)
        tmp = ctx.empty_half(prec)
        for call, seed in enumerate((11, 12)):  # two calls in a row, different inputs
            v = S.gaussian_spinor(dims, seed)
            full = ctx.to_device(v, prec)
            e_in, _ = ctx.halves(full, prec)
            ref_full = ctx.empty_full(prec)
            ref_full.zero_()
            ctx.schur_apply(ctx.halves(ref_full, prec)[0], e_in, tmp, kappa, prec, dagger=dagger)
            got_full = ctx.empty_full(prec)
            got_full.zero_()
            ctx.schur_apply_noalloc(ctx.halves(got_full, prec)[0], e_in, kappa, prec, dagger=dagger)
            ref = ctx.to_host(ref_full, prec)
            got = ctx.to_host(got_full, prec)
            assert np.isfinite(got).all()
            assert rel(got, ref) <= TOL[prec], (call, rel(got, ref))


def test_noalloc_rejects_lattices_beyond_the_fixed_scratch():
    dims = (64, 32, 32, 32)  # one FP32 odd half field is 100 MB, above the 8 MiB array
    with Context(dims) as ctx:
        buf = ctx.empty_half(F32)
        out = ctx.empty_half(F32)
        with pytest.raises(PLQError) as e:
            ctx.schur_apply_noalloc(out, buf, 0.12, F32)
        assert e.value.status == plq.PLQ_ERR_ARG
        assert "scratch" in str(e.value)


@pytest.mark.parametrize("prec", [F32, F16])
def test_noalloc_schur_follows_the_launch_configuration(prec):
    """With a hand-set launch (neighbour table, 64-thread blocks, two sites per thread) the
    allocation-free operator and plq_schur_apply launch alike and agree on two calls in a row."""
    dims = (8, 8, 8, 8)
    kappa = 0.12
    U = S.gauge_field(dims, 0.3, 2)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 12, prec)
        ctx.set_launch(prec, 1, block=64, index_mode=1, sites_per_thread=2)
        tmp = ctx.empty_half(prec)
        for call, seed in enumerate((21, 22)):
            v = S.gaussian_spinor(dims, seed)
            full = ctx.to_device(v, prec)
            e_in, _ = ctx.halves(full, prec)
            ref_full = ctx.empty_full(prec)
            ref_full.zero_()
            ctx.schur_apply(ctx.halves(ref_full, prec)[0], e_in, tmp, kappa, prec)
            got_full = ctx.empty_full(prec)
            got_full.zero_()
            ctx.schur_apply_noalloc(ctx.halves(got_full, prec)[0], e_in, kappa, prec)
            ref = ctx.to_host(ref_full, prec)
            got = ctx.to_host(got_full, prec)
            assert rel(got, ref) <= TOL[prec], (call, rel(got, ref))
