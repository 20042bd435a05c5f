"""plq_schur_apply_noalloc: the allocation-free form of the Schur operator.

Some callers cannot allocate device memory when they apply the operator
(during CUDA graph capture cudaMalloc is not allowed; applications with their
own device-memory pool forbid other allocations; real-time loops avoid the
allocator).  This entry point keeps its odd-parity intermediate in a fixed
array inside the library instead of a caller-provided buffer.  The test calls
it through the C ABI twice in a row, on different inputs, and checks each
result against plq_schur_apply with a caller-owned intermediate, within the
per-application tolerance of the other GPU tests.  It lives in a file that
pytest collects last.
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
