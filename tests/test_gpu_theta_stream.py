"""Two-pass theta schedule (Eq. (2)) and the link x spinor streaming kernel."""
import numpy as np
import pytest

import synthetic as S
from oracle import wilson as W
from gpuhelp import TOL, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1405_0700_gb300 import F32, F64, Context  # noqa: E402
from paper_1405_0700_gb300 import plq  # noqa: E402


@pytest.mark.parametrize("prec,reals", [(F64, 18), (F32, 18), (F32, 12)])
@pytest.mark.parametrize("dims", [(10, 4, 6, 8), (2, 2, 2, 2)])
def test_theta_schedule_matches_oracle(prec, reals, dims):
    U, phi = S.gauge_and_spinor(dims, 0.3, 31)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, reals, prec)
        full = ctx.to_device(phi, prec)
        e_in, o_in = ctx.halves(full, prec)
        out = ctx.empty_full(prec)
        e_out, o_out = ctx.halves(out, prec)
        theta = torch.empty(ctx.theta_bytes(prec), dtype=torch.uint8, device="cuda")
        ctx.hopping_eo_theta(0, e_out, o_in, theta, prec)
        ctx.hopping_eo_theta(1, o_out, e_in, theta, prec)
        got = ctx.to_host(out, prec)
    assert rel(got, W.hopping(U, phi)) <= TOL[prec]


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("prec", [F64, F32])
def test_link_spinor_stream(mode, prec):
    n = 5000
    rng = np.random.default_rng(7)
    Uc = S.su3_from_hermitian(rng.standard_normal((n, 3, 3)), rng.standard_normal((n, 3, 3)), 0.5)
    ph = rng.standard_normal((n, 4, 3)) + 1j * rng.standard_normal((n, 4, 3))
    expect = W.link_spinor_product(Uc, ph)  # the oracle's kernel of the prefetch experiment
    dt = torch.float64 if prec == F64 else torch.float32
    U = torch.from_numpy(Uc.view(np.float64).reshape(n, 18)).to("cuda", dt).contiguous()
    P = torch.from_numpy(ph.view(np.float64).reshape(n, 24)).to("cuda", dt).contiguous()
    out = torch.zeros_like(P)
    perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    ptrs = None
    if mode == 2:
        es = P.element_size()
        base = lambda t, w: t.data_ptr() + perm.long() * (w * es)
        ptrs = torch.cat([base(out, 24), base(U, 18), base(P, 24)]).to(torch.int64).contiguous()
    plq.link_spinor_stream(mode, n, U, P, out, perm if mode == 1 else None, ptrs, prec)
    torch.cuda.synchronize()
    got = out.cpu().double().numpy().reshape(n, 4, 3, 2)
    got = got[..., 0] + 1j * got[..., 1]
    tol = 1e-14 if prec == F64 else 1e-6
    assert np.max(np.abs(got - expect)) < tol * np.max(np.abs(expect)) * 10
