"""Runs the library's kernels through the C ABI on small lattices and checks each
result against the oracle and the context's device status word.

Started by test_gpu_debug_build.py in a child process whose PLQ_LIBRARY names the
PLQ_DEBUG build (device bounds guards that record PLQ_ERR_BOUNDS instead of
accessing out of range), so that a guard that fires anywhere in these launches
shows up as a status, not as a fault.  Prints one JSON line and exits 0 when every
check passed.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main():
    import numpy as np
    import torch  # noqa: F401  (device memory)

    import synthetic as S
    from gpuhelp import TOL, gpu_hopping_full, rel
    from oracle import c_oracle as C
    from oracle import wilson as W
    from paper_1405_0700_gb300 import F16, F32, F64, Context
    from paper_1405_0700_gb300 import plq

    failures, checks = [], 0

    def check(name, ok, status):
        nonlocal checks
        checks += 1
        if not ok or status != plq.PLQ_OK:
            failures.append({"check": name, "ok": bool(ok), "status": int(status)})

    # single and multi-right-hand-side operator, every format, ragged lattices, every launch kind
    for dims in [(6, 2, 4, 2), (14, 6, 2, 10), (8, 8, 4, 4)]:
        U = S.gauge_field(dims, 0.3, 31)
        for prec, reals in [(F64, 18), (F64, 12), (F32, 18), (F32, 12), (F16, 18), (F16, 12)]:
            with Context(dims) as ctx:
                ctx.gauge_upload(U, reals, prec)
                phi = S.gaussian_spinor(dims, 32)
                got = gpu_hopping_full(ctx, phi, prec)
                check(f"hop {dims} {prec} {reals}", rel(got, W.hopping(U, phi)) <= TOL[prec], ctx.device_status())
                if prec == F64:
                    continue
                n = 5
                phis = np.stack([S.gaussian_spinor(dims, 40 + r) for r in range(n)])
                lxh = dims[1] // 2
                launches = [(96, 0, 1, 0, 0), (64, 1, 1, 0, 0), (96, 0, 1, 0, 1), (96, 0, 1, 0, 2), (96, 0, 1, 0, 3)]
                if n * lxh <= 512 and not (prec == F16 and (lxh * n) % 4):
                    launches.append((0, 0, 1, 0, 4))
                for blk, mode, tile, zc, sm in launches:
                    ctx.set_launch(prec, n, blk, mode, tile, zc, sm)
                    got = gpu_hopping_full(ctx, phis, prec, n).reshape(phis.shape)
                    ok = all(rel(got[r], W.hopping(U, phis[r])) <= TOL[prec] for r in range(n))
                    check(f"mrhs {dims} {prec} {reals} {(blk, mode, tile, zc, sm)}", ok, ctx.device_status())
    # solvers: mixed CG (single and multi), BiCGstab, batched
    dims = (8, 4, 4, 4)
    kappa = 0.12
    U, b = S.gauge_and_spinor(dims, 0.3, 33)
    with Context(dims) as ctx:
        ctx.gauge_upload(U, 18, F64)
        ctx.gauge_upload(U, 12, F32)
        bd = ctx.to_device(b, F64)
        x = ctx.empty_full(F64)
        for fn in (ctx.cg_solve, ctx.bicgstab_solve):
            fn(x, bd, kappa, inner_prec=F32)
            xs = ctx.to_host(x, F64)
            res = np.linalg.norm(b - C.wilson(U, xs, kappa)) / np.linalg.norm(b)
            check(f"{fn.__name__}", res <= 1e-10, ctx.device_status())
        n = 3
        srcs = np.stack([S.gaussian_spinor(dims, 50 + r) for r in range(n)])
        bm = ctx.to_device(srcs, F64, n)
        xm = ctx.empty_full(F64, n)
        ctx.cg_solve_multi(xm, bm, kappa, n, inner_prec=F32)
        xs = ctx.to_host(xm, F64, n).reshape(srcs.shape)
        ok = all(np.linalg.norm(srcs[r] - C.wilson(U, xs[r], kappa)) / np.linalg.norm(srcs[r]) <= 1e-10
                 for r in range(n))
        check("cg_solve_multi", ok, ctx.device_status())
    specs = S.batch_solve_specs(n=3, sizes=((8, 4, 4, 4), (16, 8, 8, 8), (10, 4, 6, 8)))
    ctxs, xs, bs, Us, srcs = [], [], [], [], []
    for sp in specs:
        Uk, bk = S.gauge_and_spinor(sp["dims"], sp["eps"], sp["seed"])
        c = Context(sp["dims"])
        c.gauge_upload(Uk, 18, F64)
        c.gauge_upload(Uk, 12, F32)
        ctxs.append(c)
        bs.append(c.to_device(bk, F64))
        xs.append(c.empty_full(F64))
        Us.append(Uk)
        srcs.append(bk)
    st = plq.lib().plq_cg_solve_batched  # noqa: F841  (loaded from the debug library)
    infos, _ = plq.cg_solve_batched(ctxs, xs, bs, [sp["kappa"] for sp in specs], inner_prec=F32,
                                    raise_on_error=False)
    ok = all(int(i.status) == plq.PLQ_OK for i in infos)
    for k, sp in enumerate(specs):
        xk = ctxs[k].to_host(xs[k], F64)
        ok = ok and np.linalg.norm(srcs[k] - C.wilson(Us[k], xk, sp["kappa"])) / np.linalg.norm(srcs[k]) <= 1e-10
    check("cg_solve_batched", ok, plq.PLQ_OK)
    for c in ctxs:
        c.close()
    print(json.dumps({"library": plq.LIB_PATH, "checks": checks, "failures": failures}))
    return 0 if not failures else 1


if __name__ == "__main__":
    sys.exit(main())
