"""Helpers for the GPU parity tests: run the library through its C ABI."""
import numpy as np

TOL = {0: 1e-13, 1: 2e-6, 2: 5e-3, 3: 1e-13}  # relative L2 per operator application: FP64, FP32, FP16, DF64


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_hopping_full(ctx, phi, prec, nrhs=1):
    """H phi on the whole lattice through two plq_hopping_eo calls."""
    full = ctx.to_device(phi, prec, nrhs)
    e_in, o_in = ctx.halves(full, prec, nrhs)
    out = ctx.empty_full(prec, nrhs)
    e_out, o_out = ctx.halves(out, prec, nrhs)
    ctx.hopping_eo(0, e_out, o_in, prec, nrhs)
    ctx.hopping_eo(1, o_out, e_in, prec, nrhs)
    return ctx.to_host(out, prec, nrhs)
