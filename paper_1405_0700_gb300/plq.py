"""Thin ctypes binding of libplq.so (the C ABI declared in include/plq.h).

Only argument marshalling happens here: every step of the operator and of the
solvers runs in the library's CUDA kernels.  PyTorch provides device memory
(``torch.uint8`` tensors sized by ``field_bytes``) and the current CUDA stream.
If ``libplq.so`` is missing the import of this module fails: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PLQ_LIBRARY may name another build of the same library (the PLQ_DEBUG build,
# libplq_debug.so); there is no fallback if the file is missing.
LIB_PATH = os.environ.get("PLQ_LIBRARY") or os.path.join(_HERE, "libplq.so")

PLQ_OK = 0
PLQ_ERR_ARG = 1
PLQ_ERR_CUDA = 2
PLQ_ERR_NOMEM = 3
PLQ_ERR_NOT_CONVERGED = 4
PLQ_ERR_BREAKDOWN = 5
PLQ_ERR_NAN = 6
PLQ_ERR_TIMEOUT = 7
PLQ_ERR_STATE = 8
PLQ_ERR_BOUNDS = 9

F64, F32, F16, DF64 = 0, 1, 2, 3
MAX_RHS = 12
NOALLOC_SCRATCH_BYTES = 8 << 20
SITE_BYTES = {F64: 192, F32: 96, F16: 52, DF64: 192}
PREC_NAMES = {"f64": F64, "f32": F32, "f16": F16, "df64": DF64}

# Every function declared in include/plq.h, with (restype, argtypes).
_c_int, _c_double, _vp, _c_long, _c_size = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_long, ctypes.c_size_t


class SolverParams(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("maxit", ctypes.c_int),
        ("inner_prec", ctypes.c_int),
        ("delta", ctypes.c_double),
        ("use_x0", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("mu", ctypes.c_double),
        ("residual_prec", ctypes.c_int),
        ("wait_limit_s", ctypes.c_double),
    ]


class TuneResult(ctypes.Structure):
    _fields_ = [
        ("block", ctypes.c_int),
        ("index_mode", ctypes.c_int),
        ("rhs_tile", ctypes.c_int),
        ("z_chunk", ctypes.c_int),
        ("smem_links", ctypes.c_int),
        ("us_per_launch", ctypes.c_double),
        ("from_cache", ctypes.c_int),
        ("candidates", ctypes.c_int),
        ("sites_per_thread", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("grid", ctypes.c_int),
        ("block", ctypes.c_int),
        ("graph_captured", ctypes.c_int),
        ("launches", ctypes.c_int),
        ("seconds", ctypes.c_double),
        ("blocks_per_sm", ctypes.c_int),
        ("graph_reused", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iterations", ctypes.c_int),
        ("n_reliable", ctypes.c_int),
        ("true_rel_residual", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("hop_applications", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


SIGNATURES = {
    "plq_last_error": (ctypes.c_char_p, []),
    "plq_version": (_c_int, []),
    "plq_init": (_c_int, [ctypes.POINTER(_vp), _vp, _c_int, _c_int]),
    "plq_finalize": (_c_int, [_vp]),
    "plq_half_volume": (_c_long, [_vp]),
    "plq_set_wait_limit": (_c_int, [_vp, _c_double]),
    "plq_device_status": (_c_int, [_vp, _c_int]),
    "plq_field_bytes": (_c_size, [_vp, _c_int, _c_int]),
    "plq_gauge_upload": (_c_int, [_vp, _vp, _c_int, _c_int, _c_int, _vp]),
    "plq_pack_spinor": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _vp]),
    "plq_unpack_spinor": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _vp]),
    "plq_hopping_eo": (_c_int, [_vp, _c_int, _vp, _vp, _c_int, _c_int, _vp]),
    "plq_hopping_eo_host": (_c_int, [_vp, _c_int, _vp, _vp, _c_int, _c_int, _vp]),
    "plq_wilson_apply": (_c_int, [_vp, _vp, _vp, _c_double, _c_int, _vp]),
    "plq_twisted_apply": (_c_int, [_vp, _vp, _vp, _c_double, _c_double, _c_int, _vp]),
    "plq_schur_apply": (_c_int, [_vp, _vp, _vp, _vp, _c_double, _c_int, _c_int, _vp]),
    "plq_cg_solve": (_c_int, [_vp, _vp, _vp, _c_double, ctypes.POINTER(SolverParams), ctypes.POINTER(SolveInfo), _vp]),
    "plq_bicgstab_solve": (_c_int, [_vp, _vp, _vp, _c_double, ctypes.POINTER(SolverParams),
                                    ctypes.POINTER(SolveInfo), _vp]),
    "plq_cg_solve_multi": (_c_int, [_vp, _vp, _vp, _c_double, _c_int, ctypes.POINTER(SolverParams),
                                    ctypes.POINTER(SolveInfo), _vp]),
    "plq_bicgstab_solve_multi": (_c_int, [_vp, _vp, _vp, _c_double, _c_int, ctypes.POINTER(SolverParams),
                                          ctypes.POINTER(SolveInfo), _vp]),
    "plq_cg_solve_batched": (_c_int, [ctypes.POINTER(_vp), _c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolverParams),
                                      ctypes.POINTER(SolveInfo), ctypes.POINTER(BatchInfo), _vp]),
    "plq_set_batched_launch": (_c_int, [_vp, _c_int, _c_int]),
    "plq_autotune_batched": (_c_int, [ctypes.POINTER(_vp), _c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolverParams), ctypes.c_char_p,
                                      ctypes.POINTER(BatchInfo)]),
    "plq_theta_bytes": (_c_size, [_vp, _c_int]),
    "plq_hopping_eo_theta": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _c_int, _vp]),
    "plq_link_spinor_stream": (_c_int, [_c_int, ctypes.c_longlong, _vp, _vp, _vp, _vp, _vp, _c_int, _vp]),
    "plq_eigcg_create": (_c_int, [_vp, _c_int, _c_int, _c_int, ctypes.POINTER(_vp)]),
    "plq_eigcg_destroy": (_c_int, [_vp]),
    "plq_eigcg_vectors": (_c_int, [_vp]),
    "plq_eigcg_projected_matrix": (_c_int, [_vp, _vp, _c_int]),
    "plq_eigcg_solve": (_c_int, [_vp, _vp, _vp, _c_double, ctypes.POINTER(SolverParams), _c_int,
                                 ctypes.POINTER(SolveInfo), _vp]),
    "plq_measure_fma_rate": (_c_int, [_c_int, _c_int, ctypes.POINTER(ctypes.c_double)]),
    "plq_schur_apply_noalloc": (_c_int, [_vp, _vp, _vp, _c_double, _c_int, _c_int, _vp]),
    "plq_autotune": (_c_int, [_vp, _c_int, _c_int, ctypes.c_char_p, ctypes.POINTER(TuneResult)]),
    "plq_set_launch": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int]),
    "plq_host_slabs": (_c_int, [_c_int, ctypes.POINTER(_c_int)]),
}

_lib = None


def lib():
    """Load libplq.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: build it with paper_1405_0700_gb300._build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PLQError(RuntimeError):
    def __init__(self, status, message, info=None):
        super().__init__(f"plq status {status}: {message}")
        self.status = status
        self.info = info


def last_error():
    return lib().plq_last_error().decode()


def check(status, info=None):
    if status != PLQ_OK:
        raise PLQError(status, last_error(), info)
    return status


def _ptr(t):
    """Device (or host) address of a torch tensor or numpy array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch

    return torch.cuda.current_stream().cuda_stream


def prec_of(p):
    return PREC_NAMES[p] if isinstance(p, str) else int(p)


def spinor_shape(dims, nrhs=1):
    """Shape of `nrhs` canonical spinor fields of lattice dims = (T, Lx, Ly, Lz)."""
    T, Lx, Ly, Lz = dims
    return ((nrhs,) if nrhs > 1 else ()) + (T, Lz, Ly, Lx, 4, 3)


def read_spinors(path, dims, nrhs=1):
    """Canonical complex128 spinor field(s) from a NumPy .npy file, checked against
    the lattice and the number of right-hand sides."""
    a = np.load(path, allow_pickle=False)
    want = spinor_shape(dims, nrhs)
    if a.shape != want:
        raise ValueError(f"{path}: shape {a.shape}, expected {want} for lattice {tuple(dims)} and nrhs={nrhs}")
    if a.dtype != np.complex128:
        raise ValueError(f"{path}: dtype {a.dtype}, expected complex128")
    return a


class Context:
    """A lattice on one GPU: ``dims = (T, Lx, Ly, Lz)``, time boundary ``t_bc``."""

    def __init__(self, dims, t_bc=-1, device=0):
        self.dims = tuple(int(d) for d in dims)
        self.t_bc = t_bc
        self.device = device
        h = _vp()
        arr = (ctypes.c_int * 4)(*self.dims)
        check(lib().plq_init(ctypes.byref(h), ctypes.cast(arr, _vp), t_bc, device))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().plq_finalize(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ sizes
    @property
    def half_volume(self):
        return int(lib().plq_half_volume(self._h))

    def set_wait_limit(self, seconds):
        """Longest time a bounded wait inside this context's kernels may take."""
        check(lib().plq_set_wait_limit(self._h, float(seconds)))

    def device_status(self, clear=True):
        """Status word of this context's kernels (PLQ_OK, or the error a kernel recorded)."""
        return int(lib().plq_device_status(self._h, int(bool(clear))))

    @property
    def volume(self):
        return 2 * self.half_volume

    def field_bytes(self, prec, nrhs=1):
        return int(lib().plq_field_bytes(self._h, prec_of(prec), nrhs))

    def empty_half(self, prec, nrhs=1):
        import torch

        return torch.empty(self.field_bytes(prec, nrhs), dtype=torch.uint8, device=f"cuda:{self.device}")

    def empty_full(self, prec, nrhs=1):
        import torch

        return torch.empty(2 * self.field_bytes(prec, nrhs), dtype=torch.uint8, device=f"cuda:{self.device}")

    def halves(self, full, prec, nrhs=1):
        n = self.field_bytes(prec, nrhs)
        return full[:n], full[n:]

    # ------------------------------------------------------------ data
    def gauge_upload(self, U, link_reals=18, prec=F64, stream=None):
        """U: canonical gauge field (complex128 NumPy array on the host, or a
        float64/complex128 torch tensor on the device)."""
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
            check(lib().plq_gauge_upload(self._h, U.ctypes.data, 0, link_reals, prec_of(prec), _stream(stream)))
        else:
            check(lib().plq_gauge_upload(self._h, U.data_ptr(), 1, link_reals, prec_of(prec), _stream(stream)))

    def pack_spinor(self, out, phi_dev, prec, nrhs=1, stream=None):
        check(lib().plq_pack_spinor(self._h, _ptr(out), _ptr(phi_dev), prec_of(prec), nrhs, _stream(stream)))
        return out

    def unpack_spinor(self, out_dev, field, prec, nrhs=1, stream=None):
        check(lib().plq_unpack_spinor(self._h, _ptr(out_dev), _ptr(field), prec_of(prec), nrhs, _stream(stream)))
        return out_dev

    def to_device(self, phi, prec, nrhs=1, stream=None):
        """Canonical complex128 NumPy spinor(s) -> packed full field on the device."""
        import torch

        src = torch.from_numpy(np.ascontiguousarray(phi, dtype=np.complex128).view(np.float64).ravel())
        src = src.to(f"cuda:{self.device}")
        out = self.empty_full(prec, nrhs)
        self.pack_spinor(out, src, prec, nrhs, stream)
        return out

    def to_host(self, field, prec, nrhs=1, stream=None):
        """Packed full field on the device -> canonical complex128 NumPy array."""
        import torch

        out = torch.empty(nrhs * self.volume * 24, dtype=torch.float64, device=f"cuda:{self.device}")
        self.unpack_spinor(out, field, prec, nrhs, stream)
        torch.cuda.synchronize(self.device)
        a = out.cpu().numpy().view(np.complex128)
        return a.reshape(spinor_shape(self.dims, nrhs))

    def save_field(self, path, field, prec, nrhs=1):
        """Checkpoint: write a packed field to `path` as a NumPy .npy array of canonical
        complex128 spinors (exact for FP64 fields); a solve resumes from it through
        load_field and use_x0."""
        np.save(path, self.to_host(field, prec, nrhs), allow_pickle=False)

    def load_field(self, path, prec, nrhs=1):
        """A new packed field of precision `prec` from a file written by save_field (or any
        canonical complex128 array of this lattice's shape)."""
        return self.to_device(read_spinors(path, self.dims, nrhs), prec, nrhs)

    # ------------------------------------------------------------ operators
    def hopping_eo(self, out_parity, out, inp, prec, nrhs=1, stream=None):
        check(lib().plq_hopping_eo(self._h, out_parity, _ptr(out), _ptr(inp), prec_of(prec), nrhs, _stream(stream)))
        return out

    def hopping_eo_host(self, out_parity, out_host, in_host, prec, nrhs=1, stream=None):
        check(lib().plq_hopping_eo_host(self._h, out_parity, _ptr(out_host), _ptr(in_host), prec_of(prec), nrhs,
                                        _stream(stream)))
        return out_host

    def wilson_apply(self, out, inp, kappa, prec, stream=None):
        check(lib().plq_wilson_apply(self._h, _ptr(out), _ptr(inp), float(kappa), prec_of(prec), _stream(stream)))
        return out

    def twisted_apply(self, out, inp, kappa, mu, prec, stream=None):
        check(lib().plq_twisted_apply(self._h, _ptr(out), _ptr(inp), float(kappa), float(mu), prec_of(prec),
                                      _stream(stream)))
        return out

    def schur_apply(self, out, inp, tmp, kappa, prec, dagger=False, stream=None):
        check(lib().plq_schur_apply(self._h, _ptr(out), _ptr(inp), _ptr(tmp), float(kappa), int(bool(dagger)),
                                    prec_of(prec), _stream(stream)))
        return out

    def schur_apply_noalloc(self, out, inp, kappa, prec, dagger=False, stream=None):
        """Mhat (or Mhat^dagger) on an even half field without any allocation in
        the call: the odd intermediate lives in the library's fixed device array
        (at most NOALLOC_SCRATCH_BYTES); concurrent calls on one GPU race."""
        check(lib().plq_schur_apply_noalloc(self._h, _ptr(out), _ptr(inp), float(kappa), int(bool(dagger)),
                                            prec_of(prec), _stream(stream)))
        return out

    def theta_bytes(self, prec):
        return int(lib().plq_theta_bytes(self._h, prec_of(prec)))

    def hopping_eo_theta(self, out_parity, out, inp, theta, prec, stream=None):
        """Two-pass (theta-field) schedule of the half-lattice hopping operator."""
        check(lib().plq_hopping_eo_theta(self._h, out_parity, _ptr(out), _ptr(inp), _ptr(theta), prec_of(prec),
                                         _stream(stream)))
        return out

    # ------------------------------------------------------------ tuning
    def autotune(self, prec, nrhs=1, cache_path=None):
        r = TuneResult()
        path = cache_path.encode() if cache_path else None
        check(lib().plq_autotune(self._h, prec_of(prec), nrhs, path, ctypes.byref(r)))
        return r.as_dict()

    def set_launch(self, prec, nrhs=1, block=0, index_mode=0, rhs_tile=1, z_chunk=0, smem_links=0,
                   sites_per_thread=0):
        check(lib().plq_set_launch(self._h, prec_of(prec), nrhs, block, index_mode, rhs_tile, z_chunk, smem_links,
                                   sites_per_thread))

    # ------------------------------------------------------------ solvers
    def _solve(self, fn, x, b, kappa, tol, maxit, inner_prec, delta, use_x0, check_every, stream, raise_on_error,
               mu=0.0, residual_prec=F64):
        p = SolverParams(tol, maxit, prec_of(inner_prec), delta, int(use_x0), check_every, mu, prec_of(residual_prec))
        info = SolveInfo()
        st = fn(self._h, _ptr(x), _ptr(b), float(kappa), ctypes.byref(p), ctypes.byref(info), _stream(stream))
        if raise_on_error:
            check(st, info)
        return info

    def cg_solve(self, x, b, kappa, tol=1e-10, maxit=20000, inner_prec=F64, delta=0.0, use_x0=False,
                 check_every=16, stream=None, raise_on_error=True, mu=0.0, residual_prec=F64):
        """CG on the even-odd normal equations; x, b packed full FP64 fields (mu: twisted mass;
        residual_prec: FP64 or DF64 arithmetic of the reliable-update residuals)."""
        return self._solve(lib().plq_cg_solve, x, b, kappa, tol, maxit, inner_prec, delta, use_x0, check_every,
                           stream, raise_on_error, mu, residual_prec)

    def _solve_multi(self, fn, x, b, kappa, nrhs, tol, maxit, inner_prec, delta, use_x0, check_every, stream,
                     raise_on_error, residual_prec=F64):
        p = SolverParams(tol, maxit, prec_of(inner_prec), delta, int(use_x0), check_every, 0.0,
                         prec_of(residual_prec))
        infos = (SolveInfo * nrhs)()
        st = fn(self._h, _ptr(x), _ptr(b), float(kappa), nrhs, ctypes.byref(p), infos, _stream(stream))
        if raise_on_error:
            check(st, list(infos))
        return list(infos)

    def cg_solve_multi(self, x, b, kappa, nrhs, tol=1e-10, maxit=20000, inner_prec=F64, delta=0.0, use_x0=False,
                       check_every=16, stream=None, raise_on_error=True, residual_prec=F64):
        """CG for nrhs interleaved right-hand sides (links loaded once per operator application)."""
        return self._solve_multi(lib().plq_cg_solve_multi, x, b, kappa, nrhs, tol, maxit, inner_prec, delta, use_x0,
                                 check_every, stream, raise_on_error, residual_prec)

    def bicgstab_solve_multi(self, x, b, kappa, nrhs, tol=1e-10, maxit=20000, inner_prec=F64, delta=0.0,
                             use_x0=False, check_every=16, stream=None, raise_on_error=True, residual_prec=F64):
        return self._solve_multi(lib().plq_bicgstab_solve_multi, x, b, kappa, nrhs, tol, maxit, inner_prec, delta,
                                 use_x0, check_every, stream, raise_on_error, residual_prec)

    def bicgstab_solve(self, x, b, kappa, tol=1e-10, maxit=20000, inner_prec=F64, delta=0.0, use_x0=False,
                       check_every=16, stream=None, raise_on_error=True, mu=0.0, residual_prec=F64):
        """BiCGstab on the even-odd Schur system; x, b packed full FP64 fields (mu: twisted mass)."""
        return self._solve(lib().plq_bicgstab_solve, x, b, kappa, tol, maxit, inner_prec, delta, use_x0,
                           check_every, stream, raise_on_error, mu, residual_prec)


def cg_solve_batched(ctxs, xs, bs, kappas, tol=1e-10, maxit=20000, inner_prec=F64, delta=0.0, use_x0=False,
                     stream=None, raise_on_error=True, wait_limit_s=0.0):
    """One persistent launch solving len(ctxs) independent systems (see plq_cg_solve_batched).
    wait_limit_s bounds each grid-barrier wait (0: the library default, about 5 s)."""
    n = len(ctxs)
    H = (_vp * n)(*[c.handle.value for c in ctxs])
    X = (_vp * n)(*[_ptr(x) for x in xs])
    B = (_vp * n)(*[_ptr(b) for b in bs])
    K = (ctypes.c_double * n)(*[float(k) for k in kappas])
    p = SolverParams(tol, maxit, prec_of(inner_prec), delta, int(use_x0), 16, 0.0, F64, float(wait_limit_s))
    infos = (SolveInfo * n)()
    bi = BatchInfo()
    st = lib().plq_cg_solve_batched(H, n, X, B, K, ctypes.byref(p), infos, ctypes.byref(bi), _stream(stream))
    if raise_on_error:
        check(st, (list(infos), bi))
    return list(infos), bi.as_dict()


def set_batched_launch(ctx, block=0, blocks_per_sm=0):
    """Launch shape of the persistent batched kernel for batches led by ``ctx``."""
    check(lib().plq_set_batched_launch(ctx.handle, int(block), int(blocks_per_sm)))


def autotune_batched(ctxs, xs, bs, kappas, tol=1e-10, maxit=20000, inner_prec=F64, delta=0.0, cache_path=None,
                     wait_limit_s=0.0):
    """Time the persistent batched CG's launch shapes on these systems (see
    plq_autotune_batched) and keep the fastest in ctxs[0]; returns its launch report."""
    n = len(ctxs)
    H = (_vp * n)(*[c.handle.value for c in ctxs])
    X = (_vp * n)(*[_ptr(x) for x in xs])
    B = (_vp * n)(*[_ptr(b) for b in bs])
    K = (ctypes.c_double * n)(*[float(k) for k in kappas])
    p = SolverParams(tol, maxit, prec_of(inner_prec), delta, 0, 16, 0.0, F64, float(wait_limit_s))
    bi = BatchInfo()
    path = cache_path.encode() if cache_path else None
    check(lib().plq_autotune_batched(H, n, X, B, K, ctypes.byref(p), path, ctypes.byref(bi)))
    return bi.as_dict()


class EigCG:
    """Incremental EigCG deflation on a context (see plq_eigcg_create / plq_eigcg_solve)."""

    def __init__(self, ctx, nev=10, m=60, max_vectors=300):
        h = _vp()
        check(lib().plq_eigcg_create(ctx.handle, nev, m, max_vectors, ctypes.byref(h)))
        self._h = h
        self.ctx = ctx

    @property
    def vectors(self):
        return int(lib().plq_eigcg_vectors(self._h))

    def projected_matrix(self):
        """H = U^H A U of the deflation basis as a (k, k) complex128 array."""
        k = int(lib().plq_eigcg_projected_matrix(self._h, None, 0))
        if k < 0:
            check(PLQ_ERR_ARG)
        H = np.zeros((max(k, 1), max(k, 1), 2), dtype=np.float64)
        got = int(lib().plq_eigcg_projected_matrix(self._h, H.ctypes.data, max(k, 1)))
        if got < 0:
            check(PLQ_ERR_ARG)
        return (H[..., 0] + 1j * H[..., 1])[:k, :k]

    def solve(self, x, b, kappa, tol=1e-8, maxit=20000, accumulate=True, stream=None, raise_on_error=True):
        p = SolverParams(tol, maxit, F64, 0.0, 0, 16, 0.0, F64)
        info = SolveInfo()
        st = lib().plq_eigcg_solve(self._h, _ptr(x), _ptr(b), float(kappa), ctypes.byref(p), int(bool(accumulate)),
                                   ctypes.byref(info), _stream(stream))
        if raise_on_error:
            check(st, info)
        return info

    def close(self):
        if getattr(self, "_h", None):
            lib().plq_eigcg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def link_spinor_stream(mode, nsites, U, phi, psi, index=None, pointers=None, prec=F32, stream=None):
    """psi(i) = U(i) phi(i) over nsites site records (see plq_link_spinor_stream)."""
    check(lib().plq_link_spinor_stream(int(mode), int(nsites), _ptr(U), _ptr(phi), _ptr(psi), _ptr(index),
                                       _ptr(pointers), prec_of(prec), _stream(stream)))


def measure_fma_rate(prec, device=0):
    """Sustained FMA throughput (flop/s) of the CUDA cores in FP64 or FP32."""
    out = ctypes.c_double()
    check(lib().plq_measure_fma_rate(device, prec_of(prec), ctypes.byref(out)))
    return out.value


def canonical_gauge_device(U, device=0):
    """Copy a canonical complex128 NumPy gauge field to the device as float64."""
    import torch

    return torch.from_numpy(np.ascontiguousarray(U, dtype=np.complex128).view(np.float64).ravel()).to(f"cuda:{device}")
