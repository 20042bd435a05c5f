"""Seeded synthetic inputs for the Wilson-Dirac hot path.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
random-field generation only and none of the arithmetic of the operator or of
the solvers, so that the oracle and the CUDA path stay independent: both are
handed the same arrays and compute their results separately.

Conventions (canonical layout, used by every caller):

* ``dims = (T, Lx, Ly, Lz)``; direction ``mu`` indexes ``dims[mu]`` with
  ``mu = 0`` the time direction and ``mu = 1, 2, 3`` the x, y, z directions.
* Lattice arrays have shape ``(T, Lz, Ly, Lx, ...)`` so that x runs fastest; the
  lexicographic site index is ``((t*Lz + z)*Ly + y)*Lx + x``.
* A gauge field has shape ``(T, Lz, Ly, Lx, 4, 3, 3)`` complex128:
  ``U[t, z, y, x, mu, row, col]`` is the SU(3) link leaving site x in
  direction +mu.
* A spinor field has shape ``(T, Lz, Ly, Lx, 4, 3)`` complex128:
  ``phi[..., spin, colour]``.

The gauge links follow the recipe U = exp(i*eps*H) with H a Gaussian Hermitian
traceless 3x3 matrix, then reunitarised (Gram-Schmidt on rows 0 and 1 and
row 2 = conj(row0 x row1)), so det U = 1 to rounding.  Random numbers come from
``numpy.random.default_rng(seed)`` (PCG64) and are drawn time slice by time
slice (real parts then imaginary parts of that slice), which lets large
lattices be generated in bounded memory while giving exactly the same field as
an unchunked run.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "lattice_shape",
    "volume",
    "su3_from_hermitian",
    "gauge_field",
    "gaussian_spinor",
    "gauge_and_spinor",
    "point_source",
    "random_gauge_transform",
    "reunitarise",
    "batch_solve_specs",
]


def lattice_shape(dims):
    """Array shape (T, Lz, Ly, Lx) of a lattice with ``dims = (T, Lx, Ly, Lz)``."""
    T, Lx, Ly, Lz = (int(d) for d in dims)
    return (T, Lz, Ly, Lx)


def volume(dims):
    T, Lx, Ly, Lz = (int(d) for d in dims)
    return T * Lx * Ly * Lz


def reunitarise(U):
    """Project a stack of 3x3 complex matrices back onto SU(3).

    Row 0 is normalised, row 1 is orthogonalised against row 0 and normalised,
    and row 2 is the complex conjugate of the cross product of rows 0 and 1,
    which fixes the determinant to 1.
    """
    U = np.array(U, dtype=np.complex128, copy=True)
    r0 = U[..., 0, :]
    r0 /= np.sqrt(np.sum(np.abs(r0) ** 2, axis=-1, keepdims=True))
    r1 = U[..., 1, :]
    r1 -= np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 /= np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1, keepdims=True))
    U[..., 0, :] = r0
    U[..., 1, :] = r1
    U[..., 2, :] = np.conj(np.cross(r0, r1))
    return U


def su3_from_hermitian(A_re, A_im, eps):
    """exp(i*eps*H) for H the traceless Hermitian part of A = A_re + i*A_im.

    H = (A + A^dagger)/2 - tr(A + A^dagger)/6 * 1, and the exponential is taken
    through the eigendecomposition H = V diag(lam) V^dagger, which is exact for
    Hermitian H.  The result is reunitarised.
    """
    A = A_re + 1j * A_im
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1)
    H = H - (tr / 3.0)[..., None, None] * np.eye(3)
    lam, V = np.linalg.eigh(H)
    E = np.exp(1j * eps * lam)
    U = np.matmul(V * E[..., None, :], np.conj(np.swapaxes(V, -1, -2)))
    return reunitarise(U)


def _gauge_slices(rng, dims, eps):
    T, Lx, Ly, Lz = (int(d) for d in dims)
    out = np.empty(lattice_shape(dims) + (4, 3, 3), dtype=np.complex128)
    slab = (Lz, Ly, Lx, 4, 3, 3)
    for t in range(T):
        a_re = rng.standard_normal(slab)
        a_im = rng.standard_normal(slab)
        out[t] = su3_from_hermitian(a_re, a_im, eps)
    return out


def _spinor_slices(rng, dims):
    T, Lx, Ly, Lz = (int(d) for d in dims)
    out = np.empty(lattice_shape(dims) + (4, 3), dtype=np.complex128)
    slab = (Lz, Ly, Lx, 4, 3)
    for t in range(T):
        re = rng.standard_normal(slab)
        im = rng.standard_normal(slab)
        out[t] = re + 1j * im
    return out


def gauge_field(dims, eps, seed):
    """Synthetic SU(3) gauge field U = reunitarise(exp(i*eps*H)), seeded."""
    rng = np.random.default_rng(seed)
    return _gauge_slices(rng, dims, eps)


def gauge_and_spinor(dims, eps, seed):
    """Gauge field and then a Gaussian complex spinor from the same generator."""
    rng = np.random.default_rng(seed)
    U = _gauge_slices(rng, dims, eps)
    phi = _spinor_slices(rng, dims)
    return U, phi


def gaussian_spinor(dims, seed):
    """Gaussian complex spinor (re and im standard normal), seeded."""
    rng = np.random.default_rng(seed)
    return _spinor_slices(rng, dims)


def point_source(dims, spin, colour, site=(0, 0, 0, 0)):
    """Unit vector at one site, spin and colour; ``site = (t, x, y, z)``."""
    phi = np.zeros(lattice_shape(dims) + (4, 3), dtype=np.complex128)
    t, x, y, z = site
    phi[t, z, y, x, spin, colour] = 1.0
    return phi


def random_gauge_transform(dims, seed):
    """A random SU(3) matrix per site, G = exp(i*H) with H Gaussian traceless."""
    rng = np.random.default_rng(seed)
    shape = lattice_shape(dims) + (3, 3)
    return su3_from_hermitian(rng.standard_normal(shape), rng.standard_normal(shape), 1.0)


def batch_solve_specs(n=16, sizes=((16, 8, 8, 8), (32, 16, 16, 16), (48, 24, 24, 24)),
                      kappa_lo=0.110, kappa_hi=0.124, eps=0.3, seed0=5000):
    """Descriptors of a batch of uneven solves: lattice, kappa, eps and seed.

    Solve i uses lattice ``sizes[i % len(sizes)]`` (dims order T, Lx, Ly, Lz),
    seed ``seed0 + i`` and kappa = kappa_lo + (kappa_hi - kappa_lo) * u_i with
    u_i uniform from ``default_rng(5)``.
    """
    u = np.random.default_rng(5).random(n)
    return [
        {
            "dims": tuple(sizes[i % len(sizes)]),
            "kappa": float(kappa_lo + (kappa_hi - kappa_lo) * u[i]),
            "eps": float(eps),
            "seed": int(seed0 + i),
        }
        for i in range(n)
    ]
