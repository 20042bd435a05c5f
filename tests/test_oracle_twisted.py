"""Pins of the twisted-mass oracle (no GPU)."""
import numpy as np
import pytest

import synthetic as S
from oracle import wilson as W

from pins import free_field_eigenvalues, _multiset_distance


def test_mu_zero_is_wilson():
    dims = (4, 4, 2, 2)
    U, phi = S.gauge_and_spinor(dims, 0.3, 1)
    assert np.array_equal(W.twisted(U, phi, 0.12, 0.0), W.wilson(U, phi, 0.12))


def test_gamma5_hermiticity_flips_mu():
    # gamma5 M_tm(mu) gamma5 = M_tm(-mu)^dagger: <chi, g5 M(mu) g5 phi> = <M(-mu) chi, phi>
    dims = (4, 4, 4, 4)
    U, phi = S.gauge_and_spinor(dims, 0.3, 2)
    chi = S.gaussian_spinor(dims, 3)
    k, mu = 0.12, 0.05
    a = W.inner(chi, W.gamma5(W.twisted(U, W.gamma5(phi), k, mu)))
    b = W.inner(W.twisted(U, chi, k, -mu), phi)
    assert abs(a - b) < 1e-12 * np.linalg.norm(chi) * np.linalg.norm(phi)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 2)])
def test_free_field_twisted_spectrum(dims):
    # U = 1: (sum gamma_mu s_mu + nu gamma5)^2 = |s|^2 + nu^2, so the eigenvalues are
    # 1 - 2 kappa sum cos p +/- i sqrt(4 kappa^2 |sin p|^2 + (2 kappa mu)^2).
    kappa, mu = 0.12, 0.3
    shape = S.lattice_shape(dims)
    U = np.broadcast_to(np.eye(3, dtype=complex), shape + (4, 3, 3)).copy()
    M = W.dense(lambda v: W.twisted(U, v, kappa, mu), shape + (4, 3))
    wil = free_field_eigenvalues(dims, kappa)
    expect = wil.real + 1j * np.sign(wil.imag + 1e-300) * np.sqrt(wil.imag ** 2 + (2 * kappa * mu) ** 2)
    assert _multiset_distance(np.linalg.eigvals(M), expect) < 1e-12


def test_schur_tm_block_algebra():
    dims = (2, 2, 2, 4)
    kappa, mu = 0.13, 0.07
    U = S.gauge_field(dims, 0.3, 4)
    shape = S.lattice_shape(dims) + (4, 3)
    M = W.dense(lambda v: W.twisted(U, v, kappa, mu), shape)
    par = np.repeat(W.parity(S.lattice_shape(dims)).ravel(), 12)
    e, o = par == 0, par == 1
    blocks = M[np.ix_(e, e)] - M[np.ix_(e, o)] @ np.linalg.solve(M[np.ix_(o, o)], M[np.ix_(o, e)])
    Mhat = W.dense(lambda v: W.schur_tm(U, v, kappa, mu), shape)[np.ix_(e, e)]
    assert np.max(np.abs(Mhat - blocks)) < 1e-14


def test_tm_cg_matches_dense_solve():
    dims = (4, 4, 4, 4)
    kappa, mu = 0.12, 0.02
    U, b = S.gauge_and_spinor(dims, 0.3, 5)
    M = W.dense(lambda v: W.twisted(U, v, kappa, mu), b.shape)
    x_ref = np.linalg.solve(M, b.ravel()).reshape(b.shape)
    res = W.solve_cg_eo_tm(U, b, kappa, mu)
    assert res.status == "ok"
    assert np.linalg.norm(res.x - x_ref) / np.linalg.norm(x_ref) < 1e-8
