"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

The paper prints no worked example, so every pin is derived from the operator
of Eq. (1) itself: Clifford algebra of the stated gamma basis, the half-spinor
redundancy noted after Eq. (2), Eq. (1) == Eq. (2), a dense matrix assembled by
explicit site loops, the free-field plane-wave spectrum (closed form), gauge
covariance, gamma5-hermiticity, translation covariance and the even-odd
structure.  ``test_oracle_mutants.py`` plants mistakes in copies of the oracle
and checks that these pins catch them.
"""
import itertools

import numpy as np
import pytest

import synthetic as S
from oracle import c_oracle as C
from oracle import wilson as W

from pins import (
    brute_force_error,
    eq1_eq2_error,
    free_field_spectrum_error,
    gamma5_hermiticity_error,
    gauge_covariance_error,
    time_translation_error,
    space_translation_error,
)


# ---------------------------------------------------------------- gamma basis
def test_clifford_algebra():
    G = W.GAMMA
    for mu, nu in itertools.product(range(4), repeat=2):
        anti = G[mu] @ G[nu] + G[nu] @ G[mu]
        assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=0, rtol=0)


def test_gammas_hermitian_and_gamma5_diagonal():
    for g in W.GAMMA:
        assert np.array_equal(g, g.conj().T)
    assert np.array_equal(W.GAMMA5, np.diag([1, 1, -1, -1]).astype(complex))


def test_chiral_block_form():
    # gamma_mu = [[0, A], [A^dagger, 0]] with A unitary (the form behind the half-spinor trick).
    for g in W.GAMMA:
        assert np.all(g[:2, :2] == 0) and np.all(g[2:, 2:] == 0)
        A = g[:2, 2:]
        assert np.allclose(g[2:, :2], A.conj().T)
        assert np.allclose(A @ A.conj().T, np.eye(2))


def test_half_spinor_redundancy():
    # Sec. 2 after Eq. (2): the lower two spin components of (1 -/+ gamma_mu) phi follow from the upper two.
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    for mu in range(4):
        A = W.GAMMA[mu][:2, 2:]
        for sign in (-1, +1):
            full = (np.eye(4) + sign * W.GAMMA[mu]) @ phi
            upper = full[:2]
            assert np.allclose(full[2:], sign * A.conj().T @ upper, atol=1e-15)


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (8, 4, 6, 2), (10, 4, 6, 8)])
def test_eq1_equals_eq2(dims):
    U, phi = S.gauge_and_spinor(dims, 0.3, 1)
    assert eq1_eq2_error(W.hopping, U, phi) < 1e-14


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (8, 4, 6, 2), (10, 4, 6, 8)])
def test_c_oracle_matches_numpy(dims):
    U, phi = S.gauge_and_spinor(dims, 0.3, 2)
    a = W.hopping(U, phi)
    assert np.linalg.norm(C.hopping(U, phi) - a) / np.linalg.norm(a) < 1e-14
    m = W.wilson(U, phi, 0.12)
    assert np.linalg.norm(C.wilson(U, phi, 0.12) - m) / np.linalg.norm(m) < 1e-14
    sites = np.array([0, 5, U[..., 0, 0, 0].size - 1])
    ref = a.reshape(-1, 4, 3)[sites]
    assert np.allclose(C.hopping_sites(U, phi, sites), ref, atol=1e-13)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (4, 2, 2, 4)])
def test_brute_force_dense(dims):
    U = S.gauge_field(dims, 0.3, 3)
    assert brute_force_error(W.hopping, U) < 1e-14


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 2), (2, 4, 2, 2), (4, 4, 2, 2), (4, 4, 4, 4)])
def test_free_field_plane_wave_spectrum(dims):
    # the whole dense spectrum (3072 eigenvalues on 4^4) as a multiset against the closed form
    assert free_field_spectrum_error(W.hopping, dims, kappa=0.12) < 1e-12


def test_free_field_plane_wave_eigenvector():
    # H e^{ipx} u = [sum_mu 2 cos p_mu - 2 i gamma_mu sin p_mu] e^{ipx} u, on a bigger lattice.
    dims = (8, 4, 6, 4)
    T, Lx, Ly, Lz = dims
    shape = S.lattice_shape(dims)
    U = np.broadcast_to(np.eye(3, dtype=complex), shape + (4, 3, 3)).copy()
    p = np.array([3 * np.pi / T, 2 * np.pi / Lx, 4 * np.pi / Ly, 2 * np.pi * 3 / Lz])
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    phase = np.exp(1j * (p[0] * t + p[1] * x + p[2] * y + p[3] * z))
    rng = np.random.default_rng(4)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    phi = phase[..., None, None] * u
    K = sum(2 * np.cos(p[m]) * np.eye(4) - 2j * np.sin(p[m]) * W.GAMMA[m] for m in range(4))
    expect = phase[..., None, None] * (K @ u)
    assert np.max(np.abs(W.hopping(U, phi) - expect)) < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 4, 6, 2)])
def test_gauge_covariance(dims):
    U, phi = S.gauge_and_spinor(dims, 0.3, 5)
    G = S.random_gauge_transform(dims, 6)
    assert gauge_covariance_error(W.hopping, U, phi, G) < 1e-14


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 4, 6, 2)])
def test_gamma5_hermiticity(dims):
    U, phi = S.gauge_and_spinor(dims, 0.3, 7)
    chi = S.gaussian_spinor(dims, 8)
    assert gamma5_hermiticity_error(W.hopping, U, phi, chi) < 1e-14


def test_gamma5_hermiticity_dense():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.3, 9)
    shape = S.lattice_shape(dims) + (4, 3)
    M = W.dense(lambda v: W.wilson(U, v, 0.12), shape)
    g5 = np.kron(np.eye(S.volume(dims)), np.kron(W.GAMMA5, np.eye(3)))
    assert np.max(np.abs(g5 @ M - (g5 @ M).conj().T)) < 1e-15


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 4, 6, 2)])
def test_translation_covariance(dims):
    U, phi = S.gauge_and_spinor(dims, 0.3, 10)
    assert space_translation_error(W.hopping, U, phi) < 1e-14
    assert time_translation_error(W.hopping, U, phi) < 1e-14


# ---------------------------------------------------------------- even-odd
def test_hopping_flips_parity():
    dims = (4, 4, 2, 6)
    U, phi = S.gauge_and_spinor(dims, 0.3, 11)
    for par in (0, 1):
        out = W.hopping(U, W.restrict(phi, par))
        assert np.max(np.abs(W.restrict(out, par))) == 0.0  # H_ee = H_oo = 0


def test_schur_identity():
    # With x_o = b_o + kappa H_oe x_e the odd residual vanishes and the even one is bhat - Mhat x_e.
    dims = (4, 4, 2, 6)
    U, b = S.gauge_and_spinor(dims, 0.3, 12)
    x_e = W.restrict(S.gaussian_spinor(dims, 13), 0)
    kappa = 0.12
    x = x_e + W.reconstruct_odd(U, x_e, b, kappa)
    r = b - W.wilson(U, x, kappa)
    assert np.max(np.abs(W.restrict(r, 1))) < 1e-13
    r_hat = W.schur_rhs(U, b, kappa) - W.schur(U, x_e, kappa)
    assert np.max(np.abs(W.restrict(r, 0) - r_hat)) < 1e-13


def test_schur_dense_block_algebra():
    dims = (2, 2, 2, 4)
    kappa = 0.13
    U = S.gauge_field(dims, 0.3, 14)
    shape = S.lattice_shape(dims) + (4, 3)
    M = W.dense(lambda v: W.wilson(U, v, kappa), shape)
    par = np.repeat(W.parity(S.lattice_shape(dims)).ravel(), 12)
    e, o = par == 0, par == 1
    Mhat_blocks = M[np.ix_(e, e)] - M[np.ix_(e, o)] @ np.linalg.solve(M[np.ix_(o, o)], M[np.ix_(o, e)])
    Mhat = W.dense(lambda v: W.schur(U, v, kappa), shape)[np.ix_(e, e)]
    assert np.max(np.abs(Mhat - Mhat_blocks)) < 1e-14
    Mhat_dag = W.dense(lambda v: W.schur_dag(U, v, kappa), shape)[np.ix_(e, e)]
    assert np.max(np.abs(Mhat_dag - Mhat.conj().T)) < 1e-15


def test_link_spinor_product_pins():
    """The link x spinor kernel of the prefetch experiment (Sec. 2.2): brute force
    on a few records, the identity link, and unitarity (|U v| = |v| for every spin
    component's colour vector when U is in SU(3))."""
    rng = np.random.default_rng(3)
    n = 7
    U = S.su3_from_hermitian(rng.standard_normal((n, 3, 3)), rng.standard_normal((n, 3, 3)), 0.7)
    phi = rng.standard_normal((n, 4, 3)) + 1j * rng.standard_normal((n, 4, 3))
    got = W.link_spinor_product(U, phi)
    brute = np.zeros_like(phi)
    for i in range(n):
        for s in range(4):
            for a in range(3):
                for b in range(3):
                    brute[i, s, a] += U[i, a, b] * phi[i, s, b]
    assert np.max(np.abs(got - brute)) < 1e-14
    eye = np.broadcast_to(np.eye(3, dtype=complex), (n, 3, 3))
    assert np.array_equal(W.link_spinor_product(eye, phi), phi)
    assert np.allclose(np.linalg.norm(got, axis=2), np.linalg.norm(phi, axis=2), rtol=1e-13, atol=0)
