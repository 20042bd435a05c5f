"""The seeded input generators: SU(3) links, reproducibility, chunk-independence."""
import numpy as np

import synthetic as S


def test_links_are_su3():
    U = S.gauge_field((4, 2, 2, 2), 0.3, 1)
    assert U.shape == (4, 2, 2, 2, 4, 3, 3)
    eye = np.eye(3)
    UUd = U @ np.conj(np.swapaxes(U, -1, -2))
    assert np.max(np.abs(UUd - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(U) - 1.0)) < 1e-14


def test_small_eps_is_near_identity():
    # exp(i eps H) -> 1 as eps -> 0: the link is built from the exponential, not a random unitary.
    U = S.gauge_field((2, 2, 2, 2), 1e-6, 3)
    assert np.max(np.abs(U - np.eye(3))) < 1e-4


def test_reproducible_and_seed_sensitive():
    a = S.gauge_and_spinor((2, 4, 2, 2), 0.2, 7)
    b = S.gauge_and_spinor((2, 4, 2, 2), 0.2, 7)
    c = S.gauge_and_spinor((2, 4, 2, 2), 0.2, 8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.allclose(a[0], c[0])


def test_gaussian_spinor_moments():
    phi = S.gaussian_spinor((8, 8, 8, 8), 11)
    assert abs(np.mean(phi.real)) < 0.02 and abs(np.var(phi.real) - 1) < 0.02
    assert abs(np.var(phi.imag) - 1) < 0.02


def test_point_source():
    phi = S.point_source((4, 2, 2, 2), 2, 1)
    assert phi[0, 0, 0, 0, 2, 1] == 1 and np.count_nonzero(phi) == 1


def test_batch_specs():
    specs = S.batch_solve_specs()
    assert len(specs) == 16
    assert all(0.110 <= s["kappa"] <= 0.124 for s in specs)
    assert [s["dims"][0] for s in specs[:3]] == [16, 32, 48]


def test_parallel_generation_matches_serial():
    dims = (4, 4, 2, 2)
    a = S.gauge_field(dims, 0.3, 5, workers=1)
    b = S.gauge_field(dims, 0.3, 5, workers=2)
    assert np.array_equal(a, b)
    assert np.array_equal(S.gaussian_spinor(dims, 5, workers=1), S.gaussian_spinor(dims, 5, workers=2))


def test_time_slices_are_independent_streams():
    # slice t of a T=4 lattice equals slice t of a T=2 lattice with the same seed (t < 2)
    a = S.gauge_field((4, 2, 2, 2), 0.3, 9)
    b = S.gauge_field((2, 2, 2, 2), 0.3, 9)
    assert np.array_equal(a[:2], b)
