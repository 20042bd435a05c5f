"""Field checkpoint files (host logic, no GPU): the canonical spinor shape and the
checks that reading a saved field applies."""
import numpy as np
import pytest

import synthetic as S
from paper_1405_0700_gb300.plq import read_spinors, spinor_shape


def test_spinor_shape_is_the_canonical_layout():
    dims = (8, 4, 6, 2)  # (T, Lx, Ly, Lz)
    assert spinor_shape(dims) == S.lattice_shape(dims) + (4, 3) == (8, 2, 6, 4, 4, 3)
    assert spinor_shape(dims, 12) == (12, 8, 2, 6, 4, 4, 3)


def test_round_trip_is_exact(tmp_path):
    dims = (4, 4, 2, 2)
    phi = np.stack([S.gaussian_spinor(dims, 30 + r) for r in range(3)])
    path = tmp_path / "x.npy"
    np.save(path, phi, allow_pickle=False)
    back = read_spinors(path, dims, 3)
    assert back.dtype == np.complex128 and np.array_equal(back, phi)


@pytest.mark.parametrize("bad", ["lattice", "nrhs", "dtype"])
def test_mismatched_files_are_rejected(tmp_path, bad):
    dims = (4, 4, 2, 2)
    phi = S.gaussian_spinor(dims, 31)
    path = tmp_path / "x.npy"
    if bad == "lattice":
        np.save(path, S.gaussian_spinor((4, 2, 4, 2), 31))
    elif bad == "nrhs":
        np.save(path, np.stack([phi, phi]))
    else:
        np.save(path, phi.astype(np.complex64))
    with pytest.raises(ValueError):
        read_spinors(path, dims, 1)
