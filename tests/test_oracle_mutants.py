"""Plant plausible mistakes in copies of the oracle's Eq. (1) and check the pins catch them.

Each mutant differs from ``oracle.wilson.hopping`` in one place (a dropped
boundary sign, swapped projectors, U instead of U^dagger, a transposed link, a
dropped direction, a link read at the wrong site, a mixed-up axis).  A pin set
that let one of them through would not be pinning the oracle.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import wilson as W

from pins import (
    brute_force_error,
    eq1_eq2_error,
    free_field_spectrum_error,
    gamma5_hermiticity_error,
    gauge_covariance_error,
    time_translation_error,
)

ONE4 = np.eye(4, dtype=complex)


def _mutant(*, bc=True, fwd_sign=-1, bwd_sign=+1, bwd_link="dagger", dirs=4, bwd_site="x-mu", axes=(0, 3, 2, 1)):
    def shift(f, mu, step, t_bc):
        out = np.roll(f, -step, axis=axes[mu])
        if mu == 0 and bc and t_bc != 1:
            out[f.shape[0] - 1 if step > 0 else 0] *= t_bc
        return out

    def hop(U, phi, t_bc=-1):
        psi = np.zeros_like(phi)
        for mu in range(dirs):
            U_mu = U[..., mu, :, :]
            psi += np.einsum("...ab,st,...tb->...sa", U_mu, ONE4 + fwd_sign * W.GAMMA[mu], shift(phi, mu, +1, t_bc))
            Ub = np.roll(U_mu, 1, axis=axes[mu]) if bwd_site == "x-mu" else U_mu
            if bwd_link == "dagger":
                L = np.conj(np.swapaxes(Ub, -1, -2))
            elif bwd_link == "plain":
                L = Ub
            else:  # transpose without conjugation
                L = np.swapaxes(Ub, -1, -2)
            psi += np.einsum("...ab,st,...tb->...sa", L, ONE4 + bwd_sign * W.GAMMA[mu], shift(phi, mu, -1, t_bc))
        return psi

    return hop


MUTANTS = {
    "no_time_bc": _mutant(bc=False),
    "swapped_projectors": _mutant(fwd_sign=+1, bwd_sign=-1),
    "backward_U_not_daggered": _mutant(bwd_link="plain"),
    "backward_U_transposed": _mutant(bwd_link="transpose"),
    "dropped_direction": _mutant(dirs=3),
    "backward_link_at_x": _mutant(bwd_site="x"),
    "x_and_z_axes_swapped": _mutant(axes=(0, 1, 2, 3)),
}


def _pin_errors(hop):
    dims = (4, 2, 2, 4)
    U, phi = S.gauge_and_spinor(dims, 0.3, 21)
    chi = S.gaussian_spinor(dims, 22)
    G = S.random_gauge_transform(dims, 23)
    return {
        "eq1_eq2": eq1_eq2_error(hop, U, phi),
        "brute_force": brute_force_error(hop, U),
        "free_field": free_field_spectrum_error(hop, (4, 2, 2, 2)),
        "gauge_cov": gauge_covariance_error(hop, U, phi, G),
        "gamma5_herm": gamma5_hermiticity_error(hop, U, phi, chi),
        "time_translation": time_translation_error(hop, U, phi),
    }


def test_unmutated_copy_passes_every_pin():
    errs = _pin_errors(_mutant())
    assert max(errs.values()) < 1e-12, errs


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    errs = _pin_errors(MUTANTS[name])
    caught = [k for k, v in errs.items() if v > 1e-6]
    assert caught, f"{name} passed every pin: {errs}"
    # the independent dense assembly of Eq. (1) catches every mutant on its own
    assert "brute_force" in caught


def test_gamma_sign_flip_caught_by_basis_pin(monkeypatch):
    flipped = W.GAMMA.copy()
    flipped[1] = -flipped[1]
    # Clifford relations survive a sign flip; gamma5 = g0 g1 g2 g3 = diag(1,1,-1,-1) does not.
    g5 = flipped[0] @ flipped[1] @ flipped[2] @ flipped[3]
    assert not np.allclose(g5, np.diag([1, 1, -1, -1]))
