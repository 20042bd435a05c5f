"""Pin checks for a hopping-operator implementation ``hop(U, phi, t_bc=-1)``.

Each function returns an error (0 for an exact operator up to rounding).  They
are used on the oracle itself (test_oracle_pins.py) and on copies of it with a
planted mistake (test_oracle_mutants.py), which must fail at least one pin.
"""
import numpy as np

import synthetic as S
from oracle import wilson as W

AX = (0, 3, 2, 1)  # array axis of direction mu in (T, Lz, Ly, Lx, ...) fields


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def eq1_eq2_error(hop, U, phi):
    """Eq. (1) against the theta-field form of Eq. (2)."""
    return _rel(hop(U, phi, -1), W.hopping_theta(U, phi, -1))


def brute_force_error(hop, U):
    """Dense matrix of ``hop`` against the site-loop assembly of Eq. (1)."""
    shape = U.shape[:4] + (4, 3)
    D = W.dense(lambda v: hop(U, v, -1), shape)
    B = W.brute_force_hopping_dense(U, -1)
    return float(np.max(np.abs(D - B)))


def free_field_eigenvalues(dims, kappa):
    """Closed-form spectrum of M = 1 - kappa H at U = 1 (periodic space, antiperiodic time).

    A plane wave e^{ipx} u has H -> sum_mu (2 cos p_mu - 2 i gamma_mu sin p_mu);
    (sum gamma_mu s_mu)^2 = |s|^2, so M has eigenvalues
    1 - 2 kappa sum cos p_mu +/- 2 i kappa |sin p|, each twice in spin and thrice in colour.
    """
    T, Lx, Ly, Lz = dims
    out = []
    for n0 in range(T):
        for n1 in range(Lx):
            for n2 in range(Ly):
                for n3 in range(Lz):
                    p = [(2 * n0 + 1) * np.pi / T, 2 * np.pi * n1 / Lx, 2 * np.pi * n2 / Ly, 2 * np.pi * n3 / Lz]
                    re = 1 - 2 * kappa * sum(np.cos(q) for q in p)
                    im = 2 * kappa * np.sqrt(sum(np.sin(q) ** 2 for q in p))
                    out += [re + 1j * im] * 6 + [re - 1j * im] * 6
    return np.array(out)


def _multiset_distance(a, b):
    from scipy.optimize import linear_sum_assignment

    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return float(np.max(cost[r, c]))


def free_field_spectrum_error(hop, dims, kappa=0.12):
    shape = S.lattice_shape(dims)
    U = np.broadcast_to(np.eye(3, dtype=complex), shape + (4, 3, 3)).copy()
    H = W.dense(lambda v: hop(U, v, -1), shape + (4, 3))
    M = np.eye(H.shape[0]) - kappa * H
    return _multiset_distance(np.linalg.eigvals(M), free_field_eigenvalues(dims, kappa))


def gauge_covariance_error(hop, U, phi, G):
    """H[U'] G phi = G H[U] phi with U'_mu(x) = G(x) U_mu(x) G(x + mu)^dagger."""
    Up = np.empty_like(U)
    for mu in range(4):
        G_fwd = np.roll(G, -1, axis=AX[mu])
        Up[..., mu, :, :] = G @ U[..., mu, :, :] @ np.conj(np.swapaxes(G_fwd, -1, -2))
    lhs = hop(Up, np.einsum("...ab,...sb->...sa", G, phi), -1)
    rhs = np.einsum("...ab,...sb->...sa", G, hop(U, phi, -1))
    return _rel(lhs, rhs)


def gamma5_hermiticity_error(hop, U, phi, chi, kappa=0.12):
    """<chi, g5 M g5 phi> = <M chi, phi> for M = 1 - kappa H."""
    g5 = np.diag([1, 1, -1, -1]).astype(complex)
    g = lambda v: np.einsum("st,...tc->...sc", g5, v)
    M = lambda v: v - kappa * hop(U, v, -1)
    a = np.vdot(chi, g(M(g(phi))))
    b = np.vdot(M(chi), phi)
    return float(abs(a - b) / (np.linalg.norm(chi) * np.linalg.norm(phi)))


def space_translation_error(hop, U, phi):
    """Shifting phi and U by one site in x shifts the result (periodic in space)."""
    sh = lambda f: np.roll(f, 1, axis=3)
    return _rel(hop(sh(U), sh(phi), -1), sh(hop(U, phi, -1)))


def time_translation_error(hop, U, phi):
    """A one-step shift in t of the antiperiodic extension commutes with H."""

    def sh(f, sign):
        g = np.roll(f, 1, axis=0)
        g[0] *= sign
        return g

    return _rel(hop(sh(U, 1), sh(phi, -1), -1), sh(hop(U, phi, -1), -1))
