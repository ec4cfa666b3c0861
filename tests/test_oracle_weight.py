"""Pins of the Weight-N oracle (App. B): <Z_P> after n forward steps at theta_h and n inverse
steps at pi/2 is <psi(theta_h, n)| U^n(pi/2) Z_P U^dagger(pi/2)^n |psi(theta_h, n)>.

Pinned against: that definition built from dense unitaries (a 10-qubit tree); the Pauli string of
Clifford propagation (the App. B Weight-N string, up to its dropped sign); the state vector of the
literal back-evolution on a 16-qubit tree where the untruncated simple update is exact; exact light
cones on the full 127-qubit lattice; theta_h = pi/2, where |omega> = |0...0>; and planted
mistakes in the inverse step (gate sign, colour order, kick before the ZZ layer) that must fail.
"""
import math

import numpy as np
import pytest

from oracle import statevector as sv
from oracle import su, weight
from oracle.lightcone import lightcone_weight_z
from oracle.pauli import forward_conjugate
from workloads import EAGLE, heavy_hex, induced_subgraph

M127, E127 = heavy_hex(*EAGLE)


def _expect_pauli(psi, x, z):
    """<psi| X^x Z^z-string (Y = XZ up to phase) |psi> with the phase of each Y as i X Z."""
    m = psi.ndim
    phi = psi.copy()
    for q in range(m):
        if z[q]:
            sgn = np.array([1.0, -1.0]).reshape([2 if k == q else 1 for k in range(m)])
            phi = phi * sgn
        if x[q]:
            phi = np.flip(phi, axis=q)
        if x[q] and z[q]:
            phi = phi * 1j
    return complex(np.vdot(psi.reshape(-1), phi.reshape(-1)))


def test_back_evolution_is_the_conjugated_operator_dense():
    """10-qubit heavy-hex tree: <omega|Z_P|omega> = <psi|U^n Z_P U^{dagger n}|psi> with U(pi/2) and
    psi(theta_h, n) built from dense 2^10 x 2^10 unitaries (Eq. 2)."""
    m, e, _ = induced_subgraph(E127, range(10))
    theta, n = 0.6, 3
    Ut = sv.dense_unitary(m, e, theta)
    Uc = sv.dense_unitary(m, e, math.pi / 2)
    psi = np.zeros(2 ** m, dtype=complex)
    psi[0] = 1.0
    for _ in range(n):
        psi = Ut @ psi
    Un = np.linalg.matrix_power(Uc, n)
    zb = sv.back_evolved_z(m, e, theta, n)
    for p in range(m):
        zd = np.array([1.0 - 2.0 * ((k >> (m - 1 - p)) & 1) for k in range(2 ** m)])
        W = Un @ np.diag(zd) @ Un.conj().T
        assert abs(np.vdot(psi, W @ psi) - zb[p]) < 1e-12


def test_weight_string_from_clifford_propagation():
    """The Pauli string U^n Z_P U^{dagger n} of Clifford propagation (signs dropped) has the same
    expectation in |psi(theta_h, n)> up to sign (16-qubit tree, n = 2 and 3)."""
    m, e, _ = induced_subgraph(E127, range(16))
    theta = 0.7
    for n in (2, 3):
        psi = None
        for psi in sv.kicked_ising_states(m, e, theta, n):
            pass
        zb = sv.back_evolved_z(m, e, theta, n)
        for p in (0, 5, 9, 14):
            x, z = forward_conjugate(m, e, p, n)
            val = _expect_pauli(psi, x, z)
            assert abs(val.imag) < 1e-12
            assert abs(abs(val.real) - abs(zb[p])) < 1e-12


@pytest.mark.parametrize("n", [1, 2])
def test_simple_update_exact_on_tree(n):
    """Untruncated simple update (D = 2^(2n)) on a 16-qubit tree equals the state vector."""
    m, e, _ = induced_subgraph(E127, range(16))
    z = weight.weight_z(m, e, 2 ** (2 * n), 0.6, n)
    assert np.abs(z - sv.back_evolved_z(m, e, 0.6, n)).max() < 1e-12


def test_full_lattice_matches_lightcone():
    """127 qubits, n = 2, D = 16: every qubit equals its exact light-cone value (radius-2 balls are
    trees), among them P = 13 and Q = 58 of App. B."""
    z = weight.weight_z(M127, E127, 16, 0.6, 2)
    for q in list(range(0, M127, 7)) + [13, 58, 62]:
        assert abs(z[q] - lightcone_weight_z(M127, E127, 0.6, q, 2)) < 1e-10, q


def test_clifford_point_returns_to_the_product_state():
    """theta_h = pi/2: U^dagger(pi/2)^n U(pi/2)^n = 1, so every <Z> is 1 (n = 2, D = 16)."""
    z = weight.weight_z(M127, E127, 16, math.pi / 2, 2)
    assert np.abs(z - 1.0).max() < 1e-12


# ------------------------------------------------------------------ planted mistakes
def _weight_z_variant(m, e, D, theta, n, sign=-1.0, reverse=True, kick_first=False):
    peps = su.GPEPS(m, e, D)
    for _ in range(n):
        peps.step(theta)
    peps.g = su.zz_phase(sign)
    order = list(reversed(range(peps.n_colours))) if reverse else list(range(peps.n_colours))
    for _ in range(n):
        if kick_first:
            peps.kick(-math.pi / 2)
        for c in order:
            peps.zz_layer(c)
        if not kick_first:
            peps.kick(-math.pi / 2)
    return peps.expect_z()


def test_unmodified_variant_equals_oracle():
    m, e, _ = induced_subgraph(E127, range(16))
    assert np.abs(_weight_z_variant(m, e, 16, 0.6, 2) - weight.weight_z(m, e, 16, 0.6, 2)).max() < 1e-14


@pytest.mark.parametrize("mistake", [dict(sign=+1.0), dict(kick_first=True)])
def test_planted_mistakes_fail_the_state_vector(mistake):
    m, e, _ = induced_subgraph(E127, range(16))
    ref = sv.back_evolved_z(m, e, 0.6, 2)
    assert np.abs(_weight_z_variant(m, e, 16, 0.6, 2, **mistake) - ref).max() > 1e-3


def test_colour_order_is_a_reading_not_a_pin():
    """Untruncated, the ZZ factors commute, so the order of the classes in the inverse step
    changes nothing (it is a reading of the paper, not pinned); truncated it does."""
    m, e, _ = induced_subgraph(E127, range(16))
    a = _weight_z_variant(m, e, 16, 0.6, 2, reverse=False)
    assert np.abs(a - sv.back_evolved_z(m, e, 0.6, 2)).max() < 1e-12
    b1 = _weight_z_variant(M127, E127, 4, 0.6, 3, reverse=True)
    b2 = _weight_z_variant(M127, E127, 4, 0.6, 3, reverse=False)
    assert np.abs(b1 - b2).max() > 1e-8
