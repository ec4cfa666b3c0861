"""Pins of the brute-force state vector against closed forms and a second construction."""
import math

import numpy as np
import pytest

from oracle import statevector as sv
from oracle.lightcone import lightcone_z
from workloads import EAGLE, heavy_hex, induced_subgraph


def test_single_qubit_closed_form():
    th = 0.37
    z = sv.kicked_ising_z(1, np.zeros((0, 2), int), th, 6)
    assert np.allclose(z[:, 0], [math.cos((k + 1) * th) for k in range(6)], atol=1e-14)


def test_two_qubit_closed_form():
    """Two coupled qubits: <Z_0> = cos(theta) after one step and cos(theta)^2 after two."""
    th = 0.81
    z = sv.kicked_ising_z(2, np.array([[0, 1]]), th, 2)
    assert abs(z[0, 0] - math.cos(th)) < 1e-14
    assert abs(z[1, 0] - math.cos(th) ** 2) < 1e-14


@pytest.mark.parametrize("th,expect", [(0.0, lambda n: 1.0), (math.pi, lambda n: (-1.0) ** n)])
def test_trivial_angles(th, expect):
    m, e = 6, np.array([[0, 1], [1, 2], [2, 3], [3, 4], [4, 5], [5, 0]])
    z = sv.kicked_ising_z(m, e, th, 4)
    for n in range(4):
        assert np.allclose(z[n], expect(n + 1), atol=1e-13)


def test_against_dense_unitary_on_a_loop():
    """Axis-by-axis evolution equals the dense Kronecker-product U of Eq. 2 (6-cycle + chord)."""
    m = 7
    e = np.array([[0, 1], [1, 2], [2, 3], [3, 4], [4, 5], [0, 5], [2, 6]])
    th = np.linspace(0.2, 1.1, m)
    U = sv.dense_unitary(m, e, th)
    assert np.allclose(U.conj().T @ U, np.eye(2 ** m), atol=1e-12)
    psi = np.zeros(2 ** m, complex); psi[0] = 1
    zs = sv.kicked_ising_z(m, e, th, 3)
    for n in range(3):
        psi = U @ psi
        p = np.abs(psi) ** 2
        for q in range(m):
            bit = (np.arange(2 ** m) >> (m - 1 - q)) & 1
            assert abs((p * (1 - 2 * bit)).sum() - zs[n, q]) < 1e-12


def test_clifford_point_zero_magnetisation():
    """theta_h = pi/2 (App. B Clifford point): <Z_q> = 0 on a heavy-hex fragment."""
    m0, e0 = heavy_hex(*EAGLE)
    m, sub, _ = induced_subgraph(e0, range(18))
    z = sv.kicked_ising_z(m, sub, math.pi / 2, 4)
    assert np.abs(z).max() < 1e-12


def test_lightcone_equals_full_state_on_a_loopy_fragment():
    """Restricting the circuit to the radius-(n-1) ball of q leaves <Z_q> unchanged."""
    m0, e0 = heavy_hex(*EAGLE)
    # 20 qubits that contain the first hexagon of the lattice (a 12-cycle)
    m, sub, verts = induced_subgraph(e0, list(range(0, 6)) + [14, 15, 18, 19, 20, 21, 22] + list(range(23, 30)))
    assert len(sub) >= m                                          # has a loop
    th = np.linspace(0.3, 1.0, m)
    full = sv.kicked_ising_z(m, sub, th, 4)
    for q in (0, 3, 7, 12):
        for n in (1, 2, 3, 4):
            assert abs(lightcone_z(m, sub, th, q, n) - full[n - 1, q]) < 1e-12
