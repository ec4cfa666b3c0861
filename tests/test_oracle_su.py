"""Pins of the simple-update oracle against values that do not come from it.

* Trees, untruncated (D >= 2^n): simple update applies each gate exactly and keeps
  the Vidal canonical form, so the mean-field <Z_i> equals the state-vector value
  and lambda_e equals the Schmidt spectrum across e.
* Full lattices, n <= 5: every light cone is a tree (App. C), so with D >= 2^n
  the oracle matches the light-cone brute force (the paper's ~1e-15 claim of the
  "Benchmarking" section).
* theta_h = 0 (identity), pi (bit flips: product state) and pi/2 (Clifford:
  <Z> = 0, App. B) invariants.
* Planted mistakes in the oracle must break at least one pin.
"""
import math

import networkx as nx
import numpy as np
import pytest

from oracle import statevector as sv
from oracle import su
from oracle.lightcone import lightcone_z
from workloads import EAGLE, OSPREY, heavy_hex, induced_subgraph

M127, E127 = heavy_hex(*EAGLE)


def fragment(verts):
    return induced_subgraph(E127, verts)


TREE16 = fragment(range(16))                    # row 0 + two bridges: a tree with degree-3 sites
TREE20 = fragment(list(range(18)) + [18, 22])   # row 0, four bridges, two qubits of row 1


@pytest.mark.parametrize("frag,theta,steps", [(TREE16, 0.6, 5), (TREE20, 1.0, 4), (TREE16, 0.3, 3)])
def test_tree_matches_statevector(frag, theta, steps):
    m, e, _ = frag
    assert len(e) == m - 1
    D = 2 ** steps
    means, zs, peps = su.evolve(m, e, D, theta, steps, per_site=True)
    ref = sv.kicked_ising_z(m, e, theta, steps)
    assert np.abs(zs - ref).max() < 1e-12
    assert np.abs(means - ref.mean(axis=1)).max() < 1e-12


def test_tree16_printed_means():
    """Mean <Z> of the 16-qubit tree at theta=0.6 (independent state vector, 8 digits)."""
    m, e, _ = TREE16
    means, _, _ = su.evolve(m, e, 32, 0.6, 5)
    assert np.allclose(means, [0.82533561, 0.84405954, 0.79485539, 0.79597706, 0.76800776], atol=5e-9)


def test_tree_lambda_equals_schmidt_values():
    m, e, _ = TREE20
    steps, theta = 3, 0.75
    D = 2 ** steps
    _, _, peps = su.evolve(m, e, D, theta, steps)
    psi = None
    for psi in sv.kicked_ising_states(m, e, theta, steps):
        pass
    g = nx.Graph([tuple(map(int, x)) for x in e])
    for k, (a, b) in enumerate(e):
        h = g.copy(); h.remove_edge(int(a), int(b))
        part = nx.node_connected_component(h, int(a))
        s = sv.schmidt_values(psi, part)[:D]
        lam = np.zeros(D); lam[:len(s)] = s
        assert np.abs(peps.lambdas()[k] - lam).max() < 1e-12


@pytest.mark.parametrize("theta,expect", [(0.0, lambda n: 1.0), (math.pi, lambda n: (-1.0) ** n)])
def test_trivial_angles_full_lattice(theta, expect):
    means, zs, peps = su.evolve(M127, E127, 4, theta, 3, per_site=True)
    for n in range(3):
        assert np.abs(zs[n] - expect(n + 1)).max() < 1e-12
    lam0 = np.zeros(4); lam0[0] = 1
    assert np.abs(peps.lambdas() - lam0).max() < 1e-12


def test_clifford_point_full_lattice():
    """theta_h = pi/2 is Clifford: U^-n Z_i U^n keeps an X or Y factor, so <Z_i> = 0 (D >= 2^n)."""
    from oracle.pauli import backward_conjugate
    for q in range(M127):
        x, _ = backward_conjugate(M127, E127, q, 4)
        assert x.any()
    _, zs, _ = su.evolve(M127, E127, 16, math.pi / 2, 4, per_site=True)
    assert np.abs(zs).max() < 1e-12


@pytest.mark.parametrize("theta", [0.3, 0.6, 1.0])
def test_full_lattice_matches_lightcone(theta):
    steps = 4
    _, zs, _ = su.evolve(M127, E127, 16, theta, steps, per_site=True)
    for n in range(1, steps + 1):
        ref = np.array([lightcone_z(M127, E127, theta, q, n) for q in range(M127)])
        assert np.abs(zs[n - 1] - ref).max() < 1e-12


def test_full_lattice_matches_lightcone_step5():
    """n = 5, D = 32: the setting of the paper's ~1e-15 benchmark (sampled qubits)."""
    theta = 0.8
    _, zs, _ = su.evolve(M127, E127, 32, theta, 5, per_site=True)
    for q in range(0, M127, 9):
        assert abs(zs[4, q] - lightcone_z(M127, E127, theta, q, 5)) < 1e-12


def test_osprey_matches_lightcone():
    m, e = heavy_hex(*OSPREY)
    theta = 0.9
    _, zs, _ = su.evolve(m, e, 8, theta, 3, per_site=True)
    for q in range(0, m, 17):
        assert abs(zs[2, q] - lightcone_z(m, e, theta, q, 3)) < 1e-12


def test_truncation_changes_result_and_conserves_norm():
    """D < 2^n truncates: the result departs from the exact value; lambda stays unit-norm."""
    theta = 1.0
    _, zs, peps = su.evolve(M127, E127, 2, theta, 3, per_site=True)
    ref = np.array([lightcone_z(M127, E127, theta, q, 3) for q in range(M127)])
    assert np.abs(zs[2] - ref).max() > 1e-4
    assert np.allclose(np.linalg.norm(peps.lam, axis=1), 1.0, atol=1e-13)


# ------------------------------------------------------------------ planted mistakes
def _tree_error(cls):
    """Max deviation of <Z_i> and of lambda_e from the state vector (3 steps, D = 8)."""
    m, e, _ = TREE16
    peps = cls(m, e, 8)
    err = 0.0
    g = nx.Graph([tuple(map(int, x)) for x in e])
    for n, psi in enumerate(sv.kicked_ising_states(m, e, 0.7, 3)):
        peps.step(0.7)
        err = max(err, float(np.abs(peps.expect_z() - sv.z_expectations(psi)).max()))
        for k, (a, b) in enumerate(e):
            h = g.copy(); h.remove_edge(int(a), int(b))
            s = sv.schmidt_values(psi, nx.node_connected_component(h, int(a)))[:8]
            lam = np.zeros(8); lam[:len(s)] = s
            err = max(err, float(np.abs(peps.lambdas()[k] - lam).max()))
    return err


def test_unmodified_oracle_is_exact_on_the_tree():
    assert _tree_error(su.GPEPS) < 1e-12


def test_planted_mistake_no_absorb():
    class Bad(su.GPEPS):
        def _absorb(self, i, skip):
            return self.gamma[i]
    assert _tree_error(Bad) > 1e-6


def test_planted_mistake_no_strip():
    class Bad(su.GPEPS):
        def _strip(self, T, i, skip):
            return T
    assert _tree_error(Bad) > 1e-6


def test_planted_mistake_readout_sqrt_lambda():
    class Bad(su.GPEPS):
        def expect_z(self):
            saved = self.lam
            self.lam = np.sqrt(saved)
            try:
                return su.GPEPS.expect_z(self)
            finally:
                self.lam = saved
    assert _tree_error(Bad) > 1e-6


def test_planted_mistake_transposed_gate_phase():
    class Bad(su.GPEPS):
        def __init__(self, *a, **k):
            super().__init__(*a, **k)
            z = np.array([1.0, -1.0])
            self.g = np.exp(1j * math.pi / 4 * np.add.outer(z, np.zeros(2)))   # single-site phase only
    assert _tree_error(Bad) > 1e-6


def test_planted_mistake_zz_before_kick():
    """A trailing ZZ layer commutes with Z_q, so only the lambda spectra can catch this one."""
    class Bad(su.GPEPS):
        def step(self, theta):
            for c in range(self.n_colours):
                self.zz_layer(c)
            self.kick(theta)
    assert _tree_error(Bad) > 1e-6


def test_oracle_gradient_matches_parameter_shift_on_a_tree():
    """Exact regime: central differences of the oracle equal the parameter-shift derivative
    of the state vector (a second, independent derivative)."""
    from oracle.gradient import fd_gradient, parameter_shift_gradient
    m, e, _ = TREE16
    rng = np.random.default_rng(7)
    theta = rng.uniform(0.5, 0.9, m)
    w = np.full(m, 1.0 / m)
    steps = 3
    ps = parameter_shift_gradient(m, e, theta, steps, w)
    fd = fd_gradient(m, e, 8, theta, steps, w, qubits=[0, 3, 4, 9, 14, 15])
    for q, v in fd.items():
        assert abs(v - ps[q]) < 1e-8 * max(1.0, abs(ps[q])), (q, v, ps[q])


def test_parameter_shift_single_qubit_closed_form():
    """One qubit: <Z> = cos(n theta), d/dtheta = -n sin(n theta)."""
    from oracle.gradient import parameter_shift_gradient
    th = 0.41
    g = parameter_shift_gradient(1, np.zeros((0, 2), int), [th], 3, np.ones(1))
    assert abs(g[0] + 3 * math.sin(3 * th)) < 1e-13


# ------------------------------------------------------------------ truncation (Eckart-Young)
# Trees where exactly one edge can exceed the bond dimension D: every other edge
# has a side of at most log2(D) qubits, so its Schmidt rank never exceeds D and
# its updates are exact.  The first update of the chosen edge whose Schmidt rank
# exceeds D is therefore the first truncation of the run, applied to a tree in
# exact Vidal canonical form, where the bond's SVD is the Schmidt decomposition
# of the whole state across that edge.  By Eckart-Young the truncated update must
# keep the D largest Schmidt values of the state-vector state after that gate,
# renormalised to unit 2-norm, and the mean-field <Z> of both ends must be the
# <Z> of the state vector projected onto those D Schmidt components.
EY_CASES = [
    ([1, 2, 3, 4, 5, 6, 15], (3, 4), 4, 0.7),        # degree-3 end (site 4) and degree-2 end
    ([0, 1, 2, 3, 4, 5], (2, 3), 4, 0.9),            # chain: two degree-2 ends
    ([0, 1, 2, 3, 4, 5, 6, 7, 15], (3, 4), 8, 0.8),  # D = 8, rank 16 before the cut
]


def _eckart_young(cls, verts, edge, D, theta):
    """Run ``cls`` gate by gate next to the state vector until the first update of
    ``edge`` whose Schmidt rank exceeds D.  Returns (max |lambda - top-D Schmidt
    values renormalised|, max |<Z>| error at the two ends against the projected
    state, the same ends' |<Z>| change caused by the projection)."""
    m, e, labels = fragment(verts)
    loc = {int(g): k for k, g in enumerate(labels)}
    a, b = loc[edge[0]], loc[edge[1]]
    peps = cls(m, e, D)
    k_e = next(k for k, (x, y) in enumerate(e) if {int(x), int(y)} == {a, b})
    g = nx.Graph([tuple(map(int, x)) for x in e])
    for k, (x, y) in enumerate(e):
        if k != k_e:   # every other edge has a side of <= log2(D) qubits
            h = g.copy(); h.remove_edge(int(x), int(y))
            assert 2 ** min(len(c) for c in nx.connected_components(h)) <= D
    h = g.copy(); h.remove_edge(a, b)
    side = sorted(nx.node_connected_component(h, a))
    rest = [q for q in range(m) if q not in side]
    psi = np.zeros((2,) * m, dtype=np.complex128)
    psi[(0,) * m] = 1.0
    for _ in range(8):
        peps.kick(theta)
        psi = sv._kick_all(psi, theta)
        for c in range(peps.n_colours):
            order = [int(k) for k in np.nonzero(peps.colour == c)[0] if k != k_e]
            if peps.colour[k_e] == c:
                order.append(k_e)            # a colour class is a matching: any order
            for k in order:
                peps.bond_update(k)
                psi = psi * sv._zz_diagonal(m, e[k:k + 1], 1.0)
                if k != k_e:
                    continue
                mat = np.transpose(psi, side + rest).reshape(2 ** len(side), -1)
                U, S, Vh = np.linalg.svd(mat, full_matrices=False)
                if int((S > 1e-12).sum()) <= D:
                    continue
                lam = S[:D] / np.linalg.norm(S[:D])
                lam_err = float(np.abs(peps.lambdas()[k_e] - lam).max())
                proj = (U[:, :D] * S[:D]) @ Vh[:D]
                proj = np.transpose((proj / np.linalg.norm(proj)).reshape((2,) * m), np.argsort(side + rest))
                z_proj, z_full, z = sv.z_expectations(proj), sv.z_expectations(psi), peps.expect_z()
                z_err = max(abs(z[a] - z_proj[a]), abs(z[b] - z_proj[b]))
                moved = min(abs(z_full[a] - z_proj[a]), abs(z_full[b] - z_proj[b]))
                return lam_err, z_err, moved
    raise AssertionError("the edge never exceeded D")


@pytest.mark.parametrize("verts,edge,D,theta", EY_CASES)
def test_truncation_keeps_the_largest_schmidt_values(verts, edge, D, theta):
    lam_err, z_err, moved = _eckart_young(su.GPEPS, verts, edge, D, theta)
    assert lam_err < 1e-13
    assert z_err < 1e-13
    assert moved > 1e-5        # the truncation is visible in <Z>: the pin is not vacuous


class _KeepSmallest(su.GPEPS):
    def _truncate(self, e, U, S, Vh):
        keep = min(self.D, S.size)
        lam = np.zeros(self.D)
        lam[:keep] = S[-keep:] / np.linalg.norm(S[-keep:])
        return U[:, -keep:], Vh[-keep:], lam


class _NormaliseBeforeCut(su.GPEPS):
    def _truncate(self, e, U, S, Vh):
        keep = min(self.D, S.size)
        lam = np.zeros(self.D)
        lam[:keep] = (S / np.linalg.norm(S))[:keep]
        return U[:, :keep], Vh[:keep], lam


class _NoRenormalisation(su.GPEPS):
    def _truncate(self, e, U, S, Vh):
        keep = min(self.D, S.size)
        lam = np.zeros(self.D)
        lam[:keep] = S[:keep]
        return U[:, :keep], Vh[:keep], lam


@pytest.mark.parametrize("bad", [_KeepSmallest, _NormaliseBeforeCut, _NoRenormalisation])
@pytest.mark.parametrize("verts,edge,D,theta", EY_CASES[:2])
def test_planted_truncation_mistakes_fail_eckart_young(bad, verts, edge, D, theta):
    try:
        lam_err, z_err, _ = _eckart_young(bad, verts, edge, D, theta)
    except (np.linalg.LinAlgError, FloatingPointError):
        return   # keeping the smallest values keeps zeros before the first cut: the run breaks down
    assert lam_err > 1e-5 or z_err > 1e-5
