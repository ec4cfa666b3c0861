"""Pins of the BP-regauging oracle (``oracle.bp``) against values that do not come from it.

* A gauge transformation leaves the state unchanged: on the 10-site torus cell
  (short loops, truncated) the contracted state vector before and after the
  regauge is the same ray.
* On a tree, BP is exact: from a random gauge (random invertible matrices on
  every bond, random lambda), the regauge recovers the Schmidt spectrum of the
  state vector across every bond, and the mean-field <Z_i> becomes the exact
  value (Vidal canonical form).
* On a loopy lattice, the BP gauge is the fixed point of the simple update
  with identity gates (the equivalence of simple update and BP gauging cited
  by the paper): both give the same lambda and <Z>.
* After the gauge the BP messages are the identity (normalised), and a second
  regauge changes nothing; the iteration stays at its fixed point.
* Planted mistakes in the oracle break at least one pin.
"""
import copy
import string

import networkx as nx
import numpy as np
import pytest

from oracle import bp, su
from oracle import statevector as sv
from workloads import EAGLE, heavy_hex, heavy_hex_cell, induced_subgraph

M127, E127 = heavy_hex(*EAGLE)
TREE16 = induced_subgraph(E127, range(16))
_ORIG_MESSAGE = bp.message


def peps_state(peps):
    """The state vector of a small gPEPS: every Gamma contracted, lambda_e on each bond."""
    letters = iter(string.ascii_letters)
    phys = [next(letters) for _ in range(peps.n)]
    bond = [next(letters) for _ in range(len(peps.edges))]
    ops, subs = [], []
    for i in range(peps.n):
        T = peps.gamma[i]
        for p, k in enumerate(peps.nb[i]):
            if i < k:
                shape = [1] * T.ndim
                shape[p + 1] = peps.D
                T = T * peps.lam[peps.edge_of[(i, k)]].reshape(shape)
        ops.append(T)
        subs.append(phys[i] + "".join(bond[peps.edge_of[(i, k)]] for k in peps.nb[i]))
    return np.einsum(",".join(subs) + "->" + "".join(phys), *ops, optimize="greedy").reshape(-1)


def cell_state(D=4, steps=3, theta=0.7):
    m, e = heavy_hex_cell()
    peps = su.GPEPS(m, e, D)
    for _ in range(steps):
        peps.step(theta)
    return peps


def ray_distance(a, b):
    return 1.0 - abs(np.vdot(a, b)) / (np.linalg.norm(a) * np.linalg.norm(b))


def random_gauge(peps, rng):
    """Gamma_i lambda Gamma_j^T = (Gamma_i X) diag(mu) (X^-1 diag(lambda / mu)) Gamma_j^T:
    a random invertible X and random positive weights mu on every bond."""
    D = peps.D
    for k, (a, b) in enumerate(peps.edges):
        i, j = int(a), int(b)
        X = rng.normal(size=(D, D)) + 1j * rng.normal(size=(D, D)) + 3 * np.eye(D)
        mu = rng.uniform(0.2, 1.0, D)
        mu /= np.linalg.norm(mu)
        peps.gamma[i] = bp._leg_product(peps.gamma[i], peps.leg(i, j), X)
        peps.gamma[j] = bp._leg_product(peps.gamma[j], peps.leg(j, i),
                                        (np.diag(1.0 / mu) @ np.linalg.inv(X) @ np.diag(peps.lam[k])).T)
        peps.lam[k] = mu


def tree_errors():
    """(max |<Z> - exact|, max |lambda - Schmidt|) after a regauge of a randomly gauged tree."""
    m, e, _ = TREE16
    steps, theta, D = 3, 0.75, 8
    peps = su.GPEPS(m, e, D)
    for _ in range(steps):
        peps.step(theta)
    psi = list(sv.kicked_ising_states(m, e, theta, steps))[-1]
    random_gauge(peps, np.random.default_rng(3))
    bp.regauge(peps, 100, 1e-14)
    z_err = float(np.abs(peps.expect_z() - sv.z_expectations(psi)).max())
    g = nx.Graph([tuple(map(int, x)) for x in e])
    lam_err = 0.0
    for k, (a, b) in enumerate(e):
        h = g.copy()
        h.remove_edge(int(a), int(b))
        s = sv.schmidt_values(psi, nx.node_connected_component(h, int(a)))[:D]
        lam = np.zeros(D)
        lam[:len(s)] = s
        lam_err = max(lam_err, float(np.abs(peps.lambdas()[k] - lam).max()))
    return z_err, lam_err


def test_regauge_keeps_the_state_on_a_loopy_lattice():
    peps = cell_state()
    psi0, z0 = peps_state(peps), peps.expect_z()
    it, res = bp.regauge(peps, 200, 1e-13)
    assert res <= 1e-13 and it < 200
    assert ray_distance(psi0, peps_state(peps)) < 1e-13
    assert np.abs(np.linalg.norm(peps.lam, axis=1) - 1.0).max() < 1e-13
    # the mean-field readout does change on a lattice with loops
    assert np.abs(peps.expect_z() - z0).max() > 1e-4


def test_regauge_recovers_schmidt_values_and_exact_z_on_a_tree():
    z_err, lam_err = tree_errors()
    assert z_err < 1e-12
    assert lam_err < 1e-11


def test_bp_gauge_equals_simple_update_with_identity_gates():
    peps = su.GPEPS(M127, E127, 4)
    for _ in range(6):
        peps.step(0.8)
    gauged = copy.deepcopy(peps)
    it, res = bp.regauge(gauged, 200, 1e-13)
    assert res <= 1e-13
    peps.g = np.ones((2, 2), dtype=np.complex128)          # identity two-site gate
    prev = peps.lambdas().copy()
    for _ in range(200):
        for c in range(peps.n_colours):
            peps.zz_layer(c)
        cur = peps.lambdas()
        done = np.abs(cur - prev).max() < 1e-14
        prev = cur.copy()
        if done:
            break
    assert np.abs(peps.lambdas() - gauged.lambdas()).max() < 1e-12
    assert np.abs(peps.expect_z() - gauged.expect_z()).max() < 1e-12


def test_gauged_state_is_a_fixed_point():
    peps = cell_state(D=4, steps=4, theta=0.9)
    bp.regauge(peps, 200, 1e-13)
    lam, z = peps.lambdas().copy(), peps.expect_z()
    msgs, _, _ = bp.messages(peps, 1)
    for (i, p), m in msgs.items():
        r = int(np.count_nonzero(peps.lam[peps.edge_of[(i, peps.nb[i][p])]] > 1e-12))
        ref = np.zeros((peps.D, peps.D))
        ref[:r, :r] = np.eye(r) / r
        assert np.abs(m - ref).max() < 1e-12, (i, p)
    it, _ = bp.regauge(peps, 200, 1e-13)
    assert it <= 2
    assert np.abs(peps.lambdas() - lam).max() < 1e-12
    assert np.abs(peps.expect_z() - z).max() < 1e-12


def test_iteration_stays_at_its_fixed_point():
    peps = cell_state()
    _, _, res = bp.messages(peps, 150, 0.0)
    assert res < 1e-14


def test_exact_regime_needs_no_work():
    """theta = 0: a product state; every message is the projector on the first index."""
    peps = su.GPEPS(M127, E127, 4)
    peps.step(0.0)
    it, res = bp.regauge(peps, 50, 1e-14)
    assert it <= 2
    assert np.all(np.abs(peps.expect_z() - 1.0) < 1e-14)


# ------------------------------------------------------------------ planted mistakes
def test_planted_mistake_environment_without_lambda(monkeypatch):
    def bad(peps, i, p, msgs, support_cut=su.LAMBDA_CUT):
        saved = peps.lam
        peps.lam = np.ones_like(saved)
        try:
            return _ORIG_MESSAGE(peps, i, p, msgs, support_cut)
        finally:
            peps.lam = saved
    monkeypatch.setattr(bp, "message", bad)
    z_err, lam_err = tree_errors()
    assert max(z_err, lam_err) > 1e-6


def test_planted_mistake_environment_conjugated(monkeypatch):
    def bad(peps, i, p, msgs, support_cut=su.LAMBDA_CUT):
        return _ORIG_MESSAGE(peps, i, p, {k: v.conj() for k, v in msgs.items()}, support_cut)
    monkeypatch.setattr(bp, "message", bad)
    z_err, lam_err = tree_errors()
    assert max(z_err, lam_err) > 1e-6


def test_planted_mistake_same_unitary_on_both_ends(monkeypatch):
    peps = cell_state()
    psi0 = peps_state(peps)
    orig_svd = np.linalg.svd

    def bad_svd(C, *a, **k):
        U, S, Vh = orig_svd(C, *a, **k)
        return U, S, U.T                       # conj(V) replaced by U
    with monkeypatch.context() as mp:
        mp.setattr(np.linalg, "svd", bad_svd)
        bp.regauge(peps, 200, 1e-13)
    assert ray_distance(psi0, peps_state(peps)) > 1e-6


def test_planted_mistake_no_hermitian_projection(monkeypatch):
    def bad(peps, i, p, msgs, support_cut=su.LAMBDA_CUT):
        G = peps.gamma[i]
        X = G.conj()
        for q, k in enumerate(peps.nb[i]):
            if q == p:
                continue
            lam = peps.lam[peps.edge_of[(i, k)]]
            E = lam[:, None] * msgs[(k, peps.leg(k, i))] * lam[None, :]
            X = bp._leg_product(X, q, E.T)
        axes = [ax for ax in range(G.ndim) if ax != p + 1]
        m = np.tensordot(G, X, axes=(axes, axes))
        return m / float(np.trace(m).real)
    monkeypatch.setattr(bp, "message", bad)
    peps = cell_state()
    try:
        _, _, res = bp.messages(peps, 150, 0.0)
    except FloatingPointError:
        res = np.inf
    assert res > 1e-6





class _Residue(su.GPEPS):
    """Simple update that leaves rounding residue in the empty directions of a rank-deficient
    bond, as an FP32 eigensolver does: lambda ~ 1e-16 .. 1e-8 there, with random Gamma columns
    at one end (the state changes by less than 1e-8)."""

    def __init__(self, *a, **k):
        self.rng = np.random.default_rng(5)
        super().__init__(*a, **k)

    def bond_update(self, e):
        super().bond_update(e)
        lam = self.lam[e]
        empty = lam <= 1e-10 * lam.max()
        if not empty.any():
            return
        lam[empty] = 10.0 ** self.rng.uniform(-16, -8, int(empty.sum()))
        i, j = int(self.edges[e][0]), int(self.edges[e][1])
        p = self.leg(i, j)
        T = np.moveaxis(self.gamma[i], p + 1, -1).copy()
        idx = np.nonzero(empty)[0]
        shape = T[..., idx].shape
        T[..., idx] = self.rng.normal(size=shape) + 1j * self.rng.normal(size=shape)
        self.gamma[i] = np.moveaxis(T, -1, p + 1)


def _residue_error(support_cut):
    clean = su.GPEPS(M127, E127, 16)
    dirty = _Residue(M127, E127, 16)
    for _ in range(2):                                  # Schmidt rank <= 4 < D
        clean.step(0.6)
        dirty.step(0.6)
    assert np.abs(dirty.expect_z() - clean.expect_z()).max() < 1e-6
    bp.regauge(clean, 100, 1e-13)
    bp.regauge(dirty, 100, 1e-13, support_cut=support_cut)
    return float(np.abs(dirty.expect_z() - clean.expect_z()).max())


def test_messages_live_on_the_lambda_support():
    """Rank-deficient bonds with rounding residue below the support cut in their empty
    directions: the regauge does not see the residue (the FP32 resolution 1e-7)."""
    assert _residue_error(1e-7) < 1e-8


def test_planted_mistake_no_support_restriction():
    assert _residue_error(0.0) > 1e-3
