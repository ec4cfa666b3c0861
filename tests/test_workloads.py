"""Pins of the heavy-hex input graphs against the paper's printed facts."""
import json
import os

import networkx as nx
import numpy as np
import pytest

from oracle.pauli import forward_conjugate, support
from workloads import CONDOR, EAGLE, LATTICES, OSPREY, graph_ball, heavy_hex, induced_subgraph

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "weight_operators.json")))


@pytest.mark.parametrize("n,edges_expected,deg", [
    (127, 144, (2, 89, 36)), (433, 504, (2, 287, 144)), (1121, 1320, (2, 719, 400))])
def test_sizes_and_degrees(n, edges_expected, deg):
    m, e = heavy_hex(*LATTICES[n])
    assert m == n and len(e) == edges_expected
    d = np.bincount(e.ravel(), minlength=m)
    assert tuple(np.bincount(d)[1:]) == deg
    assert len({tuple(x) for x in e}) == len(e) and np.all(e[:, 0] < e[:, 1])
    g = nx.Graph([tuple(x) for x in e])
    assert nx.is_connected(g) and nx.is_bipartite(g)
    # every coupler has an end of degree <= 2 (no edge joins two degree-3 qubits)
    assert np.all(np.minimum(d[e[:, 0]], d[e[:, 1]]) <= 2)


@pytest.mark.parametrize("key", ["W10_127", "W17_127"])
def test_weight_operators_app_b(key):
    """App. B, Eqs. (4)-(5): U^5 Z_q U^-5 at theta_h = pi/2 is exactly the printed operator."""
    w = GOLD[key]
    m, e = heavy_hex(*EAGLE)
    x, z = forward_conjugate(m, e, w["q"], w["steps"])
    sup = support(x, z)
    assert sup == {"X": w["X"], "Y": w["Y"], "Z": w["Z"]}


@pytest.mark.parametrize("size", ["127", "433", "1121"])
def test_table1_P_labels_have_weight_10(size):
    m, e = heavy_hex(*LATTICES[int(size)])
    x, z = forward_conjugate(m, e, GOLD["table1_P"][size], 5)
    assert int(np.count_nonzero(x | z)) == GOLD["table1_P_weight"]


def test_reverse_gate_order_does_not_reproduce_w10():
    """The kick-then-ZZ order of Eq. (2) matters: conjugating ZZ first gives another operator."""
    from oracle import pauli
    m, e = heavy_hex(*EAGLE)
    e64 = np.asarray(e, dtype=np.int64)
    x = np.zeros(m, np.uint8); z = np.zeros(m, np.uint8); z[13] = 1
    for _ in range(5):
        pauli._zz(x, z, e64)
        pauli._kick(x, z)
    assert int(np.count_nonzero(x | z)) != 10


def test_local_tree_structure_app_c():
    """App. C: on the 127 lattice every ball of radius <= 5 is a tree; loops appear beyond."""
    m, e = heavy_hex(*EAGLE)
    for r in (1, 2, 3, 4, 5):
        for q in range(m):
            k, sub, _ = induced_subgraph(e, graph_ball(m, e, q, r))
            assert len(sub) == k - 1          # connected with k-1 edges: a tree
    loops = 0
    for q in range(m):
        k, sub, _ = induced_subgraph(e, graph_ball(m, e, q, 6))
        loops += len(sub) >= k
    assert loops > 0
