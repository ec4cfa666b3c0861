"""Heavy-hexagon coupling graphs of the 127-, 433- and 1121-qubit processors.

Paper, section "Method" and Fig. 1: finite heavy-hexagon lattices with open
boundaries whose vertices (qubits) and links (couplers) match Eagle (127),
Osprey (433) and Condor (1121).  Fig. 2 caption: qubits are labelled "left to
right and top to bottom, starting with 0".

The figure itself is not machine readable, so the graph is built from a
row/bridge rule:

* ``rows`` rows of ``width`` columns.  Row 0 holds columns 0..width-2, the
  last row holds columns 1..width-1, every other row holds 0..width-1;
  neighbouring columns of a row are coupled.
* Between row r and row r+1 sits a layer of bridge qubits, at columns
  0, 4, 8, ... when r is even and 2, 6, 10, ... when r is odd.  A bridge is
  coupled to the qubit of row r and the qubit of row r+1 in its column.
* Labels: row 0 left to right, then the bridges between rows 0 and 1 left to
  right, then row 1, and so on.

(7, 15) gives 127 qubits / 144 couplers, (13, 27) gives 433 / 504 and
(21, 43) gives 1121 / 1320.  The tests pin this rule against the Weight-10 and
Weight-17 operators of App. B, Eq. (4) and the P labels of Table I.
"""
from __future__ import annotations

from collections import deque

import numpy as np

EAGLE = (7, 15)
OSPREY = (13, 27)
CONDOR = (21, 43)
LATTICES = {127: EAGLE, 433: OSPREY, 1121: CONDOR}


def heavy_hex(rows: int, width: int):
    """Return ``(n_qubits, edges)`` of the heavy-hex lattice.

    ``edges`` is an int32 array of shape (E, 2) with ``edges[e, 0] < edges[e, 1]``,
    sorted lexicographically.
    """
    if rows < 2 or width < 3:
        raise ValueError("heavy_hex needs rows >= 2 and width >= 3")
    label = 0
    row_label = []          # per row: {column: label}
    bridge_cols = []        # per layer: list of (column, label)
    for r in range(rows):
        lo = 1 if r == rows - 1 else 0
        hi = width - 2 if r == 0 else width - 1
        cols = {}
        for c in range(lo, hi + 1):
            cols[c] = label
            label += 1
        row_label.append(cols)
        if r < rows - 1:
            start = 0 if r % 2 == 0 else 2
            layer = []
            for c in range(start, width, 4):
                layer.append((c, label))
                label += 1
            bridge_cols.append(layer)
    edges = []
    for r in range(rows):
        cols = sorted(row_label[r])
        for a, b in zip(cols[:-1], cols[1:]):
            edges.append((row_label[r][a], row_label[r][b]))
    for r, layer in enumerate(bridge_cols):
        for c, b in layer:
            if c not in row_label[r] or c not in row_label[r + 1]:
                raise ValueError(f"bridge column {c} of layer {r} has no row qubit")
            edges.append((row_label[r][c], b))
            edges.append((b, row_label[r + 1][c]))
    e = np.array(sorted((min(a, b), max(a, b)) for a, b in edges), dtype=np.int32)
    return label, e


def induced_subgraph(edges, vertices):
    """Relabel ``vertices`` (sorted) to 0..m-1 and keep only the edges inside them.

    Returns ``(m, sub_edges, vertex_list)``; ``vertex_list[k]`` is the original
    label of new vertex k.
    """
    vs = sorted(int(v) for v in vertices)
    index = {v: k for k, v in enumerate(vs)}
    sub = [(index[int(a)], index[int(b)]) for a, b in np.asarray(edges)
           if int(a) in index and int(b) in index]
    sub = np.array(sorted(sub), dtype=np.int32).reshape(-1, 2)
    return len(vs), sub, vs


def graph_ball(n_qubits, edges, centre, radius):
    """Vertices within graph distance ``radius`` of ``centre`` (breadth-first search)."""
    adj = [[] for _ in range(n_qubits)]
    for a, b in np.asarray(edges):
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    dist = {int(centre): 0}
    q = deque([int(centre)])
    while q:
        v = q.popleft()
        if dist[v] == radius:
            continue
        for w in adj[v]:
            if w not in dist:
                dist[w] = dist[v] + 1
                q.append(w)
    return sorted(dist)
