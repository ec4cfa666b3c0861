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
CELL = "cell"      # the infinite lattice as its 10-site unit cell (heavy_hex_cell)
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


def heavy_hex_coords(rows: int, width: int):
    """Per label of ``heavy_hex(rows, width)``: ``("row", r, c)`` for the qubit of row r in column
    c, ``("bridge", r, c)`` for the bridge of layer r (between rows r and r+1) in column c."""
    out = []
    for r in range(rows):
        lo = 1 if r == rows - 1 else 0
        hi = width - 2 if r == 0 else width - 1
        out += [("row", r, c) for c in range(lo, hi + 1)]
        if r < rows - 1:
            out += [("bridge", r, c) for c in range(0 if r % 2 == 0 else 2, width, 4)]
    return out


# The infinite lattice of the same rule repeats every 4 columns and every 2 rows (the
# bridge offsets alternate 0, 2 between successive row pairs): a unit cell of 8 row qubits
# and 2 bridges, the 10-site cell of the paper's infinite-lattice simulations ("Method").
CELL_COORDS = ([("row", 0, c) for c in range(4)] + [("bridge", 0, 0)]
               + [("row", 1, c) for c in range(4)] + [("bridge", 1, 2)])


def heavy_hex_cell():
    """The infinite heavy-hex lattice as its translation-invariant 10-site unit cell with
    periodic couplers (a 10-vertex, 12-edge graph on a torus).

    Labels left to right, top to bottom (``CELL_COORDS``): row 0 = 0..3, the bridge of layer 0
    (column 0, between rows 0 and 1) = 4, row 1 = 5..8, the bridge of layer 1 (column 2, between
    row 1 and row 0 of the next cell down) = 9.  Rows close on themselves after 4 columns.  The
    simple update of a translation-invariant state on the infinite lattice updates each coupler
    class of this cell once per colour, so it is the simple update of this graph.
    Returns ``(10, edges)`` like :func:`heavy_hex`."""
    e = [(0, 1), (1, 2), (2, 3), (3, 0), (5, 6), (6, 7), (7, 8), (8, 5),
         (0, 4), (4, 5), (7, 9), (9, 2)]
    return 10, np.array(sorted((min(a, b), max(a, b)) for a, b in e), dtype=np.int32)


# Colour class of each coupler of heavy_hex_cell() (in its sorted edge order): the pattern that
# the greedy colouring of the finite lattices (edges sorted by label, first fit) takes in their
# interior, which repeats with the cell's period, so the infinite lattice is updated in the same
# order as the bulk of the finite ones.  The greedy rule applied to the 12 cell edges themselves
# would need a fourth colour.
CELL_COLOUR = {(0, 1): 1, (0, 3): 0, (0, 4): 2, (1, 2): 2, (2, 3): 1, (2, 9): 0,
               (4, 5): 0, (5, 6): 1, (5, 8): 2, (6, 7): 0, (7, 8): 1, (7, 9): 2}


def heavy_hex_cell_colour():
    """int array of the colour class of every edge of heavy_hex_cell(), in its edge order."""
    _, e = heavy_hex_cell()
    return np.array([CELL_COLOUR[(int(a), int(b))] for a, b in e], dtype=np.int64)


def equivalent_site(rows: int, width: int, cell_site: int, row_near: int, col_near: int):
    """A label of ``heavy_hex(rows, width)`` occupying the place of cell site ``cell_site`` (same
    kind, row parity and column modulo 4), near (row_near, col_near)."""
    kind, r0, c0 = CELL_COORDS[cell_site]
    best = None
    for lab, (k, r, c) in enumerate(heavy_hex_coords(rows, width)):
        if k == kind and r % 2 == r0 % 2 and c % 4 == c0:
            d = abs(r - row_near) + abs(c - col_near)
            if best is None or d < best[0]:
                best = (d, lab)
    return best[1]


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
