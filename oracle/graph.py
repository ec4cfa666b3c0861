"""Edge colouring and leg order (oracle side).

The paper's first-order Trotter step (Eq. 2) applies exp(i pi/4 Z_i Z_j) on
every edge; those gates commute, so the exact circuit does not depend on their
order, but truncated simple update does.  The paper does not state an order.
Reading taken here: greedy first-fit edge colouring over the edges sorted by
(smaller label, larger label); colours are applied 0, 1, 2, ...  Each colour
class is a matching, so its bond updates are independent.

Leg order of site i: its neighbours sorted by label.
"""
from __future__ import annotations

import numpy as np


def greedy_colouring(edges):
    """First-fit colour of each edge (edges visited in (min, max) label order).

    Returns an int array aligned with ``edges`` (input order preserved).
    """
    edges = np.asarray(edges)
    order = sorted(range(len(edges)), key=lambda e: (min(edges[e]), max(edges[e])))
    used = {}           # vertex -> set of colours on its edges
    colour = np.full(len(edges), -1, dtype=np.int64)
    for e in order:
        a, b = int(edges[e][0]), int(edges[e][1])
        taken = used.get(a, set()) | used.get(b, set())
        c = 0
        while c in taken:
            c += 1
        colour[e] = c
        used.setdefault(a, set()).add(c)
        used.setdefault(b, set()).add(c)
    return colour


def neighbours(n_qubits, edges):
    """Sorted neighbour list of every site: its leg order."""
    nb = [[] for _ in range(n_qubits)]
    for a, b in np.asarray(edges):
        nb[int(a)].append(int(b))
        nb[int(b)].append(int(a))
    return [sorted(x) for x in nb]
