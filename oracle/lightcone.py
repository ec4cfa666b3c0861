"""Exact <Z_q> after n steps from the backward light cone of q (App. C argument).

In the Heisenberg picture U^{dagger n} Z_q U^n only involves gates inside the
graph ball of radius n-1 around q (each step's ZZ layer widens the support of
the evolved operator by one edge; the kick does not).  So the circuit restricted
to that ball, with its induced edges, gives <Z_q> exactly.  On the heavy-hex
lattices those balls hold at most 19 qubits for n <= 5.
"""
from __future__ import annotations

import numpy as np

from workloads.heavyhex import graph_ball, induced_subgraph

from .statevector import back_evolved_z_cancelled, kicked_ising_states


def lightcone_z(n_qubits, edges, theta, q, n):
    """Exact <Z_q> after n Trotter steps; ``theta`` scalar or per qubit (full lattice)."""
    if n == 0:
        return 1.0
    ball = graph_ball(n_qubits, edges, q, n - 1)
    m, sub, verts = induced_subgraph(edges, ball)
    th = np.broadcast_to(np.asarray(theta, dtype=np.float64), (n_qubits,))[verts]
    psi = None
    for psi in kicked_ising_states(m, sub, th, n):
        pass
    k = verts.index(int(q))
    p = np.abs(psi) ** 2
    pq = np.ascontiguousarray(np.moveaxis(p, k, 0)).reshape(2, -1).sum(axis=1)
    return float((pq[0] - pq[1]) / (pq[0] + pq[1]))


def lightcone_weight_z(n_qubits, edges, theta, q, n):
    """Exact <Z_q> of |omega(theta, n)> = U^dagger(pi/2)^n |psi(theta, n)> (App. B).

    The last forward and the first inverse ZZ layer cancel, leaving 2n - 2 ZZ
    layers and a kick last, so U-conjugation of Z_q reaches the ball of radius
    2n - 2 around q and no further; the circuit on that ball with its induced
    edges gives the value exactly."""
    if n == 0:
        return 1.0
    ball = graph_ball(n_qubits, edges, q, max(2 * n - 2, 0))
    m, sub, verts = induced_subgraph(edges, ball)
    th = np.broadcast_to(np.asarray(theta, dtype=np.float64), (n_qubits,))[verts]
    z = back_evolved_z_cancelled(m, sub, th, n)
    return float(z[verts.index(int(q))])
