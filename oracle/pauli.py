"""Clifford Pauli propagation of the kicked Ising step at theta_h = pi/2 (App. B).

At theta_h = pi/2 every factor of U (Eq. 2) is Clifford, so U P U^dagger of a
Pauli string P is again a Pauli string (up to sign).  A string is stored as
bit vectors (x, z): X = (1,0), Z = (0,1), Y = (1,1).

Conjugation rules (derived from the commutation relations, signs dropped):
  exp(-i pi/4 X_q):          x_q ^= z_q
  exp(+i pi/4 Z_a Z_b):      if x_a xor x_b: z_a ^= 1 and z_b ^= 1
"""
from __future__ import annotations

import numpy as np


def _kick(x, z):
    x ^= z


def _zz(x, z, edges):
    flip = x[edges[:, 0]] ^ x[edges[:, 1]]
    # every ZZ factor commutes with every other, so the layer acts at once
    np.bitwise_xor.at(z, edges[flip.astype(bool), 0], 1)
    np.bitwise_xor.at(z, edges[flip.astype(bool), 1], 1)


def forward_conjugate(m, edges, q, n):
    """U^n Z_q U^{dagger n} at theta_h = pi/2 (App. B, Eq. 5): returns (x, z) bit arrays."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    x = np.zeros(m, dtype=np.uint8)
    z = np.zeros(m, dtype=np.uint8)
    z[q] = 1
    for _ in range(n):
        _kick(x, z)          # U P U^+ = ZZ (K P K^+) ZZ^+: kick conjugation first
        _zz(x, z, edges)
    return x, z


def backward_conjugate(m, edges, q, n):
    """U^{dagger n} Z_q U^n at theta_h = pi/2: <0|.|0> is nonzero iff no X or Y remains."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    x = np.zeros(m, dtype=np.uint8)
    z = np.zeros(m, dtype=np.uint8)
    z[q] = 1
    for _ in range(n):
        _zz(x, z, edges)     # U^+ P U = K^+ (ZZ^+ P ZZ) K: ZZ conjugation first
        _kick(x, z)
    return x, z


def support(x, z):
    """Dict {'X': [...], 'Y': [...], 'Z': [...]} of qubit labels."""
    return {
        "X": [int(q) for q in np.nonzero((x == 1) & (z == 0))[0]],
        "Y": [int(q) for q in np.nonzero((x == 1) & (z == 1))[0]],
        "Z": [int(q) for q in np.nonzero((x == 0) & (z == 1))[0]],
    }
