"""Brute-force state vectors of the kicked Ising circuit (paper Eqs. 2-3).

|psi(theta, n)> = U(theta)^n |0>^m with U = (prod_edges exp(i pi/4 Z_i Z_j)) (prod_i exp(-i theta_i X_i / 2)).
Only for small m (<= ~22 qubits).  Two independent constructions:
``kicked_ising_z`` works on the (2,)*m tensor axis by axis; ``dense_unitary``
builds U as a 2^m x 2^m matrix from Kronecker products (m <= ~10).
"""
from __future__ import annotations

import math

import numpy as np


def _rx(theta):
    c, s = math.cos(theta / 2.0), math.sin(theta / 2.0)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def _zz_diagonal(m, edges, sign):
    """exp(sign * i pi/4 * sum_edges z_a z_b) over the computational basis, shape (2,)*m."""
    z = np.array([1.0, -1.0])
    acc = np.zeros((2,) * m)
    for a, b in np.asarray(edges).reshape(-1, 2):
        shape = [1] * m
        sa = list(shape); sa[int(a)] = 2
        sb = list(shape); sb[int(b)] = 2
        acc = acc + z.reshape(sa) * z.reshape(sb)
    return np.exp(sign * 1j * math.pi / 4.0 * acc)


def kicked_ising_states(m, edges, theta, steps, zz_sign=+1.0):
    """Yield the state tensor (shape (2,)*m) after each Trotter step.

    ``theta``: scalar, per qubit (m,), or per step and qubit (steps, m)."""
    th = np.asarray(theta, dtype=np.float64)
    th = th if th.ndim == 2 else np.broadcast_to(th, (m,))[None, :].repeat(steps, axis=0)
    psi = np.zeros((2,) * m, dtype=np.complex128)
    psi[(0,) * m] = 1.0
    phase = _zz_diagonal(m, edges, zz_sign)
    for t in range(steps):
        for q in range(m):
            psi = np.moveaxis(np.tensordot(_rx(th[t, q]), psi, axes=(1, q)), 0, q)
        psi = psi * phase
        yield psi


def z_expectations(psi):
    """<Z_q> for every axis q of the state tensor."""
    m = psi.ndim
    p = np.abs(psi) ** 2
    out = np.empty(m)
    for q in range(m):
        # contiguous rows so that numpy sums pairwise (a plain running sum over
        # 2^19 terms loses ~1e-12)
        pq = np.ascontiguousarray(np.moveaxis(p, q, 0)).reshape(2, -1).sum(axis=1)
        out[q] = (pq[0] - pq[1]) / (pq[0] + pq[1])
    return out


def kicked_ising_z(m, edges, theta, steps, zz_sign=+1.0):
    """<Z_q> after each step: array of shape (steps, m)."""
    return np.array([z_expectations(psi) for psi in kicked_ising_states(m, edges, theta, steps, zz_sign)])


def dense_unitary(m, edges, theta, zz_sign=+1.0):
    """U(theta) of Eq. 2 as a dense 2^m x 2^m matrix (qubit 0 = most significant bit)."""
    th = np.broadcast_to(np.asarray(theta, dtype=np.float64), (m,))
    K = np.array([[1.0 + 0j]])
    for q in range(m):
        K = np.kron(K, _rx(th[q]))
    z = np.array([1.0, -1.0])
    diag = np.zeros(2 ** m)
    for a, b in np.asarray(edges).reshape(-1, 2):
        za = np.ones(1)
        for q in range(m):
            za = np.kron(za, z if q in (int(a), int(b)) else np.ones(2))
        diag += za
    return np.diag(np.exp(zz_sign * 1j * math.pi / 4.0 * diag)) @ K


def _kick_all(psi, theta):
    m = psi.ndim
    th = np.broadcast_to(np.asarray(theta, dtype=np.float64), (m,))
    for q in range(m):
        psi = np.moveaxis(np.tensordot(_rx(th[q]), psi, axes=(1, q)), 0, q)
    return psi


def back_evolved_z(m, edges, theta_h, n):
    """<Z_q> of |omega> = U^dagger(pi/2)^n U(theta_h)^n |0> (App. B), built literally: n forward
    steps, then n inverse steps (the ZZ layer with the opposite phase, then the kick by -pi/2)."""
    psi = None
    for psi in kicked_ising_states(m, edges, theta_h, n):
        pass
    if psi is None:
        psi = np.zeros((2,) * m, dtype=np.complex128)
        psi[(0,) * m] = 1.0
    inv_phase = _zz_diagonal(m, edges, -1.0)
    for _ in range(n):
        psi = _kick_all(psi * inv_phase, -math.pi / 2)
    return z_expectations(psi)


def back_evolved_z_cancelled(m, edges, theta_h, n):
    """The same state built from U^dagger(pi/2) U(theta_h) = K(theta_h - pi/2) (the ZZ layers of
    the last forward and first inverse step cancel): U^dagger(pi/2)^(n-1) K(theta_h - pi/2)
    U(theta_h)^(n-1) |0>.  ``theta_h`` scalar or per qubit."""
    psi = np.zeros((2,) * m, dtype=np.complex128)
    psi[(0,) * m] = 1.0
    if n >= 2:
        for psi in kicked_ising_states(m, edges, theta_h, n - 1):
            pass
    th = np.broadcast_to(np.asarray(theta_h, dtype=np.float64), (m,))
    psi = _kick_all(psi, th - math.pi / 2)
    inv_phase = _zz_diagonal(m, edges, -1.0)
    for _ in range(n - 1):
        psi = _kick_all(psi * inv_phase, -math.pi / 2)
    return z_expectations(psi)


def schmidt_values(psi, part_a):
    """Schmidt coefficients of the state tensor across (part_a | rest), sorted descending."""
    m = psi.ndim
    a = sorted(part_a)
    b = [q for q in range(m) if q not in set(a)]
    M = np.transpose(psi, a + b).reshape(2 ** len(a), 2 ** len(b))
    return np.linalg.svd(M, compute_uv=False)
