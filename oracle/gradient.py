"""Derivatives of <Z> with respect to the kick angles (oracle side).

The paper computes no gradients; these are the references of the library's
reverse mode.  ``fd_gradient`` differentiates the FP64 simple-update oracle
(``oracle/su.py``) by central differences.  ``parameter_shift_gradient``
differentiates the exact state vector (``oracle/statevector.py``): each kick
exp(-i theta X/2) has generator X/2 with eigenvalues +-1/2, so the derivative
of an expectation value with respect to one occurrence of theta_i is
[f(theta_i + pi/2) - f(theta_i - pi/2)] / 2 at that occurrence; a per-qubit
angle shared by all steps sums this over the steps.
"""
from __future__ import annotations

import math

import numpy as np

from . import statevector as sv
from . import su


def oracle_loss(n, edges, D, theta, steps, weights):
    """sum_i weights_i <Z_i> after ``steps`` steps of the oracle simple update."""
    peps = su.GPEPS(n, edges, D)
    for _ in range(steps):
        peps.step(theta)
    return float(np.dot(weights, peps.expect_z()))


def fd_gradient(n, edges, D, theta, steps, weights, h=1e-5, qubits=None):
    """Central differences of :func:`oracle_loss` in the angles of ``qubits`` (default all)."""
    theta = np.asarray(theta, dtype=np.float64)
    qubits = range(n) if qubits is None else qubits
    out = {}
    for q in qubits:
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        out[int(q)] = (oracle_loss(n, edges, D, tp, steps, weights) -
                       oracle_loss(n, edges, D, tm, steps, weights)) / (2 * h)
    return out


def statevector_loss(m, edges, theta_steps, weights):
    psi = None
    for psi in sv.kicked_ising_states(m, edges, theta_steps, theta_steps.shape[0]):
        pass
    return float(np.dot(weights, sv.z_expectations(psi)))


def parameter_shift_gradient(m, edges, theta, steps, weights):
    """Exact d(sum_i weights_i <Z_i>)/dtheta_q of the state vector, every qubit q."""
    base = np.broadcast_to(np.asarray(theta, dtype=np.float64), (m,))[None, :].repeat(steps, axis=0)
    g = np.zeros(m)
    for q in range(m):
        for t in range(steps):
            tp, tm = base.copy(), base.copy()
            tp[t, q] += math.pi / 2
            tm[t, q] -= math.pi / 2
            g[q] += 0.5 * (statevector_loss(m, edges, tp, weights) - statevector_loss(m, edges, tm, weights))
    return g
