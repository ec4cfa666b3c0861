"""Weight-N observables by Clifford back-evolution (App. B).  TEST INFRASTRUCTURE ONLY.

At theta_h = pi/2 every factor of U (Eq. 2) is Clifford, so W = U^n(pi/2) Z_P
U^{dagger n}(pi/2) is a Pauli string of higher weight (App. B gives the
Weight-10 and Weight-17 strings of the 127-qubit lattice for n = 5, P = 13 and
58; Table I lists P and Q for the other lattices).  Its expectation in
|psi(theta_h, n)> is the single-site <Z_P> of

    |omega(theta_h, n)> = U^{dagger}(pi/2)^n |psi(theta_h, n)>,

which the simple update computes like any other state: n forward steps at
theta_h, then n inverse steps.  U(theta) applies the kick first and then the
ZZ layer, so U^dagger(theta) applies the ZZ layer with the opposite phase
exp(-i pi/4 Z Z) first and then the kick exp(+i theta X / 2).  Reading (the
paper is silent on it): in the inverse step the colour classes are taken in
the reverse order of the forward step.
"""
from __future__ import annotations

import math

import numpy as np

from .su import GPEPS, zz_phase


def inverse_steps(peps, theta, n):
    """Apply U^dagger(theta)^n to the oracle state ``peps`` (App. B)."""
    g_forward = peps.g
    peps.g = zz_phase(-1.0)
    try:
        for _ in range(n):
            for c in reversed(range(peps.n_colours)):
                peps.zz_layer(c)
            peps.kick(-np.asarray(theta, dtype=np.float64))
    finally:
        peps.g = g_forward


def weight_z(n_qubits, edges, D, theta_h, n, colour=None):
    """<Z_i> of |omega(theta_h, n)> for every qubit i (simple update, mean-field readout)."""
    peps = GPEPS(n_qubits, edges, D, colour=colour)
    for _ in range(n):
        peps.step(theta_h)
    inverse_steps(peps, math.pi / 2, n)
    return peps.expect_z()
