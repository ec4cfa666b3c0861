"""Simple update of a graph PEPS (gPEPS) with mean-field <Z> readout, FP64/complex128.

Paper, section "Method": the state is a gPEPS with one tensor per qubit and one
bond per coupler, bond dimension chi (called D here), evolved by the *simple
update* of tensors; expectation values use a *mean-field* approximation of the
environment; chi is also the truncation parameter.  Section "Model", Eqs. (2)-(3):
each Trotter step applies exp(-i theta_h X_i / 2) to every qubit, then
exp(+i pi/4 Z_i Z_j) on every edge; the start is |0...0>.

The paper names these steps but prints no formulas, so this module spells out
the textbook simple update in its usual order, one bond (i, j) at a time:

  absorb   A_i = Gamma_i with the lambda of every other leg of i multiplied in
  QR       A_i = Q_i R_i  (rows: other legs; columns: physical s, bond k)
  gate     Theta[(a,s),(b,t)] = g(s,t) sum_k R_i[a,s,k] lambda_ij[k] R_j[b,t,k]
           with g(s,t) = exp(i pi/4 z_s z_t), z = (+1, -1)
  SVD      Theta = U S V^dagger
  truncate keep the D largest singular values
  renorm   lambda_ij' = S[:D] / ||S[:D]||_2
  strip    Gamma_i' = (Q_i U)[:, :D] divided by the lambda of i's other legs
           (pseudo-inverse: 1/lambda := 0 when lambda <= 1e-13 max(lambda)),
           Gamma_j' likewise from V^dagger.

Mean-field readout of site i: psi_i = Gamma_i times lambda on every leg,
p_s = sum |psi_i[s, ...]|^2, <Z_i> = (p_0 - p_1) / (p_0 + p_1).

Readings where the paper is silent (also listed in the design notes):
lambda normalised to unit 2-norm; lambda (not sqrt(lambda)) on every leg in the
readout; the kick is applied to all sites before the first ZZ layer of a step;
colours are applied in increasing order (``oracle.graph``); leg order of a site
is its neighbours sorted by label; ties at the truncation cut follow LAPACK's
order.

Parity pins: ``tests/test_oracle_su.py`` (state vectors on trees, light cones on
the full lattices, the theta_h = 0, pi/2, pi invariants, and the truncation
branch by Eckart-Young: the first truncated update on a tree in canonical form
keeps the D largest Schmidt values of the state vector, renormalised, and the
<Z> of both ends equals that of the state vector projected onto them).
"""
from __future__ import annotations

import math

import numpy as np

from .graph import greedy_colouring, neighbours

LAMBDA_CUT = 1e-13


def rx(theta):
    """exp(-i theta X / 2) (Eq. 2, single-site factor)."""
    c, s = math.cos(theta / 2.0), math.sin(theta / 2.0)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def zz_phase(sign=+1.0):
    """g[s, t] = exp(sign * i pi/4 z_s z_t) with z = (+1, -1): the diagonal of the
    two-site factor of Eq. 2 (sign = +1 is the paper's)."""
    z = np.array([1.0, -1.0])
    return np.exp(sign * 1j * math.pi / 4.0 * np.outer(z, z))


def _pinv(lam):
    cut = LAMBDA_CUT * float(np.max(lam)) if lam.size else 0.0
    out = np.zeros_like(lam)
    nz = lam > cut
    out[nz] = 1.0 / lam[nz]
    return out


class GPEPS:
    """Graph PEPS of ``n_qubits`` sites on the coupling graph ``edges`` (E x 2)."""

    def __init__(self, n_qubits, edges, D, colour=None, zz_sign=+1.0):
        self.n = int(n_qubits)
        self.edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
        self.D = int(D)
        if self.D < 1:
            raise ValueError("D must be >= 1")
        self.nb = neighbours(self.n, self.edges)
        self.edge_of = {}
        for e, (a, b) in enumerate(self.edges):
            self.edge_of[(int(a), int(b))] = e
            self.edge_of[(int(b), int(a))] = e
        self.colour = (greedy_colouring(self.edges) if colour is None
                       else np.asarray(colour, dtype=np.int64))
        self.n_colours = int(self.colour.max()) + 1 if len(self.edges) else 0
        self.g = zz_phase(zz_sign)
        self.reset()

    # ----------------------------------------------------------------- state
    def reset(self):
        """|0...0>: Gamma_i[0, 0, ..., 0] = 1, lambda_e = (1, 0, ..., 0)."""
        D = self.D
        self.gamma = []
        for i in range(self.n):
            t = np.zeros((2,) + (D,) * len(self.nb[i]), dtype=np.complex128)
            t[(0,) * t.ndim] = 1.0
            self.gamma.append(t)
        self.lam = np.zeros((len(self.edges), D), dtype=np.float64)
        self.lam[:, 0] = 1.0

    def leg(self, i, j):
        """Position of neighbour j among the legs of site i."""
        return self.nb[i].index(j)

    # ----------------------------------------------------------------- gates
    def kick(self, theta):
        """Apply exp(-i theta_i X_i / 2) to every site (Eq. 2); ``theta`` scalar or per qubit."""
        th = np.broadcast_to(np.asarray(theta, dtype=np.float64), (self.n,))
        for i in range(self.n):
            self.gamma[i] = np.tensordot(rx(th[i]), self.gamma[i], axes=(1, 0))

    def _absorb(self, i, skip):
        A = self.gamma[i]
        for p, nbr in enumerate(self.nb[i]):
            if p == skip:
                continue
            lam = self.lam[self.edge_of[(i, nbr)]]
            shape = [1] * A.ndim
            shape[p + 1] = self.D
            A = A * lam.reshape(shape)
        return A

    def _strip(self, T, i, skip):
        for p, nbr in enumerate(self.nb[i]):
            if p == skip:
                continue
            inv = _pinv(self.lam[self.edge_of[(i, nbr)]])
            shape = [1] * T.ndim
            shape[p + 1] = self.D
            T = T * inv.reshape(shape)
        return T

    def bond_update(self, e):
        """Simple update of edge e with the gate exp(i pi/4 Z_i Z_j)."""
        D = self.D
        i, j = int(self.edges[e][0]), int(self.edges[e][1])
        pi, pj = self.leg(i, j), self.leg(j, i)
        mats = []
        for site, p in ((i, pi), (j, pj)):
            A = self._absorb(site, p)                                   # absorb
            nd = A.ndim
            A = np.moveaxis(A, [0, p + 1], [nd - 2, nd - 1])             # (other legs..., s, k)
            other = A.shape[:-2]
            Q, R = np.linalg.qr(A.reshape(-1, 2 * D))                   # QR
            mats.append((Q, R.reshape(R.shape[0], 2, D), other, p))
        (Qi, Ri, oth_i, _), (Qj, Rj, oth_j, _) = mats
        ri, rj = Ri.shape[0], Rj.shape[0]
        lam = self.lam[e]
        theta = np.einsum("ask,k,btk->asbt", Ri, lam, Rj) * self.g[None, :, None, :]   # gate
        theta = theta.reshape(2 * ri, 2 * rj)
        U, S, Vh = np.linalg.svd(theta, full_matrices=False)           # SVD
        U, Vh, lam_new = self._truncate(e, U, S, Vh)                    # truncate + renormalise
        keep = U.shape[1]
        Gi = np.zeros((Qi.shape[0], 2, D), dtype=np.complex128)
        Gi[:, :, :keep] = np.einsum("ma,ask->msk", Qi, U.reshape(ri, 2, keep))
        Gj = np.zeros((Qj.shape[0], 2, D), dtype=np.complex128)
        Gj[:, :, :keep] = np.einsum("mb,kbt->mtk", Qj, Vh.reshape(keep, rj, 2))
        for site, G, oth, p in ((i, Gi, oth_i, pi), (j, Gj, oth_j, pj)):
            nd = len(oth) + 2
            T = np.moveaxis(G.reshape(oth + (2, D)), [nd - 2, nd - 1], [0, p + 1])
            self.gamma[site] = self._strip(T, site, p)                  # strip lambda^-1
        self.lam[e] = lam_new

    def _truncate(self, e, U, S, Vh):
        """Keep the D largest singular values (LAPACK returns them in decreasing
        order) and their vectors; the new lambda is the kept values divided by their
        own 2-norm, zero-padded to D ("Method": chi is the truncation parameter).
        Returns (U[:, :keep], Vh[:keep], lambda')."""
        D = self.D
        keep = min(D, S.size)                                           # truncate
        U, S, Vh = U[:, :keep], S[:keep], Vh[:keep, :]
        nrm = float(np.linalg.norm(S))
        if not np.isfinite(nrm) or nrm == 0.0:
            raise FloatingPointError(f"bond {e}: singular values vanish or are not finite")
        lam_new = np.zeros(D)
        lam_new[:keep] = S / nrm                                        # renormalise
        return U, Vh, lam_new

    def zz_layer(self, c):
        """Simple update of every edge of colour class c (a matching)."""
        for e in np.nonzero(self.colour == c)[0]:
            self.bond_update(int(e))

    def step(self, theta):
        """One Trotter step U(theta) of Eq. 2: kicks first, then ZZ colour by colour."""
        self.kick(theta)
        for c in range(self.n_colours):
            self.zz_layer(c)

    # --------------------------------------------------------------- readout
    def expect_z(self):
        """Mean-field <Z_i> of every site (float64 array of length n)."""
        out = np.empty(self.n)
        for i in range(self.n):
            psi = self.gamma[i]
            for p, nbr in enumerate(self.nb[i]):
                lam = self.lam[self.edge_of[(i, nbr)]]
                shape = [1] * psi.ndim
                shape[p + 1] = self.D
                psi = psi * lam.reshape(shape)
            w = np.abs(psi.reshape(2, -1)) ** 2
            p0, p1 = float(w[0].sum()), float(w[1].sum())
            out[i] = (p0 - p1) / (p0 + p1)
        return out

    def lambdas(self):
        """Bond weights, one row per edge, sorted in decreasing order."""
        return -np.sort(-self.lam, axis=1)


def evolve(n_qubits, edges, D, theta, steps, colour=None, per_site=False, zz_sign=+1.0):
    """Run ``steps`` Trotter steps from |0...0>.

    Returns ``(mean_z[steps], z[steps, n] or None, peps)``.
    """
    peps = GPEPS(n_qubits, edges, D, colour=colour, zz_sign=zz_sign)
    means = np.empty(steps)
    zs = np.empty((steps, peps.n)) if per_site else None
    for t in range(steps):
        peps.step(theta)
        z = peps.expect_z()
        means[t] = z.mean()
        if per_site:
            zs[t] = z
    return means, zs, peps
