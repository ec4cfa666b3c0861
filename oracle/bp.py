"""Belief-propagation (BP) regauging of a gPEPS, FP64/complex128.  TEST INFRASTRUCTURE ONLY.

Paper, section "Method": as a comparison, the PEPS is re-gauged with belief
propagation after each Trotter step, following the BP gauging scheme of the
cited tensor-network study of the same circuit; section "Results",
"Benchmarking": five steps with a BP gauging after each, which leaves the
accuracy unchanged.  The paper prints no formulas, so this module states the
standard BP gauge of the norm network <psi|psi> in the Gamma-lambda form of
``oracle.su``, step by step.

Messages.  Every site i sends along each of its legs (edge e to neighbour j) a
D x D Hermitian matrix over the (ket a, bra a') index pair of that leg:

    m_{i->e}[a, a'] = sum  Gamma_i[s, .., a, .., b, .., c] conj(Gamma_i[s, .., a', .., b', .., c'])
                           E_f[b, b'] E_g[c, c']          (s and every other leg summed)

where E_f = diag(lambda_f) m_{k->f} diag(lambda_f) is the environment of i's
other leg f, built from the message that the neighbour k across f sends along
f.  A message lives on the support of its own bond's lambda_e: the rows and
columns k with lambda_e[k] <= LAMBDA_CUT * max(lambda_e) are zero (the
pseudo-inverse convention of ``oracle.su``, which already treats those
directions as absent; ``support_cut`` sets the threshold).  A low-precision
simple update leaves rounding residue in the empty directions of a
rank-deficient bond: lambda far below its resolution, with Gamma columns that
are rounding noise.  Kept in the messages, that residue sends BP to another
fixed point (a wrong mean-field readout after the gauge), so a path that
stores Gamma in FP32 restricts the messages at its own resolution (1e-7).  All messages start at identity / D; an iteration
recomputes every message from the previous iteration's (parallel schedule),
keeps its Hermitian part (m + m^H) / 2, restricts it to the support and
normalises it to unit trace; iterations stop when the largest
elementwise change is <= tol, or after max_iter.  The exact message is
Hermitian; its rounding noise is not, and an anti-Hermitian multiple of a
message is not removed by the trace normalisation: it spreads along the loops
of the lattice and grows by the growth rate of non-backtracking walks (about
1.4 per iteration on heavy-hex), so without the projection the iteration
leaves its fixed point after a few dozen iterations.

Gauge.  For edge e = (i, j), G_i = conj(m_{i->e}) is the Gram matrix A_i^H A_i
of i's side seen through its environment (A_i = Gamma_i with the square roots
of the other environments absorbed, leg e as columns), likewise G_j.  With the
Hermitian square root R = G^{1/2} and its pseudo-inverse R^+ (eigenvalues of G
<= GRAM_CUT times the largest dropped):

    C = R_i diag(lambda_e) R_j^T = U S V^H            (SVD)
    lambda_e' = S / ||S||_2
    Gamma_i  <- Gamma_i x_e (R_i^+ U)                 Gamma_j <- Gamma_j x_e (R_j^+ conj(V))

with (T x_e P)[.., k, ..] = sum_a T[.., a, ..] P[a, k] on leg e.  The columns
k with S_k <= LAMBDA_CUT * S_max are set to zero (the pseudo-inverse convention
of ``oracle.su``).  Gamma_i lambda_e Gamma_j^T is unchanged up to the factor
1/||S|| and the projectors on the ranges of G, so the state is unchanged; every
edge uses the messages of the same converged iteration.  After the gauge, BP
messages are proportional to the identity (the Vidal gauge on a tree).

Readings where the paper is silent (also in the design notes): messages start
at identity / D, are made Hermitian, restricted to the support of their
bond's lambda and normalised to unit trace; parallel update schedule;
convergence test on the largest elementwise change; the gauge uses the
converged messages of every edge at once; GRAM_CUT = 1e-13 relative.

Parity pins: ``tests/test_oracle_bp.py`` (state unchanged on a loopy lattice,
exact Schmidt values and <Z> on a tree from a random gauge, BP fixed point ==
simple update with identity gates, planted mistakes).
"""
from __future__ import annotations

import numpy as np

from .su import LAMBDA_CUT

GRAM_CUT = 1e-13


def _leg_product(T, p, M):
    """(T x_p M)[.., k, ..] = sum_a T[.., a, ..] M[a, k] on leg p (axis p + 1 of T)."""
    return np.moveaxis(np.tensordot(T, M, axes=(p + 1, 0)), -1, p + 1)


def identity_messages(peps):
    D = peps.D
    return {(i, p): np.eye(D, dtype=np.complex128) / D
            for i in range(peps.n) for p in range(len(peps.nb[i]))}


def message(peps, i, p, msgs, support_cut=LAMBDA_CUT):
    """m_{i->e} for leg p of site i from the messages ``msgs`` of i's other legs (unit trace),
    restricted to the support of lambda_e (entries k with lambda_e[k] <= support_cut * max zero)."""
    G = peps.gamma[i]
    X = G.conj()
    for q, k in enumerate(peps.nb[i]):
        if q == p:
            continue
        lam = peps.lam[peps.edge_of[(i, k)]]
        E = lam[:, None] * msgs[(k, peps.leg(k, i))] * lam[None, :]
        X = _leg_product(X, q, E.T)          # X[.., b, ..] = sum_b' E[b, b'] X[.., b', ..]
    axes = [ax for ax in range(G.ndim) if ax != p + 1]
    m = np.tensordot(G, X, axes=(axes, axes))
    m = 0.5 * (m + m.conj().T)
    lam_e = peps.lam[peps.edge_of[(i, peps.nb[i][p])]]
    keep = lam_e > support_cut * float(lam_e.max())
    m = m * np.outer(keep, keep)
    tr = float(np.trace(m).real)
    if not np.isfinite(tr) or tr <= 0.0:
        raise FloatingPointError(f"message of site {i}, leg {p}: trace {tr}")
    return m / tr


def messages(peps, max_iter=50, tol=1e-12, start=None, support_cut=LAMBDA_CUT):
    """Iterate BP to a fixed point.  Returns (messages, iterations run, last residual)."""
    msgs = identity_messages(peps) if start is None else start
    it, res = 0, float("inf")
    for it in range(1, max_iter + 1):
        new = {key: message(peps, key[0], key[1], msgs, support_cut) for key in msgs}
        res = max((float(np.abs(new[k] - msgs[k]).max()) for k in msgs), default=0.0)
        msgs = new
        if res <= tol:
            break
    return msgs, it, res


def sqrt_and_pinv(G):
    """Hermitian square root of the PSD matrix G and its pseudo-inverse."""
    G = 0.5 * (G + G.conj().T)
    w, W = np.linalg.eigh(G)
    wmax = max(float(w.max()), 0.0)
    keep = w > GRAM_CUT * wmax
    r = np.where(keep, np.sqrt(np.where(keep, w, 1.0)), 0.0)
    rinv = np.where(keep, 1.0 / r.clip(min=np.finfo(float).tiny), 0.0)
    return (W * r) @ W.conj().T, (W * rinv) @ W.conj().T


def gauge(peps, msgs):
    """Bring ``peps`` to the gauge of the converged ``msgs`` (every edge at once)."""
    P = {}
    lam_new = np.zeros_like(peps.lam)
    for e, (a, b) in enumerate(peps.edges):
        i, j = int(a), int(b)
        pi, pj = peps.leg(i, j), peps.leg(j, i)
        Ri, Ri_inv = sqrt_and_pinv(msgs[(i, pi)].conj())
        Rj, Rj_inv = sqrt_and_pinv(msgs[(j, pj)].conj())
        C = Ri @ np.diag(peps.lam[e]) @ Rj.T
        U, S, Vh = np.linalg.svd(C)
        nrm = float(np.linalg.norm(S))
        if not np.isfinite(nrm) or nrm == 0.0:
            raise FloatingPointError(f"edge {e}: the gauged bond vanishes")
        drop = S <= LAMBDA_CUT * S[0]
        Vc = Vh.T.copy()                                   # conj(V)
        U = U.copy()
        U[:, drop] = 0.0
        Vc[:, drop] = 0.0
        P[(i, pi)] = Ri_inv @ U
        P[(j, pj)] = Rj_inv @ Vc
        lam_new[e] = S / nrm
    for i in range(peps.n):
        for p in range(len(peps.nb[i])):
            peps.gamma[i] = _leg_product(peps.gamma[i], p, P[(i, p)])
    peps.lam = lam_new


def regauge(peps, max_iter=50, tol=1e-12, support_cut=LAMBDA_CUT):
    """BP messages to convergence, then the gauge.  Returns (iterations, residual)."""
    msgs, it, res = messages(peps, max_iter, tol, support_cut=support_cut)
    gauge(peps, msgs)
    return it, res


def evolve_bp(n_qubits, edges, D, theta, steps, max_iter=50, tol=1e-12, colour=None):
    """Trotter steps with a BP regauge after each (paper, "Benchmarking").

    Returns (mean <Z> per step, <Z_i> per step [steps, n], iterations per step, state)."""
    from .su import GPEPS
    peps = GPEPS(n_qubits, edges, D, colour=colour)
    means, zs, iters = [], [], []
    for _ in range(steps):
        peps.step(theta)
        it, _ = regauge(peps, max_iter, tol)
        iters.append(it)
        z = peps.expect_z()
        zs.append(z)
        means.append(float(z.mean()))
    return np.array(means), np.array(zs), iters, peps
