"""Reverse mode (gpeps_grad) against exact and finite-difference derivatives.

References: the parameter-shift derivative of the exact state vector (exact
regime: a heavy-hex tree, D = 2^n), central differences of the FP64 oracle
(truncated 127-qubit lattice), and, at the 127-qubit, D = 16, 20-step workload
with per-qubit angles, the oracle's central differences (h = 1e-5) for 24 angles
spread over the lattice (committed values of tests/golden/make_oracle_golden.py)
plus central differences of the library's own forward for six of them.
Tolerance 1e-6 relative to the largest derivative.
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle.gradient import fd_gradient, parameter_shift_gradient
from workloads import EAGLE, heavy_hex, induced_subgraph, kick_angles, workload

from ._gpu_util import gpu_lib

pytestmark = pytest.mark.gpu

M127, E127 = heavy_hex(*EAGLE)
REL = 1e-6


def _grad(graph, D, theta, steps, ckpt=5, weights=None):
    g = gpu_lib()([graph], D, dtype="c128")
    n = graph[0]
    w = np.full(n, 1.0 / n) if weights is None else weights
    z, dth = g.grad(torch.tensor(theta, dtype=torch.float64, device="cuda"), steps, ckpt,
                    dL_dz=torch.tensor(w, dtype=torch.float64, device="cuda"))
    assert g.status() == 0
    out = (float(np.dot(w, z.cpu().numpy())), dth.cpu().numpy())
    g.close()
    return out


def test_grad_exact_regime_parameter_shift():
    m, e, _ = induced_subgraph(E127, range(16))
    rng = np.random.default_rng(3)
    theta = rng.uniform(0.5, 0.9, m)
    w = np.full(m, 1.0 / m)
    _, g = _grad((m, e), 8, theta, 3, ckpt=2)
    ref = parameter_shift_gradient(m, e, theta, 3, w)
    assert np.abs(g - ref).max() < REL * np.abs(ref).max()


def test_grad_truncated_127_vs_oracle_fd():
    rng = np.random.default_rng(11)
    theta = rng.uniform(0.5, 0.9, M127)
    w = np.full(M127, 1.0 / M127)
    _, g = _grad((M127, E127), 4, theta, 3, ckpt=1)
    qs = [0, 5, 13, 20, 37, 58, 62, 90, 113, 126]
    fd = fd_gradient(M127, E127, 4, theta, 3, w, qubits=qs)
    scale = max(abs(v) for v in fd.values())
    for q, v in fd.items():
        assert abs(g[q] - v) < REL * scale, (q, g[q], v)


def test_grad_workload_d16_vs_oracle_fd():
    """127 q, D = 16, 20 steps, theta_i ~ U[0.5, 0.9] (seeded), checkpoint every 5: the loss and
    the derivative in every committed angle against the oracle's central differences."""
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_eagle_grad_d16.json")
    gold = json.load(open(path))
    w = workload("eagle_grad_d16")
    (n, e), th = w.graphs()[0], kick_angles(w)[0]
    L, g = _grad((n, e), w.D, th, w.steps, ckpt=5)
    assert len(gold["dloss_dtheta"]) >= 20 and gold["h"] == 1e-5
    assert abs(L - gold["loss"]) < 1e-10
    scale = max(abs(v) for v in gold["dloss_dtheta"].values())
    for q, v in gold["dloss_dtheta"].items():
        assert abs(g[int(q)] - v) < REL * scale, (q, g[int(q)], v)


def test_grad_workload_d16_vs_library_fd():
    """The same workload against central differences of the library's own forward (six angles)."""
    w = workload("eagle_grad_d16")
    (n, e), th = w.graphs()[0], kick_angles(w)[0]
    weights = np.full(n, 1.0 / n)
    L, g = _grad((n, e), w.D, th, w.steps, ckpt=5)
    G = gpu_lib()([(n, e)], w.D, dtype="c128")
    h = 1e-5
    qs = [0, 13, 37, 62, 100, 126]
    fd = {}
    for q in qs:
        vals = []
        for sgn in (1, -1):
            tq = th.copy()
            tq[q] += sgn * h
            z, _ = G.grad(torch.tensor(tq, dtype=torch.float64, device="cuda"), w.steps, 5)
            vals.append(float(np.dot(weights, z.cpu().numpy())))
        fd[q] = (vals[0] - vals[1]) / (2 * h)
    G.close()
    scale = np.abs(g).max()
    for q in qs:
        assert abs(g[q] - fd[q]) < REL * scale, (q, g[q], fd[q])


def test_grad_checkpoint_spacing_does_not_change_the_result():
    rng = np.random.default_rng(5)
    theta = rng.uniform(0.5, 0.9, M127)
    ref = _grad((M127, E127), 8, theta, 6, ckpt=1)[1]
    for k in (2, 5, 6):
        g = _grad((M127, E127), 8, theta, 6, ckpt=k)[1]
        assert np.abs(g - ref).max() < 1e-12 * np.abs(ref).max()


def test_autograd_function():
    from paper_2309_15642_gb300.gpeps import KickedIsingZ
    m, e, _ = induced_subgraph(E127, range(16))
    g = gpu_lib()([(m, e)], 8, dtype="c128")
    rng = np.random.default_rng(9)
    theta = torch.tensor(rng.uniform(0.5, 0.9, m), dtype=torch.float64, device="cuda", requires_grad=True)
    z = KickedIsingZ.apply(theta, g, 3, 2)
    loss = (z * torch.linspace(0.5, 1.5, m, dtype=torch.float64, device="cuda")).sum()
    loss.backward()
    _, direct = g.grad(theta.detach(), 3, 2, dL_dz=torch.linspace(0.5, 1.5, m, dtype=torch.float64, device="cuda"))
    assert torch.allclose(theta.grad, direct, rtol=0, atol=1e-14)
    g.close()


def test_grad_rejects_unsupported_handles():
    from paper_2309_15642_gb300 import GpepsError
    th = torch.full((M127,), 0.7, dtype=torch.float64, device="cuda")
    for dtype, D in (("mixed", 8), ("c128", 32)):
        g = gpu_lib()([(M127, E127)], D, dtype=dtype)
        with pytest.raises(GpepsError):
            g.grad(th, 2, 1)
        g.close()
