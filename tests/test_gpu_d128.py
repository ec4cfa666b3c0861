"""Bond dimension D = 128 (complex128): the large-chi runs of the paper's long-time study.

The paper's Figs. 5-7 evolve the 127-, 433- and 1121-qubit lattices for 37-39
steps at chi up to 560/370/270.  Here D = 128 (256 x 256 bond cores, degree-3
ends of 16384 rows) runs on the complex128 path, whose unsquared bond SVD needs
no squared eigensolver.  Pins: the exact regime (a heavy-hex tree at D = 2^7
against the state vector; every qubit of the 127-qubit lattice against its
light cone for 4 steps) and the truncated regime, where the oracle's own update
of sampled bonds of every kind, from the GPU's state after 8 steps (the first
truncation falls in step 8), must agree with the GPU's update of the same bonds
in step 9 (lambda 1e-9, <Z> of both ends 1e-10).  The mixed path and BP
regauging reject D > 64.
"""
import numpy as np
import pytest
import torch

from oracle import statevector as sv
from oracle.graph import greedy_colouring
from oracle.lightcone import lightcone_z
from workloads import EAGLE, heavy_hex, induced_subgraph

from ._gpu_util import gpu_lib, run_layers
from .test_gpu_d64 import _oracle_bond

pytestmark = pytest.mark.gpu

D = 128
M127, E127 = heavy_hex(*EAGLE)


def test_d128_tree_exact():
    """16-qubit heavy-hex tree, D = 128, 7 steps (Schmidt ranks <= 2^7): the state vector."""
    m, e, _ = induced_subgraph(E127, range(16))
    zg, _, g = run_layers([(m, e)], D, "c128", [0.9], 7)
    ref = sv.kicked_ising_z(m, e, 0.9, 7)
    assert np.abs(zg - ref).max() < 1e-10
    assert g.status() == 0
    g.close()


def test_d128_full_lattice_lightcone_exact():
    """127 qubits, D = 128, 4 steps: every qubit equals its light-cone value (balls are trees)."""
    theta = 0.8
    zg, _, g = run_layers([(M127, E127)], D, "c128", [theta], 4)
    for n in (1, 2, 3, 4):
        ref = np.array([lightcone_z(M127, E127, theta, q, n) for q in range(M127)])
        assert np.abs(zg[n - 1] - ref).max() < 1e-10
    g.close()


@pytest.mark.parametrize("schedule", [0, 4])
def test_d128_truncated_sampled_bonds(schedule):
    """127 qubits, D = 128, theta = 1.0 (the paper's long-time angle): 8 Trotter steps (layered
    launches or the fused step), then kick + colour class 0 explicitly; sampled bonds of every
    kind against the oracle's update of the same bond from the same state; every lambda stays
    normalised."""
    theta = 1.0
    n, edges = M127, E127
    g = gpu_lib()([(n, edges)], D, dtype="c128")
    g.set_schedule(schedule)
    g.reset()
    th = torch.tensor([theta], dtype=torch.float64, device="cuda")
    g.step(8, th)
    assert g.status() == 0
    col = greedy_colouring(edges)
    deg = np.bincount(np.asarray(edges).reshape(-1), minlength=n)
    kinds = {}
    for k in (k for k in range(len(edges)) if col[k] == 0):
        a, b = (int(x) for x in edges[k])
        kinds.setdefault(tuple(sorted((deg[a], deg[b]))), []).append(k)
    sample = sorted({ks[i] for ks in kinds.values() for i in (0, len(ks) // 2, -1)})
    g.kick(th)
    refs = {k: _oracle_bond(g, (n, edges), int(edges[k][0]), int(edges[k][1]), theta, D) for k in sample}
    g.zz_layer(0)
    z, _ = g.expect_z()
    z = z.cpu().numpy()
    assert g.status() == 0
    truncated = 0
    for k, (lam_o, zi, zj) in refs.items():
        a, b = (int(x) for x in edges[k])
        lam_g = g.lambdas(0, k)
        assert np.abs(np.sort(lam_g)[::-1] - np.sort(lam_o)[::-1]).max() < 1e-9, k
        assert abs(z[a] - zi) < 1e-10, (k, z[a], zi)
        assert abs(z[b] - zj) < 1e-10, (k, z[b], zj)
        truncated += int(np.count_nonzero(lam_o > 1e-12) == D)
    assert truncated > 0          # the sample includes bonds cut to D
    lam = np.array([g.lambda_tensor(0, k).cpu().numpy() for k in range(len(edges))])
    assert np.abs((lam ** 2).sum(axis=1) - 1.0).max() < 1e-12
    g.close()


def test_d128_rejected_where_unsupported():
    from paper_2309_15642_gb300 import GpepsError
    with pytest.raises(GpepsError):
        gpu_lib()([(M127, E127)], D, dtype="mixed")
    with pytest.raises(GpepsError):
        gpu_lib()([(M127, E127)], 129, dtype="c128")
    m, e, _ = induced_subgraph(E127, range(16))
    g = gpu_lib()([(m, e)], D, dtype="c128")
    g.reset()
    with pytest.raises(GpepsError):
        g.bp_regauge(10)
    g.close()
