"""BP regauging on the GPU (``gpeps_bp_regauge``) against the oracle (``oracle.bp``).

* Tree, random gauge: the regauge must recover the exact Schmidt values of the
  state vector across every bond and the exact <Z_i> (BP is exact on trees).
* 127 qubits and the 10-site torus cell, Trotter steps with a regauge after each
  (the paper's BP comparison): mean <Z>, per-qubit <Z> and lambda spectra against
  the oracle's evolution, step by step.
* The full 1121-qubit lattice at D = 32 (mixed): after the regauge every
  sampled message that the oracle computes from the GPU's state and identity
  incoming messages is the normalised identity (the defining property of the
  BP gauge), and the lambda stay normalised.
Tolerances: |d<Z>| <= 1e-10 (complex128), 1e-4 (mixed), as for the Trotter step.
"""
import networkx as nx
import numpy as np
import pytest
import torch

from oracle import bp, su
from oracle import statevector as sv
from workloads import CONDOR, EAGLE, heavy_hex, heavy_hex_cell, induced_subgraph

from ._gpu_util import gpu_lib

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "mixed": 1e-4}
TOL_LAM = {"c128": 1e-9, "mixed": 2e-3}
M127, E127 = heavy_hex(*EAGLE)


def read_state(g, n, edges):
    gam = [g.site_tensor(0, v)[0].cpu().numpy().astype(np.complex128) for v in range(n)]
    lam = np.array([g.lambda_tensor(0, k).cpu().numpy() for k in range(len(edges))])
    return gam, lam


def write_state(g, n, edges, gam, lam):
    for v in range(n):
        t, _ = g.site_tensor(0, v)
        t.copy_(torch.as_tensor(gam[v]).to(t.dtype))
    for k in range(len(edges)):
        g.lambda_tensor(0, k).copy_(torch.as_tensor(lam[k]))
    torch.cuda.synchronize()


def sorted_lam(x):
    return -np.sort(-np.asarray(x), axis=-1)


def lam_close(gpu, ref, dtype, truncated=False):
    """Sorted spectra: complex128 to 1e-6 everywhere and 1e-9 (5e-8 once truncated) where
    lambda > 1e-3 (after a regauge the bond weights come from the eigenproblem of the
    squared matrix C C^H of the gauge, so the small ones are resolved to ~sqrt(eps) of
    the largest); mixed to 2e-3."""
    d = np.abs(sorted_lam(gpu) - np.asarray(ref))
    if dtype != "c128":
        return d.max() < TOL_LAM["mixed"]
    big = np.asarray(ref) > 1e-3
    return d.max() < 1e-6 and (not big.any() or d[big].max() < (5e-8 if truncated else 1e-9))


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_tree_random_gauge_recovers_schmidt_values(dtype):
    m, e, _ = induced_subgraph(E127, range(16))
    steps, theta, D = 3, 0.75, 8
    g = gpu_lib()([(m, e)], D, dtype=dtype)
    g.reset()
    g.step(steps, torch.tensor([theta], dtype=torch.float64, device="cuda"))
    gam, lam = read_state(g, m, e)
    nb = [g.site_tensor(0, v)[1] for v in range(m)]
    rng = np.random.default_rng(11)
    for k, (a, b) in enumerate(e):
        i, j = int(a), int(b)
        X = rng.normal(size=(D, D)) + 1j * rng.normal(size=(D, D)) + 3 * np.eye(D)
        mu = rng.uniform(0.2, 1.0, D)
        mu /= np.linalg.norm(mu)
        gam[i] = bp._leg_product(gam[i], nb[i].index(j), X)
        gam[j] = bp._leg_product(gam[j], nb[j].index(i), (np.diag(1.0 / mu) @ np.linalg.inv(X) @ np.diag(lam[k])).T)
        lam[k] = mu
    write_state(g, m, e, gam, lam)
    it, res = g.bp_regauge(100)
    assert it < 100, (it, res)
    psi = list(sv.kicked_ising_states(m, e, theta, steps))[-1]
    z, _ = g.expect_z()
    assert np.abs(z.cpu().numpy() - sv.z_expectations(psi)).max() < TOL[dtype]
    graph = nx.Graph([tuple(map(int, x)) for x in e])
    for k, (a, b) in enumerate(e):
        h = graph.copy()
        h.remove_edge(int(a), int(b))
        s = sv.schmidt_values(psi, nx.node_connected_component(h, int(a)))[:D]
        ref = np.zeros(D)
        ref[:len(s)] = s
        assert np.abs(sorted_lam(g.lambdas(0, k)) - ref).max() < TOL_LAM[dtype], k
    assert g.status() == 0
    g.close()


def _evolve_and_compare(n, e, D, theta, steps, dtype, colours=None):
    means_o, zs_o, _, peps = bp.evolve_bp(n, e, D, theta, steps, max_iter=200, tol=1e-13, colour=colours)
    g = gpu_lib()([(n, e)], D, dtype=dtype, colours=[colours] if colours is not None else None)
    g.reset()
    th = torch.tensor([theta], dtype=torch.float64, device="cuda")
    lam_o = None
    for s in range(steps):
        g.step(1, th)
        it, res = g.bp_regauge(200)
        assert it < 200, (s, it, res)
        z, mean = g.expect_z()
        z = z.cpu().numpy()
        assert np.abs(z - zs_o[s]).max() < TOL[dtype], s
        assert abs(float(mean.cpu().numpy()[0]) - means_o[s]) < TOL[dtype], s
    lam_o = peps.lambdas()
    for k in range(len(e)):
        assert np.abs(sorted_lam(g.lambdas(0, k)) - lam_o[k]).max() < TOL_LAM[dtype], k
    assert g.status() == 0
    g.close()


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_eagle_bp_evolution_matches_oracle(dtype):
    """127 qubits, D = 4, theta = 0.8, 7 steps with a regauge after each (truncated from step 3)."""
    _evolve_and_compare(M127, E127, 4, 0.8, 7, dtype)


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_eagle_d16_bp_evolution_matches_oracle(dtype):
    """127 qubits, D = 16, theta = 0.6, 6 steps: deg-3 messages of 2 x 16^3 tensors."""
    _evolve_and_compare(M127, E127, 16, 0.6, 6, dtype)


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_cell_bp_evolution_matches_oracle(dtype):
    """The 10-site torus cell of the infinite lattice (loops of length 4 and 6), D = 8."""
    from workloads import heavy_hex_cell_colour
    m, e = heavy_hex_cell()
    _evolve_and_compare(m, e, 8, 0.9, 5, dtype, colours=heavy_hex_cell_colour())


def test_odd_bond_dimension():
    """D = 5: the gauge eigenproblems are padded to an even size."""
    m, e, _ = induced_subgraph(E127, range(24))
    _evolve_and_compare(m, e, 5, 0.7, 4, "c128")


def test_condor_d32_full_size_gauge_property():
    """1121 qubits, D = 32, mixed, 6 steps then a regauge: sampled messages from identity are the
    normalised identity, lambda normalised, <Z> finite and within [-1, 1]."""
    n, edges = heavy_hex(*CONDOR)
    D = 32
    g = gpu_lib()([(n, edges)], D, dtype="mixed")
    g.reset()
    g.step(6, torch.tensor([0.7], dtype=torch.float64, device="cuda"))
    it, res = g.bp_regauge(200)
    assert it < 200 and res <= 1e-6, (it, res)
    assert g.status() == 0
    nbrs = {}
    for a, b in edges:
        nbrs.setdefault(int(a), []).append(int(b))
        nbrs.setdefault(int(b), []).append(int(a))
    deg3 = [v for v in range(n) if len(nbrs[v]) == 3]
    deg2 = [v for v in range(n) if len(nbrs[v]) == 2]
    full = {(min(int(a), int(b)), max(int(a), int(b))): k for k, (a, b) in enumerate(edges)}
    for v in deg3[::97] + deg2[::181]:
        t, nb = g.site_tensor(0, v)
        sites = sorted([v] + nb)
        loc = {s: k for k, s in enumerate(sites)}
        sub = np.array(sorted((min(loc[v], loc[u]), max(loc[v], loc[u])) for u in nb))
        peps = su.GPEPS(len(sites), sub, D)
        peps.gamma[loc[v]] = t.cpu().numpy().astype(np.complex128)
        for k, (a, b) in enumerate(sub):
            peps.lam[k] = g.lambda_tensor(0, full[(min(sites[a], sites[b]), max(sites[a], sites[b]))]).cpu().numpy()
        msgs = bp.identity_messages(peps)
        for p in range(len(nb)):
            m = bp.message(peps, loc[v], p, msgs)
            lam_e = peps.lam[peps.edge_of[(loc[v], peps.nb[loc[v]][p])]]
            r = int(np.count_nonzero(lam_e > 1e-13 * lam_e.max()))   # the columns the gauge keeps
            ref = np.zeros((D, D))
            ref[:r, :r] = np.eye(r) / r
            assert np.abs(m - ref).max() < 1e-4, (v, p)
    lam = np.array([g.lambda_tensor(0, k).cpu().numpy() for k in range(len(edges))])
    assert np.abs((lam ** 2).sum(axis=1) - 1.0).max() < 1e-12
    z, _ = g.expect_z()
    z = z.cpu().numpy()
    assert np.all(np.isfinite(z)) and np.abs(z).max() <= 1.0 + 1e-6
    g.close()


def test_workspace_errors():
    g = gpu_lib()([(M127, E127)], 4, dtype="c128")
    import ctypes
    nbytes = ctypes.c_size_t()
    assert g.lib.gpeps_query_bp_workspace(g.h, 0, ctypes.byref(nbytes)) == 1
    assert g.lib.gpeps_query_bp_workspace(g.h, 10, ctypes.byref(nbytes)) == 0
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    it, res = ctypes.c_int32(), ctypes.c_double()
    assert g.lib.gpeps_bp_regauge(g.h, 10, 1e-12, ctypes.c_void_p(small.data_ptr()), 256, ctypes.byref(it),
                                  ctypes.byref(res), None) == 1
    assert g.lib.gpeps_bp_regauge(g.h, 10, -1.0, ctypes.c_void_p(small.data_ptr()), nbytes.value,
                                  ctypes.byref(it), ctypes.byref(res), None) == 1
    g.close()


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_eagle_bp_d32_matches_oracle_golden(dtype):
    """127 qubits at the benchmark's D = 32, theta = 0.7, 8 steps with a regauge after each
    (truncation from step 6): mean <Z> of every step, every qubit and sampled lambda at the
    committed steps of ``tests/golden/make_oracle_golden.py eagle_bp_d32``."""
    import json
    import os
    from workloads import workload
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_eagle_bp_d32.json")) as f:
        inst = json.load(f)["instances"][0]
    w = workload("eagle_bp_d32")
    g = gpu_lib()(w.graphs(), w.D, dtype=dtype)
    g.reset()
    th = torch.tensor([w.theta[0]], dtype=torch.float64, device="cuda")
    for s in range(1, w.steps + 1):
        g.step(1, th)
        it, res = g.bp_regauge(300)
        assert it < 300, (s, it, res)
        z, mean = g.expect_z()
        assert abs(float(mean.cpu().numpy()[0]) - inst["mean_z"][s - 1]) < TOL[dtype], s
        if str(s) in inst["z"]:
            assert np.abs(z.cpu().numpy() - np.array(inst["z"][str(s)])).max() < TOL[dtype], s
            for e, lam in inst["lambda"][str(s)].items():
                assert lam_close(g.lambdas(0, int(e)), lam, dtype, truncated=2 ** s > w.D), (s, e)
    assert g.status() == 0
    g.close()


@pytest.mark.parametrize("D", [1, 2])
def test_small_bond_dimensions(D):
    """D = 1 (a product state: every message and gauge is 1 x 1, padded to 2 x 2 in the gauge)
    and D = 2, on a 24-qubit fragment with a regauge after each of 3 steps."""
    m, e, _ = induced_subgraph(E127, range(24))
    _evolve_and_compare(m, e, D, 0.7, 3, "c128")


def test_isolated_qubit_and_single_edge():
    """A qubit without couplers (no messages, no gauge) next to one edge and a path."""
    edges = np.array([[0, 1], [2, 3], [3, 4]], dtype=np.int32)
    _evolve_and_compare(6, edges, 2, 0.9, 3, "c128")
