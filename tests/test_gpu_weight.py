"""Weight-N observables by Clifford back-evolution (App. B) on the GPU: n forward steps at
theta_h, n inverse steps at pi/2 (gpeps_inverse_steps: colour classes reversed with the
conjugate gate, then the kick by -pi/2), single-site <Z> readout.

Against exact light cones in the untruncated regime (127 qubits, n = 2, D = 16), the identity
|omega> = |0...0> at theta_h = pi/2, and the oracle in the paper's setting (n = 5, the Weight-10
and Weight-17 sites of App. B and the P/Q labels of Table I on all three lattices, truncated).
Tolerances as in test_gpu_parity.
"""
import math

import numpy as np
import pytest
import torch

from oracle import weight
from oracle.lightcone import lightcone_weight_z
from workloads import CONDOR, EAGLE, OSPREY, heavy_hex

from ._gpu_util import gpu_lib

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "mixed": 1e-4}
TOL_TRUNC = {"c128": 1e-10, "mixed": 1e-4}
M127, E127 = heavy_hex(*EAGLE)


def _gpu_weight_z(graph, D, dtype, theta, n, schedule=0):
    g = gpu_lib()([graph], D, dtype=dtype)
    g.set_schedule(schedule)
    z = g.weight_z(torch.tensor([theta], dtype=torch.float64, device="cuda"), n).cpu().numpy()
    assert g.status() == 0
    g.close()
    return z


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_weight_exact_regime_lightcone(dtype):
    z = _gpu_weight_z((M127, E127), 16, dtype, 0.6, 2)
    for q in list(range(0, M127, 9)) + [13, 58, 62]:
        assert abs(z[q] - lightcone_weight_z(M127, E127, 0.6, q, 2)) < TOL[dtype], q


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_weight_clifford_point_identity(dtype):
    z = _gpu_weight_z((M127, E127), 16, dtype, math.pi / 2, 2)
    assert np.abs(z - 1.0).max() < TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
@pytest.mark.parametrize("theta", [0.3, 0.6])
def test_weight_127_n5_matches_oracle(dtype, theta):
    """127 qubits, D = 16, n = 5 (10 simple-update steps, truncated): every qubit, among them the
    Weight-10 (P = 13) and Weight-17 (Z_58) sites; the forward half runs as the fused step."""
    z = _gpu_weight_z((M127, E127), 16, dtype, theta, 5, schedule=4)
    ref = weight.weight_z(M127, E127, 16, theta, 5)
    assert np.abs(z - ref).max() < TOL_TRUNC[dtype]


@pytest.mark.parametrize("lattice, P, Q", [(OSPREY, 25, 181), (CONDOR, 41, 505)])
def test_weight_table1_sites_larger_lattices(lattice, P, Q):
    """433 and 1121 qubits (Table I labels), D = 8, n = 5, complex128."""
    n_q, e = heavy_hex(*lattice)
    z = _gpu_weight_z((n_q, e), 8, "c128", 0.6, 5)
    ref = weight.weight_z(n_q, e, 8, 0.6, 5)
    assert abs(z[P] - ref[P]) < TOL_TRUNC["c128"] and abs(z[Q] - ref[Q]) < TOL_TRUNC["c128"]
    assert np.abs(z - ref).max() < TOL_TRUNC["c128"]
