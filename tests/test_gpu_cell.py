"""The infinite heavy-hex lattice (10-site unit cell with periodic couplers, its periodic
colouring) on the GPU: the 16-angle sweep of 16 cell instances in one batch (D = 32, 5 steps)
against the committed oracle values, a 20-step truncated run against the oracle, the untruncated
regime against exact light cones of the equivalent interior sites of the 1121-qubit lattice, and
the Table I site Q(infinity) = 2 by Clifford back-evolution.  Tolerances as in test_gpu_parity.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import su, weight
from oracle.lightcone import lightcone_z
from workloads import CONDOR, equivalent_site, heavy_hex, heavy_hex_cell, heavy_hex_cell_colour, kick_angles, workload

from ._gpu_util import gpu_lib, split

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "mixed": 1e-4}
TOL_TRUNC = {"c128": 1e-10, "mixed": 1e-4}
CELL = heavy_hex_cell()
COL = heavy_hex_cell_colour()


def _cell(D, dtype, n_inst=1):
    return gpu_lib()([CELL] * n_inst, D, dtype=dtype, colours=[COL] * n_inst)


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_infinite_sweep16_matches_oracle(dtype):
    w = workload("infinite_sweep16_d32")
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_infinite_sweep16_d32.json")) as f:
        gold = json.load(f)
    theta = [th[0] for th in kick_angles(w)]
    g = _cell(w.D, dtype, len(theta))
    g.reset()
    means = g.step(w.steps, torch.tensor(theta, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert g.status() == 0
    ref = np.array([inst["mean_z"] for inst in gold["instances"]]).T
    assert np.abs(means - ref).max() < TOL[dtype]
    z, _ = g.expect_z()
    zi = split(z.cpu().numpy(), w.graphs())
    for k, inst in enumerate(gold["instances"]):
        assert np.abs(zi[k] - np.array(inst["z"][str(w.steps)])).max() < TOL[dtype], k
    g.close()


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
@pytest.mark.parametrize("schedule", [0, 4])
def test_infinite_truncated_20_steps(dtype, schedule):
    n, e = CELL
    g = _cell(32, dtype)
    g.set_schedule(schedule)
    g.reset()
    means = g.step(20, torch.tensor([0.7], dtype=torch.float64, device="cuda")).cpu().numpy()[:, 0]
    z, _ = g.expect_z()
    assert g.status() == 0
    peps = su.GPEPS(n, e, 32, colour=COL)
    ref = []
    for _ in range(20):
        peps.step(0.7)
        ref.append(peps.expect_z().mean())
    assert np.abs(means - np.array(ref)).max() < TOL[dtype]
    assert np.abs(z.cpu().numpy() - peps.expect_z()).max() < TOL_TRUNC[dtype]
    g.close()


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_infinite_exact_regime_lightcone(dtype):
    N, E = heavy_hex(*CONDOR)
    g = _cell(16, dtype)
    g.reset()
    th = torch.tensor([0.6], dtype=torch.float64, device="cuda")
    for steps in range(1, 5):
        g.step(1, th)
        z, _ = g.expect_z()
        z = z.cpu().numpy()
        for s in range(10):
            ref = lightcone_z(N, E, 0.6, equivalent_site(*CONDOR, s, 10, 20), steps)
            assert abs(z[s] - ref) < TOL[dtype], (steps, s)
    g.close()


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_infinite_weight_at_q(dtype):
    """Table I: Q(infinity) = 2; n = 5, D = 32, every cell site against the oracle."""
    n, e = CELL
    g = _cell(32, dtype)
    z = g.weight_z(torch.tensor([0.6], dtype=torch.float64, device="cuda"), 5).cpu().numpy()
    assert g.status() == 0
    ref = weight.weight_z(n, e, 32, 0.6, 5, colour=COL)
    assert abs(z[2] - ref[2]) < TOL_TRUNC[dtype] and np.abs(z - ref).max() < TOL_TRUNC[dtype]
    g.close()
