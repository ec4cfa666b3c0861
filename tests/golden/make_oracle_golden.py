"""Write the oracle's expected values for the larger workloads (calls only ``oracle/``).

    python tests/golden/make_oracle_golden.py eagle_sweep16_d16
    python tests/golden/make_oracle_golden.py heavyhex_mix_d32
    python tests/golden/make_oracle_golden.py eagle_d64
    python tests/golden/make_oracle_golden.py infinite_sweep16_d32
    python tests/golden/make_oracle_golden.py eagle_bp_d32

Each run writes ``tests/golden/oracle_<workload>.json``: the mean <Z> of every
instance after every Trotter step, the per-qubit <Z> after a few sampled steps
and the sorted lambda spectra of a few sampled edges.  The oracle is the plain
FP64 simple update of ``oracle/su.py`` (the workload's colouring: greedy, or the
unit cell's periodic one; same inputs as the GPU tests from ``workloads``); for a
workload with ``bp`` set, followed after every step by the BP regauge of
``oracle/bp.py`` (to a residual of 1e-13), whose iteration counts are recorded.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import bp  # noqa: E402
from oracle.su import GPEPS  # noqa: E402
from workloads import kick_angles, workload  # noqa: E402

SAMPLE_STEPS = {"eagle_sweep16_d16": [1, 4, 5, 10, 20], "heavyhex_mix_d32": [1, 5, 6, 10, 25, 50],
                "eagle_d64": [1, 5, 6, 7, 8], "infinite_sweep16_d32": [1, 3, 5], "eagle_bp_d32": [1, 5, 6, 7, 8]}


def sampled_edges(n_edges, k=8):
    return sorted(set(np.linspace(0, n_edges - 1, k).astype(int).tolist()))


def run(name, steps=None):
    w = workload(name)
    steps = steps or w.steps
    thetas = kick_angles(w)
    sample = [s for s in SAMPLE_STEPS.get(name, [steps]) if s <= steps]
    out = {"workload": name, "D": w.D, "steps": steps, "instances": []}
    t0 = time.time()
    for k, ((n, edges), th, col) in enumerate(zip(w.graphs(), thetas, w.colours())):
        peps = GPEPS(n, edges, w.D, colour=col)
        inst = {"n_qubits": int(n), "theta": float(th[0]) if w.per_qubit_seed is None else None,
                "mean_z": [], "z": {}, "lambda": {}}
        if w.bp:
            inst["bp_iterations"] = []
        ed = sampled_edges(len(edges))
        for t in range(1, steps + 1):
            peps.step(th)
            if w.bp:
                it, res = bp.regauge(peps, 500, 1e-13)
                if res > 1e-13:
                    raise RuntimeError(f"BP did not converge at step {t}: residual {res}")
                inst["bp_iterations"].append(it)
            z = peps.expect_z()
            inst["mean_z"].append(float(z.mean()))
            if t in sample:
                inst["z"][str(t)] = [float(v) for v in z]
                lam = peps.lambdas()
                inst["lambda"][str(t)] = {str(e): [float(v) for v in lam[e]] for e in ed}
            print(f"{name} instance {k} step {t} mean {z.mean():.12f} ({time.time() - t0:.0f}s)", flush=True)
        out["instances"].append(inst)
    path = os.path.join(HERE, f"oracle_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path)


# 24 kick angles spread over the 127-qubit lattice (rows, bridges, both ends)
GRAD_QUBITS = sorted(set(np.linspace(0, 126, 24).round().astype(int).tolist()))


def run_grad(name):
    """Oracle gradient (central differences, h = 1e-5) of the mean <Z> after all steps with
    respect to the per-qubit kick angles of GRAD_QUBITS."""
    from oracle.gradient import fd_gradient, oracle_loss
    w = workload(name)
    (n, edges), th = w.graphs()[0], kick_angles(w)[0]
    weights = np.full(n, 1.0 / n)
    t0 = time.time()
    loss = oracle_loss(n, edges, w.D, th, w.steps, weights)
    g = fd_gradient(n, edges, w.D, th, w.steps, weights, h=1e-5, qubits=GRAD_QUBITS)
    out = {"workload": name, "D": w.D, "steps": w.steps, "h": 1e-5, "loss": loss,
           "dloss_dtheta": {str(q): v for q, v in g.items()}}
    path = os.path.join(HERE, f"oracle_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, f"({time.time() - t0:.0f}s)")


if __name__ == "__main__":
    if workload(sys.argv[1]).per_qubit_seed is not None:
        run_grad(sys.argv[1])
    else:
        run(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else None)
