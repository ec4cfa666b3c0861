"""The named synthetic workloads: lattice(s), bond dimension D, steps and kick angles.

Every workload is the kicked Ising circuit of the paper's Eqs. (2)-(3) started
from |0...0>; nothing is random except the per-qubit kick angles of the
gradient workload, drawn from ``numpy.random.default_rng(15642)`` uniformly in
[0.5, 0.9] in qubit-label order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .heavyhex import CELL, CONDOR, EAGLE, OSPREY, heavy_hex, heavy_hex_cell, heavy_hex_cell_colour


@dataclass(frozen=True)
class Workload:
    name: str
    lattices: tuple          # one (rows, width) per instance
    D: int
    steps: int
    theta: tuple             # one kick angle per instance (ignored when per_qubit_seed is set)
    per_qubit_seed: int | None = None
    note: str = ""
    bp: bool = False         # a BP regauge after every Trotter step

    def graphs(self):
        """List of ``(n_qubits, edges)``, one per instance."""
        cache = {}
        out = []
        for lat in self.lattices:
            if lat not in cache:
                cache[lat] = heavy_hex_cell() if lat == CELL else heavy_hex(*lat)
            out.append(cache[lat])
        return out

    def colours(self):
        """Per instance: the edge colour classes to use (the unit cell's periodic colouring), or
        None for the greedy colouring of the library and the oracle."""
        return [heavy_hex_cell_colour() if lat == CELL else None for lat in self.lattices]

    @property
    def n_instances(self):
        return len(self.lattices)


def kick_angles(w: Workload):
    """Per-instance list of per-qubit kick angles (float64 arrays)."""
    out = []
    for k, (n, _) in enumerate(w.graphs()):
        if w.per_qubit_seed is not None:
            rng = np.random.default_rng(w.per_qubit_seed)
            out.append(rng.uniform(0.5, 0.9, size=n).astype(np.float64))
        else:
            out.append(np.full(n, float(w.theta[k]), dtype=np.float64))
    return out


WORKLOADS = {
    "eagle_d4": Workload("eagle_d4", (EAGLE,), 4, 5, (0.6,),
                         note="127 q, D=4, 5 steps, theta=0.6, complex128"),
    "eagle_sweep16_d16": Workload(
        "eagle_sweep16_d16", (EAGLE,) * 16, 16, 20,
        tuple(float(t) for t in np.linspace(0.0, math.pi / 2, 16)),
        note="127 q x 16 instances, theta evenly spaced in [0, pi/2], D=16, 20 steps"),
    "heavyhex_mix_d32": Workload(
        "heavyhex_mix_d32", (EAGLE, OSPREY, CONDOR), 32, 50, (0.7, 0.7, 0.7),
        note="127 + 433 + 1121 q in one batch, D=32, 50 steps, theta=0.7"),
    "eagle_grad_d16": Workload("eagle_grad_d16", (EAGLE,), 16, 20, (0.0,), per_qubit_seed=15642,
                               note="127 q, D=16, 20 steps, theta_i ~ U[0.5, 0.9] seeded 15642"),
    "condor_d64": Workload("condor_d64", (CONDOR,), 64, 100, (0.8,),
                           note="1121 q, D=64, 100 steps, theta=0.8"),
    "infinite_sweep16_d32": Workload(
        "infinite_sweep16_d32", (CELL,) * 16, 32, 5,
        tuple(float(t) for t in np.linspace(0.0, math.pi / 2, 16)),
        note="infinite heavy-hex lattice (10-site unit cell, periodic couplers) x 16 instances, "
             "theta evenly spaced in [0, pi/2], D=32, 5 steps"),
    "eagle_d64": Workload("eagle_d64", (EAGLE,), 64, 8, (0.8,),
                          note="127 q, D=64, 8 steps, theta=0.8: the 128 x 128 bond eigenproblems of "
                               "condor_d64 on a lattice the oracle finishes in minutes (truncation from step 7)"),
    "eagle_d128": Workload("eagle_d128", (EAGLE,), 128, 39, (1.0,),
                           note="127 q, D=128, theta=1.0: the paper's long-time runs (Figs. 5-7, 37-39 steps) "
                                "at chi = 128 on the complex128 path (truncation from step 8)"),
    "eagle_bp_d32": Workload("eagle_bp_d32", (EAGLE,), 32, 8, (0.7,), bp=True,
                             note="127 q, D=32, 8 steps, theta=0.7, a BP regauge after every step (the paper's "
                                  "BP comparison at the benchmark's bond dimension; truncation from step 6)"),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]
