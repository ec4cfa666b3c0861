"""Seeded, synthetic inputs shared by the oracle and the CUDA path.

This package holds no arithmetic of the simulation method: only the coupling
graphs of the lattices (a deterministic construction rule) and the kick angles
of the named workloads.  Both ``oracle/`` and the product package read their
inputs from here; neither imports the other.
"""
from .heavyhex import (EAGLE, OSPREY, CONDOR, CELL, LATTICES, heavy_hex, heavy_hex_cell,
                       heavy_hex_cell_colour, heavy_hex_coords, equivalent_site, induced_subgraph,
                       graph_ball)
from .configs import WORKLOADS, Workload, workload, kick_angles

__all__ = ["EAGLE", "OSPREY", "CONDOR", "CELL", "LATTICES", "heavy_hex", "heavy_hex_cell",
           "heavy_hex_cell_colour", "heavy_hex_coords", "equivalent_site", "induced_subgraph",
           "graph_ball", "WORKLOADS", "Workload", "workload", "kick_angles"]
