"""The infinite heavy-hex lattice as a translation-invariant 10-site unit cell (paper, "Method":
gPEPS of the thermodynamic limit with a unit cell of 10 sites; the cell's shape is not printed).

The finite lattices' row/bridge rule repeats every 4 columns and every 2 rows, so the cell holds
8 row qubits and 2 bridges with periodic couplers.  Pinned here: its structure; its colouring is
the pattern the finite lattices' greedy colouring takes in their interior; and, the strong pin,
the oracle's simple update of the cell (untruncated, D = 2^n) equals for n <= 5 the exact
light-cone value of the equivalent interior site of the 1121-qubit lattice (every ball of radius
<= 4 is a tree) -- a wrong cell (shape, periodic couplers, colouring) breaks that equality.
"""
import numpy as np
import pytest

from oracle import su
from oracle.graph import greedy_colouring
from oracle.lightcone import lightcone_z
from workloads import (CONDOR, OSPREY, equivalent_site, heavy_hex, heavy_hex_cell, heavy_hex_cell_colour,
                       heavy_hex_coords)
from workloads.heavyhex import CELL_COORDS


def test_cell_structure():
    n, e = heavy_hex_cell()
    assert n == 10 and len(e) == 12 and len({tuple(x) for x in e.tolist()}) == 12
    deg = np.bincount(e.reshape(-1), minlength=n)
    assert sorted(deg.tolist()) == [2] * 6 + [3] * 4
    assert all(not (deg[a] == 3 and deg[b] == 3) for a, b in e)
    col = heavy_hex_cell_colour()
    assert set(col.tolist()) == {0, 1, 2}
    for c in range(3):
        ends = e[col == c].reshape(-1)
        assert len(ends) == len(set(ends.tolist()))   # a matching
    assert greedy_colouring(e).max() + 1 == 4          # why the colouring is given explicitly


@pytest.mark.parametrize("lattice", [OSPREY, CONDOR])
def test_cell_colouring_is_the_interior_pattern(lattice):
    N, E = heavy_hex(*lattice)
    col = greedy_colouring(E)
    co = heavy_hex_coords(*lattice)
    cell_index = {c: k for k, c in enumerate(CELL_COORDS)}
    _, ce = heavy_hex_cell()
    ccol = {tuple(x): int(c) for x, c in zip(ce.tolist(), heavy_hex_cell_colour())}
    checked = 0
    for k, (a, b) in enumerate(E):
        ka, kb = co[a], co[b]
        if not (3 <= min(ka[1], kb[1]) and max(ka[1], kb[1]) <= lattice[0] - 4 and 4 <= ka[2] <= lattice[1] - 5):
            continue
        ia = cell_index[(ka[0], ka[1] % 2, ka[2] % 4)]
        ib = cell_index[(kb[0], kb[1] % 2, kb[2] % 4)]
        assert ccol[(min(ia, ib), max(ia, ib))] == col[k]
        checked += 1
    assert checked > 100


@pytest.mark.parametrize("theta", [0.3, 0.7])
def test_cell_simple_update_is_the_infinite_lattice(theta):
    n, e = heavy_hex_cell()
    col = heavy_hex_cell_colour()
    N, E = heavy_hex(*CONDOR)
    sites = [equivalent_site(*CONDOR, s, 10, 20) for s in range(n)]
    for steps in range(1, 6):
        peps = su.GPEPS(n, e, 2 ** steps, colour=col)
        for _ in range(steps):
            peps.step(theta)
        z = peps.expect_z()
        for s in range(n):
            assert abs(z[s] - lightcone_z(N, E, theta, sites[s], steps)) < 1e-10, (steps, s)


def test_planted_mistake_wrong_bridge_column():
    """A 10-site cell whose second bridge sits one column off (column 3 instead of 2) is not the
    heavy-hex lattice: the pin above must fail for it."""
    n = 10
    e = np.array(sorted([(0, 1), (1, 2), (2, 3), (0, 3), (5, 6), (6, 7), (7, 8), (5, 8),
                         (0, 4), (4, 5), (8, 9), (3, 9)]), dtype=np.int32)
    N, E = heavy_hex(*CONDOR)
    peps = su.GPEPS(n, e, 8)
    for _ in range(3):
        peps.step(0.7)
    z = peps.expect_z()
    ref = [lightcone_z(N, E, 0.7, equivalent_site(*CONDOR, s, 10, 20), 3) for s in range(n)]
    assert np.abs(z - np.array(ref)).max() > 1e-3
