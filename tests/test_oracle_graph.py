"""Edge colouring (update order) of the oracle."""
import numpy as np
import pytest

from oracle.graph import greedy_colouring, neighbours
from workloads import LATTICES, heavy_hex


@pytest.mark.parametrize("n,sizes", [(127, (54, 51, 39)), (433, (180, 174, 150)), (1121, (460, 450, 410))])
def test_three_colours_matchings(n, sizes):
    m, e = heavy_hex(*LATTICES[n])
    col = greedy_colouring(e)
    assert col.max() == 2
    assert tuple(np.bincount(col)) == sizes
    for c in range(3):
        ends = e[col == c].ravel()
        assert len(np.unique(ends)) == len(ends)      # a matching


def test_neighbours_sorted():
    m, e = heavy_hex(*LATTICES[127])
    nb = neighbours(m, e)
    assert all(x == sorted(x) for x in nb)
    assert sum(len(x) for x in nb) == 2 * len(e)
