"""The fused step (schedule 4): every bond update of a Trotter step in one persistent launch,
bonds taken colour class by colour class, each waiting only for the earlier bonds on its two
sites.  Its arithmetic is the layered launches' (the Gram pass summed in FP64 in tile order),
so the results must equal theirs bit for bit; a wait that gives up (here forced with a zero
wait limit: no GPU fault, no hang) must raise GPEPS_FLAG_TIMEOUT and leave the context usable.
"""
import numpy as np
import pytest
import torch

from workloads import EAGLE, heavy_hex, workload

from ._gpu_util import gpu_lib

pytestmark = pytest.mark.gpu

M127, E127 = heavy_hex(*EAGLE)
FLAG_TIMEOUT = 4


def _run(graphs, D, dtype, theta, steps, schedule):
    g = gpu_lib()(graphs, D, dtype=dtype)
    g.set_schedule(schedule)
    g.reset()
    m = g.step(steps, torch.tensor(theta, dtype=torch.float64, device="cuda")).cpu().numpy()
    z, _ = g.expect_z()
    lam = g.state.clone()
    flags = g.status()
    g.close()
    return m, z.cpu().numpy(), lam, flags


def test_four_ctas_per_sm_fused_step_bit_identical_benchmark_batch():
    """The benchmark batch at D = 32 (mixed) with four 192-thread fused-step CTAs per SM
    (schedule 6): the same state as the layered launches after 7 steps."""
    w = workload("heavyhex_mix_d32")
    a = _run(w.graphs(), 32, "mixed", [0.7] * 3, 7, 2)
    b = _run(w.graphs(), 32, "mixed", [0.7] * 3, 7, 6)
    assert a[3] == 0 and b[3] == 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert torch.equal(a[2], b[2])


@pytest.mark.parametrize("dtype", ["mixed", "c128"])
def test_fused_step_bit_identical_benchmark_batch(dtype):
    """127 + 433 + 1121 qubits, D = 32, theta = 0.7, 7 steps: the whole state after the fused
    steps equals the state after the layered launches (schedule 2)."""
    w = workload("heavyhex_mix_d32")
    a = _run(w.graphs(), 32, dtype, [0.7] * 3, 7, 2)
    b = _run(w.graphs(), 32, dtype, [0.7] * 3, 7, 4)
    assert a[3] == 0 and b[3] == 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert torch.equal(a[2], b[2])


def test_three_ctas_per_sm_fused_step_bit_identical_benchmark_batch():
    """The benchmark batch at D = 32 (mixed) with three 192-thread fused-step CTAs per SM
    (schedule 5, the autotuner's choice): the same state as the layered launches after 7 steps."""
    w = workload("heavyhex_mix_d32")
    a = _run(w.graphs(), 32, "mixed", [0.7] * 3, 7, 2)
    b = _run(w.graphs(), 32, "mixed", [0.7] * 3, 7, 5)
    assert a[3] == 0 and b[3] == 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert torch.equal(a[2], b[2])


@pytest.mark.parametrize("dtype", ["mixed", "c128"])
def test_fused_step_bit_identical_d64(dtype):
    """127 qubits, D = 64 (128 x 128 eigenproblems, one CTA per SM), 7 steps."""
    a = _run([(M127, E127)], 64, dtype, [0.8], 7, 0)
    b = _run([(M127, E127)], 64, dtype, [0.8], 7, 4)
    assert a[3] == 0 and b[3] == 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert torch.equal(a[2], b[2])


def test_fused_step_wait_timeout_is_reported():
    """A zero wait limit makes every wait on a running dependency give up at once: the launch
    ends, GPEPS_FLAG_TIMEOUT is raised, and the device stays usable (a new handle then runs
    clean and agrees with the layered launches)."""
    g = gpu_lib()([(M127, E127)], 8, dtype="mixed")
    g.set_schedule(4)
    g.set_wait_limit(0)
    g.reset()
    g.step(2, torch.tensor([0.7], dtype=torch.float64, device="cuda"))
    assert g.status() & FLAG_TIMEOUT
    g.close()
    a = _run([(M127, E127)], 8, "mixed", [0.7], 3, 0)
    b = _run([(M127, E127)], 8, "mixed", [0.7], 3, 4)
    assert a[3] == 0 and b[3] == 0 and np.array_equal(a[0], b[0])
