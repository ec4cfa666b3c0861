"""The mixed path with its two streaming products on the tensor cores.

gpeps_set_tensor_cores moves the Gram blocks of the larger end and its update
(the absorb/reduce/contract products of the simple update, "Method") onto
tcgen05 kind::tf32 products with FP32 accumulators in tensor memory, each FP32
operand split into a TF32 pair (3xTF32, about 2^-22 relative per product).  The
bond eigenproblem, lambda and lambda^-1 stay FP64.  Tolerances are the mixed
path's: every qubit within 1e-4 of the FP64 oracle; lambda as in test_gpu_parity.
The fused step and the layered launches share the per-tile arithmetic, so the
two schedules must give the same state bit for bit, as they do on CUDA cores.
"""
import json
import os

import numpy as np
import pytest
import torch

from workloads import EAGLE, heavy_hex, workload

from ._gpu_util import gpu_lib, split
from .test_gpu_parity import lam_check

pytestmark = pytest.mark.gpu

TOL = 1e-4
M127, E127 = heavy_hex(*EAGLE)
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLD, f"oracle_{name}.json")) as f:
        return json.load(f)


def _run(graphs, D, theta, steps, schedule, tensor, layered=False):
    g = gpu_lib()(graphs, D, dtype="mixed")
    g.set_schedule(schedule)
    g.set_tensor_cores(tensor)
    g.reset()
    th = torch.tensor(theta, dtype=torch.float64, device="cuda")
    if layered:
        for _ in range(steps):
            g.kick(th)
            for c in range(g.n_colours):
                g.zz_layer(c)
    else:
        g.step(steps, th)
    z, _ = g.expect_z()
    state = g.state.clone()
    flags = g.status()
    g.close()
    return z.cpu().numpy(), state, flags


@pytest.mark.parametrize("D", [32, 64])
def test_tensor_cores_agree_with_cuda_cores(D):
    """127 qubits, theta = 0.7, 7 steps (truncated from step 6 at D = 32): the tensor-core
    products move no qubit by more than 1e-5 against the CUDA-core products (both FP32-level;
    the difference is rounding, well inside the 1e-4 budget of the mixed path)."""
    a = _run([(M127, E127)], D, [0.7], 7, 0, False, layered=True)
    b = _run([(M127, E127)], D, [0.7], 7, 0, True, layered=True)
    assert a[2] == 0 and b[2] == 0
    d = np.abs(a[0] - b[0]).max()
    assert d < 1e-5, d


@pytest.mark.parametrize("schedule", [6, 5, 4])
def test_tensor_cores_fused_step_bit_identical_benchmark_batch(schedule):
    """The benchmark batch (127 + 433 + 1121 qubits, D = 32), 7 steps: the fused step with four
    (schedule 6), three (schedule 5) or two (schedule 4) CTAs per SM and the layered launches give
    the same state bit for bit on the tensor cores (four CTAs hold 4 x 128 of the SM's 512 TMEM
    columns)."""
    w = workload("heavyhex_mix_d32")
    a = _run(w.graphs(), 32, [0.7] * 3, 7, 2, True, layered=True)
    b = _run(w.graphs(), 32, [0.7] * 3, 7, schedule, True)
    assert a[2] == 0 and b[2] == 0
    assert np.array_equal(a[0], b[0])
    assert torch.equal(a[1], b[1])


def test_tensor_cores_fused_step_bit_identical_d64():
    """127 qubits, D = 64 (N = 256 update products, two Gram products per tile), 7 steps."""
    a = _run([(M127, E127)], 64, [0.8], 7, 0, True, layered=True)
    b = _run([(M127, E127)], 64, [0.8], 7, 4, True)
    assert a[2] == 0 and b[2] == 0
    assert torch.equal(a[1], b[1])


@pytest.mark.parametrize("floor32,floor_rel", [(2e-7, 1e-7), (1e-7, 7e-8)])
def test_tensor_cores_benchmark_setting_matches_oracle(floor32, floor_rel):
    """The benchmark batch in the settings the autotuner chooses between for bench.py with the
    tensor cores on (fused step, three CTAs per SM, FP32 / FP64 stopping floors 2e-7 / 1e-7 or
    1e-7 / 7e-8 of the trace, four extra FP32 levels): every qubit at the committed steps 5, 6,
    10, 25 and 50 within 1e-4 of the FP64 oracle, and the sampled lambda spectra."""
    gold = _golden("heavyhex_mix_d32")
    w = workload("heavyhex_mix_d32")
    graphs = w.graphs()
    g = gpu_lib()(graphs, w.D, dtype="mixed")
    g.set_schedule(5)
    g.set_tensor_cores(True)
    g.set_jacobi(floor_rel=floor_rel, floor32=floor32)
    g.set_levels(level_ratio=1e-5, levels=4)
    g.reset()
    th = torch.tensor([0.7] * 3, dtype=torch.float64, device="cuda")
    done = 0
    for s in (5, 6, 10, 25, 50):
        g.step(s - done, th)
        done = s
        z, _ = g.expect_z()
        zi = split(z.cpu().numpy(), graphs)
        for k, inst in enumerate(gold["instances"]):
            d = float(np.abs(zi[k] - np.array(inst["z"][str(s)])).max())
            assert d < TOL, (s, k, d)
            for e, lam in inst["lambda"][str(s)].items():
                lam_check(g.lambdas(k, int(e)), np.array(lam), "mixed", truncated=2 ** s > w.D)
    assert g.status() == 0
    g.close()


def test_tensor_cores_eagle_d64_matches_oracle():
    """127 qubits, D = 64, theta = 0.8, 8 steps of the fused step on the tensor cores: every
    qubit and the sampled lambda at the committed steps, the mean of every step."""
    inst = _golden("eagle_d64")["instances"][0]
    w = workload("eagle_d64")
    g = gpu_lib()(w.graphs(), w.D, dtype="mixed")
    g.set_schedule(4)
    g.set_tensor_cores(True)
    g.reset()
    th = torch.tensor([0.8], dtype=torch.float64, device="cuda")
    done, means = 0, []
    for s in sorted(int(k) for k in inst["z"]):
        means.append(g.step(s - done, th).cpu().numpy()[:, 0])
        done = s
        z, _ = g.expect_z()
        assert np.abs(z.cpu().numpy() - np.array(inst["z"][str(s)])).max() < TOL, s
        for e, lam in inst["lambda"][str(s)].items():
            lam_check(g.lambdas(0, int(e)), np.array(lam), "mixed", truncated=2 ** s > w.D)
    means = np.concatenate(means)
    assert np.abs(means - np.array(inst["mean_z"][:done])).max() < TOL
    assert g.status() == 0
    g.close()


def test_tensor_cores_ragged_tiles_and_small_ends():
    """Sites of degree 1 and 2 as the larger end (32-row tiles at D = 32), a tree fragment and
    a 2-qubit graph, against the CUDA-core products (1e-5) and the oracle (1e-4)."""
    from oracle import su
    from workloads import induced_subgraph
    n, e, _ = induced_subgraph(E127, list(range(20)))
    for graph in ((n, e), (2, np.array([[0, 1]], dtype=np.int32))):
        a = _run([graph], 32, [0.9], 6, 0, False, layered=True)
        b = _run([graph], 32, [0.9], 6, 0, True, layered=True)
        assert a[2] == 0 and b[2] == 0
        assert np.abs(a[0] - b[0]).max() < 1e-5
        peps = su.GPEPS(graph[0], graph[1], 32)
        for _ in range(6):
            peps.step(0.9)
        assert np.abs(b[0] - peps.expect_z()).max() < TOL


def test_tensor_cores_rejected_where_unsupported():
    """complex128 handles and bond dimensions other than 32 and 64 keep the CUDA-core products."""
    G = gpu_lib()
    for dtype, D in (("c128", 32), ("mixed", 16), ("mixed", 8)):
        g = G([(M127, E127)], D, dtype=dtype)
        with pytest.raises(RuntimeError):
            g.set_tensor_cores(True)
        g.set_tensor_cores(False)
        g.close()


def test_tensor_cores_bp_regauge_matches_oracle_golden():
    """BP regauging with the message products on the tensor cores (leg products and message
    Gram, 3xTF32) and the simple update's passes too: 127 qubits, D = 32, theta = 0.7, a regauge
    to convergence after each of 8 steps; the mean of every step, every qubit and the sampled
    lambda at the committed steps against the FP64 oracle (the mixed path's tolerances)."""
    from workloads import workload
    from .test_gpu_bp import lam_close
    inst = _golden("eagle_bp_d32")["instances"][0]
    w = workload("eagle_bp_d32")
    g = gpu_lib()(w.graphs(), w.D, dtype="mixed")
    g.set_tensor_cores(True)
    g.reset()
    th = torch.tensor([w.theta[0]], dtype=torch.float64, device="cuda")
    for s in range(1, w.steps + 1):
        g.step(1, th)
        it, res = g.bp_regauge(300)
        assert it < 300, (s, it, res)
        z, mean = g.expect_z()
        assert abs(float(mean.cpu().numpy()[0]) - inst["mean_z"][s - 1]) < TOL, s
        if str(s) in inst["z"]:
            assert np.abs(z.cpu().numpy() - np.array(inst["z"][str(s)])).max() < TOL, s
            for e, lam in inst["lambda"][str(s)].items():
                assert lam_close(g.lambdas(0, int(e)), lam, "mixed", truncated=2 ** s > w.D), (s, e)
    assert g.status() == 0
    g.close()


def test_tensor_core_messages_agree_with_cuda_cores():
    """From one state (127 qubits, D = 32, 7 steps: sites of degree 1, 2 and 3, truncated bonds),
    a regauge with the tensor-core message products and one with the CUDA-core products reach
    the same <Z_i> within 1e-5 and the same lambda spectra within 1e-4."""
    g = gpu_lib()([(M127, E127)], 32, dtype="mixed")
    g.reset()
    th = torch.tensor([0.7], dtype=torch.float64, device="cuda")
    g.step(7, th)
    saved = g.save_state()
    out = {}
    for tc in (False, True):
        g.load_state(saved)
        g.set_tensor_cores(tc)
        it, res = g.bp_regauge(300)
        assert it < 300, (tc, it, res)
        z, _ = g.expect_z()
        out[tc] = (z.cpu().numpy(), np.array([g.lambdas(0, e) for e in (0, 50, 100, 143)]))
    assert g.status() == 0
    g.close()
    assert np.abs(out[True][0] - out[False][0]).max() < 1e-5
    assert np.abs(out[True][1] - out[False][1]).max() < 1e-4
