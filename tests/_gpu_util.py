"""Helpers of the GPU tests: run the CUDA path through the Python binding of the C ABI."""
import numpy as np
import torch


def gpu_lib():
    from paper_2309_15642_gb300 import _build
    _build.build()
    from paper_2309_15642_gb300 import GPEPS
    return GPEPS


def run_layers(graphs, D, dtype, theta, steps, per_qubit=False, colours=None):
    """Explicit calls: kick, every colour class, expect_z, per step.

    Returns (z[steps, total_qubits], mean[steps, n_inst], object)."""
    GPEPS = gpu_lib()
    g = GPEPS(graphs, D, dtype=dtype, colours=colours)
    g.reset()
    th = torch.as_tensor(np.asarray(theta, dtype=np.float64), device="cuda")
    zs, ms = [], []
    for _ in range(steps):
        g.kick(th, per_qubit=per_qubit)
        for c in range(g.n_colours):
            g.zz_layer(c)
        z, m = g.expect_z()
        zs.append(z.cpu().numpy())
        ms.append(m.cpu().numpy())
    assert g.status() == 0
    return np.array(zs), np.array(ms), g


def run_step(graphs, D, dtype, theta, steps, per_qubit=False, check_status=True):
    """gpeps_step (captured CUDA graph replay), the launch configuration of bench.py."""
    GPEPS = gpu_lib()
    g = GPEPS(graphs, D, dtype=dtype)
    g.reset()
    th = torch.as_tensor(np.asarray(theta, dtype=np.float64), device="cuda")
    means = g.step(steps, th, per_qubit=per_qubit)
    out = means.cpu().numpy()
    if check_status:
        assert g.status() == 0
    return out, g


def split(z, graphs):
    """Per-instance slices of a [.., total_qubits] array."""
    out, o = [], 0
    for n, _ in graphs:
        out.append(z[..., o:o + n])
        o += n
    return out
