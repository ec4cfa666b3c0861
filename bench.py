#!/usr/bin/env python
"""Benchmark of the simple-update Trotter step (bond updates/s) on one GB300 per rank.

Workload (default ``heavyhex_mix_d32``): one batch of the 127-, 433- and
1121-qubit heavy-hex lattices (1968 bond updates per Trotter step), bond
dimension D = 32, theta_h = 0.7, started from |0...0>, synthetic (the lattices
stand in for the processors' coupling maps).  A step is one Trotter step of
the whole batch: kick, three colour classes of bond updates, mean-field <Z>.

``--impl gpeps`` (default) times the CUDA library: W warm-up steps, then K
steps replayed from the captured step graph, bracketed by CUDA events on the
library's stream; the state (>= 307 MB) is larger than L2, so no flush is
needed.  It also reports the complex128 path on the same batch, per-kernel
times of the dominant kernel against the FP64 ALU roofline, an end-to-end
number through the public API with host buffers, and the FP64 CPU oracle
timed on a bounded sample.  ``--impl reference`` times the oracle alone.

``--bp`` times Trotter steps with a belief-propagation regauge after each (the
paper's BP comparison): value = Trotter steps/s of the batch, with the BP
iterations, the per-phase device times and the message kernel's roofline.

Multi-GPU (torchrun): replicas only.  Every rank evolves its own copy of the
batch; there is no collective on the data path; value = all ranks' bond
updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bond updates/s at D=32 (mixed vs FP64 plain, |d<Z>|<=1e-4); % of roofline"
# FP64 vector peak from the unit counts and the maximum SM clock: 152 SMs x 2 FP64 FMA per clock
# x 2 flops x 2.07 GHz (an FP64 FMA loop on this part measured 1197 GFLOP/s)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpeps", choices=["gpeps", "reference"])
    ap.add_argument("--workload", default="heavyhex_mix_d32")
    ap.add_argument("--dtype", default="mixed", choices=["mixed", "c128"])
    ap.add_argument("--no-plain", action="store_true", help="skip the complex128 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--profile-steps", type=int, default=2, help="profiled steps after the timed region (>= 1)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default schedule and thresholds")
    ap.add_argument("--schedule", type=int, default=None,
                    help="with --no-autotune: bond schedule (0 one CTA per bond; 1, 2, 3 work queue with 1, 2, 4 "
                         "CTAs per SM; 4, 5, 6 the fused step with up to 2, 3, 4 CTAs per SM)")
    ap.add_argument("--bp", action="store_true",
                    help="time Trotter steps with a belief-propagation regauge after each (the paper's BP "
                         "comparison) instead of the plain step")
    ap.add_argument("--bp-max-iter", type=int, default=200)
    ap.add_argument("--no-condor", action="store_true",
                    help="skip the sub-records (1121-qubit D = 64, BP regauging, D = 128)")
    ap.add_argument("--cpu-leg", action="store_true",
                    help="internal: time one leg of the CPU oracle baseline and print it as JSON")
    ap.add_argument("--tensor", action="store_true",
                    help="with --no-autotune: Gram and update passes on the tensor cores (mixed, D = 32 or 64)")
    ap.add_argument("--floor-rel", type=float, default=None,
                    help="with --no-autotune: FP64 Jacobi floor (fraction of the trace) of the mixed path")
    ap.add_argument("--floor32", type=float, default=None,
                    help="with --no-autotune and --floor-rel: FP32-level floor (fraction of the trace) of the "
                         "mixed path")
    return ap.parse_args()


# ------------------------------------------------------------------ replicas (N > 1)
def max_over_ranks(ms, device=None):
    """The largest of every rank's time (all-reduce MAX); the time itself without a process
    group.  ``device``: where the reduction tensor lives (the rank's GPU under NCCL, the CPU
    under gloo)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ms_max, world):
    """Units of every replica over the slowest rank's time: the whole job's rate."""
    return world * units_per_rank / (ms_max * 1e-3)


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampler (200 ms) running while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons, power = [], [], set(), []
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                pass
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows),
                "power_w_max": max(power) if power else None}


# DRAM bytes per launch of the dominant kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by workload, dtype and schedule; reported as the roofline's
# `traffic` only for that configuration (profiles/step_kernel_heavyhex_mix_d32.md)
# and whether the Gram and update passes ran on the tensor cores
NCU_TRAFFIC = {
    # one steady-state launch (Trotter step 8) of the fused step, floors 1e-7 / 7e-8: three and four
    # CTAs per SM, each with the CUDA-core and with the tensor-core Gram and update passes
    ("heavyhex_mix_d32", "mixed", 5, False): 2253342208 + 2040923904,
    ("heavyhex_mix_d32", "mixed", 5, True): 2443752000 + 2472390000,
    ("heavyhex_mix_d32", "mixed", 6, False): 2417434000 + 2293279000,
    ("heavyhex_mix_d32", "mixed", 6, True): 2693205760 + 2721358336}

# TF32 tensor peak: the measured bf16 burst (MEASURED_PEAKS.json) x the nominal TF32 : BF16 dense ratio
# (1.1 : 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25

# ------------------------------------------------------------------ algorithmic counts
def bond_fixed_flops(graphs, D, dtype):
    """(FP64, FP32) flops of one Trotter step's bond eigenproblems that do not depend on how the
    Jacobi sweeps converge, per bond with its own n = 2 D^(deg - 1) (deg of the smaller end;
    8 flops per complex MAC).  Mixed path (squared form): of the re-orthonormalisation of the FP32
    eigenvectors, E = V^dagger V - I (n^3 / 2 MACs) and Q = V R^-1 (n^3 / 2) in FP64 and the
    E-sized products X1^dagger X1 and X^2 (n^3 / 6 MACs each) in FP32; rho' = V^dagger rho V
    3 n^3 / 2 MACs in FP64; the rho formation 2 (n D^2 + n(n+1)/2 D) MACs and the Y matrices
    2 D^2 n MACs in FP32.  Complex128
    (unsquared form, all FP64): the pivoted Cholesky roots of the two D x D Gram blocks 2 D^3 / 3
    MACs, the core M = 2D x n, 2D n D MACs, the re-orthonormalisation 4 n^3 / 3, B = M V0 2D n^2
    and the Y matrices 2 D^2 n MACs.  The Jacobi sweeps and the levels are counted in the kernel."""
    import numpy as np
    f64 = f32 = 0.0
    for n_q, edges in graphs:
        deg = np.bincount(np.asarray(edges).ravel(), minlength=n_q)
        for a, b in edges:
            n = 2 * D ** (int(min(deg[a], deg[b])) - 1)
            if dtype == "c128":
                f64 += (2.0 * D ** 3 / 3 + 2 * D * n * D + 4.0 * n ** 3 / 3 + 2 * D * n * n + 2 * D * D * n) * 8
                continue
            f64 += (n ** 3 + 1.5 * n ** 3) * 8
            f32 += (2 * (n * D * D + n * (n + 1) / 2 * D) + 2 * D * D * n + n ** 3 / 3.0) * 8
    return f64, f32


# flops of one executed Jacobi 2x2 block update (both sides) and one eigenvector pair update
# (two-sided, mixed path)
JACOBI_BLOCK_FLOPS, JACOBI_VEC_FLOPS = 72, 18


def one_sided_flops(D, checks, rotations):
    """Real flops of the complex128 one-sided sweeps: a pair check forms |b_p|^2, |b_q|^2 and
    b_p^H b_q over the 2D rows (16 flops per row), a rotation updates 2D rows of B and n <= 2D
    rows of V (18 flops per row pair; counted at n = 2D)."""
    return checks * 16 * 2 * D + rotations * 18 * 4 * D


# ------------------------------------------------------------------ committed oracle values
def load_golden(w):
    """The committed FP64 oracle values of workload ``w`` (tests/golden), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{w.name}.json")
    return json.load(open(path)) if os.path.exists(path) else None


def golden_z(gold, step):
    """Per-qubit <Z> of every instance after ``step`` steps, concatenated (or None)."""
    import numpy as np
    if gold is None or any(str(step) not in inst["z"] for inst in gold["instances"]):
        return None
    return np.concatenate([np.asarray(inst["z"][str(step)], dtype=np.float64) for inst in gold["instances"]])


# FP32 vector peak from the unit counts and the maximum SM clock: 152 SMs x 128 FP32 FMA per
# clock x 2 flops x 2.07 GHz
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07


def bp_message_flops(graphs, D):
    """Real flops of one BP iteration (every message of the batch): per message of a site of
    degree z, (z - 1) leg products of 2 D^(z+1) complex MACs and the upper triangle of the Gram,
    D (D + 1) / 2 entries of 2 D^(z-1) complex MACs; 8 real flops per complex MAC."""
    import numpy as np
    total = 0
    for n, edges in graphs:
        deg = np.bincount(np.asarray(edges).reshape(-1), minlength=n)
        for z in deg:
            z = int(z)
            if z == 0:
                continue
            cmac = (z - 1) * 2 * D ** (z + 1) + D * (D + 1) // 2 * 2 * D ** (z - 1)
            total += z * 8 * cmac
    return float(total)


def cpu_oracle_bp(w, seconds_cap=10.0):
    """The FP64 oracle's BP messages on a bounded sample: the first lattice of the batch after
    two Trotter steps, message updates (the half-edges in turn, degree-3 sites first, from
    identity messages) until ``seconds_cap`` seconds have passed.  Returns BP message updates/s."""
    import numpy as np
    from oracle import bp
    from oracle.su import GPEPS as OraclePEPS
    from workloads import kick_angles
    (n, edges) = w.graphs()[0]
    th = kick_angles(w)[0]
    peps = OraclePEPS(n, edges, w.D)
    for _ in range(2):
        peps.step(th)
    msgs = bp.identity_messages(peps)
    keys = sorted(msgs, key=lambda k: -len(peps.nb[k[0]]))
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < seconds_cap:
        i, p = keys[done % len(keys)]
        bp.message(peps, i, p, msgs)
        done += 1
    dt = time.perf_counter() - t0
    deg = np.array([len(peps.nb[keys[k % len(keys)][0]]) for k in range(done)])
    return {"value": done / dt, "unit": "BP message updates/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} message updates ({int((deg == 3).sum())} of degree-3 sites) of the {n}-qubit "
                      f"lattice at D={w.D} after 2 steps, numpy FP64, {dt:.1f} s"}


def run_bp(args, local_rank):
    """Trotter steps with a BP regauge after each: W untimed, then K timed (CUDA events on the
    library's stream around step + regauge, the regauge's per-iteration convergence test
    included)."""
    import torch
    from paper_2309_15642_gb300 import _build
    _build.build()
    from paper_2309_15642_gb300 import GPEPS
    from workloads import kick_angles, workload

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = workload(args.workload)
    graphs = w.graphs()
    theta = [float(t[0]) for t in kick_angles(w)]
    K, W = args.steps, args.warmup
    g = GPEPS(graphs, w.D, dtype=args.dtype, device=str(dev))
    tuning = None
    if not args.no_autotune:
        from paper_2309_15642_gb300.autotune import autotune
        best, _ = autotune(g, theta)
        tuning = best
    else:
        if args.tensor and args.dtype == "mixed":
            g.set_tensor_cores(True)
        g.set_schedule(args.schedule or 0)
        if args.floor_rel is not None and args.dtype == "mixed":
            g.set_jacobi(floor_rel=args.floor_rel, **({} if args.floor32 is None else {"floor32": args.floor32}))
    g.reset()
    th = torch.tensor(theta, dtype=torch.float64, device=dev)
    out = torch.empty((1, g.n_instances), dtype=torch.float64, device=dev)
    for _ in range(W):
        g.step(1, th, out=out)
        g.bp_regauge(args.bp_max_iter)
    torch.cuda.synchronize(dev)
    clocks = Clocks(local_rank)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, phases, su_ms = [], [0.0, 0.0, 0.0], 0.0
    means = []
    # every step: the kick angles from pinned host memory, the Trotter step, the regauge and
    # the mean <Z> back to the host (the regauge's convergence test synchronises anyway)
    th_host = torch.tensor(theta, dtype=torch.float64).pin_memory()
    mean_host = torch.empty(g.n_instances, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e0.record(g.stream)
    for _ in range(K):
        th.copy_(th_host, non_blocking=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(g.stream)
        g.step(1, th, out=out)
        b.record(g.stream)
        it, res, ms3 = g.bp_regauge(args.bp_max_iter, profile=True)
        b.synchronize()
        su_ms += a.elapsed_time(b)
        iters.append(it)
        phases = [x + y for x, y in zip(phases, ms3)]
        z, m = g.expect_z()
        mean_host.copy_(m, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        means.append(mean_host.numpy().tolist())
    e1.record(g.stream)
    e1.synchronize()
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    flags = g.status()
    n_msg = sum(2 * len(e) for _, e in graphs)
    flops_iter = bp_message_flops(graphs, w.D)
    msg_launch_ms = phases[0] / max(sum(iters), 1)
    achieved = flops_iter / (msg_launch_ms * 1e-3) / 1e9
    peak = FP64_PEAK_GFLOPS if args.dtype == "c128" else FP32_PEAK_GFLOPS
    roofline = {"kernel": "bp_message_kernel (every BP message of the batch: leg products with the neighbours' "
                          "environments and the Hermitian Gram, one launch per iteration)",
                "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "GFLOP/s (FP64)" if args.dtype == "c128" else "GFLOP/s (FP32)",
                "frac": achieved / peak,
                "peak_source": ("derived: 152 SMs x 2 FP64 FMA/clock x 2 flops x 2.07 GHz" if args.dtype == "c128"
                                else "derived: 152 SMs x 128 FP32 FMA/clock x 2 flops x 2.07 GHz"),
                "traffic": None, "flops_per_launch": flops_iter, "launch_ms": msg_launch_ms,
                "units_per_launch": n_msg}
    e2e = {"value": K / wall, "unit": "Trotter steps/s with BP regauging",
           "h2d_bytes_per_step": th_host.numel() * 8, "d2h_bytes_per_step": mean_host.numel() * 8}
    g.close()
    return dict(value=K / (ms * 1e-3), ms=ms, clocks=ck, flags=flags, roofline=roofline, iters=iters,
                phases_ms=[x / K for x in phases], su_ms=su_ms / K, n_msg=n_msg, means=means, w=w,
                tuning=tuning, e2e=e2e)


def big_end_flops(graphs, D):
    """FP32 flops of the Gram and update passes over the larger ends of one Trotter step: per
    bond 4 D^2 R complex MACs (8 flops each), R = D^(deg - 1) rows of the larger end."""
    import numpy as np
    tot = 0
    for n, edges in graphs:
        deg = np.bincount(np.asarray(edges).ravel(), minlength=n)
        for a, b in edges:
            rows = D ** (int(max(deg[a], deg[b])) - 1)
            tot += 4 * D * D * rows * 8
    return float(tot)


def tc_executed_flops(graphs, D):
    """TF32 flops the tensor-core Gram and update passes execute in one Trotter step (3xTF32: three
    products per operand pair).  Gram: per 32-row chunk of the larger end (rows padded to a multiple
    of 8), one 128 x 128 product (D = 32: over all 4D columns) or two (D = 64: one per spin).
    Update: per 128 rows, an M = 128 x N = 4D x K = 4D product."""
    import numpy as np
    tot = 0
    for n, edges in graphs:
        deg = np.bincount(np.asarray(edges).ravel(), minlength=n)
        for a, b in edges:
            rows = D ** (int(max(deg[a], deg[b])) - 1)
            ngm = 2 if D == 64 else 1
            for r0 in range(0, rows, 32):
                kc8 = (min(32, rows - r0) + 7) // 8 * 8
                tot += ngm * 2 * 128 * 128 * kc8
            tot += ((rows + 127) // 128) * 2 * 128 * (4 * D) * (4 * D)
    return 3.0 * tot


def tf32_peak_tflops():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        v = json.load(open(path)).get("bf16_tflops")
        if v:
            return float(v) * TF32_OVER_BF16, "measured bf16 burst x nominal TF32/BF16 ratio 1.1/2.25"
    return 1900.0 * TF32_OVER_BF16, "fallback bf16 1.9 PFLOP/s x nominal TF32/BF16 ratio 1.1/2.25"


def tensor_pipe_record(graphs, D, kernel_ms, on):
    """Tensor-pipe use of the dominant kernel: the TF32 flops its tensor-core passes executed over
    its launch time, against the TF32 peak (a kernel-average figure: the step is FP64-bound)."""
    if not on:
        return {"tensor_cores": False, "utilisation": 0.0,
                "note": "Gram and update passes on CUDA cores (the autotuner's or the caller's choice)"}
    f = tc_executed_flops(graphs, D)
    peak, src = tf32_peak_tflops()
    achieved = f / (kernel_ms * 1e-3) / 1e12
    return {"tensor_cores": True, "tf32_flops_per_launch": f, "achieved_tflops": achieved, "peak_tflops": peak,
            "frac": achieved / peak, "peak_source": src,
            "note": "tcgen05 kind::tf32 (3xTF32) Gram and update passes; kernel-average rate over the whole "
                    "launch, which the FP64 bond eigenproblems dominate"}


def step_bytes(graphs, D, elt):
    """Algorithmic HBM bytes of one Trotter step: every bond reads and writes both site
    tensors once (its larger end twice: Gram and update pass), the readout reads every
    tensor once; lambda vectors are negligible."""
    tot = 0
    for n, edges in graphs:
        import numpy as np
        deg = np.bincount(np.asarray(edges).ravel(), minlength=n)
        size = {int(d): 2 * D ** int(d) * elt for d in set(deg.tolist())}
        for a, b in edges:
            sa, sb = size[int(deg[a])], size[int(deg[b])]
            big, small = max(sa, sb), min(sa, sb)
            tot += 3 * big + 2 * small
        tot += sum(size[int(d)] for d in deg)
    return tot


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_leg(w, warmup, seconds_cap):
    """The FP64 oracle on the first lattice of the batch, in the GPU arm's steady-state window:
    ``warmup`` Trotter steps from |0...0> untimed, then whole Trotter steps (kick, every colour
    class, readout) timed while fewer than ``seconds_cap`` seconds have passed (at least one)."""
    import numpy as np
    from oracle.su import GPEPS as OraclePEPS
    from workloads import kick_angles
    (n, edges) = w.graphs()[0]
    th = kick_angles(w)[0]
    peps = OraclePEPS(n, edges, w.D)
    for _ in range(warmup):
        peps.step(th)
    t0 = time.perf_counter()
    steps = 0
    while steps == 0 or (time.perf_counter() - t0 < seconds_cap and warmup + steps < w.steps):
        peps.step(th)
        peps.expect_z()
        steps += 1
    dt = time.perf_counter() - t0
    return {"bond_updates_per_s": len(edges) * steps / dt, "trotter_steps_per_s": steps / dt,
            "window": f"{warmup + 1}..{warmup + steps}", "seconds": dt, "qubits": n, "bonds_per_step": len(edges)}


def cpu_oracle(w, warmup, seconds_cap=10.0):
    """Oracle baseline, two legs over the same window: numpy/LAPACK with its default thread
    count, and a child process whose BLAS/OpenMP pools are set to one thread before numpy loads."""
    allt = cpu_oracle_leg(w, warmup, seconds_cap)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    single = None
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", "--workload", w.name,
                            "--warmup", str(warmup)], env=env, capture_output=True, text=True, timeout=900)
        if r.returncode == 0 and r.stdout.strip():
            single = json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.TimeoutExpired, ValueError):
        single = None
    def sample(leg):
        return (f"{leg['qubits']}-qubit lattice of the batch, D={w.D}, Trotter steps {leg['window']} after "
                f"{warmup} untimed warm-up steps from |0...0> (the GPU arm's steady-state window), "
                f"numpy/LAPACK FP64")
    return {"value": allt["bond_updates_per_s"], "unit": "bond updates/s", "cores": os.cpu_count(),
            "kind": "oracle", "sample": sample(allt) + ", default BLAS threads",
            "trotter_steps_per_s_of_sample": allt["trotter_steps_per_s"], "seconds": allt["seconds"],
            "single_thread": None if single is None else {
                "value": single["bond_updates_per_s"], "unit": "bond updates/s", "cores": 1,
                "window": single["window"], "seconds": single["seconds"],
                "sample": sample(single) + ", OMP/OPENBLAS/MKL_NUM_THREADS=1"}}


def golden_parity(w, means, W, K):
    """max |mean <Z> - oracle| over the timed steps W+1..W+K, from the committed oracle values."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{w.name}.json")
    if not os.path.exists(path):
        return None
    gold = json.load(open(path))
    ref = np.array([inst["mean_z"] for inst in gold["instances"]]).T      # [steps, instances]
    if W + K > ref.shape[0]:
        return None
    d = float(np.abs(means[:K] - ref[W:W + K]).max())
    return {"max_abs_dmean_z": d, "steps": f"{W + 1}..{W + K}", "reference": "FP64 CPU oracle (committed values)"}


def site_parity(g, w, th, first, last):
    """Per-qubit parity of the setting just timed: the handle (as tuned) is reset and stepped to
    every step s in [first, last] that has committed oracle values; max_i |<Z_i> - oracle| over
    those steps and max |lambda - oracle| over the committed edges.  Runs after the timed region."""
    import numpy as np
    gold = load_golden(w)
    if gold is None:
        return None
    steps = sorted(int(k) for k in gold["instances"][0]["z"] if first <= int(k) <= last)
    if not steps:
        return None
    g.reset()
    done, dz, dl = 0, 0.0, 0.0
    for st in steps:
        g.step(st - done, th)
        done = st
        z, _ = g.expect_z()
        dz = max(dz, float(np.abs(z.cpu().numpy() - golden_z(gold, st)).max()))
        for k, inst in enumerate(gold["instances"]):
            for e, lam in inst["lambda"].get(str(st), {}).items():
                dl = max(dl, float(np.abs(g.lambdas(k, int(e)) - np.asarray(lam)).max()))
    return {"max_abs_dz_per_qubit": dz, "max_abs_dlambda_sampled": dl, "steps": steps}


def parity_record(g, w, th, means, W, K):
    """Mean <Z> of every timed step and every qubit at the committed steps inside the window."""
    out = golden_parity(w, means, W, K)
    site = site_parity(g, w, th, W + 1, W + K)
    if out is None:
        return site
    if site is not None:
        out.update(max_abs_dz_per_qubit=site["max_abs_dz_per_qubit"], per_qubit_steps=site["steps"],
                   max_abs_dlambda_sampled=site["max_abs_dlambda_sampled"])
    return out


# ------------------------------------------------------------------ GPU arm
def run_gpeps(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2309_15642_gb300 import _build
    _build.build()
    from paper_2309_15642_gb300 import GPEPS
    from workloads import kick_angles, workload

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = workload(args.workload)
    graphs = w.graphs()
    theta = [float(t[0]) for t in kick_angles(w)]
    K, W = args.steps, args.warmup
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def timed(dtype, K, W, tune):
        g = GPEPS(graphs, w.D, dtype=dtype, device=str(dev))
        tuning = None
        if not tune:
            if args.schedule is not None:
                g.set_schedule(args.schedule)
            if args.floor_rel is not None and dtype == "mixed":
                g.set_jacobi(floor_rel=args.floor_rel, **({} if args.floor32 is None else {"floor32": args.floor32}))
            if args.tensor and dtype == "mixed":
                g.set_schedule(0)
                g.set_tensor_cores(True)
                g.set_schedule(args.schedule or 0)
        if tune:
            from paper_2309_15642_gb300.autotune import autotune
            # candidates are also held to the committed oracle values after the tuner's 6 + 4 steps
            best, table = autotune(g, theta, warm_steps=6, steps=4, reference_z=golden_z(load_golden(w), 10))
            tuning = {"chosen": best, "candidates": table}
        g.reset()
        th = torch.tensor(theta, dtype=torch.float64, device=dev)
        out = torch.empty((max(K, 1), g.n_instances), dtype=torch.float64, device=dev)
        g.step(W, th)
        torch.cuda.synchronize(dev)
        if dist:
            tdist.barrier()
        clocks = Clocks(local_rank) if rank == 0 else None
        if clocks:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(g.stream)
        g.step(K, th, out=out)
        e1.record(g.stream)
        e1.synchronize()
        torch.cuda.synchronize(dev)
        ck = clocks.stop() if clocks else None
        ms = max_over_ranks(e0.elapsed_time(e1), device=dev)
        flags = g.status()
        return g, th, out, ms, ck, flags, tuning

    g, th, out, ms, clocks, flags, tuning = timed(args.dtype, K, W, not args.no_autotune)
    bonds_step = g.bonds_per_step
    value = whole_job_rate(bonds_step * K, ms, world)
    mean_last = out[K - 1].cpu().numpy().tolist() if K else []

    # per-kernel durations of profiled steps right after the timed region, under the schedule
    # of the timed region (fused: one launch per step; layered: three per colour class)
    sched = (tuning["chosen"].get("persistent", 0) if tuning else (args.schedule or 0))
    tensor = bool(tuning["chosen"].get("tensor", False)) if tuning else (args.tensor and args.dtype == "mixed")
    fused = sched >= 4          # schedules 4, 5 and 6: the fused step (two, three or four CTAs per SM)
    prof = {"gram": [], "bond": [], "update": []} if not fused else {"kick": [], "bond_updates": [], "readout": []}
    s0, q0, b0 = g.sweeps()
    c0 = g.bond_counters()
    w0 = g.jacobi_work()
    for _ in range(args.profile_steps):
        if fused:
            for k, v in zip(("kick", "bond_updates", "readout"), g.step_profiled(th)):
                prof[k].append(v)
            continue
        g.kick(th)
        for c in range(g.n_colours):
            t3 = g.zz_layer_profiled(c)
            for k, v in zip(("gram", "bond", "update"), t3):
                prof[k].append(v)
        g.expect_z()
    s1, q1, b1 = g.sweeps()
    c1 = g.bond_counters()
    w1 = g.jacobi_work()
    work_step = [(b - a) / max(args.profile_steps, 1) for a, b in zip(w0, w1)]
    phase_names = ["rho", "fp32_jacobi", "fp64_orthonormalise", "rotate_and_fp32_levels", "fp64_jacobi",
                   "epilogue"]
    phase_cycles = {k: (b - a) / max(b1 - b0, 1) for k, a, b in zip(phase_names, c0, c1)}
    if fused:  # the Gram and update passes of the larger end inside the fused step
        phase_cycles["gram_pass"] = (c1[22] - c0[22]) / max(b1 - b0, 1)
        phase_cycles["update_pass"] = (c1[23] - c0[23]) / max(b1 - b0, 1)
    sweeps_per_bond = (s1 - s0) / max(b1 - b0, 1)
    sweeps32_per_bond = (q1 - q0) / max(b1 - b0, 1)
    layer_ms = {k: sum(v) / max(args.profile_steps, 1) for k, v in prof.items()}   # per step, all colours
    # flops of one step's bond eigenproblems: the fixed dense phases plus the Jacobi work the
    # kernel executed (counted in the kernel; converged pairs are skipped and not counted)
    fix64, fix32 = bond_fixed_flops(graphs, w.D, args.dtype)
    if args.dtype == "c128":   # one-sided sweeps: the counters are pair checks and rotations
        f64_step = fix64 + one_sided_flops(w.D, work_step[0], work_step[1]) + work_step[4] * 8
        f32_step = fix32 + one_sided_flops(w.D, work_step[2], work_step[3])
    else:
        f64_step = fix64 + work_step[0] * JACOBI_BLOCK_FLOPS + work_step[1] * JACOBI_VEC_FLOPS + work_step[4] * 8
        f32_step = fix32 + work_step[2] * JACOBI_BLOCK_FLOPS + work_step[3] * JACOBI_VEC_FLOPS
    if fused:
        launch_ms = sum(prof["bond_updates"]) / max(len(prof["bond_updates"]), 1)
        bonds_per_launch = bonds_step
        launches_step = 1
        f32_big = big_end_flops(graphs, w.D)          # Gram and update passes inside the launch
        kernel = ("step_kernel (fused step: Gram pass, 2D x 2D bond eigenproblem with FP64 Jacobi and update "
                  f"of every bond of a Trotter step, one launch, {({5: 3, 6: 4}).get(sched, 2)} CTAs per SM where they fit)")
    else:
        launch_ms = sum(prof["bond"]) / max(len(prof["bond"]), 1)
        bonds_per_launch = bonds_step / g.n_colours
        launches_step = g.n_colours
        f32_big = 0.0
        kernel = "bond_kernel (2D x 2D bond eigenproblem, FP64 Jacobi)"
    flops_launch = f64_step / launches_step
    achieved = flops_launch / (launch_ms * 1e-3) / 1e9
    roofline = {"kernel": kernel, "bound": "alu",
                "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (FP64)",
                "frac": achieved / FP64_PEAK_GFLOPS,
                "traffic": NCU_TRAFFIC.get((w.name, args.dtype, sched, tensor)),
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clock x 2 flops x 2.07 GHz (MEASURED_PEAKS.json has "
                               "no FP64 figure; an FP64 FMA loop measured 1197 GFLOP/s)",
                "fp64_sweeps_per_bond": sweeps_per_bond, "fp32_sweeps_per_bond": sweeps32_per_bond,
                "fp32_gflops": (f32_step / launches_step + f32_big) / (launch_ms * 1e-3) / 1e9,
                "fp64_flops_per_launch": flops_launch,
                "jacobi_work_per_step": dict(zip(("fp64_blocks", "fp64_vector_pairs", "fp32_blocks",
                                                  "fp32_vector_pairs", "fp64_level_macs"), work_step)),
                "launch_ms": launch_ms, "units_per_launch": bonds_per_launch, "schedule": sched,
                "cycles_per_bond_by_phase": phase_cycles, "per_step_ms": layer_ms,
                "tensor_pipe": tensor_pipe_record(graphs, w.D, launch_ms if fused else
                                                  layer_ms.get("gram", 0.0) + layer_ms.get("update", 0.0), tensor)}
    elt = 8 if args.dtype == "mixed" else 16
    sb = step_bytes(graphs, w.D, elt)
    hbm = {"algorithmic_bytes_per_step": sb, "achieved_gbs_whole_step": sb / (ms / K * 1e-3) / 1e9}

    # end to end through the public API with host buffers
    th_host = torch.tensor(theta, dtype=torch.float64).pin_memory()
    res_host = torch.empty(g.n_instances, dtype=torch.float64).pin_memory()
    th_dev = torch.empty_like(th_host, device=dev)
    res_dev = torch.empty((1, g.n_instances), dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    Ke = max(min(K, 10), 1)
    t0 = time.perf_counter()
    for _ in range(Ke):
        th_dev.copy_(th_host, non_blocking=True)
        g.step(1, th_dev, out=res_dev)
        res_host.copy_(res_dev[0], non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * bonds_step * Ke / e2e_s, "unit": "bond updates/s",
           "h2d_bytes_per_step": th_host.numel() * 8, "d2h_bytes_per_step": res_host.numel() * 8}
    parity = parity_record(g, w, th, out.cpu().numpy(), W, K)
    g.close()

    plain = None
    if not args.no_plain and args.dtype == "mixed":
        Kp, Wp = max(min(K, 10), 1), W
        gp, thp, outp, msp, _, flp, tunp = timed("c128", Kp, Wp, not args.no_autotune)
        plain = {"dtype": "c128", "value": world * bonds_step * Kp / (msp * 1e-3), "unit": "bond updates/s",
                 "ms_per_step": msp / Kp, "steps": Kp, "warmup": Wp, "flags": flp,
                 "schedule": (tunp or {}).get("chosen"),
                 "parity": parity_record(gp, w, thp, outp.cpu().numpy(), Wp, Kp)}
        gp.close()
    # kernels of ours per timed step: kick, the bond updates (one fused launch, or Gram + bond +
    # update per colour class), readout, mean
    launches_per_step = 1 + (1 if fused else 3 * g.n_colours) + 2
    return dict(value=value, ms=ms, bonds_step=bonds_step, clocks=clocks, flags=flags, roofline=roofline,
                launches_per_step=launches_per_step,
                e2e=e2e, plain=plain, hbm=hbm, mean_last=mean_last, w=w, tuning=tuning, parity=parity)


def measured_hbm_gbs():
    """The measured copy bandwidth of this GPU model (MEASURED_PEAKS.json at the repository root),
    else an earlier measurement on a GB300, 6.8 TB/s."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        v = json.load(open(path)).get("hbm_gbs")
        if v:
            return float(v), "measured"
    return 6800.0, "fallback"


def run_condor_d64(dev, Kc=3, Wc=6):
    """The large configuration: 1121 qubits, D = 64, theta_h = 0.8 (workload condor_d64), in both
    precisions on the fused step (schedule 4; mixed with FP64 floor 3e-8, its tuned setting at
    D = 64).  Each: Wc warm-up steps from |0...0> (bonds saturate at step 6), Kc timed steps (CUDA
    events on the library stream), then one profiled step for the step kernel's time and the FP64
    work it executed.  Reports bond updates/s, Trotter steps/s, algorithmic HBM GB/s against the
    measured copy bandwidth, the step kernel's FP64 rate against the derived FP64 peak, the tensor
    pipe (the mixed path with its Gram and update passes on the tensor cores, beside the same path
    on CUDA cores), and the largest per-qubit differences between the paths after the timed steps.  The complex128 path is held to the oracle at
    1e-10 per qubit at D = 64 on the 127-qubit lattice; the oracle itself needs minutes per step
    of this lattice, so there are no committed oracle values for it."""
    import numpy as np
    import torch
    from paper_2309_15642_gb300 import GPEPS
    from workloads import kick_angles, workload
    wc = workload("condor_d64")
    graphs = wc.graphs()
    th = torch.tensor([float(t[0]) for t in kick_angles(wc)], dtype=torch.float64, device=dev)
    hbm_peak, hbm_src = measured_hbm_gbs()
    out, zs = {"workload": wc.name, "lattice_qubits": [n for n, _ in graphs], "D": wc.D,
               "theta": list(wc.theta)}, {}
    for key, dtype, tensor in (("mixed", "mixed", True), ("mixed_cuda_cores", "mixed", False), ("c128", "c128", False)):
        g = GPEPS(graphs, wc.D, dtype=dtype, device=str(dev))
        g.set_tensor_cores(tensor)
        g.set_schedule(4)
        if dtype == "mixed":
            g.set_jacobi(floor_rel=3e-8)
        g.reset()
        g.step(Wc, th)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(g.stream)
        g.step(Kc, th)
        e1.record(g.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        z, _ = g.expect_z()
        zs[key] = z.cpu().numpy()
        w0 = g.jacobi_work()
        kernel_ms = g.step_profiled(th)[1]
        work = [b - a for a, b in zip(w0, g.jacobi_work())]
        fix64, _ = bond_fixed_flops(graphs, wc.D, dtype)
        f64 = fix64 + work[4] * 8 + (one_sided_flops(wc.D, work[0], work[1]) if dtype == "c128"
                                     else work[0] * JACOBI_BLOCK_FLOPS + work[1] * JACOBI_VEC_FLOPS)
        sb = step_bytes(graphs, wc.D, 8 if dtype == "mixed" else 16)
        gbs = sb / (ms / Kc * 1e-3) / 1e9
        gf = f64 / (kernel_ms * 1e-3) / 1e9
        out[key] = {"value": g.bonds_per_step * Kc / (ms * 1e-3), "unit": "bond updates/s",
                      "trotter_steps_per_s": Kc / (ms * 1e-3), "ms_per_step": ms / Kc,
                      "timed_steps": f"{Wc + 1}..{Wc + Kc}",
                      "hbm": {"algorithmic_bytes_per_step": sb, "achieved_gbs": gbs, "peak_gbs": hbm_peak,
                              "frac": gbs / hbm_peak, "peak_source": hbm_src},
                      "fp64": {"kernel": "step_kernel", "kernel_ms": kernel_ms, "flops_per_launch": f64,
                               "achieved_gflops": gf, "peak_gflops": FP64_PEAK_GFLOPS,
                               "frac": gf / FP64_PEAK_GFLOPS},
                      "tensor_pipe": tensor_pipe_record(graphs, wc.D, kernel_ms, tensor),
                      "flags": g.status()}
        g.close()
    out["max_abs_dz_per_qubit_mixed_vs_c128"] = float(np.abs(zs["mixed"] - zs["c128"]).max())
    out["max_abs_dz_per_qubit_tensor_vs_cuda_cores"] = float(np.abs(zs["mixed"] - zs["mixed_cuda_cores"]).max())
    return out


def run_bp_record(dev, W=5, K=3, tensor=True):
    """BP regauging after each Trotter step (the paper's BP comparison) on workload eagle_bp_d32
    (127 q, D = 32, theta_h = 0.7), mixed path, fused step (three CTAs per SM where they fit, FP64
    floor 1e-7 as in the headline's tuned setting), the simple update's passes and the
    message products on the tensor cores (tensor=True) or on CUDA cores: W steps each followed by
    a regauge to convergence, then K timed steps (CUDA events on the library stream around step +
    regauge, the regauge's per-iteration convergence read-back included).  Reports Trotter
    steps/s with BP, BP iterations and per-phase device times, the message kernel's algorithmic
    FP32 work rate against the derived FP32 peak, and every qubit after the last step against the
    committed FP64 oracle values (BP included)."""
    import numpy as np
    import torch
    from paper_2309_15642_gb300 import GPEPS
    from workloads import kick_angles, workload
    wb = workload("eagle_bp_d32")
    graphs = wb.graphs()
    th = torch.tensor([float(t[0]) for t in kick_angles(wb)], dtype=torch.float64, device=dev)
    g = GPEPS(graphs, wb.D, dtype="mixed", device=str(dev))
    g.set_tensor_cores(tensor)
    from paper_2309_15642_gb300._abi import GpepsError
    try:
        g.set_schedule(5)      # the fused step with three CTAs per SM, as timed in the headline
    except GpepsError:
        g.set_schedule(4)
    g.set_jacobi(floor_rel=1e-7)
    g.reset()
    for _ in range(W):
        g.step(1, th)
        g.bp_regauge(200)
    torch.cuda.synchronize(dev)
    iters, phases = [], [0.0, 0.0, 0.0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    for _ in range(K):
        g.step(1, th)
        it, _, ms3 = g.bp_regauge(200, profile=True)
        iters.append(it)
        phases = [x + y for x, y in zip(phases, ms3)]
    e1.record(g.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    z, _ = g.expect_z()
    gold = golden_z(load_golden(wb), W + K)
    dz = None if gold is None else float(np.abs(z.cpu().numpy() - gold).max())
    flops = bp_message_flops(graphs, wb.D)
    msg_ms = phases[0] / max(sum(iters), 1)
    gf = flops / (msg_ms * 1e-3) / 1e9
    out = {"workload": wb.name, "dtype": "c64+f64", "tensor_cores": tensor,
           "value": K / (ms * 1e-3), "unit": "Trotter steps/s with BP",
           "ms_per_step": ms / K, "timed_steps": f"{W + 1}..{W + K}", "bp_iterations": iters,
           "ms_per_step_by_phase": {"messages": phases[0] / K, "gauge": phases[1] / K, "apply": phases[2] / K},
           "message_kernel": {"launch_ms": msg_ms, "flops_per_launch": flops, "achieved_gflops": gf,
                              "peak_gflops": FP32_PEAK_GFLOPS, "frac": gf / FP32_PEAK_GFLOPS, "bound": "alu (FP32)"},
           "max_abs_dz_per_qubit": dz, "parity_step": W + K, "flags": g.status()}
    g.close()
    return out


def run_large_chi_record(dev, W=7, K=2):
    """The large-chi path (the paper's long-time runs, Figs. 5-7, at chi = 128): workload
    eagle_d128, 127 q, D = 128 (256 x 256 bond cores, degree-3 ends of 16384 rows), theta_h = 1.0,
    complex128, layered launches (faster than the fused step at this size, where one CTA would
    hold a whole Gram pass).  W warm-up steps from |0...0> (the first truncation falls in step
    8), K timed steps (CUDA events on the library stream).  Reports bond updates/s, Trotter
    steps/s and the FP64 rate of the whole step by the counted work (Gram and update products,
    the bond SVDs' dense phases and the Jacobi work executed)."""
    import torch
    from paper_2309_15642_gb300 import GPEPS
    from workloads import kick_angles, workload
    wl = workload("eagle_d128")
    graphs = wl.graphs()
    th = torch.tensor([float(t[0]) for t in kick_angles(wl)], dtype=torch.float64, device=dev)
    g = GPEPS(graphs, wl.D, dtype="c128", device=str(dev))
    g.reset()
    g.step(W, th)
    torch.cuda.synchronize(dev)
    w0 = g.jacobi_work()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    g.step(K, th)
    e1.record(g.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    work = [b - a for a, b in zip(w0, g.jacobi_work())]
    fix64, _ = bond_fixed_flops(graphs, wl.D, "c128")
    f64 = K * (fix64 + big_end_flops(graphs, wl.D)) + one_sided_flops(wl.D, work[0], work[1]) + work[4] * 8
    gf = f64 / (ms * 1e-3) / 1e9
    out = {"workload": wl.name, "dtype": "c128", "D": wl.D, "value": g.bonds_per_step * K / (ms * 1e-3),
           "unit": "bond updates/s", "trotter_steps_per_s": K / (ms * 1e-3), "ms_per_step": ms / K,
           "timed_steps": f"{W + 1}..{W + K}", "schedule": 0,
           "fp64": {"whole_step_gflops": gf, "peak_gflops": FP64_PEAK_GFLOPS, "frac": gf / FP64_PEAK_GFLOPS,
                    "flops_per_step": f64 / K},
           "flags": g.status()}
    g.close()
    return out


def main():
    args = parse()
    args.profile_steps = max(args.profile_steps, 1)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    from workloads import workload
    w = workload(args.workload)

    if args.cpu_leg:
        print(json.dumps(cpu_oracle_leg(w, args.warmup, 10.0)))
        return

    if args.impl == "reference":
        if rank != 0:
            return
        K, W = args.steps, args.warmup
        # each step: one Trotter step of the oracle on the 127-qubit lattice of the batch
        from oracle.su import GPEPS as OraclePEPS
        from workloads import kick_angles
        (n, edges) = w.graphs()[0]
        th = kick_angles(w)[0]
        peps = OraclePEPS(n, edges, w.D)
        for _ in range(W):
            peps.step(th)
            peps.expect_z()
        t0 = time.perf_counter()
        for _ in range(K):
            peps.step(th)
            peps.expect_z()
        dt = time.perf_counter() - t0
        v = len(edges) * K / dt
        sample = (f"{n}-qubit lattice of the batch, D={w.D}, one Trotter step per step, steps {W + 1}..{W + K} "
                  f"after {W} untimed warm-up steps from |0...0> (numpy/LAPACK FP64, default BLAS threads)")
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": "bond updates/s", "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": dt / max(K, 1) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "lattices": [list(l) for l in w.lattices], "D": w.D,
                       "theta": list(w.theta), "sample": sample},
            "cpu_baseline": {"value": v, "unit": "bond updates/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "bond updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    if args.bp:
        if rank != 0:
            return
        r = run_bp(args, local_rank)
        cpu = None if args.no_cpu else cpu_oracle_bp(r["w"])
        K = args.steps
        it_mean = sum(r["iters"]) / max(len(r["iters"]), 1)
        msg_rate = r["n_msg"] * sum(r["iters"]) / max(r["phases_ms"][0] * K * 1e-3, 1e-12)
        print(json.dumps({
            "metric": "Trotter steps/s with a BP regauge after each step (the paper's BP comparison)",
            "value": r["value"], "unit": "Trotter steps/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
            "ms_per_step": r["ms"] / max(K, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+f64" if args.dtype == "mixed" else "c128", "data": "synthetic",
            "config": {"workload": r["w"].name, "lattices": [list(l) for l in r["w"].lattices], "D": r["w"].D,
                       "theta": list(r["w"].theta), "messages_per_iteration": r["n_msg"],
                       "timed_steps": f"{args.warmup + 1}..{args.warmup + K} from |0...0>",
                       "l2": "state larger than L2 (no flush)"},
            "bp": {"iterations_per_step": r["iters"], "mean_iterations": it_mean,
                   "ms_per_step": {"trotter_step": r["su_ms"], "messages": r["phases_ms"][0],
                                   "gauge": r["phases_ms"][1], "apply": r["phases_ms"][2]},
                   "message_updates_per_s": msg_rate},
            "roofline": r["roofline"], "clocks": r["clocks"], "cpu_baseline": cpu,
            "e2e": r["e2e"],
            # per step: the fused Trotter step (kick, step kernel, readout, mean), the regauge
            # (identity messages, one message launch per iteration, gauge, apply), expect_z (2)
            "gpu_launches": sum(r["iters"]) + 9 * K, "device_flags": r["flags"],
            "tuning": r["tuning"], "mean_z_last_step": r["means"][-1] if r["means"] else None}))
        return

    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    r = run_gpeps(args, rank, world, local_rank)
    condor = bp_rec = large = None
    if rank == 0 and world == 1 and not args.no_condor and args.workload == "heavyhex_mix_d32":
        import torch
        dev = torch.device("cuda", local_rank)
        condor = run_condor_d64(dev)
        bp_rec = run_bp_record(dev)
        cc = run_bp_record(dev, tensor=False)
        bp_rec["cuda_cores"] = {k: cc[k] for k in ("value", "ms_per_step", "ms_per_step_by_phase", "message_kernel",
                                                   "max_abs_dz_per_qubit")}
        large = run_large_chi_record(dev)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle(w, args.warmup)
    if rank == 0:
        line = {
            "metric": METRIC, "value": r["value"], "unit": "bond updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64+f64" if args.dtype == "mixed" else "c128", "data": "synthetic",
            "config": {"workload": w.name, "lattices": [list(l) for l in w.lattices], "D": w.D,
                       "theta": list(w.theta), "bonds_per_step": r["bonds_step"],
                       "trotter_steps_per_s": world * 1e3 * args.steps / r["ms"] / world,
                       "l2": "state larger than L2 (no flush)", "parallelism": f"replicas x{world}",
                       "timed_steps": f"{args.warmup + 1}..{args.warmup + args.steps} from |0...0>"},
            "roofline": r["roofline"], "hbm": r["hbm"], "clocks": r["clocks"], "e2e": r["e2e"],
            "plain_c128": r["plain"], "condor_d64": condor, "bp_regauge": bp_rec, "large_chi_d128": large,
            "cpu_baseline": cpu, "parity": r["parity"],
            "tuning": (r["tuning"] or {}).get("chosen"),
            "gpu_launches": r["launches_per_step"] * args.steps, "device_flags": r["flags"],
            "mean_z_last_step": r["mean_last"],
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
