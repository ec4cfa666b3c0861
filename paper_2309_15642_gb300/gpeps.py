"""Thin Python binding of the C ABI: the same calls, with torch for device memory and streams.

Every step of the evolution runs in ``libgpeps.so``; this module only packs
arguments, allocates the two caller-owned device buffers as torch tensors and
orders the library's stream against torch's current stream.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _abi
from ._abi import GPEPS_C128, GPEPS_MIXED_C64, GraphC, check

DTYPES = {"c128": GPEPS_C128, "mixed": GPEPS_MIXED_C64}


class GPEPS:
    """A batch of graph PEPS, one per graph in ``graphs`` (list of ``(n_qubits, edges)``).

    ``dtype``: ``"c128"`` (FP64 everywhere) or ``"mixed"`` (complex64 tensors,
    FP32 Gram/contract products, FP64 bond eigensolver and lambda).
    ``colours``: optional list (one int8 array per graph) of edge colour classes.
    """

    def __init__(self, graphs, D, dtype="mixed", device="cuda:0", colours=None):
        if not torch.cuda.is_available():
            raise RuntimeError("GPEPS needs a CUDA device; there is no CPU path")
        self.lib = _abi.load()
        self.device = torch.device(device)
        self.D = int(D)
        self.dtype = dtype
        self.n_instances = len(graphs)
        self._keep = []
        arr = (GraphC * self.n_instances)()
        for k, (n, edges) in enumerate(graphs):
            e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
            self._keep.append(e)
            arr[k].n_qubits = int(n)
            arr[k].n_edges = int(e.shape[0])
            arr[k].edges = e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            if colours is not None and colours[k] is not None:
                c = np.ascontiguousarray(np.asarray(colours[k], dtype=np.int8))
                self._keep.append(c)
                arr[k].colour = c.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
            else:
                arr[k].colour = None
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.Stream(self.device)
        h = ctypes.c_void_p()
        check(self.lib.gpeps_create(ctypes.cast(arr, ctypes.c_void_p), self.n_instances, self.D,
                                    DTYPES[dtype], ctypes.c_void_p(self.stream.cuda_stream),
                                    ctypes.byref(h)), "gpeps_create")
        self.h = h
        sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        check(self.lib.gpeps_query_workspace(self.h, ctypes.byref(sb), ctypes.byref(wb)), "gpeps_query_workspace")
        self.state_bytes, self.work_bytes = sb.value, wb.value
        self.state = torch.zeros(self.state_bytes, dtype=torch.uint8, device=self.device)  # padding defined
        self.work = torch.empty(self.work_bytes, dtype=torch.uint8, device=self.device)
        check(self.lib.gpeps_bind(self.h, ctypes.c_void_p(self.state.data_ptr()),
                                  ctypes.c_void_p(self.work.data_ptr())), "gpeps_bind")
        q, e = ctypes.c_int64(), ctypes.c_int64()
        check(self.lib.gpeps_sizes(self.h, ctypes.byref(q), ctypes.byref(e)), "gpeps_sizes")
        self.total_qubits, self.total_edges = q.value, e.value
        nc = ctypes.c_int32()
        check(self.lib.gpeps_n_colours(self.h, ctypes.byref(nc)), "gpeps_n_colours")
        self.n_colours = nc.value
        self.bonds_per_step = self.total_edges
        self._bp_work, self._bp_iter = None, 0

    # -------------------------------------------------------------- stream order
    def _after_torch(self):
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def _before_torch(self):
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _theta(self, theta, per_qubit):
        t = torch.as_tensor(theta, dtype=torch.float64)
        if t.device != self.device:
            t = t.to(self.device)
        t = t.contiguous()
        n = self.total_qubits if per_qubit else self.n_instances
        if t.numel() != n:
            raise ValueError(f"theta must have {n} entries (per_qubit={per_qubit})")
        return t

    # -------------------------------------------------------------- the C calls
    def reset(self):
        self._after_torch()
        check(self.lib.gpeps_reset(self.h), "gpeps_reset")

    def kick(self, theta, per_qubit=False):
        t = self._theta(theta, per_qubit)
        self._after_torch()
        check(self.lib.gpeps_kick(self.h, ctypes.c_void_p(t.data_ptr()), int(bool(per_qubit))), "gpeps_kick")
        t.record_stream(self.stream)

    def zz_layer(self, colour):
        check(self.lib.gpeps_zz_layer(self.h, int(colour)), "gpeps_zz_layer")

    def zz_layer_profiled(self, colour):
        """Run colour class ``colour`` with events around its three launches; returns ms[3]
        (Gram partials, bond eigenproblems, larger-end update)."""
        ms = (ctypes.c_float * 3)()
        check(self.lib.gpeps_zz_layer_profiled(self.h, int(colour), ms), "gpeps_zz_layer_profiled")
        return [float(x) for x in ms]

    def step_profiled(self, theta, per_qubit=False):
        """One Trotter step under the current schedule, launched directly with events around its
        parts; returns ms[3] (kick, bond updates of every colour class, readout and mean)."""
        t = self._theta(theta, per_qubit)
        self._after_torch()
        ms = (ctypes.c_float * 3)()
        check(self.lib.gpeps_step_profiled(self.h, ctypes.c_void_p(t.data_ptr()), int(bool(per_qubit)), ms),
              "gpeps_step_profiled")
        return [float(x) for x in ms]

    def expect_z(self):
        """Return ``(z[total_qubits], mean[n_instances])`` as float64 CUDA tensors."""
        z = torch.empty(self.total_qubits, dtype=torch.float64, device=self.device)
        m = torch.empty(self.n_instances, dtype=torch.float64, device=self.device)
        self._after_torch()
        check(self.lib.gpeps_expect_z(self.h, ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(m.data_ptr())),
              "gpeps_expect_z")
        self._before_torch()
        return z, m

    def step(self, n_steps, theta, per_qubit=False, out=None):
        """Run ``n_steps`` Trotter steps; returns the mean <Z> per step and instance."""
        t = self._theta(theta, per_qubit)
        if out is None:
            out = torch.empty((n_steps, self.n_instances), dtype=torch.float64, device=self.device)
        self._after_torch()
        check(self.lib.gpeps_step(self.h, int(n_steps), ctypes.c_void_p(t.data_ptr()), int(bool(per_qubit)),
                                  ctypes.c_void_p(out.data_ptr())), "gpeps_step")
        self._before_torch()
        self._last_theta = t  # the captured graph reads this buffer
        return out

    def inverse_steps(self, n_steps, theta, per_qubit=False):
        """Apply U^dagger(theta)^n_steps (App. B: colour classes in reverse order with the conjugate
        gate, then the kick by -theta); see gpeps_inverse_steps."""
        t = self._theta(theta, per_qubit)
        self._after_torch()
        check(self.lib.gpeps_inverse_steps(self.h, int(n_steps), ctypes.c_void_p(t.data_ptr()),
                                           int(bool(per_qubit))), "gpeps_inverse_steps")
        t.record_stream(self.stream)

    def weight_z(self, theta_h, n_steps, per_qubit=False):
        """Weight-N observables by Clifford back-evolution (App. B): from |0...0>, n_steps Trotter
        steps at theta_h, then n_steps inverse steps at pi/2; returns <Z_i> of that state for every
        qubit (float64 tensor), i.e. <U^n(pi/2) Z_i U^dagger(pi/2)^n> in |psi(theta_h, n)>.  Qubit
        P = 13 of the 127-qubit lattice gives the Weight-10 operator of App. B."""
        self.reset()
        self.step(n_steps, theta_h, per_qubit=per_qubit)
        half_pi = torch.full_like(self._theta(theta_h, per_qubit), math.pi / 2)
        self.inverse_steps(n_steps, half_pi, per_qubit=per_qubit)
        z, _ = self.expect_z()
        return z

    def status(self):
        f = ctypes.c_int32()
        check(self.lib.gpeps_status(self.h, ctypes.byref(f)), "gpeps_status")
        return f.value

    def lambdas(self, instance, edge):
        out = (ctypes.c_double * self.D)()
        check(self.lib.gpeps_lambda(self.h, int(instance), int(edge), out), "gpeps_lambda")
        return np.array(out[:], dtype=np.float64)

    def sweeps(self):
        """(FP64 Jacobi sweeps, FP32 warm-start sweeps, bond updates) since the last reset."""
        s, s32, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(self.lib.gpeps_sweeps(self.h, ctypes.byref(s), ctypes.byref(s32), ctypes.byref(b)), "gpeps_sweeps")
        return s.value, s32.value, b.value

    def bond_phase_cycles(self):
        """SM cycles per phase of the bond kernel since the last reset (summed over bonds)."""
        return self.bond_counters()[:6]

    def jacobi_work(self):
        """(FP64 block updates, FP64 eigenvector pair updates, FP32 block updates, FP32 pair
        updates, FP64 complex MACs of the extra FP32 levels) executed since the last reset (see
        gpeps_jacobi_work)."""
        w = (ctypes.c_int64 * 5)()
        check(self.lib.gpeps_jacobi_work(self.h, w), "gpeps_jacobi_work")
        return [int(x) for x in w]

    def pass_cycles(self):
        """SM cycles of the fused step's Gram and update passes of the larger ends since the last
        reset (summed over bonds; zero for the layered launches)."""
        return self.bond_counters()[22:24]

    def bond_counters(self):
        """All counters of the bond kernel: 6 phase cycle sums, rotations per FP32 sweep (8),
        rotations per FP64 sweep (8), cycles of the fused step's Gram and update passes (2)."""
        c = (ctypes.c_int64 * 24)()
        check(self.lib.gpeps_bond_phase_cycles(self.h, c), "gpeps_bond_phase_cycles")
        return [int(x) for x in c]

    def set_schedule(self, schedule):
        """Bond eigenproblems: 0 one CTA per bond; 1, 2, 3 work queue with one, two or four CTAs
        per SM; 4 one fused persistent launch per Trotter step in :meth:`step`, 5 and 6 the same
        with three or four CTAs per SM (see gpeps_set_schedule)."""
        check(self.lib.gpeps_set_schedule(self.h, int(schedule)), "gpeps_set_schedule")

    def set_tensor_cores(self, on: bool = True) -> None:
        """Gram and update products of the larger ends on the tensor cores
        (mixed path, D = 32 or 64; see gpeps_set_tensor_cores)."""
        check(self.lib.gpeps_set_tensor_cores(self.h, 1 if on else 0), "gpeps_set_tensor_cores")

    def set_jacobi(self, tol=None, floor_rel=None, tol32=1e-6, floor32=2e-7, max_sweeps=40, max_sweeps32=20):
        """Thresholds of the bond eigensolver (see gpeps_set_jacobi); None = the dtype's default."""
        if tol is None:
            tol = 1e-14 if self.dtype == "c128" else 1e-9
        if floor_rel is None:
            floor_rel = 1e-20 if self.dtype == "c128" else 1e-8
        check(self.lib.gpeps_set_jacobi(self.h, float(tol), float(floor_rel), float(tol32), float(floor32),
                                        int(max_sweeps), int(max_sweeps32)), "gpeps_set_jacobi")

    def set_wait_limit(self, cycles=4000000000):
        """Wait limit of the fused step in SM cycles (see gpeps_set_wait_limit)."""
        check(self.lib.gpeps_set_wait_limit(self.h, int(cycles)), "gpeps_set_wait_limit")

    def set_levels(self, level_ratio=1e-5, levels=4):
        """Extra FP32 levels of the bond eigensolver (see gpeps_set_levels)."""
        check(self.lib.gpeps_set_levels(self.h, float(level_ratio), int(levels)), "gpeps_set_levels")

    # -------------------------------------------------------------- gradient
    def grad(self, theta, n_steps, ckpt_every=5, dL_dz=None):
        """Gradient path (complex128, D <= 16): returns ``(z, dtheta)`` with z = <Z_i> after
        ``n_steps`` steps from |0...0> with per-qubit kick angles ``theta`` and, when the weights
        ``dL_dz`` are given, dtheta = d(sum_i dL_dz_i <Z_i>)/dtheta (else None)."""
        t = self._theta(theta, per_qubit=True)
        nbytes = ctypes.c_size_t()
        check(self.lib.gpeps_query_grad_workspace(self.h, int(n_steps), int(ckpt_every), ctypes.byref(nbytes)),
              "gpeps_query_grad_workspace")
        work = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=self.device)
        z = torch.empty(self.total_qubits, dtype=torch.float64, device=self.device)
        w = dth = None
        if dL_dz is not None:
            w = torch.as_tensor(dL_dz, dtype=torch.float64).to(self.device).contiguous()
            dth = torch.empty(self.total_qubits, dtype=torch.float64, device=self.device)
        self._after_torch()
        check(self.lib.gpeps_grad(self.h, ctypes.c_void_p(t.data_ptr()), int(n_steps), int(ckpt_every),
                                  ctypes.c_void_p(w.data_ptr()) if w is not None else None,
                                  ctypes.c_void_p(z.data_ptr()),
                                  ctypes.c_void_p(dth.data_ptr()) if dth is not None else None,
                                  ctypes.c_void_p(work.data_ptr()), nbytes.value), "gpeps_grad")
        self._before_torch()
        self.stream.synchronize()
        return z, dth

    def bp_regauge(self, max_iter=100, tol=None, profile=False):
        """Belief-propagation regauging of the state (see ``gpeps_bp_regauge``).  ``tol``
        defaults to 1e-12 (complex128) or 1e-6 (mixed: FP32 message contractions).  Returns
        ``(iterations, residual)``, and with ``profile`` also the device milliseconds of the
        message launches, the gauge and the apply."""
        if tol is None:
            tol = 1e-12 if self.dtype == "c128" else 1e-6
        if self._bp_work is None or self._bp_iter < max_iter:
            nbytes = ctypes.c_size_t()
            check(self.lib.gpeps_query_bp_workspace(self.h, int(max_iter), ctypes.byref(nbytes)),
                  "gpeps_query_bp_workspace")
            self._bp_work = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=self.device)
            self._bp_iter = int(max_iter)
        it = ctypes.c_int32()
        res = ctypes.c_double()
        ms = (ctypes.c_float * 3)()
        self._after_torch()
        check(self.lib.gpeps_bp_regauge(self.h, int(max_iter), float(tol), ctypes.c_void_p(self._bp_work.data_ptr()),
                                        self._bp_work.numel(), ctypes.byref(it), ctypes.byref(res),
                                        ctypes.cast(ms, ctypes.c_void_p) if profile else None),
              "gpeps_bp_regauge")
        self._before_torch()
        if profile:
            return it.value, res.value, tuple(float(x) for x in ms)
        return it.value, res.value

    # -------------------------------------------------------------- state access
    def site_tensor(self, instance, site):
        """View of Gamma of a site inside the state buffer: complex tensor [2] + [D] * deg, and
        the site's neighbours in leg order."""
        off, deg = ctypes.c_int64(), ctypes.c_int32()
        nb = (ctypes.c_int32 * 3)()
        check(self.lib.gpeps_site_layout(self.h, int(instance), int(site), ctypes.byref(off), ctypes.byref(deg),
                                         nb), "gpeps_site_layout")
        cdt = torch.complex128 if self.dtype == "c128" else torch.complex64
        esz = 16 if self.dtype == "c128" else 8
        n = 2 * self.D ** deg.value
        t = self.state[off.value: off.value + n * esz].view(cdt).view([2] + [self.D] * deg.value)
        return t, [x for x in nb[:deg.value]]

    def lambda_tensor(self, instance, edge):
        """View of lambda (float64[D], unsorted) of an edge inside the state buffer."""
        off = ctypes.c_int64()
        check(self.lib.gpeps_lambda_layout(self.h, int(instance), int(edge), ctypes.byref(off)),
              "gpeps_lambda_layout")
        return self.state[off.value: off.value + self.D * 8].view(torch.float64)

    def save_state(self):
        """Host copy of the whole state (every Gamma and lambda): a checkpoint taken after a
        full Trotter step, when no kick is pending."""
        self.stream.synchronize()
        return self.state.cpu().clone()

    def load_state(self, saved):
        """Restore a checkpoint of :meth:`save_state` (same graphs, D and dtype)."""
        if saved.numel() != self.state.numel():
            raise ValueError("checkpoint of another layout")
        self._after_torch()
        with torch.cuda.stream(self.stream):
            self.state.copy_(saved.to(self.device, non_blocking=False))
        self.stream.synchronize()

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "h", None) is not None:
            self.stream.synchronize()
            self.lib.gpeps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KickedIsingZ(torch.autograd.Function):
    """<Z_i> after ``n_steps`` Trotter steps as a differentiable function of the per-qubit kick
    angles: ``z = KickedIsingZ.apply(theta, g, n_steps, ckpt_every)``; backward runs the
    library's reverse mode (checkpointed, recomputing each segment)."""

    @staticmethod
    def forward(ctx, theta, g, n_steps, ckpt_every=5):
        z, _ = g.grad(theta.detach(), n_steps, ckpt_every)
        ctx.save_for_backward(theta.detach())
        ctx.g, ctx.n_steps, ctx.ckpt_every = g, n_steps, ckpt_every
        return z

    @staticmethod
    def backward(ctx, grad_z):
        (theta,) = ctx.saved_tensors
        _, dth = ctx.g.grad(theta, ctx.n_steps, ctx.ckpt_every, dL_dz=grad_z.detach())
        return dth.to(theta.dtype), None, None, None
