/*
 * gpeps.h -- C ABI of the GB300 (sm_103a) simple-update Trotter evolution of
 * the kicked Ising circuit on heavy-hexagon graph PEPS.
 *
 * The method (paper, sections "Model" and "Method", Eqs. 1-3): a graph PEPS
 * with one tensor Gamma_i per qubit (physical dimension 2, one virtual leg of
 * dimension D per coupler) and one weight vector lambda_e per coupler is
 * evolved by U(theta_h) = (prod_edges exp(i pi/4 Z_i Z_j)) (prod_i exp(-i theta_h X_i / 2))
 * with the *simple update* of tensors, truncating every bond to D ("chi" in the
 * paper), and read out with a *mean-field* approximation of the environment.
 *
 * Conventions for every entry point
 *   - Every function returns an int status: GPEPS_OK (0) or a GPEPS_E* code.
 *     gpeps_error_string() names it.  No entry point aborts or traps.
 *   - All GPU work is enqueued asynchronously on the stream given to
 *     gpeps_create (NULL = legacy default stream) unless stated otherwise.
 *   - Device memory is owned by the caller: gpeps_query_workspace() reports the
 *     two sizes, the caller allocates them (e.g. torch tensors) and passes them
 *     to gpeps_bind().  The handle owns only host metadata and, after the first
 *     gpeps_step(), one instantiated CUDA graph.  The library never calls
 *     cudaMalloc.
 *   - "host" pointers are read (or written) before the call returns; "device"
 *     pointers must stay valid until the enqueued work has finished.
 *   - Errors found on the device (Jacobi sweep cap, NaN/Inf, vanishing norm)
 *     set bits in a device flag word; gpeps_status() synchronises the stream
 *     and returns them.  Device code never traps and every loop is bounded.
 *
 * Scope: graphs in which every edge has an end of degree <= 2 and every vertex
 * has degree <= 3 (true of the heavy-hex lattices of the paper, Fig. 1);
 * 1 <= D <= 64, and D <= 128 for GPEPS_C128 (gpeps_grad: D <= 16; BP regauging:
 * D <= 64; gpeps_bond_update_noalloc: D <= 32).
 */
#ifndef GPEPS_H
#define GPEPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GPEPS_OK 0
#define GPEPS_EINVAL 1   /* bad argument: graph, D, dtype, colour, pointer, call order */
#define GPEPS_ECUDA 2    /* a CUDA runtime call failed (the message is kept, see gpeps_last_cuda_error) */
#define GPEPS_ENOCONV 3  /* device flag: a Jacobi eigensolver hit its sweep cap (results still written) */
#define GPEPS_ENUMERIC 4 /* device flag: NaN/Inf or a vanishing bond spectrum */
#define GPEPS_ENOMEM 5   /* host allocation failed */

/* device flag bits returned by gpeps_status */
#define GPEPS_FLAG_NOCONV 1
#define GPEPS_FLAG_NUMERIC 2
#define GPEPS_FLAG_TIMEOUT 4  /* a wait of the fused step kernel gave up (schedule 4) */

/* storage / arithmetic of the evolution */
#define GPEPS_C128 0       /* complex128 tensors; every product and the eigensolver in FP64 */
#define GPEPS_MIXED_C64 1  /* complex64 tensors; Gram/contract products in FP32; bond
                              eigensolver, lambda renormalisation and lambda^-1 in FP64 */

/*
 * One coupling graph.  edges: host, int32[2*n_edges], pairs (a, b) with
 * 0 <= a, b < n_qubits, a != b, no duplicates.  colour: host, int8[n_edges]
 * giving the update class of every edge (each class must be a matching), or
 * NULL for the library's greedy first-fit colouring over edges sorted by
 * (smaller label, larger label).  The paper does not fix an update order; the
 * ZZ gates of Eq. 2 commute, so only truncated results depend on it.
 */
typedef struct {
  int32_t n_qubits;
  int32_t n_edges;
  const int32_t* edges;
  const int8_t* colour;
} gpeps_graph;

typedef struct gpeps_handle gpeps_handle;

/*
 * Create a batch of n_instances independent gPEPS, instance k living on
 * graphs[k] (the same graph may be passed for several instances, e.g. a sweep
 * of theta_h).  D: bond dimension (paper's chi, section "Method").  dtype:
 * GPEPS_C128 or GPEPS_MIXED_C64.  stream: a cudaStream_t or NULL.  The graph
 * arrays are copied; *out receives the handle (free with gpeps_destroy).
 * Errors: GPEPS_EINVAL for a malformed graph, a colouring that is not a
 * matching, a vertex of degree > 3, an edge joining two degree-3 vertices,
 * D outside [1, 64] (GPEPS_MIXED_C64) or [1, 128] (GPEPS_C128), or an unknown
 * dtype.
 */
int gpeps_create(const gpeps_graph* graphs, int32_t n_instances, int32_t D, int32_t dtype,
                 void* stream, gpeps_handle** out);

/*
 * Bytes of the two caller-owned device buffers.  state: every Gamma_i (complex,
 * physical index outermost, legs in sorted-neighbour order, last leg fastest)
 * and every lambda_e (float64[D]).  work: kick angles, bond work lists,
 * per-bond scratch (the complex128 bond SVD's matrices, 264 KB per bond of the
 * largest colour class at D = 32 and 4.2 MB at D = 128; in the mixed path for
 * D > 34 the 2D x 2D bond eigenproblems that do not fit in shared memory, 772 KB
 * at D = 64), Gram partials of the larger ends (2 D^2 complex per tile of 64
 * rows, 32 rows in complex128 beyond D = 64),
 * <Z> outputs and the flag word.  Both need 256-byte alignment (cudaMalloc and
 * torch give it).
 */
int gpeps_query_workspace(const gpeps_handle* h, size_t* state_bytes, size_t* work_bytes);

/* Attach the two device buffers (sizes from gpeps_query_workspace) and upload
 * the work lists; enqueues copies on the stream.  Re-binding invalidates a
 * captured step graph.  Errors: GPEPS_EINVAL for NULL or misaligned pointers,
 * or a current device with less than 227 KB of opt-in shared memory per block. */
int gpeps_bind(gpeps_handle* h, void* d_state, void* d_work);

/* Product state |0...0> of Eq. 3 on every instance: Gamma_i[0,0,...,0] = 1,
 * lambda_e = (1, 0, ..., 0), no pending kick; clears the flag word. */
int gpeps_reset(gpeps_handle* h);

/*
 * Kick: apply exp(-i theta X_i / 2) (Eq. 2, single-site factor) to every qubit
 * of every instance.  theta: device float64, [n_instances] when per_qubit == 0,
 * else [total qubits] in instance-then-label order.  The rotation is not
 * applied to the tensors here: it is accumulated per site and fused into the
 * next bond update that touches the site (and applied on the fly by
 * gpeps_expect_z while still pending).
 */
int gpeps_kick(gpeps_handle* h, const double* theta, int32_t per_qubit);

/*
 * Simple update (section "Method") with the gate exp(i pi/4 Z_i Z_j) of Eq. 2
 * on every edge of colour class `colour` of every instance; the edges of a
 * class are independent and run concurrently.  Per bond: absorb the lambda of
 * the other legs, reduce both site tensors, apply the gate, solve the 2D x 2D
 * bond eigenproblem, keep the D largest Schmidt values, renormalise lambda to
 * unit 2-norm and strip lambda^-1 (pseudo-inverse below 1e-13 max(lambda)).
 * Every Schmidt value with a positive squared value is kept (up to D).
 * Errors: GPEPS_EINVAL for colour outside [0, n_colours).
 */
int gpeps_zz_layer(gpeps_handle* h, int32_t colour);

/*
 * Same work as gpeps_zz_layer, with CUDA events recorded on the handle's
 * stream around its three launches; synchronises and writes the durations in
 * milliseconds to host ms[3]: [0] Gram partials of the larger ends, [1] bond
 * eigenproblems (one CTA per bond), [2] update of the larger ends.
 */
int gpeps_zz_layer_profiled(gpeps_handle* h, int32_t colour, float* ms);

/*
 * One Trotter step as gpeps_step runs it under the current schedule, launched
 * directly (no graph) with CUDA events around its parts: ms (host float[3])
 * receives [0] the kick, [1] the bond updates of every colour class (the fused
 * launch of schedule 4, or the Gram, bond and update launches of each class),
 * [2] the readout and mean.  Synchronises the stream.  Errors: GPEPS_EINVAL for
 * a NULL pointer or an unbound handle.
 */
int gpeps_step_profiled(gpeps_handle* h, const double* theta, int32_t per_qubit, float* ms);

/*
 * Thresholds of the bond eigensolver (defaults in parentheses).  Mixed path: its
 * FP64 sweeps on the squared bond matrix stop rotating a pair when |a_pq| <=
 * max(tol sqrt(a_pp a_qq), floor_rel * trace) (1e-9, 1e-8).  Complex128 path: its
 * FP64 one-sided sweeps on the bond core B stop rotating a column pair when
 * |b_p^H b_q| <= max(tol |b_p| |b_q|, floor_rel ||B||_F^2) (1e-14, 1e-20).  The
 * FP32 stages use tol32 (1e-6; complex128: relative to the two columns) and
 * floor32 (2e-7; mixed only); sweep caps
 * max_sweeps (40; hitting it sets GPEPS_FLAG_NOCONV) and max_sweeps32 (20).
 * Host-only; drops a captured step graph.  Errors: GPEPS_EINVAL for
 * non-positive thresholds or caps outside [1, 200] (FP64) / [0, 200] (FP32).
 */
int gpeps_set_jacobi(gpeps_handle* h, double tol, double floor_rel, double tol32, double floor32,
                     int32_t max_sweeps, int32_t max_sweeps32);

/*
 * Extra FP32 levels of the bond eigensolver: after the first FP32 solve and
 * the FP64 re-orthonormalisation, up to `levels` (4; at most 8) further FP32
 * solves, each on the rescaled block of the (at most 32) largest eigenvalues
 * that lie below level_ratio (1e-5) x the scale of the last block that held
 * them, so that small eigenvalues start the FP64 sweeps resolved to FP32
 * accuracy relative to their own size.  Host-only; drops a captured step
 * graph.  Errors: GPEPS_EINVAL for level_ratio outside (0, 1) or levels
 * outside [0, 8].
 */
int gpeps_set_levels(gpeps_handle* h, double level_ratio, int32_t levels);

/*
 * Wait limit of the fused step (schedule 4), in SM clock cycles (default
 * 4e9, about 2 s, where a bond update takes at most ~0.2 s (D <= 64); 6.4e10
 * beyond D = 64, where one takes about a second): a bond that waits longer for an earlier bond on one of its
 * sites gives up, raises GPEPS_FLAG_TIMEOUT and runs on what it finds, so a
 * launch always ends.  0 gives up at once whenever a dependency is still
 * running (failure-detection tests use it).  Host-only; drops a captured step
 * graph.  Errors: GPEPS_EINVAL for a negative value.
 */
int gpeps_set_wait_limit(gpeps_handle* h, int64_t cycles);

/*
 * Schedule of the bond eigenproblems: 0 launches one CTA per bond (default);
 * 1 launches one CTA per SM that takes bonds from a work queue in the work
 * buffer; 2 and 3 launch two (256 threads each) or four (128 threads) CTAs per
 * SM on the queue, each with its n x n FP64 matrices in a slot of the work
 * buffer (held in L2) and its FP32 level in shared memory, so that one bond's
 * latency-bound phases overlap another's FP64 work.  Every schedule runs the
 * bonds of a colour class largest first and gives bit-identical results.
 * 4 makes gpeps_step run every bond update of a Trotter step in one persistent
 * launch (two CTAs per SM where they fit, else one): the Gram pass of the
 * larger end, the bond eigenproblem and the update of the larger end run in the
 * CTA that takes the bond, bonds are taken colour class by colour class, and a
 * bond waits only until the earlier bonds on its two sites are done, so the
 * classes need no barrier between them (same results; a wait that gives up
 * after ~2 s raises GPEPS_FLAG_TIMEOUT instead of hanging); gpeps_zz_layer
 * then uses schedule 2 (or 1 where 2 does not fit).  5 is the fused step with
 * three 192-thread CTAs per SM (where their shared memory fits, D <= 32), 6
 * with four (GPEPS_MIXED_C64 where their shared memory fits, D <= 32; with the
 * tensor cores on, their TMEM, four times 4D columns, must fit the SM's 512).
 * Host-only; drops a captured step graph.  Errors: GPEPS_EINVAL for other
 * values, and for 2 to 6 on an unbound handle, when the FP32 level does not
 * fit the CTA's share of shared memory (D above 47 for 2, above 32 for 3, 5
 * and 6), for 6 with complex128, or on a device with more than 256 SMs.
 */
int gpeps_set_schedule(gpeps_handle* h, int32_t schedule);  /* 0..6 */

/*
 * Tensor cores for the two streaming products of every bond update in the
 * mixed path ("Method": the absorb/reduce/contract products of the simple
 * update, here as TF32 products with FP32 accumulation): the
 * Gram blocks G_s of the larger end and its update Gamma_a' = A~ Y_s run as
 * tcgen05.mma (kind::tf32) products with FP32 accumulators in tensor memory,
 * each FP32 operand split as hi + lo in TF32 (three products per pair, about
 * 2^-22 relative error, FP32-level), the Gram read out per 64-row tile and
 * summed in FP64 as the CUDA-core form does.  The bond eigenproblem, lambda
 * and lambda^-1 stay FP64.  on = 0 returns to the CUDA-core products (the
 * default).  Applies to the layered launches and to the fused step
 * (schedules 4 and 5), and at D = 32 also to the message products of
 * gpeps_bp_regauge (leg products and message Gram, 3xTF32).  Host-only; drops a captured step graph.  Errors:
 * GPEPS_EINVAL unless the handle is GPEPS_MIXED_C64 with D = 32 or 64, or if
 * the fused schedule in use would no longer fit its shared memory (or, under
 * schedule 6, four CTAs' TMEM).
 */
int gpeps_set_tensor_cores(gpeps_handle* h, int32_t on);

/* Number of colour classes (the largest over the instances). */
int gpeps_n_colours(const gpeps_handle* h, int32_t* n_colours);

/*
 * Mean-field <Z_i> (section "Method"; App. B): psi_i = Gamma_i with lambda on
 * every leg, p_s = sum |psi_i[s,...]|^2, <Z_i> = (p_0 - p_1)/(p_0 + p_1), pending
 * kicks applied on the fly.  d_z: device float64[total qubits] or NULL;
 * d_mean: device float64[n_instances] (mean over the instance's qubits) or NULL.
 */
int gpeps_expect_z(gpeps_handle* h, double* d_z, double* d_mean);

/*
 * n_steps inverse Trotter steps U^dagger(theta)^n (App. B): since
 * U(theta) = ZZ K(theta) (Eq. 2), one inverse step applies every colour class
 * with the conjugate gate exp(-i pi/4 Z Z), in the reverse order of a forward
 * step, and then the kick exp(+i theta X / 2) (pending, like gpeps_kick).
 * With theta = pi/2 after n forward steps this gives the state
 * |omega(theta_h, n)> = U^dagger(pi/2)^n |psi(theta_h, n)> whose single-site
 * <Z_P> (gpeps_expect_z) is the Weight-N observable <U^n(pi/2) Z_P
 * U^dagger(pi/2)^n> of App. B (e.g. P = 13 gives Weight 10 on the 127-qubit
 * lattice).  theta: device, as in gpeps_kick.  Launched directly on the stream
 * (no graph).  Errors: GPEPS_EINVAL for a NULL pointer, an unbound handle or
 * n_steps < 0.
 */
int gpeps_inverse_steps(gpeps_handle* h, int32_t n_steps, const double* theta, int32_t per_qubit);

/*
 * n_steps Trotter steps U(theta) of Eq. 2: kick with theta (device, as in
 * gpeps_kick), then every colour class in increasing order, then the mean
 * <Z> of every instance into d_mean_per_step[t * n_instances + k] (device
 * float64, or NULL).  One step is captured once as a CUDA graph and replayed.
 */
int gpeps_step(gpeps_handle* h, int32_t n_steps, const double* theta, int32_t per_qubit,
               double* d_mean_per_step);

/* Synchronise the stream and return the device flag word (GPEPS_FLAG_* bits)
 * in *flags; also returns GPEPS_ECUDA if a CUDA error is pending. */
int gpeps_status(gpeps_handle* h, int32_t* flags);

/* Copy lambda of edge `edge` (index into that instance's edge list) of
 * instance `instance` to host out[D], sorted in decreasing order; synchronises. */
int gpeps_lambda(gpeps_handle* h, int32_t instance, int32_t edge, double* out);

/*
 * Layout of the state buffer, for reading, checkpointing or writing tensors.
 * gpeps_site_layout: byte offset of Gamma of site `site` of instance
 * `instance` inside the state buffer, its degree, and its neighbours in leg
 * order (host int32[3], -1 past the degree).  Gamma is complex (16 bytes per
 * element for GPEPS_C128, 8 for GPEPS_MIXED_C64), laid out [s][leg0][leg1][leg2]
 * with the physical index s in {0, 1} outermost and the last leg fastest,
 * 2 * D^deg elements.  gpeps_lambda_layout: byte offset of lambda (float64[D])
 * of edge `edge`.  Host-only; the handle need not be bound.  Saving the state
 * buffer after a full Trotter step (no kick pending) and copying it back into
 * a bound handle of the same graphs, D and dtype restores the evolution.
 */
int gpeps_site_layout(const gpeps_handle* h, int32_t instance, int32_t site, int64_t* byte_offset, int32_t* deg,
                      int32_t* neighbours);
int gpeps_lambda_layout(const gpeps_handle* h, int32_t instance, int32_t edge, int64_t* byte_offset);

/*
 * Gradient of L = sum_i c_i <Z_i> after n_steps Trotter steps with respect to
 * per-qubit kick angles theta_i (the same angles at every step), by a
 * hand-written reverse mode of the simple update (no counterpart in the
 * paper).  complex128 handles with D <= 16 only.
 *
 * The forward applies the kicks exp(-i theta_i X_i / 2) explicitly, then the
 * colour classes; Schmidt values whose square is <= 1e-14 of the largest are
 * zero in both directions.  The reverse is first-order perturbation theory of
 * the bond eigenproblem over all its eigenvectors with Lorentzian broadening
 * 1/(e_k - e_j) -> (e_k - e_j) / ((e_k - e_j)^2 + (1e-12 e_max)^2), chained
 * through the Gram, update, lambda renormalisation and lambda^-1 steps, the
 * kicks and the mean-field readout.  Checkpoints: the state every ckpt_every
 * steps; each segment is recomputed with one state snapshot per colour class.
 *   theta:   device float64[total qubits] (instance-then-label order)
 *   dL_dz:   device float64[total qubits] (the weights c_i), or NULL for the
 *            forward alone
 *   z_out:   device float64[total qubits] or NULL: <Z_i> after n_steps
 *   dtheta:  device float64[total qubits] (required with dL_dz): dL/dtheta_i
 *   d_grad_work: device, 256-byte aligned, >= gpeps_query_grad_workspace bytes
 * The handle's state is left at a recomputed intermediate state.  Errors:
 * GPEPS_EINVAL (dtype, D, sizes, pointers).
 */
int gpeps_query_grad_workspace(const gpeps_handle* h, int32_t n_steps, int32_t ckpt_every, size_t* bytes);
int gpeps_grad(gpeps_handle* h, const double* theta, int32_t n_steps, int32_t ckpt_every, const double* dL_dz,
               double* z_out, double* dtheta, void* d_grad_work, size_t grad_work_bytes);

/*
 * Belief-propagation (BP) regauging of the state (paper, section "Method":
 * the PEPS re-gauged with BP after each Trotter step, for comparison;
 * "Results", "Benchmarking").  Messages of the norm network, one D x D
 * Hermitian matrix per leg of every site:
 *   m_{i->e}[a][a'] = sum Gamma_i[.., a, ..] conj(Gamma_i[.., a', ..]) prod_f E_f
 * over s and every other leg f of i, with E_f = diag(lambda_f) m_{k->f}
 * diag(lambda_f) built from the message of the neighbour k across f.  They
 * start at identity / D; an iteration recomputes all of them from the previous
 * iteration's, keeps them Hermitian, restricts them to the support of their
 * bond's lambda (entries k with lambda[k] <= cut * max zero; cut = 1e-13 for
 * GPEPS_C128, 1e-7 for GPEPS_MIXED_C64, below which a rank-deficient bond holds
 * only rounding residue) and normalises them to unit trace, until the largest
 * elementwise change is <= tol or after max_iter iterations.  Then
 * every edge e = (i, j) is gauged with the converged messages: with
 * R = conj(m)^{1/2} at both ends (pseudo-inverse below 1e-13 of the largest
 * eigenvalue), C = R_i diag(lambda_e) R_j^T = U S V^H, lambda_e' = S / ||S||,
 * Gamma_i <- Gamma_i (R_i^+ U) and Gamma_j <- Gamma_j (R_j^+ conj(V)) on leg e
 * (columns with S <= 1e-13 S_max zeroed).  The state is unchanged; the
 * mean-field readout afterwards uses the new gauge.  Messages, gauge matrices
 * and lambda are FP64; the message contractions run in the storage precision
 * (FP32 for GPEPS_MIXED_C64, where the eigenproblems of the gauge are also
 * warm-started in FP32 before FP64 sweeps, and the gauge is applied in FP32
 * when its matrices are well conditioned).  A pending kick commutes with the
 * regauge and stays pending.
 *   d_bp_work:  device, 256-byte aligned, >= gpeps_query_bp_workspace(max_iter)
 *               bytes (the messages of two iterations, the gauge matrices, the
 *               work lists and one global scratch slot per CTA)
 *   iterations: host, or NULL: BP iterations run
 *   residual:   host, or NULL: the largest elementwise change of the last one
 *   phase_ms:   host float[3], or NULL: device milliseconds (CUDA events) of the
 *               message launches (summed over iterations), the gauge and the apply
 * Synchronises the stream once per iteration (the convergence test), so it
 * cannot be captured into a CUDA graph.  Device flags: GPEPS_FLAG_NOCONV (a
 * gauge eigenproblem hit its sweep cap), GPEPS_FLAG_NUMERIC (a message with
 * non-positive or non-finite trace, or a vanishing gauged bond: that edge keeps
 * its gauge).  Errors: GPEPS_EINVAL for an unbound handle, D > 64, max_iter < 1,
 * negative or NaN tol, a NULL, misaligned or too small workspace.
 */
int gpeps_query_bp_workspace(gpeps_handle* h, int32_t max_iter, size_t* bytes);
int gpeps_bp_regauge(gpeps_handle* h, int32_t max_iter, double tol, void* d_bp_work, size_t bp_work_bytes,
                     int32_t* iterations, double* residual, float* phase_ms);

/* Totals of the batch: qubits, edges, bond updates per Trotter step. */
int gpeps_sizes(const gpeps_handle* h, int64_t* total_qubits, int64_t* total_edges);

/* Work counters since the last gpeps_reset, summed over bonds: FP64 Jacobi
 * sweeps, FP32 warm-start sweeps, and bond updates launched.  Host pointers
 * (any may be NULL); synchronises. */
int gpeps_sweeps(gpeps_handle* h, int64_t* sweeps64, int64_t* sweeps32, int64_t* total_bonds);

/*
 * Jacobi work executed since gpeps_reset, summed over every bond eigenproblem:
 * work (host int64[5]) = FP64 2x2 block updates (each rotates a 2x2 block of
 * the matrix from both sides, 72 flops), FP64 eigenvector pair updates (one row
 * of V, 18 flops), the same two counts of the FP32 levels, and the FP64 complex
 * multiply-adds with which the extra FP32 levels' rotations are applied to V
 * and rho' (8 flops each).  Converged pairs are skipped and not counted.  Synchronises the stream.  Errors: GPEPS_EINVAL
 * for NULL pointers or an unbound handle.
 */
int gpeps_jacobi_work(gpeps_handle* h, int64_t* work);

/* Counters of the bond-eigenproblem kernel since the last gpeps_reset, summed
 * over bonds, host int64[24].  [0..5] SM cycles (clock64 of one thread per
 * CTA) of its phases: [0] the bond matrix (mixed: the reduced density matrix
 * rho; complex128: the pivoted Cholesky roots of the Gram blocks, the core M
 * and rho = M^H M), [1] first FP32 Jacobi level, [2] FP64 re-orthonormalisation
 * of the FP32 eigenvectors, [3] mixed: V^dagger rho V and the further FP32
 * levels on small-eigenvalue blocks; complex128: B = M V and the further FP32
 * levels on blocks of small columns of B, [4] FP64 Jacobi sweeps (complex128:
 * one-sided, on B), [5] truncation, Y matrices and the smaller end.  [6..13]
 * rotations applied in sweep 0..7 of the first FP32 level, [14..21] in FP64
 * sweep 0..7, [22] and [23] SM cycles of the Gram pass and of the update pass
 * of the larger end inside the fused step (schedules 4 and 5; 0 otherwise).
 * Synchronises. */
int gpeps_bond_phase_cycles(gpeps_handle* h, int64_t* cycles);

/*
 * One simple-update bond step on two caller-owned site tensors, allocating
 * nothing.  The paper has no counterpart: this is a variant of the batched
 * layer for callers that cannot allocate device memory once they run, e.g. a
 * host framework that owns every device allocation through its own pool and
 * does not let libraries call cudaMalloc/cudaFree (which also synchronise the
 * device), or a latency-critical loop that must not pay for an allocation.
 *
 * Same arithmetic as gpeps_zz_layer for one bond: kick, absorb, gate, bond
 * eigenproblem, truncation to D, renormalisation, lambda^-1 strip.
 *   D, dtype      as in gpeps_create (1 <= D <= 32).
 *   gamma_a/b     device, the two site tensors (layout of gpeps_site_layout:
 *                 [s][leg0][leg1][leg2], last leg fastest), updated in place;
 *                 aligned to their element size, distinct.
 *   deg_a/b       degrees (1..3, not both 3); leg_a/b: position of the bond leg.
 *   lam           device float64[5][D]: row 0 lambda of the bond (replaced by
 *                 the new one, unsorted), rows 1-2 lambda of a's other legs in
 *                 leg order, rows 3-4 those of b (rows past the degree unused).
 *   theta         host float64[2] or NULL: kick angles exp(-i theta X/2) applied
 *                 to a and b before the gate (0 = none).
 *   stream        cudaStream_t or NULL; flags_out: host or NULL; when given the
 *                 call synchronises the stream and stores the GPEPS_FLAG_* bits.
 * Scratch: a file-scope device array of GPEPS_NOALLOC_SCRATCH_BYTES that every
 * GPU loading this library holds until the process exits; enough for D <= 32
 * in either dtype (larger sizes return GPEPS_EINVAL).  The first call on a
 * device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) and opts the kernels in to their shared memory; make
 * that first call before any stream capture.  Every call shares the array and
 * it keeps the last call's contents: calls whose work overlaps on the GPU (on
 * different streams, or from several threads) race and must be serialised by
 * the caller.  No cudaMalloc, cudaFree or allocating library call is made.
 */
#define GPEPS_NOALLOC_SCRATCH_BYTES (1u << 20)
int gpeps_bond_update_noalloc(int32_t D, int32_t dtype, void* gamma_a, int32_t deg_a, int32_t leg_a,
                              void* gamma_b, int32_t deg_b, int32_t leg_b, double* lam, const double* theta,
                              void* stream, int32_t* flags_out);

/*
 * Diagnostic, no part of the paper's method: the FP64 Jacobi rotation helpers
 * against the textbook formulas in CUDA's own FP64 hypot, sqrt and rsqrt.  For
 * k < n, in[4k..4k+3] = (a, b, Re g, Im g) (device float64; g != 0) describes the
 * 2 x 2 Hermitian [[a, g], [conj(g), b]]; out[8k..8k+7] (device float64)
 * receives the helper's (c, s, Re e, Im e) and then the reference's.  which: 0
 * the two-sided helper of the squared eigensolver (|g|^2 must be above FP32's
 * smallest normal), 1 the one-sided helper of the complex128 bond SVD (any
 * finite scale).  Asynchronous on stream.  Errors: GPEPS_EINVAL for n < 0, an
 * unknown `which` or NULL arrays; GPEPS_ECUDA for a failed launch.
 */
int gpeps_selftest_rotation(int32_t which, int32_t n, const double* in, double* out, void* stream);

int gpeps_destroy(gpeps_handle* h);
const char* gpeps_error_string(int status);
const char* gpeps_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GPEPS_H */
