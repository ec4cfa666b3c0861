// Internal device-side data structures of the gPEPS simple-update library.
//
// Site tensors live in one state buffer, each Gamma_i as [s][leg0][leg1][leg2]
// (physical index outermost, legs in sorted-neighbour order, last leg fastest),
// followed by lambda_e as float64[D] per edge.  A bond update views each end as
// a matrix A[(other legs), (s, k)] through the strides of a SideDesc.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gpeps {

constexpr int kMaxD = 64;          // bond dimension limit of the mixed path, BP regauging and the no-alloc update
constexpr int kMaxDc128 = 128;     // bond dimension limit of the complex128 simple update
constexpr int kMaxLevel = 32;      // indices of one extra FP32 level (one per lane of a warp)
constexpr size_t kSmemOptin = 232448;  // opt-in shared memory per CTA of sm_100/sm_103 (227 KB)
constexpr size_t kBondSmemMax = kSmemOptin - 1024;  // dynamic part of a bond CTA (static variables need the rest)
constexpr int kTileRows = 64;      // rows of a big-side tile (Gram and update launches)
// Rows of a big-side tile at (D, element bytes): kTileRows, or 32 for complex128
// beyond D = 64, where a 64-row tile of 2D + 1 complex doubles (263 KB at D = 128)
// would not fit the shared memory of a CTA
__host__ __device__ constexpr int tile_rows(int D, size_t elt) { return (D > kMaxD && elt == 16) ? 32 : kTileRows; }
// Columns of Y_s that the update passes hold in shared memory at once
__host__ __device__ constexpr int y_cols(int D) { return D > kMaxD ? 32 : D; }
constexpr int kThreads = 256;      // threads of the streaming and readout CTAs
constexpr int kBondThreads = 512;  // threads of the bond-eigenproblem CTA (one CTA per SM: more warps hide FP64 latency)
constexpr double kLambdaCut = 1e-13;  // pseudo-inverse threshold relative to max(lambda)
constexpr int kPhases = 6;            // phases of the bond kernel with SM-cycle counters
constexpr int kRotSweeps = 8;         // rotation counters kept for the first sweeps of a solve
constexpr int kPassCounters = 2;     // fused step: SM cycles of the Gram pass and of the update pass of end a
constexpr int kCounters = kPhases + 2 * kRotSweeps + kPassCounters;  // cycles, FP32 rotations, FP64 rotations, passes
// Work counters of the bond kernels (u64 each): [0] FP64 sweeps, [1] FP32 sweeps of the first
// level, [2] extra FP32 levels, [3] FP64 complex MACs of the extra levels, [4] FP64 2x2 block
// updates, [5] FP64 eigenvector
// pair updates, [6] FP32 2x2 block updates, [7] FP32 eigenvector pair updates (all levels)
constexpr int kWorkCounters = 8;
constexpr int kMaxExtraLevels = 8;    // FP32 warm-start levels after the first (small-eigenvalue blocks)
constexpr double kNoiseRel = 1e-15;   // ... and above this fraction of the trace (FP64 rounding noise)

// One end of a bond seen as a matrix: row r = (r1, r2) runs over the other legs,
// column (s, k) over the physical index and the bond leg.
struct SideDesc {
  int64_t off;      // element offset of Gamma in the tensor area of the state
  int32_t rows;     // D^(deg-1)
  int32_t n2;       // extent of the faster other leg (1 if none)
  int32_t str_s;    // element stride of the physical index
  int32_t str_k;    // element stride of the bond leg
  int32_t str_o1;   // element stride of the slower other leg (0 if none)
  int32_t str_o2;   // element stride of the faster other leg (0 if none)
  int32_t lam_o1;   // lambda offset (float64 elements) of the slower other leg, -1 if none
  int32_t lam_o2;   // lambda offset of the faster other leg, -1 if none
  int32_t site;     // global site index (kick angles)
  int32_t pad;
};

// Bond (a, b): a is the end with more rows (Gram + update launches), b the end
// whose (row, s) space carries the bond eigenproblem (2 * b.rows <= 2D).
struct BondDesc {
  SideDesc a;
  SideDesc b;
  int32_t lam_e;    // lambda offset of the bond itself
  int32_t part0;    // first Gram-partial slot of side a
  int32_t n_parts;  // row tiles of side a
  int32_t pad;
};

struct TileDesc {
  int32_t bond;     // index into the colour class's bond list
  int32_t row0;     // first row of side a in this tile
  int32_t nrows;    // rows in this tile (<= kTileRows)
  int32_t part;     // Gram-partial slot written by this tile
};

// One bond update of the fused step: the bond, and the earlier tasks of the
// same step on its two sites (-1: none) that must be complete before it starts.
struct StepTask {
  BondDesc bd;
  int32_t dep_a;
  int32_t dep_b;
  int32_t colour;
  int32_t pad;
};

struct SiteDesc {
  int64_t off;      // element offset of Gamma
  int32_t deg;
  int32_t lam[3];   // lambda offsets of the legs in leg order (-1 past deg)
};

struct JacobiParams {
  double tol;        // FP64 sweeps: relative off-diagonal threshold |a_pq| <= tol sqrt(a_pp a_qq)
  double floor_rel;  // FP64 sweeps: absolute threshold |a_pq| <= floor_rel * trace
  double tol32;      // FP32 warm-start sweeps: the same two thresholds
  double floor32;
  double ev_cut;     // eigenvalues <= ev_cut * max eigenvalue are dropped (lambda = 0)
  int max_sweeps;    // FP64 cap (hitting it sets GPEPS_FLAG_NOCONV)
  int max_sweeps32;  // FP32 cap (hitting it only costs FP64 sweeps)
  double level_ratio;  // an extra FP32 level takes the diagonals below this fraction of their block's scale
  int levels;          // extra FP32 levels at most (0..kMaxExtraLevels)
  long long wait_cycles;  // fused step: a wait for an earlier task gives up after this many SM cycles
  int gate_sign;          // +1: the paper's exp(+i pi/4 Z Z); -1: its inverse exp(-i pi/4 Z Z)
};

// Tensor-core passes of the mixed path (bigend_tc.cuh): D = 32 or 64.
constexpr int kTcKc = 32;  // Gram pass: rows (the K extent) of one staged chunk
constexpr int kTcKu = 16;  // update pass: K values of one operand chunk (8 complex k of one spin)
__host__ __device__ constexpr bool tc_supported(int D) { return D == 32 || D == 64; }
// a wait for committed tensor-core products gives up after this many SM cycles (~2 s; a chunk takes microseconds)
constexpr long long kTcWaitCycles = 4000000000LL;
// TMEM columns of a CTA using the tensor-core passes (a power of two >= 32)
__host__ __device__ constexpr uint32_t tc_cols(int D) { return (uint32_t)(4 * D); }
// Shared memory of the Gram pass: the operand (hi | lo, 4D rows x kTcKc), the
// readout dump aliasing it (128 rows x (2D + 1) floats), the bulk-copy staging
// area (two spins x kTcKc rows x D complex) after both, one weight per row.
struct TcGramSmem {
  size_t stage, weight, total;
  __host__ __device__ constexpr TcGramSmem(int D)
      : stage((((size_t)4 * D * kTcKc * 8 > (size_t)128 * (2 * D + 1) * 4) ? (size_t)4 * D * kTcKc * 8
                                                                            : (size_t)128 * (2 * D + 1) * 4) +
                  15 & ~(size_t)15),
        weight(stage + (size_t)2 * kTcKc * D * 8),
        total(weight + (size_t)kTcKc * 4) {}
};
__host__ __device__ constexpr size_t tc_gram_smem(int D) { return TcGramSmem(D).total; }
// shared memory of the update chunk: hi and lo of A (128 rows) and of W (4D rows), kTcKu each, and the row mask
__host__ __device__ constexpr size_t tc_update_smem(int D) {
  return (size_t)(128 + 4 * D) * kTcKu * 4 * 2 + 128 * 4;
}

// Launchers (su_kernels.cu).  T = float for GPEPS_MIXED_C64, double for GPEPS_C128.
template <typename T>
struct Launch {
  static cudaError_t init();
  static cudaError_t reset(void* gamma, double* lam, int64_t n_gamma, int64_t n_lam_edges, int D,
                           const int64_t* d_site_off, int n_sites, double* pending, cudaStream_t st);
  // pending[i] += scale * theta (scale = -1: the inverse kick exp(+i theta X / 2))
  static cudaError_t kick(double* pending, const double* theta, const int32_t* site_inst, int n_sites,
                          int per_qubit, cudaStream_t st, double scale = 1.0);
  static cudaError_t gram(const TileDesc* tiles, int n_tiles, const BondDesc* bonds, const void* gamma,
                          const double* lam, const double* pending, void* partials, int D, cudaStream_t st);
  static cudaError_t bond(const BondDesc* bonds, int n_bonds, const void* partials, void* gamma, double* lam,
                          double* pending, void* Y, double* theta_a, int* flags,
                          unsigned long long* sweeps, unsigned long long* cycles, void* vsave, int D,
                          JacobiParams jp, cudaStream_t st, unsigned int* queue = nullptr, int n_ctas = 0,
                          void* scratch = nullptr, int per_sm = 1);
  static cudaError_t update(const TileDesc* tiles, int n_tiles, const BondDesc* bonds, void* gamma,
                            const double* lam, const void* Y, const double* theta_a, int D, cudaStream_t st);
  // The same two passes on the tensor cores (tcgen05, 3xTF32; complex64 storage, D = 32 or 64 only), one
  // CTA per bond over its row tiles; a wait that runs past kTcWaitCycles raises GPEPS_FLAG_TIMEOUT.
  static cudaError_t gram_tc(const BondDesc* bonds, int n_bonds, const void* gamma, const double* lam,
                             const double* pending, void* partials, int* flags, int D, cudaStream_t st);
  static cudaError_t update_tc(const BondDesc* bonds, int n_bonds, void* gamma, const double* lam, const void* Y,
                               const double* theta_a, int* flags, int D, cudaStream_t st);
  static cudaError_t readout(const SiteDesc* sites, int n_sites, const void* gamma, const double* lam,
                             const double* pending, double* z, int D, cudaStream_t st);
  // Every bond update of one Trotter step in one persistent launch (per_sm CTAs
  // per SM over the ordered task list; `done` holds one flag per task).
  static cudaError_t step(const StepTask* tasks, int n_tasks, unsigned int* queue, int* done, void* gamma,
                          double* lam, double* pending, int* flags, unsigned long long* sweeps,
                          unsigned long long* cycles, int D, JacobiParams jp, cudaStream_t st, int n_ctas,
                          void* scratch, size_t slot, int per_sm, bool tc = false);
};


constexpr int kMaxGradD = 16;  // bond dimension limit of the reverse mode (shared memory of its bond kernel)

// Reverse mode (complex128 only), su_kernels.cu.
struct Adjoint {
  static cudaError_t init();
  static cudaError_t layer(const TileDesc* tiles, int n_tiles, const BondDesc* bonds, int n_bonds, const void* gamma,
                           const double* lam, void* gbar, double* lbar, void* partG, void* partY, void* Gbar,
                           void* Ybuf, const void* vsave, int D, JacobiParams jp, cudaStream_t st);
  static cudaError_t apply_kick(const SiteDesc* sites, int n_sites, void* gamma, const double* theta, int D,
                                cudaStream_t st);
  static cudaError_t kick(const SiteDesc* sites, int n_sites, const void* gamma_post, void* gbar,
                          const double* theta, double* dtheta, int D, cudaStream_t st);
  static cudaError_t readout(const SiteDesc* sites, int n_sites, const void* gamma, const double* lam,
                             const double* cz, void* gbar, double* lbar, int D, cudaStream_t st);
};

cudaError_t launch_mean(const double* z, const int32_t* inst_site0, int n_inst, double* mean, cudaStream_t st);

// Memory of one bond-eigenproblem CTA at bond dimension D: the dynamic shared
// memory of its launch and, when the n x n matrices (n = 2D) do not fit the
// device's opt-in shared memory `smem_optin`, the bytes of the global scratch
// slot that holds them (0 otherwise; one slot per concurrently running bond).
struct BondFootprint {
  size_t smem;
  size_t slot;
};
// elt: bytes of a stored complex element (8: complex64, squared form; 16:
// complex128, whose unsquared form always keeps its matrices in a global slot).
BondFootprint bond_footprint(int D, size_t smem_optin, size_t elt);
// The same with the n x n matrices always in a global slot (the FP32 level in
// shared memory): the layout of the two-CTAs-per-SM schedule.
BondFootprint bond_footprint_global(int D, size_t elt);
// CTAs of the bond kernel sharing an SM in the global-matrix schedules: 2 of
// 256 threads or 4 of 128 threads, each with at most 1/k of the SM's 228 KB of
// shared memory (less 1 KB for the CTA's own reservation)
constexpr size_t kSmemPerSm = 233472;
constexpr size_t bond_share_smem(int k) { return kSmemPerSm / k - 1024 - 1024; }
constexpr int kMaxSms = 256;          // SMs the shared-SM schedules have scratch slots for

// Memory of a fused-step CTA: dynamic shared memory, and the bytes of its
// global slot (n x n matrices of the bond eigenproblem, FP64 Gram sums, Y and
// the kick angle of end a).
// tc: the Gram and update passes on the tensor cores (their staged operands set the floor).
BondFootprint step_footprint(int D, size_t elt, bool tc = false);
constexpr long long kWaitCycles = 4000000000LL;  // default wait limit of the fused step (~2 s of SM cycles)

// ---------------------------------------------------------------- BP regauging
// Messages live per half-edge h (a leg of a site), D x D complex FP64 each at
// msgs + h * D * D; the gauge matrices of the half-edges likewise.
struct BpMsgTask {
  int64_t off;     // element offset of Gamma_i
  int32_t deg;     // legs of site i
  int32_t leg;     // the leg p the message is sent along
  int32_t out;     // half-edge index of (i, p)
  int32_t in[3];   // per leg q != p: half-edge index of the neighbour's message towards i
  int32_t lam[3];  // per leg: lambda offset (float64 elements) of its edge
  int32_t pad;
};
struct BpEdgeTask {
  int32_t hi, hj;  // half-edge indices of the edge at its two ends
  int32_t lam;     // lambda offset of the edge
  int32_t pad;
};
struct BpSiteTask {
  int64_t off;     // element offset of Gamma_i
  int32_t deg;
  int32_t h0;      // half-edge index of leg 0 (legs are h0 .. h0 + deg - 1)
};
constexpr int kBpThreads = 256;      // threads of the BP apply CTA
constexpr int kBpMsgThreads = 256;   // threads of a BP message CTA (288, two upper-triangle entries per
                                     // thread at D = 32 instead of up to three, measured slower: 4.95
                                     // against 4.76 ms, one CTA per SM fewer)
constexpr double kBpGramCut = 1e-13; // eigenvalues of G below this fraction of the largest: pseudo-inverse 0
constexpr double kBpSupportCutF32 = 1e-7;  // complex64 storage: message support lambda_k > cut * max(lambda)
constexpr size_t kGaugeSmemMax = 2 * 32 * 32 * 16;  // the gauge CTA's Jacobi pair in shared memory up to D = 32
constexpr int kGaugeThreads = 128;                  // threads of a gauge CTA (four per SM)

// Launchers (bp_kernels.cu).  T is the storage type of Gamma; messages, gauge
// and lambda are FP64.
template <typename T>
struct BpLaunch {
  static cudaError_t init();
  static size_t message_smem(int D);
  static int resident(int D);  // message CTAs per SM (occupancy at D)
  static cudaError_t identity(double2* msgs, int n_half, int D, cudaStream_t st);
  static cudaError_t message(const BpMsgTask* tasks, int n_tasks, const void* gamma, const double* lam,
                             const double2* msg_in, double2* msg_out, void* scratch, int64_t slot_elems, int D,
                             unsigned long long* residual, int* flags, int n_ctas, cudaStream_t st,
                             bool tensor = false);  // tensor: tcgen05 products (complex64, D = 32 only)
  static cudaError_t apply(const BpSiteTask* sites, int n_sites, void* gamma, const double2* P, int D,
                           cudaStream_t st);
  // gauge of every edge in the arithmetic of T; scratch: 7 n x n complex of T per CTA, n = D
  // rounded up to even (up to D = 32 two of them sit in shared memory instead)
  static cudaError_t gauge(const BpEdgeTask* edges, int n_edges, const double2* msgs, double* lam, double2* P,
                           double2* scratch, int64_t slot_elems, int D, int* flags, int n_ctas, cudaStream_t st);
};

}  // namespace gpeps
