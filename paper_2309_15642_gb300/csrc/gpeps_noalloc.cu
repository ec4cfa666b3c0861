// gpeps_bond_update_noalloc: one simple-update bond step on two caller-owned
// site tensors without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a host
// framework that owns every device allocation through its own pool and does
// not let libraries call cudaMalloc/cudaFree (which also synchronise the
// device), or a latency-critical loop that must not pay for an allocation.
// Such a caller passes only its tensors; the scratch of the three launches
// (Gram partials of the larger end, the Y matrices, the descriptors, the kick
// angles, the flag word and, in complex128, the bond kernel's matrices) lives in
// the file-scope device array below, which every GPU that loads this library
// holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "gpeps.h"
#include "gpeps_internal.cuh"

using namespace gpeps;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GPEPS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

// Layout of the scratch (bytes).
constexpr size_t kFlagsOff = 0;                                  // int flags[4]
constexpr size_t kSweepsOff = 16;                                // u64[kWorkCounters]
constexpr size_t kCyclesOff = 80;                                // u64[kCounters]
constexpr size_t kPendingOff = 320;                              // double pending[2], theta_a[1]
constexpr size_t kDescOff = 512;                                 // BondDesc, TileDesc[...]
constexpr int kNoallocMaxD = 32;                                 // bond dimension limit of this entry point
constexpr size_t kMaxTiles = (kNoallocMaxD * kNoallocMaxD + kTileRows - 1) / kTileRows;
constexpr size_t kYOff = 1024;                                   // 2 D^2 complex
constexpr size_t kPartOff = kYOff + (size_t)2 * kNoallocMaxD * kNoallocMaxD * 16;  // tiles x 2 D^2 complex
// complex128: the global slot of the bond kernel's matrices (its size depends on D; checked per call)
constexpr size_t kSlotOff = (kPartOff + kMaxTiles * 2 * kNoallocMaxD * kNoallocMaxD * 16 + 255) & ~(size_t)255;

static_assert(kSweepsOff + kWorkCounters * sizeof(unsigned long long) <= kCyclesOff, "work counters");
static_assert(kCyclesOff + kCounters * sizeof(unsigned long long) <= kPendingOff, "counter area");
static_assert(sizeof(BondDesc) + kMaxTiles * sizeof(TileDesc) <= kYOff - kDescOff, "descriptor area");
static_assert(kPartOff + kMaxTiles * 2 * kNoallocMaxD * kNoallocMaxD * 16 <= GPEPS_NOALLOC_SCRATCH_BYTES, "scratch size");

int fail_cuda(cudaError_t) { return GPEPS_ECUDA; }

// First call on a device (with that device current): the device address of the
// scratch array and the shared-memory opt-in of the kernels.
int scratch_for_current_device(void** out, int dtype) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e);
  if (dev < 0 || dev >= kMaxDevices) return GPEPS_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return fail_cuda(e);
    e = Launch<double>::init();
    if (e != cudaSuccess) return fail_cuda(e);
    e = Launch<float>::init();
    if (e != cudaSuccess) return fail_cuda(e);
    g_scratch[dev] = p;
  }
  (void)dtype;
  *out = g_scratch[dev];
  return GPEPS_OK;
}

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Side descriptor of a site of degree d whose bond leg is `leg`; lambda rows
// of its other legs are `row0`, `row0 + 1` of the caller's [5][D] array.
SideDesc side(int64_t off, int d, int leg, int D, int row0, int site) {
  SideDesc sd{};
  auto stride = [&](int q) { return (int32_t)ipow(D, d - 1 - q); };
  sd.off = off;
  sd.site = site;
  sd.str_s = (int32_t)ipow(D, d);
  sd.str_k = stride(leg);
  sd.rows = (int32_t)ipow(D, d - 1);
  int others[2], no = 0;
  for (int q = 0; q < d; ++q)
    if (q != leg) others[no++] = q;
  sd.lam_o1 = sd.lam_o2 = -1;
  sd.str_o1 = sd.str_o2 = 0;
  sd.n2 = 1;
  if (no == 2) {
    sd.str_o1 = stride(others[0]);
    sd.lam_o1 = row0 * D;
    sd.str_o2 = stride(others[1]);
    sd.lam_o2 = (row0 + 1) * D;
    sd.n2 = D;
  } else if (no == 1) {
    sd.str_o2 = stride(others[0]);
    sd.lam_o2 = row0 * D;
    sd.n2 = D;
  }
  return sd;
}

template <typename T>
int run(char* scratch, int D, void* base, const BondDesc& bd, int n_tiles, double* lam, JacobiParams jp,
        cudaStream_t st) {
  const TileDesc* tiles = reinterpret_cast<const TileDesc*>(scratch + kDescOff + sizeof(BondDesc));
  const BondDesc* bonds = reinterpret_cast<const BondDesc*>(scratch + kDescOff);
  double* pending = reinterpret_cast<double*>(scratch + kPendingOff);
  double* theta_a = pending + 2;
  int* flags = reinterpret_cast<int*>(scratch + kFlagsOff);
  auto* sweeps = reinterpret_cast<unsigned long long*>(scratch + kSweepsOff);
  auto* cycles = reinterpret_cast<unsigned long long*>(scratch + kCyclesOff);
  void* Y = scratch + kYOff;
  void* partials = scratch + kPartOff;
  cudaError_t e = Launch<T>::gram(tiles, n_tiles, bonds, base, lam, pending, partials, D, st);
  if (e == cudaSuccess)
    e = Launch<T>::bond(bonds, 1, partials, base, lam, pending, Y, theta_a, flags, sweeps, cycles, nullptr, D, jp,
                        st, nullptr, 0, scratch + kSlotOff);
  if (e == cudaSuccess) e = Launch<T>::update(tiles, n_tiles, bonds, base, lam, Y, theta_a, D, st);
  (void)bd;
  return e == cudaSuccess ? GPEPS_OK : GPEPS_ECUDA;
}

}  // namespace

extern "C" int gpeps_bond_update_noalloc(int32_t D, int32_t dtype, void* gamma_a, int32_t deg_a, int32_t leg_a,
                                         void* gamma_b, int32_t deg_b, int32_t leg_b, double* lam,
                                         const double* theta, void* stream, int32_t* flags_out) {
  if (D < 1 || D > kNoallocMaxD) return GPEPS_EINVAL;
  if (dtype != GPEPS_C128 && dtype != GPEPS_MIXED_C64) return GPEPS_EINVAL;
  if (!gamma_a || !gamma_b || !lam || gamma_a == gamma_b) return GPEPS_EINVAL;
  if (deg_a < 1 || deg_a > 3 || deg_b < 1 || deg_b > 3) return GPEPS_EINVAL;
  if (leg_a < 0 || leg_a >= deg_a || leg_b < 0 || leg_b >= deg_b) return GPEPS_EINVAL;
  if (deg_a == 3 && deg_b == 3) return GPEPS_EINVAL;
  const size_t elt = dtype == GPEPS_C128 ? 16 : 8;
  if (kSlotOff + bond_footprint(D, kBondSmemMax, elt).slot > GPEPS_NOALLOC_SCRATCH_BYTES) return GPEPS_EINVAL;
  const uintptr_t pa = reinterpret_cast<uintptr_t>(gamma_a), pb = reinterpret_cast<uintptr_t>(gamma_b);
  if ((pa % elt) || (pb % elt) || (reinterpret_cast<uintptr_t>(lam) % 8)) return GPEPS_EINVAL;
  void* sp = nullptr;
  int st = scratch_for_current_device(&sp, dtype);
  if (st) return st;
  char* scratch = static_cast<char*>(sp);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);

  // the larger end runs the Gram and update launches; tensors are addressed
  // from its pointer (the other end by its element distance)
  const bool a_big = deg_a >= deg_b;
  const uintptr_t pbig = a_big ? pa : pb, psmall = a_big ? pb : pa;
  const int64_t small_off = (int64_t)(psmall - pbig) / (int64_t)elt;
  BondDesc bd{};
  bd.a = a_big ? side(0, deg_a, leg_a, D, 1, 0) : side(0, deg_b, leg_b, D, 3, 0);
  bd.b = a_big ? side(small_off, deg_b, leg_b, D, 3, 1) : side(small_off, deg_a, leg_a, D, 1, 1);
  bd.lam_e = 0;
  bd.part0 = 0;
  bd.n_parts = (bd.a.rows + kTileRows - 1) / kTileRows;
  if ((size_t)bd.n_parts > kMaxTiles) return GPEPS_EINVAL;
  unsigned char host[kYOff];
  std::memset(host, 0, sizeof(host));
  double pend[3] = {0.0, 0.0, 0.0};
  if (theta) {
    pend[0] = a_big ? theta[0] : theta[1];
    pend[1] = a_big ? theta[1] : theta[0];
  }
  std::memcpy(host + kPendingOff, pend, sizeof(pend));
  std::memcpy(host + kDescOff, &bd, sizeof(bd));
  for (int p = 0; p < bd.n_parts; ++p) {
    TileDesc t{};
    t.bond = 0;
    t.row0 = p * kTileRows;
    t.nrows = bd.a.rows - t.row0 < kTileRows ? bd.a.rows - t.row0 : kTileRows;
    t.part = p;
    std::memcpy(host + kDescOff + sizeof(BondDesc) + p * sizeof(TileDesc), &t, sizeof(t));
  }
  // control words start at zero on every call; descriptors and angles replaced
  cudaError_t e = cudaMemcpyAsync(scratch, host, sizeof(host), cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return GPEPS_ECUDA;
  // Jacobi thresholds of the batched path for this dtype
  JacobiParams jp{};
  jp.tol = dtype == GPEPS_C128 ? 1e-14 : 1e-9;
  jp.floor_rel = dtype == GPEPS_C128 ? 1e-20 : 1e-8;
  jp.tol32 = 1e-6;
  jp.floor32 = 2e-7;
  jp.ev_cut = 0.0;
  jp.max_sweeps = 40;
  jp.max_sweeps32 = 20;
  jp.level_ratio = 1e-5;
  jp.levels = 4;
  jp.wait_cycles = kWaitCycles;
  jp.gate_sign = 1;
  void* base = reinterpret_cast<void*>(pbig);
  st = dtype == GPEPS_C128 ? run<double>(scratch, D, base, bd, bd.n_parts, lam, jp, cs)
                           : run<float>(scratch, D, base, bd, bd.n_parts, lam, jp, cs);
  if (st) return st;
  if (flags_out) {
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return GPEPS_ECUDA;
    int f = 0;
    e = cudaMemcpy(&f, scratch + kFlagsOff, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return GPEPS_ECUDA;
    *flags_out = f;
  }
  return GPEPS_OK;
}
