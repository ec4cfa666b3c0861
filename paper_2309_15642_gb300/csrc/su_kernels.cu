// CUDA kernels of the simple-update Trotter step (sm_103a).
//
// One bond update (paper, section "Method": simple update; gate of Eq. 2) is
// split over three batched launches per colour class:
//
//   gram    per row tile of the big end a: kick (Eq. 2, single-site factor) and
//           lambda of the other legs fused on load, partial Gram blocks
//           G_s[k][l] = sum_r conj(A[r][s][k]) A[r][s][l]          (T arithmetic)
//   bond    per bond: reduced density matrix of the small end b,
//           rho[x][y] = sum_s conj(g(s,t_x)) g(s,t_y) sum_{k,l} conj(F[x][k]) lam_k G_s[k][l] lam_l F[y][l]
//           with x = (row of b, t), F = kicked A_b; its Hermitian eigenproblem by
//           parallel cyclic Jacobi in FP64; keep the D largest eigenvalues
//           (Schmidt values s^2), lambda' = s / ||s||, Gamma_b' = conj(V) / lambda_other
//           (pseudo-inverse), and the small matrices
//           Y_s[k][k'] = lam_k sum_x F[x][k] g(s,t_x) V[x][k'] / s_k'
//   update  per row tile of a: Gamma_a'[r][s][k'] = sum_k A~[r][s][k] Y_s[k][k'] in place
//           (A~ = kicked Gamma_a without lambda: the lambda absorbed into the
//           Gram cancels against the lambda^-1 strip; rows whose lambda is below
//           the pseudo-inverse cut are zeroed).
//
// This is the textbook QR + SVD simple update rewritten around Gram matrices:
// the singular values and vectors of the gated two-site matrix are those of
// the eigenproblem of rho, so no panel QR is ever formed, and the only FP64
// work is the 2D x 2D bond eigenproblem (and, in complex128 mode, the products).
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "gpeps_internal.cuh"
#include "jacobi.cuh"

namespace gpeps {

// exp(-i theta X / 2) applied to the pair (g0, g1) of physical components.
template <typename T>
__device__ __forceinline__ void kick2(T c, T s, V2<T> g0, V2<T> g1, V2<T>& a0, V2<T>& a1) {
  a0 = mk<T>(c * g0.x + s * g1.y, c * g0.y - s * g1.x);
  a1 = mk<T>(s * g0.y + c * g1.x, -s * g0.x + c * g1.y);
}

struct RowPos {
  int r1, r2;
};
__device__ __forceinline__ RowPos row_pos(const SideDesc& sd, int r) {
  RowPos p;
  p.r1 = r / sd.n2;
  p.r2 = r - p.r1 * sd.n2;
  return p;
}
__device__ __forceinline__ int64_t elem(const SideDesc& sd, int s, RowPos p, int k) {
  return sd.off + (int64_t)s * sd.str_s + (int64_t)p.r1 * sd.str_o1 + (int64_t)p.r2 * sd.str_o2 +
         (int64_t)k * sd.str_k;
}
// Loads of state that another CTA of the same launch may have written (the
// fused step kernel) go around L1, which is not coherent between SMs; the
// layered kernels read state written by earlier launches only.
template <bool kCG, typename X>
__device__ __forceinline__ X ldst(const X* p) {
  if constexpr (kCG) return __ldcg(p);
  else return *p;
}
template <bool kCG = false>
__device__ __forceinline__ double row_weight(const SideDesc& sd, const double* lam, RowPos p) {
  double w = 1.0;
  if (sd.lam_o1 >= 0) w *= ldst<kCG>(lam + sd.lam_o1 + p.r1);
  if (sd.lam_o2 >= 0) w *= ldst<kCG>(lam + sd.lam_o2 + p.r2);
  return w;
}

}  // namespace gpeps
// tensor-core passes (they use the row/element helpers above)
#include "bigend_tc.cuh"
namespace gpeps {

// ---------------------------------------------------------------- reset / kick
template <typename T>
__global__ void reset_kernel(V2<T>* gamma, double* lam, const int64_t* site_off, int n_sites,
                             int64_t n_edges, int D, double* pending) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n_sites) {
    gamma[site_off[i]] = mk<T>((T)1, (T)0);
    pending[i] = 0.0;
  }
  if (i < n_edges) lam[i * D] = 1.0;
}

__global__ void kick_kernel(double* pending, const double* theta, const int32_t* site_inst, int n_sites,
                            int per_qubit, double scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_sites) pending[i] += scale * (per_qubit ? theta[i] : theta[site_inst[i]]);
}

// ---------------------------------------------------------------- Gram partials
template <typename T>
__global__ void __launch_bounds__(kThreads)
    gram_kernel(const TileDesc* __restrict__ tiles, const BondDesc* __restrict__ bonds,
                const V2<T>* __restrict__ gamma, const double* __restrict__ lam,
                const double* __restrict__ pending, V2<T>* __restrict__ partials, int D) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V2<T>* A = reinterpret_cast<V2<T>*>(smem_raw);  // [nrows][2D+1]
  const TileDesc t = tiles[blockIdx.x];
  const SideDesc sa = bonds[t.bond].a;
  const int ld = 2 * D + 1;
  const double th = pending[sa.site];
  const T c = (T)cos(0.5 * th), s = (T)sin(0.5 * th);
  const int nel = t.nrows * D;
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    int r, k;
    if (sa.str_k == 1) {
      r = idx / D;
      k = idx - r * D;
    } else {
      k = idx / t.nrows;
      r = idx - k * t.nrows;
    }
    const RowPos p = row_pos(sa, t.row0 + r);
    const int64_t e = elem(sa, 0, p, k);
    const T w = (T)row_weight(sa, lam, p);
    V2<T> a0, a1;
    kick2<T>(c, s, gamma[e], gamma[e + sa.str_s], a0, a1);
    A[r * ld + k] = mk<T>(a0.x * w, a0.y * w);
    A[r * ld + D + k] = mk<T>(a1.x * w, a1.y * w);
  }
  __syncthreads();
  const int D2 = D * D;
  const int nout = 2 * D2;
  V2<T>* out = partials + (int64_t)t.part * nout;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int sidx = o / D2;
    const int kl = o - sidx * D2;
    const int k = kl / D;
    const int l = kl - k * D;
    const V2<T>* ck = A + sidx * D + k;
    const V2<T>* cl = A + sidx * D + l;
    V2<T> acc = mk<T>(0, 0);
    for (int r = 0; r < t.nrows; ++r) fma_conj<T>(acc, ck[r * ld], cl[r * ld]);
    out[o] = acc;
  }
}

// ---------------------------------------------------------------- bond eigenproblem

// Memory layout of bond_kernel for a bond whose small end has nb rows
// (n = 2 nb).  Three large regions of complex doubles (the big part):
//   R    [n][n+1]                 the bond matrix rho, later V^dagger rho V
//   Vr   max(n*n, 2D^2 + n*D)     Gram blocks C_s and H while rho is formed, then V
//   X    max(n*(n+1), n*D)        F; then the FP32 copies rho32 [n][n+1] and V32 [n][n+1];
//                                 then the Gram/Cholesky factor of V; then rho V; then F again
// and the small arrays (rotations of both precisions, eigenvalues, indices).
// Both parts sit in shared memory when they fit (D <= 34); beyond that the big
// part is a slot of a global scratch buffer (held in L2 by the running CTAs)
// and only the small arrays stay in shared memory.  Offsets of the big part
// are relative to its base, offsets of the small arrays to theirs.
struct BondSmem {
  size_t off_R, off_V, off_X, big, off_re, off_re32, off_lamo, off_ev, off_sv, off_rc, off_rs, off_scal, off_rc32,
      off_rs32, off_int, small;
  __host__ __device__ BondSmem(int D, int n) {
    const int m = n / 2;
    size_t v = (size_t)n * n;
    if ((size_t)2 * D * D + (size_t)n * D > v) v = (size_t)2 * D * D + (size_t)n * D;
    size_t x = (size_t)n * (n + 1);
    if ((size_t)n * D > x) x = (size_t)n * D;
    off_R = 0;
    off_V = off_R + (size_t)n * (n + 1) * 16;
    off_X = off_V + v * 16;
    big = off_X + x * 16;
    off_re = 0;
    off_re32 = off_re + (size_t)m * 16;
    off_lamo = off_re32 + (size_t)((m + 1) / 2) * 16;
    off_ev = off_lamo + (size_t)D * 8;
    off_sv = off_ev + (size_t)n * 8;
    off_rc = off_sv + (size_t)D * 8;
    off_rs = off_rc + (size_t)m * 8;
    off_scal = off_rs + (size_t)m * 8;
    off_rc32 = off_scal + 8 * 8;
    off_rs32 = off_rc32 + (size_t)((m + 1) / 2) * 8;
    off_int = off_rs32 + (size_t)((m + 1) / 2) * 8;
    small = (off_int + (size_t)(n + 2 * m + 8 + 144) * 4 + 15) & ~(size_t)15;  // order, rp, rq, iflag, Jacobi lists
    // global-memory mode: the FP32 level's packed rho32 and V32 follow the small
    // arrays, and later the scratch of the extra levels (lv = min(n/2, 32)
    // indices: W64 [lv][lv], Gw [lv][lv+1] complex double, B32 [lv][lv+1],
    // W32 [lv][lv] complex float)
    f32 = ((size_t)n * (n + 1) / 2 + (size_t)n * (n + 1)) * 8;
    const size_t lv = (size_t)(m < kMaxLevel ? m : kMaxLevel);
    const size_t lvl = lv * (48 * lv + 24);
    if (lvl > f32) f32 = lvl;
  }
  size_t f32;
};

// Big part of the bond layout: the squared form (BondSmem) for complex64 storage,
// the unsquared SVD form (SvdLayout, declared below) for complex128.
__host__ __device__ size_t bond_big(int D, size_t elt);
// Shared scratch after the small arrays: the FP32 level of the squared form, or
// the FP32 warm start and levels of the unsquared form (svd_f32_bytes, below).
__host__ __device__ size_t svd_f32_bytes(int D);
static size_t bond_f32(int D, size_t elt) { return elt == 16 ? svd_f32_bytes(D) : BondSmem(D, 2 * D).f32; }

BondFootprint bond_footprint(int D, size_t smem_optin, size_t elt) {
  const BondSmem L(D, 2 * D);
  if (elt == 8 && L.big + L.small <= smem_optin) return BondFootprint{L.big + L.small, 0};
  return BondFootprint{L.small + bond_f32(D, elt), (bond_big(D, elt) + 255) & ~(size_t)255};
}

BondFootprint bond_footprint_global(int D, size_t elt) {
  const BondSmem L(D, 2 * D);
  return BondFootprint{L.small + bond_f32(D, elt), (bond_big(D, elt) + 255) & ~(size_t)255};
}


// Bijection from [0, n(n+1)/2) onto the upper triangle i <= j of an n x n
// matrix (n even): row r is paired with row n-1-r (lengths n-r and r+1), so a
// loop over the triangle keeps every lane busy.
__device__ __forceinline__ void upper_index(int idx, int n, int& i, int& j) {
  const int w = n + 1;
  const int r = idx / w, c = idx - (idx / w) * w;
  if (c < n - r) {
    i = r;
    j = r + c;
  } else {
    i = n - 1 - r;
    j = i + (c - (n - r));
  }
}

// Re-orthonormalise the columns of V (n x n, row stride n) in FP64.  V is a
// product of FP32 rotations, so G = V^dagger V = I + E with |E| ~ 1e-6 and the
// Cholesky factor R (G = R^dagger R) and its inverse follow from short series
// that are exact to O(|E|^3) ~ 1e-18, with only parallel products:
//   X1 = P(E), X = P(E - X1^dagger X1), R = I + X, R^-1 = I - X + X^2,
// where P keeps the strict upper triangle and half the diagonal.  Q = V R^-1
// is formed row by row in place (one warp per row).  G holds E and X in its
// upper triangle and X1^dagger X1, X^2 in its strict lower triangle (row
// stride ldg); dg[n] holds their diagonals.  Returns max |E_ij|.
//
// kF32Products (the complex64 path, whose bond matrix carries FP32 rounding):
// the two products of E-sized factors, X1^dagger X1 and X^2, run in FP32 on
// FP32 copies of X1 and X.  Their entries are O(n |E|^2) ~ 1e-10, so FP32's
// relative 1e-7 leaves absolute errors at or below the FP64 rounding of E itself
// at the |E| ~ 1e-6 of a 64-wide FP32 solve; E = V^dagger V - I and Q = V R^-1
// stay FP64.  The FP32 copy of upper entry (i, j) sits in the otherwise unused
// 16 bytes mirrored below the diagonal, (j, i) for i < j and the padding column
// (i, n) for i = j (ldg >= n + 1): X1 in its first 8 bytes, X in its last 8.
// Q pairs the columns j and n-1-j on one lane (n <= 128).
__device__ __forceinline__ float2* tri32(double2* G, int ldg, int n, int i, int j) {
  return reinterpret_cast<float2*>(i < j ? G + j * ldg + i : G + i * ldg + n);
}

template <bool kF32Products>
__device__ double orthonormalise(double2* V, int n, double2* G, int ldg, double* dg, double* scal) {
  if constexpr (kF32Products) {
    // E = V^dagger V - I (upper triangle, FP64) and the FP32 copy of X1 = P(E)
    for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
      int i, j;
      upper_index(idx, n, i, j);
      double2 acc = make_double2(i == j ? -1.0 : 0.0, 0.0);
      for (int r = 0; r < n; ++r) fma_conj<double>(acc, V[r * n + i], V[r * n + j]);
      if (i == j) acc.y = 0.0;
      G[i * ldg + j] = acc;
      tri32(G, ldg, n, i, j)[0] =
          i == j ? make_float2((float)(0.5 * acc.x), 0.f) : make_float2((float)acc.x, (float)acc.y);
    }
    if (threadIdx.x == 0) scal[6] = 0.0;
    __syncthreads();
    // K = X1^dagger X1 (FP32, K_ij = sum_{k <= i} conj(X1_ki) X1_kj), X = P(E - K) in FP64
    // over E, and its FP32 copy; record max |E|
    for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
      int i, j;
      upper_index(idx, n, i, j);
      float2 k32 = make_float2(0.f, 0.f);
      for (int k = 0; k <= i; ++k) fma_conj<float>(k32, tri32(G, ldg, n, k, i)[0], tri32(G, ldg, n, k, j)[0]);
      const double2 e = G[i * ldg + j];
      const double ae = fabs(e.x) + fabs(e.y);
      if (ae > scal[6]) atomicMax(reinterpret_cast<unsigned long long*>(scal + 6), __double_as_longlong(ae));
      const double2 x = i == j ? make_double2(0.5 * (e.x - (double)k32.x), 0.0)
                               : make_double2(e.x - (double)k32.x, e.y - (double)k32.y);
      G[i * ldg + j] = x;
      tri32(G, ldg, n, i, j)[1] = make_float2((float)x.x, (float)x.y);
    }
    __syncthreads();
    // M = X^2 - X in the upper triangle (X^2 upper triangular, FP32: (X^2)_ij = sum_{i<=k<=j} X_ik X_kj)
    for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
      int i, j;
      upper_index(idx, n, i, j);
      float2 s32 = make_float2(0.f, 0.f);
      for (int k = i; k <= j; ++k) fma_c<float>(s32, tri32(G, ldg, n, i, k)[1], tri32(G, ldg, n, k, j)[1]);
      const double2 x = G[i * ldg + j];
      G[i * ldg + j] = i == j ? make_double2((double)s32.x - x.x, 0.0)
                              : make_double2((double)s32.x - x.x, (double)s32.y - x.y);
    }
    __syncthreads();
  } else {
    // E = V^dagger V - I (upper triangle)
    for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
      int i, j;
      upper_index(idx, n, i, j);
      double2 acc = make_double2(i == j ? -1.0 : 0.0, 0.0);
      for (int r = 0; r < n; ++r) fma_conj<double>(acc, V[r * n + i], V[r * n + j]);
      if (i == j) acc.y = 0.0;
      G[i * ldg + j] = acc;
    }
    if (threadIdx.x == 0) scal[6] = 0.0;
    __syncthreads();
    // K = X1^dagger X1 with X1 = P(E): K_ij = sum_{k <= i} conj(X1_ki) X1_kj  (i <= j)
    for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
      int i, j;
      upper_index(idx, n, i, j);
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k <= i; ++k) {
        double2 xki = G[k * ldg + i], xkj = G[k * ldg + j];
        if (k == i) xki = cscale(xki, 0.5);
        if (k == j) xkj = cscale(xkj, 0.5);
        fma_conj<double>(acc, xki, xkj);
      }
      if (i == j) dg[i] = acc.x;
      else G[j * ldg + i] = acc;
    }
    __syncthreads();
    // X = P(E - K) in the upper triangle; record max |E|
    for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
      int i, j;
      upper_index(idx, n, i, j);
      const double2 e = G[i * ldg + j];
      const double ae = fabs(e.x) + fabs(e.y);
      if (ae > scal[6]) atomicMax(reinterpret_cast<unsigned long long*>(scal + 6), __double_as_longlong(ae));
      if (i == j) G[i * ldg + i] = make_double2(0.5 * (e.x - dg[i]), 0.0);
      else G[i * ldg + j] = csub(e, G[j * ldg + i]);
    }
    __syncthreads();
    // X^2 (upper triangular) into the strict lower triangle and dg
    for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
      int i, j;
      upper_index(idx, n, i, j);
      double2 acc = make_double2(0.0, 0.0);
      for (int k = i; k <= j; ++k) fma_c<double>(acc, G[i * ldg + k], G[k * ldg + j]);
      if (i == j) dg[i] = acc.x;
      else G[j * ldg + i] = acc;
    }
    __syncthreads();
    // M = X^2 - X in the upper triangle
    for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
      int i, j;
      upper_index(idx, n, i, j);
      if (i == j) G[i * ldg + i] = make_double2(dg[i] - G[i * ldg + i].x, 0.0);
      else G[i * ldg + j] = csub(G[j * ldg + i], G[i * ldg + j]);
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (kF32Products && n <= 128) {
    // Q[r][j] = V[r][j] + sum_{i <= j} V[r][i] M[i][j], one warp per row, in place: lane l
    // forms the column pairs (j, n-1-j) for j = l and l + 32 (below n/2) in one pass of n + 1
    // products each (i = t for column j while t <= j, then i = t - j - 1 for column n-1-j),
    // so that no lane of an FP64 instruction idles on a shorter column, and writes after
    // the whole warp has read the row
    const int h = n >> 1;
    for (int r = warp; r < n; r += nw) {
      double2* v = V + r * n;
      double2 out[4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = lane + 32 * u;
        if (j < h) {
          const int j2 = n - 1 - j;
          double2 acc = v[j];
          for (int t = 0; t <= n; ++t) {
            if (t == j + 1) {
              out[2 * u] = acc;
              acc = v[j2];
            }
            const bool first = t <= j;
            const int i = first ? t : t - j - 1;
            fma_c<double>(acc, v[i], G[i * ldg + (first ? j : j2)]);
          }
          out[2 * u + 1] = acc;
        }
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = lane + 32 * u;
        if (j < h) {
          v[j] = out[2 * u];
          v[n - 1 - j] = out[2 * u + 1];
        }
      }
      __syncwarp();
    }
  } else {
    // Q[r][j] = V[r][j] + sum_{i <= j} V[r][i] M[i][j], one warp per row, in place:
    // 32-column chunks from the right, since a chunk reads only columns at or
    // left of its own (each lane computes its column before any lane writes)
    for (int r = warp; r < n; r += nw) {
      double2* v = V + r * n;
      for (int c = (n - 1) >> 5; c >= 0; --c) {
        const int j = lane + 32 * c;
        double2 acc = make_double2(0.0, 0.0);
        if (j < n) {
          acc = v[j];
          for (int i = 0; i <= j; ++i) fma_c<double>(acc, v[i], G[i * ldg + j]);
        }
        __syncwarp();
        if (j < n) v[j] = acc;
        __syncwarp();
      }
    }
  }
  __syncthreads();
  return scal[6];
}

// FP32 warm start of a Hermitian eigenproblem: the FP64 n x n matrix RHO (row
// stride n+1) rounded to FP32 and diagonalised there by parallel cyclic Jacobi
// to convergence, its eigenvectors widened into Vm [n][n] and re-orthonormalised
// in FP64 (`orthonormalise`, X as scratch).  The FP32 copies live in X, or
// (f32s given: the n x n matrices are in global memory) packed in shared memory
// at f32s.  Returns the FP32 sweeps.
__device__ int fp32_warm_start(const double2* RHO, double2* Vm, double2* X, int n, double trace,
                               const JacobiParams& jp, float2* re32, double* ev, double* scal, float* rc32,
                               float* rs32, int* rp, int* rq, int* iflag, unsigned long long* sweeps_out,
                               unsigned long long* cycles, int* flags, long long& t_prev, float2* f32s) {
  const int ldr = n + 1;
  const bool packed = f32s != nullptr;
  float2* R32 = packed ? f32s : reinterpret_cast<float2*>(X);
  float2* V32 = packed ? f32s + (size_t)n * (n + 1) / 2 : R32 + (size_t)n * (n + 1);
  const int ldv32 = n + 1;  // odd row stride: the eigenvector updates run conflict-free down the rows
  auto mark = [&](int phase) {
    if (threadIdx.x == 0 && cycles) {
      const long long t = clock64();
      atomicAdd(cycles + phase, (unsigned long long)(t - t_prev));
      t_prev = t;
    }
  };
  const HermPacked<float> P32{R32, n};
  if (packed) {
    for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
      int i, j;
      upper_index(idx, n, i, j);
      const double2 v = RHO[i * ldr + j];
      R32[P32.at(i, j)] = make_float2((float)v.x, (float)v.y);
    }
  } else {
    for (int idx = threadIdx.x; idx < n * ldr; idx += blockDim.x) {
      const double2 v = RHO[idx];
      R32[idx] = make_float2((float)v.x, (float)v.y);
    }
  }
  for (int idx = threadIdx.x; idx < n * ldv32; idx += blockDim.x)
    V32[idx] = make_float2((idx / ldv32) == (idx % ldv32) ? 1.f : 0.f, 0.f);
  __syncthreads();
  unsigned long long* rc32_count = cycles ? cycles + kPhases : nullptr;
  const int sw32 =
      packed ? jacobi_hermitian<float, true, HermPacked<float>, true>(
                   P32, V32, ldv32, n, (float)jp.tol32, (float)(jp.floor32 * trace), jp.max_sweeps32, rc32, rs32,
                   re32, rp, rq, iflag, rc32_count, sweeps_out + 6)
             : jacobi_hermitian<float, true, HermFull<float>, true>(
                   HermFull<float>{R32, ldr}, V32, ldv32, n, (float)jp.tol32, (float)(jp.floor32 * trace),
                   jp.max_sweeps32, rc32, rs32, re32, rp, rq, iflag, rc32_count, sweeps_out + 6);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - (idx / n) * n;
    const float2 v = V32[i * ldv32 + j];
    Vm[idx] = make_double2((double)v.x, (double)v.y);
  }
  __syncthreads();
  mark(1);
  const double emax = orthonormalise<true>(Vm, n, X, ldr, ev, scal);
  if (threadIdx.x == 0 && !(emax < 1e-4)) atomicOr(flags, 1);  // FP32 basis too far from unitary
  mark(2);
  return sw32;
}

// Mixed-precision Jacobi eigensolver of the Hermitian n x n matrix RHO (FP64,
// row stride n+1, trace > 0) in shared memory: FP32 sweeps to convergence on a
// rounded copy, FP64 re-orthonormalisation of their eigenvectors, rho' =
// V^dagger rho V in FP64, further FP32 levels on rescaled small-eigenvalue
// blocks, FP64 sweeps to the thresholds of jp.  On return RHO is diagonal (the
// eigenvalues) and Vm [n][n] holds the eigenvectors.  X is scratch of
// max(n(n+1), n D) complex doubles; the small arrays as in bond_kernel.
// Returns the FP64 sweeps (max_sweeps + 1 = cap hit).
__device__ int eig_mixed(double2* RHO, double2* Vm, double2* X, int n, int D, double trace, const JacobiParams& jp,
                         double2* re, float2* re32, double* ev, double* rc, double* rs, double* scal, float* rc32,
                         float* rs32, int* order, int* rp, int* rq, int* iflag, unsigned long long* sweeps_out,
                         unsigned long long* cycles, int* flags, long long& t_prev, float2* f32s) {
  const int ldr = n + 1;
  const bool packed = f32s != nullptr;
  auto mark = [&](int phase) {
    if (threadIdx.x == 0 && cycles) {
      const long long t = clock64();
      atomicAdd(cycles + phase, (unsigned long long)(t - t_prev));
      t_prev = t;
    }
  };
  const int sw32 = fp32_warm_start(RHO, Vm, X, n, trace, jp, re32, ev, scal, rc32, rs32, rp, rq, iflag, sweeps_out,
                                   cycles, flags, t_prev, f32s);
  // rho' = V^dagger rho V: W = rho V into X, then the upper triangle of V^dagger W into RHO
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - (idx / n) * n;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < n; ++k) fma_c<double>(acc, RHO[i * ldr + k], Vm[k * n + j]);
    X[i * ldr + j] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
    int i, j;
    upper_index(idx, n, i, j);
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < n; ++k) fma_conj<double>(acc, Vm[k * n + i], X[k * ldr + j]);
    RHO[i * ldr + j] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - (idx / n) * n;
    if (j > i) RHO[j * ldr + i] = cconj(RHO[i * ldr + j]);
    if (j == i) RHO[i * ldr + i].y = 0.0;
  }
  __syncthreads();
  // Further FP32 levels for the eigenvalues the previous level could not
  // resolve (FP32 rounding ~1e-7 of that level's largest entry).  Every index
  // remembers the scale of the last block that held it (the whole matrix at
  // first); a level takes the largest indices (at most min(n/2, 32)) whose
  // diagonal lies below jp.level_ratio x that scale and above rounding noise of
  // the whole matrix, diagonalises their block again in FP32 on a rescaled copy,
  // and applies the rotation, re-orthonormalised in FP64, to V and to rho' in FP64.
  {
    int* cand = order;    // [n] candidate indices of this level, largest first
    double* dcur = ev;
    double* rscale = rc;  // [n] (rc and rs are contiguous and idle until the FP64 sweeps)
    int* mark_c = rp;     // [n] (rp and rq likewise, idle during the selection)
    const int cap = (n / 2 < kMaxLevel) ? n / 2 : kMaxLevel;
    // level scratch for ns <= lv indices: in X, or in the free FP32 shared memory
    // (sized for min(n/2, 32) indices)
    const int lv = packed ? cap : n / 2;
    double2* W64 = packed ? reinterpret_cast<double2*>(f32s) : X;   // [ns][ns]
    double2* Gw = W64 + (size_t)lv * lv;                             // [ns][ns+1]
    float2* B32 = reinterpret_cast<float2*>(Gw + (size_t)lv * (lv + 1));  // [ns][ns+1]
    float2* W32 = B32 + (size_t)lv * (lv + 1);                            // [ns][ns]
    const double lo = kNoiseRel * trace;
    for (int level = 0; level < jp.levels; ++level) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) dcur[i] = RHO[i * ldr + i].x;
      __syncthreads();
      if (level == 0) {
        if (threadIdx.x == 0) {
          double s0 = 0.0;
          for (int i = 0; i < n; ++i) s0 = fmax(s0, dcur[i]);
          scal[3] = s0;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) rscale[i] = scal[3];
      }
      for (int i = threadIdx.x; i < n; i += blockDim.x)
        mark_c[i] = (dcur[i] > lo && dcur[i] <= jp.level_ratio * rscale[i]) ? 1 : 0;
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (!mark_c[i]) continue;
        const double di = dcur[i];
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += mark_c[j] && (dcur[j] > di || (dcur[j] == di && j < i));
        if (rank < cap) cand[rank] = i;
      }
      if (threadIdx.x == 0) {
        int cnt = 0;
        for (int j = 0; j < n; ++j) cnt += mark_c[j];
        iflag[1] = (cnt < cap ? cnt : cap) & ~1;  // even: drop the smallest
      }
      __syncthreads();
      if (threadIdx.x == 0) scal[7] = iflag[1] > 0 ? dcur[cand[0]] : 0.0;
      __syncthreads();
      const int ns = iflag[1];
      const double bscale = scal[7];
      if (ns < 2 || !(bscale > 0.0)) break;
      const int ldb = ns + 1;
      const double inv = 1.0 / bscale;
      double btr = 0.0;
      for (int idx = threadIdx.x; idx < ns * ns; idx += blockDim.x) {
        const int a = idx / ns, b = idx - (idx / ns) * ns;
        const double2 v = RHO[cand[a] * ldr + cand[b]];
        B32[a * ldb + b] = make_float2((float)(v.x * inv), (float)(v.y * inv));
        W32[a * ns + b] = make_float2(a == b ? 1.f : 0.f, 0.f);
      }
      for (int a = 0; a < ns; ++a) btr += dcur[cand[a]] * inv;
      __syncthreads();
      const int swl = jacobi_hermitian<float, true>(HermFull<float>{B32, ldb}, W32, ns, ns, (float)jp.tol32,
                                                    (float)(jp.floor32 * btr), jp.max_sweeps32, rc32, rs32, re32,
                                                    rp, rq, iflag, nullptr, sweeps_out + 6);
      (void)swl;
      for (int idx = threadIdx.x; idx < ns * ns; idx += blockDim.x) {
        const float2 v = W32[idx];
        W64[idx] = make_double2((double)v.x, (double)v.y);
      }
      __syncthreads();
      orthonormalise<true>(W64, ns, Gw, ldb, dcur, scal);
      // rows of V and rho': X[r][cand] <- X[r][cand] W, then the columns of rho':
      // rho'[cand][c] <- W^dagger rho'[cand][c]; a row (column) per segment of seg >= ns
      // lanes, 32 / seg of them per warp, so that a small level does not leave most
      // lanes of each FP64 instruction idle
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      const int seg = ns <= 8 ? 8 : (ns <= 16 ? 16 : 32), per = 32 / seg;
      const int sub = lane / seg, sl = lane - (lane / seg) * seg;
      for (int r0 = warp * per; r0 < 2 * n; r0 += nw * per) {
        const int rr = r0 + sub;
        const bool on = rr < 2 * n && sl < ns;
        double2* row = rr < n ? Vm + rr * n : RHO + (rr - n) * ldr;
        double2 out = make_double2(0.0, 0.0);
        if (on) {
          for (int a = 0; a < ns; ++a) fma_c<double>(out, row[cand[a]], W64[a * ns + sl]);
        }
        __syncwarp();
        if (on) row[cand[sl]] = out;
        __syncwarp();
      }
      __syncthreads();
      for (int c0 = warp * per; c0 < n; c0 += nw * per) {
        const int c = c0 + sub;
        const bool on = c < n && sl < ns;
        double2 out = make_double2(0.0, 0.0);
        if (on) {
          for (int a = 0; a < ns; ++a) fma_conj<double>(out, W64[a * ns + sl], RHO[cand[a] * ldr + c]);
        }
        __syncwarp();
        if (on) RHO[cand[sl] * ldr + c] = out;
        __syncwarp();
      }
      for (int a = threadIdx.x; a < ns; a += blockDim.x) rscale[cand[a]] = bscale;
      __syncthreads();
      if (threadIdx.x == 0) {
        atomicAdd(sweeps_out + 2, 1ull);
        // FP64 complex MACs of this level: rows of V and rho' (2n x ns x ns), columns of
        // rho' (n x ns x ns), the re-orthonormalisation of W (its Gram and Q = W R^-1,
        // about ns^3 / 2 each; its other products run in FP32)
        const unsigned long long nsl = (unsigned long long)ns;
        atomicAdd(sweeps_out + 3, 3ull * n * nsl * nsl + nsl * nsl * nsl);
      }
    }
  }
  mark(3);
  const int sweeps = jacobi_hermitian<double, false>(HermFull<double>{RHO, ldr}, Vm, n, n, jp.tol,
                                                     jp.floor_rel * trace,
                                                     jp.max_sweeps, rc, rs, re, rp, rq, iflag,
                                                     cycles ? cycles + kPhases + kRotSweeps : nullptr,
                                                     sweeps_out + 4);
  mark(4);
  if (threadIdx.x == 0) {
    if (sweeps > jp.max_sweeps) atomicOr(flags, 1);
    atomicAdd(sweeps_out, (unsigned long long)(sweeps > jp.max_sweeps ? jp.max_sweeps : sweeps));
    atomicAdd(sweeps_out + 1, (unsigned long long)(sw32 > jp.max_sweeps32 ? jp.max_sweeps32 : sw32));
  }
  return sweeps;
}

// A bond whose spectrum is not usable (NaN/Inf or zero norm) is left as it
// was: Y = identity so that the update launch only applies the pending kick
// to end a, lambda and end b untouched; the flag word reports it.
template <typename T, bool kCG>
__device__ void bond_fail(const BondDesc& bd, V2<T>* Y, double* theta_a, double* pending, int* flags, int D) {
  const int D2 = D * D;
  for (int o = threadIdx.x; o < 2 * D2; o += blockDim.x) {
    const int kl = o % D2;
    Y[o] = mk<T>((T)((kl / D) == (kl % D) ? 1 : 0), (T)0);
  }
  if (threadIdx.x == 0) {
    atomicOr(flags, 2);
    *theta_a = ldst<kCG>(pending + bd.a.site);
    pending[bd.a.site] = 0.0;
  }
}

// F[(row, t)][k]: kicked Gamma_b with the lambda of its other legs, in the
// storage precision T.
template <typename T, bool kCG>
__device__ void load_F(const SideDesc& sb, const V2<T>* gamma, const double* lam, double th, V2<T>* F, int D) {
  const T c = (T)cos(0.5 * th), s = (T)sin(0.5 * th);
  for (int idx = threadIdx.x; idx < sb.rows * D; idx += blockDim.x) {
    const int rj = idx / D, k = idx - (idx / D) * D;
    const RowPos p = row_pos(sb, rj);
    const int64_t e = elem(sb, 0, p, k);
    V2<T> a0, a1;
    kick2<T>(c, s, ldst<kCG>(gamma + e), ldst<kCG>(gamma + e + sb.str_s), a0, a1);
    const T w = (T)row_weight<kCG>(sb, lam, p);
    F[(rj * 2 + 0) * D + k] = c_scale<T>(a0, w);
    F[(rj * 2 + 1) * D + k] = c_scale<T>(a1, w);
  }
}

// ---------------------------------------------------------------- unsquared bond SVD (complex128)
// The squared form above resolves Schmidt values below ~sqrt(eps) of the
// largest only approximately (rho = Psi^H Psi carries rounding of eps ||rho||).
// The complex128 path takes the SVD of a 2D x n core of Psi itself.  Writing the
// gated two-site matrix block by block in the physical index s of end a,
//   Psi_s[r_a][x] = g(s, t_x) sum_k A~_s[r_a][k] lam_k F[x][k]  (x = (row of b, t)),
// and G_s = R_s^H R_s for the Gram blocks G_s = A~_s^H A~_s of end a,
// Psi = blockdiag(Q_0, Q_1) M with M[(s, j)][x] = g(s, t_x) sum_k R_s[j][k] lam_k F[x][k]
// and Q_s isometric on the range of A~_s: Psi and M have the same singular
// values and right singular vectors.  R_s is the pivoted Cholesky factor of G_s
// (the bond's own lam enters only through M, so a pivot cut on G_s never drops a
// bond index of small lam); the SVD of M is one-sided (Hestenes) Jacobi on B = M V0, preconditioned
// by V0, the FP32 eigenvectors of M^H M re-orthonormalised in FP64, and by FP32
// levels on rescaled blocks of B^H B whose columns are small (the Gram of B is
// accurate relative to each column, unlike rho).  The Schmidt values are the
// column norms of B, accurate to eps of the largest.

constexpr double kCholCut = 1e-15;     // pivoted Cholesky stops below this fraction of the largest diagonal
constexpr double kNoiseRelSvd = 1e-30; // columns of B with |b|^2 below this fraction of ||M||_F^2 are rounding

// Global-slot layout (complex doubles) of the unsquared bond update, fixed for
// n = 2D so that every bond of a launch shares it:
//   Mt  [2D][2D]     M^T (Mt[x][s D + j]); F [n][D] again for the epilogue
//   RB  [2D][2D+1]   rho = M^H M (row stride n + 1); then B^T (Bt[j][r] = B[r][j], row stride 2D)
//   Vx  [2D][2D]     F [n][D] first; then V0 and finally V (row x, column j)
//   Xs  [2D][2D+1]   G_s [2][D][D+1] and R_s [2][D][D] first; then the FP32
//                    level's scratch; then V^T (Vt[j][x], row stride n)
struct SvdLayout {
  size_t off_Mt, off_RB, off_V, off_X, big;
  __host__ __device__ explicit SvdLayout(int D) {
    const size_t nm = (size_t)2 * D;
    off_Mt = 0;
    off_RB = off_Mt + nm * nm * 16;
    off_V = off_RB + nm * (nm + 1) * 16;
    off_X = off_V + nm * nm * 16;
    big = off_X + nm * (nm + 1) * 16;
  }
};

__host__ __device__ size_t bond_big(int D, size_t elt) {
  return elt == 16 ? SvdLayout(D).big : BondSmem(D, 2 * D).big;
}

// Pivoted Cholesky of the two Hermitian positive semi-definite D x D matrices
// G_0, G_1 (Cw, row stride D + 1, overwritten by their Schur complements), in
// outer-product form with diagonal pivoting (the semi-definite Cholesky analysed
// by Higham, 1990): step k takes the largest remaining diagonal C[p][p], row k of
// R_s is C[p][j] / sqrt(C[p][p]) on the columns j not yet pivoted (sqrt(C[p][p])
// at p, zero on the pivoted ones), and the unpivoted block is updated by
// C[i][j] -= conj(R[k][i]) R[k][j].  A factor stops when its largest remaining
// diagonal is <= kCholCut times its largest initial one (the rest is rounding);
// its remaining rows are zero, so R_s^H R_s = G_s up to that cut.  Warps 0 and 1
// choose the pivots of s = 0 and 1.  mask: 2D ints; piv: 4 ints; dk: 4 doubles.
__device__ void pivoted_cholesky2(double2* Cw, double2* Rr, int D, int* mask, int* piv, double* dk) {
  const int ldc = D + 1, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int idx = threadIdx.x; idx < 2 * D * D; idx += blockDim.x) Rr[idx] = make_double2(0.0, 0.0);
  for (int idx = threadIdx.x; idx < 2 * D; idx += blockDim.x) mask[idx] = 1;
  if (warp < 2) {
    double mx = 0.0;
    for (int i = lane; i < D; i += 32) mx = fmax(mx, Cw[(size_t)warp * D * ldc + i * ldc + i].x);
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) {
      dk[2 + warp] = mx;  // largest initial diagonal
      piv[2 + warp] = 1;  // factor still running
    }
  }
  __syncthreads();
  for (int k = 0; k < D; ++k) {
    if (warp < 2) {
      const int sidx = warp;
      const double2* C = Cw + (size_t)sidx * D * ldc;
      double best = -1.0;
      int bi = D;
      for (int i = lane; i < D; i += 32) {
        if (mask[sidx * D + i]) {
          const double d = C[i * ldc + i].x;
          if (d > best) {
            best = d;
            bi = i;
          }
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        const bool go = piv[2 + sidx] && bi < D && best > kCholCut * dk[2 + sidx] && best > 0.0;  // NaN stops
        piv[sidx] = go ? bi : -1;
        dk[sidx] = go ? best : 0.0;
        if (go) mask[sidx * D + bi] = 0;
        else piv[2 + sidx] = 0;
      }
    }
    __syncthreads();
    if (piv[0] < 0 && piv[1] < 0) break;
    for (int idx = threadIdx.x; idx < 2 * D; idx += blockDim.x) {
      const int sidx = idx / D, j = idx - (idx / D) * D, pv = piv[sidx];
      if (pv < 0) continue;
      const double r = sqrt(dk[sidx]);
      double2 v = make_double2(0.0, 0.0);
      if (j == pv) v = make_double2(r, 0.0);
      else if (mask[sidx * D + j]) v = cscale(Cw[(size_t)sidx * D * ldc + pv * ldc + j], 1.0 / r);
      Rr[(size_t)sidx * D * D + (size_t)k * D + j] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * D * D; idx += blockDim.x) {
      const int sidx = idx / (D * D), ij = idx - sidx * D * D, i = ij / D, j = ij - (ij / D) * D;
      if (piv[sidx] < 0 || !mask[sidx * D + i] || !mask[sidx * D + j]) continue;
      const double2* r = Rr + (size_t)sidx * D * D + (size_t)k * D;
      const double2 ri = r[i], rj = r[j];
      double2& c = Cw[(size_t)sidx * D * ldc + i * ldc + j];
      c.x -= ri.x * rj.x + ri.y * rj.y;
      c.y -= ri.x * rj.y - ri.y * rj.x;
    }
    __syncthreads();
  }
}

// Sum of a double over the lanes of a warp (every lane gets the total).
__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// |b_j|^2 of the n columns of B (Bt [n][rows]) into alpha, one warp per column.
__device__ void column_norms(const double2* Bt, int rows, int n, double* alpha) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < n; j += nw) {
    const double2* b = Bt + (size_t)j * rows;
    double a = 0.0;
    for (int i = lane; i < rows; i += 32) a = fma(b[i].x, b[i].x, fma(b[i].y, b[i].y, a));
    a = warp_sum(a);
    if (lane == 0) alpha[j] = a;
  }
  __syncthreads();
}

// Pair k of round r of the round-robin pairing of n indices (as jacobi_hermitian).
__device__ __forceinline__ void round_pair(int r, int k, int n, int& p, int& q) {
  if (k == 0) {
    p = r;
    q = n - 1;
  } else {
    p = r + k;
    if (p >= n - 1) p -= n - 1;
    q = r - k;
    if (q < 0) q += n - 1;
  }
}

// Rotation of a column pair in FP32 (the warm start and the levels): the same
// angle as `os_rotation`, in plain FP32 arithmetic (the FP32 stages work on
// matrices scaled to unit Frobenius norm and skip pairs with |g| below 1e-13,
// so nothing underflows).  1/|g| and c = 1/sqrt(1+t^2) get one Newton step each
// so that |e| = 1 and c^2 + s^2 = 1 to FP32 rounding: a column of a 128-wide
// solve takes ~1500 rotations, and the ~2e-7 of rsqrtf alone would leave the
// accumulated rotation ~3e-4 away from unitary.
__device__ __forceinline__ void os_rot(float a, float b, float2 g, float& c, float& s, float2& e) {
  const float g2 = fmaf(g.x, g.x, g.y * g.y);
  float ig = rsqrtf(g2);
  ig = ig * fmaf(-0.5f * g2, ig * ig, 1.5f);
  const float zeta = (b - a) * (0.5f * ig);
  const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
  const float u = fmaf(t, t, 1.f);
  float cc = rsqrtf(u);
  cc = cc * fmaf(-0.5f * u, cc * cc, 1.5f);
  c = cc;
  s = t * cc;
  e = make_float2(g.x * ig, -g.y * ig);
}
__device__ __forceinline__ void os_rot(double a, double b, double2 g, double& c, double& s, double2& e) {
  double ag;
  os_rotation(a, b, g, c, s, e, ag);
}

// One-sided (Hestenes) Jacobi on the n columns of B (Bt [n][rows]), with V^T
// (Vt [n][n]) rotated alongside, in the arithmetic of R (FP32 for the warm start
// and the levels, FP64 for the final sweeps).  A sweep runs the n - 1 rounds of
// the round-robin pairing; a round (1) forms |b_p|^2, |b_q|^2 and g = b_p^H b_q
// of its n/2 disjoint pairs from the columns themselves (8 lanes per pair), (2)
// decides and builds every rotation with one thread per pair (`os_rot`): pair
// (p, q) rotates when |g| > max(tol |b_p| |b_q|, floor_abs), by
// b_p <- c b_p - s e b_q, b_q <- s b_p + c e b_q, (3) applies the rotations of
// the active pairs only, over the rows of B and V.  Norms are never carried
// over from earlier rotations (a closed-form update loses digits when a pair is
// nearly parallel, and every later angle of that column would inherit the
// error).  A sweep without rotations ends the solve.  Returns the sweeps
// (max_sweeps + 1 = cap hit); work[0] += pair checks, work[1] += rotations,
// rot_count[sweep] += rotations of the first kRotSweeps sweeps (either may be
// null).  rc, rs: n/2 reals; re: n/2 complex; iflag: the integer scratch of
// jacobi_hermitian.  n <= 256, blockDim.x >= n/2 rounded up to 32.
template <typename R>
__device__ int one_sided_jacobi(V2<R>* Bt, int rows, V2<R>* Vt, int n, R tol, R floor_abs, int max_sweeps, R* rc,
                                R* rs, V2<R>* re, int* iflag, unsigned long long* work,
                                unsigned long long* rot_count) {
  const int m = n / 2, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int sub = lane & 7, grp = lane >> 3;
  int* act = iflag + 8;     // [4 warps][32] active pairs of the round
  int* wcnt = iflag + 136;  // active pairs per warp
  const int npw = (m + 31) >> 5;  // warps that build the rotations (n <= 256: at most 4)
  const R tol2 = tol * tol, floor2 = floor_abs * floor_abs;
  const int len = rows + n;
  unsigned long long n_chk = 0, n_rot = 0;
  int result = max_sweeps + 1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) iflag[3] = 0;
    for (int r = 0; r < n - 1; ++r) {
      // (1) norms and inner product of every pair: rc[k] = |b_p|^2, rs[k] = |b_q|^2, re[k] = g
      for (int k0 = warp * 4; k0 < m; k0 += nw * 4) {
        const int k = k0 + grp;
        R a = 0, b = 0;
        V2<R> g = mk<R>(0, 0);
        if (k < m) {
          int p, q;
          round_pair(r, k, n, p, q);
          const V2<R>* bp = Bt + (size_t)p * rows;
          const V2<R>* bq = Bt + (size_t)q * rows;
          for (int i = sub; i < rows; i += 8) {
            const V2<R> u = bp[i], v = bq[i];
            a = fma(u.x, u.x, fma(u.y, u.y, a));
            b = fma(v.x, v.x, fma(v.y, v.y, b));
            fma_conj<R>(g, u, v);
          }
        }
        for (int off = 4; off > 0; off >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, off);
          b += __shfl_xor_sync(0xffffffffu, b, off);
          g.x += __shfl_xor_sync(0xffffffffu, g.x, off);
          g.y += __shfl_xor_sync(0xffffffffu, g.y, off);
        }
        if (k < m && sub == 0) {
          rc[k] = a;
          rs[k] = b;
          re[k] = g;
        }
      }
      __syncthreads();
      // (2) one thread per pair: test, rotation (c, s, e) into rc, rs, re, compacted active list
      if (warp < npw) {
        const int k = threadIdx.x;
        bool on = false;
        if (k < m) {
          const V2<R> g = re[k];
          const R a = rc[k], b = rs[k];
          const R g2 = fma(g.x, g.x, g.y * g.y);
          on = g2 > tol2 * a * b && g2 > floor2;
          if (on) {
            R c, sn;
            V2<R> e;
            os_rot(a, b, g, c, sn, e);
            rc[k] = c;
            rs[k] = sn;
            re[k] = e;
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (on) act[warp * 32 + __popc(bal & ((1u << lane) - 1u))] = k;
        if (lane == 0) wcnt[warp] = __popc(bal);
      }
      __syncthreads();
      // prefix counts of the warps' lists (scalars: a runtime-indexed array would live in local memory)
      const int p1 = wcnt[0], p2 = p1 + (npw > 1 ? wcnt[1] : 0), p3 = p2 + (npw > 2 ? wcnt[2] : 0);
      const int na = p3 + (npw > 3 ? wcnt[3] : 0);
      if (threadIdx.x == 0) {
        iflag[3] += na;
        n_chk += (unsigned long long)m;
        n_rot += (unsigned long long)na;
      }
      if (na == 0) continue;  // nothing below reads this round's scratch
      // (3) the active rotations over the rows of B, then of V
      for (int t = threadIdx.x; t < na * len; t += blockDim.x) {
        const int ia = t / len, i = t - ia * len;
        const int k = ia < p1 ? act[ia] : ia < p2 ? act[32 + ia - p1] : ia < p3 ? act[64 + ia - p2] : act[96 + ia - p3];
        int p, q;
        round_pair(r, k, n, p, q);
        V2<R>* xp = i < rows ? Bt + (size_t)p * rows + i : Vt + (size_t)p * n + (i - rows);
        V2<R>* xq = i < rows ? Bt + (size_t)q * rows + i : Vt + (size_t)q * n + (i - rows);
        const R c = rc[k], sn = rs[k];
        const V2<R> u = *xp, v = c_mul<R>(*xq, re[k]);
        *xp = mk<R>(c * u.x - sn * v.x, c * u.y - sn * v.y);
        *xq = mk<R>(sn * u.x + c * v.x, sn * u.y + c * v.y);
      }
      __syncthreads();
    }
    const int total = iflag[3];
    if (threadIdx.x == 0 && rot_count && sweep < kRotSweeps) atomicAdd(rot_count + sweep, (unsigned long long)total);
    __syncthreads();
    if (total == 0) {
      result = sweep + 1;
      break;
    }
  }
  if (work && threadIdx.x == 0) {
    atomicAdd(work, n_chk);
    atomicAdd(work + 1, n_rot);
  }
  return result;
}

// FP32 one-sided stages: relative threshold jp.tol32 (at the rounding of an FP32 dot product) and
// this absolute one, in units of the largest squared column norm
constexpr float kOsFloor32 = 1e-13f;

// Shared scratch (bytes) after the small arrays of the unsquared bond update:
// the FP32 warm start's B32 [n][2D] and V^T32 [n][n] (complex float) when D <= 32
// (beyond, they use the global slot), and the FP32 levels' block of at most
// lv = min(D, kMaxLevel) columns: B32 [lv][2D], W^T32 [lv][lv] (complex float),
// W64 [lv][lv] and Gw [lv][lv+1] (complex double).
__host__ __device__ size_t svd_level_w64_off(int cap, int rows) {
  return ((size_t)cap * rows * 8 + (size_t)cap * cap * 8 + 15) & ~(size_t)15;
}
__host__ __device__ size_t svd_f32_bytes(int D) {
  const size_t n = (size_t)2 * D, lv = D < kMaxLevel ? (size_t)D : (size_t)kMaxLevel;
  const size_t lvl = svd_level_w64_off((int)lv, (int)n) + lv * lv * 16 + lv * (lv + 1) * 16;
  const size_t warm = D <= 32 ? 2 * n * n * 8 : 0;
  return lvl > warm ? lvl : warm;
}

// FP32 levels on the small columns of B: the columns whose squared norms lie
// below jp.level_ratio x the scale of the last block that held them (the
// largest column at first) and above rounding (kNoiseRelSvd of ||M||_F^2); the
// largest ns <= lv of them form one block.  The block is copied to FP32, scaled
// by the power of two that brings its largest column to norm ~1; FP32 one-sided
// Jacobi makes those columns orthogonal to FP32 accuracy relative to each
// column; the accumulated rotation W, re-orthonormalised in FP64, rotates those
// columns of B and of V in FP64.  Meant to run after an FP64 sweep, which has
// removed from the small columns their components along the large ones (else
// the block would be their contamination).  lvl: as svd_f32_bytes.
__device__ void svd_levels(double2* Bt, int rows, double2* Vt, int n, double tr, const JacobiParams& jp,
                           double* alpha, double* rscale, int* mark_c, int* cand, double* scal, float2* re32,
                           float* rc32, float* rs32, int* iflag, unsigned char* lvl, unsigned long long* sweeps_out) {
  const int cap = (n / 2 < kMaxLevel) ? n / 2 : kMaxLevel;
  float2* B32 = reinterpret_cast<float2*>(lvl);                                // [cap][rows]
  float2* W32 = B32 + (size_t)cap * rows;                                      // [cap][cap], W^T
  double2* W64 = reinterpret_cast<double2*>(lvl + svd_level_w64_off(cap, rows));  // [cap][cap]
  double2* Gw = W64 + (size_t)cap * cap;                                       // [cap][cap+1]
  const double lo = kNoiseRelSvd * tr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int level = 0; level < jp.levels; ++level) {
    column_norms(Bt, rows, n, alpha);
    if (level == 0) {
      if (threadIdx.x == 0) {
        double s0 = 0.0;
        for (int i = 0; i < n; ++i) s0 = fmax(s0, alpha[i]);
        scal[3] = s0;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) rscale[i] = scal[3];
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      mark_c[i] = (alpha[i] > lo && alpha[i] <= jp.level_ratio * rscale[i]) ? 1 : 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (!mark_c[i]) continue;
      const double ai = alpha[i];
      int rank = 0;
      for (int j = 0; j < n; ++j) rank += mark_c[j] && (alpha[j] > ai || (alpha[j] == ai && j < i));
      if (rank < cap) cand[rank] = i;
    }
    if (threadIdx.x == 0) {
      int cnt = 0;
      for (int j = 0; j < n; ++j) cnt += mark_c[j];
      iflag[1] = (cnt < cap ? cnt : cap) & ~1;  // even: the round-robin pairing needs it
    }
    __syncthreads();
    if (threadIdx.x == 0) scal[7] = iflag[1] > 0 ? alpha[cand[0]] : 0.0;
    __syncthreads();
    const int ns = iflag[1];
    const double bscale = scal[7];
    if (ns < 2 || !(bscale > 0.0)) break;
    int ex;
    frexp(bscale, &ex);
    const double sc = ldexp(1.0, -(ex >> 1));  // the block's largest squared norm -> [1/2, 2)
    for (int idx = threadIdx.x; idx < ns * rows; idx += blockDim.x) {
      const int a = idx / rows, r = idx - (idx / rows) * rows;
      const double2 v = Bt[(size_t)cand[a] * rows + r];
      B32[idx] = make_float2((float)(v.x * sc), (float)(v.y * sc));
    }
    for (int idx = threadIdx.x; idx < ns * ns; idx += blockDim.x)
      W32[idx] = make_float2((idx / ns) == (idx % ns) ? 1.f : 0.f, 0.f);
    __syncthreads();
    one_sided_jacobi<float>(B32, rows, W32, ns, (float)jp.tol32, kOsFloor32, jp.max_sweeps32, rc32, rs32, re32,
                            iflag, sweeps_out + 6, nullptr);
    for (int idx = threadIdx.x; idx < ns * ns; idx += blockDim.x) {
      const int a = idx / ns, b = idx - (idx / ns) * ns;
      const float2 v = W32[(size_t)b * ns + a];
      W64[idx] = make_double2((double)v.x, (double)v.y);
    }
    __syncthreads();
    orthonormalise<false>(W64, ns, Gw, ns + 1, alpha, scal);
    // rows of B (r < rows) and of V (x < n): new column cand[b] = sum_a old column cand[a] W[a][b]
    for (int rr = warp; rr < rows + n; rr += nw) {
      double2* base = rr < rows ? Bt + rr : Vt + (rr - rows);
      const int ld = rr < rows ? rows : n;
      double2 out = make_double2(0.0, 0.0);
      if (lane < ns)
        for (int a = 0; a < ns; ++a) fma_c<double>(out, base[(size_t)cand[a] * ld], W64[a * ns + lane]);
      __syncwarp();
      if (lane < ns) base[(size_t)cand[lane] * ld] = out;
      __syncwarp();
    }
    for (int a = threadIdx.x; a < ns; a += blockDim.x) rscale[cand[a]] = bscale;
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicAdd(sweeps_out + 2, 1ull);
      const unsigned long long nsl = (unsigned long long)ns;
      atomicAdd(sweeps_out + 3, (unsigned long long)(rows + n) * nsl * nsl + 4ull * nsl * nsl * nsl / 3ull);
    }
  }
}

// Front half of the unsquared bond update (complex128): from the Gram blocks of
// end a (FP64 sums in gsum, or this bond's partials) and end b, the right
// singular vectors V (Vm [n][n], row x, column j) and squared singular values
// (ev[j]) of the gated two-site matrix.  Returns false when M vanishes or is not
// finite (the bond is then left unchanged by the caller).  lvl: the level
// scratch in shared memory.
template <bool kCG>
__device__ bool bond_front_svd(const BondDesc& bd, const double2* __restrict__ partials, const double2* gsum,
                               const double2* gamma, const double* lam, double th_b, int D, const JacobiParams& jp,
                               unsigned char* big, double* lamo, double* ev, double* rc, double* rs, double2* re,
                               double* scal, float2* re32, float* rc32, float* rs32, int* order, int* rp, int* rq,
                               int* iflag,
                               unsigned char* lvl, unsigned long long* sweeps_out, unsigned long long* cycles,
                               int* flags, long long& t_prev, double2** Vm_out) {
  const SideDesc& sb = bd.b;
  const int n = 2 * sb.rows, rows = 2 * D, D2 = D * D, ldr = n + 1;
  const SvdLayout L(D);
  double2* Mt = reinterpret_cast<double2*>(big + L.off_Mt);
  double2* RB = reinterpret_cast<double2*>(big + L.off_RB);
  double2* Vx = reinterpret_cast<double2*>(big + L.off_V);
  double2* Xs = reinterpret_cast<double2*>(big + L.off_X);
  double2* Cw = Xs;                        // [2][D][D+1] Gram blocks G_s of end a
  double2* Rr = Xs + (size_t)2 * D * (D + 1);  // [2][D][D]
  double2* F = Vx;                         // [n][D]
  int* mask = reinterpret_cast<int*>(Mt);  // [2][D] while the factors run
  auto mark = [&](int phase) {
    if (threadIdx.x == 0) {
      const long long t = clock64();
      atomicAdd(cycles + phase, (unsigned long long)(t - t_prev));
      t_prev = t;
    }
  };
  // G_s, FP64
  for (int o = threadIdx.x; o < 2 * D2; o += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    if (gsum) {
      acc = gsum[o];
    } else {
      for (int p = 0; p < bd.n_parts; ++p) {
        const double2 v = partials[(int64_t)p * 2 * D2 + o];
        acc.x += v.x;
        acc.y += v.y;
      }
    }
    const int sidx = o / D2, kl = o - sidx * D2, k = kl / D, l = kl - (kl / D) * D;
    Cw[(size_t)sidx * D * (D + 1) + k * (D + 1) + l] = acc;
  }
  load_F<double, kCG>(sb, gamma, lam, th_b, F, D);
  __syncthreads();
  pivoted_cholesky2(Cw, Rr, D, mask, iflag + 8, scal + 4);
  // M^T[x][s D + j] = g(s, t_x) sum_k R_s[j][k] lam_k F[x][k], g(s, t) = (1 + i sign) / sqrt 2 for
  // s = t, (1 - i sign) / sqrt 2 otherwise (sign = gate_sign: exp(+-i pi/4 z_s z_t))
  const double r2 = 0.70710678118654752440;
  for (int idx = threadIdx.x; idx < n * rows; idx += blockDim.x) {
    const int x = idx / rows, r = idx - (idx / rows) * rows, sidx = r / D, j = r - (r / D) * D;
    const double2* Rj = Rr + (size_t)sidx * D2 + (size_t)j * D;
    const double2* Fx = F + (size_t)x * D;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < D; ++k) fma_c<double>(acc, Rj[k], cscale(Fx[k], lamo[k]));
    const double gi = ((sidx == (x & 1)) == (jp.gate_sign > 0)) ? r2 : -r2;
    Mt[idx] = make_double2(r2 * acc.x - gi * acc.y, r2 * acc.y + gi * acc.x);
  }
  __syncthreads();
  // ||M||_F^2
  {
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < n * rows; idx += blockDim.x)
      acc = fma(Mt[idx].x, Mt[idx].x, fma(Mt[idx].y, Mt[idx].y, acc));
    acc = warp_sum(acc);
    if (threadIdx.x == 0) scal[0] = 0.0;
    __syncthreads();
    if (lane == 0) atomicAdd(scal, acc);
    __syncthreads();
  }
  const double trace = scal[0];
  if (!(trace > 0.0) || !isfinite(trace)) return false;
  mark(0);
  // FP32 one-sided warm start on M scaled by the power of two that brings ||M||_F
  // to ~1: its rotations leave a column of Schmidt value s_j at a cosine of
  // ~1e-7 s_max / s_j against the others (the eigenvectors of the squared M^H M
  // in FP32 would leave ~1e-7 (s_max / s_j)^3).  B32 [n][2D] and V^T32 [n][n] in
  // shared memory up to D = 32, else over the free rho and scratch regions.
  float2* B32 = D <= 32 ? reinterpret_cast<float2*>(lvl) : reinterpret_cast<float2*>(RB);
  float2* Vt32 = D <= 32 ? B32 + (size_t)n * rows : reinterpret_cast<float2*>(Xs);
  {
    int ex;
    frexp(trace, &ex);
    const double sc = ldexp(1.0, -(ex >> 1));
    for (int idx = threadIdx.x; idx < n * rows; idx += blockDim.x)
      B32[idx] = make_float2((float)(Mt[idx].x * sc), (float)(Mt[idx].y * sc));
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x)
      Vt32[idx] = make_float2((idx / n) == (idx % n) ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  const int sw32 = one_sided_jacobi<float>(B32, rows, Vt32, n, (float)jp.tol32, kOsFloor32, jp.max_sweeps32, rc32,
                                           rs32, re32, iflag, sweeps_out + 6, cycles ? cycles + kPhases : nullptr);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int x = idx / n, j = idx - (idx / n) * n;
    const float2 v = Vt32[(size_t)j * n + x];
    Vx[idx] = make_double2((double)v.x, (double)v.y);
  }
  __syncthreads();
  mark(1);
  {
    // The series of `orthonormalise` is exact to O(|E|^3), below 1e-12 for the
    // |E| ~ 2e-5 that the FP32 warm start leaves at n = 64 (~400 rotations per
    // column; measured <Z> parity 3e-14).  A wide solve drifts further (n = 256:
    // ~2500 rotations per column leave |E| ~ 1e-4), so from 1e-4 on a second
    // pass, which starts from ~|E|^3, finishes the job; a basis beyond the
    // series' range is flagged.
    const double emax = orthonormalise<false>(Vx, n, Xs, ldr, ev, scal);
    const double emax2 = emax > 1e-4 ? orthonormalise<false>(Vx, n, Xs, ldr, ev, scal) : 0.0;
    if (threadIdx.x == 0 && (!(emax < 1e-2) || !(emax2 < 1e-8))) atomicOr(flags, 1);
  }
  mark(2);
  // B = M V0 (Bt[j][r] = sum_x V0[x][j] M[r][x]) and V^T, over the free regions
  double2* Bt = RB;
  double2* Vt = Xs;
  for (int idx = threadIdx.x; idx < n * rows; idx += blockDim.x) {
    const int j = idx / rows, r = idx - (idx / rows) * rows;
    double2 acc = make_double2(0.0, 0.0);
    for (int x = 0; x < n; ++x) fma_c<double>(acc, Vx[(size_t)x * n + j], Mt[(size_t)x * rows + r]);
    Bt[idx] = acc;
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int j = idx / n, x = idx - (idx / n) * n;
    Vt[idx] = Vx[(size_t)x * n + j];
  }
  __syncthreads();
  // One FP64 sweep first: it converges the pairs of large columns and removes
  // from the small columns their FP32-level components along the large ones
  // (~1e-7 of the largest Schmidt value, which can exceed a small column's own
  // size).  Only then are the small columns a clean block for the FP32 levels,
  // whose rotations leave the last sweeps little to do.
  unsigned long long* rot = cycles ? cycles + kPhases + kRotSweeps : nullptr;
  const int sw1 = one_sided_jacobi(Bt, rows, Vt, n, jp.tol, jp.floor_rel * trace, 1, rc, rs, re, iflag,
                                   sweeps_out + 4, rot);
  mark(4);
  // level marks in rp/rq (n ints, free until a level's Jacobi), candidates in order
  svd_levels(Bt, rows, Vt, n, trace, jp, ev, rc, rp, order, scal, re32, rc32, rs32, iflag, lvl, sweeps_out);
  mark(3);
  const int sweeps = sw1 == 1 ? 1
                              : 1 + one_sided_jacobi(Bt, rows, Vt, n, jp.tol, jp.floor_rel * trace, jp.max_sweeps - 1,
                                                     rc, rs, re, iflag, sweeps_out + 4, rot ? rot + 1 : nullptr);
  mark(4);
  if (threadIdx.x == 0) {
    if (sweeps > jp.max_sweeps) atomicOr(flags, 1);
    atomicAdd(sweeps_out, (unsigned long long)(sweeps > jp.max_sweeps ? jp.max_sweeps : sweeps));
    atomicAdd(sweeps_out + 1, (unsigned long long)(sw32 > jp.max_sweeps32 ? jp.max_sweeps32 : sw32));
  }
  // squared singular values (the column norms of B) and V back in row-major order
  column_norms(Bt, rows, n, ev);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int x = idx / n, j = idx - (idx / n) * n;
    Vx[idx] = Vt[(size_t)j * n + x];
  }
  __syncthreads();
  *Vm_out = Vx;
  return true;
}

// Bond eigenproblem: rho (FP64), eigenvectors by FP32 Jacobi to convergence
// (the FP32 pipe is 64x the FP64 pipe on this part), FP64 Cholesky-QR of the
// FP32 eigenvectors, rho' = V^dagger rho V and FP64 Jacobi sweeps on rho' until
// every off-diagonal is at FP64 rounding level (mixed-precision Jacobi: a
// low-precision eigenbasis as preconditioner of the high-precision sweeps).
// The Gram blocks of end a come either as bd.n_parts storage-precision
// partials (partials: this bond's first) summed here in FP64, or already summed
// (gsum, FP64).  Outputs: Y (2 D^2, this bond's), *theta_a (the kick of end a,
// consumed), vs (sorted eigenpairs for the reverse mode, or null), the new
// Gamma_b and lambda of the bond.
template <typename T, bool kCG>
__device__ void bond_body(const BondDesc bd, const V2<T>* __restrict__ partials, const double2* gsum, V2<T>* gamma,
                          double* lam, double* pending, V2<T>* __restrict__ Y, double* __restrict__ theta_a,
                          int* flags, unsigned long long* sweeps_out, unsigned long long* cycles, double2* vs, int D,
                          JacobiParams jp, unsigned char* big) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SideDesc sb = bd.b;
  const int nb = sb.rows;
  const int n = 2 * nb;
  const int D2 = D * D;
  const BondSmem L(D, n);
  unsigned char* bigp = big ? big : smem_raw;                   // R, Vr, X
  unsigned char* smallp = big ? smem_raw : smem_raw + L.big;   // the small arrays
  double2* RHO = reinterpret_cast<double2*>(bigp + L.off_R);  // [n][n+1]
  double2* Vr = reinterpret_cast<double2*>(bigp + L.off_V);
  double2* X = reinterpret_cast<double2*>(bigp + L.off_X);
  V2<T>* Cs = reinterpret_cast<V2<T>*>(Vr);  // [2][D][D], storage precision
  V2<T>* H = Cs + 2 * D2;                     // [n][D]
  double2* Vm = Vr;                           // [n][n]
  V2<T>* F = reinterpret_cast<V2<T>*>(X);     // [n][D]
  double2* re = reinterpret_cast<double2*>(smallp + L.off_re);
  float2* re32 = reinterpret_cast<float2*>(smallp + L.off_re32);
  double* lamo = reinterpret_cast<double*>(smallp + L.off_lamo);
  double* ev = reinterpret_cast<double*>(smallp + L.off_ev);
  double* sv = reinterpret_cast<double*>(smallp + L.off_sv);
  double* rc = reinterpret_cast<double*>(smallp + L.off_rc);
  double* rs = reinterpret_cast<double*>(smallp + L.off_rs);
  double* scal = reinterpret_cast<double*>(smallp + L.off_scal);  // [0] trace [1] norm [2] max lambda_o [4] tmp
  float* rc32 = reinterpret_cast<float*>(smallp + L.off_rc32);
  float* rs32 = reinterpret_cast<float*>(smallp + L.off_rs32);
  int* order = reinterpret_cast<int*>(smallp + L.off_int);
  int* rp = order + n;
  int* rq = rp + n / 2;
  int* iflag = rq + n / 2;  // [4]
  const int ldr = n + 1;
  const double th_b = ldst<kCG>(pending + sb.site);
  long long t_prev = clock64();
  auto mark = [&](int phase) {
    if (threadIdx.x == 0) {
      const long long t = clock64();
      atomicAdd(cycles + phase, (unsigned long long)(t - t_prev));
      t_prev = t;
    }
  };

  for (int k = threadIdx.x; k < D; k += blockDim.x) lamo[k] = ldst<kCG>(lam + bd.lam_e + k);
  __syncthreads();
  if constexpr (sizeof(T) == 8) {
    // complex128: the unsquared SVD of the bond core, in the CTA's global slot
    // (every launcher passes one for this dtype)
    if (!big || !bond_front_svd<kCG>(bd, partials, gsum, gamma, lam, th_b, D, jp, big, lamo, ev, rc, rs, re, scal,
                                     re32, rc32, rs32, order, rp, rq, iflag, smallp + L.small, sweeps_out, cycles,
                                     flags, t_prev, &Vm)) {
      bond_fail<T, kCG>(bd, Y, theta_a, pending, flags, D);
      return;
    }
    F = reinterpret_cast<V2<T>*>(big + SvdLayout(D).off_Mt);
    __syncthreads();
  } else {
    for (int o = threadIdx.x; o < 2 * D2; o += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      if (gsum) {
        acc = gsum[o];
      } else {
        for (int p = 0; p < bd.n_parts; ++p) {
          const V2<T> v = partials[(int64_t)p * 2 * D2 + o];
          acc.x += (double)v.x;
          acc.y += (double)v.y;
        }
      }
      const int kl = o % D2;
      const int k = kl / D, l = kl - (kl / D) * D;
      const double2 v = cscale(acc, lamo[k] * lamo[l]);
      Cs[o] = mk<T>((T)v.x, (T)v.y);
    }
    load_F<T, kCG>(sb, gamma, lam, th_b, F, D);
    for (int idx = threadIdx.x; idx < n * ldr; idx += blockDim.x) RHO[idx] = make_double2(0.0, 0.0);
    __syncthreads();
    // rho = sum_s phase(s) o (conj(F) C_s F^T), upper triangle, then mirrored;
    // products in the storage precision (the inputs carry no more), sum in FP64
    for (int sidx = 0; sidx < 2; ++sidx) {
      const V2<T>* C = Cs + sidx * D2;
      for (int idx = threadIdx.x; idx < n * D; idx += blockDim.x) {
        const int x = idx / D, l = idx - (idx / D) * D;
        V2<T> acc = mk<T>(0, 0);
        for (int k = 0; k < D; ++k) fma_conj<T>(acc, F[x * D + k], C[k * D + l]);
        H[x * D + l] = acc;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < n * (n + 1) / 2; idx += blockDim.x) {
        int x, y;
        upper_index(idx, n, x, y);
        V2<T> acc = mk<T>(0, 0);
        for (int l = 0; l < D; ++l) fma_c<T>(acc, H[x * D + l], F[y * D + l]);
        const int tx = x & 1, ty = y & 1;
        double2 v;
        if (tx == ty) {
          v = make_double2((double)acc.x, (double)acc.y);
        } else if ((sidx == ty) == (jp.gate_sign > 0)) {  // +i (the conjugate gate swaps +i and -i)
          v = make_double2(-(double)acc.y, (double)acc.x);
        } else {  // -i
          v = make_double2((double)acc.y, -(double)acc.x);
        }
        RHO[x * ldr + y] = cadd(RHO[x * ldr + y], v);
      }
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int x = idx / n, y = idx - (idx / n) * n;
      if (y > x) RHO[y * ldr + x] = cconj(RHO[x * ldr + y]);
      if (y == x) RHO[x * ldr + x].y = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0.0;
      for (int i = 0; i < n; ++i) tr += RHO[i * ldr + i].x;
      scal[0] = tr;
    }
    __syncthreads();
    const double trace = scal[0];
    if (!(trace > 0.0) || !isfinite(trace)) {
      bond_fail<T, kCG>(bd, Y, theta_a, pending, flags, D);
      return;
    }
    mark(0);
    eig_mixed(RHO, Vm, X, n, D, trace, jp, re, re32, ev, rc, rs, scal, rc32, rs32, order, rp, rq, iflag, sweeps_out,
              cycles, flags, t_prev, big ? reinterpret_cast<float2*>(smallp + L.small) : nullptr);
    // eigenvalues sorted in decreasing order (ties by index)
    for (int i = threadIdx.x; i < n; i += blockDim.x) ev[i] = RHO[i * ldr + i].x;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int rank = 0;
    const double vi = ev[i];
    for (int j = 0; j < n; ++j) rank += (ev[j] > vi) || (ev[j] == vi && j < i);
    order[rank] = i;
  }
  __syncthreads();
  if (vs) {  // sorted eigenvectors and eigenvalues for the reverse mode (slot of 2D x 2D + 2D)
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int x = idx / n, j = idx - (idx / n) * n;
      vs[x * n + j] = Vm[x * n + order[j]];
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) vs[n * n + j] = make_double2(ev[order[j]], 0.0);
  }
  const int keep = n < D ? n : D;
  if (threadIdx.x == 0) {
    const double emax = ev[order[0]];
    double nrm2 = 0.0;
    for (int kk = 0; kk < D; ++kk) {
      double sval = 0.0;
      if (kk < keep) {
        const double e = ev[order[kk]];
        if (e > jp.ev_cut * emax && e > 0.0) sval = sqrt(e);
      }
      sv[kk] = sval;
      nrm2 += sval * sval;
    }
    scal[1] = sqrt(nrm2);
    double mx = 0.0;
    const int lo = sb.lam_o1 >= 0 ? sb.lam_o1 : sb.lam_o2;
    if (lo >= 0)
      for (int k = 0; k < D; ++k) mx = fmax(mx, ldst<kCG>(lam + lo + k));
    scal[2] = mx;
  }
  load_F<T, kCG>(sb, gamma, lam, th_b, F, D);
  __syncthreads();
  const double nrm = scal[1];
  if (!(nrm > 0.0) || !isfinite(nrm)) {
    bond_fail<T, kCG>(bd, Y, theta_a, pending, flags, D);
    return;
  }
  // Y_s[k][kk] = lam_k sum_x F[x][k] g(s, t_x) V[x][order[kk]] / sv[kk], in the
  // storage precision (Y feeds the storage-precision update of end a).  In FP32
  // the kept eigenvectors are rounded once into Vk [n][D], after F in X.
  V2<T>* Vk = F + (size_t)n * D;
  if constexpr (sizeof(T) == 4) {
    for (int idx = threadIdx.x; idx < n * D; idx += blockDim.x) {
      const int x = idx / D, kk = idx - (idx / D) * D;
      V2<T> v = mk<T>(0, 0);
      if (sv[kk] > 0.0) {
        const double2 vd = Vm[x * n + order[kk]];
        v = mk<T>((T)vd.x, (T)vd.y);
      }
      Vk[idx] = v;
    }
    __syncthreads();
  }
  const T r2 = (T)0.70710678118654752440;
  for (int o = threadIdx.x; o < 2 * D2; o += blockDim.x) {
    const int sidx = o / D2;
    const int kl = o - sidx * D2;
    const int k = kl / D, kk = kl - (kl / D) * D;
    V2<T> acc = mk<T>(0, 0);
    if (sv[kk] > 0.0) {
      const int col = order[kk];
      for (int x = 0; x < n; ++x) {
        const V2<T> fv = F[x * D + k];
        const V2<T> g = mk<T>(r2, ((sidx == (x & 1)) == (jp.gate_sign > 0)) ? r2 : -r2);
        V2<T> vv;
        if constexpr (sizeof(T) == 4) {
          vv = Vk[x * D + kk];
        } else {
          const double2 vd = Vm[x * n + col];
          vv = mk<T>((T)vd.x, (T)vd.y);
        }
        fma_c<T>(acc, c_mul<T>(fv, g), vv);
      }
      acc = c_scale<T>(acc, (T)(lamo[k] / sv[kk]));
    }
    Y[o] = acc;
  }
  // Gamma_b'[t][row][kk] = conj(V[(row, t)][order[kk]]) / lambda_other(row)
  {
    const double mx = scal[2];
    for (int idx = threadIdx.x; idx < n * D; idx += blockDim.x) {
      const int x = idx / D, kk = idx - (idx / D) * D;
      const int rj = x >> 1, t = x & 1;
      const RowPos p = row_pos(sb, rj);
      double winv = 1.0;
      const int lo = sb.lam_o1 >= 0 ? sb.lam_o1 : sb.lam_o2;
      if (lo >= 0) {
        const double lv = ldst<kCG>(lam + lo + (sb.lam_o1 >= 0 ? p.r1 : p.r2));
        winv = lv > kLambdaCut * mx ? 1.0 / lv : 0.0;
      }
      double2 v = make_double2(0.0, 0.0);
      if (sv[kk] > 0.0) v = cscale(cconj(Vm[x * n + order[kk]]), winv);
      gamma[elem(sb, t, p, kk)] = mk<T>((T)v.x, (T)v.y);
    }
  }
  __syncthreads();
  // new lambda of the bond; kick angles consumed
  for (int kk = threadIdx.x; kk < D; kk += blockDim.x) lam[bd.lam_e + kk] = sv[kk] / nrm;
  if (threadIdx.x == 0) {
    *theta_a = ldst<kCG>(pending + bd.a.site);
    pending[bd.a.site] = 0.0;
    pending[sb.site] = 0.0;
  }
  mark(5);
}

template <typename T>
__device__ __forceinline__ void bond_body_layered(int bi, const BondDesc* __restrict__ bonds,
                                                  const V2<T>* __restrict__ partials, V2<T>* gamma, double* lam,
                                                  double* pending, V2<T>* __restrict__ Yout,
                                                  double* __restrict__ theta_a, int* flags,
                                                  unsigned long long* sweeps_out, unsigned long long* cycles,
                                                  double2* vsave, int D, JacobiParams jp, unsigned char* big) {
  const BondDesc bd = bonds[bi];
  const int D2 = D * D, nm = 2 * D;
  bond_body<T, false>(bd, partials + (int64_t)bd.part0 * 2 * D2, nullptr, gamma, lam, pending,
                      Yout + (int64_t)bi * 2 * D2, theta_a + bi, flags, sweeps_out, cycles,
                      vsave ? vsave + (int64_t)bi * (nm * nm + nm) : nullptr, D, jp, big);
}

// One CTA per bond.  `scratch` (null when everything fits in shared memory):
// one slot of `slot` bytes per CTA for the big part of the layout.
template <typename T>
__global__ void __launch_bounds__(kBondThreads, 1)
    bond_kernel(const BondDesc* __restrict__ bonds, const V2<T>* __restrict__ partials, V2<T>* gamma, double* lam,
                double* pending, V2<T>* __restrict__ Yout, double* __restrict__ theta_a, int* flags,
                unsigned long long* sweeps_out, unsigned long long* cycles, double2* vsave, int D, JacobiParams jp,
                unsigned char* scratch, size_t slot) {
  bond_body_layered<T>(blockIdx.x, bonds, partials, gamma, lam, pending, Yout, theta_a, flags, sweeps_out, cycles,
                       vsave, D, jp, scratch ? scratch + (size_t)blockIdx.x * slot : nullptr);
}

// Persistent form: kMinB CTAs per SM take bonds from a work queue (bonds are
// ordered by decreasing size, so the large ones go first and the small ones
// fill the tail).  The queue counter is zeroed before every launch.
template <typename T, int kThr, int kMinB>
__global__ void __launch_bounds__(kThr, kMinB)
    bond_kernel_persistent(int n_bonds, unsigned int* queue, const BondDesc* __restrict__ bonds,
                           const V2<T>* __restrict__ partials, V2<T>* gamma, double* lam, double* pending,
                           V2<T>* __restrict__ Yout, double* __restrict__ theta_a, int* flags,
                           unsigned long long* sweeps_out, unsigned long long* cycles, double2* vsave, int D,
                           JacobiParams jp, unsigned char* scratch, size_t slot) {
  __shared__ int next;
  unsigned char* big = scratch ? scratch + (size_t)blockIdx.x * slot : nullptr;
  for (;;) {
    if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int bi = next;
    __syncthreads();
    if (bi >= n_bonds) break;
    bond_body_layered<T>(bi, bonds, partials, gamma, lam, pending, Yout, theta_a, flags, sweeps_out, cycles, vsave,
                         D, jp, big);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- fused step
// Every bond update of one Trotter step in one persistent launch.  The tasks
// are ordered colour by colour; a CTA takes the next one from the queue and
// waits until the earlier tasks on both of its sites are done (they were taken
// before it by running CTAs, so the wait ends), then runs, for end a, the Gram
// pass of the gram launch (same per-tile arithmetic, summed in FP64 in tile
// order as the bond launch sums the partials), the bond eigenproblem, and the
// update pass of the update launch.  So the results equal those of the layered
// launches bit for bit, and a colour class needs no barrier: its tail overlaps
// the next class.

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: wait (bounded) until task d is done; a wait that gives up raises
// GPEPS_FLAG_TIMEOUT and lets the task run on what it finds.
__device__ void wait_done(const int* done, int d, int* flags, long long limit) {
  if (d < 0) return;
  const long long t0 = clock64();
  while (ld_acquire(done + d) == 0) {
    if (clock64() - t0 >= limit) {
      atomicOr(flags, 4);
      return;
    }
    __nanosleep(256);
  }
}

template <typename T>
__device__ void fused_gram(const SideDesc& sa, const V2<T>* gamma, const double* lam, double th, double2* gsum, int D,
                           unsigned char* sm) {
  V2<T>* A = reinterpret_cast<V2<T>*>(sm);  // [nrows][2D+1]
  const int ld = 2 * D + 1;
  const int D2 = D * D, nout = 2 * D2;
  const T c = (T)cos(0.5 * th), s = (T)sin(0.5 * th);
  for (int o = threadIdx.x; o < nout; o += blockDim.x) gsum[o] = make_double2(0.0, 0.0);
  const int tr = tile_rows(D, sizeof(V2<T>));
  const int ntiles = (sa.rows + tr - 1) / tr;
  for (int tp = 0; tp < ntiles; ++tp) {
    const int row0 = tp * tr;
    const int nrows = sa.rows - row0 < tr ? sa.rows - row0 : tr;
    const int nel = nrows * D;
    for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
      int r, k;
      if (sa.str_k == 1) {
        r = idx / D;
        k = idx - r * D;
      } else {
        k = idx / nrows;
        r = idx - k * nrows;
      }
      const RowPos p = row_pos(sa, row0 + r);
      const int64_t e = elem(sa, 0, p, k);
      const T w = (T)row_weight<true>(sa, lam, p);
      V2<T> a0, a1;
      kick2<T>(c, s, __ldcg(gamma + e), __ldcg(gamma + e + sa.str_s), a0, a1);
      A[r * ld + k] = mk<T>(a0.x * w, a0.y * w);
      A[r * ld + D + k] = mk<T>(a1.x * w, a1.y * w);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
      const int sidx = o / D2;
      const int kl = o - sidx * D2;
      const int k = kl / D;
      const int l = kl - k * D;
      const V2<T>* ck = A + sidx * D + k;
      const V2<T>* cl = A + sidx * D + l;
      V2<T> acc = mk<T>(0, 0);
      for (int r = 0; r < nrows; ++r) fma_conj<T>(acc, ck[r * ld], cl[r * ld]);
      double2 g = gsum[o];
      g.x += (double)acc.x;
      g.y += (double)acc.y;
      gsum[o] = g;
    }
    __syncthreads();
  }
}

template <typename T>
__device__ void fused_update(const SideDesc& sa, V2<T>* gamma, const double* lam, const V2<T>* Y, double th, int D,
                             unsigned char* sm) {
  __shared__ double cut[2];
  const int D2 = D * D, yc = y_cols(D), tr = tile_rows(D, sizeof(V2<T>));
  V2<T>* Ys = reinterpret_cast<V2<T>*>(sm);  // [D][yc]
  V2<T>* A = Ys + (size_t)D * yc;
  const size_t a_elems_r = (size_t)tr * (2 * D + 1), a_elems_c = (size_t)(2 * D) * (tr + 1);
  float* mask = reinterpret_cast<float*>(A + (a_elems_r > a_elems_c ? a_elems_r : a_elems_c));
  const bool kfast = sa.str_k == 1;
  if (threadIdx.x < 2) {
    const int lo = threadIdx.x == 0 ? sa.lam_o1 : sa.lam_o2;
    double mx = 0.0;
    if (lo >= 0)
      for (int k = 0; k < D; ++k) mx = fmax(mx, __ldcg(lam + lo + k));
    cut[threadIdx.x] = kLambdaCut * mx;
  }
  const T c = (T)cos(0.5 * th), s = (T)sin(0.5 * th);
  const int ntiles = (sa.rows + tr - 1) / tr;
  for (int tp = 0; tp < ntiles; ++tp) {
    const int row0 = tp * tr;
    const int nrows = sa.rows - row0 < tr ? sa.rows - row0 : tr;
    const int ldr = 2 * D + 1, ldc = nrows + 1;
    const int nel = nrows * D;
    for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
      int r, k;
      if (kfast) {
        r = idx / D;
        k = idx - r * D;
      } else {
        k = idx / nrows;
        r = idx - k * nrows;
      }
      const RowPos p = row_pos(sa, row0 + r);
      const int64_t e = elem(sa, 0, p, k);
      V2<T> a0, a1;
      kick2<T>(c, s, __ldcg(gamma + e), __ldcg(gamma + e + sa.str_s), a0, a1);
      if (kfast) {
        A[r * ldr + k] = a0;
        A[r * ldr + D + k] = a1;
      } else {
        A[k * ldc + r] = a0;
        A[(D + k) * ldc + r] = a1;
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
      const RowPos p = row_pos(sa, row0 + r);
      bool ok = true;
      if (sa.lam_o1 >= 0) ok = ok && __ldcg(lam + sa.lam_o1 + p.r1) > cut[0];
      if (sa.lam_o2 >= 0) ok = ok && __ldcg(lam + sa.lam_o2 + p.r2) > cut[1];
      mask[r] = ok ? 1.f : 0.f;
    }
    const int nout = nrows * yc;
    for (int sidx = 0; sidx < 2; ++sidx) {
      for (int kb = 0; kb < D; kb += yc) {
        for (int o = threadIdx.x; o < D * yc; o += blockDim.x) {
          const int k = o / yc, cc = o - (o / yc) * yc;
          Ys[o] = Y[sidx * D2 + k * D + kb + cc];
        }
        __syncthreads();
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
          int r, kc;
          if (kfast) {
            r = o / yc;
            kc = o - r * yc;
          } else {
            kc = o / nrows;
            r = o - kc * nrows;
          }
          V2<T> acc = mk<T>(0, 0);
          const V2<T>* Yc = Ys + kc;
          if (kfast) {
            const V2<T>* Ar = A + r * ldr + sidx * D;
            for (int k = 0; k < D; ++k) fma_c<T>(acc, Ar[k], Yc[k * yc]);
          } else {
            const V2<T>* Ar = A + (sidx * D) * ldc + r;
            for (int k = 0; k < D; ++k) fma_c<T>(acc, Ar[k * ldc], Yc[k * yc]);
          }
          const T mk_ = (T)mask[r];
          const RowPos p = row_pos(sa, row0 + r);
          gamma[elem(sa, sidx, p, kb + kc)] = mk<T>(acc.x * mk_, acc.y * mk_);
        }
        __syncthreads();
      }
    }
  }
}

// ---------------------------------------------------------------- tensor-core passes (mixed path)
// Allocate the CTA's TMEM (warp 0) and set up its two mbarriers (MMA commits,
// bulk-copy staging); every thread then holds the TMEM base address.
__device__ __forceinline__ uint32_t tc_setup(uint32_t* slot, uint64_t* bars, uint32_t ncols) {
  if (threadIdx.x < 32) {
    tc::tmem_alloc(slot, ncols);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(bars, 1);
    tc::mbar_init(bars + 1, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  return *slot;
}
__device__ __forceinline__ void tc_teardown(uint32_t tmem, uint32_t ncols) {
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, ncols);
  }
}

// Row mask of the update: rows whose lambda on an other leg is at or below the
// pseudo-inverse cut are zeroed (as in update_kernel).
template <bool kCG>
__device__ void tc_row_mask(const SideDesc& sa, const double* lam, int row0, int nrows, int D, float* mask,
                            double* cut) {
  if (threadIdx.x < 2) {
    const int lo = threadIdx.x == 0 ? sa.lam_o1 : sa.lam_o2;
    double mx = 0.0;
    if (lo >= 0)
      for (int k = 0; k < D; ++k) mx = fmax(mx, ldst<kCG>(lam + lo + k));
    cut[threadIdx.x] = kLambdaCut * mx;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
    const RowPos p = row_pos(sa, row0 + r);
    bool ok = true;
    if (sa.lam_o1 >= 0) ok = ok && ldst<kCG>(lam + sa.lam_o1 + p.r1) > cut[0];
    if (sa.lam_o2 >= 0) ok = ok && ldst<kCG>(lam + sa.lam_o2 + p.r2) > cut[1];
    mask[r] = ok ? 1.f : 0.f;
  }
  __syncthreads();
}

// Update pass over all rows of end a, 128 rows at a time.
template <bool kCG>
__device__ bool tc_update_pass(const SideDesc& sa, float2* gamma, const double* lam, const float2* Y, double th,
                               int D, unsigned char* sm, const TcCtx& cx, uint32_t& phase) {
  __shared__ double cut[2];
  float* mask = reinterpret_cast<float*>(sm + tc_update_smem(D) - 128 * 4);
  const float c = (float)cos(0.5 * th), s = (float)sin(0.5 * th);
  bool ok = true;
  for (int row0 = 0; row0 < sa.rows && ok; row0 += 128) {
    const int nrows = sa.rows - row0 < 128 ? sa.rows - row0 : 128;
    tc_row_mask<kCG>(sa, lam, row0, nrows, D, mask, cut);
    ok = tc_update_rows<kCG>(sa, gamma, Y, c, s, mask, row0, nrows, D, sm, cx, phase);
  }
  return ok;
}

// Gram partials of one bond on the tensor cores, one partial per 64-row tile
// (layered form of the mixed path; the partial layout of gram_kernel).
__global__ void __launch_bounds__(128)
    tc_gram_kernel(const BondDesc* __restrict__ bonds, const float2* __restrict__ gamma,
                   const double* __restrict__ lam, const double* __restrict__ pending, float2* __restrict__ partials,
                   int* flags, int D, long long limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tslot;
  const uint32_t ncols = tc_cols(D);
  const TcCtx cx{tc_setup(&tslot, bars, ncols), bars, bars + 1, limit};
  uint32_t mphase = 0, sphase = 0;
  const BondDesc& bd = bonds[blockIdx.x];
  const SideDesc sa = bd.a;
  const double th = pending[sa.site];
  const float c = (float)cos(0.5 * th), s = (float)sin(0.5 * th);
  const int D2 = D * D;
  const bool ok = tc_gram_pass<false>(sa, gamma, lam, c, s, D, smem_raw, cx, mphase, sphase, nullptr,
                                      partials + (int64_t)bd.part0 * 2 * D2);
  if (!ok && threadIdx.x == 0) atomicOr(flags, 4);
  tc_teardown(cx.tmem, ncols);
}

// Update of one bond's end a on the tensor cores (layered form of the mixed
// path; the same product as update_kernel).
__global__ void __launch_bounds__(128)
    tc_update_kernel(const BondDesc* __restrict__ bonds, float2* gamma, const double* __restrict__ lam,
                     const float2* __restrict__ Y, const double* __restrict__ theta_a, int* flags, int D,
                     long long limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tslot;
  const uint32_t ncols = tc_cols(D);
  const TcCtx cx{tc_setup(&tslot, bars, ncols), bars, bars + 1, limit};
  uint32_t phase = 0;
  const SideDesc sa = bonds[blockIdx.x].a;
  const bool ok = tc_update_pass<false>(sa, gamma, lam, Y + (int64_t)blockIdx.x * 2 * D * D, theta_a[blockIdx.x], D,
                                        smem_raw, cx, phase);
  if (!ok && threadIdx.x == 0) atomicOr(flags, 4);
  tc_teardown(cx.tmem, ncols);
}

// The fused step's Gram pass on the tensor cores: per 64-row tile read out and
// summed in FP64 in tile order, as the layered partials are.  kNb: see
// tc_gram_pass (1 where three CTAs share an SM and registers are scarce).
// With gsum null the tiles' FP32 partials go to part instead (see StepSlot).
template <int kNb>
__device__ bool tc_fused_gram(const SideDesc& sa, const float2* gamma, const double* lam, double th, double2* gsum,
                              float2* part, int D, unsigned char* sm, const TcCtx& cx, uint32_t& mphase,
                              uint32_t& sphase) {
  const int D2 = D * D, nout = 2 * D2;
  if (gsum) {
    for (int o = threadIdx.x; o < nout; o += blockDim.x) gsum[o] = make_double2(0.0, 0.0);
    __syncthreads();
  }
  const float c = (float)cos(0.5 * th), s = (float)sin(0.5 * th);
  return tc_gram_pass<true, kNb>(sa, gamma, lam, c, s, D, sm, cx, mphase, sphase, gsum, part);
}

// Layout of a fused-step CTA's global slot: the big part of the bond layout at
// n = 2D, then the FP64 Gram sums [2][D][D], Y [2][D][D] and the kick angle of end a.
// Complex64 storage up to D = 32 adds the FP32 Gram partials of the tensor-core
// pass, one per 64-row tile of the largest end (ceil(D^2 / 64) x 2 D^2 complex):
// stored per tile and summed by the bond eigenproblem in tile order, as the
// layered launches do, with no read-modify-write of an FP64 sum per tile.
struct StepSlot {
  size_t off_gsum, off_Y, off_th, off_part, total;
  __host__ __device__ StepSlot(int D, size_t elt) {
    off_gsum = (bond_big(D, elt) + 255) & ~(size_t)255;
    off_Y = off_gsum + (size_t)2 * D * D * 16;
    off_th = off_Y + (size_t)2 * D * D * elt;
    off_part = (off_th + 16 + 255) & ~(size_t)255;
    const size_t part = (elt == 8 && D <= 32) ? (size_t)((D * D + kTileRows - 1) / kTileRows) * 2 * D * D * 8 : 0;
    total = (off_part + part + 255) & ~(size_t)255;
  }
};

BondFootprint step_footprint(int D, size_t elt, bool tc) {
  const BondSmem L(D, 2 * D);
  size_t sm = L.small + bond_f32(D, elt);
  if (tc) {
    if (tc_gram_smem(D) > sm) sm = tc_gram_smem(D);
    if (tc_update_smem(D) > sm) sm = tc_update_smem(D);
    return BondFootprint{(sm + 15) & ~(size_t)15, StepSlot(D, elt).total};
  }
  const size_t tr = (size_t)tile_rows(D, elt);
  const size_t gram = tr * (2 * D + 1) * elt;
  const size_t r = tr * (2 * D + 1), c = (size_t)(2 * D) * (tr + 1);
  const size_t upd = (size_t)D * y_cols(D) * elt + (r > c ? r : c) * elt + tr * 4;
  if (gram > sm) sm = gram;
  if (upd > sm) sm = upd;
  return BondFootprint{(sm + 15) & ~(size_t)15, StepSlot(D, elt).total};
}

template <typename T, int kThr, int kMinB, bool kTC>
__global__ void __launch_bounds__(kThr, kMinB)
    step_kernel(const StepTask* __restrict__ tasks, int n_tasks, unsigned int* queue, int* done, V2<T>* gamma,
                double* lam, double* pending, int* flags, unsigned long long* sweeps_out, unsigned long long* cycles,
                int D, JacobiParams jp, unsigned char* scratch, size_t slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int next;
  unsigned char* mine = scratch + (size_t)blockIdx.x * slot;
  const StepSlot SL(D, sizeof(V2<T>));
  double2* gsum = reinterpret_cast<double2*>(mine + SL.off_gsum);
  V2<T>* Y = reinterpret_cast<V2<T>*>(mine + SL.off_Y);
  double* th_a = reinterpret_cast<double*>(mine + SL.off_th);
  float2* tc_part = reinterpret_cast<float2*>(mine + SL.off_part);  // tensor-core Gram partials (D <= 32)
  // tensor-core passes: TMEM for the whole launch, mbarriers of the MMA commits and of the
  // staging; between the passes their state (the two phase bits, ok) lives in shared memory, so
  // that nothing of it occupies registers during the bond eigenproblem
  __shared__ __align__(8) uint64_t tc_bars[2];
  __shared__ uint32_t tc_slot, tc_state[3];
  if constexpr (kTC) {
    tc_setup(&tc_slot, tc_bars, tc_cols(D));
    if (threadIdx.x == 0) {
      tc_state[0] = 0u;
      tc_state[1] = 0u;
      tc_state[2] = 1u;
    }
    __syncthreads();
  }
  for (;;) {
    if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int ti = next;
    __syncthreads();
    if (ti >= n_tasks) break;
    const BondDesc bd = tasks[ti].bd;
    if (threadIdx.x == 0) {
      wait_done(done, tasks[ti].dep_a, flags, jp.wait_cycles);
      wait_done(done, tasks[ti].dep_b, flags, jp.wait_cycles);
    }
    __syncthreads();
    long long tp = 0;
    if (threadIdx.x == 0 && cycles) tp = clock64();
    if constexpr (kTC) {
      const TcCtx cx{tc_slot, tc_bars, tc_bars + 1, kTcWaitCycles};
      uint32_t ph = tc_state[0], sph = tc_state[1];
      bool ok = tc_state[2] != 0;
      // D <= 32: per-tile FP32 partials in the slot, summed by the bond eigenproblem; else FP64 sums
      if (ok)
        ok = tc_fused_gram<(kMinB >= 3 ? 1 : 4)>(bd.a, reinterpret_cast<const float2*>(gamma), lam,
                                                 __ldcg(pending + bd.a.site), D <= 32 ? nullptr : gsum,
                                                 D <= 32 ? tc_part : nullptr, D, smem_raw, cx, ph, sph);
      __syncthreads();
      if (threadIdx.x == 0) {
        tc_state[0] = ph;
        tc_state[1] = sph;
        tc_state[2] = ok ? 1u : 0u;
      }
      __syncthreads();
    } else {
      fused_gram<T>(bd.a, gamma, lam, __ldcg(pending + bd.a.site), gsum, D, smem_raw);
    }
    if (threadIdx.x == 0 && cycles) atomicAdd(cycles + kPhases + 2 * kRotSweeps, (unsigned long long)(clock64() - tp));
    {
      const bool parts = kTC && D <= 32;
      bond_body<T, true>(bd, parts ? reinterpret_cast<const V2<T>*>(tc_part) : nullptr, parts ? nullptr : gsum,
                         gamma, lam, pending, Y, th_a, flags, sweeps_out, cycles, nullptr, D, jp, mine);
    }
    __syncthreads();
    if (threadIdx.x == 0 && cycles) tp = clock64();
    if constexpr (kTC) {
      const TcCtx cx{tc_slot, tc_bars, tc_bars + 1, kTcWaitCycles};
      uint32_t ph = tc_state[0];
      bool ok = tc_state[2] != 0;
      if (ok)
        ok = tc_update_pass<true>(bd.a, reinterpret_cast<float2*>(gamma), lam, reinterpret_cast<const float2*>(Y),
                                  *th_a, D, smem_raw, cx, ph);
      __syncthreads();
      if (threadIdx.x == 0) {
        tc_state[0] = ph;
        tc_state[2] = ok ? 1u : 0u;
      }
    } else {
      fused_update<T>(bd.a, gamma, lam, Y, *th_a, D, smem_raw);
    }
    __syncthreads();
    if (threadIdx.x == 0 && cycles)
      atomicAdd(cycles + kPhases + 2 * kRotSweeps + 1, (unsigned long long)(clock64() - tp));
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(done + ti, 1);
    }
  }
  if constexpr (kTC) {
    __syncthreads();
    if (!tc_state[2] && threadIdx.x == 0) atomicOr(flags, 4);
    tc_teardown(tc_slot, tc_cols(D));
  }
}

// ---------------------------------------------------------------- big-end update
template <typename T>
__global__ void __launch_bounds__(kThreads)
    update_kernel(const TileDesc* __restrict__ tiles, const BondDesc* __restrict__ bonds, V2<T>* gamma,
                  const double* __restrict__ lam, const V2<T>* __restrict__ Y,
                  const double* __restrict__ theta_a, int D) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TileDesc t = tiles[blockIdx.x];
  const SideDesc sa = bonds[t.bond].a;
  const int D2 = D * D, yc = y_cols(D);
  V2<T>* Ys = reinterpret_cast<V2<T>*>(smem_raw);  // [D][yc]: columns kb.. of Y_s of the spin block being written
  V2<T>* A = Ys + (size_t)D * yc;                  // tile, layout chosen for the write order
  const size_t a_elems_r = (size_t)t.nrows * (2 * D + 1), a_elems_c = (size_t)(2 * D) * (t.nrows + 1);
  float* mask = reinterpret_cast<float*>(A + (a_elems_r > a_elems_c ? a_elems_r : a_elems_c));
  __shared__ double cut[2];
  const bool kfast = sa.str_k == 1;
  // kfast: A[r][(2D+1)] with (s, k) inside; else A[(s, k)][nrows+1] with r inside
  const int ldr = 2 * D + 1, ldc = t.nrows + 1;
  if (threadIdx.x < 2) {
    const int lo = threadIdx.x == 0 ? sa.lam_o1 : sa.lam_o2;
    double mx = 0.0;
    if (lo >= 0)
      for (int k = 0; k < D; ++k) mx = fmax(mx, lam[lo + k]);
    cut[threadIdx.x] = kLambdaCut * mx;
  }
  const double th = theta_a[t.bond];
  const T c = (T)cos(0.5 * th), s = (T)sin(0.5 * th);
  const int nel = t.nrows * D;
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    int r, k;
    if (kfast) {
      r = idx / D;
      k = idx - r * D;
    } else {
      k = idx / t.nrows;
      r = idx - k * t.nrows;
    }
    const RowPos p = row_pos(sa, t.row0 + r);
    const int64_t e = elem(sa, 0, p, k);
    V2<T> a0, a1;
    kick2<T>(c, s, gamma[e], gamma[e + sa.str_s], a0, a1);
    if (kfast) {
      A[r * ldr + k] = a0;
      A[r * ldr + D + k] = a1;
    } else {
      A[k * ldc + r] = a0;
      A[(D + k) * ldc + r] = a1;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < t.nrows; r += blockDim.x) {
    const RowPos p = row_pos(sa, t.row0 + r);
    bool ok = true;
    if (sa.lam_o1 >= 0) ok = ok && lam[sa.lam_o1 + p.r1] > cut[0];
    if (sa.lam_o2 >= 0) ok = ok && lam[sa.lam_o2 + p.r2] > cut[1];
    mask[r] = ok ? 1.f : 0.f;
  }
  __syncthreads();
  // one pass per spin block s and block of yc columns kk:
  // Gamma_a'[s][row][kk] = mask(row) sum_k A_s[row][k] Y_s[k][kk]
  const int nout = t.nrows * yc;
  for (int sidx = 0; sidx < 2; ++sidx) {
    for (int kb = 0; kb < D; kb += yc) {
      for (int o = threadIdx.x; o < D * yc; o += blockDim.x) {
        const int k = o / yc, cc = o - (o / yc) * yc;
        Ys[o] = Y[((int64_t)t.bond * 2 + sidx) * D2 + (int64_t)k * D + kb + cc];
      }
      __syncthreads();
      for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        int r, kc;
        if (kfast) {  // kk fastest
          r = o / yc;
          kc = o - r * yc;
        } else {  // r fastest
          kc = o / t.nrows;
          r = o - kc * t.nrows;
        }
        V2<T> acc = mk<T>(0, 0);
        const V2<T>* Yc = Ys + kc;
        if (kfast) {
          const V2<T>* Ar = A + r * ldr + sidx * D;
          for (int k = 0; k < D; ++k) fma_c<T>(acc, Ar[k], Yc[k * yc]);
        } else {
          const V2<T>* Ar = A + (sidx * D) * ldc + r;
          for (int k = 0; k < D; ++k) fma_c<T>(acc, Ar[k * ldc], Yc[k * yc]);
        }
        const T mk_ = (T)mask[r];
        const RowPos p = row_pos(sa, t.row0 + r);
        gamma[elem(sa, sidx, p, kb + kc)] = mk<T>(acc.x * mk_, acc.y * mk_);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- readout
template <typename T>
__global__ void __launch_bounds__(kThreads)
    readout_kernel(const SiteDesc* __restrict__ sites, const V2<T>* __restrict__ gamma,
                   const double* __restrict__ lam, const double* __restrict__ pending, double* __restrict__ z,
                   int D) {
  const SiteDesc sd = sites[blockIdx.x];
  const int deg = sd.deg;
  // lambda^2 of every leg in the storage precision, once per CTA (as each element would form it)
  __shared__ T sq[3][kMaxDc128];
  for (int t = threadIdx.x; t < deg * D; t += blockDim.x) {
    const int q = t / D, l = t - (t / D) * D;
    const T lv = (T)lam[sd.lam[q] + l];
    sq[q][l] = lv * lv;
  }
  __syncthreads();
  int nel = 1;
  for (int q = 0; q < deg; ++q) nel *= D;
  // per element: kick and weighted |psi|^2 in the storage precision (the
  // tensors carry no more); complex128 sums every element in FP64, complex64
  // sums 8 elements of a thread in FP32 (all terms are positive: relative
  // error below 8 x 2^-24) before each FP64 addition, which keeps FP64
  // conversions and adds (64 cycles of an SMSP's FP64 unit per warp
  // instruction) off the per-element path
  const double th = pending[blockIdx.x];
  const T c = (T)cos(0.5 * th), s = (T)sin(0.5 * th);
  // base-D digits of the element index (leg deg-1 fastest) and of the stride, stepped with carries
  int dg[3] = {0, 0, 0}, st[3] = {0, 0, 0};
  {
    int a = threadIdx.x, b = blockDim.x;
#pragma unroll
    for (int q = 2; q >= 0; --q) {
      if (q < deg) {
        dg[q] = a % D;
        a /= D;
        st[q] = b % D;
        b /= D;
      }
    }
  }
  double p0 = 0.0, p1 = 0.0;
  T f0 = (T)0, f1 = (T)0;
  int run = 0;
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    T w = (T)1;
#pragma unroll
    for (int q = 2; q >= 0; --q)
      if (q < deg) w *= sq[q][dg[q]];
    int carry = 0;
#pragma unroll
    for (int q = 2; q >= 0; --q) {
      if (q < deg) {
        const int v = dg[q] + st[q] + carry;
        carry = v >= D ? 1 : 0;
        dg[q] = v - (carry ? D : 0);
      }
    }
    V2<T> a0, a1;
    kick2<T>(c, s, gamma[sd.off + idx], gamma[sd.off + nel + idx], a0, a1);
    if constexpr (sizeof(T) == 8) {
      p0 += (double)(w * (a0.x * a0.x + a0.y * a0.y));
      p1 += (double)(w * (a1.x * a1.x + a1.y * a1.y));
    } else {
      f0 += w * (a0.x * a0.x + a0.y * a0.y);
      f1 += w * (a1.x * a1.x + a1.y * a1.y);
      if (++run == 8) {
        p0 += (double)f0;
        p1 += (double)f1;
        f0 = f1 = (T)0;
        run = 0;
      }
    }
  }
  p0 += (double)f0;
  p1 += (double)f1;
  __shared__ double red[2][kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    p0 += __shfl_down_sync(0xffffffffu, p0, off);
    p1 += __shfl_down_sync(0xffffffffu, p1, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][warp] = p0;
    red[1][warp] = p1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    z[blockIdx.x] = (s0 - s1) / (s0 + s1);
  }
}

__global__ void mean_kernel(const double* __restrict__ z, const int32_t* __restrict__ inst_site0,
                            double* __restrict__ mean) {
  const int k = blockIdx.x;
  const int s0 = inst_site0[k], s1 = inst_site0[k + 1];
  double acc = 0.0;
  for (int i = s0 + threadIdx.x; i < s1; i += blockDim.x) acc += z[i];
  __shared__ double red[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    mean[k] = s / (double)(s1 - s0);
  }
}

// ---------------------------------------------------------------- launchers
static size_t gram_smem(int D, size_t elt) { return (size_t)tile_rows(D, elt) * (2 * D + 1) * elt; }
static size_t update_smem(int D, size_t elt) {
  const size_t tr = (size_t)tile_rows(D, elt);
  const size_t r = tr * (2 * D + 1), c = (tr + 1) * 2 * D;
  return (size_t)D * y_cols(D) * elt + (r > c ? r : c) * elt + tr * 4 + 64;
}

// Opt in to the dynamic shared memory of the largest supported D (called once
// per handle before any launch, outside stream capture).
template <typename T>
cudaError_t Launch<T>::init() {
  cudaError_t e = cudaFuncSetAttribute(gram_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBondSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(bond_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBondSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(bond_kernel_persistent<T, kBondThreads, 1>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBondSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(bond_kernel_persistent<T, 256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bond_share_smem(2));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(bond_kernel_persistent<T, 128, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bond_share_smem(4));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(step_kernel<T, 256, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bond_share_smem(2));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(step_kernel<T, 192, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bond_share_smem(3));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(step_kernel<T, kBondThreads, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kBondSmemMax);
  if (e != cudaSuccess) return e;
  if constexpr (std::is_same<T, float>::value) {
    e = cudaFuncSetAttribute(step_kernel<T, 192, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bond_share_smem(4));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(step_kernel<T, 192, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bond_share_smem(4));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(step_kernel<T, 256, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bond_share_smem(2));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(step_kernel<T, 192, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bond_share_smem(3));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(step_kernel<T, kBondThreads, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBondSmemMax);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_gram_smem(64));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(tc_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_update_smem(64));
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(update_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBondSmemMax);
}

template <typename T>
cudaError_t Launch<T>::reset(void* gamma, double* lam, int64_t n_gamma, int64_t n_lam_edges, int D,
                             const int64_t* d_site_off, int n_sites, double* pending, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(gamma, 0, (size_t)n_gamma * sizeof(V2<T>), st);
  if (err != cudaSuccess) return err;
  err = cudaMemsetAsync(lam, 0, (size_t)n_lam_edges * D * sizeof(double), st);
  if (err != cudaSuccess) return err;
  const int64_t n = n_sites > n_lam_edges ? n_sites : n_lam_edges;
  if (n == 0) return cudaSuccess;
  reset_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(static_cast<V2<T>*>(gamma), lam, d_site_off,
                                                                 n_sites, n_lam_edges, D, pending);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::kick(double* pending, const double* theta, const int32_t* site_inst, int n_sites,
                            int per_qubit, cudaStream_t st, double scale) {
  if (n_sites == 0) return cudaSuccess;
  kick_kernel<<<(n_sites + 255) / 256, 256, 0, st>>>(pending, theta, site_inst, n_sites, per_qubit, scale);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::gram(const TileDesc* tiles, int n_tiles, const BondDesc* bonds, const void* gamma,
                            const double* lam, const double* pending, void* partials, int D, cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  const size_t sm = gram_smem(D, sizeof(V2<T>));
  gram_kernel<T><<<n_tiles, kThreads, sm, st>>>(tiles, bonds, static_cast<const V2<T>*>(gamma), lam, pending,
                                                 static_cast<V2<T>*>(partials), D);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::gram_tc(const BondDesc* bonds, int n_bonds, const void* gamma, const double* lam,
                               const double* pending, void* partials, int* flags, int D, cudaStream_t st) {
  if (n_bonds == 0) return cudaSuccess;
  if (!std::is_same<T, float>::value || !tc_supported(D)) return cudaErrorInvalidValue;
  tc_gram_kernel<<<n_bonds, 128, tc_gram_smem(D), st>>>(bonds, static_cast<const float2*>(gamma), lam, pending,
                                                          static_cast<float2*>(partials), flags, D, kTcWaitCycles);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::update_tc(const BondDesc* bonds, int n_bonds, void* gamma, const double* lam, const void* Y,
                                 const double* theta_a, int* flags, int D, cudaStream_t st) {
  if (n_bonds == 0) return cudaSuccess;
  if (!std::is_same<T, float>::value || !tc_supported(D)) return cudaErrorInvalidValue;
  tc_update_kernel<<<n_bonds, 128, tc_update_smem(D), st>>>(bonds, static_cast<float2*>(gamma), lam,
                                                              static_cast<const float2*>(Y), theta_a, flags, D,
                                                              kTcWaitCycles);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::bond(const BondDesc* bonds, int n_bonds, const void* partials, void* gamma, double* lam,
                            double* pending, void* Y, double* theta_a, int* flags, unsigned long long* sweeps,
                            unsigned long long* cycles, void* vsave, int D, JacobiParams jp, cudaStream_t st,
                            unsigned int* queue, int n_ctas, void* scratch, int per_sm) {
  if (n_bonds == 0) return cudaSuccess;
  const bool shared = per_sm > 1;
  const BondFootprint fp = shared ? bond_footprint_global(D, sizeof(V2<T>)) : bond_footprint(D, kBondSmemMax, sizeof(V2<T>));
  if (fp.slot && !scratch) return cudaErrorInvalidValue;
  if (shared && (!queue || (per_sm != 2 && per_sm != 4) || fp.smem > bond_share_smem(per_sm)))
    return cudaErrorInvalidValue;
  unsigned char* sp = fp.slot ? static_cast<unsigned char*>(scratch) : nullptr;
  if (queue) {
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int want = per_sm * n_ctas;
    const int grid = want < n_bonds ? want : n_bonds;
#define GP_BOND_PERSISTENT(THR, MINB)                                                                           \
  bond_kernel_persistent<T, THR, MINB><<<grid, THR, fp.smem, st>>>(                                             \
      n_bonds, queue, bonds, static_cast<const V2<T>*>(partials), static_cast<V2<T>*>(gamma), lam, pending,    \
      static_cast<V2<T>*>(Y), theta_a, flags, sweeps, cycles, static_cast<double2*>(vsave), D, jp, sp, fp.slot)
    if (per_sm == 4)
      GP_BOND_PERSISTENT(128, 4);
    else if (per_sm == 2)
      GP_BOND_PERSISTENT(256, 2);
    else
      GP_BOND_PERSISTENT(kBondThreads, 1);
#undef GP_BOND_PERSISTENT
    return cudaGetLastError();
  }
  bond_kernel<T><<<n_bonds, kBondThreads, fp.smem, st>>>(bonds, static_cast<const V2<T>*>(partials),
                                                      static_cast<V2<T>*>(gamma), lam, pending,
                                                      static_cast<V2<T>*>(Y), theta_a, flags, sweeps, cycles,
                                                      static_cast<double2*>(vsave), D, jp, sp, fp.slot);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::update(const TileDesc* tiles, int n_tiles, const BondDesc* bonds, void* gamma,
                              const double* lam, const void* Y, const double* theta_a, int D, cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  const size_t sm = update_smem(D, sizeof(V2<T>));
  update_kernel<T><<<n_tiles, kThreads, sm, st>>>(tiles, bonds, static_cast<V2<T>*>(gamma), lam,
                                                   static_cast<const V2<T>*>(Y), theta_a, D);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::readout(const SiteDesc* sites, int n_sites, const void* gamma, const double* lam,
                               const double* pending, double* z, int D, cudaStream_t st) {
  if (n_sites == 0) return cudaSuccess;
  readout_kernel<T><<<n_sites, kThreads, 0, st>>>(sites, static_cast<const V2<T>*>(gamma), lam, pending, z, D);
  return cudaGetLastError();
}

cudaError_t launch_mean(const double* z, const int32_t* inst_site0, int n_inst, double* mean, cudaStream_t st) {
  if (n_inst == 0) return cudaSuccess;
  mean_kernel<<<n_inst, kThreads, 0, st>>>(z, inst_site0, mean);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::step(const StepTask* tasks, int n_tasks, unsigned int* queue, int* done, void* gamma,
                            double* lam, double* pending, int* flags, unsigned long long* sweeps,
                            unsigned long long* cycles, int D, JacobiParams jp, cudaStream_t st, int n_ctas,
                            void* scratch, size_t slot, int per_sm, bool tc) {
  if (n_tasks == 0) return cudaSuccess;
  if (tc && (!std::is_same<T, float>::value || !tc_supported(D))) return cudaErrorInvalidValue;
  const BondFootprint fp = step_footprint(D, sizeof(V2<T>), tc);
  // four CTAs per SM with the tensor-core passes: 4 x tc_cols(D) TMEM columns must fit the SM's 512
  if (!scratch || slot < fp.slot || per_sm < 1 || per_sm > 4 || (per_sm == 4 && tc && 4 * tc_cols(D) > 512))
    return cudaErrorInvalidValue;
  if (fp.smem > (per_sm > 1 ? bond_share_smem(per_sm) : kBondSmemMax)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(done, 0, (size_t)n_tasks * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int want = per_sm * n_ctas;
  const int grid = want < n_tasks ? want : n_tasks;
  unsigned char* sp = static_cast<unsigned char*>(scratch);
#define GP_STEP(THR, MINB, TC)                                                                                   \
  step_kernel<T, THR, MINB, TC><<<grid, THR, fp.smem, st>>>(tasks, n_tasks, queue, done, static_cast<V2<T>*>(gamma), \
                                                            lam, pending, flags, sweeps, cycles, D, jp, sp, slot)
  if (tc) {
    if constexpr (std::is_same<T, float>::value) {
      if (per_sm == 4)
        GP_STEP(192, 4, true);
      else if (per_sm == 3)
        GP_STEP(192, 3, true);
      else if (per_sm == 2)
        GP_STEP(256, 2, true);
      else
        GP_STEP(kBondThreads, 1, true);
    }
  } else if (per_sm == 4) {
    if constexpr (std::is_same<T, float>::value) {
      GP_STEP(192, 4, false);
    } else {
      return cudaErrorInvalidValue;
    }
  } else if (per_sm == 3) {
    GP_STEP(192, 3, false);
  } else if (per_sm == 2) {
    GP_STEP(256, 2, false);
  } else {
    GP_STEP(kBondThreads, 1, false);
  }
#undef GP_STEP
  return cudaGetLastError();
}

template struct Launch<float>;
template struct Launch<double>;

// ============================================================================
// Reverse mode (gradient of a weighted sum of <Z_i> with respect to the kick
// angles), complex128, D <= kMaxGradD.  Convention: for a real loss L and a
// complex variable z, zbar = dL/dRe z + i dL/dIm z; for z = a w with a fixed,
// wbar = conj(a) zbar.  The forward of the gradient path applies the kicks
// explicitly (no kick is fused into a bond) and treats Schmidt values whose
// square is <= jp.ev_cut of the largest as zero, in both directions.
//
// One colour layer is reversed by three launches that mirror the forward:
//   adj_tile    per tile of the larger end a: the Gram partials of the forward
//               and Ybar_s = sum_r conj(A~[r][s][k]) Gbar'[r][s][l]
//   adj_bond    per bond: recompute the bond eigenproblem, then
//               Gbar_b' -> Vbar, w_b-bar;  Ybar -> lambda-bar, Vbar, sbar, Fbar;
//               lambda'-bar -> sbar;  sbar -> Ebar = sbar / 2s;
//               (Ebar, Vbar) -> rhobar = (M + M^H)/2,
//               M = V (diag(Ebar) + K) V^H, K_kj = (vbar_k^H v_j) (e_k - e_j) /
//               ((e_k - e_j)^2 + eps^2) over every eigenvector j (Lorentzian-
//               broadened first-order perturbation theory);
//               rho = sum_s B_s^H C_s B_s (B_s = F^T diag g(s,.)) ->
//               Cbar_s = B_s rhobar B_s^H, Bbar_s = 2 C_s B_s rhobar -> Fbar;
//               C_s = Lambda G_s Lambda -> Gbar_s, lambda-bar;  F -> Gbar_b, w_b-bar
//   adj_update  per tile of a: A~bar = mask (Gbar' Y_s^H) + 2 w^2 A~ Gbar_s,
//               w-bar -> lambda-bar of a's other legs
// ============================================================================

struct AdjSmem {
  size_t off_R, off_V, off_X, off_F, off_Gs, off_Cs, off_Yb, off_Ym, off_Vb, off_Fb, off_M, off_T1, off_re,
      off_re32, off_lamo, off_ev, off_sv, off_rc, off_rs, off_scal, off_lbe, off_svb, off_eb, off_wbb, off_rc32,
      off_rs32, off_int, total;
  __host__ __device__ AdjSmem(int D, int n) {
    const int m = n / 2;
    size_t x = (size_t)n * (n + 1);
    if ((size_t)n * D > x) x = (size_t)n * D;
    size_t o = 0;
    auto take = [&](size_t bytes) {
      const size_t r = o;
      o += (bytes + 15) & ~(size_t)15;
      return r;
    };
    off_R = take((size_t)n * (n + 1) * 16);
    off_V = take((size_t)n * n * 16);
    off_X = take(x * 16);
    off_F = take((size_t)n * D * 16);
    off_Gs = take((size_t)2 * D * D * 16);
    off_Cs = take((size_t)2 * D * D * 16);
    off_Yb = take((size_t)2 * D * D * 16);
    off_Ym = take((size_t)2 * D * D * 16);
    off_Vb = take((size_t)n * D * 16);
    off_Fb = take((size_t)n * D * 16);
    // M holds K and M (n x n) and Cbar_s (D x D); T1 holds Xbar (D x D) and B_s rhobar (D x n)
    off_M = take((size_t)(n * n > D * D ? n * n : D * D) * 16);
    off_T1 = take((size_t)(D * n > D * D ? D * n : D * D) * 16);
    off_re = take((size_t)m * 16);
    off_re32 = take((size_t)m * 8);
    off_lamo = take((size_t)D * 8);
    off_ev = take((size_t)n * 8);
    off_sv = take((size_t)D * 8);
    off_rc = take((size_t)m * 8);
    off_rs = take((size_t)m * 8);
    off_scal = take(8 * 8);
    off_lbe = take((size_t)D * 8);
    off_svb = take((size_t)D * 8);
    off_eb = take((size_t)n * 8);
    off_wbb = take((size_t)n * 8);
    off_rc32 = take((size_t)m * 4);
    off_rs32 = take((size_t)m * 4);
    off_int = take((size_t)(n + 2 * m + 8) * 4);
    total = o;
  }
};

size_t adj_bond_smem_bytes(int D, int n) { return AdjSmem(D, n).total; }

// Gram partials (as the forward) and Ybar partials of the larger end, per tile.
__global__ void __launch_bounds__(kThreads)
    adj_tile_kernel(const TileDesc* __restrict__ tiles, const BondDesc* __restrict__ bonds,
                    const double2* __restrict__ gamma, const double* __restrict__ lam,
                    const double2* __restrict__ gbar, double2* __restrict__ partG, double2* __restrict__ partY,
                    int D) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TileDesc t = tiles[blockIdx.x];
  const SideDesc sa = bonds[t.bond].a;
  const int ld = 2 * D + 1;
  double2* At = reinterpret_cast<double2*>(smem_raw);  // [nrows][2D+1]
  double2* Gb = At + (size_t)t.nrows * ld;              // [nrows][2D+1]
  double* w = reinterpret_cast<double*>(Gb + (size_t)t.nrows * ld);
  __shared__ double cut[2];
  if (threadIdx.x < 2) {
    const int lo = threadIdx.x == 0 ? sa.lam_o1 : sa.lam_o2;
    double mx = 0.0;
    if (lo >= 0)
      for (int k = 0; k < D; ++k) mx = fmax(mx, lam[lo + k]);
    cut[threadIdx.x] = kLambdaCut * mx;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < t.nrows; r += blockDim.x) {
    const RowPos p = row_pos(sa, t.row0 + r);
    w[r] = row_weight(sa, lam, p);
  }
  for (int idx = threadIdx.x; idx < t.nrows * D; idx += blockDim.x) {
    int r, k;
    if (sa.str_k == 1) {
      r = idx / D;
      k = idx - r * D;
    } else {
      k = idx / t.nrows;
      r = idx - k * t.nrows;
    }
    const RowPos p = row_pos(sa, t.row0 + r);
    bool ok = true;
    if (sa.lam_o1 >= 0) ok = ok && lam[sa.lam_o1 + p.r1] > cut[0];
    if (sa.lam_o2 >= 0) ok = ok && lam[sa.lam_o2 + p.r2] > cut[1];
    const int64_t e = elem(sa, 0, p, k);
    At[r * ld + k] = gamma[e];
    At[r * ld + D + k] = gamma[e + sa.str_s];
    Gb[r * ld + k] = ok ? gbar[e] : make_double2(0.0, 0.0);
    Gb[r * ld + D + k] = ok ? gbar[e + sa.str_s] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int D2 = D * D;
  for (int o = threadIdx.x; o < 2 * D2; o += blockDim.x) {
    const int sidx = o / D2, kl = o - (o / D2) * D2, k = kl / D, l = kl - (kl / D) * D;
    double2 g = make_double2(0.0, 0.0), y = make_double2(0.0, 0.0);
    for (int r = 0; r < t.nrows; ++r) {
      const double2 ak = At[r * ld + sidx * D + k];
      const double ww = w[r] * w[r];
      fma_conj<double>(g, cscale(ak, ww), At[r * ld + sidx * D + l]);
      fma_conj<double>(y, ak, Gb[r * ld + sidx * D + l]);
    }
    partG[(int64_t)t.part * 2 * D2 + o] = g;
    partY[(int64_t)t.part * 2 * D2 + o] = y;
  }
}

__device__ __forceinline__ double2 phase_g(int sidx, int t) {
  const double r2 = 0.70710678118654752440;
  return make_double2(r2, sidx == t ? r2 : -r2);
}

__global__ void __launch_bounds__(kThreads)
    adj_bond_kernel(const BondDesc* __restrict__ bonds, const double2* __restrict__ partG,
                    const double2* __restrict__ partY, const double2* __restrict__ gamma,
                    const double* __restrict__ lam, double2* gbar, double* lbar, double2* __restrict__ Gbar_out,
                    double2* __restrict__ Y_out, const double2* __restrict__ vsave, int D, JacobiParams jp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BondDesc bd = bonds[blockIdx.x];
  const SideDesc sb = bd.b;
  const int nb = sb.rows, n = 2 * nb, D2 = D * D, ldr = n + 1;
  const AdjSmem L(D, n);
  double2* RHO = reinterpret_cast<double2*>(smem_raw + L.off_R);
  double2* Vm = reinterpret_cast<double2*>(smem_raw + L.off_V);
  double2* X = reinterpret_cast<double2*>(smem_raw + L.off_X);
  double2* F = reinterpret_cast<double2*>(smem_raw + L.off_F);
  double2* Gs = reinterpret_cast<double2*>(smem_raw + L.off_Gs);
  double2* Cs = reinterpret_cast<double2*>(smem_raw + L.off_Cs);
  double2* Yb = reinterpret_cast<double2*>(smem_raw + L.off_Yb);
  double2* Ym = reinterpret_cast<double2*>(smem_raw + L.off_Ym);
  double2* Vb = reinterpret_cast<double2*>(smem_raw + L.off_Vb);  // [n][D] Vbar of the kept columns
  double2* Fb = reinterpret_cast<double2*>(smem_raw + L.off_Fb);  // [n][D]
  double2* Mm = reinterpret_cast<double2*>(smem_raw + L.off_M);   // [n][n] or [D][D]
  double2* T1 = reinterpret_cast<double2*>(smem_raw + L.off_T1);  // [D][n] or [D][D]
  double* lamo = reinterpret_cast<double*>(smem_raw + L.off_lamo);
  double* ev = reinterpret_cast<double*>(smem_raw + L.off_ev);
  double* sv = reinterpret_cast<double*>(smem_raw + L.off_sv);
  double* scal = reinterpret_cast<double*>(smem_raw + L.off_scal);
  double* lbe = reinterpret_cast<double*>(smem_raw + L.off_lbe);
  double* svb = reinterpret_cast<double*>(smem_raw + L.off_svb);
  double* eb = reinterpret_cast<double*>(smem_raw + L.off_eb);
  double* wbb = reinterpret_cast<double*>(smem_raw + L.off_wbb);
  int* order = reinterpret_cast<int*>(smem_raw + L.off_int);

  // ---- forward recomputation
  for (int k = threadIdx.x; k < D; k += blockDim.x) {
    lamo[k] = lam[bd.lam_e + k];
    lbe[k] = 0.0;
    svb[k] = 0.0;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) wbb[i] = 0.0;
  __syncthreads();
  for (int o = threadIdx.x; o < 2 * D2; o += blockDim.x) {
    double2 g = make_double2(0.0, 0.0), y = make_double2(0.0, 0.0);
    for (int p = 0; p < bd.n_parts; ++p) {
      g = cadd(g, partG[(int64_t)(bd.part0 + p) * 2 * D2 + o]);
      y = cadd(y, partY[(int64_t)(bd.part0 + p) * 2 * D2 + o]);
    }
    const int kl = o % D2, k = kl / D, l = kl - (kl / D) * D;
    Gs[o] = g;
    Cs[o] = cscale(g, lamo[k] * lamo[l]);
    Yb[o] = y;
  }
  load_F<double, false>(sb, gamma, lam, 0.0, F, D);
  // the forward's eigenvectors (sorted by decreasing eigenvalue) and eigenvalues: the
  // output adjoints are expressed in the forward's gauge, so the same V must be used
  {
    const int nm = 2 * D;
    const double2* vs = vsave + (int64_t)blockIdx.x * (nm * nm + nm);
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Vm[idx] = vs[idx];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      ev[j] = vs[n * n + j].x;
      order[j] = j;
    }
  }
  __syncthreads();
  const int kmax = n < D ? n : D;
  if (threadIdx.x == 0) {
    const double emax = ev[order[0]];
    double nrm2 = 0.0;
    for (int kk = 0; kk < D; ++kk) {
      double sval = 0.0;
      if (kk < kmax) {
        const double e = ev[order[kk]];
        if (e > jp.ev_cut * emax && e > 0.0) sval = sqrt(e);
      }
      sv[kk] = sval;
      nrm2 += sval * sval;
    }
    scal[1] = sqrt(nrm2);
    double mx = 0.0;
    const int lo = sb.lam_o1 >= 0 ? sb.lam_o1 : sb.lam_o2;
    if (lo >= 0)
      for (int k = 0; k < D; ++k) mx = fmax(mx, lam[lo + k]);
    scal[2] = mx;
    scal[3] = emax;
  }
  __syncthreads();
  const double nrm = scal[1], lmx = scal[2], emax = scal[3];
  // forward Y (FP64) for the update adjoint
  for (int o = threadIdx.x; o < 2 * D2; o += blockDim.x) {
    const int sidx = o / D2, kl = o - (o / D2) * D2, k = kl / D, kk = kl - (kl / D) * D;
    double2 acc = make_double2(0.0, 0.0);
    if (sv[kk] > 0.0) {
      for (int x = 0; x < n; ++x) fma_c<double>(acc, cmul(F[x * D + k], phase_g(sidx, x & 1)), Vm[x * n + order[kk]]);
      acc = cscale(acc, lamo[k] / sv[kk]);
    }
    Ym[o] = acc;
    Y_out[(int64_t)blockIdx.x * 2 * D2 + o] = acc;
  }
  // ---- reverse
  // Gamma_b' = conj(V_D) / w_b: Vbar and w_b-bar
  for (int idx = threadIdx.x; idx < n * D; idx += blockDim.x) {
    const int x = idx / D, kk = idx - (idx / D) * D;
    const int rj = x >> 1, t = x & 1;
    const RowPos p = row_pos(sb, rj);
    double winv = 1.0;
    const int lo = sb.lam_o1 >= 0 ? sb.lam_o1 : sb.lam_o2;
    if (lo >= 0) {
      const double lv = lam[lo + (sb.lam_o1 >= 0 ? p.r1 : p.r2)];
      winv = lv > kLambdaCut * lmx ? 1.0 / lv : 0.0;
    }
    double2 vb = make_double2(0.0, 0.0);
    if (sv[kk] > 0.0) {
      const double2 g = gbar[elem(sb, t, p, kk)];
      vb = cscale(cconj(g), winv);
    }
    Vb[x * D + kk] = vb;
  }
  __syncthreads();
  if (threadIdx.x < nb) {
    const int rj = threadIdx.x;
    const RowPos p = row_pos(sb, rj);
    const int lo = sb.lam_o1 >= 0 ? sb.lam_o1 : sb.lam_o2;
    if (lo >= 0) {
      const double lv = lam[lo + (sb.lam_o1 >= 0 ? p.r1 : p.r2)];
      if (lv > kLambdaCut * lmx) {
        double acc = 0.0;
        for (int t = 0; t < 2; ++t)
          for (int kk = 0; kk < D; ++kk)
            if (sv[kk] > 0.0) {
              const double2 g = gbar[elem(sb, t, p, kk)];
              const double2 v = Vm[(rj * 2 + t) * n + order[kk]];
              acc += g.x * v.x - g.y * v.y;  // Re(conj(gbar) conj(V)) = Re(gbar V) with conj both
            }
        wbb[rj] += -acc / (lv * lv);
      }
    }
  }
  for (int idx = threadIdx.x; idx < n * D; idx += blockDim.x) Fb[idx] = make_double2(0.0, 0.0);
  __syncthreads();
  // Y_s = Lambda B_s V_D / s
  for (int sidx = 0; sidx < 2; ++sidx) {
    // lambda_e-bar (per k) and Xbar = lambda_k Ybar / s into T1[k][kk]
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
      double acc = 0.0;
      for (int kk = 0; kk < D; ++kk) {
        if (!(sv[kk] > 0.0)) continue;
        const double2 yb = Yb[sidx * D2 + k * D + kk], ym = Ym[sidx * D2 + k * D + kk];
        // X[k][kk] = Ym * s / lambda_k: Re(conj(Yb) X) / s = Re(conj(Yb) Ym) / lambda_k
        if (lamo[k] > 0.0) acc += (yb.x * ym.x + yb.y * ym.y) / lamo[k];
      }
      lbe[k] += acc;
    }
    for (int kk = threadIdx.x; kk < D; kk += blockDim.x) {
      if (!(sv[kk] > 0.0)) continue;
      double acc = 0.0;
      for (int k = 0; k < D; ++k) {
        const double2 yb = Yb[sidx * D2 + k * D + kk], ym = Ym[sidx * D2 + k * D + kk];
        acc += yb.x * ym.x + yb.y * ym.y;
      }
      svb[kk] -= acc / sv[kk];
    }
    for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
      const int k = idx / D, kk = idx - (idx / D) * D;
      T1[k * D + kk] = sv[kk] > 0.0 ? cscale(Yb[sidx * D2 + k * D + kk], lamo[k] / sv[kk]) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    // Vbar[x][kk] += sum_k conj(B_s[k][x]) Xbar[k][kk];  Fbar[x][k] += conj(g) sum_kk Xbar[k][kk] conj(V[x][kk])
    for (int idx = threadIdx.x; idx < n * D; idx += blockDim.x) {
      const int x = idx / D, c = idx - (idx / D) * D;
      const double2 g = phase_g(sidx, x & 1);
      double2 vb = make_double2(0.0, 0.0), fb = make_double2(0.0, 0.0);
      for (int k = 0; k < D; ++k) fma_conj<double>(vb, cmul(F[x * D + k], g), T1[k * D + c]);
      for (int kk = 0; kk < D; ++kk)
        if (sv[kk] > 0.0) fma_c<double>(fb, T1[c * D + kk], cconj(Vm[x * n + order[kk]]));
      Vb[x * D + c] = cadd(Vb[x * D + c], vb);
      Fb[x * D + c] = cadd(Fb[x * D + c], cmul(cconj(g), fb));
    }
    __syncthreads();
  }
  // lambda' = s / ||s||
  if (threadIdx.x == 0) {
    double dot = 0.0;
    for (int kk = 0; kk < D; ++kk)
      if (sv[kk] > 0.0) dot += (sv[kk] / nrm) * lbar[bd.lam_e + kk];
    for (int kk = 0; kk < D; ++kk)
      if (sv[kk] > 0.0) {
        svb[kk] += (lbar[bd.lam_e + kk] - (sv[kk] / nrm) * dot) / nrm;
      }
    for (int j = 0; j < n; ++j) eb[j] = 0.0;
    for (int kk = 0; kk < D && kk < n; ++kk)
      if (sv[kk] > 0.0) eb[kk] = svb[kk] / (2.0 * sv[kk]);
  }
  __syncthreads();
  // eigen adjoint.  Sorted columns: v_j = V[:, order[j]].  Q[kk][j] = vbar_kk^H v_j (kk kept),
  // K = Q o Fm;  T = V_sorted (diag(Ebar) + K) in X [n][n];  M = T V_sorted^H in Mm.
  const double eps2 = (1e-12 * emax) * (1e-12 * emax);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int kk = idx / n, j = idx - (idx / n) * n;
    double2 q = make_double2(0.0, 0.0);
    if (kk < D && sv[kk] > 0.0 && j != kk) {
      for (int x = 0; x < n; ++x) fma_conj<double>(q, Vb[x * D + kk], Vm[x * n + order[j]]);
      const double d = ev[order[kk]] - ev[order[j]];
      q = cscale(q, d / (d * d + eps2));
    }
    Mm[kk * n + j] = q;  // K
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int x = idx / n, j = idx - (idx / n) * n;
    double2 acc = cscale(Vm[x * n + order[j]], eb[j]);
    for (int kk = 0; kk < D && kk < n; ++kk) fma_c<double>(acc, Vm[x * n + order[kk]], Mm[kk * n + j]);
    X[x * n + j] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int x = idx / n, y = idx - (idx / n) * n;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < n; ++j) fma_c<double>(acc, X[x * n + j], cconj(Vm[y * n + order[j]]));
    Mm[x * n + y] = acc;
  }
  __syncthreads();
  // rhobar = (M + M^H)/2 into RHO (the forward rho is no longer needed)
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int x = idx / n, y = idx - (idx / n) * n;
    const double2 a = Mm[x * n + y], b = Mm[y * n + x];
    RHO[x * ldr + y] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  }
  __syncthreads();
  for (int sidx = 0; sidx < 2; ++sidx) {
    // T1 = B_s rhobar  [D][n]
    for (int idx = threadIdx.x; idx < D * n; idx += blockDim.x) {
      const int k = idx / n, y = idx - (idx / n) * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int x = 0; x < n; ++x) fma_c<double>(acc, cmul(F[x * D + k], phase_g(sidx, x & 1)), RHO[x * ldr + y]);
      T1[k * n + y] = acc;
    }
    __syncthreads();
    // Cbar_s[k][l] = sum_y T1[k][y] conj(B_s[l][y]) -> Gbar_s = Lambda Cbar Lambda, lambda-bar
    for (int idx = threadIdx.x; idx < D2; idx += blockDim.x) {
      const int k = idx / D, l = idx - (idx / D) * D;
      double2 cb = make_double2(0.0, 0.0);
      for (int y = 0; y < n; ++y) fma_c<double>(cb, T1[k * n + y], cconj(cmul(F[y * D + l], phase_g(sidx, y & 1))));
      Gbar_out[(int64_t)blockIdx.x * 2 * D2 + sidx * D2 + idx] = cscale(cb, lamo[k] * lamo[l]);
      Mm[idx] = cb;  // Cbar_s, reused below
    }
    __syncthreads();
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
      double acc = 0.0;
      for (int l = 0; l < D; ++l) {
        const double2 cb = Mm[k * D + l], g = Gs[sidx * D2 + k * D + l];
        acc += (cb.x * g.x + cb.y * g.y) * lamo[l];
      }
      lbe[k] += 2.0 * acc;
    }
    // Bbar_s = 2 C_s T1 -> Fbar[x][k] += conj(g(s,t_x)) Bbar_s[k][x]
    for (int idx = threadIdx.x; idx < n * D; idx += blockDim.x) {
      const int x = idx / D, k = idx - (idx / D) * D;
      double2 acc = make_double2(0.0, 0.0);
      for (int l = 0; l < D; ++l) fma_c<double>(acc, Cs[sidx * D2 + k * D + l], T1[l * n + x]);
      Fb[x * D + k] = cadd(Fb[x * D + k], cmul(cconj(phase_g(sidx, x & 1)), cscale(acc, 2.0)));
    }
    __syncthreads();
  }
  // F = w_b Gamma_b: Gamma_b-bar, w_b-bar; write back
  for (int idx = threadIdx.x; idx < nb * D; idx += blockDim.x) {
    const int rj = idx / D, k = idx - (idx / D) * D;
    const RowPos p = row_pos(sb, rj);
    const double w = row_weight(sb, lam, p);
    for (int t = 0; t < 2; ++t) {
      const int64_t e = elem(sb, t, p, k);
      gbar[e] = cscale(Fb[(rj * 2 + t) * D + k], w);
    }
  }
  if (threadIdx.x < nb) {
    const int rj = threadIdx.x;
    const RowPos p = row_pos(sb, rj);
    double acc = wbb[rj];
    for (int t = 0; t < 2; ++t)
      for (int k = 0; k < D; ++k) {
        const double2 fb = Fb[(rj * 2 + t) * D + k], g = gamma[elem(sb, t, p, k)];
        acc += fb.x * g.x + fb.y * g.y;
      }
    if (sb.lam_o1 >= 0 && sb.lam_o2 >= 0) {
      atomicAdd(lbar + sb.lam_o1 + p.r1, acc * lam[sb.lam_o2 + p.r2]);
      atomicAdd(lbar + sb.lam_o2 + p.r2, acc * lam[sb.lam_o1 + p.r1]);
    } else if (sb.lam_o2 >= 0) {
      atomicAdd(lbar + sb.lam_o2 + p.r2, acc);
    } else if (sb.lam_o1 >= 0) {
      atomicAdd(lbar + sb.lam_o1 + p.r1, acc);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < D; k += blockDim.x) lbar[bd.lam_e + k] = lbe[k];
}

// A~bar = mask (Gbar' Y_s^H) + 2 w^2 A~ Gbar_s (in place over Gbar'), w-bar -> lambda-bar of a's other legs.
__global__ void __launch_bounds__(kThreads)
    adj_update_kernel(const TileDesc* __restrict__ tiles, const BondDesc* __restrict__ bonds,
                      const double2* __restrict__ gamma, const double* __restrict__ lam, double2* gbar, double* lbar,
                      const double2* __restrict__ Gbar_in, const double2* __restrict__ Y_in, int D) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TileDesc t = tiles[blockIdx.x];
  const SideDesc sa = bonds[t.bond].a;
  const int ld = 2 * D + 1, D2 = D * D;
  double2* Ys = reinterpret_cast<double2*>(smem_raw);  // [2][D][D]
  double2* Gg = Ys + 2 * D2;                           // [2][D][D]
  double2* At = Gg + 2 * D2;                           // [nrows][2D+1]
  double2* Gb = At + (size_t)t.nrows * ld;             // [nrows][2D+1]
  double* w = reinterpret_cast<double*>(Gb + (size_t)t.nrows * ld);
  double* wb = w + t.nrows;
  __shared__ double cut[2];
  for (int o = threadIdx.x; o < 2 * D2; o += blockDim.x) {
    Ys[o] = Y_in[(int64_t)t.bond * 2 * D2 + o];
    Gg[o] = Gbar_in[(int64_t)t.bond * 2 * D2 + o];
  }
  if (threadIdx.x < 2) {
    const int lo = threadIdx.x == 0 ? sa.lam_o1 : sa.lam_o2;
    double mx = 0.0;
    if (lo >= 0)
      for (int k = 0; k < D; ++k) mx = fmax(mx, lam[lo + k]);
    cut[threadIdx.x] = kLambdaCut * mx;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < t.nrows; r += blockDim.x) {
    const RowPos p = row_pos(sa, t.row0 + r);
    w[r] = row_weight(sa, lam, p);
    wb[r] = 0.0;
  }
  for (int idx = threadIdx.x; idx < t.nrows * D; idx += blockDim.x) {
    int r, k;
    if (sa.str_k == 1) {
      r = idx / D;
      k = idx - r * D;
    } else {
      k = idx / t.nrows;
      r = idx - k * t.nrows;
    }
    const RowPos p = row_pos(sa, t.row0 + r);
    bool ok = true;
    if (sa.lam_o1 >= 0) ok = ok && lam[sa.lam_o1 + p.r1] > cut[0];
    if (sa.lam_o2 >= 0) ok = ok && lam[sa.lam_o2 + p.r2] > cut[1];
    const int64_t e = elem(sa, 0, p, k);
    At[r * ld + k] = gamma[e];
    At[r * ld + D + k] = gamma[e + sa.str_s];
    Gb[r * ld + k] = ok ? gbar[e] : make_double2(0.0, 0.0);
    Gb[r * ld + D + k] = ok ? gbar[e + sa.str_s] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int o = threadIdx.x; o < t.nrows * 2 * D; o += blockDim.x) {
    const int r = o / (2 * D), rem = o - r * 2 * D, sidx = rem / D, k = rem - sidx * D;
    double2 y = make_double2(0.0, 0.0), a = make_double2(0.0, 0.0);
    for (int l = 0; l < D; ++l) {
      fma_c<double>(y, Gb[r * ld + sidx * D + l], cconj(Ys[sidx * D2 + k * D + l]));
      fma_c<double>(a, At[r * ld + sidx * D + l], Gg[sidx * D2 + l * D + k]);
    }
    a = cscale(a, 2.0 * w[r]);  // Abar[r][s][k] (the adjoint of A = w A~)
    const double2 at = At[r * ld + sidx * D + k];
    atomicAdd(wb + r, a.x * at.x + a.y * at.y);
    const double2 out = cadd(y, cscale(a, w[r]));
    const RowPos p = row_pos(sa, t.row0 + r);
    gbar[elem(sa, sidx, p, k)] = out;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < t.nrows; r += blockDim.x) {
    const RowPos p = row_pos(sa, t.row0 + r);
    const double v = wb[r];
    if (sa.lam_o1 >= 0 && sa.lam_o2 >= 0) {
      atomicAdd(lbar + sa.lam_o1 + p.r1, v * lam[sa.lam_o2 + p.r2]);
      atomicAdd(lbar + sa.lam_o2 + p.r2, v * lam[sa.lam_o1 + p.r1]);
    } else if (sa.lam_o2 >= 0) {
      atomicAdd(lbar + sa.lam_o2 + p.r2, v);
    } else if (sa.lam_o1 >= 0) {
      atomicAdd(lbar + sa.lam_o1 + p.r1, v);
    }
  }
}

// Explicit kick of every site: Gamma_i <- exp(-i theta_i X / 2) Gamma_i (one CTA per site).
__global__ void apply_kick_kernel(const SiteDesc* __restrict__ sites, double2* gamma, const double* __restrict__ theta,
                                  int D) {
  const SiteDesc sd = sites[blockIdx.x];
  int nel = 1;
  for (int q = 0; q < sd.deg; ++q) nel *= D;
  const double th = theta[blockIdx.x];
  const double c = cos(0.5 * th), s = sin(0.5 * th);
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    double2 a0, a1;
    kick2<double>(c, s, gamma[sd.off + idx], gamma[sd.off + nel + idx], a0, a1);
    gamma[sd.off + idx] = a0;
    gamma[sd.off + nel + idx] = a1;
  }
}

// Reverse of the explicit kick: thetabar_i += Re <Gbar, (-i/2) X Gamma_post>, Gbar <- R^H Gbar.
__global__ void adj_kick_kernel(const SiteDesc* __restrict__ sites, const double2* __restrict__ gamma_post,
                                double2* gbar, const double* __restrict__ theta, double* dtheta, int D) {
  const SiteDesc sd = sites[blockIdx.x];
  int nel = 1;
  for (int q = 0; q < sd.deg; ++q) nel *= D;
  const double th = theta[blockIdx.x];
  const double c = cos(0.5 * th), s = sin(0.5 * th);
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    const double2 g0 = gbar[sd.off + idx], g1 = gbar[sd.off + nel + idx];
    const double2 p0 = gamma_post[sd.off + idx], p1 = gamma_post[sd.off + nel + idx];
    // (-i/2) X Gamma_post: component 0 <- (-i/2) p1, component 1 <- (-i/2) p0
    acc += g0.x * (0.5 * p1.y) + g0.y * (-0.5 * p1.x) + g1.x * (0.5 * p0.y) + g1.y * (-0.5 * p0.x);
    // R^H = [[c, i s], [i s, c]]
    gbar[sd.off + idx] = make_double2(c * g0.x - s * g1.y, c * g0.y + s * g1.x);
    gbar[sd.off + nel + idx] = make_double2(-s * g0.y + c * g1.x, s * g0.x + c * g1.y);
  }
  __shared__ double red[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    dtheta[blockIdx.x] += v;
  }
}

// Reverse of the mean-field readout for L = sum_i c_i <Z_i>: Gbar_i (written) and
// lambda-bar (accumulated) of every leg.  One CTA per site.
__global__ void adj_readout_kernel(const SiteDesc* __restrict__ sites, const double2* __restrict__ gamma,
                                   const double* __restrict__ lam, const double* __restrict__ cz, double2* gbar,
                                   double* lbar, int D) {
  const SiteDesc sd = sites[blockIdx.x];
  int nel = 1;
  for (int q = 0; q < sd.deg; ++q) nel *= D;
  __shared__ double red[2][kThreads / 32];
  __shared__ double pz[2];
  __shared__ double lb[3][kMaxD];
  for (int i = threadIdx.x; i < 3 * kMaxD; i += blockDim.x) lb[i / kMaxD][i % kMaxD] = 0.0;
  double p0 = 0.0, p1 = 0.0;
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    double w = 1.0;
    int rest = idx;
    for (int q = sd.deg - 1; q >= 0; --q) {
      const double lv = lam[sd.lam[q] + rest % D];
      w *= lv * lv;
      rest /= D;
    }
    const double2 g0 = gamma[sd.off + idx], g1 = gamma[sd.off + nel + idx];
    p0 += w * (g0.x * g0.x + g0.y * g0.y);
    p1 += w * (g1.x * g1.x + g1.y * g1.y);
  }
  for (int off = 16; off > 0; off >>= 1) {
    p0 += __shfl_down_sync(0xffffffffu, p0, off);
    p1 += __shfl_down_sync(0xffffffffu, p1, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = p0;
    red[1][threadIdx.x >> 5] = p1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    const double c = cz[blockIdx.x], den = (s0 + s1) * (s0 + s1);
    pz[0] = c * 2.0 * s1 / den;   // d<Z>/dp0
    pz[1] = -c * 2.0 * s0 / den;  // d<Z>/dp1
  }
  __syncthreads();
  const double dz0 = pz[0], dz1 = pz[1];
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    int li[3] = {0, 0, 0};
    int rest = idx;
    for (int q = sd.deg - 1; q >= 0; --q) {
      li[q] = rest % D;
      rest /= D;
    }
    double l2[3] = {1.0, 1.0, 1.0};
    double w = 1.0;
    for (int q = 0; q < sd.deg; ++q) {
      const double lv = lam[sd.lam[q] + li[q]];
      l2[q] = lv * lv;
      w *= l2[q];
    }
    const double2 g0 = gamma[sd.off + idx], g1 = gamma[sd.off + nel + idx];
    gbar[sd.off + idx] = cscale(g0, 2.0 * dz0 * w);
    gbar[sd.off + nel + idx] = cscale(g1, 2.0 * dz1 * w);
    const double m = dz0 * (g0.x * g0.x + g0.y * g0.y) + dz1 * (g1.x * g1.x + g1.y * g1.y);
    for (int q = 0; q < sd.deg; ++q) {
      double other = 1.0;
      for (int q2 = 0; q2 < sd.deg; ++q2)
        if (q2 != q) other *= l2[q2];
      atomicAdd(&lb[q][li[q]], m * 2.0 * lam[sd.lam[q] + li[q]] * other);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < sd.deg * D; i += blockDim.x) {
    const int q = i / D, l = i - (i / D) * D;
    atomicAdd(lbar + sd.lam[q] + l, lb[q][l]);
  }
}

static size_t adj_tile_smem(int D) { return (size_t)2 * kTileRows * (2 * D + 1) * 16 + (size_t)kTileRows * 8; }
static size_t adj_update_smem(int D) {
  return (size_t)4 * D * D * 16 + (size_t)2 * kTileRows * (2 * D + 1) * 16 + (size_t)2 * kTileRows * 8;
}

cudaError_t Adjoint::init() {
  cudaError_t e = cudaFuncSetAttribute(adj_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)adj_tile_smem(kMaxGradD));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(adj_bond_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)adj_bond_smem_bytes(kMaxGradD, 2 * kMaxGradD));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(adj_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)adj_update_smem(kMaxGradD));
}

cudaError_t Adjoint::layer(const TileDesc* tiles, int n_tiles, const BondDesc* bonds, int n_bonds, const void* gamma,
                           const double* lam, void* gbar, double* lbar, void* partG, void* partY, void* Gbar,
                           void* Ybuf, const void* vsave, int D, JacobiParams jp, cudaStream_t st) {
  if (n_bonds == 0) return cudaSuccess;
  const double2* g = static_cast<const double2*>(gamma);
  adj_tile_kernel<<<n_tiles, kThreads, adj_tile_smem(D), st>>>(tiles, bonds, g, lam, static_cast<double2*>(gbar),
                                                                static_cast<double2*>(partG),
                                                                static_cast<double2*>(partY), D);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj_bond_kernel<<<n_bonds, kThreads, adj_bond_smem_bytes(D, 2 * D), st>>>(
      bonds, static_cast<const double2*>(partG), static_cast<const double2*>(partY), g, lam,
      static_cast<double2*>(gbar), lbar, static_cast<double2*>(Gbar), static_cast<double2*>(Ybuf),
      static_cast<const double2*>(vsave), D, jp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj_update_kernel<<<n_tiles, kThreads, adj_update_smem(D), st>>>(tiles, bonds, g, lam, static_cast<double2*>(gbar),
                                                                    lbar, static_cast<const double2*>(Gbar),
                                                                    static_cast<const double2*>(Ybuf), D);
  return cudaGetLastError();
}

cudaError_t Adjoint::apply_kick(const SiteDesc* sites, int n_sites, void* gamma, const double* theta, int D,
                                cudaStream_t st) {
  if (n_sites == 0) return cudaSuccess;
  apply_kick_kernel<<<n_sites, kThreads, 0, st>>>(sites, static_cast<double2*>(gamma), theta, D);
  return cudaGetLastError();
}

cudaError_t Adjoint::kick(const SiteDesc* sites, int n_sites, const void* gamma_post, void* gbar,
                          const double* theta, double* dtheta, int D, cudaStream_t st) {
  if (n_sites == 0) return cudaSuccess;
  adj_kick_kernel<<<n_sites, kThreads, 0, st>>>(sites, static_cast<const double2*>(gamma_post),
                                                 static_cast<double2*>(gbar), theta, dtheta, D);
  return cudaGetLastError();
}

cudaError_t Adjoint::readout(const SiteDesc* sites, int n_sites, const void* gamma, const double* lam,
                             const double* cz, void* gbar, double* lbar, int D, cudaStream_t st) {
  if (n_sites == 0) return cudaSuccess;
  adj_readout_kernel<<<n_sites, kThreads, 0, st>>>(sites, static_cast<const double2*>(gamma), lam, cz,
                                                    static_cast<double2*>(gbar), lbar, D);
  return cudaGetLastError();
}

}  // namespace gpeps
