// CUDA kernels of the belief-propagation (BP) regauging of the gPEPS state (sm_103a).
//
// Paper, section "Method": for comparison the PEPS is re-gauged with belief
// propagation after each Trotter step ("Results", "Benchmarking").  The norm
// network <psi|psi> carries one D x D Hermitian message per leg of every site
// (a half-edge); one BP iteration recomputes every message from those of the
// previous iteration (parallel schedule):
//
//   message  one CTA per half-edge (i, p): X = conj(Gamma_i) with the
//            environment E_q = diag(lambda_q) m_q diag(lambda_q) of each other
//            leg q applied (leg products through an L2-resident scratch tensor
//            of the CTA), then m[a][a'] = sum Gamma_i[.., a, ..] X[.., a', ..]
//            over s and the other legs, restricted to the support of the
//            bond's lambda (entries k with lambda[k] <= cut * max are zero: cut
//            1e-13 in complex128, 1e-7 with complex64 storage, where rounding
//            residue of rank-deficient bonds sits below that resolution and
//            would lead BP to another fixed point).  Only the upper triangle is summed: the
//            message is Hermitian by definition, and the mirrored lower triangle
//            keeps it exactly so (its rounding noise would otherwise grow along
//            the loops of the lattice).  Normalised to unit trace in FP64; the
//            largest elementwise change is reduced into the iteration's residual.
//   gauge    one 128-thread CTA per edge, FP64 (for complex64 storage the
//            eigenproblems of G are warm-started in FP32): the Hermitian square
//            root R and pseudo-inverse R^+ of G = conj(m) at both ends (Jacobi),
//            C = R_i diag(lambda) R_j^T, its left singular vectors U from the
//            eigenproblem of C C^H, and Y = C^T conj(U), whose column norms are the
//            singular values S (C = U Y^T holds exactly whatever the accuracy of
//            the smallest eigenvalues).  lambda' = S / ||S||, and the gauge
//            matrices R_i^+ U and R_j^+ Y / S of the two half-edges.
//   apply    one CTA per site: Gamma_i <- Gamma_i x_p P_p on every leg p, in place
//            (FP32 for complex64 storage when the gauge matrices are well
//            conditioned, else FP64 rounded once to the storage type).
//
// Leg products and the message Gram view a site tensor [s][leg0][leg1][leg2]
// (last leg fastest) along leg p as columns c (s and the other legs) times the
// leg index b: element (c, b) sits at (c / I) D I + c % I + b I with I the
// stride of the leg.  Tiles of 32 columns x D leg entries pass through shared
// memory, so every element of a tensor is read once per product.
#include <cuda_runtime.h>

#include <cstdint>

#include "gpeps.h"
#include "gpeps_internal.cuh"
#include "jacobi.cuh"
#include "tcgen05.cuh"

namespace gpeps {

namespace {

// Upper-triangle pairs per thread of the message Gram: D <= 32 and D <= 64.
constexpr int kGramPerSmall = (32 * 33 / 2 + kBpMsgThreads - 1) / kBpMsgThreads;
constexpr int kGramPerLarge = (kMaxD * (kMaxD + 1) / 2 + kBpMsgThreads - 1) / kBpMsgThreads;
// The apply runs in FP32 for complex64 storage when every entry of a site's
// gauge matrices is at most this large (well-conditioned gauge), else in FP64.
constexpr double kApplyF32Max = 64.0;

__device__ __forceinline__ int64_t leg_addr(int c, int b, int I, int D) {
  const int o = c / I;
  return (int64_t)o * D * I + (c - o * I) + (int64_t)b * I;
}

// Column j and leg entry b of the idx-th load of a 32-column tile: consecutive
// threads take consecutive addresses (along the leg when it is the fastest index).
__device__ __forceinline__ void tile_pos(int idx, int I, int D, int& j, int& b) {
  if (I == 1) {
    j = idx / D;
    b = idx - j * D;
  } else {
    b = idx >> 5;
    j = idx & 31;
  }
}

// dst(c, b) = sum_b' M[b][b'] src(c, b') over the columns c in [c_begin, c_end)
// of the leg with stride I (conj(src) when kConj), in the arithmetic of TC
// (src and dst hold TS).  Element (c, b) sits at leg_addr(c, b) - src_off in
// src and at leg_addr(c, b) - dst_off in dst.  M: shared [D][D + 1]; tile:
// shared [32][D + 1], both TC.  The next tile is loaded into registers (kL per
// thread, 32 D <= kL blockDim) while the current one is multiplied.  dst may be
// src: the columns of a tile are read completely before any of them is written,
// and the prefetched columns are not the ones being written.
template <typename TS, typename TC, bool kConj, int kL, bool kD32 = false>
__device__ void leg_product(V2<TS>* dst, int64_t dst_off, const V2<TS>* src, int64_t src_off, int c_begin,
                            int c_end, int I, int D, const V2<TC>* M, V2<TC>* tile) {
  const int ld = D + 1;
  constexpr int kB = kL > 0 ? kL : 1;
  V2<TS> buf[kB];
  auto fetch = [&](int c0) {
    const int nc = min(32, c_end - c0);
#pragma unroll
    for (int k = 0; k < kL; ++k) {
      const int idx = threadIdx.x + k * blockDim.x;
      int j, b;
      tile_pos(idx, I, D, j, b);
      buf[k] = (idx < 32 * D && j < nc) ? src[leg_addr(c0 + j, b, I, D) - src_off] : mk<TS>(0, 0);
    }
  };
  if (kL > 0 && c_begin < c_end) fetch(c_begin);
  for (int c0 = c_begin; c0 < c_end; c0 += 32) {
    const int nc = min(32, c_end - c0);
    if constexpr (kL > 0) {
#pragma unroll
      for (int k = 0; k < kL; ++k) {
        const int idx = threadIdx.x + k * blockDim.x;
        int j, b;
        tile_pos(idx, I, D, j, b);
        if (idx < 32 * D) tile[j * ld + b] = mk<TC>((TC)buf[k].x, kConj ? -(TC)buf[k].y : (TC)buf[k].y);
      }
    } else {
      for (int idx = threadIdx.x; idx < 32 * D; idx += blockDim.x) {
        int j, b;
        tile_pos(idx, I, D, j, b);
        if (j < nc) {
          const V2<TS> v = src[leg_addr(c0 + j, b, I, D) - src_off];
          tile[j * ld + b] = mk<TC>((TC)v.x, kConj ? -(TC)v.y : (TC)v.y);
        }
      }
    }
    __syncthreads();
    if (kL > 0 && c0 + 32 < c_end) fetch(c0 + 32);
    if (kD32 && blockDim.x == 256) {
      // D = 32: a 2 x 2 register tile per thread, columns {jb, jb + 16} x leg entries
      // {bb, bb + 16}: a half-warp reads 16 tile rows (distinct banks with the row
      // stride 33) and shares two M values, so a complex FMA costs one shared-memory
      // wavefront instead of three
      const int jb = threadIdx.x & 15, bb = threadIdx.x >> 4;
      V2<TC> a00 = mk<TC>(0, 0), a01 = a00, a10 = a00, a11 = a00;
      const V2<TC>* t0 = tile + jb * 33;
      const V2<TC>* t1 = t0 + 16 * 33;
      const V2<TC>* m0 = M + bb * 33;
      const V2<TC>* m1 = m0 + 16 * 33;
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {
        const V2<TC> x0 = t0[k], x1 = t1[k], y0 = m0[k], y1 = m1[k];
        fma_c<TC>(a00, y0, x0);
        fma_c<TC>(a01, y1, x0);
        fma_c<TC>(a10, y0, x1);
        fma_c<TC>(a11, y1, x1);
      }
      if (jb < nc) {
        dst[leg_addr(c0 + jb, bb, I, 32) - dst_off] = mk<TS>((TS)a00.x, (TS)a00.y);
        dst[leg_addr(c0 + jb, bb + 16, I, 32) - dst_off] = mk<TS>((TS)a01.x, (TS)a01.y);
      }
      if (jb + 16 < nc) {
        dst[leg_addr(c0 + jb + 16, bb, I, 32) - dst_off] = mk<TS>((TS)a10.x, (TS)a10.y);
        dst[leg_addr(c0 + jb + 16, bb + 16, I, 32) - dst_off] = mk<TS>((TS)a11.x, (TS)a11.y);
      }
    } else {
      for (int idx = threadIdx.x; idx < 32 * D; idx += blockDim.x) {
        const int b = idx >> 5, j = idx & 31;
        if (j < nc) {
          V2<TC> acc = mk<TC>(0, 0);
          const V2<TC>* mr = M + b * ld;
          const V2<TC>* tr = tile + j * ld;
          for (int k = 0; k < D; ++k) fma_c<TC>(acc, mr[k], tr[k]);
          dst[leg_addr(c0 + j, b, I, D) - dst_off] = mk<TS>((TS)acc.x, (TS)acc.y);
        }
      }
    }
    __syncthreads();
  }
}

// The upper triangle of m[a][a'] = sum_c A(c, a) B(c, a') over the columns of
// a leg (B = conj(A) when kConjB), accumulated in registers over column ranges
// (K pairs a <= a' per thread), then stored with its conjugate mirror.
template <typename T, int K>
struct GramAcc {
  int pa[K], pb[K];
  V2<T> acc[K];

  __device__ void init(int D) {
    const int npairs = D * (D + 1) / 2;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int u = threadIdx.x + k * blockDim.x;
      int r = 0, c = 0;
      if (u < npairs) {
        r = (int)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
        while (r * (r + 1) / 2 > u) --r;
        while ((r + 1) * (r + 2) / 2 <= u) ++r;
        c = u - r * (r + 1) / 2;
      }
      pa[k] = c;
      pb[k] = r;
      acc[k] = mk<T>(0, 0);
    }
  }

  // A(c, b) at A[leg_addr(c, b)], B(c, b) at B[leg_addr(c, b) - b_off], c in [c_begin, c_end)
  template <bool kConjB>
  __device__ void add(const V2<T>* A, const V2<T>* B, int64_t b_off, int c_begin, int c_end, int I, int D,
                      V2<T>* tA, V2<T>* tB) {
    const int ld = D + 1;
    const int npairs = D * (D + 1) / 2;
    for (int c0 = c_begin; c0 < c_end; c0 += 32) {
      const int nc = min(32, c_end - c0);
      for (int idx = threadIdx.x; idx < 32 * D; idx += blockDim.x) {
        int j, b;
        tile_pos(idx, I, D, j, b);
        V2<T> va = mk<T>(0, 0), vb = mk<T>(0, 0);
        if (j < nc) {
          const int64_t ad = leg_addr(c0 + j, b, I, D);
          va = A[ad];
          vb = B[ad - b_off];
          if (kConjB) vb.y = -vb.y;
        }
        tA[j * ld + b] = va;
        tB[j * ld + b] = vb;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (threadIdx.x + k * blockDim.x < npairs) {
          const V2<T>* ta = tA + pa[k];
          const V2<T>* tb = tB + pb[k];
          for (int j = 0; j < 32; ++j) fma_c<T>(acc[k], ta[j * ld], tb[j * ld]);
        }
      }
      __syncthreads();
    }
  }

  __device__ void store(double2* Mo, int D) const {
    const int npairs = D * (D + 1) / 2;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (threadIdx.x + k * blockDim.x < npairs) {
        const int a = pa[k], b = pb[k];
        if (a == b) {
          Mo[a * D + a] = make_double2((double)acc[k].x, 0.0);
        } else {
          Mo[a * D + b] = make_double2((double)acc[k].x, (double)acc[k].y);
          Mo[b * D + a] = make_double2((double)acc[k].x, -(double)acc[k].y);
        }
      }
    }
  }
};

// The Gram at D = 32 in FP32 as a 2 x 2 register tile per thread (256 threads):
// entries {ab, ab + 16} x {ap, ap + 16} of m, so a half-warp reads 16 consecutive
// entries of a tA row and shares two of tB (one shared-memory wavefront per complex
// FMA instead of about three).  The whole matrix is summed, in the same order as
// GramAcc, and only the upper triangle is stored (mirrored), as there.
struct GramAcc32 {
  float2 a00, a01, a10, a11;

  __device__ void init() { a00 = a01 = a10 = a11 = make_float2(0.f, 0.f); }

  template <bool kConjB>
  __device__ void add(const float2* A, const float2* B, int64_t b_off, int c_begin, int c_end, int I,
                      float2* tA, float2* tB) {
    constexpr int D = 32, ld = 33;
    const int ab = threadIdx.x & 15, ap = threadIdx.x >> 4;
    for (int c0 = c_begin; c0 < c_end; c0 += 32) {
      const int nc = min(32, c_end - c0);
      for (int idx = threadIdx.x; idx < 32 * D; idx += blockDim.x) {
        int j, b;
        tile_pos(idx, I, D, j, b);
        float2 va = make_float2(0.f, 0.f), vb = va;
        if (j < nc) {
          const int64_t ad = leg_addr(c0 + j, b, I, D);
          va = A[ad];
          vb = B[ad - b_off];
          if (kConjB) vb.y = -vb.y;
        }
        tA[j * ld + b] = va;
        tB[j * ld + b] = vb;
      }
      __syncthreads();
#pragma unroll 8
      for (int j = 0; j < 32; ++j) {
        const float2 x0 = tA[j * ld + ab], x1 = tA[j * ld + ab + 16];
        const float2 y0 = tB[j * ld + ap], y1 = tB[j * ld + ap + 16];
        fma_c<float>(a00, x0, y0);
        fma_c<float>(a01, x0, y1);
        fma_c<float>(a10, x1, y0);
        fma_c<float>(a11, x1, y1);
      }
      __syncthreads();
    }
  }

  __device__ void store(double2* Mo) const {
    constexpr int D = 32;
    const int ab = threadIdx.x & 15, ap = threadIdx.x >> 4;
    const int as[2] = {ab, ab + 16}, bs[2] = {ap, ap + 16};
    const float2 v[2][2] = {{a00, a01}, {a10, a11}};
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        const int a = as[u], b = bs[w];
        if (a == b) {
          Mo[a * D + a] = make_double2((double)v[u][w].x, 0.0);
        } else if (a < b) {
          Mo[a * D + b] = make_double2((double)v[u][w].x, (double)v[u][w].y);
          Mo[b * D + a] = make_double2((double)v[u][w].x, -(double)v[u][w].y);
        }
      }
  }
};

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) r = fmax(r, red[w]);
  }
  __syncthreads();
  return r;
}

__global__ void bp_identity_kernel(double2* msgs, int64_t n, int D) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = i % ((int64_t)D * D);
  const int a = (int)(e / D), b = (int)(e - (int64_t)(e / D) * D);
  msgs[i] = make_double2(a == b ? 1.0 / D : 0.0, 0.0);
}

// The end of a message: restrict Mo (the summed Gram, [D][D]) to the support of
// the bond's lambda, normalise it to unit trace, store it and fold the largest
// change against the previous iteration into my_res (bad: not finite).
__device__ void bp_message_finish(const BpMsgTask& tk, const double2* Mo, const double* __restrict__ lam,
                                  const double2* __restrict__ msg_in, double2* __restrict__ msg_out, int D,
                                  double support_cut, double& my_res, bool& bad) {
  __shared__ double s_trace, s_cut;
  // the support of lambda_e: entries k with lambda_e[k] <= support_cut * max are zero
  const double* le = lam + tk.lam[tk.leg];
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int a = 0; a < D; ++a) mx = fmax(mx, le[a]);
    const double cut = support_cut * mx;
    double tr = 0.0;
    for (int a = 0; a < D; ++a)
      if (le[a] > cut) tr += Mo[a * D + a].x;
    s_trace = tr;
    s_cut = cut;
  }
  __syncthreads();
  const double tr = s_trace, cut = s_cut;
  const bool ok = tr > 0.0 && isfinite(tr);
  const double inv = ok ? 1.0 / tr : 0.0;
  double2* mo = msg_out + (int64_t)tk.out * D * D;
  const double2* mprev = msg_in + (int64_t)tk.out * D * D;
  for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
    double2 v = Mo[idx];
    if (ok) {
      const int a = idx / D, b = idx - a * D;
      const double w = (le[a] > cut && le[b] > cut) ? inv : 0.0;
      v.x *= w;
      v.y *= w;
    } else {
      const int a = idx / D;
      v = make_double2(a * D + a == idx ? 1.0 / D : 0.0, 0.0);
    }
    const double2 o = mprev[idx];
    const double dx = v.x - o.x, dy = v.y - o.y;
    const double d = sqrt(dx * dx + dy * dy);
    if (!isfinite(d)) bad = true;
    else my_res = fmax(my_res, d);
    mo[idx] = v;
  }
  if (!ok) bad = true;
  __syncthreads();
}

// One BP iteration.  A message is computed one physical component s at a time
// (the products never mix s), so the scratch tensor X of a CTA holds D^deg
// elements and the launch's scratch stays in L2.
template <typename T, int K>
__global__ void __launch_bounds__(kBpMsgThreads, sizeof(T) == 4 && K == kGramPerSmall ? 5 : 1) bp_message_kernel(const BpMsgTask* __restrict__ tasks, int n_tasks,
                                                                const V2<T>* __restrict__ gamma,
                                                                const double* __restrict__ lam,
                                                                const double2* __restrict__ msg_in,
                                                                double2* __restrict__ msg_out, V2<T>* scratch,
                                                                int64_t slot_elems, int D, double support_cut,
                                                                unsigned long long* residual, int* flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  const int ld = D + 1;
  V2<T>* M = reinterpret_cast<V2<T>*>(smem);  // [D][D + 1]: the environment of one other leg
  V2<T>* tA = M + D * ld;                      // [32][D + 1]
  V2<T>* tB = tA + 32 * ld;                    // [32][D + 1]
  double2* Mo = reinterpret_cast<double2*>(tB + 32 * ld);  // [D][D]
  V2<T>* X = scratch + (int64_t)blockIdx.x * slot_elems;
  // tiles are loaded straight into shared memory: a register prefetch of the next
  // tile, or a 2 x D/16 register tile per thread, cost more in occupancy than
  // they saved (measured: 5.26 and 5.51 ms against 4.76 ms per launch at D = 32)
  constexpr int kL = 0;
  double my_res = 0.0;
  bool bad = false;
  for (int t = blockIdx.x; t < n_tasks; t += gridDim.x) {
    const BpMsgTask tk = tasks[t];
    const V2<T>* G = gamma + tk.off;
    const int z = tk.deg, p = tk.leg;
    int half = 1;  // columns (and elements) per physical component: D^(deg-1) and D^deg
    for (int k = 1; k < z; ++k) half *= D;
    const int64_t sz = (int64_t)half * D;
    int legs[2] = {-1, -1}, nl = 0;
    for (int q = 0; q < z; ++q)
      if (q != p) legs[nl++] = q;
    int Ip = 1;
    for (int k = p + 1; k < z; ++k) Ip *= D;
    GramAcc<T, K> gram;
    GramAcc32 gram32;
    const bool tile32 = sizeof(T) == 4 && D == 32 && blockDim.x == 256;
    if (tile32) gram32.init();
    else gram.init(D);
    for (int s = 0; s < 2; ++s) {
      const int c0 = s * half, c1 = c0 + half;
      const int64_t off = s * sz;
      for (int l = 0; l < nl; ++l) {
        // E_q = diag(lambda_q) m_q diag(lambda_q); the product's first barrier
        // (after its first tile load) orders these writes before any read of M,
        // and the previous product's last barrier orders them after its reads
        const double* lq = lam + tk.lam[legs[l]];
        const double2* mi = msg_in + (int64_t)tk.in[legs[l]] * D * D;
        for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
          const int b = idx / D, bb = idx - b * D;
          const double2 v = mi[idx];
          const double w = lq[b] * lq[bb];
          M[b * ld + bb] = mk<T>((T)(v.x * w), (T)(v.y * w));
        }
        int I = 1;
        for (int k = legs[l] + 1; k < z; ++k) I *= D;
        if (sizeof(T) == 4 && D == 32) {  // the 2 x 2 register tile (kD32); the FP64 build is
                                          // bound by the FP64 pipe and would only lose registers
          if (l == 0) leg_product<T, T, true, kL, true>(X, off, G, 0, c0, c1, I, D, M, tA);
          else leg_product<T, T, false, kL, true>(X, off, X, off, c0, c1, I, D, M, tA);
        } else {
          if (l == 0) leg_product<T, T, true, kL>(X, off, G, 0, c0, c1, I, D, M, tA);
          else leg_product<T, T, false, kL>(X, off, X, off, c0, c1, I, D, M, tA);
        }
      }
      if (tile32) {
        if constexpr (sizeof(T) == 4) {
          if (nl == 0) gram32.add<true>(G, G, 0, c0, c1, Ip, tA, tB);
          else gram32.add<false>(G, X, off, c0, c1, Ip, tA, tB);
        }
      } else {
        if (nl == 0) gram.template add<true>(G, G, 0, c0, c1, Ip, D, tA, tB);
        else gram.template add<false>(G, X, off, c0, c1, Ip, D, tA, tB);
      }
    }
    if (tile32) gram32.store(Mo);
    else gram.store(Mo, D);
    __syncthreads();
    bp_message_finish(tk, Mo, lam, msg_in, msg_out, D, support_cut, my_res, bad);
  }
  const double r = block_max(my_res, red);
  const int any_bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    if (any_bad) {
      atomicOr(flags, GPEPS_FLAG_NUMERIC);
      atomicMax(residual, 0x7FF0000000000000ULL);  // +inf
    } else {
      atomicMax(residual, (unsigned long long)__double_as_longlong(r));
    }
  }
}

// ---------------------------------------------------------------- tensor-core messages (complex64, D = 32)
// The products of bp_message_kernel on the tensor cores (tcgen05 kind::tf32 with
// FP32 accumulators in TMEM; every FP32 operand split into a TF32 pair, three
// products per pair, as in the simple update's tensor-core passes):
//   leg product  dst(c, b) = sum_b' M[b][b'] src(c, b') for 128 columns c at a
//                time: an M = 128 (c) x N = 64 ((re/im, b)) x K = 64 ((re/im, b'))
//                product whose right operand W, the realified environment M of
//                the leg, is staged once per leg;
//   Gram         m[a][a'] = sum_c A(c, a) B(c, a') over 64-column chunks of both
//                spins into a second accumulator: rows (re/im, a), columns
//                (re/im, a') (rows 64..127 of the M = 128 product unused);
//                m = (B_rr - B_ii) + i (B_ri + B_ir), summed whole and stored as
//                its upper triangle with the conjugate mirror, as the CUDA-core
//                kernel does.
// Operands are K-major without swizzle (tcgen05.cuh) with real and imaginary
// parts in separate planes, written 8 rows x 4 K values per warp (32 banks).
// Every wait is bounded; a wait that gives up raises GPEPS_FLAG_TIMEOUT and the
// CTA stops issuing products (its messages are then wrong, the flag says so).
constexpr int kBpTcD = 32;
constexpr int kBpTcThreads = 256;
constexpr int kTcBatch = 8;  // loads of a thread in flight together in the operand staging
struct BpTcSmem {  // bytes
  static constexpr size_t W = 0;                     // hi | lo of W: 64 rows x 64 K (2 x 16 KB)
  static constexpr size_t A = 32768;                 // leg product hi | lo: 128 x 64 (2 x 32 KB); Gram: A hi | lo
                                                     // 128 x 64 (2 x 32 KB, B in the region of W); readout dump
                                                     // 64 x 65 floats
  static constexpr size_t Mo = A + 65536;            // double2 [32][32]
  static constexpr size_t total = Mo + (size_t)kBpTcD * kBpTcD * 16;
};

__global__ void __launch_bounds__(kBpTcThreads, 2)
    bp_message_tc_kernel(const BpMsgTask* __restrict__ tasks, int n_tasks, const float2* __restrict__ gamma,
                         const double* __restrict__ lam, const double2* __restrict__ msg_in,
                         double2* __restrict__ msg_out, float2* scratch, int64_t slot_elems, double support_cut,
                         unsigned long long* residual, int* flags) {
  constexpr int D = kBpTcD;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  if (threadIdx.x < 32) {
    tc::tmem_alloc(&tslot, 128u);  // [0, 64): leg product, [64, 128): Gram
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  uint32_t phase = 0;
  bool tc_ok = true;
  unsigned char* Wh = smem + BpTcSmem::W;
  unsigned char* Wl = Wh + 16384;
  unsigned char* Ah = smem + BpTcSmem::A;
  unsigned char* Al = Ah + 32768;
  unsigned char* gAh = Ah;            // Gram: A hi | lo, 128 rows x 64 K (the leg product's region)
  unsigned char* gAl = gAh + 32768;
  unsigned char* gBh = Wh;            // Gram: B hi | lo, 64 rows x 64 K (W is rebuilt before its next use)
  unsigned char* gBl = gBh + 16384;
  float* dump = reinterpret_cast<float*>(smem + BpTcSmem::A);
  double2* Mo = reinterpret_cast<double2*>(smem + BpTcSmem::Mo);
  float2* X = scratch + (int64_t)blockIdx.x * slot_elems;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t idesc = tc::idesc_tf32(128, 64);
  double my_res = 0.0;
  bool bad = false;
  for (int t = blockIdx.x; t < n_tasks; t += gridDim.x) {
    const BpMsgTask tk = tasks[t];
    const float2* G = gamma + tk.off;
    const int z = tk.deg, p = tk.leg;
    int half = 1;
    for (int k = 1; k < z; ++k) half *= D;
    const int64_t sz = (int64_t)half * D;
    int legs[2] = {-1, -1}, nl = 0;
    for (int q = 0; q < z; ++q)
      if (q != p) legs[nl++] = q;
    int Ip = 1;
    for (int k = p + 1; k < z; ++k) Ip *= D;
    bool fresh_gram = true;
    for (int s = 0; s < 2; ++s) {
      const int c0 = s * half, c1 = c0 + half;
      const int64_t off = s * sz;
      for (int l = 0; l < nl; ++l) {
        // W: the environment E_q = diag(lambda_q) m_q diag(lambda_q), rounded to FP32 as in the
        // CUDA-core kernel, realified (rows (re/im, b), K (re/im, b')); a warp takes 8 b x 4 b'
        const double* lq = lam + tk.lam[legs[l]];
        const double2* mi = msg_in + (int64_t)tk.in[legs[l]] * D * D;
        for (int g = warp; g < (D / 8) * (D / 4); g += nwarps) {
          const int b = (g / (D / 4)) * 8 + (lane & 7), bp = (g % (D / 4)) * 4 + (lane >> 3);
          const double2 v = mi[b * D + bp];
          const double w = lq[b] * lq[bp];
          const float mr = (float)(v.x * w), mim = (float)(v.y * w);
          tc_put(Wh, Wl, b, bp, 64, mr);
          tc_put(Wh, Wl, b, D + bp, 64, -mim);
          tc_put(Wh, Wl, D + b, bp, 64, mim);
          tc_put(Wh, Wl, D + b, D + bp, 64, mr);
        }
        int I = 1;
        for (int k = legs[l] + 1; k < z; ++k) I *= D;
        // the first leg reads conj(Gamma), the second the scratch in place (a tile's columns are
        // read completely before any of them is written back)
        const float2* src = l == 0 ? G : X;
        const int64_t soff = l == 0 ? 0 : off;
        const float conj = l == 0 ? -1.f : 1.f;
        for (int ct = c0; ct < c1; ct += 128) {
          const int nc = c1 - ct < 128 ? c1 - ct : 128;
          const int ngroups = ((nc + 7) / 8) * (D / 4);
          for (int g0 = warp; g0 < ngroups; g0 += kTcBatch * nwarps) {
            float2 v[kTcBatch];
#pragma unroll
            for (int i = 0; i < kTcBatch; ++i) {
              const int g = g0 + i * nwarps;
              const int c = (g / (D / 4)) * 8 + (lane & 7), bp = (g % (D / 4)) * 4 + (lane >> 3);
              v[i] = (g < ngroups && c < nc) ? src[leg_addr(ct + c, bp, I, D) - soff] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < kTcBatch; ++i) {
              const int g = g0 + i * nwarps;
              if (g < ngroups) {
                const int c = (g / (D / 4)) * 8 + (lane & 7), bp = (g % (D / 4)) * 4 + (lane >> 3);
                tc_put(Ah, Al, c, bp, 64, v[i].x);
                tc_put(Ah, Al, c, D + bp, 64, conj * v[i].y);
              }
            }
          }
          tc::fence_async_smem();
          __syncthreads();
          if (tc_ok) {
            if (threadIdx.x == 0) {
              tc::fence_after_sync();
              tc_issue(tc::smem_u32(Ah), 32768u, tc::smem_u32(Wh), 16384u, 64, 64, tmem, idesc, true);
              tc::mma_commit(&bar);
            }
            tc_ok = tc_wait(&bar, phase, kTcWaitCycles);
          }
          if (tc_ok) {  // warps w and w + 4 read TMEM lanes 32 (w % 4) ..: each takes 16 of the 32 b
            tc::fence_after_sync();
            const int c = threadIdx.x & 127;
            for (int bb = (threadIdx.x >> 7) * 16; bb < D; bb += 16 * (blockDim.x >> 7)) {
              float re[16], im[16];
              tc::tmem_ld16(tmem + ((uint32_t)(32 * (c >> 5)) << 16) + (uint32_t)bb, re);
              tc::tmem_ld16(tmem + ((uint32_t)(32 * (c >> 5)) << 16) + (uint32_t)(D + bb), im);
              if (c < nc) {
#pragma unroll
                for (int q = 0; q < 16; ++q) X[leg_addr(ct + c, bb + q, I, D) - off] = make_float2(re[q], im[q]);
              }
            }
          }
          tc::fence_before_sync();
          __syncthreads();
        }
      }
      // Gram over the columns of leg p, 64 at a time (rows a and D + a of both operands: the
      // real and imaginary parts; K = the column, zero-padded to a multiple of 8)
      for (int cg = c0; cg < c1; cg += 64) {
        const int nc = c1 - cg < 64 ? c1 - cg : 64, nc8 = (nc + 7) & ~7;
        const int ngroups = (D / 8) * (nc8 / 4);
        for (int g0 = warp; g0 < ngroups; g0 += kTcBatch * nwarps) {  // a thread's loads in flight together
          float2 va[kTcBatch], vb[kTcBatch];
#pragma unroll
          for (int i = 0; i < kTcBatch; ++i) {
            const int g = g0 + i * nwarps;
            const int a = (g % (D / 8)) * 8 + (lane & 7), cc = (g / (D / 8)) * 4 + (lane >> 3);
            va[i] = make_float2(0.f, 0.f);
            vb[i] = va[i];
            if (g < ngroups && cc < nc) {
              const int64_t ad = leg_addr(cg + cc, a, Ip, D);
              va[i] = G[ad];
              vb[i] = nl == 0 ? make_float2(va[i].x, -va[i].y) : X[ad - off];
            }
          }
#pragma unroll
          for (int i = 0; i < kTcBatch; ++i) {
            const int g = g0 + i * nwarps;
            if (g >= ngroups) continue;
            const int a = (g % (D / 8)) * 8 + (lane & 7), cc = (g / (D / 8)) * 4 + (lane >> 3);
            tc_put(gAh, gAl, a, cc, 64, va[i].x);
            tc_put(gAh, gAl, D + a, cc, 64, va[i].y);
            tc_put(gBh, gBl, a, cc, 64, vb[i].x);
            tc_put(gBh, gBl, D + a, cc, 64, vb[i].y);
          }
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tc_ok) {
          if (threadIdx.x == 0) {
            tc::fence_after_sync();
            tc_issue(tc::smem_u32(gAh), 32768u, tc::smem_u32(gBh), 16384u, nc8, 64, tmem + 64u, idesc, fresh_gram);
            tc::mma_commit(&bar);
          }
          tc_ok = tc_wait(&bar, phase, kTcWaitCycles);
        }
        fresh_gram = false;
      }
    }
    // read the Gram (threads 0..63: rows (re/im, a)), combine and store the upper triangle mirrored
    if (threadIdx.x < 64 && tc_ok) {
      tc::fence_after_sync();
      const int m = threadIdx.x;
      for (int cb = 0; cb < 2 * D; cb += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * (m >> 5)) << 16) + 64u + (uint32_t)cb, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) dump[m * (2 * D + 1) + cb + q] = v[q];
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
      const int a = idx / D, b = idx - a * D;
      if (a > b) continue;
      const float* ra = dump + a * (2 * D + 1);
      const float* ia = dump + (D + a) * (2 * D + 1);
      const double re = (double)__fsub_rn(ra[b], ia[D + b]);
      const double im = (double)__fadd_rn(ra[D + b], ia[b]);
      if (a == b) {
        Mo[a * D + a] = make_double2(re, 0.0);
      } else {
        Mo[a * D + b] = make_double2(re, im);
        Mo[b * D + a] = make_double2(re, -im);
      }
    }
    __syncthreads();
    bp_message_finish(tk, Mo, lam, msg_in, msg_out, D, support_cut, my_res, bad);
  }
  const double r = block_max(my_res, red);
  const int any_bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    if (!tc_ok) atomicOr(flags, GPEPS_FLAG_TIMEOUT);
    if (any_bad) {
      atomicOr(flags, GPEPS_FLAG_NUMERIC);
      atomicMax(residual, 0x7FF0000000000000ULL);  // +inf
    } else {
      atomicMax(residual, (unsigned long long)__double_as_longlong(r));
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 128u);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBpThreads) bp_apply_kernel(const BpSiteTask* __restrict__ sites, int n_sites,
                                                              V2<T>* gamma, const double2* __restrict__ P, int D) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  const int ld = D + 1;
  // Storage-precision arithmetic when the site's gauge matrices are well
  // conditioned; FP64 otherwise (a gauge matrix with large entries, rounded to
  // FP32, would spoil the cancellation of the product)
  double2* M64 = reinterpret_cast<double2*>(smem);  // [D][D + 1]
  double2* tile64 = M64 + D * ld;                    // [32][D + 1]
  V2<T>* M32 = reinterpret_cast<V2<T>*>(smem);
  V2<T>* tile32 = M32 + D * ld;
  for (int t = blockIdx.x; t < n_sites; t += gridDim.x) {
    const BpSiteTask st = sites[t];
    V2<T>* G = gamma + st.off;
    int ncols = 2;
    for (int k = 1; k < st.deg; ++k) ncols *= D;
    bool low = false;
    if constexpr (sizeof(T) == 4) {
      double mx = 0.0;
      const double2* P0 = P + (int64_t)st.h0 * D * D;
      for (int idx = threadIdx.x; idx < st.deg * D * D; idx += blockDim.x)
        mx = fmax(mx, fmax(fabs(P0[idx].x), fabs(P0[idx].y)));
      low = block_max(mx, red) <= kApplyF32Max;  // thread 0 holds the maximum
      if (threadIdx.x == 0) red[0] = low ? 1.0 : 0.0;
      __syncthreads();
      low = red[0] != 0.0;
      __syncthreads();
    }
    for (int p = 0; p < st.deg; ++p) {
      // (G x_p P)[.., k, ..] = sum_a G[.., a, ..] P[a][k]: M[k][a] = P[a][k]
      const double2* Pp = P + (int64_t)(st.h0 + p) * D * D;
      for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
        const int a = idx / D, k = idx - a * D;
        if (low) M32[k * ld + a] = mk<T>((T)Pp[idx].x, (T)Pp[idx].y);
        else M64[k * ld + a] = Pp[idx];
      }
      __syncthreads();
      int I = 1;
      for (int k = p + 1; k < st.deg; ++k) I *= D;
      if (low) leg_product<T, T, false, 32 * kMaxD / kBpThreads>(G, 0, G, 0, 0, ncols, I, D, M32, tile32);
      else leg_product<T, double, false, 0>(G, 0, G, 0, 0, ncols, I, D, M64, tile64);
    }
  }
}

// ---------------------------------------------------------------- gauge
// The square roots of G run in the arithmetic R: FP64 for complex128, FP32 for
// complex64 storage (whose messages are FP32-accurate; the gauge preserves the
// state whatever the accuracy of the roots, which only sets how close the new
// gauge is to the BP fixed point).  Messages in, gauge matrices and lambda out
// are FP64.
template <typename R>
struct GaugeSmall {
  R rc[64], rs[64];
  V2<R> re[64];
  int rp[64], rq[64];
  int iflag[160];
  double w[64], winv[64];
  double S[64], lamv[64];
  int order[64];
  double scal[4];
};

template <typename R> struct GaugeTol;
template <> struct GaugeTol<double> {
  static constexpr double tol = 1e-15, floor = 4.4e-16;  // |a_pq| <= tol sqrt(a_pp a_qq) or <= floor * trace
};
template <> struct GaugeTol<float> {  // warm start only (FP64 sweeps finish)
  static constexpr double tol = 1e-6, floor = 2e-7;
};
constexpr int kGaugeSweeps = 40;

// Jacobi eigenproblem of the n x n Hermitian matrix in Am (destroyed), eigenvectors in W.
template <typename R>
__device__ void gauge_eig(V2<R>* Am, V2<R>* W, int n, GaugeSmall<R>& sm, int* flags) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int a = idx / n;
    W[idx] = mk<R>(a * n + a == idx ? R(1) : R(0), R(0));
  }
  for (int i = threadIdx.x; i < 160; i += blockDim.x) sm.iflag[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int a = 0; a < n; ++a) tr += (double)Am[a * n + a].x;
    sm.scal[0] = tr;
  }
  __syncthreads();
  const R floor_abs = (R)(GaugeTol<R>::floor * fmax(sm.scal[0], 0.0));
  const int sw = jacobi_hermitian<R, sizeof(R) == 4>(HermFull<R>{Am, n}, W, n, n, (R)GaugeTol<R>::tol, floor_abs,
                                                     kGaugeSweeps, sm.rc, sm.rs, sm.re, sm.rp, sm.rq, sm.iflag,
                                                     nullptr, nullptr);
  if (threadIdx.x == 0 && sw > kGaugeSweeps) atomicOr(flags, GPEPS_FLAG_NOCONV);
  __syncthreads();
}

// Eigenproblem of the FP64 Hermitian n x n matrix Hm (row stride n, left intact):
// on return region[0, nn) holds W^H Hm W, diagonal to the Jacobi thresholds (the
// eigenvalues on its diagonal), and region[nn, 2nn) the eigenvectors W, FP64 and
// orthonormal.  region: 2 n x n FP64 complex; tmp: n x n FP64 complex of scratch.
// R = double: FP64 Jacobi on a copy.  R = float: warm start by FP32 Jacobi on a
// rounded copy, its eigenvectors made orthonormal in FP64 by one Newton-Schulz step
// (W <- W (3 - W^H W) / 2), Hm rotated into that basis in FP64 (nearly diagonal)
// and FP64 sweeps to finish, accumulated into W.  Either way W is orthonormal to
// FP64 accuracy, so the gauge built from it keeps the state exactly whatever the
// conditioning of Hm (FP32 eigenvectors alone are orthonormal only to ~1e-7).
template <typename R>
__device__ void eig_warm(const double2* Hm, int n, double2* region, double2* tmp, GaugeSmall<R>& sm,
                         GaugeSmall<double>& sm64, int* flags) {
  const int nn = n * n;
  double2* A64 = region;      // FP64 matrix: [0, 16 nn) bytes
  double2* W64 = region + nn;  // FP64 eigenvectors: [16 nn, 32 nn) bytes
  if constexpr (sizeof(R) == 8) {
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) A64[idx] = Hm[idx];
    __syncthreads();
    gauge_eig<double>(A64, W64, n, sm64, flags);
  } else {
    V2<R>* Am = reinterpret_cast<V2<R>*>(region);  // FP32 pair: [0, 8 nn) and [8 nn, 16 nn) bytes
    V2<R>* W = Am + nn;
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) Am[idx] = mk<R>((R)Hm[idx].x, (R)Hm[idx].y);
    __syncthreads();
    gauge_eig<R>(Am, W, n, sm, flags);
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x)
      W64[idx] = make_double2((double)W[idx].x, (double)W[idx].y);
    __syncthreads();
    // orthonormalise: S = W^H W (in A64), then W <- 1.5 W - 0.5 W S (W S in tmp)
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int a = idx / n, b = idx - a * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < n; ++k) fma_conj<double>(acc, W64[k * n + a], W64[k * n + b]);
      A64[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int a = idx / n, b = idx - a * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < n; ++k) fma_c<double>(acc, W64[a * n + k], A64[k * n + b]);
      tmp[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const double2 w = W64[idx], t = tmp[idx];
      W64[idx] = make_double2(1.5 * w.x - 0.5 * t.x, 1.5 * w.y - 0.5 * t.y);
    }
    __syncthreads();
    // Hm W (in tmp), then A = W^H Hm W (in A64)
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int a = idx / n, l = idx - a * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int b = 0; b < n; ++b) fma_c<double>(acc, Hm[a * n + b], W64[b * n + l]);
      tmp[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int k = idx / n, l = idx - k * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int a = 0; a < n; ++a) fma_conj<double>(acc, W64[a * n + k], tmp[a * n + l]);
      A64[idx] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 160; i += blockDim.x) sm64.iflag[i] = 0;
    if (threadIdx.x == 0) {
      double tr = 0.0;
      for (int k = 0; k < n; ++k) tr += A64[k * n + k].x;
      sm64.scal[0] = tr;
    }
    __syncthreads();
    const int sw = jacobi_hermitian<double, false>(HermFull<double>{A64, n}, W64, n, n, GaugeTol<double>::tol,
                                                   GaugeTol<double>::floor * fmax(sm64.scal[0], 0.0),
                                                   kGaugeSweeps, sm64.rc, sm64.rs, sm64.re, sm64.rp, sm64.rq,
                                                   sm64.iflag, nullptr, nullptr);
    if (threadIdx.x == 0 && sw > kGaugeSweeps) atomicOr(flags, GPEPS_FLAG_NOCONV);
    __syncthreads();
  }
}

// Rt = G^{1/2} and Rinv = (G^{1/2})^+ of G = conj(m) (m: D x D FP64 message; n >= D,
// padded with zeros), both FP64, through eig_warm (G is staged in Rt, Rinv is its
// scratch until both are overwritten at the end).
template <typename R>
__device__ void gauge_root(const double2* m, int D, int n, double2* region, double2* Rt, double2* Rinv,
                           GaugeSmall<R>& sm, GaugeSmall<double>& sm64, int* flags) {
  const int nn = n * n;
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int a = idx / n, b = idx - a * n;
    double2 v = make_double2(0.0, 0.0);
    if (a < D && b < D) {
      const double2 x = m[a * D + b];
      v = make_double2(x.x, -x.y);
    }
    Rt[idx] = v;
  }
  __syncthreads();
  eig_warm<R>(Rt, n, region, Rinv, sm, sm64, flags);
  const double2* A64 = region;
  const double2* W64 = region + nn;
  if (threadIdx.x == 0) {
    double wmax = 0.0;
    for (int k = 0; k < n; ++k) wmax = fmax(wmax, A64[k * n + k].x);
    for (int k = 0; k < n; ++k) {
      const double wk = A64[k * n + k].x;
      const bool keep = wk > kBpGramCut * wmax && wk > 0.0;
      sm64.w[k] = keep ? sqrt(wk) : 0.0;
      sm64.winv[k] = keep ? 1.0 / sqrt(wk) : 0.0;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int a = idx / n, b = idx - a * n;
    double2 r = make_double2(0.0, 0.0), ri = make_double2(0.0, 0.0);
    for (int k = 0; k < n; ++k) {
      const double2 u = W64[a * n + k], v = W64[b * n + k];
      const double2 uv = make_double2(u.x * v.x + u.y * v.y, u.y * v.x - u.x * v.y);  // u conj(v)
      r.x = fma(sm64.w[k], uv.x, r.x);
      r.y = fma(sm64.w[k], uv.y, r.y);
      ri.x = fma(sm64.winv[k], uv.x, ri.x);
      ri.y = fma(sm64.winv[k], uv.y, ri.y);
    }
    Rt[idx] = r;
    Rinv[idx] = ri;
  }
  __syncthreads();
}

// 128-thread CTAs, four per SM.  The three eigenproblems (both G and C C^H) are
// warm-started in the arithmetic R (FP32 for complex64 storage) and finished in
// FP64 (eig_warm); the roots, C, the eigenproblem of C C^H (which sets
// lambda' and resolves the smallest Schmidt directions) and the gauge matrices
// are FP64.  Slot layout (n x n FP64 complex each): Ri, Ri^+, Rj, Rj^+, C; the
// Jacobi work space (2 n x n) in dynamic shared memory when it fits (in_smem),
// else after C in the slot.
template <typename R>
__global__ void __launch_bounds__(kGaugeThreads, 4) bp_gauge_kernel(const BpEdgeTask* __restrict__ edges,
                                                                   int n_edges, const double2* __restrict__ msgs,
                                                                   double* lam, double2* P, double2* scratch,
                                                                   int64_t slot_elems, int D, int in_smem,
                                                                   int* flags) {
  extern __shared__ __align__(16) unsigned char gsmem[];
  __shared__ GaugeSmall<R> sm;
  __shared__ GaugeSmall<double> sm64;
  const int n = D + (D & 1);
  const int nn = n * n;
  double2* Ri = scratch + (int64_t)blockIdx.x * slot_elems;
  double2* Rii = Ri + nn;
  double2* Rj = Rii + nn;
  double2* Rji = Rj + nn;
  double2* C = Rji + nn;
  double2* Am = in_smem ? reinterpret_cast<double2*>(gsmem) : C + nn;
  double2* W = Am + nn;
  for (int e = blockIdx.x; e < n_edges; e += gridDim.x) {
    const BpEdgeTask tk = edges[e];
    gauge_root<R>(msgs + (int64_t)tk.hi * D * D, D, n, Am, Ri, Rii, sm, sm64, flags);
    gauge_root<R>(msgs + (int64_t)tk.hj * D * D, D, n, Am, Rj, Rji, sm, sm64, flags);
    for (int k = threadIdx.x; k < n; k += blockDim.x) sm64.lamv[k] = k < D ? lam[tk.lam + k] : 0.0;
    __syncthreads();
    // C = Ri diag(lambda) Rj^T
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int a = idx / n, b = idx - a * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int c = 0; c < n; ++c) {
        const double2 x = Ri[a * n + c], y = Rj[b * n + c];
        const double l = sm64.lamv[c];
        acc.x = fma(l, x.x * y.x - x.y * y.y, acc.x);
        acc.y = fma(l, x.x * y.y + x.y * y.x, acc.y);
      }
      C[idx] = acc;
    }
    __syncthreads();
    // H = C C^H (in Ri, free now), its eigenvectors U (in W), warm-started like the roots
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int a = idx / n, b = idx - a * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int c = 0; c < n; ++c) fma_conj<double>(acc, C[b * n + c], C[a * n + c]);
      Ri[idx] = acc;
    }
    __syncthreads();
    eig_warm<R>(Ri, n, Am, Rj, sm, sm64, flags);
    // Y = C^T conj(U) (in Am, whose eigenvalues are not used), S_k = ||Y[:, k]||
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int a = idx / n, k = idx - a * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int b = 0; b < n; ++b) fma_conj<double>(acc, W[b * n + k], C[b * n + a]);
      Am[idx] = acc;
    }
    __syncthreads();
    double2* Y = Am;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      double s2 = 0.0;
      for (int a = 0; a < n; ++a) {
        const double2 y = Y[a * n + k];
        s2 += y.x * y.x + y.y * y.y;
      }
      sm64.S[k] = sqrt(s2);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      int rank = 0;
      const double sk = sm64.S[k];
      for (int j = 0; j < n; ++j) rank += (sm64.S[j] > sk) || (sm64.S[j] == sk && j < k);
      sm64.order[rank] = k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double nrm2 = 0.0;
      for (int kk = 0; kk < D; ++kk) nrm2 += sm64.S[sm64.order[kk]] * sm64.S[sm64.order[kk]];
      sm64.scal[1] = sqrt(nrm2);
      sm64.scal[2] = sm64.S[sm64.order[0]];
    }
    __syncthreads();
    const double nrm = sm64.scal[1], smax = sm64.scal[2];
    const bool ok = nrm > 0.0 && isfinite(nrm);
    if (threadIdx.x == 0 && !ok) atomicOr(flags, GPEPS_FLAG_NUMERIC);
    double2* Pi = P + (int64_t)tk.hi * D * D;
    double2* Pj = P + (int64_t)tk.hj * D * D;
    for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
      const int a = idx / D, kk = idx - a * D;
      const int k = sm64.order[kk];
      const double sk = sm64.S[k];
      double2 pi = make_double2(0.0, 0.0), pj = make_double2(0.0, 0.0);
      if (!ok) {  // leave the state as it is
        pi = make_double2(a == kk ? 1.0 : 0.0, 0.0);
        pj = pi;
      } else if (sk > kLambdaCut * smax) {
        for (int b = 0; b < n; ++b) {
          fma_c<double>(pi, Rii[a * n + b], W[b * n + k]);
          fma_c<double>(pj, Rji[a * n + b], Y[b * n + k]);
        }
        pj.x /= sk;
        pj.y /= sk;
      }
      Pi[idx] = pi;
      Pj[idx] = pj;
    }
    if (ok)
      for (int kk = threadIdx.x; kk < D; kk += blockDim.x) lam[tk.lam + kk] = sm64.S[sm64.order[kk]] / nrm;
    __syncthreads();
  }
}

}  // namespace

template <typename T>
size_t BpLaunch<T>::message_smem(int D) {
  return (size_t)(D + 64) * (D + 1) * sizeof(V2<T>) + (size_t)D * D * sizeof(double2);
}

static size_t apply_smem(int D) { return (size_t)(D + 32) * (D + 1) * sizeof(double2); }
static size_t gauge_smem(int D) {
  const int n = D + (D & 1);
  const size_t b = (size_t)2 * n * n * sizeof(double2);
  return b <= kGaugeSmemMax ? b : 0;
}

template <typename T>
cudaError_t BpLaunch<T>::init() {
  cudaError_t e = cudaFuncSetAttribute(bp_message_kernel<T, kGramPerSmall>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)message_smem(32));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(bp_message_kernel<T, kGramPerLarge>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)message_smem(kMaxD));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(bp_gauge_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGaugeSmemMax);
  if (e != cudaSuccess) return e;
  if constexpr (sizeof(T) == 4) {
    e = cudaFuncSetAttribute(bp_message_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BpTcSmem::total);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(bp_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)apply_smem(kMaxD));
}

template <typename T>
int BpLaunch<T>::resident(int D) {
  int n = 0;
  const cudaError_t e =
      D <= 32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bp_message_kernel<T, kGramPerSmall>, kBpMsgThreads,
                                                              message_smem(D))
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bp_message_kernel<T, kGramPerLarge>, kBpMsgThreads,
                                                              message_smem(D));
  return (e == cudaSuccess && n > 0) ? n : 1;
}

template <typename T>
cudaError_t BpLaunch<T>::identity(double2* msgs, int n_half, int D, cudaStream_t st) {
  const int64_t n = (int64_t)n_half * D * D;
  if (n == 0) return cudaSuccess;
  bp_identity_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(msgs, n, D);
  return cudaGetLastError();
}

template <typename T>
cudaError_t BpLaunch<T>::message(const BpMsgTask* tasks, int n_tasks, const void* gamma, const double* lam,
                                 const double2* msg_in, double2* msg_out, void* scratch, int64_t slot_elems, int D,
                                 unsigned long long* residual, int* flags, int n_ctas, cudaStream_t st,
                                 bool tensor) {
  if (n_tasks == 0) return cudaSuccess;
  int grid = n_tasks < n_ctas ? n_tasks : n_ctas;
  const double cut = sizeof(T) == 4 ? kBpSupportCutF32 : kLambdaCut;
  if (tensor) {
    if (sizeof(T) != 4 || D != kBpTcD) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (grid > 2 * sms) grid = 2 * sms;  // two 112 KB CTAs per SM; the scratch has n_ctas >= grid slots
    if constexpr (sizeof(T) == 4)
      bp_message_tc_kernel<<<grid, kBpTcThreads, BpTcSmem::total, st>>>(
          tasks, n_tasks, static_cast<const float2*>(gamma), lam, msg_in, msg_out, static_cast<float2*>(scratch),
          slot_elems, cut, residual, flags);
    return cudaGetLastError();
  }
  if (D <= 32)
    bp_message_kernel<T, kGramPerSmall><<<grid, kBpMsgThreads, message_smem(D), st>>>(
        tasks, n_tasks, static_cast<const V2<T>*>(gamma), lam, msg_in, msg_out, static_cast<V2<T>*>(scratch),
        slot_elems, D, cut, residual, flags);
  else
    bp_message_kernel<T, kGramPerLarge><<<grid, kBpMsgThreads, message_smem(D), st>>>(
        tasks, n_tasks, static_cast<const V2<T>*>(gamma), lam, msg_in, msg_out, static_cast<V2<T>*>(scratch),
        slot_elems, D, cut, residual, flags);
  return cudaGetLastError();
}

template <typename T>
cudaError_t BpLaunch<T>::apply(const BpSiteTask* sites, int n_sites, void* gamma, const double2* P, int D,
                               cudaStream_t st) {
  if (n_sites == 0) return cudaSuccess;
  bp_apply_kernel<T><<<n_sites, kBpThreads, apply_smem(D), st>>>(sites, n_sites, static_cast<V2<T>*>(gamma), P, D);
  return cudaGetLastError();
}

template <typename T>
cudaError_t BpLaunch<T>::gauge(const BpEdgeTask* edges, int n_edges, const double2* msgs, double* lam, double2* P,
                               double2* scratch, int64_t slot_elems, int D, int* flags, int n_ctas, cudaStream_t st) {
  if (n_edges == 0) return cudaSuccess;
  const size_t smem = gauge_smem(D);
  const int grid = n_edges < n_ctas ? n_edges : n_ctas;
  bp_gauge_kernel<T><<<grid, kGaugeThreads, smem, st>>>(edges, n_edges, msgs, lam, P, scratch, slot_elems, D,
                                                        smem > 0 ? 1 : 0, flags);
  return cudaGetLastError();
}

template struct BpLaunch<float>;
template struct BpLaunch<double>;

}  // namespace gpeps
