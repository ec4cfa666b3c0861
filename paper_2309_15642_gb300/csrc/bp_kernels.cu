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
//   gauge    one CTA per edge, FP64: the Hermitian square root R and pseudo-
//            inverse R^+ of G = conj(m) at both ends (Jacobi eigenproblems),
//            C = R_i diag(lambda) R_j^T, its left singular vectors U from the
//            eigenproblem of C C^H, and Y = C^T conj(U), whose column norms are the
//            singular values S (C = U Y^T holds exactly whatever the accuracy of
//            the smallest eigenvalues).  lambda' = S / ||S||, and the gauge
//            matrices R_i^+ U and R_j^+ Y / S of the two half-edges.
//   apply    one CTA per site: Gamma_i <- Gamma_i x_p P_p on every leg p, in place,
//            in FP64 arithmetic rounded once to the storage type.
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

namespace gpeps {

namespace {

constexpr int kGramPer = (kMaxD * (kMaxD + 1) / 2 + kBpThreads - 1) / kBpThreads;  // upper-triangle pairs per thread

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

// dst(c, b) = sum_b' M[b][b'] src(c, b') over the ncols columns of the leg with
// stride I (conj(src) when kConj), in the arithmetic of TC (src and dst hold TS).
// M: shared [D][D + 1]; tile: shared [32][D + 1], both TC.  dst may be src: a
// tile is read completely before any of it is written.
template <typename TS, typename TC, bool kConj>
__device__ void leg_product(V2<TS>* dst, const V2<TS>* src, int ncols, int I, int D, const V2<TC>* M,
                            V2<TC>* tile) {
  const int ld = D + 1;
  for (int c0 = 0; c0 < ncols; c0 += 32) {
    const int nc = min(32, ncols - c0);
    for (int idx = threadIdx.x; idx < 32 * D; idx += blockDim.x) {
      int j, b;
      tile_pos(idx, I, D, j, b);
      if (j < nc) {
        const V2<TS> v = src[leg_addr(c0 + j, b, I, D)];
        tile[j * ld + b] = mk<TC>((TC)v.x, kConj ? -(TC)v.y : (TC)v.y);
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * D; idx += blockDim.x) {
      const int b = idx >> 5, j = idx & 31;
      if (j < nc) {
        V2<TC> acc = mk<TC>(0, 0);
        const V2<TC>* mr = M + b * ld;
        const V2<TC>* tr = tile + j * ld;
        for (int k = 0; k < D; ++k) fma_c<TC>(acc, mr[k], tr[k]);
        dst[leg_addr(c0 + j, b, I, D)] = mk<TS>((TS)acc.x, (TS)acc.y);
      }
    }
    __syncthreads();
  }
}

// Mo[a][a'] = sum_c A(c, a) B(c, a') (B = conj(A) when kConjB) for a <= a', the
// lower triangle its conjugate mirror; FP64 result in shared Mo [D][D].
template <typename T, bool kConjB>
__device__ void leg_gram(const V2<T>* A, const V2<T>* B, int ncols, int I, int D, V2<T>* tA, V2<T>* tB,
                         double2* Mo) {
  const int ld = D + 1;
  const int npairs = D * (D + 1) / 2;
  int pa[kGramPer], pb[kGramPer];
  V2<T> acc[kGramPer];
#pragma unroll
  for (int k = 0; k < kGramPer; ++k) {
    const int u = threadIdx.x + k * blockDim.x;
    int r = 0, c = 0;
    if (u < npairs) {
      r = (int)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
      while (r * (r + 1) / 2 > u) --r;
      while ((r + 1) * (r + 2) / 2 <= u) ++r;
      c = u - r * (r + 1) / 2;
    }
    pa[k] = c;  // a <= a'
    pb[k] = r;
    acc[k] = mk<T>(0, 0);
  }
  for (int c0 = 0; c0 < ncols; c0 += 32) {
    const int nc = min(32, ncols - c0);
    for (int idx = threadIdx.x; idx < 32 * D; idx += blockDim.x) {
      int j, b;
      tile_pos(idx, I, D, j, b);
      V2<T> va = mk<T>(0, 0), vb = mk<T>(0, 0);
      if (j < nc) {
        const int64_t ad = leg_addr(c0 + j, b, I, D);
        va = A[ad];
        vb = B[ad];
        if (kConjB) vb.y = -vb.y;
      }
      tA[j * ld + b] = va;
      tB[j * ld + b] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGramPer; ++k) {
      if (threadIdx.x + k * blockDim.x < npairs) {
        const V2<T>* ta = tA + pa[k];
        const V2<T>* tb = tB + pb[k];
        for (int j = 0; j < 32; ++j) fma_c<T>(acc[k], ta[j * ld], tb[j * ld]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < kGramPer; ++k) {
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
  __syncthreads();
}

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

template <typename T>
__global__ void __launch_bounds__(kBpThreads) bp_message_kernel(const BpMsgTask* __restrict__ tasks, int n_tasks,
                                                                const V2<T>* __restrict__ gamma,
                                                                const double* __restrict__ lam,
                                                                const double2* __restrict__ msg_in,
                                                                double2* __restrict__ msg_out, V2<T>* scratch,
                                                                int64_t slot_elems, int D, double support_cut,
                                                                unsigned long long* residual, int* flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ double s_trace, s_cut;
  const int ld = D + 1;
  V2<T>* M = reinterpret_cast<V2<T>*>(smem);  // [D][D + 1]
  V2<T>* tA = M + D * ld;                      // [32][D + 1]
  V2<T>* tB = tA + 32 * ld;                    // [32][D + 1]
  double2* Mo = reinterpret_cast<double2*>(tB + 32 * ld);  // [D][D]
  V2<T>* X = scratch + (int64_t)blockIdx.x * slot_elems;
  double my_res = 0.0;
  bool bad = false;
  for (int t = blockIdx.x; t < n_tasks; t += gridDim.x) {
    const BpMsgTask tk = tasks[t];
    const V2<T>* G = gamma + tk.off;
    const int z = tk.deg, p = tk.leg;
    int ncols = 2;
    for (int k = 1; k < z; ++k) ncols *= D;
    bool first = true;
    for (int q = 0; q < z; ++q) {
      if (q == p) continue;
      const double* lq = lam + tk.lam[q];
      const double2* mi = msg_in + (int64_t)tk.in[q] * D * D;
      for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
        const int b = idx / D, bb = idx - b * D;
        const double2 v = mi[idx];
        const double w = lq[b] * lq[bb];
        M[b * ld + bb] = mk<T>((T)(v.x * w), (T)(v.y * w));
      }
      __syncthreads();
      int I = 1;
      for (int k = q + 1; k < z; ++k) I *= D;
      if (first) leg_product<T, T, true>(X, G, ncols, I, D, M, tA);
      else leg_product<T, T, false>(X, X, ncols, I, D, M, tA);
      first = false;
    }
    int Ip = 1;
    for (int k = p + 1; k < z; ++k) Ip *= D;
    if (first) leg_gram<T, true>(G, G, ncols, Ip, D, tA, tB, Mo);
    else leg_gram<T, false>(G, X, ncols, Ip, D, tA, tB, Mo);
    // the support of lambda_e: entries k with lambda_e[k] <= support_cut * max are zero
    const double* le = lam + tk.lam[p];
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

template <typename T>
__global__ void __launch_bounds__(kBpThreads) bp_apply_kernel(const BpSiteTask* __restrict__ sites, int n_sites,
                                                              V2<T>* gamma, const double2* __restrict__ P, int D) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ld = D + 1;
  // FP64 arithmetic whatever the storage: the gauge matrices of nearly null
  // directions are large, and rounding them to FP32 would spoil the cancellation
  double2* M = reinterpret_cast<double2*>(smem);  // [D][D + 1]
  double2* tile = M + D * ld;                      // [32][D + 1]
  for (int t = blockIdx.x; t < n_sites; t += gridDim.x) {
    const BpSiteTask st = sites[t];
    V2<T>* G = gamma + st.off;
    int ncols = 2;
    for (int k = 1; k < st.deg; ++k) ncols *= D;
    for (int p = 0; p < st.deg; ++p) {
      // (G x_p P)[.., k, ..] = sum_a G[.., a, ..] P[a][k]: M[k][a] = P[a][k]
      const double2* Pp = P + (int64_t)(st.h0 + p) * D * D;
      for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
        const int a = idx / D, k = idx - a * D;
        M[k * ld + a] = Pp[idx];
      }
      __syncthreads();
      int I = 1;
      for (int k = p + 1; k < st.deg; ++k) I *= D;
      leg_product<T, double, false>(G, G, ncols, I, D, M, tile);
    }
  }
}

// ---------------------------------------------------------------- gauge (FP64)
struct GaugeSmall {
  double rc[64], rs[64];
  double2 re[64];
  int rp[64], rq[64];
  int iflag[160];
  double w[64], S[64], lamv[64];
  int order[64];
  double scal[4];
};

constexpr double kGaugeTol = 1e-15;      // Jacobi: |a_pq| <= tol sqrt(a_pp a_qq) ...
constexpr double kGaugeFloor = 4.4e-16;  // ... or <= floor * trace
constexpr int kGaugeSweeps = 40;

// Jacobi eigenproblem of the n x n Hermitian matrix in Am (destroyed), eigenvectors in W.
__device__ void gauge_eig(double2* Am, double2* W, int n, GaugeSmall& sm, int* flags) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int a = idx / n;
    W[idx] = make_double2(a * n + a == idx ? 1.0 : 0.0, 0.0);
  }
  for (int i = threadIdx.x; i < 160; i += blockDim.x) sm.iflag[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int a = 0; a < n; ++a) tr += Am[a * n + a].x;
    sm.scal[0] = tr;
  }
  __syncthreads();
  const double floor_abs = kGaugeFloor * fmax(sm.scal[0], 0.0);
  const int sw = jacobi_hermitian<double, false>(HermFull<double>{Am, n}, W, n, n, kGaugeTol, floor_abs,
                                                 kGaugeSweeps, sm.rc, sm.rs, sm.re, sm.rp, sm.rq, sm.iflag,
                                                 nullptr, nullptr);
  if (threadIdx.x == 0 && sw > kGaugeSweeps) atomicOr(flags, GPEPS_FLAG_NOCONV);
  __syncthreads();
}

// R = G^{1/2} and Rinv = (G^{1/2})^+ of G = conj(m) (m: D x D message; n >= D, padded with zeros).
__device__ void gauge_root(const double2* m, int D, int n, double2* Am, double2* W, double2* R, double2* Rinv,
                           GaugeSmall& sm, int* flags) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int a = idx / n, b = idx - a * n;
    double2 v = make_double2(0.0, 0.0);
    if (a < D && b < D) {
      const double2 x = m[a * D + b];
      v = make_double2(x.x, -x.y);
    }
    Am[idx] = v;
  }
  __syncthreads();
  gauge_eig(Am, W, n, sm, flags);
  if (threadIdx.x == 0) {
    double wmax = 0.0;
    for (int k = 0; k < n; ++k) wmax = fmax(wmax, Am[k * n + k].x);
    for (int k = 0; k < n; ++k) {
      const double wk = Am[k * n + k].x;
      const bool keep = wk > kBpGramCut * wmax && wk > 0.0;
      sm.w[k] = keep ? sqrt(wk) : 0.0;
      sm.S[k] = keep ? 1.0 / sqrt(wk) : 0.0;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int a = idx / n, b = idx - a * n;
    double2 r = make_double2(0.0, 0.0), ri = make_double2(0.0, 0.0);
    for (int k = 0; k < n; ++k) {
      const double2 u = W[a * n + k], v = W[b * n + k];
      const double2 uv = make_double2(u.x * v.x + u.y * v.y, u.y * v.x - u.x * v.y);  // u conj(v)
      r.x = fma(sm.w[k], uv.x, r.x);
      r.y = fma(sm.w[k], uv.y, r.y);
      ri.x = fma(sm.S[k], uv.x, ri.x);
      ri.y = fma(sm.S[k], uv.y, ri.y);
    }
    R[idx] = r;
    Rinv[idx] = ri;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kBpThreads) bp_gauge_kernel(const BpEdgeTask* __restrict__ edges, int n_edges,
                                                              const double2* __restrict__ msgs, double* lam,
                                                              double2* P, double2* scratch, int64_t slot_elems,
                                                              int D, int* flags) {
  __shared__ GaugeSmall sm;
  const int n = D + (D & 1);
  const int nn = n * n;
  double2* Am = scratch + (int64_t)blockIdx.x * slot_elems;
  double2* W = Am + nn;
  double2* Ri = W + nn;
  double2* Rii = Ri + nn;
  double2* Rj = Rii + nn;
  double2* Rji = Rj + nn;
  double2* C = Rji + nn;
  for (int e = blockIdx.x; e < n_edges; e += gridDim.x) {
    const BpEdgeTask tk = edges[e];
    gauge_root(msgs + (int64_t)tk.hi * D * D, D, n, Am, W, Ri, Rii, sm, flags);
    gauge_root(msgs + (int64_t)tk.hj * D * D, D, n, Am, W, Rj, Rji, sm, flags);
    for (int k = threadIdx.x; k < n; k += blockDim.x) sm.lamv[k] = k < D ? lam[tk.lam + k] : 0.0;
    __syncthreads();
    // C = Ri diag(lambda) Rj^T
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int a = idx / n, b = idx - a * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int c = 0; c < n; ++c) {
        const double2 x = Ri[a * n + c], y = Rj[b * n + c];
        const double l = sm.lamv[c];
        acc.x = fma(l, x.x * y.x - x.y * y.y, acc.x);
        acc.y = fma(l, x.x * y.y + x.y * y.x, acc.y);
      }
      C[idx] = acc;
    }
    __syncthreads();
    // H = C C^H, its eigenvectors U (in W)
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int a = idx / n, b = idx - a * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int c = 0; c < n; ++c) fma_conj<double>(acc, C[b * n + c], C[a * n + c]);
      Am[idx] = acc;
    }
    __syncthreads();
    gauge_eig(Am, W, n, sm, flags);
    // Y = C^T conj(U) (in Ri), S_k = ||Y[:, k]||
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int a = idx / n, k = idx - a * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int b = 0; b < n; ++b) fma_conj<double>(acc, W[b * n + k], C[b * n + a]);
      Ri[idx] = acc;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      double s2 = 0.0;
      for (int a = 0; a < n; ++a) {
        const double2 y = Ri[a * n + k];
        s2 += y.x * y.x + y.y * y.y;
      }
      sm.S[k] = sqrt(s2);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      int rank = 0;
      const double sk = sm.S[k];
      for (int j = 0; j < n; ++j) rank += (sm.S[j] > sk) || (sm.S[j] == sk && j < k);
      sm.order[rank] = k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double nrm2 = 0.0;
      for (int kk = 0; kk < D; ++kk) nrm2 += sm.S[sm.order[kk]] * sm.S[sm.order[kk]];
      sm.scal[1] = sqrt(nrm2);
      sm.scal[2] = sm.S[sm.order[0]];
    }
    __syncthreads();
    const double nrm = sm.scal[1], smax = sm.scal[2];
    const bool ok = nrm > 0.0 && isfinite(nrm);
    if (threadIdx.x == 0 && !ok) atomicOr(flags, GPEPS_FLAG_NUMERIC);
    double2* Pi = P + (int64_t)tk.hi * D * D;
    double2* Pj = P + (int64_t)tk.hj * D * D;
    for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
      const int a = idx / D, kk = idx - a * D;
      const int k = sm.order[kk];
      const double sk = sm.S[k];
      double2 pi = make_double2(0.0, 0.0), pj = make_double2(0.0, 0.0);
      if (!ok) {  // leave the state as it is
        pi = make_double2(a == kk ? 1.0 : 0.0, 0.0);
        pj = pi;
      } else if (sk > kLambdaCut * smax) {
        for (int b = 0; b < n; ++b) {
          fma_c<double>(pi, Rii[a * n + b], W[b * n + k]);
          fma_c<double>(pj, Rji[a * n + b], Ri[b * n + k]);
        }
        pj.x /= sk;
        pj.y /= sk;
      }
      Pi[idx] = pi;
      Pj[idx] = pj;
    }
    if (ok)
      for (int kk = threadIdx.x; kk < D; kk += blockDim.x) lam[tk.lam + kk] = sm.S[sm.order[kk]] / nrm;
    __syncthreads();
  }
}

}  // namespace

template <typename T>
size_t BpLaunch<T>::message_smem(int D) {
  return (size_t)(D + 64) * (D + 1) * sizeof(V2<T>) + (size_t)D * D * sizeof(double2);
}

template <typename T>
cudaError_t BpLaunch<T>::init() {
  cudaError_t e = cudaFuncSetAttribute(bp_message_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)message_smem(kMaxD));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(bp_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)((kMaxD + 32) * (kMaxD + 1) * sizeof(double2)));
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
                                 unsigned long long* residual, int* flags, int n_ctas, cudaStream_t st) {
  if (n_tasks == 0) return cudaSuccess;
  const int grid = n_tasks < n_ctas ? n_tasks : n_ctas;
  bp_message_kernel<T><<<grid, kBpThreads, message_smem(D), st>>>(
      tasks, n_tasks, static_cast<const V2<T>*>(gamma), lam, msg_in, msg_out, static_cast<V2<T>*>(scratch),
      slot_elems, D, sizeof(T) == 4 ? kBpSupportCutF32 : kLambdaCut, residual, flags);
  return cudaGetLastError();
}

template <typename T>
cudaError_t BpLaunch<T>::apply(const BpSiteTask* sites, int n_sites, void* gamma, const double2* P, int D,
                               cudaStream_t st) {
  if (n_sites == 0) return cudaSuccess;
  const size_t smem = (size_t)(D + 32) * (D + 1) * sizeof(double2);
  bp_apply_kernel<T><<<n_sites, kBpThreads, smem, st>>>(sites, n_sites, static_cast<V2<T>*>(gamma), P, D);
  return cudaGetLastError();
}

cudaError_t bp_gauge(const BpEdgeTask* edges, int n_edges, const double2* msgs, double* lam, double2* P,
                     double2* scratch, int64_t slot_elems, int D, int* flags, int n_ctas, cudaStream_t st) {
  if (n_edges == 0) return cudaSuccess;
  const int grid = n_edges < n_ctas ? n_edges : n_ctas;
  bp_gauge_kernel<<<grid, kBpThreads, 0, st>>>(edges, n_edges, msgs, lam, P, scratch, slot_elems, D, flags);
  return cudaGetLastError();
}

template struct BpLaunch<float>;
template struct BpLaunch<double>;

}  // namespace gpeps
