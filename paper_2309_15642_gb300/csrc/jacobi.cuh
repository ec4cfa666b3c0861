// Complex helpers and the parallel cyclic Jacobi eigensolver for Hermitian
// matrices, shared by the simple-update kernels (su_kernels.cu) and the
// belief-propagation regauging kernels (bp_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "gpeps_internal.cuh"

namespace gpeps {

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };

template <typename T>
using V2 = typename vec2<T>::type;

template <typename T>
__device__ __forceinline__ V2<T> mk(T x, T y) {
  V2<T> r;
  r.x = x;
  r.y = y;
  return r;
}

// acc += conj(a) * b
template <typename T>
__device__ __forceinline__ void fma_conj(V2<T>& acc, V2<T> a, V2<T> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// acc += a * b
template <typename T>
__device__ __forceinline__ void fma_c(V2<T>& acc, V2<T> a, V2<T> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <typename T>
__device__ __forceinline__ V2<T> c_mul(V2<T> a, V2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ V2<T> c_conj(V2<T> a) {
  return mk<T>(a.x, -a.y);
}
template <typename T>
__device__ __forceinline__ V2<T> c_scale(V2<T> a, T s) {
  return mk<T>(a.x * s, a.y * s);
}
template <typename T>
__device__ __forceinline__ V2<T> c_add(V2<T> a, V2<T> b) {
  return mk<T>(a.x + b.x, a.y + b.y);
}
template <typename T>
__device__ __forceinline__ V2<T> c_sub(V2<T> a, V2<T> b) {
  return mk<T>(a.x - b.x, a.y - b.y);
}

// Rotation of the pair (p, q) (Golub & Van Loan, Alg. 8.4.1, sym.schur2, after
// the diagonal phase that makes a_pq real): J = [[c, s], [-s e, c e]],
// e = conj(a_pq)/|a_pq|.  Returns false (identity) when the pair is converged.
__device__ __forceinline__ bool rotation(float app, float aqq, float2 apq, float tol, float floor_abs, float& c,
                                         float& s, float2& e) {
  const float g2 = apq.x * apq.x + apq.y * apq.y;
  if (!(g2 > floor_abs * floor_abs && g2 > tol * tol * fabsf(app * aqq))) return false;
  const float ig = rsqrtf(g2);
  const float zeta = (aqq - app) * (0.5f * ig);
  const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  c = rsqrtf(1.f + t * t);
  s = t * c;
  e = make_float2(apq.x * ig, -apq.y * ig);
  return true;
}
// FP64 version, without FP64 divides or square roots: 1/|a_pq| and c =
// 1/sqrt(1 + t^2) start from FP32 rsqrtf and take two Newton-Raphson steps of
// the reciprocal square root, y <- y (3 - x y^2) / 2 (each step squares the
// relative error: 1e-7 -> 1e-14 -> rounding), so e and (c, s) are unit to FP64
// rounding and J is unitary; t starts from the FP32 formula and takes one
// Newton-Raphson step on f(t) = t^2 + 2 zeta t - 1 with an FP32 reciprocal of
// f'(t), which leaves a relative error of about 1e-7 x 1e-7 in the angle.
__device__ __forceinline__ bool rotation(double app, double aqq, double2 apq, double tol, double floor_abs,
                                         double& c, double& s, double2& e) {
  const double g2 = apq.x * apq.x + apq.y * apq.y;
  if (!(g2 > floor_abs * floor_abs && g2 > tol * tol * fabs(app * aqq))) return false;
  const float g2f = (float)g2;
  const float igf = rsqrtf(g2f);
  double ig = (double)igf;
  ig = ig * (1.5 - 0.5 * g2 * ig * ig);
  ig = ig * (1.5 - 0.5 * g2 * ig * ig);
  const float zetaf = (float)(aqq - app) * (0.5f * igf);
  const float tf = copysignf(1.f, zetaf) / (fabsf(zetaf) + sqrtf(1.f + zetaf * zetaf));
  // one Newton step on t^2 + 2 zeta t - 1 = 0 in FP64 (the FP32 reciprocal of the
  // derivative suffices): the angle becomes FP64-accurate, so a rotation zeroes
  // a_pq to rounding instead of shrinking it by the FP32 angle error
  const double zeta = (aqq - app) * (0.5 * ig);
  double t = (double)tf;
  const double f = fma(t, t, fma(2.0 * zeta, t, -1.0));
  t -= f * (double)__frcp_rn((float)(2.0 * (t + zeta)));
  const double u = 1.0 + t * t;
  double cc = (double)rsqrtf((float)u);
  cc = cc * (1.5 - 0.5 * u * cc * cc);
  cc = cc * (1.5 - 0.5 * u * cc * cc);
  c = cc;
  s = t * cc;
  e = make_double2(apq.x * ig, -apq.y * ig);
  return true;
}

// Rotation of the column pair with squared norms a, b and inner product
// g = b_p^H b_q (g != 0), the one that diagonalises [[a, g], [conj(g), b]]:
// the phase e = conj(g) / |g| first, then t = tan of the angle from
// t^2 + 2 zeta t - 1 = 0, zeta = (b - a) / (2 |g|) (Golub & Van Loan Alg. 8.4.1),
// for the one-sided Jacobi of the unsquared bond SVD.  The three entries are
// first rescaled by the same power of two so that |g| ~ 1 (exact; the angle is
// scale-free), so that the FP32 seeds below cannot underflow; then the
// Newton-Raphson refinements of `rotation` (two reciprocal-square-root steps
// for 1/|g| and for c = 1/sqrt(1 + t^2), one step on the angle equation) make
// the rotation unitary to FP64 rounding without FP64 divides or square roots.
// When |zeta| is beyond FP32 range t = 1 / (2 zeta).
// Also returns |g|.
__device__ __forceinline__ void os_rotation(double a, double b, double2 g, double& c, double& s, double2& e,
                                            double& ag) {
  int ex;
  frexp(fma(g.x, g.x, g.y * g.y), &ex);
  const int k = ex >> 1;  // |g| ~ 2^k
  a = ldexp(a, -k);
  b = ldexp(b, -k);
  g = make_double2(ldexp(g.x, -k), ldexp(g.y, -k));
  const double g2 = fma(g.x, g.x, g.y * g.y);  // in [1/4, 2)
  double ig = (double)rsqrtf((float)g2);
  ig = ig * (1.5 - 0.5 * g2 * ig * ig);
  ig = ig * (1.5 - 0.5 * g2 * ig * ig);
  const double zeta = (b - a) * (0.5 * ig);
  double t;
  if (fabs(zeta) < 1e18) {
    const float zf = (float)zeta;
    t = (double)(copysignf(1.f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.f))));
    const double f = fma(t, t, fma(2.0 * zeta, t, -1.0));
    t -= f * (double)__frcp_rn((float)(2.0 * (t + zeta)));
  } else {
    t = 0.5 / zeta;
  }
  const double u = fma(t, t, 1.0);
  double cc = (double)rsqrtf((float)u);
  cc = cc * (1.5 - 0.5 * u * cc * cc);
  cc = cc * (1.5 - 0.5 * u * cc * cc);
  c = cc;
  s = t * cc;
  e = make_double2(g.x * ig, -g.y * ig);
  ag = ldexp(g2 * ig, k);
}

// Storage of the Hermitian matrix of a Jacobi solve.  HermFull: n x n with row
// stride lda, both triangles kept.  HermPacked: the upper triangle row by row
// (n(n+1)/2 entries, row i starting at i(2n - i + 1)/2); the lower triangle is
// implied, so a rotated entry is written once at its upper-triangle place.
template <typename R>
struct HermFull {
  V2<R>* A;
  int lda;
  __device__ __forceinline__ V2<R> get(int i, int j) const { return A[i * lda + j]; }
  __device__ __forceinline__ void put(int i, int j, V2<R> v, bool mirror) const {
    A[i * lda + j] = v;
    if (mirror) A[j * lda + i] = c_conj<R>(v);
  }
};
template <typename R>
struct HermPacked {
  V2<R>* P;
  int n;
  __device__ __forceinline__ int at(int i, int j) const { return ((i * (2 * n - i + 1)) >> 1) + j - i; }
  __device__ __forceinline__ V2<R> get(int i, int j) const {
    return i <= j ? P[at(i, j)] : c_conj<R>(P[at(j, i)]);
  }
  __device__ __forceinline__ void put(int i, int j, V2<R> v, bool) const {
    if (i <= j) P[at(i, j)] = v;
    else P[at(j, i)] = c_conj<R>(v);
  }
};

// Parallel cyclic Jacobi for the Hermitian n x n matrix A (storage policy S:
// HermFull or HermPacked), accumulating V (row stride ldv) <- V * product of rotations
// (V is initialised by the caller).  The (n-1) rounds of a sweep use the
// round-robin pairing, so the n/2 <= 64 rotations of a round are disjoint and
// applied together: A <- J^dagger A J on 2x2 blocks, V <- V J.  A pair is
// skipped when |a_pq| <= max(tol sqrt(a_pp a_qq), floor_abs).  The active pairs
// of a round are compacted (a warp ballot per 32 pairs) and the work runs over
// them densely: the blocks {a, b} with a active (each unordered pair once, the
// diagonal block a = b included), and the rows of V times the active pairs; a
// round without active pairs does no work.  So late sweeps, where few pairs
// still rotate, do not occupy whole warps with skipped lanes.
// With kExact the off-diagonal of a rotated diagonal block is set to zero (the
// FP32 angle is exact for FP32 arithmetic); the FP64 sweeps keep the computed
// residual instead.  Returns the sweeps run; max_sweeps + 1 = cap hit.
// work (or null): adds the 2x2 block updates and the eigenvector pair updates
// executed, work[0] and work[1].  iflag: 8 ints, followed by 136 ints of scratch:
// the active and the idle pairs of the round, per warp ([2][32] each), and their
// counts, double-buffered by round parity ([2][4]).
// kRowsFastest: the eigenvector update gives consecutive threads consecutive rows of V
// for one pair (its rotation read as a broadcast); with an odd row stride ldv (in
// elements of 8 bytes) the 16 rows of a half-warp then fall in distinct banks.  The
// default gives consecutive threads the active pairs of one row.  Both perform the same
// operations on every element.
template <typename R, bool kExact, typename S, bool kRowsFastest = false>
__device__ int jacobi_hermitian(S A, V2<R>* V, int ldv, int n, R tol, R floor_abs, int max_sweeps,
                                R* rc, R* rs, V2<R>* re, int* rp, int* rq, int* iflag,
                                unsigned long long* rot_count, unsigned long long* work = nullptr) {
  const int m = n / 2;
  int* act = iflag + 8;     // [2 warps][32] active pairs
  int* idle = iflag + 72;   // [2 warps][32] idle pairs
  int* wcnt = iflag + 136;  // [2 buffers][active w0, active w1, idle w0, idle w1]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long n_blk = 0, n_vec = 0;
  int sweep = 0, result = max_sweeps + 1;
  for (; sweep < max_sweeps; ++sweep) {
    int rot_sweep = 0;  // thread 0: rotations of this sweep
    for (int r = 0; r < n - 1; ++r) {
      int* cnt = wcnt + 4 * (r & 1);
      if (warp < 2) {
        const int k = threadIdx.x;
        bool on = false;
        if (k < m) {
          int p, q;
          if (k == 0) {
            p = r;
            q = n - 1;
          } else {
            p = r + k;
            if (p >= n - 1) p -= n - 1;
            q = r - k;
            if (q < 0) q += n - 1;
          }
          if (p > q) {
            const int tmp = p;
            p = q;
            q = tmp;
          }
          R cs = 1, sn = 0;
          V2<R> e = mk<R>(1, 0);
          on = rotation(A.get(p, p).x, A.get(q, q).x, A.get(p, q), tol, floor_abs, cs, sn, e) && sn != R(0);
          rp[k] = p;
          rq[k] = q;
          rc[k] = cs;
          rs[k] = on ? sn : R(0);
          re[k] = e;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        const unsigned bid = __ballot_sync(0xffffffffu, k < m && !on);
        const unsigned below = (1u << lane) - 1u;
        if (on) act[warp * 32 + __popc(bal & below)] = k;
        if (k < m && !on) idle[warp * 32 + __popc(bid & below)] = k;
        if (lane == 0) {
          cnt[warp] = __popc(bal);
          cnt[2 + warp] = __popc(bid);
        }
      }
      __syncthreads();
      const int c0 = cnt[0], na = c0 + cnt[1], i0 = cnt[2], ni = i0 + cnt[3];
      if (threadIdx.x == 0) rot_sweep += na;
      if (na == 0) continue;  // nothing read below: the next round may overwrite at once
      auto active = [&](int i) { return i < c0 ? act[i] : act[32 + i - c0]; };
      auto idle_at = [&](int j) { return j < i0 ? idle[j] : idle[32 + j - i0]; };
      // blocks {a, b} touching an active pair, each once: a active and b idle
      // (na x ni), then both active with rank(a) <= rank(b) (triangle, diagonal included)
      const int n_ai = na * ni, n_blocks = n_ai + na * (na + 1) / 2;
      for (int t = threadIdx.x; t < n_blocks; t += blockDim.x) {
        int a, b;
        if (t < n_ai) {
          const int ia = t / ni;
          a = active(ia);
          b = idle_at(t - ia * ni);
        } else {
          const int u = t - n_ai;
          int row = (int)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
          while (row * (row + 1) / 2 > u) --row;
          while ((row + 1) * (row + 2) / 2 <= u) ++row;
          a = active(u - row * (row + 1) / 2);
          b = active(row);
        }
        ++n_blk;
        const int pa = rp[a], qa = rq[a], pb = rp[b], qb = rq[b];
        const R ca = rc[a], sa = rs[a], cb = rc[b], sb = rs[b];
        const V2<R> ea = re[a], eb = rs[b] != R(0) ? re[b] : mk<R>(1, 0);
        const V2<R> b00 = A.get(pa, pb), b01 = A.get(pa, qb);
        const V2<R> b10 = A.get(qa, pb), b11 = A.get(qa, qb);
        const V2<R> b01e = c_mul<R>(b01, eb), b11e = c_mul<R>(b11, eb);
        const V2<R> t00 = c_sub<R>(c_scale<R>(b00, cb), c_scale<R>(b01e, sb));
        const V2<R> t01 = c_add<R>(c_scale<R>(b00, sb), c_scale<R>(b01e, cb));
        const V2<R> t10 = c_sub<R>(c_scale<R>(b10, cb), c_scale<R>(b11e, sb));
        const V2<R> t11 = c_add<R>(c_scale<R>(b10, sb), c_scale<R>(b11e, cb));
        const V2<R> ce = c_conj<R>(ea);
        const V2<R> u10 = c_mul<R>(t10, ce), u11 = c_mul<R>(t11, ce);
        V2<R> n00 = c_sub<R>(c_scale<R>(t00, ca), c_scale<R>(u10, sa));
        V2<R> n01 = c_sub<R>(c_scale<R>(t01, ca), c_scale<R>(u11, sa));
        V2<R> n10 = c_add<R>(c_scale<R>(t00, sa), c_scale<R>(u10, ca));
        V2<R> n11 = c_add<R>(c_scale<R>(t01, sa), c_scale<R>(u11, ca));
        const bool diag = b == a;
        if (diag) {
          n00.y = R(0);
          n11.y = R(0);
          if (kExact) {
            n01 = mk<R>(0, 0);
          } else {
            n01 = mk<R>(R(0.5) * (n01.x + n10.x), R(0.5) * (n01.y - n10.y));
          }
          n10 = c_conj<R>(n01);
        }
        A.put(pa, pb, n00, !diag);
        A.put(pa, qb, n01, !diag);
        A.put(qa, pb, n10, !diag);
        A.put(qa, qb, n11, !diag);
      }
      auto vec_update = [&](int i, int k) {
        ++n_vec;
        const R cs = rc[k], sn = rs[k];
        const int p = rp[k], q = rq[k];
        const V2<R> vp = V[i * ldv + p];
        const V2<R> vqe = c_mul<R>(V[i * ldv + q], re[k]);
        V[i * ldv + p] = c_sub<R>(c_scale<R>(vp, cs), c_scale<R>(vqe, sn));
        V[i * ldv + q] = c_add<R>(c_scale<R>(vp, sn), c_scale<R>(vqe, cs));
      };
      if (kRowsFastest && blockDim.x % n == 0) {
        const int i = threadIdx.x % n, step = blockDim.x / n;
        for (int j = threadIdx.x / n; j < na; j += step) vec_update(i, active(j));
      } else if (kRowsFastest) {
        for (int t = threadIdx.x; t < n * na; t += blockDim.x) {
          const int j = t / n;
          vec_update(t - j * n, active(j));
        }
      } else {
        for (int t = threadIdx.x; t < n * na; t += blockDim.x) {
          const int i = t / na;
          vec_update(i, active(t - i * na));
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      iflag[3] = rot_sweep;
      if (rot_count && sweep < kRotSweeps) atomicAdd(rot_count + sweep, (unsigned long long)rot_sweep);
    }
    __syncthreads();
    const int done = iflag[3] == 0;
    __syncthreads();
    if (done) {
      result = sweep + 1;
      break;
    }
  }
  if (work) {
    for (int off = 16; off > 0; off >>= 1) {
      n_blk += __shfl_down_sync(0xffffffffu, n_blk, off);
      n_vec += __shfl_down_sync(0xffffffffu, n_vec, off);
    }
    if (lane == 0) {
      atomicAdd(work, n_blk);
      atomicAdd(work + 1, n_vec);
    }
  }
  return result;
}

}  // namespace gpeps
