// Tensor-core (tcgen05, kind::tf32) Gram and update passes of the larger end
// of a bond in the mixed path (complex64 storage), D = 32 or 64.
//
// The two streaming products of a bond update ("Method": absorb, reduce and
// contract of the simple update) are real GEMMs once complex numbers are
// split into their real and imaginary parts:
//
//   Gram    P[r][c], c = (s, k, re/im), holds the kicked, lambda-weighted end a;
//           B = P^T P accumulates in TMEM over the rows r, and
//           G_s[k][l] = (B[(s,k,re)][(s,l,re)] + B[(s,k,im)][(s,l,im)])
//                     + i (B[(s,k,re)][(s,l,im)] - B[(s,k,im)][(s,l,re)]).
//           D = 32: one 128 x 128 product over all 4D columns of P (the
//           blocks s != s' are computed and not read); D = 64: one 128 x 128
//           product per s.
//   update  Gamma_a'[s][r][k'] = mask_r sum_t sum_k Gamma_t[r][k] K_st Y_s[k][k']
//           with the kick K = exp(-i theta X / 2) folded into the right
//           operand: one M = 128 (rows) x N = 4D ((s, k', re/im)) product over
//           K = 4D ((t, k, re/im)) whose left operand is the stored tensor as it
//           is (complex numbers are (re, im) pairs, i.e. K-major already).
//
// FP32 accuracy through the 3xTF32 split: every FP32 operand x is held as
// hi = tf32(x) and lo = tf32(x - hi), and each product is
// hi_a hi_b + hi_a lo_b + lo_a hi_b (the dropped lo_a lo_b and the rounding of
// lo leave about 2^-22 of |a b|), accumulated in FP32 in TMEM.  The Gram is read
// out of TMEM after every 64-row tile and summed in FP64, as the CUDA-core
// passes do.
//
// Operands are staged by the CTA's threads in chunks of kTcKc values of K
// (core-matrix layout of tcgen05.cuh); thread 0 issues the MMAs and commits
// them to an mbarrier that every thread waits on (bounded).  Warps 0-3 read
// the accumulator (warp w: TMEM lanes 32w .. 32w + 31).
//
// Included by su_kernels.cu after its row/element helpers (row_pos, elem,
// row_weight, ldst, kick2).
#pragma once
#include "tcgen05.cuh"

namespace gpeps {


struct TcCtx {
  uint32_t tmem;    // TMEM base address (tc_cols(D) columns)
  uint64_t* bar;    // mbarrier the MMA commits arrive on
  long long limit;  // wait budget in SM cycles
};

__device__ __forceinline__ void tc_put(unsigned char* hi, unsigned char* lo, int row, int q, float x) {
  float h, l;
  tc::split_tf32(x, h, l);
  const uint32_t o = tc::kmajor_off(row, q, kTcKc);
  *reinterpret_cast<float*>(hi + o) = h;
  *reinterpret_cast<float*>(lo + o) = l;
}

// Every thread waits for the committed products; the outcome is made uniform
// over the CTA.  After a wait that gave up, a second bounded wait lets products
// still in flight finish before the caller frees TMEM.
__device__ __forceinline__ bool tc_wait_chunk(const TcCtx& cx, uint32_t& phase) {
  const bool ok = __syncthreads_and(tc::mbar_wait(cx.bar, phase, cx.limit) ? 1 : 0) != 0;
  if (!ok) tc::mbar_wait(cx.bar, phase, cx.limit);
  phase ^= 1u;
  return ok;
}

// Make the staged chunk visible to the tensor core, issue the 3xTF32 products
// of `nk` K values (a multiple of 8) from thread 0, and wait for them.
// a/b: shared addresses of hi (lo follows at +lo_a / +lo_b bytes).
__device__ __forceinline__ bool tc_mma_chunk(uint32_t a, uint32_t lo_a, uint32_t b, uint32_t lo_b, int nk,
                                             uint32_t d_tmem, uint32_t idesc, bool fresh, const TcCtx& cx,
                                             uint32_t& phase) {
  tc::fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc::fence_after_sync();
    constexpr uint32_t kLbo = 128, kSbo = kTcKc * 32;
    for (int ks = 0; ks < nk; ks += 8) {
      const uint32_t off = (uint32_t)ks * 32;
      const uint64_t ah = tc::smem_desc(a + off, kLbo, kSbo), al = tc::smem_desc(a + lo_a + off, kLbo, kSbo);
      const uint64_t bh = tc::smem_desc(b + off, kLbo, kSbo), bl = tc::smem_desc(b + lo_b + off, kLbo, kSbo);
      tc::mma_tf32(d_tmem, ah, bh, idesc, (fresh && ks == 0) ? 0u : 1u);
      tc::mma_tf32(d_tmem, ah, bl, idesc, 1u);
      tc::mma_tf32(d_tmem, al, bh, idesc, 1u);
    }
    tc::mma_commit(cx.bar);
  }
  return tc_wait_chunk(cx, phase);
}

// Gram of rows [row0, row0 + nrows) of end a into TMEM: a fresh accumulation
// if `fresh`, else added to the one there.
template <bool kCG>
__device__ bool tc_gram_rows(const SideDesc& sa, const float2* gamma, const double* lam, float c, float s, int row0,
                             int nrows, int D, unsigned char* sm, const TcCtx& cx, uint32_t& phase, bool fresh) {
  unsigned char* hi = sm;
  const uint32_t lo_off = (uint32_t)(4 * D * kTcKc * 4);
  unsigned char* lo = sm + lo_off;
  const uint32_t idesc = tc::idesc_tf32(128, 128);
  const uint32_t base = tc::smem_u32(hi);
  bool ok = true;
  for (int r0 = 0; r0 < nrows; r0 += kTcKc) {
    const int kc = nrows - r0 < kTcKc ? nrows - r0 : kTcKc;
    const int nel = kc * D;
    for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
      int r, k;
      if (sa.str_k == 1) {
        r = idx / D;
        k = idx - r * D;
      } else {
        k = idx / kc;
        r = idx - k * kc;
      }
      const RowPos p = row_pos(sa, row0 + r0 + r);
      const int64_t e = elem(sa, 0, p, k);
      const float w = (float)row_weight<kCG>(sa, lam, p);
      float2 a0, a1;
      kick2<float>(c, s, ldst<kCG>(gamma + e), ldst<kCG>(gamma + e + sa.str_s), a0, a1);
      tc_put(hi, lo, 2 * k, r, a0.x * w);
      tc_put(hi, lo, 2 * k + 1, r, a0.y * w);
      tc_put(hi, lo, 2 * (D + k), r, a1.x * w);
      tc_put(hi, lo, 2 * (D + k) + 1, r, a1.y * w);
    }
    // rows are the K extent here: pad a ragged chunk (a degree-1 end has one row) to a multiple of 8
    const int kc8 = (kc + 7) & ~7;
    for (int idx = threadIdx.x; idx < (kc8 - kc) * 4 * D; idx += blockDim.x) {
      const int r = kc + idx / (4 * D), cc = idx - (idx / (4 * D)) * 4 * D;
      tc_put(hi, lo, cc, r, 0.f);
    }
    // D = 32: rows 0..127 of P; D = 64: rows 128 g .. 128 g + 127 (spin g) into TMEM columns 128 g ..
    const int ng = D == 64 ? 2 : 1;
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      constexpr uint32_t kLbo = 128, kSbo = kTcKc * 32;
      for (int g = 0; g < ng; ++g) {
        const uint32_t rb = base + (uint32_t)g * 16u * kSbo;
        for (int ks = 0; ks < kc8; ks += 8) {
          const uint32_t off = (uint32_t)ks * 32;
          const uint64_t dh = tc::smem_desc(rb + off, kLbo, kSbo), dl = tc::smem_desc(rb + lo_off + off, kLbo, kSbo);
          const uint32_t d = cx.tmem + (uint32_t)g * 128u;
          tc::mma_tf32(d, dh, dh, idesc, (fresh && r0 == 0 && ks == 0) ? 0u : 1u);
          tc::mma_tf32(d, dh, dl, idesc, 1u);
          tc::mma_tf32(d, dl, dh, idesc, 1u);
        }
      }
      tc::mma_commit(cx.bar);
    }
    ok = tc_wait_chunk(cx, phase);
    if (!ok) break;
  }
  return ok;
}

// Read the Gram accumulator: calls out(s, k, l, reim, value) once for every
// component of G_s[k][l] (threads 0..127; the re/im rows of one (s, k) are the
// neighbouring lanes m and m ^ 1).
template <typename Out>
__device__ __forceinline__ void tc_gram_read(int D, const TcCtx& cx, Out out) {
  if (threadIdx.x < 128) {
    tc::fence_after_sync();
    const int m = threadIdx.x, warp = m >> 5, reim = m & 1;
    const int ng = D == 64 ? 2 : 1;
    for (int g = 0; g < ng; ++g) {
      const int sp = D == 64 ? g : (m >> 6);
      const int k = D == 64 ? (m >> 1) : ((m >> 1) & 31);
      const uint32_t col0 = D == 64 ? (uint32_t)g * 128u : (uint32_t)sp * 64u;
      for (int cb = 0; cb < 2 * D; cb += 32) {
        float v[32];
        tc::tmem_ld32(cx.tmem + ((uint32_t)(32 * warp) << 16) + col0 + (uint32_t)cb, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float po = __shfl_xor_sync(0xffffffffu, v[2 * j + 1], 1);
          out(sp, k, cb / 2 + j, reim, reim == 0 ? v[2 * j] + po : po - v[2 * j]);
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
}

// Update of rows [row0, row0 + nrows) of end a (nrows <= 128):
// Gamma_a'[s][r][k'] = mask[r] sum_t sum_k Gamma_t[r][k] K_st Y_s[k][k'] in place.
// Y: [2][D][D] complex of this bond; (c, s) the kick of end a.  The rows are
// written by threads 0..127 after the product completes, so the in-place write
// reads nothing it has overwritten.
template <bool kCG>
__device__ bool tc_update_rows(const SideDesc& sa, float2* gamma, const float2* Y, float c, float s,
                               const float* mask, int row0, int nrows, int D, unsigned char* sm, const TcCtx& cx,
                               uint32_t& phase) {
  unsigned char* ahi = sm;
  const uint32_t a_lo = (uint32_t)(128 * kTcKc * 4);
  unsigned char* alo = ahi + a_lo;
  unsigned char* bhi = alo + a_lo;
  const uint32_t b_lo = (uint32_t)(4 * D * kTcKc * 4);
  unsigned char* blo = bhi + b_lo;
  const int D2 = D * D, nchunks = 4 * D / kTcKc, per_t = 2 * D / kTcKc;
  const uint32_t idesc = tc::idesc_tf32(128, 4 * D);
  bool ok = true;
  for (int j = 0; j < nchunks && ok; ++j) {
    const int t = j / per_t, k0 = (j - t * per_t) * (kTcKc / 2);
    // left operand: row r, K value q = 2 (k - k0) + re/im
    const int na = nrows * (kTcKc / 2);
    for (int idx = threadIdx.x; idx < na; idx += blockDim.x) {
      int r, kk;
      if (sa.str_k == 1) {
        r = idx / (kTcKc / 2);
        kk = idx - r * (kTcKc / 2);
      } else {
        kk = idx / nrows;
        r = idx - kk * nrows;
      }
      const RowPos p = row_pos(sa, row0 + r);
      const float2 g = ldst<kCG>(gamma + elem(sa, t, p, k0 + kk));
      tc_put(ahi, alo, r, 2 * kk, g.x);
      tc_put(ahi, alo, r, 2 * kk + 1, g.y);
    }
    // right operand: row n = (s', k', re/im), K value q = 2 (k - k0) + re/im;
    // w = K_{s't} Y_{s'}[k][k'] with K_00 = K_11 = c, K_01 = K_10 = -i s
    const int nb = 2 * D * (kTcKc / 2);
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
      const int kp = idx % D, rest = idx / D;
      const int kk = rest % (kTcKc / 2), sp = rest / (kTcKc / 2);
      const float2 y = ldst<kCG>(Y + sp * D2 + (k0 + kk) * D + kp);
      const float2 w = sp == t ? make_float2(c * y.x, c * y.y) : make_float2(s * y.y, -s * y.x);
      const int n0 = sp * 2 * D + 2 * kp, q0 = 2 * kk;
      tc_put(bhi, blo, n0, q0, w.x);
      tc_put(bhi, blo, n0, q0 + 1, -w.y);
      tc_put(bhi, blo, n0 + 1, q0, w.y);
      tc_put(bhi, blo, n0 + 1, q0 + 1, w.x);
    }
    ok = tc_mma_chunk(tc::smem_u32(ahi), a_lo, tc::smem_u32(bhi), b_lo, kTcKc, cx.tmem, idesc, j == 0, cx, phase);
  }
  if (threadIdx.x < 128 && ok) {
    tc::fence_after_sync();
    const int r = threadIdx.x, warp = r >> 5;
    const bool live = r < nrows;
    RowPos p{0, 0};
    float mk = 0.f;
    if (live) {
      p = row_pos(sa, row0 + r);
      mk = mask[r];
    }
    for (int cb = 0; cb < 4 * D; cb += 32) {
      float v[32];
      tc::tmem_ld32(cx.tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, v);
      if (live) {
        const int sp = cb / (2 * D), kp0 = (cb - sp * 2 * D) / 2;
#pragma unroll
        for (int q = 0; q < 16; ++q) gamma[elem(sa, sp, p, kp0 + q)] = make_float2(v[2 * q] * mk, v[2 * q + 1] * mk);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  return ok;
}

}  // namespace gpeps
