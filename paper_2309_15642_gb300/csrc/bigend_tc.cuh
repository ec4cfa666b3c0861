// Tensor-core (tcgen05, kind::tf32) Gram and update passes of the larger end
// of a bond in the mixed path (complex64 storage), D = 32 or 64.
//
// The two streaming products of a bond update ("Method": absorb, reduce and
// contract of the simple update) are real GEMMs once complex numbers are
// split into their real and imaginary parts:
//
//   Gram    P[r][c], c = (s, re/im, k) (spin-major, real parts then imaginary
//           parts), holds the kicked, lambda-weighted end a; B = P^T P
//           accumulates in TMEM over the rows r, and
//           G_s[k][l] = (B[(s,re,k)][(s,re,l)] + B[(s,im,k)][(s,im,l)])
//                     + i (B[(s,re,k)][(s,im,l)] - B[(s,im,k)][(s,re,l)]).
//           D = 32: one 128 x 128 product over all 4D columns of P (the
//           blocks s != s' are computed and not read); D = 64: one 128 x 128
//           product per s.
//   update  Gamma_a'[s][r][k'] = mask_r sum_t sum_k Gamma_t[r][k] K_st Y_s[k][k']
//           with the kick K = exp(-i theta X / 2) folded into the right
//           operand W: one M = 128 (rows) x N = 4D ((s, re/im, k')) product
//           over K = 4D ((t, k, re/im)), staged in chunks of 8 complex k of one t.
//
// FP32 accuracy through the 3xTF32 split: every FP32 operand x is held as
// hi = tf32(x) and lo = tf32(x - hi), and each product is
// hi_a hi_b + hi_a lo_b + lo_a hi_b (the dropped lo_a lo_b and the rounding of
// lo leave about 2^-22 of |a b|), accumulated in FP32 in TMEM.  The Gram is read
// out of TMEM after every 64-row tile and summed in FP64, as the CUDA-core
// passes do.
//
// Data movement: the rows of end a for the Gram are contiguous runs of the
// state (the bond leg, or the faster other leg, is the last leg), so each
// 32-row chunk is staged by bulk copies (cp.async.bulk, the TMA engine)
// completing on an mbarrier, one chunk ahead of the conversion; the staged
// complex numbers are kicked, weighted, split and written to the operand
// layout, thread 0 issues the MMAs and commits them to a second mbarrier.
// The update's left operand is loaded in batches (every thread's loads of a
// chunk in flight at once) and its right operand is built from Y.  Lane
// assignments keep the operand writes free of shared-memory bank conflicts
// (8 consecutive operand rows x 4 consecutive K values per warp).
//
// Included by su_kernels.cu after its row/element helpers (row_pos, elem,
// row_weight, ldst).
#pragma once
#include "tcgen05.cuh"

namespace gpeps {

// exp(-i theta X / 2) on the pair (g0, g1) with the rounding pinned (explicit
// fused multiply-adds), so that every kernel that inlines it computes the same
// bits whatever the compiler would contract
__device__ __forceinline__ void tc_kick(float c, float s, float2 g0, float2 g1, float2& a0, float2& a1) {
  a0 = make_float2(__fmaf_rn(c, g0.x, __fmul_rn(s, g1.y)), __fmaf_rn(c, g0.y, -__fmul_rn(s, g1.x)));
  a1 = make_float2(__fmaf_rn(c, g1.x, __fmul_rn(s, g0.y)), __fmaf_rn(c, g1.y, -__fmul_rn(s, g0.x)));
}

// Warp 0: bulk copies of rows [r0, r0 + kc) of end a (both spins) into the
// staging area, completing on cx.sbar.  The chunk lies within one value of the
// slower other leg, so each copy is a contiguous run: with the bond leg last
// (str_k = 1) one run of kc x D elements per spin (staged [s][r][k]); else the
// faster other leg is last (str_o2 = 1) and there is one run of kc rows per
// (s, k) (staged [s][k][r]).  Every run starts on a 16-byte boundary (site
// offsets and strides are multiples of D elements, r0 of 32) and is a multiple
// of 16 bytes long.
__device__ __forceinline__ void tc_stage_rows(const SideDesc& sa, const float2* gamma, int r0, int kc, int D,
                                              float2* stg, const TcCtx& cx) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const RowPos p = row_pos(sa, r0);
  const int64_t base = sa.off + (int64_t)p.r1 * sa.str_o1 + (int64_t)p.r2 * sa.str_o2;
  if (lane == 0) tc::mbar_expect_tx(cx.sbar, (uint32_t)(2 * kc * D * 8));
  __syncwarp();
  if (sa.str_k == 1) {
    if (lane < 2)
      tc::bulk_g2s(stg + (size_t)lane * kc * D, gamma + base + (int64_t)lane * sa.str_s, (uint32_t)(kc * D * 8),
                   cx.sbar);
  } else {
    for (int i = lane; i < 2 * D; i += 32) {
      const int sp = i / D, k = i - sp * D;
      tc::bulk_g2s(stg + (size_t)i * kc, gamma + base + (int64_t)sp * sa.str_s + (int64_t)k * sa.str_k,
                   (uint32_t)(kc * 8), cx.sbar);
    }
  }
}

// Gram pass over all rows of end a: per 64-row tile the accumulator is read,
// and G_0, G_1 of the tile are either added in FP64 to gsum ([2][D][D], in tile
// order) or, with gsum null, stored in FP32 to part + tile * 2 D^2 (the
// layered partials).  kNb: entries of G per thread whose loads of gsum are in
// flight together (registers permitting).  Returns false if a wait gave up
// (the pass then stops).
template <bool kCG, int kNb = 4>
__device__ bool tc_gram_pass(const SideDesc& sa, const float2* gamma, const double* lam, float c, float s, int D,
                             unsigned char* sm, const TcCtx& cx, uint32_t& mphase, uint32_t& sphase, double2* gsum,
                             float2* part) {
  const TcGramSmem L(D);
  unsigned char* hi = sm;
  const uint32_t lo_off = (uint32_t)(4 * D * kTcKc * 4);
  unsigned char* lo = sm + lo_off;
  float* dump = reinterpret_cast<float*>(sm);
  float2* stg = reinterpret_cast<float2*>(sm + L.stage);
  float* wrow = reinterpret_cast<float*>(sm + L.weight);
  const uint32_t idesc = tc::idesc_tf32(128, 128);
  const int rows = sa.rows, nchunk = (rows + kTcKc - 1) / kTcKc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int ldd = 2 * D + 1;
  bool ok = true;
  // the tensors and the shared memory were last touched by generic loads and stores (earlier
  // bond updates, in this CTA or, ordered by the done flags, in others): order those before the
  // bulk copies
  tc::fence_async_all();
  __syncthreads();
  tc_stage_rows(sa, gamma, 0, rows < kTcKc ? rows : kTcKc, D, stg, cx);
  for (int j = 0; j < nchunk && ok; ++j) {
    const int r0 = j * kTcKc, kc = rows - r0 < kTcKc ? rows - r0 : kTcKc, kc8 = (kc + 7) & ~7;
    for (int r = threadIdx.x; r < kc; r += blockDim.x)
      wrow[r] = (float)row_weight<kCG>(sa, lam, row_pos(sa, r0 + r));
    if (!tc_wait(cx.sbar, sphase, cx.limit)) {
      ok = false;
      break;
    }
    // items (r, k): a warp takes 4 rows x 8 consecutive k
    const int ngr = (kc8 + 3) / 4, ngk = D / 8;
    for (int g = warp; g < ngr * ngk; g += nwarps) {
      const int gr = g / ngk, gk = g - gr * ngk;
      const int r = gr * 4 + (lane >> 3), k = gk * 8 + (lane & 7);
      float2 a0 = make_float2(0.f, 0.f), a1 = a0;
      if (r < kc) {
        float2 g0, g1;
        if (sa.str_k == 1) {
          g0 = stg[(size_t)r * D + k];
          g1 = stg[(size_t)(kc + r) * D + k];
        } else {
          g0 = stg[(size_t)k * kc + r];
          g1 = stg[(size_t)(D + k) * kc + r];
        }
        const float w = wrow[r];
        tc_kick(c, s, g0, g1, a0, a1);
        a0 = make_float2(__fmul_rn(a0.x, w), __fmul_rn(a0.y, w));
        a1 = make_float2(__fmul_rn(a1.x, w), __fmul_rn(a1.y, w));
      }
      if (r < kc8) {  // rows are the K extent: a ragged chunk is padded with zero rows
        tc_put(hi, lo, k, r, kTcKc, a0.x);
        tc_put(hi, lo, D + k, r, kTcKc, a0.y);
        tc_put(hi, lo, 2 * D + k, r, kTcKc, a1.x);
        tc_put(hi, lo, 3 * D + k, r, kTcKc, a1.y);
      }
    }
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      const bool fresh = (r0 % kTileRows) == 0;
      const uint32_t base = tc::smem_u32(hi);
      for (int gm = 0; gm < (D == 64 ? 2 : 1); ++gm) {
        const uint32_t rb = base + (uint32_t)gm * 16u * (uint32_t)(kTcKc * 32);
        tc_issue(rb, lo_off, rb, lo_off, kc8, kTcKc, cx.tmem + (uint32_t)gm * 128u, idesc, fresh);
      }
      tc::mma_commit(cx.bar);
    }
    // the staging area is free (every thread is past the conversion): fetch the next chunk
    if (j + 1 < nchunk) {
      const int n0 = r0 + kTcKc;
      tc_stage_rows(sa, gamma, n0, rows - n0 < kTcKc ? rows - n0 : kTcKc, D, stg, cx);
    }
    ok = tc_wait(cx.bar, mphase, cx.limit);
    if (!ok) {
      if (j + 1 < nchunk) tc_wait(cx.sbar, sphase, cx.limit);  // the copies in flight land before we return
      break;
    }
    if ((r0 + kc) % kTileRows != 0 && j + 1 < nchunk) continue;
    // tile complete: dump the same-spin columns of every accumulator row, then combine re/im rows
    tc::fence_after_sync();
    for (int gm = 0; gm < (D == 64 ? 2 : 1); ++gm) {
      if (threadIdx.x < 128) {
        const int m = threadIdx.x;
        const int sp = D == 64 ? gm : (m >> 6);
        const uint32_t col0 = D == 64 ? (uint32_t)gm * 128u : (uint32_t)sp * 64u;
        for (int cb = 0; cb < 2 * D; cb += 16) {
          float v[16];
          tc::tmem_ld16(cx.tmem + ((uint32_t)(32 * (m >> 5)) << 16) + col0 + (uint32_t)cb, v);
#pragma unroll
          for (int q = 0; q < 16; ++q) dump[m * ldd + cb + q] = v[q];
        }
      }
      tc::fence_before_sync();
      __syncthreads();
      // entries of G in index order sp * D^2 + k * D + l; a batch's loads of gsum are in flight
      // before its stores
      const int n = (D == 64 ? 1 : 2) * D * D, g0 = D == 64 ? gm * D * D : 0;
      for (int o0 = threadIdx.x; o0 < n; o0 += kNb * blockDim.x) {
        float re[kNb], im[kNb];
        double2 old[kNb];
#pragma unroll
        for (int b = 0; b < kNb; ++b) {
          const int o = o0 + b * blockDim.x;
          if (o < n) {
            const int ss = o / (D * D), kl = o - ss * D * D, k = kl / D, l = kl - k * D;
            const int rre = (D == 64 ? 0 : ss * 64) + k, rim = rre + D;
            re[b] = __fadd_rn(dump[rre * ldd + l], dump[rim * ldd + D + l]);
            im[b] = __fsub_rn(dump[rre * ldd + D + l], dump[rim * ldd + l]);
            if (gsum) old[b] = gsum[g0 + o];
          }
        }
#pragma unroll
        for (int b = 0; b < kNb; ++b) {
          const int o = o0 + b * blockDim.x;
          if (o < n) {
            if (gsum)
              gsum[g0 + o] = make_double2(old[b].x + (double)re[b], old[b].y + (double)im[b]);
            else
              part[(int64_t)(r0 / kTileRows) * 2 * D * D + g0 + o] = make_float2(re[b], im[b]);
          }
        }
      }
      __syncthreads();
    }
  }
  return ok;
}

// Update of rows [row0, row0 + nrows) of end a (nrows <= 128):
// Gamma_a'[s][r][k'] = mask[r] sum_t sum_k Gamma_t[r][k] K_st Y_s[k][k'] in place.
// Y: [2][D][D] complex of this bond; (c, s) the kick of end a.  Operand
// chunks hold 8 complex k of one t with K value q = re/im * 8 + (k - k0).
// The rows are written by threads 0..127 after the product completes, so the
// in-place write reads nothing it has overwritten.
template <bool kCG>
__device__ bool tc_update_rows(const SideDesc& sa, float2* gamma, const float2* Y, float c, float s,
                               const float* mask, int row0, int nrows, int D, unsigned char* sm, const TcCtx& cx,
                               uint32_t& phase) {
  constexpr int Ku = kTcKu, half = kTcKu / 2;
  unsigned char* ahi = sm;
  const uint32_t a_lo = (uint32_t)(128 * Ku * 4);
  unsigned char* alo = ahi + a_lo;
  unsigned char* bhi = alo + a_lo;
  const uint32_t b_lo = (uint32_t)(4 * D * Ku * 4);
  unsigned char* blo = bhi + b_lo;
  const int D2 = D * D, nchunks = 4 * D / Ku, per_t = 2 * D / Ku;
  const uint32_t idesc = tc::idesc_tf32(128, 4 * D);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  bool ok = true;
  for (int j = 0; j < nchunks && ok; ++j) {
    const int t = j / per_t, k0 = (j - t * per_t) * half;
    // left operand: a warp takes 8 rows x 4 k; all loads of a thread in flight at once
    {
      constexpr int kBatch = 4;  // loads of a thread in flight together
      const int ngroups = ((nrows + 7) / 8) * (half / 4);
      for (int g0 = warp; g0 < ngroups; g0 += kBatch * nwarps) {
        float2 gv[kBatch];
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
          const int g = g0 + i * nwarps;
          gv[i] = make_float2(0.f, 0.f);
          if (g < ngroups) {
            const int gr = g / (half / 4), gk = g - gr * (half / 4);
            const int r = gr * 8 + (lane & 7), kk = gk * 4 + (lane >> 3);
            if (r < nrows) gv[i] = ldst<kCG>(gamma + elem(sa, t, row_pos(sa, row0 + r), k0 + kk));
          }
        }
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
          const int g = g0 + i * nwarps;
          if (g < ngroups) {
            const int gr = g / (half / 4), gk = g - gr * (half / 4);
            const int r = gr * 8 + (lane & 7), kk = gk * 4 + (lane >> 3);
            tc_put(ahi, alo, r, kk, Ku, gv[i].x);
            tc_put(ahi, alo, r, half + kk, Ku, gv[i].y);
          }
        }
      }
    }
    // right operand: row n = (s', re/im, k'), K value q = re/im * 8 + (k - k0);
    // w = K_{s't} Y_{s'}[k][k'] with K_00 = K_11 = c, K_01 = K_10 = -i s.  A warp takes 8 k' x 4 k.
    {
      constexpr int kBatch = 4;
      const int ngroups = 2 * (D / 8) * (half / 4);
      for (int g0 = warp; g0 < ngroups; g0 += kBatch * nwarps) {
      float2 yv[kBatch];
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        const int g = g0 + i * nwarps;
        if (g < ngroups) {
          const int sp = g / ((D / 8) * (half / 4)), rest = g - sp * (D / 8) * (half / 4);
          const int gp = rest / (half / 4), gk = rest - gp * (half / 4);
          yv[i] = ldst<kCG>(Y + sp * D2 + (k0 + gk * 4 + (lane >> 3)) * D + gp * 8 + (lane & 7));
        }
      }
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        const int g = g0 + i * nwarps;
        if (g >= ngroups) continue;
        const int sp = g / ((D / 8) * (half / 4)), rest = g - sp * (D / 8) * (half / 4);
        const int gp = rest / (half / 4), gk = rest - gp * (half / 4);
        const int kp = gp * 8 + (lane & 7), kk = gk * 4 + (lane >> 3);
        const float2 y = yv[i];
        const float2 w = sp == t ? make_float2(__fmul_rn(c, y.x), __fmul_rn(c, y.y))
                                 : make_float2(__fmul_rn(s, y.y), -__fmul_rn(s, y.x));
        const int nre = sp * 2 * D + kp, nim = nre + D;
        tc_put(bhi, blo, nre, kk, Ku, w.x);
        tc_put(bhi, blo, nre, half + kk, Ku, -w.y);
        tc_put(bhi, blo, nim, kk, Ku, w.y);
        tc_put(bhi, blo, nim, half + kk, Ku, w.x);
      }
      }
    }
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      tc_issue(tc::smem_u32(ahi), a_lo, tc::smem_u32(bhi), b_lo, Ku, Ku, cx.tmem, idesc, j == 0);
      tc::mma_commit(cx.bar);
    }
    ok = tc_wait(cx.bar, phase, cx.limit);
  }
  if (threadIdx.x < 128 && ok) {
    tc::fence_after_sync();
    const int r = threadIdx.x, wq = r >> 5;
    const bool live = r < nrows;
    RowPos p{0, 0};
    float mk = 0.f;
    if (live) {
      p = row_pos(sa, row0 + r);
      mk = mask[r];
    }
    for (int sp = 0; sp < 2; ++sp) {
      for (int kb = 0; kb < D; kb += 16) {
        float vr[16], vi[16];
        const uint32_t col = (uint32_t)(sp * 2 * D + kb);
        tc::tmem_ld16(cx.tmem + ((uint32_t)(32 * wq) << 16) + col, vr);
        tc::tmem_ld16(cx.tmem + ((uint32_t)(32 * wq) << 16) + col + (uint32_t)D, vi);
        if (live) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            gamma[elem(sa, sp, p, kb + q)] = make_float2(__fmul_rn(vr[q], mk), __fmul_rn(vi[q], mk));
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  return ok;
}

}  // namespace gpeps
