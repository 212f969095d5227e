// Small dense double-float linear algebra of the background model (Eq. (9)
// and the iteration's covariance, Eq. (11)), one CTA per partition:
//   chol_inv_df   blocked Cholesky C = U^T U of a matrix in shared memory,
//                 with the inverse factor X = L^{-1} (L = U^T) formed in the
//                 same sweep;
//   xtx_apply_df  z = C^{-1} b = X^T (X b), X in shared memory;
//   c0inv_apply   Z = C^{-1} U for a few vectors from X in shared memory
//                 (the per-iteration solves).
// All arithmetic is double-float (mf_df.cuh); every sum has a fixed order.
#pragma once
#include "mf_common.cuh"
#include "mf_df.cuh"

namespace mf {

static_assert(kMaxB <= kThreads, "one thread per band in the vector loops");

__device__ __forceinline__ df df_shfl_xor(df v, int o) {
  return df{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// compensated accumulation of products (Dot2 of Ogita, Rump and Oishi, with
// double-float factors; the lo*lo product is dropped)
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(df x, df y) {
    const df pr = two_prod(x.hi, y.hi);
    const float err = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, pr.lo));
    const df t = two_sum(s, pr.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, err));
  }
  __device__ __forceinline__ df result() const { return fast_two_sum(s, c); }
};

// Dot2 for two sums at once on the packed f32x2 pipe: sum_j x_j (a_j, b_j)
// with a double-float x_j and the pair (a_j, b_j) given as its high parts
// yh and low parts yl
struct Dot2x2 {
  float2 s = {0.f, 0.f}, c = {0.f, 0.f};
  __device__ __forceinline__ void add(df x, float2 yh, float2 yl) {
    const float2 xh = f2(x.hi);
    const float2 ph = __fmul2_rn(xh, yh);
    const float2 pe = __ffma2_rn(xh, yh, __fmul2_rn(ph, f2(-1.f)));  // x.hi y.hi - ph, exact
    const float2 err = __ffma2_rn(xh, yl, __ffma2_rn(f2(x.lo), yh, pe));
    const float2 t = __fadd2_rn(s, ph);  // TwoSum(s, ph)
    const float2 bb = sub2(t, s);
    const float2 e = __fadd2_rn(sub2(s, sub2(t, bb)), sub2(ph, bb));
    s = t;
    c = __fadd2_rn(c, __fadd2_rn(e, err));
  }
  // add another partial sum (s2, c2) of the same two sums
  __device__ __forceinline__ void merge(float2 s2, float2 c2) {
    const float2 t = __fadd2_rn(s, s2);
    const float2 bb = sub2(t, s);
    const float2 e = __fadd2_rn(sub2(s, sub2(t, bb)), sub2(s2, bb));
    s = t;
    c = __fadd2_rn(c, __fadd2_rn(c2, e));
  }
  // merge with the partial sum of the lane whose index differs in bit 0
  // (all 32 lanes must call)
  __device__ __forceinline__ void merge_lane_pair() {
    const float2 s2 = make_float2(__shfl_xor_sync(0xffffffffu, s.x, 1), __shfl_xor_sync(0xffffffffu, s.y, 1));
    const float2 c2 = make_float2(__shfl_xor_sync(0xffffffffu, c.x, 1), __shfl_xor_sync(0xffffffffu, c.y, 1));
    merge(s2, c2);
  }
  // (high, low) of the two sums (Fast2Sum per lane)
  __device__ __forceinline__ void result(float2& h, float2& l) const {
    h = __fadd2_rn(s, c);
    l = sub2(c, sub2(h, s));
  }
};

// entry t of a packed list of rows, row r holding nb - r entries and
// starting at r nb - r (r - 1) / 2 -> (r, r + offset in the row); closed
// form, corrected by one
__device__ __forceinline__ void tri_decode(int t, int nb, int& bi, int& bj) {
  const float b2 = 2.f * nb + 1.f;
  int r = (int)((b2 - sqrtf(b2 * b2 - 8.f * (float)t)) * 0.5f);
  auto start = [&](int x) { return x * nb - (x * (x - 1)) / 2; };
  if (r < 0) r = 0;
  if (r > nb - 1) r = nb - 1;
  if (start(r) > t) --r;
  else if (r + 1 < nb && start(r + 1) <= t) ++r;
  bi = r;
  bj = r + (t - start(r));
}

namespace dense_detail {

constexpr int kPanel = 8;

// c - a for packed double-float pairs (the product 1 * a is exact)
__device__ __forceinline__ void df2_sub_inplace(float2& ch, float2& cl, float2 ah, float2 al) {
  df2_fnma(ch, cl, 1.f, -1.f, 0.f, ah, al);
}

// Steps j0 .. j1 - 1 of the elimination of [C | I] restricted to the
// diagonal block [j0, j1) x [j0, j1), by one warp: afterwards the block's
// upper triangle holds U_JJ (diagonal included), its strict lower triangle
// W = L_JJ^{-1} (diagonal invd), i.e. C_JJ = U_JJ^T U_JJ.  Step p: pivot d =
// A_pp, rows q in (p, j1) take q -= (A_pq / d) p on columns k <= p (the
// identity's half, unit diagonal implicit at k = p) and k >= q; row p - 1
// is scaled by its d^{-1/2} (no longer read).  Lanes 0..27 own (row, pair)
// of the update, lanes 28..31 the scaling.  Returns false if a pivot is not
// > 0 or not finite (uniform within the warp).
__device__ __forceinline__ bool factor_diag_block(const DfMat& A, int j0, int j1, df* invd) {
  const int lane = threadIdx.x & 31;
  const int q_off = 1 + (lane >> 2), c = j0 + 2 * (lane & 3);
  for (int p = j0; p < j1; ++p) {
    __syncwarp();
    const df d = A.get(p, p);
    if (!(d.hi > 0.f) || !df_isfinite(d)) return false;
    const df r = df_rsqrt(d);
    if (lane < 28) {
      const int q = p + q_off;
      if (q < j1 && c < j1) {
        const df w = df_mul(A.get(p, q), df_mul(r, r));
        const bool mx = c <= p || c >= q, my = c + 1 <= p || c + 1 >= q;
        if (mx || my) {
          float2 sh = A.hi2(p, c), sl = A.lo2(p, c);
          if (c == p) sh.x = 1.f, sl.x = 0.f;
          if (c + 1 == p) sh.y = 1.f, sl.y = 0.f;
          float2 ch = A.hi2(q, c), cl = A.lo2(q, c);
          const float2 oh = ch, ol = cl;
          df2_fnma(ch, cl, w.hi, -w.hi, w.lo, sh, sl);
          if (!mx) ch.x = oh.x, cl.x = ol.x;
          if (!my) ch.y = oh.y, cl.y = ol.y;
          A.set2(q, c, ch, cl);
        }
      }
    } else if (p > j0) {
      const int cs = j0 + 2 * (lane - 28);
      if (cs < j1) {
        float2 h = A.hi2(p - 1, cs), l = A.lo2(p - 1, cs);
        df2_mul1(h, l, invd[p - 1]);
        A.set2(p - 1, cs, h, l);
      }
    }
    if (lane == 0) invd[p] = r;
  }
  __syncwarp();
  if (lane < 4 && j0 + 2 * lane < j1) {
    const int cs = j0 + 2 * lane;
    float2 h = A.hi2(j1 - 1, cs), l = A.lo2(j1 - 1, cs);
    df2_mul1(h, l, invd[j1 - 1]);
    A.set2(j1 - 1, cs, h, l);
  }
  __syncwarp();
  return true;
}

// element (p, k) of W = L_JJ^{-1} from the factored diagonal block
__device__ __forceinline__ df w_elem(const DfMat& A, const df* invd, int p, int k) {
  return k < p ? A.get(p, k) : invd[p];
}

// 2 x 4 tile (rows i0, i0 + 1; columns k0 .. k0 + 3) of the rows below the
// panel [j0, j1): A_ik -= sum_p U_pi S_pk, S_pk = A_pk except in the
// panel's own columns, where S_pk = W_pk (invd[p] on the diagonal, 0 above
// it).  The sum is accumulated with compensation and subtracted once.  On
// a diagonal tile only k >= i is written: k < i holds X.
__device__ __forceinline__ void panel_update_tile(const DfMat& A, const df* invd, int j0, int j1,
                                                  int i0, int k0, bool diag) {
  Dot2x2 acc[2][2];
  const bool in_panel = k0 >= j0 && k0 < j1;
#pragma unroll 2
  for (int p = j0; p < j1; ++p) {
    const float2 uh = A.hi2(p, i0), ul = A.lo2(p, i0);
    float4 sh = A.hi4(p, k0), sl = A.lo4(p, k0);
    if (in_panel) {
      const df xd = invd[p];
      auto fix = [&](float& h, float& l, int k) {
        if (k == p) h = xd.hi, l = xd.lo;
        if (k > p) h = 0.f, l = 0.f;
      };
      fix(sh.x, sl.x, k0);
      fix(sh.y, sl.y, k0 + 1);
      fix(sh.z, sl.z, k0 + 2);
      fix(sh.w, sl.w, k0 + 3);
    }
    acc[0][0].add(df{uh.x, ul.x}, make_float2(sh.x, sh.y), make_float2(sl.x, sl.y));
    acc[0][1].add(df{uh.x, ul.x}, make_float2(sh.z, sh.w), make_float2(sl.z, sl.w));
    acc[1][0].add(df{uh.y, ul.y}, make_float2(sh.x, sh.y), make_float2(sl.x, sl.y));
    acc[1][1].add(df{uh.y, ul.y}, make_float2(sh.z, sh.w), make_float2(sl.z, sl.w));
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + a, k = k0 + 2 * h;
      float2 th, tl;
      acc[a][h].result(th, tl);
      float2 ch = A.hi2(i, k), cl = A.lo2(i, k);
      df2_sub_inplace(ch, cl, th, tl);
      if (!diag || k >= i) {
        A.set2(i, k, ch, cl);
      } else if (k + 1 >= i) {
        A.set(i, k + 1, df{ch.y, cl.y});
      }
    }
}

}  // namespace dense_detail

// In-place Cholesky factorisation C = U^T U of the symmetric leading n x n
// block of A (n a multiple of 4, n <= 2 kThreads; only the upper triangle,
// diagonal included, is read), together with X = L^{-1}, L = U^T: the
// elimination of [C | I], step p subtracting (C_pi / d_p) times row p from
// each row i > p of both halves (d_p the pivot), with row p of both halves
// scaled by d_p^{-1/2} once it is used.  The identity's strict lower part
// lives in A's strict lower triangle (its unit diagonal is implicit).
// Blocked right-looking over panels J of 8 rows [j0, j1):
//  (a) one warp runs the panel's steps on its diagonal block only, giving
//      U_JJ and W = L_JJ^{-1} (for the next panel, while the other warps
//      finish (c) below the next panel's rows: a look-ahead);
//  (b) the rest of the panel's rows is multiplied by W (the composite of
//      the same steps and scalings): U_JK = W C_JK right of the block,
//      X_JK = W R_JK left of it (R the identity half as updated so far);
//  (c) the rows below take the panel's steps at once as the rank-8 update
//      A_ik -= sum_p U_pi S_pk (S = U right of the panel, X and W left of
//      it), in 2 x 4 register tiles.
// On return: A's strict upper triangle holds U and its diagonal U_jj, the
// strict lower triangle X (A[r][j] = X[r][j], j < r), and invd[j] =
// 1/U_jj = X_jj.  Returns false (uniformly) if a pivot is not > 0 or not
// finite.
__device__ inline bool chol_inv_df(const DfMat& A, int n, df* invd) {
  using namespace dense_detail;
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += kThreads) {
    const int r = idx / n, c = idx - r * n;
    if (c < r) A.set(r, c, df{0.f, 0.f});
  }
  const int n4 = n >> 2;
  __syncthreads();
  // (a) of the first panel
  if (tid < 32) {
    const bool ok = factor_diag_block(A, 0, min(kPanel, n), invd);
    if (tid == 0) s_fail = ok ? 0 : 1;
  }
  for (int j0 = 0; j0 < n; j0 += kPanel) {
    const int j1 = min(j0 + kPanel, n), nb = j1 - j0;
    __syncthreads();
    if (s_fail) return false;
    // (b) slot = (row p of the panel, column pair outside the block); all
    // results are formed before any is written
    const int npairs = (n - nb) >> 1;
    const int slots = nb * npairs;
    float2 rh[2], rl[2];
    int rp[2], rc[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int t = tid + s * kThreads;
      rp[s] = -1;
      if (t < slots) {
        const int pi = t / npairs, pc = t - pi * npairs;
        const int c = 2 * pc < j0 ? 2 * pc : 2 * pc + nb;
        const int p = j0 + pi;
        Dot2x2 d;
        for (int m = j0; m <= p; ++m)
          d.add(w_elem(A, invd, p, m), A.hi2(m, c), A.lo2(m, c));
        d.result(rh[s], rl[s]);
        rp[s] = p;
        rc[s] = c;
      }
    }
    static_assert(2 * kThreads >= kPanel * (kMaxB / 2), "two (b) slots per thread");
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 2; ++s)
      if (rp[s] >= 0) A.set2(rp[s], rc[s], rh[s], rl[s]);
    __syncthreads();
    // (c) rows i >= j1: 4 x 4 tiles left of the panel's end (X) and on or
    // right of the diagonal (U), trailing row block I holding n4 - I of
    // them; two slots (row pairs) per tile.  Look-ahead: first the next
    // panel's rows (row blocks I < r1, a prefix of the slots), then one warp
    // factors the next panel's diagonal block while the other warps update
    // the remaining rows, which the next diagonal step does not touch.
    const int j4 = j1 >> 2, m = n4 - j4;
    const int tslots = 2 * (m * n4 - m * (m - 1) / 2);
    const int r1 = min(m, kPanel / 4);
    const int t1 = 2 * (r1 * n4 - r1 * (r1 - 1) / 2);
    auto tile = [&](int t) {
      int I, bj;
      tri_decode(t >> 1, n4, I, bj);
      const int u = bj - I, ib = j4 + I;
      const int kb = u < j4 ? u : ib + (u - j4);
      panel_update_tile(A, invd, j0, j1, 4 * ib + 2 * (t & 1), 4 * kb, kb == ib);
    };
    for (int t = tid; t < t1; t += kThreads) tile(t);
    if (j1 < n) {
      __syncthreads();
      if (tid < 32) {
        const bool ok = factor_diag_block(A, j1, min(j1 + kPanel, n), invd);
        if (tid == 0) s_fail = ok ? 0 : 1;
      } else {
        for (int t = t1 + tid - 32; t < tslots; t += kThreads - 32) tile(t);
      }
    }
  }
  __syncthreads();
  return true;
}

__device__ __forceinline__ void apply_lanes(int B, int tid, int& row, int& sub, int& nl) {
  const int r2 = max(0, 2 * B - kThreads / 2);  // rows on 2 lanes: 0 .. r2 - 1
  const int l4 = 4 * (B - r2);                  // lanes of the 4-lane rows
  if (tid < l4) {
    row = r2 + (tid >> 2);
    sub = tid & 3;
    nl = 4;
  } else if (tid < l4 + 2 * r2) {
    row = (tid - l4) >> 1;
    sub = tid & 1;
    nl = 2;
  } else {
    row = -1;
    sub = 0;
    nl = 2;
  }
}
__device__ __forceinline__ void merge_apply_lanes(Dot2x2& d, int nl) {
  d.merge_lane_pair();
  // every lane takes part in the shuffles; only the 4-lane rows merge
  const float2 s2 = make_float2(__shfl_xor_sync(0xffffffffu, d.s.x, 2),
                                __shfl_xor_sync(0xffffffffu, d.s.y, 2));
  const float2 c2 = make_float2(__shfl_xor_sync(0xffffffffu, d.c.x, 2),
                                __shfl_xor_sync(0xffffffffu, d.c.y, 2));
  if (nl == 4) d.merge(s2, c2);
}
// a scalar Dot2 partial sum merged with that of the lane whose index differs
// in bit `o` (every lane calls; `apply`: this lane takes the merge)
__device__ __forceinline__ void dot2_merge_xor(Dot2& d, int o, bool apply) {
  const float s2 = __shfl_xor_sync(0xffffffffu, d.s, o);
  const float c2 = __shfl_xor_sync(0xffffffffu, d.c, o);
  if (apply) {
    const df t = two_sum(d.s, s2);
    d.s = t.hi;
    d.c = __fadd_rn(d.c, __fadd_rn(c2, t.lo));
  }
}

// z = C^{-1} b = X^T (X b), X from chol_inv_df (strict lower triangle of
// A, diagonal invd); y is scratch; neither may alias b.  Rows (then
// columns) on 4 or 2 lanes as in apply_lanes, compensated sums.
__device__ inline void xtx_apply_df(const DfMat& A, int n, const df* invd, const df* b, df* y, df* z) {
  int r, sub, nl;
  apply_lanes(n, threadIdx.x, r, sub, nl);
  {
    Dot2 d;
    if (r >= 0)
      for (int j = sub; j <= r; j += nl) d.add(j == r ? invd[r] : A.get(r, j), b[j]);
    dot2_merge_xor(d, 1, true);
    dot2_merge_xor(d, 2, nl == 4);
    if (r >= 0 && sub == 0) y[r] = d.result();
  }
  __syncthreads();
  {
    // column j = n - 1 - r holds n - j = r + 1 terms, like row r above
    const int j = n - 1 - r;
    Dot2 d;
    if (r >= 0)
      for (int i = j + sub; i < n; i += nl) d.add(i == j ? invd[j] : A.get(i, j), y[i]);
    dot2_merge_xor(d, 1, true);
    dot2_merge_xor(d, 2, nl == 4);
    if (r >= 0 && sub == 0) z[j] = d.result();
  }
  __syncthreads();
}

// row stride (double-floats) of the B x B scratch matrix the solve kernels
// keep in the region that first holds L^{-1}
__host__ __device__ inline int linv_ld(int B) { return B + 1; }
// The stored inverse factor X = L^{-1} is packed: row i (its i + 1 entries
// j <= i, the diagonal last) starts at i (i + 1) / 2, B (B + 1) / 2
// double-floats in all (a multiple of 16 bytes for B a multiple of 4), half
// the bytes the iteration solves copy per partition of a padded square.
__host__ __device__ inline int linv_row(int i) { return i * (i + 1) / 2; }
__host__ __device__ inline size_t linv_packed(int B) { return (size_t)B * (B + 1) / 2; }

// Z = C^{-1} [a, b] for NP pairs of vectors, with X = L^{-1} packed by rows
// in shared memory (linv_row, as stored by the initial solve).  Pair q comes interleaved,
// UP[q][j] = (a_j.hi, b_j.hi, a_j.lo, b_j.lo); YP[q] is scratch of the same
// form; the results go to Z[2q] (a) and Z[2q + 1] (b).  Y = X U row by row,
// then Z = X^T Y column by column, with packed compensated sums.  A row of
// i + 1 terms (a column of B - i) is split over 4 lanes, each taking every
// fourth term, or over 2 lanes for the first r2 rows (the shortest), so that
// one pass of the block covers all B rows: 4 (B - r2) + 2 r2 <= kThreads.
// The 4-lane rows fill whole warps first, so that no row's lanes straddle a
// warp; the lanes' partial sums are merged by shuffles, always in the same
// order.
template <int NP>
__device__ void c0inv_apply(const df* X, int B, const float4* const* UP, float4* const* YP,
                            df* const* Z) {
  static_assert(kThreads >= 2 * kMaxB, "two lanes per row at the widest window");
  const int tid = threadIdx.x;
  int r, sub, nl;
  apply_lanes(B, tid, r, sub, nl);
  for (int q = 0; q < NP; ++q) {
    Dot2x2 d;
    if (r >= 0) {
      const int i = r;
      const df* row = X + linv_row(i);
      const float4* u = UP[q];
#pragma unroll 4
      for (int j = sub; j <= i; j += nl) {
        const float4 uu = u[j];
        d.add(row[j], make_float2(uu.x, uu.y), make_float2(uu.z, uu.w));
      }
    }
    merge_apply_lanes(d, nl);
    if (r >= 0 && sub == 0) {
      float2 rh, rl;
      d.result(rh, rl);
      YP[q][r] = make_float4(rh.x, rh.y, rl.x, rl.y);
    }
  }
  __syncthreads();
  for (int q = 0; q < NP; ++q) {
    Dot2x2 d;
    // column j = B - 1 - r holds B - j = r + 1 terms, like row r above
    const int j = B - 1 - r;
    if (r >= 0) {
      const float4* y = YP[q];
#pragma unroll 4
      for (int i = j + sub; i < B; i += nl) {
        const float4 yy = y[i];
        d.add(X[linv_row(i) + j], make_float2(yy.x, yy.y), make_float2(yy.z, yy.w));
      }
    }
    merge_apply_lanes(d, nl);
    if (r >= 0 && sub == 0) {
      float2 rh, rl;
      d.result(rh, rl);
      Z[2 * q][j] = df{rh.x, rl.x};
      Z[2 * q + 1][j] = df{rh.y, rl.y};
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float4 pack_pair(df a, df b) { return make_float4(a.hi, b.hi, a.lo, b.lo); }

}  // namespace mf
