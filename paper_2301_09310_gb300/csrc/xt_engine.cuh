// xt_engine.cuh -- strip-wavefront extension of one pair by a group of P lanes.
//
// Layout (cf. the intra-query scheme of arXiv 2301.09310 Sec. IV-A, here on
// a band and with the boundary row passed by warp shuffles):
//   * the target rows are cut into strips of R rows; a chunk is P consecutive
//     strips, lane p of the group owns strip p of every chunk;
//   * within a chunk the lanes sweep the chunk's band columns [lo, hi], lane p
//     one column behind lane p-1 (anti-diagonal wavefront); each step a lane
//     updates its R cells of one column, keeping H, H - alpha and E of its
//     rows in registers and receiving the row above (H, F) from lane p-1 by
//     __shfl_up_sync;
//   * the bottom row of the chunk (lane P-1) goes to a ring of (H, F) pairs
//     indexed by column, which lane 0 reads back for the next chunk -- the
//     band keeps the live span of columns below P*R + 2w + 2, so the ring is
//     a small power of two in shared memory (or a global slab for huge bands);
//   * after each chunk the group walks the chunk's rows in row order through
//     RowState (row maximum with largest column, gscore, z-drop), exactly as
//     the definition orders them, and stops at the z-drop row or at a dead
//     row (every later row is then dead too).
// Row maximum and its column come from one integer max over H * 65536 + j,
// so ties resolve to the largest column for free (valid while H < 32768 and
// j < 65536; the WIDE variant keeps the pair explicitly).
#pragma once
#include "xt_common.cuh"

namespace xt {

template <int R, bool MASKED, bool WIDE>
__device__ __forceinline__ void step_cells(int32_t (&Hl)[R], int32_t (&HAl)[R], int32_t (&El)[R],
                                           int32_t (&key)[R], int32_t (&mrow)[R],
                                           int32_t (&mjrow)[R], const uint32_t (&sel)[R],
                                           uint32_t prof, uint32_t nnnn, int32_t Hdiag,
                                           int32_t Hup, int32_t Fup, int32_t c, int32_t alpha,
                                           int32_t beta, int32_t rlo, int32_t rhi,
                                           int32_t& outH, int32_t& outF) {
  int32_t D = Hdiag;          // H(i-1, c-1) of the current row
  int32_t upA = Hup - alpha;  // H(i-1, c) - alpha
  int32_t upF = Fup;          // F(i-1, c)
  int32_t upH = Hup;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int32_t Hleft = Hl[r];  // H(i, c-1): next row's diagonal
    const int32_t S = prmt_s8(prof, nnnn, sel[r]);
    // anchoring: a dead diagonal (H = 0) gives no match continuation
    const int32_t M = (D > 0) ? D + S : 0;
    int32_t E = __viaddmax_s32(El[r], -beta, HAl[r]);  // max(E(i,c-1) - beta, H(i,c-1) - alpha)
    int32_t F = __viaddmax_s32(upF, -beta, upA);       // max(F(i-1,c) - beta, H(i-1,c) - alpha)
    int32_t H = __vimax3_s32_relu(M, E, F);            // max(0, M, E, F)
    bool inb = true;
    if (MASKED) {
      inb = (r >= rlo) && (r <= rhi);
      if (!inb) { H = 0; E = 0; F = 0; }
    }
    const int32_t HA = H - alpha;
    if (WIDE) {
      if (inb && H >= mrow[r]) { mrow[r] = H; mjrow[r] = c; }
    } else {
      const int32_t kk = H * 65536 + c;
      if (MASKED) { if (inb) key[r] = max(key[r], kk); }
      else key[r] = max(key[r], kk);
    }
    D = Hleft;
    Hl[r] = H; HAl[r] = HA; El[r] = E;
    upH = H; upA = HA; upF = F;
  }
  outH = upH;
  outF = upF;
}

// Extend one pair with the P lanes of a group (lane p of P, group lanes gmask).
// ring: the group's (H, F) ring, element c at ring[(c & rmask) * stride].
// s_prof: the five query profiles in shared memory.
template <int P, int R, bool WIDE>
__device__ __forceinline__ Outcome run_pair(const Pair& pr, const Score& sc,
                                            const uint32_t* s_prof, int2* ring, int stride,
                                            int rmask, int p, unsigned gmask) {
  const int32_t qlen = pr.qlen, tlen = pr.tlen, h0 = pr.h0;
  const int32_t alpha = sc.alpha, beta = sc.beta, w = sc.w;
  const uint32_t nnnn = sc.nnnn;
  RowState st;
  st.init(h0);
  int32_t hi_prev = -1;
  for (int32_t r0 = 0; r0 < tlen; r0 += P * R) {
    const int32_t rlast = min(tlen - 1, r0 + P * R - 1);
    const int32_t lo = max(0, r0 - w);
    const int32_t hi = min(qlen - 1, rlast + w);
    if (lo > hi) break;  // every row from r0 on has an empty band
    const int32_t i0 = r0 + p * R;
    const bool lane_live = i0 < tlen;
    int32_t Hl[R], HAl[R], El[R], key[R], gval[R], mrow[R], mjrow[R];
    uint32_t sel[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int32_t i = i0 + r;
      const uint32_t tb = (i < tlen) ? clamp_code(pr.t[i]) : 4u;
      sel[r] = score_selector(tb);
      Hl[r] = (lo == 0 && i < tlen) ? col_m1(i, h0, sc) : 0;
      HAl[r] = Hl[r] - alpha;
      El[r] = 0;
      key[r] = -1;
      gval[r] = -1;
      mrow[r] = 0;
      mjrow[r] = -1;
    }
    int32_t Hdiag;  // H(i0 - 1, lo - 1)
    if (p == 0) {
      if (r0 == 0) Hdiag = h0;
      else if (lo == 0) Hdiag = col_m1(r0 - 1, h0, sc);
      else Hdiag = ring[((lo - 1) & rmask) * stride].x;
    } else {
      Hdiag = (lo == 0) ? col_m1(i0 - 1, h0, sc) : 0;
    }
    const int32_t nsteps = hi - lo + P;
    int32_t botH = 0, botF = 0;
    for (int32_t s = 0; s < nsteps; ++s) {
      int32_t nbH = 0, nbF = 0;
      if (P > 1) {
        nbH = __shfl_up_sync(gmask, botH, 1, P);
        nbF = __shfl_up_sync(gmask, botF, 1, P);
      }
      const int32_t c = lo + s - p;
      if (lane_live && c >= lo && c <= hi) {
        int32_t Hup, Fup;
        if (p == 0) {
          if (r0 == 0) {
            Hup = row_m1(c, h0, sc);
            Fup = 0;
          } else if (c <= hi_prev) {
            const int2 v = ring[(c & rmask) * stride];
            Hup = v.x;
            Fup = v.y;
          } else {
            Hup = 0;
            Fup = 0;
          }
        } else {
          Hup = nbH;
          Fup = nbF;
        }
        const uint32_t prof = s_prof[clamp_code(__ldg(pr.q + c))];
        const int32_t d0 = c - i0;
        const bool body = (d0 >= R - 1 - w) && (d0 <= w) && (i0 + R <= tlen);
        int32_t oH, oF;
        if (__all_sync(__activemask(), body)) {
          step_cells<R, false, WIDE>(Hl, HAl, El, key, mrow, mjrow, sel, prof, nnnn, Hdiag, Hup,
                                     Fup, c, alpha, beta, 0, R - 1, oH, oF);
        } else {
          const int32_t rlo = d0 - w;
          const int32_t rhi = min(d0 + w, tlen - 1 - i0);
          step_cells<R, true, WIDE>(Hl, HAl, El, key, mrow, mjrow, sel, prof, nnnn, Hdiag, Hup,
                                    Fup, c, alpha, beta, rlo, rhi, oH, oF);
        }
        if (c == qlen - 1) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int32_t i = i0 + r;
            const bool inb = (i < tlen) && (c - i <= w) && (i - c <= w);
            gval[r] = inb ? Hl[r] : -1;
          }
        }
        Hdiag = Hup;
        botH = oH;
        botF = oF;
        if (p == P - 1) ring[(c & rmask) * stride] = make_int2(oH, oF);
      } else {
        botH = 0;
        botF = 0;
      }
    }
    if (P > 1) __syncwarp(gmask);
    hi_prev = hi;
    // Row summaries of the chunk, in row order.
    int32_t last_m = 0;
    for (int pp = 0; pp < P; ++pp) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int32_t kv = key[r], gv = gval[r], mv = mrow[r], mjv = mjrow[r];
        if (P > 1) {
          gv = __shfl_sync(gmask, gv, pp, P);
          if (WIDE) {
            mv = __shfl_sync(gmask, mv, pp, P);
            mjv = __shfl_sync(gmask, mjv, pp, P);
          } else {
            kv = __shfl_sync(gmask, kv, pp, P);
          }
        }
        const int32_t i = r0 + pp * R + r;
        if (i < tlen && !st.stop) {
          int32_t m, mj;
          if (WIDE) {
            m = mv;
            mj = mjv;
          } else {
            m = kv < 0 ? 0 : (kv >> 16);
            mj = kv < 0 ? -1 : (kv & 0xFFFF);
          }
          st.feed(i, m, mj, gv, sc);
          last_m = m;
        }
      }
    }
    if (st.stop) break;
    // A dead row (all in-band H = 0, boundary cell dead) kills every later row.
    if (last_m == 0 && col_m1(rlast, h0, sc) == 0) break;
  }
  Outcome o;
  o.score = st.best;
  o.qle = st.bj + 1;
  o.tle = st.bi + 1;
  o.gscore = st.gscore;
  o.gtle = st.gtle;
  o.max_off = st.max_off;
  o.cells = band_cells_upto(st.last_live, qlen, w);
  return o;
}

}  // namespace xt
