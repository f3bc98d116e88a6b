// xt_lane.cuh -- one lane per pair: a single thread extends a whole pair.
//
// For short queries every lane of a warp runs its own pair (the batch is
// bucketed by length, so the lanes of a warp see nearly the same geometry).
// The lane sweeps its pair strip by strip: a strip is R target rows (32-bit
// mode) or two stacked strips of R rows held in the two 16-bit halves of each
// register (packed mode), the upper strip one column behind the lower one so
// that it can take the lower strip's bottom row straight from the previous
// step.  The row above a strip comes from the pair's ring of (H, F) by column
// (shared memory, or a global slab for large rings); the strip writes its own
// bottom row back in place.
//
// Cell update (Eq. 1 read as anchored, banded extension; D = H(i-1,j-1)):
//   M = min(D + S, (m+1)*D)     equals D + S for a live D >= 1 and is <= 0 for
//                               a dead D = 0: the anchoring rule without a branch
//   E = max(E - beta, H(i,j-1) - alpha, 0)   (one fused add-max with relu)
//   F = max(F - beta, H(i-1,j) - alpha, 0)
//   H = max(M, E, F)                          (>= 0 because E >= 0)
// Row maximum with the largest column: 32-bit mode takes max over
// H * 65536 + j; packed mode takes a per-half max with a ">=" predicate
// (__vibmax_s16x2) that moves the column register on ties.
#pragma once
#include <type_traits>

#include "xt_common.cuh"

namespace xt {

enum LaneMode { LM_I32 = 0, LM_P16 = 1 };

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t add16x2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("add.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  return r;
}

__device__ __forceinline__ uint32_t pack16(int32_t lo, int32_t hi) {
  return ((uint32_t)lo & 0xFFFFu) | ((uint32_t)hi << 16);
}
__device__ __forceinline__ int32_t lo16(uint32_t v) { return (int32_t)(int16_t)(v & 0xFFFFu); }
__device__ __forceinline__ int32_t hi16(uint32_t v) { return (int32_t)(int16_t)(v >> 16); }

// Ring of (H, F) for one pair: 32-bit mode keeps int2 entries, packed mode
// one uint32 (H in the low half, F in the high half).
template <bool PACKED>
struct Ring {
  using T = typename std::conditional<PACKED, uint32_t, int2>::type;
  T* base;
  int stride;
  int mask;
  __device__ __forceinline__ T& at(int32_t c) const { return base[(c & mask) * stride]; }
};

// ----------------------------------------------------------- 32-bit lane
template <int R, bool MASKED>
__device__ __forceinline__ void lane_step_i32(int32_t (&Hl)[R], int32_t (&HAl)[R],
                                              int32_t (&El)[R], int32_t (&key)[R],
                                              const uint32_t (&sel)[R], uint32_t prof,
                                              uint32_t nnnn, int32_t Hdiag, int32_t Hup,
                                              int32_t Fup, int32_t c, int32_t alpha,
                                              int32_t beta, int32_t mc, int32_t rlo, int32_t rhi,
                                              int32_t& outH, int32_t& outF) {
  int32_t D = Hdiag;
  int32_t upA = Hup - alpha;
  int32_t upF = Fup;
  int32_t upH = Hup;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int32_t Hleft = Hl[r];
    const int32_t S = prmt_s8(prof, nnnn, sel[r]);
    const int32_t M = __viaddmin_s32(D, S, D * mc);
    int32_t E = __viaddmax_s32_relu(El[r], -beta, HAl[r]);
    int32_t F = __viaddmax_s32_relu(upF, -beta, upA);
    int32_t H = __vimax3_s32(M, E, F);
    if (MASKED) {
      const bool inb = (r >= rlo) && (r <= rhi);
      if (!inb) { H = 0; E = 0; F = 0; }
      if (inb) key[r] = max(key[r], H * 65536 + c);
    } else {
      key[r] = max(key[r], H * 65536 + c);
    }
    const int32_t HA = H - alpha;
    D = Hleft;
    Hl[r] = H; HAl[r] = HA; El[r] = E;
    upH = H; upA = HA; upF = F;
  }
  outH = upH;
  outF = upF;
}

// Extend one pair with one lane, 32-bit (requires h0 + match*min(qlen,tlen)
// <= 32767 and qlen <= 65535 for the row key).
template <int R>
__device__ __forceinline__ Outcome lane_pair_i32(const Pair& pr, const Score& sc,
                                                 const uint32_t* s_prof, const Ring<false>& ring,
                                                 int32_t mc) {
  const int32_t qlen = pr.qlen, tlen = pr.tlen, h0 = pr.h0;
  const int32_t alpha = sc.alpha, beta = sc.beta, w = sc.w;
  const uint32_t nnnn = sc.nnnn;
  RowState st;
  st.init(h0);
  int32_t hi_prev = -1;
  for (int32_t i0 = 0; i0 < tlen; i0 += R) {
    const int32_t rlast = min(tlen - 1, i0 + R - 1);
    const int32_t lo = max(0, i0 - w);
    const int32_t hi = min(qlen - 1, rlast + w);
    if (lo > hi) break;
    int32_t Hl[R], HAl[R], El[R], key[R];
    uint32_t sel[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int32_t i = i0 + r;
      sel[r] = score_selector(i < tlen ? clamp_code(pr.t[i]) : 4u);
      Hl[r] = (lo == 0 && i < tlen) ? col_m1(i, h0, sc) : 0;
      HAl[r] = Hl[r] - alpha;
      El[r] = 0;
      key[r] = -1;
    }
    int32_t Hdiag;
    if (i0 == 0) Hdiag = h0;
    else if (lo == 0) Hdiag = col_m1(i0 - 1, h0, sc);
    else Hdiag = ring.at(lo - 1).x;
    for (int32_t c = lo; c <= hi; ++c) {
      int32_t Hup, Fup;
      if (i0 == 0) {
        Hup = row_m1(c, h0, sc);
        Fup = 0;
      } else {
        const int2 v = ring.at(c);
        const bool ok = c <= hi_prev;
        Hup = ok ? v.x : 0;
        Fup = ok ? v.y : 0;
      }
      const uint32_t prof = s_prof[clamp_code(__ldg(pr.q + c))];
      const int32_t d0 = c - i0;
      const bool body = (d0 >= R - 1 - w) && (d0 <= w) && (i0 + R <= tlen);
      int32_t oH, oF;
      if (__all_sync(__activemask(), body)) {
        lane_step_i32<R, false>(Hl, HAl, El, key, sel, prof, nnnn, Hdiag, Hup, Fup, c, alpha,
                                beta, mc, 0, R - 1, oH, oF);
      } else {
        lane_step_i32<R, true>(Hl, HAl, El, key, sel, prof, nnnn, Hdiag, Hup, Fup, c, alpha,
                               beta, mc, d0 - w, min(d0 + w, tlen - 1 - i0), oH, oF);
      }
      Hdiag = Hup;
      ring.at(c) = make_int2(oH, oF);
    }
    hi_prev = hi;
    // rows in order; H(i, qlen-1) is the last column's H when the sweep reached it
    int32_t last_m = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int32_t i = i0 + r;
      if (i < tlen && !st.stop) {
        const int32_t kv = key[r];
        const int32_t m = kv < 0 ? 0 : (kv >> 16);
        const int32_t mj = kv < 0 ? -1 : (kv & 0xFFFF);
        const bool g_in = hi == qlen - 1 && (qlen - 1 - i <= w) && (i - (qlen - 1) <= w);
        st.feed(i, m, mj, g_in ? Hl[r] : -1, sc);
        last_m = m;
      }
    }
    if (st.stop) break;
    if (last_m == 0 && col_m1(rlast, h0, sc) == 0) break;
  }
  Outcome o;
  o.score = st.best; o.qle = st.bj + 1; o.tle = st.bi + 1; o.gscore = st.gscore;
  o.gtle = st.gtle; o.max_off = st.max_off;
  o.cells = band_cells_upto(st.last_live, qlen, w);
  return o;
}

// ------------------------------------------------------------- packed lane
// One step of the two stacked strips: the lower strip (low halves) at column
// c, the upper strip (high halves) at column c - 1.  All values are packed
// int16x2; H, E, F are >= 0 and bounded ((h0 + match*min(qlen,tlen) + 1) << k
// <= 32767), so no half ever wraps.
//   MASKED: only rows lrlo..lrhi (lower) and hrlo..hrhi (upper) are in band;
//           the others become dead and leave the row maximum alone.
//   KEEP:   0 normal; 1 the upper strip has not started (its state is kept);
//           2 the lower strip has finished (its state is kept).
// sel[r]: byte selector of row r in bits 0-15; bits 16-23 / 24-31 are 0xFF
// when the lower / upper strip's target base is N (score n_score).
// Mj[r]: column of the row maximum, lower strip in bits 0-15, upper in 16-31.
template <int R, bool MASKED, bool HAS_N, int KEEP>
__device__ __forceinline__ void lane_step_p16(uint32_t (&Hl)[R], uint32_t (&HAl)[R],
                                              uint32_t (&El)[R], uint32_t (&Mx)[R],
                                              uint32_t (&Mj)[R], const uint32_t (&sel)[R],
                                              uint32_t prof_lo, uint32_t prof_hi, uint32_t nn2,
                                              uint32_t D, uint32_t Hup, uint32_t Fup, uint32_t C2,
                                              uint32_t na2, uint32_t nb2, uint32_t mcm,
                                              int32_t lrlo, int32_t lrhi, int32_t hrlo,
                                              int32_t hrhi, uint32_t& outH, uint32_t& outF) {
  uint32_t upA = add16x2(Hup, na2);
  uint32_t upF = Fup;
  uint32_t upH = Hup;
  constexpr uint32_t kKeepMask = KEEP == 1 ? 0xFFFF0000u : 0x0000FFFFu;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t Hleft = Hl[r];
    uint32_t S = prmt(prof_lo, prof_hi, sel[r]);
    if (HAS_N) {
      const uint32_t nm = prmt(sel[r], 0u, 0x3322u);  // 0xFFFF in each N half
      S = (S & ~nm) | (nn2 & nm);
    }
    const uint32_t M = __viaddmin_s16x2(D, S, D * mcm);
    uint32_t E = __viaddmax_s16x2_relu(El[r], nb2, HAl[r]);
    uint32_t F = __viaddmax_s16x2_relu(upF, nb2, upA);
    uint32_t H = __vimax3_s16x2(M, E, F);
    bool inl = true, inh = true;
    if (MASKED) {
      inl = r >= lrlo && r <= lrhi;
      inh = r >= hrlo && r <= hrhi;
      const uint32_t bm = (inl ? 0x0000FFFFu : 0u) | (inh ? 0xFFFF0000u : 0u);
      H &= bm;
      E &= bm;
      F &= bm;
    }
    bool ph, pl;
    Mx[r] = __vibmax_s16x2(H, Mx[r], &ph, &pl);
    if (MASKED) {
      pl = pl && inl;
      ph = ph && inh;
    }
    if (pl) Mj[r] = prmt(Mj[r], C2, 0x3254u);  // low half from C2
    if (ph) Mj[r] = prmt(Mj[r], C2, 0x7610u);  // high half from C2
    const uint32_t HA = add16x2(H, na2);
    D = Hleft;
    if (KEEP) {
      Hl[r] = (Hleft & kKeepMask) | (H & ~kKeepMask);
      HAl[r] = (HAl[r] & kKeepMask) | (HA & ~kKeepMask);
      El[r] = (El[r] & kKeepMask) | (E & ~kKeepMask);
    } else {
      Hl[r] = H; HAl[r] = HA; El[r] = E;
    }
    upH = H; upA = HA; upF = F;
  }
  outH = upH;
  outF = upF;
}

// Extend one pair with one lane in packed 16-bit arithmetic.  mshift = k with
// 2^k >= match + 1; the caller guarantees (h0 + match*min(qlen,tlen) + 1) << k
// <= 32767 and qlen <= 65535.
template <int R>
__device__ __forceinline__ Outcome lane_pair_p16(const Pair& pr, const Score& sc,
                                                 const uint32_t* s_prof, const Ring<true>& ring,
                                                 int mshift) {
  const int32_t qlen = pr.qlen, tlen = pr.tlen, h0 = pr.h0;
  const int32_t alpha = sc.alpha, beta = sc.beta, w = sc.w;
  const uint32_t na2 = pack16(-alpha, -alpha), nb2 = pack16(-beta, -beta);
  const int32_t nsc = (int32_t)(int8_t)(sc.nnnn & 0xFF);
  const uint32_t nn2 = pack16(nsc, nsc);
  // halves are >= 0 and below 2^(15-k): a 32-bit multiply by 2^k shifts each half
  const uint32_t mcm = 1u << mshift;
  constexpr int RR = 2 * R;
  RowState st;
  st.init(h0);
  int32_t hi_prev = -1;
  for (int32_t i0 = 0; i0 < tlen; i0 += RR) {
    const int32_t rlast = min(tlen - 1, i0 + RR - 1);
    const int32_t lo = max(0, i0 - w);
    const int32_t hi = min(qlen - 1, rlast + w);
    if (lo > hi) break;
    uint32_t Hl[R], HAl[R], El[R], Mx[R], sel[R], Mj[R];
    uint32_t anyN = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int32_t il = i0 + r, ih = i0 + R + r;
      const uint32_t cl = il < tlen ? clamp_code(pr.t[il]) : 0u;
      const uint32_t ch = ih < tlen ? clamp_code(pr.t[ih]) : 0u;
      const uint32_t bl = cl & 3u, bh = 4u + (ch & 3u);
      const uint32_t nf = (cl == 4u ? 0x00FF0000u : 0u) | (ch == 4u ? 0xFF000000u : 0u);
      sel[r] = bl | ((bl | 8u) << 4) | (bh << 8) | ((bh | 8u) << 12) | nf;
      anyN |= nf;
      // both strips start from column lo - 1 (column -1 when lo == 0)
      const int32_t hl = (lo == 0 && il < tlen) ? col_m1(il, h0, sc) : 0;
      const int32_t hh = (lo == 0 && ih < tlen) ? col_m1(ih, h0, sc) : 0;
      Hl[r] = pack16(hl, hh);
      HAl[r] = add16x2(Hl[r], na2);
      El[r] = 0;
      Mx[r] = 0;
      Mj[r] = 0xFFFFFFFFu;  // -1 in both halves: no column yet
    }
    const bool has_n = __any_sync(__activemask(), anyN != 0);
    // lower strip's diagonal at its first column: H(i0-1, lo-1)
    int32_t dlo;
    if (i0 == 0) dlo = h0;
    else if (lo == 0) dlo = col_m1(i0 - 1, h0, sc);
    else dlo = lo16(ring.at(lo - 1));
    // lower strip's bottom row (row i0+R-1) at the previous column and the one
    // before; at column lo - 1 it is the left boundary
    const int32_t lb = (lo == 0 && i0 + R - 1 < tlen) ? col_m1(i0 + R - 1, h0, sc) : 0;
    int32_t botH1 = lb, botF1 = lb, botH2 = lb;
    uint32_t prof_prev = 0;
    const int32_t nsteps = hi - lo + 2;
    // software pipeline: query codes two columns ahead, profile and ring one ahead
    const int32_t qlast = qlen - 1;
    uint32_t code_n = clamp_code(__ldg(pr.q + min(lo + 1, qlast)));
    uint32_t prof_c = s_prof[clamp_code(__ldg(pr.q + lo))];
    uint32_t ring_c = ring.at(lo);
    for (int32_t s = 0; s < nsteps; ++s) {
      const int32_t c = lo + s;  // lower strip column; the upper strip is at c - 1
      const bool lo_act = c <= hi;
      const bool hi_act = s >= 1;
      // issue the next step's loads first
      const uint32_t code_nn = clamp_code(__ldg(pr.q + min(c + 2, qlast)));
      const uint32_t prof_n = s_prof[code_n];
      const uint32_t ring_n = ring.at(c + 1);
      int32_t tH = 0, tF = 0;  // row above the lower strip at column c
      if (lo_act) {
        if (i0 == 0) {
          tH = row_m1(c, h0, sc);
        } else if (c <= hi_prev) {
          tH = lo16(ring_c);
          tF = hi16(ring_c);
        }
      }
      const uint32_t prof = lo_act ? prof_c : 0u;
      const uint32_t Hup = pack16(tH, botH1);
      const uint32_t Fup = pack16(tF, botF1);
      const uint32_t D = pack16(dlo, botH2);
      const uint32_t C2 = pack16(c, c - 1);
      const int32_t d0 = c - i0;
      const bool body = lo_act && hi_act && d0 >= RR - w && d0 <= w && i0 + RR <= tlen;
      uint32_t oH, oF;
      if (__all_sync(__activemask(), body)) {
        if (has_n)
          lane_step_p16<R, false, true, 0>(Hl, HAl, El, Mx, Mj, sel, prof, prof_prev, nn2, D,
                                           Hup, Fup, C2, na2, nb2, mcm, 0, R - 1, 0, R - 1, oH,
                                           oF);
        else
          lane_step_p16<R, false, false, 0>(Hl, HAl, El, Mx, Mj, sel, prof, prof_prev, nn2, D,
                                            Hup, Fup, C2, na2, nb2, mcm, 0, R - 1, 0, R - 1, oH,
                                            oF);
      } else {
        // in-band rows: |i - col| <= w and i < tlen, for an active strip only
        const int32_t lrlo = lo_act ? d0 - w : R;
        const int32_t lrhi = lo_act ? min(d0 + w, tlen - 1 - i0) : -1;
        const int32_t dh = d0 - 1 - R;  // upper strip: column c-1 minus its first row
        const int32_t hrlo = hi_act ? dh - w : R;
        const int32_t hrhi = hi_act ? min(dh + w, tlen - 1 - i0 - R) : -1;
        if (s == 0)
          lane_step_p16<R, true, true, 1>(Hl, HAl, El, Mx, Mj, sel, prof, prof_prev, nn2, D, Hup,
                                          Fup, C2, na2, nb2, mcm, lrlo, lrhi, hrlo, hrhi, oH, oF);
        else if (!lo_act)
          lane_step_p16<R, true, true, 2>(Hl, HAl, El, Mx, Mj, sel, prof, prof_prev, nn2, D, Hup,
                                          Fup, C2, na2, nb2, mcm, lrlo, lrhi, hrlo, hrhi, oH, oF);
        else
          lane_step_p16<R, true, true, 0>(Hl, HAl, El, Mx, Mj, sel, prof, prof_prev, nn2, D, Hup,
                                          Fup, C2, na2, nb2, mcm, lrlo, lrhi, hrlo, hrhi, oH, oF);
      }
      if (hi_act) ring.at(c - 1) = (oH >> 16) | (oF & 0xFFFF0000u);
      botH2 = botH1;
      botH1 = lo16(oH);
      botF1 = lo16(oF);
      dlo = tH;
      prof_prev = prof;
      prof_c = prof_n;
      code_n = code_nn;
      ring_c = ring_n;
    }
    hi_prev = hi;
    int32_t last_m = 0;
    const bool reach = hi == qlen - 1;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int32_t i = i0 + half * R + r;
        if (i < tlen && !st.stop) {
          const int32_t m = half ? hi16(Mx[r]) : lo16(Mx[r]);
          const int32_t mj = half ? hi16(Mj[r]) : lo16(Mj[r]);
          // after the sweep, Hl holds H(i, hi) of both strips (each strip kept
          // its state once it had passed column hi)
          const bool g_in = reach && (qlen - 1 - i <= w) && (i - (qlen - 1) <= w);
          const int32_t g = g_in ? (half ? hi16(Hl[r]) : lo16(Hl[r])) : -1;
          st.feed(i, m, mj, g, sc);
          last_m = m;
        }
      }
    }
    if (st.stop) break;
    if (last_m == 0 && col_m1(rlast, h0, sc) == 0) break;
  }
  Outcome o;
  o.score = st.best; o.qle = st.bj + 1; o.tle = st.bi + 1; o.gscore = st.gscore;
  o.gtle = st.gtle; o.max_off = st.max_off;
  o.cells = band_cells_upto(st.last_live, qlen, w);
  return o;
}

}  // namespace xt
