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

// Query codes of one pair: read from global memory, or from a copy staged in
// shared memory (byte c of the lane at stage[c * 32], lanes of a warp
// interleaved so that a warp reading one column hits 32 consecutive bytes).
template <bool STAGED>
struct Query {
  const uint8_t* g;  // global query
  uint8_t* stage;    // this lane's column 0 in the warp's stage
  __device__ __forceinline__ void load(int32_t qlen, bool live) {
    if (STAGED && live)
      for (int32_t c = 0; c < qlen; ++c) stage[c * 32] = (uint8_t)clamp_code(__ldg(g + c));
  }
  __device__ __forceinline__ uint32_t code(int32_t c) const {
    if (STAGED) return stage[c * 32];
    return clamp_code(__ldg(g + c));
  }
};

// The previous strip's bottom row, fed column by column through shared
// memory for rings in a global slab: each lane keeps D = 8 slots (measured
// on c4_long: 8 beat 16 and 32, whose larger footprint takes L1 capacity),
// and the entry of column c sits in slot c mod D.  A strip first starts copying its
// columns lo .. lo+D-1 (cp.async, one commit group each); the step that
// consumes column c waits until that copy has landed (at most D-1 younger
// groups pending), reads the slot and refills it with column c+D.  Only
// columns the strip consumes are copied, so no copy is in flight when the
// strip ends; steps without a copy still commit an (empty) group to keep the
// count.  The copies run D steps ahead of their use instead of the two that
// registers allow.  Slot k of lane t sits at slot0 + k * kLaneThreads.
constexpr int kPipeD = 8;

template <typename T>
struct RingPipe {
  T* slot0;  // this lane's slot 0 (shared memory)
  __device__ __forceinline__ T* slot(int32_t c) const {
    return slot0 + (uint32_t)(c & (kPipeD - 1)) * kLaneThreads;
  }
  __device__ __forceinline__ void copy(const T* src, int32_t c) const {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(slot(c));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src),
                 "n"((int)sizeof(T))
                 : "memory");
  }
  __device__ __forceinline__ void commit() const {
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  // the entry of column c, once its copy has landed
  __device__ __forceinline__ T take(int32_t c) const {
    asm volatile("cp.async.wait_group %0;" ::"n"(kPipeD - 1) : "memory");
    return *slot(c);
  }
};

// Unrolling of the fast-step loop of the packed engine (a tuning knob of the
// build: the loop body is large, so unrolling trades register renaming of
// the pipelined values against instruction-cache footprint).  Two copies
// measured fastest on c3_mixed (18.6 ms of DP per 4M pairs against 19.1 for
// one copy, 20.4 for three; four spill).
#ifndef XT_FAST_UNROLL_N
#define XT_FAST_UNROLL_N 2
#endif
constexpr int kFastUnroll = XT_FAST_UNROLL_N;

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

// Extend the pairs of one warp, one pair per lane, 32-bit (requires h0 +
// match*min(qlen,tlen) <= 32767 and qlen <= 65535 for the row key).  Lanes
// walk their strips in lockstep, as in the packed form.
template <int R, bool PIPE>
__device__ __forceinline__ Outcome lane_pair_i32(const Pair& pr, bool valid, const Score& sc,
                                                 const uint32_t* s_prof, const Ring<false>& ring,
                                                 int32_t mc, const RingPipe<int2>& pipe) {
  const int32_t qlen = pr.qlen, tlen = pr.tlen, h0 = pr.h0;
  const int32_t alpha = sc.alpha, beta = sc.beta, w = sc.w;
  const uint32_t nnnn = sc.nnnn;
  RowState st;
  st.init(h0);
  bool live = valid;
  int32_t hi_prev = -1;
  for (int32_t i0 = 0;; i0 += R) {
    int32_t lo = 1, hi = 0, rlast = 0;
    if (live) {
      rlast = min(tlen - 1, i0 + R - 1);
      lo = max(0, i0 - w);
      hi = min(qlen - 1, rlast + w);
      if (i0 >= tlen || lo > hi) live = false;
    }
    if (!__any_sync(0xffffffffu, live)) break;
    int32_t Hl[R], HAl[R], El[R], key[R];
    uint32_t sel[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int32_t i = i0 + r;
      sel[r] = score_selector((live && i < tlen) ? clamp_code(pr.t[i]) : 4u);
      Hl[r] = (lo == 0 && i < tlen) ? col_m1(i, h0, sc) : 0;
      HAl[r] = Hl[r] - alpha;
      El[r] = 0;
      key[r] = -1;
    }
    int32_t Hdiag = 0;
    if (i0 == 0) Hdiag = h0;
    else if (lo == 0) Hdiag = col_m1(i0 - 1, h0, sc);
    else if (live) Hdiag = ring.at(lo - 1).x;
    const int32_t nsteps = live ? hi - lo + 1 : 0;
    const int32_t nmax = __reduce_max_sync(0xffffffffu, nsteps);
    // the unmasked range: every live lane in its band body, every row in
    // band, and the previous strip's row present at the column
    constexpr int32_t kFar = 1 << 30;
    int32_t sb_lo = 0, sb_hi = kFar;
    if (live) {
      sb_lo = max(0, R - 1 - w + i0 - lo);
      sb_hi = min(hi - lo, w + i0 - lo);
      if (i0 > 0) sb_hi = min(sb_hi, hi_prev - lo);
      if (i0 + R > tlen) sb_hi = -1;
    }
    const int32_t fs = (int32_t)__reduce_max_sync(0xffffffffu, (uint32_t)sb_lo);
    const int32_t fe = min(__reduce_min_sync(0xffffffffu, sb_hi), nmax - 1);
    const int32_t qlast = max(qlen - 1, 0);
    uint32_t code_n = live ? clamp_code(__ldg(pr.q + min(lo + 1, qlast))) : 0u;
    uint32_t prof_c = s_prof[live ? clamp_code(__ldg(pr.q + lo)) : 0u];
    int2 ring_c = make_int2(0, 0), ring_n1 = make_int2(0, 0);
    // the last column the strip consumes a ring entry of: its steps end at
    // column lo + nmax - 1, and the previous strip wrote up to hi_prev
    const int32_t last_c = min(hi_prev, lo + nmax - 1);
    if (PIPE) {
      if (i0 > 0) {  // the first strip reads row -1, not the ring
#pragma unroll
        for (int k = 0; k < kPipeD; ++k) {
          if (live && lo + k <= last_c) pipe.copy(&ring.at(lo + k), lo + k);
          pipe.commit();
        }
      }
    } else {
      ring_c = live ? ring.at(lo) : make_int2(0, 0);
      ring_n1 = live ? ring.at(lo + 1) : make_int2(0, 0);
    }
    // the entry of column c, and the copy of column c + kPipeD into its slot
    auto feed = [&](int32_t c) -> int2 {
      const int2 v = pipe.take(c);
      if (live && c + kPipeD <= last_c) pipe.copy(&ring.at(c + kPipeD), c + kPipeD);
      pipe.commit();
      return v;
    };
    auto slow_step = [&](int32_t s) {
      const int32_t c = lo + s;
      const bool act = live && c <= hi;
      const uint32_t code_nn = act ? clamp_code(__ldg(pr.q + min(c + 2, qlast))) : 0u;
      const uint32_t prof_n = s_prof[code_n];
      const int2 ring_n2 = (!PIPE && act) ? ring.at(c + 2) : make_int2(0, 0);
      int32_t Hup = 0, Fup = 0;
      if (i0 > 0 && PIPE) ring_c = feed(c);
      if (act) {
        if (i0 == 0) {
          Hup = row_m1(c, h0, sc);
        } else if (c <= hi_prev) {
          Hup = ring_c.x;
          Fup = ring_c.y;
        }
      }
      const int32_t d0 = c - i0;
      int32_t oH, oF;
      if (act)
        lane_step_i32<R, true>(Hl, HAl, El, key, sel, prof_c, nnnn, Hdiag, Hup, Fup, c, alpha,
                               beta, mc, d0 - w, min(d0 + w, tlen - 1 - i0), oH, oF);
      if (act) ring.at(c) = make_int2(oH, oF);
      Hdiag = Hup;
      prof_c = prof_n;
      code_n = code_nn;
      ring_c = ring_n1;
      ring_n1 = ring_n2;
    };
    // nothing masked or checked; lanes without a pair compute on garbage and
    // store only into their own ring, which they never read again
    auto fast_step = [&](int32_t s) {
      const int32_t c = lo + s;
      const uint32_t code_nn = live ? clamp_code(__ldg(pr.q + min(c + 2, qlast))) : 0u;
      const uint32_t prof_n = s_prof[code_n];
      const int2 ring_n2 = PIPE ? make_int2(0, 0) : ring.at(c + 2);
      int32_t Hup, Fup;
      if (i0 == 0) {
        Hup = row_m1(c, h0, sc);
        Fup = 0;
      } else {
        if (PIPE) ring_c = feed(c);
        Hup = ring_c.x;
        Fup = ring_c.y;
      }
      int32_t oH, oF;
      lane_step_i32<R, false>(Hl, HAl, El, key, sel, prof_c, nnnn, Hdiag, Hup, Fup, c, alpha, beta,
                              mc, 0, R - 1, oH, oF);
      ring.at(c) = make_int2(oH, oF);
      Hdiag = Hup;
      prof_c = prof_n;
      code_n = code_nn;
      ring_c = ring_n1;
      ring_n1 = ring_n2;
    };
    int32_t s = 0;
    while (s < nmax) {
      if (s >= fs && s <= fe) {
        for (; s <= fe; ++s) fast_step(s);
      } else {
        slow_step(s);
        ++s;
      }
    }
    hi_prev = hi;
    if (live) {
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
      if (st.stop || (last_m == 0 && col_m1(rlast, h0, sc) == 0)) live = false;
    }
  }
  Outcome o;
  o.score = st.best; o.qle = st.bj + 1; o.tle = st.bi + 1; o.gscore = st.gscore;
  o.gtle = st.gtle; o.max_off = st.max_off;
  o.cells = band_cells_upto(st.last_live, qlen, w);
  return o;
}

// ------------------------------------------------------------- packed lane
// Row maximum in packed form: within blocks of 2^TB steps each half keeps
// key = H * 2^TB + (step within the block), so one packed max keeps the
// largest H with the latest (largest) column; at the end of a block the keys
// are folded into 32-bit (H << 16 | column) per row.  TB = 6 needs H <= 511,
// TB = 4 (a fold every 16 steps) H <= 2047.
constexpr uint32_t kKeyNone = 0x80008000u;  // -32768 in both halves: no key yet

// One step of the two stacked strips: the lower strip (low halves) at column
// c, the upper strip (high halves) at column c - 1.  All values are packed
// int16x2; H, E, F are >= 0 and bounded, so no half ever wraps.
//   MASKED: bit r (lower strip) / bit 16 + r (upper strip) of `inband` says
//     whether row r's cell is in band.  An out-of-band cell gets H = F = 0:
//     that is all its in-band neighbours can read (E of a cell left of the
//     band is rebuilt from a dead H; E of a cell right of it only flows
//     further right).  Its row key may move, but only to H = 0, and a row
//     whose maximum is 0 takes its column from the band geometry instead.
//   KEEP: halves set in `keep` (a strip that has not started, or has
//     finished) keep their state.
// sel[r]: byte selector of row r in bits 0-15; bits 16-23 / 24-31 are 0xFF
// when the lower / upper strip's target base is N (score n_score).
template <int R, bool MASKED, bool HAS_N, bool KEEP, int TB = 6>
__device__ __forceinline__ void lane_step_p16(uint32_t (&Hl)[R], uint32_t (&HAl)[R],
                                              uint32_t (&El)[R], uint32_t (&K)[R],
                                              const uint32_t (&sel)[R], uint32_t prof_lo,
                                              uint32_t prof_hi, uint32_t nn2, uint32_t D,
                                              uint32_t Hup, uint32_t Fup, uint32_t pos2,
                                              uint32_t na2, uint32_t nb2, uint32_t mcm,
                                              uint32_t inband, uint32_t keep, uint32_t& outH,
                                              uint32_t& outF) {
  uint32_t upA = add16x2(Hup, na2);
  uint32_t upF = Fup;
  uint32_t upH = Hup;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t Hleft = Hl[r];
    uint32_t S = prmt(prof_lo, prof_hi, sel[r]);
    if (HAS_N) {
      const uint32_t nm = prmt(sel[r], 0u, 0x3322u);  // 0xFFFF in each N half
      S = (S & ~nm) | (nn2 & nm);
    }
    const uint32_t M = __viaddmin_s16x2(D, S, D * mcm);
    const uint32_t E = __viaddmax_s16x2_relu(El[r], nb2, HAl[r]);
    uint32_t F = __viaddmax_s16x2_relu(upF, nb2, upA);
    uint32_t H = __vimax3_s16x2(M, E, F);
    if (MASKED) {
      // bits r and 16 + r moved to the sign bits of bytes 1 and 3, then spread
      const uint32_t bm = prmt(inband << (15 - r), 0u, 0xBB99u);
      H &= bm;
      F &= bm;
    }
    // H * 2^TB + step, both halves at once (halves >= 0 and small enough that
    // neither carries into the other)
    asm("max.s16x2 %0, %0, %1;" : "+r"(K[r]) : "r"(H * (uint32_t)(1 << TB) + pos2));
    const uint32_t HA = add16x2(H, na2);
    D = Hleft;
    if (KEEP) {
      Hl[r] = (Hleft & keep) | (H & ~keep);
      HAl[r] = (HAl[r] & keep) | (HA & ~keep);
      El[r] = (El[r] & keep) | (E & ~keep);
    } else {
      Hl[r] = H; HAl[r] = HA; El[r] = E;
    }
    upH = H; upA = HA; upF = F;
  }
  outH = upH;
  outF = upF;
}

// Bits lo..hi (clamped to 0..n-1) set; 0 when the range is empty.
__device__ __forceinline__ uint32_t bit_range(int32_t lo, int32_t hi, int n) {
  lo = max(lo, 0);
  hi = min(hi, n - 1);
  if (lo > hi) return 0u;
  return ((2u << hi) - 1u) & ~((1u << lo) - 1u);
}

// Fold the block keys into the per-row (H << 16 | column) maxima; cbase is
// the lower strip's column of block step 0 (the upper strip's is cbase - 1).
template <int R, int TB>
__device__ __forceinline__ void fold_keys(uint32_t (&K)[R], int32_t (&Blo)[R], int32_t (&Bhi)[R],
                                          int32_t cbase) {
  constexpr int32_t kMask = (1 << TB) - 1;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int32_t kl = lo16(K[r]), kh = hi16(K[r]);
    if (kl >= 0) Blo[r] = max(Blo[r], ((kl >> TB) << 16) | (cbase + (kl & kMask)));
    if (kh >= 0) Bhi[r] = max(Bhi[r], ((kh >> TB) << 16) | (cbase - 1 + (kh & kMask)));
    K[r] = kKeyNone;
  }
}

// Extend the pairs of one warp, one pair per lane, in packed 16-bit
// arithmetic.  The lanes walk their strips in lockstep (the batch is ordered
// by exact query length, so the 32 pairs of a warp share one geometry) and a
// lane whose pair is done, or has no pair (valid = false), idles masked.
// mshift = k with 2^k >= match + 1.  The caller guarantees, with B = h0 +
// match*min(qlen,tlen): (B + 1) << k <= 32767, (B + 1) * 2^TB - 1 <= 32767 (the row keys),
// 1 <= qlen <= 65535 and tlen >= 1.
template <int R, bool STAGED, int TB = 6>
__device__ __forceinline__ Outcome lane_pair_p16(const Pair& pr, bool valid, const Score& sc,
                                                 const uint32_t* s_prof, const Ring<true>& ring,
                                                 int mshift, Query<STAGED> qs) {
  const int32_t qlen = pr.qlen, tlen = pr.tlen, h0 = pr.h0;
  const int32_t alpha = sc.alpha, beta = sc.beta, w = sc.w;
  const uint32_t na2 = pack16(-alpha, -alpha), nb2 = pack16(-beta, -beta);
  const int32_t nsc = (int32_t)(int8_t)(sc.nnnn & 0xFF);
  const uint32_t nn2 = pack16(nsc, nsc);
  // halves are >= 0 and below 2^(15-k): a 32-bit multiply by 2^k shifts each half
  const uint32_t mcm = 1u << mshift;
  constexpr int32_t kTagSteps = 1 << TB;  // steps per row-key block
  constexpr int RR = 2 * R;
  constexpr int32_t kFar = 1 << 30;
  RowState st;
  st.init(h0);
  bool live = valid;
  qs.load(qlen, live);
  int32_t hi_prev = -1;
  for (int32_t i0 = 0;; i0 += RR) {
    int32_t lo = 1, hi = 0, rlast = 0;
    if (live) {
      rlast = min(tlen - 1, i0 + RR - 1);
      lo = max(0, i0 - w);
      hi = min(qlen - 1, rlast + w);
      if (i0 >= tlen || lo > hi) live = false;
    }
    if (!__any_sync(0xffffffffu, live)) break;
    uint32_t Hl[R], HAl[R], El[R], K[R], sel[R];
    int32_t Blo[R], Bhi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int32_t il = i0 + r, ih = i0 + R + r;
      const uint32_t cl = (live && il < tlen) ? clamp_code(pr.t[il]) : 0u;
      const uint32_t ch = (live && ih < tlen) ? clamp_code(pr.t[ih]) : 0u;
      const uint32_t bl = cl & 3u, bh = 4u + (ch & 3u);
      const uint32_t nf = (cl == 4u ? 0x00FF0000u : 0u) | (ch == 4u ? 0xFF000000u : 0u);
      sel[r] = bl | ((bl | 8u) << 4) | (bh << 8) | ((bh | 8u) << 12) | nf;
      // both strips start from column lo - 1 (column -1 when lo == 0)
      const int32_t hl = (lo == 0 && il < tlen) ? col_m1(il, h0, sc) : 0;
      const int32_t hh = (lo == 0 && ih < tlen) ? col_m1(ih, h0, sc) : 0;
      Hl[r] = pack16(hl, hh);
      HAl[r] = add16x2(Hl[r], na2);
      El[r] = 0;
      K[r] = kKeyNone;
      Blo[r] = -1;
      Bhi[r] = -1;
    }
    // lower strip's diagonal at its first column: H(i0-1, lo-1)
    int32_t dlo = 0;
    if (i0 == 0) dlo = h0;
    else if (lo == 0) dlo = col_m1(i0 - 1, h0, sc);
    else if (live) dlo = lo16(ring.at(lo - 1));
    // lower strip's bottom row (row i0+R-1) at column lo - 1: the left boundary
    const int32_t lb = (lo == 0 && i0 + R - 1 < tlen) ? col_m1(i0 + R - 1, h0, sc) : 0;
    uint32_t oH1 = (uint32_t)lb, oF1 = (uint32_t)lb, oH2 = (uint32_t)lb;  // low halves used
    uint32_t tHF_prev = (uint32_t)dlo & 0xFFFFu;
    uint32_t prof_prev = 0;
    // steps: s = 0 .. nsteps-1 (lower strip at lo + s, upper at lo + s - 1); the
    // unmasked range is where both strips are active and every row is in band
    const int32_t nsteps = live ? hi - lo + 2 : 0;
    int32_t sb_lo = 0, sb_hi = kFar;
    if (live) {
      sb_lo = max(1, RR - w + i0 - lo);
      sb_hi = min(hi - lo, w + i0 - lo);
      // the fast steps read the previous strip's row without checking that
      // it reached the column
      if (i0 > 0) sb_hi = min(sb_hi, hi_prev - lo);
      if (i0 + RR > tlen) sb_hi = -1;
    }
    const int32_t nmax = __reduce_max_sync(0xffffffffu, nsteps);
    const int32_t fs = (int32_t)__reduce_max_sync(0xffffffffu, (uint32_t)sb_lo);
    const int32_t fe = min(__reduce_min_sync(0xffffffffu, sb_hi), nmax - 1);
    // software pipeline: ring entries and query codes three columns ahead,
    // profiles one ahead (the ring row of the previous strip is usually an
    // L2 hit by now, so one step of lead time is not enough)
    const int32_t qlast = qlen - 1;
    uint32_t code_n1 = live ? qs.code(min(lo + 1, qlast)) : 0u;
    uint32_t code_n2 = live ? qs.code(min(lo + 2, qlast)) : 0u;
    uint32_t code_n3 = live ? qs.code(min(lo + 3, qlast)) : 0u;
    uint32_t prof_c = s_prof[live ? qs.code(lo) : 0u];
    uint32_t ring_c = live ? ring.at(lo) : 0u;
    uint32_t ring_n1 = live ? ring.at(lo + 1) : 0u;
    uint32_t ring_n2 = live ? ring.at(lo + 2) : 0u;
    int32_t blk = 0;     // steps taken in the current key block
    int32_t cbase = lo;  // lower strip's column at block step 0
    // A masked step: band edges, a lane whose lower strip has finished or
    // whose upper strip has not started (those halves keep their state).
    auto slow_step = [&](int32_t s) {
      const int32_t c = lo + s;
      const bool lo_act = live && c <= hi;
      const bool hi_act = live && s >= 1 && c - 1 <= hi;
      const uint32_t code_n4 = lo_act ? qs.code(min(c + 4, qlast)) : 0u;
      const uint32_t prof_n = s_prof[code_n1];
      const uint32_t ring_n3 = lo_act ? ring.at(c + 3) : 0u;
      // (H, F) of the row above at column c: row -1 on the first strip, else the
      // previous strip's bottom row (dead where it never reached)
      uint32_t tHF;
      if (i0 == 0) tHF = lo_act ? ((uint32_t)row_m1(c, h0, sc) & 0xFFFFu) : 0u;
      else tHF = (lo_act && c <= hi_prev) ? ring_c : 0u;
      const uint32_t prof = lo_act ? prof_c : 0u;
      const uint32_t Hup = prmt(tHF, oH1, 0x5410u);
      const uint32_t Fup = prmt(tHF, oF1, 0x5432u);
      const uint32_t D = prmt(tHF_prev, oH2, 0x5410u);
      const uint32_t pos2 = (uint32_t)blk * 0x00010001u;
      uint32_t oH, oF;
      const int32_t d0 = c - i0;
      const int32_t dh = d0 - 1 - R;  // upper strip: column c-1 minus its first row
      const uint32_t inband =
          (lo_act ? bit_range(d0 - w, min(d0 + w, tlen - 1 - i0), R) : 0u) |
          ((hi_act ? bit_range(dh - w, min(dh + w, tlen - 1 - i0 - R), R) : 0u) << 16);
      const uint32_t keep = (lo_act ? 0u : 0x0000FFFFu) | (hi_act ? 0u : 0xFFFF0000u);
      lane_step_p16<R, true, true, true, TB>(Hl, HAl, El, K, sel, prof, prof_prev, nn2, D, Hup, Fup,
                                         pos2, na2, nb2, mcm, inband, keep, oH, oF);
      if (hi_act) ring.at(c - 1) = prmt(oH, oF, 0x7632u);
      oH2 = oH1;
      oH1 = oH;
      oF1 = oF;
      tHF_prev = tHF;
      prof_prev = prof;
      prof_c = prof_n;
      code_n1 = code_n2;
      code_n2 = code_n3;
      code_n3 = code_n4;
      ring_c = ring_n1;
      ring_n1 = ring_n2;
      ring_n2 = ring_n3;
      if (++blk == kTagSteps) {
        fold_keys<R, TB>(K, Blo, Bhi, cbase);
        cbase += kTagSteps;
        blk = 0;
      }
    };
    // A fast step: every live lane has both strips active, every row in band
    // and the previous strip's row present at the column, so nothing is
    // masked or checked; lanes without a pair compute on garbage and store
    // only into their own ring, which they never read again.
    auto fast_step = [&](int32_t s) {
      const int32_t c = lo + s;
      const uint32_t code_n4 = live ? qs.code(min(c + 4, qlast)) : 0u;
      const uint32_t prof_n = s_prof[code_n1];
      const uint32_t ring_n3 = ring.at(c + 3);
      uint32_t tHF;
      if (i0 == 0) tHF = live ? ((uint32_t)row_m1(c, h0, sc) & 0xFFFFu) : 0u;
      else tHF = ring_c;
      const uint32_t Hup = prmt(tHF, oH1, 0x5410u);
      const uint32_t Fup = prmt(tHF, oF1, 0x5432u);
      const uint32_t D = prmt(tHF_prev, oH2, 0x5410u);
      const uint32_t pos2 = (uint32_t)blk * 0x00010001u;
      // one code path with the N-base select (2 instructions per row) is
      // faster than a vote between two copies of the step: the instruction
      // cache, not the ALU count, decides here
      uint32_t oH, oF;
      lane_step_p16<R, false, true, false, TB>(Hl, HAl, El, K, sel, prof_c, prof_prev, nn2, D, Hup,
                                           Fup, pos2, na2, nb2, mcm, 0u, 0u, oH, oF);
      ring.at(c - 1) = prmt(oH, oF, 0x7632u);
      oH2 = oH1;
      oH1 = oH;
      oF1 = oF;
      tHF_prev = tHF;
      prof_prev = prof_c;
      prof_c = prof_n;
      code_n1 = code_n2;
      code_n2 = code_n3;
      code_n3 = code_n4;
      ring_c = ring_n1;
      ring_n1 = ring_n2;
      ring_n2 = ring_n3;
      ++blk;
    };
    // One loop, one call site per kind of step (the steps are large: code
    // size matters more than the branch).  The fast range [fs, fe] never
    // holds the first step (upper strip not started) or a step past any
    // lane's end; it runs in stretches up to the next key-block boundary.
    int32_t s = 0;
    while (s < nmax) {
      if (s >= fs && s <= fe) {
        const int32_t e = min(fe, s + (kTagSteps - 1 - blk));
#pragma unroll kFastUnroll
        for (; s <= e; ++s) fast_step(s);
        if (blk == kTagSteps) {
          fold_keys<R, TB>(K, Blo, Bhi, cbase);
          cbase += kTagSteps;
          blk = 0;
        }
      } else {
        slow_step(s);
        ++s;
      }
    }
    fold_keys<R, TB>(K, Blo, Bhi, cbase);
    hi_prev = hi;
    if (live) {
      int32_t last_m = 0;
      const bool reach = hi == qlen - 1;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int32_t i = i0 + half * R + r;
          if (i < tlen && !st.stop) {
            const int32_t bk = half ? Bhi[r] : Blo[r];
            const int32_t m = bk < 0 ? 0 : (bk >> 16);
            // a dead row's column is its last in-band column (-1: none)
            const int32_t mj = m > 0 ? (bk & 0xFFFF) : (i - w <= qlen - 1 ? min(qlen - 1, i + w) : -1);
            // after the sweep, Hl holds H(i, hi) of both strips (each strip kept
            // its state once it had passed column hi)
            const bool g_in = reach && (qlen - 1 - i <= w) && (i - (qlen - 1) <= w);
            const int32_t g = g_in ? (half ? hi16(Hl[r]) : lo16(Hl[r])) : -1;
            st.feed(i, m, mj, g, sc);
            last_m = m;
          }
        }
      }
      if (st.stop || (last_m == 0 && col_m1(rlast, h0, sc) == 0)) live = false;
    }
  }
  Outcome o;
  o.score = st.best; o.qle = st.bj + 1; o.tle = st.bi + 1; o.gscore = st.gscore;
  o.gtle = st.gtle; o.max_off = st.max_off;
  o.cells = band_cells_upto(st.last_live, qlen, w);
  return o;
}

}  // namespace xt
