// xt_bwa.cu -- the BWA-MEM-compatible extension (xt_extend_batch_bwa).
//
// The variant (stated in full in include/xt.h) opens gaps from the match value
// M rather than from H and trims each row to the live run around the row's
// best cell.  Both change how the work parallelises:
//
//  * the insertion chain E of a row depends only on that row's M values,
//    E(i,j) = max(0, max_{k<j} (M(i,k) - o_ins - e_ins*(j-k))), a max-plus
//    prefix scan over the row, and M and F depend only on the row above: a row
//    is data-parallel across its columns;
//  * trimming makes row i+1's columns depend on all of row i (the run around
//    the row maximum), so rows must go one after another -- the strip scheme
//    of the default kernels, which keeps several rows in flight, does not
//    apply.
//
// So one pair is extended by a group of G lanes that computes a whole row at
// a time: lane l holds K consecutive columns of the row in registers (slot s =
// l*K + k is column A_i + s, with the anchor A_i = max(0, i - w') the first
// in-band column of row i).  Going from row i-1 to row i the anchor moves by
// 0 or 1 column, so the row above sits at the same slot (diagonal neighbour)
// or one slot further (vertical neighbour): one shuffle across each lane
// boundary.  Per row the group runs an exclusive max-scan for the insertion
// chain, a max-reduction for the row maximum and its column, and a min/max
// reduction for the live run.  G is the smallest power of two with G*K >=
// min(qlen, 2w'+1), from 4 lanes (64 columns) to 512 lanes (8192 columns); up
// to 32 lanes a group is a warp segment (shuffles), above that a whole CTA
// (shuffles plus shared memory).  Pairs are classified by G, and each class
// runs a persistent kernel whose groups take pairs from a counter.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "xt.h"
#include "xt_common.cuh"
#include "xt_ctx.cuh"

namespace xt {
namespace {

constexpr int kBwaK = 16;                    // columns per lane
constexpr int kBwaClasses = 8;               // G = 4 << class, 64 << class columns
constexpr int kBwaWarpThreads = 128;         // CTA size of the warp-segment classes
constexpr int32_t kBwaNeg = -(1 << 29);      // below any reachable value
constexpr uint8_t kBwaDone = 0xff;           // pair finished in classify

static_assert((64 << (kBwaClasses - 1)) == XT_BWA_MAX_WIDTH, "class range must end at the limit");

struct BwaScore {
  int32_t match, mismatch, nsc;
  int32_t o_ins, e_ins, o_del, e_del;
  int32_t w, zdrop, end_bonus;
};

struct BwaArgs {
  const uint8_t* q_seq;
  const uint8_t* t_seq;
  const int64_t* q_off;
  const int64_t* t_off;
  const int32_t* q_len;
  const int32_t* t_len;
  const int32_t* h0;
  int64_t q_bytes, t_bytes;
  int32_t n;
  xt_result* out;
  int64_t* cells;
  BwaScore sc;
  uint8_t* pclass;   // [n]
  int32_t* order;    // [n] pairs grouped by class
  int32_t* counts;   // [kBwaClasses]
  int32_t* cursor;   // [kBwaClasses]
  int32_t* heads;    // [kBwaClasses] next pair of each class's persistent kernel
};

struct ClassOffsets {
  int32_t off[kBwaClasses];
};

// The narrowed band half-width of a pair with query length qlen.
__host__ __device__ inline int32_t bwa_band(const BwaScore& s, int32_t qlen) {
  const int64_t gain = (int64_t)qlen * s.match + s.end_bonus;
  const int64_t wi = gain < s.o_ins ? 1 : (gain - s.o_ins) / s.e_ins + 1;
  const int64_t wd = gain < s.o_del ? 1 : (gain - s.o_del) / s.e_del + 1;
  int64_t w = s.w;
  if (wi < w) w = wi;
  if (wd < w) w = wd;
  return (int32_t)w;
}

__device__ __forceinline__ void put_result(const BwaArgs& a, int32_t k, int32_t score, int32_t qle,
                                           int32_t tle, int32_t gscore, int32_t gtle,
                                           int32_t max_off, int32_t status, int64_t cells) {
  xt_result r;
  r.score = score; r.qle = qle; r.tle = tle; r.gscore = gscore; r.gtle = gtle;
  r.max_off = max_off; r.status = status;
  a.out[k] = r;
  if (a.cells) a.cells[k] = cells;
}

// ---------------------------------------------------------------- classify
// Checks every pair, finishes the degenerate and invalid ones, and counts the
// rest per group-size class (block-aggregated atomics).
__global__ void k_bwa_classify(BwaArgs a) {
  __shared__ int32_t s_cnt[kBwaClasses];
  if (threadIdx.x < kBwaClasses) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t ql = a.q_len[k], tl = a.t_len[k], h0 = a.h0[k];
    const int64_t qo = a.q_off[k], to = a.t_off[k];
    bool ok = h0 >= 1 && h0 <= XT_MAX_H0 && ql >= 0 && tl >= 0 && ql <= XT_MAX_LEN &&
              tl <= XT_MAX_LEN && qo >= 0 && to >= 0 && qo <= a.q_bytes - ql &&
              to <= a.t_bytes - tl;
    int32_t width = 0;
    if (ok) {
      const int64_t wb = 2 * (int64_t)bwa_band(a.sc, ql) + 1;
      width = (int32_t)(wb < ql ? wb : ql);
      ok = width <= XT_BWA_MAX_WIDTH;
    }
    uint8_t cls = kBwaDone;
    if (!ok) {
      put_result(a, (int32_t)k, 0, 0, 0, 0, 0, 0, XT_EINVAL, 0);
    } else if (ql == 0) {
      put_result(a, (int32_t)k, h0, 0, 0, h0, 0, 0, XT_OK, 0);
    } else if (tl == 0) {
      put_result(a, (int32_t)k, h0, 0, 0, -1, 0, 0, XT_OK, 0);
    } else {
      int c = 0;
      while ((64 << c) < width) ++c;
      cls = (uint8_t)c;
      atomicAdd(&s_cnt[c], 1);
    }
    a.pclass[k] = cls;
  }
  __syncthreads();
  if (threadIdx.x < kBwaClasses && s_cnt[threadIdx.x] > 0)
    atomicAdd(&a.counts[threadIdx.x], s_cnt[threadIdx.x]);
}

// Pairs grouped by class: a block reserves its pairs' positions with one
// atomic per class, then places them.
__global__ void k_bwa_scatter(BwaArgs a, ClassOffsets co) {
  __shared__ int32_t s_cnt[kBwaClasses];
  __shared__ int32_t s_base[kBwaClasses];
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n;
       base += (int64_t)gridDim.x * blockDim.x) {
    if (threadIdx.x < kBwaClasses) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t k = base + threadIdx.x;
    const int c = k < a.n ? a.pclass[k] : kBwaDone;
    int32_t rank = 0;
    if (c != kBwaDone) rank = atomicAdd(&s_cnt[c], 1);
    __syncthreads();
    if (threadIdx.x < kBwaClasses && s_cnt[threadIdx.x] > 0)
      s_base[threadIdx.x] = atomicAdd(&a.cursor[threadIdx.x], s_cnt[threadIdx.x]);
    __syncthreads();
    if (c != kBwaDone) a.order[co.off[c] + s_base[c] + rank] = (int32_t)k;
    __syncthreads();
  }
}

// ------------------------------------------------------------ lane groups
// Collectives of the G lanes that extend one pair.
template <int G, bool kSegment = (G <= 32)>
struct Group;

// A warp segment of G lanes (G <= 32).
template <int G>
struct Group<G, true> {
  unsigned mask;
  int lane;
  __device__ __forceinline__ void init() {
    const int wl = threadIdx.x & 31;
    lane = wl & (G - 1);
    mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (wl & ~(G - 1)));
  }
  __device__ __forceinline__ int index() const { return lane; }
  // value of lane l+1 (0 past the last lane)
  __device__ __forceinline__ int32_t from_next(int32_t v) const {
    const int32_t r = __shfl_down_sync(mask, v, 1, G);
    return lane == G - 1 ? 0 : r;
  }
  // value of lane l-1 (fill for lane 0)
  __device__ __forceinline__ int32_t from_prev(int32_t v, int32_t fill) const {
    const int32_t r = __shfl_up_sync(mask, v, 1, G);
    return lane == 0 ? fill : r;
  }
  // max over the lanes before this one (kBwaNeg for lane 0)
  __device__ __forceinline__ int32_t excl_max(int32_t v) const {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const int32_t t = __shfl_up_sync(mask, v, o, G);
      if (lane >= o) v = max(v, t);
    }
    const int32_t r = __shfl_up_sync(mask, v, 1, G);
    return lane == 0 ? kBwaNeg : r;
  }
  __device__ __forceinline__ int64_t all_max64(int64_t v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const int64_t t = __shfl_xor_sync(mask, v, o, G);
      v = t > v ? t : v;
    }
    return v;
  }
  // (max of a, min of b) over the group
  __device__ __forceinline__ void all_max_min(int32_t* a, int32_t* b) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      *a = max(*a, __shfl_xor_sync(mask, *a, o, G));
      *b = min(*b, __shfl_xor_sync(mask, *b, o, G));
    }
  }
  __device__ __forceinline__ int32_t bcast(int32_t v, int src) const {
    return __shfl_sync(mask, v, src, G);
  }
  // one lane takes the next pair of the class for the whole group
  __device__ __forceinline__ int32_t claim(int32_t* head) const {
    int32_t p = 0;
    if (lane == 0) p = atomicAdd(head, 1);
    return __shfl_sync(mask, p, 0, G);
  }
};

// A whole CTA of G lanes (G = 64 .. 512): shuffles inside warps, shared memory
// across them.  Each collective writes its own shared array once per row and
// ends with one barrier; at least one other barrier separates two uses of the
// same array, so a lane can never overwrite a value another lane still reads.
template <int G>
struct Group<G, false> {
  static constexpr int kW = G / 32;
  struct Shared {
    int32_t nxt[3][kW];
    int32_t prv[kW];
    int32_t scan[kW];
    int64_t key[kW];
    int32_t amax[kW], amin[kW];
    int32_t b;
    int32_t claim;
  };
  Shared* sh;
  int lane, wl, wid;
  __device__ __forceinline__ void init(Shared* s) {
    sh = s;
    lane = threadIdx.x;
    wl = lane & 31;
    wid = lane >> 5;
  }
  __device__ __forceinline__ int index() const { return lane; }
  // values of lane l+1 for three registers at once (0 past the last lane)
  __device__ __forceinline__ void from_next3(int32_t* a, int32_t* b, int32_t* c) const {
    if (wl == 0) {
      sh->nxt[0][wid] = *a;
      sh->nxt[1][wid] = *b;
      sh->nxt[2][wid] = *c;
    }
    const int32_t ra = __shfl_down_sync(0xffffffffu, *a, 1);
    const int32_t rb = __shfl_down_sync(0xffffffffu, *b, 1);
    const int32_t rc = __shfl_down_sync(0xffffffffu, *c, 1);
    __syncthreads();
    if (wl == 31) {
      const bool last = wid == kW - 1;
      *a = last ? 0 : sh->nxt[0][wid + 1];
      *b = last ? 0 : sh->nxt[1][wid + 1];
      *c = last ? 0 : sh->nxt[2][wid + 1];
    } else {
      *a = ra; *b = rb; *c = rc;
    }
  }
  __device__ __forceinline__ int32_t from_prev(int32_t v, int32_t fill) const {
    if (wl == 31) sh->prv[wid] = v;
    const int32_t r = __shfl_up_sync(0xffffffffu, v, 1);
    __syncthreads();
    if (wl == 0) return wid == 0 ? fill : sh->prv[wid - 1];
    return r;
  }
  __device__ __forceinline__ int32_t excl_max(int32_t v) const {
    int32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (wl >= o) inc = max(inc, t);
    }
    if (wl == 31) sh->scan[wid] = inc;
    int32_t ex = __shfl_up_sync(0xffffffffu, inc, 1);
    if (wl == 0) ex = kBwaNeg;
    __syncthreads();
    for (int u = 0; u < wid; ++u) ex = max(ex, sh->scan[u]);
    return ex;
  }
  __device__ __forceinline__ int64_t all_max64(int64_t v) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int64_t t = __shfl_xor_sync(0xffffffffu, v, o);
      v = t > v ? t : v;
    }
    if (wl == 0) sh->key[wid] = v;
    __syncthreads();
    int64_t r = sh->key[0];
    for (int u = 1; u < kW; ++u) r = sh->key[u] > r ? sh->key[u] : r;
    return r;
  }
  __device__ __forceinline__ void all_max_min(int32_t* a, int32_t* b) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      *a = max(*a, __shfl_xor_sync(0xffffffffu, *a, o));
      *b = min(*b, __shfl_xor_sync(0xffffffffu, *b, o));
    }
    if (wl == 0) {
      sh->amax[wid] = *a;
      sh->amin[wid] = *b;
    }
    __syncthreads();
    int32_t x = sh->amax[0], y = sh->amin[0];
    for (int u = 1; u < kW; ++u) {
      x = max(x, sh->amax[u]);
      y = min(y, sh->amin[u]);
    }
    *a = x;
    *b = y;
  }
  __device__ __forceinline__ int32_t bcast(int32_t v, int src) const {
    if (lane == src) sh->b = v;
    __syncthreads();
    return sh->b;
  }
  __device__ __forceinline__ int32_t claim(int32_t* head) const {
    __syncthreads();  // the previous pair's readers of sh->claim are done
    if (lane == 0) sh->claim = atomicAdd(head, 1);
    __syncthreads();
    return sh->claim;
  }
};

template <int G>
__device__ __forceinline__ void shift_in(const Group<G, true>& g, int32_t* a, int32_t* b,
                                         int32_t* c) {
  *a = g.from_next(*a);
  *b = g.from_next(*b);
  *c = g.from_next(*c);
}
template <int G>
__device__ __forceinline__ void shift_in(const Group<G, false>& g, int32_t* a, int32_t* b,
                                         int32_t* c) {
  g.from_next3(a, b, c);
}

// Score row for target code ti (0..4): byte c = S(ti, query code c), c = 0..4.
__device__ __forceinline__ void score_row(const BwaScore& s, uint32_t ti, uint32_t* lo,
                                          uint32_t* hi) {
  const uint32_t nb = (uint8_t)(int8_t)s.nsc;
  if (ti >= 4u) {
    *lo = nb * 0x01010101u;
  } else {
    const uint32_t xb = (uint8_t)(int8_t)s.mismatch, mb = (uint8_t)(int8_t)s.match;
    const uint32_t sh = 8u * ti;
    *lo = ((xb * 0x01010101u) & ~(0xffu << sh)) | (mb << sh);
  }
  *hi = nb;
}

// M and F of slot s from its diagonal (D) and vertical (um, uf) neighbours in
// the row above, 0 outside the row's columns [lo, hi); Y carries the lane's
// insertion chain (started from 0 at its first slot) past the slot.
__device__ __forceinline__ void cell_mf(const BwaScore& sc, int32_t s, int32_t lo, int32_t hi,
                                        uint32_t rp_lo, uint32_t rp_hi, uint32_t sel, int32_t D,
                                        int32_t um, int32_t uf, int32_t oe_del, int32_t e_del,
                                        int32_t oe_ins, int32_t e_ins, int32_t* M_out,
                                        int32_t* F_out, int32_t* Y) {
  const bool in = (uint32_t)(s - lo) < (uint32_t)(hi - lo);
  const int32_t S = prmt_s8(rp_lo, rp_hi, sel);
  const int32_t M = (in && D > 0) ? D + S : 0;
  *F_out = in ? __viaddmax_s32_relu(um, -oe_del, uf - e_del) : 0;
  *M_out = M;
  *Y = __viaddmax_s32_relu(M, -oe_ins, *Y - e_ins);
}

// --------------------------------------------------------------- the kernel
// One pair per group of G lanes; slot s = lane*K + k of row i is column
// A_i + s.  Registers per slot: H, M, F of the row above (under its anchor)
// and the query base's score selector (under the current anchor).
template <int G>
__device__ __forceinline__ void bwa_pair(const BwaArgs& a, const Group<G>& g, int32_t k) {
  constexpr int K = kBwaK;
  constexpr int C = G * K;
  const BwaScore& sc = a.sc;
  const int32_t qlen = a.q_len[k], tlen = a.t_len[k], h0 = a.h0[k];
  const uint8_t* q = a.q_seq + a.q_off[k];
  const uint8_t* t = a.t_seq + a.t_off[k];
  const int32_t w = bwa_band(sc, qlen);
  const int32_t oe_ins = sc.o_ins + sc.e_ins, oe_del = sc.o_del + sc.e_del;
  const int32_t e_ins = sc.e_ins, e_del = sc.e_del;
  const int lane = g.index();
  const int32_t sb = lane * K;  // this lane's first slot

  int32_t Hd[K], Mv[K], Fv[K];
  uint32_t qs[K];
  // row -1 under anchor 0: the insertion run from the seed, inside the band
#pragma unroll
  for (int kk = 0; kk < K; ++kk) {
    const int32_t s = sb + kk;
    const int32_t v = h0 - oe_ins - e_ins * s;
    Hd[kk] = (s < qlen && s + 1 <= w && v > 0) ? v : 0;
    Mv[kk] = 0;
    Fv[kk] = 0;
    qs[kk] = score_selector(s < qlen ? clamp_code(q[s]) : 4u);
  }
  int32_t A_prev = 0;
  int32_t hb_prev = h0;  // column -1 of the row above: the seed for row 0
  int32_t beg = 0, end = min(qlen, w + 1);
  int32_t best = h0, bi = -1, bj = -1, max_off = 0, gscore = -1, gtle = 0;
  int64_t cells = 0;

  for (int32_t i = 0; i < tlen; ++i) {
    if (beg >= end) break;  // nothing to compute: the row maximum is 0
    const int32_t A = max(0, i - w);
    const int32_t lo = beg - A, hi = end - A;
    uint32_t rp_lo, rp_hi;
    score_row(sc, clamp_code(t[i]), &rp_lo, &rp_hi);
    // pass 1: M and F per slot from the row above (diagonal and vertical
    // neighbours), and the lane's insertion carry from 0
    int32_t Y = 0;
    if (A == A_prev) {
      const int32_t in = g.from_prev(Hd[K - 1], hb_prev);
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        const int32_t D = kk > 0 ? Hd[kk - 1] : in;
        cell_mf(sc, sb + kk, lo, hi, rp_lo, rp_hi, qs[kk], D, Mv[kk], Fv[kk], oe_del, e_del,
                oe_ins, e_ins, &Mv[kk], &Fv[kk], &Y);
      }
    } else {
      // the anchor moved one column right: the row above is one slot further
      int32_t m0 = Mv[0], f0 = Fv[0], q0 = (int32_t)qs[0];
      shift_in(g, &m0, &f0, &q0);
#pragma unroll
      for (int kk = 0; kk < K; ++kk) qs[kk] = kk + 1 < K ? qs[kk + 1] : (uint32_t)q0;
      if (lane == G - 1) {
        const int32_t c = A + C - 1;
        qs[K - 1] = score_selector(c < qlen ? clamp_code(q[c]) : 4u);
      }
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        const int32_t um = kk + 1 < K ? Mv[kk + 1] : m0;
        const int32_t uf = kk + 1 < K ? Fv[kk + 1] : f0;
        cell_mf(sc, sb + kk, lo, hi, rp_lo, rp_hi, qs[kk], Hd[kk], um, uf, oe_del, e_del, oe_ins,
                e_ins, &Mv[kk], &Fv[kk], &Y);
      }
    }
    // insertion carry into this lane: max over earlier lanes l' of their
    // carry Y_l' decayed over the (l - 1 - l') * K columns in between
    const int32_t decay = e_ins * K;
    const int32_t ex = g.excl_max(Y + decay * lane);
    int32_t E = lane == 0 ? 0 : max(0, ex - decay * (lane - 1));
    // pass 2: E, H, the row maximum (largest slot on ties) and the live mask
    int32_t key = 0;
    uint32_t live = 0;
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
      const int32_t s = sb + kk;
      const bool in = (uint32_t)(s - lo) < (uint32_t)(hi - lo);
      const int32_t M = Mv[kk];
      const int32_t H = in ? __vimax3_s32(M, E, Fv[kk]) : 0;
      Hd[kk] = H;
      key = max(key, H * K + kk);
      live |= H > 0 ? 1u << kk : 0u;
      E = __viaddmax_s32_relu(M, -oe_ins, E - e_ins);
    }
    const int64_t kk64 = g.all_max64(((int64_t)(key / K) << 32) | (uint32_t)(sb + key % K));
    const int32_t m = (int32_t)(kk64 >> 32);
    const int32_t mslot = (int32_t)(kk64 & 0xffffffff);
    // end-to-end score when the row reaches the last query column
    if (end == qlen) {
      const int32_t ts = qlen - 1 - A;
      int32_t gv = 0;
#pragma unroll
      for (int kk = 0; kk < K; ++kk) gv = (sb + kk == ts) ? Hd[kk] : gv;
      gv = g.bcast(gv, ts / K);
      if (gv >= gscore) {
        gscore = gv;
        gtle = i + 1;
      }
    }
    if (m == 0) break;
    cells += end - beg;
    const int32_t mj = A + mslot;
    if (m > best) {
      best = m;
      bi = i;
      bj = mj;
      max_off = max(max_off, abs(mj - i));
    } else if (sc.zdrop > 0) {
      const int64_t di = i - bi, dj = mj - bj;
      const int64_t drop = di > dj ? (int64_t)best - m - (di - dj) * e_del
                                   : (int64_t)best - m - (dj - di) * e_ins;
      if (drop > sc.zdrop) break;
    }
    // the live run around the best slot: the last dead slot below it and the
    // first dead slot above it (slots outside [lo, hi) hold 0)
    const int32_t rel = mslot - sb;
    const uint32_t dead = ~live & ((1u << K) - 1u);
    const uint32_t below = rel <= 0 ? 0u : (rel >= K ? dead : dead & ((1u << rel) - 1u));
    const uint32_t above = rel >= K - 1 ? 0u : (rel < 0 ? dead : dead & ~((2u << rel) - 1u));
    int32_t zb = below ? sb + 31 - __clz(below) : -1;
    int32_t za = above ? sb + __ffs(above) - 1 : C;
    g.all_max_min(&zb, &za);
    // next row: the run's columns reachable in one step, within the band
    const int32_t hb = (beg == 0 && i + 1 <= w) ? max(0, h0 - oe_del - e_del * i) : 0;
    beg = max(A + zb + 1, i + 1 - w);
    end = min(min(A + za + 1, i + w + 2), qlen);
    hb_prev = hb;
    A_prev = A;
  }
  if (lane == 0) put_result(a, k, best, bj + 1, bi + 1, gscore, gtle, max_off, XT_OK, cells);
}

// Four CTAs per SM (128 registers, no spills) rather than three: the kernel
// is bound by the integer pipe and waits on short dependency chains.
template <int G>
__global__ void __launch_bounds__(kBwaWarpThreads, 4) k_bwa_seg(BwaArgs a, int cls, int32_t off,
                                                                int32_t count) {
  Group<G> g;
  g.init();
  for (;;) {
    const int32_t p = g.claim(&a.heads[cls]);
    if (p >= count) break;
    const int32_t idx = off + p;
    if (idx < 0 || idx >= a.n) break;  // defensive: order index out of range
    const int32_t k = a.order[idx];
    if (k < 0 || k >= a.n) continue;
    bwa_pair<G>(a, g, k);
  }
}

// 512 threads per SM at least (16 warps, 128 registers each).
template <int G>
__global__ void __launch_bounds__(G, 512 / G) k_bwa_cta(BwaArgs a, int cls, int32_t off,
                                                        int32_t count) {
  __shared__ typename Group<G, false>::Shared s;
  Group<G> g;
  g.init(&s);
  for (;;) {
    const int32_t p = g.claim(&a.heads[cls]);
    if (p >= count) break;
    const int32_t idx = off + p;
    if (idx < 0 || idx >= a.n) break;
    const int32_t k = a.order[idx];
    if (k < 0 || k >= a.n) continue;
    bwa_pair<G>(a, g, k);
  }
}

template <int G>
cudaError_t launch_class(xt_ctx* ctx, const BwaArgs& a, int cls, int32_t off, int32_t count,
                         cudaStream_t stream) {
  constexpr bool kSeg = G <= 32;
  const int threads = kSeg ? kBwaWarpThreads : G;
  const int per_block = kSeg ? kBwaWarpThreads / G : 1;
  int& resident = ctx->bwa_blocks[cls];
  if (resident == 0) {
    cudaError_t e;
    if constexpr (kSeg)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_bwa_seg<G>, threads, 0);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_bwa_cta<G>, threads, 0);
    if (e != cudaSuccess) return e;
    if (resident < 1) resident = 1;
  }
  const int64_t want = ((int64_t)count + per_block - 1) / per_block;
  const int grid = (int)std::min<int64_t>(want, (int64_t)resident * ctx->num_sms);
  if constexpr (kSeg)
    k_bwa_seg<G><<<grid, threads, 0, stream>>>(a, cls, off, count);
  else
    k_bwa_cta<G><<<grid, threads, 0, stream>>>(a, cls, off, count);
  return cudaGetLastError();
}

cudaError_t launch_bwa_class(xt_ctx* ctx, const BwaArgs& a, int cls, int32_t off, int32_t count,
                             cudaStream_t stream) {
  switch (cls) {
    case 0: return launch_class<4>(ctx, a, cls, off, count, stream);
    case 1: return launch_class<8>(ctx, a, cls, off, count, stream);
    case 2: return launch_class<16>(ctx, a, cls, off, count, stream);
    case 3: return launch_class<32>(ctx, a, cls, off, count, stream);
    case 4: return launch_class<64>(ctx, a, cls, off, count, stream);
    case 5: return launch_class<128>(ctx, a, cls, off, count, stream);
    case 6: return launch_class<256>(ctx, a, cls, off, count, stream);
    case 7: return launch_class<512>(ctx, a, cls, off, count, stream);
    default: return cudaErrorInvalidValue;
  }
}

bool bwa_scoring_ok(const xt_bwa_scoring* s) {
  if (!s) return false;
  if (s->match < 1 || s->match > 127) return false;
  if (s->mismatch > 0 || s->mismatch < -127) return false;
  if (s->n_score > 0 || s->n_score < -127) return false;
  if (s->o_del < 0 || s->o_del > 1023 || s->o_ins < 0 || s->o_ins > 1023) return false;
  if (s->e_del < 1 || s->e_del > 1023 || s->e_ins < 1 || s->e_ins > 1023) return false;
  if (s->w < 0) return false;
  if (s->end_bonus < 0 || s->end_bonus > (1 << 20)) return false;
  return true;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace xt

using namespace xt;

extern "C" xt_status xt_bwa_scoring_check(const xt_bwa_scoring* sc) {
  return bwa_scoring_ok(sc) ? XT_OK : XT_EINVAL;
}

extern "C" xt_status xt_extend_batch_bwa(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes,
                                         const int64_t* q_off, const int32_t* q_len,
                                         const uint8_t* t_seq, int64_t t_bytes,
                                         const int64_t* t_off, const int32_t* t_len,
                                         const int32_t* h0, int32_t n_pairs,
                                         const xt_bwa_scoring* scr, xt_result* out,
                                         int64_t* cells_out, void* stream) {
  if (!ctx) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (n_pairs < 0) return ctx_fail(ctx, XT_EINVAL, "n_pairs < 0");
  if (!bwa_scoring_ok(scr)) return ctx_fail(ctx, XT_EINVAL, "scoring record out of range");
  if (q_bytes < 0 || t_bytes < 0) return ctx_fail(ctx, XT_EINVAL, "negative buffer size");
  if (n_pairs > 0 && (!q_off || !q_len || !t_off || !t_len || !h0 || !out))
    return ctx_fail(ctx, XT_EINVAL, "null array");
  if ((q_bytes > 0 && !q_seq) || (t_bytes > 0 && !t_seq))
    return ctx_fail(ctx, XT_EINVAL, "null sequence buffer");
  if (ctx->pending.active) return ctx_fail(ctx, XT_EBUSY, "a begun call has not been finished");
  if (n_pairs == 0) return XT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaSetDevice");
  xt_status s = ctx_codes(ctx, &q_seq, q_bytes, &t_seq, t_bytes, st);
  if (s != XT_OK) return s;
  // workspace: class bytes, order, counters
  const size_t n = (size_t)n_pairs;
  const size_t o_cls = 0;
  const size_t o_order = align256(o_cls + n);
  const size_t o_cnt = align256(o_order + 4 * n);
  const size_t bytes = align256(o_cnt + 3 * 4 * kBwaClasses);
  s = ctx_alloc(ctx, &ctx->bwa_ws, &ctx->bwa_ws_bytes, bytes);
  if (s != XT_OK) return s;
  char* ws = static_cast<char*>(ctx->bwa_ws);
  BwaArgs a;
  a.q_seq = q_seq; a.t_seq = t_seq; a.q_off = q_off; a.t_off = t_off; a.q_len = q_len;
  a.t_len = t_len; a.h0 = h0; a.q_bytes = q_bytes; a.t_bytes = t_bytes; a.n = n_pairs;
  a.out = out; a.cells = cells_out;
  a.sc.match = scr->match; a.sc.mismatch = scr->mismatch; a.sc.nsc = scr->n_score;
  a.sc.o_ins = scr->o_ins; a.sc.e_ins = scr->e_ins; a.sc.o_del = scr->o_del;
  a.sc.e_del = scr->e_del;
  // a band wider than any pair changes nothing; clamp so index arithmetic stays in int32
  a.sc.w = scr->w > 2 * XT_MAX_LEN ? 2 * XT_MAX_LEN : scr->w;
  a.sc.zdrop = scr->zdrop; a.sc.end_bonus = scr->end_bonus;
  a.pclass = reinterpret_cast<uint8_t*>(ws + o_cls);
  a.order = reinterpret_cast<int32_t*>(ws + o_order);
  a.counts = reinterpret_cast<int32_t*>(ws + o_cnt);
  a.cursor = a.counts + kBwaClasses;
  a.heads = a.cursor + kBwaClasses;
  const int threads = 256;
  const int grid = (int)std::min<int64_t>(((int64_t)n_pairs + threads - 1) / threads,
                                          (int64_t)ctx->num_sms * 8);
  e = cudaMemsetAsync(a.counts, 0, 3 * 4 * kBwaClasses, st);
  if (e == cudaSuccess) {
    k_bwa_classify<<<grid, threads, 0, st>>>(a);
    e = cudaGetLastError();
  }
  // the class sizes come back to size the launches
  int32_t* cnt_host = ctx->seg_host + kSegHostBwaCounts;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cnt_host, a.counts, 4 * kBwaClasses, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->seg_ev, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(ctx->seg_ev);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "BWA classify");
  ClassOffsets co;
  int32_t total = 0;
  int32_t cnt[kBwaClasses];
  for (int c = 0; c < kBwaClasses; ++c) {
    cnt[c] = cnt_host[c];
    co.off[c] = total;
    total += cnt[c];
  }
  if (total == 0) return XT_OK;
  k_bwa_scatter<<<grid, threads, 0, st>>>(a, co);
  e = cudaGetLastError();
  // widest groups first: they hold the longest rows
  for (int c = kBwaClasses - 1; c >= 0 && e == cudaSuccess; --c)
    if (cnt[c] > 0) e = launch_bwa_class(ctx, a, c, co.off[c], cnt[c], st);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "BWA extension");
  ctx->calls++;
  return XT_OK;
}
