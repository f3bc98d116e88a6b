// xt_bwa.cu -- the BWA-MEM-compatible extension (xt_extend_batch_bwa).
//
// The variant (stated in full in include/xt.h) opens gaps from the match value
// M rather than from H and drops the dead cells at both ends of each row.
// Both change how the work parallelises:
//
//  * the insertion chain E of a row depends only on that row's M values,
//    E(i,j) = max(0, max_{k<j} (M(i,k) - o_ins - e_ins*(j-k))), a max-plus
//    prefix scan over the row, and M and F depend only on the row above: a row
//    is data-parallel across its columns;
//  * trimming makes row i+1's columns depend on all of row i (its first and
//    last live cells), so rows must go one after another -- the strip scheme
//    of the default kernels, which keeps several rows in flight, does not
//    apply.
//
// So one pair is extended by a group of G lanes that computes a whole row at
// a time, and only the row's own columns [beg, end): trimming keeps a row far
// narrower than its band (about a quarter of 2w'+1 on short reads), so the
// lanes split the row's width, k = ceil((end - beg) / G) <= K consecutive
// columns each, and the row above lives in shared memory rather than in fixed
// registers.  Per row the group runs an exclusive max-scan for the insertion
// chain, a max-reduction for the row maximum and its column, and a min/max
// reduction for the row's first and last live columns.  G*K is the smallest power of two >= min(qlen,
// 2w'+1), from 64 to 8192 columns; up to 32 lanes a group is a warp segment
// (shuffles), above that a whole CTA (shuffles plus shared memory).  Pairs are
// classified by G*K, and each class runs a persistent kernel whose groups take
// pairs from a counter.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "xt.h"
#include "xt_common.cuh"
#include "xt_ctx.cuh"

namespace xt {
namespace {

// Most columns a lane computes in a row (16 or 32): more columns per lane
// means fewer lanes per pair and cheaper per-row collectives, at two
// registers per column.
#ifndef XT_BWA_LANE_COLUMNS
#define XT_BWA_LANE_COLUMNS 32
#endif
constexpr int kBwaK = XT_BWA_LANE_COLUMNS;
static_assert(kBwaK == 16 || kBwaK == 32, "columns per lane: 16 or 32");
constexpr int kBwaClasses = 8;               // G*K = 64 << class columns
constexpr int kBwaWarpThreads = 128;         // CTA size of the warp-segment classes
constexpr int32_t kBwaNeg = -(1 << 29);      // below any reachable value
constexpr uint8_t kBwaDone = 0xff;           // pair finished in classify
// Within a class pairs go longest query first, in buckets of query length
// (capped): the groups sharing a warp then extend pairs of like length, whose
// rows are of like width, and the longest pairs do not start last.
constexpr int kBwaLenBuckets = 1024;
constexpr int kBwaScanThreads = 1024;
// A row buffer element's y word: the column's query code above F.
constexpr int kCodeShift = 28;
constexpr uint32_t kFMask = (1u << kCodeShift) - 1u;
static_assert((int64_t)XT_MAX_H0 + (int64_t)XT_MAX_LEN * 127 < (1ll << kCodeShift), "F fits below the code");
static_assert(kBwaLenBuckets * kBwaClasses % kBwaScanThreads == 0, "scan tiling");

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
  int32_t* order;    // [n] pairs by class, then by query length (longest first)
  int32_t* slots;    // [kBwaClasses * kBwaLenBuckets] pairs per (class, length), then positions
  int32_t* counts;   // [kBwaClasses] pairs per class
  int32_t* heads;    // [kBwaClasses] next pair of each class's persistent kernel
};

// Slot of a pair of class c and query length ql: classes in order, longer
// queries first within a class.
__device__ __forceinline__ int32_t bwa_slot(int c, int32_t ql) {
  const int32_t b = ql < kBwaLenBuckets - 1 ? ql : kBwaLenBuckets - 1;
  return c * kBwaLenBuckets + (kBwaLenBuckets - 1 - b);
}

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
// rest per (class, query length) slot.
__global__ void k_bwa_classify(BwaArgs a) {
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
      atomicAdd(&a.slots[bwa_slot(c, ql)], 1);
    }
    a.pclass[k] = cls;
  }
}

// One block: slot counts to first positions (exclusive scan in slot order)
// and the pairs per class.
__global__ void __launch_bounds__(kBwaScanThreads) k_bwa_scan(BwaArgs a) {
  constexpr int kPer = kBwaClasses * kBwaLenBuckets / kBwaScanThreads;
  constexpr int kPerClass = kBwaLenBuckets / kPer;  // threads per class
  __shared__ int32_t s_warp[kBwaScanThreads / 32];
  __shared__ int32_t s_class[kBwaClasses];
  const int tid = threadIdx.x;
  int32_t v[kPer];
  int32_t sum = 0;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    v[u] = a.slots[tid * kPer + u];
    sum += v[u];
  }
  if (tid < kBwaClasses) s_class[tid] = 0;
  // inclusive scan of the thread sums
  int32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if ((tid & 31) >= o) inc += t;
  }
  if ((tid & 31) == 31) s_warp[tid >> 5] = inc;
  __syncthreads();
  int32_t before = inc - sum;
  for (int u = 0; u < (tid >> 5); ++u) before += s_warp[u];
  atomicAdd(&s_class[tid / kPerClass], sum);
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    a.slots[tid * kPer + u] = before;
    before += v[u];
  }
  __syncthreads();
  if (tid < kBwaClasses) a.counts[tid] = s_class[tid];
}

// Each pair takes the next position of its slot.
__global__ void k_bwa_scatter(BwaArgs a) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int c = a.pclass[k];
    if (c == kBwaDone) continue;
    const int32_t pos = atomicAdd(&a.slots[bwa_slot(c, a.q_len[k])], 1);
    if (pos >= 0 && pos < a.n) a.order[pos] = (int32_t)k;
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
  // orders the group's shared-memory accesses before and after it
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
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
  // *m = max of v over the group, *at = the largest col among the lanes
  // holding it.  A whole warp uses the warp-reduction instructions; a warp
  // segment, whose neighbours in the warp reduce over other masks at the same
  // time, a shuffle tree (measured faster there).
  __device__ __forceinline__ void max_last(int32_t v, int32_t col, int32_t* m,
                                           int32_t* at) const {
    if constexpr (G == 32) {
      const int32_t x = __reduce_max_sync(mask, v);
      *m = x;
      *at = __reduce_max_sync(mask, v == x ? col : INT32_MIN);
    } else {
      int64_t key = ((int64_t)v << 32) | (uint32_t)col;
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        const int64_t t = __shfl_xor_sync(mask, key, o, G);
        key = t > key ? t : key;
      }
      *m = (int32_t)(key >> 32);
      *at = (int32_t)(key & 0xffffffff);
    }
  }
  // (max of a, min of b) over the group
  __device__ __forceinline__ void all_max_min(int32_t* a, int32_t* b) const {
    if constexpr (G == 32) {
      *a = __reduce_max_sync(mask, *a);
      *b = __reduce_min_sync(mask, *b);
    } else {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        *a = max(*a, __shfl_xor_sync(mask, *a, o, G));
        *b = min(*b, __shfl_xor_sync(mask, *b, o, G));
      }
    }
  }
  // one lane takes the next pair of the class for the whole group
  __device__ __forceinline__ int32_t claim(int32_t* head) const {
    int32_t p = 0;
    if (lane == 0) p = atomicAdd(head, 1);
    return __shfl_sync(mask, p, 0, G);
  }
};

// A whole CTA of G lanes (G >= 64): shuffles inside warps, shared memory
// across them.  Each collective writes its own shared array once per row and
// ends with one barrier; at least one other barrier separates two uses of the
// same array, so a lane can never overwrite a value another lane still reads.
template <int G>
struct Group<G, false> {
  static constexpr int kW = G / 32;
  struct Shared {
    int32_t scan[kW];
    int64_t key[kW];
    int32_t amax[kW], amin[kW];
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
  __device__ __forceinline__ void sync() const { __syncthreads(); }
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
  // *m = max of v over the group, *at = col of the highest lane holding it
  __device__ __forceinline__ void max_last(int32_t v, int32_t col, int32_t* m,
                                           int32_t* at) const {
    const int64_t key = all_max64(((int64_t)v << 32) | (uint32_t)col);
    *m = (int32_t)(key >> 32);
    *at = (int32_t)(key & 0xffffffff);
  }
  __device__ __forceinline__ void all_max_min(int32_t* a, int32_t* b) const {
    *a = __reduce_max_sync(0xffffffffu, *a);
    *b = __reduce_min_sync(0xffffffffu, *b);
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
  __device__ __forceinline__ int32_t claim(int32_t* head) const {
    __syncthreads();  // the previous pair's readers of sh->claim are done
    if (lane == 0) sh->claim = atomicAdd(head, 1);
    __syncthreads();
    return sh->claim;
  }
};

// Score row for target code ti (0..4) as biased bytes: byte c of {hi:lo} is
// S(ti, query code c) + 128, c = 0..4; bytes 5..7 are 0.
__device__ __forceinline__ void score_row(uint32_t ti, uint32_t mism4, uint32_t nb, uint32_t mb,
                                          uint32_t* lo, uint32_t* hi) {
  if (ti >= 4u) {
    *lo = nb * 0x01010101u;
  } else {
    const uint32_t sh = 8u * ti;
    *lo = (mism4 & ~(0xffu << sh)) | (mb << sh);
  }
  *hi = nb;
}

// --------------------------------------------------------------- the kernel
// One pair per group of G lanes.  Row i computes only its columns [beg, end):
// lane l takes k consecutive columns from beg + l*k (fewer in the last lanes),
// k = ceil((end - beg) / G) rounded up to odd while <= K.  The row above lives
// in the group's buffer of G*K + 2 elements, one per column j of [beg - 1,
// end]: x = H(i-1, j) and y = query code of column j << 28 | F(i, j), at index
// j - o(i-1) with the origin o(r) = max(-1, r - w' - 1).  The origin moves by
// 0 or 1 column a row, so a row's reads (x of column j-1, y of column j) and
// its writes (column j at index j - o(i)) touch the same window; a barrier of
// the group separates the row's reads from its writes.  Two extra elements per row hold the
// boundary: column beg-1 (x = H of column -1 for the next row: the deletion
// run from the seed, else 0) and column end (y = its query code << 28 | 0).
// F and H stay below 2^28: H <= h0 + qlen * match <= 2^20 + 2^20 * 127.
// A group's row buffer, element e at base[e * S]: the buffers of the S groups
// that share a half-warp are interleaved element by element (S = 16 / G for
// groups of up to 8 lanes, else 1).  With each lane's columns an odd count,
// the G lanes of a group then fall on distinct bank pairs of one residue
// class mod 2S, and the S groups on different classes, so a half-warp's
// 8-byte accesses meet no bank conflict whatever each group's row offsets.
template <int S>
struct RowBuf {
  int2* base;
  __device__ __forceinline__ int2& operator[](int32_t e) const { return base[e * S]; }
  __device__ __forceinline__ RowBuf operator+(int32_t e) const { return RowBuf{base + e * S}; }
};

template <int G, int K, typename Buf>
__device__ __forceinline__ void bwa_pair(const BwaArgs& a, const Group<G>& g, Buf buf,
                                         int32_t k) {
  const BwaScore& sc = a.sc;
  const int32_t qlen = a.q_len[k], tlen = a.t_len[k], h0 = a.h0[k];
  const uint8_t* q = a.q_seq + a.q_off[k];
  const uint8_t* t = a.t_seq + a.t_off[k];
  const int32_t w = bwa_band(sc, qlen);
  const int32_t oe_ins = sc.o_ins + sc.e_ins, oe_del = sc.o_del + sc.e_del;
  const int32_t e_ins = sc.e_ins, e_del = sc.e_del;
  const uint32_t mb = (uint32_t)(sc.match + 128), nb = (uint32_t)(sc.nsc + 128);
  const uint32_t mism4 = (uint32_t)(sc.mismatch + 128) * 0x01010101u;
  const int lane = g.index();

  // row -1 (origin -1): the seed at column -1, the insertion run from it
  // inside the band, no deletion state; each element carries its column's code
  int32_t end = min(qlen, w + 1);
#pragma unroll 4
  for (int32_t idx = lane; idx < end + 2; idx += G) {
    const int32_t j = idx - 1;
    int32_t x = h0;
    if (j >= 0) {
      const int32_t v = h0 - oe_ins - e_ins * j;
      x = (j < qlen && j + 1 <= w && v > 0) ? v : 0;
    }
    const uint32_t c = (j >= 0 && j < qlen) ? clamp_code(q[j]) : 4u;
    buf[idx] = make_int2(x, (int32_t)(c << kCodeShift));
  }
  g.sync();
  int32_t beg = 0;
  int32_t best = h0, bi = -1, bj = -1, max_off = 0, gscore = -1, gtle = 0;
  int64_t cells = 0;
  uint32_t t_next = tlen > 0 ? t[0] : 4u;

  for (int32_t i = 0; i < tlen; ++i) {
    if (beg >= end) break;  // nothing to compute: the row maximum is 0
    const int32_t o_up = max(-1, i - w - 2), o_row = max(-1, i - w - 1);
    uint32_t rp_lo, rp_hi;
    score_row(clamp_code(t_next), mism4, nb, mb, &rp_lo, &rp_hi);
    if (i + 1 < tlen) t_next = t[i + 1];
    // the query code of column end enters with the row's boundary element
    const uint32_t q_end = (lane == G - 1 && end < qlen) ? clamp_code(q[end]) : 4u;
    // columns per lane: ceil((end - beg) / G) <= K (end - beg <= min(qlen, 2w'+1)),
    // rounded up to odd where that stays <= K, so that the lanes of a group
    // read and write distinct shared-memory banks
    const int32_t kq = min(((end - beg + G - 1) / G) | 1, K);
    const int32_t first = beg + lane * kq;
    const int32_t cnt = max(0, min(kq, end - first));

    // pass 1: M, F and H without the insertion carry from earlier lanes;
    // Y is the lane's insertion chain, started from 0
    // The F word of column j goes to the buffer at once: its index in this
    // row's layout holds the y word of column j (origin unchanged) or of
    // column j-1 (origin moved), which this lane has read already.  Only the
    // first column's word waits for the barrier when the origin moved: the
    // lane before reads column first-1's y word in this pass.
    const bool moved = o_row != o_up;
    const Buf wr = buf + (first - o_row);
    int32_t Hp[K];
    int32_t Y = 0, y_first = 0;
    if (cnt > 0) {
      const Buf rd = buf + (first - 1 - o_up);
      int32_t Dn = rd[0].x;
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        if (kk >= cnt) break;
        const int2 e = rd[kk + 1];
        const int32_t D = Dn;
        Dn = e.x;
        const uint32_t y = (uint32_t)e.y;
        const int32_t Sb = prmt_s8(rp_lo, rp_hi, (y >> kCodeShift) + 0x5550u);
        const int32_t M = D > 0 ? D + Sb - 128 : 0;
        const int32_t F = (int32_t)(y & kFMask);
        const int32_t Fn = __viaddmax_s32_relu(M, -oe_del, F - e_del);
        const int32_t yn = (int32_t)((y & ~kFMask) | (uint32_t)Fn);
        if (kk > 0 || !moved)
          wr[kk].y = yn;
        else
          y_first = yn;
        Hp[kk] = __vimax3_s32(M, Y, F);
        Y = __viaddmax_s32_relu(M, -oe_ins, Y - e_ins);
      }
    }
    // insertion carry into this lane: max over earlier lanes l' of their
    // carry Y_l' decayed over the (l - 1 - l') * k columns in between
    const int32_t decay = e_ins * kq;
    const int32_t ex = g.excl_max(Y + decay * lane);
    int32_t E = lane == 0 ? 0 : max(0, ex - decay * (lane - 1));
    g.sync();  // every read of the row above is done
    // pass 2: H, the lane's maximum (largest column on ties), dead columns
    int32_t Hl = -1, kl = 0;
    uint32_t dead = 0;
    if (cnt > 0) {
      if (moved) wr[0].y = y_first;
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        if (kk >= cnt) break;
        const int32_t H = max(Hp[kk], E);
        E -= e_ins;
        const bool ge = H >= Hl;
        Hl = ge ? H : Hl;
        kl = ge ? kk : kl;
        dead |= H == 0 ? 1u << kk : 0u;
        wr[kk].x = H;
      }
    }
    const int32_t hb = (beg == 0 && i + 1 <= w) ? max(0, h0 - oe_del - e_del * i) : 0;
    if (lane == 0) buf[beg - 1 - o_row] = make_int2(hb, (int32_t)(4u << kCodeShift));
    if (lane == G - 1) buf[end - o_row] = make_int2(0, (int32_t)(q_end << kCodeShift));
    int32_t m, mj;
    g.max_last(Hl, first + kl, &m, &mj);
    g.sync();  // the row is stored
    // end-to-end score when the row reaches the last query column
    if (end == qlen) {
      const int32_t gv = buf[qlen - 1 - o_row].x;
      if (gv >= gscore) {
        gscore = gv;
        gtle = i + 1;
      }
    }
    if (m == 0) break;
    cells += end - beg;
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
    // the first and the last live column of the row (the row maximum is > 0,
    // so some lane holds one); the dead cells at both ends are dropped
    const uint32_t live = (cnt >= 32 ? 0xffffffffu : (1u << cnt) - 1u) & ~dead;
    int32_t ll = live ? first + 31 - __clz(live) : -1;
    int32_t fl = live ? first + __ffs(live) - 1 : INT_MAX;
    g.all_max_min(&ll, &fl);
    // next row: the columns the live cells reach in one step, within the band
    beg = max(fl, i + 1 - w);
    end = min(min(ll + 2, i + w + 2), qlen);
  }
  if (lane == 0) put_result(a, k, best, bj + 1, bi + 1, gscore, gtle, max_off, XT_OK, cells);
  g.sync();  // the buffer is free for the group's next pair
}

// Columns per lane K and lanes per pair G of a class (capacity 64 << class).
template <int C>
struct BwaClass {
  static constexpr int K = kBwaK;
  static constexpr int G = (64 << C) / K;
  static constexpr bool kSeg = G <= 32;
  static constexpr int kPairsPerBlock = kSeg ? kBwaWarpThreads / G : 1;
  static constexpr int kBufElems = G * K + 2;  // per pair
  static constexpr int kThreads = kSeg ? kBwaWarpThreads : G;
  static constexpr size_t kSmem = (size_t)kPairsPerBlock * kBufElems * sizeof(int2);
};

// Six CTAs per SM for the warp-segment classes (at most 80 registers, no
// spills; 6 x 33 KB of row buffers): more warps to cover shared-memory and
// dependency latency.
template <int C>
__global__ void __launch_bounds__(kBwaWarpThreads, 6) k_bwa_seg(BwaArgs a, int32_t off,
                                                                int32_t count) {
  using Cl = BwaClass<C>;
  constexpr int G = Cl::G;
  __shared__ int2 s_buf[Cl::kPairsPerBlock * Cl::kBufElems];
  Group<G> g;
  g.init();
  // the S groups of a half-warp interleave their buffers (see RowBuf)
  constexpr int S = G <= 8 ? 16 / G : 1;
  static_assert(Cl::kPairsPerBlock % S == 0, "groups of a block fill whole interleaved sets");
  const int gi = threadIdx.x / G;
  const RowBuf<S> buf{s_buf + (gi / S) * S * Cl::kBufElems + gi % S};
  for (;;) {
    const int32_t p = g.claim(&a.heads[C]);
    if (p >= count) break;
    const int32_t idx = off + p;
    if (idx < 0 || idx >= a.n) break;  // defensive: order index out of range
    const int32_t k = a.order[idx];
    if (k < 0 || k >= a.n) continue;
    bwa_pair<G, Cl::K>(a, g, buf, k);
  }
}

// One pair per CTA; the row buffer in dynamic shared memory.
template <int C>
__global__ void __launch_bounds__(BwaClass<C>::G, 512 / BwaClass<C>::G)
    k_bwa_cta(BwaArgs a, int32_t off, int32_t count) {
  using Cl = BwaClass<C>;
  constexpr int G = Cl::G;
  __shared__ typename Group<G, false>::Shared s;
  extern __shared__ int2 d_buf[];
  Group<G> g;
  g.init(&s);
  for (;;) {
    const int32_t p = g.claim(&a.heads[C]);
    if (p >= count) break;
    const int32_t idx = off + p;
    if (idx < 0 || idx >= a.n) break;
    const int32_t k = a.order[idx];
    if (k < 0 || k >= a.n) continue;
    bwa_pair<G, Cl::K>(a, g, RowBuf<1>{d_buf}, k);
  }
}

template <int C>
cudaError_t launch_class(xt_ctx* ctx, const BwaArgs& a, int32_t off, int32_t count,
                         cudaStream_t stream) {
  using Cl = BwaClass<C>;
  int& resident = ctx->bwa_blocks[C];
  const size_t dyn = Cl::kSeg ? 0 : Cl::kSmem;
  if (resident == 0) {
    cudaError_t e;
    if constexpr (Cl::kSeg) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_bwa_seg<C>, Cl::kThreads, 0);
    } else {
      e = cudaFuncSetAttribute(k_bwa_cta<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)dyn);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_bwa_cta<C>, Cl::kThreads,
                                                          dyn);
    }
    if (e != cudaSuccess) return e;
    if (resident < 1) resident = 1;
  }
  const int64_t want = ((int64_t)count + Cl::kPairsPerBlock - 1) / Cl::kPairsPerBlock;
  const int grid = (int)std::min<int64_t>(want, (int64_t)resident * ctx->num_sms);
  if constexpr (Cl::kSeg)
    k_bwa_seg<C><<<grid, Cl::kThreads, 0, stream>>>(a, off, count);
  else
    k_bwa_cta<C><<<grid, Cl::kThreads, dyn, stream>>>(a, off, count);
  return cudaGetLastError();
}

cudaError_t launch_bwa_class(xt_ctx* ctx, const BwaArgs& a, int cls, int32_t off, int32_t count,
                             cudaStream_t stream) {
  switch (cls) {
    case 0: return launch_class<0>(ctx, a, off, count, stream);
    case 1: return launch_class<1>(ctx, a, off, count, stream);
    case 2: return launch_class<2>(ctx, a, off, count, stream);
    case 3: return launch_class<3>(ctx, a, off, count, stream);
    case 4: return launch_class<4>(ctx, a, off, count, stream);
    case 5: return launch_class<5>(ctx, a, off, count, stream);
    case 6: return launch_class<6>(ctx, a, off, count, stream);
    case 7: return launch_class<7>(ctx, a, off, count, stream);
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
  xt_status s = ctx_codes(ctx, &q_seq, &q_bytes, &t_seq, &t_bytes, st);
  if (s != XT_OK) return s;
  // workspace: class bytes, order, counters
  const size_t n = (size_t)n_pairs;
  const size_t o_cls = 0;
  const size_t o_order = align256(o_cls + n);
  const size_t o_slots = align256(o_order + 4 * n);
  const size_t n_ctr = (size_t)kBwaClasses * kBwaLenBuckets + 2 * kBwaClasses;
  const size_t bytes = align256(o_slots + 4 * n_ctr);
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
  a.slots = reinterpret_cast<int32_t*>(ws + o_slots);
  a.counts = a.slots + kBwaClasses * kBwaLenBuckets;
  a.heads = a.counts + kBwaClasses;
  const int threads = 256;
  const int grid = (int)std::min<int64_t>(((int64_t)n_pairs + threads - 1) / threads,
                                          (int64_t)ctx->num_sms * 8);
  e = cudaMemsetAsync(a.slots, 0, 4 * n_ctr, st);
  if (e == cudaSuccess) {
    k_bwa_classify<<<grid, threads, 0, st>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_bwa_scan<<<1, kBwaScanThreads, 0, st>>>(a);
    e = cudaGetLastError();
  }
  // the class sizes come back to size the launches
  int32_t* cnt_host = ctx->seg_host + kSegHostBwaCounts;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cnt_host, a.counts, 4 * kBwaClasses, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->seg_ev, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(ctx->seg_ev);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "BWA classify");
  int32_t off[kBwaClasses];
  int32_t total = 0;
  int32_t cnt[kBwaClasses];
  for (int c = 0; c < kBwaClasses; ++c) {
    cnt[c] = cnt_host[c];
    off[c] = total;
    total += cnt[c];
  }
  if (total == 0) return XT_OK;
  k_bwa_scatter<<<grid, threads, 0, st>>>(a);
  e = cudaGetLastError();
  // widest groups first: they hold the longest rows
  for (int c = kBwaClasses - 1; c >= 0 && e == cudaSuccess; --c)
    if (cnt[c] > 0) e = launch_bwa_class(ctx, a, c, off[c], cnt[c], st);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "BWA extension");
  ctx->calls++;
  return XT_OK;
}
