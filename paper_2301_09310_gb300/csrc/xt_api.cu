// xt_api.cu -- the C ABI of include/xt.h: context, argument checks, device
// workspace, launch plan and the host-buffer (end-to-end) variant.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "xt.h"
#include "xt_ctx.cuh"
#include "xt_kernels.cuh"

using namespace xt;

namespace {

constexpr size_t kAlign = 256;
constexpr int kPlainRsCapLog2 = 13;    // plain kernel ring up to 8192 entries (64 KB)
constexpr int kQueueRsCapLog2 = 12;    // queue kernels: ring up to 4096 entries per group
constexpr size_t kPoolCap = (size_t)2 << 30;  // global ring pool cap (allocated only when a plan needs it)

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int log2_ceil(int64_t x) {
  int k = 0;
  while (((int64_t)1 << k) < x) ++k;
  return k;
}

xt_status fail(xt_ctx* ctx, xt_status s, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return s;
}

xt_status cuda_fail(xt_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, XT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool scoring_ok(const xt_scoring* sc) {
  if (!sc) return false;
  if (sc->match < 1 || sc->match > 127) return false;
  if (sc->mismatch > 0 || sc->mismatch < -127) return false;
  if (sc->n_score > 0 || sc->n_score < -127) return false;
  if (sc->gap_open < 0 || sc->gap_open > 1023) return false;
  if (sc->gap_extend < 0 || sc->gap_extend > 1023) return false;
  if (sc->w < 0) return false;
  return true;
}

Score make_score(const xt_scoring* s) {
  Score sc;
  sc.alpha = s->gap_open + s->gap_extend;
  sc.beta = s->gap_extend;
  // a band wider than any pair changes nothing; clamp so index arithmetic stays in int32
  sc.w = s->w > 2 * XT_MAX_LEN ? 2 * XT_MAX_LEN : s->w;
  sc.zdrop = s->zdrop;
  const uint32_t mb = (uint8_t)(int8_t)s->match, xb = (uint8_t)(int8_t)s->mismatch,
                 nb = (uint8_t)(int8_t)s->n_score;
  for (int qc = 0; qc < 4; ++qc) {
    uint32_t v = 0;
    for (int tb = 0; tb < 4; ++tb) v |= (tb == qc ? mb : xb) << (8 * tb);
    sc.prof[qc] = v;
  }
  sc.nnnn = nb | (nb << 8) | (nb << 16) | (nb << 24);
  sc.prof[4] = sc.nnnn;
  return sc;
}

xt_status dev_alloc(xt_ctx* ctx, void** p, size_t* have, size_t want) {
  if (*have >= want) return XT_OK;
  const size_t grow = want - *have;
  if (ctx->budget && ctx->held + grow > ctx->budget)
    return fail(ctx, XT_ENOMEM, "device memory budget exceeded");
  if (*p) {
    cudaFree(*p);
    ctx->held -= *have;
    *p = nullptr;
    *have = 0;
  }
  cudaError_t e = cudaMalloc(p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ctx, XT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  *have = want;
  ctx->held += want;
  return XT_OK;
}

}  // namespace

xt_status xt::ctx_fail(xt_ctx* ctx, xt_status s, const char* msg) { return fail(ctx, s, msg); }

xt_status xt::ctx_cuda_fail(xt_ctx* ctx, cudaError_t e, const char* where) {
  return cuda_fail(ctx, e, where);
}

xt_status xt::ctx_alloc(xt_ctx* ctx, void** p, size_t* have, size_t want) {
  return dev_alloc(ctx, p, have, want);
}


xt_status xt::ctx_codes(xt_ctx* ctx, const uint8_t** q_seq, int64_t* q_bytes,
                        const uint8_t** t_seq, int64_t* t_bytes, cudaStream_t stream) {
  if (ctx->alphabet == XT_ALPHABET_CODES) return XT_OK;
  const bool packed = ctx->alphabet == XT_ALPHABET_PACKED4;
  const int64_t qn = packed ? 2 * *q_bytes : *q_bytes, tn = packed ? 2 * *t_bytes : *t_bytes;
  const size_t qa = align_up((size_t)qn);
  xt_status s = dev_alloc(ctx, &ctx->conv, &ctx->conv_bytes, qa + (size_t)tn + kAlign);
  if (s != XT_OK) return s;
  uint8_t* cq = static_cast<uint8_t*>(ctx->conv);
  cudaError_t e;
  if (packed) {
    e = launch_unpack4(*q_seq, cq, 0, *q_bytes, ctx->num_sms, stream);
    if (e == cudaSuccess) e = launch_unpack4(*t_seq, cq + qa, 0, *t_bytes, ctx->num_sms, stream);
  } else {
    e = launch_ascii_codes(*q_seq, cq, *q_bytes, ctx->num_sms, stream);
    if (e == cudaSuccess) e = launch_ascii_codes(*t_seq, cq + qa, *t_bytes, ctx->num_sms, stream);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, packed ? "4-bit unpacking" : "ASCII conversion");
  *q_seq = cq;
  *t_seq = cq + qa;
  *q_bytes = qn;
  *t_bytes = tn;
  return XT_OK;
}

void xt::drop_graphs(xt_ctx* ctx) {
  for (auto& g : ctx->graph_cache)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  ctx->graph_cache.clear();
}

namespace {

// Carve the per-call workspace for up to n pairs (and the device batch
// descriptor).  Calls pass their capacity class n_cap, not their own n: the
// region offsets then depend only on the class, so a graph captured for one
// call of a class stays valid for every other call of that class.
xt_status get_work(xt_ctx* ctx, int32_t n, Work* w, Batch** desc) {
  size_t off = 0;
  const size_t o_desc = off; off = align_up(off + sizeof(Batch));
  const size_t o_pclass = off; off = align_up(off + (size_t)n);
  const size_t o_order = off; off = align_up(off + 4 * (size_t)n);
  const size_t o_counts = off; off = align_up(off + 4 * (size_t)kNumBuckets);
  const size_t o_cursor = off; off = align_up(off + 4 * (size_t)kNumBuckets);
  const size_t o_sb = off; off = align_up(off + 4 * (size_t)(kNumClasses * kNumJ));
  const size_t o_se = off; off = align_up(off + 4 * (size_t)(kNumClasses * kNumJ));
  const size_t o_heads = off; off = align_up(off + 4 * (size_t)kMaxLaunches);
  void* old = ctx->work;
  xt_status s = dev_alloc(ctx, &ctx->work, &ctx->work_bytes, off);
  if (s != XT_OK) return s;
  if (ctx->work != old) drop_graphs(ctx);
  char* base = (char*)ctx->work;
  *desc = (Batch*)(base + o_desc);
  w->pclass = (uint8_t*)(base + o_pclass);
  w->order = (int32_t*)(base + o_order);
  w->counts = (int32_t*)(base + o_counts);
  w->cursor = (int32_t*)(base + o_cursor);
  w->seg_begin = (int32_t*)(base + o_sb);
  w->seg_end = (int32_t*)(base + o_se);
  w->heads = (int32_t*)(base + o_heads);
  return XT_OK;
}

struct Plan {
  Launch launch[kMaxLaunches];
  int n_launch = 0;
  bool bad = false;   // count-aware planning met a bucket it cannot place
  JFlags jf = {};
  bool any_huge = false;
  int64_t slab = 0;
  bool pool_serial = true;  // global-ring launches share one pool region, in order
};

int64_t next_pow2(int64_t x) { return (int64_t)1 << log2_ceil(x); }

// Schedule of bucket j (queries of qlen + 2 <= 2^j): the fewest lanes per pair
// whose shared-memory ring fits 32 KB per CTA.  The ring needs
// min(qlen, P*R + 2w) + 2 entries.
// The tuned schedule of bucket j for band w and the size class of the call
// being planned, or nullptr (built-in rule).
const BucketSched* tuned(const xt_ctx* ctx, int w, int j) {
  if (ctx->forced_P) return nullptr;
  for (const auto& t : ctx->tuning) {
    if (t.w != w) continue;
    if (ctx->plan_small && t.small[j].P > 0) return &t.small[j];
    if (t.b[j].P > 0) return &t.b[j];
  }
  return nullptr;
}

// Ring entries (log2) of a group-engine pair of bucket j under band w.
int queue_ring_log2(int j, int w, int P, int R) {
  return log2_ceil(std::min<int64_t>((int64_t)1 << j, next_pow2((int64_t)P * R + 2 * (int64_t)w + 2)));
}

bool queue_instantiated(int P, int R) {
  if (R == 4 || R == 8) return P == 1 || P == 2 || P == 4 || P == 8 || P == 16 || P == 32;
  if (R == 16) return P == 1 || P == 2 || P == 4;
  return false;
}

void bucket_schedule(const xt_ctx* ctx, int j, int w, int* P, int* R, int* rs_log2, bool* huge,
                     bool allow_gring = true) {
  if (const BucketSched* t = tuned(ctx, w, j)) {
    if (t->P > 1) {
      *P = t->P; *R = t->R; *rs_log2 = queue_ring_log2(j, w, t->P, t->R); *huge = false;
      return;
    }
  }
  if (ctx->forced_P > 1) {
    const int64_t need = std::min<int64_t>(
        (int64_t)1 << j, next_pow2((int64_t)ctx->forced_P * ctx->forced_R + 2 * (int64_t)w + 2));
    const int lg = log2_ceil(need);
    if (lg <= kQueueRsCapLog2 &&
        queue_smem_bytes(ctx->forced_P, lg) <= (size_t)ctx->smem_optin - 1024) {
      *P = ctx->forced_P; *R = ctx->forced_R; *rs_log2 = lg; *huge = false;
      return;
    }
  }
  const int Rr = 8;
  for (int p = 1; p <= 32; p *= 2) {
    const int64_t need = std::min<int64_t>((int64_t)1 << j, next_pow2((int64_t)p * Rr + 2 * (int64_t)w + 2));
    const int lg = log2_ceil(need);
    const size_t bytes = queue_smem_bytes(p, lg);
    // a ring that leaves room for fewer than two CTAs per SM runs better
    // from the global slabs of the HUGE class (two CTAs per SM), where those
    // are allowed
    const size_t cap = allow_gring ? (size_t)ctx->smem_optin / 2 - 1024 : (size_t)ctx->smem_optin;
    if (bytes <= 32 * 1024 || (p == 32 && lg <= kQueueRsCapLog2 && bytes <= cap)) {
      *P = p; *R = Rr; *rs_log2 = lg; *huge = false;
      return;
    }
  }
  *P = 32; *R = 8; *rs_log2 = 0; *huge = true;
}

void add_huge_launch(xt_ctx* ctx, const Score& sc, Plan* pl) {
  // global slabs: ring of min(qlen, 256 + 2w) + 2 entries, qlen <= XT_MAX_LEN
  const int64_t need = std::min<int64_t>(XT_MAX_LEN, 256 + 2 * (int64_t)sc.w) + 2;
  pl->slab = next_pow2(need);
  const int64_t per_cta = (kQueueThreads / 32) * pl->slab * (int64_t)sizeof(int2);
  int64_t grid = (int64_t)kPoolCap / per_cta;
  if (grid > 2 * ctx->num_sms) grid = 2 * ctx->num_sms;
  if (grid < 1) grid = 1;
  Launch& L = pl->launch[pl->n_launch++];
  L = Launch();
  L.cls = CLS_HUGE; L.j_lo = 0; L.j_hi = kJMax; L.lane = false; L.P = 32; L.R = 8;
  L.rs_log2 = 0; L.global_ring = true; L.slab = pl->slab; L.grid = (int)grid; L.mparam = 0;
}

constexpr int kLaneJMax = 9;           // single-phase plan: one-lane engine up to 2^9 - 2 bases
// one-lane rows per strip without a tuned schedule: 16 above 510 bases (the
// long buckets' strips amortise their start over more rows)
inline int lane_default_R(int j) { return j >= 10 ? 16 : 8; }
constexpr size_t kLaneSmemCap = 48 * 1024;

// One-lane launch of bucket j for class cls (PACKED or NARROW); false if it
// needs a global ring and those are not allowed.
bool lane_launch(xt_ctx* ctx, const Score& sc, int cls, int j, bool allow_gring, Launch* L) {
  const BucketSched* t = tuned(ctx, sc.w, j);
  int R = ctx->forced_P == 1 ? ctx->forced_R : (t && t->P == 1 ? t->R : lane_default_R(j));
  // the packed engine's 16-row strips need more registers than it has (they
  // spill); its long buckets, and those with 4-bit row-key tags, keep 8
  if (cls == CLS_PACKED && R > 8 && (ctx->forced_P != 1 || packed_tag_bits(j) == 4)) R = 8;
  const int rows = cls == CLS_PACKED ? 2 * R : R;
  const int64_t need = std::min<int64_t>((int64_t)1 << j, next_pow2(rows + 2 * (int64_t)sc.w + 2));
  const int lg = log2_ceil(need);
  const size_t ring = (size_t)kLaneThreads * lane_ring_bytes(cls, lg);
  const bool gring = ring > kLaneSmemCap;
  if (gring && !allow_gring) return false;
  L->cls = cls; L->j_lo = j; L->j_hi = j; L->lane = true; L->P = 1; L->R = R;
  L->rs_log2 = lg; L->global_ring = gring; L->slab = gring ? ((int64_t)1 << lg) : 0;
  const size_t smem = (gring ? 0 : ring) + (cls == CLS_PACKED ? lane_stage_bytes(j) : 0) +
                      lane_pipe_bytes(cls, gring);
  const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(220 * 1024) / (smem + 1024)));
  L->grid = ctx->num_sms * per_sm;
  int k = 0;
  while ((1 << k) < ctx->match + 1) ++k;
  // packed: the anchoring shift and, above it, the row keys' step-tag bits
  L->mparam = cls == CLS_PACKED ? (k | packed_tag_bits(j) << 8) : ctx->match + 1;
  return true;
}

bool same_config(const Launch& a, const Launch& b) {
  return a.cls == b.cls && a.lane == b.lane && a.P == b.P && a.R == b.R &&
         a.rs_log2 == b.rs_log2 && a.global_ring == b.global_ring && a.grid == b.grid &&
         a.mparam == b.mparam;
}

void plan_batched(xt_ctx* ctx, const Score& sc, Plan* pl, bool allow_gring = true) {
  // which buckets run the one-lane engine (the same answer for every class)
  bool lane_j[kNumJ] = {false};
  for (int j = kJMin; j <= kJMax; ++j) {
    Launch L;
    const BucketSched* t = tuned(ctx, sc.w, j);
    const bool want = ctx->forced_P == 1 || (!ctx->forced_P && (t ? t->P == 1 : j <= kLaneJMax));
    lane_j[j] = want &&
                lane_launch(ctx, sc, CLS_PACKED, j, allow_gring, &L) &&
                lane_launch(ctx, sc, CLS_NARROW, j, allow_gring, &L);
    if (lane_j[j]) pl->jf.f[j] |= kJPacked;
  }
  for (int cls = CLS_PACKED; cls <= CLS_WIDE; ++cls) {
    int prev = -1;
    for (int j = kJMax; j >= kJMin; --j) {
      Launch L;
      if (lane_j[j] && cls != CLS_WIDE) {
        lane_launch(ctx, sc, cls, j, allow_gring, &L);
      } else {
        if (cls == CLS_PACKED) { prev = -1; continue; }  // no packed pairs in this bucket
        int P, R, lg;
        bool huge;
        bucket_schedule(ctx, j, sc.w, &P, &R, &lg, &huge, allow_gring);
        if (huge) {
          pl->jf.f[j] |= kJHuge;
          pl->any_huge = true;
          prev = -1;
          continue;
        }
        L.cls = cls; L.j_lo = j; L.j_hi = j; L.lane = false; L.P = P; L.R = R;
        L.rs_log2 = lg; L.global_ring = false; L.slab = 0; L.mparam = 0;
        const size_t smem = queue_smem_bytes(P, lg);
        const int per_sm = (int)std::min<size_t>(16, std::max<size_t>(1, (size_t)(220 * 1024) / std::max<size_t>(smem + 1024, 1)));
        L.grid = ctx->num_sms * per_sm;
      }
      if (prev >= 0 && same_config(pl->launch[prev], L)) {
        pl->launch[prev].j_lo = j;
        continue;
      }
      pl->launch[pl->n_launch] = L;
      prev = pl->n_launch++;
    }
    // the lowest bucket also takes the pairs below kJMin (classify clamps j)
    if (prev >= 0) pl->launch[prev].j_lo = 0;
  }
  if (pl->any_huge) add_huge_launch(ctx, sc, pl);
}

// ---- count-aware planning (the batched path): classify runs first with
// per-bucket flags that do not depend on the counts, then every non-empty
// bucket is planned from its own pair count.
constexpr int32_t kBucketSmall = XT_SMALL_BUCKET;  // fewer pairs: a bucket cannot fill the GPU
constexpr int32_t kLaneSlots = 77824;    // one-lane thread slots of a full GPU (152 x 4 x 128)
// Built-in rule: the fewest pairs of a bucket for one lane per pair.  A pair's
// time on one lane grows with its length, so a bucket of long queries needs
// close to a full wave of pairs before the one-lane engine pays; short ones
// finish fast even when a bucket leaves most lanes idle.
constexpr int kLongJ = 10;               // buckets of queries longer than 510 bases
inline int32_t lane_min_pairs(int j) { return j >= kLongJ ? 32768 : (j >= 7 ? kBucketSmall : 0); }
// The longest query of bucket j, and the in-band cells of a pair of query
// length q whose target runs to the band's end (q + w rows of at most 2w+1
// columns): the planning estimates of a pair's work.
inline double pair_cells_q(int j) { return (double)(((int64_t)1 << j) - 2); }
inline double band_cells_est(double q, int w) {
  return (q + (double)w) * std::min(q, 2.0 * (double)w + 1.0);
}

// Flags for classify: kJHuge where the default group ring does not fit
// (band geometry only), kJPacked where a one-lane schedule is possible for
// the bucket in either size class, kJTag4 on such buckets of 511-base queries
// and longer in calls of n >= kTag4MinPairs pairs.  lane_ok[j]: that one-lane
// launch exists.
void batched_flags(xt_ctx* ctx, const Score& sc, int32_t n, JFlags* jf, bool* lane_ok) {
  *jf = JFlags{};
  for (int j = 0; j < kNumJ; ++j) lane_ok[j] = false;
  const bool saved = ctx->plan_small;
  for (int j = kJMin; j <= kJMax; ++j) {
    Launch L;
    bool want = false;
    if (ctx->forced_P) {
      want = ctx->forced_P == 1;
    } else {
      for (int small = 0; small < 2; ++small) {
        ctx->plan_small = small != 0;
        const BucketSched* t = tuned(ctx, sc.w, j);
        // untuned buckets of any length may take the one-lane engine where
        // its ring fits (the count decides later)
        want |= t ? t->P == 1 : bucket_sched_ok(ctx, sc.w, j, 1, lane_default_R(j));
      }
      ctx->plan_small = false;
    }
    lane_ok[j] = want && lane_launch(ctx, sc, CLS_PACKED, j, true, &L) &&
                 lane_launch(ctx, sc, CLS_NARROW, j, true, &L);
    if (lane_ok[j])
      jf->f[j] |= kJPacked | (packed_tag_bits(j) == 4 && n >= kTag4MinPairs ? kJTag4 : 0);
    // the default rule's answer (tuned group schedules always fit, see
    // bucket_sched_ok, but a bucket's class must not depend on its count)
    const int fP = ctx->forced_P;
    int P, R, lg;
    bool huge;
    std::vector<TuneEntry> keep;
    keep.swap(ctx->tuning);
    ctx->forced_P = fP > 1 ? fP : 0;
    bucket_schedule(ctx, j, sc.w, &P, &R, &lg, &huge, true);
    ctx->forced_P = fP;
    keep.swap(ctx->tuning);
    // a bucket the group engine cannot hold runs on the one-lane engine when
    // it can; only its WIDE pairs (group engine only) then go to the HUGE class
    if (huge) jf->f[j] |= lane_ok[j] ? kJHugeWide : kJHuge;
  }
  ctx->plan_small = saved;
}

Launch queue_launch(const xt_ctx* ctx, int cls, int j, int P, int R, int lg) {
  Launch L;
  L.cls = cls; L.j_lo = j; L.j_hi = j; L.lane = false; L.P = P; L.R = R; L.rs_log2 = lg;
  const size_t smem = queue_smem_bytes(P, lg);
  const int per_sm = (int)std::min<size_t>(
      16, std::max<size_t>(1, (size_t)(220 * 1024) / std::max<size_t>(smem + 1024, 1)));
  L.grid = ctx->num_sms * per_sm;
  return L;
}

// Plan the DP launches from the pair count of every (class, bucket):
// empty buckets get no launch; a bucket too small to fill the GPU takes its
// small-batch schedule, or by default a group schedule with enough lanes per
// pair to fill it; larger buckets take the throughput schedule.
void plan_counts(xt_ctx* ctx, const Score& sc, const int32_t (*cnt)[kNumJ], const JFlags& jf,
                 const bool* lane_ok, Plan* pl) {
  pl->jf = jf;
  const bool saved = ctx->plan_small;
  // the call's estimated cells: each bucket's pairs at a query length three
  // quarters of the way up the bucket
  double est_cells = 0.0;
  for (int cls = CLS_PACKED; cls < kNumClasses; ++cls)
    for (int j = 0; j < kNumJ; ++j)
      if (cnt[cls][j]) {
        const int jj = j < kJMin ? kJMin : j;
        est_cells += (double)cnt[cls][j] * band_cells_est(0.75 * pair_cells_q(jj), sc.w);
      }
  // long queries: one lane per pair needs many pairs to fill the GPU, but
  // the long buckets of one call run side by side, so when together they
  // hold two full waves of lanes each of them takes the one-lane engine
  int64_t long_pairs = 0;
  for (int cls = CLS_PACKED; cls <= CLS_NARROW; ++cls)
    for (int j = kLongJ; j < kNumJ; ++j)
      if (lane_ok[j]) long_pairs += cnt[cls][j];
  const bool long_lanes = long_pairs >= 2 * (int64_t)kLaneSlots;
  auto min_pairs = [&](int jj) { return jj >= kLongJ && long_lanes ? 0 : lane_min_pairs(jj); };
  for (int cls = CLS_PACKED; cls <= CLS_WIDE; ++cls) {
    int prev = -1;
    for (int j = kJMax; j >= 0; --j) {
      const int32_t c = cnt[cls][j];
      if (c == 0) continue;                   // empty: the launch before it may span it
      const int jj = j < kJMin ? kJMin : j;   // classify clamps short queries into kJMin
      ctx->plan_small = c < kBucketSmall;
      Launch L;
      bool lane = false;
      if (cls != CLS_WIDE && lane_ok[jj]) {
        lane = true;
        if (ctx->forced_P > 1) {
          lane = false;
        } else if (!ctx->forced_P) {
          const BucketSched* t = tuned(ctx, sc.w, jj);
          if (t) lane = t->P == 1;
          // latency rule below; a long bucket still takes one lane per pair
          // when its longest pair on one lane takes at most half of the call's
          // whole work spread over the GPU (the one-lane engine is the
          // cheapest per cell, and the call's other buckets fill the slots it
          // leaves; without the factor two, 400k- and 1M-pair calls of the
          // c5 mix measured slower)
          else if (c < min_pairs(jj))
            lane = jj >= kLongJ && 2.0 * band_cells_est(pair_cells_q(jj), sc.w) *
                                           (double)kLaneSlots <= est_cells;
        }
      }
      if (lane) {
        lane_launch(ctx, sc, cls, jj, true, &L);
      } else {
        int P = 0, R = 8, lg = 0;
        bool huge = false;
        const BucketSched* t = ctx->forced_P ? nullptr : tuned(ctx, sc.w, jj);
        if (!ctx->forced_P && !t && c < min_pairs(jj) && cls != CLS_WIDE) {
          // enough lanes per pair that the bucket's longest pair takes no
          // longer than the call's whole work spread over the GPU's one-lane
          // slots (the call's buckets run side by side, so a small bucket
          // need not fill the GPU on its own; fewer lanes per pair waste less
          // of each chunk on the wavefront's fill), where the ring fits
          const double need = band_cells_est(pair_cells_q(jj), sc.w) * (double)kLaneSlots /
                              std::max(est_cells, 1.0);
          int want = 4;  // two-lane groups measured slower than four on every call size
          while (want < 32 && want < need) want *= 2;
          for (int q = want; q >= 2 && P == 0; q /= 2) {
            const int l = queue_ring_log2(jj, sc.w, q, 8);
            if (l <= kQueueRsCapLog2 && queue_smem_bytes(q, l) <= (size_t)ctx->smem_optin / 2 - 1024) {
              P = q;
              lg = l;
            }
          }
        }
        if (P == 0) bucket_schedule(ctx, jj, sc.w, &P, &R, &lg, &huge, true);
        if (huge && cls != CLS_WIDE && lane_ok[jj]) {
          lane_launch(ctx, sc, cls, jj, true, &L);  // no group ring fits: one lane per pair
        } else if (huge) {
          // the flags gave these pairs no HUGE class, so they would be lost
          pl->bad = true;
          continue;
        } else {
          L = queue_launch(ctx, cls, jj, P, R, lg);
        }
      }
      L.j_lo = j;
      L.j_hi = j;
      if (prev >= 0 && same_config(pl->launch[prev], L)) {
        pl->launch[prev].j_lo = j;
        continue;
      }
      if (pl->n_launch >= kMaxLaunches - 1) {  // 3 classes x 17 buckets + 1 stay below
        pl->bad = true;
        continue;
      }
      pl->launch[pl->n_launch] = L;
      prev = pl->n_launch++;
    }
  }
  ctx->plan_small = saved;
  // longest queries first: their pairs set the call's critical path, and the
  // launches after them fill the slots they leave (c5-mix call of 1M pairs:
  // 21.6 ms in class order, 19.7 ms in this order, both with the rings apart)
  std::stable_sort(pl->launch, pl->launch + pl->n_launch,
                   [](const Launch& a, const Launch& b) { return a.j_hi > b.j_hi; });
  int32_t huge_pairs = 0;
  for (int j = 0; j < kNumJ; ++j) huge_pairs += cnt[CLS_HUGE][j];
  if (huge_pairs > 0) {
    pl->any_huge = true;
    add_huge_launch(ctx, sc, pl);
  }
}

// Device bytes of one global-ring launch's slabs.
size_t ring_launch_bytes(const Launch& L) {
  if (L.lane) return (size_t)L.grid * kLaneThreads * (size_t)L.slab * lane_ring_bytes(L.cls, 0);
  return (size_t)L.grid * (kQueueThreads / L.P) * (size_t)L.slab * sizeof(int2);
}

// Lay out the global rings of a plan in the pool and return the bytes it
// needs: every global-ring launch gets its own region when they all fit the
// pool cap and the context's budget (the launches then run side by side on
// the call's branches, each filling the slots the others leave), else they
// share one region and run one after another.
size_t layout_pool(const xt_ctx* ctx, Plan* pl) {
  size_t sum = 0, most = 0;
  for (int i = 0; i < pl->n_launch; ++i) {
    Launch& L = pl->launch[i];
    if (!L.global_ring) continue;
    const size_t b = ring_launch_bytes(L);
    L.pool_off = sum;
    sum += align_up(b);
    most = std::max(most, b);
  }
  const bool fits = sum <= kPoolCap &&
                    (ctx->budget == 0 || sum <= ctx->pool_bytes ||
                     ctx->held + (sum - ctx->pool_bytes) <= ctx->budget);
  pl->pool_serial = !fits;
  if (fits) return sum;
  for (int i = 0; i < pl->n_launch; ++i) pl->launch[i].pool_off = 0;
  return most;
}

}  // namespace

// Size a context's device buffers once for calls of up to n_pairs pairs: the
// workspace of that capacity class, the global ring pool to pool_bytes (at
// most its cap, as far as the budget allows; a plan that needs more grows it
// later) and, when conv_bytes > 0, the buffer of converted sequences.  A
// long-running caller (the server's slots) then does not free and regrow them
// between calls: a cudaFree waits for the whole device.
xt_status xt::ctx_reserve(xt_ctx* ctx, int32_t n_pairs, size_t conv_bytes, size_t pool_bytes) {
  if (!ctx || n_pairs < 0) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, XT_ECUDA, "cudaSetDevice");
  int lg = 10;
  while (lg < 31 && (1 << lg) < n_pairs) ++lg;
  Work w;
  Batch* desc = nullptr;
  xt_status s = get_work(ctx, lg >= 31 ? INT32_MAX : (1 << lg), &w, &desc);
  if (s == XT_OK && conv_bytes) s = dev_alloc(ctx, &ctx->conv, &ctx->conv_bytes, conv_bytes);
  if (s != XT_OK) return s;
  size_t pool = std::min(pool_bytes, kPoolCap);
  if (ctx->budget) {
    const size_t left = ctx->budget > ctx->held ? ctx->budget - ctx->held : 0;
    pool = std::min(pool, ctx->pool_bytes + left);
  }
  if (pool > ctx->pool_bytes) {
    void* old = ctx->pool;
    s = dev_alloc(ctx, (void**)&ctx->pool, &ctx->pool_bytes, pool);
    if (ctx->pool != old) drop_graphs(ctx);
  }
  return s;
}

bool xt::bucket_sched_ok(const xt_ctx* ctx, int w, int j, int P, int R) {
  if (j < kJMin || j > kJMax || w < 0) return false;
  if (P == 1) {
    if (R != 4 && R != 8 && R != 16) return false;
    // one-lane rings beyond shared memory go to the global pool: keep it bounded
    const int64_t need = std::min<int64_t>((int64_t)1 << j, next_pow2(2 * R + 2 * (int64_t)w + 2));
    const size_t per_cta = (size_t)kLaneThreads * lane_ring_bytes(CLS_NARROW, log2_ceil(need));
    return per_cta <= kLaneSmemCap || per_cta * 4 * (size_t)ctx->num_sms <= kPoolCap;
  }
  if (!queue_instantiated(P, R)) return false;
  const int lg = queue_ring_log2(j, w, P, R);
  return lg <= kQueueRsCapLog2 && queue_smem_bytes(P, lg) <= (size_t)ctx->smem_optin - 1024;
}

namespace {

void plan_plain(xt_ctx* ctx, const Score& sc, Plan* pl, int* rs_log2) {
  const int64_t need = 256 + 2 * (int64_t)sc.w + 2;
  int lg = log2_ceil(need);
  if (lg > kPlainRsCapLog2) lg = kPlainRsCapLog2;
  *rs_log2 = lg;
  for (int j = kJMin; j <= kJMax; ++j) {
    // a pair of bucket j needs at most min(2^j, 256 + 2w + 2) ring entries
    const int64_t nj = std::min<int64_t>((int64_t)1 << j, next_pow2(need));
    if (nj > ((int64_t)1 << lg)) {
      pl->jf.f[j] |= kJHuge;
      pl->any_huge = true;
    }
  }
  if (pl->any_huge) add_huge_launch(ctx, sc, pl);
}

xt_status check_args(xt_ctx* ctx, const void* q_seq, int64_t q_bytes, const void* q_off,
                     const void* q_len, const void* t_seq, int64_t t_bytes, const void* t_off,
                     const void* t_len, const void* h0, int32_t n, const xt_scoring* sc,
                     const void* out) {
  if (!ctx) return XT_EINVAL;
  if (n < 0) return fail(ctx, XT_EINVAL, "n_pairs < 0");
  if (!scoring_ok(sc)) return fail(ctx, XT_EINVAL, "scoring record out of range");
  if (q_bytes < 0 || t_bytes < 0) return fail(ctx, XT_EINVAL, "negative buffer size");
  if (n > 0 && (!q_off || !q_len || !t_off || !t_len || !h0 || !out))
    return fail(ctx, XT_EINVAL, "null array");
  if ((q_bytes > 0 && !q_seq) || (t_bytes > 0 && !t_seq))
    return fail(ctx, XT_EINVAL, "null sequence buffer");
  return XT_OK;
}

// The front of a call: reset counters, classify, order the queue.
cudaError_t enqueue_front(const JFlags& jf, const Score& sc, int32_t match, const Work& w,
                          const Batch* desc, int32_t n_cap, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(w.counts, 0, 4 * (size_t)kNumBuckets, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.heads, 0, 4 * (size_t)kMaxLaunches, stream);
  if (e == cudaSuccess) e = launch_classify(desc, n_cap, sc, match, jf, w, stream);
  if (e == cudaSuccess) e = launch_order(desc, n_cap, w, stream);
  return e;
}

// The extension kernels of a call (and the plain kernel for the plain path).
cudaError_t enqueue_dp(xt_ctx* ctx, bool plain, const Plan& pl, int plain_rs, const Score& sc,
                       const Work& w, const Batch* desc, int32_t n_cap, cudaStream_t stream,
                       int* dp_out) {
  cudaError_t e = cudaSuccess;
  const int slot = ctx->ev_pending;
  const bool timed = ctx->timing && slot < xt_ctx::kEvRing;
  if (timed) {
    for (int k = 0; k < 2; ++k)
      if (!ctx->ev[slot][k]) cudaEventCreate(&ctx->ev[slot][k]);
    cudaEventRecord(ctx->ev[slot][0], stream);
  }
  int dp = 0;
  if (e == cudaSuccess && plain) {
    e = launch_plain(desc, n_cap, sc, w, plain_rs, stream);
    ++dp;
  }
  // The DP launches are independent (each drains its own bucket range), so
  // they fork onto the auxiliary streams: a launch's tail overlaps the next
  // launch's start, and small batches fill the GPU.  Global-ring launches
  // with regions of their own fork too; sharing one region (a plan whose
  // rings exceed the pool cap or the budget) they stay in order on branch 0.
  const int nb = std::min(ctx->branches, pl.n_launch);
  if (e == cudaSuccess && nb > 1) {
    e = cudaEventRecord(ctx->fork_ev, stream);
    for (int b = 0; e == cudaSuccess && b < nb; ++b) e = cudaStreamWaitEvent(ctx->aux[b], ctx->fork_ev, 0);
  }
  for (int i = 0, rr = 0; e == cudaSuccess && i < pl.n_launch; ++i) {
    const Launch& L = pl.launch[i];
    cudaStream_t st = stream;
    if (nb > 1) st = ctx->aux[L.global_ring && pl.pool_serial ? 0 : (rr++ % nb)];
    void* gring = L.global_ring ? static_cast<void*>(reinterpret_cast<char*>(ctx->pool) + L.pool_off)
                                : nullptr;
    e = L.lane ? launch_lane(desc, sc, w, L, i, gring, st)
               : launch_queue(desc, sc, w, L, i, static_cast<int2*>(gring), st);
    if (e != cudaSuccess) {
      char buf[192];
      std::snprintf(buf, sizeof(buf),
                    "launch %d of %d (%s cls %d buckets %d..%d P %d R %d ring 2^%d %s grid %d): ", i,
                    pl.n_launch, L.lane ? "one-lane" : "group", L.cls, L.j_lo, L.j_hi, L.P, L.R,
                    L.rs_log2, L.global_ring ? "global" : "shared", L.grid);
      ctx->launch_error = buf;
    }
    ++dp;
  }
  if (e == cudaSuccess && nb > 1) {
    for (int b = 0; e == cudaSuccess && b < nb; ++b) {
      e = cudaEventRecord(ctx->join_ev[b], ctx->aux[b]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ctx->join_ev[b], 0);
    }
  }
  if (e == cudaSuccess && timed) {
    cudaEventRecord(ctx->ev[slot][1], stream);
    ctx->ev_pending = slot + 1;
  }
  *dp_out = dp;
  return e;
}

// A signature of a plan's launches (the graph of a call depends on it).
uint64_t plan_signature(const Plan& pl) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](int64_t v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (uint64_t)((v >> (8 * b)) & 0xFF);
      h *= 1099511628211ull;
    }
  };
  mix(pl.n_launch);
  for (int i = 0; i < pl.n_launch; ++i) {
    const Launch& L = pl.launch[i];
    mix(L.cls); mix(L.j_lo); mix(L.j_hi); mix(L.lane); mix(L.P); mix(L.R); mix(L.rs_log2);
    mix(L.global_ring); mix(L.slab); mix(L.grid); mix(L.mparam); mix((int64_t)L.pool_off);
  }
  mix(pl.pool_serial);
  for (int j = 0; j < kNumJ; ++j) mix(pl.jf.f[j]);
  return h;
}

// The first half of a call: checks, workspace, descriptor, and for the
// batched path the classify pass and the copy of its bucket counts.  The
// call's state waits in ctx->pending for run_finish.
xt_status run_begin(xt_ctx* ctx, bool plain, const uint8_t* q_seq, int64_t q_bytes,
                    const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                    int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                    const int32_t* h0, int32_t n, const xt_scoring* scr, xt_result* out,
                    int64_t* cells, cudaStream_t stream) {
  xt_status s = check_args(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n,
                           scr, out);
  if (s != XT_OK) return s;
  if (ctx->pending.active) return fail(ctx, XT_EBUSY, "a begun call has not been finished");
  PendingCall& pc = ctx->pending;
  pc = PendingCall();
  pc.n = n;
  if (n == 0) {
    pc.active = true;  // finish has nothing to do
    return XT_OK;
  }
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  pc.plain = plain;
  pc.scr = *scr;
  pc.sc = make_score(scr);
  pc.n_cap_log2 = 10;
  while ((1 << pc.n_cap_log2) < n) ++pc.n_cap_log2;
  pc.n_cap = pc.n_cap_log2 >= 31 ? INT32_MAX : (1 << pc.n_cap_log2);
  pc.has_cells = cells != nullptr;
  pc.stream = stream;
  s = get_work(ctx, pc.n_cap, &pc.w, &pc.desc);
  if (s != XT_OK) return s;
  ctx->match = scr->match;
  ctx->plan_small = false;
  // raw reads or 4-bit codes: an elementwise pass writes one base code per
  // byte into the context's workspace, and the call reads those
  s = ctx_codes(ctx, &q_seq, &q_bytes, &t_seq, &t_bytes, stream);
  if (s != XT_OK) return s;
  // this call's arguments go to the device descriptor through a one-thread
  // kernel (a kernel parameter, not a copy: a host-to-device copy here would
  // queue behind bulk copies of other streams)
  Batch hb;
  hb.q_seq = q_seq; hb.t_seq = t_seq; hb.q_off = q_off; hb.t_off = t_off; hb.q_len = q_len;
  hb.t_len = t_len; hb.h0 = h0; hb.q_bytes = q_bytes; hb.t_bytes = t_bytes; hb.n = n;
  hb.out = out; hb.cells = cells;
  e = launch_store_desc(pc.desc, hb, stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "descriptor");
  if (!plain) {
    // classify and order with count-independent bucket flags, then bring the
    // pair count of every (class, bucket) back for the plan
    batched_flags(ctx, pc.sc, n, &pc.jf, pc.lane_ok);
    e = enqueue_front(pc.jf, pc.sc, scr->match, pc.w, pc.desc, pc.n_cap, stream);
    const size_t seg_bytes =
        (size_t)((const char*)(pc.w.seg_end + kNumClasses * kNumJ) - (const char*)pc.w.seg_begin);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->seg_host, pc.w.seg_begin, seg_bytes, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->seg_ev, stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "classify");
  }
  pc.active = true;
  return XT_OK;
}

// The second half: plan from the counts (waiting for them if needed) and
// enqueue the extension kernels, through a captured graph when one exists.
xt_status run_finish(xt_ctx* ctx) {
  PendingCall& pc = ctx->pending;
  if (!pc.active) return fail(ctx, XT_EINVAL, "no begun call to finish");
  pc.active = false;
  if (pc.n == 0) return XT_OK;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  const bool plain = pc.plain;
  const Score& sc = pc.sc;
  const Work& w = pc.w;
  ctx->match = pc.scr.match;
  Plan pl;
  int plain_rs = 0;
  if (plain) {
    ctx->plan_small = false;
    plan_plain(ctx, sc, &pl, &plain_rs);
  } else {
    e = cudaEventSynchronize(ctx->seg_ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "classify");
    const int32_t* sb = ctx->seg_host;
    const int32_t* se = ctx->seg_host + (w.seg_end - w.seg_begin);
    int32_t cnt[kNumClasses][kNumJ];
    for (int c = 0; c < kNumClasses; ++c)
      for (int j = 0; j < kNumJ; ++j) cnt[c][j] = se[c * kNumJ + j] - sb[c * kNumJ + j];
    plan_counts(ctx, sc, cnt, pc.jf, pc.lane_ok, &pl);
    if (pl.bad) return fail(ctx, XT_ECUDA, "internal: inconsistent bucket plan");
  }
  const size_t want = layout_pool(ctx, &pl);
  if (want) {
    void* old = ctx->pool;
    xt_status s = dev_alloc(ctx, (void**)&ctx->pool, &ctx->pool_bytes, want);
    if (s != XT_OK) return s;
    if ((void*)ctx->pool != old) drop_graphs(ctx);
  }
  // the plain path's whole call, or the batched path's extension kernels,
  // replay as one graph once a call with the same key has been seen
  auto body = [&](cudaStream_t st, int* dp) -> cudaError_t {
    cudaError_t r = cudaSuccess;
    if (plain) r = enqueue_front(pl.jf, sc, pc.scr.match, w, pc.desc, pc.n_cap, st);
    if (r == cudaSuccess) r = enqueue_dp(ctx, plain, pl, plain_rs, sc, w, pc.desc, pc.n_cap, st, dp);
    return r;
  };
  int dp = 0;
  GraphEntry* ge = nullptr;
  if (ctx->graphs && !ctx->timing) {
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.plain = plain; key.sc = pc.scr; key.forced_P = ctx->forced_P; key.forced_R = ctx->forced_R;
    key.n_cap_log2 = pc.n_cap_log2; key.work = ctx->work; key.pool = ctx->pool;
    key.has_cells = pc.has_cells;
    key.plan_sig = plan_signature(pl);
    key.branches = ctx->branches;
    key.alphabet = ctx->alphabet;
    for (auto& g : ctx->graph_cache)
      if (g.key == key) ge = &g;
    if (!ge) {
      if (ctx->graph_cache.size() >= 64) drop_graphs(ctx);
      ctx->graph_cache.push_back(GraphEntry());
      ge = &ctx->graph_cache.back();
      ge->key = key;
    }
    ge->seen += 1;
    if (!ge->exec && ge->seen >= 2) {
      // capture once on a private stream; the graph reads every per-call
      // argument from the device descriptor
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e2 = body(ctx->cap_stream, &dp);
        e = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (e == cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ge->exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        // capture is an optimisation: on failure this and later calls launch directly
        cudaGetLastError();
        if (ge->exec) cudaGraphExecDestroy(ge->exec);
        ge->exec = nullptr;
        ctx->graphs = false;
        ctx->last_error = std::string("graph capture disabled: ") + cudaGetErrorString(e);
      }
    }
  }
  if (ge && ge->exec) {
    e = cudaGraphLaunch(ge->exec, pc.stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    dp = plain ? 1 + pl.n_launch : pl.n_launch;
  } else {
    ctx->launch_error.clear();
    e = body(pc.stream, &dp);
    if (e != cudaSuccess) return cuda_fail(ctx, e, ("launch " + ctx->launch_error).c_str());
  }
  ctx->calls += 1;
  ctx->launches += 4 + dp;  // descriptor, classify, scan, scatter + DP kernels
  ctx->dp_launches += dp;
  return XT_OK;
}

xt_status run(xt_ctx* ctx, bool plain, const uint8_t* q_seq, int64_t q_bytes, const int64_t* q_off,
              const int32_t* q_len, const uint8_t* t_seq, int64_t t_bytes, const int64_t* t_off,
              const int32_t* t_len, const int32_t* h0, int32_t n, const xt_scoring* scr,
              xt_result* out, int64_t* cells, cudaStream_t stream) {
  xt_status s = run_begin(ctx, plain, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len,
                          h0, n, scr, out, cells, stream);
  if (s != XT_OK) {
    if (s != XT_EBUSY) ctx->pending.active = false;
    return s;
  }
  return run_finish(ctx);
}

// Both-direction extension of seeds whose sequences are base codes (below).
xt_status seeds_codes(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes, const int64_t* q_off,
                      const int32_t* q_len, const uint8_t* t_seq, int64_t t_bytes,
                      const int64_t* t_off, const int32_t* t_len, const int32_t* q_beg,
                      const int32_t* t_beg, const int32_t* seed_len, const int32_t* h0,
                      int32_t n_pairs, const xt_scoring* sc, xt_result* left, xt_result* right,
                      int64_t* left_cells, int64_t* right_cells, cudaStream_t st);

}  // namespace

extern "C" {

xt_status xt_ctx_create(xt_ctx** out, int device, size_t mem_budget_bytes) {
  if (!out) return XT_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return XT_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) return XT_ECUDA;
  xt_ctx* c = new xt_ctx();
  c->device = device;
  c->budget = mem_budget_bytes;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  c->smem_optin = max_smem_per_block_optin(device);
  bool ok = true;
  ok = ok && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaHostAlloc((void**)&c->seg_host, 4 * kSegHostWords, cudaHostAllocDefault) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&c->seg_ev, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) == cudaSuccess;
  for (int b = 0; ok && b < kMaxBranches; ++b) {
    ok = cudaStreamCreateWithFlags(&c->aux[b], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->join_ev[b], cudaEventDisableTiming) == cudaSuccess;
  }
  ok = ok && cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
  for (auto& ev : c->stage_ev)
    ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    xt_ctx_destroy(c);
    return XT_ECUDA;
  }
  *out = c;
  return XT_OK;
}

xt_status xt_ctx_destroy(xt_ctx* ctx) {
  if (!ctx) return XT_EINVAL;
  for (auto*& c : ctx->chunk_ctx)
    if (c) {
      xt_ctx_destroy(c);
      c = nullptr;
    }
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->work) cudaFree(ctx->work);
  if (ctx->pool) cudaFree(ctx->pool);
  if (ctx->dev_in) cudaFree(ctx->dev_in);
  if (ctx->conv) cudaFree(ctx->conv);
  if (ctx->seed_ws) cudaFree(ctx->seed_ws);
  if (ctx->seed_rev) cudaFree(ctx->seed_rev);
  if (ctx->bwa_ws) cudaFree(ctx->bwa_ws);
  for (auto& pr : ctx->ev)
    for (auto& e : pr)
      if (e) cudaEventDestroy(e);
  drop_graphs(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->seg_host) cudaFreeHost(ctx->seg_host);
  if (ctx->seg_ev) cudaEventDestroy(ctx->seg_ev);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  for (auto& ev : ctx->stage_ev)
    if (ev) cudaEventDestroy(ev);
  for (int b = 0; b < kMaxBranches; ++b) {
    if (ctx->aux[b]) cudaStreamDestroy(ctx->aux[b]);
    if (ctx->join_ev[b]) cudaEventDestroy(ctx->join_ev[b]);
  }
  delete ctx;
  return XT_OK;
}

xt_status xt_ctx_sync(xt_ctx* ctx, void* stream) {
  if (!ctx) return XT_EINVAL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  return XT_OK;
}

xt_status xt_extend_batch(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes,
                          const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                          int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                          const int32_t* h0, int32_t n_pairs, const xt_scoring* sc,
                          xt_result* out, int64_t* cells_out, void* stream) {
  if (!ctx) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  return run(ctx, false, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n_pairs,
             sc, out, cells_out, (cudaStream_t)stream);
}

xt_status xt_extend_batch_begin(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes,
                                const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                                int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                                const int32_t* h0, int32_t n_pairs, const xt_scoring* sc,
                                xt_result* out, int64_t* cells_out, void* stream) {
  if (!ctx) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  const xt_status s = run_begin(ctx, false, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off,
                                t_len, h0, n_pairs, sc, out, cells_out, (cudaStream_t)stream);
  if (s != XT_OK && s != XT_EBUSY) ctx->pending.active = false;
  return s;
}

xt_status xt_extend_batch_ready(xt_ctx* ctx, int* ready) {
  if (!ctx || !ready) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->pending.active) return fail(ctx, XT_EINVAL, "no begun call");
  if (ctx->pending.n == 0 || ctx->pending.plain) {
    *ready = 1;
    return XT_OK;
  }
  const cudaError_t e = cudaEventQuery(ctx->seg_ev);
  if (e == cudaErrorNotReady) {
    *ready = 0;
    return XT_OK;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "classify");
  *ready = 1;
  return XT_OK;
}

xt_status xt_extend_batch_finish(xt_ctx* ctx) {
  if (!ctx) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  return run_finish(ctx);
}

xt_status xt_extend_batch_plain(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes,
                                const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                                int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                                const int32_t* h0, int32_t n_pairs, const xt_scoring* sc,
                                xt_result* out, int64_t* cells_out, void* stream) {
  if (!ctx) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  return run(ctx, true, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n_pairs,
             sc, out, cells_out, (cudaStream_t)stream);
}

xt_status xt_extend_seeds(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes, const int64_t* q_off,
                          const int32_t* q_len, const uint8_t* t_seq, int64_t t_bytes,
                          const int64_t* t_off, const int32_t* t_len, const int32_t* q_beg,
                          const int32_t* t_beg, const int32_t* seed_len, const int32_t* h0,
                          int32_t n_pairs, const xt_scoring* sc, xt_result* left,
                          xt_result* right, int64_t* left_cells, int64_t* right_cells,
                          void* stream) {
  if (!ctx) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  xt_status s = check_args(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0,
                           n_pairs, sc, left);
  if (s != XT_OK) return s;
  if (n_pairs > 0 && (!q_beg || !t_beg || !seed_len || !right))
    return fail(ctx, XT_EINVAL, "null array");
  if (ctx->pending.active) return fail(ctx, XT_EBUSY, "a begun call has not been finished");
  if (n_pairs == 0) return XT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, XT_ECUDA, "cudaSetDevice");
  // 4-bit codes are unpacked first: the reversed prefixes are copied base by
  // base, and both sides then read one code per byte
  if (ctx->alphabet == XT_ALPHABET_PACKED4) {
    s = ctx_codes(ctx, &q_seq, &q_bytes, &t_seq, &t_bytes, st);
    if (s != XT_OK) return s;
    ctx->alphabet = XT_ALPHABET_CODES;
    s = seeds_codes(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, q_beg, t_beg,
                    seed_len, h0, n_pairs, sc, left, right, left_cells, right_cells, st);
    ctx->alphabet = XT_ALPHABET_PACKED4;
    return s;
  }
  return seeds_codes(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, q_beg, t_beg,
                     seed_len, h0, n_pairs, sc, left, right, left_cells, right_cells, st);
}

}  // extern "C"

namespace {

// Both-direction extension of checked, non-empty seed batches (the caller
// holds the context's lock).
xt_status seeds_codes(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes, const int64_t* q_off,
                      const int32_t* q_len, const uint8_t* t_seq, int64_t t_bytes,
                      const int64_t* t_off, const int32_t* t_len, const int32_t* q_beg,
                      const int32_t* t_beg, const int32_t* seed_len, const int32_t* h0,
                      int32_t n_pairs, const xt_scoring* sc, xt_result* left, xt_result* right,
                      int64_t* left_cells, int64_t* right_cells, cudaStream_t st) {
  xt_status s = XT_OK;
  // workspace: per-seed arrays and the block sums
  const size_t n = (size_t)n_pairs;
  const size_t nb = (n + 1023) / 1024;
  size_t off = 0;
  const size_t o_lql = off; off = align_up(off + 4 * n);
  const size_t o_ltl = off; off = align_up(off + 4 * n);
  const size_t o_lqo = off; off = align_up(off + 8 * n);
  const size_t o_lto = off; off = align_up(off + 8 * n);
  const size_t o_rql = off; off = align_up(off + 4 * n);
  const size_t o_rtl = off; off = align_up(off + 4 * n);
  const size_t o_rqo = off; off = align_up(off + 8 * n);
  const size_t o_rto = off; off = align_up(off + 8 * n);
  const size_t o_rh0 = off; off = align_up(off + 4 * n);
  const size_t o_bq = off; off = align_up(off + 8 * nb);
  const size_t o_bt = off; off = align_up(off + 8 * nb);
  const size_t o_tot = off; off = align_up(off + 16);
  s = dev_alloc(ctx, &ctx->seed_ws, &ctx->seed_ws_bytes, off);
  if (s != XT_OK) return s;
  char* d = static_cast<char*>(ctx->seed_ws);
  SeedWork sw;
  sw.lq_len = (int32_t*)(d + o_lql); sw.lt_len = (int32_t*)(d + o_ltl);
  sw.lq_off = (int64_t*)(d + o_lqo); sw.lt_off = (int64_t*)(d + o_lto);
  sw.rq_len = (int32_t*)(d + o_rql); sw.rt_len = (int32_t*)(d + o_rtl);
  sw.rq_off = (int64_t*)(d + o_rqo); sw.rt_off = (int64_t*)(d + o_rto);
  sw.rh0 = (int32_t*)(d + o_rh0);
  sw.block_q = (int64_t*)(d + o_bq); sw.block_t = (int64_t*)(d + o_bt);
  sw.totals = (int64_t*)(d + o_tot);
  sw.rev_q = sw.rev_t = nullptr;
  // lengths and the prefix sums up to their totals, which size the copies
  cudaError_t e = launch_seed_front(n_pairs, q_len, t_len, q_off, t_off, q_bytes, t_bytes, q_beg,
                                    t_beg, seed_len, sw, st);
  int64_t* tot_host = reinterpret_cast<int64_t*>(ctx->seg_host + kSegHostSeedTotals);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tot_host, sw.totals, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->seg_ev, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(ctx->seg_ev);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "seed layout");
  const int64_t tq = tot_host[0], tt = tot_host[1];
  const size_t qa = align_up((size_t)tq);
  s = dev_alloc(ctx, &ctx->seed_rev, &ctx->seed_rev_bytes, qa + align_up((size_t)tt) + kAlign);
  if (s != XT_OK) return s;
  sw.rev_q = static_cast<uint8_t*>(ctx->seed_rev);
  sw.rev_t = sw.rev_q + qa;
  e = launch_seed_reverse(n_pairs, q_seq, q_off, t_seq, t_off, sw, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "seed prefixes");
  // left: the reversed prefixes from the seed's score
  s = run(ctx, false, sw.rev_q, tq, sw.lq_off, sw.lq_len, sw.rev_t, tt, sw.lt_off, sw.lt_len, h0,
          n_pairs, sc, left, left_cells, st);
  if (s != XT_OK) return s;
  // right: the suffixes from the left side's best
  e = launch_seed_right_h0(n_pairs, h0, left, sw, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "seed right scores");
  return run(ctx, false, q_seq, q_bytes, sw.rq_off, sw.rq_len, t_seq, t_bytes, sw.rt_off,
             sw.rt_len, sw.rh0, n_pairs, sc, right, right_cells, st);
}

}  // namespace

extern "C" {

namespace {

// The two chunk contexts of ctx, created on first use, with ctx's schedule
// settings; they read base codes.
xt_status chunk_contexts(xt_ctx* ctx) {
  for (auto*& c : ctx->chunk_ctx) {
    if (!c) {
      xt_status s = xt_ctx_create(&c, ctx->device, 0);
      if (s != XT_OK) {
        c = nullptr;
        return fail(ctx, s, "chunk context");
      }
    }
    c->tuning = ctx->tuning;
    c->forced_P = ctx->forced_P;
    c->forced_R = ctx->forced_R;
    c->branches = ctx->branches;
    c->graphs = ctx->graphs;
    c->alphabet = XT_ALPHABET_CODES;
  }
  return XT_OK;
}

}  // namespace

xt_status xt_extend_batch_host(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes,
                               const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                               int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                               const int32_t* h0, int32_t n_pairs, const xt_scoring* sc,
                               xt_result* out, int64_t* cells_out, void* stream) {
  if (!ctx) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  xt_status s = check_args(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0,
                           n_pairs, sc, out);
  if (s != XT_OK) return s;
  if (ctx->pending.active) return fail(ctx, XT_EBUSY, "a begun call has not been finished");
  if (n_pairs == 0) return XT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, XT_ECUDA, "cudaSetDevice");
  const size_t n = (size_t)n_pairs;
  // 4-bit codes arrive packed (half the bytes of base codes) and are unpacked
  // on the device, chunk by chunk below
  const bool packed = ctx->alphabet == XT_ALPHABET_PACKED4;
  const int64_t qn = packed ? 2 * q_bytes : q_bytes, tn = packed ? 2 * t_bytes : t_bytes;
  size_t off = 0;
  const size_t o_q = off; off = align_up(off + (size_t)q_bytes);
  const size_t o_t = off; off = align_up(off + (size_t)t_bytes);
  const size_t o_qc = off; off = align_up(off + (packed ? (size_t)qn : 0));
  const size_t o_tc = off; off = align_up(off + (packed ? (size_t)tn : 0));
  const size_t o_qo = off; off = align_up(off + 8 * n);
  const size_t o_to = off; off = align_up(off + 8 * n);
  const size_t o_ql = off; off = align_up(off + 4 * n);
  const size_t o_tl = off; off = align_up(off + 4 * n);
  const size_t o_h0 = off; off = align_up(off + 4 * n);
  const size_t o_out = off; off = align_up(off + sizeof(xt_result) * n);
  const size_t o_cells = off; off = align_up(off + 8 * n);
  const size_t o_ends = off; off = align_up(off + 16 * kMaxChunks);
  s = dev_alloc(ctx, &ctx->dev_in, &ctx->dev_in_bytes, off);
  if (s != XT_OK) return s;
  char* d = (char*)ctx->dev_in;
  const int64_t* dqo = (const int64_t*)(d + o_qo);
  const int64_t* dto = (const int64_t*)(d + o_to);
  const int32_t* dql = (const int32_t*)(d + o_ql);
  const int32_t* dtl = (const int32_t*)(d + o_tl);
  const int32_t* dh0 = (const int32_t*)(d + o_h0);
  xt_result* dout = (xt_result*)(d + o_out);
  int64_t* dcells = cells_out ? (int64_t*)(d + o_cells) : nullptr;
  unsigned long long* dends = (unsigned long long*)(d + o_ends);
  cudaError_t e = cudaSuccess;
  auto h2d = [&](size_t o, const void* src, size_t bytes, cudaStream_t on) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(d + o, src, bytes, cudaMemcpyHostToDevice, on);
  };
  // many pairs: chunks of at least kChunkPairs pairs, each extended as soon as
  // the sequence bytes it reads are on the device, while the copy stream
  // brings the next chunk's bytes and takes the finished chunks' results back
  // chunk sizes double: the first chunk is small, so the extension starts
  // early, and each later chunk's bytes (copied about 2.5x faster than they
  // are extended) arrive while the chunk before it extends
  ChunkStarts cb{};
  cb.count = 1;
  if (ctx->alphabet != XT_ALPHABET_ASCII && n_pairs >= 2 * (int64_t)kChunkPairs) {
    int m = 2;
    while (m < kMaxChunks && (int64_t)n_pairs / ((2 << m) - 1) >= kChunkFirstMin) ++m;
    const int64_t unit = ((int64_t)n_pairs + (1 << m) - 2) / ((1 << m) - 1);
    int64_t p = 0;
    cb.count = 0;
    for (int k = 0; k < m && p < n_pairs; ++k) {
      cb.start[cb.count++] = (int32_t)p;
      p = std::min<int64_t>(n_pairs, (p + (unit << k) + 255) / 256 * 256);
    }
  }
  const int chunks = cb.count;
  if (chunks <= 1) {
    h2d(o_q, q_seq, (size_t)q_bytes, st);
    h2d(o_t, t_seq, (size_t)t_bytes, st);
    h2d(o_qo, q_off, 8 * n, st);
    h2d(o_to, t_off, 8 * n, st);
    h2d(o_ql, q_len, 4 * n, st);
    h2d(o_tl, t_len, 4 * n, st);
    h2d(o_h0, h0, 4 * n, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "host to device copy");
    s = run(ctx, false, (const uint8_t*)(d + o_q), q_bytes, dqo, dql, (const uint8_t*)(d + o_t),
            t_bytes, dto, dtl, dh0, n_pairs, sc, dout, dcells, st);
    if (s != XT_OK) return s;
    e = cudaMemcpyAsync(out, dout, sizeof(xt_result) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && cells_out)
      e = cudaMemcpyAsync(cells_out, dcells, 8 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device to host copy");
    return XT_OK;
  }
  cudaStream_t cs = ctx->copy_stream;
  cudaEvent_t* ev = ctx->stage_ev;  // [0]: start, [1]: metadata, [2+k]: chunk k's bytes,
                                    // [2+chunks+k]: chunk k extended
  e = cudaEventRecord(ev[0], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[0], 0);
  h2d(o_qo, q_off, 8 * n, cs);
  h2d(o_to, t_off, 8 * n, cs);
  h2d(o_ql, q_len, 4 * n, cs);
  h2d(o_tl, t_len, 4 * n, cs);
  h2d(o_h0, h0, 4 * n, cs);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[1], 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(dends, 0, 16 * kMaxChunks, st);
  if (e == cudaSuccess)
    e = launch_chunk_ends(dqo, dql, dto, dtl, n_pairs, cb, qn, tn, dends, st);
  unsigned long long* ends = reinterpret_cast<unsigned long long*>(ctx->seg_host + kSegHostChunkEnds);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ends, dends, 16 * kMaxChunks, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->seg_ev, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(ctx->seg_ev);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "chunk layout");
  // chunk k needs every byte below the furthest end of chunks 0..k
  int64_t need_q[kMaxChunks], need_t[kMaxChunks];
  for (int k = 0; k < chunks; ++k) {
    need_q[k] = std::max<int64_t>(k ? need_q[k - 1] : 0, (int64_t)ends[2 * k]);
    need_t[k] = std::max<int64_t>(k ? need_t[k - 1] : 0, (int64_t)ends[2 * k + 1]);
  }
  // bases [0, need) of a buffer are its bytes [0, need) as codes, or
  // [0, ceil(need / 2)) when packed; a packed chunk is unpacked on the copy
  // stream as soon as its bytes are there
  auto bytes_of = [&](int64_t bases) { return packed ? (bases + 1) / 2 : bases; };
  for (int k = 0; k < chunks && e == cudaSuccess; ++k) {
    const int64_t q0 = k ? bytes_of(need_q[k - 1]) : 0, t0 = k ? bytes_of(need_t[k - 1]) : 0;
    const int64_t q1 = bytes_of(need_q[k]), t1 = bytes_of(need_t[k]);
    h2d(o_q + (size_t)q0, q_seq + q0, (size_t)(q1 - q0), cs);
    h2d(o_t + (size_t)t0, t_seq + t0, (size_t)(t1 - t0), cs);
    if (packed && e == cudaSuccess) {
      e = launch_unpack4((const uint8_t*)(d + o_q), (uint8_t*)(d + o_qc), q0, q1, ctx->num_sms, cs);
      if (e == cudaSuccess)
        e = launch_unpack4((const uint8_t*)(d + o_t), (uint8_t*)(d + o_tc), t0, t1, ctx->num_sms,
                           cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 + k], cs);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host to device copy");
  // the chunks read the unpacked codes (the context's alphabet is codes for them)
  const uint8_t* cq = (const uint8_t*)(d + (packed ? o_qc : o_q));
  const uint8_t* ct = (const uint8_t*)(d + (packed ? o_tc : o_t));
  // Without a memory budget the chunks alternate between two contexts of
  // their own (workspace, ring pool, streams): chunk k classifies as soon as
  // the metadata is on the device, and its extension kernels wait only for
  // its own bytes, so they take the slots that chunk k-1's kernels leave as
  // they drain.  Chunk k+2 reuses chunk k's context after it in stream order.
  const bool apart = ctx->budget == 0 && !ctx->timing;
  if (apart) {
    s = chunk_contexts(ctx);
    if (s != XT_OK) {
      cudaStreamSynchronize(cs);
      cudaStreamSynchronize(st);
      return s;
    }
  }
  auto sync_all = [&]() {
    cudaStreamSynchronize(cs);
    cudaStreamSynchronize(st);
    if (apart)
      for (auto* c : ctx->chunk_ctx) cudaStreamSynchronize(c->copy_stream);
  };
  const int alphabet = ctx->alphabet;
  ctx->alphabet = XT_ALPHABET_CODES;
  for (int k = 0; k < chunks; ++k) {
    const int32_t p0 = cb.start[k];
    const int32_t p1 = k + 1 < chunks ? cb.start[k + 1] : n_pairs;
    if (p1 <= p0) continue;
    xt_ctx* cc = apart ? ctx->chunk_ctx[k & 1] : ctx;
    cudaStream_t cst = apart ? cc->copy_stream : st;
    if (apart) {
      e = cudaStreamWaitEvent(cst, ev[1], 0);
      if (e != cudaSuccess) break;
      s = run_begin(cc, false, cq, qn, dqo + p0, dql + p0, ct, tn, dto + p0, dtl + p0, dh0 + p0,
                    p1 - p0, sc, dout + p0, dcells ? dcells + p0 : nullptr, cst);
      if (s == XT_OK) {
        e = cudaStreamWaitEvent(cst, ev[2 + k], 0);
        s = e == cudaSuccess ? run_finish(cc) : cuda_fail(cc, e, "chunk bytes");
      }
      if (s != XT_OK) {
        cc->pending.active = false;
        ctx->last_error = cc->last_error;
      }
    } else {
      e = cudaStreamWaitEvent(st, ev[2 + k], 0);
      if (e != cudaSuccess) break;
      s = run(ctx, false, cq, qn, dqo + p0, dql + p0, ct, tn, dto + p0, dtl + p0, dh0 + p0,
              p1 - p0, sc, dout + p0, dcells ? dcells + p0 : nullptr, st);
    }
    if (s != XT_OK) {
      ctx->alphabet = alphabet;
      sync_all();
      return s;
    }
    e = cudaEventRecord(ev[2 + chunks + k], cst);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[2 + chunks + k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out + p0, dout + p0, sizeof(xt_result) * (size_t)(p1 - p0),
                          cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess && cells_out)
      e = cudaMemcpyAsync(cells_out + p0, dcells + p0, 8 * (size_t)(p1 - p0),
                          cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) break;
  }
  ctx->alphabet = alphabet;
  cudaError_t e2 = cudaStreamSynchronize(cs);
  if (e == cudaSuccess) e = e2;
  e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  if (apart)
    for (auto* c : ctx->chunk_ctx) {
      e2 = cudaStreamSynchronize(c->copy_stream);
      if (e == cudaSuccess) e = e2;
    }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "chunked host call");
  return XT_OK;
}

xt_status xt_ctx_set_graphs(xt_ctx* ctx, int enable) {
  if (!ctx) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->graphs = enable != 0;
  return XT_OK;
}

xt_status xt_ctx_set_bucket_schedule(xt_ctx* ctx, int w, int j, int P, int R) {
  xt_status s = xt_ctx_set_bucket_schedule_for(ctx, w, j, XT_BATCH_LARGE, P, R);
  if (s == XT_OK) s = xt_ctx_set_bucket_schedule_for(ctx, w, j, XT_BATCH_SMALL, P, R);
  return s;
}

xt_status xt_ctx_set_bucket_schedule_for(xt_ctx* ctx, int w, int j, int batch_class, int P,
                                         int R) {
  if (!ctx || w < 0 || j < kJMin || j > kJMax) return XT_EINVAL;
  if (batch_class != XT_BATCH_LARGE && batch_class != XT_BATCH_SMALL) return XT_EINVAL;
  const int wc = w > 2 * XT_MAX_LEN ? 2 * XT_MAX_LEN : w;  // the band the plan sees
  if (P != 0 && !bucket_sched_ok(ctx, wc, j, P, R))
    return fail(ctx, XT_EINVAL, "schedule not available for this bucket and band");
  std::lock_guard<std::mutex> lk(ctx->mu);
  TuneEntry* e = nullptr;
  for (auto& t : ctx->tuning)
    if (t.w == wc) e = &t;
  if (!e) {
    ctx->tuning.push_back(TuneEntry());
    e = &ctx->tuning.back();
    e->w = wc;
  }
  BucketSched& b = batch_class == XT_BATCH_SMALL ? e->small[j] : e->b[j];
  b.P = P;
  b.R = P ? R : 0;
  drop_graphs(ctx);
  return XT_OK;
}

xt_status xt_ctx_get_bucket_schedule(xt_ctx* ctx, int w, int j, int* P, int* R) {
  return xt_ctx_get_bucket_schedule_for(ctx, w, j, XT_BATCH_LARGE, P, R);
}

xt_status xt_ctx_get_bucket_schedule_for(xt_ctx* ctx, int w, int j, int batch_class, int* P,
                                         int* R) {
  if (!ctx || !P || !R || w < 0 || j < kJMin || j > kJMax) return XT_EINVAL;
  if (batch_class != XT_BATCH_LARGE && batch_class != XT_BATCH_SMALL) return XT_EINVAL;
  const int wc = w > 2 * XT_MAX_LEN ? 2 * XT_MAX_LEN : w;
  std::lock_guard<std::mutex> lk(ctx->mu);
  *P = 0;
  *R = 0;
  for (auto& t : ctx->tuning)
    if (t.w == wc) {
      const BucketSched& b = batch_class == XT_BATCH_SMALL ? t.small[j] : t.b[j];
      *P = b.P;
      *R = b.R;
    }
  return XT_OK;
}

xt_status xt_ctx_set_alphabet(xt_ctx* ctx, int alphabet) {
  if (!ctx || (alphabet != XT_ALPHABET_CODES && alphabet != XT_ALPHABET_ASCII &&
               alphabet != XT_ALPHABET_PACKED4))
    return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->alphabet = alphabet;
  return XT_OK;
}

xt_status xt_ctx_set_streams(xt_ctx* ctx, int branches) {
  if (!ctx || branches < 1 || branches > kMaxBranches) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->branches != branches) drop_graphs(ctx);
  ctx->branches = branches;
  return XT_OK;
}

xt_status xt_ctx_set_timing(xt_ctx* ctx, int enable) {
  if (!ctx) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->timing = enable != 0;
  return XT_OK;
}

xt_status xt_ctx_stats(xt_ctx* ctx, xt_stats* out) {
  if (!ctx || !out) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  double ms = 0;
  for (int i = 0; i < ctx->ev_pending; ++i) {
    cudaError_t e = cudaEventSynchronize(ctx->ev[i][1]);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ctx->ev[i][0], ctx->ev[i][1]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event timing");
    ms += t;
  }
  for (auto* c : ctx->chunk_ctx)
    if (c) {
      ctx->calls += c->calls;
      ctx->launches += c->launches;
      ctx->dp_launches += c->dp_launches;
      c->calls = c->launches = c->dp_launches = 0;
    }
  out->calls = ctx->calls;
  out->launches = ctx->launches;
  out->dp_launches = ctx->dp_launches;
  out->timed_calls = ctx->ev_pending;
  out->dp_ms = ms;
  ctx->calls = ctx->launches = ctx->dp_launches = 0;
  ctx->ev_pending = 0;
  return XT_OK;
}

xt_status xt_ctx_set_schedule(xt_ctx* ctx, int P, int R) {
  if (!ctx) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (P == 0) {
    ctx->forced_P = ctx->forced_R = 0;
    return XT_OK;
  }
  const bool p_ok = P == 1 || P == 2 || P == 4 || P == 8 || P == 16 || P == 32;
  const bool r_ok = R == 4 || R == 8 || (R == 16 && P <= 4);
  if (!p_ok || !r_ok) return fail(ctx, XT_EINVAL, "unsupported schedule");
  ctx->forced_P = P;
  ctx->forced_R = R;
  return XT_OK;
}

xt_status xt_scoring_check(const xt_scoring* sc) { return scoring_ok(sc) ? XT_OK : XT_EINVAL; }

const char* xt_status_str(xt_status s) {
  switch (s) {
    case XT_OK: return "XT_OK";
    case XT_EINVAL: return "XT_EINVAL";
    case XT_ENOMEM: return "XT_ENOMEM";
    case XT_ECUDA: return "XT_ECUDA";
    case XT_ETIMEOUT: return "XT_ETIMEOUT";
    case XT_EBUSY: return "XT_EBUSY";
  }
  return "XT_UNKNOWN";
}

const char* xt_ctx_last_error(const xt_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "";
}

}  // extern "C"

// ------------------------------------------------------------------------
// Allocation-free batched extension (xt_extend_batch_static).
//
// The scratch the batched path needs -- one class byte and one int32 queue
// slot per pair, bucket counters and cursors, the segment table, the queue
// heads and the per-bucket flags -- is carved from this one fixed device
// array instead of the context's workspace.  Host code only ever sees the
// symbol as a host-side stand-in; the kernels get its device address, looked
// up once per device below.
static __device__ __align__(256) unsigned char g_static_scratch[XT_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on
// the first call for that device and kept for the life of the process; a
// cudaDeviceReset of that device invalidates it, see include/xt.h).
cudaError_t static_scratch(int device, void** ptr) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[device] = p;
  }
  *ptr = g_static_ptr[device];
  return cudaSuccess;
}

// Carve the Work tables for n pairs out of the scratch array; false if they
// do not fit.
bool carve_static(void* base_ptr, int32_t n, Work* w, Batch** desc) {
  size_t off = 0;
  const size_t o_desc = off; off = align_up(off + sizeof(Batch));
  const size_t o_pclass = off; off = align_up(off + (size_t)n);
  const size_t o_order = off; off = align_up(off + 4 * (size_t)n);
  const size_t o_counts = off; off = align_up(off + 4 * (size_t)kNumBuckets);
  const size_t o_cursor = off; off = align_up(off + 4 * (size_t)kNumBuckets);
  const size_t o_sb = off; off = align_up(off + 4 * (size_t)(kNumClasses * kNumJ));
  const size_t o_se = off; off = align_up(off + 4 * (size_t)(kNumClasses * kNumJ));
  const size_t o_heads = off; off = align_up(off + 4 * (size_t)kMaxLaunches);
  if (off > XT_STATIC_SCRATCH_BYTES) return false;
  char* base = (char*)base_ptr;
  w->pclass = (uint8_t*)(base + o_pclass);
  w->order = (int32_t*)(base + o_order);
  w->counts = (int32_t*)(base + o_counts);
  w->cursor = (int32_t*)(base + o_cursor);
  w->seg_begin = (int32_t*)(base + o_sb);
  w->seg_end = (int32_t*)(base + o_se);
  w->heads = (int32_t*)(base + o_heads);
  *desc = (Batch*)(base + o_desc);
  return true;
}

}  // namespace

extern "C" xt_status xt_extend_batch_static(const uint8_t* q_seq, int64_t q_bytes,
                                            const int64_t* q_off, const int32_t* q_len,
                                            const uint8_t* t_seq, int64_t t_bytes,
                                            const int64_t* t_off, const int32_t* t_len,
                                            const int32_t* h0, int32_t n_pairs,
                                            const xt_scoring* scr, xt_result* out,
                                            int64_t* cells_out, void* stream) {
  // A host-side context object only: it holds the launch plan's inputs and
  // allocates nothing.
  xt_ctx host;
  xt_status s = check_args(&host, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0,
                           n_pairs, scr, out);
  if (s != XT_OK) return s;
  if (n_pairs > XT_STATIC_MAX_PAIRS) return XT_EINVAL;
  if (n_pairs == 0) return XT_OK;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kStaticMaxDevices)
    return XT_ECUDA;
  host.device = device;
  if (cudaDeviceGetAttribute(&host.num_sms, cudaDevAttrMultiProcessorCount, device) !=
      cudaSuccess)
    return XT_ECUDA;
  host.smem_optin = max_smem_per_block_optin(device);
  const Score sc = make_score(scr);
  Plan pl;
  host.match = scr->match;
  plan_batched(&host, sc, &pl, /*allow_gring=*/false);
  if (pl.any_huge) return XT_EINVAL;  // band too wide for shared-memory rings
  void* base = nullptr;
  if (static_scratch(device, &base) != cudaSuccess) return XT_ECUDA;
  Work w;
  Batch* desc = nullptr;
  if (!carve_static(base, n_pairs, &w, &desc)) return XT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Batch b;
  b.q_seq = q_seq; b.t_seq = t_seq; b.q_off = q_off; b.t_off = t_off; b.q_len = q_len;
  b.t_len = t_len; b.h0 = h0; b.q_bytes = q_bytes; b.t_bytes = t_bytes; b.n = n_pairs; b.out = out;
  b.cells = cells_out;
  // the descriptor travels to its device slot as a kernel parameter: no
  // host buffer has to outlive the call, and no copy waits behind bulk
  // copies that other streams queued on the copy engine
  cudaError_t e = launch_store_desc(desc, b, st);
  // counters and queue heads start at zero on every call; the bucket flags
  // are rewritten; everything else is written before it is read
  if (e == cudaSuccess) e = cudaMemsetAsync(w.counts, 0, 4 * (size_t)kNumBuckets, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.heads, 0, 4 * (size_t)kMaxLaunches, st);
  if (e == cudaSuccess) e = launch_classify(desc, n_pairs, sc, scr->match, pl.jf, w, st);
  if (e == cudaSuccess) e = launch_order(desc, n_pairs, w, st);
  for (int i = 0; e == cudaSuccess && i < pl.n_launch; ++i) {
    const Launch& L = pl.launch[i];
    e = L.lane ? launch_lane(desc, sc, w, L, i, nullptr, st)
               : launch_queue(desc, sc, w, L, i, nullptr, st);
  }
  return e == cudaSuccess ? XT_OK : XT_ECUDA;
}
