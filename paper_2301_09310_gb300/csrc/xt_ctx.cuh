// xt_ctx.cuh -- the library context (xt_ctx of include/xt.h) and the
// per-bucket schedule table, shared by the API and the autotuner.
#pragma once
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "xt.h"
#include "xt_kernels.cuh"

namespace xt {

// A captured call: same scoring, schedule, capacity class and workspace.
struct GraphKey {
  int plain;
  xt_scoring sc;
  int forced_P, forced_R;
  int n_cap_log2;
  void* work;
  void* pool;
  bool has_cells;
  uint64_t plan_sig;   // the plan of the extension kernels (count-aware)
  int branches;
  int alphabet;
  bool operator==(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};
struct GraphEntry {
  GraphKey key;
  int seen = 0;                   // calls with this key (captured on the second)
  cudaGraphExec_t exec = nullptr;
};
constexpr int kMaxBranches = 8;  // streams the DP launches of one call fork onto

// Schedule of one length bucket: P lanes per pair (1: the one-lane engine),
// R rows per lane.  P = 0: the built-in rule.
struct BucketSched {
  int P = 0, R = 0;
};
// The schedules of every bucket for calls whose band is w: one set for
// buckets that fill the GPU (tuned at saturation) and one for buckets of
// fewer than XT_SMALL_BUCKET pairs in a call (tuned on small trials: there a
// pair's latency on its engine, not the engine's throughput, decides).
struct TuneEntry {
  int w = 0;
  BucketSched b[kNumJ];
  BucketSched small[kNumJ];
};

// Whether (P, R) is an instantiated schedule whose ring fits for bucket j
// under band w on this context's device.
bool bucket_sched_ok(const struct ::xt_ctx* ctx, int w, int j, int P, int R);
// The context's pinned read-back area (int32 words): the bucket counts of a
// batched call first, then the small values other calls bring back.
constexpr int kSegHostWords = 1024;
constexpr int kSegHostSeedTotals = 512;  // xt_extend_seeds: 2 x int64
constexpr int kSegHostBwaCounts = 640;   // xt_extend_batch_bwa: class sizes
constexpr int kSegHostChunkEnds = 768;   // xt_extend_batch_host: 2 x kMaxChunks x uint64
// Drop every captured graph of the context.
void drop_graphs(struct ::xt_ctx* ctx);
// Record an error message on the context and return s (or XT_ECUDA for e).
xt_status ctx_fail(struct ::xt_ctx* ctx, xt_status s, const char* msg);
xt_status ctx_cuda_fail(struct ::xt_ctx* ctx, cudaError_t e, const char* where);
// Grow *p (holding *have bytes) to at least `want` bytes within the budget.
xt_status ctx_alloc(struct ::xt_ctx* ctx, void** p, size_t* have, size_t want);
// Size the workspace, the ring pool (to pool_bytes) and (conv_bytes > 0) the
// conversion buffer for calls of up to n_pairs pairs once (see xt_api.cu).
xt_status ctx_reserve(struct ::xt_ctx* ctx, int32_t n_pairs, size_t conv_bytes, size_t pool_bytes);
// With the ASCII or the 4-bit alphabet, convert both sequence buffers to one
// base code per byte in the context's workspace, point *q_seq / *t_seq at
// them and set *q_bytes / *t_bytes to their sizes in bases (no-op for codes).
xt_status ctx_codes(struct ::xt_ctx* ctx, const uint8_t** q_seq, int64_t* q_bytes,
                    const uint8_t** t_seq, int64_t* t_bytes, cudaStream_t stream);

// Host-buffer calls of many pairs run in chunks of pairs whose sequence
// bytes are copied while earlier chunks extend (xt_extend_batch_host).
constexpr int kMaxChunks = 8;
// the read-back regions do not overlap (bucket counts: two aligned tables)
static_assert(2 * (4 * kNumClasses * kNumJ + 255) / 4 <= kSegHostSeedTotals, "bucket counts");
static_assert(kSegHostSeedTotals + 4 <= kSegHostBwaCounts, "seed totals");
static_assert(kSegHostBwaCounts + 16 <= kSegHostChunkEnds, "BWA class sizes");
static_assert(kSegHostChunkEnds + 4 * kMaxChunks <= kSegHostWords, "chunk ends");
constexpr int32_t kChunkPairs = 1 << 20;   // calls of 2 x this many pairs or more are chunked
constexpr int32_t kChunkFirstMin = 1 << 18; // pairs in the first (smallest) chunk at least
// First pair of each chunk of a host-buffer call (multiples of 256).
struct ChunkStarts {
  int32_t start[kMaxChunks];
  int32_t count;
};
// ends[2k], ends[2k+1]: how far chunk k's pairs read into the query and the
// target buffer (see xt_stage.cu); ends must be zeroed first.
// Store a call's batch descriptor into device memory (one thread; the
// descriptor travels as a kernel parameter).
cudaError_t launch_store_desc(Batch* dst, const Batch& b, cudaStream_t stream);
cudaError_t launch_chunk_ends(const int64_t* q_off, const int32_t* q_len, const int64_t* t_off,
                              const int32_t* t_len, int32_t n, const ChunkStarts& cb,
                              int64_t q_bytes, int64_t t_bytes, unsigned long long* ends,
                              cudaStream_t stream);

// A call between its classify pass and its extension kernels.
struct PendingCall {
  bool active = false;
  bool plain = false;
  int32_t n = 0;
  xt_scoring scr{};
  Score sc{};
  Work w{};
  Batch* desc = nullptr;
  int32_t n_cap = 0;
  int n_cap_log2 = 0;
  bool has_cells = false;
  cudaStream_t stream = nullptr;
  JFlags jf{};
  bool lane_ok[kNumJ] = {};
};

}  // namespace xt

struct xt_ctx {
  int device = 0;
  int num_sms = 0;
  int smem_optin = 0;
  size_t budget = 0;            // 0: no cap
  size_t held = 0;              // bytes of device memory held
  // per-call workspace (grown on demand)
  void* work = nullptr;
  size_t work_bytes = 0;
  // global ring pool for pairs whose band does not fit in shared memory
  int2* pool = nullptr;
  size_t pool_bytes = 0;
  // end-to-end staging: device copies of host inputs and pinned host mirrors
  void* dev_in = nullptr;
  size_t dev_in_bytes = 0;
  // raw reads converted to base codes (XT_ALPHABET_ASCII)
  void* conv = nullptr;
  size_t conv_bytes = 0;
  // both-direction seed extension: per-seed arrays, reversed prefixes
  void* seed_ws = nullptr;
  size_t seed_ws_bytes = 0;
  void* seed_rev = nullptr;
  size_t seed_rev_bytes = 0;
  // BWA-MEM-compatible calls: class bytes, order, counters
  void* bwa_ws = nullptr;
  size_t bwa_ws_bytes = 0;
  int bwa_blocks[8] = {};        // resident CTAs per SM of each group-size kernel (0: unknown)
  // host-buffer calls: a copy stream and its events (chunked staging)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t stage_ev[2 * xt::kMaxChunks + 2] = {};
  // launch accounting and DP timing (xt_ctx_stats)
  bool timing = false;
  static constexpr int kEvRing = 256;
  cudaEvent_t ev[kEvRing][2] = {};
  int ev_pending = 0;
  int calls = 0, launches = 0, dp_launches = 0;
  // per-call batch descriptor: pinned host slots copied to a device slot

  // CUDA graphs of whole calls
  bool graphs = true;
  cudaStream_t cap_stream = nullptr;
  // the DP launches of a call fork onto these streams and join back
  int branches = xt::kMaxBranches;
  cudaStream_t aux[xt::kMaxBranches] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[xt::kMaxBranches] = {};
  std::vector<xt::GraphEntry> graph_cache;
  int match = 1;                 // scoring of the call being planned
  int forced_P = 0;              // schedule override (0: per-bucket table)
  int forced_R = 0;
  int alphabet = XT_ALPHABET_CODES;  // how sequence bytes encode bases
  std::vector<xt::TuneEntry> tuning;  // per-band bucket schedules (xt_autotune)
  bool plan_small = false;       // the bucket being planned is small (its small-batch schedule)
  // pair counts per (class, bucket) read back between classify and the plan
  int32_t* seg_host = nullptr;
  cudaEvent_t seg_ev = nullptr;
  std::mutex mu;
  std::string last_error;
  std::string launch_error;      // which launch of the call failed
  xt::PendingCall pending;       // xt_extend_batch_begin .. _finish
  // host-buffer calls in chunks: two internal contexts the chunks alternate
  // between (created on first use, contexts without a memory budget only)
  struct xt_ctx* chunk_ctx[2] = {};
};

