// xt_kernels.cuh -- kernel declarations and launch-plan types shared by the
// host API and the kernel translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "xt_common.cuh"

namespace xt {

// Pair classes after classify.
//   PACKED: two strips in the 16-bit halves of each register (one-lane engine)
//   NARROW: 32-bit, row key H*65536 + j (h0 + match*min(qlen,tlen) <= 32767)
//   WIDE:   32-bit with an explicit (max, column) pair per row
//   HUGE:   band ring too large for shared memory (global slab per group)
enum PairClass : uint8_t { CLS_PACKED = 0, CLS_NARROW = 1, CLS_WIDE = 2, CLS_HUGE = 3, CLS_DONE = 4 };
constexpr int kNumClasses = 4;           // classes that need a DP kernel
// per-bucket flags (Work::jflags)
constexpr uint8_t kJHuge = 1;            // bucket's pairs go to the HUGE class
constexpr uint8_t kJPacked = 2;          // bucket runs the one-lane engine: packed pairs allowed
constexpr uint8_t kJHugeWide = 4;        // the bucket's WIDE pairs (group engine only) are HUGE
constexpr uint8_t kJTag4 = 8;            // packed row keys of the bucket carry 4-bit step tags
// Step-tag bits of the packed row keys (H * 2^bits + step in 16 bits) in
// bucket j: 6 (H <= 511) up to queries of 510 bases, 4 (H <= 2047, folded
// every 16 steps) beyond, where a pair's score bound grows past 511.
constexpr int kTag4J = 10;
constexpr int packed_tag_bits(int j) { return j >= kTag4J ? 4 : 6; }
// Calls of at least this many pairs pack those buckets' pairs (kJTag4): only
// then are there enough of them to run one lane per pair; in smaller calls
// they go to lane groups, which run them in 32-bit anyway (c5-mix calls:
// 800k pairs 16.43 -> 16.00 ms, 4M 68.1 -> 58.8 ms; 400k 9.76 -> 11.90 ms had
// they been packed: a second group launch waited for the first).
constexpr int32_t kTag4MinPairs = 1 << 19;
constexpr int kJMin = 5;                 // length buckets j: qlen + 2 <= 2^j
constexpr int kJMax = 21;
constexpr int kNumJ = kJMax + 1;
constexpr int kNumSub = 256;             // sub-buckets per bucket: exact query length up to 2^9
constexpr int kNumBuckets = kNumClasses * kNumJ * kNumSub;
constexpr int kQueueThreads = 128;       // threads per CTA of the queue kernels
constexpr int kMaxLaunches = 64;         // queue-kernel launches per call (heads)

// Device workspace of one call (carved from the context's pool).
struct Work {
  uint8_t* pclass;      // [n]
  int32_t* order;       // [n] pairs grouped by (class, bucket desc, sub desc)
  int32_t* counts;      // [kNumBuckets]
  int32_t* cursor;      // [kNumBuckets]
  int32_t* seg_begin;   // [kNumClasses * kNumJ]
  int32_t* seg_end;     // [kNumClasses * kNumJ]
  int32_t* heads;       // [kMaxLaunches]
};

constexpr int kLaneThreads = 128;        // threads per CTA of the one-lane kernels
constexpr int kLaneStageJMax = 9;        // one-lane kernels stage queries up to 2^9 - 2 bases

// One persistent launch: pairs of class cls, buckets [j_lo, j_hi].  Every
// field has a default, so a launch built field by field never carries stack
// contents into the dispatch.
struct Launch {
  int cls = 0, j_lo = 0, j_hi = 0;
  bool lane = false;         // one-lane engine (k_lane) instead of the group engine (k_queue)
  int P = 1, R = 8;          // lanes per pair, rows per lane-strip (per half when packed)
  int rs_log2 = 0;           // ring entries per group = 1 << rs_log2
  bool global_ring = false;  // ring in a global slab per group instead of shared memory
  int64_t slab = 0;          // entries per global slab (power of two)
  int grid = 0;              // CTAs
  int mparam = 0;            // one-lane engine: match + 1 (32-bit) or shift k (packed)
  size_t pool_off = 0;       // global ring: byte offset of the launch's slabs in the pool
};

// Host-side launchers (defined in xt_kernels.cu); all enqueue on `stream`.
// Per-bucket flags (kJHuge | kJPacked), passed to classify by value.
struct JFlags {
  uint8_t f[kNumJ];
};
// Kernels read the batch arguments from a device copy (bd) so that one
// captured graph serves every call; n_cap sizes the per-pair grids (>= n).
cudaError_t launch_classify(const Batch* bd, int32_t n_cap, const Score& sc, int32_t match,
                            const JFlags& jf, const Work& w, cudaStream_t stream);
cudaError_t launch_order(const Batch* bd, int32_t n_cap, const Work& w, cudaStream_t stream);
cudaError_t launch_queue(const Batch* bd, const Score& sc, const Work& w, const Launch& L,
                         int head_id, int2* gring, cudaStream_t stream);
cudaError_t launch_plain(const Batch* bd, int32_t n_cap, const Score& sc, const Work& w,
                         int rs_log2, cudaStream_t stream);
cudaError_t launch_lane(const Batch* bd, const Score& sc, const Work& w, const Launch& L,
                        int head_id, void* gring, cudaStream_t stream);
// ASCII letters to base codes (A/C/G/T either case -> 0..3, else 4), n bytes.
cudaError_t launch_ascii_codes(const uint8_t* in, uint8_t* out, int64_t n, int num_sms,
                               cudaStream_t stream);
// 4-bit codes, two per byte, to one code per byte: bytes [b0, b1) of `in`
// become bytes [2 b0, 2 b1) of `out`.
cudaError_t launch_unpack4(const uint8_t* in, uint8_t* out, int64_t b0, int64_t b1, int num_sms,
                           cudaStream_t stream);
// Both-direction extension of seeds: device workspace (carved by the host).
struct SeedWork {
  int32_t *lq_len, *lt_len;   // left (reversed prefix) lengths, -1: invalid seed
  int64_t *lq_off, *lt_off;   // their offsets in rev_q / rev_t
  int32_t *rq_len, *rt_len;   // right (suffix) lengths, -1: invalid seed
  int64_t *rq_off, *rt_off;   // their offsets in the caller's buffers
  int32_t* rh0;               // right side's seed score
  int64_t *block_q, *block_t; // per-block sums of the left lengths
  int64_t* totals;            // [2]: bytes of rev_q and rev_t
  uint8_t *rev_q, *rev_t;     // reversed prefixes
};
// Prep, lengths, and the scan up to the totals (sw.totals, read by the host).
cudaError_t launch_seed_front(int32_t n, const int32_t* q_len, const int32_t* t_len,
                              const int64_t* q_off, const int64_t* t_off, int64_t q_bytes,
                              int64_t t_bytes, const int32_t* q_beg, const int32_t* t_beg,
                              const int32_t* seed_len, const SeedWork& sw, cudaStream_t stream);
// Offsets of the reversed prefixes and the reversed copies (sw.rev_q/rev_t set).
cudaError_t launch_seed_reverse(int32_t n, const uint8_t* q_seq, const int64_t* q_off,
                                const uint8_t* t_seq, const int64_t* t_off, const SeedWork& sw,
                                cudaStream_t stream);
// Right side's seed scores from the left results.
cudaError_t launch_seed_right_h0(int32_t n, const int32_t* h0, const xt_result* left,
                                 const SeedWork& sw, cudaStream_t stream);
// Shared memory a queue launch needs per CTA (bytes).
size_t queue_smem_bytes(int P, int rs_log2);
// Ring bytes per lane of a one-lane launch (per CTA in shared memory: x kLaneThreads).
size_t lane_ring_bytes(int cls, int rs_log2);
// Query staging bytes per CTA of a one-lane launch whose longest bucket is j_hi (0: none).
size_t lane_stage_bytes(int j_hi);
// Ring-feed slot bytes per CTA of a one-lane launch (global rings of 32-bit pairs).
size_t lane_pipe_bytes(int cls, bool global_ring);
int max_smem_per_block_optin(int device);

}  // namespace xt
