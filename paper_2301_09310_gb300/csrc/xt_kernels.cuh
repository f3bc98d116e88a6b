// xt_kernels.cuh -- kernel declarations and launch-plan types shared by the
// host API and the kernel translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "xt_common.cuh"

namespace xt {

// Pair classes after classify.
enum PairClass : uint8_t { CLS_NARROW = 0, CLS_WIDE = 1, CLS_HUGE = 2, CLS_DONE = 3 };
constexpr int kNumClasses = 3;           // classes that need a DP kernel
constexpr int kJMin = 5;                 // length buckets j: qlen + 2 <= 2^j
constexpr int kJMax = 21;
constexpr int kNumJ = kJMax + 1;
constexpr int kNumSub = 8;               // sub-buckets (finer length order) per bucket
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
  uint8_t* huge_j;      // [kNumJ] 1 if bucket j goes to the global-ring kernel
};

// One persistent queue-kernel launch: pairs of class cls, buckets [j_lo, j_hi].
struct Launch {
  int cls, j_lo, j_hi;
  int P, R;            // lanes per pair, rows per lane-strip
  int rs_log2;         // ring entries per group = 1 << rs_log2 (shared memory)
  bool global_ring;    // huge pairs: ring in a global slab per group
  int64_t slab;        // entries per global slab (power of two)
  int grid;            // CTAs
};

// Host-side launchers (defined in xt_kernels.cu); all enqueue on `stream`.
cudaError_t launch_classify(const Batch& b, const Score& sc, int32_t match, const Work& w,
                            cudaStream_t stream);
cudaError_t launch_order(const Batch& b, const Work& w, cudaStream_t stream);
cudaError_t launch_queue(const Batch& b, const Score& sc, const Work& w, const Launch& L,
                         int head_id, int2* gring, cudaStream_t stream);
cudaError_t launch_plain(const Batch& b, const Score& sc, const Work& w, int rs_log2,
                         cudaStream_t stream);
// Shared memory a queue launch needs per CTA (bytes).
size_t queue_smem_bytes(int P, int rs_log2);
int max_smem_per_block_optin(int device);

}  // namespace xt
