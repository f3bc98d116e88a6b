// xt_kernels.cu -- classify/bucket, ordering, persistent queue kernels and the
// plain one-pair-per-block kernel.
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>

#include "xt_engine.cuh"
#include "xt_kernels.cuh"
#include "xt_lane.cuh"

namespace xt {

__device__ __forceinline__ int ceil_log2(uint32_t x) {  // x >= 1
  return x <= 1 ? 0 : 32 - __clz(x - 1);
}

// Length bucket j (qlen + 2 <= 2^j, at least kJMin) and sub-bucket: the exact
// query length while a bucket spans at most kNumSub lengths, else its top bits.
__device__ __forceinline__ void bucket_of(int32_t ql, int* j_out, int* sub_out) {
  int j = ceil_log2((uint32_t)ql + 2u);
  if (j < kJMin) j = kJMin;
  int sub;
  if (j == kJMin) {
    sub = ql;
  } else {
    const int32_t off = ql + 2 - (1 << (j - 1));
    sub = j <= 9 ? off : (off >> (j - 9));
  }
  sub = sub < 0 ? 0 : (sub >= kNumSub ? kNumSub - 1 : sub);
  *j_out = j;
  *sub_out = sub;
}

// ---------------------------------------------------------------- classify
// Validates every pair, writes the results of invalid and degenerate pairs
// directly, and assigns the others a class and a (bucket, sub-bucket) by
// query length, counted for the ordering pass.  A block takes kOrdPer x
// kOrdThreads consecutive pairs and counts them in a shared-memory histogram
// of every (class, bucket, sub-bucket), then adds its non-zero bins to the
// global counts: a batch's pairs fall into a few hundred bins, and one global
// atomic per pair on those bins serialised the pass.
constexpr int kOrdThreads = 1024;
constexpr int kOrdPer = 8;
constexpr int kOrdPairs = kOrdThreads * kOrdPer;  // pairs per block

__device__ __forceinline__ void hist_clear(int32_t* s_hist) {
  for (int i = threadIdx.x; i < kNumBuckets; i += kOrdThreads) s_hist[i] = 0;
}

// Class of pair k (CLS_DONE after writing the result of an invalid or
// degenerate pair) and its histogram bin.
__device__ __forceinline__ int classify_pair(const Batch& b, int32_t k, int32_t match,
                                             int32_t mshift, const uint8_t* s_jf, int* bin) {
  const int64_t qo = b.q_off[k], to = b.t_off[k];
  const int32_t ql = b.q_len[k], tl = b.t_len[k], h0 = b.h0[k];
  const bool ok = h0 >= 1 && h0 <= XT_MAX_H0 && ql >= 0 && tl >= 0 && ql <= XT_MAX_LEN &&
                  tl <= XT_MAX_LEN && qo >= 0 && to >= 0 && qo <= b.q_bytes - ql &&
                  to <= b.t_bytes - tl;
  if (!ok) {
    write_result(b, k, 0, 0, 0, 0, 0, 0, XT_EINVAL, 0);
    return CLS_DONE;
  }
  if (ql == 0) {
    write_result(b, k, h0, 0, 0, h0, 0, 0, XT_OK, 0);
    return CLS_DONE;
  }
  if (tl == 0) {
    write_result(b, k, h0, 0, 0, -1, 0, 0, XT_OK, 0);
    return CLS_DONE;
  }
  int j, sub;
  bucket_of(ql, &j, &sub);
  const int64_t bound = (int64_t)h0 + (int64_t)match * (ql < tl ? ql : tl);
  const bool wide = bound > 32767 || ql > 65535;
  const uint8_t jf = s_jf[j];
  int cls = wide ? CLS_WIDE : CLS_NARROW;
  // packed: the anchoring multiply and the 16-bit row keys (H * 2^bits + step) fit
  const int64_t tag = (jf & kJTag4) ? 16 : 64;
  if (!wide && (jf & kJPacked) && ((bound + 1) << mshift) <= 32767 &&
      bound * tag + tag - 1 <= 32767)
    cls = CLS_PACKED;
  if ((jf & kJHuge) || (cls == CLS_WIDE && (jf & kJHugeWide))) cls = CLS_HUGE;
  *bin = (cls * kNumJ + j) * kNumSub + sub;
  return cls;
}

__global__ void __launch_bounds__(kOrdThreads) k_classify(const Batch* __restrict__ bd, Score sc,
                                                          int32_t match, int32_t mshift,
                                                          JFlags jfl, Work w) {
  extern __shared__ int32_t s_hist[];  // [kNumBuckets]
  // the bucket flags, indexed by a runtime bucket: shared memory, not a
  // local copy of the by-value argument
  __shared__ uint8_t s_jf[kNumJ];
  if (threadIdx.x < kNumJ) s_jf[threadIdx.x] = jfl.f[threadIdx.x];
  const Batch b = *bd;
  hist_clear(s_hist);
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kOrdPairs;
#pragma unroll 1
  for (int r = 0; r < kOrdPer; ++r) {
    const int64_t kk = base + r * kOrdThreads + threadIdx.x;
    if (kk < b.n) {
      const int32_t k = (int32_t)kk;
      int bin = 0;
      const int cls = classify_pair(b, k, match, mshift, s_jf, &bin);
      w.pclass[k] = (uint8_t)cls;
      if (cls < kNumClasses) atomicAdd(&s_hist[bin], 1);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kNumBuckets; i += kOrdThreads) {
    const int32_t c = s_hist[i];
    if (c) atomicAdd(&w.counts[i], c);
  }
}

// Exclusive scan of the bucket counts in queue order: per class, buckets from
// the longest down, sub-buckets from the longest down (longest work first).
// One block of kScanThreads threads, each owning a run of counters.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = (kNumBuckets + kScanThreads - 1) / kScanThreads;

__device__ __forceinline__ int scan_index(int L) {  // queue position -> counter index
  const int per_cls = kNumJ * kNumSub;
  const int cls = L / per_cls;
  const int rem = L - cls * per_cls;
  const int j = kJMax - rem / kNumSub;
  const int sub = kNumSub - 1 - rem % kNumSub;
  return (cls * kNumJ + j) * kNumSub + sub;
}

__global__ void __launch_bounds__(kScanThreads) k_scan(Work w) {
  __shared__ int32_t s_warp[kScanThreads / 32];
  const int t = threadIdx.x;
  int32_t vals[kScanPer];
  int32_t sum = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int L = t * kScanPer + k;
    vals[k] = L < kNumBuckets ? w.counts[scan_index(L)] : 0;
    sum += vals[k];
  }
  // block-wide exclusive scan of the per-thread sums
  const int lane = t & 31, wid = t >> 5;
  int32_t incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int32_t v = s_warp[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += u;
    }
    s_warp[lane] = v;  // inclusive warp totals
  }
  __syncthreads();
  int32_t acc = incl - sum + (wid > 0 ? s_warp[wid - 1] : 0);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int L = t * kScanPer + k;
    if (L < kNumBuckets) {
      const int idx = scan_index(L);
      const int cj = idx / kNumSub;  // cls * kNumJ + j
      const int sub = idx % kNumSub;
      w.cursor[idx] = acc;
      if (sub == kNumSub - 1) w.seg_begin[cj] = acc;
      acc += vals[k];
      if (sub == 0) w.seg_end[cj] = acc;
    }
  }
}

// Each block ranks its pairs within their bins in shared memory, reserves one
// run of queue slots per non-zero bin with one global atomic (the scan left
// every bin's cursor at its first slot) and writes the pairs' indices there.
__global__ void __launch_bounds__(kOrdThreads) k_scatter(const Batch* __restrict__ bd, Work w) {
  extern __shared__ int32_t s_hist[];  // [kNumBuckets]: counts, then run starts
  const int32_t n = bd->n;
  const int32_t* __restrict__ q_len = bd->q_len;
  hist_clear(s_hist);
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kOrdPairs;
  int bin[kOrdPer], rank[kOrdPer];
#pragma unroll
  for (int r = 0; r < kOrdPer; ++r) {
    const int64_t kk = base + r * kOrdThreads + threadIdx.x;
    bin[r] = -1;
    rank[r] = 0;
    if (kk < n) {
      const int cls = w.pclass[kk];
      if (cls < kNumClasses) {
        int j, sub;
        bucket_of(q_len[kk], &j, &sub);
        bin[r] = (cls * kNumJ + j) * kNumSub + sub;
        rank[r] = atomicAdd(&s_hist[bin[r]], 1);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kNumBuckets; i += kOrdThreads) {
    const int32_t c = s_hist[i];
    if (c) s_hist[i] = atomicAdd(&w.cursor[i], c);
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kOrdPer; ++r)
    if (bin[r] >= 0) w.order[s_hist[bin[r]] + rank[r]] = (int32_t)(base + r * kOrdThreads + threadIdx.x);
}

__device__ __forceinline__ Pair load_pair(const Batch& b, int32_t k) {
  Pair pr;
  pr.q = b.q_seq + b.q_off[k];
  pr.t = b.t_seq + b.t_off[k];
  pr.qlen = b.q_len[k];
  pr.tlen = b.t_len[k];
  pr.h0 = b.h0[k];
  return pr;
}

// ------------------------------------------------------- persistent queue
// Groups of P lanes pull pairs of class `cls`, buckets [j_lo, j_hi], from a
// device-side queue (one atomicAdd per pair) until it is empty.
// The score profile goes to shared memory with constant indices: indexing the
// by-value Score argument with threadIdx.x would move it to local memory.
__device__ __forceinline__ void copy_profile(const Score& sc, uint32_t* s_prof) {
#pragma unroll
  for (int c = 0; c < 5; ++c) s_prof[c] = sc.prof[c];
}

template <int P, int R, bool WIDE>
__global__ void __launch_bounds__(kQueueThreads)
    k_queue(const Batch* __restrict__ bd, Score sc, Work w, int cls, int j_lo, int j_hi,
            int head_id, int rs_log2, int2* gring, int64_t slab) {
  // batch arguments stay in shared memory and are read where used
  __shared__ Batch s_b;
  if (threadIdx.x == 0) s_b = *bd;
  __syncthreads();
  const Batch& b = s_b;
  extern __shared__ int2 s_ring[];
  __shared__ uint32_t s_prof[8];
  if (threadIdx.x == 0) copy_profile(sc, s_prof);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int p = threadIdx.x % P;
  const int g = threadIdx.x / P;
  constexpr int G = kQueueThreads / P;
  const unsigned gmask = (P == 32) ? 0xffffffffu : (((1u << P) - 1u) << (lane - p));
  const int32_t begin = w.seg_begin[cls * kNumJ + j_hi];
  const int32_t end = w.seg_end[cls * kNumJ + j_lo];
  int2* ring;
  int stride, rmask;
  if (gring) {
    ring = gring + (int64_t)(blockIdx.x * G + g) * slab;
    stride = 1;
    rmask = (int)(slab - 1);
  } else {
    ring = s_ring + g;
    stride = G;
    rmask = (1 << rs_log2) - 1;
  }
  int32_t* head = w.heads + head_id;
  for (;;) {
    int32_t idx = 0;
    if (p == 0) idx = begin + atomicAdd(head, 1);
    if (P > 1) idx = __shfl_sync(gmask, idx, 0, P);
    if (idx >= end) break;
    const int32_t k = w.order[idx];
    // an index outside the batch would mean a corrupt workspace: skip it
    // (group-uniform) rather than read outside the caller's arrays
    if ((uint32_t)k >= (uint32_t)b.n) continue;
    const Pair pr = load_pair(b, k);
    const Outcome o = run_pair<P, R, WIDE>(pr, sc, s_prof, ring, stride, rmask, p, gmask);
    if (p == 0) write_result(b, k, o.score, o.qle, o.tle, o.gscore, o.gtle, o.max_off, XT_OK,
                             o.cells);
  }
}

// --------------------------------------------------------- one-lane queue
// Every lane extends whole pairs on its own; the warp takes consecutive queue
// slots (one atomicAdd per warp per round), so neighbouring lanes get pairs
// of nearly equal length.
template <int R, bool PACKED, bool GRING, bool QSTAGE, int TB = 6>
__global__ void __launch_bounds__(kLaneThreads, 4)
    k_lane(const Batch* __restrict__ bd, Score sc, Work w, int cls, int j_lo, int j_hi,
           int head_id, int rs_log2, void* gring, int mparam, int qs_log2) {
  // batch arguments stay in shared memory and are read where used
  __shared__ Batch s_b;
  if (threadIdx.x == 0) s_b = *bd;
  const Batch& b = s_b;
  using T = typename Ring<PACKED>::T;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ uint32_t s_prof[8];
  if (threadIdx.x == 0) copy_profile(sc, s_prof);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // ring: column c of lane t at [(c & mask) * kLaneThreads + t], so the lanes
  // of a warp (which sit on the same column) touch consecutive words
  Ring<PACKED> ring;
  ring.mask = (1 << rs_log2) - 1;
  ring.stride = kLaneThreads;
  size_t ring_bytes = 0;
  if (GRING) {
    ring.base = reinterpret_cast<T*>(gring) +
                (int64_t)blockIdx.x * kLaneThreads * ((int64_t)1 << rs_log2) + threadIdx.x;
  } else {
    ring.base = reinterpret_cast<T*>(s_dyn) + threadIdx.x;
    ring_bytes = (size_t)kLaneThreads * ((size_t)1 << rs_log2) * sizeof(T);
  }
  Query<QSTAGE> qs;
  qs.stage = QSTAGE ? s_dyn + ring_bytes + (size_t)(threadIdx.x >> 5) * (32u << qs_log2) + lane
                    : nullptr;
  // 32-bit global rings feed their entries through shared-memory slots
  RingPipe<int2> pipe;
  pipe.slot0 = reinterpret_cast<int2*>(s_dyn) + threadIdx.x;
  const int32_t begin = w.seg_begin[cls * kNumJ + j_hi];
  const int32_t end = w.seg_end[cls * kNumJ + j_lo];
  int32_t* head = w.heads + head_id;
  // rounds of 32 consecutive pairs per warp, all lanes together
  for (;;) {
    int32_t base = 0;
    if (lane == 0) base = atomicAdd(head, 32);
    base = begin + __shfl_sync(0xffffffffu, base, 0);
    if (base >= end) break;
    const int32_t idx = base + lane;
    Pair pr;
    int32_t k = idx < end ? w.order[idx] : -1;
    // an index outside the batch would mean a corrupt workspace: the lane
    // idles rather than read outside the caller's arrays
    const bool valid = (uint32_t)k < (uint32_t)b.n;
    if (valid) {
      pr = load_pair(b, k);
    } else {
      pr.q = b.q_seq; pr.t = b.t_seq; pr.qlen = 0; pr.tlen = 0; pr.h0 = 1;
    }
    Outcome o;
    qs.g = pr.q;
    if (PACKED)
      o = lane_pair_p16<R, QSTAGE, TB>(pr, valid, sc, s_prof,
                                       *reinterpret_cast<Ring<true>*>(&ring), mparam & 0xFF, qs);
    else
      o = lane_pair_i32<R, GRING>(pr, valid, sc, s_prof, *reinterpret_cast<Ring<false>*>(&ring),
                                  mparam, pipe);
    if (valid)
      write_result(b, k, o.score, o.qle, o.tle, o.gscore, o.gtle, o.max_off, XT_OK, o.cells);
  }
}

// ------------------------------------------------------------------ plain
// One pair per thread block of one warp (P = 32 lanes, R = 8 rows per lane),
// 32-bit arithmetic, no bucketing: the comparison kernel.
__global__ void __launch_bounds__(32) k_plain(const Batch* __restrict__ bd, Score sc, Work w,
                                              int rs_log2) {
  extern __shared__ int2 s_ring[];
  __shared__ uint32_t s_prof[8];
  const Batch b = *bd;
  const int32_t k = blockIdx.x;
  if (k >= b.n) return;
  const int cls = w.pclass[k];
  if (cls != CLS_NARROW && cls != CLS_WIDE) return;
  if (threadIdx.x == 0) copy_profile(sc, s_prof);
  __syncwarp();
  const Pair pr = load_pair(b, k);
  const int rmask = (1 << rs_log2) - 1;
  Outcome o;
  if (cls == CLS_NARROW)
    o = run_pair<32, 8, false>(pr, sc, s_prof, s_ring, 1, rmask, threadIdx.x, 0xffffffffu);
  else
    o = run_pair<32, 8, true>(pr, sc, s_prof, s_ring, 1, rmask, threadIdx.x, 0xffffffffu);
  if (threadIdx.x == 0)
    write_result(b, k, o.score, o.qle, o.tle, o.gscore, o.gtle, o.max_off, XT_OK, o.cells);
}

// ------------------------------------------------------- ASCII -> codes
// Raw reads (ASCII letters) to base codes, four bytes per thread-step with
// per-byte SIMD compares: A, C, G, T in either case become 0, 1, 2, 3 and
// any other byte becomes 4 (N).  Grid-stride over 16-byte chunks of the
// buffer (word loads when both pointers are 4-byte aligned, else bytes).
__device__ __forceinline__ uint32_t codes4(uint32_t w) {
  const uint32_t x = w | 0x20202020u;  // lower case
  const uint32_t a = __vcmpeq4(x, 0x61616161u), c = __vcmpeq4(x, 0x63636363u);
  const uint32_t g = __vcmpeq4(x, 0x67676767u), t = __vcmpeq4(x, 0x74747474u);
  const uint32_t base = a | c | g | t;
  const uint32_t code = (c & 0x01010101u) | (g & 0x02020202u) | (t & 0x03030303u);
  return (code & base) | (0x04040404u & ~base);
}

__global__ void k_ascii_codes(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                              int64_t n) {
  const int64_t chunks = (n + 15) / 16;
  const bool words = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 3u) == 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < chunks;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b0 = k * 16;
    if (words && b0 + 16 <= n) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(in + b0);
      uint32_t* dst = reinterpret_cast<uint32_t*>(out + b0);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = codes4(__ldg(src + q));
    } else {
      for (int64_t b = b0; b < n && b < b0 + 16; ++b) out[b] = (uint8_t)(codes4(in[b]) & 0xFFu);
    }
  }
}

cudaError_t launch_ascii_codes(const uint8_t* in, uint8_t* out, int64_t n, int num_sms,
                               cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int64_t chunks = (n + 15) / 16;
  const int T = 256;
  const int64_t want = (chunks + T - 1) / T;
  const int grid = (int)(want < (int64_t)num_sms * 8 ? want : (int64_t)num_sms * 8);
  k_ascii_codes<<<grid, T, 0, stream>>>(in, out, n);
  return cudaGetLastError();
}

// ------------------------------------------------ 4-bit codes -> bytes
// Two 4-bit codes per byte (base 2k in the low nibble of byte k, base 2k+1 in
// the high nibble) to one code per byte.  A thread expands one 32-bit word
// (eight bases) into two: the low nibbles of its bytes are bases 0, 2, 4, 6,
// the high nibbles 1, 3, 5, 7, interleaved back by two byte permutes.
// Bytes [b0, b1) of `in` become bytes [2 b0, 2 b1) of `out`; grid-stride.
__device__ __forceinline__ void unpack_word(uint32_t w, uint32_t* lo, uint32_t* hi) {
  const uint32_t ev = w & 0x0F0F0F0Fu, od = (w >> 4) & 0x0F0F0F0Fu;
  uint32_t a, b;
  asm("prmt.b32 %0, %1, %2, 0x5140;" : "=r"(a) : "r"(ev), "r"(od));
  asm("prmt.b32 %0, %1, %2, 0x7362;" : "=r"(b) : "r"(ev), "r"(od));
  *lo = a;
  *hi = b;
}

__global__ void k_unpack4(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int64_t b0,
                          int64_t b1) {
  // word-aligned middle: whole 32-bit words of `in` (out is then 8-byte aligned
  // whenever both buffers start on 8-byte boundaries)
  const bool words = ((reinterpret_cast<uintptr_t>(in) & 3u) == 0) &&
                     ((reinterpret_cast<uintptr_t>(out) & 7u) == 0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t m0 = b0, m1 = b0;
  if (words) {
    m0 = (b0 + 3) & ~(int64_t)3;
    m1 = b1 & ~(int64_t)3;
    if (m1 < m0) m1 = m0;
    for (int64_t k = m0 / 4 + t; k < m1 / 4; k += stride) {
      uint32_t lo, hi;
      unpack_word(__ldg(reinterpret_cast<const uint32_t*>(in) + k), &lo, &hi);
      reinterpret_cast<uint2*>(out)[k] = make_uint2(lo, hi);
    }
  }
  // the ragged ends (or everything, unaligned) byte by byte
  auto one = [&](int64_t k) {
    const uint32_t v = in[k];
    out[2 * k] = (uint8_t)(v & 15u);
    out[2 * k + 1] = (uint8_t)(v >> 4);
  };
  for (int64_t k = b0 + t; k < (words ? m0 : b1); k += stride) one(k);
  if (words)
    for (int64_t k = m1 + t; k < b1; k += stride) one(k);
}

cudaError_t launch_unpack4(const uint8_t* in, uint8_t* out, int64_t b0, int64_t b1, int num_sms,
                           cudaStream_t stream) {
  if (b1 <= b0) return cudaSuccess;
  const int T = 256;
  const int64_t want = ((b1 - b0) / 4 + T - 1) / T + 1;
  const int grid = (int)(want < (int64_t)num_sms * 8 ? want : (int64_t)num_sms * 8);
  k_unpack4<<<grid, T, 0, stream>>>(in, out, b0, b1);
  return cudaGetLastError();
}

// ------------------------------------------------ both-direction seeds
// Seed k: an exact match of seed_len[k] bases at query q_beg[k] and target
// t_beg[k].  Left lengths are the prefixes before the seed, right views the
// suffixes after it (offsets into the caller's buffers); a seed outside its
// pair gets length -1 on both sides, which classify reports as XT_EINVAL.
__global__ void k_seed_prep(int32_t n, const int32_t* __restrict__ q_len,
                            const int32_t* __restrict__ t_len, const int64_t* __restrict__ q_off,
                            const int64_t* __restrict__ t_off, int64_t q_bytes, int64_t t_bytes,
                            const int32_t* __restrict__ q_beg, const int32_t* __restrict__ t_beg,
                            const int32_t* __restrict__ seed_len, SeedWork sw) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int32_t ql = q_len[k], tl = t_len[k], qb = q_beg[k], tb = t_beg[k], sl = seed_len[k];
  const int64_t qo = q_off[k], to = t_off[k];
  // the pair inside its buffers (the reversed copy reads them before classify
  // checks anything), the seed inside the pair
  const bool ok = ql >= 0 && tl >= 0 && ql <= XT_MAX_LEN && tl <= XT_MAX_LEN && qo >= 0 &&
                  to >= 0 && qo <= q_bytes - ql && to <= t_bytes - tl && qb >= 0 && tb >= 0 &&
                  sl >= 0 && (int64_t)qb + sl <= ql && (int64_t)tb + sl <= tl;
  sw.lq_len[k] = ok ? qb : -1;
  sw.lt_len[k] = ok ? tb : -1;
  sw.rq_len[k] = ok ? ql - qb - sl : -1;
  sw.rt_len[k] = ok ? tl - tb - sl : -1;
  sw.rq_off[k] = ok ? qo + qb + sl : 0;
  sw.rt_off[k] = ok ? to + tb + sl : 0;
}

// Exclusive prefix sums of the left lengths (both sides at once), in blocks
// of kSeedScanBlock pairs: block-local sums first, then a scan of the block
// totals, then the final offsets.
constexpr int kSeedScanBlock = 1024;

__device__ __forceinline__ void block_scan2(int64_t& a, int64_t& b, int64_t* s_a, int64_t* s_b) {
  // inclusive block-wide scan of two values (blockDim.x = kSeedScanBlock)
  const int t = threadIdx.x;
  s_a[t] = a;
  s_b[t] = b;
  __syncthreads();
  for (int d = 1; d < kSeedScanBlock; d <<= 1) {
    const int64_t va = t >= d ? s_a[t - d] : 0, vb = t >= d ? s_b[t - d] : 0;
    __syncthreads();
    s_a[t] += va;
    s_b[t] += vb;
    __syncthreads();
  }
  a = s_a[t];
  b = s_b[t];
}

__global__ void __launch_bounds__(kSeedScanBlock) k_seed_sums(int32_t n, SeedWork sw) {
  __shared__ int64_t s_a[kSeedScanBlock], s_b[kSeedScanBlock];
  const int32_t k = blockIdx.x * kSeedScanBlock + threadIdx.x;
  int64_t a = k < n ? max(sw.lq_len[k], 0) : 0, b = k < n ? max(sw.lt_len[k], 0) : 0;
  block_scan2(a, b, s_a, s_b);
  if (threadIdx.x == kSeedScanBlock - 1) {
    sw.block_q[blockIdx.x] = a;
    sw.block_t[blockIdx.x] = b;
  }
}

// One block: exclusive scan of the block totals (in place) and the grand totals.
__global__ void __launch_bounds__(kSeedScanBlock) k_seed_block_scan(int32_t nblocks, SeedWork sw) {
  __shared__ int64_t s_a[kSeedScanBlock], s_b[kSeedScanBlock];
  int64_t carry_a = 0, carry_b = 0;
  for (int32_t base = 0; base < nblocks; base += kSeedScanBlock) {
    const int32_t i = base + threadIdx.x;
    const int64_t a0 = i < nblocks ? sw.block_q[i] : 0, b0 = i < nblocks ? sw.block_t[i] : 0;
    int64_t a = a0, b = b0;
    block_scan2(a, b, s_a, s_b);
    if (i < nblocks) {
      sw.block_q[i] = carry_a + a - a0;
      sw.block_t[i] = carry_b + b - b0;
    }
    carry_a += s_a[kSeedScanBlock - 1];
    carry_b += s_b[kSeedScanBlock - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sw.totals[0] = carry_a;
    sw.totals[1] = carry_b;
  }
}

__global__ void __launch_bounds__(kSeedScanBlock) k_seed_offsets(int32_t n, SeedWork sw) {
  __shared__ int64_t s_a[kSeedScanBlock], s_b[kSeedScanBlock];
  const int32_t k = blockIdx.x * kSeedScanBlock + threadIdx.x;
  const int64_t a0 = k < n ? max(sw.lq_len[k], 0) : 0, b0 = k < n ? max(sw.lt_len[k], 0) : 0;
  int64_t a = a0, b = b0;
  block_scan2(a, b, s_a, s_b);
  if (k < n) {
    sw.lq_off[k] = sw.block_q[blockIdx.x] + a - a0;
    sw.lt_off[k] = sw.block_t[blockIdx.x] + b - b0;
  }
}

// The reversed prefixes, one warp per seed.
__global__ void k_seed_reverse(int32_t n, const uint8_t* __restrict__ q_seq,
                               const int64_t* __restrict__ q_off,
                               const uint8_t* __restrict__ t_seq,
                               const int64_t* __restrict__ t_off, SeedWork sw) {
  const int32_t k = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= n) return;
  const int32_t lq = sw.lq_len[k], lt = sw.lt_len[k];
  const uint8_t* q = q_seq + q_off[k];
  const uint8_t* t = t_seq + t_off[k];
  for (int32_t i = lane; i < lq; i += 32) sw.rev_q[sw.lq_off[k] + i] = q[lq - 1 - i];
  for (int32_t i = lane; i < lt; i += 32) sw.rev_t[sw.lt_off[k] + i] = t[lt - 1 - i];
}

// Right side's seed score: the left side's local best (the seed's own
// score where the left side had nothing to extend).
__global__ void k_seed_right_h0(int32_t n, const int32_t* __restrict__ h0,
                                const xt_result* __restrict__ left, SeedWork sw) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  sw.rh0[k] = left[k].status == XT_OK ? left[k].score : h0[k];
}

cudaError_t launch_seed_front(int32_t n, const int32_t* q_len, const int32_t* t_len,
                              const int64_t* q_off, const int64_t* t_off, int64_t q_bytes,
                              int64_t t_bytes, const int32_t* q_beg, const int32_t* t_beg,
                              const int32_t* seed_len, const SeedWork& sw, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_seed_prep<<<(n + 255) / 256, 256, 0, stream>>>(n, q_len, t_len, q_off, t_off, q_bytes, t_bytes,
                                                  q_beg, t_beg, seed_len, sw);
  const int32_t nb = (n + kSeedScanBlock - 1) / kSeedScanBlock;
  k_seed_sums<<<nb, kSeedScanBlock, 0, stream>>>(n, sw);
  k_seed_block_scan<<<1, kSeedScanBlock, 0, stream>>>(nb, sw);
  return cudaGetLastError();
}

cudaError_t launch_seed_reverse(int32_t n, const uint8_t* q_seq, const int64_t* q_off,
                                const uint8_t* t_seq, const int64_t* t_off, const SeedWork& sw,
                                cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int32_t nb = (n + kSeedScanBlock - 1) / kSeedScanBlock;
  k_seed_offsets<<<nb, kSeedScanBlock, 0, stream>>>(n, sw);
  const int64_t threads = (int64_t)n * 32;
  k_seed_reverse<<<(int)((threads + 255) / 256), 256, 0, stream>>>(n, q_seq, q_off, t_seq, t_off,
                                                                  sw);
  return cudaGetLastError();
}

cudaError_t launch_seed_right_h0(int32_t n, const int32_t* h0, const xt_result* left,
                                 const SeedWork& sw, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_seed_right_h0<<<(n + 255) / 256, 256, 0, stream>>>(n, h0, left, sw);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- launchers
// Static shared memory of the kernels (descriptor copy, profiles) stays below
// this; a launch asks for the larger dynamic limit whenever both together
// could pass the 48 KB a kernel gets without opting in.
constexpr size_t kStaticSmemMax = 1024;

// The dynamic shared-memory limit of a kernel is one attribute per (kernel,
// device) for the whole process, and calls of several contexts (or a context
// call and an allocation-free call) may launch the same kernel from several
// host threads at once.  The limit is therefore only ever raised, under a
// lock, never set back to a smaller launch's size: it is a cap, and each
// launch's occupancy still follows its own dynamic size.
std::mutex g_smem_mu;
std::map<std::pair<const void*, int>, int> g_smem_limit;  // (kernel, device) -> limit set

template <typename K>
cudaError_t raise_smem_limit(K kern, size_t smem) {
  if (smem + kStaticSmemMax <= 48 * 1024) return cudaSuccess;  // the default limit covers it
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const std::pair<const void*, int> key(reinterpret_cast<const void*>(kern), dev);
  std::lock_guard<std::mutex> lk(g_smem_mu);
  auto it = g_smem_limit.find(key);
  if (it != g_smem_limit.end() && it->second >= (int)smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) g_smem_limit[key] = (int)smem;
  return e;
}

constexpr size_t kHistBytes = sizeof(int32_t) * (size_t)kNumBuckets;

cudaError_t launch_classify(const Batch* bd, int32_t n_cap, const Score& sc, int32_t match,
                            const JFlags& jf, const Work& w, cudaStream_t stream) {
  if (n_cap == 0) return cudaSuccess;
  int mshift = 0;
  while ((1 << mshift) < match + 1) ++mshift;
  cudaError_t e = raise_smem_limit(k_classify, kHistBytes);
  if (e != cudaSuccess) return e;
  const int grid = (int)(((int64_t)n_cap + kOrdPairs - 1) / kOrdPairs);
  k_classify<<<grid, kOrdThreads, kHistBytes, stream>>>(bd, sc, match, mshift, jf, w);
  return cudaGetLastError();
}

cudaError_t launch_order(const Batch* bd, int32_t n_cap, const Work& w, cudaStream_t stream) {
  k_scan<<<1, kScanThreads, 0, stream>>>(w);
  if (n_cap > 0) {
    cudaError_t e = raise_smem_limit(k_scatter, kHistBytes);
    if (e != cudaSuccess) return e;
    const int grid = (int)(((int64_t)n_cap + kOrdPairs - 1) / kOrdPairs);
    k_scatter<<<grid, kOrdThreads, kHistBytes, stream>>>(bd, w);
  }
  return cudaGetLastError();
}

size_t queue_smem_bytes(int P, int rs_log2) {
  return (size_t)(kQueueThreads / P) * ((size_t)1 << rs_log2) * sizeof(int2);
}

template <int P, int R, bool WIDE>
static cudaError_t launch_queue_t(const Batch* b, const Score& sc, const Work& w, const Launch& L,
                                  int head_id, int2* gring, cudaStream_t stream) {
  const size_t smem = L.global_ring ? 0 : queue_smem_bytes(P, L.rs_log2);
  auto kern = k_queue<P, R, WIDE>;
  cudaError_t e = raise_smem_limit(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<L.grid, kQueueThreads, smem, stream>>>(b, sc, w, L.cls, L.j_lo, L.j_hi, head_id,
                                                L.rs_log2, L.global_ring ? gring : nullptr,
                                                L.slab);
  return cudaGetLastError();
}

template <bool WIDE>
static cudaError_t launch_queue_w(const Batch* b, const Score& sc, const Work& w, const Launch& L,
                                  int head_id, int2* gring, cudaStream_t stream) {
#define XT_Q(PP, RR) \
  if (L.P == PP && L.R == RR) return launch_queue_t<PP, RR, WIDE>(b, sc, w, L, head_id, gring, stream);
  XT_Q(1, 8) XT_Q(2, 8) XT_Q(4, 8) XT_Q(8, 8) XT_Q(16, 8) XT_Q(32, 8)
  XT_Q(1, 4) XT_Q(2, 4) XT_Q(4, 4) XT_Q(8, 4) XT_Q(16, 4) XT_Q(32, 4)
  XT_Q(1, 16) XT_Q(2, 16) XT_Q(4, 16)
#undef XT_Q
  return cudaErrorInvalidValue;
}

cudaError_t launch_queue(const Batch* b, const Score& sc, const Work& w, const Launch& L,
                         int head_id, int2* gring, cudaStream_t stream) {
  // packed pairs (score bound B <= 2047) fit the 32-bit row key H * 65536 + j
  // as NARROW pairs do; WIDE and HUGE pairs keep the explicit (max, column)
  if (L.cls == CLS_NARROW || L.cls == CLS_PACKED)
    return launch_queue_w<false>(b, sc, w, L, head_id, gring, stream);
  return launch_queue_w<true>(b, sc, w, L, head_id, gring, stream);
}

size_t lane_ring_bytes(int cls, int rs_log2) {
  return ((size_t)1 << rs_log2) * (cls == CLS_PACKED ? sizeof(uint32_t) : sizeof(int2));
}

size_t lane_stage_bytes(int j_hi) {
  return j_hi <= kLaneStageJMax ? (size_t)kLaneThreads << j_hi : 0;
}

size_t lane_pipe_bytes(int cls, bool global_ring) {
  return (global_ring && cls != CLS_PACKED) ? (size_t)kLaneThreads * kPipeD * sizeof(int2) : 0;
}

template <int R, bool PACKED, bool GRING, bool QSTAGE, int TB = 6>
static cudaError_t launch_lane_t(const Batch* b, const Score& sc, const Work& w, const Launch& L,
                                 int head_id, void* gring, cudaStream_t stream) {
  const size_t smem = (GRING ? 0 : kLaneThreads * lane_ring_bytes(L.cls, L.rs_log2)) +
                      (QSTAGE ? lane_stage_bytes(L.j_hi) : 0) + lane_pipe_bytes(L.cls, GRING);
  auto kern = k_lane<R, PACKED, GRING, QSTAGE, TB>;
  cudaError_t e = raise_smem_limit(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<L.grid, kLaneThreads, smem, stream>>>(b, sc, w, L.cls, L.j_lo, L.j_hi, head_id,
                                               L.rs_log2, gring, L.mparam, L.j_hi);
  return cudaGetLastError();
}

cudaError_t launch_lane(const Batch* b, const Score& sc, const Work& w, const Launch& L,
                        int head_id, void* gring, cudaStream_t stream) {
  const bool packed = L.cls == CLS_PACKED;
  const bool stage = packed && lane_stage_bytes(L.j_hi) > 0;
  // packed long buckets (no query stage): row keys with 4-bit step tags
  if (packed && (L.mparam >> 8) == 4) {
    if (stage || (L.R != 4 && L.R != 8)) return cudaErrorInvalidValue;
    if (L.R == 4)
      return L.global_ring ? launch_lane_t<4, true, true, false, 4>(b, sc, w, L, head_id, gring, stream)
                           : launch_lane_t<4, true, false, false, 4>(b, sc, w, L, head_id, gring, stream);
    return L.global_ring ? launch_lane_t<8, true, true, false, 4>(b, sc, w, L, head_id, gring, stream)
                         : launch_lane_t<8, true, false, false, 4>(b, sc, w, L, head_id, gring, stream);
  }
#define XT_LG(RR, PK, GR)                                                                       \
  return stage ? launch_lane_t<RR, PK, GR, true>(b, sc, w, L, head_id, gring, stream)           \
               : launch_lane_t<RR, PK, GR, false>(b, sc, w, L, head_id, gring, stream);
#define XT_L(RR)                                                                                \
  if (L.R == RR) {                                                                              \
    if (packed) {                                                                               \
      if (L.global_ring) { XT_LG(RR, true, true) } else { XT_LG(RR, true, false) }             \
    }                                                                                           \
    return L.global_ring ? launch_lane_t<RR, false, true, false>(b, sc, w, L, head_id, gring, stream) \
                         : launch_lane_t<RR, false, false, false>(b, sc, w, L, head_id, gring, stream); \
  }
  XT_L(4) XT_L(8)
  if (L.R == 16) {
    if (packed)
      return L.global_ring ? launch_lane_t<16, true, true, false>(b, sc, w, L, head_id, gring, stream)
                           : launch_lane_t<16, true, false, false>(b, sc, w, L, head_id, gring, stream);
    return L.global_ring ? launch_lane_t<16, false, true, false>(b, sc, w, L, head_id, gring, stream)
                         : launch_lane_t<16, false, false, false>(b, sc, w, L, head_id, gring, stream);
  }
#undef XT_L
#undef XT_LG
  return cudaErrorInvalidValue;
}

cudaError_t launch_plain(const Batch* b, int32_t n_cap, const Score& sc, const Work& w,
                         int rs_log2, cudaStream_t stream) {
  if (n_cap == 0) return cudaSuccess;
  const size_t smem = ((size_t)1 << rs_log2) * sizeof(int2);
  cudaError_t e = raise_smem_limit(k_plain, smem);
  if (e != cudaSuccess) return e;
  k_plain<<<n_cap, 32, smem, stream>>>(b, sc, w, rs_log2);
  return cudaGetLastError();
}

int max_smem_per_block_optin(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  return v;
}

}  // namespace xt
