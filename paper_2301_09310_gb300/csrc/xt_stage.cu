// xt_stage.cu -- staging of a call's inputs: the device descriptor of a
// batch, and for host-buffer calls (xt_extend_batch_host) how far into the
// sequence buffers each chunk of pairs reads, so that the copies of later
// chunks' bytes overlap the extension of earlier chunks.
#include <cstdint>

#include "xt_ctx.cuh"

namespace xt {
namespace {

constexpr int kStageThreads = 256;

// ends[2k] / ends[2k+1]: the largest q_off + q_len / t_off + t_len over the
// pairs of chunk k (pairs [cb.start[k], cb.start[k+1])), clamped to
// [0, q_bytes] / [0, t_bytes].  Chunk starts are multiples of the block size,
// so a block never spans two chunks; ends must start at 0.
__global__ void __launch_bounds__(kStageThreads)
k_chunk_ends(const int64_t* __restrict__ q_off, const int32_t* __restrict__ q_len,
             const int64_t* __restrict__ t_off, const int32_t* __restrict__ t_len, int32_t n,
             ChunkStarts cb, int64_t q_bytes, int64_t t_bytes,
             unsigned long long* __restrict__ ends) {
  __shared__ unsigned long long s_q[kStageThreads / 32], s_t[kStageThreads / 32];
  const int64_t p = (int64_t)blockIdx.x * kStageThreads + threadIdx.x;
  unsigned long long qe = 0, te = 0;
  if (p < n) {
    int64_t a = q_off[p] + (int64_t)q_len[p];
    int64_t b = t_off[p] + (int64_t)t_len[p];
    a = a < 0 ? 0 : (a > q_bytes ? q_bytes : a);
    b = b < 0 ? 0 : (b > t_bytes ? t_bytes : b);
    qe = (unsigned long long)a;
    te = (unsigned long long)b;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, qe, o);
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, te, o);
    qe = x > qe ? x : qe;
    te = y > te ? y : te;
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_q[wid] = qe;
    s_t[wid] = te;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int u = 1; u < kStageThreads / 32; ++u) {
      qe = s_q[u] > qe ? s_q[u] : qe;
      te = s_t[u] > te ? s_t[u] : te;
    }
    const int64_t base = (int64_t)blockIdx.x * kStageThreads;
    if (base < n) {
      int k = 0;
      while (k + 1 < cb.count && base >= cb.start[k + 1]) ++k;
      atomicMax(&ends[2 * k], qe);
      atomicMax(&ends[2 * k + 1], te);
    }
  }
}

__global__ void k_store_desc(Batch* dst, Batch b) { *dst = b; }

}  // namespace

cudaError_t launch_store_desc(Batch* dst, const Batch& b, cudaStream_t stream) {
  k_store_desc<<<1, 1, 0, stream>>>(dst, b);
  return cudaGetLastError();
}

cudaError_t launch_chunk_ends(const int64_t* q_off, const int32_t* q_len, const int64_t* t_off,
                              const int32_t* t_len, int32_t n, const ChunkStarts& cb,
                              int64_t q_bytes, int64_t t_bytes, unsigned long long* ends,
                              cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  if (cb.count < 1 || cb.count > kMaxChunks || cb.start[0] != 0) return cudaErrorInvalidValue;
  for (int k = 1; k < cb.count; ++k)
    if (cb.start[k] % kStageThreads != 0 || cb.start[k] <= cb.start[k - 1]) return cudaErrorInvalidValue;
  const int grid = (int)(((int64_t)n + kStageThreads - 1) / kStageThreads);
  k_chunk_ends<<<grid, kStageThreads, 0, stream>>>(q_off, q_len, t_off, t_len, n, cb, q_bytes,
                                                    t_bytes, ends);
  return cudaGetLastError();
}

}  // namespace xt
