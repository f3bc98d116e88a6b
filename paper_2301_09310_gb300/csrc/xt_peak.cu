// xt_peak.cu -- measurement aid: integer instruction throughput of this GPU.
//
// The extension DP is integer arithmetic, so its roofline is the rate at
// which an SM issues the integer instructions the cell update is made of.
// Each probe kernel runs one kind of instruction in 8 independent chains per
// thread (enough warps per SM and chains per warp that latency is hidden), so
// its time measures that instruction's throughput.  Empty volatile asm
// statements make every chain value opaque to the compiler after each step,
// so nothing is folded, hoisted or merged; they emit no instructions.
//
// XT_RATE_CELL_P16 runs the packed one-lane cell update itself (the fast
// step of the extension engine: 8 row pairs = 16 cells per step) on
// registers: the ceiling of that code with no memory, band or row work.
#include <cstdint>
#include <cuda_runtime.h>

#include "xt.h"
#include "xt_kernels.cuh"
#include "xt_lane.cuh"

namespace {

constexpr int kRateThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 4;  // steps of all chains per loop iteration

__device__ __forceinline__ void opaque(uint32_t& v) { asm volatile("" : "+r"(v)); }

template <int OP>
__device__ __forceinline__ uint32_t op_step(uint32_t a, uint32_t b, uint32_t c, int k) {
  uint32_t r;
  if constexpr (OP == XT_RATE_ADD16X2) {
    asm("add.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  } else if constexpr (OP == XT_RATE_MAX3_16X2) {
    r = __vimax3_s16x2(a, b, c);
  } else if constexpr (OP == XT_RATE_ADDMAX_16X2) {
    r = __viaddmax_s16x2_relu(a, b, c);
  } else if constexpr (OP == XT_RATE_PRMT) {
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  } else if constexpr (OP == XT_RATE_IADD3) {
    r = a + b + c;
  } else if constexpr (OP == XT_RATE_MAX3_32) {
    r = (uint32_t)__vimax3_s32((int)a, (int)b, (int)c);
  } else if constexpr (OP == XT_RATE_IMAD) {
    r = a * b + c;
  } else if constexpr (OP == XT_RATE_HMAX2) {
    asm("max.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  }
  return r;
}

// XT_RATE_MIX: the even chains run the 3-way packed max (ALU pipe), the odd
// chains the packed add (multiply-add pipe): the two kinds whose single-kind
// probes execute exactly as counted (ncu), now interleaved so that both
// pipes feed the issue slots.
__device__ __forceinline__ uint32_t mix_step(uint32_t a, uint32_t b, uint32_t c, int k) {
  uint32_t r;
  if (k & 1)
    asm("add.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  else
    r = __vimax3_s16x2(a, b, c);
  return r;
}

template <int OP>
__global__ void __launch_bounds__(kRateThreads) k_rate(uint32_t seed, int iters, uint32_t* sink) {
  uint32_t a[kChains], b[kChains], c[kChains];
  const uint32_t t = blockIdx.x * kRateThreads + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    a[k] = seed * (t + 2u * k + 1u);
    b[k] = seed ^ (0x01000193u * (k + 1));
    c[k] = (seed + 3u * k) | 0x01010101u;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) {
        if constexpr (OP == XT_RATE_MIX) {
          a[k] = mix_step(a[k], b[k], c[k], k);
        } else {
          a[k] = op_step<OP>(a[k], b[k], c[k], k);
        }
        opaque(a[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      opaque(b[k]);
      opaque(c[k]);
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x ^= a[k];
  if (x == seed + 0x9E3779B9u) sink[blockIdx.x] = x;  // keeps the chains live
}

// The packed cell update of the one-lane engine on registers: 8 row pairs
// (16 cells) per step, N-base select included, as the engine's fast step.
__global__ void __launch_bounds__(xt::kLaneThreads) k_rate_cell(uint32_t seed, int iters,
                                                              uint32_t* sink) {
  constexpr int R = 8;
  const uint32_t t = blockIdx.x * xt::kLaneThreads + threadIdx.x;
  uint32_t Hl[R], HAl[R], El[R], K[R], sel[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    Hl[r] = (seed * (t + r)) & 0x00FF00FFu;
    HAl[r] = Hl[r] - 0x00070007u;
    El[r] = 0;
    K[r] = 0x80008000u;
    const uint32_t bl = (t + r) & 3u, bh = 4u + ((t >> 2) + r & 3u);
    sel[r] = bl | ((bl | 8u) << 4) | (bh << 8) | ((bh | 8u) << 12);
  }
  uint32_t prof_lo = 0x01FCFCFCu ^ (seed & 0x00000300u), prof_hi = 0xFC01FCFCu;
  const uint32_t nn2 = 0xFFFFFFFFu, na2 = 0xFFF9FFF9u, nb2 = 0xFFFFFFFFu, mcm = 2u;
  uint32_t D = seed & 0x001F001Fu, Hup = D, Fup = 0, pos2 = 0;
  for (int it = 0; it < iters; ++it) {
    uint32_t oH, oF;
    xt::lane_step_p16<R, false, true, false>(Hl, HAl, El, K, sel, prof_lo, prof_hi, nn2, D, Hup,
                                             Fup, pos2, na2, nb2, mcm, 0u, 0u, oH, oF);
    D = Hup;
    Hup = oH;
    Fup = oF;
    pos2 = (pos2 + 0x00010001u) & 0x003F003Fu;
    const uint32_t p = prof_lo;
    prof_lo = prof_hi;
    prof_hi = p;
    opaque(prof_lo);
    opaque(prof_hi);
  }
  uint32_t x = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) x ^= Hl[r] ^ K[r] ^ El[r];
  if (x == seed + 0x9E3779B9u) sink[blockIdx.x] = x;
}

template <int OP>
cudaError_t launch_rate(int grid, int iters, uint32_t seed, uint32_t* sink, cudaStream_t st) {
  k_rate<OP><<<grid, kRateThreads, 0, st>>>(seed, iters, sink);
  return cudaGetLastError();
}

cudaError_t launch_op(int op, int grid, int iters, uint32_t seed, uint32_t* sink,
                      cudaStream_t st) {
  switch (op) {
    case XT_RATE_ADD16X2: return launch_rate<XT_RATE_ADD16X2>(grid, iters, seed, sink, st);
    case XT_RATE_MAX3_16X2: return launch_rate<XT_RATE_MAX3_16X2>(grid, iters, seed, sink, st);
    case XT_RATE_ADDMAX_16X2: return launch_rate<XT_RATE_ADDMAX_16X2>(grid, iters, seed, sink, st);
    case XT_RATE_PRMT: return launch_rate<XT_RATE_PRMT>(grid, iters, seed, sink, st);
    case XT_RATE_IADD3: return launch_rate<XT_RATE_IADD3>(grid, iters, seed, sink, st);
    case XT_RATE_MAX3_32: return launch_rate<XT_RATE_MAX3_32>(grid, iters, seed, sink, st);
    case XT_RATE_IMAD: return launch_rate<XT_RATE_IMAD>(grid, iters, seed, sink, st);
    case XT_RATE_MIX: return launch_rate<XT_RATE_MIX>(grid, iters, seed, sink, st);
    case XT_RATE_HMAX2: return launch_rate<XT_RATE_HMAX2>(grid, iters, seed, sink, st);
    case XT_RATE_CELL_P16:
      k_rate_cell<<<grid, xt::kLaneThreads, 0, st>>>(seed, iters, sink);
      return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

}  // namespace

extern "C" xt_status xt_int_rate(int device, int op, int reps, int64_t* units, double* ms) {
  if (!units || !ms || op < 0 || op > XT_RATE_HMAX2 || reps < 1) return XT_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return XT_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return XT_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const bool cell = op == XT_RATE_CELL_P16;
  // a full SM of warps for the instruction probes (8 x 256 threads); the cell
  // probe at the engine's own shape (4 CTAs of 128 threads per SM)
  const int threads = cell ? xt::kLaneThreads : kRateThreads;
  const int grid = sms * (cell ? 4 : 2048 / kRateThreads);
  const int iters = cell ? 20000 : 8192;
  const int64_t per_thread = cell ? (int64_t)iters * 16 : (int64_t)iters * kUnroll * kChains;
  uint32_t* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  xt_status s = XT_OK;
  float best = -1.f;
  if (cudaMalloc(&sink, sizeof(uint32_t) * (size_t)grid) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    s = XT_ECUDA;
  } else if (launch_op(op, grid, iters, 0x2301u, sink, st) != cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess) {
    s = XT_ECUDA;  // warm-up launch
  } else {
    for (int r = 0; r < reps && s == XT_OK; ++r) {
      float t = 0.f;
      if (cudaEventRecord(e0, st) != cudaSuccess ||
          launch_op(op, grid, iters, 0x2301u + r, sink, st) != cudaSuccess ||
          cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
        s = XT_ECUDA;
      } else if (best < 0.f || t < best) {
        best = t;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  cudaGetLastError();
  cudaSetDevice(prev);
  if (s != XT_OK) return s;
  *units = per_thread * threads * (int64_t)grid;
  *ms = best;
  return XT_OK;
}
