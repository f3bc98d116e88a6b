// xt_common.cuh -- device-side definitions shared by the extension kernels.
//
// Notation follows arXiv 2301.09310 Eq. 1: rows i are target bases, columns j
// query bases, alpha = gap_open + gap_extend opens a gap, beta = gap_extend
// extends it.  The seed-extension reading (seed cell h0, boundary gap runs,
// band, anchoring, z-drop) is stated in include/xt.h.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "xt.h"

namespace xt {

// Per-call scoring constants as the kernels use them.
struct Score {
  int32_t alpha;    // gap_open + gap_extend
  int32_t beta;     // gap_extend
  int32_t w;        // band half-width, clamped to [0, 2 * XT_MAX_LEN]
  int32_t zdrop;    // <= 0: disabled
  uint32_t prof[5]; // prof[qc]: byte b (b = 0..3) = S(target b, query qc) as int8; prof[4] = all n
  uint32_t nnnn;    // n_score in all four bytes (target N)
};

// Raw batch arguments as received at the C ABI (device pointers).
struct Batch {
  const uint8_t* q_seq;
  const uint8_t* t_seq;
  const int64_t* q_off;
  const int64_t* t_off;
  const int32_t* q_len;
  const int32_t* t_len;
  const int32_t* h0;
  int64_t q_bytes;
  int64_t t_bytes;
  int32_t n;
  xt_result* out;
  int64_t* cells;  // may be null
};

// One pair as the DP engine sees it.
struct Pair {
  const uint8_t* q;
  const uint8_t* t;
  int32_t qlen, tlen, h0;
};

// Final state of one extension.
struct Outcome {
  int32_t score, qle, tle, gscore, gtle, max_off;
  int64_t cells;
};

// Sign-extended byte select: byte (sel & 7) of {a: bytes 0-3, b: bytes 4-7}
// into byte 0, its sign replicated into bytes 1-3 (PTX prmt default mode).
__device__ __forceinline__ int32_t prmt_s8(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  return static_cast<int32_t>(r);
}

// Selector that picks byte `code` (0..3 from the query profile, 4 = N) and
// sign-extends it to 32 bits.
__device__ __forceinline__ uint32_t score_selector(uint32_t code) {
  const uint32_t s = code | 8u;
  return code | (s << 4) | (s << 8) | (s << 12);
}

__device__ __forceinline__ uint32_t clamp_code(uint32_t b) { return b < 4u ? b : 4u; }

// H (= F) of boundary column cell (i, -1): a deletion run of i+1 target bases
// from the seed, in band only while i + 1 <= w.
__device__ __forceinline__ int32_t col_m1(int32_t i, int32_t h0, const Score& sc) {
  if (i + 1 > sc.w) return 0;
  const int32_t v = h0 - sc.alpha - sc.beta * i;
  return v > 0 ? v : 0;
}

// H (= E) of boundary row cell (-1, c): an insertion run of c+1 query bases.
__device__ __forceinline__ int32_t row_m1(int32_t c, int32_t h0, const Score& sc) {
  if (c + 1 > sc.w) return 0;
  const int32_t v = h0 - sc.alpha - sc.beta * c;
  return v > 0 ? v : 0;
}

// Sum of in-band widths of rows 0..n (n < qlen + w, so every width is > 0):
//   sum_i min(qlen, i + w + 1) - sum_i max(0, i - w).
__host__ __device__ __forceinline__ int64_t band_cells_upto(int64_t n, int64_t qlen, int64_t w) {
  if (n < 0) return 0;
  int64_t a;
  const int64_t k = qlen - w - 1;  // rows i <= k have i + w + 1 <= qlen
  if (k < 0) {
    a = (n + 1) * qlen;
  } else if (n <= k) {
    a = (n + 1) * (w + 1) + n * (n + 1) / 2;
  } else {
    a = (k + 1) * (w + 1) + k * (k + 1) / 2 + (n - k) * qlen;
  }
  const int64_t m = n - w;
  const int64_t b = m > 0 ? m * (m + 1) / 2 : 0;
  return a - b;
}

__device__ __forceinline__ void write_result(const Batch& b, int32_t k, int32_t score, int32_t qle,
                                             int32_t tle, int32_t gscore, int32_t gtle,
                                             int32_t max_off, int32_t status, int64_t cells) {
  xt_result r;
  r.score = score; r.qle = qle; r.tle = tle; r.gscore = gscore; r.gtle = gtle;
  r.max_off = max_off; r.status = status;
  b.out[k] = r;
  if (b.cells) b.cells[k] = cells;
}

// Row-order bookkeeping of one extension: local best, z-drop, end-to-end
// score and the last live row.  Fed one row summary at a time, in row order.
struct RowState {
  int32_t best, bi, bj, max_off, gscore, gtle, last_live;
  bool stop;

  __device__ __forceinline__ void init(int32_t h0) {
    best = h0; bi = -1; bj = -1; max_off = 0; gscore = -1; gtle = 0; last_live = -1; stop = false;
  }

  // Row i with maximum m (0 if dead), mj its largest column (-1 when the row
  // has no in-band cell) and g = H(i, qlen-1) when that cell is in band, else -1.
  __device__ __forceinline__ void feed(int32_t i, int32_t m, int32_t mj, int32_t g,
                                       const Score& sc) {
    if (m > 0) last_live = i;
    if (g > 0 && g > gscore) { gscore = g; gtle = i + 1; }
    if (m > best) {
      best = m; bi = i; bj = mj;
      const int32_t off = mj > i ? mj - i : i - mj;
      max_off = off > max_off ? off : max_off;
    } else if (sc.zdrop > 0) {
      const int64_t d = (int64_t)(i - bi) - (int64_t)(mj - bj);
      const int64_t drop = (int64_t)best - m - (d < 0 ? -d : d) * (int64_t)sc.beta;
      if (drop > sc.zdrop) stop = true;
    }
  }
};

}  // namespace xt
