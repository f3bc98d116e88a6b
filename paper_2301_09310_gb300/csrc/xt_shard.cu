// xt_shard.cu -- splitting a batch over several devices (host code).
//
// Pairs are independent, so a run on several GPUs partitions them with no
// exchange between the parts beyond collecting results (the paper's remark
// on multiple GPUs, Sec. VII-C).  The parts should take equal time, and a
// pair's time follows its cells, so the split is longest-processing-time
// first (LPT) on an estimate of each pair's cells: pairs in decreasing order
// of the estimate, each to the part with the least estimated work so far.
// LPT's makespan is within 4/3 - 1/(3m) of the optimum for m parts, and with
// the many small pairs of a read batch it is balanced to within a pair.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <queue>
#include <vector>

#include "xt.h"
#include "xt_common.cuh"

namespace {

// In-band cells of a whole pair with no z-drop: every row whose band holds a
// column (rows i < min(tlen, qlen + w)), the same count the kernels report
// for a pair that stays live to its last row.
int64_t estimated_cells(int32_t qlen, int32_t tlen, int64_t w) {
  if (qlen <= 0 || tlen <= 0) return 0;
  const int64_t last = std::min<int64_t>(tlen, (int64_t)qlen + w) - 1;
  return xt::band_cells_upto(last, qlen, w);
}

}  // namespace

extern "C" xt_status xt_shard_lpt(const int32_t* q_len, const int32_t* t_len, int32_t n_pairs,
                                  int32_t w, int32_t parts, int32_t* shard, int64_t* part_cells) {
  if (n_pairs < 0 || w < 0 || parts < 1 || parts > 4096) return XT_EINVAL;
  if (n_pairs > 0 && (!q_len || !t_len || !shard)) return XT_EINVAL;
  const int64_t wc = std::min<int64_t>(w, 2 * (int64_t)XT_MAX_LEN);
  std::vector<int64_t> est((size_t)n_pairs);
  for (int32_t k = 0; k < n_pairs; ++k) {
    const int32_t ql = std::min(std::max(q_len[k], 0), XT_MAX_LEN);
    const int32_t tl = std::min(std::max(t_len[k], 0), XT_MAX_LEN);
    est[k] = estimated_cells(ql, tl, wc);
  }
  // decreasing estimate, ties by pair index: the same split on every rank
  std::vector<int32_t> order((size_t)n_pairs);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return est[a] != est[b] ? est[a] > est[b] : a < b;
  });
  // least-loaded part first, ties by part index
  using Load = std::pair<int64_t, int32_t>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int32_t p = 0; p < parts; ++p) heap.push({0, p});
  std::vector<int64_t> load((size_t)parts, 0);
  for (int32_t k : order) {
    const Load top = heap.top();
    heap.pop();
    shard[k] = top.second;
    load[top.second] = top.first + est[k];
    heap.push({load[top.second], top.second});
  }
  if (part_cells)
    for (int32_t p = 0; p < parts; ++p) part_cells[p] = load[p];
  return XT_OK;
}
