// xt_serve.cpp -- the serving loop of include/xt.h: requests of host pairs,
// continuously batched onto the batched extension path.
//
// One server thread owns every CUDA call.  Each slot is an independent
// context with its own stream, pinned staging buffer and device buffers, so
// the gather and the copies of one batch overlap the kernels of another.  A
// stream host callback wakes the thread when a slot's batch is complete (the
// thread also polls the slot's event, so a failed stream cannot stall it).
// Client threads only touch the waiting queue and the ticket table, under
// one mutex that is never held across a CUDA call.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>
#include <time.h>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "xt.h"

namespace xt {
// sizes a context's device buffers once for calls of up to n_pairs pairs (xt_api.cu)
xt_status ctx_reserve(xt_ctx* ctx, int32_t n_pairs, size_t conv_bytes, size_t pool_bytes);
}  // namespace xt

namespace {

constexpr int64_t kPairInBytes = 28;   // staged per pair: q_off, t_off (int64), q_len, t_len, h0
constexpr size_t kAlign = 256;
constexpr int kRegions = 7;            // staged regions, each 256-byte aligned
constexpr int kMaxSlots = 8;
constexpr int32_t kMaxBatchPairsCap = 1 << 24;
constexpr int kMaxGatherThreads = 16;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int64_t mono_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

// Staged bytes of a batch of `pairs` pairs and `seq` sequence bytes
// (upper bound: every region padded to the alignment).
int64_t staged_bytes(int64_t pairs, int64_t seq) {
  return pairs * kPairInBytes + seq + kRegions * (int64_t)kAlign;
}

// Result bytes of a batch of n pairs: xt_result[n], then int64 cells[n].
size_t result_bytes(int64_t n) { return align_up((size_t)n * sizeof(xt_result)) + (size_t)n * 8; }

struct Request {
  const uint8_t* q_seq; int64_t q_bytes; const int64_t* q_off; const int32_t* q_len;
  const uint8_t* t_seq; int64_t t_bytes; const int64_t* t_off; const int32_t* t_len;
  const int32_t* h0; int32_t n; xt_scoring sc;
  xt_result* out; int64_t* cells;
  int64_t staged = 0;
  xt_serve_times times{};
  bool done = false;
};
using ReqPtr = std::shared_ptr<Request>;

// A fixed pool of host threads that runs one parallel loop at a time; the
// calling thread takes part, items are handed out through an atomic counter.
class WorkerPool {
 public:
  explicit WorkerPool(int extra_threads) {
    for (int i = 0; i < extra_threads; ++i) th_.emplace_back([this] { loop(); });
  }
  ~WorkerPool() {
    {
      std::lock_guard<std::mutex> lk(m_);
      quit_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  // body(i) for every i in [0, count); returns when all have run.
  void parallel_for(int64_t count, const std::function<void(int64_t)>& body) {
    if (th_.empty() || count <= 1) {
      for (int64_t i = 0; i < count; ++i) body(i);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(m_);
      job_ = &body;
      count_ = count;
      next_.store(0);
      active_ = (int)th_.size();
      ++gen_;
    }
    cv_.notify_all();
    drain();
    std::unique_lock<std::mutex> lk(m_);
    cv_done_.wait(lk, [&] { return active_ == 0; });
    job_ = nullptr;
  }

 private:
  void drain() {
    for (;;) {
      const int64_t i = next_.fetch_add(1);
      if (i >= count_) break;
      (*job_)(i);
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return quit_ || gen_ != seen; });
        if (quit_) return;
        seen = gen_;
      }
      drain();
      std::lock_guard<std::mutex> lk(m_);
      if (--active_ == 0) cv_done_.notify_one();
    }
  }
  std::vector<std::thread> th_;
  std::mutex m_;
  std::condition_variable cv_, cv_done_;
  const std::function<void(int64_t)>* job_ = nullptr;
  int64_t count_ = 0;
  std::atomic<int64_t> next_{0};
  int active_ = 0;
  uint64_t gen_ = 0;
  bool quit_ = false;
};

struct Slot {
  xt_server* srv = nullptr;
  xt_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t start_ev = nullptr;
  cudaEvent_t done_ev = nullptr;
  int64_t gather_ns = 0;
  uint8_t* h_in = nullptr;
  uint8_t* d_in = nullptr;
  uint8_t* h_out = nullptr;
  uint8_t* d_out = nullptr;
  std::vector<ReqPtr> reqs;   // the batch in flight, in staging order
  int32_t n = 0;
  // server thread only: FREE, or RUN (the batch enqueued up to its results)
  enum State { FREE, RUN } state = FREE;
  bool signalled = false;     // set by the host callback, consumed by the server thread (mutex)
  xt_status status = XT_OK;   // error raised while enqueuing the batch
};

}  // namespace

struct xt_server {
  int device = 0;
  xt_serve_config cfg{};
  int64_t in_cap = 0;         // staging bytes per slot
  std::vector<std::unique_ptr<Slot>> slots;
  std::mutex mu;
  std::condition_variable cv_work;  // the server thread: request, completion, stop
  std::condition_variable cv_done;  // waiters
  std::deque<ReqPtr> waiting;
  int64_t waiting_bytes = 0;
  std::unordered_map<uint64_t, ReqPtr> tickets;
  uint64_t next_ticket = 1;
  bool stop = false;
  bool paused = false;
  xt_serve_stats stats{};
  std::unique_ptr<WorkerPool> gather;  // staging threads besides the server thread
  std::thread th;
};

namespace {

void CUDART_CB slot_done(void* p) {
  Slot* s = static_cast<Slot*>(p);
  {
    std::lock_guard<std::mutex> lk(s->srv->mu);
    s->signalled = true;
  }
  s->srv->cv_work.notify_one();
}

// Take the next batch from the waiting queue (caller holds the mutex):
// requests in arrival order with the oldest request's scoring, while the
// slot's pair and byte capacities hold.  Requests of another scoring keep
// their place.
std::vector<ReqPtr> take_batch(xt_server* S) {
  std::vector<ReqPtr> batch;
  if (S->waiting.empty()) return batch;
  const xt_scoring sc = S->waiting.front()->sc;
  int64_t n = 0, seq = 0;
  std::deque<ReqPtr> rest;
  bool full = false;
  for (auto& r : S->waiting) {
    const bool same = std::memcmp(&r->sc, &sc, sizeof(sc)) == 0;
    if (!full && same) {
      const int64_t n2 = n + r->n, seq2 = seq + r->q_bytes + r->t_bytes;
      if (n2 <= S->cfg.max_batch_pairs && staged_bytes(n2, seq2) <= S->in_cap) {
        batch.push_back(r);
        n = n2;
        seq = seq2;
        S->waiting_bytes -= r->staged;
        continue;
      }
      full = true;  // keep arrival order among requests of this scoring
    }
    rest.push_back(r);
  }
  S->waiting.swap(rest);
  return batch;
}

// The completion event and callback come last, whatever happened before.
void end_batch(Slot& s) {
  cudaError_t e = cudaEventRecord(s.done_ev, s.stream);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(s.stream, slot_done, &s);
  if (e != cudaSuccess && s.status == XT_OK) s.status = XT_ECUDA;
  s.state = Slot::RUN;
}

// Gather a batch into the slot's staging buffer and enqueue copy in,
// extension, copy out, event and callback on the slot's stream.
void launch_batch(xt_server* S, Slot& s) {
  int64_t n = 0, Q = 0, T = 0;
  for (auto& r : s.reqs) {
    n += r->n;
    Q += r->q_bytes;
    T += r->t_bytes;
  }
  const size_t o_qoff = 0;
  const size_t o_toff = align_up(o_qoff + 8 * (size_t)n);
  const size_t o_qlen = align_up(o_toff + 8 * (size_t)n);
  const size_t o_tlen = align_up(o_qlen + 4 * (size_t)n);
  const size_t o_h0 = align_up(o_tlen + 4 * (size_t)n);
  const size_t o_qseq = align_up(o_h0 + 4 * (size_t)n);
  const size_t o_tseq = align_up(o_qseq + (size_t)Q);
  const size_t in_bytes = o_tseq + (size_t)T;
  const int64_t g0 = mono_ns();
  uint8_t* h = s.h_in;
  int64_t* qoff = reinterpret_cast<int64_t*>(h + o_qoff);
  int64_t* toff = reinterpret_cast<int64_t*>(h + o_toff);
  // where each request lands in the batch, then the requests in parallel
  struct Place {
    int64_t k, qb, tb;
  };
  std::vector<Place> place(s.reqs.size());
  int64_t k = 0, qb = 0, tb = 0;
  for (size_t i = 0; i < s.reqs.size(); ++i) {
    place[i] = {k, qb, tb};
    k += s.reqs[i]->n;
    qb += s.reqs[i]->q_bytes;
    tb += s.reqs[i]->t_bytes;
  }
  S->gather->parallel_for((int64_t)s.reqs.size(), [&](int64_t ri) {
    const Request* r = s.reqs[ri].get();
    const int64_t k = place[ri].k, qb = place[ri].qb, tb = place[ri].tb;
    if (r->q_bytes) std::memcpy(h + o_qseq + qb, r->q_seq, (size_t)r->q_bytes);
    if (r->t_bytes) std::memcpy(h + o_tseq + tb, r->t_seq, (size_t)r->t_bytes);
    std::memcpy(h + o_qlen + 4 * k, r->q_len, 4 * (size_t)r->n);
    std::memcpy(h + o_tlen + 4 * k, r->t_len, 4 * (size_t)r->n);
    std::memcpy(h + o_h0 + 4 * k, r->h0, 4 * (size_t)r->n);
    // rebase offsets into the batch; a sequence outside its own request's
    // buffer gets offset -1, which the classify pass reports as XT_EINVAL
    for (int32_t i = 0; i < r->n; ++i) {
      const int64_t qo = r->q_off[i], to = r->t_off[i];
      const int64_t ql = r->q_len[i], tl = r->t_len[i];
      qoff[k + i] = (qo >= 0 && ql >= 0 && qo <= r->q_bytes && ql <= r->q_bytes - qo) ? qo + qb : -1;
      toff[k + i] = (to >= 0 && tl >= 0 && to <= r->t_bytes && tl <= r->t_bytes - to) ? to + tb : -1;
    }
  });
  s.gather_ns = mono_ns() - g0;
  s.n = (int32_t)n;
  s.status = XT_OK;
  uint8_t* d = s.d_in;
  xt_result* d_res = reinterpret_cast<xt_result*>(s.d_out);
  int64_t* d_cells = reinterpret_cast<int64_t*>(s.d_out + align_up((size_t)n * sizeof(xt_result)));
  cudaError_t e = cudaEventRecord(s.start_ev, s.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, h, in_bytes, cudaMemcpyHostToDevice, s.stream);
  if (e == cudaSuccess) {
    // The one-step call: the thread waits for this batch's classify pass
    // before it plans the extension kernels.  Letting the thread go on (the
    // two-step xt_extend_batch_begin / _finish) let up to `slots` batches'
    // extension kernels share the GPU at once, and measured worse on a
    // 4M-pair stream: p99 latency up from 11.7 to 18.0 ms at 25% load and
    // 26.3M down to 21.3M pairs/s sustained at 90%.
    const xt_status st = xt_extend_batch(
        s.ctx, d + o_qseq, Q, reinterpret_cast<const int64_t*>(d + o_qoff),
        reinterpret_cast<const int32_t*>(d + o_qlen), d + o_tseq, T,
        reinterpret_cast<const int64_t*>(d + o_toff), reinterpret_cast<const int32_t*>(d + o_tlen),
        reinterpret_cast<const int32_t*>(d + o_h0), (int32_t)n, &s.reqs.front()->sc, d_res, d_cells,
        s.stream);
    if (st != XT_OK) s.status = st;
  } else {
    s.status = XT_ECUDA;
  }
  if (s.status == XT_OK) {
    e = cudaMemcpyAsync(s.h_out, s.d_out, result_bytes(n), cudaMemcpyDeviceToHost, s.stream);
    if (e != cudaSuccess) s.status = XT_ECUDA;
  }
  end_batch(s);
}

// Publish a finished slot's results to its requests.
void finish_batch(xt_server* S, Slot& s, cudaError_t e) {
  xt_status status = s.status;
  if (status == XT_OK && e != cudaSuccess) status = XT_ECUDA;
  int64_t cells = 0;
  if (status == XT_OK) {
    const xt_result* res = reinterpret_cast<const xt_result*>(s.h_out);
    const int64_t* c = reinterpret_cast<const int64_t*>(
        s.h_out + align_up((size_t)s.n * sizeof(xt_result)));
    int64_t pos = 0;
    for (auto& r : s.reqs) {
      std::memcpy(r->out, res + pos, (size_t)r->n * sizeof(xt_result));
      if (r->cells) std::memcpy(r->cells, c + pos, (size_t)r->n * 8);
      pos += r->n;
    }
    for (int64_t i = 0; i < pos; ++i) cells += c[i];
  }
  float dev_ms = 0.f;
  if (status == XT_OK && cudaEventElapsedTime(&dev_ms, s.start_ev, s.done_ev) != cudaSuccess) {
    cudaGetLastError();
    dev_ms = 0.f;
  }
  const int64_t t = mono_ns();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto& r : s.reqs) {
      r->times.done_ns = t;
      r->times.status = status;
      r->done = true;
      S->stats.requests += 1;
      S->stats.pairs += r->n;
    }
    S->stats.cells += cells;
    S->stats.batches += 1;
    S->stats.gather_ns += s.gather_ns;
    S->stats.device_ns += (int64_t)(dev_ms * 1e6);
    S->stats.in_flight -= 1;
  }
  s.reqs.clear();
  s.state = Slot::FREE;
  S->cv_done.notify_all();
}

void serve_loop(xt_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    // completed batches
    for (auto& sp : S->slots) {
      Slot& s = *sp;
      if (s.state != Slot::RUN) continue;
      const cudaError_t e = cudaEventQuery(s.done_ev);
      if (e == cudaErrorNotReady) continue;
      finish_batch(S, s, e);
    }
    // new batches on free slots
    for (auto& sp : S->slots) {
      Slot& s = *sp;
      if (s.state != Slot::FREE) continue;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->paused || S->waiting.empty()) break;
        s.reqs = take_batch(S);
        if (s.reqs.empty()) break;
        const int64_t t = mono_ns();
        int64_t n = 0;
        for (auto& r : s.reqs) n += r->n;
        for (auto& r : s.reqs) {
          r->times.launch_ns = t;
          r->times.batch_pairs = (int32_t)n;
        }
        S->stats.in_flight += 1;
      }
      launch_batch(S, s);
    }
    // sleep until something can move
    std::unique_lock<std::mutex> lk(S->mu);
    bool busy = false, signalled = false, free_slot = false;
    for (auto& sp : S->slots) {
      busy |= sp->state != Slot::FREE;
      free_slot |= sp->state == Slot::FREE;
      // consume the flag: a callback of a slot's previous batch may arrive
      // after that batch was already reaped through its event
      signalled |= sp->signalled;
      sp->signalled = false;
    }
    const bool can_launch = free_slot && !S->paused && !S->waiting.empty();
    if (S->stop && S->waiting.empty() && !busy) break;
    if (S->stop && S->paused) S->paused = false;
    if (can_launch || signalled) continue;
    // a completion, a request or stop notifies; the timeout polls the events
    S->cv_work.wait_for(lk, std::chrono::microseconds(busy ? 2000 : 50000));
  }
}

void free_slot(Slot& s) {
  if (s.stream) cudaStreamSynchronize(s.stream);
  if (s.ctx) xt_ctx_destroy(s.ctx);
  if (s.h_in) cudaFreeHost(s.h_in);
  if (s.h_out) cudaFreeHost(s.h_out);
  if (s.d_in) cudaFree(s.d_in);
  if (s.d_out) cudaFree(s.d_out);
  if (s.start_ev) cudaEventDestroy(s.start_ev);
  if (s.done_ev) cudaEventDestroy(s.done_ev);
  if (s.stream) cudaStreamDestroy(s.stream);
  s = Slot();
}

void free_server(xt_server* S) {
  for (auto& sp : S->slots) free_slot(*sp);
  delete S;
}

}  // namespace

extern "C" {

int64_t xt_now_ns(void) { return mono_ns(); }

xt_status xt_serve_create(xt_server** out, int device, const xt_serve_config* cfg_in) {
  if (!out) return XT_EINVAL;
  *out = nullptr;
  xt_serve_config cfg{};
  if (cfg_in) cfg = *cfg_in;
  // defaults: two slots of 1 GiB (c5 stream at 90% of the batched peak: 43.2-43.8M pairs/s,
  // p99 57-62 ms, against 38.4M and 84 ms with three slots of 256 MiB)
  if (cfg.slots == 0) cfg.slots = 2;
  if (cfg.max_batch_pairs == 0) cfg.max_batch_pairs = 1 << 20;
  if (cfg.max_batch_bytes == 0) cfg.max_batch_bytes = (int64_t)1 << 30;
  if (cfg.max_queued_bytes == 0) cfg.max_queued_bytes = (int64_t)1 << 30;
  if (cfg.gather_threads == 0) {
    const int hw = (int)std::thread::hardware_concurrency();
    cfg.gather_threads = std::max(1, std::min(kMaxGatherThreads / 2, hw / 4));
  }
  if (cfg.slots < 1 || cfg.slots > kMaxSlots || cfg.max_batch_pairs < 1 ||
      cfg.max_batch_pairs > kMaxBatchPairsCap || cfg.max_batch_bytes < 4096 ||
      cfg.max_queued_bytes < 1 || cfg.gather_threads < 1 || cfg.gather_threads > kMaxGatherThreads)
    return XT_EINVAL;
  // requests are gathered byte by byte: codes or ASCII letters, not 4-bit codes
  if (cfg.alphabet != XT_ALPHABET_CODES && cfg.alphabet != XT_ALPHABET_ASCII) return XT_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return XT_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return XT_ECUDA;
  xt_server* S = new xt_server();
  S->device = device;
  S->cfg = cfg;
  S->in_cap = cfg.max_batch_bytes + kRegions * (int64_t)kAlign;
  const size_t out_cap = result_bytes(cfg.max_batch_pairs);
  const size_t slot_buf = (size_t)S->in_cap + out_cap;
  size_t ctx_budget = 0;
  if (cfg.mem_budget_bytes) {
    if (cfg.mem_budget_bytes <= slot_buf * cfg.slots) {
      delete S;
      return XT_ENOMEM;
    }
    ctx_budget = (cfg.mem_budget_bytes - slot_buf * cfg.slots) / cfg.slots;
  }
  for (int i = 0; i < cfg.slots; ++i) {
    S->slots.push_back(std::make_unique<Slot>());
    Slot& s = *S->slots.back();
    s.srv = S;
    xt_status st = xt_ctx_create(&s.ctx, device, ctx_budget);
    // direct launches: batches of a stream have many different plans, and a
    // graph captured on the second batch of each one put capture time into
    // the latency of that batch (c5 stream at 25% load: p99 9.0-9.1 ms
    // without graphs, 9.1-16.6 ms with them; throughput unchanged)
    if (st == XT_OK) st = xt_ctx_set_graphs(s.ctx, 0);
    if (st == XT_OK && cfg.tuning_path) st = xt_ctx_load_tuning(s.ctx, cfg.tuning_path);
    if (st == XT_OK) st = xt_ctx_set_alphabet(s.ctx, cfg.alphabet);
    // every buffer a batch can need, sized now: regrowing one mid-stream frees
    // the old buffer, and a cudaFree waits for the other slots' work
    // (ring pool: 1 GB holds the global rings of the c5 mix's plans, about
    // 0.6 GB at most)
    if (st == XT_OK)
      st = xt::ctx_reserve(s.ctx, cfg.max_batch_pairs,
                           cfg.alphabet == XT_ALPHABET_ASCII ? (size_t)S->in_cap + 4096 : 0,
                           (size_t)1 << 30);
    cudaError_t e = st == XT_OK ? cudaSuccess : cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s.start_ev);
    if (e == cudaSuccess) e = cudaEventCreate(&s.done_ev);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_in, (size_t)S->in_cap);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_out, out_cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s.d_in, (size_t)S->in_cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s.d_out, out_cap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_server(S);
      return st != XT_OK ? st : (e == cudaErrorMemoryAllocation ? XT_ENOMEM : XT_ECUDA);
    }
  }
  S->gather = std::make_unique<WorkerPool>(cfg.gather_threads - 1);
  S->th = std::thread(serve_loop, S);
  *out = S;
  return XT_OK;
}

xt_status xt_serve_submit(xt_server* S, const uint8_t* q_seq, int64_t q_bytes, const int64_t* q_off,
                          const int32_t* q_len, const uint8_t* t_seq, int64_t t_bytes,
                          const int64_t* t_off, const int32_t* t_len, const int32_t* h0,
                          int32_t n, const xt_scoring* sc, xt_result* out, int64_t* cells,
                          uint64_t* ticket) {
  if (!S || !ticket) return XT_EINVAL;
  *ticket = 0;
  if (n < 0 || q_bytes < 0 || t_bytes < 0) return XT_EINVAL;
  if (n > 0 && (!q_off || !q_len || !t_off || !t_len || !h0 || !out)) return XT_EINVAL;
  if ((q_bytes > 0 && !q_seq) || (t_bytes > 0 && !t_seq)) return XT_EINVAL;
  if (xt_scoring_check(sc) != XT_OK) return XT_EINVAL;
  if (n > S->cfg.max_batch_pairs || q_bytes > S->in_cap || t_bytes > S->in_cap) return XT_EINVAL;
  const int64_t staged = staged_bytes(n, q_bytes + t_bytes);
  if (staged > S->in_cap) return XT_EINVAL;
  auto r = std::make_shared<Request>();
  r->q_seq = q_seq; r->q_bytes = q_bytes; r->q_off = q_off; r->q_len = q_len;
  r->t_seq = t_seq; r->t_bytes = t_bytes; r->t_off = t_off; r->t_len = t_len;
  r->h0 = h0; r->n = n; r->sc = *sc; r->out = out; r->cells = cells;
  r->staged = staged;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return XT_EBUSY;
    if (!S->waiting.empty() && S->waiting_bytes + staged > S->cfg.max_queued_bytes)
      return XT_EBUSY;
    r->times.submit_ns = mono_ns();
    *ticket = S->next_ticket++;
    S->tickets[*ticket] = r;
    if (n == 0) {
      r->times.launch_ns = r->times.done_ns = r->times.submit_ns;
      r->times.status = XT_OK;
      r->done = true;
      S->stats.requests += 1;
    } else {
      S->waiting.push_back(r);
      S->waiting_bytes += staged;
    }
  }
  S->cv_work.notify_one();
  return XT_OK;
}

xt_status xt_serve_poll(xt_server* S, uint64_t ticket, int* done) {
  if (!S || !done) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return XT_EINVAL;
  *done = it->second->done ? 1 : 0;
  return XT_OK;
}

xt_status xt_serve_wait(xt_server* S, uint64_t ticket, int64_t timeout_us, xt_serve_times* times) {
  if (!S) return XT_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return XT_EINVAL;
  ReqPtr r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_us < 0) {
    S->cv_done.wait(lk, ready);
  } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
    return XT_ETIMEOUT;
  }
  if (times) *times = r->times;
  S->tickets.erase(ticket);
  return (xt_status)r->times.status;
}

xt_status xt_serve_pause(xt_server* S, int paused) {
  if (!S) return XT_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->paused = paused != 0;
  }
  S->cv_work.notify_one();
  return XT_OK;
}

xt_status xt_serve_get_stats(xt_server* S, xt_serve_stats* out) {
  if (!S || !out) return XT_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  out->waiting = (int64_t)S->waiting.size();
  return XT_OK;
}

xt_status xt_serve_destroy(xt_server* S) {
  if (!S) return XT_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->th.joinable()) S->th.join();
  S->cv_done.notify_all();
  free_server(S);
  return XT_OK;
}

}  // extern "C"
