// xt_tune.cu -- the autotuner of include/xt.h: per length bucket, time every
// available schedule (lanes per pair P, rows per lane R) on synthetic pairs of
// that bucket and keep the fastest; persist the table as JSON keyed by device.
//
// Every timed schedule must also reproduce the first schedule's results bit
// for bit (pairs are independent of the schedule); a mismatch fails the call.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "xt.h"
#include "xt_ctx.cuh"

using namespace xt;

namespace {

// ----------------------------------------------------------------- JSON
// A small reader/writer for the table: objects, arrays, strings, numbers.
struct Json {
  enum Kind { NUL, NUM, STR, ARR, OBJ, BOOL } kind = NUL;
  double num = 0;
  bool b = false;
  std::string str;
  std::vector<Json> arr;
  std::vector<std::pair<std::string, Json>> obj;
  const Json* get(const char* key) const {
    if (kind != OBJ) return nullptr;
    for (auto& kv : obj)
      if (kv.first == key) return &kv.second;
    return nullptr;
  }
};

struct Parser {
  const char* p;
  const char* end;
  bool ok = true;
  void ws() {
    while (p < end && (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t')) ++p;
  }
  bool lit(const char* s) {
    const size_t n = std::strlen(s);
    if ((size_t)(end - p) >= n && std::strncmp(p, s, n) == 0) {
      p += n;
      return true;
    }
    return false;
  }
  std::string string() {
    std::string out;
    ++p;  // opening quote
    while (p < end && *p != '"') {
      if (*p == '\\' && p + 1 < end) {
        ++p;
        switch (*p) {
          case 'n': out += '\n'; break;
          case 't': out += '\t'; break;
          case 'r': out += '\r'; break;
          case 'b': out += '\b'; break;
          case 'f': out += '\f'; break;
          case 'u':  // keep \uXXXX as written: names here are ASCII
            out += "\\u";
            break;
          default: out += *p;
        }
        ++p;
      } else {
        out += *p++;
      }
    }
    if (p >= end) ok = false;
    else ++p;  // closing quote
    return out;
  }
  Json value(int depth = 0) {
    Json v;
    ws();
    if (p >= end || depth > 32) {
      ok = false;
      return v;
    }
    if (*p == '{') {
      v.kind = Json::OBJ;
      ++p;
      ws();
      if (p < end && *p == '}') { ++p; return v; }
      while (ok) {
        ws();
        if (p >= end || *p != '"') { ok = false; break; }
        std::string k = string();
        ws();
        if (p >= end || *p != ':') { ok = false; break; }
        ++p;
        v.obj.emplace_back(k, value(depth + 1));
        ws();
        if (p < end && *p == ',') { ++p; continue; }
        if (p < end && *p == '}') { ++p; break; }
        ok = false;
      }
    } else if (*p == '[') {
      v.kind = Json::ARR;
      ++p;
      ws();
      if (p < end && *p == ']') { ++p; return v; }
      while (ok) {
        v.arr.push_back(value(depth + 1));
        ws();
        if (p < end && *p == ',') { ++p; continue; }
        if (p < end && *p == ']') { ++p; break; }
        ok = false;
      }
    } else if (*p == '"') {
      v.kind = Json::STR;
      v.str = string();
    } else if (lit("true")) {
      v.kind = Json::BOOL; v.b = true;
    } else if (lit("false")) {
      v.kind = Json::BOOL; v.b = false;
    } else if (lit("null")) {
      v.kind = Json::NUL;
    } else {
      char* q = nullptr;
      std::string tok(p, std::min<size_t>(64, (size_t)(end - p)));
      v.num = std::strtod(tok.c_str(), &q);
      if (q == tok.c_str()) { ok = false; return v; }
      v.kind = Json::NUM;
      p += (q - tok.c_str());
    }
    return v;
  }
};

bool read_file(const char* path, std::string* out) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  char buf[65536];
  size_t n;
  out->clear();
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) out->append(buf, n);
  std::fclose(f);
  return true;
}

bool parse_file(const char* path, Json* root) {
  std::string text;
  if (!read_file(path, &text)) return false;
  Parser ps{text.data(), text.data() + text.size()};
  *root = ps.value();
  ps.ws();
  return ps.ok && ps.p == ps.end && root->kind == Json::OBJ;
}

std::string quote(const std::string& s) {
  std::string o = "\"";
  for (char c : s) {
    if (c == '"' || c == '\\') o += '\\';
    o += c;
  }
  return o + "\"";
}

// One table entry: the device it was tuned on, the band, the scoring used and
// the chosen schedule (with its measured rate) of every tuned bucket.
struct Entry {
  std::string device;
  int sms = 0;
  int w = 0;
  xt_scoring sc{};
  struct B {
    int j, P, R;
    double gcups;
    int Ps, Rs;  // small-batch schedule (0: none)
    double gcups_s;
  };
  std::vector<B> buckets;
};

bool entry_from_json(const Json& e, Entry* out) {
  const Json *dev = e.get("device"), *sms = e.get("sms"), *w = e.get("w"), *bk = e.get("buckets");
  if (!dev || dev->kind != Json::STR || !sms || sms->kind != Json::NUM || !w ||
      w->kind != Json::NUM || !bk || bk->kind != Json::ARR)
    return false;
  out->device = dev->str;
  out->sms = (int)sms->num;
  out->w = (int)w->num;
  if (const Json* sc = e.get("scoring")) {
    if (sc->kind == Json::ARR && sc->arr.size() == 7) {
      int32_t* f = &out->sc.match;
      for (int k = 0; k < 7; ++k) f[k] = (int32_t)sc->arr[k].num;
    }
  }
  for (const Json& b : bk->arr) {
    const Json *j = b.get("j"), *P = b.get("P"), *R = b.get("R"), *g = b.get("gcups");
    if (!j || !P || !R || j->kind != Json::NUM || P->kind != Json::NUM || R->kind != Json::NUM)
      return false;
    const Json *Ps = b.get("Ps"), *Rs = b.get("Rs"), *gs = b.get("gcups_s");
    const bool small = Ps && Rs && Ps->kind == Json::NUM && Rs->kind == Json::NUM;
    out->buckets.push_back({(int)j->num, (int)P->num, (int)R->num, g ? g->num : 0.0,
                            small ? (int)Ps->num : 0, small ? (int)Rs->num : 0,
                            gs ? gs->num : 0.0});
  }
  return true;
}

std::string entry_to_json(const Entry& e) {
  char buf[256];
  std::string s = "    {\"device\": " + quote(e.device);
  std::snprintf(buf, sizeof(buf), ", \"sms\": %d, \"w\": %d,\n     \"scoring\": [%d, %d, %d, %d, %d, %d, %d],\n     \"buckets\": [",
                e.sms, e.w, e.sc.match, e.sc.mismatch, e.sc.gap_open, e.sc.gap_extend, e.sc.w,
                e.sc.zdrop, e.sc.n_score);
  s += buf;
  for (size_t k = 0; k < e.buckets.size(); ++k) {
    const auto& b = e.buckets[k];
    std::snprintf(buf, sizeof(buf),
                  "%s\n       {\"j\": %d, \"P\": %d, \"R\": %d, \"gcups\": %.3f, "
                  "\"Ps\": %d, \"Rs\": %d, \"gcups_s\": %.3f}",
                  k ? "," : "", b.j, b.P, b.R, b.gcups, b.Ps, b.Rs, b.gcups_s);
    s += buf;
  }
  return s + "]}";
}

bool write_table(const char* path, const std::vector<Entry>& entries) {
  std::string s = "{\"format\": \"xt-tuning\", \"version\": 1,\n  \"entries\": [\n";
  for (size_t k = 0; k < entries.size(); ++k) s += (k ? ",\n" : "") + entry_to_json(entries[k]);
  s += "\n  ]}\n";
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  const bool ok = std::fwrite(s.data(), 1, s.size(), f) == s.size();
  if (std::fclose(f) != 0 || !ok) return false;
  return std::rename(tmp.c_str(), path) == 0;
}

std::vector<Entry> read_entries(const char* path) {
  std::vector<Entry> v;
  Json root;
  if (!parse_file(path, &root)) return v;
  const Json* es = root.get("entries");
  if (!es || es->kind != Json::ARR) return v;
  for (const Json& e : es->arr) {
    Entry x;
    if (entry_from_json(e, &x)) v.push_back(x);
  }
  return v;
}

// ------------------------------------------------------ synthetic pairs
// xorshift64* (Vigna): the tuner's own generator; any mix of lengths works.
struct Rng {
  uint64_t s;
  uint64_t next() {
    s ^= s >> 12;
    s ^= s << 25;
    s ^= s >> 27;
    return s * 0x2545F4914F6CDD1DULL;
  }
  uint32_t below(uint32_t n) { return (uint32_t)((next() >> 32) * (uint64_t)n >> 32); }
};

struct HostPairs {
  std::vector<uint8_t> q, t;
  std::vector<int64_t> qo, to;
  std::vector<int32_t> ql, tl, h0;
};

// n pairs of bucket j: query length uniform over the bucket, target = the
// query's source window plus up to 2w more bases, query = that window with 1%
// substitutions (so the extension runs across the whole band).
void make_pairs(int j, int w, int n, uint64_t seed, HostPairs* hp) {
  const int qlo = j == kJMin ? 1 : (1 << (j - 1)) - 1;
  const int qhi = (1 << j) - 2;
  const int64_t extra_cap = 2 * (int64_t)qhi;
  Rng r{seed * 0x9E3779B97F4A7C15ULL + 1};
  hp->qo.resize(n); hp->to.resize(n); hp->ql.resize(n); hp->tl.resize(n); hp->h0.resize(n);
  int64_t qb = 0, tb = 0;
  for (int k = 0; k < n; ++k) {
    const int ql = qlo + (int)r.below((uint32_t)(qhi - qlo + 1));
    const int tl = ql + (int)std::min<int64_t>(2 * (int64_t)w, extra_cap);
    hp->qo[k] = qb; hp->to[k] = tb; hp->ql[k] = ql; hp->tl[k] = tl; hp->h0[k] = 30;
    qb += ql;
    tb += tl;
  }
  hp->q.resize(qb);
  hp->t.resize(tb);
  for (int k = 0; k < n; ++k) {
    uint8_t* t = hp->t.data() + hp->to[k];
    uint8_t* q = hp->q.data() + hp->qo[k];
    for (int i = 0; i < hp->tl[k]; ++i) t[i] = (uint8_t)r.below(4);
    for (int i = 0; i < hp->ql[k]; ++i)
      q[i] = r.below(100) == 0 ? (uint8_t)((t[i] + 1 + r.below(3)) & 3) : t[i];
  }
}

struct DevPairs {
  uint8_t* buf = nullptr;
  const uint8_t *q = nullptr, *t = nullptr;
  const int64_t *qo = nullptr, *to = nullptr;
  const int32_t *ql = nullptr, *tl = nullptr, *h0 = nullptr;
  xt_result* out = nullptr;
  int64_t* cells = nullptr;
  ~DevPairs() {
    if (buf) cudaFree(buf);
  }
};

size_t al(size_t x) { return (x + 255) / 256 * 256; }

cudaError_t upload(const HostPairs& hp, DevPairs* d) {
  const size_t n = hp.ql.size();
  const size_t sizes[] = {hp.q.size(), hp.t.size(), 8 * n, 8 * n, 4 * n, 4 * n, 4 * n,
                          sizeof(xt_result) * n, 8 * n};
  size_t off[9], tot = 0;
  for (int k = 0; k < 9; ++k) {
    off[k] = tot;
    tot += al(sizes[k] ? sizes[k] : 1);
  }
  cudaError_t e = cudaMalloc((void**)&d->buf, tot);
  if (e != cudaSuccess) return e;
  const void* src[] = {hp.q.data(), hp.t.data(), hp.qo.data(), hp.to.data(),
                       hp.ql.data(), hp.tl.data(), hp.h0.data()};
  for (int k = 0; k < 7 && e == cudaSuccess; ++k)
    if (sizes[k]) e = cudaMemcpy(d->buf + off[k], src[k], sizes[k], cudaMemcpyHostToDevice);
  d->q = d->buf + off[0];
  d->t = d->buf + off[1];
  d->qo = (const int64_t*)(d->buf + off[2]);
  d->to = (const int64_t*)(d->buf + off[3]);
  d->ql = (const int32_t*)(d->buf + off[4]);
  d->tl = (const int32_t*)(d->buf + off[5]);
  d->h0 = (const int32_t*)(d->buf + off[6]);
  d->out = (xt_result*)(d->buf + off[7]);
  d->cells = (int64_t*)(d->buf + off[8]);
  return e;
}

// Candidate schedules in the order they are tried.
std::vector<BucketSched> candidates(const xt_ctx* ctx, int w, int j) {
  static const int kCand[][2] = {{1, 8}, {1, 4}, {1, 16}, {2, 8}, {2, 4}, {2, 16}, {4, 8},
                                 {4, 4}, {4, 16}, {8, 8}, {8, 4}, {16, 8}, {16, 4}, {32, 8},
                                 {32, 4}};
  std::vector<BucketSched> v;
  for (auto& c : kCand)
    if (bucket_sched_ok(ctx, w, j, c[0], c[1])) v.push_back({c[0], c[1]});
  return v;
}

std::string device_name(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  return p.name;
}

void set_sched(xt_ctx* ctx, int w, int j, BucketSched s, bool small) {
  TuneEntry* e = nullptr;
  for (auto& t : ctx->tuning)
    if (t.w == w) e = &t;
  if (!e) {
    ctx->tuning.push_back(TuneEntry());
    e = &ctx->tuning.back();
    e->w = w;
  }
  (small ? e->small[j] : e->b[j]) = s;
  drop_graphs(ctx);
}

constexpr int kSmallTrialPairs = 2048;

struct Trial {
  BucketSched best{};
  double gcups = -1;
};

// Time every candidate schedule of bucket j on n synthetic pairs; every
// candidate must reproduce the first one's results.
xt_status tune_bucket(xt_ctx* ctx, const xt_scoring* sc, int w, int j, int n,
                      const std::vector<BucketSched>& cand, bool small_only, int reps, Trial* tr,
                      std::string* why) {
  HostPairs hp;
  make_pairs(j, w, n, 0x5EED0000u + (uint64_t)j + (small_only ? 77u : 0u), &hp);
  DevPairs d;
  if (upload(hp, &d) != cudaSuccess) {
    cudaGetLastError();
    *why = "tuning buffers";
    return XT_ENOMEM;
  }
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (st) cudaStreamDestroy(st);
    if (e0) cudaEventDestroy(e0);
    *why = "tuning stream";
    return XT_ECUDA;
  }
  std::vector<xt_result> first_out(n), out(n);
  std::vector<int64_t> first_cells(n), cells(n);
  xt_status status = XT_OK;
  for (size_t c = 0; c < cand.size() && status == XT_OK; ++c) {
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      set_sched(ctx, w, j, cand[c], true);
      if (!small_only) set_sched(ctx, w, j, cand[c], false);
    }
    auto call = [&] {
      return xt_extend_batch(ctx, d.q, (int64_t)hp.q.size(), d.qo, d.ql, d.t,
                             (int64_t)hp.t.size(), d.to, d.tl, d.h0, n, sc, d.out, d.cells, st);
    };
    xt_status s = call();
    if (s != XT_OK) { status = s; *why = "tuning call"; break; }
    cudaError_t e = cudaMemcpyAsync(out.data(), d.out, sizeof(xt_result) * n,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cells.data(), d.cells, 8 * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { status = XT_ECUDA; *why = cudaGetErrorString(e); break; }
    if (c == 0) {
      first_out = out;
      first_cells = cells;
    } else if (std::memcmp(out.data(), first_out.data(), sizeof(xt_result) * n) != 0 ||
               cells != first_cells) {
      status = XT_ECUDA;
      *why = "schedules disagree on bucket " + std::to_string(j);
      break;
    }
    int64_t total = 0;
    for (int64_t v : cells) total += v;
    e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
      if (call() != XT_OK) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { status = XT_ECUDA; *why = cudaGetErrorString(e); break; }
    const double gcups = (double)total / (ms / reps * 1e-3) / 1e9;
    if (gcups > tr->gcups) {
      tr->gcups = gcups;
      tr->best = cand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return status;
}

}  // namespace

extern "C" {

xt_status xt_autotune(xt_ctx* ctx, const xt_scoring* sc, int j_max, double cells_per_trial,
                      const char* table_path) {
  if (!ctx || xt_scoring_check(sc) != XT_OK || j_max < kJMin || j_max > kJMax ||
      cells_per_trial < 0)
    return XT_EINVAL;
  if (cells_per_trial == 0) cells_per_trial = 3e10;
  const int w = sc->w > 2 * XT_MAX_LEN ? 2 * XT_MAX_LEN : sc->w;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->forced_P) {
      ctx->last_error = "xt_autotune: a schedule override is set (xt_ctx_set_schedule)";
      return XT_EINVAL;
    }
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return XT_ECUDA;
  Entry entry;
  entry.device = device_name(ctx->device);
  entry.sms = ctx->num_sms;
  entry.w = w;
  entry.sc = *sc;
  const bool graphs = ctx->graphs;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->graphs = false;  // time direct launches; no capture per candidate
  }
  xt_status status = XT_OK;
  std::string why;
  for (int j = kJMin; j <= j_max && status == XT_OK; ++j) {
    std::vector<BucketSched> cand;
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      cand = candidates(ctx, w, j);
    }
    if (cand.empty()) continue;
    // large calls: a trial fills the GPU, four pairs per one-lane thread slot
    // (every schedule timed at saturation), unless that exceeds the cells
    // budget; the candidate is set for both classes, since a capped trial
    // may itself be a small call
    const double qmid = j == kJMin ? 16.0 : 0.75 * (1 << j);
    const double width = std::min<double>(2.0 * w + 1, qmid + std::min<double>(2.0 * w, 2.0 * qmid));
    const double wave = (double)ctx->num_sms * 4 * kLaneThreads;  // one pair per one-lane slot
    int n = (int)std::max(1024.0, std::min<double>({(double)(1 << 20), 4.0 * wave,
                                                    cells_per_trial / (qmid * width)}));
    std::vector<BucketSched> big_cand = cand;
    int big_reps = 3;
    bool lane_cand = false;
    for (auto& c : cand) lane_cand |= c.P == 1;
    if (lane_cand && n < wave) {
      // long pairs: below one wave the one-lane engine would be timed half
      // idle, so time one full wave, with fewer candidates and one call each
      n = (int)wave;
      big_cand.clear();
      for (auto& c : cand)
        if ((c.P == 1 && c.R >= 8) || (c.P >= 16 && c.R == 8)) big_cand.push_back(c);
      big_reps = 1;
    }
    Trial big;
    status = tune_bucket(ctx, sc, w, j, n, big_cand, /*small_only=*/false, big_reps, &big, &why);
    if (status != XT_OK) break;
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      set_sched(ctx, w, j, big.best, false);
      set_sched(ctx, w, j, big.best, true);
    }
    // small calls: a bucket's share of a call of a few thousand pairs
    Trial little;
    status = tune_bucket(ctx, sc, w, j, kSmallTrialPairs, cand, /*small_only=*/true, 10, &little,
                         &why);
    if (status != XT_OK) break;
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      set_sched(ctx, w, j, little.best, true);
    }
    entry.buckets.push_back({j, big.best.P, big.best.R, big.gcups, little.best.P, little.best.R,
                             little.gcups});
  }
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->graphs = graphs;
    if (status != XT_OK) ctx->last_error = "xt_autotune: " + why;
  }
  if (status != XT_OK) return status;
  if (table_path) {
    std::vector<Entry> all = read_entries(table_path);
    std::vector<Entry> keep;
    for (auto& x : all)
      if (!(x.device == entry.device && x.sms == entry.sms && x.w == entry.w)) keep.push_back(x);
    keep.push_back(entry);
    if (!write_table(table_path, keep)) {
      std::lock_guard<std::mutex> lk(ctx->mu);
      ctx->last_error = std::string("xt_autotune: cannot write ") + table_path;
      return XT_EINVAL;
    }
  }
  return XT_OK;
}

xt_status xt_ctx_load_tuning(xt_ctx* ctx, const char* table_path) {
  if (!ctx || !table_path) return XT_EINVAL;
  Json root;
  if (!parse_file(table_path, &root)) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_error = std::string("xt_ctx_load_tuning: cannot read or parse ") + table_path;
    return XT_EINVAL;
  }
  const std::string dev = device_name(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  for (const Entry& e : read_entries(table_path)) {
    if (e.device != dev || e.sms != ctx->num_sms || e.w < 0) continue;
    for (const auto& b : e.buckets) {
      if (b.j < kJMin || b.j > kJMax) continue;
      if (bucket_sched_ok(ctx, e.w, b.j, b.P, b.R)) set_sched(ctx, e.w, b.j, {b.P, b.R}, false);
      if (b.Ps > 0 && bucket_sched_ok(ctx, e.w, b.j, b.Ps, b.Rs))
        set_sched(ctx, e.w, b.j, {b.Ps, b.Rs}, true);
    }
  }
  return XT_OK;
}

}  // extern "C"
