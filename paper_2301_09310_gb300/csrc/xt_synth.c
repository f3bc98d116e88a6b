/*
 * xt_synth.c -- seeded synthetic seed-extension workloads.
 *
 * Input generation only: this file holds none of the extension arithmetic and
 * is shared by the tests, the bench and the oracle runs as a source of inputs.
 *
 * The paper measures on BWA-MEM seeds from GRCh38 with Illumina MiSeq reads
 * (SRR835433, 250 bp) and PacBio reads (SRP091981, ~2 kbp) (Sec. V-D), and on
 * equal-length synthetic reads from a wgsim-like simulator (Sec. V-B).  Neither
 * the genome nor the reads exist here; this generator stands in for them with
 * the same shape: a reference window of uniform A/C/G/T (a small fraction N),
 * a query copied from it with substitutions and short insertions/deletions,
 * and the target = the matching reference window, longer than the query.
 *
 * Every random draw comes from SplitMix64 keyed by (seed, pair index, stream),
 * so pair k's content does not depend on how the batch is split or threaded,
 * and the same bytes come out on any host.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

typedef struct {
  uint64_t seed;
  int32_t len_kind;      /* 0 fixed, 1 uniform [1, read length] over a read-length mix,
                            2 log-uniform [len_lo, len_hi], 3 lognormal clipped */
  int32_t qlen_fixed;    /* kind 0 */
  int32_t n_mix;         /* kind 1: number of read lengths (<= 4) */
  int32_t mix_len[4];
  double mix_frac[4];
  double len_lo, len_hi; /* kind 2 bounds, kind 3 clip bounds */
  double ln_median, ln_sigma;
  int32_t tlen_extra;    /* tlen = qlen + tlen_extra */
  double p_n;            /* fraction of N in the reference */
  double p_sub, p_ins, p_del; /* per-base mutation rates of the query copy */
  int32_t indel_max;     /* indel length uniform in [1, indel_max] */
  int32_t long_threshold; /* qlen above this uses the long-read rates below (0: never) */
  double long_p_sub, long_p_ins, long_p_del;
  double p_unrelated;    /* query and target drawn independently */
  int32_t h0_lo, h0_hi;  /* h0 uniform in [h0_lo, h0_hi] */
} xs_config;

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct { uint64_t s; } rng_t;

static inline rng_t rng_for(uint64_t seed, uint64_t pair, uint64_t stream) {
  rng_t r;
  r.s = mix64(seed * 0x9E3779B97F4A7C15ULL + mix64(pair * 4 + stream + 1));
  return r;
}
static inline uint64_t next64(rng_t* r) {
  r->s += 0x9E3779B97F4A7C15ULL;
  return mix64(r->s);
}
static inline double unif(rng_t* r) { return (double)(next64(r) >> 11) * (1.0 / 9007199254740992.0); }
static inline int32_t rint_in(rng_t* r, int32_t lo, int32_t hi) {
  return lo + (int32_t)(next64(r) % (uint64_t)(hi - lo + 1));
}

/* Reference base at position p of pair k's window: a pure function of (k, p). */
static inline uint8_t ref_base(const xs_config* c, uint64_t k, int64_t p) {
  uint64_t h = mix64(c->seed ^ mix64(k * 0x632BE59BD9B4E019ULL + (uint64_t)p * 0x85EBCA77C2B2AE63ULL));
  double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
  if (u < c->p_n) return 4;
  return (uint8_t)(h & 3);
}

static inline uint8_t rand_base(const xs_config* c, rng_t* r) {
  if (unif(r) < c->p_n) return 4;
  return (uint8_t)(next64(r) & 3);
}

typedef struct { int32_t qlen, tlen, h0, unrelated; } pair_shape;

static pair_shape shape_of(const xs_config* c, uint64_t k) {
  rng_t r = rng_for(c->seed, k, 0);
  pair_shape s;
  s.unrelated = unif(&r) < c->p_unrelated;
  int32_t q = 1;
  switch (c->len_kind) {
    case 0: q = c->qlen_fixed; break;
    case 1: {
      double u = unif(&r), acc = 0;
      int32_t rl = c->mix_len[c->n_mix - 1];
      for (int m = 0; m < c->n_mix; ++m) {
        acc += c->mix_frac[m];
        if (u < acc) { rl = c->mix_len[m]; break; }
      }
      q = rint_in(&r, 1, rl);
      break;
    }
    case 2: {
      double u = unif(&r);
      q = (int32_t)floor(exp(log(c->len_lo) + u * (log(c->len_hi) - log(c->len_lo))));
      break;
    }
    case 3: {
      /* Box-Muller normal from two uniforms */
      double u1 = unif(&r), u2 = unif(&r);
      if (u1 < 1e-300) u1 = 1e-300;
      double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
      double v = floor(c->ln_median * exp(c->ln_sigma * z));
      if (v < c->len_lo) v = c->len_lo;
      if (v > c->len_hi) v = c->len_hi;
      q = (int32_t)v;
      break;
    }
  }
  if (q < 0) q = 0;
  s.qlen = q;
  s.tlen = q + c->tlen_extra;
  s.h0 = rint_in(&r, c->h0_lo, c->h0_hi);
  return s;
}

/* Lengths and h0 of pairs [first, first+n). */
void xs_shapes(const xs_config* c, uint64_t first, int64_t n, int32_t* q_len, int32_t* t_len,
               int32_t* h0) {
  for (int64_t i = 0; i < n; ++i) {
    pair_shape s = shape_of(c, first + (uint64_t)i);
    q_len[i] = s.qlen;
    t_len[i] = s.tlen;
    h0[i] = s.h0;
  }
}

static void fill_pair(const xs_config* c, uint64_t k, uint8_t* q, uint8_t* t) {
  pair_shape s = shape_of(c, k);
  if (s.unrelated) {
    rng_t r = rng_for(c->seed, k, 1);
    for (int32_t i = 0; i < s.qlen; ++i) q[i] = rand_base(c, &r);
    for (int32_t i = 0; i < s.tlen; ++i) t[i] = rand_base(c, &r);
    return;
  }
  for (int32_t i = 0; i < s.tlen; ++i) t[i] = ref_base(c, k, i);
  double ps = c->p_sub, pi = c->p_ins, pd = c->p_del;
  if (c->long_threshold > 0 && s.qlen > c->long_threshold) {
    ps = c->long_p_sub; pi = c->long_p_ins; pd = c->long_p_del;
  }
  rng_t r = rng_for(c->seed, k, 2);
  int64_t p = 0;
  int32_t j = 0;
  while (j < s.qlen) {
    double u = unif(&r);
    if (u < ps) {
      uint8_t b = ref_base(c, k, p++);
      uint8_t x = (uint8_t)(next64(&r) % 3);
      q[j++] = (b >= 4) ? (uint8_t)(next64(&r) & 3) : (uint8_t)((b + 1 + x) & 3);
    } else if (u < ps + pi) {
      int32_t L = rint_in(&r, 1, c->indel_max);
      for (int32_t e = 0; e < L && j < s.qlen; ++e) q[j++] = (uint8_t)(next64(&r) & 3);
    } else if (u < ps + pi + pd) {
      p += rint_in(&r, 1, c->indel_max);
    } else {
      q[j++] = ref_base(c, k, p++);
    }
  }
}

typedef struct {
  const xs_config* c; uint64_t first; int64_t n;
  const int64_t* q_off; const int64_t* t_off; uint8_t* q_seq; uint8_t* t_seq;
  int64_t next;
} fill_job;

static void* fill_worker(void* arg) {
  fill_job* f = (fill_job*)arg;
  for (;;) {
    int64_t s = __atomic_fetch_add(&f->next, 256, __ATOMIC_RELAXED);
    if (s >= f->n) break;
    int64_t e = s + 256 < f->n ? s + 256 : f->n;
    for (int64_t i = s; i < e; ++i)
      fill_pair(f->c, f->first + (uint64_t)i, f->q_seq + f->q_off[i], f->t_seq + f->t_off[i]);
  }
  return NULL;
}

/* Sequences of pairs [first, first+n) at the given offsets (from xs_shapes). */
void xs_fill(const xs_config* c, uint64_t first, int64_t n, const int64_t* q_off,
             const int64_t* t_off, uint8_t* q_seq, uint8_t* t_seq, int nthreads) {
  fill_job f = {c, first, n, q_off, t_off, q_seq, t_seq, 0};
  if (nthreads < 1) nthreads = 1;
  pthread_t th[256];
  if (nthreads > 256) nthreads = 256;
  int started = 0;
  for (int k = 1; k < nthreads; ++k)
    if (pthread_create(&th[started], NULL, fill_worker, &f) == 0) ++started;
  fill_worker(&f);
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
}

/* Lengths and h0 of the pairs idx[0..n) of the workload's stream (pair k's
 * shape depends on k alone, so any subset can be drawn). */
void xs_shapes_at(const xs_config* c, const int64_t* idx, int64_t n, int32_t* q_len,
                  int32_t* t_len, int32_t* h0) {
  for (int64_t i = 0; i < n; ++i) {
    pair_shape s = shape_of(c, (uint64_t)idx[i]);
    q_len[i] = s.qlen;
    t_len[i] = s.tlen;
    h0[i] = s.h0;
  }
}

typedef struct {
  const xs_config* c; const int64_t* idx; int64_t n;
  const int64_t* q_off; const int64_t* t_off; uint8_t* q_seq; uint8_t* t_seq;
  int64_t next;
} fill_at_job;

static void* fill_at_worker(void* arg) {
  fill_at_job* f = (fill_at_job*)arg;
  for (;;) {
    int64_t s = __atomic_fetch_add(&f->next, 256, __ATOMIC_RELAXED);
    if (s >= f->n) break;
    int64_t e = s + 256 < f->n ? s + 256 : f->n;
    for (int64_t i = s; i < e; ++i)
      fill_pair(f->c, (uint64_t)f->idx[i], f->q_seq + f->q_off[i], f->t_seq + f->t_off[i]);
  }
  return NULL;
}

/* Sequences of the pairs idx[0..n) at the given offsets (from xs_shapes_at). */
void xs_fill_at(const xs_config* c, const int64_t* idx, int64_t n, const int64_t* q_off,
                const int64_t* t_off, uint8_t* q_seq, uint8_t* t_seq, int nthreads) {
  fill_at_job f = {c, idx, n, q_off, t_off, q_seq, t_seq, 0};
  if (nthreads < 1) nthreads = 1;
  pthread_t th[256];
  if (nthreads > 256) nthreads = 256;
  int started = 0;
  for (int k = 1; k < nthreads; ++k)
    if (pthread_create(&th[started], NULL, fill_at_worker, &f) == 0) ++started;
  fill_at_worker(&f);
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
}
