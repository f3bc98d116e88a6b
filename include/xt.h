/*
 * xt.h -- batched seed extension on GB300 (sm_103a): the C ABI.
 *
 * Operation (arXiv 2301.09310, Sec. II-A, Eq. 1): for every pair, extend an
 * exact-match seed of score h0 along a query q and a target (reference window)
 * t with affine-gap dynamic programming.  Rows i index the target ("reference
 * at i"), columns j the query ("query at j").  alpha = gap_open + gap_extend
 * is the cost of a gap's first base and beta = gap_extend of each further
 * base (Eq. 1's alpha and beta).  The DP runs on an extended matrix with a
 * seed cell H(-1,-1) = h0, a boundary row and column of pure gap runs from the
 * seed, a static band |i - j| <= w (cells outside it are dead), and the
 * anchoring rule that a cell of value 0 is dead and is not restarted by a
 * later match (extension stays tied to its seed).  After each target row, in
 * row order, the row maximum m_i (largest column on ties) updates the local
 * best; a row that does not improve it stops the extension when
 *   best - m_i - |(i - bi) - (mj_i - bj)| * beta > zdrop      (zdrop > 0).
 * The end-to-end score is the best H at the last query column (earliest row
 * on ties).  The paper states only plain Eq. 1; the seed, band and z-drop
 * reading above is this library's, and every result is bit-exact against the
 * scalar CPU oracle that implements it.
 *
 * Conventions of every entry point:
 *   - Sequences are uint8 base codes: 0,1,2,3 = A,C,G,T; any value >= 4 is N.
 *     Pairs are concatenated: pair k's query is q_seq[q_off[k] .. q_off[k] +
 *     q_len[k]), its target t_seq[t_off[k] .. t_off[k] + t_len[k]).
 *   - Pointers marked "device" must be device memory (cudaMalloc, torch CUDA
 *     tensors) of the context's device; the caller owns them and the library
 *     never frees them.  Work is enqueued on `stream` (a cudaStream_t; NULL is
 *     the legacy default stream) and is asynchronous: results are valid after
 *     the stream has been synchronised.  Inputs must stay alive and unchanged
 *     until then.
 *   - Argument and scoring errors are reported synchronously, before anything
 *     is enqueued (XT_EINVAL).  Per-pair input errors (h0 < 1 or > XT_MAX_H0,
 *     negative or too long lengths, a sequence outside its buffer) set that
 *     pair's status to XT_EINVAL, zero its other fields and cells, and leave
 *     the other pairs unaffected.  Device errors surface as XT_ECUDA at the
 *     call or at xt_ctx_sync.  No call aborts the process or traps the GPU.
 *   - Pairs are independent: a pair's result does not depend on the other
 *     pairs of the batch, the schedule or the kernel that computed it.
 */
#ifndef XT_H
#define XT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XT_ABI_VERSION 1
#define XT_MAX_LEN (1 << 20)  /* longest accepted query or target (bases) */
#define XT_MAX_H0 (1 << 20)   /* largest accepted seed score */

typedef enum {
  XT_OK = 0,
  XT_EINVAL = 1,   /* bad argument, scoring record or pair */
  XT_ENOMEM = 2,   /* the context's memory budget or the device is exhausted */
  XT_ECUDA = 3,    /* a CUDA call or kernel failed */
  XT_ETIMEOUT = 4, /* a bounded device-side wait expired */
  XT_EBUSY = 5     /* resource in use (e.g. serving queue full) */
} xt_status;

/*
 * Scoring record (Eq. 1's S, alpha, beta; band and z-drop of seed extension).
 *   match      in [1, 127]     score of two equal bases A/C/G/T
 *   mismatch   in [-127, 0]    score of two different bases (signed)
 *   gap_open   in [0, 1023]    a gap of k bases costs gap_open + k * gap_extend
 *   gap_extend in [0, 1023]
 *   w          >= 0            band: cell (i, j) exists iff |i - j| <= w
 *   zdrop      any             <= 0 disables the z-drop cutoff
 *   n_score    in [-127, 0]    score of any pair of bases involving N
 */
typedef struct {
  int32_t match, mismatch, gap_open, gap_extend, w, zdrop, n_score;
} xt_scoring;

/*
 * Result of one extension, 7 x int32 = 28 bytes, in input order.
 *   score    local best (>= h0)               qle  query bases consumed at it
 *   tle      target bases consumed at it      gscore end-to-end score at the
 *            last query column, -1 if never reached with a live cell
 *   gtle     target bases consumed at gscore  max_off  largest |j - i| of the
 *            rows that raised the best        status   XT_OK or XT_EINVAL
 * qlen == 0 gives {h0,0,0,h0,0,0,OK}; tlen == 0 gives {h0,0,0,-1,0,0,OK}.
 */
typedef struct {
  int32_t score, qle, tle, gscore, gtle, max_off, status;
} xt_result;

typedef struct xt_ctx xt_ctx;

/*
 * Create a context on CUDA device `device` (made current for the call).
 * mem_budget_bytes caps the device workspace the context may hold (0 = no
 * cap beyond the device).  *ctx receives the handle; XT_EINVAL on a NULL ctx
 * or a bad device, XT_ECUDA when the device cannot be used.
 */
xt_status xt_ctx_create(xt_ctx** ctx, int device, size_t mem_budget_bytes);

/* Release the context and its workspace (after synchronising its work). */
xt_status xt_ctx_destroy(xt_ctx* ctx);

/* Wait for the context's work on `stream`; reports pending device errors. */
xt_status xt_ctx_sync(xt_ctx* ctx, void* stream);

/*
 * Batched extension (the fast path).  A classify pass validates each pair
 * and sorts the batch into length buckets; persistent kernels then pull pairs
 * from device-side queues, each bucket with its own schedule (pairs per warp,
 * rows per lane, packed 16-bit or 32-bit arithmetic where a per-pair score
 * bound makes it exact).  The call waits on the host for the classify pass
 * (a few hundred bytes of bucket counts come back) before it enqueues the
 * extension kernels; those are asynchronous.
 *
 *   q_seq, t_seq       device, uint8 codes; q_bytes / t_bytes their sizes
 *   q_off, t_off       device, int64[n_pairs]
 *   q_len, t_len, h0   device, int32[n_pairs]
 *   n_pairs            >= 0
 *   sc                 host pointer to the scoring record (read during the call)
 *   out                device, xt_result[n_pairs]
 *   cells_out          device int64[n_pairs] or NULL: useful in-band cells of
 *                      each pair (rows 0 .. the last live row not after the
 *                      z-drop stop row, summed over their band widths)
 *   stream             cudaStream_t
 * Device workspace comes from the context (grown as needed within its budget;
 * XT_ENOMEM if it cannot).
 */
xt_status xt_extend_batch(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes,
                          const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                          int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                          const int32_t* h0, int32_t n_pairs, const xt_scoring* sc,
                          xt_result* out, int64_t* cells_out, void* stream);

/*
 * xt_extend_batch in two steps, for callers that must not block (one
 * thread driving several contexts and streams).  _begin checks the
 * arguments (errors as xt_extend_batch) and enqueues the classify pass and
 * the copy of its bucket counts on `stream`; _ready sets *ready = 1 once
 * those counts are on the host; _finish plans and enqueues the extension
 * kernels (waiting for the counts if they are not there yet).  Between
 * _begin and _finish the context holds the call: other calls on it return
 * XT_EBUSY.  xt_extend_batch is _begin followed by _finish.
 */
xt_status xt_extend_batch_begin(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes,
                                const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                                int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                                const int32_t* h0, int32_t n_pairs, const xt_scoring* sc,
                                xt_result* out, int64_t* cells_out, void* stream);
xt_status xt_extend_batch_ready(xt_ctx* ctx, int* ready);
xt_status xt_extend_batch_finish(xt_ctx* ctx);

/*
 * Both-direction extension of seeds (Sec. II-A: seed-and-extend grows each
 * exact-match seed to both sides).  Pair k holds a query and a target window
 * (as in xt_extend_batch) and a seed: seed_len[k] matching bases at query
 * position q_beg[k] and target position t_beg[k], with score h0[k].  The left
 * side extends the reversed prefixes (query [0, q_beg), target [0, t_beg))
 * from h0; the right side extends the suffixes (query [q_beg + seed_len,
 * qlen), target [t_beg + seed_len, tlen)) from the left side's local best
 * (h0 when the left side is empty).  left[k] and right[k] are xt_results of
 * each side, positions counted from the seed outwards; left_cells /
 * right_cells (NULL: not written) their useful cells.  A seed outside its
 * pair (or a pair outside its buffers) gives XT_EINVAL on both sides.  All
 * arrays are device memory; q_beg, t_beg, seed_len int32[n_pairs].  The
 * call reads the sizes of the reversed prefixes back before it copies them
 * into the context's workspace (the two sides' sequences: at most the
 * seeds' prefix lengths summed), then enqueues both sides on `stream`.
 */
xt_status xt_extend_seeds(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes, const int64_t* q_off,
                          const int32_t* q_len, const uint8_t* t_seq, int64_t t_bytes,
                          const int64_t* t_off, const int32_t* t_len, const int32_t* q_beg,
                          const int32_t* t_beg, const int32_t* seed_len, const int32_t* h0,
                          int32_t n_pairs, const xt_scoring* sc, xt_result* left,
                          xt_result* right, int64_t* left_cells, int64_t* right_cells,
                          void* stream);

/*
 * Plain extension: one pair per thread block (one warp), 32-bit arithmetic,
 * no bucketing and no persistent queue -- the comparison kernel.  Same
 * arguments, conventions and results as xt_extend_batch.
 */
xt_status xt_extend_batch_plain(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes,
                                const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                                int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                                const int32_t* h0, int32_t n_pairs, const xt_scoring* sc,
                                xt_result* out, int64_t* cells_out, void* stream);

/*
 * End-to-end variant of xt_extend_batch on HOST buffers (same argument
 * meaning, every pointer a host pointer; pinned memory is fastest).  Copies
 * the inputs to the device, extends, copies results (and cells when
 * cells_out != NULL) back, and returns after the stream has synchronised.
 * From 2 x 2^20 pairs the call runs in chunks of doubling size whose bytes
 * copy while earlier chunks extend; a context created without a memory
 * budget runs them on two internal contexts of its own (created on the
 * first such call, released with the context), so that a chunk's kernels
 * overlap the previous chunk's.
 */
xt_status xt_extend_batch_host(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes,
                               const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                               int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                               const int32_t* h0, int32_t n_pairs, const xt_scoring* sc,
                               xt_result* out, int64_t* cells_out, void* stream);

/*
 * Override the schedule of the batched path (testing and tuning aid).
 * P = 1 runs every bucket on the one-lane engine (one thread per pair, R rows
 * per strip; packed pairs hold two stacked strips of R rows).  P = 2, 4, 8, 16
 * or 32 runs the group engine (P lanes per pair, R rows per lane) on every
 * bucket whose ring fits in shared memory.  R is 4, 8 or 16 (16 only with
 * P <= 4).  P = 0 restores the built-in per-bucket table.  Results never
 * depend on the schedule.  XT_EINVAL for an unsupported (P, R).
 */
xt_status xt_ctx_set_schedule(xt_ctx* ctx, int P, int R);

/*
 * Launch accounting and DP timing (measurement aid).  With timing enabled,
 * every extension call records a CUDA event pair on its stream around its DP
 * (extension) kernels.  xt_ctx_stats waits for the pending events, sums their
 * durations into dp_ms, reports the number of calls and kernel launches since
 * the previous xt_ctx_stats, and resets those counters.
 */
typedef struct {
  int32_t calls;        /* extension calls since the last query */
  int32_t launches;     /* kernels those calls enqueued (classify, ordering, DP) */
  int32_t dp_launches;  /* of which extension (DP) kernels */
  int32_t timed_calls;  /* calls whose DP time is included in dp_ms */
  double dp_ms;         /* summed device time of the DP kernels, ms */
} xt_stats;

xt_status xt_ctx_set_timing(xt_ctx* ctx, int enable);

/*
 * CUDA graphs (on by default).  The second call with the same scoring,
 * schedule, capacity class (n rounded up to a power of two, at least 1024)
 * and workspace is captured as one graph; later such calls replay it, so a
 * call costs the classify pass, one descriptor-store kernel and one graph
 * launch on the host.
 * Calls with timing enabled launch directly.  enable = 0 turns capture off.
 * A context's calls must be ordered on the GPU (one stream, or synchronised):
 * they share its workspace.
 */
xt_status xt_ctx_set_graphs(xt_ctx* ctx, int enable);
xt_status xt_ctx_stats(xt_ctx* ctx, xt_stats* out);

/*
 * Concurrency of the extension kernels of one call.  The batched path's
 * per-bucket kernels are independent; they fork onto up to `branches`
 * internal streams (forked from and joined back into the call's stream, so
 * the call stays ordered on it) and run concurrently.  Kernels that share the
 * global ring pool stay in order on one branch.  1..8 (default 8); 1 runs
 * every kernel on the call's stream.  Results never depend on it.
 */
#define XT_MAX_BRANCHES 8
xt_status xt_ctx_set_streams(xt_ctx* ctx, int branches);

/*
 * Per-bucket schedules of the batched path.  The batch is bucketed by query
 * length: bucket j (5..21) holds queries of 2^(j-1) - 1 .. 2^j - 2 bases
 * (bucket 5 also the shorter ones).  A schedule runs a bucket with P lanes
 * per pair and R rows per lane: P = 1 is the one-lane engine (one thread per
 * pair, R = 4, 8 or 16; packed 16-bit where exact), P = 2..32 the group
 * engine (P lanes of a warp per pair, R = 4 or 8, or 16 with P <= 4).
 * A call classifies its pairs first and plans every non-empty bucket from
 * the number of pairs it holds.  Schedules are kept per band w and per
 * class of that count: XT_BATCH_SMALL schedules apply to buckets of fewer
 * than XT_SMALL_BUCKET pairs in the call (they cannot fill the GPU, so a
 * pair's latency on its engine decides), XT_BATCH_LARGE ones to larger
 * buckets, and to small buckets without a small schedule.  A call uses the
 * schedules set for its own scoring's w and the built-in rule for buckets
 * without one (one lane per pair where the bucket is large enough: 8192
 * pairs for queries of 63..510 bases, 32768 above; otherwise enough lanes
 * per pair to fill the GPU).  P = 0 removes a bucket's
 * schedule.  XT_EINVAL if (P, R) does not exist or its band ring does not
 * fit on this device.  Results never depend on the schedule.
 * xt_ctx_set_bucket_schedule sets both classes.
 */
#define XT_BATCH_LARGE 0
#define XT_BATCH_SMALL 1
#define XT_SMALL_BUCKET 8192
xt_status xt_ctx_set_bucket_schedule(xt_ctx* ctx, int w, int j, int P, int R);
xt_status xt_ctx_set_bucket_schedule_for(xt_ctx* ctx, int w, int j, int batch_class, int P,
                                         int R);
/* The schedule set for (w, j) (large batches, or the given class): *P = 0
 * when the built-in rule applies. */
xt_status xt_ctx_get_bucket_schedule(xt_ctx* ctx, int w, int j, int* P, int* R);
xt_status xt_ctx_get_bucket_schedule_for(xt_ctx* ctx, int w, int j, int batch_class, int* P,
                                         int* R);

/*
 * Autotuner.  For every bucket j = 5..j_max, times each available (P, R) on
 * synthetic pairs of that bucket's lengths (each query a mutated copy of its
 * target, so pairs extend over the full band) with the scoring `sc`, and
 * keeps the fastest as the bucket's schedule for sc->w on this context.  A
 * trial batch holds enough pairs to fill the GPU four times over with the
 * one-lane engine (throughput at saturation), but at most about
 * cells_per_trial useful cells (0 = 3e10); for long queries, where that
 * budget would leave the one-lane engine half idle, one full wave of pairs
 * is timed instead, over the one-lane and 16/32-lane schedules only.  When
 * table_path is not NULL the schedules are also written to that JSON file
 * (entries of other devices or bands in it are kept), for
 * xt_ctx_load_tuning.  Every schedule tried must give bit-identical results
 * on the tuning pairs (XT_ECUDA otherwise).  Needs the global override of
 * xt_ctx_set_schedule off (XT_EINVAL).  Synchronous; takes seconds.
 */
xt_status xt_autotune(xt_ctx* ctx, const xt_scoring* sc, int j_max, double cells_per_trial,
                      const char* table_path);

/*
 * Load the schedules a table written by xt_autotune holds for this
 * context's device (same name and SM count); entries of other devices are
 * ignored.  XT_EINVAL if the file cannot be read or parsed.
 */
xt_status xt_ctx_load_tuning(xt_ctx* ctx, const char* table_path);

/*
 * How the context's calls read sequence bytes.  XT_ALPHABET_CODES (default):
 * base codes 0, 1, 2, 3 = A, C, G, T, any other value N.  XT_ALPHABET_ASCII:
 * raw reads as ASCII letters -- A, C, G, T in either case are the bases and
 * any other byte (N, n, IUPAC codes, ...) is N.  A call then first runs an
 * elementwise pass that writes the base codes of both sequence buffers into
 * the context's workspace (q_bytes + t_bytes bytes, within its budget) and
 * extends from those.  Results are those of the same sequences given as
 * base codes.
 * XT_ALPHABET_PACKED4: base codes packed two to a byte, the paper's 4-bit
 * packing (Sec. II-B, eight bases per 32-bit word): base p of a buffer is the
 * low nibble of byte p / 2 when p is even and the high nibble when p is odd
 * (0..3 = A, C, G, T, any other nibble N).  Offsets and lengths count bases;
 * q_bytes / t_bytes are the buffers' sizes in bytes, so a buffer holds
 * 2 * bytes bases.  A call first unpacks both buffers to one code per byte in
 * the context's workspace (2 * (q_bytes + t_bytes) bytes, within its budget);
 * xt_extend_batch_host copies the packed bytes, half those of base codes, and
 * unpacks each chunk's bytes as they arrive.  Results are those of the same
 * sequences given as base codes.
 * (The allocation-free xt_extend_batch_static reads base codes only, and the
 * serving loop takes base codes or ASCII: XT_EINVAL at xt_serve_create.)
 */
#define XT_ALPHABET_CODES 0
#define XT_ALPHABET_ASCII 1
#define XT_ALPHABET_PACKED4 2
xt_status xt_ctx_set_alphabet(xt_ctx* ctx, int alphabet);

/* XT_OK if the scoring record is within the ranges above, else XT_EINVAL. */
xt_status xt_scoring_check(const xt_scoring* sc);

/*
 * BWA-MEM-compatible extension (opt-in; the default definition above is
 * Eq. 1 of Sec. II-A as read there).  Seed-and-extend aligners that take
 * their seeds from BWA-MEM (the seeds of the paper's real-data runs,
 * Sec. V) extend with a variant of Eq. 1; this call computes that variant,
 * stated here in full (rows i = target, columns j = query):
 *
 *   gaps open from the match value, so an insertion never touches a deletion:
 *     M(i,j) = H(i-1,j-1) + S(i,j) if H(i-1,j-1) > 0, else 0 (may be < 0)
 *     E(i,j) = max(0, M(i,j-1) - o_ins - e_ins, E(i,j-1) - e_ins)   insertion
 *     F(i,j) = max(0, M(i-1,j) - o_del - e_del, F(i-1,j) - e_del)   deletion
 *     H(i,j) = max(M, E, F); cells a row does not compute hold 0, and E is 0
 *     at a row's first computed column;
 *   boundaries: H(-1,-1) = h0; row -1 is the insertion run from the seed,
 *     max(0, h0 - o_ins - e_ins*(c+1)) inside the band (no deletion opens from
 *     it); column -1 the deletion run max(0, h0 - o_del - e_del*(r+1)), used
 *     only as the diagonal source of (r+1, 0) when row r computed column 0
 *     (no insertion opens from it);
 *   band narrowing: with gain = qlen*match + end_bonus, w_x = 1 if gain < o_x,
 *     else (gain - o_x) / e_x + 1 (x = ins, del), and the band is |i - j| <=
 *     min(w, w_ins, w_del) =: w';
 *   row trimming: row 0 computes [0, min(qlen, w'+1)); the dead cells at
 *     both ends of a row are dropped: if a and b are the first and the last
 *     computed column of row i with H > 0, row i+1 computes
 *     [max(a, i+1-w'), min(b+2, i+w'+2, qlen)) (dead columns between a and b
 *     are computed again);
 *   after each row, in order: if the row computed column qlen-1 and H(i,
 *     qlen-1) >= gscore, gscore = that value and gtle = i+1 (the latest row
 *     wins ties; gscore starts at -1); the extension stops if m = 0; a new
 *     local best needs m > best (as in the default definition); otherwise,
 *     with zdrop > 0, di = i - bi, dj = mj - bj, it stops after the row when
 *     best - m - (di - dj)*e_del > zdrop (di > dj) or best - m - (dj - di)*
 *     e_ins > zdrop (otherwise).
 *
 * Results and cells_out are as for xt_extend_batch: cells_out counts the
 * computed columns of every row with m > 0 that was evaluated.  Degenerate
 * pairs give the default definition's results.  Per-pair errors are those of
 * xt_extend_batch plus rows wider than XT_BWA_MAX_WIDTH columns
 * (min(qlen, 2w'+1) > XT_BWA_MAX_WIDTH: status XT_EINVAL).  The scoring
 * record: match in [1, 127]; mismatch and n_score in [-127, 0]; o_del and
 * o_ins in [0, 1023]; e_del and e_ins in [1, 1023]; w >= 0; end_bonus in
 * [0, 2^20]; zdrop <= 0 disables the z-drop.  Asynchronous on `stream`; the
 * context's alphabet applies.  Inputs, outputs and ownership as for
 * xt_extend_batch; the call does not use CUDA graphs or bucket schedules.
 */
typedef struct {
  int32_t match, mismatch, n_score;
  int32_t o_del, e_del, o_ins, e_ins;
  int32_t w, zdrop, end_bonus;
} xt_bwa_scoring;
#define XT_BWA_MAX_WIDTH 8192
xt_status xt_bwa_scoring_check(const xt_bwa_scoring* sc);
xt_status xt_extend_batch_bwa(xt_ctx* ctx, const uint8_t* q_seq, int64_t q_bytes,
                              const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                              int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                              const int32_t* h0, int32_t n_pairs, const xt_bwa_scoring* sc,
                              xt_result* out, int64_t* cells_out, void* stream);

/*
 * Split a batch over `parts` devices (host call, no GPU needed).  Pairs are
 * independent (Sec. VII-C: several GPUs partition the pairs and exchange
 * nothing but results), so each device extends its own part with
 * xt_extend_batch and the results are put back in input order by the
 * caller.  The split is LPT on estimated cells: each pair's estimate is its
 * in-band cells with no z-drop under band w (rows i < min(tlen, qlen + w));
 * pairs go in decreasing order of the estimate (ties: lower pair index
 * first) to the part with the smallest estimated total so far (ties: lower
 * part index), which keeps the largest part within 4/3 of the best possible
 * split and, for batches of many small pairs, within one pair of the mean.
 * Deterministic: every rank that calls it on the same lengths gets the same
 * split.  Host arrays: q_len, t_len int32[n_pairs] (negative lengths count
 * as 0); shard int32[n_pairs] receives each pair's part in [0, parts);
 * part_cells int64[parts] (may be NULL) each part's estimated cells.
 * XT_EINVAL for n_pairs < 0, w < 0, parts outside [1, 4096] or a NULL array.
 */
xt_status xt_shard_lpt(const int32_t* q_len, const int32_t* t_len, int32_t n_pairs, int32_t w,
                       int32_t parts, int32_t* shard, int64_t* part_cells);

/*
 * Measurement aid (not part of the method): the throughput of one kind of
 * integer instruction on `device`, which sets the roofline of the extension
 * DP (integer arithmetic, no dense contraction).  A probe kernel runs the
 * instruction in independent chains on every SM (8 chains per thread, a full
 * SM of warps) and is timed with CUDA events after one warm-up launch; the
 * best of `reps` launches is returned: *units instructions (thread-level) in
 * *ms milliseconds.  XT_RATE_MIX runs the 3-way packed max (integer ALU
 * pipe) in half of the chains and the packed add (multiply-add pipe) in the
 * other half, so both pipes feed the issue slots: it measures the issue rate.  XT_RATE_CELL_P16 runs the packed cell update of
 * the one-lane engine on registers (the engine's fast step, 16 cells per step
 * and thread); *units then counts cells.  Synchronous; allocates a few bytes
 * of device memory; XT_EINVAL for an unknown op or device.
 */
#define XT_RATE_ADD16X2 0      /* add.s16x2 (issues to the multiply-add pipe) */
#define XT_RATE_MAX3_16X2 1    /* 3-way packed 16-bit max */
#define XT_RATE_ADDMAX_16X2 2  /* packed 16-bit add-max with relu */
#define XT_RATE_PRMT 3         /* byte permute */
#define XT_RATE_IADD3 4        /* 32-bit three-input add */
#define XT_RATE_MAX3_32 5      /* 3-way 32-bit max */
#define XT_RATE_IMAD 6         /* 32-bit multiply-add */
#define XT_RATE_MIX 7          /* 3-way packed max and packed add, by chain */
#define XT_RATE_CELL_P16 8     /* the packed cell update (cells, not instructions) */
#define XT_RATE_HMAX2 9        /* packed half-precision max */
xt_status xt_int_rate(int device, int op, int reps, int64_t* units, double* ms);

/* Human-readable name of a status code (static storage). */
const char* xt_status_str(xt_status s);

/* Last error message recorded by the context (static per context; "" if none). */
const char* xt_ctx_last_error(const xt_ctx* ctx);

/*
 * Batched extension that allocates nothing (the paper has no counterpart:
 * this exists for callers, not for the method).
 *
 * Some callers may not call cudaMalloc at all: code running inside another
 * framework's memory pool or arena, a process that has reserved all of the
 * device memory for itself up front, or a latency-critical loop that must
 * never hit the allocator.  This entry point serves them: it takes no
 * context and never allocates device or host memory.  Its scratch (the
 * per-pair class bytes, the bucket queue and its counters) lives in one
 * fixed array inside the library, XT_STATIC_SCRATCH_BYTES long, which every
 * GPU that loads the library holds until the process exits.
 *
 * Arguments and results are those of xt_extend_batch (all arrays device
 * memory of the CURRENT device, owned by the caller; work is enqueued on
 * `stream`).  Limits, rejected with XT_EINVAL before anything is enqueued:
 *   n_pairs <= XT_STATIC_MAX_PAIRS, and a band narrow enough that every
 *   pair's boundary ring fits in shared memory (w up to about 1900; wider
 *   bands need xt_extend_batch, which can grow a global ring pool).
 * The first call on each device looks up the array's device address once
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make
 * that first call before any stream capture on that device.  The address
 * belongs to the device's primary context: after a cudaDeviceReset of that
 * device it is no longer valid, so a process that resets a device must not
 * call this entry point on it again.  All calls share the one array and it
 * keeps the previous call's contents (the call zeroes what must start at
 * zero): calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it, so order them, e.g. on one stream.  The batch
 * descriptor goes to the device as a kernel parameter, so no host memory of
 * the call has to outlive it.
 */
#define XT_STATIC_MAX_PAIRS (1 << 20)
#define XT_STATIC_SCRATCH_BYTES ((size_t)6 << 20)
xt_status xt_extend_batch_static(const uint8_t* q_seq, int64_t q_bytes, const int64_t* q_off,
                                 const int32_t* q_len, const uint8_t* t_seq, int64_t t_bytes,
                                 const int64_t* t_off, const int32_t* t_len, const int32_t* h0,
                                 int32_t n_pairs, const xt_scoring* sc, xt_result* out,
                                 int64_t* cells_out, void* stream);

/*
 * Serving loop: requests of host pairs, continuous batching on the GPU.
 *
 * Not part of the paper's method (which extends one batch per call): this is
 * the runtime that feeds a stream of small requests into the batched path.
 * A server owns one thread, `slots` contexts with a stream each, and per slot
 * a pinned host staging buffer and a device buffer of max_batch_bytes.
 * Whenever a slot is free and requests are waiting, the thread forms a batch
 * from the waiting requests in arrival order (requests with the same scoring
 * record as the oldest one, until the slot's pair or byte capacity is
 * reached), gathers their pairs into the staging buffer (offsets rebased; a
 * pair whose sequence lies outside its request's buffer gets status
 * XT_EINVAL), copies it to the device with one copy, runs xt_extend_batch,
 * and copies the results back with one copy.  While one slot's batch runs,
 * the next forms and copies on another.  When a batch completes, the thread
 * writes each request's results to the caller's output arrays and marks the
 * request done.  Results are identical to one xt_extend_batch call on the
 * request alone (pairs are independent).
 *
 * Admission: a request larger than one slot (pairs or staged bytes) is
 * rejected with XT_EINVAL; while the bytes of waiting requests would exceed
 * max_queued_bytes, xt_serve_submit returns XT_EBUSY and the caller retries.
 * Device memory: slots x (staging + result buffers + context workspace);
 * mem_budget_bytes caps the total (XT_ENOMEM at create or in a batch).
 * The slots' contexts launch directly, without CUDA graphs: batches of a
 * stream differ in their plans, and capturing a graph for each new plan
 * would add to that batch's latency.
 */
typedef struct xt_server xt_server;

typedef struct {
  int32_t slots;            /* batches in flight at once, 1..8 (0: 2) */
  int32_t max_batch_pairs;  /* pairs per batch, <= 1 << 24 (0: 1 << 20) */
  int64_t max_batch_bytes;  /* staged input bytes per batch: sequences plus
                               28 bytes per pair (0: 1 GiB) */
  int64_t max_queued_bytes; /* staged bytes of waiting requests (0: 1 GiB) */
  size_t mem_budget_bytes;  /* device memory of the whole server (0: no cap) */
  int32_t gather_threads;   /* host threads staging a batch, 1..16, the server
                               thread included (0: a quarter of the cores, <= 8) */
  const char* tuning_path;  /* a table written by xt_autotune, loaded into every
                               slot's context (NULL: built-in schedules) */
  int32_t alphabet;         /* XT_ALPHABET_CODES (0) or XT_ALPHABET_ASCII (not
                               XT_ALPHABET_PACKED4: XT_EINVAL) */
} xt_serve_config;

/* Latency stamps of one request, ns on CLOCK_MONOTONIC (see xt_now_ns). */
typedef struct {
  int64_t submit_ns;   /* xt_serve_submit accepted it */
  int64_t launch_ns;   /* its batch was formed (left the waiting queue) */
  int64_t done_ns;     /* its results were in the caller's output arrays */
  int32_t batch_pairs; /* pairs of the batch that carried it */
  int32_t status;      /* XT_OK, or the error of its batch (XT_ECUDA, XT_ENOMEM) */
} xt_serve_times;

typedef struct {
  int64_t requests;    /* completed requests */
  int64_t pairs;       /* their pairs */
  int64_t cells;       /* their useful cells */
  int64_t batches;     /* batches run */
  int64_t waiting;     /* requests waiting for a batch now */
  int64_t in_flight;   /* batches on the GPU now */
  int64_t gather_ns;   /* host time spent staging batches (summed) */
  int64_t device_ns;   /* stream time from copy-in start to copy-out end (summed) */
} xt_serve_stats;

/* Monotonic clock of the latency stamps (CLOCK_MONOTONIC, ns). */
int64_t xt_now_ns(void);

/* Start a server on `device`; cfg may be NULL (all defaults). */
xt_status xt_serve_create(xt_server** server, int device, const xt_serve_config* cfg);

/*
 * Queue one request of n_pairs >= 0 host pairs (same layout and meaning as
 * xt_extend_batch, every pointer a HOST pointer).  The caller keeps every
 * array alive and unchanged, and the output arrays (out: xt_result[n_pairs];
 * cells_out: int64[n_pairs] or NULL) untouched, until the request is done.
 * *ticket identifies it.  Errors, all synchronous: XT_EINVAL (arguments,
 * scoring, a request larger than one slot), XT_EBUSY (queue full, retry).
 */
xt_status xt_serve_submit(xt_server* server, const uint8_t* q_seq, int64_t q_bytes,
                          const int64_t* q_off, const int32_t* q_len, const uint8_t* t_seq,
                          int64_t t_bytes, const int64_t* t_off, const int32_t* t_len,
                          const int32_t* h0, int32_t n_pairs, const xt_scoring* sc,
                          xt_result* out, int64_t* cells_out, uint64_t* ticket);

/* *done = 1 when the request's results are in its output arrays. */
xt_status xt_serve_poll(xt_server* server, uint64_t ticket, int* done);

/*
 * Wait up to timeout_us microseconds (< 0: no limit) for a request.  On
 * completion the ticket is released, `times` (may be NULL) receives its
 * stamps, and the request's status is returned.  XT_ETIMEOUT if it is not
 * done in time (the ticket stays valid); XT_EINVAL for an unknown ticket.
 */
xt_status xt_serve_wait(xt_server* server, uint64_t ticket, int64_t timeout_us,
                        xt_serve_times* times);

/*
 * paused != 0: form no new batches (batches in flight finish; requests keep
 * queueing up to max_queued_bytes).  paused = 0 resumes.  xt_serve_destroy
 * resumes a paused server to finish its queue.
 */
xt_status xt_serve_pause(xt_server* server, int paused);

xt_status xt_serve_get_stats(xt_server* server, xt_serve_stats* out);

/* Finish every queued request, stop the thread and free the server. */
xt_status xt_serve_destroy(xt_server* server);

#ifdef __cplusplus
}
#endif
#endif /* XT_H */
