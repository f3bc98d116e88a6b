/*
 * xt_oracle.c -- scalar CPU oracle for banded affine-gap seed extension.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle that the CUDA
 * path is checked against.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load it; the library never does.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (arXiv 2301.09310, Sec. II-A, Eq. 1, read as seed
 * extension per Sec. II-A "extending to both directions from the found seeds";
 * one direction per call):
 *
 *   The DP runs on an extended matrix, rows r = -1..tlen-1 (target, "reference
 *   at i" of Eq. 1) and columns c = -1..qlen-1 (query, "query at j").
 *   alpha = gap_open + gap_extend (cost of a gap's first base, Eq. 1's alpha),
 *   beta  = gap_extend            (each further base,        Eq. 1's beta).
 *
 *   band      : cell (r,c) is in band iff |r - c| <= w; out-of-band cells are
 *               dead (H = E = F = 0).
 *   seed      : H(-1,-1) = h0.
 *   row -1    : H(-1,c) = E(-1,c) = max(0, h0 - alpha - beta*c) when in band,
 *               F(-1,c) = 0.
 *   column -1 : H(r,-1) = F(r,-1) = max(0, h0 - alpha - beta*r) when in band,
 *               E(r,-1) = 0.
 *   S(i,j)    : match if t_i == q_j and both are bases A,C,G,T (codes 0..3);
 *               n_score if either code is N (any byte >= 4 is N);
 *               mismatch otherwise.
 *   interior  : D = H(i-1,j-1);  M = D + S(i,j) if D > 0, else 0
 *               (a dead cell is not restarted: the extension stays anchored at
 *               the seed, which is how Eq. 1's "0" is read here);
 *               E = max(0, H(i,j-1) - alpha, E(i,j-1) - beta)      (Eq. 1, E)
 *               F = max(0, H(i-1,j) - alpha, F(i-1,j) - beta)      (Eq. 1, F)
 *               H = max(0, M, E, F)                                (Eq. 1, H)
 *
 *   After each row i (in order): m_i = max in-band H(i,j) over j >= 0, mj_i =
 *   the largest such j attaining it (m_i = 0, mj_i = -1 for an empty band).
 *   gscore: if column qlen-1 is in band, H(i,qlen-1) > 0 and > gscore, then
 *   gscore = H(i,qlen-1), gtle = i+1 (strict, so the earliest row wins).
 *   local best (best,bi,bj) starts (h0,-1,-1), max_off = 0:
 *     m_i > best           -> best = m_i, bi = i, bj = mj_i,
 *                             max_off = max(max_off, |mj_i - i|)
 *     else if zdrop > 0    -> d = (i-bi) - (mj_i-bj),
 *                             stop after row i if best - m_i - |d|*beta > zdrop.
 *   result = {best, bj+1, bi+1, gscore, gtle, max_off, OK}; gscore starts -1,
 *   gtle 0.  qlen == 0 -> {h0,0,0,h0,0,0}; tlen == 0 -> {h0,0,0,-1,0,0}.
 *   Useful cells = sum over rows 0..i_end of the in-band width of the row,
 *   i_end = the last row (not after the stop row) holding an H > 0.
 *
 * The arithmetic is int64 throughout, so no value of the definition can
 * overflow for the input limits the library accepts.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* Scoring record, laid out like the library's but declared here on its own. */
typedef struct {
  int32_t match, mismatch, gap_open, gap_extend, w, zdrop, n_score;
} xo_scoring;

enum { XO_OK = 0, XO_EINVAL = 1 };

/* Input limits shared in value (not in code) with the library's checks. */
#define XO_MAX_LEN (1 << 20)
#define XO_MAX_H0 (1 << 20)

static int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t min2(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t iabs64(int64_t a) { return a < 0 ? -a : a; }

static int in_band(int64_t r, int64_t c, int64_t w) { return iabs64(r - c) <= w; }

static int64_t score(const xo_scoring* sc, uint8_t a, uint8_t b) {
  if (a >= 4 || b >= 4) return sc->n_score;
  return a == b ? sc->match : sc->mismatch;
}

/* Number of in-band columns j in [0, qlen) of row i. */
static int64_t band_width(int64_t i, int64_t qlen, int64_t w) {
  int64_t lo = max2(0, i - w), hi = min2(qlen, i + w + 1);
  return hi > lo ? hi - lo : 0;
}

/* Returns 0 when the scoring record is acceptable. */
int xo_check_scoring(const xo_scoring* sc) {
  if (!sc) return XO_EINVAL;
  if (sc->match < 1 || sc->match > 127) return XO_EINVAL;
  if (sc->mismatch > 0 || sc->mismatch < -127) return XO_EINVAL;
  if (sc->n_score > 0 || sc->n_score < -127) return XO_EINVAL;
  if (sc->gap_open < 0 || sc->gap_open > 1023) return XO_EINVAL;
  if (sc->gap_extend < 0 || sc->gap_extend > 1023) return XO_EINVAL;
  if (sc->w < 0) return XO_EINVAL;
  return XO_OK;
}

/*
 * One extension.  out[7] = {score, qle, tle, gscore, gtle, max_off, status}.
 * *cells receives the useful-cell count.  When rows_m / rows_mj are non-NULL
 * they receive m_i and mj_i for every row that was evaluated and *n_rows the
 * number of such rows (the stop row included).  When full_H/E/F are non-NULL
 * they receive the extended matrices, (tlen+1) x (qlen+1), row-major, entry
 * [(r+1)*(qlen+1) + (c+1)] for cell (r,c); rows after the stop row stay 0.
 */
void xo_extend_one(const uint8_t* q, int32_t qlen, const uint8_t* t, int32_t tlen, int32_t h0,
                   const xo_scoring* sc, int32_t out[7], int64_t* cells, int64_t* rows_m,
                   int64_t* rows_mj, int32_t* n_rows, int64_t* full_H, int64_t* full_E,
                   int64_t* full_F) {
  const int64_t alpha = (int64_t)sc->gap_open + sc->gap_extend;
  const int64_t beta = sc->gap_extend;
  const int64_t w = sc->w;
  if (n_rows) *n_rows = 0;
  *cells = 0;
  if (qlen == 0) {
    out[0] = h0; out[1] = 0; out[2] = 0; out[3] = h0; out[4] = 0; out[5] = 0; out[6] = XO_OK;
    return;
  }
  if (tlen == 0) {
    out[0] = h0; out[1] = 0; out[2] = 0; out[3] = -1; out[4] = 0; out[5] = 0; out[6] = XO_OK;
    return;
  }
  const int64_t ncol = (int64_t)qlen + 1; /* index c+1 holds column c */
  int64_t* Hp = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Ep = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Fp = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Hc = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Ec = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Fc = calloc((size_t)ncol, sizeof(int64_t));

  /* Row -1: the seed cell and the insertion run along the query. */
  Hp[0] = h0; Ep[0] = 0; Fp[0] = 0;
  for (int64_t c = 0; c < qlen; ++c) {
    if (in_band(-1, c, w)) {
      int64_t v = max2(0, h0 - alpha - beta * c);
      Hp[c + 1] = v; Ep[c + 1] = v; Fp[c + 1] = 0;
    }
  }
  if (full_H) {
    for (int64_t c = 0; c < ncol; ++c) {
      full_H[c] = Hp[c]; full_E[c] = Ep[c]; full_F[c] = Fp[c];
    }
  }

  int64_t best = h0, bi = -1, bj = -1, max_off = 0;
  int64_t gscore = -1, gtle = 0;
  int64_t last_live = -1;
  for (int64_t i = 0; i < tlen; ++i) {
    /* Column -1: the deletion run along the target. */
    if (in_band(i, -1, w)) {
      int64_t v = max2(0, h0 - alpha - beta * i);
      Hc[0] = v; Fc[0] = v; Ec[0] = 0;
    } else {
      Hc[0] = 0; Fc[0] = 0; Ec[0] = 0;
    }
    int64_t m = 0, mj = -1;
    int any_live = 0;
    for (int64_t j = 0; j < qlen; ++j) {
      if (!in_band(i, j, w)) {
        Hc[j + 1] = 0; Ec[j + 1] = 0; Fc[j + 1] = 0;
        continue;
      }
      int64_t D = Hp[j];
      int64_t M = D > 0 ? D + score(sc, t[i], q[j]) : 0;
      int64_t E = max2(0, max2(Hc[j] - alpha, Ec[j] - beta));
      int64_t F = max2(0, max2(Hp[j + 1] - alpha, Fp[j + 1] - beta));
      int64_t H = max2(max2(0, M), max2(E, F));
      Hc[j + 1] = H; Ec[j + 1] = E; Fc[j + 1] = F;
      if (H >= m) { m = H; mj = j; }
      if (H > 0) any_live = 1;
    }
    if (full_H) {
      for (int64_t c = 0; c < ncol; ++c) {
        full_H[(i + 1) * ncol + c] = Hc[c];
        full_E[(i + 1) * ncol + c] = Ec[c];
        full_F[(i + 1) * ncol + c] = Fc[c];
      }
    }
    if (rows_m) { rows_m[i] = m; rows_mj[i] = mj; }
    if (n_rows) *n_rows = (int32_t)(i + 1);
    if (any_live) last_live = i;
    /* End-to-end score at the last query column. */
    if (in_band(i, qlen - 1, w)) {
      int64_t g = Hc[qlen];
      if (g > 0 && g > gscore) { gscore = g; gtle = i + 1; }
    }
    /* Local best and z-drop, in row order. */
    if (m > best) {
      best = m; bi = i; bj = mj;
      max_off = max2(max_off, iabs64(mj - i));
    } else if (sc->zdrop > 0) {
      int64_t d = (i - bi) - (mj - bj);
      int64_t drop = best - m - iabs64(d) * beta;
      if (drop > sc->zdrop) break;
    }
    int64_t* tmp;
    tmp = Hp; Hp = Hc; Hc = tmp;
    tmp = Ep; Ep = Ec; Ec = tmp;
    tmp = Fp; Fp = Fc; Fc = tmp;
  }
  int64_t n = 0;
  for (int64_t i = 0; i <= last_live; ++i) n += band_width(i, qlen, w);
  *cells = n;
  out[0] = (int32_t)best; out[1] = (int32_t)(bj + 1); out[2] = (int32_t)(bi + 1);
  out[3] = (int32_t)gscore; out[4] = (int32_t)gtle; out[5] = (int32_t)max_off; out[6] = XO_OK;
  free(Hp); free(Ep); free(Fp); free(Hc); free(Ec); free(Fc);
}

/* ======================================================================== *
 * BWA-MEM-compatible extension (an opt-in variant of the definition above).
 *
 * Seed-and-extend aligners that take their seeds from BWA-MEM (Sec. II-A and
 * the real-seed experiments of Sec. V) extend with a variant of Eq. 1 whose
 * differences are, in the notation above (rows i = target, columns j = query;
 * E = horizontal gap = insertion, F = vertical gap = deletion):
 *
 *   V1 gaps open from the match value M, not from H, so an insertion is
 *      never directly followed by a deletion or the reverse:
 *        M(i,j) = D + S(i,j) if D = H(i-1,j-1) > 0, else 0   (may be < 0)
 *        E(i,j) = max(0, M(i,j-1) - oe_ins, E(i,j-1) - e_ins), 0 at the
 *                 first computed column of the row
 *        F(i,j) = max(0, M(i-1,j) - oe_del, F(i-1,j) - e_del), 0 when
 *                 (i-1,j) was not computed
 *        H(i,j) = max(M, E, F)                  (>= 0, as E, F >= 0)
 *      with oe_x = o_x + e_x.  Cells that are not computed hold H = M = E =
 *      F = 0.
 *   V2 separate insertion and deletion penalties (o_ins, e_ins, o_del, e_del).
 *   V3 boundaries: row -1 is the insertion run from the seed,
 *      H(-1,c) = max(0, h0 - oe_ins - e_ins*c) inside the band, with M = F =
 *      0 there (no deletion opens from it); column -1 is the deletion run,
 *      H(r,-1) = max(0, h0 - oe_del - e_del*r), used only as the diagonal
 *      source of (r+1, 0) and only when row r computed column 0; no insertion
 *      opens from it.  H(-1,-1) = h0.
 *   V4 band narrowing: a gap longer than the whole query could pay for is
 *      never taken.  With gain = qlen*match + end_bonus,
 *        w_x = 1 if gain < o_x, else (gain - o_x) / e_x + 1   (x = ins, del)
 *        w'  = min(w, w_ins, w_del)
 *      and the band is |i - j| <= w'.
 *   V5 row trimming: row 0 computes columns [0, min(qlen, w'+1)).  After row
 *      i, the dead cells at the two ends of its computed range are dropped:
 *      with a the first and b the last computed column of row i with H > 0,
 *      row i+1 computes
 *        [max(a, i+1-w'), min(b+2, i+w'+2, qlen))
 *      i.e. the columns its live cells reach in one step (a vertical step
 *      from a, a diagonal step from b); dead columns between a and b are
 *      computed again.  (A cell with H = 0 also has M <= 0 and F = 0, so the
 *      next row's deletion state there is 0: H alone decides.)
 *   V6 rows: m_i and mj_i are taken over the computed columns (largest j on
 *      ties).  After row i, in this order:
 *        gscore: if row i computed column qlen-1 and H(i,qlen-1) >= gscore,
 *                gscore = H(i,qlen-1), gtle = i+1 (latest row on ties; a 0
 *                counts; gscore starts at -1, gtle at 0);
 *        stop if m_i = 0 (row i is not counted as useful);
 *        local best as in the default definition, else if zdrop > 0 with
 *        di = i - bi, dj = mj_i - bj: drop = best - m_i - (di - dj)*e_del
 *        when di > dj, else best - m_i - (dj - di)*e_ins; stop after row i
 *        when drop > zdrop.
 *   Useful cells: the computed widths of every row with m_i > 0 that was
 *   evaluated (the stop row of a z-drop included).  Degenerate inputs give
 *   the same results as the default definition.  A batch pair whose rows
 *   would be wider than XO_BWA_MAX_WIDTH columns (min(qlen, 2w'+1)) gets
 *   status XO_EINVAL, a limit shared in value with the library.
 *
 * The flags XO_BWA_NO_TRIM and XO_BWA_NO_NARROW switch V5 and V4 off; they
 * exist only so that the tests can pin V1-V3 and V6 on their own against an
 * enumeration of alignment paths.
 * ======================================================================== */

typedef struct {
  int32_t match, mismatch, n_score, o_del, e_del, o_ins, e_ins, w, zdrop, end_bonus;
} xo_bwa_scoring;

enum { XO_BWA_NO_TRIM = 1, XO_BWA_NO_NARROW = 2 };

#define XO_BWA_MAX_END_BONUS (1 << 20)

int xo_check_bwa_scoring(const xo_bwa_scoring* sc) {
  if (!sc) return XO_EINVAL;
  if (sc->match < 1 || sc->match > 127) return XO_EINVAL;
  if (sc->mismatch > 0 || sc->mismatch < -127) return XO_EINVAL;
  if (sc->n_score > 0 || sc->n_score < -127) return XO_EINVAL;
  if (sc->o_del < 0 || sc->o_del > 1023 || sc->o_ins < 0 || sc->o_ins > 1023) return XO_EINVAL;
  if (sc->e_del < 1 || sc->e_del > 1023 || sc->e_ins < 1 || sc->e_ins > 1023) return XO_EINVAL;
  if (sc->w < 0) return XO_EINVAL;
  if (sc->end_bonus < 0 || sc->end_bonus > XO_BWA_MAX_END_BONUS) return XO_EINVAL;
  return XO_OK;
}

static int64_t score_bwa(const xo_bwa_scoring* sc, uint8_t a, uint8_t b) {
  if (a >= 4 || b >= 4) return sc->n_score;
  return a == b ? sc->match : sc->mismatch;
}

/* V4: the band half-width after narrowing for a query of length qlen. */
int64_t xo_bwa_band(const xo_bwa_scoring* sc, int64_t qlen, int flags) {
  if (flags & XO_BWA_NO_NARROW) return sc->w;
  const int64_t gain = qlen * sc->match + sc->end_bonus;
  const int64_t wi = gain < sc->o_ins ? 1 : (gain - sc->o_ins) / sc->e_ins + 1;
  const int64_t wd = gain < sc->o_del ? 1 : (gain - sc->o_del) / sc->e_del + 1;
  return min2(sc->w, min2(wi, wd));
}

/*
 * One extension under V1-V6.  out[7] and *cells as xo_extend_one.  Optional
 * traces: rows_beg/rows_end/rows_m/rows_mj per evaluated row (*n_rows of
 * them, the stop row included); full_H/M/E/F as (tlen+1) x (qlen+1) arrays,
 * entry [(r+1)*(qlen+1) + (c+1)] for cell (r,c), 0 where not computed.
 */
void xo_extend_one_bwa(const uint8_t* q, int32_t qlen, const uint8_t* t, int32_t tlen,
                       int32_t h0, const xo_bwa_scoring* sc, int flags, int32_t out[7],
                       int64_t* cells, int64_t* rows_beg, int64_t* rows_end, int64_t* rows_m,
                       int64_t* rows_mj, int32_t* n_rows, int64_t* full_H, int64_t* full_M,
                       int64_t* full_E, int64_t* full_F) {
  const int64_t oe_ins = (int64_t)sc->o_ins + sc->e_ins, e_ins = sc->e_ins;
  const int64_t oe_del = (int64_t)sc->o_del + sc->e_del, e_del = sc->e_del;
  if (n_rows) *n_rows = 0;
  *cells = 0;
  if (qlen == 0) {
    out[0] = h0; out[1] = 0; out[2] = 0; out[3] = h0; out[4] = 0; out[5] = 0; out[6] = XO_OK;
    return;
  }
  if (tlen == 0) {
    out[0] = h0; out[1] = 0; out[2] = 0; out[3] = -1; out[4] = 0; out[5] = 0; out[6] = XO_OK;
    return;
  }
  const int64_t w = xo_bwa_band(sc, qlen, flags);
  const int64_t ncol = (int64_t)qlen + 1; /* index c+1 holds column c, index 0 column -1 */
  int64_t* Hp = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Mp = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Fp = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Hc = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Mc = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Ec = calloc((size_t)ncol, sizeof(int64_t));
  int64_t* Fc = calloc((size_t)ncol, sizeof(int64_t));

  /* Row -1 (V3): the seed and the insertion run; its cells hold no M or F. */
  Hp[0] = h0;
  for (int64_t c = 0; c < qlen; ++c)
    if (in_band(-1, c, w)) Hp[c + 1] = max2(0, h0 - oe_ins - e_ins * c);
  if (full_H) {
    for (int64_t c = 0; c < ncol; ++c) {
      full_H[c] = Hp[c]; full_M[c] = 0; full_E[c] = 0; full_F[c] = 0;
    }
  }

  int64_t best = h0, bi = -1, bj = -1, max_off = 0;
  int64_t gscore = -1, gtle = 0;
  int64_t next_beg = 0, next_end = qlen; /* V5: the columns the last run reaches */
  int64_t n_cells = 0;
  for (int64_t i = 0; i < tlen; ++i) {
    int64_t beg = max2(next_beg, i - w);
    int64_t end = min2(min2(next_end, i + w + 1), qlen);
    for (int64_t c = 0; c < ncol; ++c) { Hc[c] = 0; Mc[c] = 0; Ec[c] = 0; Fc[c] = 0; }
    /* V3: column -1 of this row, the diagonal source of (i+1, 0). */
    if (beg == 0 && in_band(i, -1, w)) Hc[0] = max2(0, h0 - oe_del - e_del * i);
    int64_t m = 0, mj = -1;
    for (int64_t j = beg; j < end; ++j) {
      const int64_t D = Hp[j];
      const int64_t M = D > 0 ? D + score_bwa(sc, t[i], q[j]) : 0;
      const int64_t E = j == beg ? 0 : max2(0, max2(Mc[j] - oe_ins, Ec[j] - e_ins));
      const int64_t F = max2(0, max2(Mp[j + 1] - oe_del, Fp[j + 1] - e_del));
      const int64_t H = max2(M, max2(E, F));
      Hc[j + 1] = H; Mc[j + 1] = M; Ec[j + 1] = E; Fc[j + 1] = F;
      if (H >= m) { m = H; mj = j; }
    }
    if (end <= beg) { m = 0; mj = -1; }
    if (full_H) {
      for (int64_t c = 0; c < ncol; ++c) {
        full_H[(i + 1) * ncol + c] = Hc[c];
        full_M[(i + 1) * ncol + c] = c == 0 ? 0 : Mc[c];
        full_E[(i + 1) * ncol + c] = Ec[c];
        full_F[(i + 1) * ncol + c] = Fc[c];
      }
    }
    if (rows_beg) { rows_beg[i] = beg; rows_end[i] = end; rows_m[i] = m; rows_mj[i] = mj; }
    if (n_rows) *n_rows = (int32_t)(i + 1);
    /* V6, in order: gscore, the dead-row stop, the local best and z-drop. */
    if (beg < end && end == qlen && Hc[qlen] >= gscore) { gscore = Hc[qlen]; gtle = i + 1; }
    if (m == 0) break;
    n_cells += end - beg;
    if (m > best) {
      best = m; bi = i; bj = mj;
      max_off = max2(max_off, iabs64(mj - i));
    } else if (sc->zdrop > 0) {
      const int64_t di = i - bi, dj = mj - bj;
      const int64_t drop = di > dj ? best - m - (di - dj) * e_del : best - m - (dj - di) * e_ins;
      if (drop > sc->zdrop) break;
    }
    /* V5: the first and the last live column of the row (m > 0 here, so both
     * exist inside [beg, end)). */
    int64_t a = beg, b = end - 1;
    while (Hc[a + 1] == 0) ++a;  /* Hc[a+1] holds column a */
    while (Hc[b + 1] == 0) --b;
    if (flags & XO_BWA_NO_TRIM) { next_beg = 0; next_end = qlen; }
    else { next_beg = a; next_end = b + 2; }
    int64_t* tmp;
    tmp = Hp; Hp = Hc; Hc = tmp;
    tmp = Mp; Mp = Mc; Mc = tmp;
    tmp = Fp; Fp = Fc; Fc = tmp;
  }
  *cells = n_cells;
  out[0] = (int32_t)best; out[1] = (int32_t)(bj + 1); out[2] = (int32_t)(bi + 1);
  out[3] = (int32_t)gscore; out[4] = (int32_t)gtle; out[5] = (int32_t)max_off; out[6] = XO_OK;
  free(Hp); free(Mp); free(Fp); free(Hc); free(Mc); free(Ec); free(Fc);
}

/* Per-pair input checks; returns XO_OK or XO_EINVAL. */
static int check_pair(int64_t qo, int32_t ql, int64_t q_bytes, int64_t to, int32_t tl,
                      int64_t t_bytes, int32_t h0) {
  if (h0 < 1 || h0 > XO_MAX_H0) return XO_EINVAL;
  if (ql < 0 || tl < 0 || ql > XO_MAX_LEN || tl > XO_MAX_LEN) return XO_EINVAL;
  if (qo < 0 || to < 0) return XO_EINVAL;
  if (qo > q_bytes - ql || to > t_bytes - tl) return XO_EINVAL;
  return XO_OK;
}

typedef struct {
  const uint8_t* q_seq; int64_t q_bytes; const int64_t* q_off; const int32_t* q_len;
  const uint8_t* t_seq; int64_t t_bytes; const int64_t* t_off; const int32_t* t_len;
  const int32_t* h0; int64_t n; const xo_scoring* sc; int32_t* out; int64_t* cells;
  int64_t next; /* next unclaimed pair, taken in chunks */
  const xo_bwa_scoring* bsc; /* non-NULL: the BWA-MEM-compatible variant with this scoring */
} batch_job;


/* The BWA-MEM-compatible variant also bounds the row width it computes:
 * min(qlen, 2w'+1) columns (w' the narrowed band), a limit shared in value
 * with the library. */
#define XO_BWA_MAX_WIDTH 8192

static int bwa_width_ok(const xo_bwa_scoring* sc, int32_t ql) {
  const int64_t w = xo_bwa_band(sc, ql, 0);
  return min2(ql, 2 * w + 1) <= XO_BWA_MAX_WIDTH;
}

static void run_pair(batch_job* b, int64_t k) {
  int32_t* o = b->out + 7 * k;
  if (check_pair(b->q_off[k], b->q_len[k], b->q_bytes, b->t_off[k], b->t_len[k], b->t_bytes,
                 b->h0[k]) != XO_OK ||
      (b->bsc && !bwa_width_ok(b->bsc, b->q_len[k]))) {
    memset(o, 0, 7 * sizeof(int32_t));
    o[6] = XO_EINVAL;
    if (b->cells) b->cells[k] = 0;
    return;
  }
  int64_t c = 0;
  if (b->bsc)
    xo_extend_one_bwa(b->q_seq + b->q_off[k], b->q_len[k], b->t_seq + b->t_off[k], b->t_len[k],
                      b->h0[k], b->bsc, 0, o, &c, NULL, NULL, NULL, NULL, NULL, NULL, NULL,
                      NULL, NULL);
  else
    xo_extend_one(b->q_seq + b->q_off[k], b->q_len[k], b->t_seq + b->t_off[k], b->t_len[k],
                  b->h0[k], b->sc, o, &c, NULL, NULL, NULL, NULL, NULL, NULL);
  if (b->cells) b->cells[k] = c;
}

static void* worker(void* arg) {
  batch_job* b = (batch_job*)arg;
  const int64_t chunk = 64;
  for (;;) {
    int64_t s = __atomic_fetch_add(&b->next, chunk, __ATOMIC_RELAXED);
    if (s >= b->n) break;
    int64_t e = s + chunk < b->n ? s + chunk : b->n;
    for (int64_t k = s; k < e; ++k) run_pair(b, k);
  }
  return NULL;
}

static int run_batch(batch_job* bp, int nthreads) {
  batch_job b = *bp;
  if (nthreads < 1) nthreads = 1;
  if (nthreads == 1) {
    worker(&b);
    return XO_OK;
  }
  pthread_t* th = malloc(sizeof(pthread_t) * (size_t)nthreads);
  int started = 0;
  for (int k = 0; k < nthreads; ++k)
    if (pthread_create(&th[started], NULL, worker, &b) == 0) ++started;
  if (started == 0) worker(&b);
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
  free(th);
  return XO_OK;
}

/*
 * Batch of independent pairs, spread over nthreads host threads (pairs are
 * independent, so the split does not change any result).  Returns XO_EINVAL
 * for an unacceptable scoring record (nothing is written), else XO_OK.
 */
int xo_extend_batch(const uint8_t* q_seq, int64_t q_bytes, const int64_t* q_off,
                    const int32_t* q_len, const uint8_t* t_seq, int64_t t_bytes,
                    const int64_t* t_off, const int32_t* t_len, const int32_t* h0, int64_t n,
                    const xo_scoring* sc, int32_t* out, int64_t* cells, int nthreads) {
  if (xo_check_scoring(sc) != XO_OK || n < 0) return XO_EINVAL;
  batch_job b = {q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n, sc, out,
                 cells, 0, NULL};
  return run_batch(&b, nthreads);
}


/* The batch runner for the BWA-MEM-compatible variant (same layout). */
int xo_extend_batch_bwa(const uint8_t* q_seq, int64_t q_bytes, const int64_t* q_off,
                        const int32_t* q_len, const uint8_t* t_seq, int64_t t_bytes,
                        const int64_t* t_off, const int32_t* t_len, const int32_t* h0, int64_t n,
                        const xo_bwa_scoring* sc, int32_t* out, int64_t* cells, int nthreads) {
  if (xo_check_bwa_scoring(sc) != XO_OK || n < 0) return XO_EINVAL;
  batch_job b = {q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n, NULL, out,
                 cells, 0, sc};
  return run_batch(&b, nthreads);
}
