/*
 * wfa_oracle.c -- plain, slow, obviously correct CPU oracle for exact
 * gap-affine pairwise alignment of (pattern, text) pairs.
 *
 * TEST INFRASTRUCTURE ONLY.  The library under test never links, loads or
 * calls this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What is computed (the method the paper aligns with, "WFA", Sec. I, which
 * it runs unmodified, Sec. I "no optimizations"):
 *   score(P, T) = min over all global alignments of P (length n, index v)
 *   and T (length m, index h) of
 *       x * (#mismatch columns) + sum over maximal gap runs of (o + L*e)
 *   where a gap run is a maximal run of L consecutive columns of the same
 *   kind: I (consumes one text char) or D (consumes one pattern char).
 *   An I run directly followed by a D run counts as two runs.  Matches cost 0.
 *
 * Four independent computations of that quantity live here:
 *   oracle_brute   enumerate every alignment path, rescore each (tiny n, m)
 *   oracle_gotoh   textbook O(nm) three-matrix DP plus a walk-back traceback
 *   oracle_wfa     the wavefront recurrences, step by step in the score
 *   oracle_rescore the cost of one given alignment (the definition above)
 *
 * Canonical alignment (tie-break; the paper is silent, this is the reading
 * every implementation in this project follows):
 *   walking backwards from the end, at a position where the alignment may
 *   continue with several optimal operations, prefer the one that ends at the
 *   largest text offset (fewest trailing matches), and among equal offsets
 *   prefer X over I over D; inside a gap, extending the gap is preferred over
 *   opening it.
 *
 * Alignment operations are written as characters:
 *   'M' match, 'X' mismatch, 'I' (consumes text only), 'D' (consumes pattern
 *   only).  Run-length words are (len << 4) | op with op 0=M 1=X 2=I 3=D.
 *
 * Ends-free alignment (the *_ef functions; not in the paper, which aligns
 * reads end to end, Sec. I -- a variant of the cited method; the reading
 * used here): up to pb leading and pe trailing pattern characters, and up to
 * tb leading and te trailing text characters, may be left unaligned at no
 * cost.  The alignment starts at (v, 0) with v <= pb or at (0, h) with
 * h <= tb, and ends at (n, h) with h >= m - te or at (v, m) with
 * v >= n - pe; a gap after the start or before the end is paid as usual.
 * The op string still covers both sequences: the skipped characters are its
 * leading / trailing D (pattern) or I (text) ops.  Among optimal end cells
 * the one on the diagonal k = h - v closest to m - n is taken, the larger k
 * on a tie.  All four lengths 0 is the global alignment above.
 *
 * Status codes per pair: 0 ok, 1 score above max_score, 2 invalid character.
 */
#include <limits.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_SCORE_LIMIT 1
#define OR_INVALID_CHAR 2

/* ------------------------------------------------------------------ chars */

/* A/C/G/T, either case -> 0/1/2/3; anything else -> -1. */
static int base_code(unsigned char c) {
  switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
  }
}

int oracle_valid(const char *s, int64_t len) {
  for (int64_t i = 0; i < len; i++)
    if (base_code((unsigned char)s[i]) < 0) return 0;
  return 1;
}

static int same(const char *P, int64_t v, const char *T, int64_t h) {
  return base_code((unsigned char)P[v]) == base_code((unsigned char)T[h]);
}

/* ---------------------------------------------------------------- rescore */

/* Cost of the alignment given by ops[0..nops) under (x, o, e), or -1 if the
 * ops are not an alignment of P and T: wrong consumption, 'M' on unequal
 * characters or 'X' on equal characters.  This is the plain definition. */
int64_t oracle_rescore(const char *P, int64_t n, const char *T, int64_t m,
                       const char *ops, int64_t nops, int64_t x, int64_t o,
                       int64_t e) {
  int64_t v = 0, h = 0, cost = 0;
  char prev = 0;
  for (int64_t i = 0; i < nops; i++) {
    char op = ops[i];
    if (op == 'M' || op == 'X') {
      if (v >= n || h >= m) return -1;
      int eq = same(P, v, T, h);
      if (op == 'M' && !eq) return -1;
      if (op == 'X' && eq) return -1;
      if (op == 'X') cost += x;
      v++; h++;
    } else if (op == 'I') {
      if (h >= m) return -1;
      cost += (prev == 'I') ? e : o + e;
      h++;
    } else if (op == 'D') {
      if (v >= n) return -1;
      cost += (prev == 'D') ? e : o + e;
      v++;
    } else {
      return -1;
    }
    prev = op;
  }
  if (v != n || h != m) return -1;
  return cost;
}

/* Cost of the alignment ops[0..nops) under the ends-free rules (pb, pe, tb,
 * te; all 0 = oracle_rescore), or -1 if ops is not an alignment of P and T.
 * The leading run of ops, if it is D (resp. I), has up to pb (resp. tb) of
 * its characters free, the trailing run up to pe (resp. te); the free
 * characters are taken at the sequence ends, and the rest of such a run is
 * one gap.  Taking as many free characters as allowed is never worse, so
 * that is the cost: the plain cost less what the free characters save (a
 * whole free run saves o + L*e, a partly free one e per free character). */
int64_t oracle_rescore_ef(const char *P, int64_t n, const char *T, int64_t m,
                          const char *ops, int64_t nops, int64_t x, int64_t o,
                          int64_t e, int64_t pb, int64_t pe, int64_t tb,
                          int64_t te) {
  int64_t cost = oracle_rescore(P, n, T, m, ops, nops, x, o, e);
  if (cost < 0 || nops == 0) return cost;
  int64_t l0 = 0, l1 = 0;
  while (l0 < nops && ops[l0] == ops[0]) l0++;
  while (l1 < nops && ops[nops - 1 - l1] == ops[nops - 1]) l1++;
  int64_t fb = ops[0] == 'D' ? pb : ops[0] == 'I' ? tb : 0;
  int64_t fe = ops[nops - 1] == 'D' ? pe : ops[nops - 1] == 'I' ? te : 0;
  if (l0 == nops) {
    /* one run: if a gap, both of its ends are free */
    int64_t f = fb + fe < nops ? fb + fe : nops;
    return f == nops ? 0 : cost - f * e;
  }
  int64_t f0 = l0 < fb ? l0 : fb, f1 = l1 < fe ? l1 : fe;
  cost -= f0 == l0 ? o + l0 * e : f0 * e;
  cost -= f1 == l1 ? o + l1 * e : f1 * e;
  return cost;
}

/* ops string -> run-length words (len << 4) | code.  Returns the number of
 * runs, or -1 if cap is too small. */
int64_t oracle_runs_encode(const char *ops, int64_t nops, uint32_t *runs,
                           int64_t cap) {
  int64_t r = 0, i = 0;
  while (i < nops) {
    int64_t j = i;
    while (j < nops && ops[j] == ops[i]) j++;
    uint32_t code = ops[i] == 'M' ? 0u : ops[i] == 'X' ? 1u : ops[i] == 'I' ? 2u : 3u;
    if (r >= cap) return -1;
    runs[r++] = ((uint32_t)(j - i) << 4) | code;
    i = j;
  }
  return r;
}

/* ------------------------------------------------------------- brute force */

/* Rank of op c in the reversed op string given the previous reversed op:
 * a gap continues before anything else; otherwise X < I < D < M. */
static int lex_rank(char c, char prev) {
  if ((prev == 'I' && c == 'I') || (prev == 'D' && c == 'D')) return 0;
  switch (c) {
    case 'X': return 1;
    case 'I': return 2;
    case 'D': return 3;
    default: return 4;
  }
}

/* Is reversed(a) (length la) smaller than reversed(b) (length lb) under
 * lex_rank?  A proper prefix is smaller. */
static int lex_less_reversed(const char *a, int la, const char *b, int lb) {
  char prev = 0;
  int i = la - 1, j = lb - 1;
  while (i >= 0 && j >= 0) {
    if (a[i] != b[j]) return lex_rank(a[i], prev) < lex_rank(b[j], prev);
    prev = a[i];
    i--;
    j--;
  }
  return i < 0 && j >= 0;
}

typedef struct {
  const char *P, *T;
  int n, m;
  int64_t x, o, e;
  int64_t pb, pe, tb, te;
  char path[32];
  int64_t best;
  char best_ops[32];
  int best_len;
  int64_t count;
} brute_t;

static void brute_rec(brute_t *b, int v, int h, int len) {
  if (v == b->n && h == b->m) {
    int64_t c = oracle_rescore_ef(b->P, b->n, b->T, b->m, b->path, len, b->x,
                                  b->o, b->e, b->pb, b->pe, b->tb, b->te);
    b->count++;
    if (c < 0) return; /* cannot happen: diagonal steps are labelled M/X by
                          character equality */
    if (b->best < 0 || c < b->best ||
        (c == b->best &&
         lex_less_reversed(b->path, len, b->best_ops, b->best_len))) {
      b->best = c;
      memcpy(b->best_ops, b->path, (size_t)len);
      b->best_len = len;
    }
    return;
  }
  if (v < b->n && h < b->m) {
    b->path[len] = same(b->P, v, b->T, h) ? 'M' : 'X';
    brute_rec(b, v + 1, h + 1, len + 1);
  }
  if (h < b->m) {
    b->path[len] = 'I';
    brute_rec(b, v, h + 1, len + 1);
  }
  if (v < b->n) {
    b->path[len] = 'D';
    brute_rec(b, v + 1, h, len + 1);
  }
}

/* Minimum cost over every alignment of P and T (n, m <= 12) under the
 * ends-free rules (oracle_rescore_ef), and the alignment whose reversed op
 * string is smallest under lex_rank among the optimal ones.  Returns the
 * cost, -1 on bad arguments.  *npaths receives the number of alignments
 * enumerated (a Delannoy number). */
int64_t oracle_brute_ef(const char *P, int n, const char *T, int m, int64_t x,
                        int64_t o, int64_t e, int64_t pb, int64_t pe, int64_t tb,
                        int64_t te, char *ops, int64_t *nops, int64_t *npaths) {
  if (n < 0 || m < 0 || n > 12 || m > 12) return -1;
  brute_t b;
  memset(&b, 0, sizeof b);
  b.P = P; b.T = T; b.n = n; b.m = m; b.x = x; b.o = o; b.e = e;
  b.pb = pb; b.pe = pe; b.tb = tb; b.te = te;
  b.best = -1;
  brute_rec(&b, 0, 0, 0);
  if (ops) memcpy(ops, b.best_ops, (size_t)b.best_len);
  if (nops) *nops = b.best_len;
  if (npaths) *npaths = b.count;
  return b.best;
}

/* The global alignment: oracle_brute_ef with no free ends. */
int64_t oracle_brute(const char *P, int n, const char *T, int m, int64_t x,
                     int64_t o, int64_t e, char *ops, int64_t *nops,
                     int64_t *npaths) {
  return oracle_brute_ef(P, n, T, m, x, o, e, 0, 0, 0, 0, ops, nops, npaths);
}

/* ------------------------------------------------------------------ Gotoh */

#define BIG (INT64_MAX / 4)

static int64_t min2(int64_t a, int64_t b) { return a < b ? a : b; }

/* Textbook gap-affine DP (Gotoh):
 *   H(0,0) = 0
 *   I(v,h) = min(H(v,h-1) + o + e, I(v,h-1) + e)     text char consumed
 *   D(v,h) = min(H(v-1,h) + o + e, D(v-1,h) + e)     pattern char consumed
 *   H(v,h) = min(H(v-1,h-1) + (P[v-1]==T[h-1] ? 0 : x), I(v,h), D(v,h))
 * out-of-range terms are +infinity; score = H(n,m).
 * Ends-free (pb, pe, tb, te): H(v,0) = 0 for v <= pb and H(0,h) = 0 for
 * h <= tb (free starts); the score is the least H over the end cells (n, h),
 * h >= m - te, and (v, m), v >= n - pe.
 * If ops is not NULL the canonical alignment is recovered by walking back
 * from the chosen end cell (see the header) with the project's tie-break
 * (mismatch, then gap, then match at each cell; inside a gap extend before
 * open) down to a free start, and written forward into ops (the skipped
 * characters as leading / trailing D or I ops), *nops receiving its length.
 * Returns the score, or -1 on allocation failure.  Memory is 3 (n+1)(m+1)
 * int64. */
int64_t oracle_gotoh_ef(const char *P, int64_t n, const char *T, int64_t m,
                        int64_t x, int64_t o, int64_t e, int64_t pb, int64_t pe,
                        int64_t tb, int64_t te, char *ops, int64_t *nops) {
  int64_t W = m + 1;
  size_t cells = (size_t)(n + 1) * (size_t)(m + 1);
  int64_t *H = malloc(cells * sizeof(int64_t));
  int64_t *I = malloc(cells * sizeof(int64_t));
  int64_t *D = malloc(cells * sizeof(int64_t));
  if (!H || !I || !D) { free(H); free(I); free(D); return -1; }
#define AT(A, v, h) A[(v) * W + (h)]
  for (int64_t v = 0; v <= n; v++) {
    for (int64_t h = 0; h <= m; h++) {
      int64_t iv = BIG, dv = BIG, hv = BIG;
      if (h > 0) iv = min2(AT(H, v, h - 1) + o + e, AT(I, v, h - 1) + e);
      if (v > 0) dv = min2(AT(H, v - 1, h) + o + e, AT(D, v - 1, h) + e);
      if ((h == 0 && v <= pb) || (v == 0 && h <= tb)) hv = 0; /* a start */
      if (v > 0 && h > 0)
        hv = min2(hv, AT(H, v - 1, h - 1) + (same(P, v - 1, T, h - 1) ? 0 : x));
      hv = min2(hv, min2(iv, dv));
      AT(I, v, h) = iv;
      AT(D, v, h) = dv;
      AT(H, v, h) = hv;
    }
  }
  /* the end cell: least H, then diagonal k = h - v nearest m - n (the
   * larger k on a tie): d = 0, 1, ... tries k = kf + d (text end, (m - k,
   * m)) before k = kf - d (pattern end, (n, n + k)) */
  int64_t score = BIG, ev = n, eh = m;
  int64_t dmax = pe > te ? pe : te;
  for (int64_t d = 0; d <= dmax; d++) {
    if (d <= pe && d <= n) {
      int64_t v = n - d; /* (v, m) on k = kf + d */
      if (AT(H, v, m) < score) { score = AT(H, v, m); ev = v; eh = m; }
    }
    if (d > 0 && d <= te && d <= m) {
      int64_t h = m - d; /* (n, h) on k = kf - d */
      if (AT(H, n, h) < score) { score = AT(H, n, h); ev = n; eh = h; }
    }
  }
  if (ops) {
    /* Walk back: state 0 = "M" (any op may come next), 1 = inside I, 2 =
     * inside D.  Ops are produced last-to-first, then reversed. */
    int64_t v = ev, h = eh, s = score, k = 0;
    for (int64_t i = 0; i < n - ev; i++) ops[k++] = 'D'; /* free pattern end */
    for (int64_t i = 0; i < m - eh; i++) ops[k++] = 'I'; /* free text end */
    int state = 0;
    for (;;) {
      if (state == 0 && s == 0 && ((h == 0 && v <= pb) || (v == 0 && h <= tb))) {
        /* a free start: the skipped prefix */
        for (int64_t i = 0; i < v; i++) ops[k++] = 'D';
        for (int64_t i = 0; i < h; i++) ops[k++] = 'I';
        break;
      }
      if (state == 0) {
        if (v > 0 && h > 0 && !same(P, v - 1, T, h - 1) &&
            AT(H, v - 1, h - 1) + x == s) {
          ops[k++] = 'X';
          v--; h--; s -= x;
        } else if (h > 0 && AT(I, v, h) == s) {
          state = 1;
        } else if (v > 0 && AT(D, v, h) == s) {
          state = 2;
        } else if (v > 0 && h > 0 && same(P, v - 1, T, h - 1) &&
                   AT(H, v - 1, h - 1) == s) {
          ops[k++] = 'M';
          v--; h--;
        } else {
          score = -2; /* inconsistent matrices: cannot happen */
          break;
        }
      } else if (state == 1) {
        ops[k++] = 'I';
        if (h > 1 && AT(I, v, h - 1) + e == s) {
          s -= e; h--;
        } else if (AT(H, v, h - 1) + o + e == s) {
          s -= o + e; h--; state = 0;
        } else {
          score = -2;
          break;
        }
      } else {
        ops[k++] = 'D';
        if (v > 1 && AT(D, v - 1, h) + e == s) {
          s -= e; v--;
        } else if (AT(H, v - 1, h) + o + e == s) {
          s -= o + e; v--; state = 0;
        } else {
          score = -2;
          break;
        }
      }
    }
    for (int64_t i = 0, j = k - 1; i < j; i++, j--) {
      char t = ops[i]; ops[i] = ops[j]; ops[j] = t;
    }
    *nops = k;
  }
#undef AT
  free(H); free(I); free(D);
  return score;
}

/* The global alignment: oracle_gotoh_ef with no free ends. */
int64_t oracle_gotoh(const char *P, int64_t n, const char *T, int64_t m,
                     int64_t x, int64_t o, int64_t e, char *ops,
                     int64_t *nops) {
  return oracle_gotoh_ef(P, n, T, m, x, o, e, 0, 0, 0, 0, ops, nops);
}

/* -------------------------------------------------------------------- WFA */

/* Offsets are text positions h on diagonal k = h - v.  A missing value is
 * NUL.  Every wavefront keeps M, I and D over its own [lo, hi]. */
#define NUL INT64_MIN

typedef struct {
  int exists;
  int64_t lo, hi;
  int64_t *M, *I, *D;
} wavefront;

typedef struct {
  int64_t cells;         /* sum of (hi - lo + 1) over existing wavefronts */
  int64_t wavefronts;    /* number of existing wavefronts */
  int64_t char_compares; /* character comparisons made by extend */
  int64_t bt_steps;      /* backtrace state visits */
} oracle_counts;

static int64_t wf_get(const wavefront *wf, int64_t s, int64_t k, char comp) {
  if (s < 0 || !wf[s].exists || k < wf[s].lo || k > wf[s].hi) return NUL;
  int64_t i = k - wf[s].lo;
  return comp == 'M' ? wf[s].M[i] : comp == 'I' ? wf[s].I[i] : wf[s].D[i];
}

static int64_t max_non_null(int64_t a, int64_t b) {
  if (a == NUL) return b;
  if (b == NUL) return a;
  return a > b ? a : b;
}

/* Extend: while v < n, h < m and P[v] == T[h], advance h (v = h - k). */
static int64_t extend(const char *P, int64_t n, const char *T, int64_t m,
                      int64_t k, int64_t h, oracle_counts *cnt) {
  while (h - k < n && h < m) {
    if (cnt) cnt->char_compares++;
    if (!same(P, h - k, T, h)) break;
    h++;
  }
  return h;
}

static void wf_free(wavefront *wf, int64_t count) {
  for (int64_t s = 0; s < count; s++) {
    free(wf[s].M); free(wf[s].I); free(wf[s].D);
  }
  free(wf);
}

/* Gap-affine WFA (Marco-Sola et al. 2021, the method cited in Sec. I):
 *   I_s[k] = max(M_{s-o-e}[k-1], I_{s-e}[k-1]) + 1
 *   D_s[k] = max(M_{s-o-e}[k+1], D_{s-e}[k+1])
 *   M_s[k] = max(M_{s-x}[k] + 1, I_s[k], D_s[k]), then extend,
 * with M_0[0] = extend(0).  A candidate past the end of a sequence
 * (h > m or v = h - k > n) is dropped before the maximum is taken.
 * lo_s/hi_s cover the sources that exist; a wavefront whose entries are all
 * missing does not exist.  s runs 0, 1, 2, ... and the result is the first
 * s with M_s[m-n] == m.
 * Ends-free (pb, pe, tb, te): the free starts are the score-0 wavefront,
 * M_0[k] = extend(max(k, 0)) on diagonals -min(pb, n) <= k <= min(tb, m);
 * the result is the first s at which some diagonal reaches an end cell:
 * M_s[k] == m for kf <= k <= kf + pe (text end), M_s[k] == n + k for
 * kf - te <= k < kf (pattern end), kf = m - n; the nearest such k to kf
 * ends the alignment (the larger on a tie).
 *
 * If max_score > 0 and no s <= max_score reaches the end, the status is
 * OR_SCORE_LIMIT.  If want_ops, the canonical alignment is written forward
 * into ops (capacity ops_cap) with its length in *nops; returns -3 if ops_cap
 * is too small, -2 on allocation failure, else the pair status. */
int oracle_wfa_ef(const char *P, int64_t n, const char *T, int64_t m, int64_t x,
                  int64_t o, int64_t e, int64_t pb, int64_t pe, int64_t tb,
                  int64_t te, int64_t max_score, int want_ops,
                  int64_t *score_out, char *ops, int64_t ops_cap, int64_t *nops,
                  oracle_counts *cnt) {
  *score_out = -1;
  if (nops) *nops = 0;
  if (!oracle_valid(P, n) || !oracle_valid(T, m)) return OR_INVALID_CHAR;
  int64_t kf = m - n;
  int64_t cap = 64, s_final = -1, k_end = kf, h_end = m;
  wavefront *wf = calloc((size_t)cap, sizeof(wavefront));
  if (!wf) return -2;

  for (int64_t s = 0;; s++) {
    if (max_score > 0 && s > max_score) {
      wf_free(wf, cap);
      return OR_SCORE_LIMIT;
    }
    if (s >= cap) {
      wavefront *nw = realloc(wf, (size_t)(2 * cap) * sizeof(wavefront));
      if (!nw) { wf_free(wf, cap); return -2; }
      memset(nw + cap, 0, (size_t)cap * sizeof(wavefront));
      wf = nw;
      cap *= 2;
    }
    wavefront *w = &wf[s];
    if (s == 0) {
      int64_t lo = -(pb < n ? pb : n), hi = tb < m ? tb : m;
      w->exists = 1;
      w->lo = lo;
      w->hi = hi;
      w->M = malloc((size_t)(hi - lo + 1) * sizeof(int64_t));
      w->I = malloc((size_t)(hi - lo + 1) * sizeof(int64_t));
      w->D = malloc((size_t)(hi - lo + 1) * sizeof(int64_t));
      if (!w->M || !w->I || !w->D) { wf_free(wf, cap); return -2; }
      for (int64_t k = lo; k <= hi; k++) {
        /* start (0, k) for k >= 0, (-k, 0) for k < 0 */
        w->M[k - lo] = extend(P, n, T, m, k, k > 0 ? k : 0, cnt);
        w->I[k - lo] = NUL;
        w->D[k - lo] = NUL;
      }
    } else {
      int64_t sx = s - x, so = s - o - e, se = s - e;
      int ex_x = sx >= 0 && wf[sx].exists;
      int ex_o = so >= 0 && wf[so].exists;
      int ex_e = se >= 0 && wf[se].exists;
      if (!ex_x && !ex_o && !ex_e) continue;
      int64_t lo = INT64_MAX, hi = INT64_MIN;
      if (ex_x) {
        if (wf[sx].lo < lo) lo = wf[sx].lo;
        if (wf[sx].hi > hi) hi = wf[sx].hi;
      }
      if (ex_o) {
        if (wf[so].lo - 1 < lo) lo = wf[so].lo - 1;
        if (wf[so].hi + 1 > hi) hi = wf[so].hi + 1;
      }
      if (ex_e) {
        if (wf[se].lo - 1 < lo) lo = wf[se].lo - 1;
        if (wf[se].hi + 1 > hi) hi = wf[se].hi + 1;
      }
      int64_t width = hi - lo + 1;
      w->lo = lo;
      w->hi = hi;
      w->M = malloc((size_t)width * sizeof(int64_t));
      w->I = malloc((size_t)width * sizeof(int64_t));
      w->D = malloc((size_t)width * sizeof(int64_t));
      if (!w->M || !w->I || !w->D) { wf_free(wf, cap); return -2; }
      int any = 0;
      for (int64_t k = lo; k <= hi; k++) {
        /* I: opens from M_{s-o-e}[k-1] or extends I_{s-e}[k-1]; +1 text */
        int64_t iv = max_non_null(wf_get(wf, so, k - 1, 'M'),
                                  wf_get(wf, se, k - 1, 'I'));
        if (iv != NUL) {
          iv += 1;
          if (iv > m) iv = NUL;
        }
        /* D: opens from M_{s-o-e}[k+1] or extends D_{s-e}[k+1]; h fixed */
        int64_t dv = max_non_null(wf_get(wf, so, k + 1, 'M'),
                                  wf_get(wf, se, k + 1, 'D'));
        if (dv != NUL && dv - k > n) dv = NUL;
        /* X: mismatch from M_{s-x}[k] */
        int64_t xv = wf_get(wf, sx, k, 'M');
        if (xv != NUL) {
          xv += 1;
          if (xv > m || xv - k > n) xv = NUL;
        }
        int64_t mv = max_non_null(xv, max_non_null(iv, dv));
        if (mv != NUL) mv = extend(P, n, T, m, k, mv, cnt);
        w->M[k - lo] = mv;
        w->I[k - lo] = iv;
        w->D[k - lo] = dv;
        if (mv != NUL || iv != NUL || dv != NUL) any = 1;
      }
      if (!any) {
        free(w->M); free(w->I); free(w->D);
        w->M = w->I = w->D = NULL;
        continue;
      }
      w->exists = 1;
    }
    if (cnt) {
      cnt->cells += w->hi - w->lo + 1;
      cnt->wavefronts++;
    }
    /* end test, nearest diagonal to kf first (the larger k on a tie) */
    int64_t dmax = pe > te ? pe : te;
    for (int64_t d = 0; d <= dmax && s_final < 0; d++) {
      if (d <= pe && wf_get(wf, s, kf + d, 'M') == m) {
        s_final = s; k_end = kf + d; h_end = m;
      } else if (d > 0 && d <= te && wf_get(wf, s, kf - d, 'M') == n + kf - d) {
        s_final = s; k_end = kf - d; h_end = n + kf - d;
      }
    }
    if (s_final >= 0) break;
  }

  *score_out = s_final;
  int rc = OR_OK;
  if (want_ops) {
    /* Backtrace from (M, s*, k_end, h_end).  Ops come out last-to-first:
     * first the free end (the pattern or text characters past the end
     * cell). */
    int64_t s = s_final, k = k_end, h = h_end, len = 0;
    char state = 'M';
    for (int64_t i = 0; i < (n - (h_end - k_end)) + (m - h_end); i++) {
      if (len >= ops_cap) { rc = -3; goto done; }
      ops[len++] = k_end > kf ? 'D' : 'I';
    }
    for (;;) {
      if (cnt) cnt->bt_steps++;
      if (state == 'M') {
        if (s == 0) {
          /* a free start on diagonal k: (0, k) or (-k, 0), then matches */
          int64_t h0 = k > 0 ? k : 0;
          for (int64_t i = 0; i < h - h0; i++) {
            if (len >= ops_cap) { rc = -3; goto done; }
            ops[len++] = 'M';
          }
          for (int64_t i = 0; i < (k > 0 ? k : -k); i++) {
            if (len >= ops_cap) { rc = -3; goto done; }
            ops[len++] = k > 0 ? 'I' : 'D';
          }
          break;
        }
        int64_t xv = wf_get(wf, s - x, k, 'M');
        if (xv != NUL) {
          xv += 1;
          if (xv > m || xv - k > n) xv = NUL;
        }
        int64_t iv = wf_get(wf, s, k, 'I');
        int64_t dv = wf_get(wf, s, k, 'D');
        /* largest offset wins; ties: X, then I, then D */
        char pick;
        int64_t c;
        if (xv != NUL && (iv == NUL || xv >= iv) && (dv == NUL || xv >= dv)) {
          pick = 'X'; c = xv;
        } else if (iv != NUL && (dv == NUL || iv >= dv)) {
          pick = 'I'; c = iv;
        } else {
          pick = 'D'; c = dv;
        }
        for (int64_t i = 0; i < h - c; i++) {
          if (len >= ops_cap) { rc = -3; goto done; }
          ops[len++] = 'M';
        }
        if (pick == 'X') {
          if (len >= ops_cap) { rc = -3; goto done; }
          ops[len++] = 'X';
          s -= x;
          h = c - 1;
        } else {
          state = pick;
          h = c;
        }
      } else if (state == 'I') {
        if (len >= ops_cap) { rc = -3; goto done; }
        ops[len++] = 'I';
        if (wf_get(wf, s - e, k - 1, 'I') == h - 1) {
          s -= e;
        } else {
          s -= o + e;
          state = 'M';
        }
        k -= 1;
        h -= 1;
      } else {
        if (len >= ops_cap) { rc = -3; goto done; }
        ops[len++] = 'D';
        if (wf_get(wf, s - e, k + 1, 'D') == h) {
          s -= e;
        } else {
          s -= o + e;
          state = 'M';
        }
        k += 1;
      }
    }
    for (int64_t i = 0, j = len - 1; i < j; i++, j--) {
      char t = ops[i]; ops[i] = ops[j]; ops[j] = t;
    }
    if (nops) *nops = len;
  }
done:
  wf_free(wf, cap);
  return rc;
}

/* The global alignment: oracle_wfa_ef with no free ends. */
int oracle_wfa(const char *P, int64_t n, const char *T, int64_t m, int64_t x,
               int64_t o, int64_t e, int64_t max_score, int want_ops,
               int64_t *score_out, char *ops, int64_t ops_cap, int64_t *nops,
               oracle_counts *cnt) {
  return oracle_wfa_ef(P, n, T, m, x, o, e, 0, 0, 0, 0, max_score, want_ops, score_out, ops, ops_cap, nops,
                       cnt);
}

/* --------------------------------------------------------------- pack2bit */

/* The packed sequence format: code A=0 C=1 G=2 T=3 (either case), 32 bases
 * per 64-bit word, base 32w+j in bits (63-2j):(62-2j) of word w, bits past
 * the sequence end zero, followed by one all-zero pad word; that is
 * ceil(len/32) + 1 words.  Returns 0, or -1 if a byte is not A/C/G/T (the
 * words are then unspecified). */
int oracle_pack2bit(const char *s, int64_t len, uint64_t *words) {
  int64_t nw = (len + 31) / 32 + 1;
  for (int64_t w = 0; w < nw; w++) words[w] = 0;
  for (int64_t i = 0; i < len; i++) {
    int c = base_code((unsigned char)s[i]);
    if (c < 0) return -1;
    words[i / 32] |= (uint64_t)c << (62 - 2 * (i % 32));
  }
  return 0;
}

/* ------------------------------------------------------------------ batch */

typedef struct {
  int64_t begin, end;
  const char *pat; const int64_t *poff; const int32_t *plen;
  const char *txt; const int64_t *toff; const int32_t *tlen;
  int64_t x, o, e, max_score;
  int64_t pb, pe, tb, te;
  int want_ops;
  int32_t *scores; int8_t *status;
  uint32_t *runs; int64_t runs_per_pair; int32_t *nruns;
  oracle_counts counts;
  int err;
} batch_job;

static void *batch_worker(void *arg) {
  batch_job *j = arg;
  char *ops = NULL;
  int64_t ops_cap = 0;
  for (int64_t i = j->begin; i < j->end; i++) {
    int64_t n = j->plen[i], m = j->tlen[i];
    const char *P = j->pat + j->poff[i];
    const char *T = j->txt + j->toff[i];
    if (j->want_ops && n + m + 1 > ops_cap) {
      free(ops);
      ops_cap = 2 * (n + m + 1);
      ops = malloc((size_t)ops_cap);
      if (!ops) { j->err = -2; return NULL; }
    }
    int64_t score, nops = 0;
    int rc = oracle_wfa_ef(P, n, T, m, j->x, j->o, j->e, j->pb, j->pe, j->tb,
                           j->te, j->max_score, j->want_ops, &score, ops,
                           ops_cap, &nops, &j->counts);
    if (rc < 0) { j->err = rc; free(ops); return NULL; }
    j->status[i] = (int8_t)rc;
    j->scores[i] = rc == OR_OK ? (int32_t)score : -1;
    if (j->nruns) j->nruns[i] = 0;
    if (rc == OR_OK && j->want_ops) {
      int64_t r = oracle_runs_encode(ops, nops, j->runs + i * j->runs_per_pair,
                                     j->runs_per_pair);
      if (r < 0) { j->err = -3; free(ops); return NULL; }
      j->nruns[i] = (int32_t)r;
    }
  }
  free(ops);
  return NULL;
}

/* Align pairs [0, n_pairs) with oracle_wfa_ef (free ends pb, pe, tb, te; all
 * 0 = global) on nthreads POSIX threads (static contiguous chunks).  Pair i
 * is pat[poff[i] .. +plen[i]) against txt[toff[i] .. +tlen[i]).  If runs !=
 * NULL the canonical alignment of pair i is written as run-length words to
 * runs[i*runs_per_pair ...] with the count in nruns[i].  counts_out (may be
 * NULL) receives the summed work counters.  Returns 0, or a negative error
 * (-2 memory, -3 runs_per_pair too small). */
int oracle_wfa_batch_ef(int64_t n_pairs, const char *pat, const int64_t *poff,
                        const int32_t *plen, const char *txt,
                        const int64_t *toff, const int32_t *tlen, int64_t x,
                        int64_t o, int64_t e, int64_t pb, int64_t pe,
                        int64_t tb, int64_t te, int64_t max_score,
                        int32_t *scores, int8_t *status, uint32_t *runs,
                        int64_t runs_per_pair, int32_t *nruns, int nthreads,
                        oracle_counts *counts_out) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 1024) nthreads = 1024;
  batch_job *jobs = calloc((size_t)nthreads, sizeof(batch_job));
  pthread_t *th = calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return -2; }
  int64_t chunk = (n_pairs + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; t++) {
    batch_job *j = &jobs[t];
    j->begin = t * chunk < n_pairs ? t * chunk : n_pairs;
    j->end = (t + 1) * chunk < n_pairs ? (t + 1) * chunk : n_pairs;
    j->pat = pat; j->poff = poff; j->plen = plen;
    j->txt = txt; j->toff = toff; j->tlen = tlen;
    j->x = x; j->o = o; j->e = e; j->max_score = max_score;
    j->pb = pb; j->pe = pe; j->tb = tb; j->te = te;
    j->want_ops = runs != NULL;
    j->scores = scores; j->status = status;
    j->runs = runs; j->runs_per_pair = runs_per_pair; j->nruns = nruns;
  }
  int started = 0;
  for (int t = 1; t < nthreads; t++) {
    if (pthread_create(&th[t], NULL, batch_worker, &jobs[t]) != 0) break;
    started = t;
  }
  batch_worker(&jobs[0]);
  for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
  /* chunks whose thread could not be started run here */
  for (int t = started + 1; t < nthreads; t++) batch_worker(&jobs[t]);
  int err = 0;
  oracle_counts total = {0, 0, 0, 0};
  for (int t = 0; t < nthreads; t++) {
    if (jobs[t].err) err = jobs[t].err;
    total.cells += jobs[t].counts.cells;
    total.wavefronts += jobs[t].counts.wavefronts;
    total.char_compares += jobs[t].counts.char_compares;
    total.bt_steps += jobs[t].counts.bt_steps;
  }
  if (counts_out) *counts_out = total;
  free(jobs);
  free(th);
  return err;
}

/* The global alignment of every pair: oracle_wfa_batch_ef with no free ends. */
int oracle_wfa_batch(int64_t n_pairs, const char *pat, const int64_t *poff,
                     const int32_t *plen, const char *txt, const int64_t *toff,
                     const int32_t *tlen, int64_t x, int64_t o, int64_t e,
                     int64_t max_score, int32_t *scores, int8_t *status,
                     uint32_t *runs, int64_t runs_per_pair, int32_t *nruns,
                     int nthreads, oracle_counts *counts_out) {
  return oracle_wfa_batch_ef(n_pairs, pat, poff, plen, txt, toff, tlen, x, o, e,
                             0, 0, 0, 0, max_score, scores, status, runs,
                             runs_per_pair, nruns, nthreads, counts_out);
}
