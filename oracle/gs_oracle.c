/*
 * GridShift mode seeking -- plain, slow, single-threaded CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * CPU legs of bench.py.  The CUDA library shares no code with this file.
 *
 * What it computes (Kumar et al., "GridShift: A Faster Mode-seeking Algorithm
 * for Image Segmentation and Object Tracking", Sec. 2.1 steps i-v, Algorithm 1,
 * Eq. 1-4; the parallel update form Eq. 6 of Sec. 2.2):
 *
 *   i)   Binning (Sec. 2.1 i, Algorithm 1 initialisation loop): the cell key of a
 *        point is floor(x / h) per coordinate; each active cell keeps its resident
 *        count C and the sum of its residents' coordinates.
 *   ii)  Update (Eq. 1-2): each active cell j moves to
 *            S'(j) = sum_v C(j+v) S(j+v) / sum_v C(j+v),  v in {-1,0,1}^d,
 *        where C(j+v) S(j+v) is the neighbour's coordinate sum.  All cells read
 *        the state before the update (Eq. 6, the parallel form).
 *   iii) Re-key (Sec. 2.1 iii): new key floor(S'(j) / h).
 *   iv)  Merge (Eq. 3-4): cells with the same new key add their counts and their
 *        count-weighted centroids C(j) S'(j); resident sets are unioned, which is
 *        kept as a map from every old cell to its merged cell.
 *   v)   Stop (Sec. 2.1 v, Theorem 2): when no active cell has another active
 *        cell in its 3^d neighbourhood, or after max_iter applied updates.
 *
 * Readings of the paper taken here:
 *   R1  State is (count, coordinate sum); the centroid is sum / count.
 *   R2  Every sum (binning, neighbourhood, merge) is formed exactly and rounded
 *       once to the nearest double, ties to even; the centroid S'(j) is the
 *       exact quotient of the exact neighbourhood sum by the neighbourhood count,
 *       rounded once.  The paper fixes no summation order; exact sums make the
 *       result independent of it.
 *   R3  floor is the mathematical floor of the exact quotient x / h; a value on
 *       a cell face belongs to the upper cell.
 *   R4  Update ii) is the parallel (Jacobi) form: all cells read the pre-update
 *       state.  The paper's listing updates in place in an unspecified order.
 *   R5  The stop test of v) is evaluated on the current state before an update;
 *       an update during which no cell has a neighbour is not applied.
 *   R6  Clusters are numbered by ascending lexicographic final key, axis 0 most
 *       significant; a mode is the final cell's sum divided by its count.
 *
 * gso_fit_sequential computes the sequential form of update ii) instead
 * (Eq. 5, Sec. 2.2; Algorithm 1 writes S'(j) in place inside its loop over the
 * cells): a cell's neighbourhood sum uses the already updated centroid of every
 * neighbour that precedes it in the sweep.  Readings:
 *   R7  The sweep order, which the paper leaves to the hash table, is by
 *       parity colour: colour(k) = sum_a (k_a mod 2) 2^(d-1-a) (axis 0 the
 *       most significant bit), colours ascending, then keys ascending.  Two
 *       distinct cells of one colour differ by an even, non-zero amount on
 *       some axis, so they are never neighbours and the order inside a colour
 *       does not change the result.
 *   R8  A neighbour updated earlier in the sweep contributes its count times
 *       its new centroid C(q) S'(q) (exact product); any other cell its stored
 *       sum, as in the parallel form.  Counts do not change during the sweep.
 *   Everything else (re-key, merge, stop test, labels) is as above.
 *
 * Exact arithmetic: an accumulator is an array of signed 64-bit "digits", digit
 * k standing for multiples of 2^(32k + XBASE).  Adding m * v (v a double, m a
 * count) splits the exact integer product of m and v's significand into 32-bit
 * pieces and adds each piece to its digit; nothing is ever rounded until the
 * accumulator is converted to a double.
 */
#include "gs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define XW 74          /* number of 32-bit digits */
#define XBASE (-1184)  /* weight exponent of digit 0: well below 2^-1074 */

typedef struct {
  int64_t dig[XW];
  int64_t nadd;
} xacc;

static void xacc_clear(xacc *a) { memset(a, 0, sizeof(*a)); }

/* Carry-propagate so that digits 0..XW-2 lie in [0, 2^32) and the top digit
 * carries the sign.  The value is unchanged. */
static void xacc_normalize(xacc *a) {
  int64_t carry = 0;
  for (int k = 0; k < XW; k++) {
    int64_t t = a->dig[k] + carry;
    int64_t lo = t & (int64_t)0xFFFFFFFF;
    carry = (t - lo) / ((int64_t)1 << 32); /* exact division */
    a->dig[k] = lo;
  }
  a->dig[XW - 1] += carry * ((int64_t)1 << 32);
  a->nadd = 0;
}

/* a += m * v, exactly. */
static void xacc_add(xacc *a, double v, uint64_t m) {
  if (v == 0.0 || m == 0) return;
  int e;
  double f = frexp(fabs(v), &e);              /* |v| = f * 2^e, 0.5 <= f < 1 */
  uint64_t M = (uint64_t)ldexp(f, 53);        /* integer significand, lsb weight 2^(e-53) */
  int64_t p = (int64_t)(e - 53) - XBASE;      /* bit position of the lsb */
  int k = (int)(p / 32), r = (int)(p % 32);
  unsigned __int128 P = (unsigned __int128)M * m;
  P <<= r;
  int64_t s = v < 0 ? -1 : 1;
  while (P != 0) {
    a->dig[k] += s * (int64_t)(uint32_t)P;
    P >>= 32;
    k++;
  }
  if (++a->nadd >= ((int64_t)1 << 28)) xacc_normalize(a);
}

/* Sign of the value (-1, 0, 1) and its magnitude as 32-bit digits in mag[]. */
static int xacc_magnitude(const xacc *a, int64_t mag[XW]) {
  xacc t = *a;
  xacc_normalize(&t);
  int sign = 0;
  if (t.dig[XW - 1] < 0) {
    sign = -1;
    for (int k = 0; k < XW; k++) t.dig[k] = -t.dig[k];
    xacc_normalize(&t);
  } else {
    for (int k = 0; k < XW; k++)
      if (t.dig[k] != 0) { sign = 1; break; }
  }
  memcpy(mag, t.dig, sizeof(t.dig));
  return sign;
}

static int mag_bit(const int64_t *mag, int64_t b) {
  if (b < 0) return 0;
  return (int)((mag[b / 32] >> (b % 32)) & 1);
}

/* Round sign * (mag * 2^XBASE + something in (0, 2^XBASE) if sticky_in) to the
 * nearest double, ties to even. */
static double round_mag(const int64_t *mag, int sign, int sticky_in) {
  int kt = XW - 1;
  while (kt >= 0 && mag[kt] == 0) kt--;
  if (kt < 0) return sign < 0 ? -0.0 : 0.0; /* below 2^XBASE: rounds to zero */
  int top = 31;
  while (((mag[kt] >> top) & 1) == 0) top--;
  int64_t P = (int64_t)kt * 32 + top;        /* position of the leading 1 */
  int64_t rp = P - 52;                       /* position of the result's lsb */
  int64_t sub_lsb = -1074 - XBASE;           /* lsb position of subnormals */
  if (rp < sub_lsb) rp = sub_lsb;
  uint64_t sig = 0;
  for (int64_t b = P; b >= rp; b--) sig = (sig << 1) | (uint64_t)mag_bit(mag, b);
  int guard = mag_bit(mag, rp - 1);
  int sticky = sticky_in;
  for (int64_t b = rp - 2; b >= 0 && !sticky; b--) sticky |= mag_bit(mag, b);
  if (guard && (sticky || (sig & 1))) sig += 1;
  double r = ldexp((double)sig, (int)(rp + XBASE));
  return sign < 0 ? -r : r;
}

static double xacc_round(const xacc *a) {
  int64_t mag[XW];
  int sign = xacc_magnitude(a, mag);
  if (sign == 0) return 0.0;
  return round_mag(mag, sign, 0);
}

/* (value / D) rounded to nearest, ties to even; 1 <= D < 2^32. */
static double xacc_div_round(const xacc *a, uint64_t D) {
  int64_t mag[XW], q[XW];
  int sign = xacc_magnitude(a, mag);
  if (sign == 0) return 0.0;
  uint64_t rem = 0;
  for (int k = XW - 1; k >= 0; k--) {
    uint64_t cur = (rem << 32) | (uint64_t)mag[k];
    q[k] = (int64_t)(cur / D);
    rem = cur % D;
  }
  return round_mag(q, sign, rem != 0);
}

int64_t gso_floor_div(double x, double h) {
  double q = floor(x / h);
  /* fma(-q, h, x) is x - q*h rounded once: its sign is that of the exact
   * difference, which is a multiple of 2^-1074 and therefore never flushes to
   * zero. */
  while (fma(-q, h, x) < 0) q -= 1.0;
  while (fma(-(q + 1.0), h, x) >= 0) q += 1.0;
  return (int64_t)q;
}

double gso_exact_sum(const double *v, const uint32_t *w, int64_t n) {
  xacc a;
  xacc_clear(&a);
  for (int64_t i = 0; i < n; i++) xacc_add(&a, v[i], w ? w[i] : 1u);
  return xacc_round(&a);
}

double gso_exact_mean(const double *v, int64_t n, uint64_t D) {
  xacc a;
  xacc_clear(&a);
  for (int64_t i = 0; i < n; i++) xacc_add(&a, v[i], 1u);
  return xacc_div_round(&a, D);
}

/* ------------------------------------------------------------------------- */
/* Cells: keys kept sorted lexicographically (axis 0 most significant).        */

static int g_d; /* dimension used by the qsort comparators */

static int key_cmp(const int64_t *a, const int64_t *b, int d) {
  for (int i = 0; i < d; i++) {
    if (a[i] < b[i]) return -1;
    if (a[i] > b[i]) return 1;
  }
  return 0;
}

typedef struct {
  const int64_t *key; /* d entries */
  int64_t idx;
} keyed;

static int keyed_cmp(const void *pa, const void *pb) {
  const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
  int c = key_cmp(a->key, b->key, g_d);
  if (c) return c;
  return (a->idx > b->idx) - (a->idx < b->idx); /* stable: original order */
}

/* Index of key in the sorted m x d array ck, or -1. */
static int64_t find_cell(const int64_t *ck, int64_t m, int d, const int64_t *key) {
  int64_t lo = 0, hi = m - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    int c = key_cmp(ck + mid * d, key, d);
    if (c == 0) return mid;
    if (c < 0) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* Parity colour of a key (R7): bit d-1-a is k_a mod 2. */
static int64_t key_colour(const int64_t *k, int d) {
  int64_t c = 0;
  for (int a = 0; a < d; a++) c = 2 * c + (k[a] % 2 != 0);
  return c;
}

static int fit_impl(const double *X, int64_t n, int d, double h, int max_iter,
                    int32_t *labels, double *modes, int64_t cap, int64_t *final_keys,
                    uint64_t *final_cnt, int64_t *m_hist, double *trace, gso_info *info,
                    int sequential) {
  if (n < 0 || d < 1 || d > 12 || !(h > 0) || !isfinite(h) || max_iter < 0 || !info) return 1;
  if (n > 0 && (!X || !labels)) return 1;
  for (int64_t i = 0; i < n * d; i++)
    if (!isfinite(X[i])) return 1;
  if ((double)n >= 4294967296.0) return 1; /* counts are kept below 2^32 */
  memset(info, 0, sizeof(*info));
  if (n == 0) return 0;

  int ret = 0;
  int64_t nv = 1;
  for (int a = 0; a < d; a++) nv *= 3;

  int64_t *K = malloc(sizeof(int64_t) * n * d);     /* point keys */
  keyed *ord = malloc(sizeof(keyed) * n);
  int64_t *cell_of = malloc(sizeof(int64_t) * n);   /* point -> initial cell */
  int64_t *ck = malloc(sizeof(int64_t) * n * d);    /* cell keys */
  uint64_t *cc = malloc(sizeof(uint64_t) * n);      /* cell counts */
  double *cs = malloc(sizeof(double) * n * d);      /* cell sums */
  int64_t *cur = malloc(sizeof(int64_t) * n);       /* initial cell -> current cell */
  double *sp = malloc(sizeof(double) * n * d);      /* updated centroids */
  int64_t *nk = malloc(sizeof(int64_t) * n * d);    /* new keys */
  int64_t *parent = malloc(sizeof(int64_t) * n);
  int64_t *ck2 = malloc(sizeof(int64_t) * n * d);
  uint64_t *cc2 = malloc(sizeof(uint64_t) * n);
  double *cs2 = malloc(sizeof(double) * n * d);
  xacc *acc = malloc(sizeof(xacc) * d);
  int64_t *probe = malloc(sizeof(int64_t) * d);
  int64_t *sweep = malloc(sizeof(int64_t) * n);     /* order of the update sweep */
  char *done = malloc((size_t)n);                   /* updated earlier in this sweep */
  if (!K || !ord || !cell_of || !ck || !cc || !cs || !cur || !sp || !nk || !parent || !ck2 ||
      !cc2 || !cs2 || !acc || !probe || !sweep || !done) {
    ret = 2;
    goto done;
  }

  /* i) binning */
  for (int64_t i = 0; i < n; i++)
    for (int a = 0; a < d; a++) {
      double q = floor(X[i * d + a] / h);
      if (!(fabs(q) < 4503599627370496.0)) { ret = 3; goto done; } /* 2^52 */
      K[i * d + a] = gso_floor_div(X[i * d + a], h);
    }
  for (int64_t i = 0; i < n; i++) { ord[i].key = K + i * d; ord[i].idx = i; }
  g_d = d;
  qsort(ord, (size_t)n, sizeof(keyed), keyed_cmp);
  int64_t m = 0;
  for (int64_t s = 0; s < n;) {
    int64_t e = s;
    while (e < n && key_cmp(ord[e].key, ord[s].key, d) == 0) e++;
    memcpy(ck + m * d, ord[s].key, sizeof(int64_t) * d);
    cc[m] = (uint64_t)(e - s);
    for (int a = 0; a < d; a++) {
      xacc_clear(&acc[a]);
      for (int64_t t = s; t < e; t++) xacc_add(&acc[a], X[ord[t].idx * d + a], 1u);
      cs[m * d + a] = xacc_round(&acc[a]);
    }
    for (int64_t t = s; t < e; t++) cell_of[ord[t].idx] = m;
    m++;
    s = e;
  }
  int64_t m0 = m;
  for (int64_t c = 0; c < m0; c++) cur[c] = c;
  if (m_hist) m_hist[0] = m;

  int t = 0, converged = 0;
  for (;;) {
    /* ii) neighbourhood-weighted centroid of every cell: from the old state
     * (parallel form), or in the sweep order of R7 reading what the sweep has
     * already updated (sequential form, R8) */
    int any_nb = 0;
    int64_t ns = 0;
    if (sequential) {
      const int64_t ncol = (int64_t)1 << d;
      for (int64_t col = 0; col < ncol; col++)
        for (int64_t j = 0; j < m; j++)
          if (key_colour(ck + j * d, d) == col) sweep[ns++] = j;
    } else {
      for (int64_t j = 0; j < m; j++) sweep[ns++] = j;
    }
    for (int64_t j = 0; j < m; j++) done[j] = 0;
    for (int64_t s = 0; s < m; s++) {
      const int64_t j = sweep[s];
      uint64_t D = 0;
      for (int a = 0; a < d; a++) xacc_clear(&acc[a]);
      for (int64_t v = 0; v < nv; v++) {
        int64_t rest = v;
        int centre = 1;
        for (int a = d - 1; a >= 0; a--) { /* axis 0 is the slowest digit */
          int off = (int)(rest % 3) - 1;
          rest /= 3;
          probe[a] = ck[j * d + a] + off;
          if (off != 0) centre = 0;
        }
        int64_t q = find_cell(ck, m, d, probe);
        if (q < 0) continue;
        D += cc[q];
        for (int a = 0; a < d; a++) {
          if (done[q]) xacc_add(&acc[a], sp[q * d + a], cc[q]);
          else xacc_add(&acc[a], cs[q * d + a], 1u);
        }
        if (!centre) any_nb = 1;
      }
      for (int a = 0; a < d; a++) sp[j * d + a] = xacc_div_round(&acc[a], D);
      if (sequential) done[j] = 1;
    }
    /* v) stop test, before the update is applied */
    if (!any_nb) { converged = 1; break; }
    if (t == max_iter) break;
    /* iii) re-key */
    for (int64_t j = 0; j < m; j++)
      for (int a = 0; a < d; a++) {
        double q = floor(sp[j * d + a] / h);
        if (!(fabs(q) < 4503599627370496.0)) { ret = 3; goto done; }
        nk[j * d + a] = gso_floor_div(sp[j * d + a], h);
      }
    if (trace) {
      for (int a = 0; a < d; a++) {
        xacc_clear(&acc[a]);
        for (int64_t j = 0; j < m; j++) xacc_add(&acc[a], sp[j * d + a], cc[j]);
        trace[((int64_t)t * 2 + 0) * d + a] = xacc_round(&acc[a]);
      }
    }
    /* iv) merge cells that share a key; members in ascending old key order */
    for (int64_t j = 0; j < m; j++) { ord[j].key = nk + j * d; ord[j].idx = j; }
    qsort(ord, (size_t)m, sizeof(keyed), keyed_cmp);
    int64_t m2 = 0;
    for (int64_t s = 0; s < m;) {
      int64_t e = s;
      while (e < m && key_cmp(ord[e].key, ord[s].key, d) == 0) e++;
      memcpy(ck2 + m2 * d, ord[s].key, sizeof(int64_t) * d);
      uint64_t cnt = 0;
      for (int a = 0; a < d; a++) xacc_clear(&acc[a]);
      for (int64_t u = s; u < e; u++) {
        int64_t j = ord[u].idx;
        cnt += cc[j];
        for (int a = 0; a < d; a++) xacc_add(&acc[a], sp[j * d + a], cc[j]);
        parent[j] = m2;
      }
      cc2[m2] = cnt;
      for (int a = 0; a < d; a++) cs2[m2 * d + a] = xacc_round(&acc[a]);
      m2++;
      s = e;
    }
    memcpy(ck, ck2, sizeof(int64_t) * m2 * d);
    memcpy(cc, cc2, sizeof(uint64_t) * m2);
    memcpy(cs, cs2, sizeof(double) * m2 * d);
    for (int64_t c = 0; c < m0; c++) cur[c] = parent[cur[c]];
    if (trace) {
      for (int a = 0; a < d; a++) {
        xacc_clear(&acc[a]);
        for (int64_t j = 0; j < m2; j++) xacc_add(&acc[a], cs[j * d + a], 1u);
        trace[((int64_t)t * 2 + 1) * d + a] = xacc_round(&acc[a]);
      }
    }
    m = m2;
    t++;
    if (m_hist) m_hist[t] = m;
  }

  if (m > cap) { ret = 4; info->k = m; goto done; }
  for (int64_t i = 0; i < n; i++) labels[i] = (int32_t)cur[cell_of[i]];
  for (int64_t c = 0; c < m; c++) {
    for (int a = 0; a < d; a++) {
      if (modes) modes[c * d + a] = cs[c * d + a] / (double)cc[c];
      if (final_keys) final_keys[c * d + a] = ck[c * d + a];
    }
    if (final_cnt) final_cnt[c] = cc[c];
  }
  info->iterations = t;
  info->converged = converged;
  info->m0 = m0;
  info->k = m;

done:
  free(K); free(ord); free(cell_of); free(ck); free(cc); free(cs); free(cur); free(sp);
  free(nk); free(parent); free(ck2); free(cc2); free(cs2); free(acc); free(probe);
  free(sweep); free(done);
  return ret;
}

int gso_fit(const double *X, int64_t n, int d, double h, int max_iter,
            int32_t *labels, double *modes, int64_t cap, int64_t *final_keys,
            uint64_t *final_cnt, int64_t *m_hist, double *trace, gso_info *info) {
  return fit_impl(X, n, d, h, max_iter, labels, modes, cap, final_keys, final_cnt, m_hist,
                  trace, info, 0);
}

int gso_fit_sequential(const double *X, int64_t n, int d, double h, int max_iter,
                       int32_t *labels, double *modes, int64_t cap, int64_t *final_keys,
                       uint64_t *final_cnt, int64_t *m_hist, double *trace, gso_info *info) {
  return fit_impl(X, n, d, h, max_iter, labels, modes, cap, final_keys, final_cnt, m_hist,
                  trace, info, 1);
}

int gso_track_window(const double *frame, int64_t width, int64_t height, int d, double h,
                     const int64_t *bins, int64_t k, int64_t x0, int64_t y0, int64_t x1,
                     int64_t y1, int64_t *out, uint8_t *present) {
  int64_t count = 0, sx = 0, sy = 0;
  int64_t mnx = INT64_MAX, mxx = INT64_MIN, mny = INT64_MAX, mxy = INT64_MIN;
  int64_t key[8];
  for (int64_t j = 0; j < k; j++) present[j] = 0;
  if (x0 < 0) x0 = 0;
  if (y0 < 0) y0 = 0;
  if (x1 > width) x1 = width;
  if (y1 > height) y1 = height;
  for (int64_t y = y0; y < y1; y++) {
    for (int64_t x = x0; x < x1; x++) {
      const double *c = frame + (y * width + x) * d;
      for (int a = 0; a < d; a++) {
        if (!(fabs(c[a]) < 4.0e15 * h)) return 1;
        key[a] = gso_floor_div(c[a], h);
      }
      int in = 0;
      for (int64_t j = 0; j < k; j++) {
        int same = 1;
        for (int a = 0; a < d; a++)
          if (bins[j * d + a] != key[a]) same = 0;
        if (same) {
          present[j] = 1;
          in = 1;
        }
      }
      if (!in) continue;
      count++;
      sx += x;
      sy += y;
      if (x < mnx) mnx = x;
      if (x > mxx) mxx = x;
      if (y < mny) mny = y;
      if (y > mxy) mxy = y;
    }
  }
  out[0] = count;
  out[1] = sx;
  out[2] = sy;
  out[3] = mnx;
  out[4] = mxx;
  out[5] = mny;
  out[6] = mxy;
  return 0;
}
