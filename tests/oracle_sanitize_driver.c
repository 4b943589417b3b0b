/*
 * Drives every entry point of the oracle (oracle/gs_oracle.c) over seeded
 * inputs and its error paths.  tests/test_oracle_sanitized.py builds it with
 * -fsanitize=address,undefined, so an out-of-bounds access, a leak or
 * undefined behaviour anywhere in the oracle fails that test.  It also checks
 * a few facts every run must satisfy (labels in range, counts summing to n).
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "../oracle/gs_oracle.h"

static uint64_t g_state = 88172645463325252ull;

/* xorshift64, uniform in [0, 1) */
static double uni(void) {
  g_state ^= g_state << 13;
  g_state ^= g_state >> 7;
  g_state ^= g_state << 17;
  return (double)(g_state >> 11) * (1.0 / 9007199254740992.0);
}

static int fail(const char *what, int trial) {
  fprintf(stderr, "oracle check failed: %s (trial %d)\n", what, trial);
  return 1;
}

static int run_fits(int trial) {
  const int d = 1 + trial % 5;
  const int64_t n = 1 + (int64_t)(uni() * 300.0);
  const double h = trial % 3 == 0 ? 1.0 : 0.75;
  const int max_iter = trial % 4 == 0 ? 2 : 50;
  double *X = malloc(sizeof(double) * (size_t)(n * d));
  int32_t *lab = malloc(sizeof(int32_t) * (size_t)n);
  double *modes = malloc(sizeof(double) * (size_t)(n * d));
  int64_t *keys = malloc(sizeof(int64_t) * (size_t)(n * d));
  uint64_t *cnt = malloc(sizeof(uint64_t) * (size_t)n);
  int64_t *mh = malloc(sizeof(int64_t) * (size_t)(max_iter + 1));
  double *tr = malloc(sizeof(double) * (size_t)(max_iter * 2 * d));
  int bad = 0;
  for (int64_t i = 0; i < n * d; i++) {
    double v = (uni() * 2.0 - 1.0) * 5.0;
    if (i % 3 == 0) v = floor(v * 4.0) / 4.0; /* on cell faces */
    X[i] = v;
  }
  for (int form = 0; form < 2 && !bad; form++) {
    gso_info info;
    const int rc = form ? gso_fit_sequential(X, n, d, h, max_iter, lab, modes, n, keys, cnt, mh,
                                             tr, &info)
                        : gso_fit(X, n, d, h, max_iter, lab, modes, n, keys, cnt, mh, tr, &info);
    if (rc != 0) { bad = fail("fit returned an error", trial); break; }
    uint64_t total = 0;
    for (int64_t c = 0; c < info.k; c++) total += cnt[c];
    if (total != (uint64_t)n) bad = fail("counts do not sum to n", trial);
    for (int64_t i = 0; i < n; i++)
      if (lab[i] < 0 || lab[i] >= info.k) bad = fail("label out of range", trial);
    if (info.iterations > max_iter) bad = fail("too many updates", trial);
    /* a modes buffer one row short: code 4, nothing written past it */
    if (info.k > 1) {
      double *small = malloc(sizeof(double) * (size_t)((info.k - 1) * d));
      gso_info i2;
      const int rc2 = form ? gso_fit_sequential(X, n, d, h, max_iter, lab, small, info.k - 1,
                                                NULL, NULL, NULL, NULL, &i2)
                           : gso_fit(X, n, d, h, max_iter, lab, small, info.k - 1, NULL, NULL,
                                     NULL, NULL, &i2);
      if (rc2 != 4) bad = fail("short modes buffer not reported", trial);
      free(small);
    }
  }
  free(X); free(lab); free(modes); free(keys); free(cnt); free(mh); free(tr);
  return bad;
}

static int run_track(int trial) {
  const int64_t W = 17 + trial % 23, H = 11 + trial % 13;
  const int d = 3;
  const double h = 16.0;
  double *frame = malloc(sizeof(double) * (size_t)(W * H * d));
  for (int64_t i = 0; i < W * H * d; i++) frame[i] = floor(uni() * 256.0);
  const int64_t k = 1 + trial % 9;
  int64_t *bins = malloc(sizeof(int64_t) * (size_t)(k * d));
  for (int64_t i = 0; i < k * d; i++) bins[i] = (int64_t)(uni() * 17.0) - 1;
  uint8_t *present = malloc((size_t)k);
  int64_t out[7];
  int bad = 0;
  /* windows inside, clipped on every side, and empty */
  const int64_t rects[4][4] = {{2, 3, W - 4, H - 2}, {-5, -7, W + 9, H + 4},
                               {W - 3, H - 2, W + 30, H + 30}, {4, 4, 4, 9}};
  for (int r = 0; r < 4; r++) {
    if (gso_track_window(frame, W, H, d, h, bins, k, rects[r][0], rects[r][1], rects[r][2],
                         rects[r][3], out, present) != 0)
      bad = fail("track window returned an error", trial);
    if (out[0] < 0 || out[0] > W * H) bad = fail("window count out of range", trial);
  }
  frame[0] = NAN;
  if (gso_track_window(frame, W, H, d, h, bins, k, 0, 0, W, H, out, present) != 1)
    bad = fail("non-finite colour not reported", trial);
  free(frame); free(bins); free(present);
  return bad;
}

int main(void) {
  int bad = 0;
  for (int trial = 0; trial < 80; trial++) bad |= run_fits(trial);
  for (int trial = 0; trial < 20; trial++) bad |= run_track(trial);
  /* empty input, and rejected arguments */
  gso_info info;
  double x[2] = {1.0, NAN};
  int32_t lab[2];
  double modes[2];
  if (gso_fit(x, 0, 1, 1.0, 5, lab, modes, 2, NULL, NULL, NULL, NULL, &info) != 0 || info.k != 0)
    bad |= fail("empty input", -1);
  if (gso_fit(x, 2, 1, 1.0, 5, lab, modes, 2, NULL, NULL, NULL, NULL, &info) != 1)
    bad |= fail("non-finite point not rejected", -1);
  if (gso_fit(x, 1, 1, -1.0, 5, lab, modes, 2, NULL, NULL, NULL, NULL, &info) != 1)
    bad |= fail("h <= 0 not rejected", -1);
  if (!bad) printf("oracle sanitized run: ok\n");
  return bad;
}
