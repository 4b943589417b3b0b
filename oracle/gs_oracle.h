/*
 * GridShift mode seeking: plain CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The product
 * library (include/gridshift.h) neither links nor calls it.
 *
 * See gs_oracle.c for what is computed and which reading of the paper each
 * step follows.
 */
#ifndef GS_ORACLE_H
#define GS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Result of one oracle run.  Arrays are caller-owned; see gs_oracle_fit. */
typedef struct {
  int32_t iterations;   /* number of applied update steps */
  int32_t converged;    /* 1: stopped because no cell had a neighbour (Theorem 2) */
  int64_t m0;           /* active cells after binning */
  int64_t k;            /* active cells at exit = number of clusters */
} gso_info;

/*
 * Runs GridShift on X (n x d, row-major, float64).
 *   labels      [n]          cluster of each point, 0..k-1 in ascending final key order
 *   modes       [cap x d]    centroid (sum / count) of each final cell, in label order
 *   final_keys  [cap x d]    final integer cell keys (may be NULL)
 *   final_cnt   [cap]        final resident counts (may be NULL)
 *   m_hist      [max_iter+1] active cells before each update (may be NULL)
 *   trace       [max_iter x 2 x d] per applied update: exact total of count-weighted
 *               centroids before the merge, and exact total of merged sums after it,
 *               each rounded to double (may be NULL)
 * cap must be >= the number of clusters (n always suffices).
 * Returns 0 on success; 1 invalid argument / non-finite input; 2 out of memory;
 * 3 a key does not fit in int64 arithmetic; 4 cap too small.
 */
int gso_fit(const double *X, int64_t n, int d, double h, int max_iter,
            int32_t *labels, double *modes, int64_t cap, int64_t *final_keys,
            uint64_t *final_cnt, int64_t *m_hist, double *trace, gso_info *info);

/* The same run with the sequential update of Eq. 5 (Sec. 2.2): the cells are
 * swept in ascending parity colour (colour bit d-1-a = k_a mod 2), then
 * ascending key, and each cell's neighbourhood sum takes the new centroid of
 * every neighbour updated earlier in the sweep, weighted by its count.
 * Arguments, outputs and return codes as gso_fit. */
int gso_fit_sequential(const double *X, int64_t n, int d, double h, int max_iter,
                       int32_t *labels, double *modes, int64_t cap, int64_t *final_keys,
                       uint64_t *final_cnt, int64_t *m_hist, double *trace, gso_info *info);

/* floor(x / h) of the exact quotient, for finite x and finite h > 0. */
int64_t gso_floor_div(double x, double h);

/* sum_i w[i] * v[i] computed exactly and rounded once to nearest-even (w may be NULL = all 1). */
double gso_exact_sum(const double *v, const uint32_t *w, int64_t n);

/* (sum_i v[i]) / D computed exactly and rounded once to nearest-even; D >= 1, D < 2^32. */
double gso_exact_mean(const double *v, int64_t n, uint64_t D);

/* The window step of GridShift-based tracking (Sec. 2.3, Algorithm 2): over
 * the pixels x0 <= x < x1, y0 <= y < y1 of a width x height frame (clipped to
 * it; pixel (x, y) is row y * width + x of the row-major frame of d colour
 * channels), R = the pixels whose colour cell floor(c / h) (per channel) is
 * one of the k keys in bins (k x d, any order).  out[0..6] = |R|, sum of x,
 * sum of y, min x, max x, min y, max y over R (min = INT64_MAX, max =
 * INT64_MIN when R is empty); present[j] = 1 if some pixel of R lies in cell
 * bins[j], else 0.  A plain double loop with a linear search of bins.
 * Returns 0, or 1 when a colour in the window is not finite or has
 * |c| >= 4e15 h (the product rounded to double). */
int gso_track_window(const double *frame, int64_t width, int64_t height, int d, double h,
                     const int64_t *bins, int64_t k, int64_t x0, int64_t y0, int64_t x1,
                     int64_t y1, int64_t *out, uint8_t *present);

#ifdef __cplusplus
}
#endif
#endif
