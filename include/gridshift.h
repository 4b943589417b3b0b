/*
 * gridshift.h -- C ABI of the GB300 (sm_103a) GridShift mode-seeking library.
 *
 * GridShift (Kumar et al., "GridShift: A Faster Mode-seeking Algorithm for
 * Image Segmentation and Object Tracking", arXiv 2206.02200) clusters n points
 * of dimension d by (Sec. 2.1, Algorithm 1):
 *   i)   binning every point into the grid cell floor(x / h) and keeping, per
 *        active cell, its resident count and the sum of its residents;
 *   ii)  moving every active cell to the count-weighted mean over its 3^d
 *        neighbouring cells (Eq. 1-2, applied in the parallel form of Eq. 6,
 *        or in the sequential form of Eq. 5: see gs_update);
 *   iii) re-keying each moved cell by floor(centroid / h);
 *   iv)  merging the cells that share a key, adding counts and count-weighted
 *        centroids (Eq. 3-4);
 *   v)   stopping when no active cell has another active cell among its 3^d
 *        neighbours (Sec. 2.1 v, Theorem 2), or after max_iter updates;
 * and returns, per point, the cluster (final cell) it belongs to, and per
 * cluster its mode (final centroid).
 *
 * Conventions shared by every entry point:
 *   - Every pointer named "device" must point to memory of the CUDA device
 *     that is current on the calling thread; "host" pointers are plain host
 *     memory.  The caller owns all input and output buffers; a gs_ctx owns its
 *     device workspace and reuses or grows it between calls.
 *   - Points are row-major n x d (point i, coordinate a at [i * d + a]) in
 *     float64 (GS_IN_F64) or float32 (GS_IN_F32).  float32 inputs are widened
 *     to float64 exactly.
 *   - All work is issued on the stream set by gs_set_stream (default: the
 *     legacy default stream); gs_fit and gs_fit_batched return after it has
 *     finished (they read the cluster count back to the host).
 *   - Labels are 0 .. k-1, numbered by ascending lexicographic order of the
 *     final integer cell key (axis 0 most significant); modes are float64,
 *     row-major k x d, in label order.
 *   - No C++ exception crosses this boundary.  A ctx is not thread-safe: use
 *     one per host thread.  On any status other than GS_OK the contents of
 *     the output buffers are unspecified, except where stated.
 *
 * Arithmetic of the GS_FP64 precision: every sum the method forms (cell sums
 * in i) and iv), neighbourhood sums in ii)) is computed exactly in integer
 * fixed point and rounded once to the nearest float64 (ties to even); the
 * centroid of ii) is the exact neighbourhood sum divided by the neighbourhood
 * count, rounded once; floor(.) is taken of the exact quotient.  The result
 * therefore does not depend on the order of the points or on thread
 * scheduling.  The fixed-point window of coordinate a spans
 * 2^(E_a - 126) .. 2^E_a with n * max_i |x_ia| < 2^E_a; a value with nonzero
 * bits below that window is truncated and counted in gs_fit_info.inexact.
 */
#ifndef GRIDSHIFT_H
#define GRIDSHIFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_E_INVALID = 1,  /* bad argument: null pointer, d out of 1..12, h not > 0, NaN/Inf input, ... */
  GS_E_NOMEM = 2,    /* a device or pinned host allocation failed */
  GS_E_KEYRANGE = 3, /* a coordinate divided by h is 4e15 or more; for gs_fit_batched,
                        gs_fit_sweep and gs_fit_noalloc also: the integer cell keys do not
                        fit the 63-bit packed key, or an axis spans more than 2^22 cells
                        (gs_fit runs such keys through its wide-key pipeline instead) */
  GS_E_CAPACITY = 4, /* modes_cap < k: *k_out is set and labels are valid */
  GS_E_CUDA = 5,     /* a CUDA runtime call failed; see gs_get_last_error */
  GS_E_INTERNAL = 6, /* a device-side bound (hash probe limit, table overflow) was hit */
  GS_E_SCRATCH = 7   /* gs_fit_noalloc only: the input needs more scratch than its static
                        device array holds (too many points, cells or cells per axis) */
} gs_status;

typedef enum {
  GS_FP64 = 0,       /* exact sums rounded once to float64 (see the header comment) */
  GS_FP32_MIXED = 1  /* float32 cell state: per-axis mean offsets from the cell's lower face,
                        neighbour sums in compensated (float-float) float32, merges and
                        binning partial sums added with float32 atomics (the result may vary
                        in its last bits from run to run); a centroid within 1e-5 h of a cell
                        face has its key decided again in float64 (gs_fit_info.face_rechecks) */
} gs_precision;

typedef enum { GS_IN_F64 = 0, GS_IN_F32 = 1 } gs_dtype;

typedef enum {
  GS_UPDATE_PARALLEL = 0,   /* Eq. 6: every cell's new centroid from the state before the
                               update (Sec. 2.2, the parallel form; the default) */
  GS_UPDATE_SEQUENTIAL = 1  /* Eq. 5: the cells updated one after another, each reading the
                               new centroid of every neighbour updated before it (Sec. 2.2;
                               Algorithm 1 updates in place).  Order: ascending parity colour
                               sum_a (k_a mod 2) 2^(d-1-a), axis 0 the most significant bit;
                               cells of one colour are never neighbours, so each colour is one
                               parallel pass (2^d passes per update).  An updated neighbour
                               contributes its count times its new centroid, exactly */
} gs_update;

typedef struct gs_ctx gs_ctx; /* opaque; owns the device workspace */

typedef struct {
  int32_t iterations;  /* update steps applied (ii-iv), 0 .. max_iter */
  int32_t converged;   /* 1 if stopped by the criterion of Sec. 2.1 v (no cell has a neighbour) */
  int64_t m0;          /* active cells after binning (i) */
  int64_t k;           /* active cells at exit = number of clusters */
  int64_t inexact;     /* values truncated by the fixed-point window, or centroids too
                          close to zero for the window to round (below about 2^-136
                          times n max|x|); 0 in normal use */
  int64_t cell_iters;  /* sum over applied updates of the active cells updated */
  int64_t launches;    /* CUDA kernels the call launched */
  int64_t face_rechecks; /* GS_FP32_MIXED: key decisions redone in float64 near a face */
} gs_fit_info;

/* Timed parts of one call, for gs_get_phase_times.  CUDA event pairs on the
 * call's stream time the launches (GS_PHASE_RANGE .. GS_PHASE_SORT, the three
 * launch groups of step i's second pass, GS_PHASE_LABELS_OUT); the loop kernel's
 * own phases are split by the device clock, read by one block at the grid
 * barriers between them. */
typedef enum {
  GS_PHASE_RANGE = 0,    /* key range and finiteness of the input, and the plan (step i,
                            set-up) */
  GS_PHASE_BIN = 1,      /* binning, first pass: cell key and count per point (step i) */
  GS_PHASE_LOOP = 2,     /* the loop kernel: steps ii-v, numbering and modes */
  GS_PHASE_SORT = 3,     /* numbering by a radix sort, when there are too many clusters
                            to number inside the loop kernel */
  GS_PHASE_K_OFFSETS = 4, /* binning, second pass: offsets of the cells in a counting
                             sort of the points by cell (step i; two launches) */
  GS_PHASE_K_SCATTER = 5, /* the points sorted by cell (one launch) */
  GS_PHASE_K_SUMS = 6,    /* exact cell sums from the sorted points (one launch) */
  GS_PHASE_K_LEVEL0 = 7,  /* in the loop kernel: the initial cells and their table */
  GS_PHASE_K_UPDATE_FIRST = 8, /* in the loop kernel: the first update step (ii-v, merge
                                  into the next level's table), over the initial cells */
  GS_PHASE_K_UPDATE_REST = 9,  /* in the loop kernel: all later update steps */
  GS_PHASE_K_COMPACT = 10, /* in the loop kernel: each next level's cell list and sums */
  GS_PHASE_K_LABELS = 11,  /* in the loop kernel: final cell of every initial cell,
                              numbering, modes */
  GS_PHASE_LABELS_OUT = 12, /* the label of every point (one launch after the loop kernel) */
  GS_NPHASES = 13
} gs_phase;

typedef struct {
  double ms[GS_NPHASES];    /* device time of each phase, summed over its occurrences */
  int32_t count[GS_NPHASES]; /* occurrences timed in each phase */
  double step_ms[16][2];    /* device clock of the first 16 update steps: the update phase
                               (ii-iv) and the compaction that follows it */
} gs_phase_times;

/* Creates a context for d-dimensional points, cell side (bandwidth) h and at
 * most max_iter update steps (Sec. 2.1; h is the cell side of step i).
 * 1 <= d <= 12, h finite and > 0, max_iter >= 0 (d > 8: gs_fit only, in
 * GS_FP64 with the parallel update).  Allocates no device memory yet.  *out receives the context (NULL on error).  Returns GS_OK,
 * GS_E_INVALID or GS_E_NOMEM. */
gs_status gs_create(int d, double h, int max_iter, gs_ctx** out);

/* Selects the arithmetic of later calls (see gs_precision; default GS_FP64).
 * Unknown values return GS_E_INVALID and leave the setting unchanged. */
gs_status gs_set_precision(gs_ctx* ctx, gs_precision p);

/* Selects the update form of later gs_fit calls (see gs_update; default
 * GS_UPDATE_PARALLEL).  GS_UPDATE_SEQUENTIAL is available for GS_FP64 runs of
 * one point set: while it is set, gs_fit with GS_FP32_MIXED and gs_fit_batched
 * with B > 1 return GS_E_INVALID.  Unknown values return GS_E_INVALID and
 * leave the setting unchanged. */
gs_status gs_set_update(gs_ctx* ctx, gs_update u);

/* Sets the CUDA stream (a cudaStream_t passed as void*, e.g.
 * torch.cuda.current_stream().cuda_stream) on which every later call issues
 * its work.  NULL selects the legacy default stream. */
gs_status gs_set_stream(gs_ctx* ctx, void* cuda_stream);

/* Runs GridShift (Sec. 2.1 steps i-v, Algorithm 1, Eq. 1-4 with the parallel
 * update of Eq. 6, or the sequential one of Eq. 5: gs_set_update) on one
 * point set.
 *   points     device, n x d row-major, dtype as given
 *   n          number of points, 0 <= n < 2^31
 *   labels     device int32[n]: cluster of every point (output)
 *   modes      device float64[modes_cap x d]: final centroid of every cluster
 *              (output; may be NULL when modes_cap == 0)
 *   modes_cap  rows available in modes
 *   k_out      host: number of clusters k (output; required)
 *   info       host: statistics (output; may be NULL)
 * n == 0 returns GS_OK with k = 0.  If k > modes_cap, returns GS_E_CAPACITY
 * with *k_out = k and labels filled; call again with a larger buffer.
 *
 * Cell keys are integer vectors of any size (Sec. 2.1).  The main pipeline
 * packs a key into 63 bits (d <= 8, at most 2^22 cells per axis); where the
 * data's keys do not fit (d > 8, an axis spanning more cells, or fields wider
 * than 63 bits together), a GS_FP64 parallel-update run goes through the
 * wide-key pipeline instead: one int64 field per axis, cells kept in key
 * order, neighbours found by binary search, merges by a stable radix sort,
 * the same exact sums (bit-identical results; slower, with one host
 * synchronisation per update step).  GS_FP32_MIXED or GS_UPDATE_SEQUENTIAL
 * runs with such keys return GS_E_KEYRANGE (d <= 8) or GS_E_INVALID (d > 8). */
gs_status gs_fit(gs_ctx* ctx, const void* points, gs_dtype dtype, int64_t n, int32_t* labels,
                 double* modes, int64_t modes_cap, int64_t* k_out, gs_fit_info* info);

/* Runs GridShift on B independent point sets (instances) in one call, with
 * the same d, h and max_iter: the result for every instance is the result
 * gs_fit gives for that instance alone (Sec. 2.1; the paper has no batched
 * form, instances simply never interact).
 *   points        device, all instances' points concatenated, n x d row-major
 *   offsets       host int64[B + 1]: instance b owns points
 *                 offsets[b] .. offsets[b + 1] - 1; offsets[0] = 0,
 *                 non-decreasing, n = offsets[B] < 2^31 (empty instances allowed)
 *   B             1 <= B <= 2^20
 *   labels        device int32[n]: cluster of every point, numbered 0 .. k_b - 1
 *                 within its instance b (output)
 *   modes         device float64[modes_cap x d]: the modes of instance 0, then
 *                 of instance 1, ... (output)
 *   modes_cap     rows available in modes
 *   mode_offsets  host int64[B + 1]: instance b's modes are rows
 *                 mode_offsets[b] .. mode_offsets[b + 1] - 1 (output)
 *   infos         host gs_fit_info[B]: per-instance iterations, converged, m0,
 *                 k and cell_iters; inexact and launches are those of the whole
 *                 call (output)
 * All instances run in one pass of the pipeline: every cell key carries its
 * instance, an instance that meets the stop criterion is frozen while the
 * others continue.  If the total number of clusters exceeds modes_cap,
 * returns GS_E_CAPACITY with labels, mode_offsets and infos filled.  Returns
 * GS_OK, GS_E_INVALID, GS_E_NOMEM, GS_E_KEYRANGE (also when the instance
 * index does not fit the packed key beside the axes), GS_E_CAPACITY,
 * GS_E_CUDA or GS_E_INTERNAL. */
gs_status gs_fit_batched(gs_ctx* ctx, const void* points, gs_dtype dtype, const int64_t* offsets,
                         int B, int32_t* labels, double* modes, int64_t modes_cap,
                         int64_t* mode_offsets, gs_fit_info* infos);

/* Runs GridShift on the pixels of an image, the input of the paper's image
 * segmentation (Sec. 4.2: each pixel's (r, g, b) values, or (r, g, b, x, y)
 * with its position).  Pixel p = y * width + x is the point
 *   (c_0, .., c_{channels-1}, x * xy_scale, y * xy_scale)   if xy_scale > 0
 *   (c_0, .., c_{channels-1})                               if xy_scale == 0
 * with every value in float64 (the channel bytes exactly, the positions
 * rounded once by the product).  The features are built on the device, in the
 * context's workspace, and fitted as gs_fit fits them: the result is the one
 * gs_fit gives for that float64 feature matrix (bit for bit in GS_FP64).
 * Only the image itself need be uploaded: one byte per channel and pixel
 * instead of eight bytes per feature.  The kernel that builds the features
 * also takes their key range (Sec. 2.1 iii's cell bounds) from the pixels,
 * so the features are not read back for it (GS_PHASE_RANGE times the build
 * and the plan together).
 *   pixels     device uint8[height x width x channels], row-major: row y,
 *              column x, then the channels
 *   height, width  >= 0, height * width < 2^31
 *   channels   1 .. 8
 *   xy_scale   0 (no position features) or finite and > 0
 *   labels, modes, modes_cap, k_out, info: as gs_fit (labels in pixel order;
 *              info->launches counts the feature build as well: one launch,
 *              two with positions)
 * The context's d must be channels + 2 (xy_scale > 0) or channels.  Returns
 * what gs_fit returns, or GS_E_INVALID for the arguments above. */
gs_status gs_fit_image(gs_ctx* ctx, const uint8_t* pixels, int64_t height, int64_t width,
                       int channels, double xy_scale, int32_t* labels, double* modes,
                       int64_t modes_cap, int64_t* k_out, gs_fit_info* info);

/* gs_fit_image on a stream of `count` images of one size held in HOST
 * memory, with host outputs: a video's frames, or images served one after
 * another.  For every image i the call uploads images[i], runs gs_fit_image
 * on it, and reads its labels and modes back into labels[i] and modes[i].
 * The upload of image i + 1 runs on a second stream while image i is
 * fitted, and the read-back of image i while image i + 1 is fitted, so the
 * copies overlap the fits (page-locked host buffers, e.g. from
 * cudaMallocHost, let them run asynchronously; other host memory works, with
 * the copies serialised).  The results are those of `count` separate gs_fit_image calls.
 *   count      >= 0 images
 *   images     host: count pointers, each to uint8[height x width x channels]
 *   height, width, channels, xy_scale: as gs_fit_image, the same for all
 *   labels     host: count pointers, each to int32[height x width] (output)
 *   modes      host: count pointers, each to float64[modes_cap x d] (output;
 *              may be NULL when modes_cap == 0)
 *   k_out      host int64[count]: clusters of every image (output; required)
 *   infos      host gs_fit_info[count] (output; may be NULL)
 * The device buffers (two of each: image, labels, modes) and the second
 * stream belong to the context and are kept for later calls.  The call
 * returns after every copy has finished.  On GS_E_CAPACITY for an image
 * (more clusters than modes_cap) the others are still fitted and the call
 * returns GS_E_CAPACITY with every k_out filled; any other error stops the
 * call.  Returns what gs_fit_image returns, GS_E_NOMEM, or GS_E_INVALID for
 * the arguments above. */
gs_status gs_fit_images_host(gs_ctx* ctx, int count, const uint8_t* const* images, int64_t height,
                             int64_t width, int channels, double xy_scale, int32_t* const* labels,
                             double* const* modes, int64_t modes_cap, int64_t* k_out,
                             gs_fit_info* infos);

/* gs_fit_batched on the pixels of B images (the channel values only: d =
 * channels, as in the (r, g, b) inputs of Sec. 4.2), built on the device as
 * gs_fit_image builds them.
 *   pixels     device uint8[n x channels]: the images' pixels concatenated
 *   channels   1 .. 8, equal to the context's d
 *   offsets    host int64[B + 1]: image b owns pixels offsets[b] ..
 *              offsets[b + 1] - 1 (as gs_fit_batched)
 *   B, labels, modes, modes_cap, mode_offsets, infos: as gs_fit_batched
 *              (every infos[b].launches counts the feature build as well)
 * Returns what gs_fit_batched returns, or GS_E_INVALID for the arguments
 * above. */
gs_status gs_fit_image_batched(gs_ctx* ctx, const uint8_t* pixels, int channels,
                               const int64_t* offsets, int B, int32_t* labels, double* modes,
                               int64_t modes_cap, int64_t* mode_offsets, gs_fit_info* infos);

/* Runs GridShift on one point set for B bandwidths h_0 .. h_{B-1} in one
 * call: instance b is the run gs_fit gives for the same points with h = hs[b]
 * (Sec. 2.1; the bandwidth study of Sec. 4.1 runs the method over a range of
 * h on the same data).  The context's d and max_iter apply, its h does not.
 *   points        device, n x d row-major, dtype as given (shared by all B runs)
 *   n             points, 0 <= n, B * n < 2^31
 *   hs            host float64[B]: the bandwidths, each finite and > 0 (repeats allowed)
 *   B             1 <= B <= 2^20
 *   labels        device int32[B * n]: labels[b * n + i] = cluster of point i
 *                 under h = hs[b], numbered 0 .. k_b - 1 within instance b (output)
 *   modes         device float64[modes_cap x d]: the modes of instance 0, then
 *                 of instance 1, ... (output)
 *   modes_cap     rows available in modes
 *   mode_offsets  host int64[B + 1]: instance b's modes are rows
 *                 mode_offsets[b] .. mode_offsets[b + 1] - 1 (output)
 *   infos         host gs_fit_info[B]: per-instance statistics, as gs_fit_batched
 * All B runs go through one pass of the batched pipeline (one launch of each
 * kernel): every instance decides its cells with its own h against its own
 * exact cell faces, and the instances share the packed-key layout.  The
 * plans are made on the host after the key-range pass (one extra round
 * trip).  GS_FP64 and GS_UPDATE_PARALLEL only (other settings return
 * GS_E_INVALID).  If the total number of clusters exceeds modes_cap, returns
 * GS_E_CAPACITY with labels, mode_offsets and infos filled.  Returns GS_OK,
 * GS_E_INVALID, GS_E_NOMEM, GS_E_KEYRANGE (the key fields of the smallest h
 * and the instance index do not fit 63 bits together), GS_E_CAPACITY,
 * GS_E_CUDA or GS_E_INTERNAL. */
gs_status gs_fit_sweep(gs_ctx* ctx, const void* points, gs_dtype dtype, int64_t n,
                       const double* hs, int B, int32_t* labels, double* modes,
                       int64_t modes_cap, int64_t* mode_offsets, gs_fit_info* infos);

/* Launch choices of the update loop.  They decide which lanes, tables and
 * phases compute a result, never the result itself (every sum is exact, so
 * the results are bit-identical under any valid choice).  This is
 * instrumentation for the autotuner (paper_2206_02200_gb300/autotune.py),
 * not a step of the paper's method. */
typedef struct {
  int32_t few_lanes_x4;  /* a level is updated with few lanes per cell (4 at d <= 3, 8 at
                            d = 4, 5, 16 at d = 6, 32 above; several cells in flight per
                            warp) when 4 x its cells exceed few_lanes_x4 x the warps of the
                            loop kernel's grid, else with 32 lanes per cell; 0 .. 2^20,
                            default 4 (more cells than warps) */
  int32_t load_shift;    /* level hash tables sized for load <= 2^-load_shift: 1 or 2
                            (default 2) */
  int32_t filter;        /* 1 (default): neighbour probes test the level's occupancy filter
                            (in shared memory) before the table; 0: every probe reads the
                            table */
  int32_t tail_enter;    /* a level of at most this many cells finishes the run in one block
                            of the loop kernel, pairwise in shared memory; 0 .. 256, default
                            128 (plain runs) */
  int32_t pencil_min;    /* the first update takes the pencil form (sums along axis 0 first,
                            d >= 3) when binning found at least this many cells; >= 0,
                            default 4096 (plain runs) */
  int32_t split_min;     /* runs of at least this many points take the second pass of
                            binning (counting sort, exact cell sums) and the label writes as
                            launches of their own, with more warps per SM; smaller runs
                            take them inside the loop kernel; >= 0, default 2^22 */
  int32_t bin_list;      /* 1 (default): binning lists the new cells of each warp 32 at a
                            time, one add on the (single) cell count for each 32, with five
                            blocks per SM; 0: one add per new cell, six blocks per SM */
  int32_t bin_sums;      /* 0 (default): a second pass sorts the points by cell (counting
                            sort) and forms the exact cell sums of Sec. 2.1 i over the
                            sorted runs; 1: binning forms them as it reads the points: the
                            points of a warp that share a cell are summed in registers and
                            added to the cell's sum with one set of atomic adds.  1 pays
                            where a warp's 32 consecutive points share few cells (measured
                            on GB300: 10% on a 321x481 image at h = 16); with about 30
                            points per cell (1080p and 4K images at d = 5, the d = 6
                            mixture) its adds cost 4 to 8 times the second pass */
} gs_tuning;

/* Sets the launch choices of later gs_fit, gs_fit_batched and gs_fit_sweep
 * calls (t == NULL: the defaults).  Values out of range return GS_E_INVALID
 * and leave the setting unchanged. */
gs_status gs_set_tuning(gs_ctx* ctx, const gs_tuning* t);

/* Copies the context's launch choices into *out (host). */
gs_status gs_get_tuning(gs_ctx* ctx, gs_tuning* out);

/* Turns per-phase device timing of later gs_fit calls on (enable != 0) or
 * off.  When on, each call records CUDA events on its stream around each
 * launch group and reads their elapsed times after its final synchronisation;
 * the result is available from gs_get_phase_times.  Off by default.  This is
 * instrumentation, not a step of the paper's method.  Returns GS_OK or
 * GS_E_INVALID (NULL ctx). */
gs_status gs_set_timing(gs_ctx* ctx, int enable);

/* Copies the per-phase times of the last gs_fit call of this context (all
 * zero if timing was off) into *out (host).  Returns GS_OK or GS_E_INVALID. */
gs_status gs_get_phase_times(gs_ctx* ctx, gs_phase_times* out);

/* gs_fit without any allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory while they run,
 * for instance a host program that fixes its whole GPU memory budget at
 * start-up and forbids later cudaMalloc/cudaFree calls (which also synchronise
 * the device), or a plug-in whose host application owns every allocation.
 *
 * It runs the same steps, with the same kernels and results, as gs_fit on a
 * context created with gs_create(d, h, max_iter) and bound to cuda_stream
 * (a cudaStream_t; NULL = legacy default stream).  The caller passes the
 * inputs and outputs exactly as for gs_fit; every other device buffer the
 * call needs is carved out of one static device array of 64 MiB that lives in
 * this library: every GPU that loads the library holds those 64 MiB until the
 * process exits.  The call allocates no device or pinned host memory and calls
 * no allocating CUDA routine.
 *
 * Set-up: every call, the first one on a device included, looks up the
 * device address of the static array (cudaGetSymbolAddress) in the context
 * current on the calling thread, so a call after a device reset, or from
 * another context on the same device, finds the array where it now is.  The
 * first call on a device also loads the library's kernels there: make it
 * before any stream capture.
 *
 * Limits: the per-point arrays (cell slot and counting-sort position) take
 * 8 bytes per point and 1 MiB is kept for the rest, so n <= 8,257,536; the
 * cell workspace (about 2.2 KB per initial active cell at d = 4 and
 * max_iter = 50, growing with d and max_iter, plus 272 KB of fixed buffers)
 * must fit what the points leave; the cell-face table holds at most 8192
 * entries (over all axes, the number of cells the data spans plus 3).
 * Beyond these the call returns GS_E_SCRATCH; use gs_fit.  GS_FP64, the
 * parallel update (GS_UPDATE_PARALLEL) and keys that fit the 63-bit packed
 * key (1 <= d <= 8) only.
 *
 * Sharing: every call uses the same array, which keeps the previous call's
 * contents; the call clears what must start at zero itself.  Calls are
 * serialised on the host by a lock and each returns only after its work on
 * cuda_stream has finished, so they do not overlap; GPU work that overlapped
 * a call's use of the array (another thread launching on the array through a
 * second copy of this library, say) would race.
 *
 * Returns GS_OK, GS_E_INVALID, GS_E_KEYRANGE, GS_E_CAPACITY (k > modes_cap:
 * *k_out and labels set, as for gs_fit), GS_E_SCRATCH, GS_E_CUDA or
 * GS_E_INTERNAL.  No error text is kept (there is no context). */
gs_status gs_fit_noalloc(int d, double h, int max_iter, void* cuda_stream, const void* points,
                         gs_dtype dtype, int64_t n, int32_t* labels, double* modes,
                         int64_t modes_cap, int64_t* k_out, gs_fit_info* info);

/* ---------------------------------------------------------------------------
 * Tracking window step (Sec. 2.3, Algorithm 2).  The tracker of Algorithm 2
 * keeps a set B of colour cells floor(c / h) (c the d colour channels of a
 * pixel, h the context's h) and, per frame, finds the pixels of a search
 * window whose colour cell lies in B:
 *     R = { pixel x in the window : floor(c(x) / h) in B },
 * then moves the window to the mean (x, y) position of R, replaces B by the
 * cells of R's pixels, and adapts the window's size from R's extent.  This
 * call computes one R: its size, the sum, mean and extent of its pixel
 * positions, and which cells of B it contains (the next B).  The loop of
 * Algorithm 2 around it (convergence of the centre, window resizing, frames)
 * is host logic: see gridshift.py (track).
 *
 * The frame is `height` x `width` pixels in row-major order (y outer, x
 * inner), d = the context's d colour channels per pixel (device, float64 or
 * float32 as dtype says); pixel (x, y) is point y * width + x.  The window is
 * the pixel rectangle x0 <= x < x1, y0 <= y < y1, clipped to the frame (an
 * empty rectangle gives an empty R).  bins is host memory, k x d integer cell
 * keys floor(c / h) per channel, in any order, duplicates allowed; k may be 0.
 * floor(c / h) is the floor of the exact quotient, as in gs_fit.
 *
 * Results (host): out->count = |R|; out->sum_x, sum_y = exact sums of the
 * positions of R's pixels; out->mean_x = sum_x / count and mean_y likewise,
 * each one IEEE division of the exact integers (NaN when count = 0);
 * out->min_x .. max_y = the bounding box of R's positions (min > max when
 * R is empty); present (host, k bytes, may be NULL): present[j] = 1 if some
 * pixel of R lies in cell bins[j], else 0.  The call synchronises the stream.
 * Returns GS_OK, GS_E_INVALID (null pointers, negative sizes, k < 0, a colour
 * in the window that is not finite or has |c| >= 4e15 h, the product rounded
 * to float64: then out->count = -1), GS_E_KEYRANGE (the keys of bins span
 * more than 2^22 cells on one channel), GS_E_NOMEM or GS_E_CUDA. */
typedef struct {
  int64_t count;
  int64_t sum_x, sum_y;
  double mean_x, mean_y;
  int64_t min_x, max_x, min_y, max_y;
} gs_track_result;

gs_status gs_track_window(gs_ctx* ctx, const void* frame, gs_dtype dtype, int64_t width,
                          int64_t height, const int64_t* bins, int64_t k, int64_t x0,
                          int64_t y0, int64_t x1, int64_t y1, gs_track_result* out,
                          uint8_t* present);

/* Copies a description of the last error of this context (NUL-terminated,
 * truncated to len bytes) into buf.  Returns GS_OK or GS_E_INVALID. */
gs_status gs_get_last_error(gs_ctx* ctx, char* buf, size_t len);

/* Static, human-readable name of a status code. */
const char* gs_status_string(gs_status s);

/* Releases the context and its device workspace.  NULL is ignored. */
void gs_destroy(gs_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GRIDSHIFT_H */
