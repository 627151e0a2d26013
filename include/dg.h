/*
 * dg.h -- C ABI of libdg, the GB300 (sm_103a) direct-geolocation library.
 *
 * Direct geolocation (Sec. III, Algorithm 1): for every candidate point of a
 * latitude/longitude grid on the Earth's surface and every snapshot, the
 * expected TDOA and FDOA follow from the two receivers' ECEF states (Eq. 3-10);
 * receiver 2's samples are aligned by that delay and receiver 1's derotated by
 * that FDOA, and the position-domain correlation of Eq. 11 is formed. The
 * per-snapshot grids are summed non-coherently and the maximum is the emitter
 * estimate.
 *
 * Conventions for every call:
 *   - Every function returns dg_status and never aborts; no C++ exception
 *     crosses this boundary. On error, outputs are left unchanged, the context
 *     stays usable and dg_last_error() describes the failure.
 *   - Device work is enqueued on the CUDA stream given to dg_create, in call
 *     order. Calls on one context must not run concurrently from several host
 *     threads.
 *   - "device pointer" means memory of the context's device (cudaMalloc,
 *     cudaMallocAsync or a torch CUDA tensor); "host pointer" means ordinary
 *     or pinned host memory.
 *   - Errors found by a kernel (see DG_EUNSUPPORTED) are latched and reported
 *     by the next dg_sync or dg_argmax_refine call.
 *   - Grids are row-major [lat][lon]: the linear index of node (i, j) is
 *     i * nlon + j, i counting latitude rows from south to north, j counting
 *     longitude columns from west to east.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_ABI_VERSION 1

typedef enum {
    DG_OK = 0,
    DG_EINVAL = 1,        /* a null pointer, a size out of range, a bad enum    */
    DG_ENOMEM = 2,        /* device allocation failed                           */
    DG_ECUDA = 3,         /* a CUDA runtime call failed                         */
    DG_ESTATE = 4,        /* call out of order (e.g. a snapshot not loaded yet) */
    DG_ETIMEOUT = 5,      /* a bounded device wait ran out                      */
    DG_EUNSUPPORTED = 6   /* valid but outside what the kernels handle          */
} dg_status;

/* Raw IQ storage, interleaved I,Q, little-endian: float32 pairs, int16 pairs,
 * int8 pairs. Integer samples are converted exactly to float, scale 1. */
enum { DG_IQ_C64 = 0, DG_IQ_CI16 = 1, DG_IQ_CI8 = 2 };

/* Delay alignment. INTEGER is Eq. 9: lag L = round(dtau * fs), half away from
 * zero (the printed "/ f_s" in Eq. 9 is read as "* f_s"). LAGRANGE4 aligns at
 * the fractional delay with 4-tap cubic Lagrange interpolation at taps
 * floor(D)-1 .. floor(D)+2 (not in the paper). Samples outside [0, N) are 0. */
enum { DG_DELAY_INTEGER = 0, DG_DELAY_LAGRANGE4 = 1 };

/* Non-coherent accumulation over snapshots (Algorithm 1, "sum the grids"):
 * POWER sums |C_k|^2; MAG sums |C_k|, the paper's S of Eq. 11. */
enum { DG_ACC_POWER = 0, DG_ACC_MAG = 1 };

/* Arithmetic of the correlation and of the cost surface. Geometry (Eq. 3-10)
 * is FP64 in both. FP32 writes float[G], FP64 writes double[G]. */
enum { DG_PREC_FP32 = 0, DG_PREC_FP64 = 1 };

/* Correlation algorithm. DIRECT evaluates Eq. 11 sample by sample for every
 * candidate. CDFT groups the candidates of a snapshot by their integer lag L
 * (Eq. 9): all of them share the lag product z_L[n] = y1[n] conj(y2[n + L]),
 * so Eq. 11 becomes, per lag, a DFT of z_L in chunks of `chunk` samples at
 * `bins` Doppler frequencies spanning that lag's FDOA range (a dense
 * contraction), followed per candidate by a 6-point Lagrange interpolation
 * between the bins around its FDOA and a sum over chunks with the FDOA phase
 * of each chunk's first sample. With LAGRANGE4 the lag is floor(D) and, the
 * interpolation being linear in y2, each candidate sums the correlations of
 * lags L - 1 .. L + 2 weighted by its 4-tap weights. Its error against the
 * definition is bounded by the bin interpolation and by the arithmetic of the
 * contraction (DG_CONTRACT_*). */
enum { DG_ALGO_DIRECT = 0, DG_ALGO_CDFT = 1 };

/* Tiles of the CDFT tensor-core contraction.
 * ROWS: 128 consecutive (lag, chunk) pairs, lag-major; each row reads its own
 * capture segments and forms its lag products. LAGS: 128 consecutive lags at
 * one chunk; the rows share one y1 segment and one y2 window, staged once per
 * tile (chunk <= 1024). ROWS and LAGS form the same lag products (the 16-bit
 * scale is a power of two), so their surfaces are identical.
 * HANKEL: 512 consecutive lags at one chunk, with the product regrouped as
 * W_b(l, q) = sum_m (y1[bM+m] e^{j 2 pi nu_q m}) conj(y2[bM+m+l]): the left
 * operand (64 bins x chunk, shared by every lag of the chunk) is formed once
 * per tile, and the right operand is y2 itself read as a Hankel matrix
 * straight from shared memory (lags in 8 phases of stride 8; chunk <= 1024).
 * It rounds y1 e^{...} and y2 to 16 bits instead of the lag products and the
 * DFT matrix, so it agrees with the others within the contraction's error.
 * On this chip HANKEL is slower than LAGS (its per-phase MMAs of N = 64
 * fetch more operand bytes per flop), so AUTO does not take it: AUTO takes
 * LAGS (chunk <= 1024 or a multiple of 1024: a longer chunk is staged in
 * windows of 1024 samples) unless padding a snapshot's lags to whole blocks
 * of 128 more than doubles its tile count, and ROWS then; when the last block
 * of a snapshot would hold fewer than 64 lags, AUTO puts those lags in ROWS
 * tiles and keeps LAGS tiles for the whole blocks. */
enum { DG_TILES_AUTO = 0, DG_TILES_ROWS = 1, DG_TILES_LAGS = 2, DG_TILES_HANKEL = 3 };

/* Arithmetic of the CDFT contraction: FP32 on CUDA cores, or 16-bit
 * tensor-core products accumulated in FP32. BF16 / FP16 round the lag products
 * and the DFT matrix once to 16 bits. The X3 forms split each into a 16-bit
 * high part and a 16-bit residual and add three products (hi*hi + lo*hi +
 * hi*lo), leaving an error of about three unit roundoffs squared. FP16 forms
 * scale int16 lag products by 2^-16 into range; c64 captures must keep
 * |y1||y2| below 6e4 for them. */
enum { DG_CONTRACT_FP32 = 0, DG_CONTRACT_BF16 = 1, DG_CONTRACT_FP16 = 2, DG_CONTRACT_BF16X3 = 3,
       DG_CONTRACT_FP16X3 = 4 };

typedef struct {
    double lat0_deg, lon0_deg; /* grid centre (node ((nlat-1)/2, (nlon-1)/2))  */
    double dlat_m, dlon_m;     /* node spacing in metres at the centre latitude:
                                  dlat = dlat_m / M(lat0), dlon = dlon_m /
                                  (N(lat0) cos lat0), with the WGS-84 meridian
                                  (M) and prime-vertical (N) radii             */
    int32_t nlat, nlon;        /* nodes per column / row, each >= 1            */
} dg_grid;

/* Receiver states at one snapshot epoch, ECEF metres and metres/second
 * (Sec. III: s_i = [p_i, v_i]). Receiver 1 is i, receiver 2 is j in Eq. 7-8. */
typedef struct {
    double p1[3], v1[3], p2[3], v2[3];
} dg_ephem;

typedef struct {
    int32_t delay;   /* DG_DELAY_*                                            */
    int32_t acc;     /* DG_ACC_*                                              */
    int32_t prec;    /* DG_PREC_*                                             */
    int32_t algo;    /* DG_ALGO_*                                             */
    int32_t row0;    /* first grid row of this context's shard                */
    int32_t nrows;   /* rows in the shard; 0 = all rows from row0             */
    int32_t timing;  /* 1: time kernels with CUDA events (dg_kernel_time)     */
    int32_t chunk;   /* CDFT: samples per chunk, a multiple of 64 in
                        [64, 16384]; 0 = chosen per batch of snapshots: the
                        longest power of two whose length x bin spacing is
                        <= 5e-2 cycles in every snapshot of the batch, up to
                        1024 (FP32 or Hankel contraction) or, on the tensor
                        cores, up to 2048 while it fits every capture and
                        the batch keeps 16 lag tiles per SM (dg_cdft_chunks);
                        at most 256 on the refinement grid of
                        dg_argmax_refine (few lags: shorter chunks give the
                        contraction more tiles). DG_TILES_LAGS needs a chunk
                        <= 1024 or a multiple of 1024, DG_TILES_HANKEL one
                        <= 1024                                               */
    int32_t bins;    /* CDFT: Doppler bins per lag; 0 = 64 (the only value)   */
    int32_t contract;/* CDFT: DG_CONTRACT_*                                   */
    int32_t tiles;   /* CDFT tensor-core tile shape: DG_TILES_*               */
    int32_t scratch_mib; /* CDFT: target for the scratch of one batch of
                        snapshots (per-candidate arrays and per-lag DFTs),
                        MiB; 0 = 12288. Fewer snapshots per batch below it
                        (at least one); many contexts sharing a GPU lower it */
    int32_t rows;    /* DIRECT: grid rows per thread, i.e. candidates per
                        thread (a CTA takes 8 warps x rows grid rows x 32
                        grid columns of one snapshot); 0 = 8 (FP32,
                        INTEGER delay) or 4 (FP32 LAGRANGE4, FP64); FP32
                        takes 4, 8 or 16 (16 with LAGRANGE4
                        spills registers), FP64 2 or 4. Changes speed
                        only: every candidate's arithmetic is the same     */
} dg_options;

typedef struct dg_ctx dg_ctx;

/* Result of dg_argmax_refine. The coarse fields refer to the context's grid
 * (global row index i, even for a shard); the refined fields to the local
 * grid of the refinement (refine_n = 0 when no refinement was asked for).
 * sub_lat_deg / sub_lon_deg (not in the paper) are a parabolic three-point
 * estimate around the final maximum (the refined one when there is a
 * refinement): along each axis the node moves by
 * 0.5 (a - d) / (a - 2 b + d) nodes (a, b, d the values before, at and after
 * it), kept within [-0.5, 0.5], and by 0 at the surface's edge (a shard's
 * first or last row included), where a - 2 b + d >= 0, or where a value is
 * not finite. It is reported beside the grid maximum and never replaces it. */
typedef struct {
    int64_t index;             /* linear index in the shard's surface         */
    int32_t i, j;              /* global row, column of the coarse maximum    */
    double lat_deg, lon_deg;   /* that node                                   */
    double cost;               /* the surface value there                     */
    int32_t refine_n;          /* side of the refinement grid (odd) or 0      */
    int32_t ri, rj;            /* maximum within the refinement grid          */
    int32_t pad;
    double refined_lat_deg, refined_lon_deg, refined_cost;
    double sub_lat_deg, sub_lon_deg;  /* parabolic sub-node estimate          */
} dg_fix;

/* Kernel classes for dg_kernel_time: the main surface's correlation and
 * accumulation, the argmax passes, grid/geometry kernels, and everything the
 * local refinement of dg_argmax_refine launches (grid, correlation, sum). */
enum { DG_K_CORR = 0, DG_K_ACCUM = 1, DG_K_ARGMAX = 2, DG_K_GRID = 3, DG_K_REFINE = 4,
       DG_K_CDFT_PLAN = 5,      /* CDFT: lag ranges, histograms, scans, scatters */
       DG_K_CDFT_CONTRACT = 6,  /* CDFT: the per-lag chunked DFT                 */
       DG_K_CDFT_COMBINE = 7,   /* CDFT: per-candidate sums over chunks          */
       DG_K_COARSE = 8,         /* dg_coarse_maps: the whole coarse pipeline     */
       DG_K_NCLASS = 9 };

/* Defaults: INTEGER delay, POWER accumulation, FP32, DIRECT, whole grid, no
 * timing, CDFT automatic chunk / 64 bins / FP32 contraction. o must not be
 * NULL. */
void dg_options_default(dg_options *o);

/* Create a context for one grid and one set of K snapshot ephemerides.
 * Converts every candidate of the shard to ECEF on the device (Algorithm 1,
 * first step; Sec. III). grid, eph (K entries) and opt are host pointers read
 * during the call; opt may be NULL for defaults. cuda_stream is a cudaStream_t
 * (NULL = the legacy default stream) on the current device; it must outlive
 * the context. fs_hz > 0 is the complex sampling rate, fc_hz > 0 the carrier
 * (lambda = c / fc in Eq. 6). The context owns its device memory (grid ECEF,
 * ephemerides, captures, scratch), allocated stream-ordered on cuda_stream.
 * On success *out is a new context; release it with dg_destroy. */
dg_status dg_create(const dg_grid *grid, const dg_ephem *eph, int32_t K, double fs_hz,
                    double fc_hz, const dg_options *opt, void *cuda_stream, dg_ctx **out);

/* Copy snapshot `step` (0 <= step < K) of both receivers into the context:
 * n_samples >= 1 complex samples each of format fmt (DG_IQ_*), stream-ordered.
 * is_device_ptr = 0: y1, y2 are host pointers (pageable memory is staged by
 * the CUDA runtime before this returns; pinned memory may be reused only after
 * the stream has passed this copy). is_device_ptr = 1: device pointers,
 * reusable after the stream has passed the copy. Reloading a step replaces it.
 * Per Sec. II (Eq. 2), sample 0 of each snapshot is t = 0. */
dg_status dg_load_capture(dg_ctx *ctx, int32_t step, int32_t fmt, const void *y1, const void *y2,
                          int64_t n_samples, int32_t is_device_ptr);

/* Move the context to another grid (no counterpart in the paper): the
 * snapshots, ephemerides and options stay, the candidate ECEF is recomputed
 * on the stream and every plan that depends on the grid is dropped, so that
 * one context with its captures loaded can search several regions in turn.
 * The grid may have any size (the ECEF buffer grows when needed, a
 * stream-ordered reallocation). Needs a context over the whole grid (no row
 * shard; DG_EUNSUPPORTED). A CUDA graph captured on the old grid, and a batch
 * holding the context, become stale (DG_ESTATE on launch until recaptured).
 * grid is a host pointer read during the call. */
dg_status dg_set_grid(dg_ctx *ctx, const dg_grid *grid);

/* Search several regions in turn (no counterpart in the paper; the dense
 * stage of a proposal-based search): for each of the n (1..256) grids in
 * regions (host array, all with the same nlat x nlon), the context moves to
 * it (dg_set_grid) and the cost surface of Algorithm 1 is written to
 * costs + r * nlat * nlon (device, the context's precision, room for
 * n * nlat * nlon values) with its argmax, all stream-ordered; then one host
 * synchronisation, and the region whose argmax holds the largest cost (ties:
 * the first) gets the dense re-evaluation of dg_argmax_refine, whose fix is
 * written to *out (host). *best (host, may be NULL) receives that region's
 * index. The context is left on that region's grid. Needs a context over the
 * whole grid and every snapshot loaded. */
dg_status dg_search_regions(dg_ctx *ctx, const dg_grid *regions, int32_t n, void *costs,
                            double refine_spacing_m, double refine_window_m, dg_fix *out, int32_t *best);

/* The cost surface of the shard (Eq. 11 summed over snapshots, Algorithm 1):
 * out[p] = sum_k |C_k(p)|^2 (or |C_k(p)|), p over the shard's nrows * nlon
 * nodes. out is a device pointer to float (FP32) or double (FP64) with room
 * for nrows * nlon values; it is written on the stream, asynchronously.
 * DG_ESTATE if any of the K snapshots is not loaded. */
dg_status dg_cost_surface(dg_ctx *ctx, void *out);

/* Argmax of a surface produced by dg_cost_surface (device pointer, same
 * precision; ties go to the lowest linear index; NaN never wins), then, if
 * refine_spacing_m > 0 and window_m >= refine_spacing_m, a dense re-evaluation
 * on a local grid centred on that node with that spacing and half-width
 * round(window_m / refine_spacing_m) nodes, and its argmax (Sec. III: the
 * maximum of S is the maximum-likelihood estimate). Synchronises the stream.
 * out is a host pointer. */
dg_status dg_argmax_refine(dg_ctx *ctx, const void *cost, double refine_spacing_m, double window_m,
                           dg_fix *out);

/* One detected emitter (dg_detect). */
typedef struct {
    int64_t index;             /* linear index in the shard's surface          */
    int32_t i, j;              /* global row, column                           */
    double lat_deg, lon_deg;   /* that node                                    */
    double value;              /* the surface value there                      */
} dg_peak;

/* Threshold detection of emitters on a surface from dg_cost_surface (device
 * pointer, the context's precision; Algorithm 1, last step: apply a threshold
 * to the summed grid). A node is reported when its value is >= the threshold
 * and it is the maximum of the (2 radius + 1)^2 window of nodes around it
 * (within the shard); among equal values the lowest linear index wins, so a
 * plateau gives one peak. relative = 1 reads threshold as a fraction of the
 * surface maximum. Peaks are ordered by value (descending, ties by index);
 * at most max_peaks (<= 2048) are written to out (host, max_peaks entries) and
 * their number to *n_out. 0 <= radius <= 64. When more than 2048 peaks pass
 * the test, the threshold is raised on the host to the max_peaks-th value of
 * the 2048 the device kept and the test repeated (at most 8 times): the
 * max_peaks largest peaks always pass it, so the result is the same.
 * DG_EUNSUPPORTED only if more than 2048 peaks share the value at which that
 * stops (raise the threshold). Synchronises the stream. */
dg_status dg_detect(dg_ctx *ctx, const void *cost, double threshold, int32_t relative, int32_t radius,
                    int32_t max_peaks, dg_peak *out, int32_t *n_out);

/* CUDA-graph replay of whole steps (the paper has no counterpart: this
 * takes the host out of the per-step loop of Algorithm 1). A step is
 * dg_cost_surface(ctx, cost), the argmax of cost and, if refine_spacing_m > 0
 * and refine_window_m >= refine_spacing_m, the refinement of
 * dg_argmax_refine, whose grid is centred on the argmax on the device.
 * dg_graph_capture runs one step uncaptured (allocating and planning
 * everything), then records the next as a CUDA graph owned by the context.
 * It needs every snapshot loaded and a context created on a non-default
 * stream (DG_EUNSUPPORTED otherwise). Captures reloaded with dg_load_capture
 * in the same formats and lengths feed the same graph; a change of format,
 * length or capacity makes dg_graph_launch return DG_ESTATE until the next
 * capture. dg_graph_launch enqueues one step on the context's stream
 * (asynchronous). dg_graph_fix waits for the stream, reports latched kernel
 * errors, and returns the fix of the last step (the same fields as
 * dg_argmax_refine; DG_EINVAL if the surface held no finite value). */
dg_status dg_graph_capture(dg_ctx *ctx, void *cost, double refine_spacing_m, double refine_window_m);
dg_status dg_graph_launch(dg_ctx *ctx);
dg_status dg_graph_fix(dg_ctx *ctx, dg_fix *out);

/* Many independent captures as one graph (the batching of many uneven
 * geolocation problems): one step of each context (its own grid, snapshots,
 * lengths, formats and options; all on one device, each on its own
 * non-default stream) is a branch forked from and joined to `stream`, so
 * independent steps run concurrently on the GPU. costs[i] is context i's
 * surface (device). dg_batch_capture runs each step once uncaptured first.
 * dg_batch_launch enqueues all n steps on `stream`, after the work queued
 * on each context's stream so far (capture loads); dg_batch_fixes waits
 * for it and writes n fixes (host); a context whose step failed gets
 * index = -1 and the first failure is returned. A context must not be used
 * by other calls while a launch of its batch is in flight.
 * When every context runs CDFT on the tensor cores (lag or row tiles) with
 * one capture format and one contraction arithmetic, the contractions of
 * the main surfaces are shared: round r is one persistent launch over the
 * tiles of the r-th snapshot batch of every context that has one (a device
 * work list over (capture, snapshot, tile)), with each context's plan
 * before it and its combine after it on the context's own branch. Rounds =
 * the most snapshot batches of any context (dg_batch_rounds; 0 when the
 * contractions are per context). Refinement surfaces stay per context. */
typedef struct dg_batch dg_batch;
dg_status dg_batch_capture(dg_ctx *const *ctxs, int32_t n, void *const *costs, double refine_spacing_m,
                           double refine_window_m, void *stream, dg_batch **out);
dg_status dg_batch_launch(dg_batch *batch);
dg_status dg_batch_fixes(dg_batch *batch, dg_fix *out);
int64_t dg_batch_launch_count(const dg_batch *batch); /* kernels per launch */
int32_t dg_batch_rounds(const dg_batch *batch);        /* shared contraction rounds */
dg_status dg_batch_destroy(dg_batch *batch);

/* Autotuning of the launch shape (no counterpart in the paper; it is the
 * successor of the paper's batch-size sweep, Sec. V-B).
 * DG_ALGO_CDFT: every chunk length 256 .. 1024 (tensor cores: .. 2048,
 * within the shortest capture), in powers of two, that the bin-spacing
 * bound admits for this grid and these snapshots, and for tensor-core
 * contractions every tile shape that takes it (DG_TILES_ROWS,
 * DG_TILES_LAGS, DG_TILES_HANKEL). Every candidate meets the same
 * interpolation bound, so the choice changes speed, not the error class.
 * DG_ALGO_DIRECT: the grid rows per thread (dg_options.rows: 4, 8, 16 in
 * FP32, 16 not with LAGRANGE4; 2, 4 in FP64), i.e. the candidates per CTA;
 * the surface is the same, bit for bit, for every value.
 * It times dg_cost_surface into cost (device, the context's precision; its
 * contents are overwritten) with CUDA events on the context's stream: one
 * untimed run, then reps >= 1 timed runs, keeping the median. The fastest
 * shape is written into the context's options (chunk and tiles, or rows)
 * and reported in *out. Results are cached per process by grid size,
 * snapshot count, lengths and formats, sampling rate, algorithm, precision,
 * delay mode and contraction: a cached shape is applied without timing
 * (out->cached = 1). Synchronises. */
typedef struct {
    int32_t chunk;    /* CDFT: samples per chunk chosen (0 for DIRECT)        */
    int32_t tiles;    /* CDFT: DG_TILES_* chosen (0 for DIRECT)               */
    double ms;        /* its median surface time (0 when cached)              */
    int32_t tried;    /* shapes timed                                         */
    int32_t cached;   /* 1: taken from the process-wide cache                 */
    int32_t rows;     /* DIRECT: grid rows per thread chosen (0 for CDFT)     */
} dg_tuning;
dg_status dg_autotune(dg_ctx *ctx, void *cost, int32_t reps, dg_tuning *out);

/* Wait for the context's stream and report any latched kernel error. */
dg_status dg_sync(dg_ctx *ctx);

/* Release the context and its device memory (stream-ordered frees, then a
 * stream synchronisation). NULL is accepted. */
dg_status dg_destroy(dg_ctx *ctx);

/* Message of the last failure on ctx (ctx NULL: the calling thread's last
 * failure in dg_create). Valid until the next call on that ctx / thread. */
const char *dg_last_error(const dg_ctx *ctx);

/* --- inspection (tests, benchmarks) ------------------------------------- */

/* Candidate ECEF of the shard, device pointer to double[3][nrows*nlon]
 * (x block, then y, then z). */
dg_status dg_grid_ecef(dg_ctx *ctx, double *xyz_out);

/* Per-candidate geometry of snapshot `step` (Eq. 3-10), device pointers, each
 * nrows*nlon long, any may be NULL: lag[] = the integer lag of the context's
 * delay mode (round(D) or floor(D)), D[] = dtau * fs in samples,
 * nu[] = dfreq / fs in cycles per sample. */
dg_status dg_step_geometry(dg_ctx *ctx, int32_t step, int32_t *lag, double *D, double *nu);

/* Accumulated CUDA-event time of one kernel class (requires opt.timing = 1;
 * synchronises the stream). ms and launches are host pointers, may be NULL. */
dg_status dg_kernel_time(dg_ctx *ctx, int32_t kernel_class, double *ms, int64_t *launches);

/* Work units of the last CDFT surface (dg_cost_surface with DG_ALGO_CDFT),
 * summed over snapshots: lag-bucket x chunk pairs contracted (each a
 * chunk-by-bins complex DFT) and candidate x super-chunk pairs combined (the
 * combine merges chunks at the bin frequencies into the longest power-of-two
 * multiple of the chunk whose length x bin spacing stays <= 5e-2 cycles).
 * Host pointers, may be NULL; zeros before the first CDFT surface. */
dg_status dg_cdft_work(const dg_ctx *ctx, int64_t *bucket_chunks, int64_t *candidate_chunks);

/* Shortest and longest chunk (samples) the last CDFT surface used, 0 if none
 * has been computed; with opt.chunk = 0 they follow each batch's FDOA spans.
 * Host only; either pointer may be NULL. */
dg_status dg_cdft_chunks(const dg_ctx *ctx, int32_t *min_chunk, int32_t *max_chunk);

/* Reset the counters behind dg_kernel_time and dg_launch_count. */
dg_status dg_reset_counters(dg_ctx *ctx);

/* Number of kernels this context has launched since creation or the last
 * dg_reset_counters. */
int64_t dg_launch_count(const dg_ctx *ctx);

/* DG_ABI_VERSION of the loaded library. */
int32_t dg_abi_version(void);

/* Test hook of the tensor-core pipeline's timeout (not in the paper). Every
 * wait of the CDFT tensor-core contraction is bounded: it gives up after 2 s
 * of the global timer or a poll limit, the kernel then stops issuing, lets
 * the MMAs and copies it issued land, frees its tensor memory and returns,
 * and the next synchronising call reports DG_ETIMEOUT (the surface values
 * are not valid; the context stays usable). polls > 0 lowers the poll limit
 * of those waits in every CDFT surface launched afterwards, in every context
 * of the process, so that a test can make them run out; 0 restores the
 * default. Not for production use. Always DG_OK. */
dg_status dg_debug_tc_wait_limit(uint32_t polls);

/* Measured FP32 peak of the current device (not in the paper: the ceiling the
 * CUDA-core kernels' rooflines are stated against). One kernel fills every SM
 * with 2048 resident threads, each running 8 independent chains of `iters` x 16
 * fused multiply-adds; *tflops = 2 x FMAs / the launch's CUDA-event time, after
 * one shorter warm-up launch. Runs on cuda_stream (NULL: legacy default) and
 * synchronises it; allocates and frees a few bytes stream-ordered. *ms (launch
 * time) and *sm_count (the device's multiprocessor count) may be NULL.
 * DG_EINVAL for iters <= 0 or tflops NULL; DG_ECUDA / DG_ENOMEM on a CUDA
 * failure. */
dg_status dg_fp32_peak(void *cuda_stream, int32_t iters, double *tflops, double *ms, int32_t *sm_count);

/* --- coarse delay-Doppler maps on the footprint ---------------------------
 * Not in the paper as such: the input of the learned proposal. For each
 * snapshot k the cross-ambiguity function (the delay-Doppler map of the
 * two-step TDOA/FDOA method of Sec. I; Eq. 11 at an integer lag l and FDOA
 * nu, before the magnitude)
 *     X(l, nu) = sum_n y1[n] conj(y2[n + l]) exp(j 2 pi nu n)
 * is sampled at every lag l0 .. l0 + nlag - 1 that the context's grid nodes
 * take (Eq. 9, round half away from zero) and at `bins` frequencies
 * nu_q = nu_lo + q delta spanning the nodes' FDOA range [nu_lo, nu_hi]
 * (Eq. 10), delta = (nu_hi - nu_lo) / (bins - 1). It is computed in chunks of
 * `chunk` samples, each turned at nu_c = (nu_lo + nu_hi) / 2 and combined at
 * the bin frequencies (each sample's phase is then off by at most
 * |nu_q - nu_c| (chunk - 1) cycles). A = |X|^2 and mu = mean(A).
 *
 * maps (device pointer, float[K][nlat - 1][nlon - 1]) receives, for each cell
 * (i, j) -- the quadrilateral of nodes (i, j), (i + 1, j), (i, j + 1),
 * (i + 1, j + 1) -- the largest A / mu over the lags from the smallest to the
 * largest of its corners' lags and the bins from
 * floor((nu_min - nu_lo) / delta) to ceil((nu_max - nu_lo) / delta), clipped
 * (every bin when delta = 0), nu_min / nu_max its corners' FDOA extremes;
 * 0 where mu = 0. bins = 0 picks 2 bins per Doppler resolution cell (1 / N)
 * over the span, 16..256; chunk = 0 picks the longest power of two <= 1024
 * with a phase error under 1/8 cycle. Needs every snapshot loaded, a context
 * over the whole grid (no row shard; DG_EUNSUPPORTED) and >= 2 x 2 nodes.
 * The context's delay mode, accumulation and precision do not apply.
 * Enqueued on the context's stream; no host synchronisation. */
typedef struct {
    int32_t l0;       /* first lag of the snapshot's map (samples)            */
    int32_t nlag;     /* lags in the map                                      */
    double nu_lo;     /* first bin frequency (cycles per sample)              */
    double delta;     /* bin spacing                                          */
    double nu_c;      /* chunk turning frequency                              */
    double mu;        /* mean of A over its nlag x bins entries               */
} dg_coarse_step;

dg_status dg_coarse_maps(dg_ctx *ctx, int32_t bins, int32_t chunk, float *maps);

/* The last coarse maps' internals (tests): shape (host int32[3], may be NULL)
 * = bins, chunk, lag capacity C; caf (device float[K][C][bins], may be NULL)
 * receives A (lag l0 + t at row t, rows t >= nlag undefined); steps (host,
 * K entries, may be NULL) receives the per-snapshot parameters, which
 * synchronises the stream and reports latched errors. DG_ESTATE before the
 * first dg_coarse_maps. */
dg_status dg_coarse_inspect(dg_ctx *ctx, float *caf, dg_coarse_step *steps, int32_t *shape);

/* --- learned proposal network: layers, forward and backward -------------
 * Not in the paper. A small convolutional network maps coarse per-snapshot
 * delay-Doppler maps, back-projected onto the footprint (dg_coarse_maps), to
 * a heatmap of where the emitter is; the dense grid is then evaluated only
 * around the heatmap's top regions. These calls are its layers, FP32, for
 * inference and for training on the GPU.
 *
 * Tensors are dense NCHW float arrays in device memory (B images, C channels,
 * H rows, W columns, W fastest). The calls are stateless and allocate
 * nothing: they enqueue kernels on `stream` (a cudaStream_t of the current
 * device, NULL = the legacy stream) and return; the caller owns every buffer
 * and keeps it alive until the stream has run the work. Outputs must not
 * alias inputs unless stated. Results are deterministic (fixed-order
 * reductions). On DG_EINVAL nothing is launched; dg_nn_last_error() (per
 * host thread) says why. */

/* 3 x 3 cross-correlation, zero padding 1, stride 1, with bias:
 *   y[n,o,i,j] = b[o] + sum_c sum_{u,v=0..2} w[o,c,u,v] x[n,c,i+u-1,j+v-1].
 * x: B*Ci*H*W, w: Co*Ci*3*3, b: Co, y: B*Co*H*W. */
dg_status dg_nn_conv3x3_forward(const float *x, const float *w, const float *b, float *y, int32_t B,
                                int32_t Ci, int32_t Co, int32_t H, int32_t W, void *stream);

/* Floats of scratch dg_nn_conv3x3_backward needs for this shape (-1 if the
 * shape is out of range). */
int64_t dg_nn_conv3x3_scratch(int32_t B, int32_t Ci, int32_t Co, int32_t H, int32_t W);

/* Gradients of sum(dy * y) for the forward above, overwritten (not added):
 *   dx[n,c,i,j] = sum_o sum_{u,v} w[o,c,u,v] dy[n,o,i-u+1,j-v+1]   (dx may be NULL: skipped)
 *   dw[o,c,u,v] = sum_{n,i,j} dy[n,o,i,j] x[n,c,i+u-1,j+v-1]
 *   db[o]       = sum_{n,i,j} dy[n,o,i,j].
 * scratch: dg_nn_conv3x3_scratch(...) floats (device), for partial sums. */
dg_status dg_nn_conv3x3_backward(const float *x, const float *w, const float *dy, float *dx, float *dw,
                                 float *db, int32_t B, int32_t Ci, int32_t Co, int32_t H, int32_t W,
                                 float *scratch, void *stream);

/* The same convolution and gradients on the tensor cores (tcgen05): x, w and
 * dy are rounded to BF16, products accumulate in FP32, outputs are FP32
 * (the learned proposal's network arithmetic: BF16 weights and
 * activations, FP32 accumulation; not in the paper). Each output then
 * differs from the exact value by at most 2^-7 times the same sum over
 * absolute values (two BF16 roundings per product) plus the FP32
 * accumulation error. The weight gradient splits the pixels over CTAs and
 * adds the partial sums in a fixed order (deterministic). Same shapes and
 * layouts as above; the backward needs Co <= 128 (DG_EUNSUPPORTED
 * otherwise). Both take scratch: dg_nn_conv3x3_tc_scratch floats (device,
 * 16-byte aligned; -1: shape out of range; with Co > 128 the forward's
 * need only), which hold the weights
 * converted to BF16 blocks (and the backward's partial sums); one scratch
 * must not serve two calls in flight at once. dg_nn_tc_check synchronises
 * the stream and returns DG_ETIMEOUT (clearing it) if a wait of one of
 * these kernels ran out since the last check (their outputs are then
 * invalid). */
dg_status dg_nn_conv3x3_forward_tc(const float *x, const float *w, const float *b, float *y, int32_t B,
                                   int32_t Ci, int32_t Co, int32_t H, int32_t W, float *scratch,
                                   void *stream);
int64_t dg_nn_conv3x3_tc_scratch(int32_t B, int32_t Ci, int32_t Co, int32_t H, int32_t W);
dg_status dg_nn_conv3x3_backward_tc(const float *x, const float *w, const float *dy, float *dx, float *dw,
                                    float *db, int32_t B, int32_t Ci, int32_t Co, int32_t H, int32_t W,
                                    float *scratch, void *stream);
dg_status dg_nn_tc_check(void *stream);

/* h = max(z, 0) over n elements (h may equal z). */
dg_status dg_nn_relu_forward(const float *z, float *h, int64_t n, void *stream);

/* dz = dh where z > 0, else 0 (dz may equal dh). */
dg_status dg_nn_relu_backward(const float *z, const float *dh, float *dz, int64_t n, void *stream);

/* Floats of scratch dg_nn_bce_logits needs for n elements. */
int64_t dg_nn_bce_scratch(int64_t n);

/* Mean weighted binary cross-entropy of sigmoid(z) against targets t in
 * [0, 1]: loss = mean(-p t log s(z) - (1 - t) log(1 - s(z))), p = pos_weight
 * > 0, and its gradient grad = (p t (s - 1) + (1 - t) s) / n. z, t, grad: n
 * floats; loss: one float (device); scratch: dg_nn_bce_scratch(n) floats. */
dg_status dg_nn_bce_logits(const float *z, const float *t, float pos_weight, int64_t n, float *grad,
                           float *loss, float *scratch, void *stream);

/* One Adam step (Kingma & Ba, 2015) in place on p, m, v (n floats each),
 * gradient g, step counting from 1:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 *   p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
dg_status dg_nn_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1,
                     float beta2, float eps, int32_t step, void *stream);

/* Message of the calling thread's last failed dg_nn_* call. */
const char *dg_nn_last_error(void);

/* --- cost surface without device allocation ---------------------------------
 * The paper has no counterpart to this call. It serves callers that may not
 * allocate GPU memory while they process data -- for example a real-time
 * receiver chain that reserves all of its device memory at start-up so that no
 * allocation can stall or fail mid-pass, or a program whose device memory is
 * owned by another allocator (a framework's caching allocator, a pool with a
 * fixed quota). dg_create allocates; this call does not.
 *
 * It computes the same surface as dg_create + dg_load_capture (every
 * snapshot) + dg_cost_surface, with the same kernels and options. Scratch
 * (candidate ECEF, per-snapshot surfaces, snapshot table, ephemerides, an
 * error word) lives in one static device array of DG_NOALLOC_SCRATCH_BYTES
 * owned by the library; it is reserved on every GPU that loads the library's
 * device code and stays reserved until the process exits. A call needs
 * 24*G + e*K*G + 128*K bytes plus alignment, with G = shard rows * nlon and
 * e = 4 (FP32) or 8 (FP64); a larger call is rejected with DG_EINVAL and
 * nothing is launched. The call makes no cudaMalloc, cudaFree or other
 * allocating call.
 *
 * Arguments: grid, eph (K entries) and opt (NULL = defaults; timing ignored)
 * are host pointers read during the call. y1 and y2 are device pointers to
 * K * n_samples samples each of format fmt, snapshot k starting at sample
 * k * n_samples. out is a device pointer as for dg_cost_surface.
 * cuda_stream is a cudaStream_t of the current device (NULL = legacy stream).
 *
 * Behaviour: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture. The call is synchronous: it returns
 * after the stream has completed the work, so kernel-detected errors
 * (DG_EUNSUPPORTED) are returned directly. Every call uses the same array and
 * leaves its contents behind (the error word is cleared at the start of each
 * call; everything else is rewritten before it is read), so calls that
 * overlap on the GPU -- from several host threads or on several streams --
 * race and must be serialised by the caller. On failure,
 * dg_noalloc_last_error() (per host thread) says why. */
#define DG_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

dg_status dg_cost_surface_noalloc(const dg_grid *grid, const dg_ephem *eph, int32_t K, double fs_hz,
                                  double fc_hz, int32_t fmt, const void *y1, const void *y2,
                                  int64_t n_samples, const dg_options *opt, void *out, void *cuda_stream);

/* Message of the calling thread's last failed dg_cost_surface_noalloc. */
const char *dg_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
