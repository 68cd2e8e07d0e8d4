/*
 * lse.h -- C ABI of the GB300 library for the fast level set evolutions
 * (LSE) of Li, Shi, Wang and Miao, "Extracting Man-Made Objects From Remote
 * Sensing Images via Fast Level Set Evolutions" (arXiv 1409.7474).
 *
 * The library evolves a level set function (LSF) phi over an image I with
 * either data term of the paper:
 *   region-based (Eq. 17):  R = D / max|D|,
 *                           D = sum_b (c+_b - c-_b)(2 I_b - c+_b - c-_b),
 *                           c+ / c- the means of I over phi >= 0 / phi < 0
 *                           (Eq. 15; per band for vector images);
 *   edge-based   (Eq. 14):  R = g(I) = 1 / (1 + |grad(G_sigma1 * I)|^2).
 * Every iteration (Table I steps 2-4, Sec. III-D Steps 2-4) applies the
 * explicit update of Eq. 18, u = phi + dt * R * |grad phi|, then the Gaussian
 * regularisation v = G_sigma * u that replaces curvature, then (on
 * re-initialisation iterations) phi = +1 where v >= 0 and -1 elsewhere.
 * Discretisation: |grad phi| by unit-spacing central differences with
 * one-sided differences on the first/last row and column; G_sigma * u is the
 * same-size convolution with a normalised TS x TS sampled Gaussian and zero
 * padding outside the image.
 *
 * Conventions shared by every call
 * --------------------------------
 * Images are band-planar: band b, row y, column x at index (b*H + y)*W + x
 * (B x H x W, rows contiguous, no padding).  phi, g and the outputs are
 * H x W, row-major, float32 unless stated.
 *
 * Ownership: the caller owns every buffer it passes; the library reads the
 * inputs and writes the outputs and never frees or keeps them.  A pointer
 * may name device memory of the context's GPU or host memory (pageable or
 * pinned); host buffers are staged through device buffers the context owns
 * (pinned host memory gives asynchronous copies).
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  All device work of a call is enqueued on it in order;
 * device outputs are valid once the stream has reached the end of the call,
 * host outputs once the caller synchronises the stream.
 *
 * Errors: argument errors are returned synchronously, before anything is
 * enqueued, and lse_last_error() describes them.  Conditions found on the
 * device (non-finite input, a device wait that ran out, a degenerate region
 * term) are reported in lse_stats.status after the stream is synchronised.
 *
 * A context serves one call at a time: calls that share a context must be
 * ordered (the same stream, or synchronised), because they share its scratch.
 */
#ifndef LSE_H
#define LSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSE_OK = 0,
    LSE_ERR_INVALID_ARG = 1,   /* a bad argument; nothing was enqueued */
    LSE_ERR_OOM = 2,           /* a device or pinned allocation failed */
    LSE_ERR_CUDA = 3,          /* a CUDA call failed; see lse_last_error */
    LSE_ERR_NONFINITE = 4,     /* NaN or Inf in image, phi0 or g (device-side) */
    LSE_ERR_TIMEOUT = 5,       /* a bounded device wait ran out (device-side) */
    LSE_WARN_DEGENERATE = 6    /* some iteration ran with R = 0 (see lse_params) */
} lse_status;

typedef enum {
    LSE_TERM_REGION = 0,       /* R_Td of Eq. 17 */
    LSE_TERM_EDGE = 1          /* E_Td = g(I) of Eq. 14 */
} lse_term;

typedef enum {
    LSE_F32 = 0,               /* float32 */
    LSE_F16 = 1,               /* IEEE half */
    LSE_BF16 = 2,              /* bfloat16 */
    LSE_U16 = 3                /* uint16, read as float32(value) / 65535.0f */
} lse_dtype;

typedef enum {
    LSE_ORDER_LISTING = 0,     /* update, smooth, re-initialise (the listing) */
    LSE_ORDER_TABLE1 = 1       /* update, re-initialise, smooth (Table I) */
} lse_order;

typedef enum {
    LSE_PAD_ZERO = 0,          /* G_sigma * u with u = 0 outside the image */
    LSE_PAD_REPLICATE = 1      /* G_sigma * u with u = its nearest image value */
} lse_padding;

/* Parameters of one evolution.
 *   term            LSE_TERM_REGION or LSE_TERM_EDGE.
 *   dt              time step of Eq. 18, > 0 (the paper uses 15-18; Sec. IV-D
 *                   reports instability above 25).
 *   sigma           standard deviation of G_sigma in Step 4 (sigma of Eq. 17,
 *                   sigma_2 of the edge term), > 0.
 *   ts              template size TS of G_sigma: odd, 1 <= ts <= 31 (Table III
 *                   uses 9 and 15).
 *   iterations      iterations to run, >= 1.
 *   reinit_period   1: re-initialise to the binary LSF after every iteration
 *                   (the listing); 0: never (region term only, Step 3 makes it
 *                   optional there); k > 1: after iterations k-1, 2k-1, ...
 *   early_stop_frac 0 disables.  Otherwise the evolution stops after the first
 *                   iteration in which fewer than early_stop_frac * H * W pixels
 *                   changed sign (Step 5: stop when phi stops varying).
 *   storage         type of the work planes in HBM: LSE_F32, or LSE_F16 /
 *                   LSE_BF16 for one band (or the edge term) with ts <= 9
 *                   (at larger radii the tile layout would start TMA copies
 *                   off the 16-byte boundary that 16-bit rows need).
 *                   16-bit storage rounds the data term (I or g) to the type
 *                   once (round to nearest even) and keeps the LSF between
 *                   iterations in it; arithmetic stays FP32 and the region
 *                   sums FP64.  A re-initialised LSF is +-1, which the 16-bit
 *                   types hold exactly, so with reinit_period = 1 the only
 *                   rounding is the data term's and that of the final v
 *                   (returned as FP32 after rounding to the type).  Other
 *                   storage values, or 16-bit storage outside those cases,
 *                   give LSE_ERR_INVALID_ARG.  Not an equation of the paper,
 *                   whose own runs are FP64 (Sec. IV-A).
 *   order           LSE_ORDER_LISTING (default): each iteration updates,
 *                   smooths, then re-initialises v, as the paper's MATLAB
 *                   listing of the edge-based LSE does.  LSE_ORDER_TABLE1:
 *                   the order of Table I (steps 2, 3, 4): on a
 *                   re-initialising iteration u is binarised (u >= 0 -> +1,
 *                   else -1) before it is smoothed, and the next iteration
 *                   starts from the real-valued v.
 *   padding         LSE_PAD_ZERO (default): the listing's conv2 'same', u = 0
 *                   outside the image.  LSE_PAD_REPLICATE: u outside the image
 *                   takes the value of the nearest image pixel.
 *                   A non-default order or padding runs on the plain
 *                   shared-memory step kernel, FP32 storage only; batches,
 *                   the server and lse_evolve_static reject it.
 * Region-term degenerate rule (the paper is silent): when phi >= 0 holds
 * nowhere or everywhere, when max_b |c+_b - c-_b| <= 1e-6 * max_b(|c+_b| +
 * |c-_b|), or when max|D| = 0, that iteration uses R = 0 and the call ends
 * with LSE_WARN_DEGENERATE. */
typedef struct {
    lse_term term;
    float dt;
    float sigma;
    int ts;
    int iterations;
    int reinit_period;
    float early_stop_frac;
    lse_dtype storage;
    lse_order order;
    lse_padding padding;
} lse_params;

/* Result statistics of the last lse_evolve on a context.
 *   iterations_run  iterations executed (< iterations after an early stop).
 *   last_flips      pixels whose sign changed in the last executed iteration.
 *   area_plus       |{v >= 0}| of the returned LSF.
 *   c_plus/c_minus  region term: Eq. 15 means of each band over v >= 0 and
 *                   v < 0 of the returned LSF (0 for an empty side); edge
 *                   term: 0.
 *   norm            region term: max|D| used by the last executed iteration
 *                   (0 when R was 0); edge term: 0.
 *   elapsed_ms      device time of the iteration loop (excludes staging,
 *                   prologue and output).
 *   status          LSE_OK, LSE_WARN_DEGENERATE, LSE_ERR_NONFINITE or
 *                   LSE_ERR_TIMEOUT. */
typedef struct {
    int iterations_run;
    long long last_flips;
    long long area_plus;
    double c_plus[8];
    double c_minus[8];
    double norm;
    float elapsed_ms;
    lse_status status;
} lse_stats;

typedef struct lse_ctx lse_ctx;

/* Creates a context on CUDA device `device` for images of at most
 * `max_pixels` = H*W pixels and `max_bands` bands (1..8).  Allocates the
 * context's device scratch (ping-pong LSF buffers, staging, per-block
 * partial sums, the device statistics record) and pinned host memory for the
 * statistics.  Larger row pitches than planned grow the scratch on first
 * use; that growth is refused while the stream is being captured.
 * Returns LSE_ERR_INVALID_ARG for a NULL out-pointer, a bad device or sizes,
 * LSE_ERR_OOM when an allocation fails; *ctx is NULL on failure.
 * The step kernel is chosen per call: the TMA tile form for one band or the
 * edge term, the TMA streaming form for 2-4 bands, the plain shared-memory
 * kernel for what neither covers.  The environment variable LSE_STEP_KERNEL
 * at creation narrows the choice, for cross-checks: "stream" skips the tile
 * form, "generic" runs every iteration on the plain kernel.
 * Two more variables at creation are failure-injection hooks for tests:
 * LSE_TEST_FAIL_ALLOC=N makes the context's next N scratch growths fail as
 * a failed cudaMalloc would (the call returns LSE_ERR_OOM, nothing is
 * enqueued past that point, and later calls work); LSE_TEST_STALL_NS=T makes
 * the first tile-form step of the next lse_evolve wait T nanoseconds (at most
 * 4e9) on an
 * mbarrier that nothing completes, so that its bounded wait runs out: the
 * call ends with status LSE_ERR_TIMEOUT and the context stays usable.  Every
 * device-side wait of the library gives up after 2^24 polls or 2 s. */
lse_status lse_create(lse_ctx **ctx, int device, size_t max_pixels,
                      int max_bands);

/* Releases everything the context owns.  The caller must have synchronised
 * the streams of its calls first.  NULL is ignored. */
void lse_destroy(lse_ctx *ctx);

/* Message for the last error on this context ("" if none).  The string
 * belongs to the context and lives until its next call or lse_destroy.
 * A NULL ctx gives the message of the last failed lse_create. */
const char *lse_last_error(const lse_ctx *ctx);

/* Edge indicator g(I) of Eq. 14, computed once per image (Sec. III-D: the
 * edge term needs the image convolved with a Gaussian, the region term does
 * not).
 *   image       B x H x W in `dtype` (see conventions), host or device.
 *   sigma1, ts1 the pre-smoothing Gaussian G_sigma1 (sigma1 > 0, odd
 *               1 <= ts1 <= 31).
 *   edge_scale  multiplies the band mean before smoothing; 255 reproduces the
 *               paper's 0..255 intensity scale for images in [0, 1].
 *   g_out       H x W float32 output, host or device.
 * Multi-band images use the equal-weight band mean (the paper converts RGB
 * to one intensity channel and argues for intensity over spectral
 * information, Sec. V-B).  Gradient and convolution as in the header above. */
lse_status lse_precompute_edge(lse_ctx *ctx, const void *image,
                               lse_dtype dtype, int H, int W, int B,
                               float sigma1, int ts1, float edge_scale,
                               float *g_out, void *stream);

/* Runs params->iterations iterations of the LSE from phi0.
 *   image     B x H x W in `dtype`, host or device (region term; for the edge
 *             term only its finiteness is checked and it may be NULL).
 *   g         H x W float32 edge indicator from lse_precompute_edge (edge
 *             term), host or device; must be NULL for the region term.
 *   phi0      H x W float32 initial LSF (Eq. 13: +1 in the initial region,
 *             -1 elsewhere; any real values are accepted), host or device.
 *   phi_out   H x W float32: the smoothed LSF v of the last executed
 *             iteration, before its re-initialisation.
 *   mask_out  H x W uint8 (may be NULL): 1 where v >= 0, else 0.
 *   stats     if non-NULL, the call synchronises `stream` and fills *stats;
 *             with NULL the call returns without waiting and lse_get_stats
 *             reads them after the caller synchronises.
 * B must not exceed the context's max_bands nor H*W its max_pixels. */
lse_status lse_evolve(lse_ctx *ctx, const void *image, lse_dtype dtype,
                      int H, int W, int B, const float *g, const float *phi0,
                      const lse_params *params, float *phi_out,
                      uint8_t *mask_out, lse_stats *stats, void *stream);

/* Statistics of the last lse_evolve on ctx.  Call after synchronising that
 * call's stream; returns LSE_ERR_INVALID_ARG if no evolve has run yet. */
lse_status lse_get_stats(lse_ctx *ctx, lse_stats *stats);

/* The number of GPU kernels that lse_evolve and lse_precompute_edge calls
 * on ctx have enqueued since lse_create (0 for NULL).  An evolution of one
 * band or of the edge term on the tile form enqueues its prologue, one
 * persistent kernel for all its iterations and its output kernel; other
 * evolutions one step kernel per iteration (and two band passes per
 * iteration for vector images).  A diagnostic: it lets a caller see which
 * path ran. */
unsigned long long lse_kernel_launches(const lse_ctx *ctx);

/* Library version string, e.g. "0.1.0". */
const char *lse_version(void);

/* lse_evolve without any allocation, for callers that cannot allocate GPU
 * memory: code that runs inside a host framework or memory pool that owns
 * all device memory, or a serving loop that must not allocate (cudaMalloc
 * can synchronise the device and its latency is unbounded).  The paper has
 * no counterpart; this is an interface of this library.
 *
 * Same computation and results as lse_evolve with the same arguments, with
 * these limits:
 *   - image (region term) or g (edge term), phi0, phi_out and mask_out (may
 *     be NULL) are device memory of the current device; image and g are
 *     float32 (dtype LSE_F32 is implied) and 16-byte aligned;
 *   - W is a multiple of 4 and H * W <= LSE_STATIC_MAX_PIXELS (262144,
 *     e.g. 512 x 512); 1 <= B <= 4;
 *   - stats->elapsed_ms is -1 (timing would need CUDA events).
 *   - stats must be NULL while `stream` is capturing (filling it
 *     synchronises the stream).
 * Anything else returns LSE_ERR_INVALID_ARG without launching work, and
 * lse_last_error(NULL) says why; a failing CUDA call (the device query,
 * the look-up of the array below, a launch) returns LSE_ERR_CUDA.
 *
 * The call allocates nothing itself: its scratch (two LSF planes, per-block
 * partial sums, the device statistics record, about 2.7 MB) is a fixed
 * array in the library's device memory that every GPU which loads the
 * library holds until the process exits.  The first call on each device
 * looks up that array's device address.  Under CUDA's lazy module loading
 * that first look-up, and the first launch of each kernel, load the
 * library's device code, and loading reserves device memory (the array
 * included); a caller that must never allocate therefore makes one warm-up
 * call on each device at start-up, before capturing any stream.  All calls
 * on a device share the array and it keeps the last call's contents: calls
 * whose work overlaps on the GPU race and must be ordered by the caller
 * (one stream, or synchronisation).  Each call clears the parts of the
 * array that must start at zero. */
#define LSE_STATIC_MAX_PIXELS 262144
lse_status lse_evolve_static(const float *image, int H, int W, int B,
                             const float *g, const float *phi0,
                             const lse_params *params, float *phi_out,
                             uint8_t *mask_out, lse_stats *stats, void *stream);

/* One image of a batched evolution (lse_evolve_batch).  Every pointer is
 * device memory of the context's GPU.
 *   image     region term: B x H x W planar of `dtype` (f32/f16/bf16/u16,
 *             u16 read as value/65535); NULL for the edge term.
 *   g         edge term: H x W FP32 g(I) (lse_precompute_edge); NULL for the
 *             region term.
 *   phi0      H x W FP32 initial LSF.
 *   params    this image's parameters (term, dt, sigma, ts, iteration cap,
 *             reinit_period, early_stop_frac); storage must be LSE_F32.
 *   phi_out   H x W FP32: v of the image's last executed iteration.
 *   mask_out  H x W uint8 mask v >= 0, or NULL. */
typedef struct {
    const void *image;
    lse_dtype dtype;
    int H, W, B;
    const float *g;
    const float *phi0;
    lse_params params;
    float *phi_out;
    uint8_t *mask_out;
} lse_problem;

#define LSE_BATCH_MAX 65536

/* Runs the n independent evolutions of `problems` together (the paper has
 * no counterpart: it extracts one object per run).  Each image keeps its own
 * statistics (Eq. 15 and 17 per image), iteration cap and early stop, and
 * its results are bit for bit those of lse_evolve on that image alone.
 * Images that need the same step kernel (term, band count, template size)
 * share one launch per iteration, so small images fill the GPU together;
 * use_graph != 0 captures the whole iteration loop in a CUDA graph and
 * launches it once.  Vector images of the region term (2-4 bands, FP32
 * storage, ts 3..15) run instead as groups of persistent evolutions: one
 * cooperative launch per band count and radius (or several, when more
 * images than the device holds CTAs), each image on its own share of the
 * CTAs with its own grid barrier, all its iterations, before the other
 * images' loop.  stats (host, n entries, may be NULL) receives each
 * image's statistics; elapsed_ms is the time of the whole iteration loop.
 * The call synchronises `stream` before it returns.  Context scratch grows
 * to hold every image's planes (about (B + 2) * 4 * H * round_up(W, 32)
 * bytes per image).  Returns LSE_ERR_INVALID_ARG (nothing enqueued) when an
 * image fails lse_evolve's checks, uses host memory, 16-bit storage, or
 * needs the plain step kernel (ts > 15, more than 4 bands); LSE_ERR_OOM
 * when scratch cannot grow; LSE_ERR_CUDA on a launch failure. */
lse_status lse_evolve_batch(lse_ctx *ctx, int n, const lse_problem *problems,
                            int use_graph, lse_stats *stats, void *stream);

/* Tile-height autotuner (the paper has no counterpart; its runs are
 * single-threaded MATLAB).  The fused step for one band or the edge term
 * works on tiles of 64 rows (8 warps per CTA, 3 CTAs per SM) or 32 rows
 * (4 warps, 6 CTAs per SM): tall tiles recompute fewer halo rows, short
 * tiles give small images enough CTAs to fill the GPU.  lse_autotune runs
 * the given problems together, `iterations` iterations each (1..1000, no
 * early stop), through lse_evolve_batch on scratch outputs (the problems'
 * phi_out and mask_out are not written), and for one shape class at a time
 * (term, storage type, template size and the power of two of the image's
 * tile count; the largest classes first) flips the tile height, keeping the
 * flip if the whole set runs at least 0.5 % faster.  So the choice fits the
 * mix it was tuned on: tune on work like what will run.  Later lse_evolve,
 * lse_evolve_batch and
 * lse_server_* calls on ctx use the table, so an image still gets the same
 * bits from each of them.  Untuned classes use 32-row tiles when the image
 * has fewer 64-row tiles than the GPU has SMs, else 64-row tiles;
 * LSE_TILE_ROWS=32 or =64 in the environment at lse_create fixes one
 * height instead.  32-row steps whose grid leaves SM slots free are
 * launched as programmatic dependents (the next step's CTAs become
 * resident while the current one finishes).  Changing an
 * image's tile height regroups the partial sums of its region statistics,
 * so its results may change in the last bits (within the parity tolerances).
 * tile_rows (host, n entries, may be NULL) receives each problem's chosen
 * height in rows, 0 where the tile form does not apply (more than four
 * bands, or more than one with 16-bit storage; ts > 15; ts = 1).  Problems
 * must pass lse_evolve_batch's checks; its errors are returned.
 * Synchronises `stream`. */
lse_status lse_autotune(lse_ctx *ctx, int n, const lse_problem *problems, int iterations,
                        int *tile_rows, void *stream);

/* ------------------------------------------------------------ serving
 * A server runs evolution requests with continuous batching (the paper has
 * no counterpart).  Requests are queued on submission and admitted, first
 * come first served, while their planes fit the server's device-memory
 * budget; every lse_server_advance call then runs the next iterations of all
 * admitted requests together (in the launches lse_evolve_batch uses) and
 * retires those that reached their cap or stopped early, writing their
 * phi_out / mask_out.  Three kinds of request skip the mix and run to
 * their end inside one advance, before the mix's iterations: vector images
 * of the region term (their own path stages the bands in one launch per
 * evolution; the mix needs three per iteration) -- the queued ones below
 * 2^21 pixels run together, up to 32, as one lse_evolve_batch whose group
 * launch gives each its own CTAs; images of 2^21 pixels or more (their
 * tiles fill the GPU alone), alone through lse_evolve, the oldest first, one
 * per advance; and,
 * under light load (nothing in the mix, at most 4 requests waiting), every
 * request: an advance then runs only the oldest, so that a lightly loaded
 * server answers as fast as a direct call per request.  Each needs H * W
 * within the context's max_pixels and B within its max_bands, else it joins
 * the mix.  A request's result is bit for bit that of
 * lse_evolve on the same image, whatever else runs beside it (in the mix,
 * a single-band or edge request keeps the CTA count, statistics and
 * reductions lse_evolve gives it; a vector image too large for the context
 * joins the mix and matches lse_evolve with LSE_PERSIST=0).  One server
 * belongs to one context; its calls are not thread-safe. */
typedef struct lse_server lse_server;

/* Creates a server on ctx's GPU whose requests share budget_bytes (>= 1 MiB)
 * of device memory, allocated here.  Returns LSE_ERR_OOM when that fails. */
lse_status lse_server_create(lse_ctx *ctx, size_t budget_bytes, lse_server **out);

/* Waits for the device, then frees the server (NULL is ignored).  Requests
 * still queued or running are dropped. */
void lse_server_destroy(lse_server *sv);

/* Queues one request and returns its id (> 0).  The request's buffers (as
 * lse_problem: device memory of the context's GPU) must stay valid until
 * lse_server_poll reports it done.  Returns LSE_ERR_INVALID_ARG for
 * lse_evolve's argument errors, host memory, storage other than LSE_F32,
 * ts > 15, more than 4 bands, or a request larger than the budget. */
lse_status lse_server_submit(lse_server *sv, const lse_problem *problem, long long *id);

/* Runs the oldest request that runs alone (see above) to its end, admits
 * queued requests of the mix that fit, runs `ticks` iterations of every
 * request in the mix on `stream`, retires the finished ones, and
 * synchronises the stream.  *running (may be NULL) receives the number of
 * requests in the mix (queued requests, and those that run alone, are not
 * counted: poll each request to see it done). */
lse_status lse_server_advance(lse_server *sv, int ticks, int *running, void *stream);

/* *state = 0 queued, 1 running, 2 done.  When done, *stats (may be NULL)
 * receives the request's statistics (elapsed_ms = -1) and the server forgets
 * the request: a later poll of the id returns LSE_ERR_INVALID_ARG. */
lse_status lse_server_poll(lse_server *sv, long long id, int *state, lse_stats *stats);

/* ------------------------------------------------------------ row strips
 * One image split by rows between processes (one GPU each).  The paper runs
 * one image in one process; these calls are this library's.  A rank owns
 * rows [y0, y1) of the H x W image and holds the strip [y0 - h, y1 + h) of
 * it, clipped to the image, with h = r + 1 halo rows, r = (ts - 1) / 2:
 * Eq. 18's central differences reach one row and Step 4's smoothing r rows,
 * so a step on the strip gives the owned rows of the whole image's step
 * exactly, provided it uses the whole image's region statistics (the means
 * of Eq. 15 and the normaliser of Eq. 17, global quantities).  The caller
 * (a driver such as the package's strips module) sums the strips'
 * partial statistics over the ranks, steps each strip with the totals,
 * and copies each strip's first and last h owned rows into its neighbours'
 * halos after every step.
 *
 * Strips of one image, given the same totals, compute the same bits
 * however the image is split: the sums are exact integers (each value
 * rounded once to a multiple of 2^-fix_k), so their total does not depend
 * on which rank added which pixel. */

/* Partial statistics of the owned rows of one strip (lse_strip_partials),
 * or their sums over all ranks (the caller adds the integer fields, takes
 * the minimum of imin and the maximum of imax and amax).
 *   npix      pixels summed.
 *   n_plus    |{phi >= 0}|.
 *   flips     pixels where (phi >= 0) differs from (phi_prev >= 0).
 *   sum_w[b]  sum of s(x) q_b(x), s = +1 where phi >= 0 and -1 elsewhere,
 *   sum_a[b]  and sum of q_b(x), where q_b(x) = I_b(x) 2^fix_k rounded to
 *             the nearest integer: sum_{phi>=0} I_b = (sum_a + sum_w) / 2
 *             and sum_{phi<0} I_b = (sum_a - sum_w) / 2, times 2^-fix_k.
 *   imin/imax range of band 0; amax = max |I_b| over all bands.
 *   fix_k     the scale the sums use (lse_strip_scale). */
typedef struct {
    long long npix;
    long long n_plus;
    long long flips;
    long long sum_w[8];
    long long sum_a[8];
    double imin, imax, amax;
    int fix_k;
    int bands;
} lse_strip_sums;

/* The fixed-point scale for an image of npix pixels whose band values are at
 * most amax in magnitude: the largest k (within -120..120) with
 * max(npix, 32) * amax * 2^k at most 2^61, so that no total, nor any sum
 * of 32 values, overflows 64 bits (30 when amax is 0 or not finite).  A
 * host function: it needs no context and no GPU. */
int lse_strip_scale(double amax, long long npix);

/* Partial statistics of rows [row0, row1) of a strip of Hs rows.
 *   image     B x Hs x W in `dtype` (see conventions), host or device; NULL
 *             for the edge term (the sums and the range are then 0).
 *   phi       Hs x W float32 LSF, host or device; NULL: only npix and the
 *             range are computed (a first call, before fix_k is known).
 *   phi_prev  Hs x W float32 LSF of the previous iteration for the flip
 *             count, or NULL (flips = 0).
 *   fix_k     the scale of the sums, from lse_strip_scale on the whole
 *             image's amax and pixel count (-120..120).
 *   out       host memory: the call synchronises `stream`, fills *out and
 *             returns the device-side conditions of earlier strip calls
 *             that did not wait (see lse_strip_status) or its own.  Device
 *             memory (of the context's GPU): the sums are written there on
 *             `stream` and the call returns at once -- the caller can then
 *             add the ranks' records on the device (the first 19 64-bit
 *             words, npix .. sum_a, are integers to sum) and pass the
 *             result to lse_strip_step with no host round trip; a NaN or
 *             Inf found is kept for lse_strip_status. */
lse_status lse_strip_partials(lse_ctx *ctx, const void *image, lse_dtype dtype, int Hs, int W,
                              int B, int row0, int row1, const float *phi,
                              const float *phi_prev, int fix_k, lse_strip_sums *out,
                              void *stream);

/* Vector images (B > 1), region term: the normaliser of Eq. 17 is the
 * maximum of |D(x)| over the whole image, D(x) = sum_b alpha_b (I_b(x) -
 * mid_b), alpha_b = 2 (c+_b - c-_b), mid_b = (c+_b + c-_b) / 2 from the
 * totals (Eq. 15).  *dmax receives that maximum over rows [row0, row1) of
 * the strip (D evaluated in FP32 as the step does); the caller takes the
 * maximum over the ranks and passes it to lse_strip_step.  0 when the
 * totals make the force zero (see lse_params' degenerate rule).  totals in
 * host memory only.  Synchronises `stream`. */
lse_status lse_strip_dmax(lse_ctx *ctx, const void *image, lse_dtype dtype, int Hs, int W,
                          int B, int row0, int row1, const lse_strip_sums *totals, float dt,
                          double *dmax, void *stream);

/* One iteration (Eq. 18 then Step 4) on a strip of Hs rows with the whole
 * image's statistics.
 *   image       region term: B x Hs x W in `dtype`, host or device.
 *   g           edge term: Hs x W float32 rows of the whole image's g
 *               (lse_precompute_edge); NULL for the region term.
 *   phi         Hs x W float32 LSF, host or device.
 *   binarise_in nonzero: the step reads phi as +1 where phi >= 0 and -1
 *               elsewhere (the re-initialisation of the previous iteration,
 *               in the listing's order).
 *   params      term, dt, sigma and ts as for lse_evolve; the iteration
 *               count, re-initialisation and early stop are the caller's
 *               (ignored here); storage F32, the listing's order and zero
 *               padding only.
 *   totals      region term: the ranks' summed lse_strip_sums of phi
 *               (npix = H * W), in host memory (checked here) or in device
 *               memory of the context's GPU (read by the step's kernels in
 *               stream order, unchecked: the caller puts the whole image's
 *               imin, imax, fix_k and bands there); NULL for the edge term.
 *   norm        B > 1 region term: the maximum over the ranks of
 *               lse_strip_dmax; ignored otherwise (one band takes max|D|
 *               in closed form from the totals' range).
 *   v_out       Hs x W float32: v of this iteration, host or device (not
 *               phi's buffer).  The r + 1 rows (r = (ts - 1) / 2) next to a
 *               cut edge of the strip (an edge that is not the image's) are
 *               not the whole image's, and each further step without an
 *               exchange spoils r + 1 more: a strip with halos k (r + 1)
 *               rows deep takes k steps before the neighbours' halo
 *               exchange must replace them.
 * Device buffers with W a multiple of 4 and 16-byte alignment (phi, v_out
 * and the image or g) are read and written in place; others are staged.
 * With v_out in host memory the call synchronises `stream` and returns
 * LSE_ERR_NONFINITE or LSE_ERR_TIMEOUT for the device-side conditions of
 * lse_stats.status; with v_out on the device it returns without waiting,
 * and the next call on the context that synchronises (lse_strip_partials
 * into host memory, lse_strip_status) returns those conditions. */
lse_status lse_strip_step(lse_ctx *ctx, const void *image, lse_dtype dtype, const float *g,
                          int Hs, int W, int B, const float *phi, int binarise_in,
                          const lse_params *params, const lse_strip_sums *totals, double norm,
                          float *v_out, void *stream);

/* Synchronises `stream` and returns the device-side conditions that strip
 * calls on ctx found since the last call that reported them:
 * LSE_ERR_TIMEOUT (a step's bounded device wait ran out), LSE_ERR_NONFINITE
 * (NaN or Inf in a strip's image or LSF), else LSE_OK.  The record is then
 * cleared. */
lse_status lse_strip_status(lse_ctx *ctx, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LSE_H */
