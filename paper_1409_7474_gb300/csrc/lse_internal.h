// lse_internal.h -- shared declarations of the GB300 LSE library (internal).
//
// Device-side state lives in one LseDevState record per context.  Every
// kernel that reduces over the image writes one LsePartial per CTA; the last
// CTA to finish (ticket counter) sums them in CTA order, so every reduction
// is deterministic for a fixed launch configuration.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lse.h"

#define LSE_MAXB 8
// Relative contrast below which c+ and c- count as equal (degenerate rule).
#define LSE_CONTRAST_TOL 1e-6

// status_bits of LseDevState
#define LSE_SBIT_NONFINITE 1u
#define LSE_SBIT_TIMEOUT 2u
#define LSE_SBIT_DEGENERATE 4u
#define LSE_SBIT_ABORT (LSE_SBIT_NONFINITE | LSE_SBIT_TIMEOUT)

// Bounded spin: try_wait polls on an mbarrier before a wait is declared
// lost, and the wall-clock limit (ns, %globaltimer) that ends it sooner.
#define LSE_WAIT_LIMIT (1u << 24)
#define LSE_WAIT_NS 2000000000ull

struct alignas(16) LseDevState {
    // constants of the call (prologue)
    double imin, imax;          // range of band 0 (single-band normaliser)
    long long npix;
    // coefficients of the next step: u = phi + s' * sum_b a[b] (I_b - m[b]),
    // with s' = 2 |grad phi| and a[b] = dt * alpha[b] / (2 M)
    float a[LSE_MAXB];
    float m[LSE_MAXB];
    float af[LSE_MAXB];         // alpha[b] as float (normaliser pass)
    double alpha[LSE_MAXB];     // 2 (c+ - c-)
    double mid[LSE_MAXB];       // (c+ + c-) / 2
    double c_plus[LSE_MAXB], c_minus[LSE_MAXB];
    double norm;                // M = max|D| for the next step
    double norm_used;           // M of the last executed step
    long long area_plus;        // |{phi >= 0}| of the current LSF
    long long last_flips;
    // band sums over phi >= 0 / phi < 0 behind c_plus / c_minus; the band
    // pass of vector images keeps them up to date from the pixels that
    // changed sign (stats_iter: iterations_run they describe)
    double run_sp[LSE_MAXB], run_sm[LSE_MAXB];
    int stats_iter;
    int iterations_run;
    int done;                   // early stop reached: later steps do nothing
    int last_buf;               // ping-pong buffer holding the latest v
    int zero_force;             // next step's force is zero (degenerate rule)
    unsigned int status_bits;
    unsigned int ticket;        // last-CTA-done counter, reset by the last CTA
    unsigned int grid_bar;      // arrivals at the persistent evolution's grid
                                // barriers (zeroed before each such launch)
    // tile-form steps: the sums over the new LSF as exact 64-bit fixed-point
    // integers (value x 2^fix_k), added up with atomics in any order --
    // sum w I_b, sum I_b, |{v >= 0}|, sign changes (lse_step_tile.cuh has
    // the layout of a slot) -- one slot per step in
    // flight (one launch per step uses slot 0; the persistent evolution
    // rotates three); and the tile queues the CTAs take tiles from
    long long acc[3][12];
    unsigned int tile_ctr[2];
    int fix_k;
};

struct alignas(16) LsePartial {
    double sp[LSE_MAXB];        // sum of I_b over phi >= 0
    double sm[LSE_MAXB];        // sum of I_b over phi < 0
    long long n_plus;
    long long flips;
    float fmax, fmin;           // normaliser / prologue range
    unsigned int bits;          // status bits seen by the CTA
    int pad;
};

// Arguments common to the step kernels.
struct StepArgs {
    int H, W, B;
    int term;                   // LSE_TERM_*
    int binarise_in;            // phi_in holds v of a re-initialised step
    int iter;                   // 0-based iteration index
    int count_flips;            // count sign changes (early stop, last step)
    int store_bin;              // store sign(v) as +-1 (this step re-initialises)
    int binary_in;              // phi_in holds +-1 only (previous step stored sign(v))
    int rad;                    // (ts - 1) / 2
    int storage;                // LSE_F32 / LSE_F16 / LSE_BF16: phi and data planes
    int order;                  // LSE_ORDER_*: LISTING, or TABLE1 (generic kernel)
    int pad;                    // LSE_PAD_*: ZERO, or REPLICATE (generic kernel)
    int reinit_u;               // Table I order: binarise u before smoothing
    float taps[16];             // 1-D taps G[0..rad] (symmetric)
    float dt;                   // time step of Eq. 18
    float half_dt;              // 0.5 * dt (edge term)
    double early_thresh;        // stop when flips < early_thresh (<= 0: off)
    long long npix;
    int pitch;                  // row pitch (elements) of phi and data
    size_t band_stride;         // elements between bands of data
    const float *phi_in;
    float *phi_out;
    int out_buf;                // index of phi_out in the ping-pong pair
    const float *data;          // image bands (region) or g (edge)
    LseDevState *st;
    LsePartial *partials;
    // work decomposition of the TMA kernel
    int useful;                 // output columns per warp strip
    int n_strips;
    int n_rowblocks;
    int th;                     // output rows per item
    int n_items;
    int nw;                     // tile form: warps per CTA (8: 64-row tiles, 4: 32-row)
    int pdl;                    // tile form: launch as a programmatic dependent
                                // (the grid leaves SM slots free)
    // vector images on the tile form: the step reads the D plane of the
    // band passes as its one data plane (data), with the coefficient
    // st->a[0] = dt / (2 M); the bands themselves are at `bands`
    int mb_split;
    const float *bands;
    // test hook (0 = off): the tile form's CTAs first wait this long (ns) on
    // an mbarrier that nothing arrives at, so the bounded wait runs out
    unsigned long long stall_ns;
};

// Vector images on the persistent evolution: M = max_x |D(x)| of Eq. 17,
// D = sum_b alpha_b (I_b - mid_b), is the maximum of a linear function of
// the pixel's colour, so it is reached at a vertex of the colour cloud's
// convex hull.  The pixels that are largest and smallest along
// LSE_MB_DIRS fixed directions seed a candidate set; every step takes M over
// the candidates (FP64) and checks |D| at every pixel against it; a pixel
// beyond it joins the candidates and the step is done again with its |D|.
#define LSE_MB_DIRS 64
#define LSE_MB_CAND 512
struct LseCandidates {
    unsigned long long key[2 * LSE_MB_DIRS];  // per direction: largest / smallest pixel
    float val[LSE_MB_CAND][4];                // band values of each candidate
    unsigned int amax_bits;                   // max |I_b| over the bands (float bits)
    int count;
    int redone;                               // steps done again (a pixel beyond M)
    int pad;
};

// The persistent evolution: every iteration of one image in one cooperative
// launch of the tile form, the CTAs meeting at a grid barrier after each
// step (lse_step_tile.cuh).  `a` holds the iteration-independent arguments;
// the per-iteration flags are derived on the device.
struct EvolveArgs {
    StepArgs a;
    float *phi[2];              // the ping-pong pair
    int cap;                    // iterations to run
    int reinit_period;
    int early_stop;
    LseCandidates *cand;        // vector images: the normaliser's candidates
};

// One vector image of a group launch of the persistent vector-image
// evolution (lse_evolve_batch), in device memory: its tensor maps (phi[0],
// phi[1], the bands), its evolution, and its CTAs [cta0, cta0 + ncta).
struct alignas(128) MbGroupItem {  // CUtensorMap needs 128-byte alignment
    CUtensorMap maps[3];
    EvolveArgs e;
    int cta0, ncta;
};

// One image of a batched evolution (lse_evolve_batch, lse_server), in device
// memory.  The CTAs [start, start + nblocks) of its class's step launch work
// on it; vector images also own the normaliser CTAs [nstart, nstart +
// nnblocks).  Launch index t runs the image's iteration t - iter0.
struct alignas(128) BatchItem {   // CUtensorMap needs 128-byte alignment
    CUtensorMap phi_maps[2];    // tensor maps of phi[0], phi[1]
    CUtensorMap data_map;
    StepArgs args;              // iteration-independent step arguments
    float *phi[2];              // the ping-pong pair
    int start, nblocks;
    int cap;                    // iterations to run
    int reinit_period;
    int early_stop;
    int nstart, nnblocks;
    long long iter0;            // launch index of the image's iteration 0
};

// Re-initialisation after iteration n (0-based) with period `period`
// (1: every iteration, 0: never, k: after iterations k-1, 2k-1, ...).
__host__ __device__ inline bool lse_reinit_after(int n, int period)
{
    if (period == 1) return true;
    if (period <= 0) return false;
    return ((n + 1) % period) == 0;
}

// The per-iteration fields of the step arguments for iteration n of an
// evolution of `cap` iterations on the ping-pong pair phi[2].  A
// re-initialising step other than the last stores sign(v) directly when the
// kernel can (`bin_out`), unless an early stop may make it the last one;
// then it stores v and the next step binarises on load.  Sign changes are
// counted for the early stop and on the last step.
struct LseStepFlags {
    int store_bin, binary_in, binarise_in, count_flips;
};

__host__ __device__ inline LseStepFlags lse_step_flags(int n, int cap, int reinit_period,
                                                       bool early_stop, bool bin_out)
{
    auto stores_bin = [&](int k) {
        return bin_out && lse_reinit_after(k, reinit_period) && k < cap - 1 && !early_stop;
    };
    LseStepFlags f;
    f.store_bin = stores_bin(n) ? 1 : 0;
    f.binary_in = (n > 0 && stores_bin(n - 1)) ? 1 : 0;
    f.binarise_in =
        (n > 0 && lse_reinit_after(n - 1, reinit_period) && !stores_bin(n - 1)) ? 1 : 0;
    f.count_flips = (early_stop || n == cap - 1) ? 1 : 0;
    return f;
}

__host__ __device__ inline void lse_iteration_flags(StepArgs &a, int n, int cap,
                                                    int reinit_period, bool early_stop,
                                                    bool bin_out, float *const phi[2])
{
    const LseStepFlags f = lse_step_flags(n, cap, reinit_period, early_stop, bin_out);
    a.iter = n;
    a.phi_in = phi[n & 1];
    a.phi_out = phi[(n + 1) & 1];
    a.out_buf = (n + 1) & 1;
    a.store_bin = f.store_bin;
    a.binary_in = f.binary_in;
    a.binarise_in = f.binarise_in;
    a.count_flips = f.count_flips;
    a.reinit_u = 0;
    if (a.order == LSE_ORDER_TABLE1) {
        // Table I: the re-initialisation (step 3) acts on u, before the
        // smoothing (step 4); the next iteration reads v as it is
        a.store_bin = 0;
        a.binary_in = 0;
        a.binarise_in = 0;
        a.reinit_u = lse_reinit_after(n, reinit_period) ? 1 : 0;
    }
}

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float lse_sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------- host side
namespace lse_detail {

// Kernel launchers, one per translation unit.  Each returns the
// cudaGetLastError() of its launch.
cudaError_t launch_convert(const void *src, int dtype, int H, int W, int B,
                           float *dst, int pitch, cudaStream_t s);
// Pitched FP32 plane -> pitched F16 / BF16 plane (16-bit storage).
cudaError_t launch_quantise(const float *src, int src_pitch, int H, int W, void *dst,
                            int pitch, int storage, cudaStream_t s);
// img, g and phi_dst are planes of the storage type (LSE_F32 / LSE_F16 /
// LSE_BF16); g_dst (FP32 storage only) receives a pitched copy of g.
cudaError_t launch_prologue(const void *img, int img_pitch, size_t band_stride,
                            const float *phi0, const void *g, int g_pitch,
                            void *phi_dst, float *g_dst, int pitch, int H,
                            int W, int B, int term, float dt, int storage,
                            LseDevState *st, LsePartial *partials, int nblocks,
                            cudaStream_t s);
// Vector images on the tile form: the statistics pass (Eq. 15) over the LSF
// the last step wrote (a no-op when no step ran since the last one, so it
// may close every evolution) and the pass that writes D (Eq. 17) into dplane
// and sets M and the step coefficient; and both for launch index n of a
// batch (the pass CTAs of each image).
cudaError_t launch_band_stats(const float *bands, int pitch, size_t band_stride,
                              float *const *bufs, int H, int W, int B, float dt,
                              LseDevState *st, LsePartial *partials, int nblocks,
                              cudaStream_t s);
cudaError_t launch_band_dterm(const float *bands, int pitch, size_t band_stride, float *dplane,
                              int H, int W, int B, float dt, LseDevState *st,
                              LsePartial *partials, int nblocks, cudaStream_t s);
cudaError_t launch_band_passes_batch(const BatchItem *items, const int *blk_item, long long n,
                                     int nblocks, cudaStream_t s);
cudaError_t launch_normaliser(const float *img, int pitch, size_t band_stride,
                              int H, int W, int B, float dt, LseDevState *st,
                              LsePartial *partials, int nblocks, cudaStream_t s);
cudaError_t launch_output(float *const *bufs, int pitch, int H, int W, int storage,
                          const LseDevState *st, float *phi_out,
                          uint8_t *mask_out, cudaStream_t s);
cudaError_t launch_edge(const float *img, int pitch, size_t band_stride, int H,
                        int W, int B, const double *taps1, int rad1,
                        double edge_scale, float *g_out, cudaStream_t s);
cudaError_t launch_step_generic(const StepArgs &a, int nblocks, cudaStream_t s);
// TMA step: returns cudaErrorNotSupported when no instantiation fits
// (radius or band count), so the caller can take the generic kernel.
cudaError_t launch_step_tma(const StepArgs &a, const CUtensorMap &phi_map,
                            const CUtensorMap &data_map, int nblocks,
                            int warps_per_block, cudaStream_t s);
// Work decomposition of the TMA step for a shape on `sm_count` SMs.
bool plan_step_tma(int H, int W, int B, int term, int rad, int sm_count,
                   StepArgs *a, int *nblocks, int *warps_per_block);
// Tile-form step (one band or the edge term): work decomposition and launch.
// nw = warps per CTA (8 or 4): tiles of 8 nw u rows; its tensor maps have
// boxes of 136 x (8 nw + 2) phi and 128 (136 for 16-bit) x 8 nw data
// elements.
bool plan_step_tile(int H, int W, int B, int term, int rad, int nw, int sm_count,
                    StepArgs *a, int *nblocks);
// Whether every TMA box of the tile form starts on 16 bytes for a radius and
// element size (false for 16-bit elements at radius 5..7).
bool tile_boxes_aligned(int rad, int elem_bytes);
cudaError_t launch_step_tile(const StepArgs &a, const CUtensorMap &phi_map,
                             const CUtensorMap &data_map, int nblocks, cudaStream_t s);
int partials_needed(int sm_count);
// The persistent evolution of the tile form (one band or the edge term):
// cudaErrorNotSupported, with nothing launched, when the call cannot take it.
cudaError_t launch_evolve_tile(const EvolveArgs &e, const CUtensorMap &pm0,
                               const CUtensorMap &pm1, const CUtensorMap &dm, int nblocks,
                               int sm_count, cudaStream_t s);
// Vector images (2-4 bands, FP32) on the persistent evolution: the candidate
// seeds of the normaliser (once per image, after the prologue), and the
// evolution itself (32-row tiles; dm maps the bands as one 3-D box).
cudaError_t launch_mb_candidates(const float *bands, int pitch, size_t band_stride, int H,
                                 int W, int B, LseCandidates *cand, LseDevState *st,
                                 int sm_count, cudaStream_t s);
cudaError_t launch_evolve_mb(const EvolveArgs &e, const CUtensorMap &pm0,
                             const CUtensorMap &pm1, const CUtensorMap &dm, int nblocks,
                             int sm_count, cudaStream_t s);
// Vector images of B bands and radius rad as one cooperative group launch
// (MbGroupItem, CTA table cta_item of nblocks entries), and the number of
// its CTAs the device holds at once (0: none).
cudaError_t launch_evolve_mb_group(int B, int rad, const MbGroupItem *items,
                                   const int *cta_item, int nblocks, cudaStream_t s);
int evolve_mb_group_capacity(int B, int rad, int sm_count);

// Batched launches (lse_evolve_batch): iteration n over every image of one
// class; CTA blockIdx.x works on image blk_item[blockIdx.x].  Step kernels
// of the tile form (one band, edge term) and of the streaming form.
cudaError_t launch_step_tile_batch(int storage, int term, int nw, int rad,
                                   const BatchItem *items, const int *blk_item, long long n,
                                   int nblocks, cudaStream_t s);
cudaError_t launch_step_tma_batch_region1(int rad, const BatchItem *items, const int *blk_item,
                                          long long n, int nblocks, int wpc, cudaStream_t s);
cudaError_t launch_step_tma_batch_edge(int rad, const BatchItem *items, const int *blk_item,
                                       long long n, int nblocks, int wpc, cudaStream_t s);
cudaError_t launch_step_tma_batch_multiband(int rad, const BatchItem *items,
                                            const int *blk_item, long long n, int nblocks, int wpc,
                                            cudaStream_t s);
cudaError_t launch_normaliser_batch(const BatchItem *items, const int *blk_item, long long n,
                                    int nblocks, cudaStream_t s);

// Which step kernel a call runs.  LSE_STEP_KERNEL=generic or =stream at
// context creation (at each call for lse_evolve_static) narrows the choice.
enum { LSE_FORM_AUTO = 0, LSE_FORM_TILE = 1, LSE_FORM_STREAM = 2, LSE_FORM_GENERIC = 3 };

struct StepPlan {
    StepArgs args;
    int form;                   // LSE_FORM_TILE / _STREAM / _GENERIC
    int nblocks, wpc;
    CUtensorMap phi_maps[2], data_map;
    float *phi[2];              // the ping-pong pair (phi_maps[i] maps phi[i])
    int iterations, reinit_period;
    bool early_stop;
};

void gauss_taps(double sigma, int rad, double *out);
int step_form_from_env();
// Warps per CTA of the tile form for untuned shapes as LSE_TILE_ROWS sets it:
// 4 for "32", 8 for "64", 0 (automatic, tile_nw_default_for) otherwise.
int tile_nw_from_env();
// The automatic choice: 32-row tiles (4 warps) when the image has fewer
// 64-row tiles than the GPU has SMs, else 64-row tiles (8 warps).
int tile_nw_default_for(int H, int W, int ts, int sm_count);
// Fills the step arguments for a call and picks its kernel (`requested` is
// LSE_FORM_AUTO, _STREAM or _GENERIC; `tile_nw` the tile form's warps per
// CTA, 8 or 4; `dplane`, H x pitch floats or NULL, lets a vector image take
// the band passes and the tile form).  Returns false when no step kernel serves the call (16-bit
// storage outside the tile form).
bool plan_step(int H, int W, int B, const lse_params &p, int pitch, size_t band_stride,
               const void *data, float *const phi[2], LseDevState *st,
               LsePartial *partials, int sm_count, int requested, int tile_nw,
               float *dplane, StepPlan *plan);
// Launches iteration n (0-based) of the plan.
cudaError_t launch_step(StepPlan &plan, int n, cudaStream_t s);
// Launches one step from phi[0] into phi[1] with the coefficients already in
// the state record: the plan's only iteration, reading phi[0] as sign(phi[0])
// when binarise_in (the caller's previous step re-initialised).
cudaError_t launch_step_once(StepPlan &plan, bool binarise_in, cudaStream_t s);
// Launches every iteration of the plan as one persistent evolution when the
// plan is of the tile form and LSE_PERSIST is not "0"; cudaErrorNotSupported
// (nothing launched) otherwise, and the caller launches one step at a time.
cudaError_t launch_evolve(StepPlan &plan, int sm_count, cudaStream_t s);
// Moves the device's ordering point of persistent evolutions to the end of
// the work enqueued on s so far (not under stream capture): lse_evolve calls
// it after the output kernel of a persistent evolution, so that the next
// persistent evolution, on whatever stream, starts after that kernel rather
// than taking every SM while it waits (which would delay the output, and the
// caller's copies behind it, by a whole evolution).
cudaError_t coop_chain_mark(cudaStream_t s);
// Vector images (2-4 bands, FP32, the listing's order, zero padding, TS
// 3..15): the persistent evolution with the bands staged by the step
// (32-row tiles), after launch_mb_candidates.  evolve_bands_applies says
// whether a call can take it (LSE_PERSIST=0 says no);
// launch_evolve_bands returns cudaErrorNotSupported, with nothing launched,
// when the grid cannot be resident.
bool evolve_bands_applies(int H, int W, int B, const lse_params &p);
cudaError_t launch_evolve_bands(int H, int W, int B, const lse_params &p, int pitch,
                                size_t band_stride, const float *bands, float *const phi[2],
                                LseDevState *st, LseCandidates *cand, int sm_count,
                                cudaStream_t s);
// The arguments, tensor maps (phi[0], phi[1], the bands) and tile count of
// that evolution, without launching it; false when it does not apply.
bool plan_evolve_bands(int H, int W, int B, const lse_params &p, int pitch,
                       size_t band_stride, const float *bands, float *const phi[2],
                       LseDevState *st, LseCandidates *cand, int sm_count, EvolveArgs *e,
                       CUtensorMap maps[3], int *nblocks);
// A group of such evolutions (one band count and radius) as one cooperative
// launch, ordered like the one-image launches.
cudaError_t launch_evolve_bands_group(int B, int rad, const MbGroupItem *items,
                                      const int *cta_item, int nblocks, cudaStream_t s);
// Sets the message lse_last_error(NULL) returns (calls without a context).
void set_contextless_error(const char *msg);

}  // namespace lse_detail
