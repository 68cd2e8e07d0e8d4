// lse_ctx.h -- the context record behind lse_ctx and the host helpers the
// C-ABI entry points share (internal).
#pragma once

#include <map>
#include <tuple>

#include "lse_internal.h"

// Key of the tile-height table: kind (region with one band, edge term, vector
// image), storage type, radius, and the bucket floor(log2(tiles)) of the
// image's tile count at 64-row tiles.
using TuneKey = std::tuple<int, int, int, int>;

struct lse_ctx {
    int device = 0;
    int sm_count = 0;
    size_t max_pixels = 0;
    int max_bands = 0;
    char err[512] = {0};
    // device scratch
    float *phi[2] = {nullptr, nullptr};
    size_t phi_cap = 0;              // elements per buffer
    float *img = nullptr;
    size_t img_cap = 0;              // elements
    float *gbuf = nullptr;
    size_t g_cap = 0;
    void *raw_in = nullptr;          // host image staging (caller dtype)
    size_t raw_cap = 0;              // bytes
    float *phi0_st = nullptr;
    size_t phi0_cap = 0;
    float *g_st = nullptr;
    size_t g_st_cap = 0;
    uint16_t *q16 = nullptr;         // data term as F16 / BF16 (16-bit storage)
    size_t q16_cap = 0;
    float *dplane = nullptr;         // vector images: D of Eq. 17, one plane
    size_t dplane_cap = 0;
    LseCandidates *cand = nullptr;   // vector images: the normaliser's candidates
    size_t cand_cap = 0;
    float *out_phi = nullptr;
    size_t out_cap = 0;
    uint8_t *out_mask = nullptr;
    size_t mask_cap = 0;
    LsePartial *partials = nullptr;
    int n_partials = 0;
    LseDevState *st = nullptr;
    LseDevState *st_host = nullptr;  // pinned mirror
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool have_stats = false;
    unsigned long long launches = 0; // kernels enqueued by lse_evolve / lse_precompute_edge
    int step_form = 0;               // LSE_STEP_KERNEL at creation (LSE_FORM_*)
    // tile form: warps per CTA (8: 64-row tiles, 4: 32-row) per shape class,
    // chosen by lse_autotune; for shapes it has not tuned, tile_nw_default
    // (LSE_TILE_ROWS at creation), or when that is 0 the automatic choice
    std::map<TuneKey, int> tile_tune;
    int tile_nw_default = 0;
    float *tune_out = nullptr;       // lse_autotune: outputs of its trial runs
    size_t tune_out_cap = 0;         // bytes
    // test hooks, from the environment at creation (see lse_create):
    // the next lse_evolve's first tile-form step waits this long (ns) on a
    // barrier nothing completes; the next N scratch growths fail
    unsigned long long test_stall_ns = 0;
    int test_fail_alloc = 0;
    // lse_evolve_batch: per-image planes, states and partials; the work list
    // and CTA tables; a pinned mirror for uploads and the states
    void *arena = nullptr;
    size_t arena_cap = 0;            // bytes
    void *tables = nullptr;
    size_t tables_cap = 0;           // bytes
    void *bhost = nullptr;
    size_t bhost_cap = 0;            // bytes (pinned)
    cudaStream_t cap_stream = nullptr;  // stream on which batches are captured
    void *mbgroup = nullptr;         // lse_evolve_batch: vector images' group items
    size_t mbgroup_cap = 0;          // and CTA tables (bytes)
    void *strip_acc = nullptr;       // lse_strip_*: the pass's device accumulator
    size_t strip_acc_cap = 0;        // bytes
    bool strip_unchecked = false;    // a strip step's status not yet read back
};

namespace lse_detail {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

enum PtrKind { PTR_NULL = 0, PTR_HOST = 1, PTR_DEVICE = 2, PTR_BAD = 3 };

// Formats the message lse_last_error returns (ctx NULL: the thread's
// context-free message).
void set_err(lse_ctx *ctx, const char *fmt, ...);
// Host, device (of `device`), or device memory of another GPU.
PtrKind classify(const void *p, int device);
size_t dtype_size(int dt);
int round_up(int v, int m);
lse_status cuda_fail(lse_ctx *ctx, cudaError_t e, const char *what);
// Grows a device buffer to at least `bytes`; refuses while capturing.
lse_status ensure(lse_ctx *ctx, void **p, size_t *cap, size_t bytes, cudaStream_t s,
                  const char *name);
bool aligned16(const void *p);
// Validates the image shape against the context.
lse_status check_image_args(lse_ctx *ctx, lse_dtype dtype, int H, int W, int B);
// Grows both LSF buffers to `elems` elements each.
lse_status ensure_phi(lse_ctx *ctx, size_t elems, cudaStream_t s);
// Makes `image` available as pitched float32 on the device (in place when it
// already is, else converted into the context's buffer).
lse_status stage_image(lse_ctx *ctx, const void *image, PtrKind kind, lse_dtype dtype, int H,
                       int W, int B, cudaStream_t s, const float **img_out, int *pitch_out,
                       size_t *band_stride);
// Validates lse_params for an image of B bands (messages via set_err).
lse_status check_params(lse_ctx *ctx, const lse_params &p, int B);
// Converts a device state record into the caller's statistics.
void fill_stats(const LseDevState &h, float elapsed_ms, lse_stats *stats);
// Warps per CTA of the tile-form step for an image on this context: the
// lse_autotune choice for its shape class, else the context's default.
int tile_nw_for(const lse_ctx *ctx, int H, int W, int B, int term, int storage, int ts);

template <typename T>
lse_status ensure_t(lse_ctx *ctx, T **p, size_t *cap_elems, size_t elems,
                    cudaStream_t s, const char *name)
{
    size_t cap_bytes = *cap_elems * sizeof(T);
    void *vp = *p;
    lse_status r = ensure(ctx, &vp, &cap_bytes, elems * sizeof(T), s, name);
    *p = static_cast<T *>(vp);
    *cap_elems = cap_bytes / sizeof(T);
    return r;
}

}  // namespace lse_detail
