// lse_api.cu -- host side of the C ABI in include/lse.h.
//
// Each call validates its arguments before touching the GPU, makes the
// context's device current (restoring the caller's afterwards), stages host
// buffers through context-owned device memory, and enqueues everything on
// the caller's stream:
//   lse_evolve:  [H2D] -> convert -> prologue -> iterations x ([normaliser]
//                -> step) -> output -> [D2H] -> D2H of the statistics record
//   lse_precompute_edge:  [H2D] -> [convert] -> edge -> [D2H]
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lse_ctx.h"

using namespace lse_detail;

namespace {

thread_local char g_create_err[512];

}  // namespace

namespace lse_detail {

void set_err(lse_ctx *ctx, const char *fmt, ...)
{
    char *buf = ctx ? ctx->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
}



PtrKind classify(const void *p, int device)
{
    if (!p) return PTR_NULL;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PTR_HOST;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return at.device == device ? PTR_DEVICE : PTR_BAD;
    return PTR_HOST;
}

size_t dtype_size(int dt)
{
    return dt == LSE_F32 ? 4 : 2;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

lse_status cuda_fail(lse_ctx *ctx, cudaError_t e, const char *what)
{
    set_err(ctx, "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LSE_ERR_OOM : LSE_ERR_CUDA;
}

// Grows a device buffer to at least `bytes`; refuses while capturing.
lse_status ensure(lse_ctx *ctx, void **p, size_t *cap, size_t bytes,
                  cudaStream_t s, const char *name)
{
    if (*cap >= bytes && *p) return LSE_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
        cs != cudaStreamCaptureStatusNone) {
        set_err(ctx, "buffer '%s' must grow to %zu bytes while the stream is "
                     "being captured; run one call of this shape uncaptured first",
                name, bytes);
        return LSE_ERR_INVALID_ARG;
    }
    if (*p) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise before growing scratch");
        cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    // test hook: the next growth fails as a failed cudaMalloc would
    cudaError_t e = cudaErrorMemoryAllocation;
    if (ctx->test_fail_alloc > 0) --ctx->test_fail_alloc;
    else e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_err(ctx, "cudaMalloc of %zu bytes for '%s' failed", bytes, name);
        return LSE_ERR_OOM;
    }
    *cap = bytes;
    return LSE_OK;
}


lse_status check_image_args(lse_ctx *ctx, lse_dtype dtype, int H, int W, int B)
{
    if (H < 1 || W < 1) {
        set_err(ctx, "H and W must be >= 1 (got %d x %d)", H, W);
        return LSE_ERR_INVALID_ARG;
    }
    if ((size_t)H * (size_t)W > ctx->max_pixels) {
        set_err(ctx, "H*W = %zu exceeds the context's max_pixels %zu",
                (size_t)H * W, ctx->max_pixels);
        return LSE_ERR_INVALID_ARG;
    }
    if (B < 1 || B > ctx->max_bands) {
        set_err(ctx, "B = %d outside 1..%d (context max_bands)", B, ctx->max_bands);
        return LSE_ERR_INVALID_ARG;
    }
    if (dtype < LSE_F32 || dtype > LSE_U16) {
        set_err(ctx, "unknown image dtype %d", (int)dtype);
        return LSE_ERR_INVALID_ARG;
    }
    return LSE_OK;
}

// Grows both LSF buffers to `elems` elements each.
lse_status ensure_phi(lse_ctx *ctx, size_t elems, cudaStream_t s)
{
    if (ctx->phi_cap >= elems && ctx->phi[0] && ctx->phi[1]) return LSE_OK;
    size_t c0 = ctx->phi_cap * 4, c1 = ctx->phi_cap * 4;
    void *p0 = ctx->phi[0], *p1 = ctx->phi[1];
    lse_status r = ensure(ctx, &p0, &c0, elems * 4, s, "lsf");
    ctx->phi[0] = static_cast<float *>(p0);
    if (r == LSE_OK) r = ensure(ctx, &p1, &c1, elems * 4, s, "lsf");
    ctx->phi[1] = static_cast<float *>(p1);
    ctx->phi_cap = (r == LSE_OK) ? elems : 0;
    return r;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Makes `image` available as pitched float32 on the device.
lse_status stage_image(lse_ctx *ctx, const void *image, PtrKind kind,
                       lse_dtype dtype, int H, int W, int B, cudaStream_t s,
                       const float **img_out, int *pitch_out, size_t *band_stride)
{
    if (kind == PTR_DEVICE && dtype == LSE_F32 && (W % 4) == 0 && aligned16(image)) {
        *img_out = static_cast<const float *>(image);
        *pitch_out = W;
        *band_stride = (size_t)H * W;
        return LSE_OK;
    }
    lse_status r;
    if (kind == PTR_HOST && dtype == LSE_F32 && (W % 4) == 0) {
        // the layout the kernels read (pitch = W): one copy, no conversion
        if ((r = ensure_t(ctx, &ctx->img, &ctx->img_cap, (size_t)B * H * W, s, "image")) != LSE_OK)
            return r;
        cudaError_t e = cudaMemcpyAsync(ctx->img, image, (size_t)B * H * W * 4,
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy image to device");
        *img_out = ctx->img;
        *pitch_out = W;
        *band_stride = (size_t)H * W;
        return LSE_OK;
    }
    const void *src = image;
    if (kind == PTR_HOST) {
        size_t bytes = (size_t)B * H * W * dtype_size(dtype);
        if ((r = ensure(ctx, &ctx->raw_in, &ctx->raw_cap, bytes, s, "image staging")) != LSE_OK)
            return r;
        cudaError_t e = cudaMemcpyAsync(ctx->raw_in, image, bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy image to device");
        src = ctx->raw_in;
    }
    const int pitch = round_up(W, 32);
    if ((r = ensure_t(ctx, &ctx->img, &ctx->img_cap, (size_t)B * H * pitch, s, "image")) != LSE_OK)
        return r;
    cudaError_t e = launch_convert(src, dtype, H, W, B, ctx->img, pitch, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "convert image");
    ++ctx->launches;
    *img_out = ctx->img;
    *pitch_out = pitch;
    *band_stride = (size_t)H * pitch;
    return LSE_OK;
}

lse_status check_params(lse_ctx *ctx, const lse_params &p, int B)
{
    if (p.term != LSE_TERM_REGION && p.term != LSE_TERM_EDGE) {
        set_err(ctx, "unknown term %d", (int)p.term);
        return LSE_ERR_INVALID_ARG;
    }
    if (!(p.dt > 0.0f) || !isfinite(p.dt) || !(p.sigma > 0.0f) || !isfinite(p.sigma)) {
        set_err(ctx, "need finite dt > 0 and sigma > 0 (got %g, %g)", p.dt, p.sigma);
        return LSE_ERR_INVALID_ARG;
    }
    if (p.ts < 1 || p.ts > 31 || (p.ts % 2) == 0) {
        set_err(ctx, "ts must be odd and in 1..31 (got %d)", p.ts);
        return LSE_ERR_INVALID_ARG;
    }
    if (p.iterations < 1 || p.reinit_period < 0) {
        set_err(ctx, "need iterations >= 1 and reinit_period >= 0");
        return LSE_ERR_INVALID_ARG;
    }
    if (!(p.early_stop_frac >= 0.0f) || !(p.early_stop_frac < 1.0f)) {
        set_err(ctx, "early_stop_frac must be in [0, 1)");
        return LSE_ERR_INVALID_ARG;
    }
    if (p.storage != LSE_F32 && p.storage != LSE_F16 && p.storage != LSE_BF16) {
        set_err(ctx, "storage must be LSE_F32, LSE_F16 or LSE_BF16 (got %d)", (int)p.storage);
        return LSE_ERR_INVALID_ARG;
    }
    if (p.storage != LSE_F32 && ((p.term == LSE_TERM_REGION && B != 1) || p.ts > 9)) {
        set_err(ctx, "16-bit storage needs one band (or the edge term) and ts <= 9");
        return LSE_ERR_INVALID_ARG;
    }
    if ((p.order != LSE_ORDER_LISTING && p.order != LSE_ORDER_TABLE1) ||
        (p.padding != LSE_PAD_ZERO && p.padding != LSE_PAD_REPLICATE)) {
        set_err(ctx, "unknown order %d or padding %d", (int)p.order, (int)p.padding);
        return LSE_ERR_INVALID_ARG;
    }
    if (p.storage != LSE_F32 && (p.order != LSE_ORDER_LISTING || p.padding != LSE_PAD_ZERO)) {
        set_err(ctx, "the Table I order and replicate padding need LSE_F32 storage");
        return LSE_ERR_INVALID_ARG;
    }
    if (p.term == LSE_TERM_EDGE && p.reinit_period != 1) {
        set_err(ctx, "the edge term needs reinit_period = 1 (Step 3: without "
                     "re-initialisation its LSF only grows)");
        return LSE_ERR_INVALID_ARG;
    }
    return LSE_OK;
}

void fill_stats(const LseDevState &h, float elapsed_ms, lse_stats *stats)
{
    memset(stats, 0, sizeof(*stats));
    stats->iterations_run = h.iterations_run;
    stats->last_flips = h.last_flips;
    stats->area_plus = h.area_plus;
    for (int b = 0; b < 8; ++b) {
        stats->c_plus[b] = h.c_plus[b];
        stats->c_minus[b] = h.c_minus[b];
    }
    stats->norm = h.norm_used;
    stats->elapsed_ms = elapsed_ms;
    if (h.status_bits & LSE_SBIT_NONFINITE) stats->status = LSE_ERR_NONFINITE;
    else if (h.status_bits & LSE_SBIT_TIMEOUT) stats->status = LSE_ERR_TIMEOUT;
    else if (h.status_bits & LSE_SBIT_DEGENERATE) stats->status = LSE_WARN_DEGENERATE;
    else stats->status = LSE_OK;
}

// Message for lse_last_error(NULL) from calls that have no context.
void set_contextless_error(const char *msg)
{
    snprintf(g_create_err, sizeof(g_create_err), "%s", msg);
}

}  // namespace lse_detail

extern "C" {

const char *lse_version(void) { return "0.1.0"; }

const char *lse_last_error(const lse_ctx *ctx)
{
    return ctx ? ctx->err : g_create_err;
}

void lse_destroy(lse_ctx *ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    void *bufs[] = {ctx->phi[0], ctx->phi[1], ctx->img, ctx->gbuf, ctx->raw_in,
                    ctx->phi0_st, ctx->g_st, ctx->out_phi, ctx->out_mask, ctx->q16,
                    ctx->partials, ctx->st, ctx->arena, ctx->tables, ctx->tune_out,
                    ctx->dplane, ctx->cand, ctx->strip_acc, ctx->mbgroup};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (ctx->st_host) cudaFreeHost(ctx->st_host);
    if (ctx->bhost) cudaFreeHost(ctx->bhost);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
}

lse_status lse_create(lse_ctx **out, int device, size_t max_pixels, int max_bands)
{
    if (!out) {
        set_err(nullptr, "lse_create: ctx out-pointer is NULL");
        return LSE_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (max_pixels < 1 || max_bands < 1 || max_bands > LSE_MAXB) {
        set_err(nullptr, "lse_create: need max_pixels >= 1 and 1 <= max_bands <= %d",
                LSE_MAXB);
        return LSE_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_err(nullptr, "lse_create: device %d not available (%d devices)", device, ndev);
        return LSE_ERR_INVALID_ARG;
    }
    DeviceGuard g(device);
    if (!g.ok) {
        set_err(nullptr, "lse_create: cannot make device %d current", device);
        return LSE_ERR_CUDA;
    }
    lse_ctx *ctx = new lse_ctx();
    ctx->device = device;
    ctx->max_pixels = max_pixels;
    ctx->max_bands = max_bands;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    ctx->n_partials = partials_needed(ctx->sm_count);
    ctx->step_form = step_form_from_env();
    ctx->tile_nw_default = tile_nw_from_env();
    if (const char *v = getenv("LSE_TEST_STALL_NS")) {
        ctx->test_stall_ns = strtoull(v, nullptr, 10);
        if (ctx->test_stall_ns > 4000000000ull) ctx->test_stall_ns = 4000000000ull;
    }
    if (const char *v = getenv("LSE_TEST_FAIL_ALLOC")) ctx->test_fail_alloc = atoi(v);
    cudaError_t e = cudaMalloc(&ctx->partials, sizeof(LsePartial) * ctx->n_partials);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->st, sizeof(LseDevState));
    if (e == cudaSuccess) e = cudaMemset(ctx->st, 0, sizeof(LseDevState));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->st_host, sizeof(LseDevState));
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e == cudaSuccess) {
        // plan for a square image of max_pixels; other shapes grow on demand
        size_t side = (size_t)ceil(sqrt((double)max_pixels));
        size_t pitch = (side + 31) / 32 * 32;
        size_t elems = side * pitch;
        if (elems < max_pixels) elems = max_pixels;
        e = cudaMalloc(&ctx->phi[0], elems * 4);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->phi[1], elems * 4);
        if (e == cudaSuccess) ctx->phi_cap = elems;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(nullptr, "lse_create: allocation failed: %s", cudaGetErrorString(e));
        lse_destroy(ctx);
        return LSE_ERR_OOM;
    }
    *out = ctx;
    return LSE_OK;
}

unsigned long long lse_kernel_launches(const lse_ctx *ctx)
{
    return ctx ? ctx->launches : 0ull;
}

lse_status lse_get_stats(lse_ctx *ctx, lse_stats *stats)
{
    if (!ctx || !stats) return LSE_ERR_INVALID_ARG;
    if (!ctx->have_stats) {
        set_err(ctx, "no lse_evolve has run on this context");
        return LSE_ERR_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) != cudaSuccess) {
        cudaGetLastError();
        ms = -1.0f;
    }
    fill_stats(*ctx->st_host, ms, stats);
    return LSE_OK;
}

lse_status lse_precompute_edge(lse_ctx *ctx, const void *image, lse_dtype dtype,
                               int H, int W, int B, float sigma1, int ts1,
                               float edge_scale, float *g_out, void *stream)
{
    if (!ctx) return LSE_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    lse_status r = check_image_args(ctx, dtype, H, W, B);
    if (r != LSE_OK) return r;
    if (!image || !g_out) {
        set_err(ctx, "image and g_out must not be NULL");
        return LSE_ERR_INVALID_ARG;
    }
    if (!(sigma1 > 0.0f) || !isfinite(sigma1) || ts1 < 1 || ts1 > 31 || (ts1 % 2) == 0) {
        set_err(ctx, "need sigma1 > 0 and odd 1 <= ts1 <= 31 (got %g, %d)", sigma1, ts1);
        return LSE_ERR_INVALID_ARG;
    }
    if (!isfinite(edge_scale)) {
        set_err(ctx, "edge_scale must be finite");
        return LSE_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return cuda_fail(ctx, cudaErrorInvalidDevice, "set device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PtrKind ki = classify(image, ctx->device), ko = classify(g_out, ctx->device);
    if (ki == PTR_BAD || ko == PTR_BAD) {
        set_err(ctx, "a device pointer belongs to another GPU than the context's");
        return LSE_ERR_INVALID_ARG;
    }
    const float *img;
    int pitch;
    size_t band_stride;
    if ((r = stage_image(ctx, image, ki, dtype, H, W, B, s, &img, &pitch, &band_stride)) != LSE_OK)
        return r;
    float *dst = g_out;
    if (ko == PTR_HOST) {
        if ((r = ensure_t(ctx, &ctx->out_phi, &ctx->out_cap, (size_t)H * W, s, "output staging")) != LSE_OK)
            return r;
        dst = ctx->out_phi;
    }
    const int rad1 = (ts1 - 1) / 2;
    double taps[16];
    gauss_taps(sigma1, rad1, taps);
    cudaError_t e = launch_edge(img, pitch, band_stride, H, W, B, taps, rad1,
                                (double)edge_scale, dst, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "edge kernel");
    ++ctx->launches;
    if (ko == PTR_HOST) {
        e = cudaMemcpyAsync(g_out, dst, (size_t)H * W * 4, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy g to host");
    }
    return LSE_OK;
}

lse_status lse_evolve(lse_ctx *ctx, const void *image, lse_dtype dtype, int H,
                      int W, int B, const float *g, const float *phi0,
                      const lse_params *params, float *phi_out, uint8_t *mask_out,
                      lse_stats *stats, void *stream)
{
    if (!ctx) return LSE_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!params) {
        set_err(ctx, "params must not be NULL");
        return LSE_ERR_INVALID_ARG;
    }
    const lse_params p = *params;
    lse_status r = check_image_args(ctx, dtype, H, W, B);
    if (r != LSE_OK) return r;
    if ((r = check_params(ctx, p, B)) != LSE_OK) return r;
    const bool region = p.term == LSE_TERM_REGION;
    if (!phi0 || !phi_out || (region && !image) || (!region && !g) || (region && g)) {
        set_err(ctx, "need phi0, phi_out, image (region) or g (edge); g must be "
                     "NULL for the region term");
        return LSE_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return cuda_fail(ctx, cudaErrorInvalidDevice, "set device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const PtrKind ki = classify(image, ctx->device), kg = classify(g, ctx->device),
                  kp = classify(phi0, ctx->device), ko = classify(phi_out, ctx->device),
                  km = classify(mask_out, ctx->device);
    if (ki == PTR_BAD || kg == PTR_BAD || kp == PTR_BAD || ko == PTR_BAD || km == PTR_BAD) {
        set_err(ctx, "a device pointer belongs to another GPU than the context's");
        return LSE_ERR_INVALID_ARG;
    }
    cudaError_t e;

    // host phi0 first: the call's copies go before its first kernel, so that
    // they overlap whatever the GPU still runs (kernels of this call cannot
    // start beside a persistent evolution that holds every SM)
    const float *phi0_src = phi0;
    if (kp == PTR_HOST) {
        if ((r = ensure_t(ctx, &ctx->phi0_st, &ctx->phi0_cap, (size_t)H * W, s, "phi0 staging")) != LSE_OK)
            return r;
        e = cudaMemcpyAsync(ctx->phi0_st, phi0, (size_t)H * W * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy phi0 to device");
        phi0_src = ctx->phi0_st;
    }

    // data term on the device: image bands (region) or g (edge)
    const float *data = nullptr;
    int pitch = 0;
    size_t band_stride = 0;
    const float *g_src = nullptr;
    int g_src_pitch = W;
    float *g_dst = nullptr;
    if (region) {
        if ((r = stage_image(ctx, image, ki, dtype, H, W, B, s, &data, &pitch, &band_stride)) != LSE_OK)
            return r;
    } else {
        g_src = g;
        if (kg == PTR_HOST) {
            if ((r = ensure_t(ctx, &ctx->g_st, &ctx->g_st_cap, (size_t)H * W, s, "g staging")) != LSE_OK)
                return r;
            e = cudaMemcpyAsync(ctx->g_st, g, (size_t)H * W * 4, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "copy g to device");
            g_src = ctx->g_st;
        }
        if (kg == PTR_DEVICE && (W % 4) == 0 && aligned16(g)) {
            data = g;
            pitch = W;
        } else {
            pitch = round_up(W, 32);
            if ((r = ensure_t(ctx, &ctx->gbuf, &ctx->g_cap, (size_t)H * pitch, s, "g")) != LSE_OK)
                return r;
            g_dst = ctx->gbuf;
            data = ctx->gbuf;
        }
        band_stride = (size_t)H * pitch;
    }
    // 16-bit storage: the data term becomes an F16 / BF16 plane, and the LSF
    // planes hold the same type
    const int sto = p.storage;
    const void *data_s = data;
    if (sto != LSE_F32) {
        const int pitch16 = round_up(W, 32);
        if ((r = ensure_t(ctx, &ctx->q16, &ctx->q16_cap, (size_t)H * pitch16, s, "16-bit data")) != LSE_OK)
            return r;
        const float *src = region ? data : g_src;
        const int src_pitch = region ? pitch : g_src_pitch;
        e = launch_quantise(src, src_pitch, H, W, ctx->q16, pitch16, sto, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "quantise");
        ++ctx->launches;
        data_s = ctx->q16;
        pitch = pitch16;
        band_stride = (size_t)H * pitch16;
        g_src = nullptr;
        g_dst = nullptr;
    }
    // LSF ping-pong buffers share the data term's pitch
    if ((r = ensure_phi(ctx, (size_t)H * pitch, s)) != LSE_OK) return r;
    float *out_phi = phi_out;
    uint8_t *out_mask = mask_out;
    if (ko == PTR_HOST) {
        if ((r = ensure_t(ctx, &ctx->out_phi, &ctx->out_cap, (size_t)H * W, s, "output staging")) != LSE_OK)
            return r;
        out_phi = ctx->out_phi;
    }
    if (km == PTR_HOST) {
        if ((r = ensure_t(ctx, &ctx->out_mask, &ctx->mask_cap, (size_t)H * W, s, "mask staging")) != LSE_OK)
            return r;
        out_mask = ctx->out_mask;
    }

    const int nred = ctx->sm_count * 4;
    e = launch_prologue(region ? data_s : nullptr, pitch, band_stride, phi0_src,
                        region ? nullptr : (sto == LSE_F32 ? (const void *)g_src : data_s),
                        sto == LSE_F32 ? g_src_pitch : pitch, ctx->phi[0], g_dst, pitch, H,
                        W, B, p.term, p.dt, sto, ctx->st, ctx->partials, nred, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "prologue");
    ++ctx->launches;

    // vector images on the persistent evolution: the step stages the bands
    // and forms D itself; M comes from candidate pixels found here, once
    bool fused_bands = false;
    if (region && B > 1 && ctx->step_form == LSE_FORM_AUTO && sto == LSE_F32 &&
        evolve_bands_applies(H, W, B, p)) {
        void *cp = ctx->cand;
        if ((r = ensure(ctx, &cp, &ctx->cand_cap, sizeof(LseCandidates), s, "candidates")) != LSE_OK)
            return r;
        ctx->cand = static_cast<LseCandidates *>(cp);
        e = launch_mb_candidates(data, pitch, band_stride, H, W, B, ctx->cand, ctx->st,
                                 ctx->sm_count, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "normaliser candidates");
        ctx->launches += 2;
        e = cudaEventRecord(ctx->ev0, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "event record");
        e = launch_evolve_bands(H, W, B, p, pitch, band_stride, data, ctx->phi, ctx->st,
                                ctx->cand, ctx->sm_count, s);
        if (e == cudaSuccess) {
            fused_bands = true;
            ++ctx->launches;
        } else if (e != cudaErrorNotSupported) {
            return cuda_fail(ctx, e, "persistent evolution of the bands");
        } else {
            cudaGetLastError();
        }
    }
    // vector images otherwise: the plane the band passes write D into, for
    // the tile form
    float *dplane = nullptr;
    if (!fused_bands && region && B > 1 && sto == LSE_F32 && ctx->step_form == LSE_FORM_AUTO) {
        if ((r = ensure_t(ctx, &ctx->dplane, &ctx->dplane_cap, (size_t)H * pitch, s, "D plane")) != LSE_OK)
            return r;
        dplane = ctx->dplane;
    }
    // the step's kernel, work decomposition and tensor maps
    StepPlan plan;
    plan.form = LSE_FORM_GENERIC;
    plan.args.mb_split = 0;
    if (!fused_bands &&
        !plan_step(H, W, B, p, pitch, band_stride, data_s, ctx->phi, ctx->st, ctx->partials,
                   ctx->sm_count, ctx->step_form, tile_nw_for(ctx, H, W, B, p.term, sto, p.ts),
                   dplane, &plan)) {
        set_err(ctx, "16-bit storage runs on the tile-form step only (LSE_STEP_KERNEL "
                     "narrowed the choice, or its tensor maps could not be encoded)");
        return LSE_ERR_INVALID_ARG;
    }

    // test hook: the first step of this call waits on a barrier that
    // nothing completes, so its bounded wait must run out (tile form only)
    if (ctx->test_stall_ns && plan.form == LSE_FORM_TILE) {
        plan.args.stall_ns = ctx->test_stall_ns;
        ctx->test_stall_ns = 0;
    }
    if (!fused_bands) {
        e = cudaEventRecord(ctx->ev0, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "event record");
    }
    const bool bands_pass = !fused_bands && plan.args.mb_split != 0;
    // one band or the edge term on the tile form: every iteration in one
    // persistent launch; otherwise (or when the grid cannot all be resident)
    // one launch per step
    bool persisted = fused_bands;
    if (!persisted && !bands_pass && !(region && B > 1)) {
        e = launch_evolve(plan, ctx->sm_count, s);
        if (e == cudaSuccess) {
            persisted = true;
            ++ctx->launches;
        }
        else if (e != cudaErrorNotSupported) return cuda_fail(ctx, e, "persistent evolution");
        else cudaGetLastError();
    }
    for (int n = 0; n < p.iterations && !persisted; ++n) {
        if (bands_pass) {
            // statistics of the LSF this step reads (the prologue made the
            // first ones), then D and its maximum
            if (n > 0) {
                e = launch_band_stats(data, pitch, band_stride, ctx->phi, H, W, B, p.dt, ctx->st,
                                      ctx->partials, nred, s);
                ++ctx->launches;
            }
            if (e == cudaSuccess)
                e = launch_band_dterm(data, pitch, band_stride, dplane, H, W, B, p.dt, ctx->st,
                                      ctx->partials, nred, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "band passes");
            ++ctx->launches;
        } else if (region && B > 1) {
            e = launch_normaliser(data, pitch, band_stride, H, W, B, p.dt, ctx->st,
                                  ctx->partials, nred, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "normaliser");
            ++ctx->launches;
        }
        e = launch_step(plan, n, s);
        plan.args.stall_ns = 0;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "step");
        ++ctx->launches;
    }
    e = cudaEventRecord(ctx->ev1, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event record");
    if (bands_pass) {
        // the statistics lse_stats reports: those of the returned LSF
        e = launch_band_stats(data, pitch, band_stride, ctx->phi, H, W, B, p.dt, ctx->st,
                              ctx->partials, nred, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "band statistics");
        ++ctx->launches;
    }
    e = launch_output(ctx->phi, pitch, H, W, sto, ctx->st, out_phi, out_mask, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "output");
    ++ctx->launches;
    if (persisted && (e = coop_chain_mark(s)) != cudaSuccess)
        return cuda_fail(ctx, e, "order persistent evolutions");
    if (ko == PTR_HOST) {
        e = cudaMemcpyAsync(phi_out, out_phi, (size_t)H * W * 4, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy phi to host");
    }
    if (km == PTR_HOST) {
        e = cudaMemcpyAsync(mask_out, out_mask, (size_t)H * W, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy mask to host");
    }
    e = cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(LseDevState), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy statistics");
    ctx->have_stats = true;
    if (stats) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
        return lse_get_stats(ctx, stats);
    }
    return LSE_OK;
}

}  // extern "C"
