// lse_step_plan.cu -- the per-call set-up of the step: its arguments, which
// step kernel runs (tile form, streaming form or the generic kernel), the
// tensor maps of the TMA forms, and the per-iteration flags.  Shared by
// lse_evolve and lse_evolve_static.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "lse_internal.h"

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t,
                                  void *, const cuuint64_t *, const cuuint64_t *,
                                  const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

// Tensor map over a pitched array of `bands` planes of the storage type
// (LSE_F32 / LSE_F16 / LSE_BF16); boxes of box_w x box_h elements (x all
// bands).  pitch and band_stride count elements.
bool encode_box(CUtensorMap *m, const void *base, int storage, int W, int H, int pitch,
                size_t band_stride, int bands, int box_w, int box_h)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const int es_bytes = storage == LSE_F32 ? 4 : 2;
    const CUtensorMapDataType ty = storage == LSE_F16    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : storage == LSE_BF16   ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)bands};
    cuuint64_t strides[2] = {(cuuint64_t)pitch * es_bytes, (cuuint64_t)band_stride * es_bytes};
    cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, (cuuint32_t)bands};
    cuuint32_t es[3] = {1, 1, 1};
    const cuuint32_t rank = bands > 1 ? 3 : 2;
    CUresult r = fn(m, ty, rank, const_cast<void *>(base), dims,
                    strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Persistent evolutions run one at a time on a device, in the order they
// were enqueued, whatever their streams: two of them resident together could
// each hold part of the SMs while their grid barriers wait for CTAs that
// cannot become resident.  Each one waits on an event the previous one
// recorded (not under stream capture, where the graph's own order applies).
constexpr int kMaxDev = 64;
std::mutex g_coop_mutex;
cudaEvent_t g_coop_event[kMaxDev];

bool persist_enabled()
{
    const char *v = getenv("LSE_PERSIST");
    return !(v && strcmp(v, "0") == 0);
}

// Runs `launch` (a cooperative launch on s) after the device's previous
// persistent evolution and makes it the one the next waits for (not under
// stream capture, where the graph's own order applies).
template <class F>
cudaError_t coop_ordered(cudaStream_t s, F launch)
{
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorNotSupported;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    err = cudaStreamIsCapturing(s, &cs);
    if (err != cudaSuccess) return err;
    const bool chain = cs == cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> lock(g_coop_mutex);
    if (chain && !g_coop_event[dev]) {
        err = cudaEventCreateWithFlags(&g_coop_event[dev], cudaEventDisableTiming);
        if (err != cudaSuccess) {
            g_coop_event[dev] = nullptr;
            return err;
        }
        err = cudaEventRecord(g_coop_event[dev], s);
        if (err != cudaSuccess) return err;
    }
    if (chain && (err = cudaStreamWaitEvent(s, g_coop_event[dev], 0)) != cudaSuccess) return err;
    err = launch();
    if (err != cudaSuccess) return err;
    return chain ? cudaEventRecord(g_coop_event[dev], s) : cudaSuccess;
}

}  // namespace

namespace lse_detail {

cudaError_t launch_evolve(StepPlan &plan, int sm_count, cudaStream_t s)
{
    if (plan.form != LSE_FORM_TILE || plan.args.mb_split || !persist_enabled())
        return cudaErrorNotSupported;
    EvolveArgs e;
    e.a = plan.args;
    e.phi[0] = plan.phi[0];
    e.phi[1] = plan.phi[1];
    e.cap = plan.iterations;
    e.reinit_period = plan.reinit_period;
    e.early_stop = plan.early_stop ? 1 : 0;
    return coop_ordered(s, [&]() {
        return launch_evolve_tile(e, plan.phi_maps[0], plan.phi_maps[1], plan.data_map,
                                  plan.nblocks, sm_count, s);
    });
}

cudaError_t coop_chain_mark(cudaStream_t s)
{
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxDev) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    err = cudaStreamIsCapturing(s, &cs);
    if (err != cudaSuccess || cs != cudaStreamCaptureStatusNone) return err;
    std::lock_guard<std::mutex> lock(g_coop_mutex);
    return g_coop_event[dev] ? cudaEventRecord(g_coop_event[dev], s) : cudaSuccess;
}

bool evolve_bands_applies(int H, int W, int B, const lse_params &p)
{
    return persist_enabled() && p.term == LSE_TERM_REGION && B >= 2 && B <= 4 &&
           p.storage == LSE_F32 && p.order == LSE_ORDER_LISTING && p.padding == LSE_PAD_ZERO &&
           p.ts >= 3 && p.ts <= 15 && (long long)H * W < 0xFFFFFFFFll;
}

bool plan_evolve_bands(int H, int W, int B, const lse_params &p, int pitch,
                       size_t band_stride, const float *bands, float *const phi[2],
                       LseDevState *st, LseCandidates *cand, int sm_count, EvolveArgs *e,
                       CUtensorMap maps[3], int *nblocks)
{
    if (!evolve_bands_applies(H, W, B, p) || !cand) return false;
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.rad = (p.ts - 1) / 2;
    a.storage = LSE_F32;
    constexpr int kNw = 4;            // 32-row tiles: the bands of a tile fill the memory
    if (!plan_step_tile(H, W, 1, LSE_TERM_EDGE, a.rad, kNw, sm_count, &a, nblocks))
        return false;
    a.H = H;
    a.W = W;
    a.B = B;
    a.term = LSE_TERM_REGION;
    double taps[16];
    gauss_taps(p.sigma, a.rad, taps);
    for (int k = 0; k < 16; ++k) a.taps[k] = k <= a.rad ? (float)taps[k] : 0.0f;
    a.dt = p.dt;
    a.half_dt = 0.5f * p.dt;
    a.early_thresh = p.early_stop_frac > 0.0f ? (double)p.early_stop_frac * H * W : 0.0;
    a.npix = (long long)H * W;
    a.pitch = pitch;
    a.band_stride = band_stride;
    a.data = bands;
    a.order = LSE_ORDER_LISTING;
    a.pad = LSE_PAD_ZERO;
    a.st = st;
    a.pdl = 0;
    const int urows = 8 * kNw;
    if (!encode_box(&maps[0], phi[0], LSE_F32, W, H, pitch, 0, 1, 136, urows + 2) ||
        !encode_box(&maps[1], phi[1], LSE_F32, W, H, pitch, 0, 1, 136, urows + 2) ||
        !encode_box(&maps[2], bands, LSE_F32, W, H, pitch, band_stride, B, 128,
                    urows - 2 * a.rad))
        return false;
    e->a = a;
    e->phi[0] = phi[0];
    e->phi[1] = phi[1];
    e->cap = p.iterations;
    e->reinit_period = p.reinit_period;
    e->early_stop = p.early_stop_frac > 0.0f ? 1 : 0;
    e->cand = cand;
    return true;
}

cudaError_t launch_evolve_bands(int H, int W, int B, const lse_params &p, int pitch,
                                size_t band_stride, const float *bands, float *const phi[2],
                                LseDevState *st, LseCandidates *cand, int sm_count,
                                cudaStream_t s)
{
    EvolveArgs e;
    CUtensorMap maps[3];
    int nblocks = 0;
    if (!plan_evolve_bands(H, W, B, p, pitch, band_stride, bands, phi, st, cand, sm_count, &e,
                           maps, &nblocks))
        return cudaErrorNotSupported;
    return coop_ordered(s, [&]() {
        return launch_evolve_mb(e, maps[0], maps[1], maps[2], nblocks, sm_count, s);
    });
}

cudaError_t launch_evolve_bands_group(int B, int rad, const MbGroupItem *items,
                                      const int *cta_item, int nblocks, cudaStream_t s)
{
    return coop_ordered(s, [&]() {
        return launch_evolve_mb_group(B, rad, items, cta_item, nblocks, s);
    });
}

void gauss_taps(double sigma, int rad, double *out)
{
    double total = 0.0;
    for (int k = 0; k <= rad; ++k) {
        out[k] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        total += k == 0 ? out[k] : 2.0 * out[k];
    }
    for (int k = 0; k <= rad; ++k) out[k] /= total;
}

int step_form_from_env()
{
    const char *k = getenv("LSE_STEP_KERNEL");
    if (!k) return LSE_FORM_AUTO;
    if (strcmp(k, "generic") == 0) return LSE_FORM_GENERIC;
    if (strcmp(k, "stream") == 0) return LSE_FORM_STREAM;
    return LSE_FORM_AUTO;
}

bool plan_step(int H, int W, int B, const lse_params &p, int pitch, size_t band_stride,
               const void *data, float *const phi[2], LseDevState *st,
               LsePartial *partials, int sm_count, int requested, int tile_nw,
               float *dplane, StepPlan *plan)
{
    StepArgs &a = plan->args;
    memset(&a, 0, sizeof(a));
    const bool region = p.term == LSE_TERM_REGION;
    a.H = H;
    a.W = W;
    a.B = region ? B : 1;
    a.term = p.term;
    a.rad = (p.ts - 1) / 2;
    double taps[16];
    gauss_taps(p.sigma, a.rad, taps);
    for (int k = 0; k < 16; ++k) a.taps[k] = k <= a.rad ? (float)taps[k] : 0.0f;
    a.dt = p.dt;
    a.half_dt = 0.5f * p.dt;
    a.early_thresh = p.early_stop_frac > 0.0f ? (double)p.early_stop_frac * H * W : 0.0;
    a.npix = (long long)H * W;
    a.pitch = pitch;
    a.band_stride = band_stride;
    a.data = static_cast<const float *>(data);
    a.storage = p.storage;
    a.order = p.order;
    a.pad = p.padding;
    a.st = st;
    a.partials = partials;
    plan->phi[0] = phi[0];
    plan->phi[1] = phi[1];
    plan->iterations = p.iterations;
    plan->reinit_period = p.reinit_period;
    plan->early_stop = p.early_stop_frac > 0.0f;
    plan->wpc = 0;

    plan->form = LSE_FORM_GENERIC;
    const int sto = p.storage;
    // 16-bit storage: the data box starts with phi's, 4 columns left of the tile
    const int data_box_w = sto == LSE_F32 ? 128 : 136;
    // the Table I order and replicate padding run on the plain kernel only
    if (p.order != LSE_ORDER_LISTING || p.padding != LSE_PAD_ZERO) {
        if (sto != LSE_F32) return false;
        requested = LSE_FORM_GENERIC;
    }
    const int urows = 8 * tile_nw;      // u rows per tile; phi adds one halo row a side
    // vector images: the band passes write D into dplane and the tile form
    // steps on that one plane (FP32, 2-4 bands)
    if (requested == LSE_FORM_AUTO && dplane && p.term == LSE_TERM_REGION && a.B > 1 &&
        a.B <= 4 && sto == LSE_F32 &&
        plan_step_tile(H, W, 1, LSE_TERM_EDGE, a.rad, tile_nw, sm_count, &a, &plan->nblocks) &&
        encode_box(&plan->phi_maps[0], phi[0], sto, W, H, pitch, 0, 1, 136, urows + 2) &&
        encode_box(&plan->phi_maps[1], phi[1], sto, W, H, pitch, 0, 1, 136, urows + 2) &&
        encode_box(&plan->data_map, dplane, sto, W, H, pitch, 0, 1, data_box_w, urows)) {
        a.mb_split = 1;
        a.bands = static_cast<const float *>(data);
        a.data = dplane;
        plan->form = LSE_FORM_TILE;
        return true;
    }
    if (requested == LSE_FORM_AUTO &&
        plan_step_tile(H, W, a.B, p.term, a.rad, tile_nw, sm_count, &a, &plan->nblocks) &&
        encode_box(&plan->phi_maps[0], phi[0], sto, W, H, pitch, 0, 1, 136, urows + 2) &&
        encode_box(&plan->phi_maps[1], phi[1], sto, W, H, pitch, 0, 1, 136, urows + 2) &&
        encode_box(&plan->data_map, data, sto, W, H, pitch, band_stride, 1, data_box_w, urows)) {
        plan->form = LSE_FORM_TILE;
    } else if (sto != LSE_F32) {
        return false;
    } else if (requested != LSE_FORM_GENERIC &&
               plan_step_tma(H, W, a.B, p.term, a.rad, sm_count, &a, &plan->nblocks,
                             &plan->wpc) &&
               encode_box(&plan->phi_maps[0], phi[0], sto, W, H, pitch, 0, 1, 136, 1) &&
               encode_box(&plan->phi_maps[1], phi[1], sto, W, H, pitch, 0, 1, 136, 1) &&
               encode_box(&plan->data_map, data, sto, W, H, pitch, band_stride, a.B, 128, 1)) {
        plan->form = LSE_FORM_STREAM;
    } else {
        plan->nblocks = sm_count * 4;
    }
    return true;
}

cudaError_t launch_step(StepPlan &plan, int n, cudaStream_t s)
{
    StepArgs &a = plan.args;
    lse_iteration_flags(a, n, plan.iterations, plan.reinit_period, plan.early_stop,
                        plan.form != LSE_FORM_GENERIC, plan.phi);
    switch (plan.form) {
    case LSE_FORM_TILE:
        return launch_step_tile(a, plan.phi_maps[n & 1], plan.data_map, plan.nblocks, s);
    case LSE_FORM_STREAM:
        return launch_step_tma(a, plan.phi_maps[n & 1], plan.data_map, plan.nblocks,
                               plan.wpc, s);
    default:
        return launch_step_generic(a, plan.nblocks, s);
    }
}

cudaError_t launch_step_once(StepPlan &plan, bool binarise_in, cudaStream_t s)
{
    StepArgs &a = plan.args;
    lse_iteration_flags(a, 0, 1, 0, false, plan.form != LSE_FORM_GENERIC, plan.phi);
    a.binarise_in = binarise_in ? 1 : 0;
    switch (plan.form) {
    case LSE_FORM_TILE:
        return launch_step_tile(a, plan.phi_maps[0], plan.data_map, plan.nblocks, s);
    case LSE_FORM_STREAM:
        return launch_step_tma(a, plan.phi_maps[0], plan.data_map, plan.nblocks, plan.wpc, s);
    default:
        return launch_step_generic(a, plan.nblocks, s);
    }
}

}  // namespace lse_detail
