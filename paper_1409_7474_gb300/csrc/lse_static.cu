// lse_static.cu -- lse_evolve_static: the evolution without allocation.
//
// Some callers cannot allocate device memory: code running inside a host
// framework or memory pool that owns all of the GPU's memory, or a serving
// loop that must not call cudaMalloc (it may synchronise the device and its
// latency is unbounded).  This entry point runs the same kernels as
// lse_evolve, but every piece of scratch they need lives in one fixed array
// of this file, `g_static_scratch`, which each GPU that loads the library
// holds until the process exits:
//   two LSF planes of LSE_STATIC_MAX_PIXELS floats (the ping-pong buffers),
//   4096 per-block partial sums, and the device statistics record
//   (about 2.7 MB in all).
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with
// that device current) and caches it.  Calls share the array: the caller
// orders calls whose work would overlap.  Each call clears the statistics
// record (its last-block ticket must start at zero); everything else is
// written before it is read.
#include <math.h>
#include <mutex>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lse_internal.h"

using namespace lse_detail;

namespace {

constexpr size_t kPlane = LSE_STATIC_MAX_PIXELS;          // floats per LSF plane
constexpr int kMaxPartials = 4096;
constexpr size_t kPhiBytes = 2 * kPlane * sizeof(float);
constexpr size_t kPartialOff = kPhiBytes;
constexpr size_t kStateOff = (kPartialOff + kMaxPartials * sizeof(LsePartial) + 255) & ~size_t(255);
constexpr size_t kScratchBytes = kStateOff + ((sizeof(LseDevState) + 255) & ~size_t(255));

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_scratch_ptr[kMaxDevices];   // device address, per device

lse_status fail(const char *fmt, ...)
{
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    set_contextless_error(msg);
    return LSE_ERR_INVALID_ARG;
}

lse_status cuda_fail(cudaError_t e, const char *what)
{
    char msg[512];
    snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
    set_contextless_error(msg);
    return LSE_ERR_CUDA;
}

bool on_device(const void *p, int dev)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
           at.device == dev;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// The array's device address on `dev` (current), looked up on first use.
unsigned char *scratch_on(int dev, cudaError_t *err)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_static_scratch);
        if (*err != cudaSuccess) return nullptr;
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *err = cudaSuccess;
    return g_scratch_ptr[dev];
}

}  // namespace

extern "C" lse_status lse_evolve_static(const float *image, int H, int W, int B,
                                        const float *g, const float *phi0,
                                        const lse_params *params, float *phi_out,
                                        uint8_t *mask_out, lse_stats *stats,
                                        void *stream)
{
    set_contextless_error("");
    if (!params) return fail("lse_evolve_static: params must not be NULL");
    const lse_params p = *params;
    if (H < 1 || W < 1 || (W % 4) != 0)
        return fail("lse_evolve_static: need H >= 1 and W a positive multiple of 4 "
                    "(got %d x %d)", H, W);
    if ((size_t)H * (size_t)W > kPlane)
        return fail("lse_evolve_static: H*W = %zu exceeds LSE_STATIC_MAX_PIXELS = %zu; "
                    "use lse_evolve", (size_t)H * W, kPlane);
    if (B < 1 || B > 4) return fail("lse_evolve_static: B = %d outside 1..4", B);
    if (p.term != LSE_TERM_REGION && p.term != LSE_TERM_EDGE)
        return fail("lse_evolve_static: unknown term %d", (int)p.term);
    if (!(p.dt > 0.0f) || !isfinite(p.dt) || !(p.sigma > 0.0f) || !isfinite(p.sigma))
        return fail("lse_evolve_static: need finite dt > 0 and sigma > 0");
    if (p.ts < 1 || p.ts > 31 || (p.ts % 2) == 0)
        return fail("lse_evolve_static: ts must be odd and in 1..31 (got %d)", p.ts);
    if (p.iterations < 1 || p.reinit_period < 0)
        return fail("lse_evolve_static: need iterations >= 1 and reinit_period >= 0");
    if (!(p.early_stop_frac >= 0.0f) || !(p.early_stop_frac < 1.0f))
        return fail("lse_evolve_static: early_stop_frac must be in [0, 1)");
    if (p.storage != LSE_F32) return fail("lse_evolve_static: storage must be LSE_F32");
    if (p.order != LSE_ORDER_LISTING || p.padding != LSE_PAD_ZERO)
        return fail("lse_evolve_static: only the listing's order and zero padding");
    const bool region = p.term == LSE_TERM_REGION;
    if (!region && p.reinit_period != 1)
        return fail("lse_evolve_static: the edge term needs reinit_period = 1");
    const float *data = region ? image : g;
    if (!data || !phi0 || !phi_out || (region && g) || (!region && image))
        return fail("lse_evolve_static: need phi0, phi_out and exactly one of image "
                    "(region term) or g (edge term)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "lse_evolve_static: no current device");
    if (dev < 0 || dev >= kMaxDevices) return fail("lse_evolve_static: device %d", dev);
    if (!on_device(data, dev) || !on_device(phi0, dev) || !on_device(phi_out, dev) ||
        (mask_out && !on_device(mask_out, dev)))
        return fail("lse_evolve_static: buffers must be device memory of the current "
                    "device (no host staging without allocation)");
    if (!aligned16(data))
        return fail("lse_evolve_static: image / g must be 16-byte aligned");
    int sm_count = 0;
    e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "lse_evolve_static: SM count");
    if (sm_count < 1) return fail("lse_evolve_static: device %d reports %d SMs", dev, sm_count);
    if (partials_needed(sm_count) > kMaxPartials)
        return fail("lse_evolve_static: %d SMs need more partial sums than the fixed %d",
                    sm_count, kMaxPartials);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (stats) {
        // reading the statistics synchronises the stream, which a capture forbids
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(s, &cap);
        if (e != cudaSuccess) return cuda_fail(e, "lse_evolve_static: stream capture status");
        if (cap != cudaStreamCaptureStatusNone)
            return fail("lse_evolve_static: stats must be NULL while the stream is capturing");
    }

    unsigned char *scratch = scratch_on(dev, &e);
    if (!scratch) return cuda_fail(e, "lse_evolve_static: cudaGetSymbolAddress");
    float *phi[2] = {reinterpret_cast<float *>(scratch),
                     reinterpret_cast<float *>(scratch) + kPlane};
    LsePartial *partials = reinterpret_cast<LsePartial *>(scratch + kPartialOff);
    LseDevState *st = reinterpret_cast<LseDevState *>(scratch + kStateOff);

    // the step's kernel and work decomposition, decided before any GPU work
    const int pitch = W;
    const size_t band_stride = (size_t)H * W;
    StepPlan plan;
    if (!plan_step(H, W, B, p, pitch, band_stride, data, phi, st, partials, sm_count,
                   step_form_from_env(),
                   tile_nw_from_env() ? tile_nw_from_env()
                                      : tile_nw_default_for(H, W, p.ts, sm_count),
                   nullptr, &plan))
        return fail("lse_evolve_static: no step kernel for this shape (LSE_STEP_KERNEL "
                    "narrowed the choice, or its tensor maps could not be encoded)");

    // the ticket and the counters of the statistics record start at zero
    e = cudaMemsetAsync(st, 0, sizeof(LseDevState), s);
    if (e != cudaSuccess) return cuda_fail(e, "lse_evolve_static: clear state");
    const int nred = sm_count * 4;
    e = launch_prologue(region ? data : nullptr, pitch, band_stride, phi0,
                        region ? nullptr : g, W, phi[0], nullptr, pitch, H, W, B,
                        p.term, p.dt, LSE_F32, st, partials, nred, s);
    if (e != cudaSuccess) return cuda_fail(e, "lse_evolve_static: prologue");

    for (int n = 0; n < p.iterations; ++n) {
        if (region && B > 1) {
            e = launch_normaliser(data, pitch, band_stride, H, W, B, p.dt, st, partials,
                                  nred, s);
            if (e != cudaSuccess) return cuda_fail(e, "lse_evolve_static: normaliser");
        }
        e = launch_step(plan, n, s);
        if (e != cudaSuccess) return cuda_fail(e, "lse_evolve_static: step");
    }
    e = launch_output(phi, pitch, H, W, LSE_F32, st, phi_out, mask_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "lse_evolve_static: output");
    if (stats) {
        LseDevState h;
        e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "lse_evolve_static: read statistics");
        memset(stats, 0, sizeof(*stats));
        stats->iterations_run = h.iterations_run;
        stats->last_flips = h.last_flips;
        stats->area_plus = h.area_plus;
        for (int b = 0; b < 8; ++b) {
            stats->c_plus[b] = h.c_plus[b];
            stats->c_minus[b] = h.c_minus[b];
        }
        stats->norm = h.norm_used;
        stats->elapsed_ms = -1.0f;
        if (h.status_bits & LSE_SBIT_NONFINITE) stats->status = LSE_ERR_NONFINITE;
        else if (h.status_bits & LSE_SBIT_TIMEOUT) stats->status = LSE_ERR_TIMEOUT;
        else if (h.status_bits & LSE_SBIT_DEGENERATE) stats->status = LSE_WARN_DEGENERATE;
        else stats->status = LSE_OK;
    }
    return LSE_OK;
}
