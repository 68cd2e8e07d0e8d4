// lse_strip.cu -- row strips of one image on several GPUs: the C-ABI entry
// points lse_strip_scale, lse_strip_partials, lse_strip_dmax and
// lse_strip_step, and their kernels.
//
// The statistics of the region term are global: c+ and c- (Eq. 15) are
// means over the whole image and the normaliser of Eq. 17 a maximum over it.
// A rank therefore contributes partial sums over the rows it owns, the
// caller adds them over the ranks, and every rank steps its strip (owned
// rows plus r + 1 halo rows a side) with the same totals.  The sums are
// exact integers: each band value is rounded once to a multiple of 2^-k
// (lse_fix), so the totals, and every result after them, do not depend on
// how the image is split.
#include <math.h>
#include <string.h>

#include "lse_ctx.h"
#include "lse_reduce.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kNv = 2 + 2 * LSE_MAXB;      // n_plus, flips, sum_w[8], sum_a[8]

// Device accumulator of one call: integer totals and float extremes as
// order-preserving bits (larger unsigned value = larger float).
struct StripAcc {
    unsigned long long v[kNv];
    unsigned int neg_min;       // ordered bits of -min(I_0)
    unsigned int max0;          // ordered bits of max(I_0)
    unsigned int amax;          // ordered bits of max |I_b|
    unsigned int nonfinite;
    unsigned int dmax, dmin;    // ordered bits of max D and of -min D (lse_strip_dmax)
    unsigned int pad[2];
};

// The whole image's totals as the coefficient kernel takes them.
struct StripTotals {
    long long npix, n_plus;
    long long sum_w[LSE_MAXB], sum_a[LSE_MAXB];
    double imin, imax;
    int fix_k;
};

__device__ __forceinline__ unsigned int ord_bits(float v)
{
    const unsigned int u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ inline float ord_value(unsigned int o)
{
    const unsigned int u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

__device__ __forceinline__ float warp_max_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The CTA's largest value of each of N floats into the accumulator word
// `dst[i]` (ordered bits), by warp shuffles, shared memory and one atomic.
template <int N>
__device__ __forceinline__ void cta_max_to(float (&v)[N], unsigned int *const (&dst)[N])
{
    __shared__ float s[kWarps][N];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        v[i] = warp_max_f(v[i]);
        if (lane == 0) s[warp][i] = v[i];
    }
    __syncthreads();
    if (threadIdx.x < N) {
        float m = -INFINITY;
        for (int w = 0; w < kWarps; ++w) m = fmaxf(m, s[w][threadIdx.x]);
        atomicMax(dst[threadIdx.x], ord_bits(m));
    }
}

// Sums over rows [row0, row1): sign counts and flips of phi, and the
// fixed-point band sums with and without the sign (see lse_strip_sums).
// Grid-stride over the owned pixels.
__global__ void __launch_bounds__(kThreads)
strip_partials_kernel(const float *__restrict__ img, int pitch, size_t band_stride,
                      const float *__restrict__ phi, int phi_pitch,
                      const float *__restrict__ prev, int prev_pitch, int W, int B,
                      int row0, int row1, int fix_k, StripAcc *acc)
{
    long long v[kNv];
#pragma unroll
    for (int i = 0; i < kNv; ++i) v[i] = 0;
    float mx[3] = {-INFINITY, -INFINITY, 0.0f};      // max I_0, max -I_0, max |I_b|
    unsigned int bad = 0;
    const long long n = (long long)(row1 - row0) * W;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kThreads) {
        const int y = row0 + (int)(i / W), x = (int)(i % W);
        bool plus = true;
        if (phi) {
            const float p = __ldg(phi + (size_t)y * phi_pitch + x);
            bad |= !isfinite(p);
            plus = p >= 0.0f;
            v[0] += plus ? 1 : 0;
            if (prev) v[1] += (__ldg(prev + (size_t)y * prev_pitch + x) >= 0.0f) != plus;
        }
        if (img) {
#pragma unroll
            for (int b = 0; b < LSE_MAXB; ++b) {
                if (b < B) {
                    const float e = __ldg(img + b * band_stride + (size_t)y * pitch + x);
                    bad |= !isfinite(e);
                    if (b == 0) {
                        mx[0] = fmaxf(mx[0], e);
                        mx[1] = fmaxf(mx[1], -e);
                    }
                    mx[2] = fmaxf(mx[2], fabsf(e));
                    if (phi) {
                        const long long q = lse_fix(e, fix_k);
                        v[2 + b] += plus ? q : -q;
                        v[2 + LSE_MAXB + b] += q;
                    }
                }
            }
        }
    }
    lse_cta_sum_i64<kNv, kWarps>(v);
    if (threadIdx.x == 0) {
        unsigned long long *dst = acc->v;
#pragma unroll
        for (int i = 0; i < kNv; ++i)
            if (v[i]) atomicAdd(dst + i, (unsigned long long)v[i]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&acc->nonfinite, 1u);
    unsigned int *const dst[3] = {&acc->max0, &acc->neg_min, &acc->amax};
    cta_max_to<3>(mx, dst);
}

// One thread: the state record for one step of a strip (or for the D pass
// of lse_strip_dmax) from the whole image's totals -- c+/c-, alpha, mid and,
// for one band, M and the step coefficient (Eqs. 15 and 17, the arithmetic
// of the whole-image path); for several bands M = norm when use_norm.
__global__ void strip_coeffs_kernel(LseDevState *st, StripTotals t, int B, int region,
                                    float dt, double norm, int use_norm)
{
    st->npix = t.npix;
    st->imin = t.imin;
    st->imax = t.imax;
    st->status_bits = 0;
    st->done = 0;
    st->ticket = 0;
    st->grid_bar = 0;
    st->last_flips = 0;
    st->iterations_run = 0;
    st->stats_iter = 0;
    st->last_buf = 0;
    st->norm_used = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 12; ++j) st->acc[i][j] = 0;
    st->tile_ctr[0] = st->tile_ctr[1] = 0;
    st->fix_k = t.fix_k;
    if (!region) {
        st->zero_force = 0;
        st->norm = 0.0;
        for (int b = 0; b < LSE_MAXB; ++b) st->a[b] = 0.0f;
        return;
    }
    LseAcc a;
    a.clear();
    for (int b = 0; b < B; ++b) {
        a.sp[b] = ldexp((double)(t.sum_a[b] + t.sum_w[b]), -(t.fix_k + 1));
        a.sm[b] = ldexp((double)(t.sum_a[b] - t.sum_w[b]), -(t.fix_k + 1));
    }
    a.n_plus = t.n_plus;
    lse_region_coeffs_v(st, a, B, dt, t.npix, t.imin, t.imax);
    if (B > 1 && use_norm && !st->zero_force) {
        if (norm > 0.0) {
            st->norm = norm;
            for (int b = 0; b < LSE_MAXB; ++b)
                st->a[b] = b < B ? (float)((double)dt * st->alpha[b] / (2.0 * norm)) : 0.0f;
        } else {
            st->zero_force = 1;
            for (int b = 0; b < LSE_MAXB; ++b) st->a[b] = 0.0f;
        }
    }
}

// Largest and smallest D = sum_b alpha_b (I_b - mid_b) over rows [row0, row1),
// in FP32 with the normaliser pass's arithmetic (nothing when the totals
// made the force zero).
__global__ void __launch_bounds__(kThreads)
strip_dmax_kernel(const float *__restrict__ img, int pitch, size_t band_stride, int W, int B,
                  int row0, int row1, const LseDevState *st, StripAcc *acc)
{
    if (st->zero_force) return;
    float af[LSE_MAXB], m[LSE_MAXB];
#pragma unroll
    for (int b = 0; b < LSE_MAXB; ++b) {
        af[b] = st->af[b];
        m[b] = st->m[b];
    }
    float mx[2] = {-INFINITY, -INFINITY};              // max D, max -D
    const long long n = (long long)(row1 - row0) * W;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kThreads) {
        const int y = row0 + (int)(i / W), x = (int)(i % W);
        const float *src = img + (size_t)y * pitch + x;
        float d = 0.0f;
#pragma unroll
        for (int b = 0; b < LSE_MAXB; ++b)
            if (b < B) d = fmaf(af[b], __ldg(src + b * band_stride) - m[b], d);
        mx[0] = fmaxf(mx[0], d);
        mx[1] = fmaxf(mx[1], -d);
    }
    unsigned int *const dst[2] = {&acc->dmax, &acc->dmin};
    cta_max_to<2>(mx, dst);
}

}  // namespace

using namespace lse_detail;

namespace {

lse_status check_rows(lse_ctx *ctx, int Hs, int W, int B, int row0, int row1)
{
    if (Hs < 1 || W < 1 || B < 1 || B > ctx->max_bands) {
        set_err(ctx, "need Hs, W >= 1 and 1 <= B <= %d (got %d x %d, B = %d)", ctx->max_bands,
                Hs, W, B);
        return LSE_ERR_INVALID_ARG;
    }
    if ((size_t)Hs * (size_t)W > ctx->max_pixels) {
        set_err(ctx, "Hs*W = %zu exceeds the context's max_pixels %zu", (size_t)Hs * W,
                ctx->max_pixels);
        return LSE_ERR_INVALID_ARG;
    }
    if (row0 < 0 || row1 < row0 || row1 > Hs) {
        set_err(ctx, "owned rows [%d, %d) outside the strip's %d rows", row0, row1, Hs);
        return LSE_ERR_INVALID_ARG;
    }
    return LSE_OK;
}

StripTotals to_totals(const lse_strip_sums &s, int B)
{
    StripTotals t;
    memset(&t, 0, sizeof(t));
    t.npix = s.npix;
    t.n_plus = s.n_plus;
    for (int b = 0; b < B && b < LSE_MAXB; ++b) {
        t.sum_w[b] = s.sum_w[b];
        t.sum_a[b] = s.sum_a[b];
    }
    t.imin = s.imin;
    t.imax = s.imax;
    t.fix_k = s.fix_k;
    return t;
}

lse_status check_totals(lse_ctx *ctx, const lse_strip_sums *t, int B)
{
    if (!t) {
        set_err(ctx, "the region term needs the ranks' totals");
        return LSE_ERR_INVALID_ARG;
    }
    if (t->npix < 1 || t->n_plus < 0 || t->n_plus > t->npix || t->fix_k < -120 ||
        t->fix_k > 120 || t->bands != B || !(t->imin <= t->imax)) {
        set_err(ctx, "totals inconsistent (npix %lld, n_plus %lld, fix_k %d, bands %d for "
                     "B = %d, range [%g, %g])",
                t->npix, t->n_plus, t->fix_k, t->bands, B, t->imin, t->imax);
        return LSE_ERR_INVALID_ARG;
    }
    return LSE_OK;
}

// A contiguous Hs x W float32 plane on the device: in place when it already
// is device memory, else copied into `stage`.
lse_status device_plane(lse_ctx *ctx, const float *src, PtrKind kind, int Hs, int W,
                        float *stage, cudaStream_t s, const float **out)
{
    if (kind == PTR_DEVICE) {
        *out = src;
        return LSE_OK;
    }
    cudaError_t e = cudaMemcpyAsync(stage, src, (size_t)Hs * W * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy LSF to device");
    *out = stage;
    return LSE_OK;
}

lse_status ensure_acc(lse_ctx *ctx, cudaStream_t s)
{
    lse_status r = ensure(ctx, &ctx->strip_acc, &ctx->strip_acc_cap, sizeof(StripAcc), s,
                          "strip sums");
    if (r != LSE_OK) return r;
    cudaError_t e = cudaMemsetAsync(ctx->strip_acc, 0, sizeof(StripAcc), s);
    return e == cudaSuccess ? LSE_OK : cuda_fail(ctx, e, "clear strip sums");
}

int pass_blocks(const lse_ctx *ctx, int rows, int W)
{
    const long long want = ((long long)rows * W + kThreads - 1) / kThreads;
    const long long cap = (long long)ctx->sm_count * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

extern "C" {

int lse_strip_scale(double amax, long long npix)
{
    return lse_fix_scale(amax, npix);
}

lse_status lse_strip_partials(lse_ctx *ctx, const void *image, lse_dtype dtype, int Hs, int W,
                              int B, int row0, int row1, const float *phi,
                              const float *phi_prev, int fix_k, lse_strip_sums *out,
                              void *stream)
{
    if (!ctx) return LSE_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!out) {
        set_err(ctx, "out must not be NULL");
        return LSE_ERR_INVALID_ARG;
    }
    lse_status r = check_rows(ctx, Hs, W, B, row0, row1);
    if (r != LSE_OK) return r;
    if (image && (r = check_image_args(ctx, dtype, Hs, W, B)) != LSE_OK) return r;
    if (phi && (fix_k < -120 || fix_k > 120)) {
        set_err(ctx, "fix_k %d outside -120..120", fix_k);
        return LSE_ERR_INVALID_ARG;
    }
    if (phi_prev && !phi) {
        set_err(ctx, "phi_prev needs phi");
        return LSE_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return cuda_fail(ctx, cudaErrorInvalidDevice, "set device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const PtrKind ki = classify(image, ctx->device), kp = classify(phi, ctx->device),
                  kq = classify(phi_prev, ctx->device);
    if (ki == PTR_BAD || kp == PTR_BAD || kq == PTR_BAD) {
        set_err(ctx, "a device pointer belongs to another GPU than the context's");
        return LSE_ERR_INVALID_ARG;
    }
    const float *img = nullptr;
    int pitch = W;
    size_t band_stride = 0;
    if (image && (r = stage_image(ctx, image, ki, dtype, Hs, W, B, s, &img, &pitch,
                                  &band_stride)) != LSE_OK)
        return r;
    const float *dphi = nullptr, *dprev = nullptr;
    if (phi || phi_prev) {
        if ((r = ensure_phi(ctx, (size_t)Hs * W, s)) != LSE_OK) return r;
        if (phi && (r = device_plane(ctx, phi, kp, Hs, W, ctx->phi[0], s, &dphi)) != LSE_OK)
            return r;
        if (phi_prev &&
            (r = device_plane(ctx, phi_prev, kq, Hs, W, ctx->phi[1], s, &dprev)) != LSE_OK)
            return r;
    }
    if ((r = ensure_acc(ctx, s)) != LSE_OK) return r;
    StripAcc *acc = static_cast<StripAcc *>(ctx->strip_acc);
    if (row1 > row0 && (img || dphi)) {
        strip_partials_kernel<<<pass_blocks(ctx, row1 - row0, W), kThreads, 0, s>>>(
            img, pitch, band_stride, dphi, W, dprev, W, W, img ? B : 0, row0, row1, fix_k, acc);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "strip partials");
        ++ctx->launches;
    }
    StripAcc h;
    unsigned int step_bits = 0;
    const bool check_step = ctx->strip_unchecked;
    cudaError_t e = cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && check_step)
        e = cudaMemcpyAsync(&step_bits, &ctx->st->status_bits, sizeof(step_bits),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read strip partials");
    ctx->strip_unchecked = false;
    if (step_bits & LSE_SBIT_TIMEOUT) {
        set_err(ctx, "a bounded device wait of the last strip step ran out");
        return LSE_ERR_TIMEOUT;
    }
    if (step_bits & LSE_SBIT_NONFINITE) {
        set_err(ctx, "the last strip step met NaN or Inf");
        return LSE_ERR_NONFINITE;
    }
    memset(out, 0, sizeof(*out));
    out->npix = (long long)(row1 - row0) * W;
    out->n_plus = (long long)h.v[0];
    out->flips = (long long)h.v[1];
    for (int b = 0; b < B && b < LSE_MAXB; ++b) {
        out->sum_w[b] = (long long)h.v[2 + b];
        out->sum_a[b] = (long long)h.v[2 + LSE_MAXB + b];
    }
    const bool any = img && row1 > row0;
    out->imin = any ? -(double)ord_value(h.neg_min) : INFINITY;
    out->imax = any ? (double)ord_value(h.max0) : -INFINITY;
    out->amax = any ? (double)ord_value(h.amax) : 0.0;
    out->fix_k = fix_k;
    out->bands = B;
    if (h.nonfinite) {
        set_err(ctx, "NaN or Inf in the image or the LSF of the owned rows");
        return LSE_ERR_NONFINITE;
    }
    return LSE_OK;
}

lse_status lse_strip_dmax(lse_ctx *ctx, const void *image, lse_dtype dtype, int Hs, int W,
                          int B, int row0, int row1, const lse_strip_sums *totals, float dt,
                          double *dmax, void *stream)
{
    if (!ctx) return LSE_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!image || !dmax) {
        set_err(ctx, "image and dmax must not be NULL");
        return LSE_ERR_INVALID_ARG;
    }
    lse_status r = check_rows(ctx, Hs, W, B, row0, row1);
    if (r == LSE_OK) r = check_image_args(ctx, dtype, Hs, W, B);
    if (r == LSE_OK) r = check_totals(ctx, totals, B);
    if (r != LSE_OK) return r;
    if (!(dt > 0.0f) || !isfinite(dt)) {
        set_err(ctx, "need a finite dt > 0 (got %g)", dt);
        return LSE_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return cuda_fail(ctx, cudaErrorInvalidDevice, "set device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const PtrKind ki = classify(image, ctx->device);
    if (ki == PTR_BAD) {
        set_err(ctx, "a device pointer belongs to another GPU than the context's");
        return LSE_ERR_INVALID_ARG;
    }
    const float *img;
    int pitch;
    size_t band_stride;
    if ((r = stage_image(ctx, image, ki, dtype, Hs, W, B, s, &img, &pitch, &band_stride)) != LSE_OK)
        return r;
    if ((r = ensure_acc(ctx, s)) != LSE_OK) return r;
    StripAcc *acc = static_cast<StripAcc *>(ctx->strip_acc);
    strip_coeffs_kernel<<<1, 1, 0, s>>>(ctx->st, to_totals(*totals, B), B, 1, dt, 0.0, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "strip coefficients");
    ++ctx->launches;
    if (row1 > row0) {
        strip_dmax_kernel<<<pass_blocks(ctx, row1 - row0, W), kThreads, 0, s>>>(
            img, pitch, band_stride, W, B, row0, row1, ctx->st, acc);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "strip D pass");
        ++ctx->launches;
    }
    StripAcc h;
    e = cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read strip D pass");
    // no contribution (zero force, or no owned rows): 0
    const double hi = h.dmax ? (double)ord_value(h.dmax) : 0.0;
    const double lo = h.dmin ? (double)ord_value(h.dmin) : 0.0;
    *dmax = fmax(fabs(hi), fabs(lo));
    return LSE_OK;
}

lse_status lse_strip_step(lse_ctx *ctx, const void *image, lse_dtype dtype, const float *g,
                          int Hs, int W, int B, const float *phi, int binarise_in,
                          const lse_params *params, const lse_strip_sums *totals, double norm,
                          float *v_out, void *stream)
{
    if (!ctx) return LSE_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!params || !phi || !v_out) {
        set_err(ctx, "params, phi and v_out must not be NULL");
        return LSE_ERR_INVALID_ARG;
    }
    lse_params p = *params;
    p.iterations = 1;
    p.reinit_period = 1;       // the caller's schedule; binarise_in carries it
    p.early_stop_frac = 0.0f;
    const bool region = p.term == LSE_TERM_REGION;
    lse_status r = check_rows(ctx, Hs, W, region ? B : 1, 0, Hs);
    if (r == LSE_OK && region) r = check_image_args(ctx, dtype, Hs, W, B);
    if (r == LSE_OK) r = check_params(ctx, p, region ? B : 1);
    if (r != LSE_OK) return r;
    if (p.storage != LSE_F32 || p.order != LSE_ORDER_LISTING || p.padding != LSE_PAD_ZERO) {
        set_err(ctx, "strips run with F32 storage, the listing's order and zero padding");
        return LSE_ERR_INVALID_ARG;
    }
    if ((region && (!image || g)) || (!region && !g)) {
        set_err(ctx, "need image (region term, g NULL) or g (edge term)");
        return LSE_ERR_INVALID_ARG;
    }
    if (region && (r = check_totals(ctx, totals, B)) != LSE_OK) return r;
    if (region && B > 1 && !(norm >= 0.0 && isfinite(norm))) {
        set_err(ctx, "norm must be finite and >= 0 (got %g)", norm);
        return LSE_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return cuda_fail(ctx, cudaErrorInvalidDevice, "set device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const PtrKind ki = classify(image, ctx->device), kg = classify(g, ctx->device),
                  kp = classify(phi, ctx->device), ko = classify(v_out, ctx->device);
    if (ki == PTR_BAD || kg == PTR_BAD || kp == PTR_BAD || ko == PTR_BAD) {
        set_err(ctx, "a device pointer belongs to another GPU than the context's");
        return LSE_ERR_INVALID_ARG;
    }
    cudaError_t e;
    // device buffers already in the kernels' layout (W a multiple of 4,
    // 16-byte aligned) are read and written in place: no staging copies
    const bool in_place =
        kp == PTR_DEVICE && ko == PTR_DEVICE && (W % 4) == 0 && aligned16(phi) &&
        aligned16(v_out) && phi != v_out &&
        (region ? ki == PTR_DEVICE && dtype == LSE_F32 && aligned16(image)
                : kg == PTR_DEVICE && aligned16(g));
    // the data plane, pitched like the LSF buffers
    const float *data;
    int pitch;
    size_t band_stride;
    if (in_place) {
        data = region ? static_cast<const float *>(image) : g;
        pitch = W;
        band_stride = (size_t)Hs * W;
    } else if (region) {
        if ((r = stage_image(ctx, image, ki, dtype, Hs, W, B, s, &data, &pitch,
                             &band_stride)) != LSE_OK)
            return r;
    } else {
        pitch = round_up(W, 32);
        if ((r = ensure_t(ctx, &ctx->gbuf, &ctx->g_cap, (size_t)Hs * pitch, s, "g")) != LSE_OK)
            return r;
        e = cudaMemcpy2DAsync(ctx->gbuf, (size_t)pitch * 4, g, (size_t)W * 4, (size_t)W * 4, Hs,
                              cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "stage g");
        data = ctx->gbuf;
        band_stride = (size_t)Hs * pitch;
    }
    float *bufs[2] = {const_cast<float *>(phi), v_out};
    if (!in_place) {
        if ((r = ensure_phi(ctx, (size_t)Hs * pitch, s)) != LSE_OK) return r;
        e = cudaMemcpy2DAsync(ctx->phi[0], (size_t)pitch * 4, phi, (size_t)W * 4, (size_t)W * 4,
                              Hs, cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "stage phi");
        bufs[0] = ctx->phi[0];
        bufs[1] = ctx->phi[1];
    }
    StripTotals t;
    memset(&t, 0, sizeof(t));
    if (region) {
        t = to_totals(*totals, B);
    } else {
        t.npix = (long long)Hs * W;
        t.fix_k = 30;
    }
    strip_coeffs_kernel<<<1, 1, 0, s>>>(ctx->st, t, region ? B : 1, region ? 1 : 0, p.dt, norm,
                                        1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "strip coefficients");
    ++ctx->launches;
    StepPlan plan;
    if (!plan_step(Hs, W, region ? B : 1, p, pitch, band_stride, data, bufs, ctx->st,
                   ctx->partials, ctx->sm_count, ctx->step_form,
                   tile_nw_for(ctx, Hs, W, region ? B : 1, p.term, LSE_F32, p.ts), nullptr,
                   &plan)) {
        set_err(ctx, "no step kernel serves this strip");
        return LSE_ERR_INVALID_ARG;
    }
    if ((e = launch_step_once(plan, binarise_in != 0, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "strip step");
    ++ctx->launches;
    if (!in_place) {
        e = cudaMemcpy2DAsync(v_out, (size_t)W * 4, ctx->phi[1], (size_t)pitch * 4,
                              (size_t)W * 4, Hs, cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy v");
    }
    if (ko != PTR_HOST) {
        // no wait: the next lse_strip_partials on this context, which
        // synchronises, reports what the device found
        ctx->strip_unchecked = true;
        return LSE_OK;
    }
    ctx->strip_unchecked = false;
    e = cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(LseDevState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
    const unsigned int bits = ctx->st_host->status_bits;
    if (bits & LSE_SBIT_TIMEOUT) {
        set_err(ctx, "a bounded device wait of the step ran out");
        return LSE_ERR_TIMEOUT;
    }
    if (bits & LSE_SBIT_NONFINITE) {
        set_err(ctx, "the step met NaN or Inf");
        return LSE_ERR_NONFINITE;
    }
    return LSE_OK;
}

}  // extern "C"
