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
#include <stddef.h>
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
    unsigned int pad;
    // status bits of strip calls that returned without waiting, kept until
    // a call that synchronises reads them (not cleared with the sums)
    unsigned int sticky;
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

// One pixel's contribution to the sums (NB bands at most, B of them used).
template <int NB>
__device__ __forceinline__ void strip_pixel(float p, float q, bool has_phi, bool has_prev,
                                            const float (&e)[NB], int B, bool has_img,
                                            int fix_k, long long (&v)[2 + 2 * NB],
                                            float (&mx)[3], unsigned int &bad)
{
    bool plus = true;
    if (has_phi) {
        bad |= !isfinite(p);
        plus = p >= 0.0f;
        v[0] += plus ? 1 : 0;
        if (has_prev) v[1] += (q >= 0.0f) != plus;
    }
    if (has_img) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b < B) {
                bad |= !isfinite(e[b]);
                if (b == 0) {
                    mx[0] = fmaxf(mx[0], e[b]);
                    mx[1] = fmaxf(mx[1], -e[b]);
                }
                mx[2] = fmaxf(mx[2], fabsf(e[b]));
                if (has_phi) {
                    const long long qv = lse_fix(e[b], fix_k);
                    v[2 + b] += plus ? qv : -qv;
                    v[2 + NB + b] += qv;
                }
            }
        }
    }
}

// Sums over rows [row0, row1): sign counts and flips of phi, and the
// fixed-point band sums with and without the sign (see lse_strip_sums).
// CTAs over rows, threads over columns; VEC: four columns a thread with
// 16-byte loads (every row and plane 16-byte aligned, W a multiple of 4),
// so that each thread has four pixels' loads in flight.  NB: the band
// count rounded up (B of them used).
template <int NB, bool VEC>
__global__ void __launch_bounds__(kThreads)
strip_partials_kernel(const float *__restrict__ img, int pitch, size_t band_stride,
                      const float *__restrict__ phi, int phi_pitch,
                      const float *__restrict__ prev, int prev_pitch, int W, int B,
                      int row0, int row1, int fix_k, StripAcc *acc)
{
    constexpr int NV = 2 + 2 * NB;
    long long v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = 0;
    float mx[3] = {-INFINITY, -INFINITY, 0.0f};      // max I_0, max -I_0, max |I_b|
    unsigned int bad = 0;
    const bool hp = phi != nullptr, hq = prev != nullptr, hi = img != nullptr;
    for (int y = row0 + blockIdx.x; y < row1; y += gridDim.x) {
        if (VEC) {
            for (int x = 4 * threadIdx.x; x < W; x += 4 * kThreads) {
                const float4 p4 = hp ? __ldg(reinterpret_cast<const float4 *>(
                                           phi + (size_t)y * phi_pitch + x))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 q4 = hq ? __ldg(reinterpret_cast<const float4 *>(
                                           prev + (size_t)y * prev_pitch + x))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                float4 e4[NB];
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    e4[b] = (hi && b < B) ? __ldg(reinterpret_cast<const float4 *>(
                                                img + b * band_stride + (size_t)y * pitch + x))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                const float pp[4] = {p4.x, p4.y, p4.z, p4.w};
                const float qq[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float e[NB];
#pragma unroll
                    for (int b = 0; b < NB; ++b)
                        e[b] = j == 0 ? e4[b].x : j == 1 ? e4[b].y : j == 2 ? e4[b].z : e4[b].w;
                    strip_pixel<NB>(pp[j], qq[j], hp, hq, e, B, hi, fix_k, v, mx, bad);
                }
            }
        } else {
            for (int x = threadIdx.x; x < W; x += kThreads) {
                const float p = hp ? __ldg(phi + (size_t)y * phi_pitch + x) : 0.0f;
                const float q = hq ? __ldg(prev + (size_t)y * prev_pitch + x) : 0.0f;
                float e[NB];
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    e[b] = (hi && b < B) ? __ldg(img + b * band_stride + (size_t)y * pitch + x)
                                         : 0.0f;
                strip_pixel<NB>(p, q, hp, hq, e, B, hi, fix_k, v, mx, bad);
            }
        }
    }
    lse_cta_sum_i64<NV, kWarps>(v);
    if (threadIdx.x == 0) {
        unsigned long long *dst = acc->v;
        if (v[0]) atomicAdd(dst + 0, (unsigned long long)v[0]);
        if (v[1]) atomicAdd(dst + 1, (unsigned long long)v[1]);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (v[2 + b]) atomicAdd(dst + 2 + b, (unsigned long long)v[2 + b]);
            if (v[2 + NB + b]) atomicAdd(dst + 2 + LSE_MAXB + b, (unsigned long long)v[2 + NB + b]);
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&acc->nonfinite, 1u);
    unsigned int *const dst[3] = {&acc->max0, &acc->neg_min, &acc->amax};
    cta_max_to<3>(mx, dst);
}

template <int NB>
cudaError_t launch_partials_nb(bool vec, int grid, cudaStream_t s, const float *img, int pitch,
                               size_t band_stride, const float *phi, const float *prev, int W,
                               int B, int row0, int row1, int fix_k, StripAcc *acc)
{
    if (vec)
        strip_partials_kernel<NB, true><<<grid, kThreads, 0, s>>>(
            img, pitch, band_stride, phi, W, prev, W, W, B, row0, row1, fix_k, acc);
    else
        strip_partials_kernel<NB, false><<<grid, kThreads, 0, s>>>(
            img, pitch, band_stride, phi, W, prev, W, W, B, row0, row1, fix_k, acc);
    return cudaGetLastError();
}

// One thread: the state record for one step of a strip (or for the D pass
// of lse_strip_dmax) from the whole image's totals -- c+/c-, alpha, mid and,
// for one band, M and the step coefficient (Eqs. 15 and 17, the arithmetic
// of the whole-image path); for several bands M = norm when use_norm.
__global__ void strip_coeffs_kernel(LseDevState *st, StripTotals t, const lse_strip_sums *dev,
                                    int B, int region, float dt, double norm, int use_norm,
                                    unsigned int *sticky, int fold)
{
    if (fold && (st->status_bits & LSE_SBIT_ABORT))
        atomicOr(sticky, st->status_bits & LSE_SBIT_ABORT);
    if (dev) {
        // the ranks' totals in device memory (summed there by the caller)
        t.npix = dev->npix;
        t.n_plus = dev->n_plus;
        for (int b = 0; b < LSE_MAXB; ++b) {
            t.sum_w[b] = b < B ? dev->sum_w[b] : 0;
            t.sum_a[b] = b < B ? dev->sum_a[b] : 0;
        }
        t.imin = dev->imin;
        t.imax = dev->imax;
        t.fix_k = dev->fix_k;
    }
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

// One thread: the pass's sums as an lse_strip_sums in device memory.
__global__ void strip_export_kernel(StripAcc *acc, lse_strip_sums *out, long long npix,
                                    int fix_k, int B, int any)
{
    out->npix = npix;
    out->n_plus = (long long)acc->v[0];
    out->flips = (long long)acc->v[1];
    for (int b = 0; b < 8; ++b) {
        out->sum_w[b] = b < B ? (long long)acc->v[2 + b] : 0;
        out->sum_a[b] = b < B ? (long long)acc->v[2 + LSE_MAXB + b] : 0;
    }
    out->imin = any ? -(double)ord_value(acc->neg_min) : INFINITY;
    out->imax = any ? (double)ord_value(acc->max0) : -INFINITY;
    out->amax = any ? (double)ord_value(acc->amax) : 0.0;
    out->fix_k = fix_k;
    out->bands = B;
    if (acc->nonfinite) atomicOr(&acc->sticky, LSE_SBIT_NONFINITE);
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
    for (int y = row0 + blockIdx.x; y < row1; y += gridDim.x)
    for (int x = threadIdx.x; x < W; x += kThreads) {
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

// The accumulator, allocated (and cleared, sticky word included) on first use.
lse_status acc_alloc(lse_ctx *ctx, cudaStream_t s)
{
    if (ctx->strip_acc) return LSE_OK;
    lse_status r = ensure(ctx, &ctx->strip_acc, &ctx->strip_acc_cap, sizeof(StripAcc), s,
                          "strip sums");
    if (r != LSE_OK) return r;
    cudaError_t e = cudaMemsetAsync(ctx->strip_acc, 0, sizeof(StripAcc), s);
    return e == cudaSuccess ? LSE_OK : cuda_fail(ctx, e, "clear strip sums");
}

// The accumulator with its sums cleared for a pass (the sticky word kept).
lse_status ensure_acc(lse_ctx *ctx, cudaStream_t s)
{
    lse_status r = acc_alloc(ctx, s);
    if (r != LSE_OK) return r;
    cudaError_t e = cudaMemsetAsync(ctx->strip_acc, 0, offsetof(StripAcc, sticky), s);
    return e == cudaSuccess ? LSE_OK : cuda_fail(ctx, e, "clear strip sums");
}

// Enqueues the reads of the device-side status of strip calls that did not
// wait (the sticky word, and the last step's bits if nothing read them
// yet) into *bits and clears the sticky word; the caller synchronises.
cudaError_t read_strip_status(lse_ctx *ctx, unsigned int *bits, unsigned int *step_bits,
                              cudaStream_t s)
{
    *bits = 0;
    *step_bits = 0;
    if (!ctx->strip_acc) return cudaSuccess;
    StripAcc *acc = static_cast<StripAcc *>(ctx->strip_acc);
    cudaError_t e = cudaMemcpyAsync(bits, &acc->sticky, sizeof(*bits), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&acc->sticky, 0, sizeof(acc->sticky), s);
    if (e == cudaSuccess && ctx->strip_unchecked)
        e = cudaMemcpyAsync(step_bits, &ctx->st->status_bits, sizeof(*step_bits),
                            cudaMemcpyDeviceToHost, s);
    return e;
}

lse_status strip_status_of(lse_ctx *ctx, unsigned int bits)
{
    if (bits & LSE_SBIT_TIMEOUT) {
        set_err(ctx, "a bounded device wait of a strip step ran out");
        return LSE_ERR_TIMEOUT;
    }
    if (bits & LSE_SBIT_NONFINITE) {
        set_err(ctx, "a strip call met NaN or Inf");
        return LSE_ERR_NONFINITE;
    }
    return LSE_OK;
}

// CTAs of a pass over `rows` rows: one per row, at most 8 per SM.
int pass_blocks(const lse_ctx *ctx, int rows, int W)
{
    (void)W;
    const int cap = ctx->sm_count * 8;
    return rows < 1 ? 1 : (rows < cap ? rows : cap);
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
                  kq = classify(phi_prev, ctx->device), ko = classify(out, ctx->device);
    if (ki == PTR_BAD || kp == PTR_BAD || kq == PTR_BAD || ko == PTR_BAD) {
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
        const int nb = img ? B : 0;
        const bool vec = (W % 4) == 0 && (pitch % 4) == 0 && (band_stride % 4) == 0 &&
                         (!img || aligned16(img)) && (!dphi || aligned16(dphi)) &&
                         (!dprev || aligned16(dprev));
        const int grid = pass_blocks(ctx, row1 - row0, W);
        cudaError_t e;
        if (nb <= 1)
            e = launch_partials_nb<1>(vec, grid, s, img, pitch, band_stride, dphi, dprev, W, nb,
                                      row0, row1, fix_k, acc);
        else if (nb <= 2)
            e = launch_partials_nb<2>(vec, grid, s, img, pitch, band_stride, dphi, dprev, W, nb,
                                      row0, row1, fix_k, acc);
        else if (nb <= 4)
            e = launch_partials_nb<4>(vec, grid, s, img, pitch, band_stride, dphi, dprev, W, nb,
                                      row0, row1, fix_k, acc);
        else
            e = launch_partials_nb<8>(vec, grid, s, img, pitch, band_stride, dphi, dprev, W, nb,
                                      row0, row1, fix_k, acc);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "strip partials");
        ++ctx->launches;
    }
    const bool any = img && row1 > row0;
    if (ko == PTR_DEVICE) {
        // the sums into the caller's device record; no wait
        strip_export_kernel<<<1, 1, 0, s>>>(acc, out, (long long)(row1 - row0) * W, fix_k, B,
                                            any ? 1 : 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "strip sums export");
        ++ctx->launches;
        return LSE_OK;
    }
    StripAcc h;
    unsigned int bits = 0, step_bits = 0;
    cudaError_t e = cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = read_strip_status(ctx, &bits, &step_bits, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read strip partials");
    ctx->strip_unchecked = false;
    if ((r = strip_status_of(ctx, bits | step_bits)) != LSE_OK) return r;
    memset(out, 0, sizeof(*out));
    out->npix = (long long)(row1 - row0) * W;
    out->n_plus = (long long)h.v[0];
    out->flips = (long long)h.v[1];
    for (int b = 0; b < B && b < LSE_MAXB; ++b) {
        out->sum_w[b] = (long long)h.v[2 + b];
        out->sum_a[b] = (long long)h.v[2 + LSE_MAXB + b];
    }
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
    if (r != LSE_OK) return r;
    {
        DeviceGuard g0(ctx->device);
        if (classify(totals, ctx->device) != PTR_HOST) {
            set_err(ctx, "lse_strip_dmax takes the totals in host memory");
            return LSE_ERR_INVALID_ARG;
        }
    }
    if ((r = check_totals(ctx, totals, B)) != LSE_OK) return r;
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
    strip_coeffs_kernel<<<1, 1, 0, s>>>(ctx->st, to_totals(*totals, B), nullptr, B, 1, dt, 0.0,
                                        0, &acc->sticky, ctx->strip_unchecked ? 1 : 0);
    ctx->strip_unchecked = false;
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
    if (v_out == phi || (const void *)v_out == image || v_out == g) {
        set_err(ctx, "v_out must not share memory with phi, the image or g");
        return LSE_ERR_INVALID_ARG;
    }
    // totals in device memory are the caller's (summed there); host ones
    // are checked here
    const PtrKind kt = region ? classify(totals, ctx->device) : PTR_NULL;
    if (kt == PTR_BAD) {
        set_err(ctx, "the totals belong to another GPU than the context's");
        return LSE_ERR_INVALID_ARG;
    }
    if (region && kt != PTR_DEVICE && (r = check_totals(ctx, totals, B)) != LSE_OK) return r;
    if (region && !totals) {
        set_err(ctx, "the region term needs the ranks' totals");
        return LSE_ERR_INVALID_ARG;
    }
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
    if (region && kt != PTR_DEVICE) {
        t = to_totals(*totals, B);
    } else if (!region) {
        t.npix = (long long)Hs * W;
        t.fix_k = 30;
    }
    if ((r = acc_alloc(ctx, s)) != LSE_OK) return r;
    strip_coeffs_kernel<<<1, 1, 0, s>>>(
        ctx->st, t, kt == PTR_DEVICE ? totals : nullptr, region ? B : 1, region ? 1 : 0, p.dt,
        norm, 1, &static_cast<StripAcc *>(ctx->strip_acc)->sticky, ctx->strip_unchecked ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "strip coefficients");
    ctx->strip_unchecked = false;
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
        // no wait: the next call on this context that synchronises
        // (lse_strip_partials into host memory, lse_strip_status) reports
        // what the device found
        ctx->strip_unchecked = true;
        return LSE_OK;
    }
    ctx->strip_unchecked = true;
    unsigned int bits = 0, step_bits = 0;
    e = read_strip_status(ctx, &bits, &step_bits, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
    ctx->strip_unchecked = false;
    return strip_status_of(ctx, bits | step_bits);
}

lse_status lse_strip_status(lse_ctx *ctx, void *stream)
{
    if (!ctx) return LSE_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return cuda_fail(ctx, cudaErrorInvalidDevice, "set device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned int bits = 0, step_bits = 0;
    cudaError_t e = read_strip_status(ctx, &bits, &step_bits, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
    ctx->strip_unchecked = false;
    return strip_status_of(ctx, bits | step_bits);
}

}  // extern "C"
