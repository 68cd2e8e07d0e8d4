// lse_bands.cu -- the region term for vector images (2-4 bands) around the
// one-plane tile-form step.  Each iteration runs
//   stats  c+_b and c-_b (Eq. 15): per-band sums over phi >= 0 / phi < 0 of
//          the current LSF and the count, then (last CTA) the means, alpha_b,
//          mid_b and the degenerate rule;
//   dterm  D(x) = sum_b alpha_b (I_b(x) - mid_b), the numerator of Eq. 17,
//          written as one plane, and its maximum M = max |D| (last CTA: the
//          step coefficient dt / (2 M));
//   step   the tile-form kernel on the D plane, t = dt D / (2 M) (Eq. 18),
//          as for the edge term's one plane g.
// The bands are read twice per iteration, the rest once, in passes that
// stream rows; at the sizes of the multi-band workloads the bands and both
// LSF planes stay in L2 between them.
#include "lse_reduce.cuh"

namespace {

constexpr int kThreads = 256;

// Sums of the bands over phi >= 0 and phi < 0 and the count, for CTA `cta`
// of `ncta`; rows stride over the CTAs, columns over the threads.  Each
// thread adds 4-pixel FP32 partials (error at most 3 * 2^-24 of their
// magnitude) into compensated FP32 sums, then the CTAs' sums meet in FP64.  phi is bufs[st->last_buf], the LSF the next step reads.
// final_pass: run even after an early stop (statistics of the returned LSF).
__device__ __forceinline__ void band_stats(const float *__restrict__ bands, int pitch,
                                           size_t band_stride, const float *const *bufs,
                                           int H, int W, int B, float dt, LseDevState *st,
                                           LsePartial *partials, int cta, int ncta,
                                           bool final_pass)
{
    if (st->status_bits & LSE_SBIT_ABORT) return;
    if (st->done && !final_pass) return;
    const float *phi = bufs[st->last_buf];
    constexpr int NBX = 4;                   // bands of this path, at most
    // per band and side, a compensated FP32 sum (lse_kahan_add) of 4-pixel
    // FP32 partials, kept in registers and turned into FP64 once
    float sp[NBX], cp[NBX], sm[NBX], cm[NBX];
#pragma unroll
    for (int b = 0; b < NBX; ++b) sp[b] = cp[b] = sm[b] = cm[b] = 0.0f;
    int npos = 0;
    const bool vec = (pitch & 3) == 0 && (band_stride & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(bands) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(phi) & 15) == 0;
    if (vec) {
        for (int y = cta; y < H; y += ncta)
        for (int x = 4 * threadIdx.x; x < W; x += 4 * blockDim.x) {
            const size_t o = (size_t)y * pitch + x;
            const float4 p4 = *reinterpret_cast<const float4 *>(phi + o);
            const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
            bool pos[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pos[j] = x + j < W && pv[j] >= 0.0f;
                npos += pos[j];
            }
#pragma unroll
            for (int b = 0; b < NBX; ++b) {
                if (b < B) {
                    const float4 e = __ldg(reinterpret_cast<const float4 *>(bands + b * band_stride + o));
                    const float ev[4] = {e.x, e.y, e.z, e.w};
                    float pp = 0.0f, pm = 0.0f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float v = x + j < W ? ev[j] : 0.0f;    // row padding
                        pp = __fadd_rn(pp, pos[j] ? v : 0.0f);
                        pm = __fadd_rn(pm, pos[j] ? 0.0f : v);
                    }
                    lse_kahan_add(sp[b], cp[b], pp);
                    lse_kahan_add(sm[b], cm[b], pm);
                }
            }
        }
    } else {
        for (int y = cta; y < H; y += ncta)
        for (int x = threadIdx.x; x < W; x += blockDim.x) {
            const size_t o = (size_t)y * pitch + x;
            const bool pos = phi[o] >= 0.0f;
            npos += pos;
#pragma unroll
            for (int b = 0; b < NBX; ++b) {
                if (b < B) {
                    const float v = __ldg(bands + b * band_stride + o);
                    lse_kahan_add(sp[b], cp[b], pos ? v : 0.0f);
                    lse_kahan_add(sm[b], cm[b], pos ? 0.0f : v);
                }
            }
        }
    }
    // the CTA's sums: float-float shuffles (the FP64 units of this part are
    // few, and every CTA reduces at the same moment at the end of the pass)
    float ks[2 * NBX], kc[2 * NBX];
    double tot[2 * NBX];
#pragma unroll
    for (int b = 0; b < NBX; ++b) {
        ks[b] = sp[b];
        kc[b] = cp[b];
        ks[NBX + b] = sm[b];
        kc[NBX + b] = cm[b];
    }
    LseAcc r;
    r.clear();
    lse_cta_reduce_ff<2 * NBX>(ks, kc, (long long)npos, 0ll, tot, &r.n_plus, &r.flips);
#pragma unroll
    for (int b = 0; b < NBX; ++b) {
        r.sp[b] = tot[b];
        r.sm[b] = tot[NBX + b];
    }
    if (!lse_publish_and_ticket_at(r, B, partials, st, cta, ncta)) return;
    LseAcc t;
    lse_sum_partials(partials, ncta, B, &t);
    if (threadIdx.x == 0) {
        lse_region_coeffs(st, t, B, dt);
        __threadfence();
        st->ticket = 0;
    }
}

// D = sum_b alpha_b (I_b - mid_b) into `dplane` (same pitch as the bands)
// and M = max |D|; last CTA: st->norm = M and st->a[0] = dt / (2 M), or 0
// with zero_force when the statistics were degenerate or M = 0.  D is
// written even then: the step multiplies it by 0, and it must be finite.
__device__ __forceinline__ void band_dterm(const float *__restrict__ bands, int pitch,
                                           size_t band_stride, float *__restrict__ dplane,
                                           int H, int W, int B, float dt, LseDevState *st,
                                           LsePartial *partials, int cta, int ncta)
{
    if (st->done || (st->status_bits & LSE_SBIT_ABORT)) return;
    float af[LSE_MAXB], m[LSE_MAXB];
#pragma unroll
    for (int b = 0; b < LSE_MAXB; ++b) {
        af[b] = st->af[b];
        m[b] = st->m[b];
    }
    LseAcc acc;
    acc.clear();
    const bool vec = (pitch & 3) == 0 && (band_stride & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(bands) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(dplane) & 15) == 0;
    if (vec) {
        for (int y = cta; y < H; y += ncta)
        for (int x = 4 * threadIdx.x; x < W; x += 4 * blockDim.x) {
            const size_t o = (size_t)y * pitch + x;
            float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int b = 0; b < LSE_MAXB; ++b) {
                if (b < B) {
                    const float4 e = __ldg(reinterpret_cast<const float4 *>(bands + b * band_stride + o));
                    d[0] = fmaf(af[b], e.x - m[b], d[0]);
                    d[1] = fmaf(af[b], e.y - m[b], d[1]);
                    d[2] = fmaf(af[b], e.z - m[b], d[2]);
                    d[3] = fmaf(af[b], e.w - m[b], d[3]);
                }
            }
            // columns past W are row padding: written as 0, kept out of M
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (x + j < W) {
                    acc.fmax = fmaxf(acc.fmax, d[j]);
                    acc.fmin = fminf(acc.fmin, d[j]);
                } else {
                    d[j] = 0.0f;
                }
            }
            *reinterpret_cast<float4 *>(dplane + o) = make_float4(d[0], d[1], d[2], d[3]);
        }
    } else {
        for (int y = cta; y < H; y += ncta)
        for (int x = threadIdx.x; x < W; x += blockDim.x) {
            const size_t o = (size_t)y * pitch + x;
            float d = 0.0f;
            for (int b = 0; b < B; ++b) d = fmaf(af[b], __ldg(bands + b * band_stride + o) - m[b], d);
            dplane[o] = d;
            acc.fmax = fmaxf(acc.fmax, d);
            acc.fmin = fminf(acc.fmin, d);
        }
    }
    LseAcc r;
    lse_cta_reduce(acc, 0, &r);
    if (!lse_publish_and_ticket_at(r, 0, partials, st, cta, ncta)) return;
    LseAcc t;
    lse_sum_partials(partials, ncta, 0, &t);
    if (threadIdx.x == 0) {
        const double M = fmax(fabs((double)t.fmax), fabs((double)t.fmin));
        st->norm = st->zero_force ? 0.0 : M;
        if (st->zero_force || !(M > 0.0)) {
            st->zero_force = 1;
            st->a[0] = 0.0f;
        } else {
            st->a[0] = (float)((double)dt / (2.0 * M));
        }
        __threadfence();
        st->ticket = 0;
    }
}

struct PlanePair {
    const float *b[2];
};

__global__ void __launch_bounds__(kThreads)
band_stats_kernel(const float *bands, int pitch, size_t band_stride, PlanePair bufs, int H,
                  int W, int B, float dt, LseDevState *st, LsePartial *partials, int final_pass)
{
    band_stats(bands, pitch, band_stride, bufs.b, H, W, B, dt, st, partials, blockIdx.x,
               gridDim.x, final_pass != 0);
}

__global__ void __launch_bounds__(kThreads)
band_dterm_kernel(const float *bands, int pitch, size_t band_stride, float *dplane, int H,
                  int W, int B, float dt, LseDevState *st, LsePartial *partials)
{
    band_dterm(bands, pitch, band_stride, dplane, H, W, B, dt, st, partials, blockIdx.x,
               gridDim.x);
}

// Launch index n of a batch: the passes of every vector image whose
// iteration n - iter0 is in [0, cap); the statistics only from its second
// iteration on (the prologue made the first one's).  CTA blockIdx.x works on
// image blk_item[blockIdx.x] with that image's pass CTAs.
__global__ void __launch_bounds__(kThreads)
band_stats_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ blk_item,
                        long long launch)
{
    const BatchItem &it = items[blk_item[blockIdx.x]];
    const long long nl = launch - it.iter0;
    if (nl < 1 || nl >= it.cap) return;
    const StepArgs &a = it.args;
    const float *bufs[2] = {it.phi[0], it.phi[1]};
    band_stats(a.bands, a.pitch, a.band_stride, bufs, a.H, a.W, a.B, a.dt, a.st, a.partials,
               blockIdx.x - it.nstart, it.nnblocks, false);
}

__global__ void __launch_bounds__(kThreads)
band_dterm_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ blk_item,
                        long long launch)
{
    const BatchItem &it = items[blk_item[blockIdx.x]];
    const long long nl = launch - it.iter0;
    if (nl < 0 || nl >= it.cap) return;
    const StepArgs &a = it.args;
    band_dterm(a.bands, a.pitch, a.band_stride, const_cast<float *>(a.data), a.H, a.W, a.B,
               a.dt, a.st, a.partials, blockIdx.x - it.nstart, it.nnblocks);
}

}  // namespace

namespace lse_detail {

cudaError_t launch_band_stats(const float *bands, int pitch, size_t band_stride,
                              float *const *bufs, int H, int W, int B, float dt,
                              LseDevState *st, LsePartial *partials, int nblocks,
                              bool final_pass, cudaStream_t s)
{
    PlanePair pp;
    pp.b[0] = bufs[0];
    pp.b[1] = bufs[1];
    const int grid = H < nblocks ? (H < 1 ? 1 : H) : nblocks;
    band_stats_kernel<<<grid, kThreads, 0, s>>>(bands, pitch, band_stride, pp, H, W, B, dt,
                                                st, partials, final_pass ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_band_dterm(const float *bands, int pitch, size_t band_stride, float *dplane,
                              int H, int W, int B, float dt, LseDevState *st,
                              LsePartial *partials, int nblocks, cudaStream_t s)
{
    const int grid = H < nblocks ? (H < 1 ? 1 : H) : nblocks;
    band_dterm_kernel<<<grid, kThreads, 0, s>>>(bands, pitch, band_stride, dplane, H, W, B, dt,
                                                st, partials);
    return cudaGetLastError();
}

cudaError_t launch_band_passes_batch(const BatchItem *items, const int *blk_item, long long n,
                                     int nblocks, cudaStream_t s)
{
    band_stats_batch_kernel<<<nblocks, kThreads, 0, s>>>(items, blk_item, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    band_dterm_batch_kernel<<<nblocks, kThreads, 0, s>>>(items, blk_item, n);
    return cudaGetLastError();
}

}  // namespace lse_detail
