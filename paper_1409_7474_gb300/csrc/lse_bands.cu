// lse_bands.cu -- the region term for vector images (2-4 bands) around the
// one-plane tile-form step.  Each iteration runs
//   stats  c+_b and c-_b (Eq. 15) of the LSF the last step wrote: the
//          per-band sums over phi >= 0 / phi < 0, updated from the pixels
//          that step changed in sign, and the count; then (last CTA) the
//          means, alpha_b, mid_b and the degenerate rule;
//   dterm  D(x) = sum_b alpha_b (I_b(x) - mid_b), the numerator of Eq. 17,
//          written as one plane, and its maximum M = max |D| (last CTA: the
//          step coefficient dt / (2 M));
//   step   the tile-form kernel on the D plane, t = dt D / (2 M) (Eq. 18),
//          as for the edge term's one plane g.
// The bands are read in full once per iteration (dterm); stats reads the two
// LSF planes and the band values of the changed pixels.
#include "lse_reduce.cuh"

namespace {

constexpr int kThreads = 256;

// The D pass follows the statistics pass as a programmatic dependent
// launch: the statistics CTAs allow it on entry, so its CTAs are resident
// and waiting when the statistics' last CTA finishes its one-thread
// finalisation, instead of being launched after it.  The D pass waits for
// the whole statistics grid (and its memory) before it reads anything.
__device__ __forceinline__ void allow_dependent_grid()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void wait_primary_grid()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Error-free sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
    return s;
}

// Statistics of the LSF the last step wrote (Eq. 15), for CTA `cta` of
// `ncta`; rows stride over the CTAs, columns over the threads (groups of 4).
//
// Update form (one step since the last statistics): the band sums over
// phi >= 0 and phi < 0 change only at pixels whose sign the step changed,
// so each thread sums +I_b (now >= 0) or -I_b (now < 0) over those pixels
// in float-float (TwoSum, error about 2^-44 of the sum of magnitudes) and
// the last CTA adds the total to the running FP64 sums in the state record.
// Only the two LSF planes are read in full; near convergence few pixels
// change sign.  The count |{phi >= 0}| is taken directly.
// Full form (any other case): the sums themselves, as compensated FP32
// sums of 4-pixel partials.
// No step since the last statistics: nothing to do, so the pass may run
// again after a stopped evolution without counting a change twice.
__device__ __forceinline__ void band_stats(const float *__restrict__ bands, int pitch,
                                           size_t band_stride, const float *buf0,
                                           const float *buf1, int H, int W, int B, float dt,
                                           LseDevState *st, LsePartial *partials, int cta,
                                           int ncta)
{
    if (st->status_bits & LSE_SBIT_ABORT) return;
    const int it = st->iterations_run;
    const int seen = st->stats_iter;
    if (it == seen) return;
    const bool update = it == seen + 1;
    const bool lb = st->last_buf != 0;
    const float *phi = lb ? buf1 : buf0;         // written by the last step
    const float *old = lb ? buf0 : buf1;         // read by it
    constexpr int NBX = 4;                       // bands of this path, at most
    // update form: (ks, -kc) per band is a float-float change of the sum
    // over phi >= 0; full form: Kahan pairs for phi >= 0 (b) and < 0 (4 + b)
    float ks[2 * NBX], kc[2 * NBX];
#pragma unroll
    for (int k = 0; k < 2 * NBX; ++k) ks[k] = kc[k] = 0.0f;
    int npos = 0;
    const bool vec = (pitch & 3) == 0 && (band_stride & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(bands) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(phi) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(old) & 15) == 0;
    for (int y = cta; y < H; y += ncta)
    for (int x = 4 * threadIdx.x; x < W; x += 4 * blockDim.x) {
        const size_t o = (size_t)y * pitch + x;
        const int nj = W - x < 4 ? W - x : 4;
        float pv[4], ov[4];
        if (vec && nj == 4) {
            const float4 p4 = *reinterpret_cast<const float4 *>(phi + o);
            pv[0] = p4.x; pv[1] = p4.y; pv[2] = p4.z; pv[3] = p4.w;
            if (update) {
                const float4 o4 = *reinterpret_cast<const float4 *>(old + o);
                ov[0] = o4.x; ov[1] = o4.y; ov[2] = o4.z; ov[3] = o4.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pv[j] = j < nj ? phi[o + j] : -1.0f;
                ov[j] = (update && j < nj) ? old[o + j] : -1.0f;
            }
        }
        bool pos[4], chg[4];
        bool any = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            pos[j] = j < nj && pv[j] >= 0.0f;
            npos += pos[j];
            chg[j] = update && j < nj && (ov[j] >= 0.0f) != pos[j];
            any |= chg[j];
        }
        if (update) {
            if (!any) continue;
#pragma unroll
            for (int b = 0; b < NBX; ++b) {
                if (b < B) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (!chg[j]) continue;
                        const float v = __ldg(bands + b * band_stride + o + j);
                        float e;
                        ks[b] = two_sum(ks[b], pos[j] ? v : -v, e);
                        kc[b] = __fsub_rn(kc[b], e);
                    }
                }
            }
        } else {
#pragma unroll
            for (int b = 0; b < NBX; ++b) {
                if (b < B) {
                    float ev[4];
                    if (vec && nj == 4) {
                        const float4 e = __ldg(reinterpret_cast<const float4 *>(bands + b * band_stride + o));
                        ev[0] = e.x; ev[1] = e.y; ev[2] = e.z; ev[3] = e.w;
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            ev[j] = j < nj ? __ldg(bands + b * band_stride + o + j) : 0.0f;
                    }
                    float pp = 0.0f, pm = 0.0f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float v = j < nj ? ev[j] : 0.0f;
                        pp = __fadd_rn(pp, pos[j] ? v : 0.0f);
                        pm = __fadd_rn(pm, pos[j] ? 0.0f : v);
                    }
                    lse_kahan_add(ks[b], kc[b], pp);
                    lse_kahan_add(ks[NBX + b], kc[NBX + b], pm);
                }
            }
        }
    }
    // the CTA's sums: float-float shuffles (the FP64 units of this part are
    // few, and every CTA reduces at the same moment at the end of the pass)
    double tot[2 * NBX];
    LseAcc r;
    r.clear();
    lse_cta_reduce_ff<2 * NBX>(ks, kc, (long long)npos, 0ll, tot, &r.n_plus, &r.flips);
#pragma unroll
    for (int b = 0; b < NBX; ++b) {
        r.sp[b] = tot[b];
        r.sm[b] = tot[NBX + b];
    }
    if (!lse_publish_and_ticket_at(r, NBX, partials, st, cta, ncta)) return;
    // the state fields the finalisation reads, in flight while the partials
    // are summed (one latency instead of a chain of them)
    double rsp[NBX], rsm[NBX], imin = 0.0, imax = 0.0;
    long long npix = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < NBX; ++b) {
            rsp[b] = st->run_sp[b];
            rsm[b] = st->run_sm[b];
        }
        npix = st->npix;
        imin = st->imin;
        imax = st->imax;
    }
    LseAcc t;
    // NBX bands (the partials of bands past B are zero): a constant count
    // lets the last CTA load and add every field at once
    lse_sum_partials<32, true>(partials, ncta, NBX, &t);
    if (threadIdx.x == 0) {
        if (update) {
#pragma unroll
            for (int b = 0; b < NBX; ++b) {
                if (b < B) {
                    const double d = t.sp[b];
                    t.sp[b] = rsp[b] + d;
                    t.sm[b] = rsm[b] - d;
                }
            }
        }
        lse_region_coeffs_v(st, t, B, dt, npix, imin, imax);
        st->stats_iter = it;
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
    const int zf = threadIdx.x == 0 ? st->zero_force : 0;   // in flight during the sum
    LseAcc t;
    lse_sum_partials(partials, ncta, 0, &t);
    if (threadIdx.x == 0) {
        const double M = fmax(fabs((double)t.fmax), fabs((double)t.fmin));
        st->norm = zf ? 0.0 : M;
        if (zf || !(M > 0.0)) {
            st->zero_force = 1;
            st->a[0] = 0.0f;
        } else {
            st->a[0] = (float)((double)dt / (2.0 * M));
        }
        __threadfence();
        st->ticket = 0;
    }
}

__global__ void __launch_bounds__(kThreads)
band_stats_kernel(const float *bands, int pitch, size_t band_stride, const float *buf0,
                  const float *buf1, int H, int W, int B, float dt, LseDevState *st,
                  LsePartial *partials)
{
    allow_dependent_grid();
    band_stats(bands, pitch, band_stride, buf0, buf1, H, W, B, dt, st, partials, blockIdx.x,
               gridDim.x);
}

__global__ void __launch_bounds__(kThreads)
band_dterm_kernel(const float *bands, int pitch, size_t band_stride, float *dplane, int H,
                  int W, int B, float dt, LseDevState *st, LsePartial *partials)
{
    wait_primary_grid();
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
    allow_dependent_grid();
    const BatchItem &it = items[blk_item[blockIdx.x]];
    const long long nl = launch - it.iter0;
    if (nl < 1 || nl >= it.cap) return;
    const StepArgs &a = it.args;
    band_stats(a.bands, a.pitch, a.band_stride, it.phi[0], it.phi[1], a.H, a.W, a.B, a.dt, a.st,
               a.partials, blockIdx.x - it.nstart, it.nnblocks);
}

__global__ void __launch_bounds__(kThreads)
band_dterm_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ blk_item,
                        long long launch)
{
    wait_primary_grid();
    const BatchItem &it = items[blk_item[blockIdx.x]];
    const long long nl = launch - it.iter0;
    if (nl < 0 || nl >= it.cap) return;
    const StepArgs &a = it.args;
    band_dterm(a.bands, a.pitch, a.band_stride, const_cast<float *>(a.data), a.H, a.W, a.B,
               a.dt, a.st, a.partials, blockIdx.x - it.nstart, it.nnblocks);
}

}  // namespace

namespace {

// A programmatic dependent launch (see allow_dependent_grid).
template <class Kern, class... Args>
cudaError_t launch_after_primary(Kern kern, int nblocks, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace

namespace lse_detail {

cudaError_t launch_band_stats(const float *bands, int pitch, size_t band_stride,
                              float *const *bufs, int H, int W, int B, float dt,
                              LseDevState *st, LsePartial *partials, int nblocks,
                              cudaStream_t s)
{
    const int grid = H < nblocks ? (H < 1 ? 1 : H) : nblocks;
    band_stats_kernel<<<grid, kThreads, 0, s>>>(bands, pitch, band_stride, bufs[0], bufs[1], H,
                                                W, B, dt, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_band_dterm(const float *bands, int pitch, size_t band_stride, float *dplane,
                              int H, int W, int B, float dt, LseDevState *st,
                              LsePartial *partials, int nblocks, cudaStream_t s)
{
    const int grid = H < nblocks ? (H < 1 ? 1 : H) : nblocks;
    return launch_after_primary(band_dterm_kernel, grid, s, bands, pitch, band_stride, dplane,
                                H, W, B, dt, st, partials);
}

cudaError_t launch_band_passes_batch(const BatchItem *items, const int *blk_item, long long n,
                                     int nblocks, cudaStream_t s)
{
    band_stats_batch_kernel<<<nblocks, kThreads, 0, s>>>(items, blk_item, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_after_primary(band_dterm_batch_kernel, nblocks, s, items, blk_item, n);
}

}  // namespace lse_detail
