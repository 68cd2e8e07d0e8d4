// lse_step_generic.cu -- one LSE iteration for any template size (TS <= 31)
// and any band count; shared-memory tiles, no TMA.
//
// Per 32 x 32 output tile (grid-stride over tiles):
//   1. phi on the tile + (r + 1) halo -> smem (binarised on load when the
//      previous iteration re-initialised; Table I step 3);
//   2. u = phi + dt R |grad phi| (Eq. 18) on the tile + r halo, with R the
//      region term of Eq. 17 or the edge term of Eq. 14, and u = 0 outside the
//      image (the zero padding of the 'same' convolution), or, with replicate
//      padding, u of the nearest image pixel; in the Table I order a
//      re-initialising iteration binarises u here (Table I step 3);
//   3. separable Gaussian G_sigma * u (Table I step 4): rows, then columns
//      (replicate padding is separable too: clamping rows and columns one
//      after the other reaches the same nearest pixel);
//   4. v -> phi_out, and the sums of the next iteration's statistics.
// It serves radii the TMA kernel does not instantiate, the Table I step
// order and replicate padding, and is the plain restatement the faster
// kernels are checked against.
#include "lse_reduce.cuh"

namespace {

constexpr int kTile = 32;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
step_generic_kernel(const __grid_constant__ StepArgs a)
{
    LseDevState *st = a.st;
    if (st->done || (st->status_bits & LSE_SBIT_ABORT)) return;
    extern __shared__ float smem[];
    const int R = a.rad;
    const int PN = kTile + 2 * R + 2;
    const int UN = kTile + 2 * R;
    float *P = smem;                // PN x PN: phi, origin (y0 - R - 1, x0 - R - 1)
    float *U = P + PN * PN;         // UN x UN: u,   origin (y0 - R, x0 - R)
    float *Hh = U + UN * UN;        // UN x kTile
    const int H = a.H, W = a.W, B = a.B;
    const bool region = a.term == LSE_TERM_REGION;

    float coef[LSE_MAXB], mid[LSE_MAXB];
#pragma unroll
    for (int b = 0; b < LSE_MAXB; ++b) {
        coef[b] = st->a[b];
        mid[b] = st->m[b];
    }
    LseAcc acc;
    acc.clear();
    const int tiles_x = (W + kTile - 1) / kTile;
    const int tiles_y = (H + kTile - 1) / kTile;
    for (int tile = blockIdx.x; tile < tiles_x * tiles_y; tile += gridDim.x) {
        const int y0 = (tile / tiles_x) * kTile;
        const int x0 = (tile % tiles_x) * kTile;
        for (int i = threadIdx.x; i < PN * PN; i += blockDim.x) {
            int py = i / PN, px = i - py * PN;
            int gy = y0 - R - 1 + py, gx = x0 - R - 1 + px;
            float v = 0.0f;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                v = a.phi_in[(size_t)gy * a.pitch + gx];
                if (a.binarise_in) v = v >= 0.0f ? 1.0f : -1.0f;
            }
            P[i] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < UN * UN; i += blockDim.x) {
            int uy = i / UN, ux = i - uy * UN;
            int gy = y0 - R + uy, gx = x0 - R + ux;
            float u = 0.0f;
            const bool inside = gy >= 0 && gy < H && gx >= 0 && gx < W;
            if (inside || a.pad == LSE_PAD_REPLICATE) {
                // replicate padding: u outside the image is u at the nearest
                // image pixel, which lies in this tile's window of P
                gy = min(max(gy, 0), H - 1);
                gx = min(max(gx, 0), W - 1);
                const float *c = P + (gy - (y0 - R - 1)) * PN + (gx - (x0 - R - 1));
                // twice the listing's gradient: central R - L, one-sided 2 (b - a)
                float dx, dy;
                if (W == 1) dx = 0.0f;
                else if (gx == 0) dx = 2.0f * (c[1] - c[0]);
                else if (gx == W - 1) dx = 2.0f * (c[0] - c[-1]);
                else dx = c[1] - c[-1];
                if (H == 1) dy = 0.0f;
                else if (gy == 0) dy = 2.0f * (c[PN] - c[0]);
                else if (gy == H - 1) dy = 2.0f * (c[0] - c[-PN]);
                else dy = c[PN] - c[-PN];
                float s2 = sqrtf(fmaf(dx, dx, dy * dy));   // 2 |grad phi|
                float t;                                     // 0.5 dt R
                const float *d = a.data + (size_t)gy * a.pitch + gx;
                if (region) {
                    t = 0.0f;
                    for (int b = 0; b < B; ++b)
                        t = fmaf(coef[b], d[b * a.band_stride] - mid[b], t);
                } else {
                    t = a.half_dt * d[0];
                }
                u = fmaf(t, s2, c[0]);
                // Table I order: re-initialise u itself, before the smoothing
                if (a.reinit_u) u = u >= 0.0f ? 1.0f : -1.0f;
            }
            U[i] = u;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < UN * kTile; i += blockDim.x) {
            int uy = i / kTile, tx = i - uy * kTile;
            const float *row = U + uy * UN + tx + R;
            float h = a.taps[0] * row[0];
            for (int k = 1; k <= R; ++k) h = fmaf(a.taps[k], row[-k] + row[k], h);
            Hh[i] = h;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kTile * kTile; i += blockDim.x) {
            int ty = i / kTile, tx = i - ty * kTile;
            int gy = y0 + ty, gx = x0 + tx;
            if (gy >= H || gx >= W) continue;
            const float *col = Hh + (ty + R) * kTile + tx;
            float v = a.taps[0] * col[0];
            for (int k = 1; k <= R; ++k)
                v = fmaf(a.taps[k], col[-k * kTile] + col[k * kTile], v);
            a.phi_out[(size_t)gy * a.pitch + gx] = v;
            const bool pos = v >= 0.0f;
            const bool was = P[(ty + R + 1) * PN + (tx + R + 1)] >= 0.0f;
            acc.n_plus += pos;
            acc.flips += (pos != was);
            if (region) {
                const float *d = a.data + (size_t)gy * a.pitch + gx;
                for (int b = 0; b < B; ++b) {
                    float iv = d[b * a.band_stride];
                    if (pos) acc.sp[b] += iv;
                    else acc.sm[b] += iv;
                }
            }
        }
        __syncthreads();
    }
    const int nb = region ? B : 0;
    LseAcc r;
    lse_cta_reduce(acc, nb, &r);
    if (!lse_publish_and_ticket(r, nb, a.partials, st)) return;
    LseAcc t;
    lse_sum_partials(a.partials, gridDim.x, nb, &t);
    if (threadIdx.x == 0) lse_step_finalize(a, t);
}

}  // namespace

namespace lse_detail {

cudaError_t launch_step_generic(const StepArgs &a, int nblocks, cudaStream_t s)
{
    const int R = a.rad;
    const int PN = kTile + 2 * R + 2, UN = kTile + 2 * R;
    size_t smem = sizeof(float) * ((size_t)PN * PN + (size_t)UN * UN + (size_t)UN * kTile);
    cudaError_t e = cudaFuncSetAttribute(
        step_generic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)((a.W + kTile - 1) / kTile) * ((a.H + kTile - 1) / kTile);
    int grid = (int)(tiles < nblocks ? tiles : nblocks);
    step_generic_kernel<<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lse_detail
