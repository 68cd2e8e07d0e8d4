// lse_prologue.cu -- once-per-call and per-iteration helper kernels:
//   convert     caller image (f32/f16/bf16/u16, B x H x W) -> pitched f32
//   quantise    pitched f32 plane -> pitched f16 / bf16 plane (16-bit storage)
//   prologue    copies phi0 (and g) into the pitched work buffers, checks
//               finiteness, reduces the statistics of phi0 (Eq. 15 sums,
//               |{phi0 >= 0}|, the range of band 0) and finalises the
//               coefficients of the first step
//   normaliser  M = max_x |D(x)| for vector images (Eq. 17), one pass over I
//   output      v of the last executed step -> caller's phi_out and mask
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lse_reduce.cuh"

namespace {

constexpr int kThreads = 256;

// A value of a work plane stored as `storage` (LSE_F32 / LSE_F16 / LSE_BF16).
__device__ __forceinline__ float load_as(const void *p, size_t i, int storage)
{
    if (storage == LSE_F16) return __half2float(static_cast<const __half *>(p)[i]);
    if (storage == LSE_BF16) return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[i]);
    return static_cast<const float *>(p)[i];
}

__device__ __forceinline__ void store_as(void *p, size_t i, float v, int storage)
{
    if (storage == LSE_F16) static_cast<__half *>(p)[i] = __float2half_rn(v);
    else if (storage == LSE_BF16) static_cast<__nv_bfloat16 *>(p)[i] = __float2bfloat16_rn(v);
    else static_cast<float *>(p)[i] = v;
}

__device__ __forceinline__ bool aligned16(const void *p)
{
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

// v[0..3] = plane[i .. i + 3] (the first nj; the rest 0), with one 16-byte
// load when `vec` (FP32 plane, i a multiple of 4 in a 16-byte aligned row)
__device__ __forceinline__ void load4(const void *p, size_t i, int nj, int storage, bool vec,
                                      float (&v)[4])
{
    if (vec && nj == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(static_cast<const float *>(p) + i));
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = j < nj ? load_as(p, i + j, storage) : 0.0f;
}

__device__ __forceinline__ void store4(void *p, size_t i, int nj, int storage, bool vec,
                                       const float (&v)[4])
{
    if (vec && nj == 4) {
        *reinterpret_cast<float4 *>(static_cast<float *>(p) + i) = make_float4(v[0], v[1], v[2], v[3]);
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (j < nj) store_as(p, i + j, v[j], storage);
}

// The kernels below walk the image by rows: rows stride over the CTAs and
// each row's columns over the threads, so no pixel index is divided.

__global__ void __launch_bounds__(kThreads)
quantise_kernel(const float *__restrict__ src, int src_pitch, int H, int W,
                void *__restrict__ dst, int pitch, int storage)
{
    for (int y = blockIdx.x; y < H; y += gridDim.x)
        for (int x = threadIdx.x; x < W; x += blockDim.x)
            store_as(dst, (size_t)y * pitch + x, src[(size_t)y * src_pitch + x], storage);
}

__global__ void __launch_bounds__(kThreads)
convert_kernel(const void *__restrict__ src, int dtype, int H, int W, int B,
               float *__restrict__ dst, int pitch)
{
    const int rows = B * H;             // row b * H + y
    for (int row = blockIdx.x; row < rows; row += gridDim.x)
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const size_t i = (size_t)row * W + x;
        float v;
        switch (dtype) {
        case LSE_F16:
            v = __half2float(static_cast<const __half *>(src)[i]);
            break;
        case LSE_BF16:
            v = __bfloat162float(static_cast<const __nv_bfloat16 *>(src)[i]);
            break;
        case LSE_U16:
            v = (float)static_cast<const uint16_t *>(src)[i] / 65535.0f;  // IEEE division
            break;
        default:
            v = static_cast<const float *>(src)[i];
        }
        dst[(size_t)row * pitch + x] = v;
    }
}

__global__ void __launch_bounds__(kThreads)
prologue_kernel(const void *__restrict__ img, int img_pitch, size_t band_stride,
                const float *__restrict__ phi0, const void *__restrict__ g,
                int g_pitch, void *__restrict__ phi_dst,
                float *__restrict__ g_dst, int pitch, int H, int W, int B,
                int term, float dt, int storage, LseDevState *st, LsePartial *partials)
{
    LseAcc acc;
    acc.clear();
    const long long n = (long long)H * W;
    // band sums over phi >= 0 / phi < 0: compensated FP32 sums
    // (lse_kahan_add) in registers, turned into FP64 once; `acc`, which the
    // reduction indexes by a run-time band count, is filled at the end
    float sp[LSE_MAXB], cp[LSE_MAXB], sm[LSE_MAXB], cm[LSE_MAXB];
    int npos = 0;
#pragma unroll
    for (int b = 0; b < LSE_MAXB; ++b) sp[b] = cp[b] = sm[b] = cm[b] = 0.0f;
    // Each thread takes groups of 4 consecutive columns, read with one
    // 16-byte access where the plane allows it (FP32, 16-byte aligned rows)
    // and value by value otherwise: the arithmetic, and so every bit of the
    // result, is the same either way.
    unsigned int bits = 0;                 // per-pixel state in registers
    float fmx = -INFINITY, fmn = INFINITY;
    const bool f32 = storage == LSE_F32;
    const bool v_phi0 = (W & 3) == 0 && aligned16(phi0);
    const bool v_dst = f32 && (pitch & 3) == 0 && aligned16(phi_dst) &&
                       (g_dst == nullptr || aligned16(g_dst));
    const bool v_img = f32 && img != nullptr && (img_pitch & 3) == 0 &&
                       (band_stride & 3) == 0 && aligned16(img);
    const bool v_g = f32 && g != nullptr && (g_pitch & 3) == 0 && aligned16(g);
    for (int y = blockIdx.x; y < H; y += gridDim.x)
    for (int x = 4 * threadIdx.x; x < W; x += 4 * blockDim.x) {
        const int nj = W - x < 4 ? W - x : 4;
        float v[4];
        load4(phi0, (size_t)y * W + x, nj, LSE_F32, v_phi0, v);
        store4(phi_dst, (size_t)y * pitch + x, nj, storage, v_dst, v);
        bool pos[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j < nj && !isfinite(v[j])) bits |= LSE_SBIT_NONFINITE;
            pos[j] = j < nj && v[j] >= 0.0f;
            npos += pos[j];
        }
        if (term == LSE_TERM_EDGE) {
            float gv[4];
            load4(g, (size_t)y * g_pitch + x, nj, storage, v_g, gv);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < nj && !isfinite(gv[j])) bits |= LSE_SBIT_NONFINITE;
            if (g_dst) store4(g_dst, (size_t)y * pitch + x, nj, LSE_F32, v_dst, gv);
        } else {
#pragma unroll
            for (int b = 0; b < LSE_MAXB; ++b) {
                if (b < B) {
                    float iv[4];
                    load4(img, b * band_stride + (size_t)y * img_pitch + x, nj, storage, v_img,
                          iv);
                    // 4-pixel partials (past the row: zero), then the
                    // compensated sums
                    float pp = 0.0f, pm = 0.0f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float e = j < nj ? iv[j] : 0.0f;
                        if (j < nj && !isfinite(e)) bits |= LSE_SBIT_NONFINITE;
                        pp = __fadd_rn(pp, pos[j] ? e : 0.0f);
                        pm = __fadd_rn(pm, pos[j] ? 0.0f : e);
                        if (b == 0 && j < nj) {
                            fmx = fmaxf(fmx, e);
                            fmn = fminf(fmn, e);
                        }
                    }
                    lse_kahan_add(sp[b], cp[b], pp);
                    lse_kahan_add(sm[b], cm[b], pm);
                }
            }
        }
    }
    acc.bits = bits;
    acc.fmax = fmx;
    acc.fmin = fmn;
    if (term != LSE_TERM_EDGE) {
#pragma unroll
        for (int b = 0; b < LSE_MAXB; ++b) {
            acc.sp[b] = lse_kahan_value(sp[b], cp[b]);
            acc.sm[b] = lse_kahan_value(sm[b], cm[b]);
        }
    }
    acc.n_plus = npos;
    const int nb = term == LSE_TERM_EDGE ? 0 : B;
    LseAcc r;
    lse_cta_reduce(acc, nb, &r);
    if (!lse_publish_and_ticket(r, nb, partials, st)) return;
    LseAcc t;
    lse_sum_partials(partials, gridDim.x, nb, &t);
    if (threadIdx.x == 0) {
        st->npix = n;
        st->status_bits = t.bits;
        st->imin = t.fmin;
        st->imax = t.fmax;
        st->last_flips = 0;
        st->iterations_run = 0;
        st->stats_iter = 0;
        st->done = 0;
        st->last_buf = 0;
        st->norm_used = 0.0;
        st->grid_bar = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 12; ++j) st->acc[i][j] = 0;
        st->tile_ctr[0] = st->tile_ctr[1] = 0;
        st->fix_k = lse_fix_scale(fmax(fabs((double)t.fmin), fabs((double)t.fmax)), n);
        if (term == LSE_TERM_REGION) {
            lse_region_coeffs_v(st, t, B, dt, n, t.fmin, t.fmax);
        } else {
            st->area_plus = t.n_plus;
            st->zero_force = 0;
            st->norm = 0.0;
            for (int b = 0; b < LSE_MAXB; ++b) {
                st->c_plus[b] = 0.0;
                st->c_minus[b] = 0.0;
            }
        }
        __threadfence();
        st->ticket = 0;
    }
}

// M = max_x |sum_b alpha_b (I_b(x) - mid_b)| for B > 1, then the step
// coefficients a_b = dt alpha_b / (2 M).  Skipped when the statistics already
// made the force zero or the evolution has stopped.
__device__ __forceinline__ void normaliser(const float *__restrict__ img, int pitch,
                                           size_t band_stride, int H, int W, int B, float dt,
                                           LseDevState *st, LsePartial *partials, int cta,
                                           int ncta)
{
    if (st->done || st->zero_force || (st->status_bits & LSE_SBIT_ABORT)) return;
    float af[LSE_MAXB], m[LSE_MAXB];
#pragma unroll
    for (int b = 0; b < LSE_MAXB; ++b) {
        af[b] = st->af[b];
        m[b] = st->m[b];
    }
    LseAcc acc;
    acc.clear();
    // four columns per thread with float4 loads where the rows allow it
    // (pitch a multiple of 4 floats, 16-byte aligned planes): more loads in
    // flight per thread; a maximum does not depend on the order it is taken
    const bool vec = (pitch & 3) == 0 && (band_stride & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(img) & 15) == 0;
    if (vec) {
        for (int y = cta; y < H; y += ncta)
        for (int x = 4 * threadIdx.x; x < W; x += 4 * blockDim.x) {
            const float *src = img + (size_t)y * pitch + x;
            float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int b = 0; b < LSE_MAXB; ++b) {
                if (b < B) {
                    const float4 e = __ldg(reinterpret_cast<const float4 *>(src + b * band_stride));
                    d[0] = fmaf(af[b], e.x - m[b], d[0]);
                    d[1] = fmaf(af[b], e.y - m[b], d[1]);
                    d[2] = fmaf(af[b], e.z - m[b], d[2]);
                    d[3] = fmaf(af[b], e.w - m[b], d[3]);
                }
            }
            // columns past W are row padding
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x + j < W) {
                    acc.fmax = fmaxf(acc.fmax, d[j]);
                    acc.fmin = fminf(acc.fmin, d[j]);
                }
        }
    } else {
        for (int y = cta; y < H; y += ncta)
        for (int x = threadIdx.x; x < W; x += blockDim.x) {
            const float *src = img + (size_t)y * pitch + x;
            float d = 0.0f;
#pragma unroll
            for (int b = 0; b < LSE_MAXB; ++b)
                if (b < B) d = fmaf(af[b], __ldg(src + b * band_stride) - m[b], d);
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
        double M = fmax(fabs((double)t.fmax), fabs((double)t.fmin));
        st->norm = M;
        if (M > 0.0) {
            for (int b = 0; b < LSE_MAXB; ++b)
                st->a[b] = b < B ? (float)((double)dt * st->alpha[b] / (2.0 * M)) : 0.0f;
        } else {
            st->zero_force = 1;
            for (int b = 0; b < LSE_MAXB; ++b) st->a[b] = 0.0f;
        }
        __threadfence();
        st->ticket = 0;
    }
}

__global__ void __launch_bounds__(kThreads)
normaliser_kernel(const float *__restrict__ img, int pitch, size_t band_stride,
                  int H, int W, int B, float dt, LseDevState *st,
                  LsePartial *partials)
{
    normaliser(img, pitch, band_stride, H, W, B, dt, st, partials, blockIdx.x, gridDim.x);
}

// The normaliser of iteration n for a batch of vector images.
__global__ void __launch_bounds__(kThreads)
normaliser_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ blk_item,
                        long long launch)
{
    const BatchItem &it = items[blk_item[blockIdx.x]];
    const long long nl = launch - it.iter0;
    if (nl < 0 || nl >= it.cap) return;
    const StepArgs &a = it.args;
    normaliser(a.data, a.pitch, a.band_stride, a.H, a.W, a.B, a.dt, a.st, a.partials,
               blockIdx.x - it.nstart, it.nnblocks);
}

struct BufPair {
    const void *b[2];
};

__global__ void __launch_bounds__(kThreads)
output_kernel(BufPair bufs, int pitch, int H, int W, int storage, const LseDevState *st,
              float *__restrict__ phi_out, uint8_t *__restrict__ mask_out)
{
    if (st->status_bits & LSE_SBIT_ABORT) return;
    const void *src = bufs.b[st->last_buf];
    for (int y = blockIdx.x; y < H; y += gridDim.x)
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const size_t p = (size_t)y * W + x;
        float v = load_as(src, (size_t)y * pitch + x, storage);
        phi_out[p] = v;
        if (mask_out) mask_out[p] = v >= 0.0f ? 1 : 0;
    }
}

// CTAs for a row-wise walk over `rows` rows, at most `cap`.
int grid_rows(long long rows, int cap)
{
    if (rows < 1) rows = 1;
    return (int)(rows < cap ? rows : cap);
}

}  // namespace

namespace lse_detail {

cudaError_t launch_convert(const void *src, int dtype, int H, int W, int B,
                           float *dst, int pitch, cudaStream_t s)
{
    int grid = grid_rows((long long)B * H, 4096);
    convert_kernel<<<grid, kThreads, 0, s>>>(src, dtype, H, W, B, dst, pitch);
    return cudaGetLastError();
}

cudaError_t launch_quantise(const float *src, int src_pitch, int H, int W, void *dst,
                            int pitch, int storage, cudaStream_t s)
{
    int grid = grid_rows(H, 4096);
    quantise_kernel<<<grid, kThreads, 0, s>>>(src, src_pitch, H, W, dst, pitch, storage);
    return cudaGetLastError();
}

cudaError_t launch_prologue(const void *img, int img_pitch, size_t band_stride,
                            const float *phi0, const void *g, int g_pitch,
                            void *phi_dst, float *g_dst, int pitch, int H,
                            int W, int B, int term, float dt, int storage,
                            LseDevState *st, LsePartial *partials, int nblocks,
                            cudaStream_t s)
{
    int grid = grid_rows(H, nblocks);
    prologue_kernel<<<grid, kThreads, 0, s>>>(img, img_pitch, band_stride, phi0,
                                              g, g_pitch, phi_dst, g_dst, pitch,
                                              H, W, B, term, dt, storage, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_normaliser(const float *img, int pitch, size_t band_stride,
                              int H, int W, int B, float dt, LseDevState *st,
                              LsePartial *partials, int nblocks, cudaStream_t s)
{
    int grid = grid_rows(H, nblocks);
    normaliser_kernel<<<grid, kThreads, 0, s>>>(img, pitch, band_stride, H, W,
                                                B, dt, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_normaliser_batch(const BatchItem *items, const int *blk_item, long long n,
                                    int nblocks, cudaStream_t s)
{
    normaliser_batch_kernel<<<nblocks, kThreads, 0, s>>>(items, blk_item, n);
    return cudaGetLastError();
}

cudaError_t launch_output(float *const *bufs, int pitch, int H, int W, int storage,
                          const LseDevState *st, float *phi_out,
                          uint8_t *mask_out, cudaStream_t s)
{
    BufPair bp;
    bp.b[0] = bufs[0];
    bp.b[1] = bufs[1];
    int grid = grid_rows(H, 4096);
    output_kernel<<<grid, kThreads, 0, s>>>(bp, pitch, H, W, storage, st, phi_out,
                                            mask_out);
    return cudaGetLastError();
}

int partials_needed(int sm_count)
{
    // the widest reducing launch: 3 CTAs of 8 warps or 6 of 4 warps per SM
    // (tile-form step) or 8 CTAs of 256 threads per SM (grid-stride kernels);
    // the persistent evolution keeps two sets (step n and step n + 1) of up
    // to 6 per SM
    return sm_count * 12;
}

}  // namespace lse_detail
