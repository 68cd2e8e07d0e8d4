// lse_edge.cu -- edge indicator g(I) = 1 / (1 + |grad(G_sigma1 * J)|^2) of
// Eq. 14, computed once per image, J = edge_scale * (band mean of I).
//
// One CTA per 32 x 32 output tile.  The band sum of I is staged with a
// (r1 + 1) halo (zero outside the image: the 'same' convolution's padding),
// smoothed separably (rows, then columns) on the tile plus a one-pixel ring,
// and differentiated with central differences, one-sided on the first/last
// row and column.  Smoothing and differences are linear, so the factor
// edge_scale / B is applied to the gradient.
//
// Precision.  g enters every iteration as dt * g * |grad phi|, so an error of
// e in g moves the LSF by up to ~20 e; keeping the LSF within 1e-5 of the
// FP64 reference needs g to ~5e-7.  The smoothed values are large (~100 in
// units of J) and their differences small, which FP32 cannot resolve.  The
// arithmetic is therefore float-float: a value is the unevaluated sum h + l
// of two floats (about 48 significant bits), built from error-free
// transformations -- Knuth's TwoSum for sums and the FMA remainder for
// products (Dekker 1971; Shewchuk 1997).  This part issues FP64 at a small
// fraction of the FP32 rate, and this formulation keeps all of the work on
// the FP32 pipes.  g itself is the FP32 reciprocal of the float-float
// denominator plus one Newton correction (within about half an ulp).
// Intensities (times edge_scale) must stay well inside the FP32 range,
// below ~1e37, for the error-free transformations to hold.
#include "lse_internal.h"

namespace {

constexpr int kTile = 32;
constexpr int kThreads = 256;
constexpr int SN = kTile + 2;              // S rows / cols (tile + 1 ring)

struct TapsFF {
    float h[16], l[16];                    // tap k = h[k] + l[k]
};

// s = fl(a + b), e = (a + b) - s exactly (TwoSum, no ordering needed)
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
    return s;
}

// (h, l) with h = fl(h + l): the normal form of a float-float value
__device__ __forceinline__ float2 renorm(float h, float l)
{
    float e;
    const float s = two_sum(h, l, e);
    return make_float2(s, e);
}

// x = t * (s + e) as (p, q), p = fl(t.h s) and q its remainder plus the
// cross terms (t.l e is below the float-float precision)
__device__ __forceinline__ float mul_tap(float th, float tl, float s, float e, float &q)
{
    const float p = __fmul_rn(th, s);
    q = __fmaf_rn(th, s, -p);
    q = __fmaf_rn(th, e, q);
    q = __fmaf_rn(tl, s, q);
    return p;
}

// acc (h, l) += (p, q): the high parts meet in TwoSum, whose error and the
// low parts collect in l (normalised once, at the end)
__device__ __forceinline__ void acc_add(float &h, float &l, float p, float q)
{
    float e;
    h = two_sum(h, p, e);
    l = __fadd_rn(l, __fadd_rn(e, q));
}

// a - b for normalised float-float values, unnormalised (s, e)
__device__ __forceinline__ float ff_sub(float2 a, float2 b, float &e)
{
    const float s = two_sum(a.x, -b.x, e);
    e = __fadd_rn(e, __fsub_rn(a.y, b.y));
    return s;
}

// Smoothing by the symmetric taps along a line of stride `st`: sum over
// |k| <= r1 of tap[|k|] * x[k * st].
__device__ __forceinline__ float2 smooth(const float2 *x, int st, int r1, const float *th,
                                         const float *tl)
{
    float l;
    const float2 c = x[0];
    float h = mul_tap(th[0], tl[0], c.x, c.y, l);
    for (int k = 1; k <= r1; ++k) {
        const float2 a = x[-k * st], b = x[k * st];
        float e;
        const float s = two_sum(a.x, b.x, e);
        e = __fadd_rn(e, __fadd_rn(a.y, b.y));
        float q;
        const float p = mul_tap(th[k], tl[k], s, e, q);
        acc_add(h, l, p, q);
    }
    return renorm(h, l);
}

__global__ void __launch_bounds__(kThreads)
edge_kernel(const float *__restrict__ img, int pitch, size_t band_stride,
            int H, int W, int B, TapsFF taps, int r1, float kh, float kl,
            float *__restrict__ g_out)
{
    extern __shared__ float2 smem[];
    __shared__ float s_th[16], s_tl[16];
    const int JN = kTile + 2 * r1 + 2;     // staged J rows / cols
    float2 *J = smem;                      // JN x JN
    float2 *Hh = J + JN * JN;              // JN x SN
    float2 *S = Hh + JN * SN;              // SN x SN
    const int x0 = blockIdx.x * kTile;
    const int y0 = blockIdx.y * kTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 16) {
        s_th[threadIdx.x] = taps.h[threadIdx.x];
        s_tl[threadIdx.x] = taps.l[threadIdx.x];
    }

    // J = sum_b I_b (exact for one band; TwoSum-accumulated otherwise)
    for (int jy = warp; jy < JN; jy += kThreads / 32) {
        const int gy = y0 - 1 - r1 + jy;
        for (int jx = lane; jx < JN; jx += 32) {
            const int gx = x0 - 1 - r1 + jx;
            float h = 0.0f, l = 0.0f;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                const float *p = img + (size_t)gy * pitch + gx;
                h = __ldg(p);
                for (int b = 1; b < B; ++b) {
                    float e;
                    h = two_sum(h, __ldg(p + b * band_stride), e);
                    l = __fadd_rn(l, e);
                }
            }
            J[jy * JN + jx] = renorm(h, l);
        }
    }
    __syncthreads();
    // rows: Hh[jy][c] = sum_k G(k) J[jy][c + r1 + k], c <-> column x0 - 1 + c
    for (int i = threadIdx.x; i < JN * SN; i += kThreads) {
        const int jy = i / SN, c = i - jy * SN;
        Hh[i] = smooth(J + jy * JN + c + r1, 1, r1, s_th, s_tl);
    }
    __syncthreads();
    // columns: S[r][c] = sum_k G(k) Hh[r + r1 + k][c], r <-> row y0 - 1 + r
    for (int i = threadIdx.x; i < SN * SN; i += kThreads) {
        const int r = i / SN, c = i - r * SN;
        S[i] = smooth(Hh + (r + r1) * SN + c, SN, r1, s_th, s_tl);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTile * kTile; i += kThreads) {
        const int ty = i / kTile, tx = i - ty * kTile;
        const int y = y0 + ty, x = x0 + tx;
        if (y >= H || x >= W) continue;
        const float2 *s = S + (ty + 1) * SN + (tx + 1);
        // gradient of the smoothed band sum, unnormalised float-float
        float sxh = 0.0f, sxl = 0.0f, syh = 0.0f, syl = 0.0f;
        if (W > 1) {
            if (x == 0) sxh = ff_sub(s[1], s[0], sxl);
            else if (x == W - 1) sxh = ff_sub(s[0], s[-1], sxl);
            else {
                sxh = __fmul_rn(0.5f, ff_sub(s[1], s[-1], sxl));   // exact halving
                sxl = __fmul_rn(0.5f, sxl);
            }
        }
        if (H > 1) {
            if (y == 0) syh = ff_sub(s[SN], s[0], syl);
            else if (y == H - 1) syh = ff_sub(s[0], s[-SN], syl);
            else {
                syh = __fmul_rn(0.5f, ff_sub(s[SN], s[-SN], syl));
                syl = __fmul_rn(0.5f, syl);
            }
        }
        // grad J = (edge_scale / B) grad S: (kh + kl) times each component
        float gxl, gyl;
        const float gxh = mul_tap(kh, kl, sxh, sxl, gxl);
        const float gyh = mul_tap(kh, kl, syh, syl, gyl);
        // q = gx^2 + gy^2
        float qxl = __fmaf_rn(gxh, gxh, -__fmul_rn(gxh, gxh));
        const float qxh = __fmul_rn(gxh, gxh);
        qxl = __fmaf_rn(__fmul_rn(2.0f, gxh), gxl, qxl);
        float qyl = __fmaf_rn(gyh, gyh, -__fmul_rn(gyh, gyh));
        const float qyh = __fmul_rn(gyh, gyh);
        qyl = __fmaf_rn(__fmul_rn(2.0f, gyh), gyl, qyl);
        float e;
        const float qh = two_sum(qxh, qyh, e);
        const float ql = __fadd_rn(e, __fadd_rn(qxl, qyl));
        // den = 1 + q (>= 1), then g = 1 / den: the FP32 quotient of the
        // leading part, corrected once by its float-float residual
        float e1;
        const float dh0 = two_sum(1.0f, qh, e1);
        const float2 den = renorm(dh0, __fadd_rn(e1, ql));
        const float r = __fdiv_rn(1.0f, den.x);
        float res = __fmaf_rn(-den.x, r, 1.0f);
        res = __fmaf_rn(-den.y, r, res);
        // a gradient beyond the FP32 range gives den = inf and g = 0, its limit
        g_out[(size_t)y * W + x] = isinf(den.x) ? 0.0f : __fmaf_rn(r, res, r);
    }
}

}  // namespace

namespace lse_detail {

cudaError_t launch_edge(const float *img, int pitch, size_t band_stride,
                          int H, int W, int B, const double *taps1, int rad1,
                          double edge_scale, float *g_out, cudaStream_t s)
{
    TapsFF t;
    for (int k = 0; k < 16; ++k) {
        const double v = k <= rad1 ? taps1[k] : 0.0;
        t.h[k] = (float)v;
        t.l[k] = (float)(v - (double)t.h[k]);
    }
    const double k = edge_scale / (double)B;
    const float kh = (float)k, kl = (float)(k - (double)kh);
    const int JN = kTile + 2 * rad1 + 2;
    size_t smem = sizeof(float2) * ((size_t)JN * JN + (size_t)JN * SN + (size_t)SN * SN);
    cudaError_t e = cudaFuncSetAttribute(
        edge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile);
    edge_kernel<<<grid, kThreads, smem, s>>>(img, pitch, band_stride, H, W, B, t, rad1, kh,
                                             kl, g_out);
    return cudaGetLastError();
}

}  // namespace lse_detail
