// lse_mb_cand.cu -- the normaliser's candidate pixels for vector images.
//
// For B > 1 bands Eq. 17 normalises D(x) = sum_b alpha_b (I_b(x) - mid_b) by
// M = max_x |D(x)|.  D is an affine function of the pixel's colour
// (I_1(x), ..., I_B(x)), so its largest and smallest values over the image
// are taken at vertices of the convex hull of the colour cloud, and alpha
// changes with every iteration.  Once per image these kernels find, for
// LSE_MB_DIRS fixed directions a_k, the pixels with the largest and the
// smallest a_k . I(x): the seeds of the candidate set over which each step
// takes M (lse_step_tile.cuh).  The seeds need not contain every vertex:
// every step checks |D| at every pixel against its M and takes a step again
// when a pixel exceeds it, adding that pixel to the candidates.  They also
// find max |I_b| over the bands, which sets the fixed-point scale of the
// step's exact sums.
#include "lse_reduce.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kDirsPerBlock = 16;      // directions a CTA follows (blockIdx.y picks them)

// Direction k: the band axes first (largest and smallest along e_b give the
// band ranges), then a Weyl sequence over [-1, 1]^B with increments
// sqrt(2), sqrt(3), sqrt(5), sqrt(7) (fractional parts), evenly spread.
__device__ __forceinline__ float dir_component(int k, int b, int B)
{
    if (k < B) return k == b ? 1.0f : 0.0f;
    const float inc[4] = {0.41421356f, 0.73205081f, 0.23606798f, 0.64575131f};
    const float f = (float)(k - B + 1) * inc[b];
    return 2.0f * (f - floorf(f)) - 1.0f;
}

// Orderable bits of a float: unsigned comparison follows the float order.
__device__ __forceinline__ unsigned int ord_bits(float v)
{
    const unsigned int u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// largest value first, then the smallest pixel index
__device__ __forceinline__ unsigned long long key_of(float v, unsigned int pix)
{
    return ((unsigned long long)ord_bits(v) << 32) | (unsigned long long)(0xFFFFFFFFu - pix);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

template <int B>
__global__ void __launch_bounds__(kThreads)
mb_extremes_kernel(const float *__restrict__ bands, int pitch, size_t band_stride, int H, int W,
                   LseCandidates *cand)
{
    __shared__ unsigned long long s_key[kThreads / 32][2 * kDirsPerBlock];
    __shared__ unsigned int s_amax[kThreads / 32];
    const int k0 = blockIdx.y * kDirsPerBlock;
    float dir[kDirsPerBlock][B];
#pragma unroll
    for (int i = 0; i < kDirsPerBlock; ++i)
#pragma unroll
        for (int b = 0; b < B; ++b) dir[i][b] = dir_component(k0 + i, b, B);
    unsigned long long kmax[kDirsPerBlock], kmin[kDirsPerBlock];
#pragma unroll
    for (int i = 0; i < kDirsPerBlock; ++i) kmax[i] = kmin[i] = 0ull;
    float amax = 0.0f;
    for (int y = blockIdx.x; y < H; y += gridDim.x)
        for (int x = threadIdx.x; x < W; x += blockDim.x) {
            float c[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                c[b] = __ldg(bands + b * band_stride + (size_t)y * pitch + x);
                amax = fmaxf(amax, fabsf(c[b]));
            }
            const unsigned int pix = (unsigned int)y * (unsigned int)W + (unsigned int)x;
#pragma unroll
            for (int i = 0; i < kDirsPerBlock; ++i) {
                float p = 0.0f;
#pragma unroll
                for (int b = 0; b < B; ++b) p = fmaf(dir[i][b], c[b], p);
                const unsigned long long hi = key_of(p, pix), lo = key_of(-p, pix);
                kmax[i] = hi > kmax[i] ? hi : kmax[i];
                kmin[i] = lo > kmin[i] ? lo : kmin[i];
            }
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kDirsPerBlock; ++i) {
        const unsigned long long a = warp_max_u64(kmax[i]), b = warp_max_u64(kmin[i]);
        if (lane == 0) {
            s_key[warp][2 * i] = a;
            s_key[warp][2 * i + 1] = b;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) s_amax[warp] = __float_as_uint(amax);
    __syncthreads();
    if (threadIdx.x < 2 * kDirsPerBlock) {
        unsigned long long m = 0ull;
        for (int w = 0; w < kThreads / 32; ++w) m = s_key[w][threadIdx.x] > m ? s_key[w][threadIdx.x] : m;
        const int i = threadIdx.x >> 1, side = threadIdx.x & 1;
        atomicMax(&cand->key[2 * (k0 + i) + side], m);
    } else if (threadIdx.x == 32 && blockIdx.y == 0) {
        unsigned int m = 0u;
        for (int w = 0; w < kThreads / 32; ++w) m = s_amax[w] > m ? s_amax[w] : m;
        atomicMax(&cand->amax_bits, m);      // non-negative floats order as their bits
    }
}

// One CTA: the band values of every seed pixel, the candidate count, and
// the fixed-point scale of the step's sums from max |I_b|.
__global__ void __launch_bounds__(kThreads)
mb_gather_kernel(const float *__restrict__ bands, int pitch, size_t band_stride, int H, int W,
                 int B, LseCandidates *cand, LseDevState *st)
{
    for (int i = threadIdx.x; i < 2 * LSE_MB_DIRS; i += blockDim.x) {
        const unsigned int pix = 0xFFFFFFFFu - (unsigned int)(cand->key[i] & 0xFFFFFFFFull);
        const int y = (int)(pix / (unsigned int)W), x = (int)(pix % (unsigned int)W);
        for (int b = 0; b < 4; ++b)
            cand->val[i][b] = (b < B && y < H) ? bands[b * band_stride + (size_t)y * pitch + x]
                                               : 0.0f;
    }
    if (threadIdx.x == 0) {
        cand->count = 2 * LSE_MB_DIRS;
        cand->redone = 0;
        st->fix_k = lse_fix_scale((double)__uint_as_float(cand->amax_bits), (long long)H * W);
    }
}

}  // namespace

namespace lse_detail {

cudaError_t launch_mb_candidates(const float *bands, int pitch, size_t band_stride, int H,
                                 int W, int B, LseCandidates *cand, LseDevState *st,
                                 int sm_count, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(cand, 0, sizeof(LseCandidates), s);
    if (e != cudaSuccess) return e;
    const int rows = H < 2 * sm_count ? H : 2 * sm_count;
    const dim3 grid(rows < 1 ? 1 : rows, LSE_MB_DIRS / kDirsPerBlock);
    switch (B) {
    case 2: mb_extremes_kernel<2><<<grid, kThreads, 0, s>>>(bands, pitch, band_stride, H, W, cand); break;
    case 3: mb_extremes_kernel<3><<<grid, kThreads, 0, s>>>(bands, pitch, band_stride, H, W, cand); break;
    case 4: mb_extremes_kernel<4><<<grid, kThreads, 0, s>>>(bands, pitch, band_stride, H, W, cand); break;
    default: return cudaErrorNotSupported;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mb_gather_kernel<<<1, kThreads, 0, s>>>(bands, pitch, band_stride, H, W, B, cand, st);
    return cudaGetLastError();
}

}  // namespace lse_detail
