// lse_step_tile.cuh -- the fused LSE iteration, tile form (one band of the
// region term, or the edge term; TS = 3..15).
//
// Same arithmetic as the streaming kernel (lse_step_tma.cuh): per pixel
//   u = phi + dt R |grad phi|                        (Eq. 18)
//   v = G_sigma * u                                  (Table I step 4)
// then v (or sign(v) on re-initialising steps, Table I step 3) is stored and
// the next iteration's region sums are accumulated (Eq. 15).  Both forms sum
// in the same order, so their v agree bit for bit.
//
// Work decomposition.  A persistent CTA of 8 warps walks a static list of
// tiles of TH = 64 - 2 RAD output rows x (128 - 8 HL) output columns.  Per
// tile:
//   1. TMA stages phi on the tile plus RAD + 1 halo rows and 4 halo columns
//      per side (136 x 66 floats) and the data term on the tile plus RAD halo
//      rows (128 x 64); ghost columns are patched in on the image's edges;
//   2. u pass: warp w takes the 8 consecutive u rows 8w .. 8w + 7, rolling
//      the three phi rows of the gradient through registers; lane l holds 4
//      columns, the horizontal Gaussian pass takes neighbouring lanes' u by
//      shuffles, and h overwrites the phi row the warp has just consumed
//      (phi rows shared with the next warp are read before a barrier);
//   3. vertical pass: warp w takes RPW consecutive output rows, sliding a
//      2 RAD + 1 row register ring down its 4 columns of h; it stores v and
//      accumulates the statistics.
// With h in the phi buffer a CTA needs 70 KB of shared memory, so three CTAs
// share an SM (radius <= 4) and cover each other's TMA waits; the next tile
// is loaded as soon as the vertical pass is done.  (Starting the edge term's
// data copy right after the u pass, which last reads it, cost that kernel
// 5 %: the split load pushed it into register spills.)
//
// FAST instantiations serve the steady state of a re-initialising evolution
// (phi = +-1 in, sign(v) out, no sign-change count): ghost columns make the
// image border a plain central difference and |grad phi| takes one of six
// values, read from a table of correctly rounded square roots.  The general
// instantiations take any input and every per-step option.
//
// Waits on the TMA mbarriers are bounded (LSE_WAIT_LIMIT polls): a wait that
// runs out sets the TIMEOUT status bit, drains the copies in flight (bounded)
// and ends the CTA's tile loop; the CTA still takes part in the reduction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "lse_f2.cuh"
#include "lse_reduce.cuh"

namespace lse_tile {

constexpr int kURowsPerWarp = 8;      // u rows each warp computes per tile
constexpr int kPhiW = 136;            // staged phi columns

// Storage of phi and of the data term in HBM: float, or half / bfloat16
// (FP32 arithmetic either way).  A lane moves its 4 columns as one 16- or
// 8-byte access.
template <class T>
struct Stor;

template <>
struct Stor<float> {
    __device__ static float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
    __device__ static float ld1(const float *p) { return *p; }
    __device__ static float from(float v) { return v; }
    __device__ static float to(float v) { return v; }
    __device__ static void st4(float *p, float a, float b, float c, float d)
    {
        *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
    }
};

template <>
struct Stor<__nv_bfloat16> {
    using T = __nv_bfloat16;
    __device__ static float4 ld4(const T *p)
    {
        const uint2 r = *reinterpret_cast<const uint2 *>(p);
        const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.x));
        const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.y));
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    __device__ static float ld1(const T *p) { return __bfloat162float(*p); }
    __device__ static float from(T v) { return __bfloat162float(v); }
    __device__ static T to(float v) { return __float2bfloat16_rn(v); }
    __device__ static void st4(T *p, float a, float b, float c, float d)
    {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(c, d);
        uint2 r;
        r.x = *reinterpret_cast<const uint32_t *>(&lo);
        r.y = *reinterpret_cast<const uint32_t *>(&hi);
        *reinterpret_cast<uint2 *>(p) = r;
    }
};

template <>
struct Stor<__half> {
    using T = __half;
    __device__ static float4 ld4(const T *p)
    {
        const uint2 r = *reinterpret_cast<const uint2 *>(p);
        const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&r.x));
        const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&r.y));
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    __device__ static float ld1(const T *p) { return __half2float(*p); }
    __device__ static float from(T v) { return __half2float(v); }
    __device__ static T to(float v) { return __float2half_rn(v); }
    __device__ static void st4(T *p, float a, float b, float c, float d)
    {
        const __half2 lo = __floats2half2_rn(a, b);
        const __half2 hi = __floats2half2_rn(c, d);
        uint2 r;
        r.x = *reinterpret_cast<const uint32_t *>(&lo);
        r.y = *reinterpret_cast<const uint32_t *>(&hi);
        *reinterpret_cast<uint2 *>(p) = r;
    }
};

// Tile geometry for NW warps per CTA: each warp takes 8 u rows, so a tile
// has UR = 8 NW u rows and TH = UR - 2 RAD output rows (56 at NW = 8,
// RAD = 4; 24 at NW = 4).  Shared-memory layout.  FP32 storage: h
// overwrites the phi rows (70 KB per CTA at NW = 8, 36 KB at NW = 4); the
// data box is the 128 tile columns.  16-bit storage: a TMA box must start on
// 16 bytes, so the data box starts with phi's, 4 columns left of the tile
// (136 wide), and h has its own FP32 buffer.
template <int RAD, class T, int NW = 8, int NB = 1>
struct TileGeo {
    static constexpr int THREADS = 32 * NW;
    static constexpr int UR = kURowsPerWarp * NW;               // u / h rows per tile
    static constexpr int PHI_ROWS = UR + 2;                     // staged phi rows
    static constexpr bool WIDE = sizeof(T) == 4;
    static constexpr int HL = (RAD + 3) / 4;                    // halo lanes per side
    static constexpr int USEFUL = 128 - 8 * HL;                 // output columns
    static constexpr int TH = UR - 2 * RAD;                     // output rows
    static constexpr int RPW = (TH + NW - 1) / NW;              // output rows per warp
    static constexpr int DATA_W = WIDE ? 128 : kPhiW;           // staged data columns
    static constexpr int DATA_X0 = WIDE ? 0 : 4;                // tile column 0 within it
    static constexpr int PHI_BYTES = PHI_ROWS * kPhiW * (int)sizeof(T);
    // NB data planes (the bands of a vector image), one box each.  A vector
    // image stages the bands of its TH output rows only (u rows RAD ..
    // RAD + TH - 1); D of the 2 RAD halo u rows is formed from global memory
    // into a buffer of its own, which leaves room for a third CTA per SM
    static constexpr int DROW0 = NB > 1 ? RAD : 0;              // first staged u row
    static constexpr int DROWS = UR - 2 * DROW0;                // staged data rows
    static constexpr int PLANE = DROWS * DATA_W;                // elements per data plane
    static constexpr int DATA_BYTES = NB * PLANE * (int)sizeof(T);
    // offsets in floats: [sqrt table 32][2 mbarriers][old-sign words 64 x 4]
    // [phi][data][h (16-bit storage only) | halo D (vector images)]
    static constexpr int SIGN_OFF = 64;
    static constexpr int PHI_OFF = SIGN_OFF + UR * 4;
    static constexpr int DATA_OFF = PHI_OFF + ((PHI_BYTES / 4 + 31) & ~31);
    static constexpr int HBUF_OFF = DATA_OFF + ((DATA_BYTES / 4 + 31) & ~31);
    static constexpr int DH_OFF = HBUF_OFF;                     // 2 RAD rows x 128
    static constexpr int FLOATS = !WIDE ? HBUF_OFF + UR * 128
                                : NB > 1 ? DH_OFF + 2 * RAD * 128
                                         : DATA_OFF + DATA_BYTES / 4;
    static constexpr int BYTES = FLOATS * 4 + 128;              // + alignment slack
    // h of u row ur: float index (ur + H_ROW0) * H_STRIDE + H_COL0 + 4 lane
    // from the phi buffer (FP32) or from the h buffer (16-bit)
    static constexpr int H_STRIDE = WIDE ? kPhiW : 128;
    static constexpr int H_ROW0 = WIDE ? 2 : 0;
    static constexpr int H_COL0 = WIDE ? 4 : 0;
    // the vertical pass reads h rows up to NW RPW - 1 + 2 RAD; past row
    // UR - 1 they lie in other shared memory (FP32) or are clamped (16-bit)
    static constexpr bool CLAMP_H = !WIDE && NW * RPW - 1 + 2 * RAD > UR - 1;
    // CTAs per SM (launch bounds): 24 warps for RAD <= 4, else 16; vector
    // images as many as their shared memory allows (228 KB per SM), at most
    // 3 (the step of a vector image needs 150-170 registers a thread)
    static constexpr int MB_BLOCKS = (227 * 1024) / (BYTES + 3072);
    static constexpr int MIN_BLOCKS =
        NB == 1 ? (RAD <= 4 ? 24 : 16) / NW
                : (MB_BLOCKS < 1 ? 1 : MB_BLOCKS > 3 ? 3 : MB_BLOCKS);
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Programmatic dependent launch, for the 32-row (4-warp) instantiations: a
// grid that leaves SM slots free (StepArgs::pdl) is launched so that the next
// one may become resident while it finishes.  Every CTA of such a launch
// waits for the previous grid's completion and memory before anything else,
// so no CTA can exit earlier and a grid's completion implies its
// predecessor's (a plain launch starts only after its predecessor
// completed); each lets the next grid launch once its tiles are done.  The
// 64-row instantiations carry neither instruction: in them alone it cost a
// full-grid launch about 1 % (measured), and images small enough to gain
// from it default to 32-row tiles.  Batches launch plainly.
__device__ __forceinline__ void wait_prior_grid()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void allow_next_grid()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Low 32 bits of %globaltimer (ns); differences are wrap-safe up to ~4.29 s.
__device__ __forceinline__ uint32_t global_ns_lo()
{
    uint32_t t;
    asm volatile("mov.u32 %0, %%globaltimer_lo;" : "=r"(t));
    return t;
}

// Bounded wait; block-uniform result (every thread polls).  Gives up after
// LSE_WAIT_LIMIT polls or limit_ns nanoseconds (at most 4e9), whichever
// comes first (the clock is read every 256 polls, from the 256th on).
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity,
                                         uint32_t limit_ns = (uint32_t)LSE_WAIT_NS)
{
    bool ok = false;
    uint32_t t0 = 0;
    for (uint32_t i = 0; i < LSE_WAIT_LIMIT; ++i) {
        if (try_wait(bar, parity)) {
            ok = true;
            break;
        }
        if ((i & 255u) == 255u) {
            const uint32_t t = global_ns_lo();
            if (i == 255u) t0 = t;
            else if (t - t0 > limit_ns) break;
        }
    }
    return __syncthreads_and(ok) != 0;
}

// One 2-D box load, issued by the calling thread.
__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap *map, int x,
                                        int y, uint32_t bar, uint32_t bytes)
{
    asm volatile(
        "fence.proxy.async.shared::cta;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%4], %5;\n\t"
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar),
          "r"(bytes)
        : "memory");
}

// One 3-D box load (x, y, plane 0 .. box depth - 1), issued by the calling
// thread: the bands of a vector image in one copy.
__device__ __forceinline__ void tma_box3(uint32_t dst, const CUtensorMap *map, int x, int y,
                                         uint32_t bar, uint32_t bytes)
{
    asm volatile(
        "fence.proxy.async.shared::cta;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%4], %5;\n\t"
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %6}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar),
          "r"(bytes), "r"(0)
        : "memory");
}

__device__ __forceinline__ float bin(float v) { return v >= 0.0f ? 1.0f : -1.0f; }

__device__ __forceinline__ float4 bin4(float4 v)
{
    return make_float4(bin(v.x), bin(v.y), bin(v.z), bin(v.w));
}

__device__ __forceinline__ float comp(const float4 &v, int j)
{
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

__device__ __forceinline__ float4 lds4(const float *p)
{
    return *reinterpret_cast<const float4 *>(p);
}

// What one step of the persistent evolution (all iterations in one launch)
// passes to tile_step and gets back.
struct TilePersist {
    LseStepFlags f;             // the step's flags (lse_step_flags)
    float *phi_out;             // the LSF plane the step writes
    unsigned long long stall_ns;   // test hook, first step only
    float coef, mid;            // step coefficients (every CTA computed them)
    uint32_t par;               // mbarrier parity, carried from step to step
    int issued;                 // boxes of the first tile already issued:
                                // 0 none, 1 data (prefetched), 2 data and phi
    int prefetch;               // issue the next step's first data box at the end
    int slot;                   // the state record's sum slot of the step
    int queue;                  // the tile queue of the step
    // vector images: D = sum_b af[b] (I_b - m[b]) (Eq. 17's numerator) and
    // the largest |D| the step's normaliser allows (beyond it a pixel is
    // reported to the slot's miss word)
    float af[4], m[4];
    float thr;
    int need_sa;                // sum I_b over the image too (a vector image's
                                // first step; the total is the same later)
};

// Slot layout of LseDevState::acc (fixed-point sums of a step): sum w I_b
// and sum I_b for up to 4 bands, the count, the sign changes, and for vector
// images the pixel whose |D| exceeded the normaliser (orderable |D| bits
// above the inverted pixel index, combined with atomicMax).
enum { LSE_ACC_SW = 0, LSE_ACC_SA = 4, LSE_ACC_NP = 8, LSE_ACC_FL = 9, LSE_ACC_MISS = 10 };

// The 128-byte aligned base (in floats) of the dynamic shared memory, the
// table of square roots the FAST code reads, and the mbarriers.  Once per
// CTA, before any box is issued.
template <int RAD, class T, int NW>
__device__ __forceinline__ void tile_smem_init()
{
    extern __shared__ float smem_f[];
    const uint32_t sm0 = smem_u32(smem_f);
    const int sb = (int)(((128u - (sm0 & 127u)) & 127u) >> 2);
    const int tid = threadIdx.x;
    if (tid < 32) {
        // sqrt table indexed by bits(q) >> 21 & 31 for q in {0,4,8,16,20,32}
        const float q = tid == 4 ? 4.f : tid == 8 ? 8.f : tid == 12 ? 16.f
                      : tid == 13 ? 20.f : tid == 16 ? 32.f : 0.f;
        smem_f[sb + tid] = sqrtf(q);
    }
    if (tid == 0) {
        const uint32_t bar_phi = sm0 + 4u * (uint32_t)(sb + 32);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_phi) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_phi + 8) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_phi + 16) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// One step over the tiles of one image, run by CTA `cta` of the `ncta` CTAs
// given to it.  PERSIST: one step of the persistent evolution (pc holds the
// coefficients and the box state; the CTA's reduced sums go to ps->slot and
// nothing is finalised here); returns whether a wait ran out.
// NB > 1: the region term of a vector image (Eq. 17 summed over NB bands,
// FP32 storage, persistent evolution only): the NB band boxes are staged
// together, D is formed per pixel in the u pass, and the band sums come from
// the staged bands.
template <int KIND_EDGE, int RAD, bool FAST, class T, int NW, bool PERSIST = false, int NB = 1>
__device__ __forceinline__ bool tile_step(const StepArgs &a, const CUtensorMap *phi_map,
                                          const CUtensorMap *data_map, int cta, int ncta,
                                          TilePersist *ps = nullptr)
{
    using G = TileGeo<RAD, T, NW, NB>;
    constexpr int kThreads = G::THREADS, kURows = G::UR, kPhiRows = G::PHI_ROWS;
    using S = Stor<T>;
    constexpr int HL = G::HL, TH = G::TH, P = 2 * RAD + 1, RPW = G::RPW;
    constexpr bool EDGE = KIND_EDGE != 0;
    constexpr bool MB = NB > 1;
    // the update takes t = coef d (edge term: d = g; vector image: d = D)
    constexpr bool DIRECT = EDGE || MB;
    static_assert(!MB || (PERSIST && !EDGE && sizeof(T) == 4 && NB <= 4),
                  "vector images: FP32 region term, persistent evolution");

    LseDevState *st = a.st;
    if constexpr (!PERSIST) {
        if (st->done || (st->status_bits & LSE_SBIT_ABORT)) return false;
    }

    extern __shared__ float smem_f[];
    const uint32_t sm0 = smem_u32(smem_f);
    const int sb = (int)(((128u - (sm0 & 127u)) & 127u) >> 2);   // 128-byte aligned base
    float *lut = smem_f + sb;
    uint32_t *sign_w = reinterpret_cast<uint32_t *>(smem_f + sb + G::SIGN_OFF);
    T *buf = reinterpret_cast<T *>(smem_f + sb + G::PHI_OFF);
    const T *dat = reinterpret_cast<const T *>(smem_f + sb + G::DATA_OFF);
    float *hbase = G::WIDE ? smem_f + sb + G::PHI_OFF : smem_f + sb + G::HBUF_OFF;
    const uint32_t bar_phi = sm0 + 4u * (uint32_t)(sb + 32);
    const uint32_t bar_dat = bar_phi + 8;
    const uint32_t bar_never = bar_phi + 16;   // test hook: nothing arrives here
    const uint32_t phi_dst = sm0 + 4u * (uint32_t)(sb + G::PHI_OFF);
    const uint32_t dat_dst = sm0 + 4u * (uint32_t)(sb + G::DATA_OFF);
    constexpr uint32_t kPhiBytes = G::PHI_BYTES;
    constexpr uint32_t kDatBytes = G::DATA_BYTES;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int H = a.H, W = a.W;
    const int tiles_x = a.n_strips, n_tiles = a.n_items;

    if constexpr (!PERSIST) {
        if (FAST && tid < 32) {
            // sqrt table indexed by bits(q) >> 21 & 31 for q in {0,4,8,16,20,32}
            const float q = tid == 4 ? 4.f : tid == 8 ? 8.f : tid == 12 ? 16.f
                          : tid == 13 ? 20.f : tid == 16 ? 32.f : 0.f;
            lut[tid] = sqrtf(q);
        }
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_phi) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_dat) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_never) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }

    float tp[RAD + 1];
#pragma unroll
    for (int k = 0; k <= RAD; ++k) tp[k] = a.taps[k];
    // edge term: dt / 2 (t = dt g / 2); the D plane of a vector image: the
    // coefficient its band pass left, dt / (2 M)
    const float coef = PERSIST ? ps->coef : EDGE ? (a.mb_split ? st->a[0] : a.half_dt) : st->a[0];
    const float mid = PERSIST ? ps->mid : EDGE ? 0.0f : st->m[0];
    const f2 coef2 = f2_pack(coef, coef), mid2 = f2_pack(mid, mid);
    float af[NB], mb_m[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        af[b] = MB ? ps->af[b] : 0.0f;
        mb_m[b] = MB ? ps->m[b] : 0.0f;
    }
    const float thr = MB ? ps->thr : 0.0f;
    const bool need_sa = MB && ps->need_sa != 0;
    unsigned long long *const miss_word = reinterpret_cast<unsigned long long *>(
        &st->acc[PERSIST ? ps->slot : 0][LSE_ACC_MISS]);
    const float sqrt8 = sqrtf(8.0f);
    const bool binarise_in = !FAST && (PERSIST ? ps->f.binarise_in : a.binarise_in) != 0;
    const bool count_flips = !FAST && (PERSIST ? ps->f.count_flips : a.count_flips) != 0;
    const bool store_bin = FAST || (PERSIST ? ps->f.store_bin : a.store_bin) != 0;
    const unsigned long long stall_ns = PERSIST ? ps->stall_ns : a.stall_ns;
    float *const phi_out = PERSIST ? ps->phi_out : a.phi_out;

    auto origin = [&](int t, int &xs, int &ys) {
        const int ty = t / tiles_x;
        xs = (t - ty * tiles_x) * G::USEFUL - 4 * HL;   // first staged data column
        ys = ty * TH - (RAD + 1);                        // first staged phi row
    };
    auto load_phi = [&](int t) {
        int xs, ys;
        origin(t, xs, ys);
        tma_box(phi_dst, phi_map, xs - 4, ys, bar_phi, kPhiBytes);
    };
    auto load_data = [&](int t) {
        int xs, ys;
        origin(t, xs, ys);
        if (MB)
            tma_box3(dat_dst, data_map, xs - G::DATA_X0, ys + 1 + G::DROW0, bar_dat, kDatBytes);
        else
            tma_box(dat_dst, data_map, xs - G::DATA_X0, ys + 1, bar_dat, kDatBytes);
    };
    auto load_tile = [&](int t) {
        load_phi(t);
        load_data(t);
    };

    // tile order.  Region term: the first tile of CTA c is tile c, the rest
    // are taken from a queue as the CTAs get to them (the three CTAs sharing
    // an SM run at different speeds, so equal static shares finish far
    // apart); the statistics are exact integer sums, the same whoever takes
    // a tile.  Edge term: CTA c takes tiles c, c + ncta, ... (the queue
    // measured slower there: 143.8 against 135.0 us per 8192 x 8192 step).
    constexpr bool QUEUE = !EDGE;
    unsigned int *const queue = &st->tile_ctr[PERSIST ? ps->queue : 0];
    __shared__ int s_next;
    const int fix_k = st->fix_k;
    int t = cta;
    if (tid == 0 && t < n_tiles) {
        if (!PERSIST || ps->issued == 0) {
            load_tile(t);
        } else if (ps->issued == 1) {
            load_phi(t);
        }
    }
    uint32_t par = PERSIST ? ps->par : 0u;
    bool failed = false;

    // 2 |{v >= 0}| over this lane's pixels: sum w + valid pixels.  fcnt is
    // an exact small integer (at most 4 x 64 in magnitude), converted in 32
    // bits: a float to 64-bit conversion issues on the FP64 pipe
    long long cnt2 = 0;
    int nflip = 0;
    long long sw_x[NB], sa_x[NB];                // fixed-point lane sums (lse_fix)
#pragma unroll
    for (int b = 0; b < NB; ++b) sw_x[b] = sa_x[b] = 0;
    const bool lane_out = lane >= HL && lane < 32 - HL;
    const int eidx = lane == 0 ? 3 : 132;        // phi column beyond the warp's edge
    const T *bl = buf + 4 + 4 * lane;            // this lane's 4 columns of a phi row
    const T *dl = dat + G::DATA_X0 + 4 * lane;   // ... of a data row
    float *hl = hbase + G::H_COL0 + 4 * lane;    // ... of an h row
    float *dhl = smem_f + sb + G::DH_OFF + 4 * lane;   // ... of a halo D row

    // D = sum_b af_b (I_b - m_b) (Eq. 17's numerator) on the lane's 4
    // columns, bands in order, on column pairs; band(b) gives I_b there
    auto mb_d = [&](auto band) {
        f2 d01 = f2_pack(0.0f, 0.0f), d23 = d01;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const float4 e = band(b);
            const f2 a2 = f2_pack(af[b], af[b]), m2 = f2_pack(mb_m[b], mb_m[b]);
            d01 = f2_fma(a2, f2_sub(f2_pack(e.x, e.y), m2), d01);
            d23 = f2_fma(a2, f2_sub(f2_pack(e.z, e.w), m2), d23);
        }
        float4 d4;
        f2_unpack(d01, d4.x, d4.y);
        f2_unpack(d23, d4.z, d4.w);
        return d4;
    };

    // test hook: a wait that cannot complete (nothing arrives on bar_never)
    // runs out into the TIMEOUT status; the first tile's copies, issued
    // above, are drained below like those of any failed wait
    // (the first step of an evolution never takes the FAST instantiation)
    if (!FAST && stall_ns && t < n_tiles) {
        (void)wait_bar(bar_never, 0, (uint32_t)stall_ns);
        failed = true;
    }
    for (; t < n_tiles && !failed;) {
        int xs, ys;
        origin(t, xs, ys);
        const int x0 = xs + 4 * lane;
        if constexpr (MB) {
            // D of the halo u rows 0 .. RAD - 1 and TH + RAD .. UR - 1 (slots
            // k = 0 .. 2 RAD - 1), from global memory while the tile's boxes
            // land; outside the image a band reads as zero, as the boxes'
            // fill gives it, so D is that of the staged rows bit for bit.
            // The slots were last read before the previous tile's vertical
            // pass; the waits below order these stores before their reads
            const bool xin = x0 >= 0 && x0 < W;       // x0 is a multiple of 4
#pragma unroll 1
            for (int k = warp; k < 2 * RAD; k += NW) {
                const int y = ys + 1 + (k < RAD ? k : TH + k);
                const bool in = xin && y >= 0 && y < H;
                const float4 d4 = mb_d([&](int b) {
                    float4 e = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (in) {
                        // x0 < W and the pitch is a multiple of 4, so the
                        // load stays in the row; columns at or past W are
                        // zeroed
                        e = __ldg(reinterpret_cast<const float4 *>(
                            a.data + b * a.band_stride + (size_t)y * a.pitch + x0));
                        if (x0 + 1 >= W) e.y = 0.0f;
                        if (x0 + 2 >= W) e.z = 0.0f;
                        if (x0 + 3 >= W) e.w = 0.0f;
                    }
                    return e;
                });
                *reinterpret_cast<float4 *>(dhl + k * 128) = d4;
            }
        }
        if (!wait_bar(bar_phi, par) || !wait_bar(bar_dat, par)) {
            failed = true;
            break;
        }
        // take the next tile while this one is worked on: the claim stays
        // in flight (nothing reads it) until the tile is done
        unsigned int claim = 0;
        if (QUEUE && tid == 0) claim = atomicAdd(queue, 1u);
        // tiles that touch column 0 or W - 1 (or lie partly outside) take the
        // border code; so do tiles whose u rows reach row 0 or H - 1
        const bool xborder = xs < 0 || xs + 128 >= W;
        const bool interior = !xborder && ys >= 0 && ys + kPhiRows <= H;
        if (FAST && xborder) {
            // ghost columns 2 phi(0) - phi(1) and 2 phi(W-1) - phi(W-2)
            const bool gl = xs <= 0, gr = xs <= W - 1 && W - 1 < xs + 128;
            for (int rr = tid; rr < kPhiRows; rr += kThreads) {
                T *row = buf + rr * kPhiW;
                if (gl) {
                    const float f0 = S::from(row[4 - xs]);
                    const float f1 = W > 1 ? S::from(row[5 - xs]) : f0;
                    row[3 - xs] = S::to(2.0f * f0 - f1);
                }
                if (gr) {
                    const float fe = S::from(row[W + 3 - xs]);
                    const float fd = W > 1 ? S::from(row[W + 2 - xs]) : fe;
                    row[W + 4 - xs] = S::to(2.0f * fe - fd);
                }
            }
            __syncthreads();
        }
        float inb[4], okf[4];
        bool oneL[4], oneR[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = x0 + j;
            inb[j] = (x >= 0 && x < W) ? 1.0f : 0.0f;
            okf[j] = (lane_out && x < W) ? 1.0f : 0.0f;
            oneL[j] = x == 0;
            oneR[j] = x == W - 1;
        }

        // ---- u pass: u rows ur0 .. ur0 + 7 (centre phi row = slot ur + 1)
        const int ur0 = warp * kURowsPerWarp;
        float4 pm = S::ld4(bl + ur0 * kPhiW);
        float4 pc = S::ld4(bl + (ur0 + 1) * kPhiW);
        float ec = S::ld1(buf + (ur0 + 1) * kPhiW + eidx);
        if (binarise_in) {
            pm = bin4(pm);
            pc = bin4(pc);
            ec = bin(ec);
        }
        __syncthreads();   // rows 8w and 8w + 1 are in registers before warp w - 1 overwrites them

        // One u row: u (Eq. 18) on the lane's 4 columns, the horizontal
        // Gaussian pass, h stored over the phi slot just read.  IN: interior
        // tile (no ghost rows, no columns outside the image or on its edge).
        auto urow = [&](auto in_tag, int ur) {
            constexpr bool IN = decltype(in_tag)::value;
            float4 pp = S::ld4(bl + (ur + 2) * kPhiW);
            float ep = S::ld1(buf + (ur + 2) * kPhiW + eidx);
            float4 d4;
            if constexpr (MB) {
                // halo rows: D from its buffer; output rows: from the
                // staged bands (row ur - RAD of each plane)
                if (ur < RAD)
                    d4 = lds4(dhl + ur * 128);
                else if (ur >= RAD + TH)
                    d4 = lds4(dhl + (ur - TH) * 128);
                else
                    d4 = mb_d([&](int b) {
                        return lds4(reinterpret_cast<const float *>(dl) + b * G::PLANE +
                                    (ur - RAD) * G::DATA_W);
                    });
            } else {
                d4 = S::ld4(dl + ur * G::DATA_W);
            }
            if (binarise_in) {
                pp = bin4(pp);
                ep = bin(ep);
            }
            if (count_flips) {
                // old signs of this row for the sign-change count
                const uint32_t s0 = __ballot_sync(0xffffffffu, pc.x >= 0.0f);
                const uint32_t s1 = __ballot_sync(0xffffffffu, pc.y >= 0.0f);
                const uint32_t s2 = __ballot_sync(0xffffffffu, pc.z >= 0.0f);
                const uint32_t s3 = __ballot_sync(0xffffffffu, pc.w >= 0.0f);
                if (lane == 0)
                    *reinterpret_cast<uint4 *>(sign_w + 4 * ur) = make_uint4(s0, s1, s2, s3);
            }
            float lft = __shfl_up_sync(0xffffffffu, pc.w, 1);
            float rgt = __shfl_down_sync(0xffffffffu, pc.x, 1);
            if (lane == 0) lft = ec;
            if (lane == 31) rgt = ec;
            const float c[6] = {lft, pc.x, pc.y, pc.z, pc.w, rgt};
            float up[4] = {pm.x, pm.y, pm.z, pm.w};
            float dn[4] = {pp.x, pp.y, pp.z, pp.w};
            bool yin = true;
            if (!IN) {
                const int y = ys + 1 + ur;
                if (y <= 0 || y >= H - 1) {             // ghost rows; rows outside
                    yin = y >= 0 && y < H;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (H == 1) {
                            up[j] = c[j + 1];
                            dn[j] = c[j + 1];
                        } else if (y == 0) {
                            up[j] = 2.f * c[j + 1] - dn[j];
                        } else if (y == H - 1) {
                            dn[j] = 2.f * c[j + 1] - up[j];
                        }
                    }
                }
            }
            float dxs[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float dx = c[j + 2] - c[j];
                if (!FAST && !IN) {
                    if (W == 1) dx = 0.0f;
                    else if (oneL[j]) dx = 2.0f * (c[j + 2] - c[j + 1]);
                    else if (oneR[j]) dx = 2.0f * (c[j + 1] - c[j]);
                }
                dxs[j] = dx;
            }
            // the update on column pairs: each packed operation rounds as
            // its scalar form, so u is bitwise the scalar u
            float u[4];
#pragma unroll
            for (int jp = 0; jp < 2; ++jp) {
                const int j0 = 2 * jp, j1 = 2 * jp + 1;
                const f2 dx = f2_pack(dxs[j0], dxs[j1]);
                const f2 dy = f2_sub(f2_pack(dn[j0], dn[j1]), f2_pack(up[j0], up[j1]));
                float q[2];
                f2_unpack(f2_fma(dx, dx, f2_mul(dy, dy)), q[0], q[1]);
                float s2[2];
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    // +-1 phi off the image border: q is 0, 4 or 8, and
                    // sqrt(q) is q / 2 (exact) or sqrt(8)
                    s2[e] = !FAST ? sqrtf(q[e])
                          : IN ? (q[e] == 8.0f ? sqrt8 : 0.5f * q[e])
                               : lut[(__float_as_uint(q[e]) >> 21) & 31u];
                const f2 d = f2_pack(comp(d4, j0), comp(d4, j1));
                const f2 t = DIRECT ? f2_mul(coef2, d) : f2_mul(coef2, f2_sub(d, mid2));
                f2_unpack(f2_fma(t, f2_pack(s2[0], s2[1]), f2_pack(c[j0 + 1], c[j1 + 1])),
                          u[j0], u[j1]);
            }
            if (!IN) {
                if (xborder) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) u[j] *= inb[j];
                }
                if (!yin) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) u[j] = 0.0f;
                }
            }
            if constexpr (MB) {
                // the normaliser must bound |D| at every pixel of the image
                // (Eq. 17); a pixel beyond it is reported (rare: the step
                // is then done again with that pixel's |D|)
                bool over = false;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    over |= (IN || (inb[j] != 0.0f && yin)) && fabsf(comp(d4, j)) > thr;
                if (over) {
                    const int y = ys + 1 + ur;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float ad = fabsf(comp(d4, j));
                        if ((IN || (inb[j] != 0.0f && yin)) && ad > thr) {
                            const unsigned int pix = (unsigned int)y * (unsigned int)W +
                                                     (unsigned int)(x0 + j);
                            atomicMax(miss_word,
                                      ((unsigned long long)__float_as_uint(ad) << 32) |
                                          (unsigned long long)(0xFFFFFFFFu - pix));
                        }
                    }
                }
            }
            float U[4 + 8 * HL];
#pragma unroll
            for (int j = 0; j < 4; ++j) U[4 * HL + j] = u[j];
#pragma unroll
            for (int o = 1; o <= HL; ++o) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j - 4 * o >= -RAD)
                        U[4 * HL + j - 4 * o] = __shfl_up_sync(0xffffffffu, u[j], o);
                    if (j + 4 * o <= 3 + RAD)
                        U[4 * HL + j + 4 * o] = __shfl_down_sync(0xffffffffu, u[j], o);
                }
            }
            float hv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float h = tp[0] * U[4 * HL + j];
#pragma unroll
                for (int q = 1; q <= RAD; ++q)
                    h = fmaf(tp[q], U[4 * HL + j - q] + U[4 * HL + j + q], h);
                hv[j] = h;
            }
            // FP32 storage: h of u row ur replaces phi slot ur + 2, read above
            // by this warp
            *reinterpret_cast<float4 *>(hl + (ur + G::H_ROW0) * G::H_STRIDE) =
                make_float4(hv[0], hv[1], hv[2], hv[3]);
            pm = pc;
            pc = pp;
            ec = ep;
        };
        if (interior) {
#pragma unroll
            for (int i = 0; i < kURowsPerWarp; ++i) urow(std::true_type{}, ur0 + i);
        } else {
#pragma unroll 2
            for (int i = 0; i < kURowsPerWarp; ++i) urow(std::false_type{}, ur0 + i);
        }
        // the buffer is refilled by TMA after the vertical pass
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();

        // ---- vertical pass: output rows r_first .. r_first + RPW - 1
        {
            const int r_first = warp * RPW;
            int rows = H - (ys + RAD + 1);               // valid output rows of the tile
            rows = rows < TH ? rows : TH;
            int rv = rows - r_first;
            rv = rv < 0 ? 0 : (rv > RPW ? RPW : rv);
            // x0 + 4 <= pitch whenever x0 < W (x0 and the pitch are multiples
            // of 4): the lane stores all 4 columns, the padding is scratch
            const bool st_ok = lane_out && x0 < W;
            T *dst = reinterpret_cast<T *>(phi_out) + (size_t)(ys + RAD + 1 + r_first) * a.pitch + x0;
            const size_t pitch = (size_t)a.pitch;
            // the ring holds the lane's 4 columns of 2 RAD + 1 h rows as
            // column pairs, so each tap of the pass is one packed
            // instruction for two columns
            f2 rg[P][2];
            f2 tp2[RAD + 1];
#pragma unroll
            for (int q = 0; q <= RAD; ++q) tp2[q] = f2_pack(tp[q], tp[q]);
            // h rows past the tile read other shared memory (finite values);
            // their outputs are never used
            auto ldh = [&](int hr, f2 *d) {
                if (G::CLAMP_H) hr = hr < kURows - 1 ? hr : kURows - 1;
                const float4 h4 = lds4(hl + (hr + G::H_ROW0) * G::H_STRIDE);
                d[0] = f2_pack(h4.x, h4.y);
                d[1] = f2_pack(h4.z, h4.w);
            };
            float fsw[NB], fsa[NB], fcnt = 0.0f;
#pragma unroll
            for (int b = 0; b < NB; ++b) fsw[b] = fsa[b] = 0.0f;
            // vector images: the band sums on column pairs (sum w I_b, and on
            // the first step sum I_b), folded per tile
            f2 psw[NB], psa[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) psw[b] = psa[b] = f2_pack(0.0f, 0.0f);
            auto vrows = [&](auto full_tag) {
                constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
                for (int i = 0; i < P - 1; ++i) ldh(r_first + i, rg[i]);
#pragma unroll
                for (int k = 0; k < RPW; ++k) {
                    ldh(r_first + k + P - 1, rg[(k + P - 1) % P]);
                    const int ro = r_first + k;
                    if (FULL || k < rv) {
                        float v[4], w[4];
#pragma unroll
                        for (int jp = 0; jp < 2; ++jp) {
                            f2 acc = f2_mul(tp2[0], rg[(k + RAD) % P][jp]);
#pragma unroll
                            for (int q = 1; q <= RAD; ++q)
                                acc = f2_fma(tp2[q],
                                             f2_add(rg[(k + RAD - q) % P][jp],
                                                    rg[(k + RAD + q) % P][jp]),
                                             acc);
                            f2_unpack(acc, v[2 * jp], v[2 * jp + 1]);
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j) w[j] = v[j] >= 0.0f ? 1.0f : -1.0f;
                        if (st_ok) {
                            if (store_bin)
                                S::st4(dst + k * pitch, w[0], w[1], w[2], w[3]);
                            else
                                S::st4(dst + k * pitch, v[0], v[1], v[2], v[3]);
                        }
                        if (count_flips) {
                            const uint4 sw =
                                *reinterpret_cast<const uint4 *>(sign_w + 4 * (ro + RAD));
                            const uint32_t wd[4] = {sw.x, sw.y, sw.z, sw.w};
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                nflip += (okf[j] != 0.0f) &&
                                         ((w[j] > 0.0f) != (((wd[j] >> lane) & 1u) != 0));
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j) fcnt = fmaf(w[j], okf[j], fcnt);
                        if (!EDGE && !MB) {
                            // outside the image the staged data is zero; halo
                            // lanes drop their sums below
                            const float4 d4 = S::ld4(dl + (ro + RAD) * G::DATA_W);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                fsw[0] = fmaf(comp(d4, j), w[j], fsw[0]);
                                fsa[0] += comp(d4, j);
                            }
                        }
                        if constexpr (MB) {
                            const f2 w01 = f2_pack(w[0], w[1]), w23 = f2_pack(w[2], w[3]);
#pragma unroll
                            for (int b = 0; b < NB; ++b) {
                                const float4 e = lds4(reinterpret_cast<const float *>(dl) +
                                                      b * G::PLANE + ro * G::DATA_W);
                                const f2 e01 = f2_pack(e.x, e.y), e23 = f2_pack(e.z, e.w);
                                psw[b] = f2_fma(e23, w23, f2_fma(e01, w01, psw[b]));
                                if (need_sa) psa[b] = f2_add(psa[b], f2_add(e01, e23));
                            }
                        }
                    }
                }
            };
            if (rv == RPW)
                vrows(std::true_type{});
            else
                vrows(std::false_type{});
            if (!EDGE && lane_out) {
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    if (MB) {
                        float lo, hi;
                        f2_unpack(psw[b], lo, hi);
                        sw_x[b] += lse_fix(__fadd_rn(lo, hi), fix_k);
                        if (need_sa) {
                            f2_unpack(psa[b], lo, hi);
                            sa_x[b] += lse_fix(__fadd_rn(lo, hi), fix_k);
                        }
                    } else {
                        sw_x[b] += lse_fix(fsw[b], fix_k);
                        sa_x[b] += lse_fix(fsa[b], fix_k);
                    }
                }
            }
            int cv = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) cv += okf[j] != 0.0f ? 1 : 0;
            cnt2 += __float2int_rn(fcnt) + cv * rv;          // int, widened
        }
        // every thread read the last claim before this tile's first barrier
        if (tid == 0) s_next = QUEUE ? ncta + (int)claim : t + ncta;
        __syncthreads();
        const int tn = s_next;
        if (tid == 0 && tn < n_tiles) load_tile(tn);
        // the data term does not change between steps: the next step's
        // first data box is in flight while the grid meets at its barrier
        if (PERSIST && tid == 0 && tn >= n_tiles && ps->prefetch) load_data(cta);
        par ^= 1u;
        t = tn;
    }
    if (NW == 4 && a.pdl) allow_next_grid();
    if (failed) {
        if (tid == 0) atomicOr(&st->status_bits, LSE_SBIT_TIMEOUT);
        // drain the copies in flight (bounded) before the CTA may exit
        wait_bar(bar_phi, par);
        wait_bar(bar_dat, par);
    }
    // the CTA's exact sums, added to the step's slot of the state record
    long long v[2 * NB + 2];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        v[b] = sw_x[b];
        v[NB + b] = sa_x[b];
    }
    v[2 * NB] = cnt2 / 2;
    v[2 * NB + 1] = nflip;
    lse_cta_sum_i64<2 * NB + 2, NW>(v);
    long long *slot = st->acc[PERSIST ? ps->slot : 0];
    auto add_sums = [&]() {
        unsigned long long *sl = reinterpret_cast<unsigned long long *>(slot);
        if (!EDGE) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                atomicAdd(sl + LSE_ACC_SW + b, (unsigned long long)v[b]);
                if (!MB || need_sa) atomicAdd(sl + LSE_ACC_SA + b, (unsigned long long)v[NB + b]);
            }
        }
        atomicAdd(sl + LSE_ACC_NP, (unsigned long long)v[2 * NB]);
        if (v[2 * NB + 1]) atomicAdd(sl + LSE_ACC_FL, (unsigned long long)v[2 * NB + 1]);
    };
    if constexpr (PERSIST) {
        // ps is in shared memory: one writer (the caller synchronises)
        if (tid == 0) {
            ps->par = par;
            ps->issued = (!failed && ps->prefetch) ? 1 : 0;
            add_sums();
        }
        return failed;
    }

    // the fields the last CTA's finalisation reads, fetched while the sums
    // are added
    __shared__ int s_last;
    LseStatePre pre;
    if (tid == 0) {
        pre = lse_state_pre(st);
        add_sums();
        __threadfence();
        s_last = atomicAdd(&st->ticket, 1u) == (unsigned int)ncta - 1;
    }
    __syncthreads();
    if (!s_last) return failed;
    if (tid == 0) {
        __threadfence();
        // the totals, and the slot and the queue cleared for the next step
        unsigned long long *sl = reinterpret_cast<unsigned long long *>(slot);
        const long long sw = (long long)atomicExch(sl + LSE_ACC_SW, 0ull);
        const long long sa = (long long)atomicExch(sl + LSE_ACC_SA, 0ull);
        const long long np = (long long)atomicExch(sl + LSE_ACC_NP, 0ull);
        const long long fl = (long long)atomicExch(sl + LSE_ACC_FL, 0ull);
        if (QUEUE) *queue = 0;
        LseAcc t;
        lse_fix_totals(sw, sa, np, fl, fix_k, t);
        lse_step_finalize(a, t, pre);
    }
    return failed;
}

template <int KIND_EDGE, int RAD, bool FAST, class T, int NW>
__global__ void __launch_bounds__(TileGeo<RAD, T, NW>::THREADS, TileGeo<RAD, T, NW>::MIN_BLOCKS)
step_tile_kernel(const __grid_constant__ StepArgs a,
                 const __grid_constant__ CUtensorMap phi_map,
                 const __grid_constant__ CUtensorMap data_map)
{
    if (NW == 4 && a.pdl) wait_prior_grid();
    tile_step<KIND_EDGE, RAD, FAST, T, NW>(a, &phi_map, &data_map, blockIdx.x, gridDim.x);
}

// FAST: the steady state of a re-initialising evolution.
__host__ __device__ inline bool is_fast(const StepArgs &a)
{
    return a.binary_in && a.store_bin && !a.count_flips && !a.binarise_in;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier of the persistent evolution: arrival `target` - 1 of the
// counter st->grid_bar (zeroed by the prologue) waits until `target` CTAs
// have arrived.  The step's stores of the LSF (generic proxy) are ordered
// before the arrival and the next step's TMA reads (async proxy) after the
// wait, with the proxy fences on both sides.  Bounded: gives up after
// LSE_WAIT_LIMIT polls or LSE_WAIT_NS, or as soon as another CTA has set an
// abort bit, and then sets TIMEOUT.  Block-uniform result.
__device__ __forceinline__ bool grid_barrier(LseDevState *st, unsigned int target)
{
    __shared__ int s_go;
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __threadfence();
        atomicAdd(&st->grid_bar, 1u);
        bool ok = false;
        const uint32_t t0 = global_ns_lo();
        for (uint32_t i = 0; i < LSE_WAIT_LIMIT; ++i) {
            if (ld_acquire_u32(&st->grid_bar) >= target) {
                ok = true;
                break;
            }
            if ((i & 31u) == 31u) {
                if (*reinterpret_cast<volatile unsigned int *>(&st->status_bits) &
                    LSE_SBIT_ABORT)
                    break;
                if (global_ns_lo() - t0 > (uint32_t)LSE_WAIT_NS) break;
            }
        }
        if (!ok) atomicOr(&st->status_bits, LSE_SBIT_TIMEOUT);
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        s_go = ok ? 1 : 0;
    }
    __syncthreads();
    return s_go != 0;
}

// Coefficients of a step of the persistent evolution (every CTA holds them).
struct PersistCoef {
    float coef, mid;            // Eq. 18: t = coef (d - mid) (region), coef d (edge)
    double norm;                // M of the step (region)
    int zero;                   // the step's force is zero (degenerate rule)
};

// The end of step n in thread 0 of every CTA of the persistent evolution:
// the grid-wide sums `t` over the new LSF give its statistics (Eq. 15) and
// the next step's coefficients (Eq. 17, one band), with the arithmetic of
// lse_step_finalize, so that one launch per step and the persistent
// evolution agree bit for bit.  CTA 0 also records them in the state
// record.  Returns whether the early stop ends the evolution here.
template <bool EDGE>
__device__ __forceinline__ bool persist_finalize(const StepArgs &a, int n, const LseAcc &t,
                                                 PersistCoef &c, double imin, double imax,
                                                 bool record)
{
    LseDevState *st = a.st;
    unsigned int bits = t.bits;
    const bool done = a.early_thresh > 0.0 && (double)t.flips < a.early_thresh;
    if (!EDGE) {
        if (c.zero) bits |= LSE_SBIT_DEGENERATE;
        const double norm_used = c.zero ? 0.0 : c.norm;
        const long long np = t.n_plus, nm = a.npix - np;
        double cp, cm, al, md;
        lse_band_coeffs(t.sp[0], t.sm[0], np, nm, cp, cm, al, md);
        const double contrast = fmax(0.0, fabs(cp - cm));
        const double scale = fmax(0.0, fabs(cp) + fabs(cm));
        int zero = (np == 0 || nm == 0 || contrast <= LSE_CONTRAST_TOL * scale);
        double norm = 0.0;
        float a0 = 0.0f;
        if (!zero && !lse_norm_one_band(cp, cm, al, imin, imax, a.dt, norm, a0)) {
            zero = 1;
            norm = 0.0;
        }
        c.coef = zero ? 0.0f : a0;
        c.mid = __double2float_rn(md);
        c.norm = norm;
        c.zero = zero;
        if (record) {
            st->norm_used = norm_used;
            st->run_sp[0] = t.sp[0];
            st->run_sm[0] = t.sm[0];
            st->c_plus[0] = cp;
            st->c_minus[0] = cm;
            st->alpha[0] = al;
            st->mid[0] = md;
            st->af[0] = __double2float_rn(al);
            st->m[0] = c.mid;
            st->area_plus = np;
            st->norm = norm;
            for (int b = 0; b < LSE_MAXB; ++b) st->a[b] = 0.0f;
            if (!zero) st->a[0] = a0;
            st->zero_force = zero;
        }
    } else if (record) {
        st->area_plus = t.n_plus;
    }
    if (record) {
        st->last_flips = t.flips;
        st->iterations_run = n + 1;
        st->last_buf = (n + 1) & 1;
        if (bits) atomicOr(&st->status_bits, bits);
        if (done) st->done = 1;
    }
    return done;
}

// Thread 0, between steps of a persistent evolution: the phi box of tile t
// for the coming step, issued as soon as the grid barrier has made the last
// step's LSF visible, so that its copy overlaps the step's finalisation
// (tile_step then issues nothing for its first tile: TilePersist::issued).
template <int RAD, class T, int NW, int NB>
__device__ __forceinline__ void issue_phi_box(const StepArgs &a, const CUtensorMap *pm, int t)
{
    using G = TileGeo<RAD, T, NW, NB>;
    extern __shared__ float smem_f[];
    const uint32_t sm0 = smem_u32(smem_f);
    const int sb = (int)(((128u - (sm0 & 127u)) & 127u) >> 2);
    const int ty = t / a.n_strips;
    const int xs = (t - ty * a.n_strips) * G::USEFUL - 4 * G::HL;
    const int ys = ty * G::TH - (RAD + 1);
    tma_box(sm0 + 4u * (uint32_t)(sb + G::PHI_OFF), pm, xs - 4, ys,
            sm0 + 4u * (uint32_t)(sb + 32), (uint32_t)G::PHI_BYTES);
}

// At the end of a persistent evolution: the boxes issued for a step that did
// not run are waited for (bounded) before the CTA exits.
__device__ __forceinline__ void drain_issued(const TilePersist &pc)
{
    extern __shared__ float smem_f[];
    const uint32_t sm0 = smem_u32(smem_f);
    const int sb = (int)(((128u - (sm0 & 127u)) & 127u) >> 2);
    const uint32_t bar_phi = sm0 + 4u * (uint32_t)(sb + 32);
    if (pc.issued >= 1) wait_bar(bar_phi + 8u, pc.par);
    if (pc.issued >= 2) wait_bar(bar_phi, pc.par);
}

// Thread 0 of every CTA after the barrier of step n: the step's totals
// (slot n mod 3) and the next coefficients; CTA 0 records them and clears
// the slot and the tile queue of step n - 1 (every CTA read that slot
// before it arrived at this barrier) for step n + 2.  A function of its
// own: inline, its FP64 code pushed the tile loops into register spills.
template <bool EDGE>
__device__ __noinline__ void persist_sum(const StepArgs &a, int n, PersistCoef *coef, int *done,
                                         bool record)
{
    LseDevState *st = a.st;
    const volatile long long *sl = st->acc[n % 3];
    LseAcc t;
    lse_fix_totals(sl[LSE_ACC_SW], sl[LSE_ACC_SA], sl[LSE_ACC_NP], sl[LSE_ACC_FL], st->fix_k, t);
    PersistCoef c = *coef;
    *done = persist_finalize<EDGE>(a, n, t, c, st->imin, st->imax, record) ? 1 : 0;
    *coef = c;
    if (record) {
        long long *old = st->acc[(n + 2) % 3];
        for (int j = 0; j < 12; ++j) old[j] = 0;
        st->tile_ctr[n & 1] = 0;
    }
}

// Every iteration of one image in one cooperative launch (the grid is at
// most the resident CTAs, so all of them run at once).  The CTAs take the
// step's tiles from its queue and add their exact sums to its slot of the
// state record; after the grid barrier every CTA reads the totals and makes
// the next step's coefficients itself, with the arithmetic of the last CTA
// of a one-step launch, so both give the same bits.  Each step takes the
// FAST or the general instantiation as its flags say.
template <int KIND_EDGE, int RAD, class T, int NW>
__global__ void __launch_bounds__(TileGeo<RAD, T, NW>::THREADS, TileGeo<RAD, T, NW>::MIN_BLOCKS)
evolve_tile_kernel(const __grid_constant__ EvolveArgs e,
                   const __grid_constant__ CUtensorMap phi_map0,
                   const __grid_constant__ CUtensorMap phi_map1,
                   const __grid_constant__ CUtensorMap data_map)
{
    constexpr bool EDGE = KIND_EDGE != 0;
    const StepArgs &a = e.a;
    LseDevState *st = a.st;
    // every CTA sees the prologue's record (the previous kernel in the stream)
    if (st->done || (st->status_bits & LSE_SBIT_ABORT)) return;
    // what lives from step to step is kept in shared memory, so that no
    // register is held across the steps' tile loops
    __shared__ TilePersist s_pc;
    __shared__ PersistCoef s_coef;
    __shared__ int s_done;
    const int cta = blockIdx.x, ncta = gridDim.x;
    if (threadIdx.x == 0) {
        s_coef.coef = EDGE ? a.half_dt : st->a[0];
        s_coef.mid = EDGE ? 0.0f : st->m[0];
        s_coef.norm = st->norm;
        s_coef.zero = st->zero_force;
        s_pc.par = 0u;
        s_pc.issued = 0;
        s_pc.stall_ns = a.stall_ns;
    }
    tile_smem_init<RAD, T, NW>();   // ends with a CTA barrier
    for (int n = 0; n < e.cap; ++n) {
        if (threadIdx.x == 0) {
            s_pc.f = lse_step_flags(n, e.cap, e.reinit_period, e.early_stop != 0, true);
            s_pc.phi_out = e.phi[(n + 1) & 1];
            s_pc.coef = s_coef.coef;
            s_pc.mid = s_coef.mid;
            s_pc.prefetch = n + 1 < e.cap;
            s_pc.slot = n % 3;
            s_pc.queue = n & 1;
        }
        __syncthreads();
        const CUtensorMap *pm = (n & 1) ? &phi_map1 : &phi_map0;
        const LseStepFlags f = s_pc.f;
        if (f.binary_in && f.store_bin && !f.count_flips && !f.binarise_in)
            tile_step<KIND_EDGE, RAD, true, T, NW, true>(a, pm, &data_map, cta, ncta, &s_pc);
        else
            tile_step<KIND_EDGE, RAD, false, T, NW, true>(a, pm, &data_map, cta, ncta, &s_pc);
        if (threadIdx.x == 0) s_pc.stall_ns = 0;
        if (!grid_barrier(st, (unsigned int)(n + 1) * (unsigned int)ncta)) break;
        if (*reinterpret_cast<volatile unsigned int *>(&st->status_bits) & LSE_SBIT_ABORT) break;
        if (threadIdx.x == 0) {
            if (s_pc.issued == 1) {
                issue_phi_box<RAD, T, NW, 1>(a, (n & 1) ? &phi_map0 : &phi_map1, cta);
                s_pc.issued = 2;
            }
            persist_sum<EDGE>(a, n, &s_coef, &s_done, cta == 0);
        }
        __syncthreads();
        if (s_done) break;
    }
    __syncthreads();
    drain_issued(s_pc);
}

// ---------------------------------------------------------------- vector images
// What a CTA of the vector-image evolution keeps from step to step: the
// FP64 factors of the coming step's D (Eq. 17's numerator), its normaliser
// M and whether its force is zero.
template <int NB>
struct MbCoef {
    double al[NB], md[NB];      // alpha_b = 2 (c+ - c-), mid_b = (c+ + c-) / 2
    double norm;                // M
    int zero;                   // R = 0 (degenerate rule, or M = 0)
};

// The band values of candidate i.
__device__ __forceinline__ float4 mb_cand_ld(const LseCandidates *cand, int i)
{
    const float *p = cand->val[i];
    return make_float4(__ldcg(p), __ldcg(p + 1), __ldcg(p + 2), __ldcg(p + 3));
}

// M = max over the n candidate pixels of |D| (FP64), by the whole CTA; v0
// holds candidate threadIdx.x (read beforehand, with other loads), the rest
// are read here.  The maximum does not depend on the order, so every CTA
// gets the same bits.
template <int NB>
__device__ __forceinline__ double mb_norm(const LseCandidates *cand, const MbCoef<NB> &c,
                                          int n, const float4 &v0)
{
    __shared__ double s_m[32];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 v = i == (int)threadIdx.x ? v0 : mb_cand_ld(cand, i);
        const float vb[4] = {v.x, v.y, v.z, v.w};
        double d = 0.0;
#pragma unroll
        for (int b = 0; b < NB; ++b) d = fma(c.al[b], (double)vb[b] - c.md[b], d);
        m = fmax(m, fabs(d));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, s_m[w]);
        s_m[0] = t;
    }
    __syncthreads();
    const double r = s_m[0];
    __syncthreads();
    return r;
}

// D of one pixel in FP64 with the step's factors.
template <int NB>
__device__ __forceinline__ double mb_d_at(const StepArgs &a, unsigned int pix,
                                          const MbCoef<NB> &c)
{
    const unsigned int y = pix / (unsigned int)a.W, x = pix % (unsigned int)a.W;
    double d = 0.0;
#pragma unroll
    for (int b = 0; b < NB; ++b)
        d = fma(c.al[b],
                (double)__ldg(a.data + b * a.band_stride + (size_t)y * a.pitch + x) - c.md[b], d);
    return d;
}

// The persistent evolution of a vector image (2-4 bands, FP32): every
// iteration in one cooperative launch, as evolve_tile_kernel does for one
// band.  Each step stages the NB band boxes, forms D per pixel (Eq. 17) and
// sums every band over v >= 0 exactly (Eq. 15).  M comes from the candidate
// pixels (LseCandidates); a pixel whose |D| exceeds it (in FP64: the step
// reports the largest FP32 |D| above M (1 + 2^-20)) joins the candidates and
// the step is done again from the same input LSF with that pixel's |D| as M,
// so every step uses M = max_x |D(x)|.  All CTAs decide a redo identically.
// The body, run by CTA `cta` of the `ncta` CTAs given to the image (the
// whole grid of a one-image launch, or the image's share of a group
// launch): its grid barrier counts those CTAs only.
template <int RAD, int NB, int NW>
__device__ __forceinline__ void mb_evolve(const EvolveArgs &e, const CUtensorMap *pm0,
                                          const CUtensorMap *pm1, const CUtensorMap *dmap,
                                          int cta, int ncta)
{
    const CUtensorMap &phi_map0 = *pm0;
    const CUtensorMap &phi_map1 = *pm1;
    const CUtensorMap &data_map = *dmap;
    const StepArgs &a = e.a;
    LseDevState *st = a.st;
    LseCandidates *cand = e.cand;
    if (st->done || (st->status_bits & LSE_SBIT_ABORT)) return;
    __shared__ TilePersist s_pc;
    __shared__ MbCoef<NB> s_c;
    __shared__ int s_done, s_redo;
    __shared__ long long s_tot[NB];     // sum I_b over the image (lse_fix units)
    __shared__ double s_cp[NB], s_cm[NB];
    // after each grid barrier: the step's slot, the status word and the
    // candidate count, read in one wave (each a round trip to L2 that every
    // CTA makes at once)
    __shared__ long long s_sl[LSE_ACC_MISS + 1];
    __shared__ unsigned int s_status;
    __shared__ int s_ncand;
    bool have_tot = false;
    if (threadIdx.x == 0) {
        // the prologue made the first step's statistics
        for (int b = 0; b < NB; ++b) {
            s_c.al[b] = st->alpha[b];
            s_c.md[b] = st->mid[b];
        }
        s_c.zero = st->zero_force;
        s_pc.par = 0u;
        s_pc.issued = 0;
        s_pc.stall_ns = a.stall_ns;
    }
    tile_smem_init<RAD, float, NW>();   // ends with a CTA barrier
    {
        const double m = mb_norm<NB>(cand, s_c,
                                     *reinterpret_cast<const volatile int *>(&cand->count),
                                     mb_cand_ld(cand, threadIdx.x));
        if (threadIdx.x == 0) {
            s_c.norm = m;
            if (!(m > 0.0)) s_c.zero = 1;
        }
    }
    int redos = 0;
    for (int n = 0, pass = 0; n < e.cap; ++pass) {
        if (threadIdx.x == 0) {
            s_pc.f = lse_step_flags(n, e.cap, e.reinit_period, e.early_stop != 0, true);
            s_pc.phi_out = e.phi[(n + 1) & 1];
            const bool z = s_c.zero != 0;
            s_pc.coef = z ? 0.0f : __double2float_rn(__ddiv_rn((double)a.dt, 2.0 * s_c.norm));
            s_pc.mid = 0.0f;
            for (int b = 0; b < 4; ++b) {
                s_pc.af[b] = b < NB ? __double2float_rn(s_c.al[b]) : 0.0f;
                s_pc.m[b] = b < NB ? __double2float_rn(s_c.md[b]) : 0.0f;
            }
            s_pc.thr = z ? INFINITY : __double2float_rn(s_c.norm * (1.0 + 0x1p-20));
            s_pc.prefetch = n + 1 < e.cap;
            s_pc.slot = pass % 3;
            s_pc.queue = pass & 1;
            s_pc.need_sa = have_tot ? 0 : 1;
        }
        __syncthreads();
        const CUtensorMap *pm = (n & 1) ? &phi_map1 : &phi_map0;
        const LseStepFlags f = s_pc.f;
        if (f.binary_in && f.store_bin && !f.count_flips && !f.binarise_in)
            tile_step<0, RAD, true, float, NW, true, NB>(a, pm, &data_map, cta, ncta, &s_pc);
        else
            tile_step<0, RAD, false, float, NW, true, NB>(a, pm, &data_map, cta, ncta, &s_pc);
        if (threadIdx.x == 0) s_pc.stall_ns = 0;
        if (!grid_barrier(st, (unsigned int)(pass + 1) * (unsigned int)ncta)) break;
        float4 cv;      // candidate threadIdx.x (blockDim <= LSE_MB_CAND)
        {
            const int tid = threadIdx.x;
            const volatile long long *slv = st->acc[pass % 3];
            if (tid <= LSE_ACC_MISS)
                s_sl[tid] = slv[tid];
            else if (tid == LSE_ACC_MISS + 1)
                s_status = *reinterpret_cast<volatile unsigned int *>(&st->status_bits);
            else if (tid == LSE_ACC_MISS + 2)
                s_ncand = *reinterpret_cast<const volatile int *>(&cand->count);
            cv = mb_cand_ld(cand, tid);
        }
        __syncthreads();
        if (s_status & LSE_SBIT_ABORT) break;
        const long long *sl = s_sl;
        if (threadIdx.x == 0) {
            const unsigned long long miss = (unsigned long long)sl[LSE_ACC_MISS];
            bool redo = false;
            const bool more = n + 1 < e.cap;
            if (miss && !s_c.zero && redos < 16) {
                const unsigned int pix = 0xFFFFFFFFu - (unsigned int)(miss & 0xFFFFFFFFull);
                const double d = fabs(mb_d_at<NB>(a, pix, s_c));
                if (d > s_c.norm) {
                    // the step used too small an M: again, with this pixel's |D|
                    redo = true;
                    s_c.norm = d;
                    if (cta == 0) {
                        const int k = cand->count;
                        if (k < LSE_MB_CAND) {
                            const unsigned int y = pix / (unsigned int)a.W;
                            const unsigned int x = pix % (unsigned int)a.W;
                            for (int b = 0; b < 4; ++b)
                                cand->val[k][b] =
                                    b < NB ? a.data[b * a.band_stride + (size_t)y * a.pitch + x]
                                           : 0.0f;
                            cand->count = k + 1;
                        }
                        cand->redone += 1;
                    }
                }
            }
            s_redo = redo ? 1 : 0;
            s_done = 0;
            // the coming step's first phi box: this step again, or the next
            if (s_pc.issued == 1 && (redo || more)) {
                issue_phi_box<RAD, float, NW, NB>(
                    a, ((redo ? n : n + 1) & 1) ? &phi_map1 : &phi_map0, cta);
                s_pc.issued = 2;
            }
        }
        __syncthreads();
        if (!s_redo && threadIdx.x < NB) {
            // the new LSF's statistics (Eq. 15), one band per thread (FP64
            // has a long latency on this part); sum I_b over the image is
            // that of the first step, whose tiles sum it the same way
            const int b = threadIdx.x;
            if (!have_tot) s_tot[b] = sl[LSE_ACC_SA + b];
            const long long np = sl[LSE_ACC_NP], nm = a.npix - np;
            const long long sw = sl[LSE_ACC_SW + b], sa = s_tot[b];
            const int k = st->fix_k;
            const double sp = ldexp((double)(sa + sw), -(k + 1));
            const double sm = ldexp((double)(sa - sw), -(k + 1));
            double al, md;
            lse_band_coeffs(sp, sm, np, nm, s_cp[b], s_cm[b], al, md);
            s_c.al[b] = al;      // the finished step's factors are read no more
            s_c.md[b] = md;
            if (cta == 0) {
                st->run_sp[b] = sp;
                st->run_sm[b] = sm;
                st->c_plus[b] = s_cp[b];
                st->c_minus[b] = s_cm[b];
                st->alpha[b] = al;
                st->mid[b] = md;
            }
        }
        have_tot = have_tot || !s_redo;
        __syncthreads();
        if (threadIdx.x == 0) {
            if (!s_redo) {
                // norm and zero of s_c are still those of the finished step
                const long long np = sl[LSE_ACC_NP], nm = a.npix - np;
                double contrast = 0.0, scale = 0.0;
                for (int b = 0; b < NB; ++b) {
                    contrast = fmax(contrast, fabs(s_cp[b] - s_cm[b]));
                    scale = fmax(scale, fabs(s_cp[b]) + fabs(s_cm[b]));
                }
                MbCoef<NB> nc = s_c;
                nc.zero = (np == 0 || nm == 0 || contrast <= LSE_CONTRAST_TOL * scale);
                nc.norm = 0.0;
                const bool done = a.early_thresh > 0.0 && (double)sl[LSE_ACC_FL] < a.early_thresh;
                if (cta == 0) {
                    st->norm_used = s_c.zero ? 0.0 : s_c.norm;
                    st->area_plus = np;
                    st->last_flips = sl[LSE_ACC_FL];
                    st->iterations_run = n + 1;
                    st->last_buf = (n + 1) & 1;
                    st->zero_force = nc.zero;
                    if (s_c.zero) atomicOr(&st->status_bits, LSE_SBIT_DEGENERATE);
                    if (done) st->done = 1;
                }
                s_c = nc;
                s_done = done ? 1 : 0;
                redos = 0;
            } else {
                ++redos;
            }
            if (cta == 0) {
                // the slot and queue of pass - 1, read by every CTA before
                // it arrived here, are cleared for pass + 2
                long long *old = st->acc[(pass + 2) % 3];
                for (int j = 0; j < 12; ++j) old[j] = 0;
                st->tile_ctr[pass & 1] = 0;
            }
        }
        __syncthreads();
        if (s_redo) continue;
        if (s_done) break;
        ++n;
        if (n < e.cap) {
            // M of the next step over the candidates (one added by a redo
            // is in place: CTA 0 wrote it before this barrier)
            const double m = mb_norm<NB>(cand, s_c, s_ncand, cv);
            if (threadIdx.x == 0) {
                s_c.norm = m;
                if (!(m > 0.0)) s_c.zero = 1;
            }
        }
    }
    __syncthreads();
    drain_issued(s_pc);
}

template <int RAD, int NB, int NW>
__global__ void __launch_bounds__(TileGeo<RAD, float, NW, NB>::THREADS,
                                  TileGeo<RAD, float, NW, NB>::MIN_BLOCKS)
evolve_mb_kernel(const __grid_constant__ EvolveArgs e,
                 const __grid_constant__ CUtensorMap phi_map0,
                 const __grid_constant__ CUtensorMap phi_map1,
                 const __grid_constant__ CUtensorMap data_map)
{
    mb_evolve<RAD, NB, NW>(e, &phi_map0, &phi_map1, &data_map, blockIdx.x, gridDim.x);
}

// Several vector images of one band count and radius in one cooperative
// launch: CTA c works on image cta_item[c], as CTA c - cta0 of its ncta.
// Each image keeps its own state record, candidates, tile queue and grid
// barrier; the exact sums make its results those of the one-image launch.
template <int RAD, int NB, int NW>
__global__ void __launch_bounds__(TileGeo<RAD, float, NW, NB>::THREADS,
                                  TileGeo<RAD, float, NW, NB>::MIN_BLOCKS)
evolve_mb_group_kernel(const MbGroupItem *__restrict__ items, const int *__restrict__ cta_item)
{
    const MbGroupItem &it = items[cta_item[blockIdx.x]];
    mb_evolve<RAD, NB, NW>(it.e, &it.maps[0], &it.maps[1], &it.maps[2],
                           (int)blockIdx.x - it.cta0, it.ncta);
}

// CTAs of the group kernel that fit on the device at once.
template <int RAD, int NB>
int evolve_mb_group_capacity_one(int sm_count)
{
    constexpr int NW = 4;
    using G = TileGeo<RAD, float, NW, NB>;
    auto kern = evolve_mb_group_kernel<RAD, NB, NW>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::BYTES) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::THREADS, G::BYTES) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sm_count;
}

template <int RAD, int NB>
cudaError_t launch_evolve_mb_group_one(const MbGroupItem *items, const int *cta_item,
                                       int nblocks, cudaStream_t s)
{
    constexpr int NW = 4;
    using G = TileGeo<RAD, float, NW, NB>;
    auto kern = evolve_mb_group_kernel<RAD, NB, NW>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           G::BYTES);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned int)nblocks);
    cfg.blockDim = dim3(G::THREADS);
    cfg.dynamicSmemBytes = G::BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, items, cta_item);
}

template <int NB>
int evolve_mb_group_capacity(int rad, int sm_count)
{
    switch (rad) {
    case 1: return evolve_mb_group_capacity_one<1, NB>(sm_count);
    case 2: return evolve_mb_group_capacity_one<2, NB>(sm_count);
    case 3: return evolve_mb_group_capacity_one<3, NB>(sm_count);
    case 4: return evolve_mb_group_capacity_one<4, NB>(sm_count);
    case 5: return evolve_mb_group_capacity_one<5, NB>(sm_count);
    case 6: return evolve_mb_group_capacity_one<6, NB>(sm_count);
    case 7: return evolve_mb_group_capacity_one<7, NB>(sm_count);
    default: return 0;
    }
}

template <int NB>
cudaError_t launch_evolve_mb_group(int rad, const MbGroupItem *items, const int *cta_item,
                                   int nblocks, cudaStream_t s)
{
    switch (rad) {
    case 1: return launch_evolve_mb_group_one<1, NB>(items, cta_item, nblocks, s);
    case 2: return launch_evolve_mb_group_one<2, NB>(items, cta_item, nblocks, s);
    case 3: return launch_evolve_mb_group_one<3, NB>(items, cta_item, nblocks, s);
    case 4: return launch_evolve_mb_group_one<4, NB>(items, cta_item, nblocks, s);
    case 5: return launch_evolve_mb_group_one<5, NB>(items, cta_item, nblocks, s);
    case 6: return launch_evolve_mb_group_one<6, NB>(items, cta_item, nblocks, s);
    case 7: return launch_evolve_mb_group_one<7, NB>(items, cta_item, nblocks, s);
    default: return cudaErrorNotSupported;
    }
}

template <int RAD, int NB>
cudaError_t launch_evolve_mb_one(const EvolveArgs &e, const CUtensorMap &pm0,
                                 const CUtensorMap &pm1, const CUtensorMap &dm, int nblocks,
                                 int sm_count, cudaStream_t s)
{
    constexpr int NW = 4;
    using G = TileGeo<RAD, float, NW, NB>;
    auto kern = evolve_mb_kernel<RAD, NB, NW>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           G::BYTES);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::THREADS, G::BYTES);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorNotSupported;
    // every resident slot, at most one CTA per tile
    long long grid = (long long)per_sm * sm_count;
    if (grid > nblocks) grid = nblocks;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned int)grid);
    cfg.blockDim = dim3(G::THREADS);
    cfg.dynamicSmemBytes = G::BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, e, pm0, pm1, dm);
}

template <int NB>
cudaError_t launch_evolve_mb_bands(const EvolveArgs &e, const CUtensorMap &pm0,
                                   const CUtensorMap &pm1, const CUtensorMap &dm, int nblocks,
                                   int sm_count, cudaStream_t s)
{
    switch (e.a.rad) {
    case 1: return launch_evolve_mb_one<1, NB>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 2: return launch_evolve_mb_one<2, NB>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 3: return launch_evolve_mb_one<3, NB>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 4: return launch_evolve_mb_one<4, NB>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 5: return launch_evolve_mb_one<5, NB>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 6: return launch_evolve_mb_one<6, NB>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 7: return launch_evolve_mb_one<7, NB>(e, pm0, pm1, dm, nblocks, sm_count, s);
    default: return cudaErrorNotSupported;
    }
}

// Iteration n of a batch of images of one class (term, radius, storage): CTA
// blockIdx.x works on image blk_item[blockIdx.x] with that image's CTA
// count, statistics and iteration cap; its per-iteration flags are derived
// here, so the launches of a whole evolution can be captured in a graph.
template <int KIND_EDGE, int RAD, class T, int NW>
__global__ void __launch_bounds__(TileGeo<RAD, T, NW>::THREADS, TileGeo<RAD, T, NW>::MIN_BLOCKS)
step_tile_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ blk_item,
                       long long launch)
{
    const BatchItem &it = items[blk_item[blockIdx.x]];
    const long long nl = launch - it.iter0;
    if (nl < 0 || nl >= it.cap) return;
    const int n = (int)nl;
    StepArgs a = it.args;
    lse_iteration_flags(a, n, it.cap, it.reinit_period, it.early_stop != 0, true, it.phi);
    tile_step<KIND_EDGE, RAD, false, T, NW>(a, &it.phi_maps[n & 1], &it.data_map,
                                            blockIdx.x - it.start, it.nblocks);
}

// Launches a step kernel with programmatic stream serialisation: it may
// start while the previous kernel in the stream finishes, and waits for it
// in wait_prior_grid().
template <typename Kern, typename... Args>
cudaError_t launch_dependent(Kern kern, int nblocks, int threads, int smem, cudaStream_t s,
                             Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// The persistent evolution as one cooperative launch of `nblocks` CTAs;
// cudaErrorNotSupported (nothing launched) when that many CTAs cannot all be
// resident on the device's `sm_count` SMs.
template <int KIND_EDGE, int RAD, class T, int NW>
cudaError_t launch_evolve_one(const EvolveArgs &e, const CUtensorMap &pm0,
                              const CUtensorMap &pm1, const CUtensorMap &dm, int nblocks,
                              int sm_count, cudaStream_t s)
{
    using G = TileGeo<RAD, T, NW>;
    auto kern = evolve_tile_kernel<KIND_EDGE, RAD, T, NW>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           G::BYTES);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::THREADS, G::BYTES);
    if (err != cudaSuccess) return err;
    if ((long long)per_sm * sm_count < nblocks) return cudaErrorNotSupported;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(G::THREADS);
    cfg.dynamicSmemBytes = G::BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, e, pm0, pm1, dm);
}

template <int KIND_EDGE, class T, int NW>
cudaError_t launch_evolve_kind(const EvolveArgs &e, const CUtensorMap &pm0,
                               const CUtensorMap &pm1, const CUtensorMap &dm, int nblocks,
                               int sm_count, cudaStream_t s)
{
    switch (e.a.rad) {
    case 1: return launch_evolve_one<KIND_EDGE, 1, T, NW>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 2: return launch_evolve_one<KIND_EDGE, 2, T, NW>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 3: return launch_evolve_one<KIND_EDGE, 3, T, NW>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 4: return launch_evolve_one<KIND_EDGE, 4, T, NW>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 5: return launch_evolve_one<KIND_EDGE, 5, T, NW>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 6: return launch_evolve_one<KIND_EDGE, 6, T, NW>(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 7: return launch_evolve_one<KIND_EDGE, 7, T, NW>(e, pm0, pm1, dm, nblocks, sm_count, s);
    default: return cudaErrorNotSupported;
    }
}


template <int KIND_EDGE, int RAD, class T, int NW>
cudaError_t launch_tile_one(const StepArgs &a, const CUtensorMap &pm, const CUtensorMap &dm,
                            int nblocks, cudaStream_t s)
{
    using G = TileGeo<RAD, T, NW>;
    auto kern = is_fast(a) ? step_tile_kernel<KIND_EDGE, RAD, true, T, NW>
                           : step_tile_kernel<KIND_EDGE, RAD, false, T, NW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         G::BYTES);
    if (e != cudaSuccess) return e;
    if (NW == 4 && a.pdl)
        return launch_dependent(kern, nblocks, G::THREADS, G::BYTES, s, a, pm, dm);
    kern<<<nblocks, G::THREADS, G::BYTES, s>>>(a, pm, dm);
    return cudaGetLastError();
}

// Instantiations for one tile height (NW warps per CTA), every radius.
template <int KIND_EDGE, class T, int NW>
cudaError_t launch_tile_kind(const StepArgs &a, const CUtensorMap &pm, const CUtensorMap &dm,
                             int nblocks, cudaStream_t s)
{
    switch (a.rad) {
    case 1: return launch_tile_one<KIND_EDGE, 1, T, NW>(a, pm, dm, nblocks, s);
    case 2: return launch_tile_one<KIND_EDGE, 2, T, NW>(a, pm, dm, nblocks, s);
    case 3: return launch_tile_one<KIND_EDGE, 3, T, NW>(a, pm, dm, nblocks, s);
    case 4: return launch_tile_one<KIND_EDGE, 4, T, NW>(a, pm, dm, nblocks, s);
    case 5: return launch_tile_one<KIND_EDGE, 5, T, NW>(a, pm, dm, nblocks, s);
    case 6: return launch_tile_one<KIND_EDGE, 6, T, NW>(a, pm, dm, nblocks, s);
    case 7: return launch_tile_one<KIND_EDGE, 7, T, NW>(a, pm, dm, nblocks, s);
    default: return cudaErrorNotSupported;
    }
}

// CTAs per SM the tile form runs at for a radius and tile height (its
// launch bounds).
inline int tile_blocks_per_sm(int rad, int nw) { return (rad <= 4 ? 24 : 16) / nw; }

template <int KIND_EDGE, int RAD, class T, int NW>
cudaError_t launch_tile_batch_one(const BatchItem *items, const int *blk_item, long long n,
                                  int nblocks, cudaStream_t s)
{
    using G = TileGeo<RAD, T, NW>;
    auto kern = step_tile_batch_kernel<KIND_EDGE, RAD, T, NW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         G::BYTES);
    if (e != cudaSuccess) return e;
    kern<<<nblocks, G::THREADS, G::BYTES, s>>>(items, blk_item, n);
    return cudaGetLastError();
}

template <int KIND_EDGE, class T, int NW>
cudaError_t launch_tile_batch(int rad, const BatchItem *items, const int *blk_item, long long n,
                              int nblocks, cudaStream_t s)
{
    switch (rad) {
    case 1: return launch_tile_batch_one<KIND_EDGE, 1, T, NW>(items, blk_item, n, nblocks, s);
    case 2: return launch_tile_batch_one<KIND_EDGE, 2, T, NW>(items, blk_item, n, nblocks, s);
    case 3: return launch_tile_batch_one<KIND_EDGE, 3, T, NW>(items, blk_item, n, nblocks, s);
    case 4: return launch_tile_batch_one<KIND_EDGE, 4, T, NW>(items, blk_item, n, nblocks, s);
    case 5: return launch_tile_batch_one<KIND_EDGE, 5, T, NW>(items, blk_item, n, nblocks, s);
    case 6: return launch_tile_batch_one<KIND_EDGE, 6, T, NW>(items, blk_item, n, nblocks, s);
    case 7: return launch_tile_batch_one<KIND_EDGE, 7, T, NW>(items, blk_item, n, nblocks, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace lse_tile
