// lse_step_tma.cuh -- the fused LSE iteration for sm_103a (TS = 3..15).
//
// One pass over the image per iteration computes, for every pixel,
//   u = phi + dt R |grad phi|                        (Eq. 18)
//   v = G_sigma * u                                  (Table I step 4)
// with R = D / max|D| (Eq. 17) or R = g (Eq. 14), stores v, and accumulates
// the sums that the next iteration's region statistics need (Eq. 15): count
// and intensity sums over v >= 0 and v < 0, plus the number of sign changes.
// The last CTA finalises c+/c- and the next step's coefficients.
//
// Work decomposition.  Each warp owns a vertical strip of 128 columns and a
// block of `th` output rows ("item").  Lane l holds columns xs + 4l .. +3.
// The outer `HL` lanes on each side only supply the horizontal halo of the
// Gaussian, so a strip yields 4 (32 - 2 HL) output columns.  The warp streams
// down the strip one row at a time:
//   * TMA (cp.async.bulk.tensor, zero fill outside the image) loads each
//     row of phi (136 floats: the strip plus 4 columns each side) and of the
//     data term (128 floats per band) into a per-warp ring of shared-memory
//     stages, each with its own mbarrier; lane 0 issues loads up to
//     `S - RAD - 2` rows ahead of use;
//   * phi rows y-1, y, y+1 sit in registers; u of row y is computed in
//     registers, its horizontal Gaussian pass takes the neighbouring lanes'
//     u by warp shuffles;
//   * the vertical pass keeps the last 2 RAD + 1 horizontally smoothed rows
//     in a register ring (the row loop is unrolled by the ring period so
//     every ring index is a compile-time constant);
//   * the output row (RAD rows behind) is written with 16-byte stores and
//     its statistics read phi and the data term from the ring.
// Nothing but the inputs' halo is recomputed, and HBM sees each input byte
// about once (halo rows/columns of neighbouring strips hit L2).
//
// Image borders cost no per-pixel logic: at x = 0 the listing's one-sided
// difference phi(1) - phi(0) equals the central difference against a ghost
// value phi(-1) = 2 phi(0) - phi(1) (and likewise at the last column and
// the first/last row; a dimension of size 1 gets ghosts equal to phi(0), so
// its difference is 0).  Ghost columns are written into the staged row in
// shared memory, ghost rows into the register window; u is zeroed outside
// the image by per-column masks and per-row flags.  Every item then runs
// the same code, so the work is balanced across warps.
//
// BIN instantiations read a binary LSF stored by the previous step (which
// wrote sign(v) because it re-initialised): |grad phi|^2 then takes only the
// values 0, 4, 8 (16, 20, 32 at borders) and its square root comes from a
// 17-entry table filled with sqrtf, exactly.  The other instantiation reads
// a real LSF (the first step, or a caller-chosen reinit period) and uses
// sqrtf.
//
// The mbarrier waits are bounded: a wait that runs out sets the TIMEOUT
// status bit, drains the loads still in flight (again bounded) and skips the
// rest of the warp's work; the CTA still reaches its reduction.
#pragma once
#include <type_traits>

#include "lse_f2.cuh"
#include "lse_reduce.cuh"

namespace lse_tma {

constexpr int kPhiBox = 136;       // phi floats per staged row
constexpr int kDataBox = 128;      // data floats per staged row and band
constexpr int kPhiBytes = kPhiBox * 4;
constexpr int kPhiSlot = 640;      // phi bytes per stage, 128-byte aligned
constexpr int kDataSlot = kDataBox * 4;

enum Kind { K_REGION1 = 0, K_REGION_MB = 1, K_EDGE = 2 };

template <int KIND>
struct KindTraits {
    static constexpr int NB = KIND == K_REGION_MB ? 4 : 1;   // bands staged
    static constexpr int PF = KIND == K_REGION_MB ? 4 : 5;   // rows of prefetch
    static constexpr bool REGION = KIND != K_EDGE;
};

template <int KIND, int RAD>
struct Geo {
    static constexpr int HL = (RAD + 3) / 4;
    static constexpr int USEFUL = 4 * (32 - 2 * HL);
    static constexpr int P = 2 * RAD + 1;
    static constexpr int S = RAD + 2 + KindTraits<KIND>::PF;
    static constexpr int STAGE = KindTraits<KIND>::NB * kDataSlot + kPhiSlot;
    static constexpr int WARP_BYTES = S * STAGE;
};

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
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

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map,
                                            int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map,
                                            int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z),
          "r"(bar)
        : "memory");
}

// Bounded wait on one stage; warp-uniform result.  Gives up after
// LSE_WAIT_LIMIT polls or LSE_WAIT_NS nanoseconds of %globaltimer (read
// every 256 polls, from the 256th on).
__device__ __forceinline__ bool wait_stage(uint32_t bar, uint32_t parity)
{
    bool ok = false;
    unsigned long long t0 = 0;
    for (uint32_t i = 0; i < LSE_WAIT_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) {
            ok = true;
            break;
        }
        if ((i & 255u) == 255u) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t0 == 0) t0 = t;
            else if (t - t0 > LSE_WAIT_NS) break;
        }
    }
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ float bin(float v) { return v >= 0.0f ? 1.0f : -1.0f; }

__device__ __forceinline__ float4 ld4(const float *p)
{
    return *reinterpret_cast<const float4 *>(p);
}

__device__ __forceinline__ float4 bin4(float4 v)
{
    return make_float4(bin(v.x), bin(v.y), bin(v.z), bin(v.w));
}

__device__ __forceinline__ float comp(const float4 &v, int j)
{
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------- kernel
// One step over the strips of one image, run by CTA `cta` of the `ncta`
// CTAs given to it.
template <int KIND, int RAD, bool BIN>
__device__ __forceinline__ void tma_step(const StepArgs &a, const CUtensorMap *phi_map,
                                         const CUtensorMap *data_map, int cta, int ncta)
{
    using G = Geo<KIND, RAD>;
    using T = KindTraits<KIND>;
    constexpr int HL = G::HL, P = G::P, S = G::S;
    constexpr int NB = T::NB;
    constexpr int SF = G::STAGE / 4;         // floats per stage
    constexpr int PHI = NB * kDataBox;       // float offset of phi in a stage

    LseDevState *st = a.st;
    if (st->done || (st->status_bits & LSE_SBIT_ABORT)) return;

    extern __shared__ float smem_f[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const uint32_t sm0 = smem_u32(smem_f);
    const int sbase = (int)(((128u - (sm0 & 127u)) & 127u) >> 2);
    const int lut = sbase;                                   // 32 floats
    const int ring = sbase + 32 + ((2 * wpc * S + 31) & ~31) + warp * S * SF;
    const uint32_t bar0 = sm0 + 4u * (uint32_t)(sbase + 32 + 2 * warp * S);
    const uint32_t ring0 = sm0 + 4u * (uint32_t)ring;

    if (BIN) {
        // sqrt table indexed by bits(q) >> 21 & 31 for q in {0,4,8,16,20,32}
        if (threadIdx.x < 32) {
            const int t = threadIdx.x;
            const float q = t == 4 ? 4.f : t == 8 ? 8.f : t == 12 ? 16.f
                          : t == 13 ? 20.f : t == 16 ? 32.f : 0.f;
            smem_f[lut + t] = sqrtf(q);
        }
        __syncthreads();
    }

    const int H = a.H, W = a.W, B = (KIND == K_REGION_MB) ? a.B : 1;
    const int th = a.th, NR = th + 2 * RAD + 2;
    const int n_per = (th + 2 * RAD) / P;    // u-rows per item = n_per * P
    const int gw = cta * wpc + warp;
    const int NW = ncta * wpc;
    const int my_items = a.n_items > gw ? (a.n_items - gw + NW - 1) / NW : 0;
    const int total_seq = my_items * NR;
    const uint32_t tx_bytes = kPhiBytes + kDataSlot * B;

    float tp[RAD + 1];
#pragma unroll
    for (int k = 0; k <= RAD; ++k) tp[k] = a.taps[k];
    float coef[NB], mid[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        coef[b] = T::REGION ? st->a[b] : 0.0f;
        mid[b] = T::REGION ? st->m[b] : 0.0f;
    }
    const float half_dt = a.half_dt;
    // the same constants as pairs, for the packed column-pair arithmetic
    f2 tp2[RAD + 1];
#pragma unroll
    for (int k = 0; k <= RAD; ++k) tp2[k] = f2_pack(tp[k], tp[k]);
    const f2 coef20 = f2_pack(coef[0], coef[0]), mid20 = f2_pack(mid[0], mid[0]);
    const f2 half_dt2 = f2_pack(half_dt, half_dt);
    const bool binarise_in = !BIN && a.binarise_in != 0;
    const bool count_flips = a.count_flips != 0;
    const bool store_bin = a.store_bin != 0;

    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(bar0 + 8 * s, 1);
        fence_mbar_init();
    }
    __syncwarp();

    // ---- producer: identical bookkeeping in every lane, lane 0 issues
    int p_seq = 0, p_stage = 0, p_rr = 0, p_k = 0, p_xs = 0, p_y = 0;
    auto origin = [&](int k, int &xs, int &ys) {
        const int item = gw + k * NW;
        const int rb = item / a.n_strips;
        xs = (item - rb * a.n_strips) * G::USEFUL - 4 * HL;
        ys = rb * th - (RAD + 1);
    };
    if (my_items > 0) origin(0, p_xs, p_y);
    auto issue_one = [&]() {
        if (lane == 0) {
            const uint32_t bar = bar0 + 8 * p_stage;
            const uint32_t dst = ring0 + (uint32_t)(p_stage * G::STAGE);
            fence_proxy_async();
            mbar_expect_tx(bar, tx_bytes);
            tma_load_2d(dst + PHI * 4, phi_map, p_xs - 4, p_y, bar);
            if (KIND == K_REGION_MB)
                tma_load_3d(dst, data_map, p_xs, p_y, 0, bar);
            else
                tma_load_2d(dst, data_map, p_xs, p_y, bar);
        }
        ++p_seq;
        ++p_y;
        p_stage = (p_stage + 1 == S) ? 0 : p_stage + 1;
        if (++p_rr == NR) {
            p_rr = 0;
            if (++p_k < my_items) origin(p_k, p_xs, p_y);
        }
    };
    // ---- consumer: waits strictly in order; returns the waited stage
    int w_seq = 0, w_stage = 0;
    uint32_t w_par = 0;
    bool failed = false;
    auto wait_one = [&]() -> int {
        const int sw = w_stage;
        if (!failed) {
            if (wait_stage(bar0 + 8 * sw, w_par)) {
                ++w_seq;
                if (++w_stage == S) {
                    w_stage = 0;
                    w_par ^= 1u;
                }
            } else {
                failed = true;     // the drain below waits for this row again
            }
        }
        return sw;
    };

    // per-lane sums: sum of w = sign(v) over output pixels (fsw_cnt), and per
    // band sum d and sum d w; FP32 within a ring period, compensated FP32
    // (lse_kahan_add) across periods, FP64 from the lane sums on
    long long cnt2 = 0;      // sum over items of (sum w + valid pixels)
    int nflip = 0;
    float fsw_cnt = 0.0f;
    float fsw[NB], fsa[NB];
    float ksw[NB], csw[NB], ksa[NB], csa[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        fsw[b] = fsa[b] = 0.0f;
        ksw[b] = csw[b] = ksa[b] = csa[b] = 0.0f;
    }
    const bool lane_out = lane >= HL && lane < 32 - HL;

    for (int k = 0; k < my_items && !failed; ++k) {
        const int base = k * NR;
        int xs, ys;
        origin(k, xs, ys);
        const int x0 = xs + 4 * lane;
        // per-column masks (1 or 0): u inside the image, output columns
        float inf[4], okf[4];
        bool oneL[4], oneR[4];
        int nvalid = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = x0 + j;
            inf[j] = (x >= 0 && x < W) ? 1.0f : 0.0f;
            okf[j] = (lane_out && x < W) ? 1.0f : 0.0f;
            nvalid += (lane_out && x < W) ? 1 : 0;
            oneL[j] = x == 0;
            oneR[j] = x == W - 1;
        }
        // uniform per item: does the strip touch the image's left/right edge,
        // and is every output lane's float4 inside the image?
        const bool xborder = xs < 0 || xs + 128 > W;
        const bool ragged = xs + 4 * (32 - HL) > W;
        const bool full = lane_out && x0 + 3 < W;
        const bool ghost_l = xs <= 0;                    // x = -1 in this strip
        const bool ghost_r = xs <= W - 1 && W - 1 < xs + 128;

        // ghost columns of a staged binary row (lane 0; BIN only)
        auto patch = [&](int stage) {
            if (BIN && (ghost_l || ghost_r)) {
                if (lane == 0) {
                    const int row = ring + stage * SF + PHI;
                    if (ghost_l) {
                        const float f0 = smem_f[row + 4 - xs];
                        const float f1 = W > 1 ? smem_f[row + 5 - xs] : f0;
                        smem_f[row + 3 - xs] = 2.0f * f0 - f1;
                    }
                    if (ghost_r) {
                        const float fe = smem_f[row + W + 3 - xs];
                        const float fd = W > 1 ? smem_f[row + W + 2 - xs] : fe;
                        smem_f[row + W + 4 - xs] = 2.0f * fe - fd;
                    }
                }
                __syncwarp();
            }
        };

        __syncwarp();   // every lane is done with the previous item's stages
        {
            int lim = base + S - 1;
            if (lim > total_seq - 1) lim = total_seq - 1;
            while (p_seq <= lim) issue_one();
        }
        const int s_a = wait_one();
        const int s_b = wait_one();
        patch(s_a);
        patch(s_b);
        float4 p0 = ld4(&smem_f[ring + s_a * SF + PHI + 4 + 4 * lane]);
        float4 pp = ld4(&smem_f[ring + s_b * SF + PHI + 4 + 4 * lane]);
        if (binarise_in) {
            p0 = bin4(p0);
            pp = bin4(pp);
        }
        float4 pm = p0;
        // h rows: as column pairs for the packed vertical pass (one band,
        // edge term); vector images keep the scalar ring, their band
        // constants already fill the register budget
        constexpr bool PK = KIND != K_REGION_MB;
        f2 ring_h[PK ? P : 1][2];
        float ring_s[PK ? 1 : P][4];

        // one u-row: u of row r, its horizontal pass into ring slot kk, and
        // (OUT) the vertical pass, store and statistics of row r - RAD
        auto row = [&](const int r, const int kk, const bool OUT) {
            __syncwarp();
            if (r > RAD && p_seq < total_seq && p_seq <= base + r - RAD + S - 1) issue_one();
            const int sn = wait_one();          // stage of row r + 1
            patch(sn);
            int sr = sn - 1;
            if (sr < 0) sr += S;
            int so = sn - 1 - RAD;
            if (so < 0) so += S;
            const int rowN = ring + sn * SF, rowR = ring + sr * SF, rowO = ring + so * SF;
            pm = p0;
            p0 = pp;
            pp = ld4(&smem_f[rowN + PHI + 4 + 4 * lane]);
            if (binarise_in) pp = bin4(pp);
            // x-neighbours of this lane's columns in row r
            float lft = __shfl_up_sync(0xffffffffu, p0.w, 1);
            float rgt = __shfl_down_sync(0xffffffffu, p0.x, 1);
            {
                float e = smem_f[rowR + PHI + (lane == 0 ? 3 : 132)];
                if (binarise_in) e = bin(e);
                if (lane == 0) lft = e;
                if (lane == 31) rgt = e;
            }
            // ghost rows (uniform per row)
            const int y = ys + r;
            float4 pmx = pm, ppx = pp;
            if (y <= 0 || y >= H - 1) {
                if (H == 1) {
                    pmx = p0;
                    ppx = p0;
                } else if (y == 0) {
                    pmx = make_float4(2.f * p0.x - pp.x, 2.f * p0.y - pp.y,
                                      2.f * p0.z - pp.z, 2.f * p0.w - pp.w);
                } else if (y == H - 1) {
                    ppx = make_float4(2.f * p0.x - pm.x, 2.f * p0.y - pm.y,
                                      2.f * p0.z - pm.z, 2.f * p0.w - pm.w);
                }
            }
            const bool yin = y >= 0 && y < H;
            // data term factor t = 0.5 dt R, on column pairs (each packed
            // operation rounds as its scalar form)
            // (vector images: per band in scalar form, which keeps the band
            // constants out of the register budget)
            f2 t2[2];
            if (KIND == K_EDGE) {
                const float4 g4 = ld4(&smem_f[rowR + 4 * lane]);
                t2[0] = f2_mul(half_dt2, f2_pack(g4.x, g4.y));
                t2[1] = f2_mul(half_dt2, f2_pack(g4.z, g4.w));
            } else if (KIND == K_REGION1) {
                const float4 d4 = ld4(&smem_f[rowR + 4 * lane]);
                t2[0] = f2_mul(coef20, f2_sub(f2_pack(d4.x, d4.y), mid20));
                t2[1] = f2_mul(coef20, f2_sub(f2_pack(d4.z, d4.w), mid20));
            } else {
                const float4 d4 = ld4(&smem_f[rowR + 4 * lane]);
                float t[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) t[j] = coef[0] * (comp(d4, j) - mid[0]);
#pragma unroll
                for (int b = 1; b < NB; ++b) {
                    if (b < B) {
                        const float4 e4 = ld4(&smem_f[rowR + b * kDataBox + 4 * lane]);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            t[j] = fmaf(coef[b], comp(e4, j) - mid[b], t[j]);
                    }
                }
                t2[0] = f2_pack(t[0], t[1]);
                t2[1] = f2_pack(t[2], t[3]);
            }
            // u = phi + t * 2|grad phi| (zero outside the image)
            const float c[6] = {lft, p0.x, p0.y, p0.z, p0.w, rgt};
            float dxs[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float dx = c[j + 2] - c[j];
                if (!BIN) {    // real LSF: one-sided differences by flags
                    if (W == 1) dx = 0.0f;
                    else if (oneL[j]) dx = 2.0f * (c[j + 2] - c[j + 1]);
                    else if (oneR[j]) dx = 2.0f * (c[j + 1] - c[j]);
                }
                dxs[j] = dx;
            }
            float u[4];
#pragma unroll
            for (int jp = 0; jp < 2; ++jp) {
                const int j0 = 2 * jp, j1 = 2 * jp + 1;
                if constexpr (!PK) {
                    // vector images: the scalar form of the same update
                    float tt[2];
                    f2_unpack(t2[jp], tt[0], tt[1]);
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int j = j0 + e;
                        const float dy = comp(ppx, j) - comp(pmx, j);
                        const float q = fmaf(dxs[j], dxs[j], dy * dy);
                        const float s2 = BIN ? smem_f[lut + ((__float_as_uint(q) >> 21) & 31u)]
                                             : sqrtf(q);
                        u[j] = fmaf(tt[e], s2, c[j + 1]);
                    }
                    continue;
                }
                const f2 dx = f2_pack(dxs[j0], dxs[j1]);
                const f2 dy = f2_sub(f2_pack(comp(ppx, j0), comp(ppx, j1)),
                                     f2_pack(comp(pmx, j0), comp(pmx, j1)));
                float q[2];
                f2_unpack(f2_fma(dx, dx, f2_mul(dy, dy)), q[0], q[1]);
                float s2[2];
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    s2[e] = BIN ? smem_f[lut + ((__float_as_uint(q[e]) >> 21) & 31u)]
                                : sqrtf(q[e]);
                f2_unpack(f2_fma(t2[jp], f2_pack(s2[0], s2[1]), f2_pack(c[j0 + 1], c[j1 + 1])),
                          u[j0], u[j1]);
            }
            if (xborder) {
#pragma unroll
                for (int j = 0; j < 4; ++j) u[j] *= inf[j];
            }
            if (!yin) {
#pragma unroll
                for (int j = 0; j < 4; ++j) u[j] = 0.0f;
            }
            // horizontal pass: U[c + 4 HL] = u at relative column c
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
            if constexpr (PK) {
                ring_h[kk][0] = f2_pack(hv[0], hv[1]);
                ring_h[kk][1] = f2_pack(hv[2], hv[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) ring_s[kk][j] = hv[j];
            }
            if (!OUT) return;
            // vertical pass of row r - RAD (on column pairs where packed)
            float v[4];
            if constexpr (PK) {
#pragma unroll
                for (int jp = 0; jp < 2; ++jp) {
                    f2 acc = f2_mul(tp2[0], ring_h[(kk - RAD + P) % P][jp]);
#pragma unroll
                    for (int q = 1; q <= RAD; ++q)
                        acc = f2_fma(tp2[q],
                                     f2_add(ring_h[(kk - RAD - q + 2 * P) % P][jp],
                                            ring_h[(kk - RAD + q + P) % P][jp]),
                                     acc);
                    f2_unpack(acc, v[2 * jp], v[2 * jp + 1]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float acc = tp[0] * ring_s[(kk - RAD + P) % P][j];
#pragma unroll
                    for (int q = 1; q <= RAD; ++q)
                        acc = fmaf(tp[q],
                                   ring_s[(kk - RAD - q + 2 * P) % P][j] +
                                       ring_s[(kk - RAD + q + P) % P][j],
                                   acc);
                    v[j] = acc;
                }
            }
            const int yo = ys + r - RAD;
            if (yo >= H) return;
            float *dst = a.phi_out + (size_t)yo * a.pitch + x0;
            if (store_bin) {
                // w = sign(v): the count is (sum w + valid) / 2 and the band sums
                // over v >= 0 are (sum d + sum d w) / 2 (d zero off the image)
                float w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) w[j] = v[j] >= 0.0f ? 1.0f : -1.0f;
                if (full) *reinterpret_cast<float4 *>(dst) = make_float4(w[0], w[1], w[2], w[3]);
                if (ragged && !full) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (okf[j] != 0.0f) dst[j] = w[j];
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) fsw_cnt = fmaf(w[j], okf[j], fsw_cnt);
                if (T::REGION) {
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        if (b < B) {
                            const float4 e4 = ld4(&smem_f[rowO + b * kDataBox + 4 * lane]);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float d = comp(e4, j) * okf[j];
                                fsw[b] = fmaf(d, w[j], fsw[b]);
                                fsa[b] += d;
                            }
                        }
                    }
                }
            } else {
                if (full) *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
                if (ragged && !full) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (okf[j] != 0.0f) dst[j] = v[j];
                }
                float w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) w[j] = v[j] >= 0.0f ? 1.0f : -1.0f;
                if (count_flips) {
                    const float4 o4 = ld4(&smem_f[rowO + PHI + 4 + 4 * lane]);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        nflip += (okf[j] != 0.0f) && ((w[j] > 0.0f) != (comp(o4, j) >= 0.0f));
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) fsw_cnt = fmaf(w[j], okf[j], fsw_cnt);
                if (T::REGION) {
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        if (b < B) {
                            const float4 e4 = ld4(&smem_f[rowO + b * kDataBox + 4 * lane]);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float d = comp(e4, j) * okf[j];
                                fsw[b] = fmaf(d, w[j], fsw[b]);
                                fsa[b] += d;
                            }
                        }
                    }
                }
            }
        };
        auto fold = [&]() {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                lse_kahan_add(ksw[b], csw[b], fsw[b]);
                lse_kahan_add(ksa[b], csa[b], fsa[b]);
                fsw[b] = fsa[b] = 0.0f;
            }
        };

        // rows 1 .. NR - 2 in whole ring periods; outputs start at 2 RAD + 1
        for (int per = 0; per < n_per && !failed; ++per) {
            const int r0 = 1 + per * P;
#pragma unroll
            for (int kk = 0; kk < P; ++kk) row(r0 + kk, kk, r0 + kk >= 2 * RAD + 1);
            fold();
        }
        // exact integer count: fsw_cnt holds sum w (|sum| <= 4 th) exactly;
        // rows at or beyond H produced no output
        {
            const int y0 = ys + RAD + 1;
            const int rows = H - y0 < th ? H - y0 : th;
            cnt2 += (long long)fsw_cnt + (long long)nvalid * (rows > 0 ? rows : 0);
        }
        fsw_cnt = 0.0f;
    }
    if (failed) {
        if (lane == 0) atomicOr(&st->status_bits, LSE_SBIT_TIMEOUT);
        // drain the loads still in flight (bounded) before the CTA may exit
        while (w_seq < p_seq) {
            wait_stage(bar0 + 8 * w_stage, w_par);
            ++w_seq;
            if (++w_stage == S) {
                w_stage = 0;
                w_par ^= 1u;
            }
        }
    }

    LseAcc acc;
    acc.clear();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const double dsw = lse_kahan_value(ksw[b], csw[b]);
        const double dsa = lse_kahan_value(ksa[b], csa[b]);
        acc.sp[b] = 0.5 * (dsa + dsw);
        acc.sm[b] = 0.5 * (dsa - dsw);
    }
    acc.n_plus = cnt2 / 2;
    acc.flips = nflip;
    const int nb = T::REGION ? B : 0;
    LseAcc r;
    lse_cta_reduce(acc, nb, &r);
    if (!lse_publish_and_ticket_at(r, nb, a.partials, st, cta, ncta)) return;
    LseAcc tot;
    lse_sum_partials(a.partials, ncta, nb, &tot);
    if (threadIdx.x == 0) lse_step_finalize(a, tot);
}

template <int KIND, int RAD, bool BIN>
__global__ void __launch_bounds__(256, 2)
step_tma_kernel(const __grid_constant__ StepArgs a,
                const __grid_constant__ CUtensorMap phi_map,
                const __grid_constant__ CUtensorMap data_map)
{
    tma_step<KIND, RAD, BIN>(a, &phi_map, &data_map, blockIdx.x, gridDim.x);
}

// Iteration n of a batch of images of one class (term, bands, radius); see
// step_tile_batch_kernel.
template <int KIND, int RAD>
__global__ void __launch_bounds__(256, 2)
step_tma_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ blk_item,
                      long long launch)
{
    const BatchItem &it = items[blk_item[blockIdx.x]];
    const long long nl = launch - it.iter0;
    if (nl < 0 || nl >= it.cap) return;
    const int n = (int)nl;
    StepArgs a = it.args;
    lse_iteration_flags(a, n, it.cap, it.reinit_period, it.early_stop != 0, true, it.phi);
    tma_step<KIND, RAD, false>(a, &it.phi_maps[n & 1], &it.data_map, blockIdx.x - it.start,
                               it.nblocks);
}

// ------------------------------------------------------------ launch
template <int KIND, int RAD>
int smem_bytes(int wpc)
{
    using G = Geo<KIND, RAD>;
    // alignment slack + sqrt table + mbarriers + per-warp rings
    return 128 + 128 + ((wpc * G::S * 8 + 127) & ~127) + wpc * G::WARP_BYTES;
}

template <int KIND, int RAD>
cudaError_t launch_one(const StepArgs &a, const CUtensorMap &pm,
                       const CUtensorMap &dm, int nblocks, int wpc,
                       cudaStream_t s)
{
    const int smem = smem_bytes<KIND, RAD>(wpc);
    auto kern = a.binary_in ? step_tma_kernel<KIND, RAD, true>
                            : step_tma_kernel<KIND, RAD, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    kern<<<nblocks, 32 * wpc, smem, s>>>(a, pm, dm);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_kind(const StepArgs &a, const CUtensorMap &pm,
                        const CUtensorMap &dm, int nblocks, int wpc,
                        cudaStream_t s)
{
    switch (a.rad) {
    case 1: return launch_one<KIND, 1>(a, pm, dm, nblocks, wpc, s);
    case 2: return launch_one<KIND, 2>(a, pm, dm, nblocks, wpc, s);
    case 3: return launch_one<KIND, 3>(a, pm, dm, nblocks, wpc, s);
    case 4: return launch_one<KIND, 4>(a, pm, dm, nblocks, wpc, s);
    case 5: return launch_one<KIND, 5>(a, pm, dm, nblocks, wpc, s);
    case 6: return launch_one<KIND, 6>(a, pm, dm, nblocks, wpc, s);
    case 7: return launch_one<KIND, 7>(a, pm, dm, nblocks, wpc, s);
    default: return cudaErrorNotSupported;
    }
}

template <int KIND, int RAD>
cudaError_t launch_batch_one(const BatchItem *items, const int *blk_item, long long n, int nblocks,
                             int wpc, cudaStream_t s)
{
    const int smem = smem_bytes<KIND, RAD>(wpc);
    auto kern = step_tma_batch_kernel<KIND, RAD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    kern<<<nblocks, 32 * wpc, smem, s>>>(items, blk_item, n);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_batch_kind(int rad, const BatchItem *items, const int *blk_item, long long n,
                              int nblocks, int wpc, cudaStream_t s)
{
    switch (rad) {
    case 1: return launch_batch_one<KIND, 1>(items, blk_item, n, nblocks, wpc, s);
    case 2: return launch_batch_one<KIND, 2>(items, blk_item, n, nblocks, wpc, s);
    case 3: return launch_batch_one<KIND, 3>(items, blk_item, n, nblocks, wpc, s);
    case 4: return launch_batch_one<KIND, 4>(items, blk_item, n, nblocks, wpc, s);
    case 5: return launch_batch_one<KIND, 5>(items, blk_item, n, nblocks, wpc, s);
    case 6: return launch_batch_one<KIND, 6>(items, blk_item, n, nblocks, wpc, s);
    case 7: return launch_batch_one<KIND, 7>(items, blk_item, n, nblocks, wpc, s);
    default: return cudaErrorNotSupported;
    }
}

template <int KIND>
int warp_bytes_for(int rad)
{
    switch (rad) {
    case 1: return Geo<KIND, 1>::WARP_BYTES + Geo<KIND, 1>::S * 8;
    case 2: return Geo<KIND, 2>::WARP_BYTES + Geo<KIND, 2>::S * 8;
    case 3: return Geo<KIND, 3>::WARP_BYTES + Geo<KIND, 3>::S * 8;
    case 4: return Geo<KIND, 4>::WARP_BYTES + Geo<KIND, 4>::S * 8;
    case 5: return Geo<KIND, 5>::WARP_BYTES + Geo<KIND, 5>::S * 8;
    case 6: return Geo<KIND, 6>::WARP_BYTES + Geo<KIND, 6>::S * 8;
    case 7: return Geo<KIND, 7>::WARP_BYTES + Geo<KIND, 7>::S * 8;
    default: return 0;
    }
}

}  // namespace lse_tma
