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
// The mbarrier waits are bounded: a wait that runs out sets the TIMEOUT
// status bit, drains the loads still in flight (again bounded) and skips the
// rest of the warp's work; the CTA still reaches its reduction.
#pragma once
#include <type_traits>

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

// Bounded wait on one stage; warp-uniform result.
__device__ __forceinline__ bool wait_stage(uint32_t bar, uint32_t parity)
{
    bool ok = false;
    for (uint32_t i = 0; i < LSE_WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) {
            ok = true;
            break;
        }
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ float bin(float v) { return v >= 0.0f ? 1.0f : -1.0f; }

__device__ __forceinline__ float4 ld4(const float *p)
{
    return *reinterpret_cast<const float4 *>(p);
}

__device__ __forceinline__ float comp(const float4 &v, int j)
{
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------- kernel
template <int KIND, int RAD>
__global__ void __launch_bounds__(256, 2)
step_tma_kernel(const __grid_constant__ StepArgs a,
                const __grid_constant__ CUtensorMap phi_map,
                const __grid_constant__ CUtensorMap data_map)
{
    using G = Geo<KIND, RAD>;
    using T = KindTraits<KIND>;
    constexpr int HL = G::HL, P = G::P, S = G::S;
    constexpr int NB = T::NB;
    constexpr float kTwoRootTwo = 2.8284271247461903f;   // sqrt(8), exactly rounded

    LseDevState *st = a.st;
    if (st->done || (st->status_bits & LSE_SBIT_ABORT)) return;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem) + warp * S;
    const unsigned char *ring = smem + ((wpc * S * 8 + 127) & ~127) + warp * G::WARP_BYTES;
    const uint32_t bar0 = smem_u32(bars);
    const uint32_t ring0 = smem_u32(ring);

    const int H = a.H, W = a.W, B = (KIND == K_REGION_MB) ? a.B : 1;
    const int th = a.th, NR = th + 2 * RAD + 2;
    const int gw = blockIdx.x * wpc + warp;
    const int NW = gridDim.x * wpc;
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
    const bool binarise = a.binarise_in != 0;
    const bool count_flips = a.count_flips != 0;

    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(bar0 + 8 * s, 1);
        fence_mbar_init();
    }
    __syncwarp();

    auto item_origin = [&](int k, int &xs, int &ys) {
        const int item = gw + k * NW;
        const int rb = item / a.n_strips;
        xs = (item - rb * a.n_strips) * G::USEFUL - 4 * HL;
        ys = rb * th - (RAD + 1);
    };

    // producer: the same bookkeeping in every lane, lane 0 issues the copies
    int p_seq = 0, p_stage = 0, p_rr = 0, p_k = 0, p_xs = 0, p_y = 0;
    if (my_items > 0) item_origin(0, p_xs, p_y);
    auto issue_upto = [&](int limit) {
        if (limit > total_seq - 1) limit = total_seq - 1;
        if (p_seq > limit) return;
        if (lane == 0) fence_proxy_async();
        while (p_seq <= limit) {
            if (lane == 0) {
                const uint32_t bar = bar0 + 8 * p_stage;
                const uint32_t dst = ring0 + p_stage * G::STAGE;
                mbar_expect_tx(bar, tx_bytes);
                tma_load_2d(dst + NB * kDataSlot, &phi_map, p_xs - 4, p_y, bar);
                if (KIND == K_REGION_MB)
                    tma_load_3d(dst, &data_map, p_xs, p_y, 0, bar);
                else
                    tma_load_2d(dst, &data_map, p_xs, p_y, bar);
            }
            ++p_seq;
            ++p_y;
            p_stage = (p_stage + 1 == S) ? 0 : p_stage + 1;
            if (++p_rr == NR) {
                p_rr = 0;
                if (++p_k < my_items) item_origin(p_k, p_xs, p_y);
            }
        }
    };
    // consumer: waits in sequence order
    int w_seq = 0, w_stage = 0;
    uint32_t w_par = 0;
    bool failed = false;
    auto wait_upto = [&](int q) {
        while (!failed && w_seq <= q) {
            if (!wait_stage(bar0 + 8 * w_stage, w_par)) {
                failed = true;     // the drain below waits for this row again
                break;
            }
            ++w_seq;
            if (++w_stage == S) {
                w_stage = 0;
                w_par ^= 1u;
            }
        }
        return !failed;
    };
    auto phi_at = [&](int stage) -> const float * {
        return reinterpret_cast<const float *>(ring + stage * G::STAGE + NB * kDataSlot);
    };
    auto data_at = [&](int stage, int b) -> const float * {
        return reinterpret_cast<const float *>(ring + stage * G::STAGE + b * kDataSlot);
    };

    int cnt = 0, nflip = 0;
    float fsp[NB], fsm[NB];
    double dsp[NB], dsm[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        fsp[b] = fsm[b] = 0.0f;
        dsp[b] = dsm[b] = 0.0;
    }
    const bool lane_out = lane >= HL && lane < 32 - HL;

    // One item: stream its NR rows.  FAST is the hot specialisation: the
    // item and its halo lie inside the image, phi is binary (the previous
    // step re-initialised) and sign changes are not counted.  Everything
    // else (image borders, a real-valued phi, flip counting) takes the
    // general instantiation, so the hot loop stays small.
    auto run_item = [&](int base, int xs, int ys, auto fast_tag) {
        constexpr bool FAST = decltype(fast_tag)::value;
        const int x0 = xs + 4 * lane;
        const bool interior = FAST || (xs >= 1 && xs + 128 < W && ys >= 0 && ys + NR - 1 < H);
        const bool bin_in = FAST || binarise;
        const bool flips = !FAST && count_flips;
        int s1 = w_stage - 1;      // stage of the newest waited row (row 1)
        if (s1 < 0) s1 += S;
        int s0 = s1 - 1;
        if (s0 < 0) s0 += S;
        float4 p0 = ld4(phi_at(s0) + 4 + 4 * lane);
        float4 pp = ld4(phi_at(s1) + 4 + 4 * lane);
        if (bin_in) {
            p0 = make_float4(bin(p0.x), bin(p0.y), bin(p0.z), bin(p0.w));
            pp = make_float4(bin(pp.x), bin(pp.y), bin(pp.z), bin(pp.w));
        }
        float4 pm = p0;
        float ring_h[P][4];
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) ring_h[i][j] = 0.0f;

        for (int r0 = 1; r0 <= NR - 2 && !failed; r0 += P) {
#pragma unroll
            for (int kk = 0; kk < P; ++kk) {
                const int r = r0 + kk;
                if (r > NR - 2 || failed) continue;
                __syncwarp();
                issue_upto(base + (r > RAD ? r - RAD : 0) + S - 1);
                if (!wait_upto(base + r + 1)) continue;
                // stages of rows r + 1, r and r - RAD
                int sn = w_stage - 1;
                if (sn < 0) sn += S;
                int sr = sn - 1;
                if (sr < 0) sr += S;
                int so = sn - 1 - RAD;
                if (so < 0) so += S;
                pm = p0;
                p0 = pp;
                pp = ld4(phi_at(sn) + 4 + 4 * lane);
                if (bin_in) pp = make_float4(bin(pp.x), bin(pp.y), bin(pp.z), bin(pp.w));
                // x-neighbours of this lane's four columns in row r
                float lft = __shfl_up_sync(0xffffffffu, p0.w, 1);
                float rgt = __shfl_down_sync(0xffffffffu, p0.x, 1);
                if (lane == 0) {
                    lft = phi_at(sr)[3];
                    if (bin_in) lft = bin(lft);
                }
                if (lane == 31) {
                    rgt = phi_at(sr)[132];
                    if (bin_in) rgt = bin(rgt);
                }
                // data term factor t = 0.5 dt R
                float t[4];
                if (KIND == K_EDGE) {
                    const float4 g4 = ld4(data_at(sr, 0) + 4 * lane);
#pragma unroll
                    for (int j = 0; j < 4; ++j) t[j] = half_dt * comp(g4, j);
                } else {
                    const float4 d4 = ld4(data_at(sr, 0) + 4 * lane);
#pragma unroll
                    for (int j = 0; j < 4; ++j) t[j] = coef[0] * (comp(d4, j) - mid[0]);
                    if (KIND == K_REGION_MB) {
#pragma unroll
                        for (int b = 1; b < NB; ++b) {
                            if (b < B) {
                                const float4 e4 = ld4(data_at(sr, b) + 4 * lane);
#pragma unroll
                                for (int j = 0; j < 4; ++j)
                                    t[j] = fmaf(coef[b], comp(e4, j) - mid[b], t[j]);
                            }
                        }
                    }
                }
                // u = phi + t * 2|grad phi|
                const float c[6] = {lft, p0.x, p0.y, p0.z, p0.w, rgt};
                float u[4];
                if (interior) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float dx = c[j + 2] - c[j];
                        const float dy = comp(pp, j) - comp(pm, j);
                        const float q = fmaf(dx, dx, dy * dy);
                        float s2;
                        if (FAST)      // binary phi: q in {0, 4, 8}, sqrt exactly
                            s2 = q > 6.0f ? kTwoRootTwo : 0.5f * q;
                        else
                            s2 = sqrtf(q);
                        u[j] = fmaf(t[j], s2, c[j + 1]);
                    }
                } else {
                    const int y = ys + r;
                    const bool yin = y >= 0 && y < H;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int x = x0 + j;
                        float dx, dy;
                        if (W == 1) dx = 0.0f;
                        else if (x == 0) dx = 2.0f * (c[j + 2] - c[j + 1]);
                        else if (x == W - 1) dx = 2.0f * (c[j + 1] - c[j]);
                        else dx = c[j + 2] - c[j];
                        if (H == 1) dy = 0.0f;
                        else if (y == 0) dy = 2.0f * (comp(pp, j) - c[j + 1]);
                        else if (y == H - 1) dy = 2.0f * (c[j + 1] - comp(pm, j));
                        else dy = comp(pp, j) - comp(pm, j);
                        const bool in = yin && x >= 0 && x < W;
                        u[j] = in ? fmaf(t[j], sqrtf(fmaf(dx, dx, dy * dy)), c[j + 1]) : 0.0f;
                    }
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
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float h = tp[0] * U[4 * HL + j];
#pragma unroll
                    for (int q = 1; q <= RAD; ++q)
                        h = fmaf(tp[q], U[4 * HL + j - q] + U[4 * HL + j + q], h);
                    ring_h[kk][j] = h;
                }
                if (r < 2 * RAD + 1) continue;
                // vertical pass and output of row r - RAD
                float v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float acc = tp[0] * ring_h[(kk - RAD + P) % P][j];
#pragma unroll
                    for (int q = 1; q <= RAD; ++q)
                        acc = fmaf(tp[q],
                                   ring_h[(kk - RAD - q + 2 * P) % P][j] +
                                       ring_h[(kk - RAD + q + P) % P][j],
                                   acc);
                    v[j] = acc;
                }
                const int yo = ys + r - RAD;
                if (!lane_out || (!FAST && yo >= H)) continue;
                float *dst = a.phi_out + (size_t)yo * a.pitch + x0;
                const bool full = FAST || x0 + 3 < W;
                if (full) {
                    *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (x0 + j < W) dst[j] = v[j];
                }
                float4 old4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (flips) old4 = ld4(phi_at(so) + 4 + 4 * lane);
                float dsel[NB][4];
                if (T::REGION) {
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        if (b < B) {
                            const float4 e4 = ld4(data_at(so, b) + 4 * lane);
#pragma unroll
                            for (int j = 0; j < 4; ++j) dsel[b][j] = comp(e4, j);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool ok = full || x0 + j < W;
                    const bool pos = ok && v[j] >= 0.0f;
                    cnt += pos;
                    if (flips) nflip += ok && (v[j] >= 0.0f) != (comp(old4, j) >= 0.0f);
                    if (T::REGION) {
#pragma unroll
                        for (int b = 0; b < NB; ++b) {
                            if (b < B) {
                                const float d = ok ? dsel[b][j] : 0.0f;
                                const float sel = pos ? d : 0.0f;
                                fsp[b] += sel;
                                fsm[b] += d - sel;
                            }
                        }
                    }
                }
            }
            // fold this period's FP32 sums into FP64
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                dsp[b] += (double)fsp[b];
                dsm[b] += (double)fsm[b];
                fsp[b] = fsm[b] = 0.0f;
            }
        }
    };

    for (int k = 0; k < my_items && !failed; ++k) {
        const int base = k * NR;
        int xs, ys;
        item_origin(k, xs, ys);
        __syncwarp();   // all lanes are done with the previous item's stages
        issue_upto(base + S - 1);
        if (!wait_upto(base + 1)) break;
        const bool fast = binarise && !count_flips && xs >= 1 && xs + 128 < W &&
                          ys >= 0 && ys + NR - 1 < H;
        if (fast)
            run_item(base, xs, ys, std::true_type{});
        else
            run_item(base, xs, ys, std::false_type{});
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
        acc.sp[b] = dsp[b];
        acc.sm[b] = dsm[b];
    }
    acc.n_plus = cnt;
    acc.flips = nflip;
    const int nb = T::REGION ? B : 0;
    LseAcc r;
    lse_cta_reduce(acc, nb, &r);
    if (!lse_publish_and_ticket(r, nb, a.partials, st)) return;
    LseAcc tot;
    lse_sum_partials(a.partials, gridDim.x, nb, &tot);
    if (threadIdx.x == 0) lse_step_finalize(a, tot);
}

// ------------------------------------------------------------ launch
template <int KIND, int RAD>
int smem_bytes(int wpc)
{
    using G = Geo<KIND, RAD>;
    return 128 + ((wpc * G::S * 8 + 127) & ~127) + wpc * G::WARP_BYTES;
}

template <int KIND, int RAD>
cudaError_t launch_one(const StepArgs &a, const CUtensorMap &pm,
                       const CUtensorMap &dm, int nblocks, int wpc,
                       cudaStream_t s)
{
    const int smem = smem_bytes<KIND, RAD>(wpc);
    cudaError_t e = cudaFuncSetAttribute(step_tma_kernel<KIND, RAD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    step_tma_kernel<KIND, RAD><<<nblocks, 32 * wpc, smem, s>>>(a, pm, dm);
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
