// lse_step_tile.cuh -- the fused LSE iteration, tile form (single-band
// region term and edge term, TS = 3..15).
//
// Same arithmetic as the streaming kernel (lse_step_tma.cuh): per pixel
//   u = phi + dt R |grad phi|                        (Eq. 18)
//   v = G_sigma * u                                  (Table I step 4)
// then v (or sign(v) on re-initialising steps, Table I step 3) is stored and
// the next iteration's region sums are accumulated (Eq. 15).
//
// Work decomposition.  A persistent CTA of 8 warps walks a static list of
// tiles of TH output rows x (128 - 8 HL) output columns.  Per tile:
//   1. TMA stages phi on the tile + (RAD + 1) halo rows and 4 halo columns
//      (136 x (TH + 2 RAD + 2) floats) and the data term on the tile + RAD
//      halo rows (128 x (TH + 2 RAD)); ghost columns are patched in for
//      tiles on the image's left/right edge;
//   2. each warp takes every 8th u-row: lane l computes u for 4 columns in
//      registers, the horizontal Gaussian pass takes neighbouring lanes' u
//      by shuffles, and the result h goes to shared memory;
//   3. each warp takes TH / 8 consecutive output rows: lane l slides a
//      2 RAD + 1 row register window of h down its 4 columns, stores v and
//      accumulates the statistics.
// The next tile's phi is loaded while step 3 runs (its buffer is free after
// step 2) and its data term right after; a second CTA on the SM overlaps
// the rest.  Per-row bookkeeping is per tile, not per row.
//
// Waits on the TMA mbarriers are bounded (LSE_WAIT_LIMIT polls): a wait
// that runs out sets the TIMEOUT status bit, drains the copies in flight
// (bounded) and stops the CTA's tile loop; the CTA still reaches its
// reduction.
#pragma once

#include "lse_reduce.cuh"

namespace lse_tile {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kURows = 64;            // u / h rows per tile (TH + 2 RAD)
constexpr int kPhiW = 136;            // staged phi columns
constexpr int kDataW = 128;           // staged data columns

template <int RAD>
struct TileGeo {
    static constexpr int HL = (RAD + 3) / 4;
    static constexpr int USEFUL = 128 - 8 * HL;                 // output columns
    static constexpr int TH = kURows - 2 * RAD;                 // output rows
    static constexpr int PHI_ROWS = kURows + 2;
    static constexpr int ROWS_PER_WARP = (TH + kWarps - 1) / kWarps;
    static constexpr int PHI_FLOATS = PHI_ROWS * kPhiW;
    static constexpr int DATA_FLOATS = kURows * kDataW;
    static constexpr int H_FLOATS = kURows * kDataW;
    // shared memory: [lut 32][2 mbarriers (4 floats), pad to 32][phi][data][h]
    static constexpr int PHI_OFF = 64;
    static constexpr int DATA_OFF = PHI_OFF + ((PHI_FLOATS + 31) & ~31);
    static constexpr int H_OFF = DATA_OFF + DATA_FLOATS;
    static constexpr int FLOATS = H_OFF + H_FLOATS;
    static constexpr int BYTES = FLOATS * 4 + 128;              // + alignment slack
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

// Bounded wait; block-uniform result (every thread polls).
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity)
{
    bool ok = false;
    for (uint32_t i = 0; i < LSE_WAIT_LIMIT; ++i)
        if (try_wait(bar, parity)) {
            ok = true;
            break;
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

__device__ __forceinline__ float bin(float v) { return v >= 0.0f ? 1.0f : -1.0f; }

__device__ __forceinline__ float comp(const float4 &v, int j)
{
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

template <int KIND_EDGE, int RAD, bool BIN>
__global__ void __launch_bounds__(kThreads, 2)
step_tile_kernel(const __grid_constant__ StepArgs a,
                 const __grid_constant__ CUtensorMap phi_map,
                 const __grid_constant__ CUtensorMap data_map)
{
    using G = TileGeo<RAD>;
    constexpr int HL = G::HL, TH = G::TH, P = 2 * RAD + 1;
    constexpr bool EDGE = KIND_EDGE != 0;

    LseDevState *st = a.st;
    if (st->done || (st->status_bits & LSE_SBIT_ABORT)) return;

    extern __shared__ float smem_f[];
    const uint32_t sm0 = smem_u32(smem_f);
    const int sb = (int)(((128u - (sm0 & 127u)) & 127u) >> 2);   // aligned base
    float *lut = smem_f + sb;
    float *phi_s = smem_f + sb + G::PHI_OFF;
    float *dat_s = smem_f + sb + G::DATA_OFF;
    float *h_s = smem_f + sb + G::H_OFF;
    const uint32_t bar_phi = sm0 + 4u * (uint32_t)(sb + 32);
    const uint32_t bar_dat = bar_phi + 8;
    const uint32_t phi_dst = sm0 + 4u * (uint32_t)(sb + G::PHI_OFF);
    const uint32_t dat_dst = sm0 + 4u * (uint32_t)(sb + G::DATA_OFF);
    constexpr uint32_t kPhiBytes = G::PHI_FLOATS * 4;
    constexpr uint32_t kDatBytes = G::DATA_FLOATS * 4;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int H = a.H, W = a.W;
    const int tiles_x = a.n_strips, n_tiles = a.n_items;

    if (tid < 32) {
        // sqrt table indexed by bits(q) >> 21 & 31 for q in {0,4,8,16,20,32}
        const float q = tid == 4 ? 4.f : tid == 8 ? 8.f : tid == 12 ? 16.f
                      : tid == 13 ? 20.f : tid == 16 ? 32.f : 0.f;
        lut[tid] = sqrtf(q);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_phi) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_dat) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    float tp[RAD + 1];
#pragma unroll
    for (int k = 0; k <= RAD; ++k) tp[k] = a.taps[k];
    const float coef = EDGE ? a.half_dt : st->a[0];
    const float mid = EDGE ? 0.0f : st->m[0];
    const bool binarise_in = !BIN && a.binarise_in != 0;
    const bool count_flips = a.count_flips != 0;
    const bool store_bin = a.store_bin != 0;

    auto origin = [&](int t, int &xs, int &ys) {
        const int ty = t / tiles_x;
        xs = (t - ty * tiles_x) * G::USEFUL - 4 * HL;   // first staged data column
        ys = ty * TH - (RAD + 1);                        // first staged phi row
    };
    auto load_phi = [&](int t) {
        int xs, ys;
        origin(t, xs, ys);
        tma_box(phi_dst, &phi_map, xs - 4, ys, bar_phi, kPhiBytes);
    };
    auto load_dat = [&](int t) {
        int xs, ys;
        origin(t, xs, ys);
        tma_box(dat_dst, &data_map, xs, ys + 1, bar_dat, kDatBytes);
    };

    int t = blockIdx.x;
    if (tid == 0 && t < n_tiles) {
        load_phi(t);
        load_dat(t);
    }
    uint32_t par = 0;
    bool failed = false;

    long long cnt2 = 0;
    int nflip = 0;
    double dsw = 0.0, dsa = 0.0;
    const bool lane_out = lane >= HL && lane < 32 - HL;

    for (; t < n_tiles; t += gridDim.x) {
        int xs, ys;
        origin(t, xs, ys);
        const int x0 = xs + 4 * lane;
        if (!wait_bar(bar_phi, par) || !wait_bar(bar_dat, par)) {
            failed = true;
            break;
        }
        // ghost columns for a binary phi on the image's left/right edge
        const bool ghost_l = xs <= 0;
        const bool ghost_r = xs <= W - 1 && W - 1 < xs + 128;
        if (BIN && (ghost_l || ghost_r)) {
            for (int rr = tid; rr < G::PHI_ROWS; rr += kThreads) {
                float *row = phi_s + rr * kPhiW;
                if (ghost_l) {
                    const float f0 = row[4 - xs];
                    const float f1 = W > 1 ? row[5 - xs] : f0;
                    row[3 - xs] = 2.0f * f0 - f1;
                }
                if (ghost_r) {
                    const float fe = row[W + 3 - xs];
                    const float fd = W > 1 ? row[W + 2 - xs] : fe;
                    row[W + 4 - xs] = 2.0f * fe - fd;
                }
            }
            // the buffer is refilled by TMA later: order these writes first
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
        // per-column masks of this lane
        float inf[4];
        bool oneL[4], oneR[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = x0 + j;
            inf[j] = (x >= 0 && x < W) ? 1.0f : 0.0f;
            oneL[j] = x == 0;
            oneR[j] = x == W - 1;
        }
        const bool xborder = xs < 0 || xs + 128 > W;

        // ---- u and horizontal pass: warp w takes u-rows w, w + 8, ...
#pragma unroll 2
        for (int ur = warp; ur < kURows; ur += kWarps) {
            const int y = ys + 1 + ur;
            const float *pr = phi_s + ur * kPhiW;      // rows y-1, y, y+1
            float4 m4 = *reinterpret_cast<const float4 *>(pr + 4 + 4 * lane);
            float4 c4 = *reinterpret_cast<const float4 *>(pr + kPhiW + 4 + 4 * lane);
            float4 p4 = *reinterpret_cast<const float4 *>(pr + 2 * kPhiW + 4 + 4 * lane);
            float e = pr[kPhiW + (lane == 0 ? 3 : 132)];
            if (binarise_in) {
                m4 = make_float4(bin(m4.x), bin(m4.y), bin(m4.z), bin(m4.w));
                c4 = make_float4(bin(c4.x), bin(c4.y), bin(c4.z), bin(c4.w));
                p4 = make_float4(bin(p4.x), bin(p4.y), bin(p4.z), bin(p4.w));
                e = bin(e);
            }
            float lft = __shfl_up_sync(0xffffffffu, c4.w, 1);
            float rgt = __shfl_down_sync(0xffffffffu, c4.x, 1);
            if (lane == 0) lft = e;
            if (lane == 31) rgt = e;
            float pm[4] = {m4.x, m4.y, m4.z, m4.w};
            float pp[4] = {p4.x, p4.y, p4.z, p4.w};
            const float c[6] = {lft, c4.x, c4.y, c4.z, c4.w, rgt};
            bool yin = true;
            if (y <= 0 || y >= H - 1) {                 // ghost rows, rows outside
                yin = y >= 0 && y < H;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (H == 1) {
                        pm[j] = c[j + 1];
                        pp[j] = c[j + 1];
                    } else if (y == 0) {
                        pm[j] = 2.f * c[j + 1] - pp[j];
                    } else if (y == H - 1) {
                        pp[j] = 2.f * c[j + 1] - pm[j];
                    }
                }
            }
            const float4 d4 = *reinterpret_cast<const float4 *>(dat_s + ur * kDataW + 4 * lane);
            float u[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float dx = c[j + 2] - c[j];
                if (!BIN) {
                    if (W == 1) dx = 0.0f;
                    else if (oneL[j]) dx = 2.0f * (c[j + 2] - c[j + 1]);
                    else if (oneR[j]) dx = 2.0f * (c[j + 1] - c[j]);
                }
                const float dy = pp[j] - pm[j];
                const float q = fmaf(dx, dx, dy * dy);
                const float s2 = BIN ? lut[(__float_as_uint(q) >> 21) & 31u] : sqrtf(q);
                const float tj = EDGE ? coef * comp(d4, j) : coef * (comp(d4, j) - mid);
                u[j] = fmaf(tj, s2, c[j + 1]);
            }
            if (xborder) {
#pragma unroll
                for (int j = 0; j < 4; ++j) u[j] *= inf[j];
            }
            if (!yin) {
#pragma unroll
                for (int j = 0; j < 4; ++j) u[j] = 0.0f;
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
            *reinterpret_cast<float4 *>(h_s + ur * kDataW + 4 * lane) =
                make_float4(hv[0], hv[1], hv[2], hv[3]);
        }
        __syncthreads();
        // the phi buffer is free (unless flips read it below): fetch the next tile's
        const int tn = t + gridDim.x;
        if (!count_flips && tid == 0 && tn < n_tiles) load_phi(tn);

        // ---- vertical pass: warp w takes output rows w*RPW .. +RPW-1
        {
            constexpr int RPW = G::ROWS_PER_WARP;
            const int r_first = warp * RPW;              // output row within the tile
            float win[P + RPW - 1][4];
#pragma unroll
            for (int i = 0; i < P + RPW - 1; ++i) {
                const int hr = r_first + i;               // h row (u-row index)
                if (hr < kURows) {
                    const float4 h4 = *reinterpret_cast<const float4 *>(h_s + hr * kDataW + 4 * lane);
                    win[i][0] = h4.x;
                    win[i][1] = h4.y;
                    win[i][2] = h4.z;
                    win[i][3] = h4.w;
                } else {
                    win[i][0] = win[i][1] = win[i][2] = win[i][3] = 0.0f;
                }
            }
            float fsw = 0.0f, fsa = 0.0f, fcnt = 0.0f;
#pragma unroll
            for (int k = 0; k < RPW; ++k) {
                const int ro = r_first + k;
                const int yo = ys + RAD + 1 + ro;
                if (ro >= TH || yo >= H) continue;
                float v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float acc = tp[0] * win[k + RAD][j];
#pragma unroll
                    for (int q = 1; q <= RAD; ++q)
                        acc = fmaf(tp[q], win[k + RAD - q][j] + win[k + RAD + q][j], acc);
                    v[j] = acc;
                }
                float w[4], okf[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    w[j] = v[j] >= 0.0f ? 1.0f : -1.0f;
                    okf[j] = (lane_out && x0 + j < W) ? 1.0f : 0.0f;
                }
                float *dst = a.phi_out + (size_t)yo * a.pitch + x0;
                const float s0 = store_bin ? w[0] : v[0], s1 = store_bin ? w[1] : v[1];
                const float s2 = store_bin ? w[2] : v[2], s3 = store_bin ? w[3] : v[3];
                if (lane_out) {
                    if (x0 + 3 < W) {
                        *reinterpret_cast<float4 *>(dst) = make_float4(s0, s1, s2, s3);
                    } else {
                        const float sv[4] = {s0, s1, s2, s3};
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (x0 + j < W) dst[j] = sv[j];
                    }
                }
                if (count_flips) {
                    const float4 o4 = *reinterpret_cast<const float4 *>(
                        phi_s + (ro + RAD + 1) * kPhiW + 4 + 4 * lane);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        nflip += (okf[j] != 0.0f) && ((w[j] > 0.0f) != (comp(o4, j) >= 0.0f));
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) fcnt = fmaf(w[j], okf[j], fcnt);
                if (!EDGE) {
                    const float4 d4 = *reinterpret_cast<const float4 *>(
                        dat_s + (ro + RAD) * kDataW + 4 * lane);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float d = comp(d4, j) * okf[j];
                        fsw = fmaf(d, w[j], fsw);
                        fsa += d;
                    }
                }
            }
            dsw += (double)fsw;
            dsa += (double)fsa;
            // valid output pixels of this lane in this tile
            int rows = TH;
            if (ys + RAD + 1 + TH > H) rows = H - (ys + RAD + 1);
            int rv = rows - r_first;
            rv = rv < 0 ? 0 : (rv > RPW ? RPW : rv);
            int cv = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) cv += (lane_out && x0 + j < W) ? 1 : 0;
            cnt2 += (long long)fcnt + (long long)cv * rv;
        }
        __syncthreads();
        if (tid == 0 && tn < n_tiles) {
            if (count_flips) load_phi(tn);
            load_dat(tn);
        }
        par ^= 1u;
    }
    if (failed) {
        if (tid == 0) atomicOr(&st->status_bits, LSE_SBIT_TIMEOUT);
        // drain the copies in flight (bounded) before the CTA may exit
        wait_bar(bar_phi, par);
        wait_bar(bar_dat, par);
    }

    LseAcc acc;
    acc.clear();
    acc.sp[0] = 0.5 * (dsa + dsw);
    acc.sm[0] = 0.5 * (dsa - dsw);
    acc.n_plus = cnt2 / 2;
    acc.flips = nflip;
    const int nb = EDGE ? 0 : 1;
    LseAcc r;
    lse_cta_reduce(acc, nb, &r);
    if (!lse_publish_and_ticket(r, nb, a.partials, st)) return;
    LseAcc tot;
    lse_sum_partials(a.partials, gridDim.x, nb, &tot);
    if (threadIdx.x == 0) lse_step_finalize(a, tot);
}

template <int KIND_EDGE, int RAD>
cudaError_t launch_tile_one(const StepArgs &a, const CUtensorMap &pm, const CUtensorMap &dm,
                            int nblocks, cudaStream_t s)
{
    using G = TileGeo<RAD>;
    auto kern = a.binary_in ? step_tile_kernel<KIND_EDGE, RAD, true>
                            : step_tile_kernel<KIND_EDGE, RAD, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         G::BYTES);
    if (e != cudaSuccess) return e;
    kern<<<nblocks, kThreads, G::BYTES, s>>>(a, pm, dm);
    return cudaGetLastError();
}

template <int KIND_EDGE>
cudaError_t launch_tile_kind(const StepArgs &a, const CUtensorMap &pm, const CUtensorMap &dm,
                             int nblocks, cudaStream_t s)
{
    switch (a.rad) {
    case 1: return launch_tile_one<KIND_EDGE, 1>(a, pm, dm, nblocks, s);
    case 2: return launch_tile_one<KIND_EDGE, 2>(a, pm, dm, nblocks, s);
    case 3: return launch_tile_one<KIND_EDGE, 3>(a, pm, dm, nblocks, s);
    case 4: return launch_tile_one<KIND_EDGE, 4>(a, pm, dm, nblocks, s);
    case 5: return launch_tile_one<KIND_EDGE, 5>(a, pm, dm, nblocks, s);
    case 6: return launch_tile_one<KIND_EDGE, 6>(a, pm, dm, nblocks, s);
    case 7: return launch_tile_one<KIND_EDGE, 7>(a, pm, dm, nblocks, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace lse_tile
