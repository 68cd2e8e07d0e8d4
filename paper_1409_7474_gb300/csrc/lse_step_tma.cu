// lse_step_tma.cu -- work decomposition and dispatch of the fused step
// kernels: the streaming form (lse_step_tma.cuh, any band count) and the tile
// form (lse_step_tile.cuh, one band or the edge term); one instantiation file
// per form and data term.
#include "lse_step_tma.cuh"

namespace lse_detail {

cudaError_t launch_step_tma_region1(const StepArgs &, const CUtensorMap &,
                                   const CUtensorMap &, int, int, cudaStream_t);
cudaError_t launch_step_tma_edge(const StepArgs &, const CUtensorMap &,
                                   const CUtensorMap &, int, int, cudaStream_t);
cudaError_t launch_step_tma_multiband(const StepArgs &, const CUtensorMap &,
                                   const CUtensorMap &, int, int, cudaStream_t);
int step_tma_warp_bytes_region1(int rad);
int step_tma_warp_bytes_edge(int rad);
int step_tma_warp_bytes_multiband(int rad);
// Tile-form instantiations, one file per storage type, term and tile
// height (lse_step_tile_<storage>_<term>_nw<warps>.cu).
#define LSE_TILE_DECL(SUF)                                                              \
    cudaError_t launch_step_tile_##SUF(const StepArgs &, const CUtensorMap &,           \
                                       const CUtensorMap &, int, cudaStream_t);         \
    cudaError_t launch_step_tile_batch_##SUF(int, const BatchItem *, const int *,       \
                                             long long, int, cudaStream_t);
LSE_TILE_DECL(f32_region_nw8)
LSE_TILE_DECL(f32_region_nw4)
LSE_TILE_DECL(f32_edge_nw8)
LSE_TILE_DECL(f32_edge_nw4)
LSE_TILE_DECL(bf16_region_nw8)
LSE_TILE_DECL(bf16_region_nw4)
LSE_TILE_DECL(bf16_edge_nw8)
LSE_TILE_DECL(bf16_edge_nw4)
LSE_TILE_DECL(f16_region_nw8)
LSE_TILE_DECL(f16_region_nw4)
LSE_TILE_DECL(f16_edge_nw8)
LSE_TILE_DECL(f16_edge_nw4)
#undef LSE_TILE_DECL
// The persistent evolution, one file per storage type, term and tile height
// (lse_evolve_tile_<storage>_<term>_nw<warps>.cu).
#define LSE_EVOLVE_DECL(SUF)                                                           \
    cudaError_t launch_evolve_tile_##SUF(const EvolveArgs &, const CUtensorMap &,      \
                                         const CUtensorMap &, const CUtensorMap &, int, \
                                         int, cudaStream_t);
LSE_EVOLVE_DECL(f32_region_nw8)
LSE_EVOLVE_DECL(f32_region_nw4)
LSE_EVOLVE_DECL(f32_edge_nw8)
LSE_EVOLVE_DECL(f32_edge_nw4)
LSE_EVOLVE_DECL(bf16_region_nw8)
LSE_EVOLVE_DECL(bf16_region_nw4)
LSE_EVOLVE_DECL(bf16_edge_nw8)
LSE_EVOLVE_DECL(bf16_edge_nw4)
LSE_EVOLVE_DECL(f16_region_nw8)
LSE_EVOLVE_DECL(f16_region_nw4)
LSE_EVOLVE_DECL(f16_edge_nw8)
LSE_EVOLVE_DECL(f16_edge_nw4)
#undef LSE_EVOLVE_DECL
cudaError_t launch_evolve_mb2(const EvolveArgs &, const CUtensorMap &, const CUtensorMap &,
                              const CUtensorMap &, int, int, cudaStream_t);
cudaError_t launch_evolve_mb3(const EvolveArgs &, const CUtensorMap &, const CUtensorMap &,
                              const CUtensorMap &, int, int, cudaStream_t);
cudaError_t launch_evolve_mb4(const EvolveArgs &, const CUtensorMap &, const CUtensorMap &,
                              const CUtensorMap &, int, int, cudaStream_t);
cudaError_t launch_evolve_mb_group2(int, const MbGroupItem *, const int *, int, cudaStream_t);
cudaError_t launch_evolve_mb_group3(int, const MbGroupItem *, const int *, int, cudaStream_t);
cudaError_t launch_evolve_mb_group4(int, const MbGroupItem *, const int *, int, cudaStream_t);
int evolve_mb_group_capacity2(int, int);
int evolve_mb_group_capacity3(int, int);
int evolve_mb_group_capacity4(int, int);

}  // namespace lse_detail

namespace {

int kind_of(int term, int B)
{
    if (term == LSE_TERM_EDGE) return lse_tma::K_EDGE;
    return B == 1 ? lse_tma::K_REGION1 : lse_tma::K_REGION_MB;
}

}  // namespace

namespace lse_detail {

bool plan_step_tma(int H, int W, int B, int term, int rad, int sm_count,
                   StepArgs *a, int *nblocks, int *warps_per_block)
{
    if (rad < 1 || rad > 7) return false;
    if (term == LSE_TERM_REGION && (B < 1 || B > 4)) return false;
    const int kind = kind_of(term, B);
    int per_warp = kind == lse_tma::K_EDGE ? step_tma_warp_bytes_edge(rad)
                 : kind == lse_tma::K_REGION1 ? step_tma_warp_bytes_region1(rad)
                                              : step_tma_warp_bytes_multiband(rad);
    // 2 CTAs of up to 8 warps per SM (16 warps of up to 128 registers): each
    // CTA gets 113 KB of the SM's 228 KB less 1 KB reserved; 6 KB of that is
    // the reduction's static shared memory
    const int budget = (113 - 6) * 1024 - 256;
    int wpc = budget / per_warp;
    if (wpc > 8) wpc = 8;
    if (wpc < 1) return false;
    const int hl = (rad + 3) / 4;
    const int useful = 128 - 8 * hl;
    const int n_strips = (W + useful - 1) / useful;
    const int max_warps = sm_count * 2 * wpc;
    int per_strip = max_warps / n_strips;
    if (per_strip < 1) per_strip = 1;
    int th = (H + per_strip - 1) / per_strip;
    if (th < 16) th = 16;
    // the kernel streams th + 2 rad u-rows per item in whole ring periods of
    // 2 rad + 1 rows: round th up so that th + 2 rad is a multiple of it
    const int period = 2 * rad + 1;
    th = ((th + 2 * rad + period - 1) / period) * period - 2 * rad;
    const int n_rowblocks = (H + th - 1) / th;
    const int n_items = n_strips * n_rowblocks;
    a->useful = useful;
    a->n_strips = n_strips;
    a->n_rowblocks = n_rowblocks;
    a->th = th;
    a->n_items = n_items;
    int blocks = (n_items + wpc - 1) / wpc;
    if (blocks > sm_count * 2) blocks = sm_count * 2;
    *nblocks = blocks;
    *warps_per_block = wpc;
    return true;
}

cudaError_t launch_step_tma(const StepArgs &a, const CUtensorMap &phi_map,
                            const CUtensorMap &data_map, int nblocks,
                            int warps_per_block, cudaStream_t s)
{
    switch (kind_of(a.term, a.B)) {
    case lse_tma::K_EDGE:
        return launch_step_tma_edge(a, phi_map, data_map, nblocks, warps_per_block, s);
    case lse_tma::K_REGION1:
        return launch_step_tma_region1(a, phi_map, data_map, nblocks, warps_per_block, s);
    default:
        return launch_step_tma_multiband(a, phi_map, data_map, nblocks, warps_per_block, s);
    }
}

// Tile form: tiles of (8 nw - 2 rad) output rows x (128 - 8 ceil(rad / 4))
// output columns (nw = warps per CTA, 8 or 4), walked by as many CTAs as fit
// on the SMs at once: 24 warps per SM for rad <= 4, else 16 (the kernels'
// launch bounds).
bool tile_boxes_aligned(int rad, int elem_bytes)
{
    // tile k's boxes start at column k * useful - 4 hl - 4 (phi, and the
    // 16-bit data box) and, for FP32, k * useful - 4 hl (the data box); a
    // tiled TMA copy must start on 16 bytes, so every such column must be a
    // multiple of 16 / elem_bytes.  16-bit elements with hl = 2 (radius
    // 5..7) fail: 112 k - 12 is 4 modulo 8.
    const int hl = (rad + 3) / 4;
    const int useful = 128 - 8 * hl;
    const int q = 16 / elem_bytes;
    const bool phi_ok = useful % q == 0 && (4 * hl + 4) % q == 0;
    const bool data_ok = elem_bytes == 4 ? (4 * hl) % q == 0 : true;   // 16-bit: phi's column
    return phi_ok && data_ok;
}

bool plan_step_tile(int H, int W, int B, int term, int rad, int nw, int sm_count,
                    StepArgs *a, int *nblocks)
{
    if (rad < 1 || rad > 7 || (nw != 8 && nw != 4)) return false;
    if (term == LSE_TERM_REGION && B != 1) return false;
    if (!tile_boxes_aligned(rad, a->storage == LSE_F32 ? 4 : 2)) return false;
    const int hl = (rad + 3) / 4;
    const int useful = 128 - 8 * hl;
    const int th = 8 * nw - 2 * rad;
    const int tiles_x = (W + useful - 1) / useful;
    const int tiles_y = (H + th - 1) / th;
    a->useful = useful;
    a->n_strips = tiles_x;
    a->n_rowblocks = tiles_y;
    a->th = th;
    a->n_items = tiles_x * tiles_y;
    a->nw = nw;
    int blocks = a->n_items;
    const int resident = sm_count * ((rad <= 4 ? 24 : 16) / nw);
    // every resident slot, even where the last round of tiles leaves most
    // CTAs idle: the fewest CTAs that need no more rounds (all finishing
    // together) measured 2.6 % slower at 8192x8192 -- the step needs every
    // resident warp's loads in flight
    if (blocks > resident) blocks = resident;
    *nblocks = blocks;
    // a grid smaller than the resident slots lets the next iteration's CTAs
    // start while this one finishes; a full grid would only hold slots that
    // other streams' kernels could use
    a->pdl = blocks < resident ? 1 : 0;
    return true;
}

namespace {

typedef cudaError_t (*TileFn)(const StepArgs &, const CUtensorMap &, const CUtensorMap &, int,
                              cudaStream_t);
typedef cudaError_t (*TileBatchFn)(int, const BatchItem *, const int *, long long, int,
                                   cudaStream_t);

// [storage: f32, f16, bf16][term: region, edge][nw: 8, 4]
const TileFn kTile[3][2][2] = {
    {{launch_step_tile_f32_region_nw8, launch_step_tile_f32_region_nw4},
     {launch_step_tile_f32_edge_nw8, launch_step_tile_f32_edge_nw4}},
    {{launch_step_tile_f16_region_nw8, launch_step_tile_f16_region_nw4},
     {launch_step_tile_f16_edge_nw8, launch_step_tile_f16_edge_nw4}},
    {{launch_step_tile_bf16_region_nw8, launch_step_tile_bf16_region_nw4},
     {launch_step_tile_bf16_edge_nw8, launch_step_tile_bf16_edge_nw4}}};
const TileBatchFn kTileBatch[3][2][2] = {
    {{launch_step_tile_batch_f32_region_nw8, launch_step_tile_batch_f32_region_nw4},
     {launch_step_tile_batch_f32_edge_nw8, launch_step_tile_batch_f32_edge_nw4}},
    {{launch_step_tile_batch_f16_region_nw8, launch_step_tile_batch_f16_region_nw4},
     {launch_step_tile_batch_f16_edge_nw8, launch_step_tile_batch_f16_edge_nw4}},
    {{launch_step_tile_batch_bf16_region_nw8, launch_step_tile_batch_bf16_region_nw4},
     {launch_step_tile_batch_bf16_edge_nw8, launch_step_tile_batch_bf16_edge_nw4}}};

typedef cudaError_t (*EvolveFn)(const EvolveArgs &, const CUtensorMap &, const CUtensorMap &,
                                const CUtensorMap &, int, int, cudaStream_t);
const EvolveFn kEvolve[3][2][2] = {
    {{launch_evolve_tile_f32_region_nw8, launch_evolve_tile_f32_region_nw4},
     {launch_evolve_tile_f32_edge_nw8, launch_evolve_tile_f32_edge_nw4}},
    {{launch_evolve_tile_f16_region_nw8, launch_evolve_tile_f16_region_nw4},
     {launch_evolve_tile_f16_edge_nw8, launch_evolve_tile_f16_edge_nw4}},
    {{launch_evolve_tile_bf16_region_nw8, launch_evolve_tile_bf16_region_nw4},
     {launch_evolve_tile_bf16_edge_nw8, launch_evolve_tile_bf16_edge_nw4}}};

bool tile_index(int storage, int term, int nw, int *si, int *ti, int *ni)
{
    *si = storage == LSE_F32 ? 0 : storage == LSE_F16 ? 1 : storage == LSE_BF16 ? 2 : -1;
    *ti = term == LSE_TERM_EDGE ? 1 : 0;
    *ni = nw == 8 ? 0 : nw == 4 ? 1 : -1;
    return *si >= 0 && *ni >= 0;
}

}  // namespace

cudaError_t launch_step_tile(const StepArgs &a, const CUtensorMap &phi_map,
                             const CUtensorMap &data_map, int nblocks, cudaStream_t s)
{
    int si, ti, ni;
    // a vector image steps on its D plane like the edge term on g
    if (!tile_index(a.storage, a.mb_split ? LSE_TERM_EDGE : a.term, a.nw, &si, &ti, &ni))
        return cudaErrorNotSupported;
    return kTile[si][ti][ni](a, phi_map, data_map, nblocks, s);
}

cudaError_t launch_evolve_tile(const EvolveArgs &e, const CUtensorMap &pm0,
                               const CUtensorMap &pm1, const CUtensorMap &dm, int nblocks,
                               int sm_count, cudaStream_t s)
{
    int si, ti, ni;
    if (e.a.mb_split || !tile_index(e.a.storage, e.a.term, e.a.nw, &si, &ti, &ni))
        return cudaErrorNotSupported;
    return kEvolve[si][ti][ni](e, pm0, pm1, dm, nblocks, sm_count, s);
}

cudaError_t launch_evolve_mb(const EvolveArgs &e, const CUtensorMap &pm0,
                             const CUtensorMap &pm1, const CUtensorMap &dm, int nblocks,
                             int sm_count, cudaStream_t s)
{
    switch (e.a.B) {
    case 2: return launch_evolve_mb2(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 3: return launch_evolve_mb3(e, pm0, pm1, dm, nblocks, sm_count, s);
    case 4: return launch_evolve_mb4(e, pm0, pm1, dm, nblocks, sm_count, s);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_evolve_mb_group(int B, int rad, const MbGroupItem *items,
                                   const int *cta_item, int nblocks, cudaStream_t s)
{
    switch (B) {
    case 2: return launch_evolve_mb_group2(rad, items, cta_item, nblocks, s);
    case 3: return launch_evolve_mb_group3(rad, items, cta_item, nblocks, s);
    case 4: return launch_evolve_mb_group4(rad, items, cta_item, nblocks, s);
    default: return cudaErrorNotSupported;
    }
}

int evolve_mb_group_capacity(int B, int rad, int sm_count)
{
    switch (B) {
    case 2: return evolve_mb_group_capacity2(rad, sm_count);
    case 3: return evolve_mb_group_capacity3(rad, sm_count);
    case 4: return evolve_mb_group_capacity4(rad, sm_count);
    default: return 0;
    }
}

cudaError_t launch_step_tile_batch(int storage, int term, int nw, int rad,
                                   const BatchItem *items, const int *blk_item, long long n,
                                   int nblocks, cudaStream_t s)
{
    int si, ti, ni;
    if (!tile_index(storage, term, nw, &si, &ti, &ni)) return cudaErrorNotSupported;
    return kTileBatch[si][ti][ni](rad, items, blk_item, n, nblocks, s);
}

}  // namespace lse_detail
