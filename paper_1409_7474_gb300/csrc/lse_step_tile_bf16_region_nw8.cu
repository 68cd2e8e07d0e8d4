// lse_step_tile_bf16_region_nw8.cu -- instantiations of the tile-form step for the single-band region term (Eq. 17),
// BF16 storage of phi and the data term, 8 warps per CTA (64-row
// tiles), every radius 1..7: alone (FAST and general) and batched.
#include "lse_step_tile.cuh"

namespace lse_detail {

cudaError_t launch_step_tile_bf16_region_nw8(const StepArgs &a, const CUtensorMap &pm,
                                             const CUtensorMap &dm, int nblocks, cudaStream_t s)
{
    return lse_tile::launch_tile_kind<0, __nv_bfloat16, 8>(a, pm, dm, nblocks, s);
}

cudaError_t launch_step_tile_batch_bf16_region_nw8(int rad, const BatchItem *items,
                                                   const int *blk_item, long long n, int nblocks,
                                                   cudaStream_t s)
{
    return lse_tile::launch_tile_batch<0, __nv_bfloat16, 8>(rad, items, blk_item, n, nblocks, s);
}

}  // namespace lse_detail
