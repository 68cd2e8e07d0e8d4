// lse_step_tile_region1.cu -- instantiations of the tile-form step for the
// single-band region term (Eq. 17), FP32 storage.
#include "lse_step_tile.cuh"

namespace lse_detail {

cudaError_t launch_step_tile_region1(const StepArgs &a, const CUtensorMap &pm,
                                     const CUtensorMap &dm, int nblocks, cudaStream_t s)
{
    return lse_tile::launch_tile_kind<0, float>(a, pm, dm, nblocks, s);
}

int step_tile_blocks_per_sm(int rad) { return lse_tile::tile_blocks_per_sm(rad); }

cudaError_t launch_step_tile_batch_region1(int rad, const BatchItem *items, const int *blk_item, long long n,
                     int nblocks, cudaStream_t s)
{
    return lse_tile::launch_tile_batch<0>(rad, items, blk_item, n, nblocks, s);
}

}  // namespace lse_detail
