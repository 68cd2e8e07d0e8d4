// lse_step_tile_edge.cu -- instantiations of the tile-form step for the edge
// term E = g (Eq. 14), FP32 storage.
#include "lse_step_tile.cuh"

namespace lse_detail {

cudaError_t launch_step_tile_edge(const StepArgs &a, const CUtensorMap &pm,
                                  const CUtensorMap &dm, int nblocks, cudaStream_t s)
{
    return lse_tile::launch_tile_kind<1, float>(a, pm, dm, nblocks, s);
}

cudaError_t launch_step_tile_batch_edge(int rad, const BatchItem *items, const int *blk_item, long long n,
                     int nblocks, cudaStream_t s)
{
    return lse_tile::launch_tile_batch<1>(rad, items, blk_item, n, nblocks, s);
}

}  // namespace lse_detail
