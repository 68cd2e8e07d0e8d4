// lse_step_tile_f16_edge_nw8.cu -- instantiations of the tile-form step for the edge term E = g (Eq. 14),
// F16 storage of phi and the data term, 8 warps per CTA (64-row
// tiles), every radius 1..7: alone (FAST and general) and batched.
#include "lse_step_tile.cuh"

namespace lse_detail {

cudaError_t launch_step_tile_f16_edge_nw8(const StepArgs &a, const CUtensorMap &pm,
                                          const CUtensorMap &dm, int nblocks, cudaStream_t s)
{
    return lse_tile::launch_tile_kind<1, __half, 8>(a, pm, dm, nblocks, s);
}

cudaError_t launch_step_tile_batch_f16_edge_nw8(int rad, const BatchItem *items,
                                                const int *blk_item, long long n, int nblocks,
                                                cudaStream_t s)
{
    return lse_tile::launch_tile_batch<1, __half, 8>(rad, items, blk_item, n, nblocks, s);
}

}  // namespace lse_detail
