// lse_step_tile_bf16_edge_nw4.cu -- instantiations of the tile-form step for the edge term E = g (Eq. 14),
// BF16 storage of phi and the data term, 4 warps per CTA (32-row
// tiles), every radius 1..7: alone (FAST and general) and batched.
#include "lse_step_tile.cuh"

namespace lse_detail {

cudaError_t launch_step_tile_bf16_edge_nw4(const StepArgs &a, const CUtensorMap &pm,
                                           const CUtensorMap &dm, int nblocks, cudaStream_t s)
{
    return lse_tile::launch_tile_kind<1, __nv_bfloat16, 4>(a, pm, dm, nblocks, s);
}

cudaError_t launch_step_tile_batch_bf16_edge_nw4(int rad, const BatchItem *items,
                                                 const int *blk_item, long long n, int nblocks,
                                                 cudaStream_t s)
{
    return lse_tile::launch_tile_batch<1, __nv_bfloat16, 4>(rad, items, blk_item, n, nblocks, s);
}

}  // namespace lse_detail
