// lse_evolve_tile_f32_edge_nw4.cu -- instantiations of the persistent
// evolution (every iteration in one cooperative launch) for the edge term (Eq. 14),
// FP32 storage of phi and the data term, 4 warps per CTA (32-row
// tiles), every radius 1..7.
#include "lse_step_tile.cuh"

namespace lse_detail {

cudaError_t launch_evolve_tile_f32_edge_nw4(const EvolveArgs &e, const CUtensorMap &pm0,
                                            const CUtensorMap &pm1, const CUtensorMap &dm,
                                            int nblocks, int sm_count, cudaStream_t s)
{
    return lse_tile::launch_evolve_kind<1, float, 4>(e, pm0, pm1, dm, nblocks, sm_count, s);
}

}  // namespace lse_detail
