// lse_evolve_tile_f16_region_nw8.cu -- instantiations of the persistent
// evolution (every iteration in one cooperative launch) for the single-band region term (Eq. 17),
// F16 storage of phi and the data term, 8 warps per CTA (64-row
// tiles), every radius 1..7.
#include "lse_step_tile.cuh"

namespace lse_detail {

cudaError_t launch_evolve_tile_f16_region_nw8(const EvolveArgs &e, const CUtensorMap &pm0,
                                              const CUtensorMap &pm1, const CUtensorMap &dm,
                                              int nblocks, int sm_count, cudaStream_t s)
{
    return lse_tile::launch_evolve_kind<0, __half, 8>(e, pm0, pm1, dm, nblocks, sm_count, s);
}

}  // namespace lse_detail
