// lse_evolve_mb4.cu -- instantiations of the persistent evolution of a
// 4-band image (the vector region term of Eq. 17), FP32 storage, 32-row
// tiles, every radius 1..7.
#include "lse_step_tile.cuh"

// At the default template (TS = 9, r = 4) a 4-band tile stages the bands of
// its 24 output rows and keeps D of its 8 halo rows apart: 72.7 KB of
// shared memory, so three CTAs share an SM (the measured 156 registers a
// thread allow three as well).
static_assert(lse_tile::TileGeo<4, float, 4, 4>::BYTES == 72704 &&
                  lse_tile::TileGeo<4, float, 4, 4>::MIN_BLOCKS == 3,
              "4-band tiles at r = 4: three CTAs per SM");

namespace lse_detail {

cudaError_t launch_evolve_mb4(const EvolveArgs &e, const CUtensorMap &pm0,
                               const CUtensorMap &pm1, const CUtensorMap &dm, int nblocks,
                               int sm_count, cudaStream_t s)
{
    return lse_tile::launch_evolve_mb_bands<4>(e, pm0, pm1, dm, nblocks, sm_count, s);
}

cudaError_t launch_evolve_mb_group4(int rad, const MbGroupItem *items, const int *cta_item,
                                    int nblocks, cudaStream_t s)
{
    return lse_tile::launch_evolve_mb_group<4>(rad, items, cta_item, nblocks, s);
}

int evolve_mb_group_capacity4(int rad, int sm_count)
{
    return lse_tile::evolve_mb_group_capacity<4>(rad, sm_count);
}

}  // namespace lse_detail
