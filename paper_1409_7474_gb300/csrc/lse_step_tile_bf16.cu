// lse_step_tile_bf16.cu -- instantiations of the tile-form step with BF16
// storage of phi and the data term (FP32 arithmetic), for the single-band
// region term (Eq. 17) and the edge term (Eq. 14).
#include "lse_step_tile.cuh"

namespace lse_detail {

cudaError_t launch_step_tile_bf16(const StepArgs &a, const CUtensorMap &pm,
                                const CUtensorMap &dm, int nblocks, cudaStream_t s)
{
    if (a.term == LSE_TERM_EDGE) return lse_tile::launch_tile_kind<1, __nv_bfloat16>(a, pm, dm, nblocks, s);
    return lse_tile::launch_tile_kind<0, __nv_bfloat16>(a, pm, dm, nblocks, s);
}

}  // namespace lse_detail
