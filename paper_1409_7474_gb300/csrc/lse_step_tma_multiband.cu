// lse_step_tma_multiband.cu -- instantiations of the fused step for one data term
// (one translation unit per term so the build compiles them in parallel).
#include "lse_step_tma.cuh"

namespace lse_detail {

cudaError_t launch_step_tma_multiband(const StepArgs &a, const CUtensorMap &pm,
                                   const CUtensorMap &dm, int nblocks, int wpc,
                                   cudaStream_t s)
{
    return lse_tma::launch_kind<lse_tma::K_REGION_MB>(a, pm, dm, nblocks, wpc, s);
}

int step_tma_warp_bytes_multiband(int rad)
{
    return lse_tma::warp_bytes_for<lse_tma::K_REGION_MB>(rad);
}

cudaError_t launch_step_tma_batch_multiband(int rad, const BatchItem *items,
                                            const int *blk_item, long long n, int nblocks, int wpc,
                                            cudaStream_t s)
{
    return lse_tma::launch_batch_kind<lse_tma::K_REGION_MB>(rad, items, blk_item, n, nblocks,
                                                           wpc, s);
}

}  // namespace lse_detail
