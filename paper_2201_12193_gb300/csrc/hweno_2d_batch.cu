// Batched persistent stage: FP64 and FP32-bulk instantiations, and the dispatch.
#include "hweno_2d_kernels.cuh"

namespace hw {

cudaError_t run_batch_stage(const HostTabs& T, int fp32, int tile_variant, const BatchStage& S, int nsm,
                            cudaStream_t st) {
  // tile shapes of the update phase (all 128 threads): 0: 32x4, 1: 16x8, 2: 64x2
  if (fp32 == PREC_DF64) return run_batch_stage_df64(T, tile_variant, S, nsm, st);
  if (fp32 == PREC_FP32) {
    if (tile_variant == 1) return launch_batch<float, 16, 8>(T.wf, T.b2f, S, nsm, st);
    if (tile_variant == 2) return launch_batch<float, 64, 2>(T.wf, T.b2f, S, nsm, st);
    return launch_batch<float, 32, 4>(T.wf, T.b2f, S, nsm, st);
  }
  if (tile_variant == 1) return launch_batch<double, 16, 8>(T.wd, T.b2d, S, nsm, st);
  if (tile_variant == 2) return launch_batch<double, 64, 2>(T.wd, T.b2d, S, nsm, st);
  return launch_batch<double, 32, 4>(T.wd, T.b2d, S, nsm, st);
}

}  // namespace hw
