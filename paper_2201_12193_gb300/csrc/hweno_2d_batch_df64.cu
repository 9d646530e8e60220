// Batched persistent stage: double-float instantiations.
#include "hweno_2d_kernels.cuh"

namespace hw {

cudaError_t run_batch_stage_df64(const HostTabs& T, int tile_variant, const BatchStage& S, int nsm, cudaStream_t st) {
  if (tile_variant == 1) return launch_batch<df64, 16, 8>(T.wx, T.b2x, S, nsm, st);
  if (tile_variant == 2) return launch_batch<df64, 64, 2>(T.wx, T.b2x, S, nsm, st);
  return launch_batch<df64, 32, 4>(T.wx, T.b2x, S, nsm, st);
}

}  // namespace hw
