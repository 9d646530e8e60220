// Double-float instantiations of the two-dimensional stage pipeline.
#include "hweno_2d_kernels.cuh"

namespace hw {

void run_stage_2d_df64(const Prob& P, const HostTabs& T, const Bufs& B, const StageCall& S, cudaStream_t st) {
  if (P.nvar == 4) stage_t<df64, 4>(P, T, T.wx, T.b2x, B, S, st);
  else stage_t<df64, 1>(P, T, T.wx, T.b2x, B, S, st);
}

}  // namespace hw
