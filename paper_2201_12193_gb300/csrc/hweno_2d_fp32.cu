// FP32-bulk instantiations of the two-dimensional stage pipeline.
#include "hweno_2d_kernels.cuh"

namespace hw {

void run_stage_2d_fp32(const Prob& P, const HostTabs& T, const Bufs& B, const StageCall& S, cudaStream_t st) {
  if (P.nvar == 4) stage_t<float, 4>(P, T, T.wf, T.b2f, B, S, st);
  else stage_t<float, 1>(P, T, T.wf, T.b2f, B, S, st);
}

bool prepare_update_tma() {
  static const bool ok = set_update_tma_attribute();
  return ok;
}

}  // namespace hw
