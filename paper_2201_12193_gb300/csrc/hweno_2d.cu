// Two-dimensional stage pipeline of the moment-based multi-resolution HWENO
// scheme (Sec. 2.2 of Li, Shu & Qiu, arXiv 2201.12193) on sm_103a.
//
// One Runge-Kutta stage is four launches on the caller's stream:
//   rec2d   (Step 1)    every cell: 3x3 moments -> 16 Gauss-Lobatto values per
//                       variable (eq. (2D-re-u)) + KXRCF face-velocity partials;
//   flag2d  (Step 2)    KXRCF (eq. (KXRCF_), (line-integral-average_)), the
//                       dimension-by-dimension first-moment modification of
//                       troubled cells (eq. (vi)) and a compacted list of them;
//   rec2d*  (Step 2.3)  the troubled cells again, from the modified moments;
//   update2d (Step 3)   HLLC/LLF fluxes at the Gauss-Lobatto points of every
//                       face (eq. (integral2), (integral3)), the cell quadrature
//                       (eq. (integral1)), L(U) of eq. (2D-equ-int-approximation)
//                       and the SSP-RK3 combination (eq. (Runge-Kutta)).
// Each cell is reconstructed once per stage (plus once more if troubled):
// FP64 arithmetic is the scarce resource on this GPU, so the pipeline keeps
// the point values in HBM rather than recomputing a halo.
//
// This unit holds the FP64 instantiations and the precision dispatch; FP32,
// double-float and the batched kernels compile in their own units.
#include "hweno_2d_kernels.cuh"

namespace hw {

void run_stage_2d(const Prob& P, const HostTabs& T, int prec, const Bufs& B, const StageCall& S, cudaStream_t st) {
  if (prec == PREC_FP32) return run_stage_2d_fp32(P, T, B, S, st);
  if (prec == PREC_DF64) return run_stage_2d_df64(P, T, B, S, st);
  if (P.nvar == 4) stage_t<double, 4>(P, T, T.wd, T.b2d, B, S, st);
  else stage_t<double, 1>(P, T, T.wd, T.b2d, B, S, st);
}

}  // namespace hw
