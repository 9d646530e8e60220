// Internal interface between the C ABI (hweno_api.cu) and the kernel files.
#pragma once

#include <cuda.h>           // CUtensorMap (the type only; maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "hweno_device.cuh"

namespace hw {

// Per-handle tables in both precisions (filled once at creation).
struct HostTabs {
  Weights<double> wd;
  Weights<float> wf;
  Weights<df64> wx;      // double-float (precision 2)
  Beta1<double> b1d;
  Beta1<float> b1f;
  Beta1<df64> b1x;
  Beta2<double> b2d;
  Beta2<float> b2f;
  Beta2<df64> b2x;
};

// Compute precision of a handle: 0 FP64, 1 FP32 bulk, 2 double-float (FP32 pairs).
enum { PREC_FP64 = 0, PREC_FP32 = 1, PREC_DF64 = 2 };

// Optional per-kernel timing: CUDA events recorded around each launch on the
// launching stream, read back (and summed per kernel kind) after a sync.
struct Prof {
  // 0 reconstruct, 1 indicator + modify, 2 reconstruct troubled, 3 flux + update,
  // 4 learned-indicator network pass, 5 fused stage (all of 0-3 in one launch)
  static constexpr int KINDS = 6;
  std::vector<cudaEvent_t> pool;
  std::vector<int> kinds;           // kind of each begin/end pair
  size_t used = 0;                  // events handed out
  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin(int kind, cudaStream_t s) { kinds.push_back(kind); cudaEventRecord(next(), s); }
  void end(cudaStream_t s) { cudaEventRecord(next(), s); }
  // Sum elapsed ms per kind into ms[n] and launches[n] (kinds >= n dropped); then reset.
  void read(double* ms, int* launches, int n) {
    for (int k = 0; k < n; ++k) { ms[k] = 0.0; launches[k] = 0; }
    for (size_t p = 0; p < kinds.size(); ++p) {
      if (kinds[p] >= n) continue;
      float t = 0.f;
      cudaEventSynchronize(pool[2 * p + 1]);
      cudaEventElapsedTime(&t, pool[2 * p], pool[2 * p + 1]);
      ms[kinds[p]] += t;
      launches[kinds[p]] += 1;
    }
    kinds.clear();
    used = 0;
  }
  ~Prof() { for (cudaEvent_t e : pool) cudaEventDestroy(e); }
};

// Work buffers owned by a handle.
struct Bufs {
  void* G;            // point values [nvar][npt][ny][gpitch] in the compute precision
  void* aux;          // KXRCF face-velocity partials and norms [5][ny][gpitch]
  int* list;          // flagged cells of the current stage (linear index j*nx+i)
  int* count;         // [3] flagged counts per stage
  unsigned* status;   // ST_* bits
  Prof* prof;         // per-kernel timing, or nullptr
  const float* mlp;   // learned indicator parameters (FP32, device), IND_MLP
  float mlp_conf;     // confidence threshold of the learned indicator
  int* mlp_stats;     // [1] cells decided by the KXRCF fallback (accumulates)
  float* mlp_prob;    // optional: the network's probability per cell of the last stage
  int* und;           // cells the learned indicator left to KXRCF (current stage)
  int* und_count;     // [3] their counts per stage
  unsigned long long* rerec;   // [1] cells reconstructed a second time (accumulates), or null
  const CUtensorMap* tmG = nullptr;   // FP32 2D Euler: tensor map of G for the TMA update kernel, or null
};

// One evaluation of the spatial operator with the troubled-cell steps and,
// unless Lout is set, the Runge-Kutta combination
//   Uout = cA * Un' + cB * (Uin' + dt * L(Uin'))
// where ' marks the first moments modified in troubled cells (eq. (vi)):
// Uin' by this stage's flags, Un' by the first stage's (maskN, ModN).
struct StageCall {
  int stage;               // 0, 1, 2 (selects counters)
  const double* Uin;
  const double* Un;        // may equal Uin (first stage)
  double* Uout;            // RK output (ignored when Lout is set)
  double dt, cA, cB;
  uint8_t* mask;           // out: this stage's flags [ny*nx]
  double* Mod;             // out: modified first moments of flagged cells [nvar][nmom-1][plane]
  const uint8_t* maskN;    // first-stage flags (for Un'); nullptr = Un unmodified
  const double* ModN;      // first-stage modified first moments
  const double* dtp;       // optional: dt read on the device (hweno_advance); < 0 = skip the step (Uout = Uin)
  double* Lout;            // optional: write L(Uin') (state layout) instead of the RK update
  double* Umod;            // optional (with Lout): write Uin'
  double* aleph;           // optional: KXRCF values [ny*nx]
  const float* U32in = nullptr;   // FP32 form: float copy of Uin (its reconstruction input), or null
  float* U32out = nullptr;        // FP32 form: float copy of Uout, written by the update
};

// FP32 form: the TMA update kernel's shared-memory attribute (once per process);
// false if it cannot be set (the caller then keeps the global-memory kernel).
bool prepare_update_tma();

void run_stage_1d(const Prob& P, const HostTabs& T, int prec, const Bufs& B, const StageCall& S, cudaStream_t st);

// ---------------------------------------------------------------- batched 2D problems
// One problem of a batch: its description and the offsets of its arrays inside
// the batch-wide buffers (elements of the respective buffer type).
struct BProb {
  Prob P;
  long long uoff;     // state buffers (doubles)
  long long goff;     // point values (elements of the compute precision)
  long long aoff;     // KXRCF partials
  long long moff;     // modified first moments (doubles)
  long long coff;     // cells before this problem (masks, troubled list)
  int rec_first;      // first reconstruction item (128 cells each)
  int upd_first;      // first update tile
  int tiles_x;        // update tiles per row
};

// Buffers and coefficients of one batched stage launch.
struct BatchStage {
  const BProb* probs;     // device array
  int nprob, n_rec, n_upd;
  const double* Uin; const double* Un; double* Uout;
  void* G; void* aux;
  double* Mod;            // this stage's modified first moments (first stage: the kept copy)
  const double* ModN;     // first-stage modified first moments (stages 2, 3), else nullptr
  uint8_t* mask;          // this stage's flags (batch cell order)
  const uint8_t* maskN;   // first-stage flags (stages 2, 3), else nullptr
  unsigned long long* list;   // troubled (problem << 32 | cell)
  int* count;
  unsigned long long* speeds; // per problem: max a_x, max a_y as FP64 bit patterns
  const double* dt_in;    // per-problem dt from the caller, or nullptr (CFL)
  double* dt_out;         // per-problem dt used (written in the first stage)
  double cfl, cA, cB;
  int stage;
  unsigned* status;       // ST_TIMEOUT of the grid barrier
  unsigned* pstatus;      // per problem: ST_NONFINITE / ST_NONPOSITIVE of its new state
  unsigned* bar;          // grid barrier {arrived, generation}
  unsigned long long spin_limit;   // polls (64 ns sleeps each) before a barrier wait gives up
  unsigned bar_extra;     // arrivals a barrier waits for beyond the launched blocks (0; > 0 only to
                          //    exercise the timeout path)
};

// Default bound of a grid-barrier wait: 2^26 polls with 64 ns sleeps, seconds.
constexpr unsigned long long BARRIER_SPIN_DEFAULT = 1ull << 26;

// Launch one batched stage as a single persistent cooperative kernel (grid =
// resident blocks); returns the CUDA error of the launch.
cudaError_t run_batch_stage(const HostTabs& T, int fp32, int tile_variant, const BatchStage& S, int nsm,
                            cudaStream_t st);
constexpr unsigned ST_TIMEOUT = 4u;   // a bounded grid-barrier wait gave up

// Learned troubled-cell indicator (hweno_mlp.cu).
int mlp_nparam();
cudaError_t run_features(const Prob& P, const double* U, const int* cells, int n, float* X, cudaStream_t st);
cudaError_t run_mlp_forward(const float* th, const float* X, int n, float* prob, int nsm, cudaStream_t st);
cudaError_t run_mlp_train(const float* th, const float* X, const float* y, const float* w, int n, float* grad,
                          float* loss, int nsm, cudaStream_t st);
cudaError_t run_adam(float* th, const float* grad, float* m1, float* m2, int step, float lr, cudaStream_t st);
cudaError_t run_mlpre2d(const Prob& P, const float* th, float conf, const double* U, uint8_t* mask, double* Mod,
                        int* und, int* und_count, int* stats, float* prob, cudaStream_t st);
void run_stage_2d(const Prob& P, const HostTabs& T, int prec, const Bufs& B, const StageCall& S, cudaStream_t st);
void run_stage_2d_fp32(const Prob& P, const HostTabs& T, const Bufs& B, const StageCall& S, cudaStream_t st);
void run_stage_2d_df64(const Prob& P, const HostTabs& T, const Bufs& B, const StageCall& S, cudaStream_t st);
cudaError_t run_batch_stage_df64(const HostTabs& T, int tile_variant, const BatchStage& S, int nsm, cudaStream_t st);

// Reductions over the cell averages (FP64): maximum wave speeds per direction
// and totals sum(ubar) per variable.  partials needs reduce_partials_len(P)
// doubles; out gets {ax, ay} or the nvar totals (unscaled sums).
int reduce_partials_len(const Prob& P);
void run_wavespeed(const Prob& P, const double* U, double* partials, double* out, cudaStream_t st);
void run_advance_dt(const Prob& P, const double* speeds, const double* par, double* st, unsigned* status,
                    cudaStream_t s);
void run_totals(const Prob& P, const double* U, double* partials, double* out, cudaStream_t st);
// FP32 form: rows [j0, j0 + nrows) of the float copy of state U, rounded to nearest.
void run_shadow32(const Prob& P, const double* U, float* U32, int j0, int nrows, cudaStream_t st);

// Fixed-state (inflow) ghost cells of a 2D Euler handle: per side, a segment
// of ghost positions whose centre coordinate along the side is below
// c0 + speed * t holds state a; the rest of an inflow side holds b.
struct FixSpec {
  int seg[4];             // segment set on the side
  int inflow[4];          // the side's kind is HWENO_BC_INFLOW
  int n[4];               // cells along the side (ny on x sides, nx on y sides)
  double c0[4], speed[4];
  double a[4][4], b[4][4];
  double x0, y0, dx, dy;
  int fixlen;             // table entries per side (positions -1 .. max(nx, ny))
};
// Fill the table Prob::fixtab for the stage at time t, or at *tn + c * *dtp
// read on the device when dtp is set (hweno_advance).
void run_fixfill(const FixSpec& F, double* tab, double t, const double* tn, const double* dtp, double c,
                 cudaStream_t st);

}  // namespace hw
