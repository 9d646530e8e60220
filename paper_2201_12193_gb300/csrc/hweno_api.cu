// C ABI of the HWENO library: handle, device buffers, stage sequencing.
// See include/hweno.h for the contract of every entry point.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

#define HWP_HOST_TABLES
#include "hweno_internal.h"
#include "hweno.h"

using hw::Prob;

struct hweno_s {
  hweno_grid g{};
  hweno_bc bc{};
  double gamma = 1.4;
  int dev = 0;
  cudaStream_t stream = nullptr;
  Prob P{};
  hw::HostTabs T{};
  int fp32 = 0;                  // compute precision (hw::PREC_*)
  double* U[3] = {nullptr, nullptr, nullptr};
  float* U32[3] = {nullptr, nullptr, nullptr};   // FP32 form (single 2D handles): float copies of U[k]
  CUtensorMap tmG{};             // FP32 2D Euler: tensor map of the point values (TMA-staged update)
  bool tma_ok = false;           // the map is encoded
  bool tma_on = false;           // the update kernel uses it (hweno_set_tma; off by default)
  int cur = 0, prev = 0;
  bool have_state = false, stepped = false;
  hw::Bufs B{};
  double* ModN = nullptr;        // first-stage modified first moments (kept for stages 2, 3)
  double* ModK = nullptr;        // modified first moments of the current stage
  uint8_t* mask3 = nullptr;      // [3][ny][nx] flags of the last step
  double* red_part = nullptr;    // reduction partials
  double* red_out = nullptr;     // reduction results (device)
  double* host_buf = nullptr;    // pinned: reduction results + status
  hw::Prof prof;                 // per-kernel event timing (hweno_profile)
  double* adv = nullptr;         // hweno_advance: device {T, cfl, max_steps, t, dt, steps, t at the step's start}
  double time = 0.0, time_prev = 0.0;   // solution time (moving fixed-state segments); before the last step
  hw::FixSpec fix{};             // fixed-state (inflow) ghost cells
  bool fix_set[4] = {false, false, false, false};
  double* fixtab = nullptr;      // their per-stage table (device), Prob::fixtab
  cudaGraphExec_t agraphs[3] = {nullptr, nullptr, nullptr};   // hweno_advance, one per state rotation
  bool adv_graph = true;         // capture works here (else direct launches)
  float* mlp = nullptr;          // learned indicator parameters (device)
  int* mlp_stats = nullptr;      // fallback counter (device)
  bool have_mlp = false;
  bool positivity = true;        // rho <= 0 or p <= 0 in a new cell average fails the step
  std::string err;
  // batch mode (hweno_create_batch): many independent 2D Euler problems
  bool batch = false;
  int nprob = 0;
  std::vector<hw::BProb> probs;  // host copy of the descriptors
  hw::BProb* dprobs = nullptr;
  long long tot_cells = 0;
  int n_rec = 0, n_upd = 0;
  int tile_variant = 0;
  unsigned long long* blist = nullptr;
  unsigned long long* speeds = nullptr;
  double* dt_out = nullptr;
  unsigned* bar = nullptr;
  unsigned* pstatus = nullptr;   // per-problem status bits (device)
  std::vector<unsigned> last_pstatus;   // per-problem bits of the last reported failure
  cudaGraphExec_t graphs[3] = {nullptr, nullptr, nullptr};   // one per state rotation
  const double* graph_dt = nullptr;
  double graph_cfl = -1.0;
  int graph_variant = -1;
  bool use_graph = true;
  int next_stage = 0;            // hweno_stage: the stage to run next (0: no step in progress)
  int stage_a = 0;               // hweno_stage: rotation of the step in progress
  double stage_dt = 0.0;         // hweno_stage: its dt
  unsigned long long spin_limit = hw::BARRIER_SPIN_DEFAULT;   // grid-barrier wait bound
  unsigned bar_extra = 0;        // extra arrivals the barrier waits for (timeout-path tests)
};

namespace {

constexpr int VERSION = 100;

hweno_status fail(hweno_t h, hweno_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

#define CK(h, call)                                                                              \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(h, HWENO_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t ncell(const hweno_s* h) { return (size_t)h->P.nx * (size_t)h->P.ny; }

// A double in the three compute precisions (the device conversions' roundings).
hw::PConst pconst(double v) {
  hw::PConst c;
  c.d = v;
  c.f = (float)v;
  c.x = hw::df64(v);
  return c;
}

// The per-precision constants of a problem (after dx, dy and gamma are set).
void fill_consts(Prob& P) {
  P.cgamma = pconst(P.gamma);
  P.cgm1 = pconst(P.gamma - 1.0);
  P.chk = pconst((P.gamma + 1.0) / (2.0 * P.gamma));
  P.cdx = pconst(P.dx);
  P.cdy = pconst(P.dy);
  P.crdx = pconst(1.0 / P.dx);
  P.crdy = pconst(1.0 / P.dy);
  P.cdx2 = pconst(P.dx * P.dx);
}
size_t nstate(const hweno_s* h) { return (size_t)h->P.nvar * h->P.nmom * ncell(h); }

// Linear weights of eq. (linear-weight) and the smoothness-indicator rows of
// eq. (beta) / (2D-beta) for p_l = (S_l q_l - S_{l-1} q_{l-1}) / g_l.
// A long double as a double-float pair (hi = nearest float, lo = nearest float of the rest).
hw::df64 dfx(long double v) {
  const float hi = (float)v;
  return hw::df64(hi, (float)(v - (long double)hi));
}

void build_tables(hweno_s* h) {
  const double* g = h->g.gamma_bar;
  long double S[5] = {0, 0, 0, 0, 0};
  for (int l = 1; l <= 4; ++l) S[l] = S[l - 1] + g[l - 1];
  auto& wd = h->T.wd;
  auto& wf = h->T.wf;
  for (int l = 1; l <= 4; ++l) {
    wd.gam[l - 1] = (double)(g[l - 1] / S[4]);
    wd.sg[l - 1] = (double)(S[l] / g[l - 1]);
    wd.s1g[l - 1] = (double)(S[l - 1] / g[l - 1]);
    wf.gam[l - 1] = (float)wd.gam[l - 1];
    wf.sg[l - 1] = (float)wd.sg[l - 1];
    wf.s1g[l - 1] = (float)wd.s1g[l - 1];
    h->T.wx.gam[l - 1] = dfx(g[l - 1] / S[4]);
    h->T.wx.sg[l - 1] = dfx(S[l] / g[l - 1]);
    h->T.wx.s1g[l - 1] = dfx(S[l - 1] / g[l - 1]);
  }
  wd.eps = 1e-10;
  wf.eps = 1e-10f;
  h->T.wx.eps = dfx(1e-10L);
  auto coef = [&](int l, long double& a, long double& b) {
    if (h->g.beta_of_q) { a = 1.0L; b = 0.0L; return; }
    a = S[l] / g[l - 1];
    b = -S[l - 1] / g[l - 1];
  };
  long double a, b;
  // flat rows: B_l[k] = a_l RC_l_l[k] + b_l RC_l_(l-1)[k]; q_1 is constant, so level 2 has no b part
  auto fill = [&](int l, const double* rl, const double* rm, int n, double* outd, float* outf, hw::df64* outx) {
    coef(l, a, b);
    for (int k = 0; k < n; ++k) {
      const long double v = a * rl[k] + (rm ? b * rm[k] : 0.0L);
      outd[k] = (double)v;
      outf[k] = (float)v;
      outx[k] = dfx(v);
    }
  };
  if (h->g.dim == 1) {
    fill(2, hwp::D1P_RC2_2, nullptr, hwp::D1_NB2, h->T.b1d.B2, h->T.b1f.B2, h->T.b1x.B2);
    fill(3, hwp::D1P_RC3_3, hwp::D1P_RC3_2, hwp::D1_NB3, h->T.b1d.B3, h->T.b1f.B3, h->T.b1x.B3);
    fill(4, hwp::D1P_RC4_4, hwp::D1P_RC4_3, hwp::D1_NB4, h->T.b1d.B4, h->T.b1f.B4, h->T.b1x.B4);
  } else {
    fill(2, hwp::D2P_RC2_2, nullptr, hwp::D2_NB2, h->T.b2d.B2, h->T.b2f.B2, h->T.b2x.B2);
    fill(3, hwp::D2P_RC3_3, hwp::D2P_RC3_2, hwp::D2_NB3, h->T.b2d.B3, h->T.b2f.B3, h->T.b2x.B3);
    fill(4, hwp::D2P_RC4_4, hwp::D2P_RC4_3, hwp::D2_NB4, h->T.b2d.B4, h->T.b2f.B4, h->T.b2x.B4);
  }
}

hweno_status validate(const hweno_grid* g, const hweno_bc* bc, double gamma, std::string& why) {
  if (!g || !bc) { why = "grid and bc must not be NULL"; return HWENO_EINVAL; }
  if (g->dim != 1 && g->dim != 2) { why = "dim must be 1 or 2"; return HWENO_EINVAL; }
  if (g->nx < 4 || (g->dim == 2 && g->ny < 4)) { why = "need at least 4 cells per direction"; return HWENO_EINVAL; }
  if ((long long)g->nx * (g->dim == 2 ? g->ny : 1) > (1LL << 31) - 1) { why = "too many cells"; return HWENO_EINVAL; }
  if (!(g->x1 > g->x0) || (g->dim == 2 && !(g->y1 > g->y0)) || !isfinite(g->x1 - g->x0)) {
    why = "empty or non-finite domain"; return HWENO_EINVAL;
  }
  if (g->eq < 0 || g->eq > 2) { why = "eq must be advection, burgers or euler"; return HWENO_EINVAL; }
  if (g->precision < 0 || g->precision > 2) {
    why = "precision must be 0 (fp64), 1 (fp32 bulk) or 2 (double-float)"; return HWENO_EINVAL;
  }
  if (g->indicator < 0 || g->indicator > 4) { why = "indicator must be none, kxrcf, all, mlp or tvb"; return HWENO_EINVAL; }
  if (g->indicator == 4 && !(g->tvb_m >= 0.0 && isfinite(g->tvb_m))) { why = "tvb_m must be finite and >= 0"; return HWENO_EINVAL; }
  if (g->charwise != 0 && (g->dim != 1 || g->eq != HWENO_EULER)) {
    why = "characteristic reconstruction (charwise) is defined for 1D Euler"; return HWENO_EINVAL;
  }
  if (g->indicator == 3 && (g->dim != 2 || g->eq != HWENO_EULER)) {
    why = "the learned indicator is defined for 2D Euler"; return HWENO_EINVAL;
  }
  for (int l = 0; l < 4; ++l)
    if (!(g->gamma_bar[l] > 0.0) || !isfinite(g->gamma_bar[l])) { why = "gamma_bar must be positive"; return HWENO_EINVAL; }
  const int k[4] = {bc->xlo, bc->xhi, bc->ylo, bc->yhi};
  for (int s = 0; s < (g->dim == 2 ? 4 : 2); ++s)
    if (k[s] != HWENO_BC_PERIODIC && k[s] != HWENO_BC_TRANSMISSIVE && k[s] != HWENO_BC_REFLECTIVE &&
        k[s] != HWENO_BC_INFLOW) {
      why = "unknown boundary kind"; return HWENO_EINVAL;
    } else if (k[s] == HWENO_BC_REFLECTIVE && g->eq != HWENO_EULER) {
      why = "reflective walls need the Euler equations"; return HWENO_EINVAL;
    } else if (k[s] == HWENO_BC_INFLOW && (g->dim != 2 || g->eq != HWENO_EULER || g->precision != 0 ||
                                           g->indicator == 3)) {
      why = "inflow sides need 2D Euler in FP64 without the learned indicator"; return HWENO_EINVAL;
    }
  if ((bc->xlo == HWENO_BC_PERIODIC) != (bc->xhi == HWENO_BC_PERIODIC) ||
      (g->dim == 2 && (bc->ylo == HWENO_BC_PERIODIC) != (bc->yhi == HWENO_BC_PERIODIC))) {
    why = "periodic sides must come in pairs"; return HWENO_EINVAL;
  }
  if (g->dim == 2) {
    const double dx = (g->x1 - g->x0) / g->nx, dy = (g->y1 - g->y0) / g->ny;
    if (fabs(dx - dy) > 1e-12 * dx) { why = "2D cells must be square (dx == dy)"; return HWENO_EINVAL; }
  }
  if (g->eq == HWENO_EULER && !(gamma > 1.0)) { why = "gamma must exceed 1"; return HWENO_EINVAL; }
  if (!isfinite(g->adv_a) || !isfinite(g->adv_b)) { why = "advection speeds must be finite"; return HWENO_EINVAL; }
  return HWENO_OK;
}

void drop_graphs(hweno_s* h) {
  for (int k = 0; k < 3; ++k) {
    if (h->graphs[k]) { cudaGraphExecDestroy(h->graphs[k]); h->graphs[k] = nullptr; }
    if (h->agraphs[k]) { cudaGraphExecDestroy(h->agraphs[k]); h->agraphs[k] = nullptr; }
  }
}

void free_all(hweno_s* h) {
  drop_graphs(h);
  cudaFree(h->mlp);
  cudaFree(h->mlp_stats);
  cudaFree(h->B.und);
  cudaFree(h->B.und_count);
  cudaFree(h->B.rerec);
  cudaFree(h->adv);
  cudaFree(h->fixtab);
  cudaFree(h->dprobs);
  cudaFree(h->blist);
  cudaFree(h->speeds);
  cudaFree(h->dt_out);
  cudaFree(h->bar);
  cudaFree(h->pstatus);
  for (int k = 0; k < 3; ++k) cudaFree(h->U[k]);
  for (int k = 0; k < 3; ++k) cudaFree(h->U32[k]);
  cudaFree(h->B.G);
  cudaFree(h->B.aux);
  cudaFree(h->B.list);
  cudaFree(h->B.count);
  cudaFree(h->B.status);
  cudaFree(h->ModN);
  cudaFree(h->ModK);
  cudaFree(h->mask3);
  cudaFree(h->red_part);
  cudaFree(h->red_out);
  if (h->host_buf) cudaFreeHost(h->host_buf);
}

// Read the status word; on a non-physical step roll the state back.
hweno_status check_status(hweno_t h) {
  CK(h, cudaMemcpyAsync(h->host_buf + 8, h->B.status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  unsigned st;
  memcpy(&st, h->host_buf + 8, sizeof st);
  if (h->batch) {   // per-problem bits
    std::vector<unsigned> ps(h->nprob);
    CK(h, cudaMemcpy(ps.data(), h->pstatus, h->nprob * sizeof(unsigned), cudaMemcpyDeviceToHost));
    unsigned any = 0;
    for (unsigned v : ps) any |= v;
    if (any) {
      h->last_pstatus = ps;
      CK(h, cudaMemsetAsync(h->pstatus, 0, h->nprob * sizeof(unsigned), h->stream));
    }
    st |= any;
  }
  if (!h->positivity) st &= ~hw::ST_NONPOSITIVE;
  if (st != 0) {
    CK(h, cudaMemsetAsync(h->B.status, 0, sizeof(unsigned), h->stream));
    if (h->stepped) { h->cur = h->prev; h->time = h->time_prev; }
    h->stepped = false;
    h->next_stage = 0;      // a step begun with hweno_stage is abandoned; U^n is intact
    char buf[200];
    snprintf(buf, sizeof buf, "last step produced a non-physical state or timed out (status 0x%x: %s%s%s%s); rolled back",
             st, (st & hw::ST_NONFINITE) ? "non-finite " : "", (st & hw::ST_NONPOSITIVE) ? "rho<=0 or p<=0 " : "",
             (st & hw::ST_NODT) ? "no CFL step length " : "", (st & hw::ST_TIMEOUT) ? "grid barrier wait limit" : "");
    return fail(h, (st & hw::ST_TIMEOUT) ? HWENO_ETIMEOUT : HWENO_ENONPHYSICAL, buf);
  }
  return HWENO_OK;
}

// every inflow side has its fixed states
bool fix_ready(const hweno_s* h) {
  const int k[4] = {h->bc.xlo, h->bc.xhi, h->bc.ylo, h->bc.yhi};
  for (int s = 0; s < 4; ++s)
    if (h->g.dim == 2 && k[s] == HWENO_BC_INFLOW && !h->fix_set[s]) return false;
  return true;
}

}  // namespace

extern "C" {

int hweno_version(void) { return VERSION; }

const char* hweno_last_error(hweno_t h) { return h ? h->err.c_str() : "null handle"; }

namespace {
bool encode_maps(hweno_t h);
}  // namespace

hweno_status hweno_create(const hweno_grid* grid, const hweno_bc* bc, double gamma, hweno_t* out) {
  if (!out) return HWENO_EINVAL;
  *out = nullptr;
  std::string why;
  if (validate(grid, bc, gamma, why) != HWENO_OK) {
    fprintf(stderr, "hweno_create: %s\n", why.c_str());
    return HWENO_EINVAL;
  }
  hweno_s* h = new hweno_s();
  h->g = *grid;
  h->bc = *bc;
  h->gamma = gamma;
  if (grid->dim == 1) { h->g.ny = 1; h->g.y0 = 0.0; h->g.y1 = 1.0; }
  if (cudaGetDevice(&h->dev) != cudaSuccess) { delete h; return HWENO_ECUDA; }
  Prob& P = h->P;
  P.nx = h->g.nx;
  P.ny = h->g.dim == 2 ? h->g.ny : 1;
  P.pitch = (P.nx + 31) / 32 * 32;
  P.plane = (long long)P.ny * P.pitch;
  P.gpitch = (P.nx + 31) / 32 * 32;
  P.gplane = (long long)P.ny * P.gpitch;
  P.nvar = h->g.eq == HWENO_EULER ? (h->g.dim == 1 ? 3 : 4) : 1;
  P.nmom = h->g.dim == 1 ? 2 : 3;
  P.eq = h->g.eq;
  P.indicator = h->g.indicator;
  P.tvb_m = h->g.tvb_m;
  P.charwise = h->g.charwise;
  P.bc[0] = bc->xlo; P.bc[1] = bc->xhi;
  P.bc[2] = h->g.dim == 2 ? bc->ylo : HWENO_BC_PERIODIC;
  P.bc[3] = h->g.dim == 2 ? bc->yhi : HWENO_BC_PERIODIC;
  P.dx = (h->g.x1 - h->g.x0) / P.nx;
  P.dy = h->g.dim == 2 ? (h->g.y1 - h->g.y0) / P.ny : 1.0;
  P.gamma = gamma;
  P.adv_a = h->g.adv_a;
  P.adv_b = h->g.adv_b;
  P.nsm = 152;
  P.positivity = 1;
  P.persist = 1;
  P.jlo = 0;
  P.jhi = P.ny;
  // 1D: the fused stage by default where it applies (bitwise the pipeline's states in one launch per stage)
  P.fused = h->g.dim == 1 && !P.charwise &&
            (P.indicator == HWENO_IND_NONE || P.indicator == HWENO_IND_KXRCF || P.indicator == HWENO_IND_ALL);
  fill_consts(P);
  cudaDeviceGetAttribute(&P.nsm, cudaDevAttrMultiProcessorCount, h->dev);
  h->fp32 = h->g.precision;
  build_tables(h);

  const size_t npt = h->g.dim == 1 ? 4 : 16;
  const size_t esz = h->fp32 == hw::PREC_FP32 ? sizeof(float) : sizeof(double);   // df64 is 8 bytes
  const size_t sbytes = (size_t)P.nvar * P.nmom * P.plane * sizeof(double);
  const size_t mbytes = (size_t)P.nvar * (P.nmom - 1) * P.plane * sizeof(double);
  const size_t nc = (size_t)P.nx * P.ny;
  bool ok = true;
  for (int k = 0; k < 3; ++k) ok = ok && cudaMalloc(&h->U[k], sbytes) == cudaSuccess;
  // FP32 form in 2D: the reconstruction reads a float copy of its input state,
  // which the update kernel writes beside each FP64 output (no per-moment
  // FP64 -> FP32 conversion in the 3 x 3 gathers)
  const bool shadow = h->fp32 == hw::PREC_FP32 && h->g.dim == 2;
  for (int k = 0; k < 3 && shadow; ++k) ok = ok && cudaMalloc(&h->U32[k], sbytes / 2) == cudaSuccess;
  ok = ok && cudaMalloc(&h->B.G, (size_t)P.nvar * npt * P.gplane * esz) == cudaSuccess;
  ok = ok && cudaMalloc(&h->B.aux, 5 * (size_t)P.gplane * esz) == cudaSuccess;
  ok = ok && cudaMalloc(&h->B.list, nc * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->B.count, 4 * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->B.status, sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->ModN, mbytes) == cudaSuccess;
  ok = ok && cudaMalloc(&h->ModK, mbytes) == cudaSuccess;
  ok = ok && cudaMalloc(&h->mask3, 3 * nc) == cudaSuccess;
  ok = ok && cudaMalloc(&h->red_part, hw::reduce_partials_len(P) * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->red_out, 8 * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMallocHost(&h->host_buf, 16 * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->B.rerec, sizeof(unsigned long long)) == cudaSuccess;
  if (grid->indicator == HWENO_IND_MLP) {
    ok = ok && cudaMalloc(&h->mlp, hw::mlp_nparam() * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->mlp_stats, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->B.und, nc * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->B.und_count, 4 * sizeof(int)) == cudaSuccess;
    if (ok) {
      cudaMemset(h->mlp_stats, 0, sizeof(int));
      cudaMemset(h->B.und_count, 0, 4 * sizeof(int));
    }
  }
  if (!ok) {
    cudaGetLastError();
    free_all(h);
    delete h;
    fprintf(stderr, "hweno_create: device allocation failed\n");
    return HWENO_ENOMEM;
  }
  cudaMemset(h->B.status, 0, sizeof(unsigned));
  cudaMemset(h->mask3, 0, 3 * nc);
  cudaMemset(h->B.count, 0, 4 * sizeof(int));
  cudaMemset(h->B.rerec, 0, sizeof(unsigned long long));
  for (int k = 0; k < 3; ++k) cudaMemset(h->U[k], 0, sbytes);
  for (int k = 0; k < 3 && shadow; ++k) cudaMemset(h->U32[k], 0, sbytes / 2);
  if (cudaDeviceSynchronize() != cudaSuccess) { free_all(h); delete h; return HWENO_ECUDA; }
  // FP32 2D Euler: the update can stage interior tiles through TMA (hweno_set_tma; off by default)
  if (shadow && P.nvar == 4) h->tma_ok = encode_maps(h);
  *out = h;
  return HWENO_OK;
}

void hweno_destroy(hweno_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

hweno_status hweno_set_stream(hweno_t h, void* s) {
  if (!h) return HWENO_EINVAL;
  h->stream = (cudaStream_t)s;
  return HWENO_OK;
}

hweno_status hweno_set_moments(hweno_t h, const double* m, size_t count, int on_device) {
  if (!h) return HWENO_EINVAL;
  if (!m || count != nstate(h)) return fail(h, HWENO_EINVAL, "set_moments: count must be nvar*nmom*ny*nx");
  const size_t rows = (size_t)h->P.nvar * h->P.nmom * h->P.ny;
  CK(h, cudaMemcpy2DAsync(h->U[h->cur], h->P.pitch * sizeof(double), m, h->P.nx * sizeof(double),
                          h->P.nx * sizeof(double), rows, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          h->stream));
  if (h->U32[h->cur]) hw::run_shadow32(h->P, h->U[h->cur], h->U32[h->cur], 0, h->P.ny, h->stream);
  CK(h, cudaMemsetAsync(h->B.status, 0, sizeof(unsigned), h->stream));
  h->have_state = true;
  h->stepped = false;
  h->next_stage = 0;
  h->time = 0.0;
  if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
  return HWENO_OK;
}

hweno_status hweno_get_moments(hweno_t h, double* m, size_t count, int on_device) {
  if (!h) return HWENO_EINVAL;
  if (!m || count != nstate(h)) return fail(h, HWENO_EINVAL, "get_moments: count must be nvar*nmom*ny*nx");
  if (!h->have_state) return fail(h, HWENO_ESTATE, "get_moments: no moments set");
  if (!on_device) {
    const hweno_status s = check_status(h);
    if (s != HWENO_OK) return s;
  }
  const size_t rows = (size_t)h->P.nvar * h->P.nmom * h->P.ny;
  CK(h, cudaMemcpy2DAsync(m, h->P.nx * sizeof(double), h->U[h->cur], h->P.pitch * sizeof(double),
                          h->P.nx * sizeof(double), rows, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          h->stream));
  if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
  return HWENO_OK;
}

namespace {

// Tensor map of the FP32 update's TMA loads: the point values as a 3D tensor
// (columns up to the padded pitch, rows, 64 planes), box 32 x 4 x 64 floats (one
// update tile).  Strides and box rows are multiples of 16 bytes (rows padded to
// 32 elements).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_maps(hweno_t h) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  const EncodeTiled enc = reinterpret_cast<EncodeTiled>(fn);
  const Prob& P = h->P;
  const cuuint32_t one[3] = {1, 1, 1};
  {
    const cuuint64_t dim[3] = {(cuuint64_t)P.gpitch, (cuuint64_t)P.ny, 64};
    const cuuint64_t stride[2] = {(cuuint64_t)P.gpitch * 4, (cuuint64_t)P.gplane * 4};
    const cuuint32_t box[3] = {32, 4, 64};
    if (enc(&h->tmG, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->B.G, dim, stride, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return false;
  }
  return hw::prepare_update_tma();
}

// Stage k (0, 1, 2) of the SSP-RK3 step from rotation a (eq. (Runge-Kutta)):
//   U^(1) = U^n' + dt L(U^n');  U^(2) = 3/4 U^n' + 1/4 (U^(1)' + dt L(U^(1)'));
//   U^{n+1} = 1/3 U^n' + 2/3 (U^(2)' + dt L(U^(2)'))
// (' marks the modified first moments where the handle's reading uses them).
void launch_stage(hweno_t h, int k, int a, double dt, double t) {
  const int b = (a + 1) % 3, c = (a + 2) % 3;
  const size_t nc = ncell(h);
  hw::StageCall S{};
  S.stage = k; S.Un = h->U[a]; S.dt = dt;
  const int in = k == 0 ? a : (k == 1 ? b : c), out = k == 1 ? c : b;
  if (k == 0) {
    S.Uin = h->U[a]; S.Uout = h->U[b]; S.cA = 0.0; S.cB = 1.0;
    S.mask = h->mask3; S.Mod = h->ModN; S.maskN = nullptr; S.ModN = nullptr;
  } else if (k == 1) {
    S.Uin = h->U[b]; S.Uout = h->U[c]; S.cA = 0.75; S.cB = 0.25;
    S.mask = h->mask3 + nc; S.Mod = h->ModK; S.maskN = h->mask3; S.ModN = h->ModN;
  } else {
    S.Uin = h->U[c]; S.Uout = h->U[b]; S.cA = 1.0 / 3.0; S.cB = 2.0 / 3.0;
    S.mask = h->mask3 + 2 * nc; S.Mod = h->ModK; S.maskN = h->mask3; S.ModN = h->ModN;
  }
  S.U32in = h->U32[in];
  S.U32out = h->U32[out];
  if (h->P.fixtab) hw::run_fixfill(h->fix, h->fixtab, t, nullptr, nullptr, 0.0, h->stream);
  if (h->g.dim == 1) hw::run_stage_1d(h->P, h->T, h->fp32, h->B, S, h->stream);
  else hw::run_stage_2d(h->P, h->T, h->fp32, h->B, S, h->stream);
}

hweno_status step_checks(hweno_t h, double dt, const char* who) {
  if (!h->have_state) return fail(h, HWENO_ESTATE, std::string(who) + ": no moments set");
  if (h->g.indicator == 3 && !h->have_mlp)
    return fail(h, HWENO_ESTATE, std::string(who) + ": learned indicator not set (hweno_set_mlp)");
  if (!(dt >= 0.0) || !isfinite(dt)) return fail(h, HWENO_EINVAL, std::string(who) + ": dt must be finite and >= 0");
  if (!fix_ready(h))
    return fail(h, HWENO_ESTATE, std::string(who) + ": an inflow side has no fixed states (hweno_set_fixed_state)");
  return HWENO_OK;
}

// the step's bookkeeping once its last stage is enqueued
void finish_step(hweno_t h, int a, double dt) {
  h->prev = a;
  h->cur = (a + 1) % 3;
  h->stepped = true;
  h->time_prev = h->time;
  h->time += dt;
}

}  // namespace

hweno_status hweno_step(hweno_t h, double dt) {
  if (!h) return HWENO_EINVAL;
  if (h->next_stage != 0) return fail(h, HWENO_ESTATE, "step: a step begun with hweno_stage is not finished");
  const hweno_status s = step_checks(h, dt, "step");
  if (s != HWENO_OK) return s;
  const int a = h->cur;
  // stage times t, t + dt, t + dt/2 (the scheme's abscissae) for moving segments
  const double tst[3] = {h->time, h->time + dt, h->time + 0.5 * dt};
  for (int k = 0; k < 3; ++k) launch_stage(h, k, a, dt, tst[k]);
  CK(h, cudaGetLastError());
  finish_step(h, a, dt);
  return HWENO_OK;
}

hweno_status hweno_stage(hweno_t h, int k, double dt) {
  if (!h) return HWENO_EINVAL;
  if (h->batch) return fail(h, HWENO_ESTATE, "stage: single-problem handles only");
  if (k != h->next_stage) return fail(h, HWENO_ESTATE, "stage: stages run in the order 0, 1, 2");
  if (k == 0) {
    const hweno_status s = step_checks(h, dt, "stage");
    if (s != HWENO_OK) return s;
    h->stage_a = h->cur;
    h->stage_dt = dt;
  } else if (dt != h->stage_dt) {
    return fail(h, HWENO_EINVAL, "stage: the three stages of a step take the same dt");
  }
  const double c[3] = {0.0, 1.0, 0.5};
  launch_stage(h, k, h->stage_a, dt, h->time + c[k] * dt);
  CK(h, cudaGetLastError());
  if (k == 2) {
    finish_step(h, h->stage_a, dt);
    h->next_stage = 0;
  } else {
    h->next_stage = k + 1;
  }
  return HWENO_OK;
}

hweno_status hweno_set_owned_rows(hweno_t h, int jlo, int jhi) {
  if (!h) return HWENO_EINVAL;
  if (h->batch || h->g.dim != 2) return fail(h, HWENO_ESTATE, "set_owned_rows: single 2D handles only");
  if (jlo < 0 || jhi > h->P.ny || jhi <= jlo) return fail(h, HWENO_EINVAL, "set_owned_rows: need 0 <= jlo < jhi <= ny");
  h->P.jlo = jlo;
  h->P.jhi = jhi;
  drop_graphs(h);
  return HWENO_OK;
}

hweno_status hweno_copy_rows(hweno_t h, int j0, int nrows, double* buf, int to_state) {
  if (!h) return HWENO_EINVAL;
  if (h->batch || h->g.dim != 2) return fail(h, HWENO_ESTATE, "copy_rows: single 2D handles only");
  if (!buf || nrows < 1 || j0 < 0 || j0 + nrows > h->P.ny) return fail(h, HWENO_EINVAL, "copy_rows: rows out of range");
  if (!h->have_state) return fail(h, HWENO_ESTATE, "copy_rows: no moments set");
  // the state the next stage reads: U^n before a step, U^(1) or U^(2) between stages
  const int a = h->next_stage == 0 ? h->cur : h->stage_a;
  double* U = h->U[(a + h->next_stage) % 3];
  const size_t w = h->P.nx * sizeof(double);
  for (int q = 0; q < h->P.nvar * h->P.nmom; ++q) {
    double* st = U + (size_t)q * h->P.plane + (size_t)j0 * h->P.pitch;
    double* bb = buf + (size_t)q * nrows * h->P.nx;
    if (to_state)
      CK(h, cudaMemcpy2DAsync(st, h->P.pitch * sizeof(double), bb, w, w, nrows, cudaMemcpyDeviceToDevice, h->stream));
    else
      CK(h, cudaMemcpy2DAsync(bb, w, st, h->P.pitch * sizeof(double), w, nrows, cudaMemcpyDeviceToDevice, h->stream));
  }
  float* U32 = h->U32[(a + h->next_stage) % 3];
  if (to_state && U32) hw::run_shadow32(h->P, U, U32, j0, nrows, h->stream);
  return HWENO_OK;
}

hweno_status hweno_wave_speeds(hweno_t h, double* ax_ay) {
  if (!h || !ax_ay) return HWENO_EINVAL;
  if (h->batch) return fail(h, HWENO_ESTATE, "wave_speeds: single-problem handles only");
  if (!h->have_state) return fail(h, HWENO_ESTATE, "wave_speeds: no moments set");
  hweno_status s = check_status(h);
  if (s != HWENO_OK) return s;
  hw::run_wavespeed(h->P, h->U[h->cur], h->red_part, h->red_out, h->stream);
  CK(h, cudaMemcpyAsync(h->host_buf, h->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  ax_ay[0] = h->host_buf[0];
  ax_ay[1] = h->host_buf[1];
  return HWENO_OK;
}

hweno_status hweno_sync(hweno_t h) {
  if (!h) return HWENO_EINVAL;
  return check_status(h);
}

namespace {

constexpr int ADV_K = 12;   // steps per replay (a multiple of 3: the buffer rotation closes)

// ADV_K steps with the step length computed on the device, from rotation a.
cudaError_t advance_steps(hweno_t h, int a, cudaStream_t st) {
  const size_t nc = ncell(h);
  double* par = h->adv;
  double* stt = h->adv + 3;
  for (int k = 0; k < ADV_K; ++k) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    hw::run_wavespeed(h->P, h->U[a], h->red_part, h->red_out, st);
    hw::run_advance_dt(h->P, h->red_out, par, stt, h->B.status, st);
    auto run = [&](const hw::StageCall& S) {
      if (h->P.fixtab) {   // stage time from the device: t_n + c dt, c = 0, 1, 1/2
        const double cst[3] = {0.0, 1.0, 0.5};
        hw::run_fixfill(h->fix, h->fixtab, 0.0, stt + 3, stt + 1, cst[S.stage], st);
      }
      if (h->g.dim == 1) hw::run_stage_1d(h->P, h->T, h->fp32, h->B, S, st);
      else hw::run_stage_2d(h->P, h->T, h->fp32, h->B, S, st);
    };
    hw::StageCall S{};
    S.dtp = stt + 1;
    S.stage = 0; S.Uin = h->U[a]; S.Un = h->U[a]; S.Uout = h->U[b]; S.cA = 0.0; S.cB = 1.0;
    S.mask = h->mask3; S.Mod = h->ModN; S.maskN = nullptr; S.ModN = nullptr;
    S.U32in = h->U32[a]; S.U32out = h->U32[b];
    run(S);
    S.stage = 1; S.Uin = h->U[b]; S.Un = h->U[a]; S.Uout = h->U[c]; S.cA = 0.75; S.cB = 0.25;
    S.mask = h->mask3 + nc; S.Mod = h->ModK; S.maskN = h->mask3; S.ModN = h->ModN;
    S.U32in = h->U32[b]; S.U32out = h->U32[c];
    run(S);
    S.stage = 2; S.Uin = h->U[c]; S.Un = h->U[a]; S.Uout = h->U[b]; S.cA = 1.0 / 3.0; S.cB = 2.0 / 3.0;
    S.mask = h->mask3 + 2 * nc; S.Mod = h->ModK;
    S.U32in = h->U32[c]; S.U32out = h->U32[b];
    run(S);
    a = b;
  }
  return cudaGetLastError();
}

cudaError_t advance_graph(hweno_t h, int a, cudaGraphExec_t* out) {
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    e = advance_steps(h, a, cs);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) *out = nullptr;
  return e;
}

}  // namespace

hweno_status hweno_advance(hweno_t h, double t_end, double cfl, long long max_steps, double* t_done,
                           long long* steps_done) {
  if (!h) return HWENO_EINVAL;
  if (h->batch) return fail(h, HWENO_ESTATE, "advance: single-problem handles only");
  if (!h->have_state) return fail(h, HWENO_ESTATE, "advance: no moments set");
  if (h->g.indicator == 3 && !h->have_mlp) return fail(h, HWENO_ESTATE, "advance: learned indicator not set");
  if (!(t_end >= 0.0) || !isfinite(t_end) || !(cfl > 0.0) || !isfinite(cfl) || max_steps < 0)
    return fail(h, HWENO_EINVAL, "advance: need t_end >= 0, cfl > 0 and max_steps >= 0");
  if (!fix_ready(h)) return fail(h, HWENO_ESTATE, "advance: an inflow side has no fixed states");
  hweno_status s0 = check_status(h);
  if (s0 != HWENO_OK) return s0;
  if (!h->adv) CK(h, cudaMalloc(&h->adv, 8 * sizeof(double)));
  double* hb = h->host_buf + 8;
  // the device clock runs on the solution time: from h->time to h->time + t_end
  const double t0 = h->time;
  hb[0] = t0 + t_end; hb[1] = cfl; hb[2] = (double)max_steps; hb[3] = t0; hb[4] = 0.0; hb[5] = 0.0;
  CK(h, cudaMemcpyAsync(h->adv, hb, 6 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  h->stepped = false;     // several steps per replay: no single-step roll-back
  double t = 0.0, steps = 0.0;
  while (steps < (double)max_steps && t_end - t > 1e-14 * fmax(1.0, fabs(t_end))) {
    const int a = h->cur;
    const bool use_graph = h->adv_graph && !h->B.prof;
    if (use_graph && !h->agraphs[a] && advance_graph(h, a, &h->agraphs[a]) != cudaSuccess) {
      h->adv_graph = false;     // capture unavailable here: launch directly
      cudaGetLastError();
    }
    if (h->adv_graph && !h->B.prof && h->agraphs[a]) CK(h, cudaGraphLaunch(h->agraphs[a], h->stream));
    else CK(h, advance_steps(h, a, h->stream));
    CK(h, cudaMemcpyAsync(hb + 3, h->adv + 3, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const hweno_status s = check_status(h);
    if (s != HWENO_OK) return s;
    const double before = steps;
    t = hb[3] - t0;
    h->time = hb[3];
    steps = hb[5];
    if (steps == before) break;           // nothing advanced (dt could not be formed)
  }
  if (t_done) *t_done = t;
  if (steps_done) *steps_done = (long long)steps;
  return HWENO_OK;
}

hweno_status hweno_max_dt(hweno_t h, double cfl, double* dt_out) {
  if (!h || !dt_out) return HWENO_EINVAL;
  if (!h->have_state) return fail(h, HWENO_ESTATE, "max_dt: no moments set");
  if (!(cfl > 0.0)) return fail(h, HWENO_EINVAL, "max_dt: cfl must be positive");
  hweno_status s = check_status(h);
  if (s != HWENO_OK) return s;
  hw::run_wavespeed(h->P, h->U[h->cur], h->red_part, h->red_out, h->stream);
  CK(h, cudaMemcpyAsync(h->host_buf, h->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  const double ax = h->host_buf[0], ay = h->host_buf[1];
  if (!isfinite(ax) || !isfinite(ay)) return fail(h, HWENO_ENONPHYSICAL, "max_dt: non-physical cell average");
  double dt;
  if (h->g.dim == 1) dt = ax > 0.0 ? cfl * h->P.dx / ax : INFINITY;
  else {
    const double r = ax / h->P.dx + ay / h->P.dy;
    dt = r > 0.0 ? cfl / r : INFINITY;
  }
  *dt_out = dt;
  return HWENO_OK;
}

hweno_status hweno_troubled_mask(hweno_t h, unsigned char* mask, size_t count) {
  if (!h) return HWENO_EINVAL;
  if (!mask || count != 3 * ncell(h)) return fail(h, HWENO_EINVAL, "troubled_mask: count must be 3*ny*nx");
  CK(h, cudaMemcpyAsync(mask, h->mask3, count, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return HWENO_OK;
}

hweno_status hweno_totals(hweno_t h, double* sums) {
  if (!h || !sums) return HWENO_EINVAL;
  if (!h->have_state) return fail(h, HWENO_ESTATE, "totals: no moments set");
  hweno_status s = check_status(h);
  if (s != HWENO_OK) return s;
  hw::run_totals(h->P, h->U[h->cur], h->red_part, h->red_out, h->stream);
  CK(h, cudaMemcpyAsync(h->host_buf, h->red_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  const double area = h->P.dx * h->P.dy;
  for (int v = 0; v < h->P.nvar; ++v) sums[v] = h->host_buf[v] * area;
  return HWENO_OK;
}

hweno_status hweno_rhs(hweno_t h, const double* U, double* Umod, double* L, unsigned char* mask, double* aleph) {
  if (!h) return HWENO_EINVAL;
  if (!U || !Umod || !L || !mask) return fail(h, HWENO_EINVAL, "rhs: U, Umod, L and mask are required");
  if (h->g.indicator == 3 && !h->have_mlp) return fail(h, HWENO_ESTATE, "rhs: learned indicator not set (hweno_set_mlp)");
  Prob P = h->P;           // caller arrays are unpadded
  P.pitch = P.nx;
  P.plane = (long long)P.ny * P.nx;
  if (!fix_ready(h)) return fail(h, HWENO_ESTATE, "rhs: an inflow side has no fixed states");
  if (h->P.fixtab) hw::run_fixfill(h->fix, h->fixtab, h->time, nullptr, nullptr, 0.0, h->stream);
  hw::StageCall S{};
  S.stage = 3; S.Uin = U; S.Un = U; S.Uout = nullptr; S.dt = 0.0; S.cA = 0.0; S.cB = 1.0;
  S.mask = mask; S.Mod = h->ModK; S.maskN = nullptr; S.ModN = nullptr;
  S.Lout = L; S.Umod = Umod; S.aleph = aleph;
  if (h->g.dim == 1) hw::run_stage_1d(P, h->T, h->fp32, h->B, S, h->stream);
  else hw::run_stage_2d(P, h->T, h->fp32, h->B, S, h->stream);
  CK(h, cudaGetLastError());
  return HWENO_OK;
}

// ---------------------------------------------------------------- learned indicator

static int device_sms() {
  int dev = 0, n = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

int hweno_mlp_nparam(void) { return hw::mlp_nparam(); }

hweno_status hweno_set_mlp(hweno_t h, const float* params, int on_device, float conf) {
  if (!h || !params || !(conf > 0.0f)) return HWENO_EINVAL;
  if (h->g.indicator != 3) return fail(h, HWENO_ESTATE, "set_mlp: the handle was not created with indicator 3 (mlp)");
  const size_t nb = hw::mlp_nparam() * sizeof(float);
  CK(h, cudaMemcpyAsync(h->mlp, params, nb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  drop_graphs(h);
  h->B.mlp = h->mlp;
  h->B.mlp_conf = conf;
  h->B.mlp_stats = h->mlp_stats;
  h->have_mlp = true;
  return HWENO_OK;
}

hweno_status hweno_mlp_probe(hweno_t h, float* prob) {
  if (!h) return HWENO_EINVAL;
  if (h->g.indicator != 3) return fail(h, HWENO_ESTATE, "mlp_probe: the handle was not created with indicator 3 (mlp)");
  h->B.mlp_prob = prob;
  drop_graphs(h);
  return HWENO_OK;
}

hweno_status hweno_mlp_fallbacks(hweno_t h, long long* cells) {
  if (!h || !cells) return HWENO_EINVAL;
  if (!h->mlp_stats) { *cells = 0; return HWENO_OK; }
  int v = 0;
  CK(h, cudaMemcpyAsync(&v, h->mlp_stats, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemsetAsync(h->mlp_stats, 0, sizeof(int), h->stream));
  *cells = v;
  return HWENO_OK;
}

hweno_status hweno_set_fixed_state(hweno_t h, int side, const hweno_fixed_state* f) {
  if (!h || !f) return HWENO_EINVAL;
  if (h->batch || h->g.dim != 2 || h->g.eq != HWENO_EULER || h->fp32 != hw::PREC_FP64 || h->g.indicator == 3)
    return fail(h, HWENO_EINVAL, "set_fixed_state: single-problem 2D Euler FP64 handles without the learned indicator");
  if (side < 0 || side > 3) return fail(h, HWENO_EINVAL, "set_fixed_state: side must be 0..3");
  const int kinds[4] = {h->bc.xlo, h->bc.xhi, h->bc.ylo, h->bc.yhi};
  const bool inflow = kinds[side] == HWENO_BC_INFLOW;
  if (kinds[side] == HWENO_BC_PERIODIC) return fail(h, HWENO_EINVAL, "set_fixed_state: the side is periodic");
  if (!inflow && !f->segment) return fail(h, HWENO_EINVAL, "set_fixed_state: only inflow sides take states without a segment");
  auto physical = [&](const double* u) {
    for (int v = 0; v < 4; ++v) if (!isfinite(u[v])) return false;
    const double p = (h->gamma - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]);
    return u[0] > 0.0 && p > 0.0;
  };
  if (f->segment && (!physical(f->a) || !isfinite(f->c0) || !isfinite(f->speed)))
    return fail(h, HWENO_EINVAL, "set_fixed_state: segment state must have rho > 0 and p > 0, c0 and speed finite");
  if (inflow && !physical(f->b)) return fail(h, HWENO_EINVAL, "set_fixed_state: inflow state must have rho > 0 and p > 0");
  hw::FixSpec& F = h->fix;
  if (!h->fixtab) {
    F.fixlen = std::max(h->P.nx, h->P.ny) + 2;
    F.n[0] = F.n[1] = h->P.ny;
    F.n[2] = F.n[3] = h->P.nx;
    F.x0 = h->g.x0; F.y0 = h->g.y0; F.dx = h->P.dx; F.dy = h->P.dy;
    for (int s = 0; s < 4; ++s) F.inflow[s] = kinds[s] == HWENO_BC_INFLOW;
    CK(h, cudaMalloc(&h->fixtab, 16 * (size_t)F.fixlen * sizeof(double)));
    CK(h, cudaMemsetAsync(h->fixtab, 0, 16 * (size_t)F.fixlen * sizeof(double), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));   // done before any later stream fills the table
    h->P.fixtab = h->fixtab;
    h->P.fixlen = F.fixlen;
  }
  F.seg[side] = f->segment ? 1 : 0;
  F.c0[side] = f->c0;
  F.speed[side] = f->speed;
  for (int v = 0; v < 4; ++v) { F.a[side][v] = f->a[v]; F.b[side][v] = f->b[v]; }
  h->fix_set[side] = true;
  drop_graphs(h);
  return HWENO_OK;
}

hweno_status hweno_set_time(hweno_t h, double t) {
  if (!h || !isfinite(t)) return HWENO_EINVAL;
  if (h->batch) return fail(h, HWENO_ESTATE, "set_time: single-problem handles only");
  h->time = t;
  h->stepped = false;
  return HWENO_OK;
}

hweno_status hweno_get_time(hweno_t h, double* t) {
  if (!h || !t) return HWENO_EINVAL;
  *t = h->time;
  return HWENO_OK;
}

hweno_status hweno_set_positivity_check(hweno_t h, int on) {
  if (!h) return HWENO_EINVAL;
  h->positivity = on != 0;
  h->P.positivity = on != 0;
  drop_graphs(h);
  if (h->batch) {
    for (auto& q : h->probs) q.P.positivity = on != 0;
    CK(h, cudaMemcpyAsync(h->dprobs, h->probs.data(), h->probs.size() * sizeof(hw::BProb), cudaMemcpyHostToDevice,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
  }
  return HWENO_OK;
}

hweno_status hweno_set_tma(hweno_t h, int on) {
  if (!h) return HWENO_EINVAL;
  if (on != 0 && on != 1) return fail(h, HWENO_EINVAL, "set_tma: on must be 0 or 1");
  if (on && !h->tma_ok)
    return fail(h, HWENO_ESTATE, "set_tma: TMA staging is for single 2D Euler FP32-bulk handles");
  h->tma_on = on != 0;
  h->B.tmG = h->tma_on ? &h->tmG : nullptr;
  drop_graphs(h);
  return HWENO_OK;
}

hweno_status hweno_set_fused(hweno_t h, int on) {
  if (!h) return HWENO_EINVAL;
  if (on != 0 && on != 1) return fail(h, HWENO_EINVAL, "set_fused: on must be 0 or 1");
  const bool ind_ok = h->g.indicator == HWENO_IND_NONE || h->g.indicator == HWENO_IND_KXRCF ||
                      h->g.indicator == HWENO_IND_ALL;
  const bool ok2 = h->g.dim == 2 && h->g.eq == HWENO_EULER && h->P.sol_j == 0;
  const bool ok1 = h->g.dim == 1 && !h->P.charwise;
  if (on && (h->batch || !ind_ok || !(ok1 || ok2)))
    return fail(h, HWENO_ESTATE, "set_fused: the fused stage is for single 1D handles (component-wise) and 2D Euler "
                                 "handles with the KXRCF, none or all indicator");
  // the fused stage keeps no float copy of the state: renew it when the pipeline takes over
  if (!on && h->P.fused && h->have_state && h->U32[h->cur])
    hw::run_shadow32(h->P, h->U[h->cur], h->U32[h->cur], 0, h->P.ny, h->stream);
  h->P.fused = on;
  drop_graphs(h);
  return HWENO_OK;
}

hweno_status hweno_set_solid(hweno_t h, int i0, int j1) {
  if (!h) return HWENO_EINVAL;
  if (h->batch || h->g.dim != 2 || h->g.eq != HWENO_EULER || h->g.precision != 0 || h->g.indicator == 3)
    return fail(h, HWENO_ESTATE, "set_solid: single 2D Euler FP64 handles without the learned indicator");
  if (j1 == 0) { h->P.sol_i = 0; h->P.sol_j = 0; drop_graphs(h); return HWENO_OK; }
  const int nx = h->P.nx, ny = h->P.ny;
  if (i0 < 0 || i0 >= nx || j1 < 1 || j1 > ny || (i0 > 0 && i0 < 4) || (j1 < ny && ny - j1 < 4))
    return fail(h, HWENO_EINVAL, "set_solid: need 0 <= i0 < nx, 1 <= j1 <= ny and 4 fluid cells beyond each face");
  if ((i0 > 0 && h->P.bc[1] == HWENO_BC_PERIODIC) || (j1 < ny && h->P.bc[2] == HWENO_BC_PERIODIC))
    return fail(h, HWENO_EINVAL, "set_solid: the sides the block touches may not be periodic");
  if (h->P.fused) return fail(h, HWENO_ESTATE, "set_solid: the fused stage has no solid block (hweno_set_fused 0)");
  h->P.sol_i = i0;
  h->P.sol_j = j1;
  drop_graphs(h);
  return HWENO_OK;
}

hweno_status hweno_set_persistence(hweno_t h, int persist) {
  if (!h) return HWENO_EINVAL;
  if (persist != 0 && persist != 1) return fail(h, HWENO_EINVAL, "set_persistence: persist must be 0 or 1");
  h->P.persist = persist;
  drop_graphs(h);
  if (h->batch) {
    for (auto& q : h->probs) q.P.persist = persist;
    CK(h, cudaMemcpyAsync(h->dprobs, h->probs.data(), h->probs.size() * sizeof(hw::BProb), cudaMemcpyHostToDevice,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
  }
  return HWENO_OK;
}

hweno_status hweno_rerecon_count(hweno_t h, long long* cells) {
  if (!h || !cells) return HWENO_EINVAL;
  if (h->batch) return fail(h, HWENO_ESTATE, "rerecon_count: single-problem handles only");
  unsigned long long v = 0;
  CK(h, cudaMemcpyAsync(&v, h->B.rerec, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemsetAsync(h->B.rerec, 0, sizeof v, h->stream));
  *cells = (long long)v;
  return HWENO_OK;
}

hweno_status hweno_features(hweno_t h, const double* U, const int* cells, int n, float* X) {
  if (!h || !U || !cells || !X || n < 0) return HWENO_EINVAL;
  if (h->g.dim != 2 || h->g.eq != HWENO_EULER) return fail(h, HWENO_EINVAL, "features: 2D Euler only");
  Prob P = h->P;
  P.pitch = P.nx;
  P.plane = (long long)P.ny * P.nx;
  CK(h, hw::run_features(P, U, cells, n, X, h->stream));
  return HWENO_OK;
}

hweno_status hweno_mlp_forward(const float* params, const float* X, int n, float* prob, void* stream) {
  if (!params || !prob || n < 0) return HWENO_EINVAL;
  if (n == 0) return HWENO_OK;
  if (!X) return HWENO_EINVAL;
  return hw::run_mlp_forward(params, X, n, prob, device_sms(), (cudaStream_t)stream) == cudaSuccess ? HWENO_OK
                                                                                                   : HWENO_ECUDA;
}

hweno_status hweno_mlp_loss_grad(const float* params, const float* X, const float* y, const float* w, int n,
                                 float* grad, float* loss, void* stream) {
  if (!params || !grad || !loss || n < 0) return HWENO_EINVAL;
  if (n == 0) return HWENO_OK;
  if (!X || !y) return HWENO_EINVAL;
  return hw::run_mlp_train(params, X, y, w, n, grad, loss, device_sms(), (cudaStream_t)stream) == cudaSuccess
             ? HWENO_OK : HWENO_ECUDA;
}

hweno_status hweno_mlp_adam(float* params, const float* grad, float* m1, float* m2, int step, float lr,
                            void* stream) {
  if (!params || !grad || !m1 || !m2 || step < 1 || !(lr > 0.0f)) return HWENO_EINVAL;
  return hw::run_adam(params, grad, m1, m2, step, lr, (cudaStream_t)stream) == cudaSuccess ? HWENO_OK : HWENO_ECUDA;
}

hweno_status hweno_profile(hweno_t h, int enable) {
  if (!h) return HWENO_EINVAL;
  CK(h, cudaStreamSynchronize(h->stream));
  double ms[hw::Prof::KINDS];
  int n[hw::Prof::KINDS];
  h->prof.read(ms, n, hw::Prof::KINDS);    // drop anything recorded so far
  h->B.prof = enable ? &h->prof : nullptr;
  return HWENO_OK;
}

hweno_status hweno_profile_read(hweno_t h, double* ms, int* launches, int nkinds) {
  if (!h) return HWENO_EINVAL;
  if (!ms || !launches || nkinds < 4) return fail(h, HWENO_EINVAL, "profile_read: need at least 4 slots");
  CK(h, cudaStreamSynchronize(h->stream));
  h->prof.read(ms, launches, std::min(nkinds, hw::Prof::KINDS));
  for (int k = hw::Prof::KINDS; k < nkinds; ++k) { ms[k] = 0.0; launches[k] = 0; }
  CK(h, cudaGetLastError());
  return HWENO_OK;
}

// ---------------------------------------------------------------- batches

namespace {

// Descriptors of every problem for the current update-tile variant.
void layout_batch(hweno_t h) {
  static const int TXS[3] = {32, 16, 64}, TYS[3] = {4, 8, 2};
  const int tx = TXS[h->tile_variant], ty = TYS[h->tile_variant];
  int rec = 0, upd = 0;
  for (auto& q : h->probs) {
    q.rec_first = rec;
    q.upd_first = upd;
    q.tiles_x = (q.P.nx + tx - 1) / tx;
    rec += (q.P.nx * q.P.ny + 127) / 128;
    upd += q.tiles_x * ((q.P.ny + ty - 1) / ty);
  }
  h->n_rec = rec;
  h->n_upd = upd;
}

size_t batch_count(const hweno_s* h, int k) {
  const Prob& P = h->probs[k].P;
  return (size_t)P.nvar * P.nmom * P.nx * P.ny;
}

hweno_status batch_graph(hweno_t h, int a, const double* dt_in, double cfl, cudaGraphExec_t* out);

}  // namespace

hweno_status hweno_create_batch(const hweno_grid* grids, const hweno_bc* bcs, int n, double gamma, hweno_t* out) {
  if (!out || !grids || !bcs || n < 1) return HWENO_EINVAL;
  *out = nullptr;
  for (int k = 0; k < n; ++k) {
    std::string why;
    if (validate(&grids[k], &bcs[k], gamma, why) != HWENO_OK) {
      fprintf(stderr, "hweno_create_batch: problem %d: %s\n", k, why.c_str());
      return HWENO_EINVAL;
    }
    const hweno_grid& g = grids[k];
    if (bcs[k].xlo == HWENO_BC_INFLOW || bcs[k].xhi == HWENO_BC_INFLOW || bcs[k].ylo == HWENO_BC_INFLOW ||
        bcs[k].yhi == HWENO_BC_INFLOW) {
      fprintf(stderr, "hweno_create_batch: problem %d: inflow sides run on single-problem handles\n", k);
      return HWENO_EINVAL;
    }
    if (g.dim != 2 || g.eq != HWENO_EULER || g.precision != grids[0].precision ||
        g.indicator != grids[0].indicator || g.beta_of_q != grids[0].beta_of_q ||
        memcmp(g.gamma_bar, grids[0].gamma_bar, sizeof g.gamma_bar) != 0) {
      fprintf(stderr, "hweno_create_batch: problem %d: batches hold 2D Euler problems sharing precision, "
              "indicator and linear weights\n", k);
      return HWENO_EINVAL;
    }
    if (g.indicator == HWENO_IND_MLP) {
      fprintf(stderr, "hweno_create_batch: the learned indicator runs on single-problem handles\n");
      return HWENO_EINVAL;
    }
  }
  hweno_s* h = new hweno_s();
  h->batch = true;
  h->nprob = n;
  h->g = grids[0];
  h->bc = bcs[0];
  h->gamma = gamma;
  h->fp32 = grids[0].precision;
  if (cudaGetDevice(&h->dev) != cudaSuccess) { delete h; return HWENO_ECUDA; }
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev);
  long long tu = 0, tg = 0, ta = 0, tm = 0, tc = 0;
  for (int k = 0; k < n; ++k) {
    hw::BProb q{};
    Prob& P = q.P;
    const hweno_grid& g = grids[k];
    P.nx = g.nx; P.ny = g.ny;
    P.pitch = (P.nx + 31) / 32 * 32; P.plane = (long long)P.ny * P.pitch;
    P.gpitch = P.pitch; P.gplane = P.plane;
    P.nvar = 4; P.nmom = 3; P.eq = HWENO_EULER; P.indicator = g.indicator; P.tvb_m = g.tvb_m;
    P.bc[0] = bcs[k].xlo; P.bc[1] = bcs[k].xhi; P.bc[2] = bcs[k].ylo; P.bc[3] = bcs[k].yhi;
    P.dx = (g.x1 - g.x0) / P.nx; P.dy = (g.y1 - g.y0) / P.ny;
    P.gamma = gamma; P.adv_a = 0.0; P.adv_b = 0.0; P.nsm = nsm; P.positivity = 1; P.persist = 1;
    P.jlo = 0; P.jhi = P.ny;
    fill_consts(P);
    q.uoff = tu; q.goff = tg; q.aoff = ta; q.moff = tm; q.coff = tc;
    tu += 12 * P.plane; tg += 64 * P.gplane; ta += 5 * P.gplane; tm += 8 * P.plane; tc += (long long)P.nx * P.ny;
    h->probs.push_back(q);
  }
  h->tot_cells = tc;
  h->P = h->probs[0].P;
  build_tables(h);
  layout_batch(h);
  const size_t esz = h->fp32 == hw::PREC_FP32 ? sizeof(float) : sizeof(double);   // df64 is 8 bytes
  bool ok = true;
  for (int k = 0; k < 3; ++k) ok = ok && cudaMalloc(&h->U[k], tu * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->B.G, tg * esz) == cudaSuccess;
  ok = ok && cudaMalloc(&h->B.aux, ta * esz) == cudaSuccess;
  ok = ok && cudaMalloc(&h->ModN, tm * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->ModK, tm * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->mask3, 3 * tc) == cudaSuccess;
  ok = ok && cudaMalloc(&h->blist, tc * sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->B.count, 4 * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->B.status, sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->speeds, 2 * n * sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->dt_out, n * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->bar, 2 * sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->pstatus, n * sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->dprobs, n * sizeof(hw::BProb)) == cudaSuccess;
  ok = ok && cudaMallocHost(&h->host_buf, 16 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_all(h);
    delete h;
    fprintf(stderr, "hweno_create_batch: device allocation failed\n");
    return HWENO_ENOMEM;
  }
  cudaMemcpy(h->dprobs, h->probs.data(), n * sizeof(hw::BProb), cudaMemcpyHostToDevice);
  cudaMemset(h->B.status, 0, sizeof(unsigned));
  cudaMemset(h->mask3, 0, 3 * tc);
  cudaMemset(h->bar, 0, 2 * sizeof(unsigned));
  cudaMemset(h->blist, 0, tc * sizeof(unsigned long long));
  cudaMemset(h->pstatus, 0, n * sizeof(unsigned));
  cudaMemset(h->dt_out, 0, n * sizeof(double));
  for (int k = 0; k < 3; ++k) cudaMemset(h->U[k], 0, tu * sizeof(double));
  if (cudaDeviceSynchronize() != cudaSuccess) { free_all(h); delete h; return HWENO_ECUDA; }
  *out = h;
  return HWENO_OK;
}

hweno_status hweno_batch_set_tile(hweno_t h, int variant) {
  if (!h || !h->batch || variant < 0 || variant > 2) return HWENO_EINVAL;
  if (variant == h->tile_variant) return HWENO_OK;
  CK(h, cudaStreamSynchronize(h->stream));
  h->tile_variant = variant;
  layout_batch(h);
  CK(h, cudaMemcpy(h->dprobs, h->probs.data(), h->nprob * sizeof(hw::BProb), cudaMemcpyHostToDevice));
  drop_graphs(h);
  return HWENO_OK;
}

hweno_status hweno_batch_set_moments(hweno_t h, int k, const double* m, size_t count, int on_device) {
  if (!h || !h->batch || k < 0 || k >= h->nprob) return HWENO_EINVAL;
  if (!m || count != batch_count(h, k)) return fail(h, HWENO_EINVAL, "batch_set_moments: count must be 12*ny*nx");
  const Prob& P = h->probs[k].P;
  CK(h, cudaMemcpy2DAsync(h->U[h->cur] + h->probs[k].uoff, P.pitch * sizeof(double), m, P.nx * sizeof(double),
                          P.nx * sizeof(double), (size_t)12 * P.ny,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemsetAsync(h->B.status, 0, sizeof(unsigned), h->stream));
  h->have_state = true;
  h->stepped = false;
  if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
  return HWENO_OK;
}

hweno_status hweno_batch_get_moments(hweno_t h, int k, double* m, size_t count, int on_device) {
  if (!h || !h->batch || k < 0 || k >= h->nprob) return HWENO_EINVAL;
  if (!m || count != batch_count(h, k)) return fail(h, HWENO_EINVAL, "batch_get_moments: count must be 12*ny*nx");
  if (!on_device) {
    const hweno_status s = check_status(h);
    if (s != HWENO_OK) return s;
  }
  const Prob& P = h->probs[k].P;
  CK(h, cudaMemcpy2DAsync(m, P.nx * sizeof(double), h->U[h->cur] + h->probs[k].uoff, P.pitch * sizeof(double),
                          P.nx * sizeof(double), (size_t)12 * P.ny,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
  return HWENO_OK;
}

hweno_status hweno_batch_troubled_mask(hweno_t h, int k, unsigned char* mask, size_t count) {
  if (!h || !h->batch || k < 0 || k >= h->nprob) return HWENO_EINVAL;
  const Prob& P = h->probs[k].P;
  const size_t nc = (size_t)P.nx * P.ny;
  if (!mask || count != 3 * nc) return fail(h, HWENO_EINVAL, "batch_troubled_mask: count must be 3*ny*nx");
  for (int st = 0; st < 3; ++st)
    CK(h, cudaMemcpyAsync(mask + st * nc, h->mask3 + st * h->tot_cells + h->probs[k].coff, nc,
                          cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return HWENO_OK;
}

hweno_status hweno_batch_status(hweno_t h, unsigned* bits, int n) {
  if (!h || !h->batch || !bits || n != h->nprob) return HWENO_EINVAL;
  for (int k = 0; k < n; ++k) bits[k] = h->last_pstatus.empty() ? 0u : h->last_pstatus[k];
  return HWENO_OK;
}

int hweno_batch_uses_graph(hweno_t h) {
  if (!h || !h->batch) return -1;
  return (h->use_graph && h->graphs[h->prev] != nullptr) ? 1 : 0;
}

hweno_status hweno_batch_dt(hweno_t h, double* dt, int n) {
  if (!h || !h->batch || !dt || n != h->nprob) return HWENO_EINVAL;
  CK(h, cudaMemcpyAsync(dt, h->dt_out, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return HWENO_OK;
}

hweno_status hweno_batch_set_barrier(hweno_t h, long long spin_limit, int extra_arrivals) {
  if (!h || !h->batch) return HWENO_EINVAL;
  if (spin_limit < 1 || extra_arrivals < 0 || extra_arrivals > 1024)
    return fail(h, HWENO_EINVAL, "batch_set_barrier: need spin_limit >= 1 and 0 <= extra_arrivals <= 1024");
  h->spin_limit = (unsigned long long)spin_limit;
  h->bar_extra = (unsigned)extra_arrivals;
  drop_graphs(h);
  return HWENO_OK;
}

hweno_status hweno_step_batch(hweno_t h, const double* dt_device, double cfl) {
  if (!h || !h->batch) return HWENO_EINVAL;
  if (!h->have_state) return fail(h, HWENO_ESTATE, "step_batch: no moments set");
  if (!dt_device && !(cfl > 0.0)) return fail(h, HWENO_EINVAL, "step_batch: need dt_device or cfl > 0");
  const int a = h->cur;
  if (h->graph_dt != dt_device || h->graph_cfl != cfl || h->graph_variant != h->tile_variant) {
    drop_graphs(h);
    h->graph_dt = dt_device;
    h->graph_cfl = cfl;
    h->graph_variant = h->tile_variant;
  }
  if (h->use_graph && !h->graphs[a]) {
    const hweno_status s = batch_graph(h, a, dt_device, cfl, &h->graphs[a]);
    if (s != HWENO_OK) {     // capture unsupported here: launch directly from now on
      h->use_graph = false;
      cudaGetLastError();
    }
  }
  if (h->use_graph && h->graphs[a]) {
    CK(h, cudaGraphLaunch(h->graphs[a], h->stream));
  } else {
    hw::BatchStage S{};
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    const long long T = h->tot_cells;
    CK(h, cudaMemsetAsync(h->speeds, 0, 2 * h->nprob * sizeof(unsigned long long), h->stream));
    CK(h, cudaMemsetAsync(h->B.count, 0, 4 * sizeof(int), h->stream));
    for (int st = 0; st < 3; ++st) {
      S.probs = h->dprobs; S.nprob = h->nprob; S.n_rec = h->n_rec; S.n_upd = h->n_upd;
      S.G = h->B.G; S.aux = h->B.aux; S.list = h->blist; S.count = h->B.count + st;
      S.speeds = h->speeds; S.dt_in = dt_device; S.dt_out = h->dt_out; S.cfl = cfl;
      S.status = h->B.status; S.pstatus = h->pstatus; S.bar = h->bar; S.stage = st;
      S.spin_limit = h->spin_limit; S.bar_extra = h->bar_extra;
      S.Un = h->U[a];
      if (st == 0) { S.Uin = h->U[a]; S.Uout = h->U[b]; S.cA = 0.0; S.cB = 1.0; S.Mod = h->ModN; S.ModN = nullptr;
                     S.mask = h->mask3; S.maskN = nullptr; }
      if (st == 1) { S.Uin = h->U[b]; S.Uout = h->U[c]; S.cA = 0.75; S.cB = 0.25; S.Mod = h->ModK; S.ModN = h->ModN;
                     S.mask = h->mask3 + T; S.maskN = h->mask3; }
      if (st == 2) { S.Uin = h->U[c]; S.Uout = h->U[b]; S.cA = 1.0 / 3.0; S.cB = 2.0 / 3.0; S.Mod = h->ModK;
                     S.ModN = h->ModN; S.mask = h->mask3 + 2 * T; S.maskN = h->mask3; }
      CK(h, cudaMemsetAsync(h->bar, 0, sizeof(unsigned), h->stream));
      CK(h, hw::run_batch_stage(h->T, h->fp32, h->tile_variant, S, h->P.nsm, h->stream));
    }
  }
  h->prev = a;
  h->cur = (a + 1) % 3;
  h->stepped = true;
  return HWENO_OK;
}

}  // extern "C"

namespace {

// Capture one batched step (memsets + three cooperative stage launches) for the
// state rotation starting at buffer a.
hweno_status batch_graph(hweno_t h, int a, const double* dt_in, double cfl, cudaGraphExec_t* out) {
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return HWENO_ECUDA;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  const int b = (a + 1) % 3, c = (a + 2) % 3;
  const long long T = h->tot_cells;
  if (e == cudaSuccess) {
    cudaMemsetAsync(h->speeds, 0, 2 * h->nprob * sizeof(unsigned long long), cs);
    cudaMemsetAsync(h->B.count, 0, 4 * sizeof(int), cs);
    for (int st = 0; st < 3 && e == cudaSuccess; ++st) {
      hw::BatchStage S{};
      S.probs = h->dprobs; S.nprob = h->nprob; S.n_rec = h->n_rec; S.n_upd = h->n_upd;
      S.G = h->B.G; S.aux = h->B.aux; S.list = h->blist; S.count = h->B.count + st;
      S.speeds = h->speeds; S.dt_in = dt_in; S.dt_out = h->dt_out; S.cfl = cfl;
      S.status = h->B.status; S.pstatus = h->pstatus; S.bar = h->bar; S.stage = st;
      S.spin_limit = h->spin_limit; S.bar_extra = h->bar_extra; S.Un = h->U[a];
      if (st == 0) { S.Uin = h->U[a]; S.Uout = h->U[b]; S.cA = 0.0; S.cB = 1.0; S.Mod = h->ModN; S.ModN = nullptr;
                     S.mask = h->mask3; S.maskN = nullptr; }
      if (st == 1) { S.Uin = h->U[b]; S.Uout = h->U[c]; S.cA = 0.75; S.cB = 0.25; S.Mod = h->ModK; S.ModN = h->ModN;
                     S.mask = h->mask3 + T; S.maskN = h->mask3; }
      if (st == 2) { S.Uin = h->U[c]; S.Uout = h->U[b]; S.cA = 1.0 / 3.0; S.cB = 2.0 / 3.0; S.Mod = h->ModK;
                     S.ModN = h->ModN; S.mask = h->mask3 + 2 * T; S.maskN = h->mask3; }
      cudaMemsetAsync(h->bar, 0, sizeof(unsigned), cs);
      e = hw::run_batch_stage(h->T, h->fp32, h->tile_variant, S, h->P.nsm, cs);
    }
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    *out = nullptr;
    return fail(h, HWENO_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  }
  return HWENO_OK;
}

}  // namespace
