// Host runtime of the propagation library: context, device layout, the
// launch sequence of one time step, and the C ABI declared in tsbz.h.
//
// Time step n -> n+1 (all sub-simulations advance together):
//   field(STEP)                          q = k + A(t_n + dt/2), q_obs = k + A(t_{n+1})
//   for m = 1..4: bra(t_{m-1}) ; stage m  Taylor recurrence, psi accumulates
//   bra_J(psi) ; observe(psi)            projections and sums at t_{n+1}
//   finalize(STEP)                       rho, norms, J(t_{n+1}); step += 1
//   hxc                                  v_Hxc[rho(t_{n+1})], v_eff
// Term buffers: stage 1 psi -> tA, stage 2 tA -> tB (psi += t1 + t2),
// stage 3 tB -> tA (psi += t3), stage 4 tA -> (psi += t4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tsbz.h"
#include "tsbz_host.h"
#include "tsbz_internal.h"
#include "tsbz_bulk.cuh"

namespace {

struct HostCell {
  tsbz_cell_desc desc;
  std::vector<double> atoms;
  CellDev dev;
  std::vector<double> vloc, pnorm;
  double2* tw[3] = {nullptr, nullptr, nullptr};
  std::vector<int> unit_ids;
  int* d_unit_ids = nullptr;
  std::vector<int> hxc_subs;   // non-frozen sub-simulations of this cell
  int* d_hxc_subs = nullptr;
  bool pa_by_stage = false;    // the last stage 4 also wrote P (next step) and Pa
  bool p_by_obs = false;       // the last observation's Pa pass also wrote P (next step)
  int variant = 0;             // kernel variant (tsbz_autotune / tsbz_set_variant)
  bool tables_step = false;    // the phase tables hold a time step's q (not J(0-/0+) tables)
  double tune_ms[TSBZ_MAX_VARIANTS] = {0, 0, 0, 0};   // ms per step measured per variant
};

struct HostSub {
  int cell = 0;
  int n_k = 0;
  std::vector<double> k;
  double dt = 0.0;
  int max_steps = 0;
  int unit0 = 0;
  std::vector<double> A;   // (2 max_steps + 1) * 3
  bool field_dirty = true;
  bool field_const = true;   // every sample of A equal (kick or no field)
  bool loaded = false;
  bool need_init = false;
  bool need_j0plus = false;
  int steps = 0;
  double* A_d = nullptr;
  double* J = nullptr;
  double* J0m = nullptr;
  double* rho = nullptr;
  double* vhxc = nullptr;
  double* norms = nullptr;
  void* veff = nullptr;
  void* veff_save = nullptr;   // the other v_eff of an ETRS step
};

}  // namespace

struct tsbz_ctx {
  int device = 0;
  int precision = TSBZ_FP64;
  cudaStream_t stream = nullptr;
  bool has_alloc = false;
  tsbz_alloc alloc{};
  std::string err;
  std::vector<HostCell> cells;
  std::vector<HostSub> subs;
  bool laid_out = false;
  std::vector<void*> owned;
  void* psi = nullptr;
  void* tA = nullptr;
  void* tB = nullptr;
  void* P = nullptr;
  void* Pa = nullptr;
  void* vnl = nullptr;     // non-local term of the tensor-core mode
  void* ph_half = nullptr;
  void* ph_obs = nullptr;
  void* ph_next = nullptr;   // tables of the next step (single-precision mode)
  long long ph_stride = 1;
  bool p_next_valid = false; // P holds the projections of psi for the coming step
  double* rho_part = nullptr;
  double* jk_part = nullptr;
  double* nrm_part = nullptr;
  double* q_half = nullptr;
  double* q_obs = nullptr;
  double* kcart = nullptr;
  void* qt_half = nullptr;
  UnitDev* d_units = nullptr;
  SubDev* d_subs = nullptr;
  CellDev* d_cells = nullptr;
  int* d_steps = nullptr;
  int* d_status = nullptr;
  int* d_mask = nullptr;
  int* d_active = nullptr;   // per sub-simulation: takes part in the current step
  int propagator = TSBZ_PROP_TAYLOR4;
  double dt_scale = 1.0;     // of the stage launches being issued (ETRS half steps: 1/2)
  void* psi_save = nullptr;  // psi(t_n) during an ETRS step (allocated on first use)
  const double* d_filt = nullptr;  // ground-state solver: filter coefficients per unit (stage m = 0)
  double* d_jtile = nullptr; // per sub-simulation: [TSBZ_FIN_MAX_TILES][3] partial currents of the finalize
  int fin_tiles = 16;        // CTAs per sub-simulation of the finalize
  int* d_jcount = nullptr;   // per sub-simulation: finalize tiles done
  double2* work_a = nullptr;
  double2* work_b = nullptr;
  double2* staging = nullptr;
  long long staging_elems = 0;
  long long n_units = 0;
  size_t psi_bytes = 0, p_bytes = 0;   // sizes of psi (= tA = tB) and P
  std::vector<long long> unit_psi_off;
  long long launches = 0;
  bool prof = false;
  bool graphs = false;
  cudaStream_t gstream = nullptr;     // the library's own stream for graph capture and replay
  cudaGraphExec_t step_graph = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  long long graph_launches = 0;       // kernels in one captured step
  double times[7] = {0, 0, 0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_marks;   // (family, event index of start)
  size_t ev_next = 0;
  size_t elem_size() const { return precision == TSBZ_FP64 ? sizeof(double2) : sizeof(float2); }
};

namespace {

enum { FAM_BRA = 0, FAM_STAGE = 1, FAM_OBS = 2, FAM_FIN = 3, FAM_HXC = 4, FAM_FIELD = 5, FAM_KET = 6 };
#define TSBZ_N_FAM 7

int set_err(tsbz_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return set_err(ctx, TSBZ_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

int dalloc(tsbz_ctx* ctx, size_t bytes, void** out) {
  bytes = bytes ? bytes : 256;
  void* p = nullptr;
  if (ctx->has_alloc) {
    p = ctx->alloc.alloc(bytes, ctx->alloc.user);
    if (!p) return set_err(ctx, TSBZ_ENOMEM, "caller allocator returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, TSBZ_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
  }
  ctx->owned.push_back(p);
  *out = p;
  return TSBZ_OK;
}

void dfree(tsbz_ctx* ctx, void* p) {
  if (!p) return;
  for (size_t i = 0; i < ctx->owned.size(); ++i)
    if (ctx->owned[i] == p) {
      ctx->owned.erase(ctx->owned.begin() + (long)i);
      break;
    }
  if (ctx->has_alloc)
    ctx->alloc.free(p, ctx->alloc.user);
  else
    cudaFree(p);
}

template <typename P> int dalloc_t(tsbz_ctx* ctx, size_t count, P** out) {
  void* p = nullptr;
  int rc = dalloc(ctx, count * sizeof(P), &p);
  *out = static_cast<P*>(p);
  return rc;
}

void ev_start(tsbz_ctx* ctx, int fam) {
  if (!ctx->prof) return;
  while (ctx->ev_pool.size() < ctx->ev_next + 2) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    ctx->ev_pool.push_back(e);
  }
  cudaEventRecord(ctx->ev_pool[ctx->ev_next], ctx->stream);
  ctx->ev_marks.push_back({fam, (int)ctx->ev_next});
  ctx->ev_next += 2;
}

void ev_stop(tsbz_ctx* ctx) {
  if (!ctx->prof) return;
  cudaEventRecord(ctx->ev_pool[ctx->ev_marks.back().second + 1], ctx->stream);
}

LaunchSet make_set(tsbz_ctx* ctx, HostCell& hc) {
  LaunchSet L;
  L.cell = hc.dev;
  L.units = ctx->d_units;
  L.unit_ids = hc.d_unit_ids;
  L.n_units = (int)hc.unit_ids.size();
  L.subs = ctx->d_subs;
  L.kcart = ctx->kcart;
  L.q_half = ctx->q_half;
  L.q_obs = ctx->q_obs;
  L.ph_half = ctx->ph_half;
  L.ph_obs = ctx->ph_obs;
  L.ph_next = ctx->ph_next;
  L.ph_stride = ctx->ph_stride;
  L.qt_half = ctx->qt_half;
  L.variant = hc.variant;
  L.dt_scale = ctx->dt_scale;
  L.filt = ctx->d_filt;
  return L;
}

int layout(tsbz_ctx* ctx) {
  if (ctx->laid_out) return TSBZ_OK;
  if (ctx->subs.empty()) return set_err(ctx, TSBZ_ESTATE, "no sub-simulation added");
  const size_t es = ctx->elem_size();
  std::vector<UnitDev> units;
  std::vector<double> kc;
  long long psi_e = 0, p_e = 0, pa_e = 0, rho_e = 0, jk_e = 0, nrm_e = 0;
  long long ph_stride = 1, stage_max = 0, work_max = 0;
  for (auto& hc : ctx->cells) {
    hc.unit_ids.clear();
    hc.hxc_subs.clear();
    ph_stride = std::max<long long>(ph_stride, (long long)hc.dev.n_atoms * 3 * hc.dev.nmax);
  }
  // finalize tiles: TSBZ_FIN_TILES per sub-simulation; with units that take a whole CTA
  // each, as many as the largest such sub-simulation has k-points (at most
  // TSBZ_FIN_MAX_TILES)
  int fin_units = TSBZ_FIN_TILES;
  for (size_t s = 0; s < ctx->subs.size(); ++s)
    if (fin_wide(ctx->cells[ctx->subs[s].cell].dev)) fin_units = std::max(fin_units, ctx->subs[s].n_k);
  ctx->fin_tiles = std::min(TSBZ_FIN_MAX_TILES, fin_units);
  for (size_t s = 0; s < ctx->subs.size(); ++s) {
    HostSub& hs = ctx->subs[s];
    HostCell& hc = ctx->cells[hs.cell];
    const CellDev& c = hc.dev;
    hs.unit0 = (int)units.size();
    for (int k = 0; k < hs.n_k; ++k) {
      UnitDev U;
      U.psi_off = psi_e;
      U.p_off = p_e;
      U.pa_off = pa_e;
      U.rho_off = rho_e;
      U.jk_off = jk_e;
      U.nrm_off = nrm_e;
      U.sub = (int)s;
      U.kloc = k;
      psi_e += (long long)c.n_bands * c.npts;
      p_e += (long long)c.n_bands * c.n_proj;
      pa_e += 4LL * c.n_bands * c.n_proj;
      rho_e += (long long)c.n_bgroups * c.npts;
      jk_e += 3LL * c.n_tiles * c.n_bgroups;
      nrm_e += (long long)c.n_tiles * c.n_bands;
      hc.unit_ids.push_back((int)units.size());
      ctx->unit_psi_off.push_back(U.psi_off);
      units.push_back(U);
      for (int ax = 0; ax < 3; ++ax) kc.push_back(hs.k[3 * k + ax]);
    }
    if (hc.desc.hxc_mode == TSBZ_HXC_SCF) hc.hxc_subs.push_back((int)s);
    stage_max = std::max<long long>(stage_max, (long long)hs.n_k * c.n_bands * c.npts);
  }
  for (auto& hc : ctx->cells) work_max = std::max<long long>(work_max, (long long)hc.hxc_subs.size() * hc.dev.npts);
  ctx->n_units = (long long)units.size();
  ctx->ph_stride = ph_stride;
  int rc;
  ctx->psi_bytes = (size_t)psi_e * es;
  ctx->p_bytes = (size_t)std::max<long long>(p_e, 1) * es;
  if ((rc = dalloc(ctx, psi_e * es, &ctx->psi))) return rc;
  if ((rc = dalloc(ctx, psi_e * es, &ctx->tA))) return rc;
  if ((rc = dalloc(ctx, psi_e * es, &ctx->tB))) return rc;
  if ((rc = dalloc(ctx, std::max<long long>(p_e, 1) * es, &ctx->P))) return rc;
  if (ctx->precision == TSBZ_FP32_TC && (rc = dalloc(ctx, psi_e * es, &ctx->vnl))) return rc;
  if ((rc = dalloc(ctx, std::max<long long>(pa_e, 1) * es, &ctx->Pa))) return rc;
  if ((rc = dalloc(ctx, ctx->n_units * ph_stride * es, &ctx->ph_half))) return rc;
  if ((rc = dalloc(ctx, ctx->n_units * ph_stride * es, &ctx->ph_obs))) return rc;
  if (ctx->precision == TSBZ_FP32 && (rc = dalloc(ctx, ctx->n_units * ph_stride * es, &ctx->ph_next))) return rc;
  if ((rc = dalloc_t(ctx, rho_e, &ctx->rho_part))) return rc;
  if ((rc = dalloc_t(ctx, std::max<long long>(jk_e, 1), &ctx->jk_part))) return rc;
  if ((rc = dalloc_t(ctx, std::max<long long>(nrm_e, 1), &ctx->nrm_part))) return rc;
  if ((rc = dalloc_t(ctx, 3 * ctx->n_units, &ctx->q_half))) return rc;
  if ((rc = dalloc_t(ctx, 3 * ctx->n_units, &ctx->q_obs))) return rc;
  if ((rc = dalloc_t(ctx, 3 * ctx->n_units, &ctx->kcart))) return rc;
  if ((rc = dalloc(ctx, 4 * ctx->n_units * (ctx->precision == TSBZ_FP64 ? 8 : 4), &ctx->qt_half))) return rc;
  if ((rc = dalloc_t(ctx, ctx->n_units, &ctx->d_units))) return rc;
  if ((rc = dalloc_t(ctx, ctx->subs.size(), &ctx->d_subs))) return rc;
  if ((rc = dalloc_t(ctx, ctx->cells.size(), &ctx->d_cells))) return rc;
  if ((rc = dalloc_t(ctx, ctx->subs.size(), &ctx->d_steps))) return rc;
  if ((rc = dalloc_t(ctx, ctx->subs.size(), &ctx->d_status))) return rc;
  if ((rc = dalloc_t(ctx, ctx->subs.size(), &ctx->d_mask))) return rc;
  if ((rc = dalloc_t(ctx, ctx->subs.size(), &ctx->d_active))) return rc;
  if ((rc = dalloc_t(ctx, 3LL * TSBZ_FIN_MAX_TILES * ctx->subs.size(), &ctx->d_jtile))) return rc;
  if ((rc = dalloc_t(ctx, ctx->subs.size(), &ctx->d_jcount))) return rc;
  if ((rc = dalloc_t(ctx, std::max<long long>(work_max, 1), &ctx->work_a))) return rc;
  if ((rc = dalloc_t(ctx, std::max<long long>(work_max, 1), &ctx->work_b))) return rc;
  if ((rc = dalloc_t(ctx, stage_max, &ctx->staging))) return rc;
  ctx->staging_elems = stage_max;
  std::vector<SubDev> sd(ctx->subs.size());
  for (size_t s = 0; s < ctx->subs.size(); ++s) {
    HostSub& hs = ctx->subs[s];
    HostCell& hc = ctx->cells[hs.cell];
    const CellDev& c = hc.dev;
    const int nf = 2 * hs.max_steps + 1;
    if ((rc = dalloc_t(ctx, 3LL * nf, &hs.A_d))) return rc;
    if ((rc = dalloc_t(ctx, 3LL * (hs.max_steps + 1), &hs.J))) return rc;
    if ((rc = dalloc_t(ctx, 3, &hs.J0m))) return rc;
    if ((rc = dalloc_t(ctx, c.npts, &hs.rho))) return rc;
    if ((rc = dalloc_t(ctx, c.npts, &hs.vhxc))) return rc;
    if ((rc = dalloc_t(ctx, (long long)hs.n_k * c.n_bands, &hs.norms))) return rc;
    if ((rc = dalloc(ctx, (size_t)c.npts * (ctx->precision == TSBZ_FP64 ? 8 : 4), &hs.veff))) return rc;
    if ((rc = dalloc(ctx, (size_t)c.npts * (ctx->precision == TSBZ_FP64 ? 8 : 4), &hs.veff_save))) return rc;
    if (hs.A.empty()) hs.A.assign(3LL * nf, 0.0);
    hs.field_dirty = true;
    SubDev& d = sd[s];
    d.cell = hs.cell;
    d.n_k = hs.n_k;
    d.unit0 = hs.unit0;
    d.max_steps = hs.max_steps;
    d.n_field = nf;
    d.hxc_frozen = hc.desc.hxc_mode == TSBZ_HXC_FROZEN;
    d.xc = hc.desc.xc;
    d.hartree = hc.desc.hartree;
    d.dt = hs.dt;
    d.A = hs.A_d;
    d.J = hs.J;
    d.J0m = hs.J0m;
    d.rho = hs.rho;
    d.vhxc = hs.vhxc;
    d.veff = hs.veff;
    d.norms = hs.norms;
    d.step = ctx->d_steps + s;
    d.status = ctx->d_status + s;
    d.active = ctx->d_active + s;
    d.veff_save = hs.veff_save;
    d.jtile = ctx->d_jtile + 3LL * TSBZ_FIN_MAX_TILES * s;
    d.jcount = ctx->d_jcount + s;
    CK(cudaMemsetAsync(hs.vhxc, 0, sizeof(double) * c.npts, ctx->stream));
    CK(cudaMemsetAsync(hs.J, 0, sizeof(double) * 3 * (hs.max_steps + 1), ctx->stream));
    CK(cudaMemsetAsync(hs.J0m, 0, sizeof(double) * 3, ctx->stream));
  }
  std::vector<CellDev> cd;
  for (auto& hc : ctx->cells) {
    if (!hc.unit_ids.empty()) {
      if ((rc = dalloc_t(ctx, hc.unit_ids.size(), &hc.d_unit_ids))) return rc;
      CK(cudaMemcpyAsync(hc.d_unit_ids, hc.unit_ids.data(), sizeof(int) * hc.unit_ids.size(), cudaMemcpyHostToDevice,
                         ctx->stream));
    }
    if (!hc.hxc_subs.empty()) {
      if ((rc = dalloc_t(ctx, hc.hxc_subs.size(), &hc.d_hxc_subs))) return rc;
      CK(cudaMemcpyAsync(hc.d_hxc_subs, hc.hxc_subs.data(), sizeof(int) * hc.hxc_subs.size(),
                         cudaMemcpyHostToDevice, ctx->stream));
    }
    cd.push_back(hc.dev);
  }
  CK(cudaMemcpyAsync(ctx->d_units, units.data(), sizeof(UnitDev) * units.size(), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_subs, sd.data(), sizeof(SubDev) * sd.size(), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_cells, cd.data(), sizeof(CellDev) * cd.size(), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->kcart, kc.data(), sizeof(double) * kc.size(), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_steps, 0, sizeof(int) * ctx->subs.size(), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int) * ctx->subs.size(), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_mask, 0, sizeof(int) * ctx->subs.size(), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_jcount, 0, sizeof(int) * ctx->subs.size(), ctx->stream));
  {
    const std::vector<int> ones(ctx->subs.size(), 1);
    CK(cudaMemcpyAsync(ctx->d_active, ones.data(), sizeof(int) * ones.size(), cudaMemcpyHostToDevice, ctx->stream));
  }
  CK(cudaMemsetAsync(ctx->rho_part, 0, sizeof(double) * std::max<long long>(rho_e, 1), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->laid_out = true;
  return TSBZ_OK;
}

int upload_fields(tsbz_ctx* ctx) {
  for (auto& hs : ctx->subs)
    if (hs.field_dirty) {
      CK(cudaMemcpyAsync(hs.A_d, hs.A.data(), sizeof(double) * hs.A.size(), cudaMemcpyHostToDevice, ctx->stream));
      hs.field_dirty = false;
      hs.field_const = true;
      for (size_t i = 3; i < hs.A.size() && hs.field_const; ++i) hs.field_const = hs.A[i] == hs.A[i % 3];
    }
  return TSBZ_OK;
}

// A constant field makes q at t_{n+1} + dt/2 and at t_{n+1} equal bit for bit, so
// the next step's projections are the first-order sums of the current's.
bool cell_field_const(const tsbz_ctx* ctx, const HostCell& hc) {
  for (const auto& hs : ctx->subs)
    if (&ctx->cells[hs.cell] == &hc && !hs.field_const) return false;
  return true;
}

// Kernel families, dispatched on the precision.
template <typename T> int run_field(tsbz_ctx* ctx, int mode) {
  ev_start(ctx, FAM_FIELD);
  for (auto& hc : ctx->cells) {
    if (hc.unit_ids.empty()) continue;
    // a constant field leaves the phase tables of the last step current
    const bool keep = mode == TSBZ_FIELD_STEP && hc.tables_step && cell_field_const(ctx, hc) &&
                      ctx->propagator == TSBZ_PROP_TAYLOR4;
    launch_field<T>(make_set(ctx, hc), keep ? TSBZ_FIELD_STEP_KEEP : mode, ctx->stream);
    hc.tables_step = mode == TSBZ_FIELD_STEP;
    ++ctx->launches;
  }
  ev_stop(ctx);
  return TSBZ_OK;
}

template <typename T> int run_observe(tsbz_ctx* ctx, int fin_mode) {
  for (auto& hc : ctx->cells) {
    if (hc.unit_ids.empty()) continue;
    LaunchSet L = make_set(ctx, hc);
    const bool sep = ctx->precision == TSBZ_FP32 && sep_supported(hc.dev);
    // the projections for the current (not needed for the density-only ETRS predictor)
    bool wrote_p = false;
    if (fin_mode != TSBZ_FIN_RHO && !(fin_mode == TSBZ_FIN_STEP && hc.pa_by_stage)) {
      ev_start(ctx, FAM_BRA);
      // after a Taylor step under a constant field the slab pass also leaves in P
      // the projections the next step starts from (same q, same operations)
      const bool p_next = fin_mode == TSBZ_FIN_STEP && ctx->propagator == TSBZ_PROP_TAYLOR4 &&
                          cell_field_const(ctx, hc);
      if (ctx->precision == TSBZ_FP32_TC)
        launch_bra_tc(L, ctx->psi, ctx->Pa, 1, ctx->stream);
      else if (sep)
        launch_bra_sep(L, ctx->psi, ctx->Pa, 1, 1, ctx->stream);
      else if (ctx->precision == TSBZ_FP32 &&
               launch_bra_slab(L, ctx->psi, ctx->Pa, 1, 1, ctx->stream, p_next ? ctx->P : nullptr))
        wrote_p = p_next && hc.dev.use_proj;
      else
        launch_bra<T>(L, ctx->psi, ctx->Pa, 1, 1, ctx->stream);
      ev_stop(ctx);
      if (hc.dev.use_proj) ++ctx->launches;
    }
    hc.p_by_obs = wrote_p;
    ev_start(ctx, FAM_OBS);
    if (!(sep && launch_observe_fused(L, ctx->psi, ctx->rho_part, ctx->jk_part, ctx->nrm_part, ctx->stream)) &&
        !(ctx->precision != TSBZ_FP64 &&
          launch_observe_zf(L, ctx->psi, ctx->rho_part, ctx->jk_part, ctx->nrm_part, ctx->stream)) &&
        !(ctx->precision == TSBZ_FP32 &&
          launch_observe_slab(L, ctx->psi, ctx->rho_part, ctx->jk_part, ctx->nrm_part, ctx->stream)))
      launch_observe<T>(L, ctx->psi, ctx->rho_part, ctx->jk_part, ctx->nrm_part, ctx->stream);
    ev_stop(ctx);
    ++ctx->launches;
  }
  ev_start(ctx, FAM_FIN);
  launch_finalize_t<T>(ctx->d_subs, (int)ctx->subs.size(), ctx->d_units, ctx->d_cells, ctx->q_obs, ctx->Pa,
                       ctx->rho_part, ctx->jk_part, ctx->nrm_part, ctx->d_mask, fin_mode, ctx->fin_tiles,
                       ctx->stream);
  ev_stop(ctx);
  ++ctx->launches;
  return TSBZ_OK;
}

template <typename T> int run_hxc(tsbz_ctx* ctx) {
  ev_start(ctx, FAM_HXC);
  for (auto& hc : ctx->cells) {
    if (hc.hxc_subs.empty()) continue;
    ctx->launches += launch_hxc_t<T>(ctx->d_subs, hc.d_hxc_subs, (int)hc.hxc_subs.size(), hc.dev, ctx->work_a,
                                     ctx->work_b, hc.tw, ctx->stream);
  }
  ev_stop(ctx);
  return TSBZ_OK;
}

int run_step_tc(tsbz_ctx* ctx) {
  run_field<float>(ctx, TSBZ_FIELD_STEP);
  void* srcs[4] = {ctx->psi, ctx->tA, ctx->tB, ctx->tA};
  void* dsts[4] = {ctx->tA, ctx->tB, ctx->tA, nullptr};
  for (auto& hc : ctx->cells) {
    if (hc.unit_ids.empty()) continue;
    LaunchSet L = make_set(ctx, hc);
    ev_start(ctx, FAM_BRA);
    launch_bra_tc(L, ctx->psi, ctx->P, 0, ctx->stream);
    ev_stop(ctx);
    if (hc.dev.use_proj) ++ctx->launches;
    for (int m = 1; m <= 4; ++m) {
      ev_start(ctx, FAM_KET);
      launch_ket_tc(L, ctx->P, ctx->vnl, ctx->stream);
      ev_stop(ctx);
      ev_start(ctx, FAM_STAGE);
      launch_stage_v(L, srcs[m - 1], dsts[m - 1], ctx->psi, ctx->vnl, m, ctx->stream);
      ev_stop(ctx);
      ctx->launches += 2;
      if (m < 4 && hc.dev.use_proj) {
        ev_start(ctx, FAM_BRA);
        launch_bra_tc(L, dsts[m - 1], ctx->P, 0, ctx->stream);
        ev_stop(ctx);
        ++ctx->launches;
      }
    }
  }
  run_observe<float>(ctx, TSBZ_FIN_STEP);
  run_hxc<float>(ctx);
  return TSBZ_OK;
}

// The four Taylor stages of every cell (after the field launch): psi advances by
// dt * ctx->dt_scale.  fresh_p: the projections of psi are recomputed first
// (else they are taken from P when the last step left them there).
template <typename T> int run_stages(tsbz_ctx* ctx, bool fresh_p, int same_next_allowed) {
  void* srcs[4] = {ctx->psi, ctx->tA, ctx->tB, ctx->tA};
  void* dsts[4] = {ctx->tA, ctx->tB, ctx->tA, nullptr};
  for (auto& hc : ctx->cells) {
    if (hc.unit_ids.empty()) continue;
    LaunchSet L = make_set(ctx, hc);
    if (ctx->precision == TSBZ_FP32 && sep_supported(hc.dev)) {
      // Four fused stages; each leaves the projections of its t_m in P, and the
      // bulk-staged stage 4 those of psi(t_{n+1}) for the next step and of the
      // current (Pa).  The projections of psi are computed here only when P does
      // not hold them already (first step, or after the state or field changed).
      if (fresh_p || !ctx->p_next_valid || !hc.pa_by_stage) {
        ev_start(ctx, FAM_BRA);
        launch_bra_sep(L, ctx->psi, ctx->P, 0, 0, ctx->stream);
        ev_stop(ctx);
        if (hc.dev.use_proj) ++ctx->launches;
      }
      const int same_next = (same_next_allowed && cell_field_const(ctx, hc)) ? 1 : 0;
      ev_start(ctx, FAM_STAGE);
      const bool whole = launch_step_fused(L, ctx->psi, ctx->P, ctx->Pa, same_next, ctx->stream);
      ev_stop(ctx);
      if (whole) {
        hc.pa_by_stage = true;
        ++ctx->launches;
        continue;
      }
      for (int m = 1; m <= 4; ++m) {
        ev_start(ctx, FAM_STAGE);
        const bool fused4 = launch_stage_sep(L, srcs[m - 1], dsts[m - 1], ctx->psi, ctx->P, ctx->Pa, m,
                                             same_next, ctx->stream);
        if (m == 4) hc.pa_by_stage = fused4;
        ev_stop(ctx);
        ++ctx->launches;
      }
      continue;
    }
    // single precision on 32-point rows: variant 0 is the slab z-march stage, the
    // point-parallel stage takes the variants after it
    const bool slab = ctx->precision == TSBZ_FP32 && slab_supported(hc.dev);
    LaunchSet Lp = L;
    if (slab && L.variant > 0) Lp.variant = L.variant == 3 ? 0 : L.variant;
    for (int m = 1; m <= 4; ++m) {
      // stage 1 starts from P when the last observation left the projections of psi there
      if (!(m == 1 && !fresh_p && ctx->p_next_valid && hc.p_by_obs)) {
        ev_start(ctx, FAM_BRA);
        if (!(slab && launch_bra_slab(L, srcs[m - 1], ctx->P, 0, 0, ctx->stream)))
          launch_bra<T>(L, srcs[m - 1], ctx->P, 0, 0, ctx->stream);
        ev_stop(ctx);
        if (hc.dev.use_proj) ++ctx->launches;
      }
      ev_start(ctx, FAM_STAGE);
      if (!(slab && launch_stage_slab(L, srcs[m - 1], dsts[m - 1], ctx->psi, ctx->P, m, ctx->stream)))
        launch_stage<T>(Lp, srcs[m - 1], dsts[m - 1], ctx->psi, ctx->P, m, ctx->stream);
      ev_stop(ctx);
      ++ctx->launches;
    }
  }
  return TSBZ_OK;
}

// Enforced-time-reversal-symmetry step: a Taylor-4 predictor gives rho~(t_{n+1})
// and v~_eff; then psi(t_{n+1}) = T4(dt/2; A(t_{n+1}), v~_eff) T4(dt/2; A(t_n),
// v_eff(t_n)) psi(t_n).  psi(t_n) and v_eff(t_n) are kept on the device.
template <typename T> int run_step_etrs(tsbz_ctx* ctx) {
  int rc;
  if (!ctx->psi_save && (rc = dalloc(ctx, ctx->psi_bytes, &ctx->psi_save))) return rc;
  const int ns = (int)ctx->subs.size();
  CK(cudaMemcpyAsync(ctx->psi_save, ctx->psi, ctx->psi_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  launch_veff_keep_t<T>(ctx->d_subs, ctx->d_cells, ns, 0, ctx->stream);
  ++ctx->launches;
  // predictor: the Taylor-4 step, then rho~ and v~_eff (no current, step unchanged)
  ctx->dt_scale = 1.0;
  run_field<T>(ctx, TSBZ_FIELD_STEP);
  if ((rc = run_stages<T>(ctx, true, 0))) return rc;
  run_observe<T>(ctx, TSBZ_FIN_RHO);
  run_hxc<T>(ctx);
  launch_veff_keep_t<T>(ctx->d_subs, ctx->d_cells, ns, 1, ctx->stream);   // v_eff(t_n) back, v~_eff kept
  ++ctx->launches;
  CK(cudaMemcpyAsync(ctx->psi, ctx->psi_save, ctx->psi_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  // the two half steps
  ctx->dt_scale = 0.5;
  run_field<T>(ctx, TSBZ_FIELD_AT_NOW);
  if ((rc = run_stages<T>(ctx, true, 0))) return rc;
  launch_veff_keep_t<T>(ctx->d_subs, ctx->d_cells, ns, 1, ctx->stream);   // v~_eff in place
  ++ctx->launches;
  run_field<T>(ctx, TSBZ_FIELD_AT_NEXT);
  if ((rc = run_stages<T>(ctx, true, 0))) return rc;
  ctx->dt_scale = 1.0;
  run_observe<T>(ctx, TSBZ_FIN_STEP);
  run_hxc<T>(ctx);
  ctx->p_next_valid = false;
  return TSBZ_OK;
}

template <typename T> int run_step(tsbz_ctx* ctx) {
  if (ctx->precision == TSBZ_FP32_TC) return run_step_tc(ctx);
  if (ctx->propagator == TSBZ_PROP_ETRS) return run_step_etrs<T>(ctx);
  run_field<T>(ctx, TSBZ_FIELD_STEP);
  int rc = run_stages<T>(ctx, false, 1);
  if (rc) return rc;
  run_observe<T>(ctx, TSBZ_FIN_STEP);
  run_hxc<T>(ctx);
  ctx->p_next_valid = true;
  return TSBZ_OK;
}

template <typename T> int run_init(tsbz_ctx* ctx, bool minus, bool plus) {
  ctx->p_next_valid = false;
  std::vector<int> mask(ctx->subs.size(), 0);
  if (minus) {
    for (size_t s = 0; s < ctx->subs.size(); ++s) mask[s] = ctx->subs[s].need_init ? 1 : 0;
    CK(cudaMemcpyAsync(ctx->d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, ctx->stream));
    run_field<T>(ctx, TSBZ_FIELD_J0MINUS);
    run_observe<T>(ctx, TSBZ_FIN_J0MINUS);
    run_hxc<T>(ctx);
    for (size_t s = 0; s < ctx->subs.size(); ++s) {
      HostSub& hs = ctx->subs[s];
      if (ctx->cells[hs.cell].desc.hxc_mode == TSBZ_HXC_FROZEN) {
        launch_veff_frozen_t<T>(ctx->d_subs, (int)s, ctx->cells[hs.cell].dev, ctx->stream);
        ++ctx->launches;
      }
    }
  }
  if (plus) {
    for (size_t s = 0; s < ctx->subs.size(); ++s)
      mask[s] = (ctx->subs[s].need_j0plus || ctx->subs[s].need_init) ? 1 : 0;
    CK(cudaMemcpyAsync(ctx->d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, ctx->stream));
    run_field<T>(ctx, TSBZ_FIELD_J0PLUS);
    run_observe<T>(ctx, TSBZ_FIN_J0PLUS);
  }
  return TSBZ_OK;
}

// One time step captured once as a CUDA graph on the library's own stream
// and replayed n times; the caller's stream and the library stream are
// ordered by events on both sides.  The first step runs uncaptured, so
// one-time set-up (kernel attributes) happens outside the capture.
int run_steps_graph(tsbz_ctx* ctx, int n_steps) {
  if (!ctx->gstream) {
    CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming));
  }
  int done = 0;
  if (ctx->step_graph && !ctx->p_next_valid) {
    // the captured step assumes P already holds the projections of psi
    int rc = ctx->precision == TSBZ_FP64 ? run_step<double>(ctx) : run_step<float>(ctx);
    if (rc) return rc;
    done = 1;
  }
  if (!ctx->step_graph) {
    int rc = ctx->precision == TSBZ_FP64 ? run_step<double>(ctx) : run_step<float>(ctx);
    if (rc) return rc;
    CK(cudaGetLastError());
    done = 1;
    CK(cudaEventRecord(ctx->ev_in, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0));
    cudaStream_t user = ctx->stream;
    const long long launches0 = ctx->launches;
    ctx->stream = ctx->gstream;
    CK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal));
    rc = ctx->precision == TSBZ_FP64 ? run_step<double>(ctx) : run_step<float>(ctx);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->gstream, &graph);
    ctx->stream = user;
    ctx->graph_launches = ctx->launches - launches0;
    ctx->launches = launches0;
    if (rc) return rc;
    if (ec != cudaSuccess) return set_err(ctx, TSBZ_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    const cudaError_t ei = cudaGraphInstantiate(&ctx->step_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return set_err(ctx, TSBZ_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
  }
  CK(cudaEventRecord(ctx->ev_in, ctx->stream));
  CK(cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0));
  for (int i = done; i < n_steps; ++i) {
    CK(cudaGraphLaunch(ctx->step_graph, ctx->gstream));
    ctx->launches += ctx->graph_launches;
  }
  CK(cudaEventRecord(ctx->ev_out, ctx->gstream));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_out, 0));
  return TSBZ_OK;
}

int ensure_ready(tsbz_ctx* ctx) {
  if (!ctx->laid_out) return set_err(ctx, TSBZ_ESTATE, "no ground state loaded");
  for (size_t s = 0; s < ctx->subs.size(); ++s)
    if (!ctx->subs[s].loaded)
      return set_err(ctx, TSBZ_ESTATE, "sub-simulation " + std::to_string(s) + " has no ground state");
  int rc = upload_fields(ctx);
  if (rc) return rc;
  bool minus = false, plus = false;
  for (auto& hs : ctx->subs) {
    minus = minus || hs.need_init;
    plus = plus || hs.need_init || (hs.need_j0plus && hs.steps == 0);
  }
  if (minus || plus) {
    rc = ctx->precision == TSBZ_FP64 ? run_init<double>(ctx, minus, plus) : run_init<float>(ctx, minus, plus);
    if (rc) return rc;
    CK(cudaGetLastError());
    for (auto& hs : ctx->subs) {
      hs.need_init = false;
      if (hs.steps == 0) hs.need_j0plus = false;
    }
  }
  return TSBZ_OK;
}

int check_sub(tsbz_ctx* ctx, int s) {
  if (!ctx) return TSBZ_EINVAL;
  if (s < 0 || s >= (int)ctx->subs.size()) return set_err(ctx, TSBZ_EINVAL, "bad sub-simulation id");
  return TSBZ_OK;
}

int copy_state_in(tsbz_ctx* ctx, int s, const double* psi, size_t n_elems, int on_device) {
  HostSub& hs = ctx->subs[s];
  const CellDev& c = ctx->cells[hs.cell].dev;
  const long long need = (long long)hs.n_k * c.n_bands * c.npts;
  if (!psi) return set_err(ctx, TSBZ_EINVAL, "psi is NULL");
  if ((long long)n_elems != need)
    return set_err(ctx, TSBZ_EINVAL, "psi has " + std::to_string(n_elems) + " complex values, expected " +
                                         std::to_string(need));
  // page-locked host memory mapped into the device's address space is read by
  // the conversion kernel over the host link directly; anything else goes
  // through the staging buffer by one copy
  const double2* src = (const double2*)ctx->staging;
  cudaPointerAttributes at{};
  if (!on_device && cudaPointerGetAttributes(&at, psi) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer) {
    src = (const double2*)at.devicePointer;
  } else {
    cudaGetLastError();   // a query on memory CUDA does not know may leave an error behind
    CK(cudaMemcpyAsync(ctx->staging, psi, sizeof(double2) * need,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  }
  char* dst = (char*)ctx->psi + ctx->unit_psi_off[hs.unit0] * ctx->elem_size();
  if (ctx->precision == TSBZ_FP64)
    launch_convert_in_t<double>(src, dst, need, ctx->stream);
  else
    launch_convert_in_t<float>(src, dst, need, ctx->stream);
  ++ctx->launches;
  CK(cudaGetLastError());
  return TSBZ_OK;
}

int sync_and_check(tsbz_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  return TSBZ_OK;
}

// Kernel variants a cell can run (the autotuner's search space):
//   FP32 on 16^3 / 8^3 cells: 0 fused tensor-core / bulk-staged stage, 1 z-march
//     stage with CUDA-core projections;
//   point-parallel path (FP64, and FP32 on shapes without a z-march kernel):
//     bands per staged projection chunk 8 (0), 4 (1), 16 (2, when its shared
//     memory fits);
//   FP32 on grids with 32-point rows (slab_supported): 0 slab z-march stage,
//     then the point-parallel stage with 4 (1), 16 (2, when it fits) or 8 (3)
//     bands per chunk;
//   FP32_TC on 16^3 grids: stage with the band of t bulk-staged in shared
//     memory and V, psi read per plane (0) or bulk-staged too (1), z-march
//     stage with a halo plane per z (2);
//   everything else: one variant.
int n_variants(const tsbz_ctx* ctx, const HostCell& hc) {
  const CellDev& c = hc.dev;
  if (ctx->precision == TSBZ_FP32_TC) return (c.n1 == 16 && c.n2 == 16 && c.n3 == 16) ? 3 : 1;
  if (ctx->precision == TSBZ_FP32 && sep_supported(c)) return sep_variants(c);
  const size_t big = (size_t)16 * (c.n_proj > 0 ? c.n_proj : 1) * ctx->elem_size();
  if (ctx->precision == TSBZ_FP32 && slab_supported(c)) return big <= 160 * 1024 ? 4 : 2;
  return big <= 160 * 1024 ? 3 : 2;
}

// Everything a time step changes that outlives the step, so that trial steps
// can be undone bit for bit: psi, P, the step counters, status words and the
// per-sub-simulation rho, v_Hxc, v_eff and norms.
struct Snapshot {
  void* psi = nullptr;
  void* P = nullptr;
  std::vector<int> steps, status;
  std::vector<std::vector<double>> rho, vhxc, norms;
  std::vector<std::vector<unsigned char>> veff;
  bool p_next_valid = false;
  std::vector<bool> pa_by_stage, p_by_obs;
};

int snapshot_take(tsbz_ctx* ctx, Snapshot& sn) {
  int rc;
  if ((rc = dalloc(ctx, ctx->psi_bytes, &sn.psi))) return rc;
  if ((rc = dalloc(ctx, ctx->p_bytes, &sn.P))) return rc;
  CK(cudaMemcpyAsync(sn.psi, ctx->psi, ctx->psi_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(sn.P, ctx->P, ctx->p_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  const size_t ns = ctx->subs.size();
  sn.steps.resize(ns);
  sn.status.resize(ns);
  sn.rho.resize(ns);
  sn.vhxc.resize(ns);
  sn.norms.resize(ns);
  sn.veff.resize(ns);
  CK(cudaMemcpyAsync(sn.steps.data(), ctx->d_steps, sizeof(int) * ns, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(sn.status.data(), ctx->d_status, sizeof(int) * ns, cudaMemcpyDeviceToHost, ctx->stream));
  const size_t rs = ctx->precision == TSBZ_FP64 ? 8 : 4;
  for (size_t s = 0; s < ns; ++s) {
    const HostSub& hs = ctx->subs[s];
    const CellDev& c = ctx->cells[hs.cell].dev;
    sn.rho[s].resize(c.npts);
    sn.vhxc[s].resize(c.npts);
    sn.norms[s].resize((size_t)hs.n_k * c.n_bands);
    sn.veff[s].resize((size_t)c.npts * rs);
    CK(cudaMemcpyAsync(sn.rho[s].data(), hs.rho, sizeof(double) * c.npts, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(sn.vhxc[s].data(), hs.vhxc, sizeof(double) * c.npts, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(sn.norms[s].data(), hs.norms, sizeof(double) * sn.norms[s].size(), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(sn.veff[s].data(), hs.veff, sn.veff[s].size(), cudaMemcpyDeviceToHost, ctx->stream));
  }
  sn.p_next_valid = ctx->p_next_valid;
  for (auto& hc : ctx->cells) {
    sn.pa_by_stage.push_back(hc.pa_by_stage);
    sn.p_by_obs.push_back(hc.p_by_obs);
  }
  return sync_and_check(ctx);
}

int snapshot_restore(tsbz_ctx* ctx, Snapshot& sn) {
  CK(cudaMemcpyAsync(ctx->psi, sn.psi, ctx->psi_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->P, sn.P, ctx->p_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  const size_t ns = ctx->subs.size();
  CK(cudaMemcpyAsync(ctx->d_steps, sn.steps.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_status, sn.status.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, ctx->stream));
  for (size_t s = 0; s < ns; ++s) {
    HostSub& hs = ctx->subs[s];
    CK(cudaMemcpyAsync(hs.rho, sn.rho[s].data(), sizeof(double) * sn.rho[s].size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(hs.vhxc, sn.vhxc[s].data(), sizeof(double) * sn.vhxc[s].size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(hs.norms, sn.norms[s].data(), sizeof(double) * sn.norms[s].size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(hs.veff, sn.veff[s].data(), sn.veff[s].size(), cudaMemcpyHostToDevice, ctx->stream));
  }
  ctx->p_next_valid = sn.p_next_valid;
  for (size_t i = 0; i < ctx->cells.size(); ++i) {
    ctx->cells[i].pa_by_stage = sn.pa_by_stage[i];
    ctx->cells[i].p_by_obs = sn.p_by_obs[i];
  }
  const int rc = sync_and_check(ctx);
  dfree(ctx, sn.psi);
  dfree(ctx, sn.P);
  sn.psi = sn.P = nullptr;
  return rc;
}

// Self-test of the bounded device wait: thread 0 announces a 16-byte
// transaction on an mbarrier and, if `deliver`, issues the bulk copy that
// completes it; every thread then waits at most `polls` polls.  Without the
// copy the wait runs out and the kernel records BK_STATUS_TIMEOUT and returns,
// with no copy in flight.
__device__ __align__(16) unsigned char g_selftest_src[16];

__global__ void k_selftest_wait(int polls, int deliver, int* status) {
  __shared__ __align__(16) unsigned char dst[16];
  __shared__ __align__(8) unsigned long long mbar;
  const uint32_t bar = bk_smem(&mbar);
  if (threadIdx.x == 0) bk_mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    bk_mbar_expect_tx(bar, 16);
    if (deliver) bk_copy_g2s(bk_smem(dst), g_selftest_src, 16, bar);
  }
  const bool ok = bk_mbar_wait(bar, 0, polls);
  if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(status, BK_STATUS_TIMEOUT);
}

// A captured step holds the kernels of the variants it was captured with.
void drop_step_graph(tsbz_ctx* ctx) {
  if (ctx->step_graph) {
    cudaGraphExecDestroy(ctx->step_graph);
    ctx->step_graph = nullptr;
  }
}

}  // namespace

extern "C" {

int tsbz_version(void) { return 10000; }

int tsbz_create(tsbz_ctx** out, int device, int precision, void* cuda_stream, const tsbz_alloc* alloc) {
  if (!out) return TSBZ_EINVAL;
  *out = nullptr;
  if (precision != TSBZ_FP64 && precision != TSBZ_FP32 && precision != TSBZ_FP32_TC) return TSBZ_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return TSBZ_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return TSBZ_ECUDA;
  tsbz_ctx* ctx = new (std::nothrow) tsbz_ctx();
  if (!ctx) return TSBZ_ENOMEM;
  ctx->device = device;
  ctx->precision = precision;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (alloc && alloc->alloc && alloc->free) {
    ctx->has_alloc = true;
    ctx->alloc = *alloc;
  }
  *out = ctx;
  return TSBZ_OK;
}

int tsbz_init_cell(tsbz_ctx* ctx, const tsbz_cell_desc* d, int* cell_id) {
  if (!ctx || !d || !cell_id) return TSBZ_EINVAL;
  if (ctx->laid_out) return set_err(ctx, TSBZ_ESTATE, "cells must be added before the first ground state");
  if (d->fd_nd < 1 || d->fd_nd > TSBZ_MAX_ND) return set_err(ctx, TSBZ_EINVAL, "fd_nd must be 1..6");
  for (int ax = 0; ax < 3; ++ax) {
    // the stencil wraps at most once: n > fd_nd
    if (d->n[ax] < d->fd_nd + 1 || d->n[ax] > 1024)
      return set_err(ctx, TSBZ_EINVAL, "grid size must be in [fd_nd + 1, 1024]");
    if (!(d->a[ax] > 0.0)) return set_err(ctx, TSBZ_EINVAL, "cell edges must be positive");
  }
  if (d->n_bands < 1 || d->n_atoms < 0 || (d->n_atoms > 0 && !d->atom_frac))
    return set_err(ctx, TSBZ_EINVAL, "bad band or atom count");
  if (d->use_projectors && (d->n_atoms == 0 || !(d->proj_half > 0.0) || !(d->r_proj > 0.0)))
    return set_err(ctx, TSBZ_EINVAL, "projectors need atoms, r_proj > 0 and proj_half > 0");
  if (d->hxc_mode != TSBZ_HXC_SCF && d->hxc_mode != TSBZ_HXC_FROZEN) return set_err(ctx, TSBZ_EINVAL, "bad hxc_mode");
  const long long npts = (long long)d->n[0] * d->n[1] * d->n[2];
  if (npts > (1LL << 30)) return set_err(ctx, TSBZ_EINVAL, "grid too large");
  if (ctx->precision == TSBZ_FP32_TC &&
      (d->fd_nd != 4 || d->n_bands > 16 || (d->use_projectors && 4 * d->n_atoms > 32) ||
       std::max(d->n[0], std::max(d->n[1], d->n[2])) > 32))
    return set_err(ctx, TSBZ_EINVAL,
                   "the tensor-core mode needs fd_nd = 4, n_bands <= 16, at most 32 projectors and "
                   "grid edges <= 32 per cell");
  HostCell hc;
  hc.desc = *d;
  hc.atoms.assign(d->atom_frac, d->atom_frac + 3 * d->n_atoms);
  hc.desc.atom_frac = hc.atoms.data();
  CellDev& c = hc.dev;
  std::memset(&c, 0, sizeof(c));
  c.n1 = d->n[0];
  c.n2 = d->n[1];
  c.n3 = d->n[2];
  c.npts = (int)npts;
  c.nmax = std::max(c.n1, std::max(c.n2, c.n3));
  c.n_atoms = d->n_atoms;
  c.use_proj = d->use_projectors ? 1 : 0;
  c.n_proj = c.use_proj ? 4 * d->n_atoms : 0;
  c.n_bands = d->n_bands;
  c.nd = d->fd_nd;
  c.n_tiles = (c.npts + TSBZ_PT - 1) / TSBZ_PT;
  c.n_bgroups = (c.n_bands + TSBZ_BG - 1) / TSBZ_BG;
  c.omega = d->a[0] * d->a[1] * d->a[2];
  c.dv = c.omega / (double)npts;
  c.occ = d->occ;
  double cw[TSBZ_MAX_ND + 1], dw[TSBZ_MAX_ND + 1];
  tsbz::fd_weights(d->fd_nd, cw, dw);
  for (int ax = 0; ax < 3; ++ax) {
    const double h = d->a[ax] / d->n[ax];
    for (int m = 0; m <= d->fd_nd; ++m) {
      c.lapw[ax][m] = cw[m] / (h * h);
      c.gradw[ax][m] = dw[m] / h;
      c.hlapf[ax][m] = (float)(-0.5 * cw[m] / (h * h));
      c.gradwf[ax][m] = (float)(dw[m] / h);
      c.hlap2[ax][m] = make_float2(c.hlapf[ax][m], c.hlapf[ax][m]);
      c.gradw2[ax][m] = make_float2(c.gradwf[ax][m], c.gradwf[ax][m]);
    }
    c.gsq_scale[ax] = 2.0 * 3.14159265358979323846 / d->a[ax];
  }
  tsbz::local_potential(hc.desc, hc.vloc);
  std::vector<double> g1, d1, ekb;
  if (c.use_proj) {
    tsbz::projector_tables(hc.desc, g1, d1, hc.pnorm, c.nmax);
  } else {
    g1.assign(1, 0.0);
    d1.assign(std::max(1, d->n_atoms * 3 * c.nmax), 0.0);
    hc.pnorm.assign(std::max(1, 4 * d->n_atoms), 0.0);
  }
  if (d1.size() < (size_t)std::max(1, d->n_atoms * 3 * c.nmax)) d1.resize(std::max(1, d->n_atoms * 3 * c.nmax), 0.0);
  for (int a = 0; a < d->n_atoms; ++a) {
    ekb.push_back(d->e_kb_s);
    for (int t = 0; t < 3; ++t) ekb.push_back(d->e_kb_p);
  }
  if (ekb.empty()) ekb.push_back(0.0);
  // pnorm_j * E_j per projector (the ket weight)
  std::vector<double> wkb(ekb.size(), 0.0);
  if (c.use_proj)
    for (int j = 0; j < c.n_proj; ++j) wkb[j] = hc.pnorm[j] * ekb[j];
  auto to_f = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
  const std::vector<float> g1f = to_f(g1), d1f = to_f(d1), pnf = to_f(hc.pnorm), wkf = to_f(wkb), ekf = to_f(ekb);
  double *vl, *gg, *dd, *pn, *ek, *wk;
  float *ggf, *ddf, *pnff, *wkff, *ekff;
  int rc;
  if ((rc = dalloc_t(ctx, hc.vloc.size(), &vl))) return rc;
  if ((rc = dalloc_t(ctx, g1.size(), &gg))) return rc;
  if ((rc = dalloc_t(ctx, d1.size(), &dd))) return rc;
  if ((rc = dalloc_t(ctx, hc.pnorm.size(), &pn))) return rc;
  if ((rc = dalloc_t(ctx, ekb.size(), &ek))) return rc;
  if ((rc = dalloc_t(ctx, wkb.size(), &wk))) return rc;
  if ((rc = dalloc_t(ctx, g1f.size(), &ggf))) return rc;
  if ((rc = dalloc_t(ctx, d1f.size(), &ddf))) return rc;
  if ((rc = dalloc_t(ctx, pnf.size(), &pnff))) return rc;
  if ((rc = dalloc_t(ctx, wkf.size(), &wkff))) return rc;
  if ((rc = dalloc_t(ctx, ekf.size(), &ekff))) return rc;
  CK(cudaMemcpy(vl, hc.vloc.data(), sizeof(double) * hc.vloc.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(gg, g1.data(), sizeof(double) * g1.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dd, d1.data(), sizeof(double) * d1.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pn, hc.pnorm.data(), sizeof(double) * hc.pnorm.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ek, ekb.data(), sizeof(double) * ekb.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(wk, wkb.data(), sizeof(double) * wkb.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ggf, g1f.data(), sizeof(float) * g1f.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ddf, d1f.data(), sizeof(float) * d1f.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pnff, pnf.data(), sizeof(float) * pnf.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(wkff, wkf.data(), sizeof(float) * wkf.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ekff, ekf.data(), sizeof(float) * ekf.size(), cudaMemcpyHostToDevice));
  c.vloc = vl;
  c.g1 = gg;
  c.d1 = dd;
  c.pnorm = pn;
  c.ekb = ek;
  c.wkb = wk;
  c.g1f = ggf;
  c.d1f = ddf;
  c.pnormf = pnff;
  c.wkbf = wkff;
  c.ekbf = ekff;
  // projector boxes from the double Gaussian tables: the smallest periodic index
  // range of each atom and axis that holds every nonzero factor
  c.pbox = nullptr;
  c.pbox_ok = 0;
  if (c.use_proj) {
    std::vector<int> box(6 * (size_t)d->n_atoms, 0);
    bool ok = true;
    const int nn[3] = {c.n1, c.n2, c.n3};
    for (int a = 0; a < d->n_atoms; ++a)
      for (int ax = 0; ax < 3; ++ax) {
        const int n = nn[ax];
        const double* gr = g1.data() + ((size_t)a * 3 + ax) * c.nmax;
        int cnt = 0;
        for (int i = 0; i < n; ++i) cnt += gr[i] != 0.0;
        int start = 0, len = n;
        if (cnt > 0 && cnt < n) {
          // a start after which cnt consecutive (periodic) entries hold every nonzero
          for (int s0 = 0; s0 < n; ++s0) {
            if (gr[s0] == 0.0 || gr[(s0 + n - 1) % n] != 0.0) continue;
            int inside = 0;
            for (int j = 0; j < cnt; ++j) inside += gr[(s0 + j) % n] != 0.0;
            if (inside == cnt) {
              start = s0;
              len = cnt;
              break;
            }
          }
        }
        box[(a * 3 + ax) * 2] = start;
        box[(a * 3 + ax) * 2 + 1] = len;
        if (ax < 2 && len > 16) ok = false;
      }
    int* db = nullptr;
    if ((rc = dalloc_t(ctx, box.size(), &db))) return rc;
    CK(cudaMemcpy(db, box.data(), sizeof(int) * box.size(), cudaMemcpyHostToDevice));
    c.pbox = db;
    c.pbox_ok = ok ? 1 : 0;
  }
  // z groups: atoms with bit-identical z rows of the float factor tables
  const int nm_z = c.nmax;
  auto same_z = [&](int a, int b) {
    for (int i = 0; i < nm_z; ++i) {
      const size_t ia = (size_t)(a * 3 + 2) * nm_z + i, ib = (size_t)(b * 3 + 2) * nm_z + i;
      if (g1f[ia] != g1f[ib] || d1f[ia] != d1f[ib]) return false;
    }
    return true;
  };
  c.zs_n = 0;
  for (int i = 0; i <= 8; ++i) c.zs_off[i] = 0;
  for (int i = 0; i < 64; ++i) c.zs_mem[i] = 0;
  if (c.use_proj && d->n_atoms <= 64) {
    std::vector<int> rep, grp(d->n_atoms, -1);
    for (int a = 0; a < d->n_atoms; ++a) {
      for (size_t h = 0; h < rep.size() && grp[a] < 0; ++h)
        if (same_z(a, rep[h])) grp[a] = (int)h;
      if (grp[a] < 0) {
        grp[a] = (int)rep.size();
        rep.push_back(a);
      }
    }
    if (rep.size() <= 8) {
      c.zs_n = (int)rep.size();
      int k = 0;
      for (int g = 0; g < c.zs_n; ++g) {
        c.zs_off[g] = k;
        for (int a = 0; a < d->n_atoms; ++a)
          if (grp[a] == g) c.zs_mem[k++] = a;
      }
      for (int g = c.zs_n; g <= 8; ++g) c.zs_off[g] = k;
    }
  }
  c.n_zg = 0;
  for (int i = 0; i < 8; ++i) c.zg_of[i] = c.zg_rep[i] = c.zg_mem[i] = 0;
  for (int i = 0; i <= 8; ++i) c.zg_off[i] = 0;
  if (c.use_proj && d->n_atoms <= 8) {
    for (int a = 0; a < 8; ++a) c.zg_of[a] = 0;
    for (int a = 0; a < d->n_atoms; ++a) {
      int g = -1;
      for (int h = 0; h < c.n_zg && g < 0; ++h)
        if (same_z(a, c.zg_rep[h])) g = h;
      if (g < 0) {
        g = c.n_zg++;
        c.zg_rep[g] = a;
      }
      c.zg_of[a] = g;
    }
    int k = 0;
    for (int g = 0; g < c.n_zg; ++g) {
      c.zg_off[g] = k;
      for (int a = 0; a < d->n_atoms; ++a)
        if (c.zg_of[a] == g) c.zg_mem[k++] = a;
    }
    for (int g = c.n_zg; g <= 8; ++g) c.zg_off[g] = k;
    for (int g = c.n_zg; g < 8; ++g) c.zg_rep[g] = 0;
  }
  const int nn[3] = {c.n1, c.n2, c.n3};
  for (int ax = 0; ax < 3; ++ax) {
    std::vector<double2> tw(nn[ax]);
    for (int m = 0; m < nn[ax]; ++m) {
      const double ang = 2.0 * 3.14159265358979323846 * m / nn[ax];
      tw[m] = make_double2(std::cos(ang), std::sin(ang));
    }
    if ((rc = dalloc_t(ctx, tw.size(), &hc.tw[ax]))) return rc;
    CK(cudaMemcpy(hc.tw[ax], tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice));
  }
  ctx->cells.push_back(std::move(hc));
  *cell_id = (int)ctx->cells.size() - 1;
  return TSBZ_OK;
}

int tsbz_add_subsim(tsbz_ctx* ctx, int cell_id, int n_k, const double* k_cart, double dt, int max_steps,
                    int* subsim_id) {
  if (!ctx || !subsim_id) return TSBZ_EINVAL;
  if (ctx->laid_out) return set_err(ctx, TSBZ_ESTATE, "sub-simulations must be added before the first ground state");
  if (cell_id < 0 || cell_id >= (int)ctx->cells.size()) return set_err(ctx, TSBZ_EINVAL, "bad cell id");
  if (n_k < 1 || !k_cart) return set_err(ctx, TSBZ_EINVAL, "need n_k >= 1 k-points");
  if (!(dt > 0.0) || max_steps < 0 || max_steps > 100000000) return set_err(ctx, TSBZ_EINVAL, "bad dt or max_steps");
  HostSub hs;
  hs.cell = cell_id;
  hs.n_k = n_k;
  hs.k.assign(k_cart, k_cart + 3LL * n_k);
  hs.dt = dt;
  hs.max_steps = max_steps;
  ctx->subs.push_back(std::move(hs));
  *subsim_id = (int)ctx->subs.size() - 1;
  return TSBZ_OK;
}

int tsbz_load_ground_state(tsbz_ctx* ctx, int s, const double* psi, size_t n_elems, int psi_on_device,
                           const double* v_hxc_frozen) {
  int rc = check_sub(ctx, s);
  if (rc) return rc;
  if ((rc = layout(ctx))) return rc;
  HostSub& hs = ctx->subs[s];
  HostCell& hc = ctx->cells[hs.cell];
  if (hc.desc.hxc_mode == TSBZ_HXC_FROZEN) {
    if (!v_hxc_frozen) return set_err(ctx, TSBZ_EINVAL, "frozen mode needs v_hxc_frozen");
    CK(cudaMemcpyAsync(hs.vhxc, v_hxc_frozen, sizeof(double) * hc.dev.npts, cudaMemcpyHostToDevice, ctx->stream));
  }
  if ((rc = copy_state_in(ctx, s, psi, n_elems, psi_on_device))) return rc;
  CK(cudaMemsetAsync(ctx->d_steps + s, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_status + s, 0, sizeof(int), ctx->stream));
  hs.steps = 0;
  hs.loaded = true;
  hs.need_init = true;
  hs.need_j0plus = true;
  // a caller's device buffer may be freed and reused as soon as this returns
  return psi_on_device ? sync_and_check(ctx) : TSBZ_OK;
}

int tsbz_set_kick(tsbz_ctx* ctx, int s, double k0, const double dir[3]) {
  if (!ctx || !dir) return TSBZ_EINVAL;
  if (s < -1 || s >= (int)ctx->subs.size()) return set_err(ctx, TSBZ_EINVAL, "bad sub-simulation id");
  for (size_t i = 0; i < ctx->subs.size(); ++i) {
    if (s >= 0 && (int)i != s) continue;
    HostSub& hs = ctx->subs[i];
    if (hs.steps > 0) return set_err(ctx, TSBZ_ESTATE, "the field can only change before the first step");
    const size_t nf = 2 * (size_t)hs.max_steps + 1;
    hs.A.assign(3 * nf, 0.0);
    for (size_t j = 0; j < nf; ++j)
      for (int ax = 0; ax < 3; ++ax) hs.A[3 * j + ax] = -k0 * dir[ax];
    hs.field_dirty = true;
    hs.need_j0plus = true;
  }
  return TSBZ_OK;
}

int tsbz_set_field(tsbz_ctx* ctx, int s, int n_steps, const double* a_samples) {
  int rc = check_sub(ctx, s);
  if (rc) return rc;
  HostSub& hs = ctx->subs[s];
  if (!a_samples || n_steps < 0 || n_steps > hs.max_steps)
    return set_err(ctx, TSBZ_EINVAL, "field needs 0 <= n_steps <= max_steps and samples");
  if (hs.steps > 0) return set_err(ctx, TSBZ_ESTATE, "the field can only change before the first step");
  const size_t nf = 2 * (size_t)hs.max_steps + 1;
  hs.A.assign(3 * nf, 0.0);
  std::memcpy(hs.A.data(), a_samples, sizeof(double) * 3 * (2 * (size_t)n_steps + 1));
  hs.field_dirty = true;
  hs.need_j0plus = true;
  return TSBZ_OK;
}

int tsbz_propagate(tsbz_ctx* ctx, int n_steps) {
  if (!ctx || n_steps < 0) return TSBZ_EINVAL;
  int rc = ensure_ready(ctx);
  if (rc) return rc;
  // per-sub-simulation step budgets: a sub-simulation that reaches max_steps
  // sits out the remaining steps (its units skip every kernel of the step)
  ctx->ev_marks.clear();
  ctx->ev_next = 0;
  if (ctx->graphs && !ctx->prof && n_steps > 0) {
    if ((rc = run_steps_graph(ctx, n_steps))) return rc;
  } else {
    for (int i = 0; i < n_steps; ++i) {
      rc = ctx->precision == TSBZ_FP64 ? run_step<double>(ctx) : run_step<float>(ctx);
      if (rc) return rc;
    }
  }
  CK(cudaGetLastError());
  if ((rc = sync_and_check(ctx))) return rc;
  for (auto& hs : ctx->subs) hs.steps = std::min(hs.max_steps, hs.steps + n_steps);
  if (ctx->prof) {
    for (int f = 0; f < TSBZ_N_FAM; ++f) ctx->times[f] = 0.0;
    for (auto& m : ctx->ev_marks) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ctx->ev_pool[m.second], ctx->ev_pool[m.second + 1]);
      ctx->times[m.first] += ms;
    }
  }
  std::vector<int> st(ctx->subs.size(), 0);
  CK(cudaMemcpy(st.data(), ctx->d_status, sizeof(int) * st.size(), cudaMemcpyDeviceToHost));
  for (size_t s = 0; s < st.size(); ++s)
    if (st[s] & BK_STATUS_TIMEOUT)
      return set_err(ctx, TSBZ_ETIMEOUT, "a bounded device wait gave up in sub-simulation " + std::to_string(s));
  for (size_t s = 0; s < st.size(); ++s)
    if (st[s]) return set_err(ctx, TSBZ_ENONFINITE, "non-finite current in sub-simulation " + std::to_string(s));
  return TSBZ_OK;
}

int tsbz_get_current(tsbz_ctx* ctx, int s, int first, int count, double* J, double* J0_minus) {
  if (!ctx || first < 0 || count < 0 || (count > 0 && !J)) return TSBZ_EINVAL;
  if (s < -1 || s >= (int)ctx->subs.size()) return set_err(ctx, TSBZ_EINVAL, "bad sub-simulation id");
  int rc = ensure_ready(ctx);
  if (rc) return rc;
  if ((rc = sync_and_check(ctx))) return rc;
  if (s >= 0) {
    HostSub& hs = ctx->subs[s];
    if (first + count > hs.steps + 1) return set_err(ctx, TSBZ_EINVAL, "requested steps not computed yet");
    if (count) CK(cudaMemcpy(J, hs.J + 3LL * first, sizeof(double) * 3 * count, cudaMemcpyDeviceToHost));
    if (J0_minus) CK(cudaMemcpy(J0_minus, hs.J0m, sizeof(double) * 3, cudaMemcpyDeviceToHost));
    return TSBZ_OK;
  }
  const double dt0 = ctx->subs[0].dt;
  for (auto& hs : ctx->subs) {
    if (hs.dt != dt0) return set_err(ctx, TSBZ_EINVAL, "two-step average needs equal dt");
    if (first + count > hs.steps + 1) return set_err(ctx, TSBZ_EINVAL, "requested steps not computed yet");
  }
  std::vector<double> acc(3 * (size_t)count, 0.0), buf(3 * (size_t)count), j0(3);
  for (auto& hs : ctx->subs) {
    if (count) CK(cudaMemcpy(buf.data(), hs.J + 3LL * first, sizeof(double) * 3 * count, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(j0.data(), hs.J0m, sizeof(double) * 3, cudaMemcpyDeviceToHost));
    for (int i = 0; i < count; ++i)
      for (int ax = 0; ax < 3; ++ax) acc[3 * i + ax] += buf[3 * i + ax] - j0[ax];
  }
  const double inv = 1.0 / (double)ctx->subs.size();
  for (size_t i = 0; i < acc.size(); ++i) J[i] = acc[i] * inv;
  if (J0_minus) J0_minus[0] = J0_minus[1] = J0_minus[2] = 0.0;
  return TSBZ_OK;
}

int tsbz_get_current_stats(tsbz_ctx* ctx, int first, int count, double* mean, double* stderr_out) {
  if (!ctx || first < 0 || count < 0 || (count > 0 && (!mean || !stderr_out))) return TSBZ_EINVAL;
  int rc = ensure_ready(ctx);
  if (rc) return rc;
  if ((rc = sync_and_check(ctx))) return rc;
  const double dt0 = ctx->subs[0].dt;
  for (auto& hs : ctx->subs) {
    if (hs.dt != dt0) return set_err(ctx, TSBZ_EINVAL, "two-step statistics need equal dt");
    if (first + count > hs.steps + 1) return set_err(ctx, TSBZ_EINVAL, "requested steps not computed yet");
  }
  const size_t n3 = 3 * (size_t)count, ns = ctx->subs.size();
  std::vector<double> dj(ns * n3), j0(3);
  for (size_t m = 0; m < ns; ++m) {
    const HostSub& hs = ctx->subs[m];
    if (count) CK(cudaMemcpy(dj.data() + m * n3, hs.J + 3LL * first, sizeof(double) * n3, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(j0.data(), hs.J0m, sizeof(double) * 3, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n3; ++i) dj[m * n3 + i] -= j0[i % 3];
  }
  // two passes in sub-simulation order: the mean (Eq. 9, the same arithmetic
  // as tsbz_get_current(-1)), then the squared deviations
  const double inv = 1.0 / (double)ns;
  for (size_t i = 0; i < n3; ++i) {
    double acc = 0.0;
    for (size_t m = 0; m < ns; ++m) acc += dj[m * n3 + i];
    mean[i] = acc * inv;
    double ss = 0.0;
    for (size_t m = 0; m < ns; ++m) {
      const double d = dj[m * n3 + i] - mean[i];
      ss += d * d;
    }
    stderr_out[i] = ns > 1 ? std::sqrt(ss / ((double)ns * (double)(ns - 1))) : 0.0;
  }
  return TSBZ_OK;
}

int tsbz_get_density(tsbz_ctx* ctx, int s, double* rho, size_t cap) {
  int rc = check_sub(ctx, s);
  if (rc) return rc;
  const CellDev& c = ctx->cells[ctx->subs[s].cell].dev;
  if (!rho || cap < (size_t)c.npts) return set_err(ctx, TSBZ_EINVAL, "rho buffer too small");
  if ((rc = ensure_ready(ctx))) return rc;
  if ((rc = sync_and_check(ctx))) return rc;
  CK(cudaMemcpy(rho, ctx->subs[s].rho, sizeof(double) * c.npts, cudaMemcpyDeviceToHost));
  return TSBZ_OK;
}

int tsbz_get_norms(tsbz_ctx* ctx, int s, double* norms, size_t cap) {
  int rc = check_sub(ctx, s);
  if (rc) return rc;
  const HostSub& hs = ctx->subs[s];
  const size_t n = (size_t)hs.n_k * ctx->cells[hs.cell].dev.n_bands;
  if (!norms || cap < n) return set_err(ctx, TSBZ_EINVAL, "norms buffer too small");
  if ((rc = ensure_ready(ctx))) return rc;
  if ((rc = sync_and_check(ctx))) return rc;
  CK(cudaMemcpy(norms, hs.norms, sizeof(double) * n, cudaMemcpyDeviceToHost));
  return TSBZ_OK;
}

int tsbz_get_step(tsbz_ctx* ctx, int s, int* step) {
  int rc = check_sub(ctx, s);
  if (rc) return rc;
  if (!step) return TSBZ_EINVAL;
  *step = ctx->subs[s].steps;
  return TSBZ_OK;
}

int tsbz_get_state(tsbz_ctx* ctx, int s, double* psi, size_t cap, int* step) {
  int rc = check_sub(ctx, s);
  if (rc) return rc;
  if (!ctx->laid_out) return set_err(ctx, TSBZ_ESTATE, "no state");
  const HostSub& hs = ctx->subs[s];
  const CellDev& c = ctx->cells[hs.cell].dev;
  const long long n = (long long)hs.n_k * c.n_bands * c.npts;
  if (!psi || (long long)cap < n) return set_err(ctx, TSBZ_EINVAL, "psi buffer too small");
  const char* src = (const char*)ctx->psi + ctx->unit_psi_off[hs.unit0] * ctx->elem_size();
  if (ctx->precision == TSBZ_FP64)
    launch_convert_out_t<double>(src, ctx->staging, n, ctx->stream);
  else
    launch_convert_out_t<float>(src, ctx->staging, n, ctx->stream);
  ++ctx->launches;
  CK(cudaMemcpyAsync(psi, ctx->staging, sizeof(double2) * n, cudaMemcpyDeviceToHost, ctx->stream));
  if ((rc = sync_and_check(ctx))) return rc;
  if (step) *step = hs.steps;
  return TSBZ_OK;
}

int tsbz_load_state(tsbz_ctx* ctx, int s, const double* psi, size_t n_elems, int step) {
  int rc = check_sub(ctx, s);
  if (rc) return rc;
  if (!ctx->laid_out || !ctx->subs[s].loaded) return set_err(ctx, TSBZ_ESTATE, "load a ground state first");
  HostSub& hs = ctx->subs[s];
  if (step < 0 || step > hs.max_steps) return set_err(ctx, TSBZ_EINVAL, "bad step");
  if ((rc = ensure_ready(ctx))) return rc;
  if ((rc = copy_state_in(ctx, s, psi, n_elems, 0))) return rc;
  ctx->p_next_valid = false;
  CK(cudaMemcpyAsync(ctx->d_steps + s, &step, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  hs.steps = step;
  // rho, norms and v_Hxc from the restored orbitals (no current is written)
  std::vector<int> mask(ctx->subs.size(), 0);
  CK(cudaMemcpyAsync(ctx->d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->precision == TSBZ_FP64) {
    run_field<double>(ctx, TSBZ_FIELD_J0MINUS);
    run_observe<double>(ctx, TSBZ_FIN_J0MINUS);
    run_hxc<double>(ctx);
  } else {
    run_field<float>(ctx, TSBZ_FIELD_J0MINUS);
    run_observe<float>(ctx, TSBZ_FIN_J0MINUS);
    run_hxc<float>(ctx);
  }
  return sync_and_check(ctx);
}

int tsbz_get_cell_tables(tsbz_ctx* ctx, int cell_id, double* vloc, size_t cap, double* proj_norms, size_t ncap) {
  if (!ctx || cell_id < 0 || cell_id >= (int)ctx->cells.size()) return TSBZ_EINVAL;
  const HostCell& hc = ctx->cells[cell_id];
  if (vloc) {
    if (cap < hc.vloc.size()) return set_err(ctx, TSBZ_EINVAL, "vloc buffer too small");
    std::memcpy(vloc, hc.vloc.data(), sizeof(double) * hc.vloc.size());
  }
  if (proj_norms) {
    const size_t n = 4 * (size_t)hc.desc.n_atoms;
    if (ncap < n) return set_err(ctx, TSBZ_EINVAL, "norm buffer too small");
    if (hc.dev.use_proj) std::memcpy(proj_norms, hc.pnorm.data(), sizeof(double) * n);
  }
  return TSBZ_OK;
}

int tsbz_get_launch_count(tsbz_ctx* ctx, long long* launches) {
  if (!ctx || !launches) return TSBZ_EINVAL;
  *launches = ctx->launches;
  return TSBZ_OK;
}

int tsbz_set_graphs(tsbz_ctx* ctx, int on) {
  if (!ctx) return TSBZ_EINVAL;
  ctx->graphs = on != 0;
  return TSBZ_OK;
}

int tsbz_set_profiling(tsbz_ctx* ctx, int on) {
  if (!ctx) return TSBZ_EINVAL;
  ctx->prof = on != 0;
  return TSBZ_OK;
}

int tsbz_get_timings(tsbz_ctx* ctx, double* times_ms, int n) {
  if (!ctx || !times_ms || n < 0) return TSBZ_EINVAL;
  for (int i = 0; i < n && i < TSBZ_N_FAM; ++i) times_ms[i] = ctx->times[i];
  return TSBZ_OK;
}

int tsbz_autotune(tsbz_ctx* ctx, int budget_ms, int* n_tried) {
  if (!ctx || budget_ms < 0) return TSBZ_EINVAL;
  int rc = ensure_ready(ctx);
  if (rc) return rc;
  bool any = false;
  for (auto& hs : ctx->subs) any = any || hs.steps < hs.max_steps;
  if (!any) return set_err(ctx, TSBZ_ESTATE, "every sub-simulation has spent its step budget: nothing to time");
  Snapshot sn;
  if ((rc = snapshot_take(ctx, sn))) {
    if (sn.psi) dfree(ctx, sn.psi);
    if (sn.P) dfree(ctx, sn.P);
    return rc;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool prof = ctx->prof;
  ctx->prof = false;
  const long long launches0 = ctx->launches;
  constexpr int kTimed = 2, kRounds = 2;   // timed windows of steps per variant, after one untimed step
  float spent = 0.f;
  int tried = 0;
  std::vector<int> before;
  for (auto& hc : ctx->cells) before.push_back(hc.variant);
  for (auto& hc : ctx->cells) {
    if (hc.unit_ids.empty()) continue;
    const int nv = n_variants(ctx, hc);
    for (int v = 0; v < TSBZ_MAX_VARIANTS; ++v) hc.tune_ms[v] = 0.0;
    const int keep = hc.variant < nv ? hc.variant : 0;
    int best = keep;
    if (nv > 1) {
      double best_ms = 0.0;
      for (int v = 0; v < nv; ++v) {
        // the default variant is always timed; the others while the budget lasts
        if (v > 0 && spent >= (float)budget_ms) break;
        hc.variant = v;
        rc = ctx->precision == TSBZ_FP64 ? run_step<double>(ctx) : run_step<float>(ctx);
        if (rc) break;
        // the faster of kRounds windows of kTimed steps (the first window of a
        // fresh variant can include one-time costs of its first launches)
        float best_win = 0.f;
        for (int r = 0; r < kRounds && !rc; ++r) {
          cudaEventRecord(e0, ctx->stream);
          for (int i = 0; i < kTimed && !rc; ++i)
            rc = ctx->precision == TSBZ_FP64 ? run_step<double>(ctx) : run_step<float>(ctx);
          cudaEventRecord(e1, ctx->stream);
          if (rc) break;
          const cudaError_t es = cudaEventSynchronize(e1);
          if (es != cudaSuccess) {
            rc = set_err(ctx, TSBZ_ECUDA, std::string("autotune: ") + cudaGetErrorString(es));
            break;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          spent += ms;
          best_win = (r == 0 || ms < best_win) ? ms : best_win;
        }
        if (rc) break;
        spent += best_win / kTimed;   // the untimed step
        hc.tune_ms[v] = best_win / kTimed;
        ++tried;
        if (v == 0 || hc.tune_ms[v] < best_ms) {
          best_ms = hc.tune_ms[v];
          best = v;
        }
      }
    }
    hc.variant = best;
    if (rc) break;
  }
  ctx->prof = prof;
  ctx->launches = launches0;   // trial steps are not part of the run
  for (size_t i = 0; i < ctx->cells.size(); ++i)
    if (ctx->cells[i].variant != before[i]) sn.p_next_valid = false;   // P of the old variant's pass
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int rr = snapshot_restore(ctx, sn);
  drop_step_graph(ctx);
  if (n_tried) *n_tried = tried;
  return rc ? rc : rr;
}

int tsbz_ground_state(tsbz_ctx* ctx, int max_iter, double tol, int degree, double mix, int* iters_out,
                      double* err_out) {
  if (!ctx || max_iter < 1 || !(tol > 0.0) || degree < 2 || degree > 200 || !(mix > 0.0 && mix <= 1.0))
    return TSBZ_EINVAL;
  if (ctx->precision != TSBZ_FP64)
    return set_err(ctx, TSBZ_EINVAL, "the ground-state solver runs in TSBZ_FP64 contexts");
  if (!ctx->laid_out) return set_err(ctx, TSBZ_ESTATE, "load starting orbitals first");
  for (auto& hs : ctx->subs) {
    if (!hs.loaded) return set_err(ctx, TSBZ_ESTATE, "every sub-simulation needs starting orbitals");
    if (hs.steps != 0) return set_err(ctx, TSBZ_ESTATE, "the ground state is solved before the first step");
  }
  int max_units = 0;
  size_t max_mat = 0;   // complex entries of one cell's n_units n_b^2 matrices
  for (auto& hc : ctx->cells) {
    if (hc.dev.n_bands > scf_max_bands())
      return set_err(ctx, TSBZ_EINVAL, "the ground-state solver takes at most 256 bands per cell");
    max_units = std::max(max_units, (int)hc.unit_ids.size());
    max_mat = std::max(max_mat, hc.unit_ids.size() * (size_t)hc.dev.n_bands * hc.dev.n_bands);
  }
  int rc = ensure_ready(ctx);
  if (rc) return rc;
  const size_t ns = ctx->subs.size();
  // scratch: Gram matrices, coefficients, bounds
  void *dS = nullptr, *dH = nullptr, *dC = nullptr, *dW1 = nullptr, *dW2 = nullptr;
  double *dlam = nullptr, *dfa = nullptr, *dfb = nullptr, *dfc = nullptr;
  int* dbad = nullptr;
  const size_t mat = std::max<size_t>(max_mat, 1) * sizeof(double2);
  auto cleanup = [&]() {
    for (void* p : {dS, dH, dC, dW1, dW2, (void*)dlam, (void*)dfa, (void*)dfb, (void*)dfc, (void*)dbad})
      dfree(ctx, p);
    ctx->d_filt = nullptr;
  };
  if ((rc = dalloc(ctx, mat, &dS)) || (rc = dalloc(ctx, mat, &dH)) || (rc = dalloc(ctx, mat, &dC)) ||
      (rc = dalloc(ctx, mat, &dW1)) || (rc = dalloc(ctx, mat, &dW2)) ||
      (rc = dalloc_t(ctx, (size_t)max_units, &dlam)) || (rc = dalloc_t(ctx, 3 * (size_t)ctx->n_units, &dfa)) ||
      (rc = dalloc_t(ctx, 3 * (size_t)ctx->n_units, &dfb)) || (rc = dalloc_t(ctx, 3 * (size_t)ctx->n_units, &dfc)) ||
      (rc = dalloc_t(ctx, 1, &dbad))) {
    cleanup();
    return rc;
  }
  CK(cudaMemsetAsync(dbad, 0, sizeof(int), ctx->stream));
  // h times the block in `out`: filter coefficients (1, 0, 0)
  std::vector<double> ones(3 * ctx->n_units, 0.0);
  for (long long u = 0; u < ctx->n_units; ++u) ones[3 * u] = 1.0;
  CK(cudaMemcpyAsync(dfc, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice, ctx->stream));
  auto apply = [&](HostCell& hc, const double* filt, void* in, void* out, void* prev) {
    ctx->d_filt = filt;
    LaunchSet L = make_set(ctx, hc);
    launch_bra<double>(L, in, ctx->P, 0, 0, ctx->stream);
    launch_stage<double>(L, in, out, prev, ctx->P, 0, ctx->stream);
    ctx->launches += 2;
  };
  // Orthonormalisation of the block in `y` by shifted CholeskyQR3, then the
  // largest Ritz value from h applied to the orthonormal block.  The three
  // rotations alternate y -> hy -> y -> hy, h Q goes into `y`, and the result
  // is copied back into `y` once every cell is done.  The first pass shifts
  // the Gram matrix by 11 (m n + n (n + 1)) u tr(S) (m points, n bands,
  // u = 2^-53).
  std::vector<double> lam_u(ctx->n_units, 0.0);
  auto orthonormalise = [&](void* y, void* hy) -> int {
    for (auto& hc : ctx->cells) {
      if (hc.unit_ids.empty()) continue;
      LaunchSet L = make_set(ctx, hc);
      const int nb = hc.dev.n_bands;
      const double m = (double)hc.dev.npts, n = (double)nb;
      const double shift_coef = 11.0 * (m * n + n * (n + 1.0)) * std::ldexp(1.0, -53);
      void* src = y;
      void* dst = hy;
      for (int pass = 0; pass < 3; ++pass) {
        launch_scf_gram(L, src, nullptr, dS, nullptr, ctx->stream);
        launch_scf_ortho(L.n_units, nb, pass == 0 ? shift_coef : 0.0, 0, dS, dH, dC, dW1, dW2, dlam, dbad,
                         ctx->stream);
        launch_scf_rotate(L, src, dC, dst, ctx->stream);
        std::swap(src, dst);
      }
      // the orthonormal block is in `src` (= hy); h Q into `dst` (= y)
      apply(hc, dfc, src, dst, nullptr);
      L = make_set(ctx, hc);
      launch_scf_gram(L, src, dst, dS, dH, ctx->stream);
      launch_scf_ortho(L.n_units, nb, 0.0, 1, dS, dH, dC, dW1, dW2, dlam, dbad, ctx->stream);
      ctx->launches += 11;
      std::vector<double> lam(L.n_units);
      CK(cudaMemcpyAsync(lam.data(), dlam, sizeof(double) * lam.size(), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      for (size_t i = 0; i < lam.size(); ++i) lam_u[hc.unit_ids[i]] = lam[i];
    }
    CK(cudaMemcpyAsync(y, hy, ctx->psi_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    return TSBZ_OK;
  };
  // upper bound of the spectrum of h_k (A = 0) per unit: FD kinetic with the
  // q terms, the largest v_eff of the sub-simulation, and sum_j |E_j|
  auto upper_bound = [&](std::vector<double>& ub) -> int {
    ub.assign(ctx->n_units, 0.0);
    std::vector<double> kc(3 * ctx->n_units);
    CK(cudaMemcpyAsync(kc.data(), ctx->kcart, sizeof(double) * kc.size(), cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<std::vector<double>> vmax_sub(ns);
    for (size_t s = 0; s < ns; ++s) {
      const HostSub& hs = ctx->subs[s];
      const CellDev& c = ctx->cells[hs.cell].dev;
      std::vector<double> v(c.npts);
      CK(cudaMemcpyAsync(v.data(), hs.veff, sizeof(double) * c.npts, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      double vm = v[0];
      for (double x : v) vm = std::max(vm, x);
      vmax_sub[s] = {vm};
    }
    for (size_t s = 0; s < ns; ++s) {
      const HostSub& hs = ctx->subs[s];
      const HostCell& hc = ctx->cells[hs.cell];
      const CellDev& c = hc.dev;
      double enl = 0.0;
      if (c.use_proj) enl = c.n_atoms * (std::fabs(hc.desc.e_kb_s) + 3.0 * std::fabs(hc.desc.e_kb_p));
      for (int k = 0; k < hs.n_k; ++k) {
        const long long u = hs.unit0 + k;
        double kin = 0.0, q2 = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
          double lap = -c.lapw[ax][0], grd = 0.0;
          for (int m = 1; m <= c.nd; ++m) {
            lap += 2.0 * std::fabs(c.lapw[ax][m]);
            grd += 2.0 * std::fabs(c.gradw[ax][m]);
          }
          const double q = kc[3 * u + ax];
          kin += 0.5 * lap + std::fabs(q) * grd;
          q2 += q * q;
        }
        ub[u] = 1.02 * (kin + 0.5 * q2 + vmax_sub[s][0] + enl) + 0.1;
      }
    }
    return TSBZ_OK;
  };
  // density mixing (Pulay, as the reference solver), per sub-simulation
  struct Mix {
    std::vector<std::vector<double>> rin, res;
  };
  std::vector<Mix> mixes(ns);
  std::vector<std::vector<double>> rho_in(ns);
  for (size_t s = 0; s < ns; ++s) {
    const HostSub& hs = ctx->subs[s];
    const HostCell& hc = ctx->cells[hs.cell];
    const double ne = hc.desc.occ * hc.desc.n_bands;
    rho_in[s].assign(hc.dev.npts, ne / hc.dev.omega);
    CK(cudaMemcpyAsync(hs.rho, rho_in[s].data(), sizeof(double) * hc.dev.npts, cudaMemcpyHostToDevice,
                       ctx->stream));
  }
  run_hxc<double>(ctx);
  run_field<double>(ctx, TSBZ_FIELD_J0MINUS);
  if ((rc = orthonormalise(ctx->psi, ctx->tA))) {
    cleanup();
    return rc;
  }
  double err = 1e300;
  int it = 0;
  std::vector<double> ub, fa(3 * ctx->n_units), fb(3 * ctx->n_units);
  for (it = 1; it <= max_iter; ++it) {
    if ((rc = upper_bound(ub))) break;
    for (long long u = 0; u < ctx->n_units; ++u) {
      // the filter damps [a, b]: a a little above the block's largest Ritz value,
      // so that the top occupied state is amplified against the first empty one
      const double a = lam_u[u] + 0.1, b = std::max(ub[u], a + 1.0);
      const double e = 0.5 * (b - a), cc = 0.5 * (b + a);
      fa[3 * u] = 1.0 / e;
      fa[3 * u + 1] = -cc / e;
      fa[3 * u + 2] = 0.0;
      fb[3 * u] = 2.0 / e;
      fb[3 * u + 1] = -2.0 * cc / e;
      fb[3 * u + 2] = -1.0;
    }
    CK(cudaMemcpyAsync(dfa, fa.data(), sizeof(double) * fa.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dfb, fb.data(), sizeof(double) * fb.size(), cudaMemcpyHostToDevice, ctx->stream));
    // Chebyshev filter of the block: Y_1 = (h - c)/e Y_0, Y_{j+1} = 2 (h - c)/e Y_j - Y_{j-1}
    void* buf[3] = {ctx->psi, ctx->tA, ctx->tB};
    int prev = 0, cur = 1;
    for (auto& hc : ctx->cells)
      if (!hc.unit_ids.empty()) apply(hc, dfa, buf[0], buf[1], nullptr);
    for (int j = 1; j < degree; ++j) {
      const int next = 3 - prev - cur;
      for (auto& hc : ctx->cells)
        if (!hc.unit_ids.empty()) apply(hc, dfb, buf[cur], buf[next], buf[prev]);
      prev = cur;
      cur = next;
    }
    if ((rc = orthonormalise(buf[cur], buf[3 - prev - cur]))) break;
    if (buf[cur] != ctx->psi)
      CK(cudaMemcpyAsync(ctx->psi, buf[cur], ctx->psi_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    // output density, then the mixed input density and its v_Hxc
    run_observe<double>(ctx, TSBZ_FIN_RHO);
    err = 0.0;
    for (size_t s = 0; s < ns; ++s) {
      HostSub& hs = ctx->subs[s];
      const HostCell& hc = ctx->cells[hs.cell];
      const int np = hc.dev.npts;
      std::vector<double> rout(np);
      CK(cudaMemcpyAsync(rout.data(), hs.rho, sizeof(double) * np, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      const double ne = hc.desc.occ * hc.desc.n_bands;
      double e = 0.0;
      for (int r = 0; r < np; ++r) e += std::fabs(rout[r] - rho_in[s][r]);
      e *= hc.dev.dv / ne;
      err = std::max(err, e);
      Mix& mx = mixes[s];
      std::vector<double> f(np);
      for (int r = 0; r < np; ++r) f[r] = rout[r] - rho_in[s][r];
      mx.rin.push_back(rho_in[s]);
      mx.res.push_back(f);
      if (mx.rin.size() > 8) {
        mx.rin.erase(mx.rin.begin());
        mx.res.erase(mx.res.begin());
      }
      const int m = (int)mx.res.size();
      // bordered system [B 1; 1 0][c; l] = [0; 1], B_ij = <f_i, f_j>
      std::vector<double> A((m + 1) * (m + 1), 0.0), x(m + 1, 0.0);
      for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) {
          double d = 0.0;
          for (int r = 0; r < np; ++r) d += mx.res[i][r] * mx.res[j][r];
          A[i * (m + 1) + j] = d;
        }
        A[i * (m + 1) + m] = 1.0;
        A[m * (m + 1) + i] = 1.0;
      }
      x[m] = 1.0;
      // Gaussian elimination with partial pivoting
      bool solved = true;
      const int n = m + 1;
      for (int col = 0; col < n && solved; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
          if (std::fabs(A[r * n + col]) > std::fabs(A[piv * n + col])) piv = r;
        if (std::fabs(A[piv * n + col]) < 1e-300) {
          solved = false;
          break;
        }
        if (piv != col) {
          for (int k2 = 0; k2 < n; ++k2) std::swap(A[col * n + k2], A[piv * n + k2]);
          std::swap(x[col], x[piv]);
        }
        for (int r = col + 1; r < n; ++r) {
          const double fct = A[r * n + col] / A[col * n + col];
          for (int k2 = col; k2 < n; ++k2) A[r * n + k2] -= fct * A[col * n + k2];
          x[r] -= fct * x[col];
        }
      }
      std::vector<double> coef(m, 0.0);
      if (solved) {
        for (int r = n - 1; r >= 0; --r) {
          double t = x[r];
          for (int k2 = r + 1; k2 < n; ++k2) t -= A[r * n + k2] * x[k2];
          x[r] = t / A[r * n + r];
        }
        for (int i = 0; i < m; ++i) coef[i] = x[i];
      } else {
        coef[m - 1] = 1.0;
      }
      for (int r = 0; r < np; ++r) {
        double v = 0.0;
        for (int i = 0; i < m; ++i) v += coef[i] * (mx.rin[i][r] + mix * mx.res[i][r]);
        rho_in[s][r] = std::max(v, 0.0);
      }
      CK(cudaMemcpyAsync(hs.rho, rho_in[s].data(), sizeof(double) * np, cudaMemcpyHostToDevice, ctx->stream));
    }
    if (err < tol) break;
    run_hxc<double>(ctx);
  }
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  cleanup();
  if (rc) return rc;
  // the orbitals are the new ground state: rho, v_Hxc, J(0-) and J(0+) follow from them
  for (auto& hs : ctx->subs) {
    hs.need_init = true;
    hs.need_j0plus = true;
  }
  ctx->p_next_valid = false;
  drop_step_graph(ctx);
  if (iters_out) *iters_out = std::min(it, max_iter);
  if (err_out) *err_out = err;
  if (bad) return set_err(ctx, TSBZ_ENONFINITE, "the block lost rank (overlap matrix not positive definite)");
  if ((rc = ensure_ready(ctx))) return rc;
  if ((rc = sync_and_check(ctx))) return rc;
  return err < tol ? TSBZ_OK : set_err(ctx, TSBZ_ESTATE, "ground state not converged within max_iter");
}

int tsbz_set_propagator(tsbz_ctx* ctx, int propagator) {
  if (!ctx) return TSBZ_EINVAL;
  if (propagator != TSBZ_PROP_TAYLOR4 && propagator != TSBZ_PROP_ETRS)
    return set_err(ctx, TSBZ_EINVAL, "unknown propagator");
  if (propagator == TSBZ_PROP_ETRS && ctx->precision == TSBZ_FP32_TC)
    return set_err(ctx, TSBZ_EINVAL, "the ETRS propagator runs in TSBZ_FP64 and TSBZ_FP32 modes");
  if (propagator != ctx->propagator) {
    ctx->propagator = propagator;
    ctx->p_next_valid = false;
    drop_step_graph(ctx);
  }
  return TSBZ_OK;
}

int tsbz_get_variant(tsbz_ctx* ctx, int cell_id, int* variant, int* n_variants_out, double* ms, int n_ms) {
  if (!ctx || cell_id < 0 || cell_id >= (int)ctx->cells.size()) return TSBZ_EINVAL;
  const HostCell& hc = ctx->cells[cell_id];
  if (variant) *variant = hc.variant;
  if (n_variants_out) *n_variants_out = n_variants(ctx, hc);
  for (int v = 0; ms && v < n_ms && v < TSBZ_MAX_VARIANTS; ++v) ms[v] = hc.tune_ms[v];
  return TSBZ_OK;
}

int tsbz_set_variant(tsbz_ctx* ctx, int cell_id, int variant) {
  if (!ctx || cell_id < 0 || cell_id >= (int)ctx->cells.size()) return TSBZ_EINVAL;
  HostCell& hc = ctx->cells[cell_id];
  if (variant < 0 || variant >= n_variants(ctx, hc))
    return set_err(ctx, TSBZ_EINVAL, "variant out of range for this cell and precision");
  if (hc.variant != variant) {
    hc.variant = variant;
    ctx->p_next_valid = false;   // the projections in P may come from the other variant's pass
    drop_step_graph(ctx);
  }
  return TSBZ_OK;
}

int tsbz_selftest_bounded_wait(int device, int polls, int deliver, int* status_out) {
  if (polls < 1 || polls > (1 << 24)) return TSBZ_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return TSBZ_ECUDA;
  int* d_status = nullptr;
  if (cudaMalloc(&d_status, sizeof(int)) != cudaSuccess) return TSBZ_ENOMEM;
  int st = 0;
  cudaError_t e = cudaMemset(d_status, 0, sizeof(int));
  if (e == cudaSuccess) {
    k_selftest_wait<<<1, 64>>>(polls, deliver ? 1 : 0, d_status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_status);
  if (e != cudaSuccess) return TSBZ_ECUDA;
  if (status_out) *status_out = st;
  return (st & BK_STATUS_TIMEOUT) ? TSBZ_ETIMEOUT : TSBZ_OK;
}

const char* tsbz_last_error(tsbz_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void tsbz_destroy(tsbz_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  for (void* p : ctx->owned) {
    if (ctx->has_alloc)
      ctx->alloc.free(p, ctx->alloc.user);
    else
      cudaFree(p);
  }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->step_graph) cudaGraphExecDestroy(ctx->step_graph);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->gstream) {
    cudaStreamSynchronize(ctx->gstream);
    cudaStreamDestroy(ctx->gstream);
  }
  delete ctx;
}

}  // extern "C"
