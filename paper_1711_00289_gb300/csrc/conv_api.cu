// conv_api.cu -- the extern "C" entry points of include/conv.h: argument
// validation on the host, packing of kernel parameters, dispatch to a kernel
// path.  Nothing here allocates or synchronises.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "compact.h"
#include "validate.h"

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

namespace cvg {

bool deep_params_ok(const conv_deep_params* p) {
  return p && finite_pos(p->capelmt + 1.0) && p->capelmt >= 0.0 && p->lambda_default >= 0.0 &&
         std::isfinite(p->lambda_default) && finite_pos(p->tau_default) && p->c0 >= 0.0 &&
         std::isfinite(p->c0) && p->alpha_dd >= 0.0 && p->alpha_dd <= 1.0 &&
         finite_pos(p->p_launch_min) && finite_pos(p->p_top_lim) && p->q_min >= 0.0 &&
         p->q_min < 1e-3 && finite_pos(p->ent_zscale) && p->n_newton_lcl >= 1 &&
         p->n_newton_lcl <= 32 && p->n_newton_h >= 0 && p->n_newton_h <= 32 &&
         p->n_plumes >= 1 && p->n_plumes <= CONV_MAX_PLUMES && std::isfinite(p->plume_spread) &&
         p->plume_spread >= 1.0;
}

bool shallow_params_ok(const conv_shallow_params* p) {
  return p && p->eps_s >= 0.0 && std::isfinite(p->eps_s) && finite_pos(p->tke) && p->c_m >= 0.0 &&
         std::isfinite(p->c_m) && finite_pos(p->cin_scale) && p->cin_max >= 0.0 &&
         std::isfinite(p->a_w) && p->b_w >= 0.0 && std::isfinite(p->b_w) && p->ql_crit >= 0.0 &&
         finite_pos(p->p_lcl_min) && finite_pos(p->p_lfc_min) && finite_pos(p->p_top_lim) &&
         p->n_newton_lcl >= 1 && p->n_newton_lcl <= 32 && p->n_newton_h >= 0 &&
         p->n_newton_h <= 32 && std::isfinite(p->evap_k) && p->evap_k >= 0.0;
}

}  // namespace cvg

namespace {

using cvg::deep_params_ok;
using cvg::RunArgs;
using cvg::shallow_params_ok;

conv_status fill_grid(const conv_grid* g, RunArgs& a) {
  if (!g || g->pver < 4 || g->pver > CONV_MAX_LEVELS || g->n_cols < 0 || g->ld < g->n_cols ||
      !g->hyai || !g->hybi || !finite_pos(g->p0))
    return CONV_ERR_ARG;
  a.L.pver = g->pver;
  a.L.p0 = g->p0;
  for (int i = 0; i <= CONV_MAX_LEVELS; ++i) {
    a.L.a[i] = i <= g->pver ? g->hyai[i] : 0.0;
    a.L.b[i] = i <= g->pver ? g->hybi[i] : 0.0;
    a.L.ap0f[i] = (float)(a.L.a[i] * g->p0);
    a.L.bf[i] = (float)a.L.b[i];
  }
  for (int i = 0; i <= g->pver; ++i)  // all pver + 1 interfaces, the surface included
    if (!std::isfinite(g->hyai[i]) || !std::isfinite(g->hybi[i])) return CONV_ERR_ARG;
  for (int i = 0; i < g->pver; ++i) {  // interfaces must be ordered top -> surface
    if (g->hyai[i + 1] * g->p0 + g->hybi[i + 1] * 1e5 <= g->hyai[i] * g->p0 + g->hybi[i] * 1e5)
      return CONV_ERR_ARG;
  }
  a.n = g->n_cols;
  a.ld = g->ld;
  return CONV_OK;
}

bool out_ok(const conv_out* o) { return o && o->dTdt && o->dqdt && o->prec && o->flags; }

cvg::OutP to_outp(const conv_out* o) {
  cvg::OutP p;
  std::memset(&p, 0, sizeof p);
  if (!o) return p;
  p.dTdt = o->dTdt;
  p.dqdt = o->dqdt;
  p.prec = o->prec;
  p.flags = o->flags;
  p.kb = o->kb;
  p.klcl = o->klcl;
  p.ktop = o->ktop;
  p.kaux = o->kaux;
  p.cape = o->cape;
  p.mb = o->mb;
  p.cons_err = o->cons_err;
  p.mu = o->mu;
  p.du = o->du;
  p.md = o->md;
  return p;
}

bool has_flux(const cvg::OutP& o) { return o.mu || o.du || o.md; }

// AUTO selects the compacted path; a shallow-only run has nothing to compact
// (no deep trigger) and always uses the plain kernel.
int pick_path(const conv_launch* l, int mode) {
  if (!(mode & cvg::MODE_DEEP)) return CONV_PATH_PLAIN;
  const int p = l ? l->path : CONV_PATH_AUTO;
  return p == CONV_PATH_AUTO ? CONV_PATH_COMPACT : p;
}

size_t needed_ws(int n, int pver, conv_precision prec, int path) {
  return path == CONV_PATH_COMPACT ? cvg::compact_workspace_bytes(n, pver, prec == CONV_FP64)
                                   : 0;
}

conv_status dispatch(RunArgs& a, conv_precision prec, const conv_launch* launch, void* ws,
                     size_t ws_bytes) {
  cvg::fill_q(a);
  if (prec != CONV_FP64 && prec != CONV_MIXED) return CONV_ERR_ARG;
  if (launch && (launch->path < CONV_PATH_AUTO || launch->path > CONV_PATH_COMPACT))
    return CONV_ERR_ARG;
  if (launch && (launch->block_threads < 0 || launch->block_threads > 1024)) return CONV_ERR_ARG;
  if (launch && (launch->mapping < CONV_MAP_DEFAULT || launch->mapping > CONV_MAP_WARP))
    return CONV_ERR_ARG;
  const int path = pick_path(launch, a.mode);
  const bool spectrum = (a.mode & cvg::MODE_DEEP) && a.dp.n_plumes > 1;
  if (spectrum && (has_flux(a.od) || has_flux(a.os))) return CONV_ERR_UNSUPPORTED;
  a.ext = has_flux(a.od) || has_flux(a.os) || ((a.mode & cvg::MODE_SHALLOW) && a.sp.evap_k > 0.0) ||
          spectrum;
  a.block = launch ? launch->block_threads : 0;
  a.mapping = launch ? launch->mapping : CONV_MAP_DEFAULT;
  for (int i = 0; i < 3; ++i)
    a.ev[i] = (launch && launch->stage_events)
                  ? static_cast<cudaEvent_t>(launch->stage_events[i])
                  : nullptr;
  const size_t need = needed_ws(a.n, a.L.pver, prec, path);
  if (need > 0) {
    if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
      return CONV_ERR_WORKSPACE;
  }
  cudaError_t e;
  if (path == CONV_PATH_PLAIN) {
    e = cvg::launch_plain(a, prec == CONV_FP64);
  } else {
    e = cvg::launch_compact(a, prec == CONV_FP64, ws, ws_bytes);
  }
  return e == cudaSuccess ? CONV_OK : CONV_ERR_CUDA;
}

conv_status common_in(const conv_grid* grid, const conv_in* in, double dt, RunArgs& a) {
  std::memset(&a, 0, sizeof a);
  conv_status s = fill_grid(grid, a);
  if (s != CONV_OK) return s;
  if (!in || !in->T || !in->q || !in->ps) return CONV_ERR_ARG;
  if (!(std::isfinite(dt) && dt > 0.0)) return CONV_ERR_ARG;
  a.T = in->T;
  a.q = in->q;
  a.ps = in->ps;
  a.lam = in->lambda;
  a.tau = in->tau;
  a.dt = dt;
  return CONV_OK;
}

}  // namespace

bool cvg::grid_ok(const conv_grid* g) {
  RunArgs a;
  std::memset(&a, 0, sizeof a);
  return fill_grid(g, a) == CONV_OK;
}

namespace {
conv_status transport_run(const conv_grid* grid, const double* ps, const conv_out* deep_out,
                          const conv_out* shallow_out, double dt, int ntr, const void* tracers,
                          void* tend_deep, void* tend_shallow, conv_precision prec,
                          conv_stream stream, bool mom, double cp_up, double cp_down) {
  if (prec != CONV_FP64 && prec != CONV_MIXED) return CONV_ERR_ARG;
  RunArgs g;
  std::memset(&g, 0, sizeof g);
  conv_status s = fill_grid(grid, g);
  if (s != CONV_OK) return s;
  if (!ps || ntr < 0 || (!deep_out && !shallow_out)) return CONV_ERR_ARG;
  if (ntr > 0 && !tracers) return CONV_ERR_ARG;
  if (deep_out && shallow_out && !(std::isfinite(dt) && dt > 0.0)) return CONV_ERR_ARG;
  if (ntr > 0 && ((deep_out && !tend_deep) || (shallow_out && !tend_shallow)))
    return CONV_ERR_ARG;
  cvg::TrArgs a;
  std::memset(&a, 0, sizeof a);
  a.L = g.L;
  a.n = g.n;
  a.ld = g.ld;
  a.pver = g.L.pver;
  a.ntr = ntr;
  a.tstride = (size_t)g.L.pver * (size_t)g.ld;
  a.ps = ps;
  a.tr = tracers;
  a.dt = dt;
  a.stream = reinterpret_cast<cudaStream_t>(stream);
  const conv_out* outs[2] = {deep_out, shallow_out};
  cvg::TrScheme* sch[2] = {&a.d, &a.s};
  void* tends[2] = {tend_deep, tend_shallow};
  for (int m = 0; m < 2; ++m) {
    const conv_out* o = outs[m];
    if (!o) continue;
    if (!o->mu || !o->du || !o->flags || !o->kb || !o->ktop) return CONV_ERR_ARG;
    const bool down = m == 0 && o->md;
    if (down && !o->kaux) return CONV_ERR_ARG;
    *sch[m] = cvg::TrScheme{o->mu, o->du, down ? o->md : nullptr, o->flags, o->kb, o->ktop,
                            down ? o->kaux : nullptr, tends[m]};
  }
  a.has_d = deep_out != nullptr;
  a.has_s = shallow_out != nullptr;
  a.mom = mom;
  a.cp_up = cp_up;
  a.cp_down = cp_down;
  return cvg::launch_transport(a, prec == CONV_FP64) == cudaSuccess ? CONV_OK : CONV_ERR_CUDA;
}
}  // namespace

extern "C" {

void conv_deep_defaults(conv_deep_params* p) {
  if (!p) return;
  p->capelmt = 70.0;
  p->lambda_default = 1e-3;
  p->tau_default = 3600.0;
  p->c0 = 2e-3;
  p->alpha_dd = 0.2;
  p->p_launch_min = 60000.0;
  p->p_top_lim = 4000.0;
  p->q_min = 1e-12;
  p->ent_zscale = 1000.0;
  p->n_newton_lcl = 6;
  p->n_newton_h = 15;
  p->n_plumes = 1;
  p->reserved = 0;
  p->plume_spread = 4.0;
}

void conv_shallow_defaults(conv_shallow_params* p) {
  if (!p) return;
  p->eps_s = 2e-3;
  p->tke = 1.0;
  p->c_m = 0.03;
  p->cin_scale = 10.0;
  p->cin_max = 50.0;
  p->a_w = 1.0;
  p->b_w = 2.0;
  p->ql_crit = 1e-3;
  p->p_lcl_min = 70000.0;
  p->p_lfc_min = 50000.0;
  p->p_top_lim = 4000.0;
  p->n_newton_lcl = 6;
  p->n_newton_h = 15;
  p->evap_k = 0.0;
}

const char* conv_status_str(conv_status s) {
  switch (s) {
    case CONV_OK: return "CONV_OK";
    case CONV_ERR_ARG: return "CONV_ERR_ARG: invalid argument";
    case CONV_ERR_CUDA: return "CONV_ERR_CUDA: CUDA launch or runtime error";
    case CONV_ERR_WORKSPACE: return "CONV_ERR_WORKSPACE: workspace missing, small or misaligned";
    case CONV_ERR_UNSUPPORTED: return "CONV_ERR_UNSUPPORTED: not implemented for these arguments";
    case CONV_ERR_TIMEOUT: return "CONV_ERR_TIMEOUT: bounded device wait gave up";
  }
  return "unknown conv_status";
}

size_t conv_workspace_bytes(const conv_grid* grid, conv_precision prec, const conv_launch* launch) {
  if (!grid || grid->n_cols < 0 || grid->pver < 1 || grid->pver > CONV_MAX_LEVELS) return 0;
  if (prec != CONV_FP64 && prec != CONV_MIXED) return 0;
  return needed_ws(grid->n_cols, grid->pver, prec, pick_path(launch, cvg::MODE_DEEP));
}

conv_status conv_deep_run(const conv_grid* grid, const conv_in* in, const conv_deep_params* par,
                          double dt, conv_precision prec, const conv_out* out,
                          const conv_launch* launch, void* ws, size_t ws_bytes,
                          conv_stream stream) {
  RunArgs a;
  conv_status s = common_in(grid, in, dt, a);
  if (s != CONV_OK) return s;
  if (!deep_params_ok(par) || !out_ok(out)) return CONV_ERR_ARG;
  a.dp = *par;
  conv_shallow_defaults(&a.sp);
  a.od = to_outp(out);
  a.mode = cvg::MODE_DEEP;
  a.stream = reinterpret_cast<cudaStream_t>(stream);
  return dispatch(a, prec, launch, ws, ws_bytes);
}

conv_status conv_shallow_run(const conv_grid* grid, const conv_in* in,
                             const conv_shallow_params* par, conv_precision prec,
                             const conv_out* out, const conv_launch* launch, void* ws,
                             size_t ws_bytes, conv_stream stream) {
  RunArgs a;
  conv_status s = common_in(grid, in, 1.0, a);
  if (s != CONV_OK) return s;
  if (!shallow_params_ok(par) || !out_ok(out)) return CONV_ERR_ARG;
  a.lam = a.tau = nullptr;
  conv_deep_defaults(&a.dp);
  a.sp = *par;
  a.os = to_outp(out);
  a.mode = cvg::MODE_SHALLOW;
  a.stream = reinterpret_cast<cudaStream_t>(stream);
  return dispatch(a, prec, launch, ws, ws_bytes);
}

conv_status conv_deep_shallow_run(const conv_grid* grid, const conv_in* in,
                                  const conv_deep_params* dpar, const conv_shallow_params* spar,
                                  double dt, conv_precision prec, const conv_out* deep_out,
                                  const conv_out* shallow_out, const conv_launch* launch,
                                  void* ws, size_t ws_bytes, conv_stream stream) {
  RunArgs a;
  conv_status s = common_in(grid, in, dt, a);
  if (s != CONV_OK) return s;
  if (!deep_params_ok(dpar) || !shallow_params_ok(spar) || !out_ok(deep_out) ||
      !out_ok(shallow_out))
    return CONV_ERR_ARG;
  a.dp = *dpar;
  a.sp = *spar;
  a.od = to_outp(deep_out);
  a.os = to_outp(shallow_out);
  a.mode = cvg::MODE_DEEP | cvg::MODE_SHALLOW;
  a.stream = reinterpret_cast<cudaStream_t>(stream);
  return dispatch(a, prec, launch, ws, ws_bytes);
}

conv_status conv_tracer_transport(const conv_grid* grid, const double* ps,
                                  const conv_out* deep_out, const conv_out* shallow_out,
                                  double dt, int ntr, const void* tracers, void* tend_deep,
                                  void* tend_shallow, conv_precision prec, conv_stream stream) {
  return transport_run(grid, ps, deep_out, shallow_out, dt, ntr, tracers, tend_deep,
                       tend_shallow, prec, stream, false, 0.0, 0.0);
}

conv_status conv_momentum_transport(const conv_grid* grid, const double* ps,
                                    const conv_out* deep_out, const conv_out* shallow_out,
                                    double dt, double cp_up, double cp_down, const void* uv,
                                    void* tend_deep, void* tend_shallow, conv_precision prec,
                                    conv_stream stream) {
  if (!(cp_up >= 0.0 && cp_up <= 1.0) || !(cp_down >= 0.0 && cp_down <= 1.0))
    return CONV_ERR_ARG;
  if (!uv) return CONV_ERR_ARG;
  return transport_run(grid, ps, deep_out, shallow_out, dt, 2, uv, tend_deep, tend_shallow,
                       prec, stream, true, cp_up, cp_down);
}



conv_status conv_deep_adjoint(const conv_grid* grid, const conv_in* in,
                              const conv_deep_params* par, double dt, conv_precision prec,
                              const double* gP, const double* gH, const double* w_heat,
                              double* gT, double* gq, double* glambda, double* gtau,
                              double* P_out, double* H_out, conv_stream stream) {
  if (prec != CONV_FP64) return prec == CONV_MIXED ? CONV_ERR_UNSUPPORTED : CONV_ERR_ARG;
  RunArgs a;
  conv_status s = common_in(grid, in, dt, a);
  if (s != CONV_OK) return s;
  if (!deep_params_ok(par)) return CONV_ERR_ARG;
  if (par->n_plumes > 1) return CONV_ERR_UNSUPPORTED;  // no adjoint of the variant
  const int n_grad = (gT != nullptr) + (gq != nullptr) + (glambda != nullptr) + (gtau != nullptr);
  if (n_grad != 0 && n_grad != 4) return CONV_ERR_ARG;
  if (n_grad == 0 && !P_out && !H_out) return CONV_ERR_ARG;
  cvg::AdjW w;
  w.given = w_heat != nullptr;
  for (int k = 0; k < CONV_MAX_LEVELS; ++k) {
    w.w[k] = (w_heat && k < grid->pver) ? w_heat[k] : 0.0;
    if (!std::isfinite(w.w[k])) return CONV_ERR_ARG;
  }
  a.dp = *par;
  a.mode = cvg::MODE_DEEP;
  a.stream = reinterpret_cast<cudaStream_t>(stream);
  cvg::fill_q(a);
  const cudaError_t e =
      cvg::launch_deep_adjoint(a, gP, gH, w, gT, gq, glambda, gtau, P_out, H_out);
  return e == cudaSuccess ? CONV_OK : CONV_ERR_CUDA;
}

conv_status conv_deep_shallow_adjoint(const conv_grid* grid, const conv_in* in,
                                      const conv_deep_params* dpar,
                                      const conv_shallow_params* spar, double dt,
                                      conv_precision prec, const double* gPd, const double* gHd,
                                      const double* gPs, const double* gHs,
                                      const double* w_heat, double* gT, double* gq,
                                      double* glambda, double* gtau, double* obj, int gradient,
                                      conv_stream stream) {
  if (prec != CONV_FP64) return prec == CONV_MIXED ? CONV_ERR_UNSUPPORTED : CONV_ERR_ARG;
  RunArgs a;
  conv_status s = common_in(grid, in, dt, a);
  if (s != CONV_OK) return s;
  if (!deep_params_ok(dpar) || !shallow_params_ok(spar) || !gT || !gq) return CONV_ERR_ARG;
  if (spar->evap_k > 0.0 || dpar->n_plumes > 1) return CONV_ERR_UNSUPPORTED;  // no adjoint
  if (gradient && (!glambda || !gtau)) return CONV_ERR_ARG;
  if (!gradient && !obj) return CONV_ERR_ARG;
  cvg::AdjW w;
  w.given = w_heat != nullptr;
  for (int k = 0; k < CONV_MAX_LEVELS; ++k) {
    w.w[k] = (w_heat && k < grid->pver) ? w_heat[k] : 0.0;
    if (!std::isfinite(w.w[k])) return CONV_ERR_ARG;
  }
  a.dp = *dpar;
  a.sp = *spar;
  a.mode = cvg::MODE_DEEP | cvg::MODE_SHALLOW;
  a.stream = reinterpret_cast<cudaStream_t>(stream);
  cvg::fill_q(a);
  const double* g[4] = {gPd, gHd, gPs, gHs};
  const cudaError_t e =
      cvg::launch_step_adjoint(a, g, w, gT, gq, glambda, gtau, obj, gradient != 0);
  return e == cudaSuccess ? CONV_OK : CONV_ERR_CUDA;
}

conv_status conv_advance(const conv_grid* grid, void* T, void* q, const void* T_relax,
                         const void* q_relax, double tau_relax, const conv_out* deep_out,
                         const conv_out* shallow_out, double dt, conv_precision prec,
                         conv_stream stream) {
  if (prec != CONV_FP64 && prec != CONV_MIXED) return CONV_ERR_ARG;
  RunArgs a;
  std::memset(&a, 0, sizeof a);
  conv_status s = fill_grid(grid, a);
  if (s != CONV_OK) return s;
  if (!T || !q || !(std::isfinite(dt) && dt > 0.0) || !std::isfinite(tau_relax)) return CONV_ERR_ARG;
  if (tau_relax > 0.0 && (!T_relax || !q_relax)) return CONV_ERR_ARG;
  if (!deep_out || !shallow_out || !deep_out->dTdt || !deep_out->dqdt || !shallow_out->dTdt ||
      !shallow_out->dqdt)
    return CONV_ERR_ARG;
  a.od = to_outp(deep_out);
  a.os = to_outp(shallow_out);
  a.dt = dt;
  a.stream = reinterpret_cast<cudaStream_t>(stream);
  const cudaError_t e = cvg::launch_advance(a, prec == CONV_FP64, T, q,
                                            tau_relax > 0.0 ? T_relax : T,
                                            tau_relax > 0.0 ? q_relax : q, tau_relax);
  return e == cudaSuccess ? CONV_OK : CONV_ERR_CUDA;
}

}  // extern "C"

// ================================================================ batches
struct conv_batch {
  conv_precision prec;
  int n_members;
  int total;
  int sms;
  cvg::BatchShape shape;
  float tune_ms[7];  // the last autotune's measurements (conv_batch_tune_record)
  bool tuned;
  cvg::RunArgs* d_members;
  int* d_offsets;
  std::vector<int> h_offsets;
};

namespace {

// Autotuner cache: (precision, largest level count, active-fraction decile).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, cvg::BatchShape> g_tune_cache;
std::map<std::pair<int, int>, int> g_last_bucket;  // (prec, pver) -> last measured decile

cvg::BatchShape default_shape(bool fp64, int max_pver, int sms) {
  cvg::BatchShape sh;
  sh.max_pver = max_pver;
  sh.trigger_mapping = 0;
  sh.trigger_block = 128;
  sh.plume_block = 128;
  sh.plume_grid = sms * cvg::batch_plume_occupancy(fp64, 128, max_pver);
  return sh;
}

}  // namespace

extern "C" {

conv_status conv_batch_plan(const conv_member* members, int n_members, conv_precision prec,
                            conv_batch** out) {
  if (!out) return CONV_ERR_ARG;
  *out = nullptr;
  if (!members || n_members < 1 || (prec != CONV_FP64 && prec != CONV_MIXED)) return CONV_ERR_ARG;
  std::vector<RunArgs> h(n_members);
  std::vector<int> off(n_members + 1, 0);
  long long total = 0;
  int max_pver = 0;
  for (int m = 0; m < n_members; ++m) {
    const conv_member& mb = members[m];
    RunArgs& a = h[m];
    conv_status st = common_in(&mb.grid, &mb.in, mb.dt, a);
    if (st != CONV_OK) return st;
    if (!deep_params_ok(&mb.deep) || !shallow_params_ok(&mb.shallow) || !out_ok(&mb.deep_out) ||
        !out_ok(&mb.shallow_out))
      return CONV_ERR_ARG;
    a.dp = mb.deep;
    a.sp = mb.shallow;
    a.od = to_outp(&mb.deep_out);
    a.os = to_outp(&mb.shallow_out);
    if (has_flux(a.od) || has_flux(a.os) || mb.shallow.evap_k > 0.0 || mb.deep.n_plumes > 1)
      return CONV_ERR_UNSUPPORTED;
    a.mode = cvg::MODE_DEEP | cvg::MODE_SHALLOW;
    a.stream = nullptr;
    cvg::fill_q(a);
    off[m] = (int)total;
    total += a.n;
    if (a.L.pver > max_pver) max_pver = a.L.pver;
  }
  if (total >= (1ll << 31)) return CONV_ERR_ARG;
  off[n_members] = (int)total;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CONV_ERR_CUDA;
  conv_batch* b = new conv_batch();
  b->prec = prec;
  b->n_members = n_members;
  b->total = (int)total;
  b->sms = sms;
  b->h_offsets = off;
  b->d_members = nullptr;
  b->d_offsets = nullptr;
  if (cudaMalloc(&b->d_members, sizeof(RunArgs) * n_members) != cudaSuccess ||
      cudaMalloc(&b->d_offsets, sizeof(int) * (n_members + 1)) != cudaSuccess ||
      cudaMemcpy(b->d_members, h.data(), sizeof(RunArgs) * n_members, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(b->d_offsets, off.data(), sizeof(int) * (n_members + 1),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    conv_batch_free(b);
    return CONV_ERR_CUDA;
  }
  const bool fp64 = prec == CONV_FP64;
  b->shape = default_shape(fp64, max_pver, sms);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto lb = g_last_bucket.find({(int)prec, max_pver});
    if (lb != g_last_bucket.end()) {
      auto it = g_tune_cache.find(std::make_tuple((int)prec, max_pver, lb->second));
      if (it != g_tune_cache.end()) b->shape = it->second;
    }
  }
  *out = b;
  return CONV_OK;
}

size_t conv_batch_workspace_bytes(const conv_batch* b) {
  if (!b) return 0;
  return cvg::ws_offsets(b->total, b->shape.max_pver, b->prec == CONV_FP64 ? 8 : 4).total;
}

conv_status conv_batch_run(const conv_batch* b, void* ws, size_t ws_bytes, conv_stream stream,
                           void* const* stage_events) {
  if (!b) return CONV_ERR_ARG;
  const size_t need = conv_batch_workspace_bytes(b);
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
    return CONV_ERR_WORKSPACE;
  cvg::BatchDev d{b->d_members, b->d_offsets, b->n_members, b->total};
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (stage_events)
    for (int i = 0; i < 3; ++i) ev[i] = static_cast<cudaEvent_t>(stage_events[i]);
  const cudaError_t e = cvg::launch_batch(d, b->shape, b->prec == CONV_FP64, ws, ws_bytes,
                                          reinterpret_cast<cudaStream_t>(stream), ev);
  return e == cudaSuccess ? CONV_OK : CONV_ERR_CUDA;
}

conv_status conv_batch_autotune(conv_batch* b, void* ws, size_t ws_bytes, conv_stream stream,
                                int reps) {
  if (!b || reps < 1) return CONV_ERR_ARG;
  const size_t need = conv_batch_workspace_bytes(b);
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
    return CONV_ERR_WORKSPACE;
  const bool fp64 = b->prec == CONV_FP64;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return CONV_ERR_CUDA;
  }
  cvg::BatchDev d{b->d_members, b->d_offsets, b->n_members, b->total};
  auto time_shape = [&](const cvg::BatchShape& sh, float* ms) -> cudaError_t {
    cudaError_t err = cvg::launch_batch(d, sh, fp64, ws, ws_bytes, s, nullptr);  // warm-up
    if (err != cudaSuccess) return err;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && err == cudaSuccess; ++r)
      err = cvg::launch_batch(d, sh, fp64, ws, ws_bytes, s, nullptr);
    cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
    return err;
  };
  static const int kBlocks[3] = {64, 128, 256};
  cvg::BatchShape best = b->shape;
  float best_ms = 1e30f;
  cudaError_t err = cudaSuccess;
  float rec[7] = {0.f};
  for (int j = 0; j < 4 && err == cudaSuccess; ++j) {  // trigger: 3 block sizes, warp mapping
    cvg::BatchShape sh = best;
    sh.trigger_mapping = j == 3 ? 1 : 0;
    if (j < 3) sh.trigger_block = kBlocks[j];
    float ms = 0.f;
    err = time_shape(sh, &ms);
    if (err != cudaSuccess) break;
    rec[j] = ms / reps;
    if (ms < best_ms) { best_ms = ms; best = sh; }
  }
  for (int j = 0; j < 3 && err == cudaSuccess; ++j) {
    const int pb = kBlocks[j];
    cvg::BatchShape sh = best;
    sh.plume_block = pb;
    sh.plume_grid = b->sms * cvg::batch_plume_occupancy(fp64, pb, best.max_pver);
    float ms = 0.f;
    err = time_shape(sh, &ms);
    if (err != cudaSuccess) break;
    rec[4 + j] = ms / reps;
    if (ms < best_ms) { best_ms = ms; best = sh; }
  }
  int count = 0;
  if (err == cudaSuccess) {  // active fraction of this batch: the queue length
    const cvg::WsOffsets off = cvg::ws_offsets(b->total, b->shape.max_pver, fp64 ? 8 : 4);
    err = cudaMemcpy(&count, static_cast<char*>(ws) + off.count, sizeof(int),
                     cudaMemcpyDeviceToHost);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return CONV_ERR_CUDA;
  b->shape = best;
  for (int j = 0; j < 7; ++j) b->tune_ms[j] = rec[j];
  b->tuned = true;
  const int bucket = b->total > 0 ? (int)(10.0 * count / b->total) : 0;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[std::make_tuple((int)b->prec, best.max_pver, bucket)] = best;
  g_last_bucket[{(int)b->prec, best.max_pver}] = bucket;
  return CONV_OK;
}

conv_status conv_batch_set_config(conv_batch* b, int32_t trigger_mapping, int32_t trigger_block,
                                  int32_t plume_block) {
  auto ok_block = [](int32_t x) { return x == 64 || x == 128 || x == 256; };
  if (!b || (trigger_mapping != CONV_MAP_THREAD && trigger_mapping != CONV_MAP_WARP) ||
      !ok_block(trigger_block) || !ok_block(plume_block))
    return CONV_ERR_ARG;
  const bool fp64 = b->prec == CONV_FP64;
  b->shape.trigger_mapping = trigger_mapping == CONV_MAP_WARP ? 1 : 0;
  b->shape.trigger_block = trigger_block;
  b->shape.plume_block = plume_block;
  b->shape.plume_grid = b->sms * cvg::batch_plume_occupancy(fp64, plume_block, b->shape.max_pver);
  return CONV_OK;
}

conv_status conv_batch_tune_record(const conv_batch* b, float* ms) {
  if (!b || !ms || !b->tuned) return CONV_ERR_ARG;
  for (int j = 0; j < 7; ++j) ms[j] = b->tune_ms[j];
  return CONV_OK;
}

conv_status conv_batch_config(const conv_batch* b, int32_t* trigger_block, int32_t* plume_block,
                              int32_t* plume_grid, int32_t* trigger_mapping) {
  if (!b) return CONV_ERR_ARG;
  if (trigger_mapping) *trigger_mapping = b->shape.trigger_mapping ? CONV_MAP_WARP : CONV_MAP_THREAD;
  if (trigger_block) *trigger_block = b->shape.trigger_block;
  if (plume_block) *plume_block = b->shape.plume_block;
  if (plume_grid) *plume_grid = b->shape.plume_grid;
  return CONV_OK;
}

void conv_batch_free(conv_batch* b) {
  if (!b) return;
  if (b->d_members) cudaFree(b->d_members);
  if (b->d_offsets) cudaFree(b->d_offsets);
  delete b;
}

}  // extern "C"
