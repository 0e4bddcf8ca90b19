// conv_api.cu -- the extern "C" entry points of include/conv.h: argument
// validation on the host, packing of kernel parameters, dispatch to a kernel
// path.  Nothing here allocates or synchronises.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "compact.h"

namespace {

using cvg::RunArgs;

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

bool deep_params_ok(const conv_deep_params* p) {
  return p && finite_pos(p->capelmt + 1.0) && p->capelmt >= 0.0 && p->lambda_default >= 0.0 &&
         std::isfinite(p->lambda_default) && finite_pos(p->tau_default) && p->c0 >= 0.0 &&
         std::isfinite(p->c0) && p->alpha_dd >= 0.0 && p->alpha_dd <= 1.0 &&
         finite_pos(p->p_launch_min) && finite_pos(p->p_top_lim) && p->q_min >= 0.0 &&
         p->q_min < 1e-3 && finite_pos(p->ent_zscale) && p->n_newton_lcl >= 1 &&
         p->n_newton_lcl <= 32 && p->n_newton_h >= 0 && p->n_newton_h <= 32;
}

bool shallow_params_ok(const conv_shallow_params* p) {
  return p && p->eps_s >= 0.0 && std::isfinite(p->eps_s) && finite_pos(p->tke) && p->c_m >= 0.0 &&
         std::isfinite(p->c_m) && finite_pos(p->cin_scale) && p->cin_max >= 0.0 &&
         std::isfinite(p->a_w) && p->b_w >= 0.0 && std::isfinite(p->b_w) && p->ql_crit >= 0.0 &&
         finite_pos(p->p_lcl_min) && finite_pos(p->p_lfc_min) && finite_pos(p->p_top_lim) &&
         p->n_newton_lcl >= 1 && p->n_newton_lcl <= 32 && p->n_newton_h >= 0 &&
         p->n_newton_h <= 32;
}

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
  for (int i = 0; i < g->pver; ++i) {  // interfaces must be ordered top -> surface
    if (!std::isfinite(g->hyai[i]) || !std::isfinite(g->hybi[i])) return CONV_ERR_ARG;
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
  return p;
}

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
  if (prec != CONV_FP64 && prec != CONV_MIXED) return CONV_ERR_ARG;
  if (launch && (launch->path < CONV_PATH_AUTO || launch->path > CONV_PATH_COMPACT))
    return CONV_ERR_ARG;
  if (launch && (launch->block_threads < 0 || launch->block_threads > 1024)) return CONV_ERR_ARG;
  const int path = pick_path(launch, a.mode);
  a.block = launch ? launch->block_threads : 0;
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
  p->n_newton_h = 4;
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
  p->n_newton_h = 4;
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

}  // extern "C"
