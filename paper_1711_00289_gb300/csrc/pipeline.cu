// pipeline.cu -- conv_pipeline_*: the fused deep -> shallow run on HOST buffers,
// in column chunks whose host-to-device copies, kernels and device-to-host
// copies run on three streams, so chunk j+1 copies in while chunk j computes and
// chunk j-1 copies out (the Grace-Blackwell host link carries both directions
// at once).  The plan owns the device staging slots, streams and events; runs
// allocate nothing.
#include <cmath>
#include <cstring>
#include <vector>

#include "compact.h"
#include "validate.h"

namespace {

constexpr int kSlots = 3;

struct Slot {
  void* mem = nullptr;
  void *T = nullptr, *q = nullptr;
  double *ps = nullptr, *lam = nullptr, *tau = nullptr;
  conv_out od{}, os{};
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaEvent_t in_done = nullptr, comp_done = nullptr, out_done = nullptr;
  bool used = false;
};

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct conv_pipeline {
  conv_grid grid;  // n_cols, ld of the host arrays; hyai/hybi point into a/b
  std::vector<double> a, b;
  conv_precision prec;
  int chunk;  // columns per chunk (= device leading dimension of a slot)
  size_t es;  // bytes per profile element
  cudaStream_t sh = nullptr, sc = nullptr, sd = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  Slot slot[kSlots];
};

namespace {

void destroy(conv_pipeline* p) {
  for (Slot& s : p->slot) {
    if (s.in_done) cudaEventDestroy(s.in_done);
    if (s.comp_done) cudaEventDestroy(s.comp_done);
    if (s.out_done) cudaEventDestroy(s.out_done);
    if (s.mem) cudaFree(s.mem);
  }
  if (p->start) cudaEventDestroy(p->start);
  if (p->done) cudaEventDestroy(p->done);
  if (p->sh) cudaStreamDestroy(p->sh);
  if (p->sc) cudaStreamDestroy(p->sc);
  if (p->sd) cudaStreamDestroy(p->sd);
  delete p;
}

// Device layout of one slot: T, q [pver][chunk]; ps, lam, tau [chunk]; for each
// scheme dTdt, dqdt [pver][chunk], prec, cape, mb, cons_err [chunk] (double),
// flags, kb, klcl, ktop, kaux [chunk] (int32); the compacted path's workspace.
size_t carve(Slot& s, char* base, int pver, int chunk, size_t es, size_t ws_bytes) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* ptr = base ? base + off : nullptr;
    off += up256(bytes);
    return static_cast<void*>(ptr);
  };
  const size_t prof = (size_t)pver * chunk * es, col8 = (size_t)chunk * 8, col4 = (size_t)chunk * 4;
  s.T = take(prof);
  s.q = take(prof);
  s.ps = static_cast<double*>(take(col8));
  s.lam = static_cast<double*>(take(col8));
  s.tau = static_cast<double*>(take(col8));
  for (conv_out* o : {&s.od, &s.os}) {
    o->dTdt = take(prof);
    o->dqdt = take(prof);
    o->prec = static_cast<double*>(take(col8));
    o->cape = static_cast<double*>(take(col8));
    o->mb = static_cast<double*>(take(col8));
    o->cons_err = static_cast<double*>(take(col8));
    o->flags = static_cast<int32_t*>(take(col4));
    o->kb = static_cast<int32_t*>(take(col4));
    o->klcl = static_cast<int32_t*>(take(col4));
    o->ktop = static_cast<int32_t*>(take(col4));
    o->kaux = static_cast<int32_t*>(take(col4));
  }
  s.ws = take(ws_bytes);
  s.ws_bytes = ws_bytes;
  return off;
}

// Columns [c0, c0+cols) of a host [pver][ld] array <-> a slot's [pver][chunk].
cudaError_t copy_prof(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width,
                      int pver, cudaMemcpyKind kind, cudaStream_t s) {
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, (size_t)pver, kind, s);
}

}  // namespace

extern "C" {

conv_status conv_pipeline_plan(const conv_grid* grid, conv_precision prec, int chunk_cols,
                               conv_pipeline** out) {
  if (!out) return CONV_ERR_ARG;
  *out = nullptr;
  if (!cvg::grid_ok(grid) || grid->n_cols < 1) return CONV_ERR_ARG;
  if (prec != CONV_FP64 && prec != CONV_MIXED) return CONV_ERR_ARG;
  if (chunk_cols < 1) return CONV_ERR_ARG;
  conv_pipeline* p = new conv_pipeline();
  p->grid = *grid;
  p->a.assign(grid->hyai, grid->hyai + grid->pver + 1);
  p->b.assign(grid->hybi, grid->hybi + grid->pver + 1);
  p->grid.hyai = p->a.data();
  p->grid.hybi = p->b.data();
  p->prec = prec;
  p->chunk = chunk_cols < grid->n_cols ? chunk_cols : grid->n_cols;
  p->es = prec == CONV_FP64 ? 8 : 4;
  conv_grid cg = p->grid;
  cg.n_cols = cg.ld = p->chunk;
  const size_t ws = conv_workspace_bytes(&cg, prec, nullptr);
  Slot probe;
  const size_t bytes = carve(probe, nullptr, grid->pver, p->chunk, p->es, ws);
  bool ok = cudaStreamCreateWithFlags(&p->sh, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&p->sc, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&p->sd, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) == cudaSuccess;
  for (Slot& s : p->slot) {
    if (!ok) break;
    ok = cudaMalloc(&s.mem, bytes) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.comp_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming) == cudaSuccess;
    if (ok) carve(s, static_cast<char*>(s.mem), grid->pver, p->chunk, p->es, ws);
  }
  if (!ok) {
    destroy(p);
    return CONV_ERR_CUDA;
  }
  *out = p;
  return CONV_OK;
}

conv_status conv_pipeline_run(conv_pipeline* p, const conv_in* host_in,
                              const conv_deep_params* dpar, const conv_shallow_params* spar,
                              double dt, const conv_out* host_deep, const conv_out* host_shallow,
                              conv_stream stream) {
  // Everything a chunk's run would refuse is refused here, before the first copy
  // is enqueued: an error return never leaves copies of the caller's buffers in
  // flight.
  if (!p || !host_in || !host_in->T || !host_in->q || !host_in->ps || !host_deep ||
      !host_shallow || !host_deep->dTdt || !host_deep->dqdt || !host_deep->prec ||
      !host_deep->flags || !host_shallow->dTdt || !host_shallow->dqdt || !host_shallow->prec ||
      !host_shallow->flags || !cvg::deep_params_ok(dpar) || !cvg::shallow_params_ok(spar) ||
      !(std::isfinite(dt) && dt > 0.0))
    return CONV_ERR_ARG;
  for (const conv_out* h : {host_deep, host_shallow})
    if (h->mu || h->du || h->md) return CONV_ERR_UNSUPPORTED;
  const int n = p->grid.n_cols, pver = p->grid.pver, ch = p->chunk;
  const size_t es = p->es, hp = (size_t)p->grid.ld * es, dp = (size_t)ch * es;
  const cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
#define CK(x)                                 \
  do {                                        \
    if ((x) != cudaSuccess) return CONV_ERR_CUDA; \
  } while (0)
  CK(cudaEventRecord(p->start, user));
  // The slots are reused from the first chunk on: copies in wait for the
  // previous run's last copy out even when that run went through another user
  // stream (before any run, `done` has never been recorded and this is a no-op).
  CK(cudaStreamWaitEvent(p->sh, p->done, 0));
  CK(cudaStreamWaitEvent(p->sh, p->start, 0));
  CK(cudaStreamWaitEvent(p->sc, p->start, 0));
  CK(cudaStreamWaitEvent(p->sd, p->start, 0));
  for (Slot& s : p->slot) s.used = false;
  for (int j = 0, c0 = 0; c0 < n; ++j, c0 += ch) {
    Slot& s = p->slot[j % kSlots];
    const int cols = n - c0 < ch ? n - c0 : ch;
    const size_t w = (size_t)cols * es;
    const char* hT = static_cast<const char*>(host_in->T) + (size_t)c0 * es;
    const char* hq = static_cast<const char*>(host_in->q) + (size_t)c0 * es;
    // copy in (once the slot's previous chunk has been copied out)
    if (s.used) CK(cudaStreamWaitEvent(p->sh, s.out_done, 0));
    CK(copy_prof(s.T, dp, hT, hp, w, pver, cudaMemcpyHostToDevice, p->sh));
    CK(copy_prof(s.q, dp, hq, hp, w, pver, cudaMemcpyHostToDevice, p->sh));
    CK(cudaMemcpyAsync(s.ps, host_in->ps + c0, (size_t)cols * 8, cudaMemcpyHostToDevice, p->sh));
    if (host_in->lambda)
      CK(cudaMemcpyAsync(s.lam, host_in->lambda + c0, (size_t)cols * 8, cudaMemcpyHostToDevice,
                         p->sh));
    if (host_in->tau)
      CK(cudaMemcpyAsync(s.tau, host_in->tau + c0, (size_t)cols * 8, cudaMemcpyHostToDevice,
                         p->sh));
    CK(cudaEventRecord(s.in_done, p->sh));
    // compute
    CK(cudaStreamWaitEvent(p->sc, s.in_done, 0));
    conv_grid cg = p->grid;
    cg.n_cols = cols;
    cg.ld = ch;
    const conv_in din = {s.T, s.q, s.ps, host_in->lambda ? s.lam : nullptr,
                         host_in->tau ? s.tau : nullptr};
    const conv_status st = conv_deep_shallow_run(&cg, &din, dpar, spar, dt, p->prec, &s.od, &s.os,
                                                 nullptr, s.ws, s.ws_bytes,
                                                 reinterpret_cast<conv_stream>(p->sc));
    if (st != CONV_OK) return st;
    CK(cudaEventRecord(s.comp_done, p->sc));
    // copy out
    CK(cudaStreamWaitEvent(p->sd, s.comp_done, 0));
    const conv_out* hos[2] = {host_deep, host_shallow};
    const conv_out* dos[2] = {&s.od, &s.os};
    for (int m = 0; m < 2; ++m) {
      const conv_out& h = *hos[m];
      const conv_out& d = *dos[m];
      CK(copy_prof(static_cast<char*>(h.dTdt) + (size_t)c0 * es, hp, d.dTdt, dp, w, pver,
                   cudaMemcpyDeviceToHost, p->sd));
      CK(copy_prof(static_cast<char*>(h.dqdt) + (size_t)c0 * es, hp, d.dqdt, dp, w, pver,
                   cudaMemcpyDeviceToHost, p->sd));
      double* const hd[4] = {h.prec, h.cape, h.mb, h.cons_err};
      const double* const dd[4] = {d.prec, d.cape, d.mb, d.cons_err};
      for (int v = 0; v < 4; ++v)
        if (hd[v])
          CK(cudaMemcpyAsync(hd[v] + c0, dd[v], (size_t)cols * 8, cudaMemcpyDeviceToHost, p->sd));
      int32_t* const hi[5] = {h.flags, h.kb, h.klcl, h.ktop, h.kaux};
      const int32_t* const di[5] = {d.flags, d.kb, d.klcl, d.ktop, d.kaux};
      for (int v = 0; v < 5; ++v)
        if (hi[v])
          CK(cudaMemcpyAsync(hi[v] + c0, di[v], (size_t)cols * 4, cudaMemcpyDeviceToHost, p->sd));
    }
    CK(cudaEventRecord(s.out_done, p->sd));
    s.used = true;
  }
  CK(cudaEventRecord(p->done, p->sd));
  CK(cudaStreamWaitEvent(user, p->done, 0));
#undef CK
  return CONV_OK;
}

void conv_pipeline_free(conv_pipeline* p) {
  if (p) destroy(p);
}

}  // extern "C"
