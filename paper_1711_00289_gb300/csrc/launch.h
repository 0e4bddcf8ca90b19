// launch.h -- internal interface between the C ABI (conv_api.cu) and the kernel
// translation units.  Not installed; the public interface is include/conv.h.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>

#include "column.cuh"

namespace cvg {

// A named NVTX range around the host-side enqueue of one pass (what Nsight
// Systems shows beside the kernels; without a tool attached the calls return
// at once).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

enum : int { MODE_DEEP = 1, MODE_SHALLOW = 2 };

struct OutP {
  void* dTdt;
  void* dqdt;
  double* prec;
  int32_t* flags;
  int32_t* kb;
  int32_t* klcl;
  int32_t* ktop;
  int32_t* kaux;
  double* cape;
  double* mb;
  double* cons_err;
  void* mu;  // mass-flux profiles (optional; extended instantiations only)
  void* du;
  void* md;
};

struct RunArgs {
  Levels L;
  int n, ld;
  const void* T;
  const void* q;
  const double* ps;
  const double* lam;
  const double* tau;
  conv_deep_params dp;
  conv_shallow_params sp;
  double dt;
  // working-precision copies (fill_q, on the host)
  DeepQ<float> dqf;
  DeepQ<double> dqd;
  ShalQ<float> sqf;
  ShalQ<double> sqd;
  OutP od, os;
  bool ext;  // profile outputs or a scheme variant requested: the extended instantiations
  int mode;
  int block;
  int mapping;  // conv_mapping of the compacted trigger pass
  cudaStream_t stream;
  cudaEvent_t ev[3];  // optional stage events (nullptr = none)
};

// Fill the working-precision parameter copies from dp, sp and dt (host).
inline void fill_q(RunArgs& a) {
  a.dqf = make_deep_q<float>(a.dp, a.dt);
  a.dqd = make_deep_q<double>(a.dp, a.dt);
  a.sqf = make_shal_q<float>(a.sp);
  a.sqd = make_shal_q<double>(a.sp);
}
__device__ __forceinline__ const DeepQ<float>& deep_q(const RunArgs& a, float) { return a.dqf; }
__device__ __forceinline__ const DeepQ<double>& deep_q(const RunArgs& a, double) { return a.dqd; }
__device__ __forceinline__ const ShalQ<float>& shal_q(const RunArgs& a, float) { return a.sqf; }
__device__ __forceinline__ const ShalQ<double>& shal_q(const RunArgs& a, double) {
  return a.sqd;
}

inline void record_stage(const RunArgs& a, int i) {
  if (a.ev[i]) cudaEventRecord(a.ev[i], a.stream);
}

// Column i of a run's input profile (no update).
template <class R>
__device__ __forceinline__ Src<R> input_src(const RunArgs& a, int i) {
  return Src<R>{static_cast<const R*>(a.T), static_cast<const R*>(a.q), nullptr, nullptr, R(0),
                (size_t)a.ld, i, false};
}
// The same column advanced by dt times the deep tendencies written to od (the
// shallow scheme's input, Alg. 1); q floored at 0 unless the column was rejected.
template <class R>
__device__ __forceinline__ Src<R> after_deep_src(const RunArgs& a, int i, bool bad) {
  return Src<R>{static_cast<const R*>(a.T), static_cast<const R*>(a.q),
                static_cast<const R*>(a.od.dTdt), static_cast<const R*>(a.od.dqdt), (R)a.dt,
                (size_t)a.ld, i, !bad};
}
template <class R, bool F>
struct OutSel {
  using type = OutCol<R>;
};
template <class R>
struct OutSel<R, true> {
  using type = FluxCol<R>;
};
template <class R, bool F = false>
__device__ __forceinline__ typename OutSel<R, F>::type out_col(const OutP& o, const RunArgs& a,
                                                               int i) {
  if constexpr (F)
    return FluxCol<R>{static_cast<R*>(o.dTdt), static_cast<R*>(o.dqdt), (size_t)a.ld, i,
                      static_cast<R*>(o.mu), static_cast<R*>(o.du), static_cast<R*>(o.md)};
  else
    return OutCol<R>{static_cast<R*>(o.dTdt), static_cast<R*>(o.dqdt), (size_t)a.ld, i};
}

__device__ __forceinline__ void store_deep_scalars(const RunArgs& a, int i, const DeepOut& o) {
  a.od.prec[i] = o.prec;
  a.od.flags[i] = o.flags;
  if (a.od.kb) a.od.kb[i] = o.kb;
  if (a.od.klcl) a.od.klcl[i] = o.klcl;
  if (a.od.ktop) a.od.ktop[i] = o.ktop;
  if (a.od.kaux) a.od.kaux[i] = o.kaux;
  if (a.od.cape) a.od.cape[i] = o.cape;
  if (a.od.mb) a.od.mb[i] = o.mb;
  if (a.od.cons_err) a.od.cons_err[i] = o.cons;
}

__device__ __forceinline__ void store_shallow_scalars(const RunArgs& a, int i, const ShalOut& o) {
  const bool bad = (o.flags & CONV_FLAG_BADINPUT) != 0;
  a.os.prec[i] = o.prec;
  a.os.flags[i] = o.flags;
  if (a.os.kb) a.os.kb[i] = bad ? -1 : a.L.pver - 1;
  if (a.os.klcl) a.os.klcl[i] = o.klcl;
  if (a.os.ktop) a.os.ktop[i] = o.ktop;
  if (a.os.kaux) a.os.kaux[i] = o.klfc;
  if (a.os.cape) a.os.cape[i] = o.cin;
  if (a.os.mb) a.os.mb[i] = o.mb;
  if (a.os.cons_err) a.os.cons_err[i] = o.cons;
}

// Plain path: one thread per column, whole scheme, no compaction.
cudaError_t launch_plain(const RunArgs& a, bool fp64);

// Tracer transport (transport.cu): one scheme's plume as a tracer sees it.
struct TrScheme {
  const void* mu;
  const void* du;
  const void* md;  // deep downdraft (nullptr: none)
  const int32_t* flags;
  const int32_t* kb;
  const int32_t* ktop;
  const int32_t* kaux;
  void* tend;
};
struct TrArgs {
  Levels L;
  int n, ld, pver, ntr;
  size_t tstride;  // pver * ld: offset between tracers
  const double* ps;
  const void* tr;
  double dt;
  TrScheme d, s;
  bool has_d, has_s;
  bool mom;               // momentum transport: ntr = 2 (u, v), pressure-gradient terms
  double cp_up, cp_down;  // their coefficients (updrafts, downdraft)
  cudaStream_t stream;
};
cudaError_t launch_transport(const TrArgs& a, bool fp64);

// Heating weights of the adjoint's objective, passed by value in the launch.
struct AdjW {
  double w[MAXL];
  bool given;  // false: w_k = p_mid_k / ps
};
// Deep-scheme adjoint (FP64): one thread per column.  gT == nullptr: no
// reverse sweep (gq, glam, gtau unused); Pout, Hout may be nullptr.
cudaError_t launch_deep_adjoint(const RunArgs& a, const double* gP, const double* gH,
                                const AdjW& w, double* gT, double* gq, double* glam,
                                double* gtau, double* Pout, double* Hout);
// State advance of the multi-step driver (in place on T, q).
cudaError_t launch_advance(const RunArgs& a, bool fp64, void* T, void* q, const void* Tr,
                           const void* qr, double tau);

// Fused deep -> shallow step adjoint (FP64): one thread per column.  gT, gq are
// also the scratch of the deep tendencies (always written); obj may be nullptr.
cudaError_t launch_step_adjoint(const RunArgs& a, const double* const g[4], const AdjW& w,
                                double* gT, double* gq, double* glam, double* gtau, double* obj,
                                bool rev);

}  // namespace cvg
