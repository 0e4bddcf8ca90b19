// launch.h -- internal interface between the C ABI (conv_api.cu) and the kernel
// translation units.  Not installed; the public interface is include/conv.h.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "column.cuh"

namespace cvg {

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
  OutP od, os;
  int mode;
  int block;
  cudaStream_t stream;
  cudaEvent_t ev[3];  // optional stage events (nullptr = none)
};

inline void record_stage(const RunArgs& a, int i) {
  if (a.ev[i]) cudaEventRecord(a.ev[i], a.stream);
}

// Plain path: one thread per column, whole scheme, no compaction.
cudaError_t launch_plain(const RunArgs& a, bool fp64);

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

}  // namespace cvg
