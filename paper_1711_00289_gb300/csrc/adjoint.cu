// adjoint.cu -- kernel and launch of the deep-scheme adjoint (FP64): one
// thread per column loads its profiles, runs deep_adjoint_column (adjoint.cuh)
// and stores dJ/dT, dJ/dq, dJ/dlambda, dJ/dtau and/or the objective pieces P, H.
#include "adjoint.cuh"
#include "launch.h"

namespace cvg {

struct AdjArgs {
  RunArgs a;
  const double* gP;
  const double* gH;
  AdjW w;
  double* gT;
  double* gq;
  double* glam;
  double* gtau;
  double* Pout;
  double* Hout;
};

__global__ void __launch_bounds__(64) k_deep_adjoint(const __grid_constant__ AdjArgs A) {
  const RunArgs& a = A.a;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int pver = a.L.pver, ld = a.ld;
  Column<double> c;
  LevelBuf<double> cbuf;
  init_column(c, a.L, input_src<double>(a, i), a.ps[i], cbuf);
  const double lam = a.lam ? a.lam[i] : a.dp.lambda_default;
  const double tau = a.tau ? a.tau[i] : a.dp.tau_default;
  const double gP = A.gP ? A.gP[i] : 0.0, gH = A.gH ? A.gH[i] : 0.0;
  const bool rev = A.gT != nullptr;
  double bT[MAXL], bq[MAXL], blam, btau, Pv, Hv;
  deep_adjoint_column(a.dp, a.dqd, lam, tau, c, gP, gH, A.w.given ? A.w.w : nullptr, rev, bT,
                      bq, blam, btau, Pv, Hv);
  if (rev) {
    for (int k = 0; k < pver; ++k) {
      A.gT[(size_t)k * ld + i] = bT[k];
      A.gq[(size_t)k * ld + i] = bq[k];
    }
    A.glam[i] = blam;
    A.gtau[i] = btau;
  }
  if (A.Pout) A.Pout[i] = Pv;
  if (A.Hout) A.Hout[i] = Hv;
}

struct StepArgs {
  RunArgs a;
  const double* g[4];  // seeds on Pd, Hd, Ps, Hs ([ld] each, nullptr = 0)
  AdjW w;
  double* gT;  // also the scratch for the deep tendencies the shallow scheme reads
  double* gq;
  double* glam;
  double* gtau;
  double* obj;  // [4][ld] or nullptr
  bool rev;
};

__global__ void __launch_bounds__(64) k_step_adjoint(const __grid_constant__ StepArgs A) {
  const RunArgs& a = A.a;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int pver = a.L.pver, ld = a.ld;
  Column<double> c, c2;
  LevelBuf<double> cbuf, cbuf2;
  init_column(c, a.L, input_src<double>(a, i), a.ps[i], cbuf);
  init_column(c2, a.L,
              Src<double>{static_cast<const double*>(a.T), static_cast<const double*>(a.q), A.gT,
                          A.gq, a.dt, (size_t)ld, i, true},
              a.ps[i], cbuf2);
  const double lam = a.lam ? a.lam[i] : a.dp.lambda_default;
  const double tau = a.tau ? a.tau[i] : a.dp.tau_default;
  double g[4];
  for (int j = 0; j < 4; ++j) g[j] = A.g[j] ? A.g[j][i] : 0.0;
  double bT[MAXL], bq[MAXL], blam, btau, obj[4];
  step_adjoint_column(a.dp, a.dqd, a.sp, a.sqd, a.dt, lam, tau, c, c2, A.gT + i, A.gq + i,
                      (size_t)ld, g, A.w.given ? A.w.w : nullptr, A.rev, bT, bq, blam, btau,
                      obj);
  if (A.rev) {
    for (int k = 0; k < pver; ++k) {
      A.gT[(size_t)k * ld + i] = bT[k];
      A.gq[(size_t)k * ld + i] = bq[k];
    }
    A.glam[i] = blam;
    A.gtau[i] = btau;
  }
  if (A.obj)
    for (int j = 0; j < 4; ++j) A.obj[(size_t)j * ld + i] = obj[j];
}

cudaError_t launch_step_adjoint(const RunArgs& a, const double* const g[4], const AdjW& w,
                                double* gT, double* gq, double* glam, double* gtau, double* obj,
                                bool rev) {
  if (a.n == 0) return cudaSuccess;
  NvtxRange r("conv: fused-step adjoint");
  StepArgs A{a, {g[0], g[1], g[2], g[3]}, w, gT, gq, glam, gtau, obj, rev};
  const int block = 64;
  k_step_adjoint<<<(a.n + block - 1) / block, block, 0, a.stream>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_deep_adjoint(const RunArgs& a, const double* gP, const double* gH,
                                const AdjW& w, double* gT, double* gq, double* glam,
                                double* gtau, double* Pout, double* Hout) {
  if (a.n == 0) return cudaSuccess;
  NvtxRange r("conv: deep adjoint");
  AdjArgs A{a, gP, gH, w, gT, gq, glam, gtau, Pout, Hout};
  const int block = 64;
  k_deep_adjoint<<<(a.n + block - 1) / block, block, 0, a.stream>>>(A);
  return cudaGetLastError();
}

}  // namespace cvg
