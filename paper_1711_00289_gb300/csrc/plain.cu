// plain.cu -- the baseline kernel: one thread per column runs deep convection
// and then shallow convection on the deep-updated state (Alg. 1 order), with the
// column profile held in per-thread arrays.  No compaction: a warp whose columns
// do not convect still pays for the ones that do, exactly the load imbalance the
// paper reports for its OpenMP loops (Sec. III-A).
#include "launch.h"

namespace cvg {

template <class R>
__device__ __forceinline__ R add_mul(R a, double dt, R b);
template <>
__device__ __forceinline__ double add_mul<double>(double a, double dt, double b) {
  return __dadd_rn(a, __dmul_rn(dt, b));  // T + dt*dTdt without contraction
}
template <>
__device__ __forceinline__ float add_mul<float>(float a, double dt, float b) {
  return a + (float)dt * b;
}

template <class R>
__global__ void __launch_bounds__(128) k_plain(RunArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int ld = a.ld, pver = a.L.pver;
  const R* __restrict__ T = static_cast<const R*>(a.T);
  const R* __restrict__ q = static_cast<const R*>(a.q);
  Column<R> c;
  c.pver = pver;
  c.ps = a.ps[i];
  for (int k = 0; k < pver; ++k) {
    c.T[k] = T[(size_t)k * ld + i];
    c.q[k] = q[(size_t)k * ld + i];
  }
  if (a.mode & MODE_DEEP) {
    DeepOut<R> o;
    const R lam = (R)(a.lam ? a.lam[i] : a.dp.lambda_default);
    const R tau = (R)(a.tau ? a.tau[i] : a.dp.tau_default);
    deep_column(a.L, a.dp, a.dt, lam, tau, c, o);
    R* dT = static_cast<R*>(a.od.dTdt);
    R* dq = static_cast<R*>(a.od.dqdt);
    for (int k = 0; k < pver; ++k) {
      dT[(size_t)k * ld + i] = o.dT[k];
      dq[(size_t)k * ld + i] = o.dq[k];
    }
    a.od.prec[i] = o.prec;
    a.od.flags[i] = o.flags;
    if (a.od.kb) a.od.kb[i] = o.kb;
    if (a.od.klcl) a.od.klcl[i] = o.klcl;
    if (a.od.ktop) a.od.ktop[i] = o.ktop;
    if (a.od.kaux) a.od.kaux[i] = o.kaux;
    if (a.od.cape) a.od.cape[i] = o.cape;
    if (a.od.mb) a.od.mb[i] = o.mb;
    if (a.od.cons_err) a.od.cons_err[i] = o.cons;
    if (a.mode & MODE_SHALLOW) {
      // the limiter keeps q >= q_min up to rounding; a rejected column passes unchanged
      const bool bad = (o.flags & CONV_FLAG_BADINPUT) != 0;
      for (int k = 0; k < pver; ++k) {
        c.T[k] = add_mul(c.T[k], a.dt, o.dT[k]);
        const R qn = add_mul(c.q[k], a.dt, o.dq[k]);
        c.q[k] = (!bad && qn < R(0)) ? R(0) : qn;
      }
    }
  }
  if (a.mode & MODE_SHALLOW) {
    ShalOut<R> o;
    shallow_column(a.L, a.sp, c, o);
    R* dT = static_cast<R*>(a.os.dTdt);
    R* dq = static_cast<R*>(a.os.dqdt);
    for (int k = 0; k < pver; ++k) {
      dT[(size_t)k * ld + i] = o.dT[k];
      dq[(size_t)k * ld + i] = o.dq[k];
    }
    const bool bad = (o.flags & CONV_FLAG_BADINPUT) != 0;
    a.os.prec[i] = o.prec;
    a.os.flags[i] = o.flags;
    if (a.os.kb) a.os.kb[i] = bad ? -1 : pver - 1;
    if (a.os.klcl) a.os.klcl[i] = o.klcl;
    if (a.os.ktop) a.os.ktop[i] = o.ktop;
    if (a.os.kaux) a.os.kaux[i] = o.klfc;
    if (a.os.cape) a.os.cape[i] = o.cin;
    if (a.os.mb) a.os.mb[i] = o.mb;
    if (a.os.cons_err) a.os.cons_err[i] = o.cons;
  }
}

cudaError_t launch_plain(const RunArgs& a, bool fp64) {
  if (a.n == 0) return cudaSuccess;
  const int block = 128;
  const int grid = (a.n + block - 1) / block;
  record_stage(a, 0);
  if (fp64)
    k_plain<double><<<grid, block, 0, a.stream>>>(a);
  else
    k_plain<float><<<grid, block, 0, a.stream>>>(a);
  const cudaError_t e = cudaGetLastError();
  record_stage(a, 1);
  record_stage(a, 2);
  return e;
}

}  // namespace cvg
