// driver.cu -- state advance of the multi-step column driver: apply the deep
// and shallow tendencies of one physics step and a Newtonian relaxation towards
// a reference profile (the single-column stand-in for the rest of the model),
// in place, level-major, one thread per (level, column).
#include "launch.h"

namespace cvg {

template <class R>
struct AdvArgs {
  R* T;
  R* q;
  const R* Tr;
  const R* qr;
  const R* dTd;
  const R* dqd;
  const R* dTs;
  const R* dqs;
  R dt, rtau;  // rtau = 1 / tau_relax (0: no relaxation)
  int n, ld, pver;
};

template <class R>
__global__ void __launch_bounds__(256) k_advance(AdvArgs<R> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (i >= a.n || k >= a.pver) return;
  const size_t o = (size_t)k * a.ld + i;
  const R T = a.T[o], q = a.q[o];
  const R fT = (a.dTd[o] + a.dTs[o]) + (a.Tr[o] - T) * a.rtau;
  const R fq = (a.dqd[o] + a.dqs[o]) + (a.qr[o] - q) * a.rtau;
  a.T[o] = T + a.dt * fT;
  const R qn = q + a.dt * fq;
  a.q[o] = qn < R(0) ? R(0) : qn;
}

template <class R>
static cudaError_t advance_t(const RunArgs& a, void* T, void* q, const void* Tr, const void* qr,
                             double tau) {
  AdvArgs<R> x{static_cast<R*>(T),
               static_cast<R*>(q),
               static_cast<const R*>(Tr),
               static_cast<const R*>(qr),
               static_cast<const R*>(a.od.dTdt),
               static_cast<const R*>(a.od.dqdt),
               static_cast<const R*>(a.os.dTdt),
               static_cast<const R*>(a.os.dqdt),
               (R)a.dt,
               tau > 0.0 ? (R)(1.0 / tau) : R(0),
               a.n,
               a.ld,
               a.L.pver};
  const dim3 grid((a.n + 255) / 256, a.L.pver);
  k_advance<R><<<grid, 256, 0, a.stream>>>(x);
  return cudaGetLastError();
}

cudaError_t launch_advance(const RunArgs& a, bool fp64, void* T, void* q, const void* Tr,
                           const void* qr, double tau) {
  if (a.n == 0) return cudaSuccess;
  return fp64 ? advance_t<double>(a, T, q, Tr, qr, tau) : advance_t<float>(a, T, q, Tr, qr, tau);
}

}  // namespace cvg
