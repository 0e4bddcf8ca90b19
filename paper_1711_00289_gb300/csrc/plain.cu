// plain.cu -- the baseline kernel: one thread per column runs deep convection
// and then shallow convection on the deep-updated state (Alg. 1 order).  No
// compaction: a warp whose columns do not convect still pays for the ones that
// do, exactly the load imbalance the paper reports for its OpenMP loops
// (Sec. IV-A).
#include "launch.h"

namespace cvg {

// Resident threads per SM the plain kernel is compiled for: the FP64 kernel,
// bound by the FP64 pipe, needs enough warps in flight to keep that pipe fed
// (7 blocks of 128: at most 72 registers).
template <class R>
struct PlainThreads {
  static constexpr int sm = 896;
};
template <>
struct PlainThreads<float> {
  static constexpr int sm = 1024;
};

// EXT: the extended instantiation (mass-flux profile outputs, scheme variants),
// launched only for runs that ask for them.
template <class R, bool EXT>
__global__ void __launch_bounds__(128, PlainThreads<R>::sm / 128)
    k_plain(const __grid_constant__ RunArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  Column<R> c;
  LevelBuf<R> cbuf;
  init_column(c, a.L, input_src<R>(a, i), a.ps[i], cbuf);
  DeepBound bound;
  bool bound_ok = false;
  if (a.mode & MODE_DEEP) {
    DeepOut o;
    const DeepQ<R>& Q = deep_q(a, R(0));
    const R lam = a.lam ? (R)a.lam[i] : Q.lambda_default;
    const R tau = a.tau ? (R)a.tau[i] : Q.tau_default;
    deep_column(a.dp, Q, lam, tau, c, o, out_col<R, EXT>(a.od, a, i), &bound, &bound_ok);
    store_deep_scalars(a, i, o);
    // the limiter keeps q >= q_min up to rounding; a rejected column passes
    // unchanged.  A column that did not trigger has zero tendencies: the shallow
    // scheme sees the state the deep trigger saw.
    if (a.mode & MODE_SHALLOW)
      c.s = after_deep_src<R>(a, i, (o.flags & CONV_FLAG_BADINPUT) != 0);
  }
  if (a.mode & MODE_SHALLOW) {
    ShalOut o;
    shallow_column(a.sp, shal_q(a, R(0)), c, o, out_col<R, EXT>(a.os, a, i),
                   (const ShallowSeed<R>*)nullptr, false,
                   bound_ok ? &bound : nullptr);
    store_shallow_scalars(a, i, o);
  }
}

cudaError_t launch_plain(const RunArgs& a, bool fp64) {
  if (a.n == 0) return cudaSuccess;
  const int block = 128;
  const int grid = (a.n + block - 1) / block;
  record_stage(a, 0);
  NvtxRange r("conv: plain pass (whole scheme per column)");
  if (fp64) {
    if (a.ext)
      k_plain<double, true><<<grid, block, 0, a.stream>>>(a);
    else
      k_plain<double, false><<<grid, block, 0, a.stream>>>(a);
  } else {
    if (a.ext)
      k_plain<float, true><<<grid, block, 0, a.stream>>>(a);
    else
      k_plain<float, false><<<grid, block, 0, a.stream>>>(a);
  }
  const cudaError_t e = cudaGetLastError();
  record_stage(a, 1);
  record_stage(a, 2);
  return e;
}

}  // namespace cvg
