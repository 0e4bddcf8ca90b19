// transport.cu -- convective transport of passive tracers (conv_tracer_transport)
// from the mass-flux profiles a scheme run wrote (mu, du, md).  Each scheme
// mixes a tracer as it mixes its conserved moist static energy, without a
// source term: a variant both schemes the paper cites carry (Sec. II-A), on the
// same column-parallel path.
//
// The work is a few operations per level against one read and one write of the
// tracer per level: HBM-bound.  One thread handles one (column, tracer) pair;
// the grid's x index is the tracer, so the blocks that run one after another
// cover the same columns for successive tracers and re-read that column block's
// profiles, flags and indices from L2 instead of HBM.  Threads of a warp hold
// adjacent columns, so every level access is one coalesced line per warp.  A
// thread reads the tracer only on the levels its column's plumes touch and
// writes every level (zeros elsewhere).
#include "launch.h"

namespace cvg {

namespace {

constexpr int kTrBlock = 128;

// Layer mass (kg m-2) of layer k, with the interface pressures the scheme
// kernels use for the same precision.
template <class R>
__device__ __forceinline__ R layer_mass(const Levels& L, double ps, int k) {
  if constexpr (sizeof(R) == 8) {
    const PressFP64 P{L, ps};
    return (P.pi(k + 1) - P.pi(k)) * (1.0 / GRAV);
  } else {
    const PressFP32 P{L, (float)ps};
    return (P.pi(k + 1) - P.pi(k)) * (float)(1.0 / GRAV);
  }
}

// The tracer a scheme sees at level k: c, or max(c + dt prior, 0) after the
// deep stage's update (prior = the deep tendency this thread just wrote).
template <class R>
struct TrCol {
  const R* c;
  const R* prior;
  R dt;
  size_t ld;
  __device__ __forceinline__ R operator()(int k) const {
    const size_t o = (size_t)k * ld;
    R v = c[o];
    if (prior) {
      v = v + dt * prior[o];
      if (v < R(0)) v = R(0);
    }
    return v;
  }
};

// One scheme's tendency of one tracer column (out at out[k * ld]).
template <class R>
__device__ __forceinline__ void scheme_transport(const TrScheme& S, bool down, const Levels& L,
                                                 double ps, int pver, size_t ld, int i,
                                                 const TrCol<R>& C, R* out) {
  const int kb = S.kb[i], kt = S.ktop[i];
  const bool active = (S.flags[i] & CONV_FLAG_ACTIVE) != 0 && kt >= 0 && kt <= kb && kb < pver;
  if (!active) {
    for (int k = 0; k < pver; ++k) out[(size_t)k * ld] = R(0);
    return;
  }
  const R* mu = static_cast<const R*>(S.mu) + i;
  const R* du = static_cast<const R*>(S.du) + i;
  const R* md = down ? static_cast<const R*>(S.md) + i : nullptr;
  const int jd = down ? S.kaux[i] : -1;
  for (int k = 0; k < kt; ++k) out[(size_t)k * ld] = R(0);
  for (int k = kb + 1; k < pver; ++k) out[(size_t)k * ld] = R(0);
  // downdraft value arriving at the launch layer: mixed from jd down to kb-1,
  // entraining md[k] - md[k-1] at layer k
  R cd = R(0), mdl = R(0);
  const bool dd = md != nullptr && jd >= 0 && jd <= kb - 1;
  if (dd) {
    R mprev = R(0);
    for (int k = jd; k <= kb - 1; ++k) {
      const R mk = md[(size_t)k * ld];
      if (mk > R(0)) cd = cd + Mth<R>::dv(mk - mprev, mk) * (C(k) - cd);
      mprev = mk;
    }
    mdl = mprev;
  }
  // launch layer upwards: tendency of layer k from the updraft value arriving
  // from k+1, then the updraft value leaving k (entraining mu[k] - mu[k+1] +
  // du[k] at layer k)
  R cu = R(0), mu1 = R(0), cbelow = R(0);
  R ck = C(kb);
  for (int k = kb; k >= kt; --k) {
    const size_t o = (size_t)k * ld;
    const R muk = mu[o], duk = du[o];
    const R cup = (k > kt || (muk != R(0) && k > 0)) ? C(k - 1) : R(0);
    R t = muk * (cup - ck) + duk * (cu - ck);
    if (dd) {
      if (k >= jd && k <= kb - 1) t += md[o] * (cbelow - ck);
      if (k == kb) t += mdl * (cd - ck);
    }
    out[o] = Mth<R>::dv(t, layer_mass<R>(L, ps, k));
    cu = muk > R(0) ? cu + Mth<R>::dv(muk - mu1 + duk, muk) * (ck - cu) : R(0);
    mu1 = muk;
    cbelow = ck;
    ck = cup;
  }
}

template <class R>
__global__ void __launch_bounds__(kTrBlock) k_transport(const __grid_constant__ TrArgs a) {
  const int n = blockIdx.x;  // tracer
  const size_t ld = (size_t)a.ld;
  for (int cb = blockIdx.y; cb * kTrBlock < a.n; cb += gridDim.y) {
    const int i = cb * kTrBlock + threadIdx.x;
    if (i >= a.n) continue;
    const size_t base = (size_t)n * a.tstride + i;
    const R* c = static_cast<const R*>(a.tr) + base;
    const double ps = a.ps[i];
    R* td = a.has_d ? static_cast<R*>(a.d.tend) + base : nullptr;
    if (a.has_d)
      scheme_transport<R>(a.d, a.d.md != nullptr, a.L, ps, a.pver, ld, i,
                          TrCol<R>{c, nullptr, R(0), ld}, td);
    if (a.has_s)
      scheme_transport<R>(a.s, false, a.L, ps, a.pver, ld, i, TrCol<R>{c, td, (R)a.dt, ld},
                          static_cast<R*>(a.s.tend) + base);
  }
}

}  // namespace

cudaError_t launch_transport(const TrArgs& a, bool fp64) {
  if (a.n == 0 || a.ntr == 0) return cudaSuccess;
  const int blocks = (a.n + kTrBlock - 1) / kTrBlock;
  const dim3 grid((unsigned)a.ntr, (unsigned)(blocks < 65535 ? blocks : 65535));
  if (fp64)
    k_transport<double><<<grid, kTrBlock, 0, a.stream>>>(a);
  else
    k_transport<float><<<grid, kTrBlock, 0, a.stream>>>(a);
  return cudaGetLastError();
}

}  // namespace cvg
