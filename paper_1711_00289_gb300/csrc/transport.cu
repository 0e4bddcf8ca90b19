// transport.cu -- convective transport of passive tracers (conv_tracer_transport)
// from the mass-flux profiles a scheme run wrote (mu, du, md).  Each scheme
// mixes a tracer as it mixes its conserved moist static energy, without a
// source term: a variant both schemes the paper cites carry (Sec. II-A), on the
// same column-parallel path.
//
// A few operations per level against one read and one write of the tracer per
// level: HBM-bound in bytes, latency-bound in practice (each level's updraft
// value depends on the level below), so the design is about loads in flight
// per thread.  A thread handles one column and a group of 4 tracers: a level's
// mass fluxes, layer mass and mixing ratio are loaded and divided once for the
// group, whose 4 recurrences run side by side, and the loads of two levels are
// issued together before either is used (measured on 884,736 columns x 25
// tracers: 1.58 ms, against 1.94 level by level, 1.73 with four levels at a
// time and 2.2 with one tracer per thread; groups of 2 and 8 were slower).
// The grid's fast index is the tracer group, so the blocks of one column block
// run close together and its profiles come from L2 after the first.  Threads
// of a warp hold adjacent columns: every level access is one coalesced line
// per warp.  A thread reads a tracer only on the levels its column's plumes
// touch and writes every level (zeros elsewhere).
#include "launch.h"

namespace cvg {

namespace {

constexpr int kTrBlock = 128;
constexpr int kTrGroup = 4;  // tracers per thread

// Interface pressure p_k = a_k p0 + b_k ps from block-shared coefficients
// (threads of a warp sit at different levels: shared memory serves them in one
// pass, where indexed kernel parameters would serialise on the constant cache).
// Same arithmetic as the scheme kernels' interface pressures.
template <class R>
struct ShLevels {
  R ap0[MAXL + 1];
  R b[MAXL + 1];
};

template <class R>
__device__ __forceinline__ R layer_mass(const ShLevels<R>& S, R ps, int k) {
  if constexpr (sizeof(R) == 8) {
    const double hi = __dadd_rn(S.ap0[k + 1], __dmul_rn(S.b[k + 1], ps));
    const double lo = __dadd_rn(S.ap0[k], __dmul_rn(S.b[k], ps));
    return (hi - lo) * (1.0 / GRAV);
  } else {
    return (fmaf(S.b[k + 1], ps, S.ap0[k + 1]) - fmaf(S.b[k], ps, S.ap0[k])) *
           (float)(1.0 / GRAV);
  }
}

struct Plume {
  int kb, kt;
  bool active;
};
__device__ __forceinline__ Plume plume_of(const TrScheme& S, int i, int pver) {
  Plume p{S.kb[i], S.ktop[i], false};
  p.active = (S.flags[i] & CONV_FLAG_ACTIVE) != 0 && p.kt >= 0 && p.kt <= p.kb && p.kb < pver;
  return p;
}

// The tracer a scheme sees: tracer g of the thread's group at level k is c, or
// max(c + dt prior, 0) after the deep stage (prior = the deep tendency this
// thread wrote earlier in the same launch, so it is read through L2, not the
// read-only path); `floor` alone where the deep stage left the column as it was.
template <class R>
struct TrSrc {
  const R* __restrict__ c;
  const R* prior;
  R dt;
  bool floor;
  size_t ld, ts;
  __device__ __forceinline__ R operator()(int g, int k) const {
    const size_t o = (size_t)g * ts + (size_t)k * ld;
    R v = c[o];
    if (prior) v = v + dt * __ldcg(prior + o);
    if (floor && v < R(0)) v = R(0);
    return v;
  }
};

// One scheme's tendencies of the thread's G tracers (ng of them live) of one
// column, level by level: the level's mass fluxes, layer mass and mixing ratios
// are loaded and divided once for all G tracers, whose recurrences then run side
// by side (G independent loads per level in flight).
// MOM: the momentum variant (conv_momentum_transport): a plume crossing layer k
// from its neighbour j gains cp (flux continuing from j) (c_k - c_j) -- the
// convective-scale pressure gradient, coefficient cp_up for the updraft and
// cp_down for the downdraft -- and the environment of layer k loses the same
// (the pressure force the plume exerts), so column momentum is conserved.
// Quotients of the transport recurrences: the tracer instantiation divides with
// IEEE a / b (25 FP32 tracers on the 884,736-column grid: 1.57 ms, against
// 1.66 ms with the schemes' div.full.f32), the momentum instantiation with the
// schemes' FP32 quotient (0.168 ms against 0.179).
template <class R, bool MOM>
__device__ __forceinline__ R tq(R a, R b) {
  if constexpr (MOM) return Mth<R>::dv(a, b);
  else return a / b;
}

template <class R, int G, bool MOM = false>
__device__ __forceinline__ void stage(const TrScheme& S, bool down, const ShLevels<R>& L, R ps,
                                      int pver, size_t ld, size_t tstr, int i, const Plume& p,
                                      const TrSrc<R>& C, R* __restrict__ out, int ng,
                                      R cp_up = R(0), R cp_down = R(0)) {
  auto put = [&](int g, int k, R v) { out[(size_t)g * tstr + (size_t)k * ld] = v; };
  if (!p.active) {
    for (int k = 0; k < pver; ++k)
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (g < ng) put(g, k, R(0));
    return;
  }
  const int kb = p.kb, kt = p.kt;
  for (int k = 0; k < kt; ++k)
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < ng) put(g, k, R(0));
  for (int k = kb + 1; k < pver; ++k)
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < ng) put(g, k, R(0));
  const R* __restrict__ mu = static_cast<const R*>(S.mu) + i;
  const R* __restrict__ du = static_cast<const R*>(S.du) + i;
  const R* __restrict__ md = down ? static_cast<const R*>(S.md) + i : nullptr;
  const int jd = down ? S.kaux[i] : -1;
  const bool dd = jd >= 0 && jd <= kb - 1;
  constexpr int D = 2;  // levels whose loads are issued together
  // downdraft values arriving at the launch layer: mixed from jd down to kb-1,
  // entraining md[k] - md[k-1] at layer k
  R cd[G];
  R cpv[MOM ? G : 1];  // momentum: the tracer one level up the downdraft
#pragma unroll
  for (int g = 0; g < G; ++g) cd[g] = R(0);
  if constexpr (MOM)
#pragma unroll
    for (int g = 0; g < G; ++g) cpv[g] = R(0);
  R mdl = R(0);
  if (dd) {
    R mprev = R(0);
    for (int k0 = jd; k0 <= kb - 1; k0 += D) {
      R mv[D], cv[G][D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int k = k0 + j;
        const bool ok = k <= kb - 1;
        mv[j] = ok ? md[(size_t)k * ld] : R(0);
#pragma unroll
        for (int g = 0; g < G; ++g) cv[g][j] = (ok && g < ng) ? C(g, k) : R(0);
      }
#pragma unroll
      for (int j = 0; j < D; ++j) {
        if (k0 + j > kb - 1) break;
        const R mk = mv[j];
        if (mk > R(0)) {
          const R r = tq<R, MOM>(mk - mprev, mk);
#pragma unroll
          for (int g = 0; g < G; ++g) {
            cd[g] = cd[g] + r * (cv[g][j] - cd[g]);
            if constexpr (MOM)
              if (mprev > R(0)) cd[g] = cd[g] + (R(1) - r) * cp_down * (cv[g][j] - cpv[g]);
          }
        }
        if constexpr (MOM)
#pragma unroll
          for (int g = 0; g < G; ++g) cpv[g] = cv[g][j];
        mprev = mk;
      }
    }
    mdl = mprev;
  }
  // launch layer upwards: tendency of layer k from the updraft value arriving
  // from k+1, then the updraft value leaving k (entraining mu[k] - mu[k+1] +
  // du[k] at layer k); mu is zero at the top layer kt and above
  R cu[G], ck[G], cb[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    cu[g] = cb[g] = R(0);
    ck[g] = g < ng ? C(g, kb) : R(0);
  }
  R mu1 = R(0);
  for (int k0 = kb; k0 >= kt; k0 -= D) {
    R muv[D], duv[D], mdv[D], mdu[MOM ? D : 1], cv[G][D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int k = k0 - j;
      const bool ok = k >= kt;
      const size_t o = (size_t)(ok ? k : kt) * ld;
      muv[j] = ok ? mu[o] : R(0);
      duv[j] = ok ? du[o] : R(0);
      mdv[j] = (ok && dd && k >= jd && k <= kb - 1) ? md[o] : R(0);
      // the downdraft flux arriving from the layer above (momentum only)
      if constexpr (MOM) mdu[j] = (ok && dd && k > jd && k <= kb - 1) ? md[o - ld] : R(0);
#pragma unroll
      for (int g = 0; g < G; ++g) cv[g][j] = (k > kt && g < ng) ? C(g, k - 1) : R(0);
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int k = k0 - j;
      if (k < kt) break;
      const R muk = muv[j], duk = duv[j], mdk = mdv[j];
      const R rm = tq<R, MOM>(R(1), layer_mass<R>(L, ps, k));
      const R ru = muk > R(0) ? tq<R, MOM>(muk - mu1 + duk, muk) : R(0);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (g >= ng) continue;
        const R cup = cv[g][j];
        R t = duk * (cu[g] - ck[g]) + muk * (cup - ck[g]);
        if (dd) {
          t += mdk * (cb[g] - ck[g]);
          if (k == kb) t += mdl * (cd[g] - ck[g]);
        }
        if constexpr (MOM) {
          // pressure forces of the updraft (from below) and the downdraft (from
          // above) in this layer; the updraft carries its own away
          const R pu = cp_up * (mu1 - duk) * (ck[g] - cb[g]);
          t -= pu + cp_down * mdu[j] * (ck[g] - cup);
          put(g, k, t * rm);
          cu[g] = muk > R(0) ? cu[g] + ru * (ck[g] - cu[g]) + tq<R, MOM>(pu, muk) : R(0);
        } else {
          put(g, k, t * rm);
          cu[g] = muk > R(0) ? cu[g] + ru * (ck[g] - cu[g]) : R(0);
        }
        cb[g] = ck[g];
        ck[g] = cup;
      }
      mu1 = muk;
    }
  }
}

template <class R, int G, bool MOM = false>
__global__ void __launch_bounds__(kTrBlock) k_transport(const __grid_constant__ TrArgs a) {
  __shared__ ShLevels<R> L;
  for (int k = threadIdx.x; k <= a.pver; k += blockDim.x) {
    if constexpr (sizeof(R) == 8) {
      L.ap0[k] = __dmul_rn(a.L.a[k], a.L.p0);
      L.b[k] = a.L.b[k];
    } else {
      L.ap0[k] = a.L.ap0f[k];
      L.b[k] = a.L.bf[k];
    }
  }
  __syncthreads();
  const int n0 = blockIdx.x * G;  // the thread's tracers n0 .. n0+ng-1
  const int ng = a.ntr - n0 < G ? a.ntr - n0 : G;
  const int pver = a.pver;
  const size_t ld = (size_t)a.ld, tstr = a.tstride;
  for (int cb = blockIdx.y; cb * kTrBlock < a.n; cb += gridDim.y) {
    const int i = cb * kTrBlock + threadIdx.x;
    if (i >= a.n) continue;
    const size_t base = (size_t)n0 * tstr + i;
    const R* c = static_cast<const R*>(a.tr) + base;
    const R ps = (R)a.ps[i];
    R* td = a.has_d ? static_cast<R*>(a.d.tend) + base : nullptr;
    bool deep_active = false;
    const R cpu = (R)a.cp_up, cpd = (R)a.cp_down;
    if (a.has_d) {
      const Plume p = plume_of(a.d, i, pver);
      deep_active = p.active;
      stage<R, G, MOM>(a.d, a.d.md != nullptr, L, ps, pver, ld, tstr, i, p,
                       TrSrc<R>{c, nullptr, R(0), false, ld, tstr}, td, ng, cpu, cpd);
    }
    if (a.has_s) {
      // the shallow scheme sees the deep-updated field: a tracer floored at 0,
      // a wind component as it is
      const Plume p = plume_of(a.s, i, pver);
      stage<R, G, MOM>(a.s, false, L, ps, pver, ld, tstr, i, p,
                       TrSrc<R>{c, deep_active ? td : nullptr, (R)a.dt, a.has_d && !MOM, ld,
                                tstr},
                       static_cast<R*>(a.s.tend) + base, ng, cpu, cpd);
    }
  }
}

}  // namespace

cudaError_t launch_transport(const TrArgs& a, bool fp64) {
  if (a.n == 0 || a.ntr == 0) return cudaSuccess;
  NvtxRange r(a.mom ? "conv: momentum transport" : "conv: tracer transport");
  const int blocks = (a.n + kTrBlock - 1) / kTrBlock;
  const dim3 grid((unsigned)((a.ntr + kTrGroup - 1) / kTrGroup),
                  (unsigned)(blocks < 65535 ? blocks : 65535));
  if (a.mom) {  // the two wind components as one group
    const dim3 g2(1, grid.y);
    if (fp64)
      k_transport<double, 2, true><<<g2, kTrBlock, 0, a.stream>>>(a);
    else
      k_transport<float, 2, true><<<g2, kTrBlock, 0, a.stream>>>(a);
  } else if (fp64) {
    k_transport<double, kTrGroup><<<grid, kTrBlock, 0, a.stream>>>(a);
  } else {
    k_transport<float, kTrGroup><<<grid, kTrBlock, 0, a.stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace cvg
