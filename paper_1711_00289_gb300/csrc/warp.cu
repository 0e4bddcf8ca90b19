// warp.cu -- the trigger pass with one column per warp (lane k = level k), the
// alternative mapping to one column per thread (compact.cu: k_trigger).
//
// Level-parallel in this mapping: the prologue of every level (pressures, log-
// thicknesses, virtual temperature, moist static energy), the heights (a
// suffix sum over levels: a warp scan), the launch level (an argmax: a warp
// reduction), the LCL layer (a ballot), the undilute parcel (every level's
// moist inversion at once, each started from the environment), the
// equilibrium level and the buoyancy bound (ballots).  Serial in it: the LCL
// solve (every lane computes it), the CAPE sum (shuffled level by level, in the
// thread mapping's order) and, for the columns that do not trigger, the shallow
// scheme where the deep trigger's bounds do not settle it (exits E1 and E2 by
// bounds are level-parallel; anything else runs the thread mapping's column
// code on lane 0).  The plume pass and the outputs' layout are unchanged, so a
// run picks either trigger pass (conv_launch.mapping; the batch autotuner
// times both).
#include "compact.h"

namespace cvg {

namespace {

constexpr int kWarpCols = 8;  // columns (warps) per block

template <class R>
__device__ __forceinline__ R shfl(R v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

// One column spread over a warp: lane k holds level k.
template <class R>
struct WarpCol {
  R T, q, pm, dl, zm, tv, h;  // this lane's level (zero on lanes >= pver)
  R Tref, qref;               // MSE reference (mixed path: the lowest layer)
  int pver, ktl;
  bool lvl;    // lane < pver and the column is live
  bool valid;  // the column passed the input check
};

template <class R>
__device__ __forceinline__ void warp_prologue(const RunArgs& a, int i, bool live, int lane,
                                              R ptl, WarpCol<R>& c) {
  using Pr = typename PressOf<R>::type;
  c.pver = a.L.pver;
  const int k = lane;
  c.lvl = live && k < c.pver;
  R Tk = R(0), qk = R(0);
  if (c.lvl) {
    Tk = __ldg(static_cast<const R*>(a.T) + (size_t)k * a.ld + i);
    qk = __ldg(static_cast<const R*>(a.q) + (size_t)k * a.ld + i);
  }
  c.T = Tk;
  c.q = qk;
  c.Tref = Mth<R>::anomaly ? shfl(Tk, c.pver - 1) : R(0);
  c.qref = Mth<R>::anomaly ? shfl(qk, c.pver - 1) : R(0);
  const double ps = live ? a.ps[i] : 1e5;
  const Pr P{a.L, (R)ps};
  const int kk = k < c.pver ? k : c.pver - 1;  // idle lanes mirror the top layer
  const R pi_lo = P.pi(kk + 1), pi_hi = P.pi(kk);
  c.pm = P.mid(pi_lo, pi_hi);
  const bool ok_lane = !c.lvl || in_range(Tk, qk);
  c.valid = live && ps > 5.0e4 && ps < 1.2e5 && __all_sync(0xffffffffu, ok_lane);
  c.tv = virt(Tk, qk);
  const R scale = R(RD / GRAV) * c.tv;
  c.dl = Mth<R>::lg(Mth<R>::dv(pi_lo, pi_hi));
  const R lzm = Mth<R>::lg(Mth<R>::dv(pi_lo, c.pm));
  // heights: z at the interface below layer k is the sum of the layer depths
  // below it (an inclusive suffix sum over lanes, shifted by one)
  R s = c.lvl ? scale * c.dl : R(0);
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const R u = __shfl_down_sync(0xffffffffu, s, off);
    if (lane + off < 32) s += u;
  }
  R zi = __shfl_down_sync(0xffffffffu, s, 1);
  if (lane == 31) zi = R(0);
  c.zm = zi + scale * lzm;
  c.h = mse(Tk, qk, c.zm, c.Tref, c.qref);
  const unsigned top = __ballot_sync(0xffffffffu, c.lvl && c.pm >= ptl);
  c.ktl = top ? __ffs(top) - 1 : c.pver - 1;
}

// Largest level k <= kstart whose mid-layer pressure is at or below b, or -1.
template <class R>
__device__ __forceinline__ int warp_level_at_or_above(const WarpCol<R>& c, int lane, int kstart,
                                                      R b) {
  const unsigned m = __ballot_sync(0xffffffffu, c.lvl && lane <= kstart && c.pm <= b);
  return m ? 31 - __clz(m) : -1;
}

// The LCL of the parcel at layer kstart, as lcl_solve computes it (every lane
// computes it; the layer search is a ballot).
__device__ __forceinline__ Lcl warp_lcl(const WarpCol<double>& c, int lane, int kstart, int n_newton,
                                        float& newton, double) {
  const double Tb = shfl(c.T, kstart), qb = shfl(c.q, kstart), pb = shfl(c.pm, kstart);
  Lcl r;
  r.pL = lcl_p(Tb, qb, pb, n_newton, newton);
  r.klcl = warp_level_at_or_above(c, lane, kstart, cmp_bound(r.pL, 0.0));
  r.exact = true;
  return r;
}
__device__ __forceinline__ Lcl warp_lcl(const WarpCol<float>& c, int lane, int kstart, int n_newton,
                                        float& newton, float guard) {
  const float Tb = shfl(c.T, kstart), qb = shfl(c.q, kstart), pb = shfl(c.pm, kstart);
  const LclF32 s = lcl_f32(Tb, qb, pb, n_newton, newton);
  Lcl r;
  if (s.saturated) {
    r.pL = (double)pb;
    r.klcl = kstart;
    r.exact = true;
    return r;
  }
  const float pLf = s.pL;
  const int k = warp_level_at_or_above(c, lane, kstart, pLf);
  const float lo = pLf * (1.f - kLclBand), hi = pLf * (1.f + kLclBand);
  const float pmk = shfl(c.pm, k >= 0 ? k : 0), pmk1 = shfl(c.pm, k + 1 <= 31 ? k + 1 : 31);
  const bool near_level = (k >= 0 && pmk > lo) || (k < kstart && pmk1 <= hi);
  const bool near_guard = guard > 0.f && fabsf(guard - pLf) <= kLclBand * pLf;
  if (!(near_level || near_guard)) {
    r.pL = (double)pLf;
    r.klcl = k;
    r.exact = false;
    return r;
  }
  r.pL = lcl_fp64_correction(Tb, qb, pb, s, newton);
  r.klcl = warp_level_at_or_above(c, lane, kstart, cmp_bound(r.pL, 0.f));
  r.exact = true;
  return r;
}

// tangent_not_buoyant of lane k's level (see column.cuh).
template <class R>
__device__ __forceinline__ bool warp_tangent_not_buoyant(const WarpCol<R>& c, R h) {
  const R Te = c.T, pm = c.pm;
  const R rt = Mth<R>::dv(R(1), Te - R(EST1));
  const R es0 = R(ES0) * Mth<R>::es(R(ESA) * (Te - R(EST0)) * rt);
  const R D0 = pm - R(ONE_M_EPS) * es0;
  if (!(D0 >= R(1e-3) * pm)) return false;
  const R qs0 = Mth<R>::dv(R(EPSV) * es0, D0);
  const R dqs0 = Mth<R>::dv(qs0 * pm, D0) * (R(ESA * ESC) * rt * rt);
  const R f0 = R(CP) * (Te - c.Tref) + R(GRAV) * c.zm + R(LV) * (qs0 - c.qref) - h;
  const R T1 = Te - Mth<R>::dv(f0, R(CP) + R(LV) * dqs0);
  const R es1 = R(ES0) * Mth<R>::es(Mth<R>::dv(R(ESA) * (T1 - R(EST0)), T1 - R(EST1)));
  const R D1 = pm - R(ONE_M_EPS) * es1;
  if (!(D1 >= R(1e-3) * pm)) return false;
  const R bup = virt(T1, Mth<R>::dv(R(EPSV) * es1, D1)) - c.tv;
  return bup < R(-kBuoyMargin);
}

template <class R, bool EXT>
__device__ __forceinline__ void zero_level(const OutP& o, const RunArgs& a, int i, int k) {
  const auto out = out_col<R, EXT>(o, a, i);
  out.put(k, R(0), R(0));
  out.flux(k, R(0), R(0), R(0));
}

// The trigger pass of the warp's column.  Every lane of every warp of the block
// calls it: the queue append is one atomic per block (s_trig, s_base: the
// block's shared flags of its warps' columns and queue base).
template <class R, bool EXT>
__device__ __forceinline__ void trigger_warp_body(const RunArgs& a, const CompactWs<R>& w, int i,
                                                  bool live, int tag, int* s_trig, int* s_base) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const DeepQ<R>& Q = deep_q(a, R(0));
  WarpCol<R> c;
  warp_prologue(a, i, live, lane, Q.p_top_lim, c);
  DeepOut o;
  o.prec = o.cape = o.mb = o.cons = 0.0;
  o.flags = c.valid ? 0 : CONV_FLAG_BADINPUT;
  o.kb = o.klcl = o.ktop = o.kaux = -1;
  bool triggered = false;
  float newton = 0.f;
  int kb = -1, klcl = -1, kel = -1;
  double cape = 0.0, pL = 0.0;
  bool pL_exact = false;
  uint32_t maybe_buoy = 0u;
  if (c.valid) {
    // launch level: largest h over the layers below p_launch_min (and the lowest
    // layer), ties to the lowest
    const bool cand = c.lvl && (lane == c.pver - 1 || c.pm >= Q.p_launch_min);
    R hk = cand ? c.h : R(-1e30);
    int kk = cand ? lane : -1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const R oh = __shfl_xor_sync(0xffffffffu, hk, off);
      const int ok = __shfl_xor_sync(0xffffffffu, kk, off);
      if (oh > hk || (oh == hk && ok > kk)) {
        hk = oh;
        kk = ok;
      }
    }
    kb = kk;
    const R hb = hk;
    const Lcl l = warp_lcl(c, lane, kb, a.dp.n_newton_lcl, newton, R(-1));
    pL = l.pL;
    pL_exact = l.exact;
    klcl = l.klcl;
    if (klcl >= c.ktl) {
      // the undilute parcel on every level from the LCL layer up, at once
      const bool par = c.lvl && lane <= klcl && lane >= c.ktl;
      R term = R(0);
      R b = R(0);
      float nl = 0.f;
      if (par) {
        MoistSeq<R> seq;
        seq.have = false;
        R qsp;
        const R Tp = moist_invert(hb, R(GRAV) * c.zm, c.pm, c.T, a.dp.n_newton_h, seq, nl, c.Tref,
                                  c.qref, sizeof(R) == 8 ? nullptr : &qsp);
        if constexpr (sizeof(R) == 8) qsp = sat_qs(Tp, c.pm);
        w.Tp[(size_t)lane * w.cap + tag] = Tp;
        b = virt(Tp, qsp) - c.tv;
        term = R(RD) * b * c.dl;
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
        nl = fmaxf(nl, __shfl_xor_sync(0xffffffffu, nl, off));
      newton = fmaxf(newton, nl);
      maybe_buoy = __ballot_sync(0xffffffffu, par && b > R(-kBuoyMargin));
      const unsigned pos = __ballot_sync(0xffffffffu, par && b > R(0));
      kel = pos ? __ffs(pos) - 1 : -1;
      if (kel >= 0) {
        // CAPE from the LCL layer up to the equilibrium level, in that order
        Acc<R> run;
        for (int k = klcl; k >= kel; --k) run.add(shfl(term, k));
        cape = run.value();
        if (cape < 0.0) cape = 0.0;
        triggered = cape > a.dp.capelmt;
      }
    }
    o.kb = kb;
    o.klcl = klcl;
    o.cape = cape;
    if (triggered) o.flags |= CONV_FLAG_TRIGGERED;
    if (newton > Mth<R>::newton_tol) o.flags |= CONV_FLAG_NEWTON;
  }
  // queue append: one atomic per block
  if (lane == 0) s_trig[warp] = triggered ? 1 : 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int j = 0; j < kWarpCols; ++j) cnt += s_trig[j];
    *s_base = cnt ? atomicAdd(w.count, cnt) : 0;
  }
  __syncthreads();
  if (!live) return;
  if (triggered) {
    if (lane == 0) {
      int slot = *s_base;
      for (int j = 0; j < warp; ++j) slot += s_trig[j];
      w.queue[slot] = tag;
      w.levels[slot] = kb | (klcl << 8) | (kel << 16);
      w.cape[slot] = cape;
      store_deep_scalars(a, i, o);
    }
    return;
  }
  if (c.lvl) zero_level<R, EXT>(a.od, a, i, lane);
  if (lane == 0) store_deep_scalars(a, i, o);
  if (!(a.mode & MODE_SHALLOW)) return;
  // the shallow scheme on the unchanged state
  const ShalQ<R>& SQ = shal_q(a, R(0));
  const bool same_src = kb == c.pver - 1 && a.sp.p_top_lim == a.dp.p_top_lim &&
                        a.sp.n_newton_lcl == a.dp.n_newton_lcl &&
                        a.sp.n_newton_h == a.dp.n_newton_h && klcl >= c.ktl;
  const bool bound_ok = newton <= Mth<R>::newton_tol;
  int settled = 0;  // 1: exit E1, 2: exit E2 by bounds, level-parallel
  float newton_s = 0.f;
  Lcl ls{0.0, -1, false};
  if (c.valid && !same_src && bound_ok && a.sp.p_top_lim == a.dp.p_top_lim) {
    const int ks = c.pver - 1;
    ls = warp_lcl(c, lane, ks, a.sp.n_newton_lcl, newton_s, SQ.p_lcl_min);
    if (ls.pL < a.sp.p_lcl_min || ls.klcl < c.ktl) {
      settled = 1;
    } else {
      const R hsrc = shfl(c.h, ks);
      const bool rel = c.lvl && lane >= c.ktl && lane <= ls.klcl && c.pm >= SQ.p_lfc_min;
      const bool covered = lane <= klcl && lane >= c.ktl && !((maybe_buoy >> lane) & 1u);
      const bool ok = !rel || covered || warp_tangent_not_buoyant(c, hsrc);
      if (__all_sync(0xffffffffu, ok)) settled = 2;
    }
  }
  if (settled) {
    if (c.lvl) zero_level<R, EXT>(a.os, a, i, lane);
    if (lane == 0) {
      ShalOut s;
      s.prec = s.cin = s.mb = s.cons = 0.0;
      s.flags = (settled << CONV_EXIT_SHIFT) |
                (newton_s > Mth<R>::newton_tol ? CONV_FLAG_NEWTON : 0);
      s.klcl = ls.klcl;
      s.ktop = -1;
      s.klfc = -1;
      store_shallow_scalars(a, i, s);
    }
    return;
  }
  // everything else: the thread mapping's column code, on lane 0
  if (lane == 0) {
    Column<R> cc;
    LevelBuf<R> cbuf;
    init_column(cc, a.L, input_src<R>(a, i), a.ps[i], cbuf);
    ShalOut s;
    const auto so = out_col<R, EXT>(a.os, a, i);
    if (!c.valid) {
      shallow_column(a.sp, SQ, cc, s, so);  // flags the column as bad input
    } else {
      prologue(SQ.p_top_lim, cc);
      const ShallowSeed<R> seed{pL, klcl, pL_exact, w.Tp + tag, (size_t)w.cap};
      const DeepBound bound{klcl, c.ktl, maybe_buoy};
      shallow_column(a.sp, SQ, cc, s, so, same_src ? &seed : nullptr, true,
                     bound_ok ? &bound : nullptr);
    }
    store_shallow_scalars(a, i, s);
  }
}

template <class R, bool EXT>
__global__ void __launch_bounds__(32 * kWarpCols, 4) k_trigger_warp(const __grid_constant__ RunArgs a,
                                                                 CompactWs<R> w) {
  __shared__ int s_trig[kWarpCols];
  __shared__ int s_base;
  const int i = blockIdx.x * kWarpCols + (threadIdx.x >> 5);
  trigger_warp_body<R, EXT>(a, w, i, i < a.n, i, s_trig, &s_base);
}

__device__ __forceinline__ int find_member_w(const int* off, int M, int g) {
  int lo = 0, hi = M;  // invariant: off[lo] <= g < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <class R>
__global__ void __launch_bounds__(32 * kWarpCols, 4) k_batch_trigger_warp(BatchDev b, const RunArgs* __restrict__ members,
                                                                      CompactWs<R> w) {
  __shared__ int s_trig[kWarpCols];
  __shared__ int s_base;
  const int g = blockIdx.x * kWarpCols + (threadIdx.x >> 5);
  const bool live = g < b.total;
  const int m = live ? find_member_w(b.offsets, b.n_members, g) : 0;
  trigger_warp_body<R, false>(members[m], w, live ? g - b.offsets[m] : 0, live, g, s_trig,
                              &s_base);
}

}  // namespace

cudaError_t launch_trigger_warp(const RunArgs& a, const CompactWs<float>& w) {
  const int grid = (a.n + kWarpCols - 1) / kWarpCols;
  NvtxRange r("conv: trigger pass, warp per column");
  if (a.ext)
    k_trigger_warp<float, true><<<grid, 32 * kWarpCols, 0, a.stream>>>(a, w);
  else
    k_trigger_warp<float, false><<<grid, 32 * kWarpCols, 0, a.stream>>>(a, w);
  return cudaGetLastError();
}
cudaError_t launch_trigger_warp(const RunArgs& a, const CompactWs<double>& w) {
  const int grid = (a.n + kWarpCols - 1) / kWarpCols;
  NvtxRange r("conv: trigger pass, warp per column");
  if (a.ext)
    k_trigger_warp<double, true><<<grid, 32 * kWarpCols, 0, a.stream>>>(a, w);
  else
    k_trigger_warp<double, false><<<grid, 32 * kWarpCols, 0, a.stream>>>(a, w);
  return cudaGetLastError();
}
cudaError_t launch_batch_trigger_warp(const BatchDev& b, const CompactWs<float>& w,
                                      cudaStream_t s) {
  k_batch_trigger_warp<float><<<(b.total + kWarpCols - 1) / kWarpCols, 32 * kWarpCols, 0, s>>>(
      b, b.members, w);
  return cudaGetLastError();
}
cudaError_t launch_batch_trigger_warp(const BatchDev& b, const CompactWs<double>& w,
                                      cudaStream_t s) {
  k_batch_trigger_warp<double><<<(b.total + kWarpCols - 1) / kWarpCols, 32 * kWarpCols, 0, s>>>(
      b, b.members, w);
  return cudaGetLastError();
}

}  // namespace cvg
