// column.cuh -- per-column deep and shallow convection for the GB300 kernels.
//
// Device code only; included by the kernel translation units.  Every routine is
// a template over the working precision R:
//   R = double  the FP64 path: every operation FP64, every Newton solve as the
//               scheme defines it (fixed LCL count; moist inversions stop on a
//               1e-7 K convergence test);
//   R = float   the mixed path: bulk FP32 with FP64 islands where a decision
//               turns on a small difference: the LCL (FP32 Newton iterations,
//               then one FP64 Newton correction with an FP64 residual where p_L
//               lies within kLclBand of a comparison), shallow rain near the
//               autoconversion threshold (kDrizzleBand) and deep condensate near
//               zero (kDeepDrizzleBand).  CAPE, CIN and the column conservation
//               sums add FP32 terms in compensated (TwoSum) arithmetic.  Moist
//               inversions are warm-started from the previous level's solution
//               by a tangent predictor and take up to kWarmSteps Newton steps to
//               FP32 convergence.
//
// The schemes (paper Sec. II-A; Alg. 1 deep then shallow; Alg. 2 entrainment and
// precipitation loops; Alg. 3 shallow early exits with zeroed outputs) follow the
// column equations frozen for this library:
//  * levels  p_i = A_i p0 + B_i ps, p_k = (p_k + p_k+1)/2, m_k = dp_k/g;
//  * heights hypsometric from the virtual temperature, z = 0 at the surface;
//  * es      Bolton (1980) eq. 10, qs = eps es/max(p - (1-eps) es, 1e-3 p);
//  * LCL     root of ln es(T) - ln e_b - (cp/Rd) ln(T/T_b), Newton from Bolton eq. 22;
//  * parcel  dry adiabat below the LCL layer, saturated MSE conservation above,
//            inverted by Newton from the environment temperature until a
//            correction falls below 1e-7 K (at most 1 + n_h steps);
//  * CAPE    sum of Rd (Tv_p - Tv) dln p from the LCL layer up to the highest
//            positively buoyant layer; trigger CAPE > capelmt;
//  * updraft eta = (1 + dz/z_e)^(lambda z_e); MSE and total water mixed per unit
//            cloud-base flux; implicit rain eta c0 dz l/(1 + c0 dz); cloud top the
//            first layer at/above the minimum-h* layer with h_u <= h*;
//  * downdraft from the minimum-h* layer between top and LCL down to the launch
//            layer, saturated by rain evaporation, scaled so that P >= 0;
//  * tendencies in flux form with upwind compensating motion;
//  * closure M_b = -CAPE/(tau F), F the parcel-fixed d(CAPE)/d(M_b), limited so
//            that q + dt dq/dt >= q_min;
//  * shallow source = lowest layer, exits E1 (LCL above p_lcl_min), E2 (no LFC
//            below p_lfc_min), E3 (CIN > cin_max), E4 (plume dies at the LCL);
//            M_b = rho c_m sqrt(tke) exp(-CIN/(cin_scale tke)); constant-mass-flux
//            plume mixing 1 - exp(-eps dz) per layer; w2 from the LFC with
//            dw2/dz = 2 a B - 2 b eps w2 integrated exactly per layer.
#pragma once

#include <cmath>
#include <cstdint>

#include "conv.h"

namespace cvg {

// ---------------------------------------------------------------- constants
constexpr double GRAV = 9.80616;
constexpr double RD = 287.04;
constexpr double RV = 461.5;
constexpr double CP = 1004.64;
constexpr double LV = 2.501e6;
constexpr double EPSV = RD / RV;
constexpr double ZVIR = RV / RD - 1.0;
constexpr double ONE_M_EPS = 1.0 - EPSV;
constexpr double INV_KAPPA = CP / RD;
constexpr double KAPPA = RD / CP;
constexpr double ES0 = 611.2;
constexpr double ESA = 17.67;
constexpr double EST0 = 273.15;
constexpr double EST1 = 29.65;
constexpr double ESC = 243.5;
constexpr double LN_ES0 = 6.415424237852311;  // ln(611.2), correctly rounded
constexpr int MAXL = CONV_MAX_LEVELS;
// Newton steps after the tangent predictor (mixed path), at most.  The
// iteration converges quadratically, e_{n+1} = (f''/2f') e_n^2 with
// f''/2f' <= 0.1 / K for the saturated MSE residual (about 0.02 / K at 300 K,
// 1000 hPa): on 30 levels the predictor is off by ~0.5 K and two steps leave
// ~1e-7 K; on coarse grids (8 levels, ~120 hPa layers) it is off by several
// kelvin and takes up to four.  The stop at kWarmStop ends most solves earlier.
constexpr int kWarmSteps = 4;
// A warm-started solve stops after a correction below kWarmStop (K): the error
// left, ~kNewtonQuad * step^2 <= 1e-5 K, is below FP32 resolution at
// atmospheric temperatures, so the next step would not change the result
// (measured: identical outputs on the 884,736-column grid, step 4% faster).
constexpr double kWarmStop = 1e-2;
constexpr float kNewtonQuad = 0.1f;  // bound on f''/2f' (1/K) used by the mixed flag

// Kernel-parameter copy of the vertical grid (FP64 and FP32 forms of A p0, B).
struct Levels {
  double a[MAXL + 1];
  double b[MAXL + 1];
  float ap0f[MAXL + 1];
  float bf[MAXL + 1];
  double p0;
  int pver;
};

// ---------------------------------------------------------------- FP32 quotient
// The mixed path's FP32 division, a build option.  CVG_F32_DIV = 2 (default):
// PTX div.full.f32, a full-range approximation within 2 ulp of a / b.
// 1: Markstein's FMA correction (P. Markstein, IBM J. Res. Dev. 34, 1990):
// from the hardware reciprocal estimate y ~ 1/b (PTX rcp.approx.f32) the
// quotient q0 = a y, its residual r = a - b q0 (one FMA, exact) and
// q1 = q0 + r y, within 1 ulp of a / b for normal operands; where q1 is not
// finite (b = 0, overflow) the estimate's own quotient q0 stands.  0: IEEE
// a / b, correctly rounded.  Step times on the 884,736-column grid: 0.858 ms
// (2), 0.896 ms (1), 0.952 ms (0); the mixed path's errors against the FP64
// definition are the same to two digits under all three.
#ifndef CVG_F32_DIV
#define CVG_F32_DIV 2
#endif
__device__ __forceinline__ float div_f32(float a, float b) {
#if CVG_F32_DIV == 2
  float q;
  asm("div.full.f32 %0, %1, %2;" : "=f"(q) : "f"(a), "f"(b));
  return q;
#elif CVG_F32_DIV == 1
  float y;
  asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(b));
  const float q0 = __fmul_rn(a, y);
  const float r = __fmaf_rn(-b, q0, a);
  const float q1 = __fmaf_rn(r, y, q0);
  return isfinite(q1) ? q1 : q0;
#else
  return a / b;
#endif
}

// ---------------------------------------------------------------- math per precision
// ex: fast where the result only scales a quantity.  es (the saturation
// exponential, which sets the Newton fixed point of every moist inversion), lg
// (layer thicknesses, accumulated into heights and moist static energy) and pw
// (the dry adiabat of the parcel, integrated into CIN) feed thresholds and the
// exp(-CIN) closure, so they use the accurate FP32 library functions.
template <class R>
struct Mth;
// newton_tol (K): a Newton solve whose remaining error exceeds it sets
// CONV_FLAG_NEWTON.  FP64: the remaining error is taken as the last correction
// (below cold_stop = 1e-7 K once the convergence test has ended the loop).
// cold_stop (K): a solve started from the environment stops after the first
// correction below it -- FP64: the scheme's convergence test; mixed: the same
// 0.01 K stop as the warm-started solves.  Mixed: the error the
// last step leaves, kNewtonQuad * (last correction)^2 by quadratic convergence
// -- the last correction itself measures the error before that step; in FP32
// a converged residual cp T + gz + Lv qs - h still carries ~0.05 J/kg of
// rounding, i.e. ~5e-5 K.
template <>
struct Mth<double> {
  static constexpr bool warm = false;
  static constexpr bool anomaly = false;
  static constexpr float newton_tol = 1e-4f;
  static constexpr double cold_stop = 1e-7;
  static __device__ __forceinline__ float left(double step) { return (float)fabs(step); }
  static __device__ __forceinline__ double es(double x) { return exp(x); }
  static __device__ __forceinline__ double ex(double x) { return exp(x); }
  static __device__ __forceinline__ double lg(double x) { return log(x); }
  static __device__ __forceinline__ double dv(double a, double b) { return a / b; }
  static __device__ __forceinline__ double pw(double a, double b) { return pow(a, b); }
  static __device__ __forceinline__ double ab(double a) { return fabs(a); }
};
template <>
struct Mth<float> {
  static constexpr bool warm = true;
  static constexpr bool anomaly = true;
  static constexpr float newton_tol = 1e-3f;
  static constexpr double cold_stop = kWarmStop;
  static __device__ __forceinline__ float left(float step) { return kNewtonQuad * step * step; }
  static __device__ __forceinline__ float es(float x) { return expf(x); }
  static __device__ __forceinline__ float ex(float x) { return __expf(x); }
  // logf, not __logf: with __logf (absolute error ~4e-7 on layer log-thicknesses
  // of 0.03-0.3) the tendency column integrals on rough soundings doubled to
  // 6e-5 of relative error.
  static __device__ __forceinline__ float lg(float x) { return logf(x); }
  static __device__ __forceinline__ float dv(float a, float b) { return div_f32(a, b); }
  static __device__ __forceinline__ float pw(float a, float b) { return powf(a, b); }
  static __device__ __forceinline__ float ab(float a) { return fabsf(a); }
};

// Virtual temperature T (1 + z q) with every operation rounded on its own (no
// contraction into FMA): parcel and environment values of the same air must be
// bit-identical so that their difference is exactly zero, as it is in FP64 math.
__device__ __forceinline__ double virt(double T, double q) {
  return __dmul_rn(T, __dadd_rn(1.0, __dmul_rn(ZVIR, q)));
}
__device__ __forceinline__ float virt(float T, float q) {
  return __fmul_rn(T, __fadd_rn(1.0f, __fmul_rn((float)ZVIR, q)));
}

__device__ __forceinline__ float fdiv_ieee(float a, float b) { return a / b; }

// ---------------------------------------------------------------- thermodynamics
// Saturation specific humidity, its T derivative (branch-consistent clamp) and
// 1/D, D = max(p - (1-eps) es, 1e-3 p).
template <class R>
__device__ __forceinline__ void sat_qs_dqs(R T, R p, R& qs, R& dqs, R& rD) {
  const R rt = Mth<R>::dv(R(1), T - R(EST1));
  const R es = R(ES0) * Mth<R>::es(R(ESA) * (T - R(EST0)) * rt);
  const R D = p - R(ONE_M_EPS) * es;
  const R Dmin = R(1e-3) * p;
  const R dlnes = R(ESA * ESC) * rt * rt;
  if (D < Dmin) {
    rD = Mth<R>::dv(R(1), Dmin);
    qs = R(EPSV) * es * rD;
    dqs = qs * dlnes;
  } else {
    rD = Mth<R>::dv(R(1), D);
    qs = R(EPSV) * es * rD;
    dqs = qs * p * rD * dlnes;
  }
}
template <class R>
__device__ __forceinline__ R sat_qs(R T, R p) {
  const R es = R(ES0) * Mth<R>::es(Mth<R>::dv(R(ESA) * (T - R(EST0)), T - R(EST1)));
  R D = p - R(ONE_M_EPS) * es;
  const R Dmin = R(1e-3) * p;
  if (D < Dmin) D = Dmin;
  return Mth<R>::dv(R(EPSV) * es, D);
}

// Saturated MSE inversion, cp T + gz + Lv qs(T,p) = h.  A solve either starts
// from the environment temperature and takes Newton steps until a correction
// falls below Mth::cold_stop, at most 1 + n_h of them (the scheme definition,
// whose loops test convergence for termination; always in FP64), or -- mixed
// path, later levels of a vertical sequence -- from the tangent prediction off
// the previous level's solution
//   dT = (dh - d(gz) + Lv qs dp/D) / (cp + Lv dqs/dT)
// followed by up to kWarmSteps Newton steps (fewer once a correction falls
// below kWarmStop).  Tracks the largest remaining error
// (Mth::left of the last correction).
template <class R>
struct MoistSeq {
  bool have;
  R T, qs, dqs, rD, p, gz, h;
};

// h is relative to the column reference cp Tref + Lv qref (see Column).
// qsol (optional): qs at the solution, qs - dqs * step from the last iterate
// (the second-order remainder is ~1e-15 relative once converged).
template <class R>
__device__ __forceinline__ R moist_invert(R h, R gz, R p, R T_env, int n_h, MoistSeq<R>& s,
                                          float& newton, R Tref, R qref, R* qsol = nullptr) {
  R T;
  int steps;
  const bool warm = Mth<R>::warm && s.have;
  if (warm) {
    T = s.T + Mth<R>::dv((h - s.h) - (gz - s.gz) + R(LV) * s.qs * (p - s.p) * s.rD,
                         R(CP) + R(LV) * s.dqs);
    steps = kWarmSteps;
  } else {
    T = T_env;
    steps = n_h + 1;
  }
  R step = R(0), qs = R(0), dqs = R(0), rD = R(0);
  for (int it = 0; it < steps; ++it) {
    sat_qs_dqs(T, p, qs, dqs, rD);
    const R f = R(CP) * (T - Tref) + gz + R(LV) * (qs - qref) - h;
    const R fp = R(CP) + R(LV) * dqs;
    step = Mth<R>::dv(f, fp);
    T -= step;
    if (Mth<R>::ab(step) < (warm ? R(kWarmStop) : R(Mth<R>::cold_stop))) break;
  }
  s.have = true;
  s.T = T;
  s.qs = qs;
  s.dqs = dqs;
  s.rD = rD;
  s.p = p;
  s.gz = gz;
  s.h = h;
  newton = fmaxf(newton, Mth<R>::left(step));
  if (qsol) *qsol = qs - dqs * step;
  return T;
}

// LCL of a parcel (Tb, qb, pb): pressure p_L where the dry adiabat saturates.
// FP64 path: FP64 Newton from the Bolton eq. 22 guess, n_newton steps.
__device__ __forceinline__ double lcl_p(double Tb, double qb, double pb, int n_newton,
                                        float& newton) {
  const double esb = ES0 * exp(ESA * (Tb - EST0) / (Tb - EST1));
  double Db = pb - ONE_M_EPS * esb;
  if (Db < 1e-3 * pb) Db = 1e-3 * pb;
  if (qb >= EPSV * esb / Db) return pb;
  const double eb = qb * pb / (EPSV + ONE_M_EPS * qb);
  const double rh = eb / esb;
  double T = 1.0 / (1.0 / (Tb - 55.0) - log(rh) / 2840.0) + 55.0;
  const double c0 = LN_ES0 - log(eb);
  double step = 0.0;
  for (int it = 0; it < n_newton; ++it) {
    const double r = 1.0 / (T - EST1);
    const double G = c0 + ESA * (T - EST0) * r - INV_KAPPA * log(T / Tb);
    const double Gp = ESA * ESC * r * r - INV_KAPPA / T;
    step = G / Gp;
    T -= step;
  }
  newton = fmaxf(newton, (float)fabs(step));
  return pb * pow(T / Tb, INV_KAPPA);
}

// ln(x/y) for x/y near 1 by the atanh series ln r = 2 atanh((r-1)/(r+1)) =
// 2u(1 + u^2/3 + u^4/5 + ...), u = (x-y)/(x+y); |u| <= 0.12 keeps the truncation
// below 1e-16 relative; otherwise the library logarithm.
__device__ __forceinline__ double ln_ratio(double x, double y) {
  const double u = (x - y) / (x + y);
  if (fabs(u) > 0.12) return log(x / y);
  const double u2 = u * u;
  double s = 1.0 / 15.0;
  s = fma(s, u2, 1.0 / 13.0);
  s = fma(s, u2, 1.0 / 11.0);
  s = fma(s, u2, 1.0 / 9.0);
  s = fma(s, u2, 1.0 / 7.0);
  s = fma(s, u2, 1.0 / 5.0);
  s = fma(s, u2, 1.0 / 3.0);
  s = fma(s, u2, 1.0);
  return 2.0 * u * s;
}

// Mixed path LCL, FP32 part: the same root, written in the difference form
// ln es(T) - ln es(Tb) - ln RH - (cp/Rd) ln(T/Tb) = 0 (exactly equivalent), by
// FP32 Newton iterations from the same first guess.  The FP32 pressure is good
// to ~5e-7 relative (ln RH and ln es carry ~1e-6 of FP32 rounding, i.e. 2e-5 K
// in T_L, and p_L ~ T_L^3.5).
struct LclF32 {
  float T, rGp;  // solution and 1/G' at the last iterate
  float pL;      // FP32 LCL pressure
  bool saturated;  // parcel saturated at its level: p_L = p_b exactly
};
// The FP32 LCL Newton iteration stops after a correction below kLclStop (K),
// or after n_newton steps.
constexpr float kLclStop = 1e-4f;
__device__ __forceinline__ LclF32 lcl_f32(float Tb, float qb, float pb, int n_newton,
                                          float& newton) {
  LclF32 s;
  const float esb =
      (float)ES0 * expf(div_f32((float)ESA * (Tb - (float)EST0), Tb - (float)EST1));
  float Db = pb - (float)ONE_M_EPS * esb;
  if (Db < 1e-3f * pb) Db = 1e-3f * pb;
  s.saturated = qb >= div_f32((float)EPSV * esb, Db);
  if (s.saturated) {
    s.T = Tb;
    s.rGp = 0.f;
    s.pL = pb;
    return s;
  }
  const float eb = div_f32(qb * pb, (float)EPSV + (float)ONE_M_EPS * qb);
  const float lnrh =
      logf(eb) - ((float)LN_ES0 + div_f32((float)ESA * (Tb - (float)EST0), Tb - (float)EST1));
  const float c1 = div_f32((float)(ESA * ESC), Tb - (float)EST1);
  float T = div_f32(1.f, div_f32(1.f, Tb - 55.f) - lnrh * (1.f / 2840.f)) + 55.f;
  float rGp = 0.f, step = 0.f;
  for (int it = 0; it < n_newton; ++it) {
    const float r = div_f32(1.f, T - (float)EST1);
    const float G = c1 * (T - Tb) * r - lnrh - (float)INV_KAPPA * logf(div_f32(T, Tb));
    const float Gp = (float)(ESA * ESC) * r * r - div_f32((float)INV_KAPPA, T);
    rGp = div_f32(1.f, Gp);
    step = G * rGp;
    T -= step;
    // converged: the error left, ~(G''/2G') step^2, is far below FP32 resolution
    // of T, and p_L moves by < 1e-8 relative, inside the 2e-5 decision band
    if (fabsf(step) < kLclStop) break;
  }
  newton = fmaxf(newton, fabsf(step));
  s.T = T;
  s.rGp = rGp;
  s.pL = pb * expf((float)INV_KAPPA * logf(div_f32(T, Tb)));
  return s;
}

// Mixed path LCL, FP64 island: one FP64 Newton correction of the FP32 root with
// the residual, the relative humidity and the logarithms in FP64; returns p_L.
__device__ __forceinline__ double lcl_fp64_correction(float Tb, float qb, float pb,
                                                      const LclF32& s, float& newton) {
  const double Tbd = Tb, qbd = qb, pbd = pb;
  const double eb = qbd * pbd / (EPSV + ONE_M_EPS * qbd);
  const double lnrh = log(eb) - (LN_ES0 + ESA * (Tbd - EST0) / (Tbd - EST1));
  const double Td = s.T;
  const double lr = ln_ratio(Td, Tbd);
  const double G = ESA * ESC * (Td - Tbd) / ((Td - EST1) * (Tbd - EST1)) - lnrh - INV_KAPPA * lr;
  const double step = G * (double)s.rGp;
  newton = fmaxf(newton, (float)fabs(step));
  // ln(TL/Tb) = ln(T/Tb) - step/T to second order in the (tiny) step
  return pbd * exp(INV_KAPPA * (lr - step * (double)fdiv_ieee(1.f, s.T)));
}

// LCL layer comparisons p_mid[k] <= pL.  In FP32 the comparison runs against pL
// rounded towards -inf to float: for a float x and a double y, x <= y exactly
// when x <= round_down(y), so the decision is the FP64 one without a conversion
// per level on the FP64 pipe.
__device__ __forceinline__ float cmp_bound(double pL, float) { return __double2float_rd(pL); }
__device__ __forceinline__ double cmp_bound(double pL, double) { return pL; }

// Entraining mass-flux profile (1 + dz/z_e)^(lambda z_e).
template <class R>
__device__ __forceinline__ R entrain_growth(R lam, R ze, R dz) {
  return Mth<R>::ex(lam * ze * Mth<R>::lg(R(1) + Mth<R>::dv(dz, ze)));
}

// ---------------------------------------------------------------- column sums
// Running sum of working-precision terms (CAPE, CIN, the conservation sums),
// accurate to FP64.  FP64 path: a plain FP64 sum.  Mixed path: a compensated
// FP32 pair -- Knuth's TwoSum carries the rounding error of every addition into
// a second FP32 word -- which keeps the sum of the FP32 terms to ~2^-48
// relative without occupying the FP64 pipe (on this device 1/64 of the FP32
// rate, and the pipe that bounds the trigger pass).
template <class R>
struct Acc;
template <>
struct Acc<double> {
  double s;
  __device__ __forceinline__ Acc() : s(0.0) {}
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  float hi, lo;
  __device__ __forceinline__ Acc() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---------------------------------------------------------------- parameters
// Scheme parameters in the working precision, with the parameter-only
// expressions the schemes need, computed once on the host: in a kernel, a
// double-to-float conversion or an FP64 operation runs on the FP64 pipe, at
// 1/67 of the FP32 rate on this device.
template <class R>
struct DeepQ {
  R p_launch_min, p_top_lim, ent_zscale, c0, alpha_dd, q_min, dt, lambda_default, tau_default;
  int n_plumes;                // plume-spectrum variant (1: bulk plume)
  R plume_f[CONV_MAX_PLUMES];  // entrainment-rate factor of each plume
};
template <class R>
struct ShalQ {
  R p_top_lim, p_lfc_min, p_lcl_min, eps, w2_0, m2beps, aw_beps, aw2, ql_crit;
  R cm_sqrt_tke;  // c_m sqrt(tke)
  R m_inv_cin;    // -1 / (cin_scale tke)
  R evap_k;       // rain evaporation coefficient (0: off)
  bool drag;      // b_w eps_s > 0
};
template <class R>
inline DeepQ<R> make_deep_q(const conv_deep_params& P, double dt) {
  DeepQ<R> q{(R)P.p_launch_min, (R)P.p_top_lim, (R)P.ent_zscale, (R)P.c0, (R)P.alpha_dd,
             (R)P.q_min, (R)dt, (R)P.lambda_default, (R)P.tau_default, 1, {}};
  q.n_plumes = P.n_plumes > 1 ? P.n_plumes : 1;
  for (int i = 0; i < CONV_MAX_PLUMES; ++i)
    q.plume_f[i] = i < q.n_plumes && q.n_plumes > 1
                       ? (R)std::pow(P.plume_spread, (double)i / (q.n_plumes - 1) - 0.5)
                       : R(1);
  return q;
}
template <class R>
inline ShalQ<R> make_shal_q(const conv_shallow_params& P) {
  const double beps = P.b_w * P.eps_s;
  ShalQ<R> q;
  q.p_top_lim = (R)P.p_top_lim;
  q.p_lfc_min = (R)P.p_lfc_min;
  q.p_lcl_min = (R)P.p_lcl_min;
  q.eps = (R)P.eps_s;
  q.w2_0 = (R)(2.0 / 3.0 * P.tke);
  q.drag = beps > 0.0;
  q.m2beps = (R)(-2.0 * beps);
  q.aw_beps = q.drag ? (R)(P.a_w / beps) : R(0);
  q.aw2 = (R)(2.0 * P.a_w);
  q.ql_crit = (R)P.ql_crit;
  q.cm_sqrt_tke = (R)(P.c_m * std::sqrt(P.tke));
  q.m_inv_cin = (R)(-1.0 / (P.cin_scale * P.tke));
  q.evap_k = (R)P.evap_k;
  return q;
}

// Conservation residual ratio of a scheme's outputs, a diagnostic:
// (|E_s - Lv P| + Lv |E_w + P|) / (cp sum m |dT| + Lv P), E_s = cp sum m dT and
// E_w = sum m dq from the column sums, P the precipitation.  The numerator is a
// cancellation.  FP64: in FP64.  Mixed: in FP32 with error-free
// transformations -- the sums are compensated pairs (hi, lo), P is the FP32
// value the scheme stores, and cp hi and Lv P are split into product and
// rounding error by FMA -- so the differences keep the accuracy of their FP32
// terms without the FP64 pipe (measured: 3% of the plume pass).
__device__ __forceinline__ double cons_ratio(const Acc<double>& sea, const Acc<double>& swa,
                                             double sc, double P) {
  const double se = CP * sea.value(), sw = swa.value();
  return (fabs(se - LV * P) + LV * fabs(sw + P)) / (CP * sc + LV * P + 1e-300);
}
__device__ __forceinline__ double cons_ratio(const Acc<float>& sea, const Acc<float>& swa,
                                             float sc, float P) {
  const float cp = (float)CP, lv = (float)LV;
  const float es = cp * sea.hi, es_e = __fmaf_rn(cp, sea.hi, -es) + cp * sea.lo;
  const float lp = lv * P, lp_e = __fmaf_rn(lv, P, -lp);
  const float ds = (es - lp) + (es_e - lp_e);
  const float dw = (swa.hi + P) + swa.lo;
  return (double)((fabsf(ds) + lv * fabsf(dw)) / (cp * sc + lp + 1e-30f));
}

// ---------------------------------------------------------------- column state
// T + dt*dT/dt as the schemes chain it (Alg. 1): FP64 without contraction.
// (dt already in the working precision: the mixed path converts it once.)
__device__ __forceinline__ double add_mul(double a, double dt, double b) {
  return __dadd_rn(a, __dmul_rn(dt, b));
}
__device__ __forceinline__ float add_mul(float a, float dt, float b) {
  return __fmaf_rn(dt, b, a);
}

// Moist static energy cp (T - Tref) + g z + Lv (q - qref), every operation rounded
// explicitly so that each re-evaluation of a level's h is bit-identical.
__device__ __forceinline__ double mse(double T, double q, double z, double Tref, double qref) {
  return __dadd_rn(__dadd_rn(__dmul_rn(CP, T - Tref), __dmul_rn(GRAV, z)),
                   __dmul_rn(LV, q - qref));
}
__device__ __forceinline__ float mse(float T, float q, float z, float Tref, float qref) {
  return __fmaf_rn((float)LV, __fsub_rn(q, qref),
                   __fmaf_rn((float)CP, __fsub_rn(T, Tref), __fmul_rn((float)GRAV, z)));
}

// Where a column's T and q come from: the caller's input arrays, optionally
// advanced by dt times the tendencies an earlier scheme has just written
// (read back from its output arrays), with q floored at zero.
template <class R>
struct Src {
  const R* T;
  const R* q;
  const R* dT;  // nullptr: no update
  const R* dq;
  R dt;
  size_t ld;
  int i;
  bool floor_q;
  __device__ __forceinline__ R Tk(int k) const {
    const size_t o = (size_t)k * ld + i;
    const R t = __ldg(T + o);
    return dT ? add_mul(t, dt, dT[o]) : t;
  }
  __device__ __forceinline__ R qk(int k) const {
    const size_t o = (size_t)k * ld + i;
    const R v = __ldg(q + o);
    if (!dq) return v;
    const R u = add_mul(v, dt, dq[o]);
    return (floor_q && u < R(0)) ? R(0) : u;
  }
};

// Interface pressures: FP64 path rounds each operation as the definition reads
// (no contraction); mixed path in FP32.
struct PressFP64 {
  const Levels& L;
  double ps;
  __device__ __forceinline__ double pi(int i) const {
    return __dadd_rn(__dmul_rn(L.a[i], L.p0), __dmul_rn(L.b[i], ps));
  }
  __device__ __forceinline__ double mid(double lo, double hi) const {
    return __dmul_rn(0.5, __dadd_rn(hi, lo));
  }
};
struct PressFP32 {
  const Levels& L;
  float ps;
  __device__ __forceinline__ float pi(int i) const { return fmaf(L.bf[i], ps, L.ap0f[i]); }
  __device__ __forceinline__ float mid(float lo, float hi) const {
    return __fmul_rn(0.5f, __fadd_rn(hi, lo));
  }
};
template <class R>
struct PressOf {
  using type = PressFP64;
};
template <>
struct PressOf<float> {
  using type = PressFP32;
};

// Column state.  The profile T, q stays where it is (Src: global memory, read
// again where needed, L2-resident while the column is worked on); the thread
// keeps only what costs a logarithm to rebuild: mid-layer heights z_mid and layer
// log-thicknesses ln(p_k+1/p_k).  Pressures, layer masses, virtual temperatures,
// moist static energies and layer depths are re-evaluated from those.
// Moist static energies h, hs (and every plume MSE derived from them) are
// relative to cp Tref + Lv qref: in the mixed path (Tref, qref) is the lowest
// layer's (T, q), so FP32 resolves MSE differences to ~1e-3 J/kg instead of the
// 0.03 J/kg ulp of 3.4e5 J/kg; in the FP64 path the reference is zero.  The
// reference cancels in every mixing rule, difference and Newton residual.
// Per-level values the FP64 path keeps instead of re-evaluating: there every
// re-evaluation runs on the FP64 pipe (a mid-layer pressure is eight FP64
// operations, an updated T two), whose throughput bounds the FP64 kernels; in
// the mixed path they cost a few FP32 operations and are re-evaluated.
template <class R>
struct ColCache {
  static constexpr bool on = false;
};
template <>
struct ColCache<double> {
  static constexpr bool on = true;
  double T[MAXL], q[MAXL], pm[MAXL], m[MAXL], Tv[MAXL], h[MAXL];
};

// A per-thread array over levels, element k at p[k * stride]: either the
// thread's own local array (stride 1) or the thread's slice of a shared-memory
// array of its block, level-major with the thread index innermost (stride =
// block size), where the 32 threads of a warp reading one level touch 32
// consecutive words -- one access, no bank conflict.
template <class R>
struct LevelArr {
  R* p;
  int stride;
  __device__ __forceinline__ R& operator[](int k) const { return p[k * stride]; }
};

// A thread's own storage for a column's level arrays (kept outside Column, so
// that stores through the views cannot alias the views themselves).
template <class R>
struct LevelBuf {
  R v[2 * MAXL];
};

template <class R>
struct Column {
  using Pr = typename PressOf<R>::type;
  Src<R> s;
  const Levels* L;
  LevelArr<R> zm, dl;  // mid-layer heights and layer log-thicknesses
  ColCache<R> cc;
  R Tref, qref;
  R psR;  // ps in the working precision
  int pver, ktl;
  double ps;
  __device__ __forceinline__ Pr press() const { return Pr{*L, psR}; }
  __device__ __forceinline__ R T(int k) const {
    if constexpr (ColCache<R>::on) return cc.T[k];
    else return s.Tk(k);
  }
  __device__ __forceinline__ R q(int k) const {
    if constexpr (ColCache<R>::on) return cc.q[k];
    else return s.qk(k);
  }
  __device__ __forceinline__ R pm(int k) const {
    if constexpr (ColCache<R>::on) {
      return cc.pm[k];
    } else {
      const Pr P = press();
      return P.mid(P.pi(k + 1), P.pi(k));
    }
  }
  __device__ __forceinline__ R m(int k) const {
    if constexpr (ColCache<R>::on) {
      return cc.m[k];
    } else {
      const Pr P = press();
      return (P.pi(k + 1) - P.pi(k)) * R(1.0 / GRAV);
    }
  }
  __device__ __forceinline__ R Tv(int k) const {
    if constexpr (ColCache<R>::on) return cc.Tv[k];
    else return virt(T(k), q(k));
  }
  __device__ __forceinline__ R h(int k) const {
    if constexpr (ColCache<R>::on) return cc.h[k];
    else return mse(T(k), q(k), zm[k], Tref, qref);
  }
  // saturation moist static energy h*
  __device__ __forceinline__ R hs(int k) const {
    const R Tk = T(k);
    return mse(Tk, sat_qs(Tk, pm(k)), zm[k], Tref, qref);
  }
  // layer depth z_int,k - z_int,k+1 = (Rd Tv / g) ln(p_k+1/p_k)
  __device__ __forceinline__ R dz(int k) const { return R(RD / GRAV) * Tv(k) * dl[k]; }
};

// buf: the thread's own storage for zm and dl.
template <class R>
__device__ __forceinline__ void init_column(Column<R>& c, const Levels& L, const Src<R>& s,
                                            double ps, LevelBuf<R>& buf) {
  c.s = s;
  c.L = &L;
  c.pver = L.pver;
  c.ps = ps;
  c.psR = (R)ps;
  c.zm = LevelArr<R>{buf.v, 1};
  c.dl = LevelArr<R>{buf.v + MAXL, 1};
}

// Keep zm and dl in a block-shared array instead: lv = this thread's first word
// of 2 pver levels x stride words (zm on levels 0..pver-1, then dl); which = 2
// (zm) or 3 (dl): only that array, pver levels x stride words.
template <class R>
__device__ __forceinline__ void bind_levels(Column<R>& c, R* lv, int stride, int which = 1) {
  if (which == 1) {
    c.zm = LevelArr<R>{lv, stride};
    c.dl = LevelArr<R>{lv + c.pver * stride, stride};
  } else if (which == 2) {
    c.zm = LevelArr<R>{lv, stride};
  } else {
    c.dl = LevelArr<R>{lv, stride};
  }
}

__device__ __forceinline__ bool in_range(double T, double q) {
  return (T > 100.0 && T < 400.0) && (q >= 0.0 && q < 0.1);
}
__device__ __forceinline__ bool in_range(float T, float q) {
  return (T > 100.f && T < 400.f) && (q >= 0.f && q < 0.1f);
}

// Heights, log-thicknesses and top limit (shared by both schemes), in the same
// pass over the profile as the input check: returns false for a column whose
// ps, T or q is out of range or not finite (CONV_FLAG_BADINPUT), whose derived
// values are then meaningless and unused.  DL = false keeps the log-thicknesses
// already in c.dl: they depend on ps alone, so a column whose T and q have
// been updated (the shallow scheme after the deep one) needs only new heights.
template <class R, bool DL = true>
__device__ __forceinline__ bool prologue(R ptl, Column<R>& c) {
  const auto P = c.press();
  const int pver = c.pver;
  R pi_lo = P.pi(pver);
  R zi = R(0);
  if constexpr (ColCache<R>::on) {
    for (int k = 0; k < pver; ++k) {
      c.cc.T[k] = c.s.Tk(k);
      c.cc.q[k] = c.s.qk(k);
    }
  }
  c.Tref = Mth<R>::anomaly ? c.T(pver - 1) : R(0);
  c.qref = Mth<R>::anomaly ? c.q(pver - 1) : R(0);
  int ktl = pver - 1;
  bool ok = c.ps > 5.0e4 && c.ps < 1.2e5;
  for (int k = pver - 1; k >= 0; --k) {
    const R pi_hi = P.pi(k);
    const R pm = P.mid(pi_lo, pi_hi);
    const R Tk = c.T(k), qk = c.q(k);
    ok = ok && in_range(Tk, qk);
    const R tv = virt(Tk, qk);
    const R scale = R(RD / GRAV) * tv;
    R dl;
    if constexpr (DL) {
      dl = Mth<R>::lg(Mth<R>::dv(pi_lo, pi_hi));
      c.dl[k] = dl;
    } else {
      dl = c.dl[k];
    }
    const R zm = zi + scale * Mth<R>::lg(Mth<R>::dv(pi_lo, pm));
    zi = zi + scale * dl;
    c.zm[k] = zm;
    if constexpr (ColCache<R>::on) {
      c.cc.pm[k] = pm;
      c.cc.m[k] = (pi_lo - pi_hi) * R(1.0 / GRAV);
      c.cc.Tv[k] = tv;
      c.cc.h[k] = mse(Tk, qk, zm, c.Tref, c.qref);
    }
    if (pm >= ptl) ktl = k;
    pi_lo = pi_hi;
  }
  c.ktl = ktl;
  return ok;
}

// Largest k <= kstart with p_mid[k] <= pL, or -1 (see cmp_bound).
template <class R>
__device__ __forceinline__ int lcl_level(const Column<R>& c, int kstart, double pL) {
  const R b = cmp_bound(pL, R(0));
  for (int k = kstart; k >= 0; --k)
    if (c.pm(k) <= b) return k;
  return -1;
}

// LCL pressure and layer of the parcel at layer kstart.  `guard`: a pressure the
// caller compares with p_L (the shallow E1 threshold), or <= 0.
// FP64 path: the FP64 Newton solve.  Mixed path: the FP32 solve decides the
// layer, and the FP64 correction runs only where the FP32 value could decide
// differently from the FP64 one -- a layer mid-point or the guard within
// kLclBand (40 times the FP32 error) of the FP32 p_L.  Elsewhere every
// comparison the scheme makes with p_L comes out as with the FP64 value.
// `exact`: p_L is the FP64 (or exactly saturated) value.
constexpr float kLclBand = 2e-5f;
struct Lcl {
  double pL;
  int klcl;
  bool exact;
};
__device__ __forceinline__ Lcl lcl_solve(const Column<double>& c, int kstart, int n_newton,
                                         float& newton, double) {
  Lcl r;
  r.pL = lcl_p(c.T(kstart), c.q(kstart), c.pm(kstart), n_newton, newton);
  r.klcl = lcl_level(c, kstart, r.pL);
  r.exact = true;
  return r;
}
__device__ __forceinline__ Lcl lcl_solve(const Column<float>& c, int kstart, int n_newton,
                                         float& newton, float guard) {
  const float Tb = c.T(kstart), qb = c.q(kstart), pb = c.pm(kstart);
  const LclF32 s = lcl_f32(Tb, qb, pb, n_newton, newton);
  Lcl r;
  if (s.saturated) {
    r.pL = (double)pb;
    r.klcl = kstart;  // p_mid[kstart] = p_b
    r.exact = true;
    return r;
  }
  const float pLf = s.pL;
  int k = kstart;
  for (; k >= 0; --k)
    if (c.pm(k) <= pLf) break;
  const float lo = pLf * (1.f - kLclBand), hi = pLf * (1.f + kLclBand);
  const bool near_level = (k >= 0 && c.pm(k) > lo) || (k < kstart && c.pm(k + 1) <= hi);
  const bool near_guard = guard > 0.f && fabsf(guard - pLf) <= kLclBand * pLf;
  if (!(near_level || near_guard)) {
    r.pL = (double)pLf;
    r.klcl = k;
    r.exact = false;
    return r;
  }
  r.pL = lcl_fp64_correction(Tb, qb, pb, s, newton);
  r.klcl = lcl_level(c, kstart, r.pL);
  r.exact = true;
  return r;
}

// Tendency output of one scheme for one column: [pver][ld] arrays, written
// level by level as the scheme produces them.
template <class R>
struct OutCol {
  static constexpr bool kFlux = false;
  static constexpr bool kExt = false;  // the extended instantiation (FluxCol)
  R* dT;
  R* dq;
  size_t ld;
  int i;
  __device__ __forceinline__ void put(int k, R a, R b) const {
    const size_t o = (size_t)k * ld + i;
    dT[o] = a;
    dq[o] = b;
  }
  __device__ __forceinline__ void zero(int k0, int k1) const {  // levels k0..k1-1
    for (int k = k0; k < k1; ++k) put(k, R(0), R(0));
  }
  __device__ __forceinline__ void flux(int, R, R, R) const {}
};

// The extended instantiation's writer: tendencies plus the plume's mass-flux
// profiles (any of the three pointers may be null): mu = updraft flux leaving
// layer k through its top, du = updraft air detrained into layer k (carrying
// the plume value from layer k+1), md = downdraft flux leaving layer k through
// its bottom.  Kernels instantiated with it also run the scheme variants
// (shallow rain evaporation); the default kernels are compiled without either.
template <class R>
struct FluxCol {
  static constexpr bool kFlux = true;
  static constexpr bool kExt = true;
  R* dT;
  R* dq;
  size_t ld;
  int i;
  R* mu;
  R* du;
  R* md;
  __device__ __forceinline__ void put(int k, R a, R b) const {
    const size_t o = (size_t)k * ld + i;
    dT[o] = a;
    dq[o] = b;
  }
  __device__ __forceinline__ void flux(int k, R u, R d, R m) const {
    const size_t o = (size_t)k * ld + i;
    if (mu) mu[o] = u;
    if (du) du[o] = d;
    if (md) md[o] = m;
  }
  // read back and increment a level this thread has written
  __device__ __forceinline__ R dT_at(int k) const { return dT[(size_t)k * ld + i]; }
  __device__ __forceinline__ void add(int k, R a, R b) const {
    const size_t o = (size_t)k * ld + i;
    dT[o] += a;
    dq[o] += b;
  }
  __device__ __forceinline__ void zero(int k0, int k1) const {
    for (int k = k0; k < k1; ++k) {
      put(k, R(0), R(0));
      flux(k, R(0), R(0), R(0));
    }
  }
};

// Discards tendencies (the adjoint recomputes the scheme for its tape only).
template <class R>
struct NoOut {
  static constexpr bool kFlux = false;
  static constexpr bool kExt = false;
  __device__ __forceinline__ void put(int, R, R) const {}
  __device__ __forceinline__ void zero(int, int) const {}
  __device__ __forceinline__ void flux(int, R, R, R) const {}
};

// ---------------------------------------------------------------- deep scheme
// Column scalars of the deep scheme (the tendencies go straight to OutCol).
struct DeepOut {
  double prec, cape, mb, cons;
  int flags, kb, klcl, ktop, kaux;
};

template <class R>
struct DeepTrig {
  int kb, klcl, kel;
  double cape, pL;
  bool pL_exact;
  bool triggered;
  float newton;
  uint32_t maybe_buoy;  // bit k: parcel buoyancy > -kBuoyMargin at layer k (klcl..ktl)
  R* Tp;                // parcel temperature of layer k at Tp[k * tps] (caller's storage)
  size_t tps;
};

// Margin (K) of the buoyancy bound the shallow scheme takes from the deep
// trigger (DeepBound): far above the rounding of either parcel's virtual
// temperature (~1e-5 K in FP32).
constexpr double kBuoyMargin = 1e-2;

// What the deep trigger on the same column state tells the shallow scheme about
// buoyancy.  The deep parcel starts from the launch layer, whose MSE is the
// largest below p_launch_min, so at least that of the shallow source (the
// lowest layer); at every layer above both LCLs the saturated parcel
// temperature grows with the parcel's MSE, and so does its buoyancy.  Where the
// deep parcel is not buoyant even within kBuoyMargin, the shallow parcel is not
// buoyant either.  The shallow scheme uses this (certainly_no_lfc) to settle
// exit E2 (no LFC) -- the outcome of the full search -- without its moist
// inversions when it can.
struct DeepBound {
  int klcl, ktl;        // the deep parcel's LCL layer and top limit
  uint32_t maybe_buoy;  // DeepTrig::maybe_buoy
};

// Launch level, LCL, undilute parcel, CAPE and trigger (deep "stage A").
// Writes the parcel temperature on ktl..klcl to t.Tp whenever klcl >= ktl.
template <class R>
__device__ __forceinline__ void deep_trigger(const Column<R>& c, const conv_deep_params& P,
                                             const DeepQ<R>& Q, DeepTrig<R>& t) {
  const int pver = c.pver, ktl = c.ktl;
  const R plaunch = Q.p_launch_min;
  int kb = pver - 1;
  R hb = c.h(kb);
  for (int k = pver - 2; k >= 0 && c.pm(k) >= plaunch; --k) {
    const R hk = c.h(k);
    if (hk > hb) {
      kb = k;
      hb = hk;
    }
  }
  t.kb = kb;
  t.kel = -1;
  t.cape = 0.0;
  t.triggered = false;
  t.newton = 0.f;
  t.maybe_buoy = 0u;
  const Lcl lcl = lcl_solve(c, kb, P.n_newton_lcl, t.newton, R(-1));
  t.pL = lcl.pL;
  t.pL_exact = lcl.exact;
  const int klcl = lcl.klcl;
  t.klcl = klcl;
  if (klcl < ktl) return;
  // Undilute parcel up from the LCL layer; CAPE accumulated in FP64, bottom up,
  // and captured at the highest positively buoyant layer.
  MoistSeq<R> seq;
  seq.have = false;
  Acc<R> run, at_el;
  int kel = -1;
  for (int k = klcl; k >= ktl; --k) {
    const R pm = c.pm(k), Tk = c.T(k);
    // the parcel's qs: the scheme's definition qs(Tp) in FP64 (exact also when
    // the iteration stops short of convergence, as with few Newton steps); the
    // mixed path takes it from the last linearisation, qs - dqs * step, which
    // its converged solves give to rounding (unconverged ones are flagged)
    R qsp;
    const R Tp = moist_invert(hb, R(GRAV) * c.zm[k], pm, Tk, P.n_newton_h, seq, t.newton, c.Tref,
                              c.qref, sizeof(R) == 8 ? nullptr : &qsp);
    if constexpr (sizeof(R) == 8) qsp = sat_qs(Tp, pm);
    t.Tp[(size_t)k * t.tps] = Tp;
    const R b = virt(Tp, qsp) - virt(Tk, c.q(k));
    run.add(R(RD) * b * c.dl[k]);
    if (b > R(-kBuoyMargin)) t.maybe_buoy |= 1u << k;
    if (b > R(0)) {
      kel = k;
      at_el = run;
    }
  }
  t.kel = kel;
  if (kel < 0) return;
  double cape = at_el.value();
  if (cape < 0.0) cape = 0.0;
  t.cape = cape;
  t.triggered = cape > P.capelmt;
}

// Mixed path, FP64 island for rain near a threshold: the shallow scheme's rain
// above the autoconversion threshold, and the deep updraft's condensate
// (threshold 0).
// The rain of a saturated plume layer, qt - qs(T_sat) - ql_crit, is a small
// difference of quantities near ql_crit where the plume barely exceeds the
// threshold ("drizzle"); there the FP32 saturation temperature's residual
// rounding (~5e-5 K, i.e. ~5e-8 kg/kg of qs) would be a large part of the rain.
// Where the FP32 rain lies within kDrizzleBand of zero, one FP64 Newton
// correction of T_sat with an FP64 residual, and qs at the corrected
// temperature in FP64, give the rain to the rounding of the FP32 plume state.
constexpr float kDrizzleBand = 1e-4f;  // kg/kg
// The deep updraft's condensate takes the FP64 island in a narrower band: it
// crosses zero in the first cloudy layer of nearly every plume, and an FP32
// condensate of 3e-6 kg/kg already carries only ~3e-4 of relative error.
// Measured (884,736-column step / 64-member ensemble): no island 0.758 /
// 3.59 ms, 3e-6 0.761 / 3.70, 1e-5 0.774 / 3.98, 1e-4 0.791 / 4.38; without
// it, trace deep precipitation on 8-level columns missed the mixed budget
// (4.2e-3 against 1e-3; 4.7e-4 with it).
#ifndef CVG_DEEP_DRIZZLE_BAND
#define CVG_DEEP_DRIZZLE_BAND 3e-6f
#endif
constexpr float kDeepDrizzleBand = CVG_DEEP_DRIZZLE_BAND;  // kg/kg
__device__ __forceinline__ float drizzle_fp64(float hu, float gz, float pm, float Tsat, float qt,
                                              float qlc, float Tref, float qref) {
  const double p = pm, T0 = Tsat;
  double qs, dqs, rD;
  sat_qs_dqs<double>(T0, p, qs, dqs, rD);
  const double f = CP * (T0 - (double)Tref) + (double)gz + LV * (qs - (double)qref) - (double)hu;
  const double T = T0 - f / (CP + LV * dqs);
  return (float)((double)qt - sat_qs<double>(T, p) - (double)qlc);
}

// Intermediate state of deep_plume, recorded only for the adjoint kernel (the
// forward kernels instantiate NoTape and record nothing).
struct NoTape {
  static constexpr bool kOn = false;
};
template <class R>
struct DeepTape {
  static constexpr bool kOn = true;
  R eta[MAXL], hu[MAXL], qt[MAXL], Ts[MAXL], rain[MAXL], dz[MAXL], qtu[MAXL];
  R etad[MAXL], hd[MAXL], Td[MAXL], qd[MAXL];
  R dh[MAXL], dq[MAXL], dT[MAXL];
  bool lpos[MAXL];
  R sumR, sumE, alpha, F, mb, net;
  int jt, jd, kstar;
  bool capped, limited, active, net_pos;
};

// Updraft, downdraft, tendencies, closure and limiter of a triggered column
// (deep "stage B": the entrainment and precipitation loops of Alg. 2).  hs: the
// column's saturation MSE; writes every level of `out`.
template <class R, class TP = NoTape, class OUT = OutCol<R>>
__device__ __forceinline__ void deep_plume(const Column<R>& c, const conv_deep_params& P,
                                           const DeepQ<R>& Q, R lam, R tau, DeepTrig<R>& t,
                                           DeepOut& o, const OUT& out, TP* tape = nullptr) {
  if constexpr (TP::kOn) tape->active = false;
  const int pver = c.pver, ktl = c.ktl, kb = t.kb, klcl = t.klcl, kel = t.kel;
  const R ze = Q.ent_zscale;
  // minimum h* layer above the LCL (ties: lowest); am[k] = argmin of h* over
  // layers k .. klcl-1, which at k = cloud top + 1 is the downdraft start
  int8_t am[MAXL];
  int khmin = -1;
  R hsmin = R(0);
  for (int k = klcl - 1; k >= ktl; --k) {
    const R v = c.hs(k);
    if (khmin < 0 || v < hsmin) {
      khmin = k;
      hsmin = v;
    }
    am[k] = (int8_t)khmin;
  }
  R eta[MAXL];
  eta[kb] = R(1);
  R hu1 = c.h(kb), qtu1 = c.q(kb);  // updraft MSE and total water at level k+1
  if constexpr (TP::kOn) {
    tape->hu[kb] = hu1;
    tape->qtu[kb] = qtu1;
  }
  const R zb = c.zm[kb];
  const R c0 = Q.c0;
  int jt = -1;
  R sumR = R(0);
  MoistSeq<R> seq;
  seq.have = false;
  // Variant (extended instantiation, n_plumes > 1): a spectrum of plumes with
  // entrainment rates lam * plume_f[i], each carrying 1/n of the cloud-base
  // mass flux and detraining at its own top; a plume whose top is at or below
  // the LCL layer drops out.  Per level: eS = the members' summed eta below
  // their tops, dtr = their detrainment terms at their tops; jt = highest top.
  bool ens = false;
  R eS[OUT::kExt ? MAXL : 1], dtr_h[OUT::kExt ? MAXL : 1], dtr_q[OUT::kExt ? MAXL : 1];
  if constexpr (OUT::kExt) {
    if (Q.n_plumes > 1) {
      ens = true;
      for (int k = 0; k < pver; ++k) eS[k] = dtr_h[k] = dtr_q[k] = R(0);
      const R w = Mth<R>::dv(R(1), (R)Q.n_plumes);
      for (int ip = 0; ip < Q.n_plumes; ++ip) {
        const R lam_i = lam * Q.plume_f[ip];
        R h1 = c.h(kb), q1 = c.q(kb), sr = R(0);
        int jt_i = -1;
        seq.have = false;
        for (int k = kb - 1; k >= ktl; --k) {
          const R e = entrain_growth(lam_i, ze, c.zm[k] - zb);
          eta[k] = e;
          const R de = e - eta[k + 1];
          const R re = Mth<R>::dv(R(1), e);
          const R hu = (eta[k + 1] * h1 + de * c.h(k)) * re;
          if ((k <= khmin && hu <= c.hs(k)) || k == ktl) {
            jt_i = k;
            break;
          }
          const R pm = c.pm(k);
          const R qt = (eta[k + 1] * q1 + de * c.q(k)) * re;
          const R Ts = moist_invert(hu, R(GRAV) * c.zm[k], pm, c.T(k), P.n_newton_h, seq,
                                    t.newton, c.Tref, c.qref);
          R l = qt - sat_qs(Ts, pm);
          if constexpr (sizeof(R) == 4)
            if (fabsf(l) < kDeepDrizzleBand)
              l = drizzle_fp64(hu, R(GRAV) * c.zm[k], pm, Ts, qt, 0.f, c.Tref, c.qref);
          if (l < R(0)) l = R(0);
          const R dz = c.dz(k);
          const R rain = Mth<R>::dv(e * c0 * dz * l, R(1) + c0 * dz);
          sr += rain;
          h1 = hu;
          q1 = qt - rain * re;
        }
        if (jt_i < 0 || jt_i >= klcl) continue;  // no cloud above the LCL
        if (jt < 0 || jt_i < jt) jt = jt_i;
        sumR += w * sr;
        for (int k = jt_i + 1; k <= kb; ++k) eS[k] += w * eta[k];
        dtr_h[jt_i] += w * eta[jt_i + 1] * (h1 - c.h(jt_i));
        dtr_q[jt_i] += w * eta[jt_i + 1] * (q1 - c.q(jt_i));
      }
    }
  }
  for (int k = kb - 1; !ens && k >= ktl; --k) {
    const R e = entrain_growth(lam, ze, c.zm[k] - zb);
    eta[k] = e;
    const R de = e - eta[k + 1];
    const R re = Mth<R>::dv(R(1), e);
    const R hu = (eta[k + 1] * hu1 + de * c.h(k)) * re;
    if constexpr (TP::kOn) tape->hu[k] = hu;
    if ((k <= khmin && hu <= c.hs(k)) || k == ktl) {
      jt = k;
      break;
    }
    const R pm = c.pm(k);
    const R qt = (eta[k + 1] * qtu1 + de * c.q(k)) * re;
    const R Ts = moist_invert(hu, R(GRAV) * c.zm[k], pm, c.T(k), P.n_newton_h, seq, t.newton,
                              c.Tref, c.qref);
    R l = qt - sat_qs(Ts, pm);
    if constexpr (sizeof(R) == 4)
      if (fabsf(l) < kDeepDrizzleBand)
        l = drizzle_fp64(hu, R(GRAV) * c.zm[k], pm, Ts, qt, 0.f, c.Tref, c.qref);
    const bool lpos = l > R(0);
    if (l < R(0)) l = R(0);
    const R dz = c.dz(k);
    const R rain = Mth<R>::dv(e * c0 * dz * l, R(1) + c0 * dz);
    const R qtu = qt - rain * re;
    sumR += rain;
    if constexpr (TP::kOn) {
      tape->qt[k] = qt;
      tape->Ts[k] = Ts;
      tape->lpos[k] = lpos;
      tape->rain[k] = rain;
      tape->dz[k] = dz;
      tape->qtu[k] = qtu;
    }
    hu1 = hu;
    qtu1 = qtu;
  }
  if (jt < 0 || jt >= klcl) {
    out.zero(0, pver);
    return;
  }

  // downdraft start: minimum h* strictly between cloud top and LCL (ties: lowest)
  const int jd = jt + 1 <= klcl - 1 ? am[jt + 1] : -1;
  R etad[MAXL];
  R hd1 = R(0), qd1 = R(0);  // downdraft MSE and humidity at the level above
  R sumE = R(0), alpha = R(0);
  if (jd >= 0) {
    const R zd = c.zm[jd];
    R eprev = R(0);
    seq.have = false;
    for (int k = jd; k <= kb - 1; ++k) {
      const R e = entrain_growth(lam, ze, zd - c.zm[k]);
      etad[k] = e;
      const R hk = c.h(k), qk = c.q(k), pm = c.pm(k);
      const R hd = (k == jd) ? hk : Mth<R>::dv(eprev * hd1 + (e - eprev) * hk, e);
      const R Td =
          moist_invert(hd, R(GRAV) * c.zm[k], pm, c.T(k), P.n_newton_h, seq, t.newton, c.Tref,
                       c.qref);
      const R qd = sat_qs(Td, pm);
      if constexpr (TP::kOn) {
        tape->Td[k] = Td;
        tape->hd[k] = hd;
        tape->qd[k] = qd;
      }
      sumE += e * qd - eprev * qd1 - (e - eprev) * qk;
      hd1 = hd;
      qd1 = qd;
      eprev = e;
    }
    alpha = Q.alpha_dd;
    const bool capped = alpha * sumE > sumR;
    if (capped) alpha = Mth<R>::dv(sumR, sumE);
    if constexpr (TP::kOn) tape->capped = capped;
  }

  // unit tendencies (per M_b) in flux form, from the launch layer up; dT, dq are
  // zero outside jt..kb.  The same pass accumulates the closure's F (the
  // parcel-fixed dCAPE/dM_b, summed from the LCL up as on k_el..klcl) and finds
  // the limiter's bound min (q - q_min)/(-dt dq) (first layer from the top
  // on ties).
  R dT[MAXL], dq[MAXL];
  for (int k = 0; k < jt; ++k) dT[k] = dq[k] = R(0);
  for (int k = kb + 1; k < pver; ++k) dT[k] = dq[k] = R(0);
  R dhkb = R(0), F = R(0), mlmin = R(0);
  int kml = -1;
  const R qmin = Q.q_min, mdt = -Q.dt;
  auto f_term = [&](int k, R dTk, R dqk) {
    R qsp, dqsp, rD;
    const R Tpk = t.Tp[(size_t)k * t.tps];
    sat_qs_dqs(Tpk, c.pm(k), qsp, dqsp, rD);
    const R dTvp = Mth<R>::dv((R(1) + R(ZVIR) * qsp) + R(ZVIR) * Tpk * dqsp,
                              R(CP) + R(LV) * dqsp);
    const R dTv = (R(1) + R(ZVIR) * c.q(k)) * dTk + R(ZVIR) * c.T(k) * dqk;
    F += R(RD) * c.dl[k] * (dTvp * dhkb - dTv);
  };
  for (int k = kb; k >= jt; --k) {
    const R hk = c.h(k), qk = c.q(k);
    R dh, dqk;
    bool done = false;
    if constexpr (OUT::kExt) {
      if (ens) {  // the spectrum's summed subsidence and detrainment terms
        dh = dtr_h[k];
        dqk = dtr_q[k];
        if (k > jt) {
          dh += eS[k] * (c.h(k - 1) - hk);
          dqk += eS[k] * (c.q(k - 1) - qk);
        }
        done = true;
      }
    }
    if (done) {
    } else if (k == jt) {
      dh = eta[jt + 1] * (hu1 - hk);
      dqk = eta[jt + 1] * (qtu1 - qk);
    } else {
      dh = eta[k] * (c.h(k - 1) - hk);
      dqk = eta[k] * (c.q(k - 1) - qk);
    }
    if (jd >= 0 && k >= jd) {
      if (k <= kb - 1) {
        const R D = alpha * etad[k];
        dh += D * (c.h(k + 1) - hk);
        dqk += D * (c.q(k + 1) - qk);
      } else {
        const R D = alpha * etad[kb - 1];
        dh += D * (hd1 - hk);
        dqk += D * (qd1 - qk);
      }
    }
    const R rm = Mth<R>::dv(R(1), c.m(k));
    dh *= rm;
    dqk *= rm;
    const R dTk = (dh - R(LV) * dqk) * R(1.0 / CP);
    dq[k] = dqk;
    dT[k] = dTk;
    if (k == kb) dhkb = dh;
    if constexpr (TP::kOn) tape->dh[k] = dh;
    if (k <= klcl && k >= kel) f_term(k, dTk, dqk);
    if (dqk < R(0)) {
      const R ml = Mth<R>::dv(qk - qmin, mdt * dqk);
      if (kml < 0 || ml <= mlmin) {
        mlmin = ml;
        kml = k;
      }
    }
  }
  // closure terms above the cloud top (dT = dq = 0 there)
  for (int k = (jt - 1 < klcl ? jt - 1 : klcl); k >= kel; --k) f_term(k, R(0), R(0));
  if (!(F < R(0))) {
    out.zero(0, pver);
    return;
  }
  R mb = Mth<R>::dv((R)(-t.cape), tau * F);
  const bool limited = kml >= 0 && mlmin < mb;
  const int kstar = limited ? kml : -1;
  if (limited) mb = mlmin;
  if (!(mb > R(0))) {
    out.zero(0, pver);
    return;
  }
  R net = sumR - alpha * sumE;
  const bool net_pos = net >= R(0);
  if (net < R(0)) net = R(0);
  if constexpr (TP::kOn) {
    tape->active = true;
    tape->jt = jt;
    tape->jd = jd;
    tape->kstar = kstar;
    tape->limited = limited;
    tape->net_pos = net_pos;
    tape->sumR = sumR;
    tape->sumE = sumE;
    tape->alpha = alpha;
    tape->F = F;
    tape->mb = mb;
    tape->net = net;
    if (jd < 0) tape->capped = false;
    for (int k = 0; k < pver; ++k) {
      tape->eta[k] = eta[k];
      tape->dq[k] = dq[k];
      tape->dT[k] = dT[k];
      if (jd >= 0) tape->etad[k] = etad[k];
    }
  }
  o.flags |= CONV_FLAG_ACTIVE | (limited ? CONV_FLAG_LIMITED : 0);
  o.mb = (double)mb;
  const R pr = mb * net;  // precipitation in the working precision
  o.prec = (double)pr;
  o.ktop = jt;
  o.kaux = jd;
  Acc<R> sea, swa;
  R sc = R(0);
  out.zero(0, jt);
  for (int k = jt; k <= kb; ++k) {
    const R a = mb * dT[k];
    const R b = mb * dq[k];
    out.put(k, a, b);
    if constexpr (OUT::kFlux)  // mu = M_b eta above the top, all of it detrains at jt
      out.flux(k, k > jt ? mb * eta[k] : R(0), k == jt ? mb * eta[jt + 1] : R(0),
               (jd >= 0 && k >= jd && k < kb) ? mb * alpha * etad[k] : R(0));
    const R mk = c.m(k);
    sea.add(mk * a);
    swa.add(mk * b);
    sc += mk * Mth<R>::ab(a);
  }
  out.zero(kb + 1, pver);
  o.cons = cons_ratio(sea, swa, sc, pr);
}

// Whole deep scheme for one column (T, q, ps set in c); writes every level of out.
// bound (may be nullptr): set valid when the column did not trigger, the deep
// trigger converged and the state is unchanged for the shallow scheme.
template <class R, class OUT>
__device__ __forceinline__ void deep_column(const conv_deep_params& P, const DeepQ<R>& Q, R lam,
                                            R tau, Column<R>& c, DeepOut& o, const OUT& out,
                                            DeepBound* bound = nullptr, bool* bound_ok = nullptr) {
  o.prec = o.cape = o.mb = o.cons = 0.0;
  o.flags = 0;
  o.kb = o.klcl = o.ktop = o.kaux = -1;
  if (bound_ok) *bound_ok = false;
  if (!prologue(Q.p_top_lim, c)) {
    o.flags = CONV_FLAG_BADINPUT;
    out.zero(0, c.pver);
    return;
  }
  R Tp[MAXL];
  DeepTrig<R> t;
  t.Tp = Tp;
  t.tps = 1;
  deep_trigger(c, P, Q, t);
  o.kb = t.kb;
  o.klcl = t.klcl;
  o.cape = t.cape;
  if (t.triggered) {
    o.flags |= CONV_FLAG_TRIGGERED;
    deep_plume(c, P, Q, lam, tau, t, o, out);
  } else {
    out.zero(0, c.pver);
    if (bound && t.newton <= Mth<R>::newton_tol) {
      *bound = DeepBound{t.klcl, c.ktl, t.maybe_buoy};
      *bound_ok = true;
    }
  }
  if (t.newton > Mth<R>::newton_tol) o.flags |= CONV_FLAG_NEWTON;
}

// ---------------------------------------------------------------- shallow scheme
struct ShalOut {
  double prec, cin, mb, cons;
  int flags, klcl, ktop, klfc;
};

// Results of the deep trigger the shallow scheme may reuse: when the deep
// launch layer is the lowest layer of the same (unmodified) column, the
// shallow source, its LCL and its saturated parcel are the deep ones.
template <class R>
struct ShallowSeed {
  double pL;
  int klcl;
  bool pL_exact;  // pL is FP64 (see lcl_solve); else checked against p_lcl_min here
  const R* Tp;    // parcel temperature of layer k (ktl..klcl) at Tp[k * tps]
  size_t tps;
};

// Upper bound on the saturated parcel's buoyancy at layer k, below -kBuoyMargin?
// The residual f(T) = cp (T - Tref) + g z + Lv (qs(T) - qref) - h of the
// saturated parcel is increasing and convex in T (es is convex for T < 2000 K
// and qs a convex increasing function of es while unclamped), so the zero of
// its tangent at any point -- one Newton step, here from the environment
// temperature -- lies at or above the parcel temperature, and buoyancy grows
// with the parcel temperature.  Declines (returns false) where the qs clamp
// could be active.
template <class R>
__device__ __forceinline__ bool tangent_not_buoyant(const Column<R>& c, int k, R pm, R h) {
  const R Te = c.T(k);
  const R rt = Mth<R>::dv(R(1), Te - R(EST1));
  const R es0 = R(ES0) * Mth<R>::es(R(ESA) * (Te - R(EST0)) * rt);
  const R D0 = pm - R(ONE_M_EPS) * es0;
  if (!(D0 >= R(1e-3) * pm)) return false;
  const R qs0 = Mth<R>::dv(R(EPSV) * es0, D0);
  const R dqs0 = Mth<R>::dv(qs0 * pm, D0) * (R(ESA * ESC) * rt * rt);
  const R f0 = R(CP) * (Te - c.Tref) + R(GRAV) * c.zm[k] + R(LV) * (qs0 - c.qref) - h;
  const R T1 = Te - Mth<R>::dv(f0, R(CP) + R(LV) * dqs0);
  const R es1 = R(ES0) * Mth<R>::es(Mth<R>::dv(R(ESA) * (T1 - R(EST0)), T1 - R(EST1)));
  const R D1 = pm - R(ONE_M_EPS) * es1;
  if (!(D1 >= R(1e-3) * pm)) return false;
  const R bup = virt(T1, Mth<R>::dv(R(EPSV) * es1, D1)) - c.Tv(k);
  return bup < R(-kBuoyMargin);
}

// True when no layer the shallow LFC search can reach (k <= klcl, p_mid >= plfc,
// k >= ktl) can hold a buoyant parcel of MSE h: layers the deep parcel covers
// by the deep bound, the others by the tangent bound.  False does not mean an
// LFC exists, only that the full search must decide.
template <class R>
__device__ __forceinline__ bool certainly_no_lfc(const Column<R>& c, const DeepBound& b, R h,
                                                 int klcl, R plfc) {
  for (int k = klcl; k >= c.ktl; --k) {
    const R pm = c.pm(k);
    if (!(pm >= plfc)) return true;
    if (k <= b.klcl && k >= b.ktl && !((b.maybe_buoy >> k) & 1u)) continue;
    if (!tangent_not_buoyant(c, k, pm, h)) return false;
  }
  return true;
}


// Intermediate state of shallow_column, recorded only for the adjoint kernel.
template <class R>
struct ShalTape {
  static constexpr bool kOn = true;
  R Tp[MAXL], b[MAXL];                 // undilute parcel temperature and buoyancy
  R hu[MAXL], qt[MAXL], qtu[MAXL];     // plume MSE, total water before / after rain
  R Tsat[MAXL], r[MAXL], chi[MAXL];    // saturated temperature, rain, mixing
  R dT[MAXL];                          // dT/dt output
  bool sat[MAXL];
  R mb, rho, sumr;
  double cin;
  int klcl, klfc, kts;
  bool active;
};

// Whole shallow scheme for one column in c (Alg. 3); writes every level of out.
// When `prologue_done` the column has been validated and its prologue computed
// already.  The plume's tendencies go out level by level as the plume rises:
// a level's is written once the level above has shown that the plume goes on,
// the top layer's when the plume stops; a plume that dies at its LCL (exit E4)
// overwrites what it wrote with zeros.
template <class R, class TP = NoTape, class OUT = OutCol<R>>
__device__ __forceinline__ void shallow_column(const conv_shallow_params& P, const ShalQ<R>& Q,
                                               Column<R>& c, ShalOut& o, const OUT& out,
                                               const ShallowSeed<R>* seed = nullptr,
                                               bool prologue_done = false,
                                               const DeepBound* bound = nullptr,
                                               TP* tape = nullptr) {
  if constexpr (TP::kOn) tape->active = false;
  const int pver = c.pver;
  o.prec = o.cin = o.mb = o.cons = 0.0;
  o.flags = 0;
  o.klcl = o.ktop = o.klfc = -1;
  if (!prologue_done && !prologue(Q.p_top_lim, c)) {
    o.flags = CONV_FLAG_BADINPUT;
    out.zero(0, pver);
    return;
  }
  const int ks = pver - 1, ktl = c.ktl;
  float newton = 0.f;
  double pL;
  int klcl;
  const R Tsrc = c.T(ks), qsrc = c.q(ks), psrc = c.pm(ks);
  // a seed whose FP32 p_L sits too close to the E1 threshold is not reused
  if (seed && !seed->pL_exact &&
      fabs(P.p_lcl_min - seed->pL) <= (double)kLclBand * seed->pL)
    seed = nullptr;
  if (seed) {
    pL = seed->pL;
    klcl = seed->klcl;
  } else {
    const Lcl lcl = lcl_solve(c, ks, P.n_newton_lcl, newton, Q.p_lcl_min);
    pL = lcl.pL;
    klcl = lcl.klcl;
  }
  o.klcl = klcl;
  if constexpr (TP::kOn) tape->klcl = klcl;
  int exit_code = 0;
  R mb = R(0);
  int klfc = -1, kts = -1;
  const R plfc = Q.p_lfc_min;
  const R hsrc = c.h(ks);
  Acc<R> sea, swa;
  R sc = R(0), sumr = R(0);
  R pevap = R(-1);  // precipitation after evaporation (variant; < 0: none)
  if (pL < P.p_lcl_min || klcl < ktl) {
    exit_code = 1;
  } else {
    // undilute parcel up to the LFC; CIN in FP64
    Acc<R> cina;
    MoistSeq<R> seq;
    seq.have = false;
    // a column the deep scheme found stable: first try to settle exit E2 (no LFC)
    // by bounds alone.  With a seed the parcel above the LCL is the deep parcel
    // itself (same source layer, LCL and temperatures; the mixed path's q_s
    // differs from the deep trigger's linearised one by ~1e-9 kg/kg, far inside
    // kBuoyMargin), so the deep trigger's buoyancy bits decide every layer.
    const bool no_lfc = bound != nullptr && certainly_no_lfc(c, *bound, hsrc, klcl, plfc);
    for (int k = ks; !no_lfc && k >= ktl; --k) {
      const R pm = c.pm(k);
      if (!(pm >= plfc)) break;
      R Tp, qp;
      if (k > klcl) {
        Tp = Tsrc * Mth<R>::pw(Mth<R>::dv(pm, psrc), R(KAPPA));
        qp = qsrc;
      } else {
        Tp = seed ? seed->Tp[(size_t)k * seed->tps]
                  : moist_invert(hsrc, R(GRAV) * c.zm[k], pm, c.T(k), P.n_newton_h, seq,
                                 newton, c.Tref, c.qref);
        qp = sat_qs(Tp, pm);
      }
      const R b = virt(Tp, qp) - c.Tv(k);
      if constexpr (TP::kOn) {
        tape->Tp[k] = Tp;
        tape->b[k] = b;
      }
      if (k <= klcl && b > R(0)) {
        klfc = k;
        break;
      }
      if (b < R(0)) cina.add(R(RD) * (-b) * c.dl[k]);
    }
    const double cin = cina.value();
    o.klfc = klfc;
    if (klfc < 0) {
      exit_code = 2;
    } else {
      o.cin = cin;
      if (cin > P.cin_max) {
        exit_code = 3;
      } else {
        const R rho = Mth<R>::dv(psrc, R(RD) * c.Tv(ks));
        mb = rho * Q.cm_sqrt_tke * Mth<R>::ex((R)cin * Q.m_inv_cin);
        if constexpr (TP::kOn) {
          tape->rho = rho;
          tape->mb = mb;
          tape->cin = cin;
          tape->hu[ks] = hsrc;
          tape->qtu[ks] = qsrc;
        }
        // plume, with a two-level window: (hu2, qtu2) at k+2, (hu1, qtu1, qp1, rf1) at k+1
        const R hsrc_env = hsrc;
        R hu2 = R(0), qtu2 = R(0);
        R hu1 = hsrc_env, qtu1 = qsrc, qp1 = qsrc, rf1 = R(0);
        R h_up = c.h(ks - 1), q_up = c.q(ks - 1);  // environment one level up
        R h_k1 = hsrc_env, q_k1 = qsrc;            // environment at k+1
        // fu, fd: the level's mass-flux profile values (profile outputs only)
        auto emit = [&](int k, R dh, R dqv, R fu, R fd) {
          const R rm = Mth<R>::dv(R(1), c.m(k));
          const R dqk = dqv * rm;
          const R dTk = (dh * rm - R(LV) * dqk) * R(1.0 / CP);
          out.put(k, dTk, dqk);
          if constexpr (OUT::kFlux) out.flux(k, fu, fd, R(0));
          if constexpr (TP::kOn) tape->dT[k] = dTk;
          const R mk = c.m(k);
          sea.add(mk * dTk);
          swa.add(mk * dqk);
          sc += mk * Mth<R>::ab(dTk);
        };
        // the source layer's tendency (its formula does not depend on the top)
        emit(ks, mb * (h_up - hsrc_env), mb * (q_up - qsrc), mb, R(0));
        R chi1 = R(0);  // mixing fraction of level k+1 (its detrainment per M_b)
        R rfv[OUT::kExt ? MAXL : 1];  // rain made per level (evaporation variant)
        R w2 = Q.w2_0;
        const R eps = Q.eps;
        const bool drag = Q.drag;
        const R m2beps = Q.m2beps, aw_beps = Q.aw_beps, aw2 = Q.aw2, qlc = Q.ql_crit;
        seq.have = false;
        for (int k = ks - 1; k >= ktl; --k) {
          const R dz = c.dz(k);
          const R hk = h_up, qk = q_up;  // environment at k
          if (k >= 1) {
            h_up = c.h(k - 1);
            q_up = c.q(k - 1);
          }
          R hu, qt, chik = R(0);
          if (k >= klcl) {
            hu = hu1;
            qt = qtu1;
            if constexpr (TP::kOn) tape->chi[k] = R(0);
          } else {
            const R chi = R(1) - Mth<R>::ex(-eps * dz);
            hu = hu1 + chi * (hk - hu1);
            qt = qtu1 + chi * (qk - qtu1);
            chik = chi;
            if constexpr (TP::kOn) tape->chi[k] = chi;
          }
          const R pm = c.pm(k);
          const R Tk = c.T(k);
          const R gz = R(GRAV) * c.zm[k];
          const R Tsat = moist_invert(hu, gz, pm, Tk, P.n_newton_h, seq, newton, c.Tref, c.qref);
          const R qsu = sat_qs(Tsat, pm);
          R Tu, qv;
          if constexpr (TP::kOn) {
            tape->hu[k] = hu;
            tape->qt[k] = qt;
            tape->Tsat[k] = Tsat;
            tape->sat[k] = qt >= qsu;
          }
          if (qt >= qsu) {
            Tu = Tsat;
            qv = qsu;
          } else {
            Tu = c.Tref + (hu - gz - R(LV) * (qt - c.qref)) * R(1.0 / CP);
            qv = qt;
          }
          if (k < klfc) {
            const R Tvk = virt(Tk, qk);
            const R B = R(GRAV) * Mth<R>::dv(virt(Tu, qv) - Tvk, Tvk);
            if (drag) {
              const R decay = Mth<R>::ex(m2beps * dz);
              w2 = w2 * decay + aw_beps * B * (R(1) - decay);
            } else {
              w2 = w2 + aw2 * B * dz;
            }
            if (!(w2 > R(0))) {
              kts = k + 1;
              break;
            }
          }
          if (k == ktl) {
            kts = k;
            // level k+1 (if not the source) is a regular level below the top
            if (k + 1 <= ks - 1) {
              emit(k + 1, mb * ((hu2 - hu1) + (hk - h_k1)), mb * ((qtu2 - qp1) + (qk - q_k1)),
                   mb, mb * chi1);
              sumr += rf1;
              if constexpr (OUT::kExt) rfv[k + 1] = rf1;
            }
            hu2 = hu1;
            qtu2 = qtu1;
            h_k1 = hk;
            q_k1 = qk;
            break;
          }
          R r = qt - qv - qlc;
          if constexpr (sizeof(R) == 4)
            if (qt >= qsu && fabsf(r) < kDrizzleBand)
              r = drizzle_fp64(hu, gz, pm, Tsat, qt, qlc, c.Tref, c.qref);
          if (r < R(0)) r = R(0);
          if constexpr (TP::kOn) {
            tape->r[k] = r;
            tape->qtu[k] = qt - r;
          }
          // the plume goes on above k: level k+1 is a regular level
          if (k + 1 <= ks - 1) {
            emit(k + 1, mb * ((hu2 - hu1) + (hk - h_k1)), mb * ((qtu2 - qp1) + (qk - q_k1)),
                 mb, mb * chi1);
            sumr += rf1;
            if constexpr (OUT::kExt) rfv[k + 1] = rf1;
          }
          chi1 = chik;
          hu2 = hu1;
          qtu2 = qtu1;
          hu1 = hu;
          qtu1 = qt - r;
          qp1 = qt;
          rf1 = r;
          h_k1 = hk;
          q_k1 = qk;
        }
        if (kts < 0 || kts >= klcl) {
          exit_code = 4;
        } else {
          // top layer: detrainment of the plume arriving from kts+1
          emit(kts, mb * (hu2 - h_k1), mb * (qtu2 - q_k1), R(0), mb);
          if constexpr (OUT::kExt) {
            // Variant: evaporation of the falling rain (Q.evap_k > 0).  Rain made
            // in plume layer j (kts < j < ks) falls through the layers below it;
            // layer j takes the fraction 1 - exp(-k max(qs - q, 0) dz) of the
            // flux arriving from above, moistening and cooling that layer; what
            // reaches the surface is the precipitation.
            if (Q.evap_k > R(0)) {
              R F = R(0);
              for (int j = kts + 1; j <= ks; ++j) {
                const R pm = c.pm(j), qj = c.q(j);
                R def = sat_qs(c.T(j), pm) - qj;
                if (def < R(0)) def = R(0);
                const R E = F * (R(1) - Mth<R>::ex(-Q.evap_k * def * c.dz(j)));
                F -= E;
                const R mk = c.m(j);
                const R ddq = Mth<R>::dv(E, mk);
                const R ddT = R(-LV / CP) * ddq;
                const R told = out.dT_at(j);
                out.add(j, ddT, ddq);
                sea.add(mk * ddT);
                swa.add(mk * ddq);
                sc += mk * (Mth<R>::ab(told + ddT) - Mth<R>::ab(told));
                if (j < ks) F += mb * rfv[j];
              }
              pevap = F;
            }
          }
        }
      }
    }
  }
  if (exit_code == 0 || exit_code == 4) o.flags |= CONV_FLAG_TRIGGERED;
  o.flags |= exit_code << CONV_EXIT_SHIFT;
  if (newton > Mth<R>::newton_tol) o.flags |= CONV_FLAG_NEWTON;
  if (exit_code != 0) {
    out.zero(0, pver);
    return;
  }
  out.zero(0, kts);
  o.flags |= CONV_FLAG_ACTIVE;
  o.mb = (double)mb;
  R pr = mb * sumr;  // precipitation in the working precision
  if constexpr (OUT::kExt)
    if (pevap >= R(0)) pr = pevap;
  o.prec = (double)pr;
  o.ktop = kts;
  if constexpr (TP::kOn) {
    tape->active = true;
    tape->klfc = klfc;
    tape->kts = kts;
    tape->sumr = sumr;
  }
  o.cons = cons_ratio(sea, swa, sc, pr);
}

}  // namespace cvg
