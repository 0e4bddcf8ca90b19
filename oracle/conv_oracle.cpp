// conv_oracle.cpp -- plain, slow FP64 CPU oracle of the column-convection hot path.
//
// TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
// CPU-baseline leg load this code; the CUDA library shares nothing with it
// (no headers, helpers, constants or tables).
//
// What the paper fixes: the physics step runs deep convection and then shallow
// convection on every column of a chunk, each column independent of the others
// (Sec. II-A, Alg. 1).  The deep scheme (Zhang-McFarlane) has an entrainment loop
// and a precipitation loop over levels, each inverting a conserved thermodynamic
// variable for temperature (Alg. 2, `ientropy`); the shallow scheme (University
// of Washington) leaves a column early at several thermodynamic checks and sets
// that column's outputs to zero (Alg. 3).  The paper prints no equations, so the
// column equations below are this project's frozen reading; each function says
// which step it implements.  Published formulas: saturation vapour pressure and
// the LCL first guess from Bolton (1980, Mon. Wea. Rev. 108, eqs. 10 and 22).
//
// Every routine is a template over the real type R:
//   R = double : the oracle proper (compiled with -ffp-contract=off);
//   R = Dual   : forward-mode tangent of the same code (deep-scheme gradients);
//   R = Cnt    : the same code counting its floating-point operations.
// Discrete decisions (level scans, branches) always compare the value part.
//
// Parity pins (tests/test_oracle_pins.py): closed-form dry adiabat CAPE,
// Bolton cross-checks, Newton residuals, brute-force level scans on tiny columns
// (launch level, EL, LFC also over superadiabatic surface layers, cloud and
// downdraft tops from h* computed by its definition), column energy/water
// conservation, non-negativity, shallow rain bounded by the plume's condensate,
// exact zeros outside the trigger, linearity of the closure in 1/tau, and
// finite differences for the tangent.  Randomised columns (inversions,
// superadiabatic, moist and dry layers; tests/test_oracle_random.py): budgets
// closed, exact zeros off the trigger, ordered level indices, the humidity
// limiter holding.  Tracer transport (tests/test_oracle_transport.py): uniform tracers
// unchanged, column tracer mass conserved, upwind monotone transport matrices,
// the moist static energy transported as each scheme transports it, and the
// mass-flux profiles carrying the same transport when it is written as a budget
// of inflow and outflow.  Rain evaporation (tests/test_oracle_evaporation.py):
// closed enthalpy and water, monotone in the coefficient, total loss into
// unsaturated air and none into saturated air, the first-order loss.  Plume
// spectrum (tests/test_oracle_spectrum.py): one plume and identical plumes are
// the bulk plume, superposition without a downdraft, the least entraining
// member's top.  tests/test_oracle_mutants.py plants plausible mistakes in a
// copy of this file; each must fail one of these pins.

#include "conv_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

namespace {

// ---------------------------------------------------------------- constants
// SI units; standard values chosen by this project (the paper gives none).
constexpr double GRAV = 9.80616;
constexpr double RD = 287.04;
constexpr double RV = 461.5;
constexpr double CP = 1004.64;
constexpr double LV = 2.501e6;
constexpr double EPS = RD / RV;
constexpr double ZVIR = RV / RD - 1.0;
constexpr double ONE_M_EPS = 1.0 - EPS;
constexpr double INV_KAPPA = CP / RD;  // cp/Rd
constexpr double KAPPA = RD / CP;      // Rd/cp
// Bolton (1980) eq. 10: es = 611.2 exp(17.67 (T-273.15)/(T-29.65)) Pa.
constexpr double ES0 = 611.2;
constexpr double ESA = 17.67;
constexpr double EST0 = 273.15;
constexpr double EST1 = 29.65;
constexpr double ESC = 243.5;  // 273.15 - 29.65
constexpr double NEWTON_FLAG_TOL = 1e-4;  // K: last Newton step above this sets bit 3
constexpr int MAXLEV = 32;

constexpr int F_TRIGGERED = 1, F_ACTIVE = 2, F_LIMITED = 4, F_NEWTON = 8, F_BADINPUT = 16;
constexpr int EXIT_SHIFT = 8;  // shallow exit stage (1..4) in bits 8-10

// ---------------------------------------------------------------- real types
inline double val(double x) { return x; }

// Forward-mode dual number with ND tangent directions (2*32 profile entries
// plus lambda and tau).
constexpr int ND = 2 * MAXLEV + 2;
struct Dual {
  double v;
  double d[ND];
  Dual() : v(0.0) { std::memset(d, 0, sizeof d); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof d); }  // NOLINT: implicit by design
};
inline double val(const Dual& x) { return x.v; }
inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v);
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v);
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
inline Dual operator-(const Dual& a) {
  Dual r(-a.v);
  for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i];
  return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v);
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
inline Dual operator+(const Dual& a, double b) { return a + Dual(b); }
inline Dual operator+(double a, const Dual& b) { return Dual(a) + b; }
inline Dual operator-(const Dual& a, double b) { return a - Dual(b); }
inline Dual operator-(double a, const Dual& b) { return Dual(a) - b; }
inline Dual operator*(const Dual& a, double b) { return a * Dual(b); }
inline Dual operator*(double a, const Dual& b) { return Dual(a) * b; }
inline Dual operator/(const Dual& a, double b) { return a / Dual(b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
inline Dual exp(const Dual& a) {
  Dual r(std::exp(a.v));
  for (int i = 0; i < ND; ++i) r.d[i] = r.v * a.d[i];
  return r;
}
inline Dual log(const Dual& a) {
  Dual r(std::log(a.v));
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] / a.v;
  return r;
}
inline Dual sqrt(const Dual& a) {
  Dual r(std::sqrt(a.v));
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
  return r;
}
inline Dual pow(const Dual& a, double e) {
  Dual r(std::pow(a.v, e));
  const double s = e * std::pow(a.v, e - 1.0);
  for (int i = 0; i < ND; ++i) r.d[i] = s * a.d[i];
  return r;
}

// Counting real: same arithmetic as double, tallies each operation.
enum { C_ADD = 0, C_MUL, C_DIV, C_EXP, C_LOG, C_POW, C_SQRT, C_NCAT = 8 };
thread_local double g_count[C_NCAT];
struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  Cnt(double x) : v(x) {}  // NOLINT
};
inline double val(const Cnt& x) { return x.v; }
inline Cnt operator+(const Cnt& a, const Cnt& b) { g_count[C_ADD] += 1; return Cnt(a.v + b.v); }
inline Cnt operator-(const Cnt& a, const Cnt& b) { g_count[C_ADD] += 1; return Cnt(a.v - b.v); }
inline Cnt operator-(const Cnt& a) { return Cnt(-a.v); }
inline Cnt operator*(const Cnt& a, const Cnt& b) { g_count[C_MUL] += 1; return Cnt(a.v * b.v); }
inline Cnt operator/(const Cnt& a, const Cnt& b) { g_count[C_DIV] += 1; return Cnt(a.v / b.v); }
inline Cnt operator+(const Cnt& a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, const Cnt& b) { return Cnt(a) + b; }
inline Cnt operator-(const Cnt& a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, const Cnt& b) { return Cnt(a) - b; }
inline Cnt operator*(const Cnt& a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, const Cnt& b) { return Cnt(a) * b; }
inline Cnt operator/(const Cnt& a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, const Cnt& b) { return Cnt(a) / b; }
inline Cnt exp(const Cnt& a) { g_count[C_EXP] += 1; return Cnt(std::exp(a.v)); }
inline Cnt log(const Cnt& a) { g_count[C_LOG] += 1; return Cnt(std::log(a.v)); }
inline Cnt sqrt(const Cnt& a) { g_count[C_SQRT] += 1; return Cnt(std::sqrt(a.v)); }
inline Cnt pow(const Cnt& a, double e) { g_count[C_POW] += 1; return Cnt(std::pow(a.v, e)); }

// FP64-island work of the mixed-precision design, tallied by the counting
// instantiation only: LCL solves (each ends with one FP64 Newton correction),
// CAPE terms and CIN terms accumulated in FP64, conservation-sum terms, and
// saturated shallow plume layers whose rain lies within 1e-4 kg/kg of zero
// (the mixed path refines their saturation temperature in FP64).
enum { I_LCL = 0, I_CAPE, I_CIN, I_CONS, I_DRIZZLE, I_NCAT };
thread_local double g_island[I_NCAT];
// Snapshot of g_count when the deep trigger stage ends (launch level through
// the CAPE trigger): splits the deep work between the trigger and plume passes.
thread_local double g_mark[C_NCAT];
template <class R>
inline void island(int, double) {}
template <>
inline void island<Cnt>(int cat, double n) { g_island[cat] += n; }
template <class R>
inline void mark_trigger_end() {}
template <>
inline void mark_trigger_end<Cnt>() {
  for (int c = 0; c < C_NCAT; ++c) g_mark[c] = g_count[c];
}
// Snapshots of g_count around the shallow scheme's undilute-parcel LFC search
// (begin, end): the search's work, which in a column that ends at exit E2 (no
// LFC) an implementation may settle by cheaper bounds.
thread_local double g_lfc0[C_NCAT], g_lfc1[C_NCAT];
template <class R>
inline void mark_lfc_search(bool) {}
template <>
inline void mark_lfc_search<Cnt>(bool end) {
  for (int c = 0; c < C_NCAT; ++c) (end ? g_lfc1 : g_lfc0)[c] = g_count[c];
}

// ---------------------------------------------------------------- parameters
struct DeepP {
  double capelmt, lambda_default, tau_default, c0, alpha_dd, p_launch_min, p_top_lim, q_min,
      ent_zscale;
  int n_lcl, n_h;
  int n_plumes;
  double plume_spread;
};
struct ShalP {
  double eps_s, tke, c_m, cin_scale, cin_max, a_w, b_w, ql_crit, p_lcl_min, p_lfc_min, p_top_lim;
  int n_lcl, n_h;
  double evap_k;
};
DeepP to_deep(const oracle_deep_params* p) {
  return DeepP{p->capelmt, p->lambda_default, p->tau_default, p->c0, p->alpha_dd,
               p->p_launch_min, p->p_top_lim, p->q_min, p->ent_zscale, p->n_newton_lcl,
               p->n_newton_h, p->n_plumes < 1 ? 1 : p->n_plumes, p->plume_spread};
}
ShalP to_shal(const oracle_shallow_params* p) {
  return ShalP{p->eps_s, p->tke, p->c_m, p->cin_scale, p->cin_max, p->a_w, p->b_w,
               p->ql_crit, p->p_lcl_min, p->p_lfc_min, p->p_top_lim, p->n_newton_lcl,
               p->n_newton_h, p->evap_k};
}

// ---------------------------------------------------------------- thermodynamics
// Saturation vapour pressure over liquid, Bolton (1980) eq. 10.  Ice ignored.
template <class R>
R sat_es(const R& T) {
  using std::exp;
  return ES0 * exp(ESA * (T - EST0) / (T - EST1));
}

// Saturation specific humidity qs = eps es / max(p - (1-eps) es, 1e-3 p) and its
// temperature derivative (differentiating the branch that is taken).
template <class R>
void sat_qs_dqs(const R& T, const R& p, R& qs, R& dqs) {
  const R es = sat_es(T);
  R D = p - ONE_M_EPS * es;
  const R Dmin = 1e-3 * p;
  const R dlnes = ESA * ESC / ((T - EST1) * (T - EST1));
  if (val(D) < val(Dmin)) {
    qs = EPS * es / Dmin;
    dqs = qs * dlnes;
  } else {
    qs = EPS * es / D;
    dqs = qs * (p / D) * dlnes;
  }
}
// The saturation specific humidity alone (the same clamped denominator).
template <class R>
R sat_qs(const R& T, const R& p) {
  const R es = sat_es(T);
  R D = p - ONE_M_EPS * es;
  const R Dmin = 1e-3 * p;
  if (val(D) < val(Dmin)) D = Dmin;
  return EPS * es / D;
}

// Interface pressures p_i = A_i p0 + B_i ps and mid-layer p_k = (p_k + p_k+1)/2
// (hybrid sigma-pressure coordinate of the 30-level grid, Sec. V-A).
template <class R>
void levels(int pver, const double* hyai, const double* hybi, double p0, const R& ps, R* p_int,
            R* p_mid) {
  for (int i = 0; i <= pver; ++i) p_int[i] = hyai[i] * p0 + hybi[i] * ps;
  for (int k = 0; k < pver; ++k) p_mid[k] = 0.5 * (p_int[k] + p_int[k + 1]);
}

// Hypsometric heights from the virtual temperature, z = 0 at the surface.
template <class R>
void heights(int pver, const R* T, const R* q, const R* p_int, const R* p_mid, R* z_int,
             R* z_mid, R* dlnp, R* Tv) {
  using std::log;
  z_int[pver] = R(0.0);
  for (int k = pver - 1; k >= 0; --k) {
    Tv[k] = T[k] * (1.0 + ZVIR * q[k]);
    const R scale = RD * Tv[k] / GRAV;
    dlnp[k] = log(p_int[k + 1] / p_int[k]);
    z_int[k] = z_int[k + 1] + scale * dlnp[k];
    z_mid[k] = z_int[k + 1] + scale * log(p_int[k + 1] / p_mid[k]);
  }
}

// Newton inversion of moist static energy for a saturated parcel: find T with
// cp T + g z + Lv qs(T, p) = h.  Newton from T_start (the environment); the
// loop tests convergence for termination, as the scheme loops the paper times
// do (Sec. V-C): it stops after the first correction smaller than H_STOP, and
// after at most 1 + n_extra steps.  The residual is increasing and convex in T
// with f''/2f' <= 0.1 / K, so the error left after a correction c is about
// 0.1 c^2: below H_STOP = 1e-7 K it is ~1e-15 K, under the rounding of T.
// Solves far from their start (a parcel 10-50 K warmer than the environment)
// take up to ten steps; most take three to five.  This is the column model's
// analogue of `ientropy` (Alg. 2).  The tangent of the solution (Dual) is taken
// by the implicit function theorem at the final iterate (ift_tangent).
constexpr double H_STOP = 1e-7;  // K

template <class R>
inline R ift_tangent(const R&, const R&, const R&, const R& T) {
  return T;
}
// dT = -(df/dtheta)/(df/dT) at the solution: one Newton correction applied to the
// tangent part only (f's tangent carries df/dT dT_iterate + df/dtheta dtheta, so
// the result no longer depends on how the iterate's tangent was built).
template <>
inline Dual ift_tangent<Dual>(const Dual& h, const Dual& gz, const Dual& p, const Dual& T) {
  Dual qs, dqs;
  sat_qs_dqs(T, p, qs, dqs);
  const Dual f = CP * T + gz + LV * qs - h;
  const double fp = CP + LV * dqs.v;
  Dual r = T;
  for (int i = 0; i < ND; ++i) r.d[i] = T.d[i] - f.d[i] / fp;
  return r;
}

template <class R>
R moist_invert(const R& h, const R& gz, const R& p, R T, int n_extra, double* last_step) {
  for (int it = 0; it <= n_extra; ++it) {
    R qs, dqs;
    sat_qs_dqs(T, p, qs, dqs);
    const R f = CP * T + gz + LV * qs - h;
    const R fp = CP + LV * dqs;
    const R step = f / fp;
    T = T - step;
    if (last_step) *last_step = std::fabs(val(step));
    if (std::fabs(val(step)) < H_STOP) break;
  }
  return ift_tangent(h, gz, p, T);
}

// Lifting condensation level of a parcel (Tb, qb, pb) lifted dry-adiabatically.
// Saturation is reached where es(T) = e_b (T/Tb)^(cp/Rd), e_b the parcel vapour
// pressure; Newton on G(T) = ln es(T) - ln e_b - (cp/Rd) ln(T/Tb) from the Bolton
// (1980) eq. 22 first guess, n_newton steps.  A parcel already saturated has its
// LCL at the launch point.  Returns the last |step|.
template <class R>
double lcl(const R& Tb, const R& qb, const R& pb, int n_newton, R& TL, R& pL) {
  using std::log;
  using std::pow;
  const R qsb = sat_qs(Tb, pb);
  if (val(qb) >= val(qsb)) {
    TL = Tb;
    pL = pb;
    return 0.0;
  }
  const R eb = qb * pb / (EPS + ONE_M_EPS * qb);
  const R rh = eb / sat_es(Tb);
  R T = 1.0 / (1.0 / (Tb - 55.0) - log(rh) / 2840.0) + 55.0;
  const R lneb = log(eb);
  const double lnes0 = std::log(ES0);
  double last = 0.0;
  for (int it = 0; it < n_newton; ++it) {
    const R G = lnes0 + ESA * (T - EST0) / (T - EST1) - lneb - INV_KAPPA * log(T / Tb);
    const R Gp = ESA * ESC / ((T - EST1) * (T - EST1)) - INV_KAPPA / T;
    const R step = G / Gp;
    T = T - step;
    last = std::fabs(val(step));
  }
  TL = T;
  pL = pb * pow(TL / Tb, INV_KAPPA);
  return last;
}

// Largest k <= kstart with p_mid[k] <= pL (first layer at or above the LCL), or -1.
template <class R>
int lcl_level(const R* p_mid, int kstart, const R& pL) {
  for (int k = kstart; k >= 0; --k)
    if (val(p_mid[k]) <= val(pL)) return k;
  return -1;
}

// Input check of one column (flag bit 4, "bad input", of the frozen interface):
// surface pressure within 500-1200 hPa, every temperature within 100-400 K and
// every humidity within [0, 0.1) kg/kg, NaN failing each test.  A column that
// fails is left with zero outputs and only that flag.
template <class R>
bool column_valid(int pver, const R* T, const R* q, const R& ps) {
  if (!(val(ps) > 5.0e4 && val(ps) < 1.2e5)) return false;
  for (int k = 0; k < pver; ++k) {
    if (!(val(T[k]) > 100.0 && val(T[k]) < 400.0)) return false;
    if (!(val(q[k]) >= 0.0 && val(q[k]) < 0.1)) return false;
  }
  return true;
}

// Normalised mass flux of an entraining plume after rising (or, for the
// downdraft, sinking) a distance dz >= 0 from its origin, with fractional
// entrainment eps = lambda z_e/(dz + z_e): lambda at the origin, decaying
// inversely with distance (the common "entrainment ~ 1/z" closure).
// d ln(eta)/d dz = eps  =>  eta = (1 + dz/z_e)^(lambda z_e).
template <class R>
R entrain_growth(const R& lambda, double z_e, const R& dz) {
  using std::exp;
  using std::log;
  return exp(lambda * z_e * log(1.0 + dz / z_e));
}

// ---------------------------------------------------------------- deep scheme
template <class R>
struct DeepState {
  int ktl = -1, kb = -1, klcl = -1, kel = -1, khmin = -1, jt = -1, jd = -1;
  bool triggered = false, active = false, limited = false, bad = false;
  double newton_max = 0.0;
  R TL, pL, cape, F, mb, sumR, sumE, alpha, prec;
  R Tp[MAXLEV], qp[MAXLEV], b[MAXLEV], eta[MAXLEV], hu[MAXLEV], qtu[MAXLEV], rain[MAXLEV];
  R etad[MAXLEV], hd[MAXLEV], qd[MAXLEV], E1[MAXLEV];
  R dh[MAXLEV], dq[MAXLEV], dT[MAXLEV], dTdt[MAXLEV], dqdt[MAXLEV];
  R m[MAXLEV], z_mid[MAXLEV], z_int[MAXLEV + 1], h[MAXLEV], hs[MAXLEV], p_mid[MAXLEV],
      p_int[MAXLEV + 1], dlnp[MAXLEV], Tv[MAXLEV];
  double cons_err = 0.0;
};

// Deep convection of one column (Sec. II-A; Alg. 2).  Steps:
//  launch level kb = argmax of moist static energy below p_launch_min (ties:
//  lowest); LCL; undilute parcel (dry adiabat below the LCL, saturated MSE
//  conservation at and above it); buoyancy of virtual temperatures; highest
//  positively buoyant level k_el; CAPE = sum of Rd b dln p over k_el..klcl
//  (serial, bottom up, negative areas included); trigger CAPE > capelmt.
//  Triggered columns: entraining bulk updraft (eta = entrain_growth(z - z_kb)),
//  MSE and total water mixed per unit cloud-base flux, implicit rain
//  R = eta c0 dz l/(1 + c0 dz)) up to the cloud top jt: the first layer, at or
//  above the minimum-h* layer, where the plume MSE has fallen to the saturated
//  environmental MSE ("entrainment loop"); a
//  saturated downdraft from the minimum-h* level jd down to kb, driven by rain
//  evaporation and scaled so precipitation stays non-negative ("precipitation
//  loop"); flux-form environment tendencies with upwind compensating
//  subsidence; CAPE-relaxation closure M_b = -CAPE/(tau F), F the parcel-fixed
//  linearised CAPE change per unit M_b; a limiter keeping q >= q_min.
template <class R>
void deep_column(int pver, const double* hyai, const double* hybi, double p0, const R* T,
                 const R* q, const R& ps, const R& lambda, const R& tau, const DeepP& P,
                 double dt, DeepState<R>& s) {
  using std::exp;
  using std::log;
  using std::pow;
  s.TL = s.pL = s.cape = s.F = s.mb = s.sumR = s.sumE = s.alpha = s.prec = R(0.0);
  for (int k = 0; k < pver; ++k) {
    s.dh[k] = s.dq[k] = s.dT[k] = s.dTdt[k] = s.dqdt[k] = R(0.0);
    s.Tp[k] = s.qp[k] = s.b[k] = s.eta[k] = s.hu[k] = s.qtu[k] = s.rain[k] = R(0.0);
    s.etad[k] = s.hd[k] = s.qd[k] = s.E1[k] = R(0.0);
  }
  if (!column_valid(pver, T, q, ps)) {
    s.bad = true;
    return;
  }
  levels(pver, hyai, hybi, p0, ps, s.p_int, s.p_mid);
  heights(pver, T, q, s.p_int, s.p_mid, s.z_int, s.z_mid, s.dlnp, s.Tv);
  for (int k = 0; k < pver; ++k) {
    s.m[k] = (s.p_int[k + 1] - s.p_int[k]) / GRAV;
    const R qsk = sat_qs(T[k], s.p_mid[k]);
    const R sdry = CP * T[k] + GRAV * s.z_mid[k];
    s.h[k] = sdry + LV * q[k];
    s.hs[k] = sdry + LV * qsk;
  }
  int ktl = pver - 1;
  for (int k = 0; k < pver; ++k)
    if (val(s.p_mid[k]) >= P.p_top_lim) { ktl = k; break; }
  s.ktl = ktl;

  // Launch level: most unstable (max h) layer below p_launch_min.
  int kb = pver - 1;
  for (int k = pver - 2; k >= 0 && val(s.p_mid[k]) >= P.p_launch_min; --k)
    if (val(s.h[k]) > val(s.h[kb])) kb = k;
  s.kb = kb;

  const R Tb = T[kb], qb = q[kb], pb = s.p_mid[kb];
  s.newton_max = std::max(s.newton_max, lcl(Tb, qb, pb, P.n_lcl, s.TL, s.pL));
  island<R>(I_LCL, 1);
  const int klcl = lcl_level(s.p_mid, kb, s.pL);
  s.klcl = klcl;
  mark_trigger_end<R>();
  if (klcl < ktl) return;  // LCL missing or above the top limit: no convection

  // Undilute parcel on levels ktl..klcl (saturated branch) and buoyancy.
  for (int k = klcl; k >= ktl; --k) {
    double st = 0.0;
    s.Tp[k] = moist_invert(s.h[kb], GRAV * s.z_mid[k], s.p_mid[k], T[k], P.n_h, &st);
    s.newton_max = std::max(s.newton_max, st);
    s.qp[k] = sat_qs(s.Tp[k], s.p_mid[k]);
    s.b[k] = s.Tp[k] * (1.0 + ZVIR * s.qp[k]) - s.Tv[k];
  }
  // Dry levels below the LCL (not used by the CAPE integral; reported).
  for (int k = kb; k > klcl; --k) {
    s.Tp[k] = Tb * pow(s.p_mid[k] / pb, KAPPA);
    s.qp[k] = qb;
    s.b[k] = s.Tp[k] * (1.0 + ZVIR * s.qp[k]) - s.Tv[k];
  }
  int kel = -1;
  for (int k = ktl; k <= klcl; ++k)
    if (val(s.b[k]) > 0.0) { kel = k; break; }
  s.kel = kel;
  mark_trigger_end<R>();
  if (kel < 0) return;
  R cape(0.0);
  for (int k = klcl; k >= kel; --k) cape = cape + RD * s.b[k] * s.dlnp[k];
  island<R>(I_CAPE, klcl - kel + 1);
  if (val(cape) < 0.0) cape = R(0.0);
  s.cape = cape;
  mark_trigger_end<R>();
  if (!(val(cape) > P.capelmt)) return;
  s.triggered = true;

  // Shallowest admissible detrainment level: minimum h* above the LCL (ties:
  // lowest); a plume is carried through any layer below it.
  int khmin = -1;
  for (int k = klcl - 1; k >= ktl; --k)
    if (khmin < 0 || val(s.hs[k]) < val(s.hs[khmin])) khmin = k;
  s.khmin = khmin;
  // Entraining updraft (entrainment loop).  Variant (n_plumes > 1): a spectrum
  // of plumes with entrainment rates lambda * spread^(i/(n-1) - 1/2), each
  // carrying the share 1/n of the cloud-base mass flux and detraining at its
  // own top; a plume whose top is at or below the LCL layer drops out.  The
  // unit tendencies of every plume are summed here; the ensemble's top (the
  // highest plume top) starts the downdraft.  n_plumes = 1 is the bulk plume.
  const int NP = P.n_plumes;
  int jt = -1;
  R sumR(0.0);
  for (int ip = 0; ip < NP; ++ip) {
    R lam_i = lambda;
    double w = 1.0;
    if (NP > 1) {
      lam_i = lambda * std::pow(P.plume_spread, (double)ip / (NP - 1) - 0.5);
      w = 1.0 / NP;
    }
    s.eta[kb] = R(1.0);
    s.hu[kb] = s.h[kb];
    s.qtu[kb] = q[kb];
    int jt_i = -1;
    R sumR_i(0.0);
    for (int k = kb - 1; k >= ktl; --k) {
      s.eta[k] = entrain_growth(lam_i, P.ent_zscale, s.z_mid[k] - s.z_mid[kb]);
      const R deta = s.eta[k] - s.eta[k + 1];
      s.hu[k] = (s.eta[k + 1] * s.hu[k + 1] + deta * s.h[k]) / s.eta[k];
      if ((k <= khmin && val(s.hu[k]) <= val(s.hs[k])) || k == ktl) {
        jt_i = k;
        break;
      }
      const R qt = (s.eta[k + 1] * s.qtu[k + 1] + deta * q[k]) / s.eta[k];
      double st = 0.0;
      const R Tsat = moist_invert(s.hu[k], GRAV * s.z_mid[k], s.p_mid[k], T[k], P.n_h, &st);
      s.newton_max = std::max(s.newton_max, st);
      const R qsu = sat_qs(Tsat, s.p_mid[k]);
      R l = qt - qsu;
      if (val(l) < 0.0) l = R(0.0);
      const R dz = s.z_int[k] - s.z_int[k + 1];
      s.rain[k] = s.eta[k] * P.c0 * dz * l / (1.0 + P.c0 * dz);
      s.qtu[k] = qt - s.rain[k] / s.eta[k];
      sumR_i = sumR_i + s.rain[k];
    }
    if (jt_i < 0 || jt_i >= klcl) continue;  // no cloud above the LCL
    if (jt < 0 || jt_i < jt) jt = jt_i;
    sumR = sumR + w * sumR_i;
    // this plume's environment tendencies per unit M_b (flux form, upwind
    // subsidence below its top, detrainment at its top)
    for (int k = jt_i + 1; k <= kb; ++k) {
      s.dh[k] = s.dh[k] + (w * s.eta[k]) * (s.h[k - 1] - s.h[k]);
      s.dq[k] = s.dq[k] + (w * s.eta[k]) * (q[k - 1] - q[k]);
    }
    s.dh[jt_i] = s.dh[jt_i] + (w * s.eta[jt_i + 1]) * (s.hu[jt_i + 1] - s.h[jt_i]);
    s.dq[jt_i] = s.dq[jt_i] + (w * s.eta[jt_i + 1]) * (s.qtu[jt_i + 1] - q[jt_i]);
  }
  s.jt = jt;
  s.sumR = sumR;
  if (jt < 0) return;

  // Downdraft (precipitation loop): starts at the minimum-h* level above the LCL.
  int jd = -1;
  for (int k = klcl - 1; k > jt; --k)
    if (jd < 0 || val(s.hs[k]) < val(s.hs[jd])) jd = k;
  s.jd = jd;
  R sumE(0.0);
  R alpha(0.0);
  if (jd >= 0) {
    for (int k = jd; k <= kb - 1; ++k)
      s.etad[k] = entrain_growth(lambda, P.ent_zscale, s.z_mid[jd] - s.z_mid[k]);
    s.hd[jd] = s.h[jd];
    for (int k = jd + 1; k <= kb - 1; ++k)
      s.hd[k] = (s.etad[k - 1] * s.hd[k - 1] + (s.etad[k] - s.etad[k - 1]) * s.h[k]) / s.etad[k];
    for (int k = jd; k <= kb - 1; ++k) {
      double st = 0.0;
      const R Td = moist_invert(s.hd[k], GRAV * s.z_mid[k], s.p_mid[k], T[k], P.n_h, &st);
      s.newton_max = std::max(s.newton_max, st);
      s.qd[k] = sat_qs(Td, s.p_mid[k]);
    }
    s.E1[jd] = s.etad[jd] * (s.qd[jd] - q[jd]);
    for (int k = jd + 1; k <= kb - 1; ++k)
      s.E1[k] = s.etad[k] * s.qd[k] - s.etad[k - 1] * s.qd[k - 1] - (s.etad[k] - s.etad[k - 1]) * q[k];
    for (int k = jd; k <= kb - 1; ++k) sumE = sumE + s.E1[k];
    alpha = R(P.alpha_dd);
    if (val(alpha * sumE) > val(sumR)) alpha = sumR / sumE;
  }
  s.sumE = sumE;
  s.alpha = alpha;

  // Environment tendencies per unit M_b: the plumes' terms are in already; the
  // downdraft's compensating ascent and its detrainment into the launch layer.
  if (jd >= 0) {
    for (int k = jd; k <= kb - 1; ++k) {
      const R D = alpha * s.etad[k];
      s.dh[k] = s.dh[k] + D * (s.h[k + 1] - s.h[k]);
      s.dq[k] = s.dq[k] + D * (q[k + 1] - q[k]);
    }
    const R D = alpha * s.etad[kb - 1];
    s.dh[kb] = s.dh[kb] + D * (s.hd[kb - 1] - s.h[kb]);
    s.dq[kb] = s.dq[kb] + D * (s.qd[kb - 1] - q[kb]);
  }
  for (int k = jt; k <= kb; ++k) {
    s.dh[k] = s.dh[k] / s.m[k];
    s.dq[k] = s.dq[k] / s.m[k];
    s.dT[k] = (s.dh[k] - LV * s.dq[k]) / CP;
  }

  // Closure: F = d(CAPE)/d(M_b) with the parcel path and level indices fixed.
  R F(0.0);
  for (int k = klcl; k >= kel; --k) {
    R qsp, dqsp;
    sat_qs_dqs(s.Tp[k], s.p_mid[k], qsp, dqsp);
    const R dTvp = ((1.0 + ZVIR * qsp) + ZVIR * s.Tp[k] * dqsp) / (CP + LV * dqsp);
    const R dTv = (1.0 + ZVIR * q[k]) * s.dT[k] + ZVIR * T[k] * s.dq[k];
    F = F + RD * s.dlnp[k] * (dTvp * s.dh[kb] - dTv);
  }
  s.F = F;
  if (!(val(F) < 0.0)) return;
  R mb = -cape / (tau * F);
  for (int k = 0; k < pver; ++k) {
    if (val(s.dq[k]) < 0.0) {
      const R ml = (q[k] - P.q_min) / (-dt * s.dq[k]);
      if (val(ml) < val(mb)) {
        mb = ml;
        s.limited = true;
      }
    }
  }
  if (!(val(mb) > 0.0)) {
    s.limited = false;
    return;
  }
  s.active = true;
  s.mb = mb;
  island<R>(I_CONS, 2.0 * (kb - jt + 1));
  for (int k = 0; k < pver; ++k) {
    s.dTdt[k] = mb * s.dT[k];
    s.dqdt[k] = mb * s.dq[k];
  }
  R net = sumR - alpha * sumE;
  if (val(net) < 0.0) net = R(0.0);
  s.prec = mb * net;

  // Column conservation residual (enthalpy and water), FP64.
  double se = 0.0, sw = 0.0, scale = 0.0;
  for (int k = 0; k < pver; ++k) {
    se += val(s.m[k]) * CP * val(s.dTdt[k]);
    sw += val(s.m[k]) * val(s.dqdt[k]);
    scale += val(s.m[k]) * CP * std::fabs(val(s.dTdt[k]));
  }
  const double P_ = val(s.prec);
  s.cons_err = (std::fabs(se - LV * P_) + LV * std::fabs(sw + P_)) / (scale + LV * P_ + 1e-300);
}

// ---------------------------------------------------------------- shallow scheme
template <class R>
struct ShalState {
  int ktl = -1, klcl = -1, klfc = -1, kts = -1, exit_code = 0;
  bool triggered = false, active = false, bad = false;
  double newton_max = 0.0;
  R TL, pL, cin, mb, prec;
  R b[MAXLEV], hu[MAXLEV], qtu[MAXLEV], qtpre[MAXLEV], w2[MAXLEV], rf[MAXLEV], Tu[MAXLEV];
  R dh[MAXLEV], dq[MAXLEV], dT[MAXLEV];
  R m[MAXLEV], z_mid[MAXLEV], z_int[MAXLEV + 1], h[MAXLEV], p_mid[MAXLEV], p_int[MAXLEV + 1],
      dlnp[MAXLEV], Tv[MAXLEV];
  double cons_err = 0.0;
};

// Shallow convection of one column (Sec. II-A; Alg. 3 with its early exits).
//  Source = lowest layer.  E1: LCL pressure below p_lcl_min.  Undilute parcel;
//  LFC = first positively buoyant level at or above the LCL, scanning up; E2: no
//  LFC at pressures >= p_lfc_min.  CIN = sum of Rd max(0,-b) dln p from the
//  source up to (not including) the LFC; E3: CIN > cin_max.  Closure M_b =
//  rho_src c_m sqrt(tke) exp(-CIN/(cin_scale tke)).  Constant-mass-flux plume,
//  undilute up to the LCL layer, above it relaxing towards the environment by
//  1 - exp(-eps_s dz) per layer; rain = M_b max(0, l - ql_crit).  The
//  closure's exp(-CIN/...) factor already selects the updrafts strong enough to
//  cross the CIN, so w2 = (2/3) tke from the source up to the LFC layer; above
//  it w2 follows dw2/dz = 2 a B - 2 b eps_s w2, integrated exactly across each
//  layer with the layer's plume buoyancy B = g (Tv_u - Tv)/Tv held fixed; cloud
//  top kts = highest layer of the run with w2 > 0; E4: kts at or below the LCL
//  layer.  Exits leave every output zero.
template <class R>
void shallow_column(int pver, const double* hyai, const double* hybi, double p0, const R* T,
                    const R* q, const R& ps, const ShalP& P, ShalState<R>& s) {
  using std::exp;
  using std::pow;
  using std::sqrt;
  s.TL = s.pL = s.cin = s.mb = s.prec = R(0.0);
  for (int k = 0; k < pver; ++k) {
    s.b[k] = s.hu[k] = s.qtu[k] = s.qtpre[k] = s.w2[k] = s.rf[k] = s.Tu[k] = R(0.0);
    s.dh[k] = s.dq[k] = s.dT[k] = R(0.0);
  }
  if (!column_valid(pver, T, q, ps)) {
    s.bad = true;
    return;
  }
  levels(pver, hyai, hybi, p0, ps, s.p_int, s.p_mid);
  heights(pver, T, q, s.p_int, s.p_mid, s.z_int, s.z_mid, s.dlnp, s.Tv);
  for (int k = 0; k < pver; ++k) {
    s.m[k] = (s.p_int[k + 1] - s.p_int[k]) / GRAV;
    s.h[k] = CP * T[k] + GRAV * s.z_mid[k] + LV * q[k];
  }
  int ktl = pver - 1;
  for (int k = 0; k < pver; ++k)
    if (val(s.p_mid[k]) >= P.p_top_lim) { ktl = k; break; }
  s.ktl = ktl;

  const int ks = pver - 1;
  const R Ts = T[ks], qsrc = q[ks], psrc = s.p_mid[ks];
  s.newton_max = std::max(s.newton_max, lcl(Ts, qsrc, psrc, P.n_lcl, s.TL, s.pL));
  island<R>(I_LCL, 1);
  const int klcl = lcl_level(s.p_mid, ks, s.pL);
  s.klcl = klcl;
  if (val(s.pL) < P.p_lcl_min || klcl < ktl) { s.exit_code = 1; return; }

  // Undilute parcel from the source up to the LFC search limit.
  int klfc = -1;
  mark_lfc_search<R>(false);
  for (int k = ks; k >= ktl && val(s.p_mid[k]) >= P.p_lfc_min; --k) {
    R Tp, qp;
    if (k > klcl) {
      Tp = Ts * pow(s.p_mid[k] / psrc, KAPPA);
      qp = qsrc;
    } else {
      double st = 0.0;
      Tp = moist_invert(s.h[ks], GRAV * s.z_mid[k], s.p_mid[k], T[k], P.n_h, &st);
      s.newton_max = std::max(s.newton_max, st);
      qp = sat_qs(Tp, s.p_mid[k]);
    }
    s.b[k] = Tp * (1.0 + ZVIR * qp) - s.Tv[k];
    if (k <= klcl && val(s.b[k]) > 0.0) { klfc = k; break; }
  }
  mark_lfc_search<R>(true);
  s.klfc = klfc;
  if (klfc < 0) { s.exit_code = 2; return; }
  R cin(0.0);
  for (int k = ks; k > klfc; --k) {
    R neg = -s.b[k];
    if (val(neg) < 0.0) neg = R(0.0);
    if (val(neg) > 0.0) island<R>(I_CIN, 1);
    cin = cin + RD * neg * s.dlnp[k];
  }
  s.cin = cin;
  if (val(cin) > P.cin_max) { s.exit_code = 3; return; }
  s.triggered = true;
  const R rho = psrc / (RD * s.Tv[ks]);
  const R mb = rho * P.c_m * std::sqrt(P.tke) * exp(-cin / (P.cin_scale * P.tke));

  // Plume.
  s.hu[ks] = s.h[ks];
  s.qtu[ks] = qsrc;
  s.qtpre[ks] = qsrc;
  s.Tu[ks] = Ts;
  const double w2_0 = 2.0 / 3.0 * P.tke;
  s.w2[ks] = R(w2_0);
  int kts = -1;
  for (int k = ks - 1; k >= ktl; --k) {
    const R dz = s.z_int[k] - s.z_int[k + 1];
    R qt;
    if (k >= klcl) {
      s.hu[k] = s.hu[k + 1];
      qt = s.qtu[k + 1];
    } else {
      const R chi = 1.0 - exp(-P.eps_s * dz);
      s.hu[k] = s.hu[k + 1] + chi * (s.h[k] - s.hu[k + 1]);
      qt = s.qtu[k + 1] + chi * (q[k] - s.qtu[k + 1]);
    }
    s.qtpre[k] = qt;
    const R gz = GRAV * s.z_mid[k];
    double st = 0.0;
    const R Tsat = moist_invert(s.hu[k], gz, s.p_mid[k], T[k], P.n_h, &st);
    s.newton_max = std::max(s.newton_max, st);
    const R qsu = sat_qs(Tsat, s.p_mid[k]);
    R Tu, qv;
    if (val(qt) >= val(qsu)) {
      Tu = Tsat;
      qv = qsu;
    } else {
      Tu = (s.hu[k] - gz - LV * qt) / CP;
      qv = qt;
    }
    s.Tu[k] = Tu;
    const R l = qt - qv;
    const R B = GRAV * (Tu * (1.0 + ZVIR * qv) - s.Tv[k]) / s.Tv[k];
    if (k >= klfc) {
      s.w2[k] = w2_0;
    } else {
      // dw2/dz = 2 a B - 2 b eps_s w2 integrated exactly over the layer (B constant).
      const double beps = P.b_w * P.eps_s;
      if (beps > 0.0) {
        const R decay = exp(-2.0 * beps * dz);
        s.w2[k] = s.w2[k + 1] * decay + (P.a_w / beps) * B * (1.0 - decay);
      } else {
        s.w2[k] = s.w2[k + 1] + 2.0 * P.a_w * B * dz;
      }
      if (!(val(s.w2[k]) > 0.0)) { kts = k + 1; break; }
    }
    if (k == ktl) { kts = k; break; }
    if (val(qt) >= val(qsu) && std::fabs(val(l) - P.ql_crit) < 1e-4) island<R>(I_DRIZZLE, 1);
    R r = l - P.ql_crit;
    if (val(r) < 0.0) r = R(0.0);
    s.rf[k] = r;
    s.qtu[k] = qt - r;
  }
  s.kts = kts;
  if (kts < 0 || kts >= klcl) {
    s.exit_code = 4;
    s.triggered = true;
    return;
  }
  s.active = true;
  s.mb = mb;
  island<R>(I_CONS, 2.0 * (ks - kts + 1));

  // Tendencies: m_k dphi_k = [U_k+1 phi_u,k+1 - U_k phi~_k] + [U_k phi_k-1 - U_k+1 phi_k],
  // U = M_b through the interfaces kts+1..ks, phi~ the pre-rain plume value.
  s.dh[ks] = mb * (s.h[ks - 1] - s.h[ks]);
  s.dq[ks] = mb * (q[ks - 1] - q[ks]);
  for (int k = kts + 1; k <= ks - 1; ++k) {
    s.dh[k] = mb * ((s.hu[k + 1] - s.hu[k]) + (s.h[k - 1] - s.h[k]));
    s.dq[k] = mb * ((s.qtu[k + 1] - s.qtpre[k]) + (q[k - 1] - q[k]));
  }
  s.dh[kts] = mb * (s.hu[kts + 1] - s.h[kts]);
  s.dq[kts] = mb * (s.qtu[kts + 1] - q[kts]);
  for (int k = kts; k <= ks; ++k) {
    s.dh[k] = s.dh[k] / s.m[k];
    s.dq[k] = s.dq[k] / s.m[k];
    s.dT[k] = (s.dh[k] - LV * s.dq[k]) / CP;
  }
  R sumr(0.0);
  for (int k = ks - 1; k > kts; --k) sumr = sumr + s.rf[k];
  s.prec = mb * sumr;

  // Variant (off when evap_k = 0): evaporation of the falling rain.  Rain made
  // in plume layer k (kts < k < ks) falls through the environment layers below
  // it; each layer j takes the fraction 1 - exp(-evap_k max(qs_j - q_j, 0) dz_j)
  // of the flux arriving from above, which moistens and cools that layer
  // (dq = E/m, dT = -Lv E/(cp m)); what reaches the surface is the precipitation.
  if (P.evap_k > 0.0) {
    R F(0.0);
    for (int j = kts + 1; j <= ks; ++j) {
      const R dz = s.z_int[j] - s.z_int[j + 1];
      R def = sat_qs(T[j], s.p_mid[j]) - q[j];
      if (val(def) < 0.0) def = R(0.0);
      const R E = F * (1.0 - exp(-P.evap_k * def * dz));
      F = F - E;
      s.dq[j] = s.dq[j] + E / s.m[j];
      s.dT[j] = s.dT[j] - LV * E / (CP * s.m[j]);
      if (j < ks) F = F + mb * s.rf[j];
    }
    s.prec = F;
  }

  double se = 0.0, sw = 0.0, scale = 0.0;
  for (int k = 0; k < pver; ++k) {
    se += val(s.m[k]) * CP * val(s.dT[k]);
    sw += val(s.m[k]) * val(s.dq[k]);
    scale += val(s.m[k]) * CP * std::fabs(val(s.dT[k]));
  }
  const double P_ = val(s.prec);
  s.cons_err = (std::fabs(se - LV * P_) + LV * std::fabs(sw + P_)) / (scale + LV * P_ + 1e-300);
}

// ---------------------------------------------------------------- tracer transport
// Convective transport of passive tracers (a variant both cited schemes carry,
// Sec. II-A: ZM and UW move constituents with their plume mass fluxes; the paper
// itself times only the thermodynamic loops).  This project's reading: a tracer
// c (mixing ratio) is mixed exactly like each scheme's conserved moist static
// energy in its own flux-form tendency equations above, with no source term
// (no rain-out, no phase change), so every step below repeats the matching MSE
// step with h replaced by c.  Inactive columns have zero tendencies.
//
// Mass-flux profiles (kg m-2 s-1) that describe the same transport:
//   mu[k]  updraft mass flux leaving layer k through its top interface;
//   du[k]  updraft air detrained into layer k, carrying the plume value
//          arriving from layer k+1;
//   md[k]  downdraft mass flux leaving layer k through its bottom interface
//          (downward positive); the downdraft detrains all of it into the layer
//          below its lowest level.
// Deep: mu = M_b eta on jt+1..kb, du[jt] = M_b eta[jt+1], md = M_b alpha etad
// on jd..kb-1.  Shallow: mu = M_b on kts+1..ks, du = M_b (1 - exp(-eps dz)) on
// kts+1..klcl-1 and du[kts] = M_b, md = 0.

// Deep tracer tendency of one column (s from deep_column; c this column's tracer).
void deep_transport(int pver, const DeepState<double>& s, const double* c, double* tend) {
  for (int k = 0; k < pver; ++k) tend[k] = 0.0;
  if (!s.active) return;
  const int kb = s.kb, jt = s.jt, jd = s.jd;
  double cu[MAXLEV], cd[MAXLEV], dc[MAXLEV];
  for (int k = 0; k < pver; ++k) cu[k] = cd[k] = dc[k] = 0.0;
  // updraft, mixed as the plume MSE is
  cu[kb] = c[kb];
  for (int k = kb - 1; k > jt; --k)
    cu[k] = (s.eta[k + 1] * cu[k + 1] + (s.eta[k] - s.eta[k + 1]) * c[k]) / s.eta[k];
  // downdraft, mixed as the downdraft MSE is
  if (jd >= 0) {
    cd[jd] = c[jd];
    for (int k = jd + 1; k <= kb - 1; ++k)
      cd[k] = (s.etad[k - 1] * cd[k - 1] + (s.etad[k] - s.etad[k - 1]) * c[k]) / s.etad[k];
  }
  // flux-form terms per unit M_b: subsidence, detrainment at the top, the
  // downdraft's compensating ascent and its detrainment into the launch layer
  for (int k = jt + 1; k <= kb; ++k) dc[k] = dc[k] + s.eta[k] * (c[k - 1] - c[k]);
  dc[jt] = dc[jt] + s.eta[jt + 1] * (cu[jt + 1] - c[jt]);
  if (jd >= 0) {
    for (int k = jd; k <= kb - 1; ++k) dc[k] = dc[k] + s.alpha * s.etad[k] * (c[k + 1] - c[k]);
    dc[kb] = dc[kb] + s.alpha * s.etad[kb - 1] * (cd[kb - 1] - c[kb]);
  }
  for (int k = jt; k <= kb; ++k) tend[k] = s.mb * (dc[k] / s.m[k]);
}

// Shallow tracer tendency of one column (s from shallow_column on the state the
// shallow scheme saw; c the tracer it sees).
void shallow_transport(int pver, const ShalState<double>& s, const ShalP& P, const double* c,
                       double* tend) {
  for (int k = 0; k < pver; ++k) tend[k] = 0.0;
  if (!s.active) return;
  const int ks = pver - 1, kts = s.kts;
  double cu[MAXLEV], dc[MAXLEV];
  for (int k = 0; k < pver; ++k) cu[k] = dc[k] = 0.0;
  // constant-mass-flux plume: undilute up to the LCL layer, relaxing towards
  // the environment by 1 - exp(-eps dz) per layer above it
  cu[ks] = c[ks];
  for (int k = ks - 1; k > kts; --k) {
    if (k >= s.klcl) {
      cu[k] = cu[k + 1];
    } else {
      const double dz = s.z_int[k] - s.z_int[k + 1];
      const double chi = 1.0 - std::exp(-P.eps_s * dz);
      cu[k] = cu[k + 1] + chi * (c[k] - cu[k + 1]);
    }
  }
  dc[ks] = s.mb * (c[ks - 1] - c[ks]);
  for (int k = kts + 1; k <= ks - 1; ++k)
    dc[k] = s.mb * ((cu[k + 1] - cu[k]) + (c[k - 1] - c[k]));
  dc[kts] = s.mb * (cu[kts + 1] - c[kts]);
  for (int k = kts; k <= ks; ++k) tend[k] = dc[k] / s.m[k];
}

// ---------------------------------------------------------------- momentum transport
// Convective momentum transport (a variant the cited schemes carry, Sec. II-A:
// the ZM and UW schemes move horizontal momentum with their plumes).  This
// project's reading: a wind component is carried like a tracer, except that
// inside a plume the convective-scale pressure gradient pushes the plume's
// momentum towards the environment's by a fraction of the environmental wind
// change it rises (or sinks) through -- the pressure-gradient term of Gregory,
// Kershaw and Inness (1997, Q. J. R. Meteorol. Soc. 123), with coefficients
// c_up (updrafts) and c_down (downdraft); with both 0 this is the tracer
// transport.  Discretely, per unit cloud-base flux: a plume crossing layer k from
// its neighbour j (k+1 for updrafts, k-1 for the downdraft) gains
// c (flux continuing from j) (u_k - u_j) on top of the mixing of the tracer
// recurrence.  The environment's tendency is the divergence of the eddy fluxes
// through the layer interfaces, with the upwind values of the tracer transport:
//   updraft, interface k (top of layer k):  F_k = eta_k (u_u,k - u_k-1), jt < k <= kb,
//   downdraft, interface k+1 (bottom of k): G_k+1 = alpha etad_k (u_d,k - u_k+1), jd <= k < kb,
//   m_k du_k/dt = M_b [(F_k+1 - F_k) + (G_k - G_k+1)],
// zero through the top of the cloud-top layer, the bottom of the launch layer
// and the top of the downdraft's first layer; so the column's momentum is
// conserved exactly, whatever the coefficients.  Equivalently: the tracer
// tendency with the plumes' momenta, minus the pressure force each plume exerts
// in each layer it crosses.

// Deep momentum tendency of one column for one wind component c.
void deep_momentum(int pver, const DeepState<double>& s, const double* c, double c_up,
                   double c_down, double* tend) {
  for (int k = 0; k < pver; ++k) tend[k] = 0.0;
  if (!s.active) return;
  const int kb = s.kb, jt = s.jt, jd = s.jd;
  double cu[MAXLEV], cd[MAXLEV], F[MAXLEV + 1], G[MAXLEV + 1];
  for (int k = 0; k <= pver; ++k) F[k] = G[k] = 0.0;
  for (int k = 0; k < pver; ++k) cu[k] = cd[k] = 0.0;
  cu[kb] = c[kb];
  for (int k = kb - 1; k > jt; --k)
    cu[k] = (s.eta[k + 1] * (cu[k + 1] + c_up * (c[k] - c[k + 1])) +
             (s.eta[k] - s.eta[k + 1]) * c[k]) / s.eta[k];
  for (int k = jt + 1; k <= kb; ++k) F[k] = s.eta[k] * (cu[k] - c[k - 1]);
  if (jd >= 0) {
    cd[jd] = c[jd];
    for (int k = jd + 1; k <= kb - 1; ++k)
      cd[k] = (s.etad[k - 1] * (cd[k - 1] + c_down * (c[k] - c[k - 1])) +
               (s.etad[k] - s.etad[k - 1]) * c[k]) / s.etad[k];
    for (int k = jd; k <= kb - 1; ++k) G[k + 1] = s.alpha * s.etad[k] * (cd[k] - c[k + 1]);
  }
  for (int k = jt; k <= kb; ++k)
    tend[k] = s.mb * (((F[k + 1] - F[k]) + (G[k] - G[k + 1])) / s.m[k]);
}

// Shallow momentum tendency of one column (s from shallow_column on the state
// the shallow scheme saw; c the wind component it sees).
void shallow_momentum(int pver, const ShalState<double>& s, const ShalP& P, const double* c,
                      double c_up, double* tend) {
  for (int k = 0; k < pver; ++k) tend[k] = 0.0;
  if (!s.active) return;
  const int ks = pver - 1, kts = s.kts;
  double cu[MAXLEV], F[MAXLEV + 1];
  for (int k = 0; k <= pver; ++k) F[k] = 0.0;
  cu[ks] = c[ks];
  for (int k = ks - 1; k > kts; --k) {
    const double ustar = cu[k + 1] + c_up * (c[k] - c[k + 1]);
    if (k >= s.klcl) {
      cu[k] = ustar;
    } else {
      const double dz = s.z_int[k] - s.z_int[k + 1];
      const double chi = 1.0 - std::exp(-P.eps_s * dz);
      cu[k] = ustar + chi * (c[k] - ustar);
    }
  }
  for (int k = kts + 1; k <= ks; ++k) F[k] = s.mb * (cu[k] - c[k - 1]);
  for (int k = kts; k <= ks; ++k) tend[k] = (F[k + 1] - F[k]) / s.m[k];
}

void deep_fluxes(int pver, const DeepState<double>& s, double* mu, double* du, double* md) {
  for (int k = 0; k < pver; ++k) mu[k] = du[k] = md[k] = 0.0;
  if (!s.active) return;
  for (int k = s.jt + 1; k <= s.kb; ++k) mu[k] = s.mb * s.eta[k];
  du[s.jt] = s.mb * s.eta[s.jt + 1];
  if (s.jd >= 0)
    for (int k = s.jd; k <= s.kb - 1; ++k) md[k] = s.mb * s.alpha * s.etad[k];
}

void shallow_fluxes(int pver, const ShalState<double>& s, const ShalP& P, double* mu, double* du,
                    double* md) {
  for (int k = 0; k < pver; ++k) mu[k] = du[k] = md[k] = 0.0;
  if (!s.active) return;
  const int ks = pver - 1;
  for (int k = s.kts + 1; k <= ks; ++k) mu[k] = s.mb;
  for (int k = s.kts + 1; k <= s.klcl - 1 && k <= ks - 1; ++k) {
    const double dz = s.z_int[k] - s.z_int[k + 1];
    du[k] = s.mb * (1.0 - std::exp(-P.eps_s * dz));
  }
  du[s.kts] = s.mb;
}

void store_flux(const oracle_flux* f, int pver, int ld, int i, const double* mu, const double* du,
                const double* md) {
  if (!f) return;
  for (int k = 0; k < pver; ++k) {
    if (f->mu) f->mu[k * ld + i] = mu[k];
    if (f->du) f->du[k * ld + i] = du[k];
    if (f->md) f->md[k * ld + i] = md[k];
  }
}

// ---------------------------------------------------------------- grid drivers
inline void set_i(int32_t* a, int i, int v) { if (a) a[i] = v; }
inline void set_d(double* a, int i, double v) { if (a) a[i] = v; }

template <class R>
void store_deep(const DeepState<R>& s, int pver, int ld, int i, const oracle_out* o) {
  for (int k = 0; k < pver; ++k) {
    set_d(o->dTdt, k * ld + i, val(s.dTdt[k]));
    set_d(o->dqdt, k * ld + i, val(s.dqdt[k]));
  }
  set_d(o->prec, i, val(s.prec));
  int fl = 0;
  if (s.bad) fl |= F_BADINPUT;
  if (s.triggered) fl |= F_TRIGGERED;
  if (s.active) fl |= F_ACTIVE;
  if (s.limited) fl |= F_LIMITED;
  if (s.newton_max > NEWTON_FLAG_TOL) fl |= F_NEWTON;
  set_i(o->flags, i, fl);
  set_i(o->kb, i, s.kb);
  set_i(o->klcl, i, s.klcl);
  set_i(o->ktop, i, s.active ? s.jt : -1);
  set_i(o->kaux, i, s.active ? s.jd : -1);
  set_d(o->cape, i, val(s.cape));
  set_d(o->mb, i, val(s.mb));
  set_d(o->cons_err, i, s.cons_err);
}

template <class R>
void store_shallow(const ShalState<R>& s, int pver, int ld, int i, const oracle_out* o) {
  for (int k = 0; k < pver; ++k) {
    set_d(o->dTdt, k * ld + i, s.active ? val(s.dT[k]) : 0.0);
    set_d(o->dqdt, k * ld + i, s.active ? val(s.dq[k]) : 0.0);
  }
  set_d(o->prec, i, s.active ? val(s.prec) : 0.0);
  int fl = 0;
  if (s.bad) fl |= F_BADINPUT;
  if (s.triggered) fl |= F_TRIGGERED;
  if (s.active) fl |= F_ACTIVE;
  if (s.newton_max > NEWTON_FLAG_TOL) fl |= F_NEWTON;
  fl |= s.exit_code << EXIT_SHIFT;
  set_i(o->flags, i, fl);
  set_i(o->kb, i, s.bad ? -1 : pver - 1);
  set_i(o->klcl, i, s.klcl);
  set_i(o->ktop, i, s.active ? s.kts : -1);
  set_i(o->kaux, i, s.klfc);
  set_d(o->cape, i, val(s.cin));
  set_d(o->mb, i, s.active ? val(s.mb) : 0.0);
  set_d(o->cons_err, i, s.active ? s.cons_err : 0.0);
}

bool grid_ok(int n_cols, int pver, int ld) {
  return n_cols >= 0 && pver >= 4 && pver <= MAXLEV && ld >= n_cols;
}

int threads_for(int n) { return n < 1 ? 1 : n; }

}  // namespace

// ================================================================ C interface
extern "C" {

double oracle_es(double T) { return sat_es(T); }
double oracle_qs(double T, double p) { return sat_qs(T, p); }
double oracle_dqsdT(double T, double p) {
  double qs, dqs;
  sat_qs_dqs(T, p, qs, dqs);
  return dqs;
}
double oracle_lcl(double Tb, double qb, double pb, int n_newton, double* TL, double* pL) {
  return lcl(Tb, qb, pb, n_newton, *TL, *pL);
}
double oracle_hinv(double h, double gz, double p, double T_start, int n_extra, double* last_step) {
  return moist_invert(h, gz, p, T_start, n_extra, last_step);
}
void oracle_heights(int pver, const double* T, const double* q, const double* p_int,
                    const double* p_mid, double* z_int, double* z_mid) {
  double dlnp[MAXLEV], Tv[MAXLEV];
  heights(pver, T, q, p_int, p_mid, z_int, z_mid, dlnp, Tv);
}
void oracle_levels(int pver, const double* hyai, const double* hybi, double p0, double ps,
                   double* p_int, double* p_mid) {
  levels(pver, hyai, hybi, p0, ps, p_int, p_mid);
}

void oracle_deep_column_diag(int pver, const double* hyai, const double* hybi, double p0,
                             const double* T, const double* q, double ps, double lambda,
                             double tau, const oracle_deep_params* par, double dt,
                             oracle_deep_diag* d) {
  DeepState<double> s;
  deep_column<double>(pver, hyai, hybi, p0, T, q, ps, lambda, tau, to_deep(par), dt, s);
  std::memset(d, 0, sizeof *d);
  d->k_top_lim = s.ktl; d->kb = s.kb; d->klcl = s.klcl; d->kel = s.kel; d->khmin = s.khmin;
  d->jt = s.jt;
  d->jd = s.jd; d->triggered = s.triggered; d->active = s.active; d->limited = s.limited;
  d->TL = s.TL; d->pL = s.pL; d->cape = s.cape; d->F = s.F; d->mb = s.mb; d->sumR = s.sumR;
  d->sumE = s.sumE; d->alpha_eff = s.alpha; d->prec = s.prec;
  for (int k = 0; k < pver; ++k) {
    d->Tp[k] = s.Tp[k]; d->qp[k] = s.qp[k]; d->b[k] = s.b[k]; d->eta[k] = s.eta[k];
    d->hu[k] = s.hu[k]; d->qtu[k] = s.qtu[k]; d->rain[k] = s.rain[k]; d->etad[k] = s.etad[k];
    d->hd[k] = s.hd[k]; d->qd[k] = s.qd[k]; d->E1[k] = s.E1[k]; d->dh[k] = s.dh[k];
    d->dq[k] = s.dq[k]; d->dT[k] = s.dT[k]; d->m[k] = s.m[k]; d->z_mid[k] = s.z_mid[k];
    d->h[k] = s.h[k]; d->hs[k] = s.hs[k]; d->p_mid[k] = s.p_mid[k];
  }
  for (int k = 0; k <= pver; ++k) { d->z_int[k] = s.z_int[k]; d->p_int[k] = s.p_int[k]; }
}

void oracle_shallow_column_diag(int pver, const double* hyai, const double* hybi, double p0,
                                const double* T, const double* q, double ps,
                                const oracle_shallow_params* par, oracle_shallow_diag* d) {
  ShalState<double> s;
  shallow_column<double>(pver, hyai, hybi, p0, T, q, ps, to_shal(par), s);
  std::memset(d, 0, sizeof *d);
  d->k_top_lim = s.ktl; d->klcl = s.klcl; d->klfc = s.klfc; d->kts = s.kts;
  d->exit_code = s.exit_code; d->active = s.active;
  d->TL = s.TL; d->pL = s.pL; d->cin = s.cin; d->mb = s.mb; d->prec = s.prec;
  for (int k = 0; k < pver; ++k) {
    d->b[k] = s.b[k]; d->hu[k] = s.hu[k]; d->qtu[k] = s.qtu[k]; d->qtpre[k] = s.qtpre[k];
    d->w2[k] = s.w2[k]; d->rf[k] = s.rf[k]; d->Tu[k] = s.Tu[k]; d->dh[k] = s.dh[k];
    d->dq[k] = s.dq[k]; d->dT[k] = s.dT[k]; d->m[k] = s.m[k]; d->z_mid[k] = s.z_mid[k];
    d->h[k] = s.h[k]; d->p_mid[k] = s.p_mid[k];
  }
  for (int k = 0; k <= pver; ++k) { d->z_int[k] = s.z_int[k]; d->p_int[k] = s.p_int[k]; }
}

int oracle_deep(int n_cols, int pver, int ld, const double* hyai, const double* hybi, double p0,
                const double* T, const double* q, const double* ps, const double* lambda,
                const double* tau, const oracle_deep_params* par, double dt,
                const oracle_out* out, int n_threads) {
  if (!grid_ok(n_cols, pver, ld) || !par || !out) return 1;
  const DeepP P = to_deep(par);
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads_for(n_threads))
  for (int i = 0; i < n_cols; ++i) {
    double Tc[MAXLEV], qc[MAXLEV];
    for (int k = 0; k < pver; ++k) { Tc[k] = T[k * ld + i]; qc[k] = q[k * ld + i]; }
    DeepState<double> s;
    deep_column<double>(pver, hyai, hybi, p0, Tc, qc, ps[i], lambda ? lambda[i] : P.lambda_default,
                        tau ? tau[i] : P.tau_default, P, dt, s);
    store_deep(s, pver, ld, i, out);
  }
  return 0;
}

int oracle_shallow(int n_cols, int pver, int ld, const double* hyai, const double* hybi,
                   double p0, const double* T, const double* q, const double* ps,
                   const oracle_shallow_params* par, const oracle_out* out, int n_threads) {
  if (!grid_ok(n_cols, pver, ld) || !par || !out) return 1;
  const ShalP P = to_shal(par);
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads_for(n_threads))
  for (int i = 0; i < n_cols; ++i) {
    double Tc[MAXLEV], qc[MAXLEV];
    for (int k = 0; k < pver; ++k) { Tc[k] = T[k * ld + i]; qc[k] = q[k * ld + i]; }
    ShalState<double> s;
    shallow_column<double>(pver, hyai, hybi, p0, Tc, qc, ps[i], P, s);
    store_shallow(s, pver, ld, i, out);
  }
  return 0;
}

int oracle_deep_shallow(int n_cols, int pver, int ld, const double* hyai, const double* hybi,
                        double p0, const double* T, const double* q, const double* ps,
                        const double* lambda, const double* tau,
                        const oracle_deep_params* dpar, const oracle_shallow_params* spar,
                        double dt, const oracle_out* deep, const oracle_out* shallow,
                        int n_threads) {
  if (!grid_ok(n_cols, pver, ld) || !dpar || !spar || !deep || !shallow) return 1;
  const DeepP DP = to_deep(dpar);
  const ShalP SP = to_shal(spar);
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads_for(n_threads))
  for (int i = 0; i < n_cols; ++i) {
    double Tc[MAXLEV], qc[MAXLEV], T2[MAXLEV], q2[MAXLEV];
    for (int k = 0; k < pver; ++k) { Tc[k] = T[k * ld + i]; qc[k] = q[k * ld + i]; }
    DeepState<double> s;
    deep_column<double>(pver, hyai, hybi, p0, Tc, qc, ps[i],
                        lambda ? lambda[i] : DP.lambda_default, tau ? tau[i] : DP.tau_default,
                        DP, dt, s);
    store_deep(s, pver, ld, i, deep);
    // Shallow input: the deep-updated state, humidity floored at zero (the deep
    // limiter keeps it >= q_min up to rounding of q - (q - q_min)); a column the
    // deep scheme rejected as bad input is passed on unchanged.
    for (int k = 0; k < pver; ++k) {
      T2[k] = Tc[k] + dt * s.dTdt[k];
      q2[k] = qc[k] + dt * s.dqdt[k];
      if (!s.bad && q2[k] < 0.0) q2[k] = 0.0;
    }
    ShalState<double> t;
    shallow_column<double>(pver, hyai, hybi, p0, T2, q2, ps[i], SP, t);
    store_shallow(t, pver, ld, i, shallow);
  }
  return 0;
}

int oracle_deep_shallow_tracers(int n_cols, int pver, int ld, const double* hyai,
                                const double* hybi, double p0, const double* T, const double* q,
                                const double* ps, const double* lambda, const double* tau,
                                const oracle_deep_params* dpar, const oracle_shallow_params* spar,
                                double dt, int ntr, const double* tracers, double* tend_deep,
                                double* tend_shallow, const oracle_flux* flux_deep,
                                const oracle_flux* flux_shallow, int n_threads) {
  if (!grid_ok(n_cols, pver, ld) || !dpar || !spar || ntr < 0 || (ntr > 0 && !tracers) ||
      (ntr > 0 && (!tend_deep || !tend_shallow)))
    return 1;
  if (dpar->n_plumes > 1) return 1;  // the transport reading covers the bulk plume
  const DeepP DP = to_deep(dpar);
  const ShalP SP = to_shal(spar);
  const size_t tstride = (size_t)pver * ld;
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads_for(n_threads))
  for (int i = 0; i < n_cols; ++i) {
    double Tc[MAXLEV], qc[MAXLEV], T2[MAXLEV], q2[MAXLEV];
    for (int k = 0; k < pver; ++k) { Tc[k] = T[k * ld + i]; qc[k] = q[k * ld + i]; }
    DeepState<double> s;
    deep_column<double>(pver, hyai, hybi, p0, Tc, qc, ps[i],
                        lambda ? lambda[i] : DP.lambda_default, tau ? tau[i] : DP.tau_default,
                        DP, dt, s);
    for (int k = 0; k < pver; ++k) {
      T2[k] = Tc[k] + dt * s.dTdt[k];
      q2[k] = qc[k] + dt * s.dqdt[k];
      if (!s.bad && q2[k] < 0.0) q2[k] = 0.0;
    }
    ShalState<double> t;
    shallow_column<double>(pver, hyai, hybi, p0, T2, q2, ps[i], SP, t);
    double mu[MAXLEV], du[MAXLEV], md[MAXLEV];
    deep_fluxes(pver, s, mu, du, md);
    store_flux(flux_deep, pver, ld, i, mu, du, md);
    shallow_fluxes(pver, t, SP, mu, du, md);
    store_flux(flux_shallow, pver, ld, i, mu, du, md);
    // each tracer: deep transport, then the shallow transport of the
    // deep-updated tracer (floored at zero, as the humidity is)
    for (int n = 0; n < ntr; ++n) {
      double c[MAXLEV], c2[MAXLEV], td[MAXLEV], ts[MAXLEV];
      for (int k = 0; k < pver; ++k) c[k] = tracers[n * tstride + k * ld + i];
      deep_transport(pver, s, c, td);
      for (int k = 0; k < pver; ++k) {
        c2[k] = c[k] + dt * td[k];
        if (c2[k] < 0.0) c2[k] = 0.0;
      }
      shallow_transport(pver, t, SP, c2, ts);
      for (int k = 0; k < pver; ++k) {
        tend_deep[n * tstride + k * ld + i] = td[k];
        tend_shallow[n * tstride + k * ld + i] = ts[k];
      }
    }
  }
  return 0;
}

int oracle_deep_shallow_momentum(int n_cols, int pver, int ld, const double* hyai,
                                 const double* hybi, double p0, const double* T,
                                 const double* q, const double* ps, const double* lambda,
                                 const double* tau, const oracle_deep_params* dpar,
                                 const oracle_shallow_params* spar, double dt, double c_up,
                                 double c_down, const double* uv, double* tend_deep,
                                 double* tend_shallow, int n_threads) {
  if (!grid_ok(n_cols, pver, ld) || !dpar || !spar || !uv || !tend_deep || !tend_shallow)
    return 1;
  if (dpar->n_plumes > 1) return 1;  // the transport reading covers the bulk plume
  const DeepP DP = to_deep(dpar);
  const ShalP SP = to_shal(spar);
  const size_t cstride = (size_t)pver * ld;
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads_for(n_threads))
  for (int i = 0; i < n_cols; ++i) {
    double Tc[MAXLEV], qc[MAXLEV], T2[MAXLEV], q2[MAXLEV];
    for (int k = 0; k < pver; ++k) { Tc[k] = T[k * ld + i]; qc[k] = q[k * ld + i]; }
    DeepState<double> s;
    deep_column<double>(pver, hyai, hybi, p0, Tc, qc, ps[i],
                        lambda ? lambda[i] : DP.lambda_default, tau ? tau[i] : DP.tau_default,
                        DP, dt, s);
    for (int k = 0; k < pver; ++k) {
      T2[k] = Tc[k] + dt * s.dTdt[k];
      q2[k] = qc[k] + dt * s.dqdt[k];
      if (!s.bad && q2[k] < 0.0) q2[k] = 0.0;
    }
    ShalState<double> t;
    shallow_column<double>(pver, hyai, hybi, p0, T2, q2, ps[i], SP, t);
    // each component: deep transport, then the shallow transport of the
    // deep-updated wind (no floor: a wind component may take either sign)
    for (int n = 0; n < 2; ++n) {
      double c[MAXLEV], c2[MAXLEV], td[MAXLEV], ts[MAXLEV];
      for (int k = 0; k < pver; ++k) c[k] = uv[n * cstride + k * ld + i];
      deep_momentum(pver, s, c, c_up, c_down, td);
      for (int k = 0; k < pver; ++k) c2[k] = c[k] + dt * td[k];
      shallow_momentum(pver, t, SP, c2, c_up, ts);
      for (int k = 0; k < pver; ++k) {
        tend_deep[n * cstride + k * ld + i] = td[k];
        tend_shallow[n * cstride + k * ld + i] = ts[k];
      }
    }
  }
  return 0;
}

int oracle_deep_adjoint(int n_cols, int pver, int ld, const double* hyai, const double* hybi,
                        double p0, const double* T, const double* q, const double* ps,
                        const double* lambda, const double* tau,
                        const oracle_deep_params* par, double dt, const double* gP,
                        const double* gH, const double* w_heat, double* gT, double* gq,
                        double* glambda, double* gtau, int n_threads) {
  if (!grid_ok(n_cols, pver, ld) || !par) return 1;
  const DeepP P = to_deep(par);
#pragma omp parallel for schedule(dynamic, 4) num_threads(threads_for(n_threads))
  for (int i = 0; i < n_cols; ++i) {
    Dual Tc[MAXLEV], qc[MAXLEV];
    for (int k = 0; k < pver; ++k) {
      Tc[k] = Dual(T[k * ld + i]);
      Tc[k].d[k] = 1.0;
      qc[k] = Dual(q[k * ld + i]);
      qc[k].d[pver + k] = 1.0;
    }
    Dual lam(lambda ? lambda[i] : P.lambda_default);
    lam.d[2 * pver] = 1.0;
    Dual ta(tau ? tau[i] : P.tau_default);
    ta.d[2 * pver + 1] = 1.0;
    std::unique_ptr<DeepState<Dual>> sp(new DeepState<Dual>());  // ~0.5 MB: keep off the stack
    DeepState<Dual>& s = *sp;
    deep_column<Dual>(pver, hyai, hybi, p0, Tc, qc, Dual(ps[i]), lam, ta, P, dt, s);
    Dual J = gP[i] * s.prec;
    if (s.active) {
      for (int k = 0; k < pver; ++k) {
        const double w = w_heat ? w_heat[k] : s.p_mid[k].v / ps[i];
        J = J + (gH[i] * w) * (s.m[k] * CP * s.dTdt[k]);
      }
    }
    for (int k = 0; k < pver; ++k) {
      gT[k * ld + i] = J.d[k];
      gq[k * ld + i] = J.d[pver + k];
    }
    glambda[i] = J.d[2 * pver];
    gtau[i] = J.d[2 * pver + 1];
  }
  return 0;
}

// Tangent of the fused step (deep convection, then shallow convection on the
// deep-updated state with q floored at zero, as oracle_deep_shallow):
//   J = gPd Pd + gHd Hd + gPs Ps + gHs Hs,  H = sum_k w_k m_k cp dT/dt_k of each
// scheme (w = w_heat, or p_mid/ps), differentiated in forward mode with respect
// to T, q, lambda and tau (Dual: 2 pver + 2 directions at once).
int oracle_deep_shallow_adjoint(int n_cols, int pver, int ld, const double* hyai,
                                const double* hybi, double p0, const double* T, const double* q,
                                const double* ps, const double* lambda, const double* tau,
                                const oracle_deep_params* dpar, const oracle_shallow_params* spar,
                                double dt, const double* gPd, const double* gHd,
                                const double* gPs, const double* gHs, const double* w_heat,
                                double* gT, double* gq, double* glambda, double* gtau,
                                int n_threads) {
  if (!grid_ok(n_cols, pver, ld) || !dpar || !spar) return 1;
  const DeepP DP = to_deep(dpar);
  const ShalP SP = to_shal(spar);
#pragma omp parallel for schedule(dynamic, 4) num_threads(threads_for(n_threads))
  for (int i = 0; i < n_cols; ++i) {
    Dual Tc[MAXLEV], qc[MAXLEV], T2[MAXLEV], q2[MAXLEV];
    for (int k = 0; k < pver; ++k) {
      Tc[k] = Dual(T[k * ld + i]);
      Tc[k].d[k] = 1.0;
      qc[k] = Dual(q[k * ld + i]);
      qc[k].d[pver + k] = 1.0;
    }
    Dual lam(lambda ? lambda[i] : DP.lambda_default);
    lam.d[2 * pver] = 1.0;
    Dual ta(tau ? tau[i] : DP.tau_default);
    ta.d[2 * pver + 1] = 1.0;
    std::unique_ptr<DeepState<Dual>> sp(new DeepState<Dual>());
    std::unique_ptr<ShalState<Dual>> tp(new ShalState<Dual>());
    DeepState<Dual>& s = *sp;
    ShalState<Dual>& t = *tp;
    deep_column<Dual>(pver, hyai, hybi, p0, Tc, qc, Dual(ps[i]), lam, ta, DP, dt, s);
    for (int k = 0; k < pver; ++k) {
      T2[k] = Tc[k] + dt * s.dTdt[k];
      q2[k] = qc[k] + dt * s.dqdt[k];
      if (!s.bad && q2[k].v < 0.0) q2[k] = Dual(0.0);
    }
    shallow_column<Dual>(pver, hyai, hybi, p0, T2, q2, Dual(ps[i]), SP, t);
    const double gpd = gPd ? gPd[i] : 0.0, ghd = gHd ? gHd[i] : 0.0;
    const double gps = gPs ? gPs[i] : 0.0, ghs = gHs ? gHs[i] : 0.0;
    Dual J = gpd * s.prec;
    if (s.active) {
      for (int k = 0; k < pver; ++k) {
        const double w = w_heat ? w_heat[k] : s.p_mid[k].v / ps[i];
        J = J + (ghd * w) * (s.m[k] * CP * s.dTdt[k]);
      }
    }
    if (t.active) {
      J = J + gps * t.prec;
      for (int k = 0; k < pver; ++k) {
        const double w = w_heat ? w_heat[k] : t.p_mid[k].v / ps[i];
        J = J + (ghs * w) * (t.m[k] * CP * t.dT[k]);
      }
    }
    for (int k = 0; k < pver; ++k) {
      gT[k * ld + i] = J.d[k];
      gq[k * ld + i] = J.d[pver + k];
    }
    glambda[i] = J.d[2 * pver];
    gtau[i] = J.d[2 * pver + 1];
  }
  return 0;
}

int oracle_deep_shallow_counted(int n_cols, int pver, int ld, const double* hyai,
                                const double* hybi, double p0, const double* T, const double* q,
                                const double* ps, const oracle_deep_params* dpar,
                                const oracle_shallow_params* spar, double dt,
                                const oracle_out* deep, const oracle_out* shallow) {
  if (!grid_ok(n_cols, pver, ld) || !dpar || !spar || !deep || !shallow) return 1;
  const DeepP DP = to_deep(dpar);
  const ShalP SP = to_shal(spar);
  std::unique_ptr<DeepState<Cnt>> sp(new DeepState<Cnt>());
  std::unique_ptr<ShalState<Cnt>> tp(new ShalState<Cnt>());
  for (int i = 0; i < n_cols; ++i) {
    Cnt Tc[MAXLEV], qc[MAXLEV], T2[MAXLEV], q2[MAXLEV];
    for (int k = 0; k < pver; ++k) { Tc[k] = Cnt(T[k * ld + i]); qc[k] = Cnt(q[k * ld + i]); }
    *sp = DeepState<Cnt>();
    *tp = ShalState<Cnt>();
    deep_column<Cnt>(pver, hyai, hybi, p0, Tc, qc, Cnt(ps[i]), Cnt(DP.lambda_default),
                     Cnt(DP.tau_default), DP, dt, *sp);
    store_deep(*sp, pver, ld, i, deep);
    for (int k = 0; k < pver; ++k) {
      T2[k] = Tc[k] + dt * sp->dTdt[k].v;
      q2[k] = qc[k] + dt * sp->dqdt[k].v;
      if (!sp->bad && q2[k].v < 0.0) q2[k] = Cnt(0.0);
    }
    shallow_column<Cnt>(pver, hyai, hybi, p0, T2, q2, Cnt(ps[i]), SP, *tp);
    store_shallow(*tp, pver, ld, i, shallow);
  }
  return 0;
}

int oracle_count_ops(int n_cols, int pver, int ld, const double* hyai, const double* hybi,
                     double p0, const double* T, const double* q, const double* ps,
                     const oracle_deep_params* dpar, const oracle_shallow_params* spar,
                     double dt, double* counts_deep, double* counts_total) {
  if (!grid_ok(n_cols, pver, ld) || !dpar || !spar) return 1;
  const DeepP DP = to_deep(dpar);
  const ShalP SP = to_shal(spar);
  double tot[C_NCAT] = {0};
  double deep[C_NCAT] = {0};
  for (int i = 0; i < n_cols; ++i) {
    Cnt Tc[MAXLEV], qc[MAXLEV], T2[MAXLEV], q2[MAXLEV];
    for (int k = 0; k < pver; ++k) { Tc[k] = Cnt(T[k * ld + i]); qc[k] = Cnt(q[k * ld + i]); }
    for (int c = 0; c < C_NCAT; ++c) g_count[c] = 0.0;
    DeepState<Cnt> s;
    deep_column<Cnt>(pver, hyai, hybi, p0, Tc, qc, Cnt(ps[i]), Cnt(DP.lambda_default),
                     Cnt(DP.tau_default), DP, dt, s);
    for (int c = 0; c < C_NCAT; ++c) deep[c] += g_count[c];
    for (int k = 0; k < pver; ++k) {
      T2[k] = Tc[k] + dt * s.dTdt[k].v;
      q2[k] = qc[k] + dt * s.dqdt[k].v;
      if (!s.bad && q2[k].v < 0.0) q2[k] = Cnt(0.0);
    }
    ShalState<Cnt> t;
    shallow_column<Cnt>(pver, hyai, hybi, p0, T2, q2, Cnt(ps[i]), SP, t);
    for (int c = 0; c < C_NCAT; ++c) tot[c] += g_count[c];
  }
  if (counts_deep)
    for (int c = 0; c < C_NCAT; ++c) counts_deep[c] = deep[c];
  if (counts_total)
    for (int c = 0; c < C_NCAT; ++c) counts_total[c] = tot[c];
  return 0;
}

int oracle_count_ops_by_pass(int n_cols, int pver, int ld, const double* hyai,
                             const double* hybi, double p0, const double* T, const double* q,
                             const double* ps, const oracle_deep_params* dpar,
                             const oracle_shallow_params* spar, double dt, double* trigger_pass,
                             double* plume_pass, double* n_triggered, double* e2_search) {
  if (!grid_ok(n_cols, pver, ld) || !dpar || !spar || !trigger_pass || !plume_pass) return 1;
  const DeepP DP = to_deep(dpar);
  const ShalP SP = to_shal(spar);
  const int W = C_NCAT + I_NCAT;
  for (int c = 0; c < W; ++c) trigger_pass[c] = plume_pass[c] = 0.0;
  if (e2_search)
    for (int c = 0; c < C_NCAT; ++c) e2_search[c] = 0.0;
  double ntrig = 0.0;
  std::unique_ptr<DeepState<Cnt>> sp(new DeepState<Cnt>());
  std::unique_ptr<ShalState<Cnt>> tp(new ShalState<Cnt>());
  for (int i = 0; i < n_cols; ++i) {
    Cnt Tc[MAXLEV], qc[MAXLEV], T2[MAXLEV], q2[MAXLEV];
    for (int k = 0; k < pver; ++k) { Tc[k] = Cnt(T[k * ld + i]); qc[k] = Cnt(q[k * ld + i]); }
    for (int c = 0; c < C_NCAT; ++c) g_count[c] = g_mark[c] = 0.0;
    for (int c = 0; c < I_NCAT; ++c) g_island[c] = 0.0;
    *sp = DeepState<Cnt>();  // the column routines expect freshly constructed states
    *tp = ShalState<Cnt>();
    DeepState<Cnt>& s = *sp;
    deep_column<Cnt>(pver, hyai, hybi, p0, Tc, qc, Cnt(ps[i]), Cnt(DP.lambda_default),
                     Cnt(DP.tau_default), DP, dt, s);
    double deep_ops[C_NCAT], deep_isl[I_NCAT];
    for (int c = 0; c < C_NCAT; ++c) deep_ops[c] = g_count[c];
    for (int c = 0; c < I_NCAT; ++c) deep_isl[c] = g_island[c];
    const bool trig = s.triggered;
    // trigger stage (all columns); the rest of the deep scheme runs in the plume pass
    for (int c = 0; c < C_NCAT; ++c) {
      const double mark = s.bad ? 0.0 : (trig ? g_mark[c] : deep_ops[c]);
      trigger_pass[c] += mark;
      plume_pass[c] += deep_ops[c] - mark;
    }
    for (int c = 0; c < I_NCAT; ++c) {
      if (c == I_CONS) plume_pass[C_NCAT + c] += deep_isl[c];
      else trigger_pass[C_NCAT + c] += deep_isl[c];
    }
    // the deep-updated state the shallow scheme reads: counted with it
    for (int c = 0; c < C_NCAT; ++c) g_count[c] = g_lfc0[c] = g_lfc1[c] = 0.0;
    for (int c = 0; c < I_NCAT; ++c) g_island[c] = 0.0;
    for (int k = 0; k < pver; ++k) {
      T2[k] = Tc[k] + dt * s.dTdt[k].v;
      q2[k] = qc[k] + dt * s.dqdt[k].v;
      if (!s.bad && q2[k].v < 0.0) q2[k] = Cnt(0.0);
    }
    shallow_column<Cnt>(pver, hyai, hybi, p0, T2, q2, Cnt(ps[i]), SP, *tp);
    double* dst = trig ? plume_pass : trigger_pass;
    for (int c = 0; c < C_NCAT; ++c) dst[c] += g_count[c];
    for (int c = 0; c < I_NCAT; ++c) dst[C_NCAT + c] += g_island[c];
    // the LFC search of a trigger-pass column that ends at exit E2
    if (e2_search && !trig && tp->exit_code == 2)
      for (int c = 0; c < C_NCAT; ++c) e2_search[c] += g_lfc1[c] - g_lfc0[c];
    ntrig += trig ? 1.0 : 0.0;
  }
  if (n_triggered) *n_triggered = ntrig;
  return 0;
}

}  // extern "C"
