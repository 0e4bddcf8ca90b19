// adjoint.cuh -- reverse-mode adjoint of the deep scheme (FP64), one thread per
// column.  For J = gP P + gH H, H = sum_k w_k m_k cp dT/dt_k, it returns
// dJ/dT_k, dJ/dq_k, dJ/dlambda and dJ/dtau.  The column is first recomputed
// forward in the thread (the plume state is recomputed, never stored between
// kernels) with deep_plume recording its intermediates; then the reverse sweep
// runs through closure, tendencies, downdraft, updraft, parcel, moist static
// energy and heights.  Newton solves are differentiated by the implicit
// function theorem, dT = (dh - g dz) / (cp + Lv dqs/dT); level choices, the
// saturation, alpha and limiter branches are held at their forward values
// (the scheme is piecewise smooth).
#pragma once

#include "column.cuh"

namespace cvg {

// qs, dqs/dT and d2qs/dT2 at (T, p), same branch as sat_qs_dqs.
__device__ __forceinline__ void qs_derivs(double T, double p, double& qs, double& dqs,
                                          double& d2qs) {
  const double r = 1.0 / (T - EST1);
  const double es = ES0 * exp(ESA * (T - EST0) * r);
  const double a = ESA * ESC * r * r;  // d ln es / dT
  const double ap = -2.0 * a * r;      // d a / dT
  const double D = p - ONE_M_EPS * es;
  if (D < 1e-3 * p) {
    qs = EPSV * es / (1e-3 * p);
    dqs = qs * a;
    d2qs = qs * (a * a + ap);
  } else {
    qs = EPSV * es / D;
    dqs = qs * p * a / D;
    d2qs = EPSV * p * es / (D * D) * (ap + a * a + 2.0 * a * a * ONE_M_EPS * es / D);
  }
}

// Adjoint of T = hinv(h, g z, p): dT = (dh - g dz) / (cp + Lv dqs(T)).
__device__ __forceinline__ void inv_adj(double T, double p, double bT, double& bh, double& bz) {
  double qs, dqs, d2;
  qs_derivs(T, p, qs, dqs, d2);
  const double B = CP + LV * dqs;
  bh += bT / B;
  bz -= GRAV * bT / B;
}

// Deep scheme with its tape, for column c (T, q, ps, pver set); false for a
// rejected column.  t.Tp must point at per-layer storage.
__device__ __forceinline__ bool deep_forward(const conv_deep_params& P, const DeepQ<double>& Q,
                                             double lam, double tau, Column<double>& c,
                                             DeepTrig<double>& t, DeepTape<double>& tp) {
  tp.active = false;
  t.triggered = false;
  if (!prologue(Q.p_top_lim, c)) return false;
  deep_trigger(c, P, Q, t);
  if (t.triggered) {
    DeepOut o;
    o.flags = 0;
    deep_plume<double, DeepTape<double>>(c, P, Q, lam, tau, t, o, NoOut<double>(), &tp);
  }
  return true;
}

// Reverse sweep of the deep scheme recorded in (t, tp) for the seeds gP on the
// precipitation and sT, sq ([pver], either may be nullptr) on the dT/dt, dq/dt
// outputs; adds the gradient to bT, bq, blam, btau.
__device__ __forceinline__ void deep_reverse(const conv_deep_params& P, const DeepQ<double>& Q,
                                             double lam, double tau, const Column<double>& c,
                                             const DeepTrig<double>& t,
                                             const DeepTape<double>& tp, double gP,
                                             const double* sT, const double* sq, double* bT,
                                             double* bq, double& blam, double& btau) {
  if (!tp.active) return;
  const int pver = c.pver;
  const int kb = t.kb, klcl = t.klcl, kel = t.kel, jt = tp.jt, jd = tp.jd;
  const double mb = tp.mb, ze = P.ent_zscale;
  {
    double bTv[MAXL], bzm[MAXL], bzi[MAXL + 1], bh[MAXL], beta[MAXL], bhu[MAXL], bqtu[MAXL];
    double betad[MAXL], bhd[MAXL], bqd[MAXL], bdh[MAXL], bdq[MAXL], bdT[MAXL], bTp[MAXL];
    for (int k = 0; k < pver; ++k) {
      bTv[k] = bzm[k] = bzi[k] = bh[k] = beta[k] = bhu[k] = bqtu[k] = 0.0;
      betad[k] = bhd[k] = bqd[k] = bdh[k] = bdq[k] = bdT[k] = bTp[k] = 0.0;
    }
    bzi[pver] = 0.0;
    double bMb = 0.0, bCAPE = 0.0, bF = 0.0, bsumR = 0.0, bsumE = 0.0, balpha = 0.0;

    // seeds on the outputs: dT/dt = mb dT, dq/dt = mb dq, P = mb max(0, sumR - alpha sumE)
    for (int k = jt; k <= kb; ++k) {
      if (sT) {
        bdT[k] += sT[k] * mb;
        bMb += sT[k] * tp.dT[k];
      }
      if (sq) {
        bdq[k] += sq[k] * mb;
        bMb += sq[k] * tp.dq[k];
      }
    }
    if (tp.net_pos) {
      bMb += gP * tp.net;
      const double bnet = gP * mb;
      bsumR += bnet;
      balpha -= bnet * tp.sumE;
      bsumE -= bnet * tp.alpha;
    }

    // closure or limiter
    if (tp.limited) {
      const int ks = tp.kstar;
      const double N = c.q(ks) - P.q_min, Dn = -Q.dt * tp.dq[ks];
      bq[ks] += bMb / Dn;
      bdq[ks] += bMb * N * Q.dt / (Dn * Dn);
    } else {
      const double F = tp.F, cape = t.cape;
      bCAPE += -bMb / (tau * F);
      btau += bMb * cape / (tau * tau * F);
      bF += bMb * cape / (tau * F * F);
      const double dhkb = tp.dh[kb];
      for (int k = kel; k <= klcl; ++k) {
        const double Tp = t.Tp[(size_t)k * t.tps];
        double qsp, dqsp, d2qsp;
        qs_derivs(Tp, c.pm(k), qsp, dqsp, d2qsp);
        const double Av = (1.0 + ZVIR * qsp) + ZVIR * Tp * dqsp, Bv = CP + LV * dqsp;
        const double w1 = bF * RD * c.dl[k];
        bdh[kb] += w1 * Av / Bv;
        const double bdTvp = w1 * dhkb;
        const double bdTv = -w1;
        const bool in_plume = k >= jt && k <= kb;  // dT, dq are constant zero elsewhere
        const double dTk = in_plume ? tp.dT[k] : 0.0, dqk = in_plume ? tp.dq[k] : 0.0;
        bq[k] += bdTv * ZVIR * dTk;
        bT[k] += bdTv * ZVIR * dqk;
        if (in_plume) {
          bdT[k] += bdTv * (1.0 + ZVIR * c.q(k));
          bdq[k] += bdTv * ZVIR * c.T(k);
        }
        const double bA = bdTvp / Bv, bB = -bdTvp * Av / (Bv * Bv);
        const double bqsp = bA * ZVIR, bdqsp = bA * ZVIR * Tp + bB * LV;
        bTp[k] += bA * ZVIR * dqsp + bqsp * dqsp + bdqsp * d2qsp;
      }
    }

    // tendencies: dT = (dh - Lv dq)/cp, dh = dh_raw/m
    double bhr[MAXL], bqr[MAXL];
    for (int k = 0; k < pver; ++k) bhr[k] = bqr[k] = 0.0;
    for (int k = jt; k <= kb; ++k) {
      bdh[k] += bdT[k] / CP;
      bdq[k] -= LV * bdT[k] / CP;
      bhr[k] = bdh[k] / c.m(k);
      bqr[k] = bdq[k] / c.m(k);
    }
    if (jd >= 0) {
      const double al = tp.alpha;
      for (int k = jd; k <= kb - 1; ++k) {
        const double D = al * tp.etad[k];
        const double bD = bhr[k] * (c.h(k + 1) - c.h(k)) + bqr[k] * (c.q(k + 1) - c.q(k));
        bh[k + 1] += bhr[k] * D;
        bh[k] -= bhr[k] * D;
        bq[k + 1] += bqr[k] * D;
        bq[k] -= bqr[k] * D;
        balpha += bD * tp.etad[k];
        betad[k] += bD * al;
      }
      const double D = al * tp.etad[kb - 1];
      const double bD = bhr[kb] * (tp.hd[kb - 1] - c.h(kb)) + bqr[kb] * (tp.qd[kb - 1] - c.q(kb));
      bhd[kb - 1] += bhr[kb] * D;
      bh[kb] -= bhr[kb] * D;
      bqd[kb - 1] += bqr[kb] * D;
      bq[kb] -= bqr[kb] * D;
      balpha += bD * tp.etad[kb - 1];
      betad[kb - 1] += bD * al;
    }
    for (int k = jt + 1; k <= kb; ++k) {
      const double e = tp.eta[k];
      bh[k - 1] += bhr[k] * e;
      bh[k] -= bhr[k] * e;
      bq[k - 1] += bqr[k] * e;
      bq[k] -= bqr[k] * e;
      beta[k] += bhr[k] * (c.h(k - 1) - c.h(k)) + bqr[k] * (c.q(k - 1) - c.q(k));
    }
    beta[jt + 1] += bhr[jt] * (tp.hu[jt + 1] - c.h(jt)) + bqr[jt] * (tp.qtu[jt + 1] - c.q(jt));
    bhu[jt + 1] += bhr[jt] * tp.eta[jt + 1];
    bh[jt] -= bhr[jt] * tp.eta[jt + 1];
    bqtu[jt + 1] += bqr[jt] * tp.eta[jt + 1];
    bq[jt] -= bqr[jt] * tp.eta[jt + 1];

    // downdraft: alpha, evaporation sum (telescoped), saturation, mixing, mass flux
    if (jd >= 0) {
      const double sR = tp.sumR, sE = tp.sumE;
      if (tp.capped) {
        bsumR += balpha / sE;
        bsumE -= balpha * sR / (sE * sE);
      }
      betad[kb - 1] += bsumE * tp.qd[kb - 1];
      bqd[kb - 1] += bsumE * tp.etad[kb - 1];
      for (int k = jd; k <= kb - 1; ++k) {
        const double eprev = k > jd ? tp.etad[k - 1] : 0.0;
        bq[k] -= bsumE * (tp.etad[k] - eprev);
        betad[k] -= bsumE * c.q(k);
        if (k > jd) betad[k - 1] += bsumE * c.q(k);
      }
      for (int k = kb - 1; k >= jd; --k) {
        if (bqd[k] != 0.0) {
          double qs, dqs, d2;
          qs_derivs(tp.Td[k], c.pm(k), qs, dqs, d2);
          inv_adj(tp.Td[k], c.pm(k), bqd[k] * dqs, bhd[k], bzm[k]);
        }
        if (k > jd) {
          const double e = tp.etad[k], ep = tp.etad[k - 1];
          betad[k - 1] += bhd[k] * (tp.hd[k - 1] - c.h(k)) / e;
          bhd[k - 1] += bhd[k] * ep / e;
          bh[k] += bhd[k] * (e - ep) / e;
          betad[k] += bhd[k] * (c.h(k) - tp.hd[k]) / e;
        } else {
          bh[jd] += bhd[jd];
        }
      }
      for (int k = jd; k <= kb - 1; ++k) {
        const double u = 1.0 + (c.zm[jd] - c.zm[k]) / ze;
        blam += betad[k] * tp.etad[k] * ze * log(u);
        const double bu = betad[k] * tp.etad[k] * lam * ze / u;
        bzm[jd] += bu / ze;
        bzm[k] -= bu / ze;
      }
    }

    // updraft, reverse of its upward recurrence
    const double c0 = P.c0;
    for (int k = jt + 1; k <= kb - 1; ++k) {
      const double e = tp.eta[k], e1 = tp.eta[k + 1];
      double bqt = bqtu[k];
      const double bR = bsumR - bqtu[k] / e;
      beta[k] += bqtu[k] * tp.rain[k] / (e * e);
      const double dz = tp.dz[k];
      const double g = c0 * dz / (1.0 + c0 * dz), gp = c0 / ((1.0 + c0 * dz) * (1.0 + c0 * dz));
      const double l = (e * g) != 0.0 ? tp.rain[k] / (e * g) : 0.0;
      beta[k] += bR * l * g;
      const double bl = bR * e * g;
      const double bdz = bR * e * l * gp;
      bTv[k] += bdz * (RD / GRAV) * c.dl[k];  // dz = (Rd Tv / g) ln(p_k+1/p_k)
      if (tp.lpos[k]) {
        bqt += bl;
        double qs, dqs, d2;
        qs_derivs(tp.Ts[k], c.pm(k), qs, dqs, d2);
        inv_adj(tp.Ts[k], c.pm(k), -bl * dqs, bhu[k], bzm[k]);
      }
      beta[k + 1] += bqt * (tp.qtu[k + 1] - c.q(k)) / e;
      bqtu[k + 1] += bqt * e1 / e;
      bq[k] += bqt * (e - e1) / e;
      beta[k] += bqt * (c.q(k) - tp.qt[k]) / e;
      beta[k + 1] += bhu[k] * (tp.hu[k + 1] - c.h(k)) / e;
      bhu[k + 1] += bhu[k] * e1 / e;
      bh[k] += bhu[k] * (e - e1) / e;
      beta[k] += bhu[k] * (c.h(k) - tp.hu[k]) / e;
    }
    bh[kb] += bhu[kb];
    bq[kb] += bqtu[kb];
    for (int k = jt + 1; k <= kb - 1; ++k) {
      const double u = 1.0 + (c.zm[k] - c.zm[kb]) / ze;
      blam += beta[k] * tp.eta[k] * ze * log(u);
      const double bu = beta[k] * tp.eta[k] * lam * ze / u;
      bzm[k] += bu / ze;
      bzm[kb] -= bu / ze;
    }

    // undilute parcel and CAPE (closure branch only)
    for (int k = kel; k <= klcl; ++k) {
      const double Tp = t.Tp[(size_t)k * t.tps];
      double qp, dqp, d2;
      qs_derivs(Tp, c.pm(k), qp, dqp, d2);
      const double bb = bCAPE * RD * c.dl[k];
      bTp[k] += bb * ((1.0 + ZVIR * qp) + Tp * ZVIR * dqp);
      bTv[k] -= bb;
      inv_adj(Tp, c.pm(k), bTp[k], bh[kb], bzm[k]);
    }

    // moist static energy, heights, virtual temperature
    for (int k = 0; k < pver; ++k) {
      bT[k] += CP * bh[k];
      bzm[k] += GRAV * bh[k];
      bq[k] += LV * bh[k];
    }
    const PressFP64 Pr = c.press();
    for (int k = 0; k < pver; ++k) {
      bzi[k + 1] += bzi[k] + bzm[k];
      const double L2 = log(Pr.pi(k + 1) / c.pm(k));
      const double bs = bzi[k] * c.dl[k] + bzm[k] * L2;
      bTv[k] += bs * (RD / GRAV);
    }
    for (int k = 0; k < pver; ++k) {
      bT[k] += bTv[k] * (1.0 + ZVIR * c.q(k));
      bq[k] += bTv[k] * c.T(k) * ZVIR;
    }
  }
}

// Adjoint of the column state shared by both schemes: h = cp T + g z_mid + Lv q,
// hypsometric heights from Tv, Tv = T (1 + zv q).  Consumes bh, bzm, bTv (they are
// modified) and adds to bT, bq.
__device__ __forceinline__ void state_adjoint(const Column<double>& c, double* bh, double* bzm,
                                              double* bTv, double* bT, double* bq) {
  const int pver = c.pver;
  double bzi[MAXL + 1];
  for (int k = 0; k <= pver; ++k) bzi[k] = 0.0;
  for (int k = 0; k < pver; ++k) {
    bT[k] += CP * bh[k];
    bzm[k] += GRAV * bh[k];
    bq[k] += LV * bh[k];
  }
  const PressFP64 Pr = c.press();
  for (int k = 0; k < pver; ++k) {
    bzi[k + 1] += bzi[k] + bzm[k];
    const double L2 = log(Pr.pi(k + 1) / c.pm(k));
    const double bs = bzi[k] * c.dl[k] + bzm[k] * L2;
    bTv[k] += bs * (RD / GRAV);
  }
  for (int k = 0; k < pver; ++k) {
    bT[k] += bTv[k] * (1.0 + ZVIR * c.q(k));
    bq[k] += bTv[k] * c.T(k) * ZVIR;
  }
}

// Reverse sweep of the shallow scheme recorded in st (column c after its
// prologue) for the seeds gP on the precipitation and sT ([pver]) on the dT/dt
// output; adds the gradient with respect to the column's T, q to bT, bq.
// Level choices (LCL, LFC, cloud top), saturation and rain on/off are held.
__device__ __forceinline__ void shallow_reverse(const Column<double>& c, const ShalQ<double>& Q,
                                                const ShalTape<double>& st, double gP,
                                                const double* sT, double* bT, double* bq) {
  if (!st.active) return;
  const int pver = c.pver, ks = pver - 1, kts = st.kts, klcl = st.klcl, klfc = st.klfc;
  const double mb = st.mb;
  double bh[MAXL], bzm[MAXL], bTv[MAXL], bhu[MAXL], bqtu[MAXL], bqt[MAXL], br[MAXL];
  for (int k = 0; k < pver; ++k) bh[k] = bzm[k] = bTv[k] = bhu[k] = bqtu[k] = bqt[k] = br[k] = 0.0;
  double bmb = 0.0;
  // outputs: dT/dt_k = (dh_k - Lv dq_k) / (cp m_k), dh, dq = mb * (flux differences)
  bmb += gP * st.sumr;
  for (int k = kts + 1; k <= ks - 1; ++k) br[k] += gP * mb;
  for (int k = kts; k <= ks; ++k) {
    const double bdT = sT ? sT[k] : 0.0;
    if (bdT == 0.0) continue;
    const double rm = 1.0 / c.m(k);
    const double bAh = bdT * rm / CP, bAq = -bdT * LV * rm / CP;  // per unit (mb x bracket)
    double Ah, Aq;
    if (k == ks) {
      Ah = c.h(ks - 1) - c.h(ks);
      Aq = c.q(ks - 1) - c.q(ks);
      bh[ks - 1] += bAh * mb;
      bh[ks] -= bAh * mb;
      bq[ks - 1] += bAq * mb;
      bq[ks] -= bAq * mb;
    } else if (k == kts) {
      Ah = st.hu[kts + 1] - c.h(kts);
      Aq = st.qtu[kts + 1] - c.q(kts);
      bhu[kts + 1] += bAh * mb;
      bh[kts] -= bAh * mb;
      bqtu[kts + 1] += bAq * mb;
      bq[kts] -= bAq * mb;
    } else {
      Ah = (st.hu[k + 1] - st.hu[k]) + (c.h(k - 1) - c.h(k));
      Aq = (st.qtu[k + 1] - st.qt[k]) + (c.q(k - 1) - c.q(k));
      bhu[k + 1] += bAh * mb;
      bhu[k] -= bAh * mb;
      bh[k - 1] += bAh * mb;
      bh[k] -= bAh * mb;
      bqtu[k + 1] += bAq * mb;
      bqt[k] -= bAq * mb;
      bq[k - 1] += bAq * mb;
      bq[k] -= bAq * mb;
    }
    bmb += bAh * Ah + bAq * Aq;
  }
  // plume, reverse of its upward recurrence
  const double eps = Q.eps;
  for (int k = kts + 1; k <= ks - 1; ++k) {
    const double pm = c.pm(k);
    bqt[k] += bqtu[k];
    br[k] -= bqtu[k];
    double bqv = 0.0;
    if (st.r[k] > 0.0) {
      bqt[k] += br[k];
      bqv -= br[k];
    }
    if (st.sat[k]) {
      double qs, dqs, d2;
      qs_derivs(st.Tsat[k], pm, qs, dqs, d2);
      inv_adj(st.Tsat[k], pm, bqv * dqs, bhu[k], bzm[k]);
    } else {
      bqt[k] += bqv;
    }
    if (k >= klcl) {
      bhu[k + 1] += bhu[k];
      bqtu[k + 1] += bqt[k];
    } else {
      const double chi = st.chi[k];
      bhu[k + 1] += bhu[k] * (1.0 - chi);
      bh[k] += bhu[k] * chi;
      bqtu[k + 1] += bqt[k] * (1.0 - chi);
      bq[k] += bqt[k] * chi;
      const double bchi = bhu[k] * (c.h(k) - st.hu[k + 1]) + bqt[k] * (c.q(k) - st.qtu[k + 1]);
      const double bdz = bchi * eps * (1.0 - chi);
      bTv[k] += bdz * (RD / GRAV) * c.dl[k];
    }
  }
  double bhsrc = bhu[ks], bTsrc = 0.0, bqsrc = bqtu[ks];
  // closure M_b = rho c_m sqrt(tke) exp(-CIN/(cin_scale tke)), rho = p_src/(Rd Tv_src)
  const double bcin = bmb * mb * Q.m_inv_cin;
  bTv[ks] -= bmb * mb / c.Tv(ks);
  // CIN over the parcel's negatively buoyant layers below the LFC
  const double psrc = c.pm(ks);
  for (int k = ks; k > klfc; --k) {
    const double b = st.b[k];
    if (!(b < 0.0)) continue;
    const double bb = -bcin * RD * c.dl[k];
    const double Tp = st.Tp[k];
    const double pm = c.pm(k);
    bTv[k] -= bb;
    if (k > klcl) {
      const double qp = c.q(ks);
      bTsrc += bb * (1.0 + ZVIR * qp) * pow(pm / psrc, KAPPA);
      bqsrc += bb * ZVIR * Tp;
    } else {
      double qp, dqp, d2;
      qs_derivs(Tp, pm, qp, dqp, d2);
      const double bTp = bb * ((1.0 + ZVIR * qp) + ZVIR * Tp * dqp);
      inv_adj(Tp, pm, bTp, bhsrc, bzm[k]);
    }
  }
  bh[ks] += bhsrc;
  bT[ks] += bTsrc;
  bq[ks] += bqsrc;
  state_adjoint(c, bh, bzm, bTv, bT, bq);
}

// For the column loaded in c (T, q, ps, pver): P (surface precipitation) and
// H = sum_k w_k m_k cp dTdt_k into Pv, Hv, and -- when `reverse` -- the gradient
// of J = gP P + gH H into bT, bq [pver], blam, btau (all zeroed first).
// w_heat: [pver] weights, or nullptr for w_k = p_mid_k / ps.
__device__ __forceinline__ void deep_adjoint_column(const conv_deep_params& P,
                                                    const DeepQ<double>& Q, double lam, double tau,
                                                    Column<double>& c, double gP, double gH,
                                                    const double* w_heat, bool reverse,
                                                    double* bT, double* bq, double& blam,
                                                    double& btau, double& Pv, double& Hv) {
  const int pver = c.pver;
  for (int k = 0; k < pver; ++k) bT[k] = bq[k] = 0.0;
  blam = btau = Pv = Hv = 0.0;
  DeepTape<double> tp;
  double Tpa[MAXL];
  DeepTrig<double> t;
  t.Tp = Tpa;
  t.tps = 1;
  deep_forward(P, Q, lam, tau, c, t, tp);
  if (!tp.active) return;
  double sT[MAXL], Hs = 0.0;
  for (int k = 0; k < pver; ++k) {
    const double wm = (w_heat ? w_heat[k] : c.pm(k) / c.ps) * c.m(k);
    sT[k] = gH * CP * wm;
    Hs += wm * tp.dT[k];
  }
  Pv = tp.mb * tp.net;
  Hv = CP * tp.mb * Hs;
  if (reverse) deep_reverse(P, Q, lam, tau, c, t, tp, gP, sT, nullptr, bT, bq, blam, btau);
}

// The fused step for one column (deep, then shallow on T + dt dT/dt_deep,
// max(q + dt dq/dt_deep, 0)): the four objective pieces Pd, Hd, Ps, Hs into obj
// and -- when `reverse` -- the gradient of J = gPd Pd + gHd Hd + gPs Ps + gHs Hs
// (seeds g[4]) into bT, bq, blam, btau.  c: the column on the input state;
// c2: an initialised column whose source is the input advanced by dt times the
// deep tendencies, which this function writes to dTs, dqs ([pver], the source
// of c2) before the shallow scheme reads them.
__device__ __forceinline__ void step_adjoint_column(
    const conv_deep_params& P, const DeepQ<double>& Q, const conv_shallow_params& SP,
    const ShalQ<double>& SQ, double dt, double lam, double tau, Column<double>& c,
    Column<double>& c2, double* dTs, double* dqs, size_t dstride, const double g[4],
    const double* w_heat, bool reverse, double* bT, double* bq, double& blam, double& btau,
    double obj[4]) {
  const int pver = c.pver;
  for (int k = 0; k < pver; ++k) bT[k] = bq[k] = 0.0;
  blam = btau = 0.0;
  obj[0] = obj[1] = obj[2] = obj[3] = 0.0;
  DeepTape<double> tp;
  double Tpa[MAXL];
  DeepTrig<double> t;
  t.Tp = Tpa;
  t.tps = 1;
  const bool valid = deep_forward(P, Q, lam, tau, c, t, tp);
  double wm[MAXL];
  for (int k = 0; k < pver; ++k) {
    const double dTk = tp.active ? tp.mb * tp.dT[k] : 0.0;
    const double dqk = tp.active ? tp.mb * tp.dq[k] : 0.0;
    dTs[(size_t)k * dstride] = dTk;
    dqs[(size_t)k * dstride] = dqk;
    wm[k] = valid ? (w_heat ? w_heat[k] : c.pm(k) / c.ps) * c.m(k) : 0.0;
    obj[1] += wm[k] * dTk;
  }
  obj[0] = tp.active ? tp.mb * tp.net : 0.0;
  obj[1] *= CP;
  c2.s.floor_q = valid;
  ShalTape<double> st;
  ShalOut so;
  shallow_column<double, ShalTape<double>, NoOut<double>>(SP, SQ, c2, so, NoOut<double>(),
                                                          nullptr, false, nullptr, &st);
  if (st.active) {
    obj[2] = st.mb * st.sumr;
    for (int k = st.kts; k < pver; ++k) obj[3] += wm[k] * st.dT[k];
    obj[3] *= CP;
  }
  if (!reverse) return;
  // shallow: gradient with respect to its input state T', q'
  double b2T[MAXL], b2q[MAXL], sT[MAXL], sq[MAXL];
  for (int k = 0; k < pver; ++k) {
    b2T[k] = b2q[k] = 0.0;
    sT[k] = g[3] * CP * wm[k];
  }
  shallow_reverse(c2, SQ, st, g[2], sT, b2T, b2q);
  // T' = T + dt dT/dt, q' = max(q + dt dq/dt, 0) (no floor for a rejected column)
  for (int k = 0; k < pver; ++k) {
    const bool floored = valid && add_mul(c.q(k), dt, dqs[(size_t)k * dstride]) < 0.0;
    const double bqk = floored ? 0.0 : b2q[k];
    bT[k] += b2T[k];
    bq[k] += bqk;
    sT[k] = g[1] * CP * wm[k] + dt * b2T[k];
    sq[k] = dt * bqk;
  }
  deep_reverse(P, Q, lam, tau, c, t, tp, g[0], sT, sq, bT, bq, blam, btau);
}

}  // namespace cvg
