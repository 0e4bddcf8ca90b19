/*
 * conv_oracle.h -- C interface of the FP64 CPU oracle for the column-convection
 * hot path (deep convection then shallow convection over independent columns).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links or includes
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load the shared object built from conv_oracle.cpp.
 *
 * The paper (Sec. II-A, Alg. 1-3) names the two schemes -- Zhang-McFarlane deep
 * convection and the University of Washington shallow plume -- but prints no
 * equations.  The oracle implements the column equations this project freezes
 * (levels, Bolton saturation, LCL Newton, undilute parcel/CAPE, entraining
 * updraft, downdraft, flux-form tendencies, CAPE-relaxation closure, CIN-based
 * shallow plume, deep adjoint).  Each function in conv_oracle.cpp says which
 * part of the paper it stands for and which published formula it uses.
 *
 * Layout of every profile array: level-major, element (k, i) at [k*ld + i],
 * k = 0 (model top) .. pver-1 (lowest layer).  Interfaces: k and k+1 bound
 * layer k; hyai/hybi hold pver+1 interface coefficients.
 */
#ifndef CONV_ORACLE_H
#define CONV_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double capelmt, lambda_default, tau_default, c0, alpha_dd;
  double p_launch_min, p_top_lim, q_min, ent_zscale;
  int32_t n_newton_lcl, n_newton_h;
  int32_t n_plumes, reserved; /* plume spectrum: number of plumes (1 = bulk plume) */
  double plume_spread;        /* largest / smallest entrainment rate of the spectrum */
} oracle_deep_params;

typedef struct {
  double eps_s, tke, c_m, cin_scale, cin_max, a_w, b_w, ql_crit;
  double p_lcl_min, p_lfc_min, p_top_lim;
  int32_t n_newton_lcl, n_newton_h;
  double evap_k; /* rain evaporation coefficient, 1/(kg/kg)/m; 0 = off */
} oracle_shallow_params;

/* Outputs of one scheme over n_cols columns (any pointer but flags may be NULL). */
typedef struct {
  double *dTdt, *dqdt;         /* [pver][ld] K/s, kg/kg/s                          */
  double *prec;                /* [ld] kg m-2 s-1                                  */
  int32_t *flags, *kb, *klcl, *ktop, *kaux;  /* [ld]                               */
  double *cape, *mb, *cons_err;              /* [ld] (shallow: cape holds CIN)     */
} oracle_out;

/* Mass-flux profiles of one scheme ([pver][ld] kg m-2 s-1, any pointer may be
 * NULL): mu = updraft flux leaving layer k through its top; du = updraft air
 * detrained into layer k (carrying the plume value from layer k+1); md =
 * downdraft flux leaving layer k through its bottom (downward positive), all
 * detrained into the layer below the downdraft's lowest level.  Zero in
 * inactive columns. */
typedef struct {
  double *mu, *du, *md;
} oracle_flux;

/* Scalar thermodynamics (for pin tests). */
double oracle_es(double T);
double oracle_qs(double T, double p);
double oracle_dqsdT(double T, double p);
/* LCL by Newton on the vapour-pressure form; returns last |dT| step. */
double oracle_lcl(double Tb, double qb, double pb, int n_newton, double* TL, double* pL);
/* Moist-static-energy inversion: T with cp T + gz + Lv qs(T,p) = h by Newton from T_start,
 * stopping after the first correction below 1e-7 K, at most 1+n_extra steps. */
double oracle_hinv(double h, double gz, double p, double T_start, int n_extra, double* last_step);
/* Hypsometric heights of one column (arrays of this column only). */
void oracle_heights(int pver, const double* T, const double* q, const double* p_int,
                    const double* p_mid, double* z_int, double* z_mid);
/* Interface/mid pressures of one column. */
void oracle_levels(int pver, const double* hyai, const double* hybi, double p0, double ps,
                   double* p_int, double* p_mid);

/* Per-column internals of the deep scheme (for pin tests). */
typedef struct {
  int32_t k_top_lim, kb, klcl, kel, khmin, jt, jd, triggered, active, limited;
  double TL, pL, cape, F, mb, sumR, sumE, alpha_eff, prec;
  double Tp[32], qp[32], b[32], eta[32], hu[32], qtu[32], rain[32];
  double etad[32], hd[32], qd[32], E1[32];
  double dh[32], dq[32], dT[32];     /* unit (per M_b) tendencies  */
  double m[32], z_mid[32], z_int[33], h[32], hs[32], p_mid[32], p_int[33];
} oracle_deep_diag;
void oracle_deep_column_diag(int pver, const double* hyai, const double* hybi, double p0,
                             const double* T, const double* q, double ps, double lambda,
                             double tau, const oracle_deep_params* par, double dt,
                             oracle_deep_diag* d);

typedef struct {
  int32_t k_top_lim, klcl, klfc, kts, exit_code, active;
  double TL, pL, cin, mb, prec;
  double b[32], hu[32], qtu[32], qtpre[32], w2[32], rf[32], Tu[32];
  double dh[32], dq[32], dT[32];     /* already scaled by M_b        */
  double m[32], z_mid[32], z_int[33], h[32], p_mid[32], p_int[33];
} oracle_shallow_diag;
void oracle_shallow_column_diag(int pver, const double* hyai, const double* hybi, double p0,
                                const double* T, const double* q, double ps,
                                const oracle_shallow_params* par, oracle_shallow_diag* d);

/* Whole-grid drivers.  n_threads <= 1 runs serially; otherwise OpenMP
 * schedule(dynamic,8) over columns (the paper's load-balancing device,
 * Sec. IV-A).  lambda/tau may be NULL (defaults).  Return 0 on success. */
int oracle_deep(int n_cols, int pver, int ld, const double* hyai, const double* hybi, double p0,
                const double* T, const double* q, const double* ps, const double* lambda,
                const double* tau, const oracle_deep_params* par, double dt,
                const oracle_out* out, int n_threads);
int oracle_shallow(int n_cols, int pver, int ld, const double* hyai, const double* hybi,
                   double p0, const double* T, const double* q, const double* ps,
                   const oracle_shallow_params* par, const oracle_out* out, int n_threads);
/* Deep, then shallow on T + dt*dTdt_deep, q + dt*dqdt_deep (Alg. 1 order). */
int oracle_deep_shallow(int n_cols, int pver, int ld, const double* hyai, const double* hybi,
                        double p0, const double* T, const double* q, const double* ps,
                        const double* lambda, const double* tau,
                        const oracle_deep_params* dpar, const oracle_shallow_params* spar,
                        double dt, const oracle_out* deep, const oracle_out* shallow,
                        int n_threads);

/* Deep-scheme gradients by forward-mode (tangent) differentiation of the same
 * column code: for J = gP*P + gH*sum_k w_k m_k cp dTdt_k, returns dJ/dT, dJ/dq
 * ([pver][ld]), dJ/dlambda and dJ/dtau ([ld]).  w_heat NULL -> w_k = p_mid_k/ps. */
int oracle_deep_adjoint(int n_cols, int pver, int ld, const double* hyai, const double* hybi,
                        double p0, const double* T, const double* q, const double* ps,
                        const double* lambda, const double* tau,
                        const oracle_deep_params* par, double dt, const double* gP,
                        const double* gH, const double* w_heat, double* gT, double* gq,
                        double* glambda, double* gtau, int n_threads);

/* Forward-mode tangent of the fused deep -> shallow step (shallow on the
 * deep-updated state, q floored at 0): gradients of
 *   J = gPd*Pd + gHd*sum w m cp dTdt_deep + gPs*Ps + gHs*sum w m cp dTdt_shallow
 * (w = w_heat, or p_mid/ps) with respect to T, q ([pver][ld]), lambda, tau
 * ([ld]).  Any of gPd, gHd, gPs, gHs may be NULL (zero). */
int oracle_deep_shallow_adjoint(int n_cols, int pver, int ld, const double* hyai,
                                const double* hybi, double p0, const double* T, const double* q,
                                const double* ps, const double* lambda, const double* tau,
                                const oracle_deep_params* dpar, const oracle_shallow_params* spar,
                                double dt, const double* gPd, const double* gHd,
                                const double* gPs, const double* gHs, const double* w_heat,
                                double* gT, double* gq, double* glambda, double* gtau,
                                int n_threads);

/* Floating-point operation counts of the path, by category:
 * [0] add/sub, [1] mul, [2] div, [3] exp, [4] log, [5] pow, [6] sqrt, [7] unused.
 * counts_deep: the deep scheme alone; counts_total: deep + shallow; both summed
 * over the given columns (8 doubles each, either may be NULL). */
/* Convective transport of ntr passive tracers ([ntr][pver][ld], stride
 * pver*ld) by the fused step: tend_deep = the deep scheme's tendency of each
 * tracer; tend_shallow = the shallow scheme's tendency of max(c + dt*tend_deep,
 * 0), the tracer the shallow scheme sees after the deep update (Alg. 1 order).
 * Each scheme mixes a tracer as it mixes its conserved moist static energy.
 * flux_deep / flux_shallow (may be NULL) receive the mass-flux profiles. */
int oracle_deep_shallow_tracers(int n_cols, int pver, int ld, const double* hyai,
                                const double* hybi, double p0, const double* T, const double* q,
                                const double* ps, const double* lambda, const double* tau,
                                const oracle_deep_params* dpar, const oracle_shallow_params* spar,
                                double dt, int ntr, const double* tracers, double* tend_deep,
                                double* tend_shallow, const oracle_flux* flux_deep,
                                const oracle_flux* flux_shallow, int n_threads);

/* Convective momentum transport of the fused step: the two wind components
 * uv [2][pver][ld] (u then v) carried by the plumes like tracers, plus the
 * pressure-gradient term of Gregory et al. (1997) inside each plume (c_up for
 * the updrafts, c_down for the downdraft; 0 gives the tracer transport), the
 * environment's tendency the divergence of the interface eddy fluxes (column
 * momentum conserved).  tend_deep, tend_shallow: [2][pver][ld] m/s2; the
 * shallow scheme transports u + dt tend_deep (no floor). */
int oracle_deep_shallow_momentum(int n_cols, int pver, int ld, const double* hyai,
                                 const double* hybi, double p0, const double* T,
                                 const double* q, const double* ps, const double* lambda,
                                 const double* tau, const oracle_deep_params* dpar,
                                 const oracle_shallow_params* spar, double dt, double c_up,
                                 double c_down, const double* uv, double* tend_deep,
                                 double* tend_shallow, int n_threads);

/* Floating-point operation counts of the fused deep -> shallow step, summed over
 * the columns, by category (add/sub, mul, div, exp, log, pow, sqrt, unused):
 * the deep scheme alone and the whole step.  Default lambda and tau. */
int oracle_count_ops(int n_cols, int pver, int ld, const double* hyai, const double* hybi,
                     double p0, const double* T, const double* q, const double* ps,
                     const oracle_deep_params* dpar, const oracle_shallow_params* spar,
                     double dt, double* counts_deep, double* counts_total);

/* The fused step computed by the counting instantiation (default lambda and
 * tau, serial): its outputs must equal oracle_deep_shallow's bit for bit. */
int oracle_deep_shallow_counted(int n_cols, int pver, int ld, const double* hyai,
                                const double* hybi, double p0, const double* T, const double* q,
                                const double* ps, const oracle_deep_params* dpar,
                                const oracle_shallow_params* spar, double dt,
                                const oracle_out* deep, const oracle_out* shallow);

/* The same counts split by the two passes of a compacted GPU implementation:
 * trigger_pass = deep trigger stage of every column + the shallow scheme of the
 * columns that do not trigger; plume_pass = the rest of the deep scheme and the
 * shallow scheme of the triggered columns.  Each array has 13 entries: the 8
 * operation categories, then FP64-island tallies of the mixed-precision design:
 * [8] LCL solves, [9] CAPE terms, [10] CIN terms, [11] conservation-sum terms,
 * [12] saturated shallow plume layers with rain within 1e-4 kg/kg of zero.
 * e2_search (8 entries, may be NULL): the operations of the shallow scheme's
 * undilute-parcel LFC search in trigger-pass columns that end at exit E2 (part
 * of trigger_pass; work an implementation may settle by bounds). */
int oracle_count_ops_by_pass(int n_cols, int pver, int ld, const double* hyai,
                             const double* hybi, double p0, const double* T, const double* q,
                             const double* ps, const oracle_deep_params* dpar,
                             const oracle_shallow_params* spar, double dt, double* trigger_pass,
                             double* plume_pass, double* n_triggered, double* e2_search);

#ifdef __cplusplus
}
#endif
#endif
