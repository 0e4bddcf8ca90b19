/*
 * conv.h -- C ABI of the GB300 column-convection library (libconvgb.so).
 *
 * What is computed.  The physics step of the atmosphere model applies deep
 * convection and then shallow convection to every vertical column, each column
 * independently of all others (paper Sec. II-A and Alg. 1).  Deep convection is
 * the Zhang-McFarlane mass-flux scheme with an entrainment loop and a
 * precipitation loop over levels that each invert a conserved thermodynamic
 * variable (Alg. 2); shallow convection is the University of Washington plume,
 * which leaves a column at several thermodynamic checks and then zeroes that
 * column's outputs (Alg. 3).  The paper gives no equations; this library
 * implements the column equations it freezes (listed with every reading of the
 * paper in the design notes): launch level of maximum moist static energy,
 * Newton LCL, undilute parcel and CAPE trigger, entraining updraft with
 * implicit rain, saturated downdraft, flux-form tendencies, CAPE-relaxation
 * closure with a moisture limiter, and a CIN-closed shallow plume.
 *
 * Data layout (the paper's transposed, padded layout, Sec. IV-C, turned for
 * a GPU: columns innermost so that a warp reads 32 adjacent columns of one
 * level in one coalesced access):
 *   profile arrays  [pver][ld], element (k, i) at k*ld + i,
 *                   k = 0 model top .. pver-1 lowest layer, i = column;
 *   column arrays   [ld];
 *   ld >= n_cols (a multiple of 32 is recommended); columns n_cols..ld-1 are
 *   neither read nor written.
 *
 * Precision.  CONV_FP64: T, q, dTdt, dqdt are double; everything is computed in
 * FP64.  CONV_MIXED: T, q, dTdt, dqdt are float and the arithmetic is FP32
 * except where a decision or an integral needs FP64 accuracy:
 *   - LCL: FP32 Newton iterations; one FP64 Newton correction (FP64 residual,
 *     relative humidity, logarithms and pressure) where the FP32 LCL pressure
 *     lies within 2e-5 (relative) of a layer mid-point or of the shallow E1
 *     threshold, so that every comparison made with it comes out as in FP64;
 *   - CAPE, CIN and the column conservation sums: FP32 terms added in
 *     compensated FP32 arithmetic (TwoSum; the sum of the terms is exact to
 *     ~2^-48 relative, each term carrying its own FP32 rounding, ~1e-7); the
 *     conservation ratio cons_err from them in FP32 with error-free products;
 *   - shallow rain within 1e-4 kg/kg of the autoconversion threshold: one FP64
 *     correction of the plume's saturation temperature and q_s in FP64;
 *   - deep updraft condensate within 3e-6 kg/kg of zero: the same FP64
 *     correction, so that the cloud top and the rain profile are decided as
 *     in FP64;
 *   - moist inversions: FP32 Newton, warm-started along each vertical sequence
 *     by a tangent predictor, at most four steps, stopping after a correction
 *     below 0.01 K;
 *   - FP32 quotients: PTX div.full.f32, within 2 ulp of IEEE division
 *     (conv_bench_f32_quotient applies it to arrays, for checking).
 * Measured against the FP64 oracle (the tests): trigger flips on at most 0.1%
 * of the columns, tendency column integrals within 1e-4 and precipitation
 * within 1e-3 relative where decisions agree.  Column scalars (ps, lambda, tau,
 * prec, cape, mb, cons_err) are double in both modes.
 *
 * Ownership and blocking.  Every pointer in conv_in / conv_out / workspace is a
 * DEVICE pointer owned by the caller; hyai/hybi in conv_grid are HOST pointers
 * read during the call.  Run calls are asynchronous on the given stream: they
 * validate arguments on the host, enqueue kernels and return.  The library
 * never allocates on a run path and never synchronises the stream.  Calls on
 * different streams with disjoint buffers may run concurrently.  Output arrays
 * must not overlap the inputs (the kernels re-read T and q through the
 * read-only cache while they write tendencies).
 *
 * Errors.  Argument errors are detected on the host before anything is
 * enqueued (CONV_ERR_ARG / CONV_ERR_WORKSPACE / CONV_ERR_UNSUPPORTED); a launch
 * failure returns CONV_ERR_CUDA.  Data problems never abort: they are reported
 * per column in `flags`:
 *   bit 0  CONV_FLAG_TRIGGERED  deep: CAPE > capelmt; shallow: passed exits E1-E3
 *   bit 1  CONV_FLAG_ACTIVE     scheme produced non-zero tendencies
 *   bit 2  CONV_FLAG_LIMITED    deep mass flux cut by the q >= q_min limiter
 *   bit 3  CONV_FLAG_NEWTON     a Newton solve did not converge: FP64, its last
 *                               correction exceeded 1e-4 K; mixed path, the error
 *                               its last step leaves (0.1/K x correction^2 by
 *                               quadratic convergence) exceeded 1e-3 K
 *   bit 4  CONV_FLAG_BADINPUT   T outside (100, 400) K, q outside [0, 0.1),
 *                               ps outside (5e4, 1.2e5) Pa or not finite;
 *                               all outputs of the column are zero
 *   bits 8-10 (shallow)         exit stage: 1 LCL too high, 2 no LFC,
 *                               3 CIN too large, 4 plume dies at the LCL; 0 none
 */
#ifndef CONV_H
#define CONV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* conv_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  CONV_OK = 0,
  CONV_ERR_ARG = 1,         /* invalid argument (NULL, size, range)          */
  CONV_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed          */
  CONV_ERR_WORKSPACE = 3,   /* workspace missing, too small or misaligned    */
  CONV_ERR_UNSUPPORTED = 4, /* valid request the library does not implement  */
  CONV_ERR_TIMEOUT = 5      /* reserved: a bounded device wait gave up       */
} conv_status;

typedef enum { CONV_FP64 = 0, CONV_MIXED = 1 } conv_precision;

enum {
  CONV_FLAG_TRIGGERED = 1,
  CONV_FLAG_ACTIVE = 2,
  CONV_FLAG_LIMITED = 4,
  CONV_FLAG_NEWTON = 8,
  CONV_FLAG_BADINPUT = 16,
  CONV_EXIT_SHIFT = 8
};

#define CONV_MAX_LEVELS 32
#define CONV_MAX_PLUMES 8

/* Vertical grid.  Interface pressure p_i = hyai[i]*p0 + hybi[i]*ps for
 * i = 0 (model top) .. pver (surface); mid-layer p_k = (p_k + p_k+1)/2.
 * hyai/hybi: HOST arrays of pver+1 doubles, copied into kernel parameters. */
typedef struct {
  int32_t pver;   /* 4 .. 32 levels                                   */
  int32_t n_cols; /* columns to process (>= 0)                        */
  int32_t ld;     /* leading dimension of profile arrays, >= n_cols   */
  int32_t reserved;
  const double* hyai;
  const double* hybi;
  double p0; /* Pa */
} conv_grid;

/* Deep scheme parameters (defaults in brackets; conv_deep_defaults fills them). */
typedef struct {
  double capelmt;        /* CAPE trigger threshold, J/kg [70]                      */
  double lambda_default; /* entrainment rate at the launch level, 1/m [1e-3]       */
  double tau_default;    /* CAPE relaxation time, s [3600]                         */
  double c0;             /* rain conversion rate, 1/m [2e-3]                       */
  double alpha_dd;       /* downdraft evaporation fraction [0.2]                   */
  double p_launch_min;   /* launch level searched where p_mid >= this, Pa [6e4]    */
  double p_top_lim;      /* no plume/parcel above p_mid < this, Pa [4e3]           */
  double q_min;          /* limiter floor on q + dt dq/dt, kg/kg [1e-12]           */
  double ent_zscale;     /* entrainment decays as zscale/(dz + zscale), m [1000]   */
  int32_t n_newton_lcl;  /* LCL Newton steps [6]                                   */
  int32_t n_newton_h;    /* moist inversions: Newton from the environment
                            temperature until a correction falls below 1e-7 K
                            (the convergence test), at most 1 + n_newton_h steps
                            [15]; a solve whose last correction stays above 1e-4 K
                            sets CONV_FLAG_NEWTON (mixed path: see the precision
                            contract above)                                     */
  int32_t n_plumes;      /* plume-spectrum variant, 1..CONV_MAX_PLUMES [1 = bulk
                            plume]: n plumes with entrainment rates lambda *
                            spread^(i/(n-1) - 1/2), each carrying 1/n of the
                            cloud-base mass flux and detraining at its own top
                            (a plume whose top is at or below the LCL layer drops
                            out); the highest top starts the downdraft and is
                            reported as ktop.  > 1 runs the extended kernel
                            instantiations; refused by conv_batch_*, the
                            adjoints and mass-flux profile outputs
                            (CONV_ERR_UNSUPPORTED). */
  int32_t reserved;      /* 0 */
  double plume_spread;   /* largest / smallest entrainment rate of the spectrum, >= 1 [4] */
} conv_deep_params;

/* Shallow scheme parameters. */
typedef struct {
  double eps_s;     /* plume mixing rate, 1/m [2e-3]                           */
  double tke;       /* boundary-layer TKE, m2/s2 [1]                           */
  double c_m;       /* cloud-base mass-flux coefficient [0.03]                 */
  double cin_scale; /* CIN e-folding in units of tke [10]                      */
  double cin_max;   /* exit E3 above this CIN, J/kg [50]                       */
  double a_w;       /* buoyancy coefficient of the w2 equation [1]             */
  double b_w;       /* drag coefficient of the w2 equation [2]                 */
  double ql_crit;   /* liquid left in the plume, kg/kg [1e-3]                  */
  double p_lcl_min; /* exit E1 if the LCL pressure is below, Pa [7e4]          */
  double p_lfc_min; /* exit E2 if no LFC at p >= this, Pa [5e4]                */
  double p_top_lim; /* Pa [4e3]                                                */
  int32_t n_newton_lcl;  /* [6], as in conv_deep_params                         */
  int32_t n_newton_h;    /* [15], as in conv_deep_params                         */
  double evap_k;    /* rain evaporation variant, 1/((kg/kg) m) [0 = off]: rain made
                       in a plume layer falls through the layers below it, each
                       taking the fraction 1 - exp(-evap_k max(qs - q, 0) dz) of
                       the flux arriving from above (moistening and cooling it);
                       the rest is the precipitation.  > 0 runs the extended
                       kernel instantiations; not supported by conv_batch_* and
                       the adjoints (CONV_ERR_UNSUPPORTED). */
} conv_shallow_params;

/* Inputs (DEVICE pointers). T,q: [pver][ld] double (FP64) or float (MIXED);
 * ps, lambda, tau: [ld] double.  lambda/tau may be NULL (parameter defaults). */
typedef struct {
  const void* T;
  const void* q;
  const double* ps;
  const double* lambda;
  const double* tau;
} conv_in;

/* Outputs of one scheme (DEVICE pointers).  dTdt (K/s), dqdt (kg/kg/s):
 * [pver][ld], element type as T.  prec (kg m-2 s-1), cape (deep: CAPE J/kg;
 * shallow: CIN J/kg), mb (cloud-base mass flux, kg m-2 s-1), cons_err (relative
 * column enthalpy + water residual; FP64, or in MIXED the compensated FP32
 * evaluation listed under Precision): [ld] double.  flags and
 * level indices: [ld] int32; kb = launch/source layer, klcl = LCL layer,
 * ktop = cloud-top layer (-1 unless active), kaux = deep: downdraft top layer
 * (-1 unless active) / shallow: LFC layer (-1 if none).
 * Mass-flux profiles (kg m-2 s-1, [pver][ld], element type as T) describe the
 * plume as a passive tracer sees it (conv_tracer_transport):
 *   mu: updraft mass flux leaving layer k through its top interface;
 *   du: updraft air detrained into layer k, carrying the plume value that
 *       arrives from layer k+1;
 *   md: downdraft mass flux leaving layer k through its bottom interface
 *       (downward positive), all of which detrains into the layer below the
 *       downdraft's lowest level.
 * Deep: mu = M_b eta on ktop+1..kb, du = M_b eta(ktop+1) at ktop, md = M_b
 * alpha eta_d on kaux..kb-1.  Shallow: mu = M_b on ktop+1..kb, du = M_b (1 -
 * exp(-eps_s dz)) on the layers between ktop and the LCL layer and M_b at ktop,
 * md = 0.  Every element is written (zero outside the plume and in inactive
 * columns).  Writing them selects separate kernel instantiations, so runs
 * without them are unaffected.  Not supported by conv_batch_* and
 * conv_pipeline_* (CONV_ERR_UNSUPPORTED).
 * dTdt, dqdt, prec and flags are required; the rest may be NULL. */
typedef struct {
  void* dTdt;
  void* dqdt;
  double* prec;
  int32_t* flags;
  int32_t* kb;
  int32_t* klcl;
  int32_t* ktop;
  int32_t* kaux;
  double* cape;
  double* mb;
  double* cons_err;
  void* mu;
  void* du;
  void* md;
} conv_out;

/* Kernel variant.  CONV_PATH_PLAIN: one thread per column runs the whole scheme
 * (no compaction; the FP64 baseline).  CONV_PATH_COMPACT: a trigger pass over
 * all columns compacts the convecting ones into device queues (warp ballot,
 * one atomic per warp) and plume passes run only over the queues.  AUTO is
 * COMPACT for runs that include the deep scheme, PLAIN for shallow-only runs.
 * block_threads 0 = library default.
 * mapping (compacted path): how the trigger pass maps columns to threads --
 * CONV_MAP_THREAD one column per thread (the default, also for 0), or
 * CONV_MAP_WARP one column per warp, lane k taking level k (the level-parallel
 * parts of the pass at once: prologue, height scan, launch-level reduction, the
 * undilute parcel's inversions; measured slower on the benchmark grid, kept as
 * the autotuner's alternative).  Results agree to rounding: FP64 decisions and
 * outputs as the thread mapping's within the parity tolerances.
 * stage_events (optional, may be NULL): three caller-created cudaEvent_t the
 * library records on `stream` -- [0] before its first kernel, [1] after the
 * trigger pass (plain path: after its only kernel), [2] after its last kernel
 * -- so a caller can time each pass; recording changes no work. */
typedef enum { CONV_PATH_AUTO = 0, CONV_PATH_PLAIN = 1, CONV_PATH_COMPACT = 2 } conv_path;
typedef enum { CONV_MAP_DEFAULT = 0, CONV_MAP_THREAD = 1, CONV_MAP_WARP = 2 } conv_mapping;
typedef struct {
  int32_t path;
  int32_t block_threads;
  int32_t mapping; /* conv_mapping */
  int32_t reserved1;
  void* const* stage_events;
} conv_launch;

/* Fill parameter structs with the defaults listed above. */
void conv_deep_defaults(conv_deep_params* p);
void conv_shallow_defaults(conv_shallow_params* p);

/* Human-readable name of a status code (static string). */
const char* conv_status_str(conv_status s);

/* Device workspace a run call needs for this grid, precision and launch
 * (launch may be NULL = defaults).  Zero for the plain path.  The workspace
 * must be 256-byte aligned; its contents need not be initialised. */
size_t conv_workspace_bytes(const conv_grid* grid, conv_precision prec,
                            const conv_launch* launch);

/* Deep convection (Alg. 2) on the state in `in`; writes `out`. dt (s) is used
 * by the moisture limiter.  Returns after enqueueing on `stream`. */
conv_status conv_deep_run(const conv_grid* grid, const conv_in* in, const conv_deep_params* par,
                          double dt, conv_precision prec, const conv_out* out,
                          const conv_launch* launch, void* ws, size_t ws_bytes,
                          conv_stream stream);

/* Shallow convection (Alg. 3) on the state in `in` (lambda/tau ignored). */
conv_status conv_shallow_run(const conv_grid* grid, const conv_in* in,
                             const conv_shallow_params* par, conv_precision prec,
                             const conv_out* out, const conv_launch* launch, void* ws,
                             size_t ws_bytes, conv_stream stream);

/* Deep convection, then shallow convection on T + dt*dTdt_deep, q + dt*dqdt_deep
 * (the order of Alg. 1), fused: the intermediate state never leaves the chip. */
conv_status conv_deep_shallow_run(const conv_grid* grid, const conv_in* in,
                                  const conv_deep_params* dpar, const conv_shallow_params* spar,
                                  double dt, conv_precision prec, const conv_out* deep_out,
                                  const conv_out* shallow_out, const conv_launch* launch,
                                  void* ws, size_t ws_bytes, conv_stream stream);

/* ------------------------------------------------------------------ adjoint
 * Reverse-mode gradient of the deep scheme, for tuning lambda and tau or for
 * sensitivity studies.  No counterpart in the paper (it gives the forward
 * scheme only); the forward scheme it differentiates is the one conv_deep_run
 * computes (Alg. 2: launch level, LCL, undilute parcel and CAPE, entraining
 * updraft with rain, saturated downdraft, flux-form tendencies, CAPE closure
 * and moisture limiter).  Per column i it evaluates
 *   P_i  surface precipitation (kg m-2 s-1, = prec of conv_deep_run)
 *   H_i  = sum_k w_k * m_k * cp * dTdt_k,i   (W m-2 for w = 1)
 * (m_k = dp_k / g: layer mass per unit area; w_k = w_heat[k], or p_mid_k / ps_i
 * when w_heat is NULL) and the gradient of J_i = gP[i] * P_i + gH[i] * H_i:
 *   gT, gq  [pver][ld] doubles: dJ/dT (per K), dJ/dq (per kg/kg)
 *   glambda, gtau  [ld] doubles: dJ/dlambda, dJ/dtau
 * gT, gq, glambda, gtau: all four DEVICE buffers (gradient wanted) or all NULL
 * (P_out / H_out only).  P_out, H_out: DEVICE [ld] doubles or NULL; at least one
 * output must be requested.  gP, gH: DEVICE [ld] doubles, either may be NULL
 * (zero).  w_heat: HOST [pver] doubles or NULL, copied into the launch.  FP64
 * only (CONV_MIXED -> CONV_ERR_UNSUPPORTED); in->T, in->q are doubles;
 * in->lambda / in->tau may be NULL (defaults).  Outputs are owned by the caller
 * and written for every column: zeros where the scheme is not active (not
 * triggered, no cloud, closure off, bad input).  Discrete choices (levels,
 * saturation, the downdraft cap and the moisture limiter) are held at their
 * forward values: the result is the derivative of the smooth piece the inputs
 * lie on.  One thread per column recomputes the forward scheme (nothing is
 * kept between calls), then runs the reverse sweep; Newton solves are
 * differentiated by the implicit function theorem.  Asynchronous on `stream`;
 * allocates nothing; no workspace. */
conv_status conv_deep_adjoint(const conv_grid* grid, const conv_in* in,
                              const conv_deep_params* par, double dt, conv_precision prec,
                              const double* gP, const double* gH, const double* w_heat,
                              double* gT, double* gq, double* glambda, double* gtau,
                              double* P_out, double* H_out, conv_stream stream);

/* Adjoint of the fused step (no counterpart in the paper): deep convection,
 * then shallow convection on T + dt*dTdt_deep, max(q + dt*dqdt_deep, 0), as
 * conv_deep_shallow_run computes it.  Per column it evaluates
 *   Pd, Hd, Ps, Hs   precipitation and H = sum_k w_k m_k cp dTdt_k of the deep
 *                    and of the shallow scheme (w as for conv_deep_adjoint)
 * into obj ([4][ld] DEVICE doubles: rows Pd, Hd, Ps, Hs; NULL = not wanted) and,
 * when `gradient` is non-zero, the gradient of
 *   J = gPd*Pd + gHd*Hd + gPs*Ps + gHs*Hs
 * with respect to T, q (gT, gq: [pver][ld]), lambda and tau (glambda, gtau:
 * [ld]).  gT and gq are required in both modes: they also hold the deep
 * tendencies the shallow scheme reads.  gPd..gHs: DEVICE [ld] doubles or NULL
 * (zero).  The gradient flows through the shallow scheme into its input state,
 * and from there into T, q directly and through the deep tendencies (the q
 * floor at zero passes no gradient where it binds).  Shallow level choices
 * (LCL, LFC, cloud top), saturation and rain on/off are held, as the deep
 * scheme's are in conv_deep_adjoint; the shallow closure is differentiated
 * through CIN and the source density.  FP64 only; one thread per column
 * recomputes both schemes with tapes; no workspace; asynchronous on `stream`. */
conv_status conv_deep_shallow_adjoint(const conv_grid* grid, const conv_in* in,
                                      const conv_deep_params* dpar,
                                      const conv_shallow_params* spar, double dt,
                                      conv_precision prec, const double* gPd, const double* gHd,
                                      const double* gPs, const double* gHs,
                                      const double* w_heat, double* gT, double* gq,
                                      double* glambda, double* gtau, double* obj, int gradient,
                                      conv_stream stream);

/* ------------------------------------------------------------------ driver
 * State advance of a multi-step column driver (no counterpart in the paper,
 * whose scheme runs inside a full model): after one conv_deep_shallow_run on
 * (T, q), update in place, level by level,
 *   T <- T + dt*((dTdt_deep + dTdt_shallow) + (T_relax - T)/tau_relax)
 *   q <- max(q + dt*((dqdt_deep + dqdt_shallow) + (q_relax - q)/tau_relax), 0)
 * The Newtonian relaxation towards reference profiles stands in for the large
 * scale forcing the rest of the model would supply; tau_relax <= 0 switches it
 * off (T_relax, q_relax may then be NULL).  T, q, T_relax, q_relax and the
 * output tendencies are DEVICE [pver][ld] arrays of the precision's type;
 * asynchronous on `stream`. */
conv_status conv_advance(const conv_grid* grid, void* T, void* q, const void* T_relax,
                         const void* q_relax, double tau_relax, const conv_out* deep_out,
                         const conv_out* shallow_out, double dt, conv_precision prec,
                         conv_stream stream);

/* ------------------------------------------------------------------ tracer transport
 * Convective transport of passive tracers (a variant both cited schemes carry:
 * ZM and UW move constituents with their plume mass fluxes, Sec. II-A; the
 * paper times only the thermodynamic loops).  Each scheme mixes a tracer as it
 * mixes its conserved moist static energy, with no source term, in flux form
 * with upwind compensating subsidence, per layer
 *   m_k dc_k/dt = mu_k (c_{k-1} - c_k) + du_k (cu_{k+1} - c_k)
 *               + md_k (c_{k+1} - c_k) [+ md_{kb-1} (cd_{kb-1} - c_kb) at kb],
 * with the updraft value cu (from kb upwards) and the downdraft value cd (from
 * kaux downwards) mixed by their entrainment.
 *
 * deep_out / shallow_out: the conv_out of a run that wrote mu and du (deep also
 * md), with flags, kb and ktop (deep also kaux); either may be NULL, not both.
 * tracers: DEVICE [ntr][pver][ld] of the precision's type (tracer n at offset
 * n*pver*ld); tend_deep / tend_shallow: the same layout, required with their
 * scheme's outputs when ntr > 0; every element of the first n_cols columns is
 * written.  With both schemes the shallow
 * scheme transports max(c + dt*tend_deep, 0), the tracer after the deep update
 * (Alg. 1 order, as conv_deep_shallow_run treats humidity).  ps: [ld] double
 * (layer masses).  ntr >= 0; dt > 0 when both schemes are given.  Validation
 * errors: CONV_ERR_ARG.  Asynchronous on `stream`; allocates nothing. */
conv_status conv_tracer_transport(const conv_grid* grid, const double* ps,
                                  const conv_out* deep_out, const conv_out* shallow_out,
                                  double dt, int ntr, const void* tracers, void* tend_deep,
                                  void* tend_shallow, conv_precision prec, conv_stream stream);

/* ------------------------------------------------------------------ momentum transport
 * Convective momentum transport (a variant the cited schemes carry: the ZM and
 * UW schemes move horizontal momentum with their plumes, Sec. II-A).  A wind
 * component is carried like a tracer (conv_tracer_transport, same mass-flux
 * profiles and layout), except that inside each plume the convective-scale
 * pressure gradient pushes the plume's momentum towards the environment's
 * (Gregory, Kershaw and Inness 1997): a plume crossing layer k from its
 * neighbour j (the layer below for the updrafts, above for the downdraft) gains
 *   cp * (plume flux continuing from j) * (u_k - u_j),
 * cp = cp_up for the updrafts, cp_down for the downdraft, and the layer's
 * environment loses the same.  Per layer this is the tracer budget above with
 * the plumes' momenta, minus those pressure forces; equivalently the divergence
 * of the interface eddy fluxes, so the column's momentum is conserved exactly.
 * cp_up = cp_down = 0 is the tracer transport; at 1 a plume's momentum equals
 * the environment's at every layer it crosses.
 *
 * uv: DEVICE [2][pver][ld] of the precision's type, u then v (component n at
 * offset n*pver*ld); tend_deep / tend_shallow: the same layout (m/s2), required
 * with their scheme's outputs; every element of the first n_cols columns is
 * written.  With both schemes the shallow scheme transports u + dt*tend_deep
 * (no floor: a wind component takes either sign).  cp_up, cp_down in [0, 1];
 * the other arguments as for conv_tracer_transport.  Validation errors:
 * CONV_ERR_ARG.  Asynchronous on `stream`; allocates nothing. */
conv_status conv_momentum_transport(const conv_grid* grid, const double* ps,
                                    const conv_out* deep_out, const conv_out* shallow_out,
                                    double dt, double cp_up, double cp_down, const void* uv,
                                    void* tend_deep, void* tend_shallow, conv_precision prec,
                                    conv_stream stream);

/* ------------------------------------------------------------------ host pipeline
 * conv_deep_shallow_run on HOST buffers (no counterpart in the paper: there the
 * data never leaves the host).  A plan splits the grid's columns into chunks of
 * chunk_cols; a run copies chunk j+1 in while chunk j computes and chunk j-1
 * copies out, on three streams of the plan, so the host link carries both
 * directions at once.  Plan time allocates (device staging for three chunks,
 * streams, events); runs allocate nothing and are asynchronous with respect to
 * the host: they are ordered after earlier work on `stream`, and later work on
 * `stream` waits for the last copy out.  Host arrays: conv_in / conv_out
 * layouts of the plan's grid (n_cols, ld), HOST pointers, page-locked for the
 * copies to be asynchronous; the optional outputs (kb ... cons_err) and
 * lambda/tau may be NULL.  The grid's hyai/hybi are copied at plan time. */
typedef struct conv_pipeline conv_pipeline;
conv_status conv_pipeline_plan(const conv_grid* grid, conv_precision prec, int chunk_cols,
                               conv_pipeline** out);
conv_status conv_pipeline_run(conv_pipeline* p, const conv_in* host_in,
                              const conv_deep_params* dpar, const conv_shallow_params* spar,
                              double dt, const conv_out* host_deep, const conv_out* host_shallow,
                              conv_stream stream);
void conv_pipeline_free(conv_pipeline* p);

/* ------------------------------------------------------------------ batches
 * Many grids / ensemble members of uneven column counts and level counts in one
 * trigger launch over all their columns and one persistent launch over a common
 * device queue of convecting columns (the GPU answer to the load imbalance the
 * paper meets with OpenMP dynamic scheduling, Sec. IV-A).  Each member is a
 * complete fused deep->shallow problem with its own grid, parameters and
 * buffers; results equal those of conv_deep_shallow_run on the compacted path
 * for that member alone. */
typedef struct {
  conv_grid grid; /* hyai/hybi: host arrays, copied at plan time */
  conv_in in;
  conv_out deep_out;
  conv_out shallow_out;
  conv_deep_params deep;
  conv_shallow_params shallow;
  double dt;
} conv_member;

typedef struct conv_batch conv_batch; /* opaque plan */

/* Validate every member as conv_deep_shallow_run would (CONV_ERR_ARG names no
 * member; check them singly to find it), copy the descriptors to the device and
 * choose a launch shape (from the autotuner's process-wide cache when it holds
 * one for this precision, level count and active-fraction bucket).  Plan time
 * allocates: host memory for the plan and a device descriptor table
 * (cudaMalloc + synchronous copy); runs allocate nothing.  n_members >= 1,
 * total columns < 2^31. */
conv_status conv_batch_plan(const conv_member* members, int n_members, conv_precision prec,
                            conv_batch** out);

/* Device workspace a run of this plan needs (256-byte aligned). */
size_t conv_batch_workspace_bytes(const conv_batch* b);

/* Enqueue the batched run on `stream`: queue reset, trigger pass, persistent
 * plume pass.  No host synchronisation and no allocation, so it may be captured
 * into a CUDA graph and replayed (the member buffers must stay valid).
 * stage_events: optional three cudaEvent_t recorded as for conv_launch. */
conv_status conv_batch_run(const conv_batch* b, void* ws, size_t ws_bytes, conv_stream stream,
                           void* const* stage_events);

/* Time candidate launch shapes on this plan's own data -- the trigger pass with
 * one column per thread in blocks of 64/128/256 and with one column per warp
 * (CONV_MAP_WARP), then the plume pass in blocks of 64/128/256 with its
 * persistent grid -- `reps` runs each after one warm-up, keep the fastest in
 * the plan and in the process-wide cache.  Synchronises `stream`; not
 * capturable.  Outputs hold the last run's results. */
conv_status conv_batch_autotune(conv_batch* b, void* ws, size_t ws_bytes, conv_stream stream,
                                int reps);

/* Launch shape currently chosen (any pointer may be NULL); trigger_mapping is a
 * conv_mapping (CONV_MAP_THREAD or CONV_MAP_WARP). */
conv_status conv_batch_config(const conv_batch* b, int32_t* trigger_block, int32_t* plume_block,
                              int32_t* plume_grid, int32_t* trigger_mapping);

/* Set the launch shape by hand: trigger_mapping CONV_MAP_THREAD or
 * CONV_MAP_WARP, trigger_block and plume_block 64, 128 or 256 (the plume pass's
 * persistent grid follows from its block and this device's occupancy).
 * CONV_ERR_ARG for other values. */
conv_status conv_batch_set_config(conv_batch* b, int32_t trigger_mapping, int32_t trigger_block,
                                  int32_t plume_block);

/* The last autotune's measurements, ms per batched run: ms[0..2] trigger blocks
 * 64/128/256 (one column per thread), ms[3] one column per warp, ms[4..6] plume
 * blocks 64/128/256 (each with the best trigger shape); ms holds 7 floats.
 * CONV_ERR_ARG if the plan has not been autotuned. */
conv_status conv_batch_tune_record(const conv_batch* b, float* ms);

/* Release the plan and its device descriptor table (NULL is a no-op). */
void conv_batch_free(conv_batch* b);

/* ---------------------------------------------------------------- sharding
 * One grid's columns split over several GPUs by convective work: the GPU
 * counterpart of the paper's proportional partitioning of the column
 * computations between devices (Sec. IV-D).  The columns are independent, so
 * each GPU runs the fused step on its own contiguous range (the inputs and
 * outputs offset by the range's first column, ld unchanged) with no exchange
 * on the data path; the ranges are chosen so that each holds about the same
 * cost  w_all * columns + w_active * triggered columns,  the triggered columns
 * counted from the flags of a previous run (the deep scheme's trigger varies
 * slowly from step to step, and the plume pass only runs on those columns).
 *
 * conv_count_triggered: counts[j] = number of columns among j*block ..
 * min((j+1)*block, n_cols) - 1 whose deep flags have CONV_FLAG_TRIGGERED.
 * flags: DEVICE int32[n_cols] (a deep conv_out.flags); counts: DEVICE
 * int32[ceil(n_cols/block)], overwritten.  Asynchronous on `stream` (one memset,
 * one kernel); CONV_ERR_ARG for n_cols < 0, block < 1 or missing pointers.
 *
 * conv_partition_columns: HOST function.  block_triggered: HOST
 * int32[ceil(n_cols/block)] (each 0 .. the block's column count), e.g. the
 * element-wise sum of every rank's counts; w_all, w_active >= 0, not both 0.
 * Writes bounds[0 .. n_parts] (HOST int32): bounds[0] = 0, bounds[n_parts] =
 * n_cols, non-decreasing, every inner bound a multiple of block at the block
 * boundary closest to r/n_parts of the total cost.  Part r is columns
 * bounds[r] .. bounds[r+1] - 1 (possibly empty).  Deterministic: every rank
 * given the same counts computes the same bounds.  CONV_ERR_ARG on invalid
 * arguments (bounds untouched then). */
conv_status conv_count_triggered(const int32_t* flags, int32_t n_cols, int32_t block,
                                 int32_t* counts, conv_stream stream);
conv_status conv_partition_columns(int32_t n_cols, int32_t block,
                                   const int32_t* block_triggered, double w_all,
                                   double w_active, int32_t n_parts, int32_t* bounds);

/* Largest n_cols accepted by conv_deep_shallow_run_noalloc. */
#define CONV_NOALLOC_MAX_COLS 65536

/* conv_deep_shallow_run without a caller workspace.  No counterpart in the paper:
 * it exists for callers that cannot allocate device memory where they call --
 * a host model whose memory manager owns the whole device pool, or code that
 * must not call cudaMalloc because it may synchronise the device or is not
 * allowed while a stream is being captured.  The caller still owns and passes
 * every input and output; the compacted path's scratch (queue and per-slot
 * trigger state) lives in a library-owned static device array sized for
 * CONV_NOALLOC_MAX_COLS columns of up to CONV_MAX_LEVELS levels in FP64
 * (about 17 MB), held on every GPU that loads the library until the process
 * exits.  Nothing here calls cudaMalloc, cudaFree or any allocating routine.
 *   - n_cols > CONV_NOALLOC_MAX_COLS returns CONV_ERR_ARG before anything runs;
 *     all other arguments are validated as for conv_deep_shallow_run.
 *   - The first call on a device looks up that device's address of the array
 *     (for the device current at the call) and caches it with the identity of
 *     the device's context; make that first call before any stream capture.
 *     After a device reset (a new context) the next call looks the address up
 *     again, so make that call outside a capture too.  The stream must belong
 *     to the current device.
 *   - Every call shares the one array, which keeps the last call's contents;
 *     the queue length is reset at the start of each call.  Calls that overlap
 *     on the GPU (other streams, other host threads) race on it: serialise them.
 * Outputs are those of conv_deep_shallow_run on the compacted path. */
conv_status conv_deep_shallow_run_noalloc(const conv_grid* grid, const conv_in* in,
                                          const conv_deep_params* dpar,
                                          const conv_shallow_params* spar, double dt,
                                          conv_precision prec, const conv_out* deep_out,
                                          const conv_out* shallow_out, conv_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* CONV_H */
