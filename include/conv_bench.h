/*
 * conv_bench.h -- measurement support of libconvgb.so (no counterpart in the
 * paper, whose timings are wall-clock seconds of CESM loops, Sec. V).
 *
 * The column schemes are bound by floating-point throughput, not by a dense
 * contraction or by HBM, so the roofline of a kernel is the time its
 * algorithmic operation counts need at the device's measured per-operation
 * throughput.  This entry point measures that throughput on the current device.
 */
#ifndef CONV_BENCH_H
#define CONV_BENCH_H

#include "conv.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CONV_OP_FMA = 0, /* a*b + c              */
  CONV_OP_EXP = 1, /* exp                  */
  CONV_OP_LOG = 2, /* log                  */
  CONV_OP_DIV = 3, /* a / b                */
  CONV_OP_POW = 4, /* pow(a, b)            */
  CONV_OP_SQRT = 5 /* sqrt                 */
} conv_op;

typedef enum {
  CONV_ARITH_FP64 = 0,      /* double, library functions                       */
  CONV_ARITH_FP32 = 1,      /* float, accurate library functions               */
  CONV_ARITH_FP32_FAST = 2  /* float, hardware approximations (__expf, ...)    */
} conv_arith;

/* Measure how many `op` evaluations per second the current device sustains in
 * `arith` (a grid of 8 independent dependency chains per thread, sized to fill
 * every SM; `iters` evaluations per chain; timed with CUDA events on a private
 * stream, synchronised).  Writes the rate to *ops_per_s.  Allocates and frees
 * 8 MB of device memory internally.  CONV_ERR_ARG for an unknown op/arith or
 * iters < 1; CONV_ERR_CUDA on a CUDA failure. */
conv_status conv_bench_op_rate(int op, int arith, int iters, double* ops_per_s);

/* The mixed path's FP32 quotient -- the division in every FP32 step of the
 * schemes -- applied elementwise, q[i] = a[i] / b[i] for 0 <= i < n, so that
 * it can be checked against IEEE division.  a, b, q: device arrays of n floats
 * (q overlapping neither a nor b); asynchronous on `stream`, no allocation.
 * CONV_ERR_ARG for n < 0 or a null array with n > 0; CONV_ERR_CUDA when the
 * launch fails. */
conv_status conv_bench_f32_quotient(const float* a, const float* b, float* q, int64_t n,
                                    conv_stream stream);

/* The LCL pressure of n parcels (T [K], q [kg/kg], p [Pa]; device arrays) by the
 * mixed path's FP32 solve (pL32, without its FP64 correction; p itself for a
 * parcel saturated where it is) and by the FP64 solve (pL64), each with at most
 * n_newton Newton steps from the Bolton first guess (the schemes' lifting
 * condensation level, Sec. II-A), so that the FP32 error can be checked against the band in
 * which the mixed path corrects it in FP64.  Asynchronous on `stream`, no
 * allocation.  CONV_ERR_ARG for n < 0, n_newton < 1 or a null array with
 * n > 0; CONV_ERR_CUDA when the launch fails. */
conv_status conv_bench_lcl(const float* T, const float* q, const float* p, float* pL32,
                           double* pL64, int64_t n, int n_newton, conv_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* CONV_BENCH_H */
