// microbench.cu -- per-operation throughput of the current device and a check
// of the mixed path's FP32 quotient (conv_bench.h).  Each thread of the rate
// kernel advances 8 independent chains; every chain step is one evaluation of
// the measured operation plus one FMA that keeps the argument bounded.  The
// FP32 operations are the schemes' own (column.cuh: Mth<float>, div_f32), so
// the rates weigh what the kernels execute.
#include <cuda_runtime.h>

#include "column.cuh"
#include "conv_bench.h"

namespace {

template <class R>
struct Ops;
template <>
struct Ops<double> {
  static __device__ double ex(double x) { return exp(x); }
  static __device__ double lg(double x) { return log(x); }
  static __device__ double dv(double a, double b) { return a / b; }
  static __device__ double pw(double a, double b) { return pow(a, b); }
  static __device__ double sq(double a) { return sqrt(a); }
};
template <>
struct Ops<float> {
  static __device__ float ex(float x) { return cvg::Mth<float>::es(x); }
  static __device__ float lg(float x) { return cvg::Mth<float>::lg(x); }
  static __device__ float dv(float a, float b) { return cvg::Mth<float>::dv(a, b); }
  static __device__ float pw(float a, float b) { return cvg::Mth<float>::pw(a, b); }
  static __device__ float sq(float a) { return sqrtf(a); }
};
struct FastF {
  static __device__ float ex(float x) { return __expf(x); }
  static __device__ float lg(float x) { return __logf(x); }
  static __device__ float dv(float a, float b) { return __fdividef(a, b); }
  static __device__ float pw(float a, float b) { return __powf(a, b); }
  static __device__ float sq(float a) { return sqrtf(a); }
};

template <class R, class O, int OP>
__global__ void k_rate(int iters, R seed, R* sink) {
  R x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = seed + R(0.01) * R(j) + R(1e-6) * R(threadIdx.x);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      R y;
      if (OP == CONV_OP_FMA) y = x[j] * R(0.999999) + R(1e-7);
      if (OP == CONV_OP_EXP) y = O::ex(x[j]) * R(0.25) + R(0.1);
      if (OP == CONV_OP_LOG) y = O::lg(x[j]) * R(0.25) + R(1.5);
      if (OP == CONV_OP_DIV) y = O::dv(R(1.7), x[j]) * R(0.5) + R(0.8);
      if (OP == CONV_OP_POW) y = O::pw(x[j], R(0.2857)) * R(0.5) + R(0.6);
      if (OP == CONV_OP_SQRT) y = O::sq(x[j]) * R(0.5) + R(0.6);
      x[j] = y;
    }
  }
  R s = R(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == R(-12345.0)) sink[0] = s;  // keeps the chains live
}

template <class R, class O>
cudaError_t run(int op, int iters, double* rate) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int block = 256, grid = sms * 8;
  R* sink = nullptr;
  e = cudaMalloc(&sink, 8 << 20);
  if (e != cudaSuccess) return e;
  cudaStream_t s;
  cudaEvent_t a, b;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto launch = [&](int n) {
    switch (op) {
      case CONV_OP_FMA: k_rate<R, O, CONV_OP_FMA><<<grid, block, 0, s>>>(n, R(1.1), sink); break;
      case CONV_OP_EXP: k_rate<R, O, CONV_OP_EXP><<<grid, block, 0, s>>>(n, R(0.3), sink); break;
      case CONV_OP_LOG: k_rate<R, O, CONV_OP_LOG><<<grid, block, 0, s>>>(n, R(1.3), sink); break;
      case CONV_OP_DIV: k_rate<R, O, CONV_OP_DIV><<<grid, block, 0, s>>>(n, R(1.2), sink); break;
      case CONV_OP_POW: k_rate<R, O, CONV_OP_POW><<<grid, block, 0, s>>>(n, R(1.2), sink); break;
      default: k_rate<R, O, CONV_OP_SQRT><<<grid, block, 0, s>>>(n, R(1.2), sink); break;
    }
  };
  launch(iters / 10 + 1);  // warm-up
  cudaEventRecord(a, s);
  launch(iters);
  cudaEventRecord(b, s);
  e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaStreamDestroy(s);
  cudaFree(sink);
  if (e == cudaSuccess) *rate = (double)grid * block * 8.0 * iters / (ms * 1e-3);
  return e;
}

__global__ void k_quotient(const float* __restrict__ a, const float* __restrict__ b,
                           float* __restrict__ q, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    q[i] = cvg::div_f32(a[i], b[i]);
}

__global__ void k_lcl(const float* __restrict__ T, const float* __restrict__ q,
                      const float* __restrict__ p, float* __restrict__ pL32,
                      double* __restrict__ pL64, int64_t n, int n_newton) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float nf = 0.f, nd = 0.f;
    const cvg::LclF32 s = cvg::lcl_f32(T[i], q[i], p[i], n_newton, nf);
    pL32[i] = s.saturated ? p[i] : s.pL;
    pL64[i] = cvg::lcl_p((double)T[i], (double)q[i], (double)p[i], n_newton, nd);
  }
}

}  // namespace

extern "C" conv_status conv_bench_lcl(const float* T, const float* q, const float* p,
                                      float* pL32, double* pL64, int64_t n, int n_newton,
                                      conv_stream stream) {
  if (n < 0 || n_newton < 1 || (n > 0 && (!T || !q || !p || !pL32 || !pL64))) return CONV_ERR_ARG;
  if (n == 0) return CONV_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CONV_ERR_CUDA;
  const int64_t want = (n + 255) / 256, cap = (int64_t)sms * 8;
  k_lcl<<<(unsigned)(want < cap ? want : cap), 256, 0, (cudaStream_t)stream>>>(T, q, p, pL32, pL64,
                                                                             n, n_newton);
  return cudaGetLastError() == cudaSuccess ? CONV_OK : CONV_ERR_CUDA;
}

extern "C" conv_status conv_bench_f32_quotient(const float* a, const float* b, float* q,
                                               int64_t n, conv_stream stream) {
  if (n < 0 || (n > 0 && (!a || !b || !q))) return CONV_ERR_ARG;
  if (n == 0) return CONV_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CONV_ERR_CUDA;
  const int64_t want = (n + 255) / 256, cap = (int64_t)sms * 8;
  k_quotient<<<(unsigned)(want < cap ? want : cap), 256, 0, (cudaStream_t)stream>>>(a, b, q, n);
  return cudaGetLastError() == cudaSuccess ? CONV_OK : CONV_ERR_CUDA;
}

extern "C" conv_status conv_bench_op_rate(int op, int arith, int iters, double* ops_per_s) {
  if (!ops_per_s || iters < 1 || op < CONV_OP_FMA || op > CONV_OP_SQRT) return CONV_ERR_ARG;
  cudaError_t e;
  switch (arith) {
    case CONV_ARITH_FP64: e = run<double, Ops<double>>(op, iters, ops_per_s); break;
    case CONV_ARITH_FP32: e = run<float, Ops<float>>(op, iters, ops_per_s); break;
    case CONV_ARITH_FP32_FAST: e = run<float, FastF>(op, iters, ops_per_s); break;
    default: return CONV_ERR_ARG;
  }
  return e == cudaSuccess ? CONV_OK : CONV_ERR_CUDA;
}
