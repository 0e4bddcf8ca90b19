// compact.h -- workspace layout of the compacted path (internal).
#pragma once

#include "launch.h"

namespace cvg {

constexpr int kCompactBlock = 128;

// Resident threads per SM the compacted kernels are compiled for (register cap
// 65536 / threads).  The mixed kernels are latency-bound chains of dependent
// FP32 operations: more resident warps hide more of that latency, until the
// spills of a tighter cap cost more.  Measured sweeps of the caps put the
// trigger pass at 1408 threads per SM (40 registers; 1664 threads, 32
// registers, was 21% slower) and the plume pass at 896 (72 registers; 768 was
// 18% slower, 1024 2% slower).  The FP64 kernels are bound by the FP64 pipe and
// need enough warps in flight to keep it fed: 896 threads (72 registers).
template <class R>
struct SmThreads {
  static constexpr int trigger = 896, plume = 896;
};
template <>
struct SmThreads<float> {
  static constexpr int trigger = 1408, plume = 896;
};

// Device workspace of the compacted path, carved from one caller buffer:
//   count  int32      queue length (zeroed at the start of every run)
//   queue  int32[n]   column index of each queued (deep-triggered) column
//   levels int32[n]   kb | klcl << 8 | kel << 16 of the queued column
//   cape   double[n]  CAPE of the queued column
//   Tp     R[pver][n] undilute parcel temperature on ktl..klcl, by column (the
//                     trigger pass writes it for every column with a parcel)
// (n = queue capacity: the columns of the run, or of all members of a batch)
template <class R>
struct CompactWs {
  int* count;
  int* queue;
  int* levels;
  double* cape;
  R* Tp;
  int cap;  // queue capacity (columns); row stride of Tp
};

struct WsOffsets {
  size_t count, queue, levels, cape, Tp, total;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline WsOffsets ws_offsets(int n, int pver, size_t real_bytes) {
  WsOffsets o;
  const size_t nn = n < 1 ? 1 : (size_t)n;
  o.count = 0;
  o.queue = 256;
  o.levels = o.queue + align256(4 * nn);
  o.cape = o.levels + align256(4 * nn);
  o.Tp = o.cape + align256(8 * nn);
  o.total = o.Tp + align256(real_bytes * (size_t)pver * nn);
  return o;
}

size_t compact_workspace_bytes(int n, int pver, bool fp64);
cudaError_t launch_compact(const RunArgs& a, bool fp64, void* ws, size_t ws_bytes);

// Batched ensemble: device copies of the members' run descriptors and the
// prefix sums of their column counts (offsets[n_members] = total).
struct BatchDev {
  const RunArgs* members;
  const int* offsets;
  int n_members;
  int total;
};
// Launch shape chosen by the plan (and the autotuner).
struct BatchShape {
  int max_pver;
  int trigger_block;  // 64, 128 or 256
  int plume_block;    // 64, 128 or 256
  int plume_grid;     // persistent grid: SMs x resident blocks per SM
};
int batch_plume_occupancy(bool fp64, int block);
cudaError_t launch_batch(const BatchDev& b, const BatchShape& sh, bool fp64, void* ws,
                         size_t ws_bytes, cudaStream_t s, cudaEvent_t* ev);

}  // namespace cvg
