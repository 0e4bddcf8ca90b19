// compact.h -- workspace layout of the compacted path (internal).
#pragma once

#include "launch.h"

namespace cvg {

constexpr int kCompactBlock = 128;
// Block sizes of the single-grid trigger and plume passes.
#ifndef CVG_TRIGGER_BLOCK
#define CVG_TRIGGER_BLOCK 128
#endif
#ifndef CVG_PLUME_BLOCK
#define CVG_PLUME_BLOCK 128
#endif
constexpr int kTriggerBlock = CVG_TRIGGER_BLOCK, kPlumeBlock = CVG_PLUME_BLOCK;

// Resident threads per SM the compacted kernels are compiled for (register cap
// 65536 / threads).  The mixed kernels are latency-bound chains of dependent
// FP32 operations: more resident warps hide more of that latency, until the
// spills of a tighter cap cost more.  Measured sweeps of the caps put the
// trigger pass at 1280 threads per SM (48 registers: 0.433 ms, against 0.445 at
// 1408 threads and 40 registers, and 0.461 at 1024 threads and 64 registers,
// with the FP32 quotients and shared-memory log-thicknesses of the current
// kernel; 256-thread blocks at the same caps were no faster) and the plume
// pass at 896 (72 registers; 768 was 18% slower, 1024 2% slower).  The
// FP64 kernels are bound by the FP64 pipe and need enough warps in flight to
// keep it fed: 896 threads (72 registers).  (Build-time overrides, for sweeps.)
#ifndef CVG_TRIGGER_SM_THREADS
#define CVG_TRIGGER_SM_THREADS 1280
#endif
#ifndef CVG_PLUME_SM_THREADS
#define CVG_PLUME_SM_THREADS 896
#endif
// Where each pass of the mixed path keeps a column's level arrays zm (mid-layer
// heights) and dl (layer log-thicknesses): 0 both in the thread's local array,
// 1 both in shared memory, 2 zm in shared memory, 3 dl in shared memory.
// Measured on the 884,736-column step (trigger / plume pass, ms): 0: 0.473 /
// 0.383; 1: 0.537 / 0.383 (30 KB per 128-thread block leaves the trigger pass
// 7 resident blocks per SM); 2: 0.454 / 0.384; 3: 0.446 / 0.384 (measured at
// 1408 threads per SM).  With dl in shared memory (15 KB per 128-thread block,
// 10-11 blocks per SM) the trigger pass's local traffic drops; the plume pass,
// at 7 blocks per SM, already hits L1 on 57% of its local loads and gains
// nothing.
#ifndef CVG_SMEM_LEVELS_TRIGGER
#define CVG_SMEM_LEVELS_TRIGGER 3
#endif
#ifndef CVG_SMEM_LEVELS_PLUME
#define CVG_SMEM_LEVELS_PLUME 0
#endif
// The batched trigger pass (256-thread blocks after autotuning, 5 per SM: 30 KB
// of shared memory each for dl) keeps both arrays local: the 64-member
// ensemble ran 3.86 ms per step that way, 4.00 ms with dl shared, 4.05 with zm.
#ifndef CVG_SMEM_LEVELS_BATCH_TRIGGER
#define CVG_SMEM_LEVELS_BATCH_TRIGGER 0
#endif
#ifndef CVG_SHALLOW_SM_THREADS
#define CVG_SHALLOW_SM_THREADS 1408
#endif
template <class R>
struct SmThreads {
  static constexpr int trigger = 896, plume = 896, shallow = 896;
};
template <>
struct SmThreads<float> {
  static constexpr int trigger = CVG_TRIGGER_SM_THREADS, plume = CVG_PLUME_SM_THREADS,
                       shallow = CVG_SHALLOW_SM_THREADS;
};

// ShalInfo: what the three-pass trigger pass hands the shallow pass per column.
enum : int {
  kShalTriggered = 1,  // the deep scheme triggered: shallow on the updated state
  kShalValid = 2,      // valid input (otherwise the shallow pass flags bad input)
  kShalSameSrc = 4,    // the deep launch layer is the shallow source: reuse its LCL, parcel
  kShalExact = 8,      // the deep p_L is the FP64 value
  kShalBoundOk = 16    // the deep trigger converged: its buoyancy bound holds
  // bits 8-15: the deep parcel's LCL layer; bits 16-23: the deep top limit
};

// Shared-memory placement of the level arrays per pass (kPassTrigger: the
// trigger kernels, kPassPlume: the plume kernels): level-major, the thread
// index innermost, pver levels x block words per array.  FP64 keeps both in
// the threads' local arrays: its 8-byte words would leave room for too few
// blocks per SM.
enum : int { kPassTrigger = 0, kPassPlume = 1, kPassBatchTrigger = 2 };
template <class R, int PASS>
struct SmemLevels {
  static constexpr int which = 0;
  static constexpr bool on = false;
};
template <int PASS>
struct SmemLevels<float, PASS> {
  static constexpr int which = PASS == kPassTrigger        ? CVG_SMEM_LEVELS_TRIGGER
                               : PASS == kPassBatchTrigger ? CVG_SMEM_LEVELS_BATCH_TRIGGER
                                                           : CVG_SMEM_LEVELS_PLUME;
  static constexpr bool on = which != 0;
};
template <class R, int PASS>
inline size_t smem_levels_bytes(int pver, int block) {
  if constexpr (SmemLevels<R, PASS>::on) {
    const size_t arrays = SmemLevels<R, PASS>::which == 1 ? 2 : 1;
    return sizeof(R) * arrays * (size_t)pver * (size_t)block;
  } else {
    return 0;
  }
}

// Device workspace of the compacted path, carved from one caller buffer:
//   count  int32      queue length (zeroed at the start of every run)
//   queue  int32[n]   column index of each queued (deep-triggered) column
//   levels int32[n]   kb | klcl << 8 | kel << 16 of the queued column
//   cape   double[n]  CAPE of the queued column
//   Tp     R[pver][n] undilute parcel temperature on ktl..klcl, by column (the
//                     trigger pass writes it for every column with a parcel)
// (n = queue capacity: the columns of the run, or of all members of a batch)
#ifndef CVG_THREE_PASS
#define CVG_THREE_PASS 0
#endif
constexpr bool kThreePass = CVG_THREE_PASS != 0;

// CVG_PLUME_SORT = 1: the plume pass regroups the queue slots of each block by
// plume depth (kb - kel of the undilute parcel) before it runs them, so that
// the columns of a warp take level loops of similar length; the block's set of
// columns, and so its memory locality, stays as the trigger pass queued it.
// Measured on the 884,736-column grid: k_plume 0.3826 ms sorted and unsorted.
// Off by default; the batched plume pass never sorts (a block-synchronised
// sort took the ensemble from 3.92 to 4.55 ms, a warp-synchronised one over
// 256-slot windows to 7.9 ms: on its uncorrelated columns, regrouping a
// window's slots breaks the coalescing of the per-level column loads).
#ifndef CVG_PLUME_SORT
#define CVG_PLUME_SORT 0
#endif
constexpr bool kPlumeSort = CVG_PLUME_SORT != 0;

template <class R>
struct CompactWs {
  int* count;
  int* queue;
  int* levels;
  double* cape;
  R* Tp;
  int cap;  // queue capacity (columns); row stride of Tp
  // three-pass layout: what the shallow pass takes from the trigger pass, by column
  double* s_pL;     // deep LCL pressure
  uint32_t* s_buoy; // DeepTrig::maybe_buoy
  int32_t* s_info;  // packed flags and levels (ShalInfo)
};

struct WsOffsets {
  size_t count, queue, levels, cape, Tp, s_pL, s_buoy, s_info, total;
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
  o.s_pL = o.Tp + align256(real_bytes * (size_t)pver * nn);
  o.s_buoy = o.s_pL + (kThreePass ? align256(8 * nn) : 0);
  o.s_info = o.s_buoy + (kThreePass ? align256(4 * nn) : 0);
  o.total = o.s_info + (kThreePass ? align256(4 * nn) : 0);
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
  int trigger_mapping;  // 0: one column per thread; 1: one column per warp
  int trigger_block;  // 64, 128 or 256
  int plume_block;    // 64, 128 or 256
  int plume_grid;     // persistent grid: SMs x resident blocks per SM
};
int batch_plume_occupancy(bool fp64, int block, int max_pver);
// The trigger pass with one column per warp (warp.cu).
cudaError_t launch_trigger_warp(const RunArgs& a, const CompactWs<float>& w);
cudaError_t launch_trigger_warp(const RunArgs& a, const CompactWs<double>& w);
cudaError_t launch_batch_trigger_warp(const BatchDev& b, const CompactWs<float>& w,
                                      cudaStream_t s);
cudaError_t launch_batch_trigger_warp(const BatchDev& b, const CompactWs<double>& w,
                                      cudaStream_t s);
cudaError_t launch_batch(const BatchDev& b, const BatchShape& sh, bool fp64, void* ws,
                         size_t ws_bytes, cudaStream_t s, cudaEvent_t* ev);

}  // namespace cvg
