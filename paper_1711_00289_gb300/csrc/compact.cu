// compact.cu -- the compacted path: the GPU answer to the load imbalance the
// paper fights with OpenMP dynamic scheduling (Sec. IV-A), which arises because
// the deep scheme's column work is skipped wherever no deep cloud forms.
// Instead of letting a warp carry idle lanes through the plume code:
//
//  k_trigger (all columns, one thread each): prologue, launch level, LCL,
//    undilute parcel and CAPE.  A column that does not trigger deep convection
//    is finished here: zero deep outputs, then the shallow scheme on the
//    unchanged state, reusing the prologue and -- when its launch layer is the
//    lowest layer -- the deep LCL and saturated parcel.  Triggered columns are
//    appended to a device queue (warp ballot, one atomic per warp) with their
//    trigger state (launch/LCL/EL levels, CAPE, parcel temperatures).
//  k_plume (one thread per queue slot): entraining updraft, downdraft,
//    closure and deep outputs, then the shallow scheme on the deep-updated
//    state.  Its grid covers every possible slot and reads the queue length
//    from device memory, so no host synchronisation is needed (capturable).
#include "compact.h"

namespace cvg {

// This thread's slice of the block's shared level arrays (nullptr: none).
template <class R, int PASS>
__device__ __forceinline__ R* smem_levels() {
  if constexpr (SmemLevels<R, PASS>::on) {
    extern __shared__ __align__(16) unsigned char cvg_smem[];
    return reinterpret_cast<R*>(cvg_smem) + threadIdx.x;
  } else {
    return nullptr;
  }
}

// Trigger pass of one column (all lanes of the warp must call it: the queue
// append is a warp ballot).  `tag` is what the queue records for the column
// (the column index, or a batch-wide index), `live` false for padding lanes.
// SMEM: the column's level arrays live in the block's shared memory
// (smem_levels), not in the thread's local arrays.
template <class R, bool EXT = false, bool SMEM = false, int PASS = kPassTrigger>
__device__ __forceinline__ void trigger_body(const RunArgs& a, const CompactWs<R>& w, int i,
                                             bool live, int tag) {
  Column<R> c;
  LevelBuf<R> cbuf;
  DeepOut o;
  DeepTrig<R> t;
  t.triggered = false;
  t.Tp = w.Tp + tag;  // parcel temperatures go straight to the workspace, by column
  t.tps = (size_t)w.cap;
  bool valid = false;
  if (live) {
    init_column(c, a.L, input_src<R>(a, i), a.ps[i], cbuf);
    if constexpr (SMEM)
      bind_levels(c, smem_levels<R, PASS>(), blockDim.x, SmemLevels<R, PASS>::which);
    o.prec = o.cape = o.mb = o.cons = 0.0;
    o.flags = 0;
    o.kb = o.klcl = o.ktop = o.kaux = -1;
    valid = prologue(deep_q(a, R(0)).p_top_lim, c);
    if (!valid) {
      o.flags = CONV_FLAG_BADINPUT;
    } else {
      deep_trigger(c, a.dp, deep_q(a, R(0)), t);
      o.kb = t.kb;
      o.klcl = t.klcl;
      o.cape = t.cape;
      if (t.triggered) o.flags |= CONV_FLAG_TRIGGERED;
      if (t.newton > Mth<R>::newton_tol) o.flags |= CONV_FLAG_NEWTON;
    }
  }
  // queue append: one atomic per warp, slots in lane order
  const unsigned ball = __ballot_sync(0xffffffffu, t.triggered);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (ball) {
    const int leader = __ffs(ball) - 1;
    if (lane == leader) base = atomicAdd(w.count, __popc(ball));
    base = __shfl_sync(0xffffffffu, base, leader);
  }
  if (!live) return;
  if (t.triggered) {
    const int slot = base + __popc(ball & ((1u << lane) - 1u));
    w.queue[slot] = tag;
    w.levels[slot] = t.kb | (t.klcl << 8) | (t.kel << 16);
    w.cape[slot] = t.cape;
    store_deep_scalars(a, i, o);  // scalars now; tendencies and the rest in the plume pass
    if constexpr (kThreePass) w.s_info[tag] = kShalTriggered;
    return;
  }
  out_col<R, EXT>(a.od, a, i).zero(0, c.pver);
  store_deep_scalars(a, i, o);
  if (!(a.mode & MODE_SHALLOW)) return;
  if constexpr (kThreePass) {
    // the shallow pass runs later: hand it what it can reuse
    int info = 0;
    if (valid) {
      const bool same_src = t.kb == c.pver - 1 && a.sp.p_top_lim == a.dp.p_top_lim &&
                            a.sp.n_newton_lcl == a.dp.n_newton_lcl &&
                            a.sp.n_newton_h == a.dp.n_newton_h && t.klcl >= c.ktl;
      info = kShalValid | (same_src ? kShalSameSrc : 0) | (t.pL_exact ? kShalExact : 0) |
             (t.newton <= Mth<R>::newton_tol ? kShalBoundOk : 0) | ((t.klcl & 0xff) << 8) |
             ((c.ktl & 0xff) << 16);
      w.s_pL[tag] = t.pL;
      w.s_buoy[tag] = t.maybe_buoy;
    }
    w.s_info[tag] = info;
    return;
  }
  ShalOut s;
  const auto so = out_col<R, EXT>(a.os, a, i);
  if (!valid) {
    shallow_column(a.sp, shal_q(a, R(0)), c, s, so);  // flags the column as bad input
  } else {
    // same state as the deep scheme saw: reuse the prologue, and the LCL/parcel
    // when the deep launch layer is the shallow source layer
    const bool same_src = t.kb == c.pver - 1 && a.sp.p_top_lim == a.dp.p_top_lim &&
                          a.sp.n_newton_lcl == a.dp.n_newton_lcl &&
                          a.sp.n_newton_h == a.dp.n_newton_h && t.klcl >= c.ktl;
    const DeepBound bound{t.klcl, c.ktl, t.maybe_buoy};
    const bool bound_ok = t.newton <= Mth<R>::newton_tol;
    if (a.sp.p_top_lim != a.dp.p_top_lim) prologue(shal_q(a, R(0)).p_top_lim, c);
    ShallowSeed<R> seed{t.pL, t.klcl, t.pL_exact, t.Tp, t.tps};
    shallow_column(a.sp, shal_q(a, R(0)), c, s, so, same_src ? &seed : nullptr, true,
                   bound_ok ? &bound : nullptr);
  }
  store_shallow_scalars(a, i, s);
}

template <class R, bool EXT>
__global__ void __launch_bounds__(kTriggerBlock, SmThreads<R>::trigger / kTriggerBlock)
    k_trigger(const __grid_constant__ RunArgs a, CompactWs<R> w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  trigger_body<R, EXT, SmemLevels<R, kPassTrigger>::on>(a, w, i, i < a.n, i);
}

// Plume pass of the column in queue slot `slot`: column i of member a, queued
// under `tag` (its index in the workspace's per-column arrays).
template <class R, bool EXT = false, bool SMEM = false>
__device__ __forceinline__ void plume_body(const RunArgs& a, const CompactWs<R>& w, int slot,
                                           int i, int tag) {
  Column<R> c;
  LevelBuf<R> cbuf;
  init_column(c, a.L, input_src<R>(a, i), a.ps[i], cbuf);
  if constexpr (SMEM)
    bind_levels(c, smem_levels<R, kPassPlume>(), blockDim.x, SmemLevels<R, kPassPlume>::which);
  DeepTrig<R> t;
  const int lvl = w.levels[slot];
  t.kb = lvl & 0xff;
  t.klcl = (lvl >> 8) & 0xff;
  t.kel = (lvl >> 16) & 0xff;
  t.cape = w.cape[slot];
  t.triggered = true;
  t.newton = 0.f;
  t.Tp = w.Tp + tag;
  t.tps = (size_t)w.cap;
  DeepOut o;
  o.prec = o.mb = o.cons = 0.0;
  o.cape = t.cape;
  o.flags = a.od.flags[i];  // trigger-stage bits written by the trigger pass
  o.kb = t.kb;
  o.klcl = t.klcl;
  o.ktop = o.kaux = -1;
  const DeepQ<R>& Q = deep_q(a, R(0));
  const R lam = a.lam ? (R)a.lam[i] : Q.lambda_default;
  const R tau = a.tau ? (R)a.tau[i] : Q.tau_default;
  prologue(Q.p_top_lim, c);
  deep_plume(c, a.dp, Q, lam, tau, t, o, out_col<R, EXT>(a.od, a, i));
  if (t.newton > Mth<R>::newton_tol) o.flags |= CONV_FLAG_NEWTON;
  store_deep_scalars(a, i, o);
  if (!(a.mode & MODE_SHALLOW) || kThreePass) return;
  c.s = after_deep_src<R>(a, i, false);  // limiter keeps q >= q_min up to rounding
  // Same ps, so the deep prologue's log-thicknesses stand: only the heights are
  // rebuilt.  An updated state out of range leaves the full check to the scheme,
  // which flags the column as bad input.
  const ShalQ<R>& SQ = shal_q(a, R(0));
  const bool ok = prologue<R, false>(SQ.p_top_lim, c);
  ShalOut s;
  shallow_column(a.sp, SQ, c, s, out_col<R, EXT>(a.os, a, i), (const ShallowSeed<R>*)nullptr, ok);
  store_shallow_scalars(a, i, s);
}

// Counting sort of the queue slots [base, min(base + BLOCK, count)) of one block
// by plume depth kb - kel (0 .. CONV_MAX_LEVELS - 1, one bin per lane of warp
// 0): returns the slot this thread runs, -1 for none.  Every thread of the
// block calls it (it synchronises the block); within a depth the order is that
// of the shared-memory atomics, which only decides which thread runs a column.
// Plume depth of a queued column, kb - kel of its undilute parcel (levels word).
__device__ __forceinline__ int depth_key(int lvl) {
  return min(31, max(0, (lvl & 0xff) - ((lvl >> 16) & 0xff)));
}

template <int BLOCK>
struct DepthSort {
  int off[32];
  int slot[BLOCK];
};
static_assert(CONV_MAX_LEVELS <= 32, "one depth bin per lane");
template <int BLOCK>
__device__ __forceinline__ int depth_sorted_slot(const int* __restrict__ levels, int base,
                                                 int count, DepthSort<BLOCK>& s) {
  static_assert(BLOCK >= 32 && BLOCK <= 1024, "block of whole warps");
  const int t = threadIdx.x;
  const int nv = min(BLOCK, count - base);
  if (t < 32) s.off[t] = 0;
  __syncthreads();
  int key = 0, rank = 0;
  if (t < nv) {
    key = depth_key(levels[base + t]);
    rank = atomicAdd(&s.off[key], 1);
  }
  __syncthreads();
  if (t < 32) {  // exclusive scan of the 32 bin counts
    const int v = s.off[t];
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (t >= d) x += y;
    }
    s.off[t] = x - v;
  }
  __syncthreads();
  if (t < nv) s.slot[s.off[key] + rank] = base + t;
  __syncthreads();
  return t < nv ? s.slot[t] : -1;
}

template <class R, bool EXT>
__global__ void __launch_bounds__(kPlumeBlock, SmThreads<R>::plume / kPlumeBlock)
    k_plume(const __grid_constant__ RunArgs a, CompactWs<R> w) {
  const int count = *w.count;
  const int base = blockIdx.x * kPlumeBlock;
  if (base >= count) return;  // whole block: nothing queued this far
  int slot = base + (int)threadIdx.x;
  if constexpr (kPlumeSort) {
    __shared__ DepthSort<kPlumeBlock> ds;
    slot = depth_sorted_slot<kPlumeBlock>(w.levels, base, count, ds);
    if (slot < 0) return;
  } else {
    if (slot >= count) return;
  }
  const int i = w.queue[slot];
  plume_body<R, EXT, SmemLevels<R, kPassPlume>::on>(a, w, slot, i, i);
}

// Shallow pass of the three-pass layout (column i, workspace index tag): a
// triggered column on its deep-updated state; a column the deep scheme left as
// it was on its own state, reusing the deep trigger's LCL and parcel (when its
// launch layer is the lowest) and its buoyancy bound, as the trigger pass would.
template <class R, bool EXT = false>
__device__ __forceinline__ void shallow_body(const RunArgs& a, const CompactWs<R>& w, int i,
                                             int tag) {
  const int info = w.s_info[tag];
  Column<R> c;
  LevelBuf<R> cbuf;
  ShalOut s;
  const auto so = out_col<R, EXT>(a.os, a, i);
  const ShalQ<R>& SQ = shal_q(a, R(0));
  if (info & kShalTriggered) {
    init_column(c, a.L, after_deep_src<R>(a, i, false), a.ps[i], cbuf);
    shallow_column(a.sp, SQ, c, s, so);
  } else if (!(info & kShalValid)) {
    init_column(c, a.L, input_src<R>(a, i), a.ps[i], cbuf);
    shallow_column(a.sp, SQ, c, s, so);  // flags the column as bad input
  } else {
    init_column(c, a.L, input_src<R>(a, i), a.ps[i], cbuf);
    prologue(SQ.p_top_lim, c);
    const int klcl = (info >> 8) & 0xff;
    const ShallowSeed<R> seed{w.s_pL[tag], klcl, (info & kShalExact) != 0, w.Tp + tag,
                              (size_t)w.cap};
    const DeepBound bound{klcl, (info >> 16) & 0xff, w.s_buoy[tag]};
    shallow_column(a.sp, SQ, c, s, so, (info & kShalSameSrc) ? &seed : nullptr, true,
                   (info & kShalBoundOk) ? &bound : nullptr);
  }
  store_shallow_scalars(a, i, s);
}

template <class R, bool EXT>
__global__ void __launch_bounds__(kCompactBlock, SmThreads<R>::shallow / kCompactBlock)
    k_shallow(const __grid_constant__ RunArgs a, CompactWs<R> w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) shallow_body<R, EXT>(a, w, i, i);
}

// Kernels that keep level arrays in shared memory get a carve-out that fits
// their resident blocks at the largest level count (plus the 1 KB the device
// reserves per block), the rest of the unified L1 / shared memory staying L1
// for the local arrays.  Set once per kernel, before its first launch.
template <class R, int PASS>
static void set_carveout(const void* f, int block, int blocks_per_sm) {
  if constexpr (SmemLevels<R, PASS>::on) {
    int dev = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        per_sm <= 0)
      return;
    const size_t most = smem_levels_bytes<R, PASS>(CONV_MAX_LEVELS, block);
    const size_t need = (size_t)blocks_per_sm * (most + 1024);
    const size_t pct = (100 * need + per_sm - 1) / per_sm;
    cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)(pct > 100 ? 100 : pct));
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
  } else {
    (void)f, (void)block, (void)blocks_per_sm;
  }
}

template <class R>
static void prefer_shared() {
  static const bool done = [] {
    constexpr int tb = SmThreads<R>::trigger / kTriggerBlock;
    constexpr int pb = SmThreads<R>::plume / kPlumeBlock;
    set_carveout<R, kPassTrigger>((const void*)k_trigger<R, false>, kTriggerBlock, tb);
    set_carveout<R, kPassTrigger>((const void*)k_trigger<R, true>, kTriggerBlock, tb);
    set_carveout<R, kPassPlume>((const void*)k_plume<R, false>, kPlumeBlock, pb);
    set_carveout<R, kPassPlume>((const void*)k_plume<R, true>, kPlumeBlock, pb);
    return true;
  }();
  (void)done;
}

size_t compact_workspace_bytes(int n, int pver, bool fp64) {
  const size_t rb = fp64 ? 8 : 4;
  return ws_offsets(n, pver, rb).total;
}

template <class R>
static cudaError_t launch_t(const RunArgs& a, void* ws, size_t ws_bytes) {
  const WsOffsets off = ws_offsets(a.n, a.L.pver, sizeof(R));
  if (ws_bytes < off.total) return cudaErrorInvalidValue;
  char* base = static_cast<char*>(ws);
  CompactWs<R> w;
  w.count = reinterpret_cast<int*>(base + off.count);
  w.queue = reinterpret_cast<int*>(base + off.queue);
  w.levels = reinterpret_cast<int*>(base + off.levels);
  w.cape = reinterpret_cast<double*>(base + off.cape);
  w.Tp = reinterpret_cast<R*>(base + off.Tp);
  w.s_pL = reinterpret_cast<double*>(base + off.s_pL);
  w.s_buoy = reinterpret_cast<uint32_t*>(base + off.s_buoy);
  w.s_info = reinterpret_cast<int32_t*>(base + off.s_info);
  w.cap = a.n;
  record_stage(a, 0);
  cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(int), a.stream);
  if (e != cudaSuccess) return e;
  const int grid = (a.n + kCompactBlock - 1) / kCompactBlock;
  const int grid_t = (a.n + kTriggerBlock - 1) / kTriggerBlock;
  const int grid_p = (a.n + kPlumeBlock - 1) / kPlumeBlock;
  const size_t sm_t = smem_levels_bytes<R, kPassTrigger>(a.L.pver, kTriggerBlock);
  const size_t sm_p = smem_levels_bytes<R, kPassPlume>(a.L.pver, kPlumeBlock);
  prefer_shared<R>();
  if (a.mapping == CONV_MAP_WARP) {
    e = launch_trigger_warp(a, w);
  } else {
    NvtxRange r("conv: trigger pass (all columns)");
    if (a.ext)
      k_trigger<R, true><<<grid_t, kTriggerBlock, sm_t, a.stream>>>(a, w);
    else
      k_trigger<R, false><<<grid_t, kTriggerBlock, sm_t, a.stream>>>(a, w);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  record_stage(a, 1);
  {
    NvtxRange r("conv: plume pass (queued columns)");
    if (a.ext)
      k_plume<R, true><<<grid_p, kPlumeBlock, sm_p, a.stream>>>(a, w);
    else
      k_plume<R, false><<<grid_p, kPlumeBlock, sm_p, a.stream>>>(a, w);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (kThreePass && (a.mode & MODE_SHALLOW)) {
    NvtxRange r("conv: shallow pass (all columns)");
    if (a.ext)
      k_shallow<R, true><<<grid, kCompactBlock, 0, a.stream>>>(a, w);
    else
      k_shallow<R, false><<<grid, kCompactBlock, 0, a.stream>>>(a, w);
    e = cudaGetLastError();
  }
  record_stage(a, 2);
  return e;
}

cudaError_t launch_compact(const RunArgs& a, bool fp64, void* ws, size_t ws_bytes) {
  if (a.n == 0) return cudaSuccess;
  return fp64 ? launch_t<double>(a, ws, ws_bytes) : launch_t<float>(a, ws, ws_bytes);
}

// ---------------------------------------------------------------- batched ensemble
// Members of uneven column and level counts share one trigger launch over the
// concatenation of their columns (column g belongs to the member m with
// offsets[m] <= g < offsets[m+1]) and one persistent plume launch that walks the
// common queue of triggered columns with a grid-stride loop until the queue
// length read from device memory is exhausted -- no host synchronisation, no
// waiting on other blocks.

__device__ __forceinline__ int find_member(const int* off, int M, int g) {
  int lo = 0, hi = M;  // invariant: off[lo] <= g < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <class R, int BLOCK>
__global__ void __launch_bounds__(BLOCK, SmThreads<R>::trigger / BLOCK)
    k_batch_trigger(BatchDev b, const RunArgs* __restrict__ members, CompactWs<R> w) {
  const int g = blockIdx.x * BLOCK + threadIdx.x;
  const bool live = g < b.total;
  int m = 0, i = 0;
  if (live) {
    m = find_member(b.offsets, b.n_members, g);
    i = g - b.offsets[m];
  }
  trigger_body<R, false, SmemLevels<R, kPassBatchTrigger>::on, kPassBatchTrigger>(members[m], w, i,
                                                                                 live, g);
}

template <class R, int BLOCK>
__global__ void __launch_bounds__(BLOCK, SmThreads<R>::plume / BLOCK)
    k_batch_plume(BatchDev b, const RunArgs* __restrict__ members, CompactWs<R> w) {
  const int count = *w.count;
  for (int slot = blockIdx.x * BLOCK + threadIdx.x; slot < count; slot += gridDim.x * BLOCK) {
    const int g = w.queue[slot];
    const int m = find_member(b.offsets, b.n_members, g);
    plume_body<R, false, SmemLevels<R, kPassPlume>::on>(members[m], w, slot, g - b.offsets[m],
                                                        g);
  }
}

// Shared-memory set-up of the batch kernels at one block size: the carve-out
// and the dynamic size of the largest level count (set_carveout).
template <class R, int BLOCK>
static void batch_smem_setup() {
  static const bool done = [] {
    set_carveout<R, kPassBatchTrigger>((const void*)k_batch_trigger<R, BLOCK>, BLOCK,
                                       SmThreads<R>::trigger / BLOCK);
    set_carveout<R, kPassPlume>((const void*)k_batch_plume<R, BLOCK>, BLOCK,
                                SmThreads<R>::plume / BLOCK);
    return true;
  }();
  (void)done;
}

template <class R, int BLOCK>
__global__ void __launch_bounds__(BLOCK, SmThreads<R>::shallow / BLOCK)
    k_batch_shallow(BatchDev b, const RunArgs* __restrict__ members, CompactWs<R> w) {
  const int g = blockIdx.x * BLOCK + threadIdx.x;
  if (g >= b.total) return;
  const int m = find_member(b.offsets, b.n_members, g);
  if (members[m].mode & MODE_SHALLOW) shallow_body<R>(members[m], w, g - b.offsets[m], g);
}

template <class R, int BLOCK>
static int plume_occupancy(int max_pver) {
  batch_smem_setup<R, BLOCK>();
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_batch_plume<R, BLOCK>, BLOCK,
                                                    smem_levels_bytes<R, kPassPlume>(max_pver, BLOCK)) !=
      cudaSuccess)
    return 1;
  return blocks < 1 ? 1 : blocks;
}

int batch_plume_occupancy(bool fp64, int block, int max_pver) {
  switch (block) {
    case 64:
      return fp64 ? plume_occupancy<double, 64>(max_pver) : plume_occupancy<float, 64>(max_pver);
    case 256:
      return fp64 ? plume_occupancy<double, 256>(max_pver)
                  : plume_occupancy<float, 256>(max_pver);
    default:
      return fp64 ? plume_occupancy<double, 128>(max_pver)
                  : plume_occupancy<float, 128>(max_pver);
  }
}

template <class R, int BLOCK>
static void launch_trig(const BatchDev& b, const CompactWs<R>& w, int max_pver,
                        cudaStream_t s) {
  batch_smem_setup<R, BLOCK>();
  k_batch_trigger<R, BLOCK><<<(b.total + BLOCK - 1) / BLOCK, BLOCK,
                              smem_levels_bytes<R, kPassBatchTrigger>(max_pver, BLOCK), s>>>(b, b.members,
                                                                                     w);
}
template <class R, int BLOCK>
static void launch_plume(const BatchDev& b, const CompactWs<R>& w, int grid, int max_pver,
                         cudaStream_t s) {
  batch_smem_setup<R, BLOCK>();
  k_batch_plume<R, BLOCK><<<grid, BLOCK, smem_levels_bytes<R, kPassPlume>(max_pver, BLOCK), s>>>(
      b, b.members, w);
}

template <class R>
static cudaError_t batch_t(const BatchDev& b, const BatchShape& sh, void* ws, size_t ws_bytes,
                           cudaStream_t s, cudaEvent_t* ev) {
  const WsOffsets off = ws_offsets(b.total, sh.max_pver, sizeof(R));
  if (ws_bytes < off.total) return cudaErrorInvalidValue;
  char* base = static_cast<char*>(ws);
  CompactWs<R> w;
  w.count = reinterpret_cast<int*>(base + off.count);
  w.queue = reinterpret_cast<int*>(base + off.queue);
  w.levels = reinterpret_cast<int*>(base + off.levels);
  w.cape = reinterpret_cast<double*>(base + off.cape);
  w.Tp = reinterpret_cast<R*>(base + off.Tp);
  w.s_pL = reinterpret_cast<double*>(base + off.s_pL);
  w.s_buoy = reinterpret_cast<uint32_t*>(base + off.s_buoy);
  w.s_info = reinterpret_cast<int32_t*>(base + off.s_info);
  w.cap = b.total;
  NvtxRange r("conv: batched run (trigger + persistent plume pass)");
  if (ev && ev[0]) cudaEventRecord(ev[0], s);
  cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (sh.trigger_mapping == 1) {
    launch_batch_trigger_warp(b, w, s);
  } else {
    switch (sh.trigger_block) {
      case 64: launch_trig<R, 64>(b, w, sh.max_pver, s); break;
      case 256: launch_trig<R, 256>(b, w, sh.max_pver, s); break;
      default: launch_trig<R, 128>(b, w, sh.max_pver, s); break;
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev && ev[1]) cudaEventRecord(ev[1], s);
  switch (sh.plume_block) {
    case 64: launch_plume<R, 64>(b, w, sh.plume_grid, sh.max_pver, s); break;
    case 256: launch_plume<R, 256>(b, w, sh.plume_grid, sh.max_pver, s); break;
    default: launch_plume<R, 128>(b, w, sh.plume_grid, sh.max_pver, s); break;
  }
  e = cudaGetLastError();
  if (kThreePass && e == cudaSuccess) {
    k_batch_shallow<R, 128><<<(b.total + 127) / 128, 128, 0, s>>>(b, b.members, w);
    e = cudaGetLastError();
  }
  if (ev && ev[2]) cudaEventRecord(ev[2], s);
  return e;
}

cudaError_t launch_batch(const BatchDev& b, const BatchShape& sh, bool fp64, void* ws,
                         size_t ws_bytes, cudaStream_t s, cudaEvent_t* ev) {
  if (b.total == 0) return cudaSuccess;
  return fp64 ? batch_t<double>(b, sh, ws, ws_bytes, s, ev)
              : batch_t<float>(b, sh, ws, ws_bytes, s, ev);
}

}  // namespace cvg
