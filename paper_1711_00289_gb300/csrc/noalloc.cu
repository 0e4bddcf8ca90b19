// noalloc.cu -- conv_deep_shallow_run_noalloc: the fused deep->shallow run on
// the compacted path with its scratch (device queue, queue length, per-slot
// trigger state) in a file-scope device array instead of a caller workspace.
//
// For callers that cannot allocate device memory at the point of the call: a
// host model whose memory manager owns the whole device pool, or code that must
// not call cudaMalloc because it can synchronise the device or is not allowed
// while a stream is being captured.  Such callers still pass their inputs and
// outputs; only the scratch comes from here.
#include <mutex>

#include "compact.h"

namespace {

// Scratch of the compacted path sized for CONV_NOALLOC_MAX_COLS columns of up
// to CONV_MAX_LEVELS levels in FP64 (the larger of the two precisions).  Every
// GPU that loads the library holds it until the process exits.
constexpr size_t kScratchBytes =
    256 + 4 * CONV_NOALLOC_MAX_COLS + 4 * CONV_NOALLOC_MAX_COLS + 8 * CONV_NOALLOC_MAX_COLS +
    8 * (size_t)CONV_MAX_LEVELS * CONV_NOALLOC_MAX_COLS;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device.  In host code the symbol
// is only a host-side stand-in, so the address is looked up once per device
// (with that device current) and cached.
conv_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CONV_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return CONV_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return CONV_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return CONV_OK;
}

}  // namespace

extern "C" conv_status conv_deep_shallow_run_noalloc(const conv_grid* grid, const conv_in* in,
                                                     const conv_deep_params* dpar,
                                                     const conv_shallow_params* spar, double dt,
                                                     conv_precision prec,
                                                     const conv_out* deep_out,
                                                     const conv_out* shallow_out,
                                                     conv_stream stream) {
  if (!grid) return CONV_ERR_ARG;
  if (grid->n_cols > CONV_NOALLOC_MAX_COLS || grid->pver > CONV_MAX_LEVELS) return CONV_ERR_ARG;
  conv_launch launch = {CONV_PATH_COMPACT, 0, 0, 0, nullptr};
  conv_grid g = *grid;
  if (g.pver < 1) return CONV_ERR_ARG;
  const size_t need = conv_workspace_bytes(&g, prec, &launch);
  if (need == 0 || need > kScratchBytes) return CONV_ERR_ARG;
  void* ws = nullptr;
  const conv_status s = scratch_for_current_device(&ws);
  if (s != CONV_OK) return s;
  // The compacted path zeroes its queue length at the start of every run.
  return conv_deep_shallow_run(grid, in, dpar, spar, dt, prec, deep_out, shallow_out, &launch,
                               ws, kScratchBytes, stream);
}
