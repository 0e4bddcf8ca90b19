// noalloc.cu -- conv_deep_shallow_run_noalloc: the fused deep->shallow run on
// the compacted path with its scratch (device queue, queue length, per-slot
// trigger state) in a file-scope device array instead of a caller workspace.
//
// For callers that cannot allocate device memory at the point of the call: a
// host model whose memory manager owns the whole device pool, or code that must
// not call cudaMalloc because it can synchronise the device or is not allowed
// while a stream is being captured.  Such callers still pass their inputs and
// outputs; only the scratch comes from here.
#include <cuda.h>

#include <mutex>

#include "compact.h"

namespace {

// Scratch of the compacted path sized for CONV_NOALLOC_MAX_COLS columns of up
// to CONV_MAX_LEVELS levels in FP64 (the larger of the two precisions).  Every
// GPU that loads the library holds it until the process exits.
constexpr size_t kScratchBytes =
    256 + 4 * CONV_NOALLOC_MAX_COLS + 4 * CONV_NOALLOC_MAX_COLS + 8 * CONV_NOALLOC_MAX_COLS +
    8 * (size_t)CONV_MAX_LEVELS * CONV_NOALLOC_MAX_COLS +
    (cvg::kThreePass ? (8 + 4 + 4) * (size_t)CONV_NOALLOC_MAX_COLS : 0);
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
  void* ptr;
  unsigned long long ctx_id;  // the context the address belongs to (0: unknown)
};
Cached g_cache[kMaxDevices] = {};

// The current context's process-unique id, through driver entry points the
// runtime hands out (the library does not link the driver library itself);
// 0 if the driver cannot say.  A device reset or a destroyed and re-created
// context gives a new id, so an address cached for the old one is not reused.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  struct Entry {
    GetCurrent get_current = nullptr;
    GetId get_id = nullptr;
  };
  // looked up once, by the first caller (a function-local static's
  // initialisation is thread-safe)
  static const Entry e = [] {
    Entry r;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                         &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      r.get_current = reinterpret_cast<GetCurrent>(f1);
      r.get_id = reinterpret_cast<GetId>(f2);
    }
    return r;
  }();
  if (!e.get_current || !e.get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (e.get_current(&ctx) != CUDA_SUCCESS || !ctx || e.get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of g_scratch in the current device's context.  In host code
// the symbol is only a host-side stand-in, so the address is looked up with
// that device current and cached per device together with the context it
// belongs to; a different context (after a device reset) is looked up anew.
conv_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CONV_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return CONV_ERR_UNSUPPORTED;
  // make the device's primary context current on this thread (initialising it
  // if needed; no allocation), so that it has an id to compare
  if (cudaSetDevice(dev) != cudaSuccess) return CONV_ERR_CUDA;
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(g_mu);
  Cached& c = g_cache[dev];
  if (!c.ptr || id == 0 || c.ctx_id != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return CONV_ERR_CUDA;
    c.ptr = p;
    c.ctx_id = id;
  }
  *out = c.ptr;
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
