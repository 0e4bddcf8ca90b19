// shard.cu -- splitting one grid's columns over several GPUs by convective
// work, the GPU counterpart of the paper's proportional partitioning of the
// column computations between Xeon and Xeon Phi cores (Sec. IV-D).  There the
// split follows each device's measured speed; here every device is the same and
// what varies is the work per column: the trigger pass costs about the same on
// every column, while the plume pass runs only on triggered columns.  So the
// columns are cut into contiguous ranges of near-equal cost
//     cost(column) = w_all + w_active * [column triggered],
// with the triggered columns of a previous step (or of a trigger-only pass)
// counted per block of columns on the device.
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "conv.h"

namespace {

// Triggered deep columns per block of `block` columns: one warp ballot per 32
// columns, one atomic per warp on the block's counter.  counts[] must hold
// ceil(n / block) zeroed ints.
__global__ void k_count_triggered(const int32_t* __restrict__ flags, int n, int block,
                                  int32_t* __restrict__ counts) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  const bool trig = live && (__ldg(flags + i) & CONV_FLAG_TRIGGERED) != 0;
  // a warp's 32 columns can straddle two count blocks when block is not a
  // multiple of 32: ballot per destination block
  const int b = live ? (int)(i / block) : -1;
  const unsigned live_mask = __ballot_sync(0xffffffffu, live);
  if (!live) return;
  const int lane = threadIdx.x & 31;
  const unsigned same = __match_any_sync(live_mask, b);
  const unsigned hits = __ballot_sync(live_mask, trig) & same;
  if (lane == __ffs(same) - 1 && hits) atomicAdd(counts + b, __popc(hits));
}

}  // namespace

extern "C" conv_status conv_count_triggered(const int32_t* flags, int32_t n_cols, int32_t block,
                                            int32_t* counts, conv_stream stream) {
  if (n_cols < 0 || block < 1 || (n_cols > 0 && (!flags || !counts))) return CONV_ERR_ARG;
  if (n_cols == 0) return CONV_OK;
  const long long nb = ((long long)n_cols + block - 1) / block;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)nb, s) != cudaSuccess)
    return CONV_ERR_CUDA;
  const int threads = 256;
  const long long grid = ((long long)n_cols + threads - 1) / threads;
  k_count_triggered<<<(unsigned)grid, threads, 0, s>>>(flags, n_cols, block, counts);
  return cudaGetLastError() == cudaSuccess ? CONV_OK : CONV_ERR_CUDA;
}

extern "C" conv_status conv_partition_columns(int32_t n_cols, int32_t block,
                                              const int32_t* block_triggered, double w_all,
                                              double w_active, int32_t n_parts, int32_t* bounds) {
  if (n_cols < 0 || block < 1 || n_parts < 1 || !bounds || !(w_all >= 0.0) ||
      !(w_active >= 0.0) || !(w_all + w_active > 0.0) || (n_cols > 0 && !block_triggered))
    return CONV_ERR_ARG;
  const long long nb = ((long long)n_cols + block - 1) / block;
  // prefix cost at each block boundary
  std::vector<double> pre((size_t)nb + 1, 0.0);
  for (long long j = 0; j < nb; ++j) {
    const long long cols = (j + 1 < nb) ? block : (long long)n_cols - j * (long long)block;
    const int32_t t = block_triggered[j];
    if (t < 0 || t > cols) return CONV_ERR_ARG;
    pre[(size_t)j + 1] = pre[(size_t)j] + w_all * (double)cols + w_active * (double)t;
  }
  const double total = pre[(size_t)nb];
  bounds[0] = 0;
  long long j = 0;
  for (int r = 1; r < n_parts; ++r) {
    // the block boundary closest to r/n_parts of the total cost, not before the
    // previous bound
    const double target = total * (double)r / (double)n_parts;
    while (j < nb && pre[(size_t)j + 1] <= target) ++j;
    long long pick = j;
    if (j < nb && pre[(size_t)j + 1] - target < target - pre[(size_t)j]) pick = j + 1;
    const long long col = pick * (long long)block;
    bounds[r] = (int32_t)(col < n_cols ? col : n_cols);
    if (bounds[r] < bounds[r - 1]) bounds[r] = bounds[r - 1];
  }
  bounds[n_parts] = n_cols;
  return CONV_OK;
}
