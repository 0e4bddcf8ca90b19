// validate.h -- host-side argument checks shared by the C-ABI entry points
// (conv_api.cu) and the host pipeline (pipeline.cu), so that a pipeline run is
// refused before it enqueues any copy.
#pragma once

#include "conv.h"

namespace cvg {

// Every field of a deep / shallow parameter block inside its documented range.
bool deep_params_ok(const conv_deep_params* p);
bool shallow_params_ok(const conv_shallow_params* p);

// The grid as conv_deep_shallow_run accepts it: 4 <= pver <= CONV_MAX_LEVELS,
// 0 <= n_cols <= ld, finite positive p0, finite level coefficients with the
// interfaces ordered top to surface.
bool grid_ok(const conv_grid* g);

}  // namespace cvg
