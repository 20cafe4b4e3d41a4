// Host-side entry points of the smoothing kernels (smooth.cu) that are not
// in mcd_internal.cuh: the shape check and the FP32-grid launcher.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "mcd_internal.cuh"

namespace mcd {

// smooth_argmax for FP32 grids: FP32 values in, FP32 smoothed values and
// argmax values out (same weights, stencil and argmax rules).
cudaError_t smooth_argmax_f32(int n_scen, int g1, int g2, const float* value, double bandwidth,
                              int degree, float* smoothed, int64_t* argmax_idx, float* argmax_val,
                              int64_t* raw_idx, float* raw_val, double* wbuf, float* wbuf32,
                              double* part_val, int64_t* part_idx, DevStatus* status, cudaStream_t stream);

// nullptr when smooth_argmax can launch n_scen grids of g1 x g2, else the
// reason it cannot.
const char* smooth_shape_error(int n_scen, int g1, int g2);

}  // namespace mcd
