// Declarations of the on-device FWER calibration (fwer.cu), used by api.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mcd_internal.cuh"

namespace mcd {

// Calibration state of one design: bracket [lo, hi] of the alpha scale with
// the estimated FWER at its ends, the current scale, the end that the last
// step replaced (-1 low, +1 high, 0 none) and whether the split is valid.
struct FwerState {
    double lo, hi, f_lo, f_hi, s;
    int32_t side;
    int32_t ok;
};

cudaError_t launch_fwer_init(int J, const DesignRec* dr, const double* w, double alpha0, FwerState* st, double* b,
                             DevStatus* status, cudaStream_t stream);
cudaError_t launch_fwer_update(int J, const DesignRec* dr, const double* w, const double* p, double alpha0, int round,
                               bool last, FwerState* st, double* b, double* scale, double* fwer,
                               cudaStream_t stream);

}  // namespace mcd
