// Declarations of the thin-plate spline fit and maximiser (tps.cu), used by api.cu.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "mcd_internal.cuh"

namespace mcd {

// Doubles of workspace that one fit of N points in k dimensions needs.
size_t tps_workspace_doubles(int N, int k);

// Fit one surface: x [N][k], y [N] (device) -> coef [N + k + 1], fitted [N]
// (may be NULL).  `bad` is a device int the fit clears and sets when the
// projected system is not positive definite (then coef and fitted are NaN
// and the status word gets MCD_ENOTSPD with index `surf`); `amax` a device
// word for max |A_ij|.
cudaError_t tps_fit_one(const double* x, const double* y, int N, int k, double s, double* coef, double* fitted,
                        double* ws, int* bad, unsigned long long* amax, DevStatus* status, int surf,
                        cudaStream_t stream);

// Doubles of workspace of tps_gcv.
size_t tps_gcv_workspace_doubles(int N, int k);

// GCV scores V(s) of one surface for the n_s smoothing values (host array)
// into score (device [n_s]); bad, amax, trace: device scratch words.
cudaError_t tps_gcv(const double* x, const double* y, int N, int k, const double* s_values, int n_s, double* score,
                    double* ws, int* bad, unsigned long long* amax, double* trace, cudaStream_t stream);

// Maximise n_surf fitted surfaces inside the box [lo, hi] (device, k each).
cudaError_t tps_argmax(const double* x, const double* coef, const double* fitted, int n_surf, int N, int k,
                       const double* lo, const double* hi, int iters, double* xbest, double* fbest,
                       cudaStream_t stream);

}  // namespace mcd
