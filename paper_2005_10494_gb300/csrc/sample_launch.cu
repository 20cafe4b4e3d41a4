// Selection and launch of the sampling kernels.
#include "mcd_internal.cuh"

namespace mcd {

const void* sample_kernel_f32_a(int d, bool grad);
const void* sample_kernel_f32_b(int d, bool grad);
const void* sample_kernel_f64_a(int d, bool grad);
const void* sample_kernel_f64_b(int d, bool grad);
const void* sample_kernel_mixed(bool grad);

namespace {

const void* select(int d_lo, int d_hi, bool grad, bool fp64) {
    if (d_lo < 1 || d_hi > kMaxD || d_lo > d_hi) return nullptr;
    if (d_lo != d_hi) return (fp64 || d_lo != 1 || d_hi != kMixedMaxD) ? nullptr : sample_kernel_mixed(grad);
    if (fp64) return d_lo <= 10 ? sample_kernel_f64_a(d_lo, grad) : sample_kernel_f64_b(d_lo, grad);
    return d_lo <= 10 ? sample_kernel_f32_a(d_lo, grad) : sample_kernel_f32_b(d_lo, grad);
}

}  // namespace

cudaError_t launch_sample(int d_lo, int d_hi, bool grad, bool fp64, const SampleParams& p, int grid,
                          int threads, cudaStream_t stream) {
    const void* fn = select(d_lo, d_hi, grad, fp64);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {const_cast<SampleParams*>(&p)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, 0, stream);
}

int sample_kernel_regs(int d_lo, int d_hi, bool grad, bool fp64) {
    const void* fn = select(d_lo, d_hi, grad, fp64);
    if (!fn) return -1;
    cudaFuncAttributes attr;
    if (cudaFuncGetAttributes(&attr, fn) != cudaSuccess) return -1;
    return attr.numRegs;
}

cudaError_t sample_occupancy(int d_lo, int d_hi, bool grad, bool fp64, int threads, int* blocks) {
    const void* fn = select(d_lo, d_hi, grad, fp64);
    if (!fn) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, 0);
}

}  // namespace mcd
