// Selection and launch of the sampling kernels.
#include "mcd_internal.cuh"

namespace mcd {

const void* sample_kernel_f32_a(int d, bool grad);
const void* sample_kernel_f32_b(int d, bool grad);
const void* sample_kernel_f64_a(int d, bool grad);
const void* sample_kernel_f64_b(int d, bool grad);
const void* sample_kernel_mixed(bool grad);
const void* shared_kernel_a(int d, bool grad, size_t* smem, int* dpt);
const void* shared_kernel_b(int d, bool grad, size_t* smem, int* dpt);

namespace {

const void* select(int d_lo, int d_hi, bool grad, bool fp64) {
    if (d_lo < 1 || d_hi > kMaxD || d_lo > d_hi) return nullptr;
    if (d_lo != d_hi) return (fp64 || d_lo != 1 || d_hi != kMixedMaxD) ? nullptr : sample_kernel_mixed(grad);
    if (fp64) return d_lo <= 10 ? sample_kernel_f64_a(d_lo, grad) : sample_kernel_f64_b(d_lo, grad);
    return d_lo <= 10 ? sample_kernel_f32_a(d_lo, grad) : sample_kernel_f32_b(d_lo, grad);
}

const void* select_shared(int d, bool grad, size_t* smem, int* dpt) {
    *smem = 0;
    *dpt = 0;
    if (d < 1 || d > kMaxD) return nullptr;
    return d <= 10 ? shared_kernel_a(d, grad, smem, dpt) : shared_kernel_b(d, grad, smem, dpt);
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

// The dynamic shared memory of the shared-draw kernels (up to 96 KB) is above
// the default 48 KB limit; the attribute is set before every occupancy query
// and launch (it is per function and cheap).
cudaError_t shared_occupancy(int d, bool grad, int* blocks) {
    size_t smem;
    int dpt;
    const void* fn = select_shared(d, grad, &smem, &dpt);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, kSharedThreads, smem);
}

cudaError_t launch_shared(int d, bool grad, const SampleParams& p, const SharedTile* tiles, const uint32_t* list,
                          int grid, cudaStream_t stream) {
    size_t smem;
    int dpt;
    const void* fn = select_shared(d, grad, &smem, &dpt);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<SampleParams*>(&p), const_cast<SharedTile**>(&tiles), const_cast<uint32_t**>(&list)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kSharedThreads), args, smem, stream);
}

int shared_designs_per_thread(int d, bool grad) {
    size_t smem;
    int dpt;
    return select_shared(d, grad, &smem, &dpt) ? dpt : 0;
}

int shared_batch_draws(int d) {
    const int g = (d % 4 == 0) ? 1 : ((d % 2 == 0) ? 2 : 4);
    return kSharedThreads * g;
}

}  // namespace mcd
