// FP32 sampling kernels for batches whose designs have different dimensions
// up to kMixedMaxD: one persistent launch switches per tile on d.
#include "sample.cuh"

namespace mcd {

const void* sample_kernel_mixed(bool grad) {
    return grad ? reinterpret_cast<const void*>(&sample_kernel_2b<1, kMixedMaxD, true, float>)
                : reinterpret_cast<const void*>(&sample_kernel_3b<1, kMixedMaxD, false, float>);
}

}  // namespace mcd
