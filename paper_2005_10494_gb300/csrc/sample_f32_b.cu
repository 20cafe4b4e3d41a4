// FP32 sampling kernels, one instantiation per dimension (11,12,13,14,15,16,17,18,19,20).
// The two-blocks-per-SM register bound (sample_kernel_2b) is used where it
// measured faster than the unbounded kernel: the adjoint at d = 7..12, 15,
// 17, 19 and the forward pass at d = 9, 13, 15, 17, 19, whose unbounded
// kernels take 160-255 registers (one block per SM); elsewhere the bounded
// kernel spills enough to lose (the adjoint at d = 13, 14, 18, 20: 11-42 %
// slower) or gains nothing (the forward pass at even d).
// The adjoint at d = 1 and 4 runs three blocks per SM (sample_kernel_3b) and
// at d = 3 four (sample_kernel_4b); the 3- and 4-block bounds lost at
// d = 5..8 (11-30 %).
#include "sample.cuh"

namespace mcd {

const void* sample_kernel_f32_b(int d, bool grad) {
    switch (d) {
        case 11: return grad ? reinterpret_cast<const void*>(&sample_kernel_2b<11, 11, true, float>) : reinterpret_cast<const void*>(&sample_kernel<11, 11, false, float>);
        case 12: return grad ? reinterpret_cast<const void*>(&sample_kernel_2b<12, 12, true, float>) : reinterpret_cast<const void*>(&sample_kernel<12, 12, false, float>);
        case 13: return grad ? reinterpret_cast<const void*>(&sample_kernel<13, 13, true, float>) : reinterpret_cast<const void*>(&sample_kernel_2b<13, 13, false, float>);
        case 14: return grad ? reinterpret_cast<const void*>(&sample_kernel<14, 14, true, float>) : reinterpret_cast<const void*>(&sample_kernel<14, 14, false, float>);
        case 15: return grad ? reinterpret_cast<const void*>(&sample_kernel_2b<15, 15, true, float>) : reinterpret_cast<const void*>(&sample_kernel_2b<15, 15, false, float>);
        case 16: return grad ? reinterpret_cast<const void*>(&sample_kernel<16, 16, true, float>) : reinterpret_cast<const void*>(&sample_kernel<16, 16, false, float>);
        case 17: return grad ? reinterpret_cast<const void*>(&sample_kernel_2b<17, 17, true, float>) : reinterpret_cast<const void*>(&sample_kernel_2b<17, 17, false, float>);
        case 18: return grad ? reinterpret_cast<const void*>(&sample_kernel<18, 18, true, float>) : reinterpret_cast<const void*>(&sample_kernel<18, 18, false, float>);
        case 19: return grad ? reinterpret_cast<const void*>(&sample_kernel_2b<19, 19, true, float>) : reinterpret_cast<const void*>(&sample_kernel_2b<19, 19, false, float>);
        case 20: return grad ? reinterpret_cast<const void*>(&sample_kernel<20, 20, true, float>) : reinterpret_cast<const void*>(&sample_kernel<20, 20, false, float>);
        default: return nullptr;
    }
}

}  // namespace mcd
