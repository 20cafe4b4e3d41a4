// FP32 sampling kernels, one instantiation per dimension (1,2,3,4,5,6,7,8,9,10).
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

const void* sample_kernel_f32_a(int d, bool grad) {
    switch (d) {
        case 1: return grad ? reinterpret_cast<const void*>(&sample_kernel_3b<1, 1, true, float>) : reinterpret_cast<const void*>(&sample_kernel<1, 1, false, float>);
        case 2: return grad ? reinterpret_cast<const void*>(&sample_kernel<2, 2, true, float>) : reinterpret_cast<const void*>(&sample_kernel<2, 2, false, float>);
        case 3: return grad ? reinterpret_cast<const void*>(&sample_kernel_4b<3, 3, true, float>) : reinterpret_cast<const void*>(&sample_kernel<3, 3, false, float>);
        case 4: return grad ? reinterpret_cast<const void*>(&sample_kernel_3b<4, 4, true, float>) : reinterpret_cast<const void*>(&sample_kernel<4, 4, false, float>);
        case 5: return grad ? reinterpret_cast<const void*>(&sample_kernel<5, 5, true, float>) : reinterpret_cast<const void*>(&sample_kernel<5, 5, false, float>);
        case 6: return grad ? reinterpret_cast<const void*>(&sample_kernel<6, 6, true, float>) : reinterpret_cast<const void*>(&sample_kernel<6, 6, false, float>);
        case 7: return grad ? reinterpret_cast<const void*>(&sample_kernel_2b<7, 7, true, float>) : reinterpret_cast<const void*>(&sample_kernel<7, 7, false, float>);
        case 8: return grad ? reinterpret_cast<const void*>(&sample_kernel_2b<8, 8, true, float>) : reinterpret_cast<const void*>(&sample_kernel<8, 8, false, float>);
        case 9: return grad ? reinterpret_cast<const void*>(&sample_kernel_2b<9, 9, true, float>) : reinterpret_cast<const void*>(&sample_kernel_2b<9, 9, false, float>);
        case 10: return grad ? reinterpret_cast<const void*>(&sample_kernel_2b<10, 10, true, float>) : reinterpret_cast<const void*>(&sample_kernel<10, 10, false, float>);
        default: return nullptr;
    }
}

}  // namespace mcd
