// FP64 sampling kernels (normals, transform and sums in FP64), dimensions 11,12,13,14,15,16,17,18,19,20.
#include "sample.cuh"

namespace mcd {

const void* sample_kernel_f64_b(int d, bool grad) {
    switch (d) {
        case 11: return grad ? reinterpret_cast<const void*>(&sample_kernel<11, 11, true, double>) : reinterpret_cast<const void*>(&sample_kernel<11, 11, false, double>);
        case 12: return grad ? reinterpret_cast<const void*>(&sample_kernel<12, 12, true, double>) : reinterpret_cast<const void*>(&sample_kernel<12, 12, false, double>);
        case 13: return grad ? reinterpret_cast<const void*>(&sample_kernel<13, 13, true, double>) : reinterpret_cast<const void*>(&sample_kernel<13, 13, false, double>);
        case 14: return grad ? reinterpret_cast<const void*>(&sample_kernel<14, 14, true, double>) : reinterpret_cast<const void*>(&sample_kernel<14, 14, false, double>);
        case 15: return grad ? reinterpret_cast<const void*>(&sample_kernel<15, 15, true, double>) : reinterpret_cast<const void*>(&sample_kernel<15, 15, false, double>);
        case 16: return grad ? reinterpret_cast<const void*>(&sample_kernel<16, 16, true, double>) : reinterpret_cast<const void*>(&sample_kernel<16, 16, false, double>);
        case 17: return grad ? reinterpret_cast<const void*>(&sample_kernel<17, 17, true, double>) : reinterpret_cast<const void*>(&sample_kernel<17, 17, false, double>);
        case 18: return grad ? reinterpret_cast<const void*>(&sample_kernel<18, 18, true, double>) : reinterpret_cast<const void*>(&sample_kernel<18, 18, false, double>);
        case 19: return grad ? reinterpret_cast<const void*>(&sample_kernel<19, 19, true, double>) : reinterpret_cast<const void*>(&sample_kernel<19, 19, false, double>);
        case 20: return grad ? reinterpret_cast<const void*>(&sample_kernel<20, 20, true, double>) : reinterpret_cast<const void*>(&sample_kernel<20, 20, false, double>);
        default: return nullptr;
    }
}

}  // namespace mcd
