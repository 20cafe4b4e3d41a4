// FP64 sampling kernels (normals, transform and sums in FP64), dimensions 1,2,3,4,5,6,7,8,9,10.
#include "sample.cuh"

namespace mcd {

const void* sample_kernel_f64_a(int d, bool grad) {
    switch (d) {
        case 1: return grad ? reinterpret_cast<const void*>(&sample_kernel<1, 1, true, double>) : reinterpret_cast<const void*>(&sample_kernel<1, 1, false, double>);
        case 2: return grad ? reinterpret_cast<const void*>(&sample_kernel<2, 2, true, double>) : reinterpret_cast<const void*>(&sample_kernel<2, 2, false, double>);
        case 3: return grad ? reinterpret_cast<const void*>(&sample_kernel<3, 3, true, double>) : reinterpret_cast<const void*>(&sample_kernel<3, 3, false, double>);
        case 4: return grad ? reinterpret_cast<const void*>(&sample_kernel<4, 4, true, double>) : reinterpret_cast<const void*>(&sample_kernel<4, 4, false, double>);
        case 5: return grad ? reinterpret_cast<const void*>(&sample_kernel<5, 5, true, double>) : reinterpret_cast<const void*>(&sample_kernel<5, 5, false, double>);
        case 6: return grad ? reinterpret_cast<const void*>(&sample_kernel<6, 6, true, double>) : reinterpret_cast<const void*>(&sample_kernel<6, 6, false, double>);
        case 7: return grad ? reinterpret_cast<const void*>(&sample_kernel<7, 7, true, double>) : reinterpret_cast<const void*>(&sample_kernel<7, 7, false, double>);
        case 8: return grad ? reinterpret_cast<const void*>(&sample_kernel<8, 8, true, double>) : reinterpret_cast<const void*>(&sample_kernel<8, 8, false, double>);
        case 9: return grad ? reinterpret_cast<const void*>(&sample_kernel<9, 9, true, double>) : reinterpret_cast<const void*>(&sample_kernel<9, 9, false, double>);
        case 10: return grad ? reinterpret_cast<const void*>(&sample_kernel<10, 10, true, double>) : reinterpret_cast<const void*>(&sample_kernel<10, 10, false, double>);
        default: return nullptr;
    }
}

}  // namespace mcd
