// Shared-draw kernels of d = 1..10.
#include "shared.cuh"

namespace mcd {

#define MCD_SHARED_CASE(D) \
    case D: *smem = grad ? shared_smem<D, true>() : shared_smem<D, false>(); \
            *dpt = grad ? SharedShape<D, true>::kDpt : SharedShape<D, false>::kDpt; \
            return grad ? shared_fn<D, true>() : shared_fn<D, false>();

const void* shared_kernel_a(int d, bool grad, size_t* smem, int* dpt) {
    switch (d) {
        MCD_SHARED_CASE(1) MCD_SHARED_CASE(2) MCD_SHARED_CASE(3) MCD_SHARED_CASE(4) MCD_SHARED_CASE(5)
        MCD_SHARED_CASE(6) MCD_SHARED_CASE(7) MCD_SHARED_CASE(8) MCD_SHARED_CASE(9) MCD_SHARED_CASE(10)
        default: return nullptr;
    }
}

}  // namespace mcd
