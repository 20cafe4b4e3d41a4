// Shared-draw kernels of d = 11..20.
#include "shared.cuh"

namespace mcd {

#define MCD_SHARED_CASE(D) \
    case D: *smem = grad ? shared_smem<D, true>() : shared_smem<D, false>(); \
            *dpt = grad ? SharedShape<D, true>::kDpt : SharedShape<D, false>::kDpt; \
            return grad ? shared_fn<D, true>() : shared_fn<D, false>();

const void* shared_kernel_b(int d, bool grad, size_t* smem, int* dpt) {
    switch (d) {
        MCD_SHARED_CASE(11) MCD_SHARED_CASE(12) MCD_SHARED_CASE(13) MCD_SHARED_CASE(14) MCD_SHARED_CASE(15)
        MCD_SHARED_CASE(16) MCD_SHARED_CASE(17) MCD_SHARED_CASE(18) MCD_SHARED_CASE(19) MCD_SHARED_CASE(20)
        default: return nullptr;
    }
}

}  // namespace mcd
