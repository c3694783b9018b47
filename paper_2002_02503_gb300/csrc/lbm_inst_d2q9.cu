// Kernel instantiations for the D2Q9 lattice (truncation orders 2,3).
#include "lbm_kernels.cuh"

namespace lbm {

const KernelSet *kernels_d2q9(int K, lbm_storage st) {
    switch (K) {
    case 2: return kernel_set_for_storage<D2Q9, 2>(st);
    case 3: return kernel_set_for_storage<D2Q9, 3>(st);
    }
    return nullptr;
}

}  // namespace lbm
