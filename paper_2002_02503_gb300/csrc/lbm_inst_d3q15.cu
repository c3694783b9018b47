// Kernel instantiations for the D3Q15 lattice (truncation orders 2,3).
#include "lbm_kernels.cuh"

namespace lbm {

const KernelSet *kernels_d3q15(int K, lbm_storage st) {
    switch (K) {
    case 2: return kernel_set_for_storage<D3Q15, 2>(st);
    case 3: return kernel_set_for_storage<D3Q15, 3>(st);
    }
    return nullptr;
}

}  // namespace lbm
