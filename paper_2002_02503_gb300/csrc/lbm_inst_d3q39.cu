// Kernel instantiations for the D3Q39 lattice (truncation orders 2,3,4,5).
#include "lbm_kernels.cuh"

namespace lbm {

const KernelSet *kernels_d3q39(int K, lbm_storage st) {
    switch (K) {
    case 2: return kernel_set_for_storage<D3Q39, 2>(st);
    case 3: return kernel_set_for_storage<D3Q39, 3>(st);
    case 4: return kernel_set_for_storage<D3Q39, 4>(st);
    case 5: return kernel_set_for_storage<D3Q39, 5>(st);
    }
    return nullptr;
}

}  // namespace lbm
