// Kernel instantiations for the D3Q39 lattice, truncation order 5 (one unit per order so
// the orders compile in parallel).
#include "lbm_kernels.cuh"

namespace lbm {

const KernelSet *kernels_d3q39_k5(lbm_storage st) { return kernel_set_for_storage<D3Q39, 5>(st); }

}  // namespace lbm
