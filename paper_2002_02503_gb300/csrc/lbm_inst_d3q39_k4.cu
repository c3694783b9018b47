// Kernel instantiations for the D3Q39 lattice, truncation order 4 (one unit per order so
// the orders compile in parallel).
#include "lbm_kernels.cuh"

namespace lbm {

const KernelSet *kernels_d3q39_k4(lbm_storage st) { return kernel_set_for_storage<D3Q39, 4>(st); }

}  // namespace lbm
