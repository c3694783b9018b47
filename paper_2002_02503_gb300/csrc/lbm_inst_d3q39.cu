// Kernel dispatch for the D3Q39 lattice (truncation orders 2..5, instantiated in
// lbm_inst_d3q39_k<K>.cu).
#include "lbm_internal.h"

namespace lbm {

const KernelSet *kernels_d3q39_k2(lbm_storage st);
const KernelSet *kernels_d3q39_k3(lbm_storage st);
const KernelSet *kernels_d3q39_k4(lbm_storage st);
const KernelSet *kernels_d3q39_k5(lbm_storage st);

const KernelSet *kernels_d3q39(int K, lbm_storage st) {
    switch (K) {
    case 2: return kernels_d3q39_k2(st);
    case 3: return kernels_d3q39_k3(st);
    case 4: return kernels_d3q39_k4(st);
    case 5: return kernels_d3q39_k5(st);
    }
    return nullptr;
}

}  // namespace lbm
