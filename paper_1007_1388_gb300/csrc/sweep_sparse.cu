// Sweep kernels over the fluid-cell list, every storage format (one
// translation unit: four small kernel families).
#include "lbm_internal.h"
#include "sweep_sparse.cuh"

namespace lbm {

cudaError_t launch_sweep_sparse(const SweepArgs &a, cudaStream_t s)
{
    switch (a.storage) {
    case 0: return launch_sweep_sparse_st<0>(a, s);
    case 1: return launch_sweep_sparse_st<1>(a, s);
    case 2: return launch_sweep_sparse_st<2>(a, s);
    case 3: return launch_sweep_sparse_st<3>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
