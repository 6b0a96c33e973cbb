// Two-cell sweep kernels for storage format f16s (one translation unit per
// format so that the build compiles them in parallel).
#include "sweep2_impl.cuh"

namespace lbm {
template cudaError_t launch_sweep2_st<1>(const SweepArgs &, cudaStream_t);
}
