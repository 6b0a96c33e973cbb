// Sweep kernels for storage format f16s (one translation unit per format
// so that the build compiles them in parallel).
#include "sweep_impl.cuh"

namespace lbm {
template cudaError_t launch_sweep_st<1>(const SweepArgs &, cudaStream_t);
}
