// Sweep kernels for storage format f64 (one translation unit per format
// so that the build compiles them in parallel).
#include "sweep_impl.cuh"

namespace lbm {
template cudaError_t launch_sweep_st<3>(const SweepArgs &, cudaStream_t);
}
