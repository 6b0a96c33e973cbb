// In-place (AA-pattern) sweep kernels for storage format f16s (one
// translation unit per format so that the build compiles them in parallel).
#include "sweep_aa.cuh"

namespace lbm {
template cudaError_t launch_sweep_aa_st<1>(const SweepArgs &, int, cudaStream_t);
}
