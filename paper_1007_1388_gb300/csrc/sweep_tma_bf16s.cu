// TMA-staged sweep kernels for storage format bf16s (one translation unit
// per format so that the build compiles them in parallel).
#include "sweep_tma.cuh"

namespace lbm {
template cudaError_t launch_sweep_tma_st<2>(const TmaSweepArgs &, const TmaMaps &, int, cudaStream_t,
                                             int *);
}
