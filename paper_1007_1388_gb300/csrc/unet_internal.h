// Internal types of the learned warm start's 3-D U-Net kernels.  Nothing here
// is part of the C ABI (include/unet.h).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lbm {

using bf16 = __nv_bfloat16;

// Grid of a batch of channels-last tensors: nb grids of nz x ny x nx voxels,
// each side a power of two (log2 given), voxel m = ((b nz + z) ny + y) nx + x.
struct VGrid {
    int nb, lz, ly, lx;
    __host__ __device__ long long voxels() const { return (long long)nb << (lz + ly + lx); }
};

// 3x3x3 convolution as an implicit GEMM on the tensor cores:
//   out[m, co] = act(bias[co] + sum_t sum_ci in[m + off_t, ci] w[co, t, ci])
// in = [src0, src1] concatenated along channels; src0 may be stored at half
// resolution (up0 = 1: nearest-neighbour upsampling on the fly).  Periodic
// along x and z, zero padding along y.  Channels multiples of 16 (c1 may be
// 0); cout a multiple of 16, at most 128.
struct ConvArgs {
    const bf16 *src0;
    const bf16 *src1;
    const bf16 *w;      // [cout][27][c0 + c1]
    const float *bias;  // [cout] or null
    void *out;          // [M][cout], bf16 or fp32
    int c0, c1, up0, cout;
    int out_f32, relu;
    VGrid g;            // output grid (src1 and non-upsampled src0 share it)
    int *err;           // set to 1 when a bounded wait gives up
};

// Weight gradient of the same convolution:
//   dw[co, t, ci] = sum_m dy[m, co] in[m + off_t, ci]
// rows (t, ci) x cout per CTA tile of 128 rows, reduced over voxel splits of
// vps voxels into partial[split][rows_pad][cout], then summed in a fixed order.
struct WgradArgs {
    const bf16 *src0;
    const bf16 *src1;
    const bf16 *dy;     // [M][cout]
    float *partial;     // [nsplit][rows_pad][cout]
    int c0, c1, up0, cout;
    int rows_pad;       // 27 (c0 + c1) rounded up to 128
    int vps;            // voxels per split, a multiple of 64
    VGrid g;
    int *err;
};

cudaError_t launch_conv3(const ConvArgs &a, cudaStream_t s);
cudaError_t launch_wgrad(const WgradArgs &a, int nsplit, float *dw, cudaStream_t s);
int wgrad_splits(const VGrid &g, int vps);
size_t conv3_smem(int cin, int cout);

}  // namespace lbm
