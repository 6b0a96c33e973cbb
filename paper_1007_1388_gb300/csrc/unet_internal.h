// Internal types of the learned warm start's 3-D U-Net kernels.  Nothing here
// is part of the C ABI (include/unet.h).
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap
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

// Halo layout of the TMA-fed kernels: a bf16 tensor of nb grids with C
// channels stored as [nb][nz + 2][ny][nx + 2][C]; padded column 0 repeats
// x = nx - 1, column nx + 1 repeats x = 0, padded plane 0 repeats z = nz - 1
// and plane nz + 1 repeats z = 0 (the periodic neighbours), so that every
// tap's operand tile is one tensor-map box (rows beyond the y walls come back
// zero-filled).  Voxel (b, z, y, x) lives at padded (b, z + 1, y, x + 1).
__host__ __device__ inline long long halo_index(const VGrid &g, long long m)
{
    const long long nx = 1ll << g.lx, ny = 1ll << g.ly, nz = 1ll << g.lz;
    const long long x = m & (nx - 1), y = (m >> g.lx) & (ny - 1), z = (m >> (g.lx + g.ly)) & (nz - 1);
    const long long b = m >> (g.lx + g.ly + g.lz);
    return ((b * (nz + 2) + z + 1) * ny + y) * (nx + 2) + x + 1;
}
__host__ __device__ inline long long halo_elems(const VGrid &g, int C)
{
    return (long long)g.nb * ((1ll << g.lz) + 2) * (1ll << g.ly) * ((1ll << g.lx) + 2) * C;
}

// A box of `count` consecutive voxels (a power of two dividing the grid's
// total) in whole rows, planes and grids: extents {bx, by, bz, bb}.
struct VBox {
    int bx, by, bz, bb;
};
__host__ __device__ inline VBox vbox(const VGrid &g, int count)
{
    VBox v{1, 1, 1, 1};
    const int nx = 1 << g.lx, ny = 1 << g.ly, nz = 1 << g.lz;
    if (count <= nx) {
        v.bx = count;
    } else if (count <= nx * ny) {
        v.bx = nx;
        v.by = count / nx;
    } else if (count <= nx * ny * nz) {
        v.bx = nx;
        v.by = ny;
        v.bz = count / (nx * ny);
    } else {
        v.bx = nx;
        v.by = ny;
        v.bz = nz;
        v.bb = count / (nx * ny * nz);
    }
    return v;
}

// TMA-fed convolution over halo-layout tensors (same result as conv3, bitwise:
// the same operands and MMA sequence).  Maps: a0 / a1 over the sources with the
// box {16 channels} x vbox(g, 128); w over the weights [cout][27][cin] with box
// {16, 1, cout}; both with 32-byte swizzle (32-byte rows, whole L2 sectors).  out: bf16 in the halo layout (periodic copies written
// too), or fp32 [M][cout] without halo.  No upsampled source.
struct ConvTmaArgs {
    CUtensorMap a0, a1, w;
    const float *bias;
    void *out;
    int c0, c1, cout;
    int out_f32, relu;
    VGrid g;
    int *err;
};

// TMA-fed weight gradient over halo-layout tensors (same result as the
// cp.async version).  Maps a0 / a1 / dy with the box {16 channels} x
// vbox(g, 64), 32-byte swizzle: 64 voxels per stage.
struct WgradTmaArgs {
    CUtensorMap a0, a1, dy;
    float *partial;
    int c0, c1, cout;
    int rows_pad, vps;
    VGrid g;
    int *err;
};

// FP32 debug mode: the same convolution on FP32 halo-layout sources with FP32
// weights [cout][27][c0 + c1] on the CUDA cores; out is FP32 in the halo
// layout (out_halo = 1, periodic copies written too) or [M][cout].
struct ConvF32Args {
    const float *src0, *src1, *w, *bias;
    float *out;
    int c0, c1, cout, out_halo, relu;
    VGrid g;
};

// FP32 weight gradient dw[co][t][ci] (ci over c0 + c1) from FP32 halo-layout
// sources and dy (halo layout, cout channels), written (not accumulated).
struct WgradF32Args {
    const float *src0, *src1, *dy;
    float *dw;
    int c0, c1, cout;
    VGrid g;
};

cudaError_t launch_conv3_f32(const ConvF32Args &a, cudaStream_t s);
cudaError_t launch_wgrad_f32(const WgradF32Args &a, cudaStream_t s);

// Tensor maps (false when the driver's encoder is unavailable or rejects the map)
// chans = channels per box row: 16 (32-byte rows, 32B swizzle; the TMA
// kernels' operand tiles) or 8 (16-byte rows, no swizzle)
bool make_halo_map(CUtensorMap *m, const void *base, int C, const VGrid &g, const VBox &box, int chans);
bool make_weight_map(CUtensorMap *m, const void *w, int cin, int cout);

cudaError_t launch_conv3(const ConvArgs &a, cudaStream_t s);
cudaError_t launch_conv3_tma(const ConvTmaArgs &a, cudaStream_t s);
cudaError_t launch_wgrad_tma(const WgradTmaArgs &a, int nsplit, float *dw, cudaStream_t s);
cudaError_t launch_wgrad(const WgradArgs &a, int nsplit, float *dw, cudaStream_t s);
int wgrad_splits(const VGrid &g, int vps);
size_t conv3_smem(int cin, int cout);

}  // namespace lbm
