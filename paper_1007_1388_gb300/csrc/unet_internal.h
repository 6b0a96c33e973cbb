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

// Planar halo layout (the network's activations): a tensor of C channels (C a
// multiple of 8) over grid g is stored as [C / 8][ptot][8], eight channels of
// one padded voxel (16 bytes in bf16) per position.  Padded voxel (b, z', y',
// x'), with z' in [0, nz + 2), y' in [0, ny + 2), x' in [0, nx + 2), is at
//   q = guard + ((b (nz + 2) + z') (ny + 2) + y') (nx + 2) + x'
// and voxel (b, z, y, x) at padded (b, z + 1, y + 1, x + 1).  Columns x' = 0
// and nx + 1 and planes z' = 0 and nz + 1 hold the periodic copies; rows y' =
// 0 and ny + 1 (beyond the walls) and the guards hold zeros.  Every run of
// positions of one 8-channel group is contiguous, so a tap of a convolution is
// a fixed offset dz sz + dy sy + dx, and operand tiles are single bulk copies.
struct Planar {
    long long sy, sz, pg, guard, ptot;  // row, plane and grid strides; guard; positions per group
};
__host__ __device__ inline Planar planar_of(const VGrid &g)
{
    Planar p;
    p.sy = (1ll << g.lx) + 2;
    p.sz = ((1ll << g.ly) + 2) * p.sy;
    p.pg = ((1ll << g.lz) + 2) * p.sz;
    p.guard = 1024 + p.sz + p.sy;  // covers a tile's or a run's overhang plus one plane, one row and one voxel
    p.ptot = 2 * p.guard + g.nb * p.pg;
    return p;
}
__host__ __device__ inline long long planar_q(const VGrid &g, const Planar &p, long long m)
{
    const long long nx = 1ll << g.lx, ny = 1ll << g.ly, nz = 1ll << g.lz;
    const long long x = m & (nx - 1), y = (m >> g.lx) & (ny - 1), z = (m >> (g.lx + g.ly)) & (nz - 1);
    const long long b = m >> (g.lx + g.ly + g.lz);
    return p.guard + b * p.pg + (z + 1) * p.sz + (y + 1) * p.sy + x + 1;
}
__host__ __device__ inline long long planar_elems(const VGrid &g, int C) { return (long long)C * planar_of(g).ptot; }

// Bulk-copy tensor-core convolution over planar tensors.  A work item is
// `tiles` x 128 consecutive positions of one grid's interior planes (columns
// and rows of the halo included and discarded); per 16 input channels it
// copies, for dz = -1, 0, 1, the contiguous run of positions its taps reach
// (one bulk copy per 8-channel group), and every tap's A operand is that slab
// at offset (dy + 1) sy + dx + 1.  Persistent CTAs, one per SM.  w: packed bf16 weights [cin / 16][9][2][3][cout][8]
// (element (k, p, h, d, co, e) = W[co][3 p + d][16 k + 8 h + e]).  out: bf16
// planar (periodic copies written too) or fp32 [M][cout].
struct ConvBulkArgs {
    const bf16 *src0, *src1, *w;
    const float *bias;
    void *out;
    int c0, c1, cout, out_f32, relu, tiles;
    VGrid g;
    int *err;
};

// Bulk-copy weight gradient over planar tensors: rows (t, ci) x cout per CTA
// tile of 128 rows; K = every position of the grids (halo and all), in runs
// of `run` (wgrad_bulk_run), split into `nsplit` ranges of pps positions (a
// multiple of run)
// whose partial sums [nsplit][rows_pad][cout] are then added in a fixed
// order.  dyz: the output gradient with zeros at every position that is not
// an interior voxel (no periodic copies), so halo positions add nothing.
struct WgradBulkArgs {
    const bf16 *src0, *src1, *dyz;
    float *partial;
    int c0, c1, cout, rows_pad, pps, run, stages;
    VGrid g;
    int *err;
};
int wgrad_bulk_splits(const VGrid &g, int pps);
void wgrad_bulk_config(int cout, int *run, int *stages);
int wgrad_bulk_pps(const VGrid &g, int row_tiles, int run);
int conv3_bulk_stages(const VGrid &g, int cin, int cout, int tiles);

cudaError_t launch_conv3_bulk(const ConvBulkArgs &a, cudaStream_t s);
cudaError_t launch_wgrad_bulk(const WgradBulkArgs &a, int nsplit, float *dw, cudaStream_t s);
size_t conv3_bulk_smem(const VGrid &g, int cin, int cout, int tiles);

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

// FP32 debug mode: the same convolution on FP32 planar sources with FP32
// weights [cout][27][c0 + c1] on the CUDA cores; out is FP32 planar
// (out_halo = 1, periodic copies written too) or [M][cout].
struct ConvF32Args {
    const float *src0, *src1, *w, *bias;
    float *out;
    int c0, c1, cout, out_halo, relu;
    VGrid g;
};

// FP32 weight gradient dw[co][t][ci] (ci over c0 + c1) from FP32 planar
// sources and dy (planar, cout channels), written (not accumulated).
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
