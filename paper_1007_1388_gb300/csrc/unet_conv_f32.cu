// FP32 debug mode of the U-Net's 3x3x3 convolutions: plain CUDA-core kernels
// over FP32 planar activations (the layout of unet_internal.h with float
// elements).  They compute the same contractions as the tensor-core kernels,
// with FP32 operands and FP32 accumulation instead of bf16 operands, so the
// whole network's gradients can be checked against an FP64 implementation to
// about 1e-6 rather than the 1e-2 that bf16 rounding allows.  Not fast: a
// check, not a training path.
#include "unet_internal.h"

namespace lbm {
namespace {

constexpr int CT = 256;

// position offset of tap t (t = 9 (dz+1) + 3 (dy+1) + (dx+1)) in the planar
// layout (rows beyond the walls hold zeros there)
__device__ __forceinline__ long long tap_offset(const Planar &p, int t)
{
    return (long long)(t / 9 - 1) * p.sz + ((t / 3) % 3 - 1) * p.sy + (t % 3 - 1);
}

__device__ __forceinline__ float at(const float *t, const Planar &p, long long q, int c)
{
    return t[((long long)(c >> 3) * p.ptot + q) * 8 + (c & 7)];
}

// one thread per (voxel, output channel)
__global__ void conv3_f32_kernel(ConvF32Args a)
{
    const long long V = a.g.voxels();
    const long long i = (long long)blockIdx.x * CT + threadIdx.x;
    if (i >= V * a.cout) return;
    const long long m = i / a.cout;
    const int co = int(i - m * a.cout);
    const Planar p = planar_of(a.g);
    const long long q = planar_q(a.g, p, m);
    const int cin = a.c0 + a.c1;
    float s = a.bias ? a.bias[co] : 0.f;
    for (int t = 0; t < 27; ++t) {
        const long long o = q + tap_offset(p, t);
        const float *w = a.w + ((long long)co * 27 + t) * cin;
        for (int ci = 0; ci < a.c0; ++ci) s = fmaf(at(a.src0, p, o, ci), w[ci], s);
        for (int ci = 0; ci < a.c1; ++ci) s = fmaf(at(a.src1, p, o, ci), w[a.c0 + ci], s);
    }
    if (a.relu) s = fmaxf(s, 0.f);
    if (!a.out_halo) {
        a.out[i] = s;
        return;
    }
    // planar: the voxel and its periodic copies along x and z
    const long long nx = 1ll << a.g.lx, nz = 1ll << a.g.lz;
    const long long x = m & (nx - 1), z = (m >> (a.g.lx + a.g.ly)) & (nz - 1);
    const long long dx = x == 0 ? nx : (x == nx - 1 ? -nx : 0);
    const long long dz = z == 0 ? nz * p.sz : (z == nz - 1 ? -nz * p.sz : 0);
    float *o = a.out + ((long long)(co >> 3) * p.ptot + q) * 8 + (co & 7);
    o[0] = s;
    if (dx) o[dx * 8] = s;
    if (dz) o[dz * 8] = s;
    if (dx && dz) o[(dx + dz) * 8] = s;
}

// one block per (co, t, group of 8 input channels): every thread sums over a
// strided set of voxels, then the block adds the threads' sums in a fixed
// tree order (deterministic)
__global__ void wgrad_f32_kernel(WgradF32Args a)
{
    __shared__ float sh[CT][9];
    const int cin = a.c0 + a.c1, groups = cin / 8;
    const int gi = blockIdx.x % groups, t = (blockIdx.x / groups) % 27, co = blockIdx.x / (groups * 27);
    const int ci0 = gi * 8;
    const float *src = ci0 < a.c0 ? a.src0 : a.src1;
    const int cs = ci0 < a.c0 ? ci0 : ci0 - a.c0;
    const long long V = a.g.voxels();
    const Planar p = planar_of(a.g);
    const long long off = tap_offset(p, t);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long m = threadIdx.x; m < V; m += CT) {
        const long long q = planar_q(a.g, p, m);
        const float d = at(a.dy, p, q, co);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = fmaf(d, at(src, p, q + off, cs + k), acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int w = CT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < 8; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + w][k];
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) a.dw[((long long)co * 27 + t) * cin + ci0 + threadIdx.x] = sh[0][threadIdx.x];
}

}  // namespace

cudaError_t launch_conv3_f32(const ConvF32Args &a, cudaStream_t s)
{
    if ((a.c0 | a.c1) & 7 || a.c0 < 8 || a.cout < 1) return cudaErrorInvalidValue;
    const long long n = a.g.voxels() * a.cout;
    conv3_f32_kernel<<<unsigned((n + CT - 1) / CT), CT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wgrad_f32(const WgradF32Args &a, cudaStream_t s)
{
    if ((a.c0 | a.c1) & 7 || a.c0 < 8 || a.cout < 1) return cudaErrorInvalidValue;
    const int blocks = a.cout * 27 * ((a.c0 + a.c1) / 8);
    wgrad_f32_kernel<<<blocks, CT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbm
