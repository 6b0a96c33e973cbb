// The learned warm start's U-Net: element-wise kernels, the forward /
// backward orchestration and the C ABI of include/unet.h.  The 3x3x3
// convolutions (the contractions) run on the tensor cores (unet_conv.cu);
// pooling, upsampling adjoints, ReLU masks, bias sums, the 1x1x1 head, the
// loss and Adam are the element-wise kernels below.  Activations are bf16
// channels-last; gradients of activations FP32 until they feed a
// convolution, where they are rounded to bf16.  In the FP32 debug mode
// (UNET_F32) activations and weight copies are FP32 and the convolutions run
// on the CUDA cores (unet_conv_f32.cu); everything else is the same code.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "unet.h"
#include "unet_internal.h"

namespace lbm {
namespace {

constexpr int EW = 256;

__host__ __device__ inline int ilog2(long long v)
{
    int l = 0;
    while ((1ll << l) < v) ++l;
    return l;
}

// Position offsets of the periodic copies of voxel m in the planar layout:
// along x (dx) and along z (dz); 0 where there is none.
__device__ __forceinline__ void halo_copies(const VGrid &g, const Planar &p, long long m, long long &dx, long long &dz)
{
    const long long nx = 1ll << g.lx, nz = 1ll << g.lz;
    const long long x = m & (nx - 1), z = (m >> (g.lx + g.ly)) & (nz - 1);
    dx = x == 0 ? nx : (x == nx - 1 ? -nx : 0);
    dz = z == 0 ? nz * p.sz : (z == nz - 1 ? -nz * p.sz : 0);
}

// first element of channels c0 .. c0 + 7 at position q of a planar tensor
template <typename A>
__device__ __forceinline__ A *planar_at(A *t, const Planar &p, long long q, int c0)
{
    return t + ((long long)(c0 >> 3) * p.ptot + q) * 8;
}

// Eight channels of an activation: bf16 (the tensor-core path; one 16-byte
// word) or float (the FP32 debug mode; two).  Values pass through float, so
// the bf16 results are those of plain bf16 rounding.
template <typename A> struct Act8;
template <> struct Act8<bf16> {
    uint4 r;
    __device__ __forceinline__ void load(const bf16 *p) { r = *reinterpret_cast<const uint4 *>(p); }
    __device__ __forceinline__ void store(bf16 *p) const { *reinterpret_cast<uint4 *>(p) = r; }
    __device__ __forceinline__ void get(float *v) const
    {
        const bf16 *h = reinterpret_cast<const bf16 *>(&r);
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __bfloat162float(h[k]);
    }
    __device__ __forceinline__ void set(const float *v)
    {
        bf16 *h = reinterpret_cast<bf16 *>(&r);
#pragma unroll
        for (int k = 0; k < 8; ++k) h[k] = __float2bfloat16(v[k]);
    }
};
template <> struct Act8<float> {
    float4 a, b;
    __device__ __forceinline__ void load(const float *p)
    {
        a = reinterpret_cast<const float4 *>(p)[0];
        b = reinterpret_cast<const float4 *>(p)[1];
    }
    __device__ __forceinline__ void store(float *p) const
    {
        reinterpret_cast<float4 *>(p)[0] = a;
        reinterpret_cast<float4 *>(p)[1] = b;
    }
    __device__ __forceinline__ void get(float *v) const
    {
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    }
    __device__ __forceinline__ void set(const float *v)
    {
        a = make_float4(v[0], v[1], v[2], v[3]);
        b = make_float4(v[4], v[5], v[6], v[7]);
    }
};

// Stores channels c0 .. c0 + 7 of voxel m of a planar tensor, and the
// voxel's periodic copies.
template <typename A>
__device__ __forceinline__ void planar_store(A *t, const VGrid &g, long long m, int c0, const Act8<A> &v)
{
    const Planar p = planar_of(g);
    long long dx, dz;
    halo_copies(g, p, m, dx, dz);
    A *at = planar_at(t, p, planar_q(g, p, m), c0);
    v.store(at);
    if (dx) v.store(at + dx * 8);
    if (dz) v.store(at + dz * 8);
    if (dx && dz) v.store(at + (dx + dz) * 8);
}

// x[m] = {solid, force of the sample, 0, ..., 0} (16 channels, planar)
template <typename A>
__global__ void make_input_kernel(const uint8_t *__restrict__ solid, const float *__restrict__ force,
                                  A *__restrict__ x, VGrid g)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.voxels()) return;
    float v[8] = {solid[i] ? 1.f : 0.f, force[i >> (g.lx + g.ly + g.lz)], 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    Act8<A> a;
    a.set(v);
    planar_store(x, g, i, 0, a);
    v[0] = v[1] = 0.f;
    a.set(v);
    planar_store(x, g, i, 8, a);
}

// Coordinates of voxel m in grid g, and the index of voxel (b, z, y, x).
__device__ __forceinline__ void coords(long long m, const VGrid &g, int &b, int &z, int &y, int &x)
{
    x = int(m & ((1ll << g.lx) - 1));
    y = int((m >> g.lx) & ((1ll << g.ly) - 1));
    z = int((m >> (g.lx + g.ly)) & ((1ll << g.lz) - 1));
    b = int(m >> (g.lx + g.ly + g.lz));
}
__device__ __forceinline__ long long vidx(const VGrid &g, int b, int z, int y, int x)
{
    return ((((long long)b << g.lz) + z) << (g.ly + g.lx)) + ((long long)y << g.lx) + x;
}

// 2x2x2 average: out (grid gh) from in (grid 2 gh), C channels, planar;
// one thread per 8 channels of an output voxel
template <typename A>
__global__ void pool_kernel(const A *__restrict__ in, A *__restrict__ out, VGrid gh, int C)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int C8 = C >> 3;
    if (i >= gh.voxels() * C8) return;
    const long long p = i / C8;
    const int c = int(i - p * C8) * 8;
    int b, z, y, x;
    coords(p, gh, b, z, y, x);
    const VGrid gf{gh.nb, gh.lz + 1, gh.ly + 1, gh.lx + 1};
    const Planar pf = planar_of(gf);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int d = 0; d < 8; ++d) {
        const long long m = vidx(gf, b, 2 * z + (d >> 2), 2 * y + ((d >> 1) & 1), 2 * x + (d & 1));
        Act8<A> a;
        a.load(planar_at(in, pf, planar_q(gf, pf, m), c));
        float h[8];
        a.get(h);
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] += h[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] *= 0.125f;
    Act8<A> o;
    o.set(s);
    planar_store(out, gh, p, c, o);
}

// nearest 2x upsampling: out (grid gf) from in (grid gf / 2), C channels,
// planar; one thread per 8 channels of an output voxel
template <typename A>
__global__ void upsample_kernel(const A *__restrict__ in, A *__restrict__ out, VGrid gf, int C)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int C8 = C >> 3;
    if (i >= gf.voxels() * C8) return;
    const long long m = i / C8;
    const int c = int(i - m * C8) * 8;
    int b, z, y, x;
    coords(m, gf, b, z, y, x);
    const VGrid gh{gf.nb, gf.lz - 1, gf.ly - 1, gf.lx - 1};
    const Planar ph = planar_of(gh);
    Act8<A> v;
    v.load(planar_at(in, ph, planar_q(gh, ph, vidx(gh, b, z >> 1, y >> 1, x >> 1)), c));
    planar_store(out, gf, m, c, v);
}

// dy = g * (y > 0) in the activation type (y, dy: planar with periodic
// copies; dyz: the same values without the copies, zeros elsewhere, for the
// weight gradient; g: [V][C] fp32); per-block channel sums of g * (y > 0) (bias
// gradient).  A thread handles 8 channels of a voxel; blockDim = EW and the
// grid stride are multiples of C / 8, so each thread keeps one channel group.
template <typename A>
__global__ void relu_bwd_kernel(const float *__restrict__ g, const A *__restrict__ y, A *__restrict__ dy,
                                A *__restrict__ dyz, float *__restrict__ part, VGrid grid, int C)
{
    __shared__ float sh[EW][9];
    const int C8 = C >> 3;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const long long n = grid.voxels() * C8;
    const Planar pl = planar_of(grid);
    for (long long i = (long long)blockIdx.x * EW + threadIdx.x; i < n; i += (long long)gridDim.x * EW) {
        const long long m = i / C8;
        const int c = int(i - m * C8) * 8;
        Act8<A> ya;
        ya.load(planar_at(y, pl, planar_q(grid, pl, m), c));
        float yv[8];
        ya.get(yv);
        const float4 g0 = *reinterpret_cast<const float4 *>(g + m * C + c);
        const float4 g1 = *reinterpret_cast<const float4 *>(g + m * C + c + 4);
        const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
        float o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            o[k] = yv[k] > 0.f ? gv[k] : 0.f;
            acc[k] += o[k];
        }
        Act8<A> oa;
        oa.set(o);
        planar_store(dy, grid, m, c, oa);
        oa.store(planar_at(dyz, pl, planar_q(grid, pl, m), c));
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < C) {
        const int grp = threadIdx.x >> 3, k = threadIdx.x & 7;
        float t = 0.f;
        for (int r = grp; r < EW; r += C8) t += sh[r][k];
        part[(long long)blockIdx.x * C + threadIdx.x] = t;
    }
}

// out[c] = sum over rows of part[row][c]: one block per column, a fixed
// tree order (deterministic)
__global__ void reduce_cols_kernel(const float *__restrict__ part, int rows, int C, float *__restrict__ out)
{
    __shared__ float sh[EW];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int r = threadIdx.x; r < rows; r += EW) s += part[(long long)r * C + c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = EW / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0];
}

// adjoint of nearest upsampling of the first c0 channels of a concatenation:
// gu[p][c] = sum over the 8 children v of p of gcat[v][c]  (gu on grid gh)
__global__ void up_bwd_kernel(const float *__restrict__ gcat, int ctot, int c0, float *__restrict__ gu, VGrid gh)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= gh.voxels() * c0) return;
    const long long p = i / c0;
    const int c = int(i - p * c0);
    int b, z, y, x;
    coords(p, gh, b, z, y, x);
    const VGrid gf{gh.nb, gh.lz + 1, gh.ly + 1, gh.lx + 1};
    float s = 0.f;
    for (int d = 0; d < 8; ++d)
        s += gcat[vidx(gf, b, 2 * z + (d >> 2), 2 * y + ((d >> 1) & 1), 2 * x + (d & 1)) * ctot + c];
    gu[i] = s;
}

// ge[v][c] = gcat[v][c0 + c] + gp[parent(v)][c] / 8: the skip connection's
// share of a concatenation gradient plus the adjoint of the 2x2x2 average
__global__ void skip_pool_kernel(const float *__restrict__ gcat, int ctot, int c0, const float *__restrict__ gp,
                                 float *__restrict__ ge, VGrid gf, int C)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= gf.voxels() * C) return;
    const long long v = i / C;
    const int c = int(i - v * C);
    int b, z, y, x;
    coords(v, gf, b, z, y, x);
    const VGrid gh{gf.nb, gf.lz - 1, gf.ly - 1, gf.lx - 1};
    ge[i] = gcat[v * ctot + c0 + c] + 0.125f * gp[vidx(gh, b, z >> 1, y >> 1, x >> 1) * C + c];
}

// 1x1x1 head y = d1 Wh^T + bh (d1 planar); with a target: loss partials, the gradient
// g_d1 = gy Wh (gy = 2 (y - target) / (V 4)), and partials of dWh (4 x 16),
// dbh (4) and the loss: part[block][72] = {dWh[64], dbh[4], sum of squared
// differences, 3 unused}.
constexpr int HEAD_PART = 72;
template <typename A>
__global__ void head_kernel(const A *__restrict__ d1, const float *__restrict__ Wh, const float *__restrict__ bh,
                            const float *__restrict__ target, float *__restrict__ out, float *__restrict__ gd1,
                            float *__restrict__ part, VGrid g)
{
    const long long V = g.voxels();
    __shared__ float sw[64], sb[4];
    __shared__ float red[EW / 32][HEAD_PART];
    if (threadIdx.x < 64) sw[threadIdx.x] = Wh[threadIdx.x];
    if (threadIdx.x < 4) sb[threadIdx.x] = bh[threadIdx.x];
    __syncthreads();
    float acc[HEAD_PART];
#pragma unroll
    for (int k = 0; k < HEAD_PART; ++k) acc[k] = 0.f;
    const float gscale = 2.f / float(V * 4);
    const Planar pl = planar_of(g);
    for (long long m = (long long)blockIdx.x * EW + threadIdx.x; m < V; m += (long long)gridDim.x * EW) {
        const long long q = planar_q(g, pl, m);
        Act8<A> h0, h1;
        h0.load(planar_at(d1, pl, q, 0));
        h1.load(planar_at(d1, pl, q, 8));
        float a[16];
        h0.get(a);
        h1.get(a + 8);
        float y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float s = sb[j];
#pragma unroll
            for (int k = 0; k < 16; ++k) s = fmaf(sw[j * 16 + k], a[k], s);
            y[j] = s;
        }
        if (out)
            reinterpret_cast<float4 *>(out)[m] = make_float4(y[0], y[1], y[2], y[3]);
        if (target) {
            const float4 t4 = reinterpret_cast<const float4 *>(target)[m];
            const float t[4] = {t4.x, t4.y, t4.z, t4.w};
            float gy[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float d = y[j] - t[j];
                acc[68] = fmaf(d, d, acc[68]);
                gy[j] = gscale * d;
                acc[64 + j] += gy[j];
#pragma unroll
                for (int k = 0; k < 16; ++k) acc[j * 16 + k] = fmaf(gy[j], a[k], acc[j * 16 + k]);
            }
            float g[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float s = 0.f;
#pragma unroll
                for (int j = 0; j < 4; ++j) s = fmaf(gy[j], sw[j * 16 + k], s);
                g[k] = s;
            }
            float4 *o = reinterpret_cast<float4 *>(gd1 + m * 16);
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = make_float4(g[4 * k], g[4 * k + 1], g[4 * k + 2], g[4 * k + 3]);
        }
    }
    if (!target || !part) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < HEAD_PART; ++k) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < HEAD_PART) {
        float s = 0.f;
        for (int w = 0; w < EW / 32; ++w) s += red[w][threadIdx.x];
        part[(long long)blockIdx.x * HEAD_PART + threadIdx.x] = s;
    }
}

// bf16 (or, in the FP32 debug mode, FP32) copies of one convolution's FP32
// weight [cout][27][cin]:
// wf [cout][27][cinp] (zero channels beyond cin) and, when wb is given, the
// tap-flipped transpose wb [cin][27][cout], wb[ci][t][co] = W[co][26 - t][ci]
// (the backward-data convolution).
template <typename A>
__global__ void prep_weights_kernel(const float *__restrict__ W, int cout, int cin, int cinp, A *__restrict__ wf,
                                    A *__restrict__ wb)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)cout * 27 * cinp) return;
    const int ci = int(i % cinp);
    const long long r = i / cinp;
    const int t = int(r % 27), co = int(r / 27);
    const float w = ci < cin ? W[((long long)co * 27 + t) * cin + ci] : 0.f;
    wf[i] = A(w);
    if (wb && ci < cin) wb[((long long)ci * 27 + (26 - t)) * cout + co] = A(w);
}

// bf16 weights of one convolution packed for the bulk-copy kernels, stage by
// stage (16 input channels), the three x taps of each (dz, dy) pair side by
// side along the output axis: wf[k][p][h][d][co][e] = W[co][3 p + d][16 k +
// 8 h + e] (0 beyond cin), and, when wb is given, the backward-data
// convolution's (input channels = cout, output channels = cin, taps flipped)
// wb[k][p][h][d][ci][e] = W[16 k + 8 h + e][26 - (3 p + d)][ci].
__global__ void pack_weights_kernel(const float *__restrict__ W, int cout, int cin, int cinp, bf16 *__restrict__ wf,
                                    bf16 *__restrict__ wb)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)cout * 27 * cinp) return;
    {
        // forward: i = ((((k 9 + p) 2 + h) 3 + d) cout + co) 8 + e
        const int e = int(i & 7);
        long long r = i >> 3;
        const int co = int(r % cout);
        r /= cout;
        const int d = int(r % 3);
        r /= 3;
        const int h = int(r & 1);
        r >>= 1;
        const int p = int(r % 9), k = int(r / 9);
        const int ci = 16 * k + 8 * h + e;
        wf[i] = __float2bfloat16(ci < cin ? W[((long long)co * 27 + 3 * p + d) * cin + ci] : 0.f);
    }
    if (wb && i < (long long)cout * 27 * cin) {
        // backward data: output channel ci, input channel 16 k + 8 h + e
        const int e = int(i & 7);
        long long r = i >> 3;
        const int ci = int(r % cin);
        r /= cin;
        const int d = int(r % 3);
        r /= 3;
        const int h = int(r & 1);
        r >>= 1;
        const int p = int(r % 9), k = int(r / 9);
        const int co = 16 * k + 8 * h + e;
        wb[i] = __float2bfloat16(W[((long long)co * 27 + (26 - (3 * p + d))) * cin + ci]);
    }
}

// dw [cout][27][cin] from the padded weight gradient [cout][27][cinp]
__global__ void unpad_grad_kernel(const float *__restrict__ src, int cout, int cin, int cinp, float *__restrict__ dst)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)cout * 27 * cin) return;
    const int ci = int(i % cin);
    const long long r = i / cin;
    dst[i] = src[r * cinp + ci];
}

// target[k][c][0..3] = {(rho - rho0) / (F_k s_rho), u_a / (F_k s_u)} (0 in solid cells)
// from the batch layout rho [nb][V], u [nb][3][V]
__global__ void targets_kernel(const float *__restrict__ rho, const float *__restrict__ u,
                               const uint8_t *__restrict__ solid, const float *__restrict__ force, long long V,
                               long long n, float rho0, float s_rho, float s_u, float *__restrict__ target)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long k = i / V, c = i - k * V;
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!solid[i]) {
        const float f = force[k];
        const float *uk = u + 3 * k * V;
        t = make_float4((rho[i] - rho0) / (f * s_rho), uk[c] / (f * s_u), uk[V + c] / (f * s_u),
                        uk[2 * V + c] / (f * s_u));
    }
    reinterpret_cast<float4 *>(target)[i] = t;
}

// the inverse map: rho = rho0 + F_k s_rho y0, u_a = F_k s_u y_{1+a}; solid cells rho0, 0
__global__ void fields_kernel(const float *__restrict__ pred, const uint8_t *__restrict__ solid,
                              const float *__restrict__ force, long long V, long long n, float rho0, float s_rho,
                              float s_u, float *__restrict__ rho, float *__restrict__ u)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long k = i / V, c = i - k * V;
    const float4 y = reinterpret_cast<const float4 *>(pred)[i];
    const bool fl = !solid[i];
    const float f = force[k];
    rho[i] = fl ? rho0 + f * s_rho * y.x : rho0;
    float *uk = u + 3 * k * V;
    uk[c] = fl ? f * s_u * y.y : 0.f;
    uk[V + c] = fl ? f * s_u * y.z : 0.f;
    uk[2 * V + c] = fl ? f * s_u * y.w : 0.f;
}

// One [1 2 1]/4 pass along axis `ax` (0 = x, 1 = y, 2 = z) of K fields of
// `comps` components on n^3 grids ([K][comps][V], x fastest): periodic along
// x and z, the edge value repeated beyond the y walls; solid cells hold 0 and
// contribute 0.
__global__ void smooth_kernel(const float *__restrict__ in, float *__restrict__ out, const uint8_t *__restrict__ solid,
                              long long n_total, int comps, int ln, int ax)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_total) return;
    const int n = 1 << ln;
    const long long V = 1ll << (3 * ln);
    const long long kc = i >> (3 * ln);        // field index k * comps + component
    const long long c = i & (V - 1);
    const long long k = kc / comps;
    if (solid[k * V + c]) {
        out[i] = 0.f;
        return;
    }
    const int x = int(c & (n - 1)), y = int((c >> ln) & (n - 1)), z = int(c >> (2 * ln));
    int m[2];
    if (ax == 0) {
        m[0] = (x - 1) & (n - 1);
        m[1] = (x + 1) & (n - 1);
    } else if (ax == 1) {
        m[0] = y > 0 ? y - 1 : y;
        m[1] = y < n - 1 ? y + 1 : y;
    } else {
        m[0] = (z - 1) & (n - 1);
        m[1] = (z + 1) & (n - 1);
    }
    const long long base = kc * V;
    auto at = [&](int j) {
        const long long cc = ax == 0 ? ((long long)z << (2 * ln)) + ((long long)y << ln) + j
                           : ax == 1 ? ((long long)z << (2 * ln)) + ((long long)j << ln) + x
                                     : ((long long)j << (2 * ln)) + ((long long)y << ln) + x;
        return in[base + cc];
    };
    out[i] = 0.25f * at(m[0]) + 0.5f * in[i] + 0.25f * at(m[1]);
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// The ten 3x3x3 convolutions in forward order (name, cin, cout).
struct ConvSpec {
    int cin, cout;
};
constexpr int NCONV = 10;
constexpr ConvSpec kConv[NCONV] = {{2, 16},  {16, 16}, {16, 32}, {32, 32}, {32, 64},
                                   {64, 64}, {96, 32}, {32, 32}, {48, 16}, {16, 16}};
enum { W1A, W1B, W2A, W2B, W3A, W3B, W4A, W4B, W5A, W5B };

struct Layout {
    long long w[NCONV], b[NCONV], wh, bh, total;
    Layout()
    {
        long long o = 0;
        for (int k = 0; k < NCONV; ++k) {
            w[k] = o;
            o += 27ll * kConv[k].cin * kConv[k].cout;
            b[k] = o;
            o += kConv[k].cout;
        }
        wh = o;
        o += 64;
        bh = o;
        o += 4;
        total = o;
    }
};
const Layout kLayout;

int cin_padded(int k) { return kConv[k].cin < 16 ? 16 : kConv[k].cin; }

// counter-based normal numbers: SplitMix64 of (seed, index), Box-Muller
uint64_t splitmix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double normal(uint64_t seed, uint64_t i)
{
    const uint64_t a = splitmix(seed * 0x100000001B3ull + 2 * i), b = splitmix(seed * 0x100000001B3ull + 2 * i + 1);
    const double u1 = (double(a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = double(b >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct unet_ctx {
    int n = 0, nb = 0;
    VGrid g1{}, g2{}, g3{};
    long long V1 = 0, V2 = 0, V3 = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *(*alloc)(size_t, void *, void *) = nullptr;
    void (*release)(void *, size_t, void *, void *) = nullptr;
    void *user = nullptr;
    std::vector<std::pair<void *, size_t>> owned;
    float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
    long long step = 0;
    int precision = UNET_BF16;  // element type of weights copies and activations: bf16 or float
    void *wf[NCONV] = {}, *wb[NCONV] = {};
    bool weights_current = false;
    void *x = nullptr, *e1h = nullptr, *e1 = nullptr, *p1 = nullptr, *e2h = nullptr, *e2 = nullptr, *p2 = nullptr,
         *e3h = nullptr, *e3 = nullptr, *d2h = nullptr, *d2 = nullptr, *d1h = nullptr, *d1 = nullptr,
         *up3 = nullptr, *up2 = nullptr;  // activations: planar layout (unet_internal.h)
    void *dy1 = nullptr, *dy2 = nullptr, *dy3 = nullptr;  // masked output gradients of levels 1, 2, 3 (planar)
    void *dyz1 = nullptr, *dyz2 = nullptr, *dyz3 = nullptr;  // the same without periodic copies
    float *gd1 = nullptr, *gcat1 = nullptr, *gd2 = nullptr, *gcat2 = nullptr, *ge3 = nullptr, *gp2 = nullptr,
          *ge2 = nullptr, *gp1 = nullptr, *ge1 = nullptr, *gh = nullptr;
    float *wpart = nullptr, *wtmp = nullptr, *bpart = nullptr, *hpart = nullptr, *dforce = nullptr;
    size_t wpart_bytes = 0;
    int relu_blocks = 0, head_blocks = 0;
    int *derr = nullptr;
    std::string err;
};

namespace {
thread_local std::string g_unet_create_error;

int ufail(unet_ctx *c, int code, const char *fmt, ...)
{
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    if (c)
        c->err = msg;
    else
        g_unet_create_error = msg;
    return code;
}

#define UCK(call, what)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return ufail(c, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

void *ualloc(unet_ctx *c, size_t bytes)
{
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->alloc) {
        p = c->alloc(bytes, (void *)c->stream, c->user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->owned.push_back({p, bytes});
    return p;
}

template <typename P>
int uown(unet_ctx *c, P **out, size_t count)
{
    void *p = ualloc(c, count * sizeof(P));
    if (!p) return ufail(c, LBM_ENOMEM, "device allocation of %zu bytes failed", count * sizeof(P));
    *out = static_cast<P *>(p);
    return LBM_OK;
}

void ufree_all(unet_ctx *c)
{
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &o : c->owned) {
        if (c->release)
            c->release(o.first, o.second, (void *)c->stream, c->user);
        else if (!c->alloc)
            cudaFree(o.first);
    }
    c->owned.clear();
}

unsigned blocks_for(long long n) { return unsigned((n + EW - 1) / EW); }

// 128-position tiles per work item of the bulk convolution: the most whose
// two accumulator buffers (cout columns a tile) fit TMEM with a ring of at
// least two stages; else one buffer
int conv_tiles(const VGrid &g, int cin, int cout)
{
    for (int t = 4; t >= 1; t >>= 1)
        if (2 * t * cout <= 512 && conv3_bulk_stages(g, cin, cout, t) >= 2) return t;
    for (int t = 4; t >= 1; t >>= 1)
        if (t * cout <= 512 && conv3_bulk_stages(g, cin, cout, t) >= 1) return t;
    return 1;
}

// one 3x3x3 convolution on the context stream (planar sources): bulk-copy
// tensor cores for bf16 (w packed per stage), the CUDA-core kernel in the
// FP32 debug mode (w [cout][27][cin])
int conv(unet_ctx *c, const bf16 *s0, int c0, const bf16 *s1, int c1, const void *w, const float *bias, void *out,
         int out_f32, int relu, int cout, VGrid g)
{
    ConvBulkArgs a{};
    a.src0 = s0;
    a.src1 = s1;
    a.w = static_cast<const bf16 *>(w);
    a.bias = bias;
    a.out = out;
    a.c0 = c0;
    a.c1 = c1;
    a.cout = cout;
    a.out_f32 = out_f32;
    a.relu = relu;
    a.tiles = conv_tiles(g, c0 + c1, cout);
    a.g = g;
    a.err = c->derr;
    UCK(launch_conv3_bulk(a, c->stream), "conv3");
    return LBM_OK;
}
int conv(unet_ctx *c, const float *s0, int c0, const float *s1, int c1, const void *w, const float *bias, void *out,
         int out_f32, int relu, int cout, VGrid g)
{
    ConvF32Args a{};
    a.src0 = s0;
    a.src1 = s1;
    a.w = static_cast<const float *>(w);
    a.bias = bias;
    a.out = static_cast<float *>(out);
    a.c0 = c0;
    a.c1 = c1;
    a.cout = cout;
    a.out_halo = !out_f32;  // activations are halo-layout, gradients [M][cout]
    a.relu = relu;
    a.g = g;
    UCK(launch_conv3_f32(a, c->stream), "conv3 (fp32)");
    return LBM_OK;
}

// voxels per split of a weight gradient: about four waves of CTAs on 152 SMs
int wgrad_vps(long long V, int tiles)
{
    long long nsplit = (608 + tiles - 1) / tiles;
    if (nsplit < 1) nsplit = 1;
    long long vps = (V + nsplit - 1) / nsplit;
    vps = (vps + 63) / 64 * 64;
    return int(vps < 64 ? 64 : vps);
}

size_t wgrad_ws_bytes(const VGrid &g, int cin, int cout)
{
    const int rows_pad = (27 * cin + 127) / 128 * 128;
    int run, stages;
    wgrad_bulk_config(cout, &run, &stages);
    const int nsplit = wgrad_bulk_splits(g, wgrad_bulk_pps(g, rows_pad / 128, run));
    return size_t(nsplit) * rows_pad * cout * sizeof(float);
}

int wgrad(unet_ctx *c, const bf16 *s0, int c0, const bf16 *s1, int c1, const bf16 *dyz, int cout, float *dw,
          VGrid g)
{
    WgradBulkArgs a{};
    a.src0 = s0;
    a.src1 = s1;
    a.dyz = dyz;
    a.c0 = c0;
    a.c1 = c1;
    a.cout = cout;
    a.rows_pad = (27 * (c0 + c1) + 127) / 128 * 128;
    wgrad_bulk_config(cout, &a.run, &a.stages);
    a.pps = wgrad_bulk_pps(g, a.rows_pad / 128, a.run);
    a.g = g;
    a.err = c->derr;
    a.partial = c->wpart;
    const int nsplit = wgrad_bulk_splits(g, a.pps);
    if (size_t(nsplit) * a.rows_pad * cout * sizeof(float) > c->wpart_bytes)
        return ufail(c, LBM_EINVAL, "weight-gradient workspace too small");
    UCK(launch_wgrad_bulk(a, nsplit, dw, c->stream), "wgrad");
    return LBM_OK;
}
int wgrad(unet_ctx *c, const float *s0, int c0, const float *s1, int c1, const float *dy, int cout, float *dw,
          VGrid g)
{
    WgradF32Args a{};
    a.src0 = s0;
    a.src1 = s1;
    a.dy = dy;
    a.dw = dw;
    a.c0 = c0;
    a.c1 = c1;
    a.cout = cout;
    a.g = g;
    UCK(launch_wgrad_f32(a, c->stream), "wgrad (fp32)");
    return LBM_OK;
}

// ReLU backward into dy (planar) and the bias gradient of layer k
template <typename A>
int relu_bwd(unet_ctx *c, const float *g, const void *y, void *dy, void *dyz, VGrid grid, int C, int k)
{
    const long long n = grid.voxels() * (C / 8);
    int nblk = int(std::min<long long>(c->relu_blocks, (n + EW - 1) / EW));
    if (nblk < 1) nblk = 1;
    relu_bwd_kernel<A><<<nblk, EW, 0, c->stream>>>(g, static_cast<const A *>(y), static_cast<A *>(dy),
                                                   static_cast<A *>(dyz), c->bpart, grid, C);
    reduce_cols_kernel<<<C, EW, 0, c->stream>>>(c->bpart, nblk, C, c->grads + kLayout.b[k]);
    UCK(cudaGetLastError(), "relu backward");
    return LBM_OK;
}

template <typename A>
int prep_weights(unet_ctx *c)
{
    if (c->weights_current) return LBM_OK;
    for (int k = 0; k < NCONV; ++k) {
        const int cp = cin_padded(k);
        const long long n = 27ll * kConv[k].cout * cp;
        if (std::is_same<A, float>::value)
            prep_weights_kernel<float><<<blocks_for(n), EW, 0, c->stream>>>(
                c->params + kLayout.w[k], kConv[k].cout, kConv[k].cin, cp, static_cast<float *>(c->wf[k]),
                static_cast<float *>(c->wb[k]));
        else
            pack_weights_kernel<<<blocks_for(n), EW, 0, c->stream>>>(c->params + kLayout.w[k], kConv[k].cout,
                                                                     kConv[k].cin, cp, static_cast<bf16 *>(c->wf[k]),
                                                                     static_cast<bf16 *>(c->wb[k]));
    }
    UCK(cudaGetLastError(), "weights");
    c->weights_current = true;
    return LBM_OK;
}

template <typename A>
int forward(unet_ctx *c, const uint8_t *solid, const float *force)
{
    int rc;
    auto T = [](void *p) { return static_cast<A *>(p); };
    UCK(cudaMemcpyAsync(c->dforce, force, sizeof(float) * c->nb, cudaMemcpyHostToDevice, c->stream), "force");
    if ((rc = prep_weights<A>(c))) return rc;
    make_input_kernel<A><<<blocks_for(c->V1), EW, 0, c->stream>>>(solid, c->dforce, T(c->x), c->g1);
    UCK(cudaGetLastError(), "input");
    const float *P = c->params;
    const Layout &L = kLayout;
    if ((rc = conv(c, T(c->x), 16, (const A *)nullptr, 0, c->wf[W1A], P + L.b[W1A], c->e1h, 0, 1, 16, c->g1))) return rc;
    if ((rc = conv(c, T(c->e1h), 16, (const A *)nullptr, 0, c->wf[W1B], P + L.b[W1B], c->e1, 0, 1, 16, c->g1))) return rc;
    pool_kernel<A><<<blocks_for(c->V2 * 2), EW, 0, c->stream>>>(T(c->e1), T(c->p1), c->g2, 16);
    if ((rc = conv(c, T(c->p1), 16, (const A *)nullptr, 0, c->wf[W2A], P + L.b[W2A], c->e2h, 0, 1, 32, c->g2))) return rc;
    if ((rc = conv(c, T(c->e2h), 32, (const A *)nullptr, 0, c->wf[W2B], P + L.b[W2B], c->e2, 0, 1, 32, c->g2))) return rc;
    pool_kernel<A><<<blocks_for(c->V3 * 4), EW, 0, c->stream>>>(T(c->e2), T(c->p2), c->g3, 32);
    if ((rc = conv(c, T(c->p2), 32, (const A *)nullptr, 0, c->wf[W3A], P + L.b[W3A], c->e3h, 0, 1, 64, c->g3))) return rc;
    if ((rc = conv(c, T(c->e3h), 64, (const A *)nullptr, 0, c->wf[W3B], P + L.b[W3B], c->e3, 0, 1, 64, c->g3))) return rc;
    upsample_kernel<A><<<blocks_for(c->V2 * 8), EW, 0, c->stream>>>(T(c->e3), T(c->up3), c->g2, 64);
    if ((rc = conv(c, T(c->up3), 64, T(c->e2), 32, c->wf[W4A], P + L.b[W4A], c->d2h, 0, 1, 32, c->g2))) return rc;
    if ((rc = conv(c, T(c->d2h), 32, (const A *)nullptr, 0, c->wf[W4B], P + L.b[W4B], c->d2, 0, 1, 32, c->g2))) return rc;
    upsample_kernel<A><<<blocks_for(c->V1 * 4), EW, 0, c->stream>>>(T(c->d2), T(c->up2), c->g1, 32);
    if ((rc = conv(c, T(c->up2), 32, T(c->e1), 16, c->wf[W5A], P + L.b[W5A], c->d1h, 0, 1, 16, c->g1))) return rc;
    if ((rc = conv(c, T(c->d1h), 16, (const A *)nullptr, 0, c->wf[W5B], P + L.b[W5B], c->d1, 0, 1, 16, c->g1))) return rc;
    UCK(cudaGetLastError(), "forward");
    return LBM_OK;
}

int check_err(unet_ctx *c)
{
    int h = 0;
    UCK(cudaStreamSynchronize(c->stream), "sync");
    UCK(cudaMemcpy(&h, c->derr, sizeof(int), cudaMemcpyDeviceToHost), "error word");
    if (h) {
        cudaMemset(c->derr, 0, sizeof(int));
        return ufail(c, LBM_ETIMEOUT, "a tensor-core wait timed out (bounded mbarrier wait)");
    }
    return LBM_OK;
}

template <typename A>
int backward(unet_ctx *c, const float *target, double *loss)
{
    int rc;
    auto T = [](void *p) { return static_cast<A *>(p); };
    const Layout &L = kLayout;
    float *G = c->grads;
    head_kernel<A><<<c->head_blocks, EW, 0, c->stream>>>(T(c->d1), c->params + L.wh, c->params + L.bh, target,
                                                         nullptr, c->gd1, c->hpart, c->g1);
    reduce_cols_kernel<<<72, EW, 0, c->stream>>>(c->hpart, c->head_blocks, 72, c->wtmp);
    UCK(cudaGetLastError(), "head");
    UCK(cudaMemcpyAsync(G + L.wh, c->wtmp, sizeof(float) * 68, cudaMemcpyDeviceToDevice, c->stream), "head grad");
    float hl = 0.f;
    UCK(cudaMemcpyAsync(&hl, c->wtmp + 68, sizeof(float), cudaMemcpyDeviceToHost, c->stream), "loss");
    // level 1 decoder
    if ((rc = relu_bwd<A>(c, c->gd1, c->d1, c->dy1, c->dyz1, c->g1, 16, W5B))) return rc;
    if ((rc = wgrad(c, T(c->d1h), 16, (const A *)nullptr, 0, T(c->dyz1), 16, G + L.w[W5B], c->g1))) return rc;
    if ((rc = conv(c, T(c->dy1), 16, (const A *)nullptr, 0, c->wb[W5B], nullptr, c->gh, 1, 0, 16, c->g1))) return rc;
    if ((rc = relu_bwd<A>(c, c->gh, c->d1h, c->dy1, c->dyz1, c->g1, 16, W5A))) return rc;
    if ((rc = wgrad(c, T(c->up2), 32, T(c->e1), 16, T(c->dyz1), 16, G + L.w[W5A], c->g1))) return rc;
    if ((rc = conv(c, T(c->dy1), 16, (const A *)nullptr, 0, c->wb[W5A], nullptr, c->gcat1, 1, 0, 48, c->g1))) return rc;
    up_bwd_kernel<<<blocks_for(c->V2 * 32), EW, 0, c->stream>>>(c->gcat1, 48, 32, c->gd2, c->g2);
    // level 2 decoder
    if ((rc = relu_bwd<A>(c, c->gd2, c->d2, c->dy2, c->dyz2, c->g2, 32, W4B))) return rc;
    if ((rc = wgrad(c, T(c->d2h), 32, (const A *)nullptr, 0, T(c->dyz2), 32, G + L.w[W4B], c->g2))) return rc;
    if ((rc = conv(c, T(c->dy2), 32, (const A *)nullptr, 0, c->wb[W4B], nullptr, c->gh, 1, 0, 32, c->g2))) return rc;
    if ((rc = relu_bwd<A>(c, c->gh, c->d2h, c->dy2, c->dyz2, c->g2, 32, W4A))) return rc;
    if ((rc = wgrad(c, T(c->up3), 64, T(c->e2), 32, T(c->dyz2), 32, G + L.w[W4A], c->g2))) return rc;
    if ((rc = conv(c, T(c->dy2), 32, (const A *)nullptr, 0, c->wb[W4A], nullptr, c->gcat2, 1, 0, 96, c->g2))) return rc;
    up_bwd_kernel<<<blocks_for(c->V3 * 64), EW, 0, c->stream>>>(c->gcat2, 96, 64, c->ge3, c->g3);
    // bottleneck
    if ((rc = relu_bwd<A>(c, c->ge3, c->e3, c->dy3, c->dyz3, c->g3, 64, W3B))) return rc;
    if ((rc = wgrad(c, T(c->e3h), 64, (const A *)nullptr, 0, T(c->dyz3), 64, G + L.w[W3B], c->g3))) return rc;
    if ((rc = conv(c, T(c->dy3), 64, (const A *)nullptr, 0, c->wb[W3B], nullptr, c->gh, 1, 0, 64, c->g3))) return rc;
    if ((rc = relu_bwd<A>(c, c->gh, c->e3h, c->dy3, c->dyz3, c->g3, 64, W3A))) return rc;
    if ((rc = wgrad(c, T(c->p2), 32, (const A *)nullptr, 0, T(c->dyz3), 64, G + L.w[W3A], c->g3))) return rc;
    if ((rc = conv(c, T(c->dy3), 64, (const A *)nullptr, 0, c->wb[W3A], nullptr, c->gp2, 1, 0, 32, c->g3))) return rc;
    skip_pool_kernel<<<blocks_for(c->V2 * 32), EW, 0, c->stream>>>(c->gcat2, 96, 64, c->gp2, c->ge2, c->g2, 32);
    // level 2 encoder
    if ((rc = relu_bwd<A>(c, c->ge2, c->e2, c->dy2, c->dyz2, c->g2, 32, W2B))) return rc;
    if ((rc = wgrad(c, T(c->e2h), 32, (const A *)nullptr, 0, T(c->dyz2), 32, G + L.w[W2B], c->g2))) return rc;
    if ((rc = conv(c, T(c->dy2), 32, (const A *)nullptr, 0, c->wb[W2B], nullptr, c->gh, 1, 0, 32, c->g2))) return rc;
    if ((rc = relu_bwd<A>(c, c->gh, c->e2h, c->dy2, c->dyz2, c->g2, 32, W2A))) return rc;
    if ((rc = wgrad(c, T(c->p1), 16, (const A *)nullptr, 0, T(c->dyz2), 32, G + L.w[W2A], c->g2))) return rc;
    if ((rc = conv(c, T(c->dy2), 32, (const A *)nullptr, 0, c->wb[W2A], nullptr, c->gp1, 1, 0, 16, c->g2))) return rc;
    skip_pool_kernel<<<blocks_for(c->V1 * 16), EW, 0, c->stream>>>(c->gcat1, 48, 32, c->gp1, c->ge1, c->g1, 16);
    // level 1 encoder
    if ((rc = relu_bwd<A>(c, c->ge1, c->e1, c->dy1, c->dyz1, c->g1, 16, W1B))) return rc;
    if ((rc = wgrad(c, T(c->e1h), 16, (const A *)nullptr, 0, T(c->dyz1), 16, G + L.w[W1B], c->g1))) return rc;
    if ((rc = conv(c, T(c->dy1), 16, (const A *)nullptr, 0, c->wb[W1B], nullptr, c->gh, 1, 0, 16, c->g1))) return rc;
    if ((rc = relu_bwd<A>(c, c->gh, c->e1h, c->dy1, c->dyz1, c->g1, 16, W1A))) return rc;
    if ((rc = wgrad(c, T(c->x), 16, (const A *)nullptr, 0, T(c->dyz1), 16, c->wtmp, c->g1))) return rc;
    unpad_grad_kernel<<<blocks_for(16 * 27 * 2), EW, 0, c->stream>>>(c->wtmp, 16, 2, 16, G + L.w[W1A]);
    UCK(cudaGetLastError(), "backward");
    if ((rc = check_err(c))) return rc;
    if (loss) *loss = double(hl) / double(c->V1 * 4);
    return LBM_OK;
}

}  // namespace

extern "C" {

long long unet_param_count(void) { return kLayout.total; }

const char *unet_last_error(const unet_ctx *c) { return c ? c->err.c_str() : g_unet_create_error.c_str(); }

void unet_destroy(unet_ctx *c)
{
    if (!c) return;
    ufree_all(c);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int unet_create(int n, int nb, unsigned long long seed, void *stream, unet_ctx **out)
{
    return unet_create_ex(n, nb, seed, UNET_BF16, stream, out);
}

int unet_create_ex(int n, int nb, unsigned long long seed, int precision, void *stream, unet_ctx **out)
{
    if (!out) return ufail(nullptr, LBM_EINVAL, "unet_create: out is NULL");
    *out = nullptr;
    if (precision != UNET_BF16 && precision != UNET_F32)
        return ufail(nullptr, LBM_EINVAL, "unet_create: precision must be UNET_BF16 or UNET_F32");
    if (n < 16 || n > 128 || (n & (n - 1)) || nb < 1 || nb > 4096 || ((long long)nb * (n / 4) * (n / 4) * (n / 4)) % 128)
        return ufail(nullptr, LBM_EINVAL, "unet_create: n must be a power of two in [16, 128], nb >= 1, and "
                     "nb (n/4)^3 a multiple of 128 (the tensor-core tile)");
    unet_ctx *c = new (std::nothrow) unet_ctx();
    if (!c) return ufail(nullptr, LBM_ENOMEM, "out of host memory");
    c->n = n;
    c->nb = nb;
    c->precision = precision;
    const size_t es = precision == UNET_F32 ? sizeof(float) : sizeof(bf16);  // activation element
    const int l = ilog2(n);
    c->g1 = VGrid{nb, l, l, l};
    c->g2 = VGrid{nb, l - 1, l - 1, l - 1};
    c->g3 = VGrid{nb, l - 2, l - 2, l - 2};
    c->V1 = c->g1.voxels();
    c->V2 = c->g2.voxels();
    c->V3 = c->g3.voxels();
    current_allocator(&c->alloc, &c->release, &c->user);
    auto bail = [&](int rc) {
        g_unet_create_error = c->err;
        unet_destroy(c);
        return rc;
    };
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(ufail(c, LBM_ECUDA, "cudaStreamCreate failed"));
        c->own_stream = true;
    }
    const long long np = kLayout.total;
    int rc = 0;
    const long long V1 = c->V1, V2 = c->V2, V3 = c->V3;
    if ((rc = uown(c, &c->params, np)) || (rc = uown(c, &c->grads, np)) || (rc = uown(c, &c->am, np)) ||
        (rc = uown(c, &c->av, np)))
        return bail(rc);
    // untyped buffers of `count` activation elements
    auto act = [&](void **p, long long count) {
        *p = ualloc(c, size_t(count) * es);
        return *p ? LBM_OK : ufail(c, LBM_ENOMEM, "device allocation of %zu bytes failed", size_t(count) * es);
    };
    for (int k = 0; k < NCONV; ++k) {
        if ((rc = act(&c->wf[k], 27ll * kConv[k].cout * cin_padded(k)))) return bail(rc);
        if (k != W1A && (rc = act(&c->wb[k], 27ll * kConv[k].cout * kConv[k].cin))) return bail(rc);
    }
    const VGrid g1 = c->g1, g2 = c->g2, g3 = c->g3;
    // planar activations, zeroed once: the wall rows and guards stay zero
    struct {
        void **p;
        VGrid g;
        int C;
    } acts[] = {{&c->x, g1, 16},   {&c->e1h, g1, 16}, {&c->e1, g1, 16},  {&c->p1, g2, 16},  {&c->e2h, g2, 32},
                {&c->e2, g2, 32},  {&c->p2, g3, 32},  {&c->e3h, g3, 64}, {&c->e3, g3, 64},  {&c->up3, g2, 64},
                {&c->d2h, g2, 32}, {&c->d2, g2, 32},  {&c->up2, g1, 32}, {&c->d1h, g1, 16}, {&c->d1, g1, 16},
                {&c->dy1, g1, 16}, {&c->dy2, g2, 32}, {&c->dy3, g3, 64}, {&c->dyz1, g1, 16},
                {&c->dyz2, g2, 32}, {&c->dyz3, g3, 64}};
    for (auto &t : acts) {
        if ((rc = act(t.p, planar_elems(t.g, t.C)))) return bail(rc);
        if (cudaMemsetAsync(*t.p, 0, size_t(planar_elems(t.g, t.C)) * es, c->stream) != cudaSuccess)
            return bail(ufail(c, LBM_ECUDA, "unet_create: clearing activations failed"));
    }
    if ((rc = uown(c, &c->gd1, V1 * 16)) || (rc = uown(c, &c->gcat1, V1 * 48)) || (rc = uown(c, &c->gd2, V2 * 32)) ||
        (rc = uown(c, &c->gcat2, V2 * 96)) || (rc = uown(c, &c->ge3, V3 * 64)) || (rc = uown(c, &c->gp2, V3 * 32)) ||
        (rc = uown(c, &c->ge2, V2 * 32)) || (rc = uown(c, &c->gp1, V2 * 16)) || (rc = uown(c, &c->ge1, V1 * 16)) ||
        (rc = uown(c, &c->gh, V1 * 16)))
        return bail(rc);
    // weight-gradient workspace: the largest of the ten layers
    const VGrid gl[NCONV] = {g1, g1, g2, g2, g3, g3, g2, g2, g1, g1};
    size_t ws = 0;
    for (int k = 0; k < NCONV; ++k) ws = std::max(ws, wgrad_ws_bytes(gl[k], cin_padded(k), kConv[k].cout));
    c->wpart_bytes = ws;
    c->relu_blocks = 1024;
    c->head_blocks = int(std::min<long long>(1024, (V1 + EW - 1) / EW));
    if ((rc = uown(c, &c->wpart, ws / sizeof(float))) || (rc = uown(c, &c->wtmp, 16 * 27 * 16)) ||
        (rc = uown(c, &c->bpart, size_t(c->relu_blocks) * 64)) ||
        (rc = uown(c, &c->hpart, size_t(c->head_blocks) * HEAD_PART)) || (rc = uown(c, &c->dforce, size_t(nb))) ||
        (rc = uown(c, &c->derr, 1)))
        return bail(rc);
    // He-normal weights (std sqrt(2 / (27 cin))), head std sqrt(1/16), zero biases
    std::vector<float> h(size_t(np), 0.f);
    for (int k = 0; k < NCONV; ++k) {
        const double sd = std::sqrt(2.0 / (27.0 * kConv[k].cin));
        for (long long i = 0; i < 27ll * kConv[k].cin * kConv[k].cout; ++i)
            h[size_t(kLayout.w[k] + i)] = float(sd * normal(seed, uint64_t(kLayout.w[k] + i)));
    }
    for (int i = 0; i < 64; ++i) h[size_t(kLayout.wh + i)] = float(0.25 * normal(seed, uint64_t(kLayout.wh + i)));
    if (cudaMemcpyAsync(c->params, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->grads, 0, sizeof(float) * np, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->am, 0, sizeof(float) * np, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->av, 0, sizeof(float) * np, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return bail(ufail(c, LBM_ECUDA, "unet_create: initialisation failed"));
    *out = c;
    return LBM_OK;
}

int unet_get_params(unet_ctx *c, float *host)
{
    if (!c || !host) return ufail(c, LBM_EINVAL, "unet_get_params: NULL argument");
    UCK(cudaMemcpyAsync(host, c->params, sizeof(float) * kLayout.total, cudaMemcpyDeviceToHost, c->stream), "params");
    UCK(cudaStreamSynchronize(c->stream), "sync");
    return LBM_OK;
}

int unet_set_params(unet_ctx *c, const float *host)
{
    if (!c || !host) return ufail(c, LBM_EINVAL, "unet_set_params: NULL argument");
    UCK(cudaMemcpyAsync(c->params, host, sizeof(float) * kLayout.total, cudaMemcpyHostToDevice, c->stream), "params");
    UCK(cudaStreamSynchronize(c->stream), "sync");
    c->weights_current = false;
    return LBM_OK;
}

int unet_predict(unet_ctx *c, const uint8_t *solid, const float *force, float *out)
{
    if (!c || !solid || !force || !out) return ufail(c, LBM_EINVAL, "unet_predict: NULL argument");
    const bool f32 = c->precision == UNET_F32;
    int rc = f32 ? forward<float>(c, solid, force) : forward<bf16>(c, solid, force);
    if (rc) return rc;
    if (f32)
        head_kernel<float><<<c->head_blocks, EW, 0, c->stream>>>(static_cast<const float *>(c->d1),
                                                                 c->params + kLayout.wh, c->params + kLayout.bh,
                                                                 nullptr, out, nullptr, nullptr, c->g1);
    else
        head_kernel<bf16><<<c->head_blocks, EW, 0, c->stream>>>(static_cast<const bf16 *>(c->d1),
                                                                c->params + kLayout.wh, c->params + kLayout.bh,
                                                                nullptr, out, nullptr, nullptr, c->g1);
    UCK(cudaGetLastError(), "head");
    return check_err(c);
}

int unet_loss_grad(unet_ctx *c, const uint8_t *solid, const float *force, const float *target, double *loss,
                   float *grad_host)
{
    if (!c || !solid || !force || !target) return ufail(c, LBM_EINVAL, "unet_loss_grad: NULL argument");
    const bool f32 = c->precision == UNET_F32;
    int rc = f32 ? forward<float>(c, solid, force) : forward<bf16>(c, solid, force);
    if (rc) return rc;
    if ((rc = f32 ? backward<float>(c, target, loss) : backward<bf16>(c, target, loss))) return rc;
    if (grad_host) {
        UCK(cudaMemcpy(grad_host, c->grads, sizeof(float) * kLayout.total, cudaMemcpyDeviceToHost), "grads");
    }
    return LBM_OK;
}

int unet_adam_step(unet_ctx *c, float lr, float b1, float b2, float eps)
{
    if (!c || !(lr >= 0.f) || !(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) || !(eps > 0.f))
        return ufail(c, LBM_EINVAL, "unet_adam_step: bad arguments");
    c->step += 1;
    const float c1 = float(1.0 - std::pow(double(b1), double(c->step)));
    const float c2 = float(1.0 - std::pow(double(b2), double(c->step)));
    adam_kernel<<<blocks_for(kLayout.total), EW, 0, c->stream>>>(c->params, c->grads, c->am, c->av, kLayout.total,
                                                                 lr, b1, b2, eps, c1, c2);
    UCK(cudaGetLastError(), "adam");
    c->weights_current = false;
    return LBM_OK;
}

// Scratch of one layer-API call (error word, weight-gradient partials):
// taken from the allocator installed with lbm_set_allocator (the caller's
// caching allocator) when there is one, else from cudaMalloc, and given back
// when the call returns (after its stream has been synchronised).
struct LayerScratch {
    void *p = nullptr;
    size_t bytes = 0;
    void *stream = nullptr;
    lbm_alloc_fn al = nullptr;
    lbm_free_fn rl = nullptr;
    void *user = nullptr;

    LayerScratch(size_t n, void *s) : bytes(n), stream(s)
    {
        current_allocator(&al, &rl, &user);
        if (al) {
            p = al(bytes, stream, user);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    ~LayerScratch()
    {
        if (!p) return;
        if (rl)
            rl(p, bytes, stream, user);
        else if (!al)
            cudaFree(p);
    }
    LayerScratch(const LayerScratch &) = delete;
    LayerScratch &operator=(const LayerScratch &) = delete;
};

int unet_conv3(const void *src0, int c0, int up0, const void *src1, int c1, const void *w, const float *bias,
               void *out, int out_f32, int relu, int cout, int nb, int lz, int ly, int lx, void *stream)
{
    if (nb < 1 || lz < 0 || ly < 0 || lx < 0 || lz + ly + lx > 30)
        return ufail(nullptr, LBM_EINVAL, "unet_conv3: bad grid");
    ConvArgs a{};
    a.src0 = static_cast<const bf16 *>(src0);
    a.src1 = static_cast<const bf16 *>(src1);
    a.w = static_cast<const bf16 *>(w);
    a.bias = bias;
    a.out = out;
    a.c0 = c0;
    a.c1 = c1;
    a.up0 = up0 ? 1 : 0;
    a.cout = cout;
    a.out_f32 = out_f32 ? 1 : 0;
    a.relu = relu ? 1 : 0;
    a.g = VGrid{nb, lz, ly, lx};
    LayerScratch scratch(256, stream);
    if (!scratch.p) return ufail(nullptr, LBM_ENOMEM, "unet_conv3: error word");
    int *err = static_cast<int *>(scratch.p);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(err, 0, sizeof(int), s);
    a.err = err;
    cudaError_t e = launch_conv3(a, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaErrorInvalidValue) return ufail(nullptr, LBM_EINVAL, "unet_conv3: invalid channels or pointers");
    if (e != cudaSuccess) return ufail(nullptr, LBM_ECUDA, "unet_conv3: %s", cudaGetErrorString(e));
    if (h) return ufail(nullptr, LBM_ETIMEOUT, "unet_conv3: a bounded wait timed out");
    return LBM_OK;
}

int unet_conv3_wgrad(const void *src0, int c0, int up0, const void *src1, int c1, const void *dy, int cout, float *dw,
                     int nb, int lz, int ly, int lx, void *stream)
{
    if (nb < 1 || lz < 0 || ly < 0 || lx < 0 || lz + ly + lx > 30 || c0 <= 0 || c1 < 0 || cout <= 0)
        return ufail(nullptr, LBM_EINVAL, "unet_conv3_wgrad: bad arguments");
    const VGrid g{nb, lz, ly, lx};
    WgradArgs a{};
    a.src0 = static_cast<const bf16 *>(src0);
    a.src1 = static_cast<const bf16 *>(src1);
    a.dy = static_cast<const bf16 *>(dy);
    a.c0 = c0;
    a.c1 = c1;
    a.up0 = up0 ? 1 : 0;
    a.cout = cout;
    a.rows_pad = (27 * (c0 + c1) + 127) / 128 * 128;
    a.vps = wgrad_vps(g.voxels(), a.rows_pad / 128);
    a.g = g;
    const int nsplit = wgrad_splits(g, a.vps);
    const size_t bytes = size_t(nsplit) * a.rows_pad * cout * sizeof(float) + 256;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LayerScratch scratch(bytes, stream);
    void *ws = scratch.p;
    if (!ws) return ufail(nullptr, LBM_ENOMEM, "unet_conv3_wgrad: workspace of %zu bytes", bytes);
    a.partial = static_cast<float *>(ws);
    a.err = reinterpret_cast<int *>(static_cast<char *>(ws) + bytes - 256);
    cudaMemsetAsync(a.err, 0, sizeof(int), s);
    cudaError_t e = launch_wgrad(a, nsplit, dw, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&h, a.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaErrorInvalidValue) return ufail(nullptr, LBM_EINVAL, "unet_conv3_wgrad: invalid channels");
    if (e != cudaSuccess) return ufail(nullptr, LBM_ECUDA, "unet_conv3_wgrad: %s", cudaGetErrorString(e));
    if (h) return ufail(nullptr, LBM_ETIMEOUT, "unet_conv3_wgrad: a bounded wait timed out");
    return LBM_OK;
}

int unet_conv3_halo(const void *src0, int c0, const void *src1, int c1, const void *w, const float *bias, void *out,
                    int out_f32, int relu, int cout, int nb, int lz, int ly, int lx, void *stream)
{
    if (nb < 1 || lz < 0 || ly < 0 || lx < 0 || lz + ly + lx > 30 || c0 <= 0 || c1 < 0 || (c1 && !src1))
        return ufail(nullptr, LBM_EINVAL, "unet_conv3_halo: bad arguments");
    const VGrid g{nb, lz, ly, lx};
    ConvTmaArgs a{};
    const VBox box = vbox(g, 128);
    if (g.voxels() % 128 || !make_halo_map(&a.a0, src0, c0, g, box, 16) ||
        (c1 && !make_halo_map(&a.a1, src1, c1, g, box, 16)) || !make_weight_map(&a.w, w, c0 + c1, cout))
        return ufail(nullptr, LBM_EINVAL, "unet_conv3_halo: tensor maps (alignment, channels or grid)");
    if (!c1) a.a1 = a.a0;
    a.bias = bias;
    a.out = out;
    a.c0 = c0;
    a.c1 = c1;
    a.cout = cout;
    a.out_f32 = out_f32 ? 1 : 0;
    a.relu = relu ? 1 : 0;
    a.g = g;
    LayerScratch scratch(256, stream);
    if (!scratch.p) return ufail(nullptr, LBM_ENOMEM, "unet_conv3_halo: error word");
    int *err = static_cast<int *>(scratch.p);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(err, 0, sizeof(int), s);
    a.err = err;
    cudaError_t e = launch_conv3_tma(a, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaErrorInvalidValue) return ufail(nullptr, LBM_EINVAL, "unet_conv3_halo: invalid channels or grid");
    if (e != cudaSuccess) return ufail(nullptr, LBM_ECUDA, "unet_conv3_halo: %s", cudaGetErrorString(e));
    if (h) return ufail(nullptr, LBM_ETIMEOUT, "unet_conv3_halo: a bounded wait timed out");
    return LBM_OK;
}

int unet_conv3_halo_wgrad(const void *src0, int c0, const void *src1, int c1, const void *dy, int cout, float *dw,
                          int nb, int lz, int ly, int lx, void *stream)
{
    if (nb < 1 || lz < 0 || ly < 0 || lx < 0 || lz + ly + lx > 30 || c0 <= 0 || c1 < 0 || cout <= 0 ||
        (c1 && !src1))
        return ufail(nullptr, LBM_EINVAL, "unet_conv3_halo_wgrad: bad arguments");
    const VGrid g{nb, lz, ly, lx};
    WgradTmaArgs a{};
    const VBox box = vbox(g, 64);
    if (g.voxels() % 64 || !make_halo_map(&a.a0, src0, c0, g, box, 16) ||
        (c1 && !make_halo_map(&a.a1, src1, c1, g, box, 16)) || !make_halo_map(&a.dy, dy, cout, g, box, 16))
        return ufail(nullptr, LBM_EINVAL, "unet_conv3_halo_wgrad: tensor maps (alignment, channels or grid)");
    if (!c1) a.a1 = a.a0;
    a.c0 = c0;
    a.c1 = c1;
    a.cout = cout;
    a.rows_pad = (27 * (c0 + c1) + 127) / 128 * 128;
    a.vps = wgrad_vps(g.voxels(), a.rows_pad / 128);
    a.g = g;
    const int nsplit = wgrad_splits(g, a.vps);
    const size_t bytes = size_t(nsplit) * a.rows_pad * cout * sizeof(float) + 256;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LayerScratch scratch(bytes, stream);
    void *ws = scratch.p;
    if (!ws) return ufail(nullptr, LBM_ENOMEM, "unet_conv3_halo_wgrad: workspace of %zu bytes", bytes);
    a.partial = static_cast<float *>(ws);
    a.err = reinterpret_cast<int *>(static_cast<char *>(ws) + bytes - 256);
    cudaMemsetAsync(a.err, 0, sizeof(int), s);
    cudaError_t e = launch_wgrad_tma(a, nsplit, dw, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&h, a.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaErrorInvalidValue) return ufail(nullptr, LBM_EINVAL, "unet_conv3_halo_wgrad: invalid channels");
    if (e != cudaSuccess) return ufail(nullptr, LBM_ECUDA, "unet_conv3_halo_wgrad: %s", cudaGetErrorString(e));
    if (h) return ufail(nullptr, LBM_ETIMEOUT, "unet_conv3_halo_wgrad: a bounded wait timed out");
    return LBM_OK;
}

long long unet_planar_positions(int nb, int lz, int ly, int lx)
{
    if (nb < 1 || lz < 1 || ly < 1 || lx < 1 || lz + ly + lx > 30) return -1;
    return planar_of(VGrid{nb, lz, ly, lx}).ptot;
}

int unet_conv3_planar(const void *src0, int c0, const void *src1, int c1, const void *wpk, const float *bias,
                      void *out, int out_f32, int relu, int cout, int nb, int lz, int ly, int lx, void *stream)
{
    if (unet_planar_positions(nb, lz, ly, lx) < 0 || c0 <= 0 || c1 < 0 || (c1 && !src1) || !src0 || !wpk || !out ||
        ((reinterpret_cast<uintptr_t>(src0) | reinterpret_cast<uintptr_t>(src1) | reinterpret_cast<uintptr_t>(wpk)) &
         15))
        return ufail(nullptr, LBM_EINVAL, "unet_conv3_planar: bad arguments");
    const VGrid g{nb, lz, ly, lx};
    ConvBulkArgs a{};
    a.src0 = static_cast<const bf16 *>(src0);
    a.src1 = static_cast<const bf16 *>(src1);
    a.w = static_cast<const bf16 *>(wpk);
    a.bias = bias;
    a.out = out;
    a.c0 = c0;
    a.c1 = c1;
    a.cout = cout;
    a.out_f32 = out_f32 ? 1 : 0;
    a.relu = relu ? 1 : 0;
    a.tiles = cout > 0 ? conv_tiles(g, c0 + c1, cout) : 1;
    a.g = g;
    LayerScratch scratch(256, stream);
    if (!scratch.p) return ufail(nullptr, LBM_ENOMEM, "unet_conv3_planar: error word");
    int *err = static_cast<int *>(scratch.p);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(err, 0, sizeof(int), s);
    a.err = err;
    cudaError_t e = launch_conv3_bulk(a, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaErrorInvalidValue) return ufail(nullptr, LBM_EINVAL, "unet_conv3_planar: invalid channels or grid");
    if (e != cudaSuccess) return ufail(nullptr, LBM_ECUDA, "unet_conv3_planar: %s", cudaGetErrorString(e));
    if (h) return ufail(nullptr, LBM_ETIMEOUT, "unet_conv3_planar: a bounded wait timed out");
    return LBM_OK;
}

int unet_conv3_planar_wgrad(const void *src0, int c0, const void *src1, int c1, const void *dy, int cout, float *dw,
                            int nb, int lz, int ly, int lx, void *stream)
{
    if (unet_planar_positions(nb, lz, ly, lx) < 0 || c0 <= 0 || c1 < 0 || cout <= 0 || (c1 && !src1) || !src0 ||
        !dy || !dw ||
        ((reinterpret_cast<uintptr_t>(src0) | reinterpret_cast<uintptr_t>(src1) | reinterpret_cast<uintptr_t>(dy)) &
         15))
        return ufail(nullptr, LBM_EINVAL, "unet_conv3_planar_wgrad: bad arguments");
    const VGrid g{nb, lz, ly, lx};
    WgradBulkArgs a{};
    a.src0 = static_cast<const bf16 *>(src0);
    a.src1 = static_cast<const bf16 *>(src1);
    a.dyz = static_cast<const bf16 *>(dy);
    a.c0 = c0;
    a.c1 = c1;
    a.cout = cout;
    a.rows_pad = (27 * (c0 + c1) + 127) / 128 * 128;
    wgrad_bulk_config(cout, &a.run, &a.stages);
    a.pps = wgrad_bulk_pps(g, a.rows_pad / 128, a.run);
    a.g = g;
    const int nsplit = wgrad_bulk_splits(g, a.pps);
    const size_t bytes = size_t(nsplit) * a.rows_pad * cout * sizeof(float) + 256;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LayerScratch scratch(bytes, stream);
    void *ws = scratch.p;
    if (!ws) return ufail(nullptr, LBM_ENOMEM, "unet_conv3_planar_wgrad: workspace of %zu bytes", bytes);
    a.partial = static_cast<float *>(ws);
    a.err = reinterpret_cast<int *>(static_cast<char *>(ws) + bytes - 256);
    cudaMemsetAsync(a.err, 0, sizeof(int), s);
    cudaError_t e = launch_wgrad_bulk(a, nsplit, dw, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&h, a.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaErrorInvalidValue) return ufail(nullptr, LBM_EINVAL, "unet_conv3_planar_wgrad: invalid channels");
    if (e != cudaSuccess) return ufail(nullptr, LBM_ECUDA, "unet_conv3_planar_wgrad: %s", cudaGetErrorString(e));
    if (h) return ufail(nullptr, LBM_ETIMEOUT, "unet_conv3_planar_wgrad: a bounded wait timed out");
    return LBM_OK;
}

int unet_targets_from_fields(const float *rho, const float *u, const uint8_t *solid, const float *force, int nb,
                             long long V, float rho0, float s_rho, float s_u, float *target, void *stream)
{
    if (!rho || !u || !solid || !force || !target || nb < 1 || V < 1 || !(s_rho != 0.f) || !(s_u != 0.f))
        return ufail(nullptr, LBM_EINVAL, "unet_targets_from_fields: bad arguments");
    const long long n = (long long)nb * V;
    targets_kernel<<<blocks_for(n), EW, 0, static_cast<cudaStream_t>(stream)>>>(rho, u, solid, force, V, n, rho0,
                                                                                s_rho, s_u, target);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : ufail(nullptr, LBM_ECUDA, "targets: %s", cudaGetErrorString(e));
}

int unet_fields_from_prediction(const float *pred, const uint8_t *solid, const float *force, int nb, long long V,
                                float rho0, float s_rho, float s_u, float *rho, float *u, void *stream)
{
    if (!pred || !solid || !force || !rho || !u || nb < 1 || V < 1)
        return ufail(nullptr, LBM_EINVAL, "unet_fields_from_prediction: bad arguments");
    const long long n = (long long)nb * V;
    fields_kernel<<<blocks_for(n), EW, 0, static_cast<cudaStream_t>(stream)>>>(pred, solid, force, V, n, rho0, s_rho,
                                                                               s_u, rho, u);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : ufail(nullptr, LBM_ECUDA, "fields: %s", cudaGetErrorString(e));
}

int unet_smooth_fields(float *f, float *scratch, const uint8_t *solid, int K, int comps, int n, int passes,
                       void *stream)
{
    if (!f || !scratch || !solid || K < 1 || comps < 1 || n < 2 || (n & (n - 1)) || passes < 0)
        return ufail(nullptr, LBM_EINVAL, "unet_smooth_fields: bad arguments");
    const int ln = ilog2(n);
    const long long tot = (long long)K * comps << (3 * ln);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int p = 0; p < passes; ++p)
        for (int ax = 0; ax < 3; ++ax) {
            smooth_kernel<<<blocks_for(tot), EW, 0, s>>>(f, scratch, solid, tot, comps, ln, ax);
            const cudaError_t e = cudaMemcpyAsync(f, scratch, sizeof(float) * tot, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return ufail(nullptr, LBM_ECUDA, "smooth: %s", cudaGetErrorString(e));
        }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : ufail(nullptr, LBM_ECUDA, "smooth: %s", cudaGetErrorString(e));
}

}  // extern "C"
