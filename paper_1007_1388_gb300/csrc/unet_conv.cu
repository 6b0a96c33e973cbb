// Tensor-core 3x3x3 convolutions of the learned warm start's U-Net
// (forward / backward-data and weight gradient), tcgen05 + TMEM.
//
// Forward (and backward-data with tap-flipped, transposed weights): an
// implicit GEMM, M = 128 voxels per CTA, N = cout, K = 27 taps x cin.  For
// every tap, each of the 128 threads gathers its voxel's shifted input row
// (cin bf16, 16-byte cp.async chunks, periodic along x and z, zero-filled
// beyond the y walls) into a K-major core-matrix tile, and the weights of that
// tap into a second one; a ring of STAGES such tiles keeps the gathers of the
// next taps in flight while one thread issues the tap's cin/16 MMAs
// (128 x cout x 16 each) into the TMEM accumulator and commits them to the
// stage's mbarrier.  The epilogue reads TMEM (32x32b), adds the bias, applies
// ReLU, rounds to bf16 (or keeps fp32) and stores 16-byte vectors.
//
// Weight gradient: M = 128 (tap, channel) rows, N = cout, K = voxels of one
// split, both operands MN-major (an input row chunk is 8 channels of one
// voxel, a gradient chunk 8 output channels of one voxel), 64 voxels per
// stage; per-split partial sums are added in a fixed order afterwards.
//
// Every mbarrier wait is bounded: one thread waits, the CTA learns the outcome
// through shared memory, and on a timeout the kernel sets the error word,
// drains its own copies, frees its TMEM and returns.
#include "umma.cuh"
#include "unet_internal.h"

namespace lbm {
namespace {

constexpr int STAGES = 4;
constexpr int THREADS = 128;
constexpr long long kWait = 2000000000ll;  // SM clocks (about one second)

__device__ __forceinline__ int tap_dz(int t) { return t / 9 - 1; }
__device__ __forceinline__ int tap_dy(int t) { return (t / 3) % 3 - 1; }
__device__ __forceinline__ int tap_dx(int t) { return t % 3 - 1; }

struct Vox {
    int b, z, y, x;
};

__device__ __forceinline__ Vox vox_of(long long m, const VGrid &g)
{
    Vox v;
    v.x = int(m & ((1ll << g.lx) - 1));
    v.y = int((m >> g.lx) & ((1ll << g.ly) - 1));
    v.z = int((m >> (g.lx + g.ly)) & ((1ll << g.lz) - 1));
    v.b = int(m >> (g.lx + g.ly + g.lz));
    return v;
}

// Element offset of channel 0 of the voxel that tap t of voxel v reads in a
// tensor with `c` channels, stored at full (half = 0) or half resolution;
// -1 beyond the y walls.
__device__ __forceinline__ long long tap_src(const Vox &v, int t, const VGrid &g, int half, int c)
{
    const int ny = 1 << g.ly;
    const int ys = v.y + tap_dy(t);
    if (ys < 0 || ys >= ny) return -1;
    const int zs = (v.z + tap_dz(t)) & ((1 << g.lz) - 1);
    const int xs = (v.x + tap_dx(t)) & ((1 << g.lx) - 1);
    const int lz = g.lz - half, ly = g.ly - half, lx = g.lx - half;
    const long long idx = ((((long long)v.b << lz) + (zs >> half)) << (ly + lx)) + ((long long)(ys >> half) << lx) +
                          (xs >> half);
    return idx * c;
}

__global__ void __launch_bounds__(THREADS) conv3_kernel(const __grid_constant__ ConvArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[STAGES];
    __shared__ uint32_t tslot;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int cin = a.c0 + a.c1, kc = cin >> 3, kc0 = a.c0 >> 3;
    const int cout = a.cout;
    const int abytes = THREADS * cin * 2;
    const int sbytes = abytes + cout * cin * 2;
    const long long M = a.g.voxels();
    const long long m = (long long)blockIdx.x * THREADS + tid;  // this thread's row
    const bool row_ok = m < M;
    const Vox v = vox_of(row_ok ? m : 0, a.g);
    const uint32_t tcols = cout <= 32 ? 32u : (cout <= 64 ? 64u : 128u);

    if (warp == 0) umma::tmem_alloc(&tslot, tcols);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) umma::mbar_init(&bar[s], 1);
        umma::mbar_fence_init();
        s_ok = 1;
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tslot;

    auto load = [&](int t, int s) {
        unsigned char *sa = smem + s * sbytes;
        unsigned char *sb = sa + abytes;
        // A: this thread's voxel row, K-major core matrices (chunk k at k*2048 + row*16)
        const long long o0 = row_ok ? tap_src(v, t, a.g, a.up0, a.c0) : -1;
        const long long o1 = (row_ok && a.c1) ? tap_src(v, t, a.g, 0, a.c1) : -1;
        for (int k = 0; k < kc; ++k) {
            const bool first = k < kc0;
            const long long o = first ? o0 : o1;
            const bf16 *src = first ? a.src0 + (o < 0 ? 0 : o + 8 * k) : a.src1 + (o < 0 ? 0 : o + 8 * (k - kc0));
            umma::cp16(sa + k * 2048 + tid * 16, src, o >= 0);
        }
        // B: the tap's weights, cout rows x kc chunks (chunk k of row n at (k*cout/8 + n/8)*128 + (n%8)*16)
        for (int i = tid; i < cout * kc; i += THREADS) {
            const int n = i / kc, k = i - n * kc;
            umma::cp16(sb + (k * (cout >> 3) + (n >> 3)) * 128 + (n & 7) * 16,
                       a.w + ((long long)(n * 27 + t) * cin + 8 * k), true);
        }
    };

    const uint32_t idesc = umma::idesc_bf16(cout, false, false);
    for (int t = 0; t < STAGES - 1; ++t) {
        load(t, t);
        umma::cp_commit();
    }
    bool ok = true;
    for (int t = 0; t < 27; ++t) {
        const int s = t % STAGES;
        const int tn = t + STAGES - 1;
        if (tn < 27 && t >= 1) {
            // stage tn % STAGES last held tap t-1: its MMAs must be done
            if (tid == 0 && !umma::mbar_wait(&bar[tn % STAGES], ((t - 1) / STAGES) & 1, kWait)) s_ok = 0;
            __syncthreads();
            if (!s_ok) {
                ok = false;
                break;
            }
        }
        if (tn < 27) load(tn, tn % STAGES);
        umma::cp_commit();
        umma::cp_wait<STAGES - 1>();
        umma::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after();
            const uint32_t sa = umma::smem_addr(smem + s * sbytes), sb = sa + abytes;
            for (int j = 0; j < (cin >> 4); ++j)
                umma::mma_bf16(tmem, umma::sdesc(sa + j * 4096, 2048, 128),
                               umma::sdesc(sb + j * cout * 32, cout * 16, 128), idesc, (t > 0 || j > 0) ? 1u : 0u);
            umma::mma_commit(&bar[s]);
        }
    }
    if (ok) {
        if (tid == 0 && !umma::mbar_wait(&bar[26 % STAGES], (26 / STAGES) & 1, kWait)) s_ok = 0;
        __syncthreads();
        ok = s_ok != 0;
    }
    if (ok) {
        umma::fence_after();
        const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
        for (int c = 0; c < cout; c += 16) {
            float r[16];
            umma::tmem_ld16(trow + c, r);
            if (!row_ok) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                float x = r[j] + (a.bias ? __ldg(a.bias + c + j) : 0.f);
                r[j] = a.relu ? fmaxf(x, 0.f) : x;
            }
            if (a.out_f32) {
                float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(a.out) + m * cout + c);
#pragma unroll
                for (int j = 0; j < 4; ++j) o[j] = make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
            } else {
                __align__(16) __nv_bfloat162 h[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(r[2 * j], r[2 * j + 1]);
                uint4 *o = reinterpret_cast<uint4 *>(static_cast<bf16 *>(a.out) + m * cout + c);
                o[0] = reinterpret_cast<const uint4 *>(h)[0];
                o[1] = reinterpret_cast<const uint4 *>(h)[1];
            }
        }
    } else if (tid == 0) {
        atomicExch(a.err, 1);
    }
    umma::cp_wait<0>();
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, tcols);
}

// Weight gradient.  Row r of the 128-row tile is (tap, channel) pair
// (r / cin, r % cin) of the flattened 27 x cin weight rows; thread tid stages,
// for every 64-voxel chunk, the 16-byte input chunks of row group tid / 8 for
// voxels 8j + tid % 8 (MN-major A, chunk (voxel k, row group g) at
// ((k/8)*16 + g)*128 + (k%8)*16) and the output-gradient chunks of the same
// voxels (MN-major B).
__global__ void __launch_bounds__(THREADS) wgrad_kernel(const __grid_constant__ WgradArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[STAGES];
    __shared__ uint32_t tslot;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cin = a.c0 + a.c1, cout = a.cout;
    const int abytes = 128 * 64 * 2;
    const int sbytes = abytes + 64 * cout * 2;
    const long long M = a.g.voxels();
    const long long vbeg = (long long)blockIdx.y * a.vps;
    const long long vend = vbeg + a.vps < M ? vbeg + a.vps : M;
    const int nchunks = int((vend - vbeg + 63) / 64);
    // this thread's A row group: 8 consecutive channels of one tap
    const int row = blockIdx.x * 128 + (tid >> 3) * 8;
    const bool row_ok = row < 27 * cin;
    const int tap = row_ok ? row / cin : 0, ch = row_ok ? row - (row / cin) * cin : 0;
    const bool first = ch < a.c0;
    const uint32_t tcols = cout <= 32 ? 32u : (cout <= 64 ? 64u : 128u);

    if (warp == 0) umma::tmem_alloc(&tslot, tcols);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) umma::mbar_init(&bar[s], 1);
        umma::mbar_fence_init();
        s_ok = 1;
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tslot;

    auto load = [&](int chunk, int s) {
        unsigned char *sa = smem + s * sbytes;
        unsigned char *sb = sa + abytes;
        const long long c0v = vbeg + (long long)chunk * 64;
        for (int j = 0; j < 8; ++j) {
            const int k = 8 * j + (tid & 7);
            const long long m = c0v + k;
            long long o = -1;
            if (row_ok && m < vend) {
                const Vox v = vox_of(m, a.g);
                o = first ? tap_src(v, tap, a.g, a.up0, a.c0) : tap_src(v, tap, a.g, 0, a.c1);
            }
            const bf16 *src = first ? a.src0 + (o < 0 ? 0 : o + ch) : a.src1 + (o < 0 ? 0 : o + ch - a.c0);
            umma::cp16(sa + (j * 16 + (tid >> 3)) * 128 + (tid & 7) * 16, src, o >= 0);
        }
        // B: 64 voxels x cout/8 chunks; chunk i: voxel k = (i/cout)*8 + i%8, group (i/8) % (cout/8)
        for (int i = tid; i < 8 * cout; i += THREADS) {
            const int kg = i / cout, ng = (i >> 3) % (cout >> 3), k = kg * 8 + (i & 7);
            const long long m = c0v + k;
            const bool ok = m < vend;
            umma::cp16(sb + (kg * (cout >> 3) + ng) * 128 + (i & 7) * 16, a.dy + (ok ? m * cout + ng * 8 : 0), ok);
        }
    };

    const uint32_t idesc = umma::idesc_bf16(cout, true, true);
    for (int c = 0; c < STAGES - 1; ++c) {
        if (c < nchunks) load(c, c);
        umma::cp_commit();
    }
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int s = c % STAGES;
        const int cn = c + STAGES - 1;
        if (cn < nchunks && c >= 1) {
            if (tid == 0 && !umma::mbar_wait(&bar[cn % STAGES], ((c - 1) / STAGES) & 1, kWait)) s_ok = 0;
            __syncthreads();
            if (!s_ok) {
                ok = false;
                break;
            }
        }
        if (cn < nchunks) load(cn, cn % STAGES);
        umma::cp_commit();
        umma::cp_wait<STAGES - 1>();
        umma::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after();
            const uint32_t sa = umma::smem_addr(smem + s * sbytes), sb = sa + abytes;
            for (int j = 0; j < 4; ++j)
                umma::mma_bf16(tmem, umma::sdesc(sa + j * 4096, 2048, 128),
                               umma::sdesc(sb + j * cout * 32, cout * 16, 128), idesc, (c > 0 || j > 0) ? 1u : 0u);
            umma::mma_commit(&bar[s]);
        }
    }
    if (ok && nchunks > 0) {
        const int last = nchunks - 1;
        if (tid == 0 && !umma::mbar_wait(&bar[last % STAGES], (last / STAGES) & 1, kWait)) s_ok = 0;
        __syncthreads();
        ok = s_ok != 0;
    }
    if (ok) {
        umma::fence_after();
        const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
        const long long prow = (long long)blockIdx.y * a.rows_pad + blockIdx.x * 128 + warp * 32 + lane;
        for (int c = 0; c < cout; c += 16) {
            float r[16];
            if (nchunks > 0) {
                umma::tmem_ld16(trow + c, r);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) r[j] = 0.f;
            }
            float4 *o = reinterpret_cast<float4 *>(a.partial + prow * cout + c);
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
        }
    } else if (tid == 0) {
        atomicExch(a.err, 1);
    }
    umma::cp_wait<0>();
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, tcols);
}

// dw[co][t][ci] = sum over splits (in order) of partial[split][t*cin + ci][co]
__global__ void wgrad_reduce_kernel(const float *__restrict__ partial, int nsplit, int rows, int rows_pad, int cout,
                                    int cin, float *__restrict__ dw)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cout) return;
    const int r = int(i / cout), co = int(i - (long long)r * cout);
    float acc = 0.f;
    for (int s = 0; s < nsplit; ++s) acc += partial[((long long)s * rows_pad + r) * cout + co];
    const int t = r / cin, ci = r - t * cin;
    dw[((long long)co * 27 + t) * cin + ci] = acc;
}
}  // namespace

// Dynamic shared memory of one conv3 CTA: the STAGES ring, and at least a
// 1/k share of the SM's 228 KB where k CTAs exhaust the 512 TMEM columns, so
// that no CTA becomes resident without TMEM to allocate.
size_t conv3_smem(int cin, int cout)
{
    const size_t ring = size_t(STAGES) * (THREADS * cin * 2 + cout * cin * 2);
    const int tcols = cout <= 32 ? 32 : (cout <= 64 ? 64 : 128);
    const size_t share = 233472 / (512 / tcols) + 1024;
    return ring > share ? ring : share;
}

static size_t wgrad_smem(int cout) { return size_t(STAGES) * (128 * 64 * 2 + 64 * cout * 2); }

cudaError_t launch_conv3(const ConvArgs &a, cudaStream_t s)
{
    const int cin = a.c0 + a.c1;
    if (a.c0 <= 0 || a.c0 % 16 || a.c1 < 0 || a.c1 % 16 || a.cout <= 0 || a.cout % 16 || a.cout > 128 ||
        (a.c1 > 0 && !a.src1) || !a.src0 || !a.w || !a.out)
        return cudaErrorInvalidValue;
    if (a.up0 && (a.g.lz < 1 || a.g.ly < 1 || a.g.lx < 1)) return cudaErrorInvalidValue;
    const size_t sm = conv3_smem(cin, a.cout);
    if (sm > 200 * 1024) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long M = a.g.voxels();
    const unsigned grid = unsigned((M + THREADS - 1) / THREADS);
    if (grid == 0) return cudaSuccess;
    conv3_kernel<<<grid, THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

int wgrad_splits(const VGrid &g, int vps) { return int((g.voxels() + vps - 1) / vps); }

cudaError_t launch_wgrad(const WgradArgs &a, int nsplit, float *dw, cudaStream_t s)
{
    const int cin = a.c0 + a.c1;
    if (a.c0 <= 0 || a.c0 % 16 || a.c1 < 0 || a.c1 % 16 || a.cout <= 0 || a.cout % 16 || a.cout > 128 ||
        a.vps <= 0 || a.vps % 64 || a.rows_pad < 27 * cin || a.rows_pad % 128 || nsplit != wgrad_splits(a.g, a.vps))
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(wgrad_smem(128)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid(unsigned(a.rows_pad / 128), unsigned(nsplit));
    if (nsplit > 0) wgrad_kernel<<<grid, THREADS, wgrad_smem(a.cout), s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = 27ll * cin * a.cout;
    wgrad_reduce_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(a.partial, nsplit, 27 * cin, a.rows_pad, a.cout,
                                                                    cin, dw);
    return cudaGetLastError();
}
}  // namespace lbm
