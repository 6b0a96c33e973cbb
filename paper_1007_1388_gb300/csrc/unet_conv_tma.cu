// TMA-fed tensor-core 3x3x3 convolutions of the U-Net on halo-layout tensors.
//
// Warp-specialised: thread 0 is the producer, issuing for every tap (forward)
// or 64-voxel chunk (weight gradient) the tensor-map box loads of the operand
// tiles into a STAGES-deep shared-memory ring (mbarrier with expect-tx); thread
// 32 issues the tcgen05 MMAs of a stage once its bytes have landed and commits
// them to the stage's "empty" barrier, which frees the slot for the producer;
// all four warps run the TMEM epilogue after the last commit.  The periodic
// halo of the inputs (x and z) makes every tap's tile one box over whole rows,
// planes or grids (vbox): rows (y) beyond the walls come back zero-filled.
// The tiles have the layouts of the cp.async kernels (unet_conv.cu), so both
// give the same result.
//
// Every wait is bounded (2e9 cycles); a thread that gives up sets the error
// word and skips its remaining work, so every thread reaches the TMEM release.
#include "lbm_internal.h"
#include "umma.cuh"
#include "unet_internal.h"

#include <cudaTypedefs.h>

namespace lbm {
namespace {

constexpr int STAGES = 4;
constexpr int THREADS = 128;
constexpr long long kWait = 2000000000ll;

__device__ __forceinline__ int tap_dz(int t) { return t / 9 - 1; }
__device__ __forceinline__ int tap_dy(int t) { return (t / 3) % 3 - 1; }
__device__ __forceinline__ int tap_dx(int t) { return t % 3 - 1; }

__global__ void __launch_bounds__(THREADS) conv3_tma_kernel(const __grid_constant__ ConvTmaArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int cin = a.c0 + a.c1, kc = cin >> 3, kc0 = a.c0 >> 3, cout = a.cout;
    const int abytes = THREADS * cin * 2, sbytes = abytes + cout * cin * 2;
    const uint32_t tcols = cout <= 32 ? 32u : (cout <= 64 ? 64u : 128u);
    const int nx = 1 << a.g.lx, ny = 1 << a.g.ly, nz = 1 << a.g.lz;
    // this CTA's 128 voxels: whole rows / planes / grids starting at (b, z, y0, 0)
    const long long m0 = (long long)blockIdx.x * THREADS;
    const int y0 = int((m0 >> a.g.lx) & (ny - 1));
    const int z = int((m0 >> (a.g.lx + a.g.ly)) & (nz - 1));
    const int b = int(m0 >> (a.g.lx + a.g.ly + a.g.lz));

    if (warp == 0) umma::tmem_alloc(&tslot, tcols);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        umma::mbar_init(&done, 1);
        umma::mbar_fence_init();
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tslot;

    if (tid == 0) {
        // producer
        const uint32_t bytes = uint32_t(kc * 2048 + kc * cout * 16);
        for (int t = 0; t < 27; ++t) {
            const int s = t % STAGES;
            if (t >= STAGES && !umma::mbar_wait(&empty[s], ((t / STAGES) - 1) & 1, kWait)) {
                atomicExch(a.err, 1);
                break;
            }
            unsigned char *sa = smem + s * sbytes;
            unsigned char *sb = sa + abytes;
            umma::mbar_arrive_expect_tx(&full[s], bytes);
            const int xs = 1 + tap_dx(t), ys = y0 + tap_dy(t), zs = 1 + z + tap_dz(t);
            // 16-channel chunks: 128 rows x 32 bytes (A), cout rows x 32 bytes (B), 32B swizzle
            for (int k = 0; k < (cin >> 4); ++k) {
                if (k < (kc0 >> 1))
                    umma::tma_load_5d(sa + k * 4096, &a.a0, 16 * k, xs, ys, zs, b, &full[s]);
                else
                    umma::tma_load_5d(sa + k * 4096, &a.a1, 16 * k - a.c0, xs, ys, zs, b, &full[s]);
            }
            for (int k = 0; k < (cin >> 4); ++k) umma::tma_load_3d(sb + k * cout * 32, &a.w, 16 * k, t, 0, &full[s]);
        }
    } else if (tid == 32) {
        // MMA issuer
        const uint32_t idesc = umma::idesc_bf16(cout, false, false);
        bool ok = true;
        for (int t = 0; t < 27; ++t) {
            const int s = t % STAGES;
            if (!umma::mbar_wait(&full[s], (t / STAGES) & 1, kWait)) {
                atomicExch(a.err, 1);
                ok = false;
                break;
            }
            umma::fence_after();
            const uint32_t sa = umma::smem_addr(smem + s * sbytes), sb = sa + abytes;
            for (int j = 0; j < (cin >> 4); ++j)
                umma::mma_bf16(tmem, umma::sdesc_sw32(sa + j * 4096), umma::sdesc_sw32(sb + j * cout * 32), idesc,
                               (t > 0 || j > 0) ? 1u : 0u);
            umma::mma_commit(&empty[s]);
        }
        if (ok) umma::mma_commit(&done);
    }
    __syncwarp();
    // epilogue: every warp reads its 32 TMEM lanes (rows)
    const bool ready = umma::mbar_wait(&done, 0, kWait);
    if (!ready && tid == 0) atomicExch(a.err, 1);
    if (ready) {
        umma::fence_after();
        const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
        const long long m = m0 + tid;
        const int x = int(m & (nx - 1)), zc = int((m >> (a.g.lx + a.g.ly)) & (nz - 1));
        // padded element offsets of this voxel and of its periodic copies
        const long long hi = halo_index(a.g, m), plane = (long long)ny * (nx + 2);
        const long long dxh = x == 0 ? nx : (x == nx - 1 ? -nx : 0);
        const long long dzh = zc == 0 ? nz * plane : (zc == nz - 1 ? -nz * plane : 0);
        for (int c = 0; c < cout; c += 16) {
            float r[16];
            umma::tmem_ld16(trow + c, r);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float v = r[j] + (a.bias ? __ldg(a.bias + c + j) : 0.f);
                r[j] = a.relu ? fmaxf(v, 0.f) : v;
            }
            if (a.out_f32) {
                float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(a.out) + m * cout + c);
#pragma unroll
                for (int j = 0; j < 4; ++j) o[j] = make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
            } else {
                __align__(16) __nv_bfloat162 h[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(r[2 * j], r[2 * j + 1]);
                const uint4 v0 = reinterpret_cast<const uint4 *>(h)[0], v1 = reinterpret_cast<const uint4 *>(h)[1];
                bf16 *base = static_cast<bf16 *>(a.out) + c;
                const long long at[4] = {hi, hi + dxh, hi + dzh, hi + dxh + dzh};
                const bool use[4] = {true, dxh != 0, dzh != 0, dxh != 0 && dzh != 0};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (use[k]) {
                        uint4 *o = reinterpret_cast<uint4 *>(base + at[k] * cout);
                        o[0] = v0;
                        o[1] = v1;
                    }
            }
        }
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, tcols);
}

// Weight gradient: block g (16 rows = channels ci0 .. ci0+15 of one tap) of
// the 128-row tile, for the chunk's 64 voxels, is one box of 64 voxels x 32
// bytes (32B swizzle) at g * 2048: MN-major A with LBO 2048 (16-row blocks)
// and SBO 256 (8-voxel groups); the output gradient likewise for B.
__global__ void __launch_bounds__(THREADS) wgrad_tma_kernel(const __grid_constant__ WgradTmaArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int cin = a.c0 + a.c1, cout = a.cout;
    const int abytes = 16 * 1024, sbytes = abytes + (cout >> 4) * 2048;
    const uint32_t tcols = cout <= 32 ? 32u : (cout <= 64 ? 64u : 128u);
    const long long M = a.g.voxels();
    const long long vbeg = (long long)blockIdx.y * a.vps;
    const long long vend = vbeg + a.vps < M ? vbeg + a.vps : M;
    const int nchunks = int((vend - vbeg + 63) / 64);
    const int nx = 1 << a.g.lx, ny = 1 << a.g.ly, nz = 1 << a.g.lz;

    if (warp == 0) umma::tmem_alloc(&tslot, tcols);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        umma::mbar_init(&done, 1);
        umma::mbar_fence_init();
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tslot;

    if (tid == 0) {
        const uint32_t bytes = uint32_t(abytes + (cout >> 4) * 2048);
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % STAGES;
            if (c >= STAGES && !umma::mbar_wait(&empty[s], ((c / STAGES) - 1) & 1, kWait)) {
                atomicExch(a.err, 1);
                break;
            }
            unsigned char *sa = smem + s * sbytes;
            unsigned char *sb = sa + abytes;
            umma::mbar_arrive_expect_tx(&full[s], bytes);
            const long long m = vbeg + (long long)c * 64;
            const int x0 = int(m & (nx - 1));
            const int y = int((m >> a.g.lx) & (ny - 1));
            const int zz = int((m >> (a.g.lx + a.g.ly)) & (nz - 1));
            const int bb = int(m >> (a.g.lx + a.g.ly + a.g.lz));
            for (int g = 0; g < 8; ++g) {
                const int row = blockIdx.x * 128 + g * 16;
                if (row < 27 * cin) {
                    const int t = row / cin, ci = row - t * cin;
                    const int xs = 1 + x0 + tap_dx(t), ys = y + tap_dy(t), zs = 1 + zz + tap_dz(t);
                    if (ci < a.c0)
                        umma::tma_load_5d(sa + g * 2048, &a.a0, ci, xs, ys, zs, bb, &full[s]);
                    else
                        umma::tma_load_5d(sa + g * 2048, &a.a1, ci - a.c0, xs, ys, zs, bb, &full[s]);
                } else {
                    // rows past the last tap: a box wholly beyond the walls (zeros)
                    umma::tma_load_5d(sa + g * 2048, &a.a0, 0, 1, -64, 0, 0, &full[s]);
                }
            }
            for (int g = 0; g < (cout >> 4); ++g)
                umma::tma_load_5d(sb + g * 2048, &a.dy, 16 * g, 1 + x0, y, 1 + zz, bb, &full[s]);
        }
    } else if (tid == 32) {
        const uint32_t idesc = umma::idesc_bf16(cout, true, true);
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % STAGES;
            if (!umma::mbar_wait(&full[s], (c / STAGES) & 1, kWait)) {
                atomicExch(a.err, 1);
                ok = false;
                break;
            }
            umma::fence_after();
            const uint32_t sa = umma::smem_addr(smem + s * sbytes), sb = sa + abytes;
            for (int j = 0; j < 4; ++j)
                umma::mma_bf16(tmem, umma::sdesc_sw32_mn(sa + j * 512, 2048), umma::sdesc_sw32_mn(sb + j * 512, 2048),
                               idesc, (c > 0 || j > 0) ? 1u : 0u);
            umma::mma_commit(&empty[s]);
        }
        if (ok && nchunks > 0) umma::mma_commit(&done);
    }
    __syncwarp();
    const bool ready = nchunks > 0 && umma::mbar_wait(&done, 0, kWait);
    if (!ready && nchunks > 0 && tid == 0) atomicExch(a.err, 1);
    if (ready) umma::fence_after();
    const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
    const long long prow = (long long)blockIdx.y * a.rows_pad + blockIdx.x * 128 + tid;
    for (int c = 0; c < cout; c += 16) {
        float r[16];
        if (ready) {
            umma::tmem_ld16(trow + c, r);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) r[j] = 0.f;
        }
        float4 *o = reinterpret_cast<float4 *>(a.partial + prow * cout + c);
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, tcols);
}

// same ordered reduction as the cp.async weight gradient
__global__ void wgrad_tma_reduce_kernel(const float *__restrict__ partial, int nsplit, int rows, int rows_pad,
                                        int cout, int cin, float *__restrict__ dw)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cout) return;
    const int r = int(i / cout), co = int(i - (long long)r * cout);
    float acc = 0.f;
    for (int s = 0; s < nsplit; ++s) acc += partial[((long long)s * rows_pad + r) * cout + co];
    const int t = r / cin, ci = r - t * cin;
    dw[((long long)co * 27 + t) * cin + ci] = acc;
}

size_t conv3_tma_smem(int cin, int cout)
{
    const size_t ring = size_t(STAGES) * (THREADS * cin * 2 + cout * cin * 2);
    const int tcols = cout <= 32 ? 32 : (cout <= 64 ? 64 : 128);
    const size_t share = 233472 / (512 / tcols) + 1024;
    return ring > share ? ring : share;
}

// the ring, plus 8 KB so that every descriptor's reach stays inside the allocation
size_t wgrad_tma_smem(int cout) { return size_t(STAGES) * (16 * 1024 + (cout >> 4) * 2048) + 8192; }

}  // namespace

bool make_halo_map(CUtensorMap *m, const void *base, int C, const VGrid &g, const VBox &bx, int chans)
{
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tma_encode_fn());
    if (!enc || !base || C % chans || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    const cuuint64_t nx = 1ull << g.lx, ny = 1ull << g.ly, nz = 1ull << g.lz;
    cuuint64_t dims[5] = {cuuint64_t(C), nx + 2, ny, nz + 2, cuuint64_t(g.nb)};
    cuuint64_t strides[4] = {cuuint64_t(C) * 2, (nx + 2) * C * 2, ny * (nx + 2) * C * 2,
                             (nz + 2) * ny * (nx + 2) * C * 2};
    cuuint32_t box[5] = {cuuint32_t(chans), cuuint32_t(bx.bx), cuuint32_t(bx.by), cuuint32_t(bx.bz),
                         cuuint32_t(bx.bb)};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, chans == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_weight_map(CUtensorMap *m, const void *w, int cin, int cout)
{
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tma_encode_fn());
    if (!enc || !w || cin % 16 || cout > 256 || (reinterpret_cast<uintptr_t>(w) & 15)) return false;
    cuuint64_t dims[3] = {cuuint64_t(cin), 27, cuuint64_t(cout)};
    cuuint64_t strides[2] = {cuuint64_t(cin) * 2, 27ull * cin * 2};
    cuuint32_t box[3] = {16, 1, cuuint32_t(cout)};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(w), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_conv3_tma(const ConvTmaArgs &a, cudaStream_t s)
{
    const int cin = a.c0 + a.c1;
    if (a.c0 <= 0 || a.c0 % 16 || a.c1 < 0 || a.c1 % 16 || a.cout <= 0 || a.cout % 16 || a.cout > 128 || !a.out ||
        a.g.voxels() % THREADS || (1 << a.g.lx) > 256)
        return cudaErrorInvalidValue;
    const size_t sm = conv3_tma_smem(cin, a.cout);
    if (sm > 200 * 1024) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const unsigned grid = unsigned(a.g.voxels() / THREADS);
    if (grid == 0) return cudaSuccess;
    conv3_tma_kernel<<<grid, THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wgrad_tma(const WgradTmaArgs &a, int nsplit, float *dw, cudaStream_t s)
{
    const int cin = a.c0 + a.c1;
    if (a.c0 <= 0 || a.c0 % 16 || a.c1 < 0 || a.c1 % 16 || a.cout <= 0 || a.cout % 16 || a.cout > 128 ||
        a.vps <= 0 || a.vps % 64 || a.rows_pad < 27 * cin || a.rows_pad % 128 ||
        nsplit != wgrad_splits(a.g, a.vps) || a.g.voxels() % 64 || (1 << a.g.lx) > 256)
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(wgrad_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(wgrad_tma_smem(128)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid(unsigned(a.rows_pad / 128), unsigned(nsplit));
    if (nsplit > 0) wgrad_tma_kernel<<<grid, THREADS, wgrad_tma_smem(a.cout), s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = 27ll * cin * a.cout;
    wgrad_tma_reduce_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(a.partial, nsplit, 27 * cin, a.rows_pad,
                                                                        a.cout, cin, dw);
    return cudaGetLastError();
}

}  // namespace lbm
