// lbm_invariants_noalloc: the FP64 invariant reduction for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine): code
// called back from inside a framework's own allocator, where a new
// allocation would re-enter it, or processes whose device memory a caching
// allocator has already reserved in full, where cudaMalloc fails.  For them
// this entry point computes the same sums as lbm_invariants, but on a plain
// array the caller owns, and keeps its per-tile partial sums in a fixed
// file-scope device array instead of allocated scratch.  It allocates
// nothing.
#include <mutex>

#include "device_common.cuh"
#include "lbm_internal.h"
#include "lbm.h"

namespace lbm {
void set_global_error(const char *msg);
}

namespace {

using namespace lbm;

constexpr long long kCellsPerPartial = 2048;   // cells reduced by one CTA
constexpr int kMaxPartials = 32768;             // slots in the scratch array
constexpr int kSlots = 8;                       // doubles per partial
constexpr int kMaxDevices = 64;

// Partial sums of the last call: kMaxPartials * kSlots doubles = 2 MiB, held
// by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kMaxPartials * kSlots];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of kSlots values; thread 0 receives the totals in acc.
__device__ __forceinline__ void block_sum(double (&acc)[kSlots])
{
    __shared__ double red[8][kSlots];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
        const double v = warp_sum_d(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < kSlots; ++k) {
            double v = 0.0;
            for (int w = 0; w < int(blockDim.x >> 5); ++w) v += red[w][k];
            acc[k] = v;
        }
}

// CTA k sums cells [k*kCellsPerPartial, (k+1)*kCellsPerPartial) of a
// direction-major FP32 array f[q*n + c]: drho, momentum, fluid and
// non-finite cell counts.
__global__ void __launch_bounds__(256) noalloc_partials(const float *f, const uint8_t *flags,
                                                        long long n, double *scratch)
{
    double acc[kSlots];
#pragma unroll
    for (int k = 0; k < kSlots; ++k) acc[k] = 0.0;
    const long long c0 = (long long)blockIdx.x * kCellsPerPartial;
    const long long c1 = min(n, c0 + kCellsPerPartial);
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        if (flags && flags[c] != LBM_FLUID) continue;
        double d = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const double v = double(f[q * n + c]);
            d += v;
            jx += ex(q) * v;
            jy += ey(q) * v;
            jz += ez(q) * v;
        }
        acc[0] += d;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jz;
        acc[4] += 1.0;
        if (!isfinite(d + jx + jy + jz)) acc[5] += 1.0;
    }
    block_sum(acc);
    if (threadIdx.x == 0)
        for (int k = 0; k < kSlots; ++k) scratch[blockIdx.x * kSlots + k] = acc[k];
}

// One CTA adds the partials in a fixed order and writes
// {mass, mom_x, mom_y, mom_z, nonfinite}.
__global__ void __launch_bounds__(256) noalloc_total(const double *scratch, int nparts, double rho0,
                                                     double fx, double fy, double fz, double *out)
{
    double acc[kSlots];
#pragma unroll
    for (int k = 0; k < kSlots; ++k) acc[k] = 0.0;
    for (int p = threadIdx.x; p < nparts; p += blockDim.x)
#pragma unroll
        for (int k = 0; k < kSlots; ++k) acc[k] += scratch[p * kSlots + k];
    block_sum(acc);
    if (threadIdx.x == 0) {
        const double nf = acc[4];
        out[0] = nf * rho0 + acc[0];
        out[1] = acc[1] - nf * 0.5 * fx;
        out[2] = acc[2] - nf * 0.5 * fy;
        out[3] = acc[3] - nf * 0.5 * fz;
        out[4] = acc[5];
    }
}

// Device address of the scratch array for the current device, looked up
// once per device (cudaGetSymbolAddress) and cached.
int scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_global_error("lbm_invariants_noalloc: device index out of range");
        return LBM_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_global_error("lbm_invariants_noalloc: cudaGetSymbolAddress failed");
            return LBM_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_invariants_noalloc(const float *f, const uint8_t *flags, long long n_cells,
                                      double rho0, const double force[3], double *out, void *stream)
{
    if (!f || !out || n_cells <= 0) {
        lbm::set_global_error("lbm_invariants_noalloc: f and out are required and n_cells > 0");
        return LBM_EINVAL;
    }
    const long long nparts = (n_cells + kCellsPerPartial - 1) / kCellsPerPartial;
    if (nparts > kMaxPartials) {
        lbm::set_global_error("lbm_invariants_noalloc: n_cells exceeds the fixed scratch limit "
                              "of 67108864 cells (32768 partials of 2048 cells)");
        return LBM_EINVAL;
    }
    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != LBM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double fx = force ? force[0] : 0.0, fy = force ? force[1] : 0.0, fz = force ? force[2] : 0.0;
    noalloc_partials<<<unsigned(nparts), 256, 0, s>>>(f, flags, n_cells, scratch);
    noalloc_total<<<1, 256, 0, s>>>(scratch, int(nparts), rho0, fx, fy, fz, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        lbm::set_global_error(cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    return LBM_OK;
}
