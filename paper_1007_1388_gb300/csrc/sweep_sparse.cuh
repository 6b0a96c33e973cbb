// The fused D3Q19 sweep over a list of fluid cells only (indirect
// addressing): the same pull stream + bounce-back + collide as the Block
// sweeps (Sec. 2.1, Sec. 3.2), on PDF arrays that hold fluid cells alone, so
// that no bytes go to solid cells of porous media.
//
// Cell i (fluid cells numbered Block by Block in (z, y, x) order) stores
// direction q at buf[q * stride + i].  The neighbour table holds, for each
// direction q = 1..18, the list index of the pull source x - e_q, or a
// negative code where that source is not fluid: -1 resting wall or solid
// cell, -2 moving wall, -3 pressure node (half-way bounce-back, Ladd's moving
// wall term, anti-bounce-back).  Periodic images and Block faces are resolved
// in the table, so no ghost exchange runs.  Row 0 of the table marks cells
// with a pressure link (bit 0).
//
// Bytes per fluid-cell update (FP32): 19 x 4 read + 19 x 4 write + 18 x 4
// neighbour indices = 224 B (PDFs as the Block sweep, indices instead of the
// solid cells' PDFs); against 153 B per cell of the Block layout it pays
// where fewer than 153 / 224 = 68% of the cells are fluid.
#pragma once

#include <algorithm>

#include "device_common.cuh"

namespace lbm {

template <int ST, int COLL, bool FORCE, int MINB, bool PRES>
__global__ void __launch_bounds__(256, MINB) sweep_sparse_kernel(const __grid_constant__ SweepArgs a)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> &K = param_consts<T>(a);  // a single instance: kernel parameters
    const CollKRef<T> KR{K};
    const S *__restrict__ src = static_cast<const S *>(a.src);
    S *__restrict__ dst = static_cast<S *>(a.dst);
    const int *__restrict__ nbr = a.nbr;
    const long long st = a.nstride, n = a.nfluid;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += gridDim.x * 256ll) {
        PresBC<T> pbc{};
        if (PRES && (__ldg(nbr + i) & 1))
            pbc = pres_setup<ST, T>(src + i, 0, int(st), param_pb<T>(a), K.ufac, K.uoff[0], K.uoff[1],
                                    K.uoff[2], K.c45, K.nc15);  // 19 stride < 2^31 (checked at create)
        T f[Q];
        f[0] = Tr::ld(src + i);
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            const int s = __ldg(nbr + q * st + i);
            if (s >= 0) {
                f[q] = Tr::ld(src + (q * st + s));
            } else {
                T v = Tr::ld(src + (opp(q) * st + i));
                if (s == -2)
                    v = vadd(v, K.bbw[q]);
                else if (PRES && s == -3)
                    v = pres_pull(q, pbc, v);
                f[q] = v;
            }
        }
        collide_v<COLL, FORCE>(f, KR);
#pragma unroll
        for (int q = 0; q < Q; ++q) Tr::st(dst + (q * st + i), f[q]);
    }
}

template <int ST, int MINB, bool PRES>
void launch_sparse_pres(const SweepArgs &a, unsigned grid, cudaStream_t s)
{
    if (a.collision == 0) {
        if (a.forced)
            sweep_sparse_kernel<ST, 0, true, MINB, PRES><<<grid, 256, 0, s>>>(a);
        else
            sweep_sparse_kernel<ST, 0, false, MINB, PRES><<<grid, 256, 0, s>>>(a);
    } else {
        if (a.forced)
            sweep_sparse_kernel<ST, 1, true, MINB, PRES><<<grid, 256, 0, s>>>(a);
        else
            sweep_sparse_kernel<ST, 1, false, MINB, PRES><<<grid, 256, 0, s>>>(a);
    }
}

template <int ST>
cudaError_t launch_sweep_sparse_st(const SweepArgs &a, cudaStream_t s)
{
    if (!a.unif) return cudaErrorInvalidConfiguration;
    if (a.nfluid == 0) return cudaSuccess;
    const long long blocks = (a.nfluid + 255) / 256;
    const unsigned grid = unsigned(a.grid > 0 ? std::min<long long>(a.grid, blocks) : blocks);
    if constexpr (ST == 3) {
        (a.pres & 1) ? launch_sparse_pres<ST, 2, true>(a, grid, s) : launch_sparse_pres<ST, 2, false>(a, grid, s);
    } else {
        if (a.minb == 4)
            (a.pres & 1) ? launch_sparse_pres<ST, 4, true>(a, grid, s) : launch_sparse_pres<ST, 4, false>(a, grid, s);
        else
            (a.pres & 1) ? launch_sparse_pres<ST, 3, true>(a, grid, s) : launch_sparse_pres<ST, 3, false>(a, grid, s);
    }
    return cudaGetLastError();
}

}  // namespace lbm
