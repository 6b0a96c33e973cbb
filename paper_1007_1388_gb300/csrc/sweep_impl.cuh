// The fused D3Q19 sweep, register version: pull stream + half-way
// bounce-back + collide, one cell per thread per z step of its tile.
//
// Sec. 3.2: one GPU thread per lattice cell, structure-of-arrays PDFs, pull
// scheme so that every store is aligned and coalesced.  For each fluid cell x
// the kernel pulls g_q = src_q[x - e_q]; when x - e_q is a wall or a solid
// cell it applies half-way bounce-back (Sec. 2.1) with the momentum-
// consistent sign, g_q = src_opp(q)[x] + s 6 w_q rho0 (e_q . u_wall).  It
// then collides (Eq. (1), BGK or TRT, Guo forcing; collide.cuh) and stores
// dst_q[x].  Solid cells are not updated.  With FP32 and 16-bit storage those
// that share a 32-byte sector of a PDF plane with fluid cells (F_FILL) store
// the rest state, 0, and (FP32) the last cells of a row zero its padding
// (F_PAD), so that every sector the sweep writes is written whole: a partly written sector
// makes the memory system read the old sector first (measured in sphere
// packings as DRAM reads well above the pulled bytes; a solid cell's PDFs are
// never read, and the interface reports them as 0).  Across x faces the
// pull reads the neighbouring Block's boundary column directly; the y/z ghost rows were
// filled by the exchange, so every Block runs the same instruction sequence
// (multi-Block runs are bitwise equal to single-Block runs).
//
// This version serves every geometry (batches of uneven instances, any Block
// size, FP64); Patches of equal 32/64/128-wide Blocks use the TMA-staged
// sweep, which gives bitwise equal results.
#pragma once

#include "device_common.cuh"

namespace lbm {

// MINB = CTAs of 256 threads per SM the register allocation must allow
// (3 -> 80 registers, 4 -> 64; FP64 uses 2 -> 128); chosen per context by
// the autotuner.  Each thread updates exactly one cell: the tile's z slices
// are the grid's y dimension.  (A per-thread loop over z made the compiler
// keep 38 strength-reduced 64-bit load and store addresses live, which
// spilled at these register budgets.)
// UNIF: a single instance whose collision constants are kernel parameters.
// MASK: near-wall cells read precomputed link masks under a warp vote (porous
// media, where near-wall and interior cells share warps).
template <int ST, int COLL, bool FORCE, int MINB, bool UNIF, bool MASK, int XBC>
__global__ void __launch_bounds__(256, MINB) sweep_kernel(const __grid_constant__ SweepArgs a)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> *__restrict__ consts = static_cast<const CollideConsts<T> *>(a.consts);

    for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const Tile tile = a.tiles[t];
        const BlockGeom &b = a.blocks[tile.block];
        const int nx = b.nx, ny = b.ny;
        int x, y, z;
        if (a.flat) {
            // a run of consecutive cells of the Block, (z, y, x) order
            const int i = tile.x0 + int(threadIdx.x);
            const int yz = quot(i, b.mnx, b.snx);  // i / nx
            x = i - yz * nx;
            z = quot(yz, b.mny, b.sny);  // yz / ny
            y = yz - z * ny;
        } else {
            x = tile.x0 + int(threadIdx.x);
            y = tile.y0 + int(threadIdx.y);
            z = tile.z0 + int(blockIdx.y);
        }
        // no lane leaves before the warp vote below
        const bool inside = x < nx && y < ny && z < b.nz;
        const int px = b.px;
        const int pxy = px * b.py;
        const int G = int(b.G);
        const CollideConsts<T> *cc = consts + b.inst;
        const CollKPtr<T> KP{cc};
        const CollKRef<T> KR{param_consts<T>(a)};
        const S *__restrict__ src = static_cast<const S *>(a.src) + b.pdf_base;
        // directions with e_x = +1 pull from x-1, e_x = -1 from x+1: on the
        // Block's first / last column those come from the x neighbour
        const S *__restrict__ srcm = src + (x == 0 ? b.xm_off : 0ll);
        const S *__restrict__ srcp = src + (x == nx - 1 ? b.xp_off : 0ll);
        S *__restrict__ dst = static_cast<S *>(a.dst) + b.pdf_base;
        const uint8_t *__restrict__ fl = a.flags + b.cell_base;

        const int pxf = b.pxf, pxyf = b.pxf * b.py;
        const int c = (z + 1) * pxy + (y + 1) * px + x;
        const int cf = (z + 1) * pxyf + (y + 1) * pxf + x + OXF;
        const uint8_t flag = inside ? fl[cf] : uint8_t(F_NOSLIP);
        // MASK: the link mask (0 for cells without a wall neighbour) is loaded
        // beside the flag, not after it, so that the pulls wait for one round
        // trip to memory instead of two
        const uint32_t lmask = MASK && inside ? __ldg(a.links + b.cell_base + cf) : 0u;
        const bool near = !(flag & F_KIND) && (flag & F_NEAR);
        // MASK: warps without a near-wall lane take the plain pull; the others
        // take one branch-free path in which each direction loads either the
        // pulled PDF or the bounced one, as the cell's link mask says.
        // Otherwise each lane branches on its own near-wall bit (no cost where
        // near-wall cells fill whole warps, as along plane walls).
        const bool take_mask = MASK ? __any_sync(0xffffffffu, near) : near;
        // solid cells (and lanes outside the Block) are not updated, but (FP32
        // and 16-bit, Patches without pressure boundaries or curved walls, whose
        // kernels keep their registers for those) cells sharing a stored sector
        // with fluid cells join the warp's stores with the rest state
        constexpr bool FILL = ST <= 2 && XBC == 0;
        const bool fill = FILL && (flag & F_FILL);
        if ((flag & F_KIND) && !fill) continue;
        T f[Q];
        if (fill) {
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = T(0);
        } else if (!take_mask) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const S *s = ex(q) > 0 ? srcm : (ex(q) < 0 ? srcp : src);
                f[q] = Tr::ld(s + (q * G + c - (ex(q) + ey(q) * px + ez(q) * pxy)));
            }
        } else if (!MASK) {
            PresBC<T> pbc{};
            if ((XBC & 1) && (__ldg(a.links + b.cell_base + cf) & L_PRESSURE))
                pbc = pres_cell<ST, UNIF, T>(param_consts<T>(a), cc, param_pb<T>(a), src, c, G);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int n = c - (ex(q) + ey(q) * px + ez(q) * pxy);
                const uint8_t nf = fl[cf - (ex(q) + ey(q) * pxf + ez(q) * pxyf)];
                if (nf & F_KIND) {
                    T v = Tr::ld(src + (opp(q) * G + c));
                    if ((nf & F_KIND) == F_MOVING)
                        v = vadd(v, UNIF ? param_consts<T>(a).bbw[q] : __ldg(&cc->bbw[q]));
                    else if ((XBC & 1) && (nf & F_KIND) == F_PRESSURE)
                        v = pres_pull(q, pbc, v);
                    f[q] = v;
                } else {
                    const S *s = ex(q) > 0 ? srcm : (ex(q) < 0 ? srcp : src);
                    f[q] = Tr::ld(s + (q * G + n));
                }
            }
        } else {
            const uint32_t lm = near ? lmask : 0u;
            const bool mv = (lm & ((XBC & 1) ? (L_MOVING | L_PRESSURE) : L_MOVING)) != 0;
            PresBC<T> pbc{};
            if ((XBC & 1) && (lm & L_PRESSURE))
                pbc = pres_cell<ST, UNIF, T>(param_consts<T>(a), cc, param_pb<T>(a), src, c, G);
            f[0] = Tr::ld(src + c);
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const bool bq = (lm >> q) & 1u;
                const S *s = ex(q) > 0 ? srcm : (ex(q) < 0 ? srcp : src);
                const S *pa = bq ? src + (opp(q) * G + c)
                                 : s + (q * G + c - (ex(q) + ey(q) * px + ez(q) * pxy));
                T v = Tr::ld(pa);
                if (mv && bq) {
                    const uint8_t nf = fl[cf - (ex(q) + ey(q) * pxf + ez(q) * pxyf)];
                    if ((nf & F_KIND) == F_MOVING)
                        v = vadd(v, UNIF ? param_consts<T>(a).bbw[q] : __ldg(&cc->bbw[q]));
                    else if ((XBC & 1) && (nf & F_KIND) == F_PRESSURE)
                        v = pres_pull(q, pbc, v);
                }
                f[q] = v;
            }
        }
        if ((XBC & 2) && near) {
            const uint32_t lmc = __ldg(a.links + b.cell_base + cf);
            if (lmc & L_CURVED)
                curved_links(f, lmc,
                             static_cast<const T *>(a.curv_q) + 18ll * __ldg(a.curv_idx + b.cell_base + cf),
                             [&](int p) { return Tr::ld(src + (p * G + c)); });
        }
        if (!fill) {
            if (UNIF)
                collide_v<COLL, FORCE>(f, KR);
            else
                collide_v<COLL, FORCE>(f, KP);
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) Tr::st(dst + (q * G + c), f[q]);
        if (FILL && (flag & F_PAD)) {  // padding element nx + j of the row, j = nx - 1 - x
            const int d = 2 * (flag >> F_PAD_SHIFT) + 1;
#pragma unroll
            for (int q = 0; q < Q; ++q) Tr::st(dst + (q * G + c + d), T(0));
        }
    }
}

template <int ST, int MINB, bool UNIF, bool MASK, int XBC>
void launch_sweep_pres(const SweepArgs &a, dim3 grid, dim3 block, cudaStream_t s)
{
    if (a.collision == 0) {
        if (a.forced)
            sweep_kernel<ST, 0, true, MINB, UNIF, MASK, XBC><<<grid, block, 0, s>>>(a);
        else
            sweep_kernel<ST, 0, false, MINB, UNIF, MASK, XBC><<<grid, block, 0, s>>>(a);
    } else {
        if (a.forced)
            sweep_kernel<ST, 1, true, MINB, UNIF, MASK, XBC><<<grid, block, 0, s>>>(a);
        else
            sweep_kernel<ST, 1, false, MINB, UNIF, MASK, XBC><<<grid, block, 0, s>>>(a);
    }
}

// Pressure boundaries (XBC bit 0) and curved walls (bit 1) are separate
// instantiations, so that the kernels of Patches without them keep the
// near-wall code they had (an extra branch there costs the 16-bit sweeps
// their load batching; the curved-wall code costs registers).
template <int ST, int MINB, bool UNIF, bool MASK>
void launch_sweep_mask(const SweepArgs &a, dim3 grid, dim3 block, cudaStream_t s)
{
    switch (a.pres & 3) {
    case 0: launch_sweep_pres<ST, MINB, UNIF, MASK, 0>(a, grid, block, s); break;
    case 1: launch_sweep_pres<ST, MINB, UNIF, MASK, 1>(a, grid, block, s); break;
    case 2: launch_sweep_pres<ST, MINB, UNIF, MASK, 2>(a, grid, block, s); break;
    default: launch_sweep_pres<ST, MINB, UNIF, MASK, 3>(a, grid, block, s); break;
    }
}

template <int ST, int MINB, bool UNIF>
void launch_sweep_unif(const SweepArgs &a, dim3 grid, dim3 block, cudaStream_t s)
{
    if (a.mask)
        launch_sweep_mask<ST, MINB, UNIF, true>(a, grid, block, s);
    else
        launch_sweep_mask<ST, MINB, UNIF, false>(a, grid, block, s);
}

template <int ST, int MINB>
void launch_sweep_minb(const SweepArgs &a, dim3 grid, dim3 block, cudaStream_t s)
{
    if (a.unif)
        launch_sweep_unif<ST, MINB, true>(a, grid, block, s);
    else
        launch_sweep_unif<ST, MINB, false>(a, grid, block, s);
}

// Register budget 5 (48 registers, five 256-thread CTAs per SM): only the
// kernels without pressure boundaries or curved walls are built with it; a
// Patch that has either runs the budget-4 kernels.
template <int ST, bool UNIF>
void launch_sweep_minb5(const SweepArgs &a, dim3 grid, dim3 block, cudaStream_t s)
{
    if (a.mask)
        launch_sweep_pres<ST, 5, UNIF, true, 0>(a, grid, block, s);
    else
        launch_sweep_pres<ST, 5, UNIF, false, 0>(a, grid, block, s);
}

template <int ST>
cudaError_t launch_sweep_st(const SweepArgs &a, cudaStream_t s)
{
    // every warp must be full: the sweep votes across its 32 lanes
    if ((a.tx * a.ty) % 32 != 0 || a.tx * a.ty > 256 || (a.flat && (a.ty != 1 || a.tz != 1)))
        return cudaErrorInvalidConfiguration;
    dim3 block(a.tx, a.ty, 1);
    const unsigned gx = unsigned(a.grid > 0 ? a.grid : a.ntiles);
    if (gx == 0) return cudaSuccess;
    const dim3 grid(gx, unsigned(a.tz), 1);
    if constexpr (ST == 3) {  // FP64 arithmetic needs the larger register budget
        launch_sweep_minb<ST, 2>(a, grid, block, s);
    } else {
        if (a.minb == 5 && (a.pres & 3) == 0) {
            if (a.unif)
                launch_sweep_minb5<ST, true>(a, grid, block, s);
            else
                launch_sweep_minb5<ST, false>(a, grid, block, s);
        } else if (a.minb >= 4) {
            launch_sweep_minb<ST, 4>(a, grid, block, s);
        } else {
            launch_sweep_minb<ST, 3>(a, grid, block, s);
        }
    }
    return cudaGetLastError();
}

}  // namespace lbm
