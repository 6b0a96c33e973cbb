// Kernels around the sweep: the ghost-layer exchange between Blocks, the
// moment (macroscopic) output, equilibrium initialisation, PDF conversion
// for checkpoints, and the FP64 invariant / residual reductions.
#include <algorithm>
#include <cstdio>

#include "device_common.cuh"
#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------- exchange
// The communication step of a Sweep (Sec. 4, Sec. 4.4): every ghost row of a
// Block that some interior cell pulls from receives, for each direction
// pointing into the Block, the post-collision PDFs of the matching boundary
// row of the neighbouring Block (or of the Block itself across a periodic
// boundary).  Only y and z faces and yz edges are copied: across x faces the
// sweep reads the neighbour directly.  Each CTA copies one slab (one
// direction plane of one face or edge) in 16-byte pieces; rows are 32-byte
// aligned and padded to whole 32-byte units, so the copy is always vectorised.
// It reads interior rows and writes ghost rows of the same buffer.
__global__ void __launch_bounds__(256) exchange_kernel(const __grid_constant__ ExchangeArgs a)
{
    const XSlab sl = a.slabs[blockIdx.x];
    const int vrow = sl.len * a.elem_bytes / 16;  // 16-byte pieces per row
    const int n = sl.rows * vrow;
    char *buf = static_cast<char *>(a.buf);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int r = k / vrow, i = k - r * vrow;
        const long long off = (long long)r * sl.stride * a.elem_bytes + (long long)i * 16;
        const uint4 v = *reinterpret_cast<const uint4 *>(buf + sl.src * a.elem_bytes + off);
        *reinterpret_cast<uint4 *>(buf + sl.dst * a.elem_bytes + off) = v;
    }
}

cudaError_t launch_exchange(const ExchangeArgs &a, cudaStream_t s)
{
    if (a.nslabs == 0) return cudaSuccess;
    exchange_kernel<<<a.nslabs, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// The in-place scheme's exchanges, one element at a time where a flag is
// fluid.  Forward (before the step from an even time): neighbours' boundary
// rows into the ghost rows, where the ghost cell is fluid (a wall or pressure
// node's slots hold what the Block's own cells stored there).  Reverse (after
// it): what the step streamed into the ghost rows to the neighbours'
// boundary rows, where the cell that streamed it is fluid (elsewhere the
// destination holds a bounce-back value its own cell wrote).
template <typename E>
__global__ void __launch_bounds__(256) exchange_flagged_kernel(const XSlabF *slabs, E *buf, const uint8_t *flags)
{
    const XSlabF sl = slabs[blockIdx.x];
    const int n = sl.rows * sl.len;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int r = k / sl.len, i = k - r * sl.len;
        if (flags[sl.fsrc + (long long)r * sl.fstride + i] & F_KIND) continue;
        const long long off = (long long)r * sl.stride + i;
        buf[sl.dst + off] = buf[sl.src + off];
    }
}

cudaError_t launch_exchange_flagged(const XSlabF *slabs, int nslabs, void *buf, int elem_bytes,
                                    const uint8_t *flags, cudaStream_t s)
{
    if (nslabs == 0) return cudaSuccess;
    if (elem_bytes == 2)
        exchange_flagged_kernel<<<nslabs, 256, 0, s>>>(slabs, static_cast<uint16_t *>(buf), flags);
    else if (elem_bytes == 4)
        exchange_flagged_kernel<<<nslabs, 256, 0, s>>>(slabs, static_cast<uint32_t *>(buf), flags);
    else
        exchange_flagged_kernel<<<nslabs, 256, 0, s>>>(slabs, static_cast<unsigned long long *>(buf), flags);
    return cudaGetLastError();
}

// ------------------------------------------------------- per-cell helpers
// storage slot of direction q (swapped in the in-place scheme's even-time layout)
__device__ __forceinline__ int slot(const FieldArgs &a, int q) { return a.swap ? opp(q) : q; }
// offset of a cell's direction-0 PDF and the direction stride: the Block
// layout, or the fluid-cell list (-1 for a solid cell there)
__device__ __forceinline__ long long cell_off(const FieldArgs &a, const BlockGeom &b, int c, int cf)
{
    return a.sidx ? (long long)a.sidx[b.cell_base + cf] : b.pdf_base + c;
}
__device__ __forceinline__ long long pstride(const FieldArgs &a, const BlockGeom &b)
{
    return a.sidx ? a.sstride : b.G;
}

struct CellPos {
    const BlockGeom *b;
    int x, y, z;   // interior coordinates inside the block
    int c;         // PDF cell index inside the block
    int cf;        // flag index inside the block
    long long o;   // cell index inside the instance's output slice
};

// Iterates the cells of the tiles (same tiling as the sweep), calling fn for
// every interior cell.
template <typename Fn>
__device__ __forceinline__ void for_each_cell(const FieldArgs &a, Fn fn)
{
    for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const Tile tile = a.tiles[t];
        const BlockGeom &b = a.blocks[tile.block];
        const int x = tile.x0 + int(threadIdx.x);
        const int y = tile.y0 + int(threadIdx.y);
        if (x >= b.nx || y >= b.ny) continue;
        const int zend = min(tile.z0 + a.tz, b.nz);
        const int pxy = b.px * b.py;
        const int pxyf = b.pxf * b.py;
        for (int z = tile.z0; z < zend; ++z) {
            CellPos p;
            p.b = &b;
            p.x = x;
            p.y = y;
            p.z = z;
            p.c = (z + 1) * pxy + (y + 1) * b.px + x;
            p.cf = (z + 1) * pxyf + (y + 1) * b.pxf + x + OXF;
            p.o = ((long long)(b.gz + z) * b.NY + (b.gy + y)) * b.NX + (b.gx + x);
            fn(p);
        }
    }
}

__device__ __forceinline__ long long inst_cells(const BlockGeom &b)
{
    return (long long)b.NX * b.NY * b.NZ;
}

// ------------------------------------------------------------ macroscopic
// Moments of the stored post-collision state (Sec. 2.1): rho = rho0 + sum f~,
// u = (sum e f~ - F/2)/rho0, which is the velocity the last collision used.
template <int ST>
__global__ void __launch_bounds__(256) macro_kernel(const __grid_constant__ FieldArgs a,
                                                    const void *buf, float *rho, float *u)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> *cs = static_cast<const CollideConsts<T> *>(a.consts);
    for_each_cell(a, [&](const CellPos &p) {
        const BlockGeom &b = *p.b;
        const CollideConsts<T> &P = cs[b.inst];
        const long long N = inst_cells(b);
        float *r = rho + b.out_base;
        float *v = u + 3 * b.out_base;
        if (a.flags[b.cell_base + p.cf] & F_KIND) {
            r[p.o] = float(P.rho0);
            v[p.o] = v[N + p.o] = v[2 * N + p.o] = 0.f;
            return;
        }
        const S *g = static_cast<const S *>(buf) + cell_off(a, b, p.c, p.cf);
        T d = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const T gq = Tr::to_t(g[(long long)slot(a, q) * pstride(a, b)]);
            d += gq;
            jx += T(ex(q)) * gq;
            jy += T(ey(q)) * gq;
            jz += T(ez(q)) * gq;
        }
        r[p.o] = float(P.rho0 + d * P.inv_s);
        v[p.o] = float(jx * P.ufac - P.uoff[0]);
        v[N + p.o] = float(jy * P.ufac - P.uoff[1]);
        v[2 * N + p.o] = float(jz * P.ufac - P.uoff[2]);
    });
}

// ------------------------------------------------------ init equilibrium
// f~ = f~eq(rho - rho0, u) of Eq. (2) in every fluid cell, 0 in solid cells.
template <int ST>
__global__ void __launch_bounds__(256) init_eq_kernel(const __grid_constant__ FieldArgs a, void *buf,
                                                      const float *rho, const float *u)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> *cs = static_cast<const CollideConsts<T> *>(a.consts);
    for_each_cell(a, [&](const CellPos &p) {
        const BlockGeom &b = *p.b;
        const CollideConsts<T> &P = cs[b.inst];
        const long long N = inst_cells(b);
        S *g = static_cast<S *>(buf) + cell_off(a, b, p.c, p.cf);
        if (a.flags[b.cell_base + p.cf] & F_KIND) {
            if (a.sidx) return;  // the fluid-cell list stores no solid cells
#pragma unroll
            for (int q = 0; q < Q; ++q) g[(long long)slot(a, q) * pstride(a, b)] = Tr::from_t(T(0));
            return;
        }
        const float *r = rho + b.out_base;
        const float *v = u + 3 * b.out_base;
        const T s = T(1) / P.inv_s;
        const T drho_s = (T(r[p.o]) - P.rho0) * s;
        const T ux = v[p.o], uy = v[N + p.o], uz = v[2 * N + p.o];
        const T usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const T eu = T(ex(q)) * ux + T(ey(q)) * uy + T(ez(q)) * uz;
            const T feq = T(wq(q)) * (drho_s + P.rho0s * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * usq));
            g[(long long)slot(a, q) * pstride(a, b)] = Tr::from_t(feq);
        }
    });
}

// f~ += f~eq(drho, u_target) - f~eq(drho, u_now) in every fluid cell: the
// velocity becomes u_target (the moments' definition of u), the density and
// the non-equilibrium part stay.  Alternated with time steps this relaxes
// the stress and density to a prescribed velocity field (consistent
// initialisation in the sense of Mei et al.).
template <int ST>
__global__ void __launch_bounds__(256) impose_u_kernel(const __grid_constant__ FieldArgs a, void *buf,
                                                       const float *u)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> *cs = static_cast<const CollideConsts<T> *>(a.consts);
    for_each_cell(a, [&](const CellPos &p) {
        const BlockGeom &b = *p.b;
        if (a.flags[b.cell_base + p.cf] & F_KIND) return;
        const CollideConsts<T> &P = cs[b.inst];
        const long long N = inst_cells(b);
        S *g = static_cast<S *>(buf) + cell_off(a, b, p.c, p.cf);
        T f[Q];
        T jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            f[q] = Tr::to_t(g[(long long)slot(a, q) * pstride(a, b)]);
            jx += T(ex(q)) * f[q];
            jy += T(ey(q)) * f[q];
            jz += T(ez(q)) * f[q];
        }
        const T n0 = jx * P.ufac - P.uoff[0], n1 = jy * P.ufac - P.uoff[1], n2 = jz * P.ufac - P.uoff[2];
        const float *v = u + 3 * b.out_base;
        const T t0 = v[p.o], t1 = v[N + p.o], t2 = v[2 * N + p.o];
        const T nsq = n0 * n0 + n1 * n1 + n2 * n2, tsq = t0 * t0 + t1 * t1 + t2 * t2;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const T en = T(ex(q)) * n0 + T(ey(q)) * n1 + T(ez(q)) * n2;
            const T et = T(ex(q)) * t0 + T(ey(q)) * t1 + T(ez(q)) * t2;
            const T d = T(wq(q)) * P.rho0s *
                        (T(3) * (et - en) + T(4.5) * (et * et - en * en) - T(1.5) * (tsq - nsq));
            g[(long long)slot(a, q) * pstride(a, b)] = Tr::from_t(f[q] + d);
        }
    });
}

// ------------------------------------------------------------ PDF in/out
template <int ST>
__global__ void __launch_bounds__(256) get_pdfs_kernel(const __grid_constant__ FieldArgs a,
                                                       const void *buf, double *f)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> *cs = static_cast<const CollideConsts<T> *>(a.consts);
    for_each_cell(a, [&](const CellPos &p) {
        const BlockGeom &b = *p.b;
        const double inv_s = double(cs[b.inst].inv_s);
        const long long N = inst_cells(b);
        double *out = f + (long long)Q * b.out_base;
        const bool solid = a.flags[b.cell_base + p.cf] & F_KIND;
        const S *g = static_cast<const S *>(buf) + cell_off(a, b, p.c, p.cf);
#pragma unroll
        for (int q = 0; q < Q; ++q)
            out[q * N + p.o] = solid ? 0.0 : double(Tr::to_t(g[(long long)slot(a, q) * pstride(a, b)])) * inv_s;
    });
}

template <int ST>
__global__ void __launch_bounds__(256) set_pdfs_kernel(const __grid_constant__ FieldArgs a, void *buf,
                                                       const double *f)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> *cs = static_cast<const CollideConsts<T> *>(a.consts);
    for_each_cell(a, [&](const CellPos &p) {
        const BlockGeom &b = *p.b;
        const double s = 1.0 / double(cs[b.inst].inv_s);
        const long long N = inst_cells(b);
        const double *in = f + (long long)Q * b.out_base;
        const bool solid = a.flags[b.cell_base + p.cf] & F_KIND;
        if (solid && a.sidx) return;  // the fluid-cell list stores no solid cells
        S *g = static_cast<S *>(buf) + cell_off(a, b, p.c, p.cf);
#pragma unroll
        for (int q = 0; q < Q; ++q)
            g[(long long)slot(a, q) * pstride(a, b)] = Tr::from_t(solid ? T(0) : T(in[q * N + p.o] * s));
    });
}

// ------------------------------------------------------------- reductions
// Sums over the fluid cells of each tile; one CTA per tile writes R_K
// partials, a second kernel adds the partials of each instance in a fixed
// order, so results are deterministic.
//  - invariants (prev == NULL): drho, momentum (before the -F/2 shift, which
//    the host applies), fluid and non-finite cell counts, every per-cell sum
//    in FP64 so that mass conservation can be checked to roundoff;
//  - residual (prev != NULL): sum |u_cur - u_prev|^2 and sum |u_cur|^2.  Each
//    cell's velocity and its change (from the per-direction differences
//    cur - prev, so the change keeps full relative precision) are formed in
//    the arithmetic type of the sweep; the norms are accumulated in FP64.
//    This keeps the check memory-bound: GB300's FP64 rate is far below its
//    FP32 rate.
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_partials(double (&acc)[R_K], double *out)
{
    __shared__ double red[8][R_K];
    const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int k = 0; k < R_K; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (warp == 0 && lane < R_K) {
        double v = 0.0;
        for (int w = 0; w < nwarps; ++w) v += red[w][lane];
        out[lane] = v;
    }
}

template <int ST>
__global__ void __launch_bounds__(256) invariants_tiles_kernel(const __grid_constant__ FieldArgs a,
                                                               const void *cur, double *partial)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> *cs = static_cast<const CollideConsts<T> *>(a.consts);
    double acc[R_K];
#pragma unroll
    for (int k = 0; k < R_K; ++k) acc[k] = 0.0;
    const long long t = blockIdx.x;
    const Tile tile = a.tiles[t];
    const BlockGeom &b = a.blocks[tile.block];
    const int x = tile.x0 + int(threadIdx.x);
    const int y = tile.y0 + int(threadIdx.y);
    if (x < b.nx && y < b.ny) {
        const double inv_s = double(cs[b.inst].inv_s);
        const int zend = min(tile.z0 + a.tz, b.nz);
        const int pxy = b.px * b.py, pxyf = b.pxf * b.py;
        for (int z = tile.z0; z < zend; ++z) {
            const int c = (z + 1) * pxy + (y + 1) * b.px + x;
            const int cf = (z + 1) * pxyf + (y + 1) * b.pxf + x + OXF;
            if (a.flags[b.cell_base + cf] & F_KIND) continue;
            const S *g = static_cast<const S *>(cur) + cell_off(a, b, c, cf);
            double d = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const double v = double(Tr::to_t(g[(long long)slot(a, q) * pstride(a, b)])) * inv_s;
                d += v;
                if (ex(q)) j[0] += ex(q) > 0 ? v : -v;
                if (ey(q)) j[1] += ey(q) > 0 ? v : -v;
                if (ez(q)) j[2] += ez(q) > 0 ? v : -v;
            }
            acc[R_DRHO] += d;
            acc[R_JX] += j[0];
            acc[R_JY] += j[1];
            acc[R_JZ] += j[2];
            acc[R_NFLUID] += 1.0;
            if (!isfinite(d + j[0] + j[1] + j[2])) acc[R_NONFINITE] += 1.0;
        }
    }
    block_partials(acc, partial + t * R_K);
}

template <int ST>
__global__ void __launch_bounds__(256) residual_tiles_kernel(const __grid_constant__ FieldArgs a,
                                                             const void *cur, const void *prev,
                                                             double *partial)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> *cs = static_cast<const CollideConsts<T> *>(a.consts);
    double acc[R_K];
#pragma unroll
    for (int k = 0; k < R_K; ++k) acc[k] = 0.0;
    const long long t = blockIdx.x;
    const Tile tile = a.tiles[t];
    const BlockGeom &b = a.blocks[tile.block];
    const int x = tile.x0 + int(threadIdx.x);
    const int y = tile.y0 + int(threadIdx.y);
    if (x < b.nx && y < b.ny) {
        const CollideConsts<T> &P = cs[b.inst];
        const T ufac = P.ufac, uo[3] = {P.uoff[0], P.uoff[1], P.uoff[2]};
        const int zend = min(tile.z0 + a.tz, b.nz);
        const int pxy = b.px * b.py, pxyf = b.pxf * b.py;
        T du2 = T(0), u2 = T(0), nf = T(0), bad = T(0);  // over this thread's few cells
        for (int z = tile.z0; z < zend; ++z) {
            const int c = (z + 1) * pxy + (y + 1) * b.px + x;
            const int cf = (z + 1) * pxyf + (y + 1) * b.pxf + x + OXF;
            if (a.flags[b.cell_base + cf] & F_KIND) continue;
            const S *g = static_cast<const S *>(cur) + cell_off(a, b, c, cf);
            const S *h = static_cast<const S *>(prev) + cell_off(a, b, c, cf);
            T j[3] = {T(0), T(0), T(0)}, dj[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const T v = Tr::to_t(g[(long long)slot(a, q) * pstride(a, b)]);
                const T dv = v - Tr::to_t(h[(long long)slot(a, q) * pstride(a, b)]);
                if (ex(q)) { j[0] += ex(q) > 0 ? v : -v; dj[0] += ex(q) > 0 ? dv : -dv; }
                if (ey(q)) { j[1] += ey(q) > 0 ? v : -v; dj[1] += ey(q) > 0 ? dv : -dv; }
                if (ez(q)) { j[2] += ez(q) > 0 ? v : -v; dj[2] += ez(q) > 0 ? dv : -dv; }
            }
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const T u = j[m] * ufac - uo[m];
                const T du = dj[m] * ufac;
                u2 += u * u;
                du2 += du * du;
            }
            nf += T(1);
            if (!isfinite(j[0] + j[1] + j[2] + dj[0] + dj[1] + dj[2])) bad += T(1);
        }
        acc[R_DU2] = double(du2);
        acc[R_U2] = double(u2);
        acc[R_NFLUID] = double(nf);
        acc[R_NONFINITE] = double(bad);
    }
    block_partials(acc, partial + t * R_K);
}

// Velocity change against a stored velocity field (the macroscopic output
// layout): per tile sum |u - u_snap|^2 and |u|^2 over fluid cells; the
// per-cell velocity is formed in the storage's arithmetic type, the sums in
// FP64.
template <int ST>
__global__ void __launch_bounds__(256) residual_snap_kernel(const __grid_constant__ FieldArgs a,
                                                            const void *cur, const float *usnap,
                                                            double *partial)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> *cs = static_cast<const CollideConsts<T> *>(a.consts);
    double acc[R_K];
#pragma unroll
    for (int k = 0; k < R_K; ++k) acc[k] = 0.0;
    const long long t = blockIdx.x;
    const Tile tile = a.tiles[t];
    const BlockGeom &b = a.blocks[tile.block];
    const int x = tile.x0 + int(threadIdx.x);
    const int y = tile.y0 + int(threadIdx.y);
    if (x < b.nx && y < b.ny) {
        const CollideConsts<T> &P = cs[b.inst];
        const T ufac = P.ufac, uo[3] = {P.uoff[0], P.uoff[1], P.uoff[2]};
        const int zend = min(tile.z0 + a.tz, b.nz);
        const int pxy = b.px * b.py, pxyf = b.pxf * b.py;
        const long long N = inst_cells(b);
        const float *us = usnap + 3 * b.out_base;
        T du2 = T(0), u2 = T(0), nf = T(0), bad = T(0);
        for (int z = tile.z0; z < zend; ++z) {
            const int c = (z + 1) * pxy + (y + 1) * b.px + x;
            const int cf = (z + 1) * pxyf + (y + 1) * b.pxf + x + OXF;
            if (a.flags[b.cell_base + cf] & F_KIND) continue;
            const long long o = ((long long)(b.gz + z) * b.NY + (b.gy + y)) * b.NX + (b.gx + x);
            const S *g = static_cast<const S *>(cur) + cell_off(a, b, c, cf);
            T j[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const T v = Tr::to_t(g[(long long)slot(a, q) * pstride(a, b)]);
                if (ex(q)) j[0] += ex(q) > 0 ? v : -v;
                if (ey(q)) j[1] += ey(q) > 0 ? v : -v;
                if (ez(q)) j[2] += ez(q) > 0 ? v : -v;
            }
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const T u = j[m] * ufac - uo[m];
                const T du = u - T(us[m * N + o]);
                u2 += u * u;
                du2 += du * du;
            }
            nf += T(1);
            if (!isfinite(j[0] + j[1] + j[2])) bad += T(1);
        }
        acc[R_DU2] = double(du2);
        acc[R_U2] = double(u2);
        acc[R_NFLUID] = double(nf);
        acc[R_NONFINITE] = double(bad);
    }
    block_partials(acc, partial + t * R_K);
}

__global__ void __launch_bounds__(256) reduce_instances_kernel(const double *partial,
                                                               const long long *begin, double *out)
{
    const int inst = blockIdx.x;
    const long long t0 = begin[inst], t1 = begin[inst + 1];
    __shared__ double red[8][R_K];
    double acc[R_K];
#pragma unroll
    for (int k = 0; k < R_K; ++k) acc[k] = 0.0;
    for (long long t = t0 + threadIdx.x; t < t1; t += blockDim.x)
#pragma unroll
        for (int k = 0; k < R_K; ++k) acc[k] += partial[t * R_K + k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < R_K; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < R_K) {
        double v = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
        out[inst * R_K + threadIdx.x] = v;
    }
}

// -------------------------------------------------------------- launchers
static dim3 field_block(const FieldArgs &a) { return dim3(a.tx, a.ty, 1); }
static unsigned field_grid(const FieldArgs &a) { return unsigned(a.ntiles); }

#define LBM_DISPATCH_ST(st, call)                   \
    switch (st) {                                   \
    case 0: call(0); break;                         \
    case 1: call(1); break;                         \
    case 2: call(2); break;                         \
    case 3: call(3); break;                         \
    default: return cudaErrorInvalidValue;          \
    }

cudaError_t launch_macroscopic(const FieldArgs &a, const void *buf, float *rho, float *u,
                               cudaStream_t s)
{
    if (a.ntiles == 0) return cudaSuccess;
#define CALL(ST) macro_kernel<ST><<<field_grid(a), field_block(a), 0, s>>>(a, buf, rho, u)
    LBM_DISPATCH_ST(a.storage, CALL)
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(const FieldArgs &a, void *buf, const float *rho, const float *u,
                                    cudaStream_t s)
{
    if (a.ntiles == 0) return cudaSuccess;
#define CALL(ST) init_eq_kernel<ST><<<field_grid(a), field_block(a), 0, s>>>(a, buf, rho, u)
    LBM_DISPATCH_ST(a.storage, CALL)
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_get_pdfs(const FieldArgs &a, const void *buf, double *f, cudaStream_t s)
{
    if (a.ntiles == 0) return cudaSuccess;
#define CALL(ST) get_pdfs_kernel<ST><<<field_grid(a), field_block(a), 0, s>>>(a, buf, f)
    LBM_DISPATCH_ST(a.storage, CALL)
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_set_pdfs(const FieldArgs &a, void *buf, const double *f, cudaStream_t s)
{
    if (a.ntiles == 0) return cudaSuccess;
#define CALL(ST) set_pdfs_kernel<ST><<<field_grid(a), field_block(a), 0, s>>>(a, buf, f)
    LBM_DISPATCH_ST(a.storage, CALL)
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_zero(void *buf, size_t bytes, cudaStream_t s)
{
    return cudaMemsetAsync(buf, 0, bytes, s);
}

cudaError_t launch_reduce(const FieldArgs &a, const void *cur, const void *prev, double *partial,
                          const long long *inst_tile_begin, int ninst, double *out, cudaStream_t s)
{
    if (a.tx * a.ty > 256) return cudaErrorInvalidValue;
    if (a.ntiles > 0) {
        if (prev) {
#define CALL(ST) residual_tiles_kernel<ST><<<field_grid(a), field_block(a), 0, s>>>(a, cur, prev, partial)
            LBM_DISPATCH_ST(a.storage, CALL)
#undef CALL
        } else {
#define CALL(ST) invariants_tiles_kernel<ST><<<field_grid(a), field_block(a), 0, s>>>(a, cur, partial)
            LBM_DISPATCH_ST(a.storage, CALL)
#undef CALL
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    reduce_instances_kernel<<<ninst, 256, 0, s>>>(partial, inst_tile_begin, out);
    return cudaGetLastError();
}

cudaError_t launch_impose_velocity(const FieldArgs &a, void *buf, const float *u, cudaStream_t s)
{
    if (a.ntiles == 0) return cudaSuccess;
#define CALL(ST) impose_u_kernel<ST><<<field_grid(a), field_block(a), 0, s>>>(a, buf, u)
    LBM_DISPATCH_ST(a.storage, CALL)
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_reduce_snap(const FieldArgs &a, const void *cur, const float *usnap, double *partial,
                               const long long *inst_tile_begin, int ninst, double *out, cudaStream_t s)
{
    if (a.tx * a.ty > 256) return cudaErrorInvalidValue;
    if (a.ntiles > 0) {
#define CALL(ST) residual_snap_kernel<ST><<<field_grid(a), field_block(a), 0, s>>>(a, cur, usnap, partial)
        LBM_DISPATCH_ST(a.storage, CALL)
#undef CALL
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    reduce_instances_kernel<<<ninst, 256, 0, s>>>(partial, inst_tile_begin, out);
    return cudaGetLastError();
}

// TMA sweep dispatch (kernels live in sweep_tma_*.cu).
template <int ST>
cudaError_t launch_sweep_tma_st(const TmaSweepArgs &, const TmaMaps &, int, cudaStream_t, int *);

cudaError_t launch_sweep_tma(const TmaSweepArgs &a, const TmaMaps &maps, int grid, cudaStream_t s)
{
    switch (a.a.storage) {
    case 0: return launch_sweep_tma_st<0>(a, maps, grid, s, nullptr);
    case 1: return launch_sweep_tma_st<1>(a, maps, grid, s, nullptr);
    case 2: return launch_sweep_tma_st<2>(a, maps, grid, s, nullptr);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t tma_occupancy(int storage, int tx, int collision, int forced, int *ctas_per_sm)
{
    TmaSweepArgs a{};
    a.a.storage = storage;
    a.a.collision = collision;
    a.a.forced = forced;
    a.nx = tx;
    TmaMaps maps{};
    switch (storage) {
    case 0: return launch_sweep_tma_st<0>(a, maps, 0, nullptr, ctas_per_sm);
    case 1: return launch_sweep_tma_st<1>(a, maps, 0, nullptr, ctas_per_sm);
    case 2: return launch_sweep_tma_st<2>(a, maps, 0, nullptr, ctas_per_sm);
    default: return cudaErrorNotSupported;
    }
}

int tma_stages(int storage) { return storage == 0 ? 4 : 5; }

// Curved walls: validate the listed links against the flags (fluid cell,
// resting-wall source), then point each cell at its table row and mark its
// link mask.  `bad` counts rejected links.
__global__ void curved_setup_kernel(const long long *fidx, const long long *sidx, const int *rows, long long n,
                                    const uint8_t *flags, uint32_t *links, int *idx, int *bad)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        if ((flags[fidx[k]] & F_KIND) != F_FLUID || (flags[sidx[k]] & F_KIND) != F_NOSLIP) {
            atomicAdd(bad, 1);
            continue;
        }
        idx[fidx[k]] = rows[k];
        atomicOr(&links[fidx[k]], L_CURVED);
    }
}

__global__ void clear_link_bit_kernel(uint32_t *links, long long n, uint32_t bit)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        links[k] &= ~bit;
}

cudaError_t launch_curved_setup(const long long *fidx, const long long *sidx, const int *rows, long long n,
                                const uint8_t *flags, uint32_t *links, long long nlinks, int *idx, int *bad,
                                cudaStream_t s)
{
    clear_link_bit_kernel<<<1024, 256, 0, s>>>(links, nlinks, L_CURVED);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || n == 0) return e;
    const long long g = std::min<long long>((n + 255) / 256, 4096);
    curved_setup_kernel<<<unsigned(g), 256, 0, s>>>(fidx, sidx, rows, n, flags, links, idx, bad);
    return cudaGetLastError();
}

// In-place sweep dispatch (kernels live in sweep_aa_*.cu).
template <int ST> cudaError_t launch_sweep_aa_st(const SweepArgs &, int, cudaStream_t);

cudaError_t launch_sweep_aa(const SweepArgs &a, int mode, cudaStream_t s)
{
    switch (a.storage) {
    case 0: return launch_sweep_aa_st<0>(a, mode, s);
    case 1: return launch_sweep_aa_st<1>(a, mode, s);
    case 2: return launch_sweep_aa_st<2>(a, mode, s);
    case 3: return launch_sweep_aa_st<3>(a, mode, s);
    default: return cudaErrorInvalidValue;
    }
}

// Sweep dispatch over the storage formats (kernels live in sweep_*.cu).
template <int ST> cudaError_t launch_sweep_st(const SweepArgs &, cudaStream_t);
template <int ST> cudaError_t launch_sweep2_st(const SweepArgs &, cudaStream_t);

cudaError_t launch_sweep(const SweepArgs &a, cudaStream_t s)
{
    if (a.pair) {
        switch (a.storage) {
        case 0: return launch_sweep2_st<0>(a, s);
        case 1: return launch_sweep2_st<1>(a, s);
        case 2: return launch_sweep2_st<2>(a, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (a.storage) {
    case 0: return launch_sweep_st<0>(a, s);
    case 1: return launch_sweep_st<1>(a, s);
    case 2: return launch_sweep_st<2>(a, s);
    case 3: return launch_sweep_st<3>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
