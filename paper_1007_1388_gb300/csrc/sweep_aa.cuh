// The fused D3Q19 sweep in place, one PDF array (the AA access pattern of
// Bailey et al., 2009): the same pull stream + bounce-back + collide of
// Sec. 2.1 and Sec. 3.2, with the streaming split over two kinds of step so
// that every thread reads and writes only locations no other thread touches
// in the same launch.
//
// The state is the two-array sweep's: S_q(x), the populations of x after its
// last collision.  Even times hold it swapped in the cell's own slots,
// A[opp(q)][x] = S_q(x); odd times hold it streamed.
//   from an even time (mode 1): f_q = A[opp(q)][x - e_q] = S_q(x - e_q), or,
//     where x - e_q is not fluid, the bounce-back of A[q][x] = S_opp(q)(x)
//     with the moving-wall or pressure term: exactly the two-array pull.
//     Collide to S'.  Push: A[q][x + e_q] = S'_q(x) for every q (into the
//     neighbour's slot when it is fluid, else into the wall or solid cell's
//     own storage, kept only so that the state can be read back), and where
//     x + e_q is not fluid also A[opp(q)][x] = the value that returns to x
//     along e_opp(q) (S'_q plus the wall term).
//   from an odd time (mode 0): f_q = A[q][x], collide, A[opp(q)][x] = f*_q.
//     Local, except for pressure links, below.
// A pressure link pulls along e_q from the pressure node P = x - e_q the
// value -S_opp(q)(x) + w_q [...](u_b), whose boundary velocity u_b comes from
// all of x's populations; in mode 1 those belong to the neighbours that pull
// them.  So the step that produces S (mode 0, or mode 4 after the state was
// written from the host) computes that value while S is in registers (or
// x's own slots) and stores it in P's slot A[opp(q)][P], the address the
// pull of mode 1 reads anyway (and x's push then overwrites).
// Each location is read and then written by exactly one thread of a launch,
// so no location is read after another thread wrote it.  Loads are plain
// (coherent) loads: the array is written in the same launch.
//
// With FP32 storage every value is the same floating-point result as in the
// two-array sweep (same pulled operands, same collision code), so the states
// are bitwise equal at every step.  With 16-bit storage a bounce-back value
// is rounded when mode 1 stores it, where the two-array sweep keeps it in
// FP32 until the collision.
//
// Across Blocks: mode 1 reaches across x faces through the Blocks' xm_off /
// xp_off like the two-array pull; beyond a wall x face (no x ghost columns)
// the slots of the wall cells live in a small side array per face; across
// y/z faces it reads and writes the ghost rows, which a forward exchange fills
// before it and a reverse exchange drains after it.
#pragma once

#include "device_common.cuh"
#include "sweep2_impl.cuh"  // Pair<ST>::st2

namespace lbm {

// Element offset in the PDF buffer of slot q of the cell (x+dx, y+dy, z+dz)
// next to cell (x, y, z) of Block b (c its index): the Block's own storage,
// the x neighbour's, or, beyond a wall x face, the face's side array.
__device__ __forceinline__ long long aa_slot(const BlockGeom &b, int q, int x, int y, int z, int c, int dx, int dy,
                                             int dz, long long xm, long long xp, int px, int pxy, int G)
{
    const int side = dx < 0 && x == 0 ? 0 : (dx > 0 && x == b.nx - 1 ? 1 : -1);
    if (side >= 0 && b.xw_base[side] >= 0)
        return b.xw_base[side] + (long long)xdir_index(q) * ((long long)b.py * (b.nz + 2)) +
               (long long)(z + dz + 1) * b.py + (y + dy + 1);
    const long long o = dx > 0 ? xp : (dx < 0 ? xm : 0ll);
    return b.pdf_base + o + ((long long)q * G + c + dx + dy * px + dz * pxy);
}

// MODE: 0 step from an odd time, 1 step from an even time, 2 the state of
// an odd time read back into the natural layout of a second array (a.dst:
// S_q(x) at slot q), 3 a natural-layout state (a.src) stored swapped into
// a.dst (an even-time array), 4 the pressure links' values of an even-time
// state that was written from the host.
//
// aa_cell: one cell (x, y, z) of Block b in the given mode; the whole work of
// the one-cell kernel, and of the two-cell kernel for cells that touch a wall
// or solid cell.
template <int ST, int COLL, bool FORCE, int MODE, bool PRES>
__device__ __forceinline__ void aa_cell(const SweepArgs &a, const BlockGeom &b, int x, int y, int z)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const CollideConsts<T> &K = param_consts<T>(a);  // a single instance: kernel parameters
    const CollKRef<T> KR{K};
    const int nx = b.nx;
    const int px = b.px, pxy = px * b.py;
    const int pxf = b.pxf, pxyf = b.pxf * b.py;
    const int G = int(b.G);
    const int c = (z + 1) * pxy + (y + 1) * px + x;
    const int cf = (z + 1) * pxyf + (y + 1) * pxf + x + OXF;
    const uint8_t *fl = a.flags + b.cell_base;
    const uint8_t flag = fl[cf];
    if (flag & F_KIND) return;  // solid and pressure cells are not updated
    const S *R0 = static_cast<const S *>(a.src);
    S *W0 = static_cast<S *>(a.dst);
    const S *R = R0 + b.pdf_base;
    S *W = W0 + b.pdf_base;
    // neighbours across the -x face (x = 0) and the +x face (x = nx - 1)
    const long long xm = x == 0 ? b.xm_off : 0ll, xp = x == nx - 1 ? b.xp_off : 0ll;
    T f[Q];

    if (MODE == 0 || MODE == 3) {
#pragma unroll
        for (int q = 0; q < Q; ++q) f[q] = Tr::to_t(R[q * G + c]);
        if (MODE == 0) collide_v<COLL, FORCE>(f, KR);
#pragma unroll
        for (int q = 0; q < Q; ++q) Tr::st(W + (opp(q) * G + c), f[q]);
        if (MODE == 0 && PRES && (flag & F_NEAR)) {
            const uint32_t lm = __ldg(a.links + b.cell_base + cf);
            if (lm & L_PRESSURE) {
                const PresBC<T> pb = pres_setup_regs<ST, T>(f, param_pb<T>(a), K.ufac, K.uoff[0], K.uoff[1],
                                                            K.uoff[2], K.c45, K.nc15);
#pragma unroll
                for (int q = 1; q < Q; ++q) {
                    if (!((lm >> q) & 1u)) continue;
                    if ((fl[cf - (ex(q) + ey(q) * pxf + ez(q) * pxyf)] & F_KIND) != F_PRESSURE) continue;
                    Tr::st(W0 + aa_slot(b, opp(q), x, y, z, c, -ex(q), -ey(q), -ez(q), xm, xp, px, pxy, G),
                           pres_pull(q, pb, Tr::to_t(Tr::from_t(f[opp(q)]))));
                }
            }
        }
        return;
    }
    if (MODE == 4) {
        if (!(flag & F_NEAR)) return;
        const uint32_t lm = __ldg(a.links + b.cell_base + cf);
        if (!(lm & L_PRESSURE)) return;
        const PresBC<T> pb = pres_cell<ST, true, T, true>(K, nullptr, param_pb<T>(a), R, c, G);
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            if (!((lm >> q) & 1u)) continue;
            if ((fl[cf - (ex(q) + ey(q) * pxf + ez(q) * pxyf)] & F_KIND) != F_PRESSURE) continue;
            Tr::st(W0 + aa_slot(b, opp(q), x, y, z, c, -ex(q), -ey(q), -ez(q), xm, xp, px, pxy, G),
                   pres_pull(q, pb, Tr::to_t(R[q * G + c])));
        }
        return;
    }
    if (MODE == 2) {  // S_q(x) was pushed to x + e_q
#pragma unroll
        for (int q = 0; q < Q; ++q)
            W[q * G + c] = R0[aa_slot(b, q, x, y, z, c, ex(q), ey(q), ez(q), xm, xp, px, pxy, G)];
        return;
    }

    const bool near = flag & F_NEAR;
    const uint32_t lm = near ? __ldg(a.links + b.cell_base + cf) : 0u;
    if (!near) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long o = ex(q) > 0 ? xm : (ex(q) < 0 ? xp : 0ll);
            f[q] = Tr::to_t(R[o + (opp(q) * G + c - (ex(q) + ey(q) * px + ez(q) * pxy))]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if ((lm >> q) & 1u) {
                const uint8_t nf = fl[cf - (ex(q) + ey(q) * pxf + ez(q) * pxyf)];
                if (PRES && (nf & F_KIND) == F_PRESSURE) {
                    // prepared by the step that produced S
                    f[q] = Tr::to_t(
                        R0[aa_slot(b, opp(q), x, y, z, c, -ex(q), -ey(q), -ez(q), xm, xp, px, pxy, G)]);
                } else {
                    T v = Tr::to_t(R[q * G + c]);  // S_opp(q)(x), stored swapped
                    if ((nf & F_KIND) == F_MOVING) v = vadd(v, K.bbw[q]);
                    f[q] = v;
                }
            } else {
                const long long o = ex(q) > 0 ? xm : (ex(q) < 0 ? xp : 0ll);
                f[q] = Tr::to_t(R[o + (opp(q) * G + c - (ex(q) + ey(q) * px + ez(q) * pxy))]);
            }
        }
    }
    collide_v<COLL, FORCE>(f, KR);
    if (!near) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long o = ex(q) > 0 ? xp : (ex(q) < 0 ? xm : 0ll);
            Tr::st(W + (o + (q * G + c + (ex(q) + ey(q) * px + ez(q) * pxy))), f[q]);
        }
    } else {
        PresBC<T> pbw{};
        if (PRES && (lm & L_PRESSURE))
            pbw = pres_setup_regs<ST, T>(f, param_pb<T>(a), K.ufac, K.uoff[0], K.uoff[1], K.uoff[2], K.c45,
                                         K.nc15);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (!((lm >> opp(q)) & 1u)) {
                const long long o = ex(q) > 0 ? xp : (ex(q) < 0 ? xm : 0ll);
                Tr::st(W + (o + (q * G + c + (ex(q) + ey(q) * px + ez(q) * pxy))), f[q]);
                continue;
            }
            // x + e_q is not fluid: S'_q is kept in that cell's slot (to read
            // the state back) and comes back to x along e_opp(q)
            Tr::st(W0 + aa_slot(b, q, x, y, z, c, ex(q), ey(q), ez(q), xm, xp, px, pxy, G), f[q]);
            T v = f[q];
            const uint8_t nf = fl[cf + (ex(q) + ey(q) * pxf + ez(q) * pxyf)];
            if ((nf & F_KIND) == F_MOVING)
                v = vadd(v, K.bbw[opp(q)]);
            else if (PRES && (nf & F_KIND) == F_PRESSURE)
                v = pres_pull(opp(q), pbw, Tr::to_t(Tr::from_t(v)));
            Tr::st(W + (opp(q) * G + c), v);
        }
    }
}

template <int ST, int COLL, bool FORCE, int MINB, int MODE, bool PRES>
__global__ void __launch_bounds__(256, MINB) sweep_aa_kernel(const __grid_constant__ SweepArgs a)
{
    for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const Tile tile = a.tiles[t];
        const BlockGeom &b = a.blocks[tile.block];
        const int nx = b.nx, ny = b.ny;
        int x, y, z;
        if (a.flat) {
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
        if (x >= nx || y >= ny || z >= b.nz) continue;
        aa_cell<ST, COLL, FORCE, MODE, PRES>(a, b, x, y, z);
    }
}

// Two cells (x even, x + 1) per thread.  A pair of fluid cells with no wall
// or solid cell among their neighbours takes the vector path in modes 0 and
// 1: the 9 directions with e_x = 0 move both cells' values with one aligned
// vector load or store, the other 10 with two scalar accesses, and the
// collision runs on the packed FP32x2 lane type (bitwise equal to the scalar
// one).  Every other pair, and every pair in modes 2..4, goes cell by cell
// through aa_cell.  Loads are plain (coherent): the array is written in the
// same launch.
template <int ST>
__device__ __forceinline__ F2 aa_ld2(const typename Traits<ST>::S *p);
template <>
__device__ __forceinline__ F2 aa_ld2<0>(const float *p)
{
    const float2 v = *reinterpret_cast<const float2 *>(p);
    return f2_pack(v.x, v.y);
}
template <>
__device__ __forceinline__ F2 aa_ld2<1>(const __half *p)
{
    const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(p));
    return f2_pack(v.x, v.y);
}
template <>
__device__ __forceinline__ F2 aa_ld2<2>(const __nv_bfloat16 *p)
{
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    return f2_pack(v.x, v.y);
}

template <int ST, int COLL, bool FORCE, int MINB, int MODE, bool PRES>
__global__ void __launch_bounds__(256, MINB) sweep_aa2_kernel(const __grid_constant__ SweepArgs a)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    const CollKRef<float> KR{a.kf};
    for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const Tile tile = a.tiles[t];
        const BlockGeom &b = a.blocks[tile.block];
        const int nx = b.nx, ny = b.ny;
        int x, y, z;  // the first (even) cell of the pair; nx is even
        if (a.flat) {
            const int i = tile.x0 + 2 * int(threadIdx.x);
            const int yz = quot(i, b.mnx, b.snx);  // i / nx
            x = i - yz * nx;
            z = quot(yz, b.mny, b.sny);  // yz / ny
            y = yz - z * ny;
        } else {
            x = tile.x0 + 2 * int(threadIdx.x);
            y = tile.y0 + int(threadIdx.y);
            z = tile.z0 + int(blockIdx.y);
        }
        if (x >= nx || y >= ny || z >= b.nz) continue;
        const int pxf = b.pxf, pxyf = b.pxf * b.py;
        const int cf = (z + 1) * pxyf + (y + 1) * pxf + x + OXF;
        const uint8_t *fl = a.flags + b.cell_base;
        const int px = b.px, pxy = px * b.py;
        const int G = int(b.G);
        const int c = (z + 1) * pxy + (y + 1) * px + x;
        const S *R = static_cast<const S *>(a.src) + b.pdf_base;
        S *W = static_cast<S *>(a.dst) + b.pdf_base;
        // cell x reaches across the -x face at x = 0, cell x + 1 across the +x face at x + 1 = nx - 1
        const long long xm0 = x == 0 ? b.xm_off : 0ll, xp1 = x + 2 == nx ? b.xp_off : 0ll;
        // modes 0 and 1: the pair's values are loaded before its flags arrive, so
        // that the loads do not wait for them (every slot read is a stored slot
        // of the Block or of its x neighbour); a pair that touches a wall or a
        // solid cell drops them and goes through the cell code
        F2 f[Q];
        if (MODE == 0) {
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = aa_ld2<ST>(R + (q * G + c));
        } else if (MODE == 1) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {  // pull from x - e_q: A[opp(q)][x - e_q]
                const long long a0 = opp(q) * G + c - (ey(q) * px + ez(q) * pxy);
                if (ex(q) == 0)
                    f[q] = aa_ld2<ST>(R + a0);
                else if (ex(q) > 0)
                    f[q] = f2_pack(Tr::to_t(R[xm0 + a0 - 1]), Tr::to_t(R[a0]));
                else
                    f[q] = f2_pack(Tr::to_t(R[a0 + 1]), Tr::to_t(R[xp1 + a0 + 2]));
            }
        }
        const uint8_t fl0 = fl[cf], fl1 = fl[cf + 1];
        if (MODE >= 2 || ((fl0 | fl1) & (F_KIND | F_NEAR))) {
#pragma unroll 1
            for (int k = 0; k < 2; ++k)  // one copy of the cell code
                if (!((k ? fl1 : fl0) & F_KIND)) aa_cell<ST, COLL, FORCE, MODE, PRES>(a, b, x + k, y, z);
            continue;
        }
        if (MODE == 0) {
            collide_v<COLL, FORCE>(f, KR);
#pragma unroll
            for (int q = 0; q < Q; ++q) Pair<ST>::st2(W + (opp(q) * G + c), f[q]);
            continue;
        }
        collide_v<COLL, FORCE>(f, KR);
#pragma unroll
        for (int q = 0; q < Q; ++q) {  // push to x + e_q: A[q][x + e_q]
            const long long b0 = q * G + c + (ey(q) * px + ez(q) * pxy);
            if (ex(q) == 0) {
                Pair<ST>::st2(W + b0, f[q]);
            } else {
                float lo, hi;
                f2_unpack(f[q], lo, hi);
                if (ex(q) > 0) {
                    Tr::st(W + (b0 + 1), lo);
                    Tr::st(W + (xp1 + b0 + 2), hi);
                } else {
                    Tr::st(W + (xm0 + b0 - 1), lo);
                    Tr::st(W + b0, hi);
                }
            }
        }
    }
}

template <int ST, int MINB, int MODE, bool PRES>
void launch_aa_mode(const SweepArgs &a, dim3 grid, dim3 block, cudaStream_t s)
{
    if constexpr (ST != 3) {  // two cells per thread: FP32 and 16-bit storage
        if (a.pair) {
            if constexpr (MODE >= 2) {
                sweep_aa2_kernel<ST, 0, false, MINB, MODE, PRES><<<grid, block, 0, s>>>(a);
            } else if (a.collision == 0) {
                if (a.forced)
                    sweep_aa2_kernel<ST, 0, true, MINB, MODE, PRES><<<grid, block, 0, s>>>(a);
                else
                    sweep_aa2_kernel<ST, 0, false, MINB, MODE, PRES><<<grid, block, 0, s>>>(a);
            } else {
                if (a.forced)
                    sweep_aa2_kernel<ST, 1, true, MINB, MODE, PRES><<<grid, block, 0, s>>>(a);
                else
                    sweep_aa2_kernel<ST, 1, false, MINB, MODE, PRES><<<grid, block, 0, s>>>(a);
            }
            return;
        }
    }
    if constexpr (MODE >= 2) {  // no collision: one instantiation serves every operator
        sweep_aa_kernel<ST, 0, false, MINB, MODE, PRES><<<grid, block, 0, s>>>(a);
    } else if (a.collision == 0) {
        if (a.forced)
            sweep_aa_kernel<ST, 0, true, MINB, MODE, PRES><<<grid, block, 0, s>>>(a);
        else
            sweep_aa_kernel<ST, 0, false, MINB, MODE, PRES><<<grid, block, 0, s>>>(a);
    } else {
        if (a.forced)
            sweep_aa_kernel<ST, 1, true, MINB, MODE, PRES><<<grid, block, 0, s>>>(a);
        else
            sweep_aa_kernel<ST, 1, false, MINB, MODE, PRES><<<grid, block, 0, s>>>(a);
    }
}

template <int ST, int MINB>
void launch_aa_minb(const SweepArgs &a, int mode, dim3 grid, dim3 block, cudaStream_t s)
{
    if (mode == 0)
        (a.pres & 1) ? launch_aa_mode<ST, MINB, 0, true>(a, grid, block, s)
               : launch_aa_mode<ST, MINB, 0, false>(a, grid, block, s);
    else if (mode == 1)
        (a.pres & 1) ? launch_aa_mode<ST, MINB, 1, true>(a, grid, block, s)
               : launch_aa_mode<ST, MINB, 1, false>(a, grid, block, s);
    else if (mode == 2)
        launch_aa_mode<ST, MINB, 2, false>(a, grid, block, s);
    else if (mode == 3)
        launch_aa_mode<ST, MINB, 3, false>(a, grid, block, s);
    else
        launch_aa_mode<ST, MINB, 4, true>(a, grid, block, s);
}

// mode 0 step from an odd time, 1 from an even time (a.src == a.dst), 2 read
// back an odd-time state, 3 store a natural-layout state swapped (a.src ->
// a.dst), 4 prepare the pressure links of an even-time state (in place)
template <int ST>
cudaError_t launch_sweep_aa_st(const SweepArgs &a, int mode, cudaStream_t s)
{
    if ((a.tx * a.ty) % 32 != 0 || a.tx * a.ty > 256 || (a.flat && (a.ty != 1 || a.tz != 1)) || !a.unif ||
        (a.pair && ST == 3))
        return cudaErrorInvalidConfiguration;
    dim3 block(a.tx, a.ty, 1);
    const unsigned gx = unsigned(a.grid > 0 ? a.grid : a.ntiles);
    if (gx == 0) return cudaSuccess;
    const dim3 grid(gx, unsigned(a.tz), 1);
    if constexpr (ST == 3) {  // FP64 arithmetic needs the larger register budget
        launch_aa_minb<ST, 2>(a, mode, grid, block, s);
    } else {
        if (a.minb == 4)
            launch_aa_minb<ST, 4>(a, mode, grid, block, s);
        else
            launch_aa_minb<ST, 3>(a, mode, grid, block, s);
    }
    return cudaGetLastError();
}

}  // namespace lbm
