// The fused sweep with two neighbouring cells (x, x + 1; x even) per thread,
// for FP32 and the 16-bit storage formats.  Same physics, pulls and rounding
// as the one-cell sweep (sweep_impl.cuh): the collision runs on the packed
// FP32x2 lane type of collide.cuh, whose rounding sequence per cell is that
// of the scalar one, so both sweeps give bitwise equal results.
//
// Why: the sweep is bound by the bytes each SM keeps in flight, and with one
// cell per thread a 16-bit PDF puts half as many bytes in flight per register
// as an FP32 one.  With two cells per thread the 9 directions with e_x = 0
// load both cells' values with one aligned vector load, the others with two
// scalar loads of adjacent elements, and the stores are vector stores.
#pragma once

#include "device_common.cuh"

namespace lbm {

template <int ST> struct Pair;
template <> struct Pair<0> {
    static __device__ __forceinline__ F2 ld2(const float *p)
    {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        return f2_pack(v.x, v.y);
    }
    static __device__ __forceinline__ void st2(float *p, F2 v)
    {
        float lo, hi;
        f2_unpack(v, lo, hi);
        *reinterpret_cast<float2 *>(p) = make_float2(lo, hi);
    }
};
template <> struct Pair<1> {
    static __device__ __forceinline__ F2 ld2(const __half *p)
    {
        const float2 v = __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
        return f2_pack(v.x, v.y);
    }
    static __device__ __forceinline__ void st2(__half *p, F2 v)
    {
        float lo, hi;
        f2_unpack(v, lo, hi);
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(lo, hi);
    }
};
template <> struct Pair<2> {
    static __device__ __forceinline__ F2 ld2(const __nv_bfloat16 *p)
    {
        const float2 v = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162 *>(p)));
        return f2_pack(v.x, v.y);
    }
    static __device__ __forceinline__ void st2(__nv_bfloat16 *p, F2 v)
    {
        float lo, hi;
        f2_unpack(v, lo, hi);
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(lo, hi);
    }
};

// The 19 pulled values of one cell from its link mask lm (bit q: the pull
// source x - e_q is a wall, so g_q comes from half-way bounce-back; lm = 0
// gives the plain pull).
template <int ST, bool UNIF, int XBC>
__device__ __forceinline__ void pull_mask(float (&v)[Q], uint32_t lm, const SweepArgs &a,
                                          const CollideConsts<float> *cc, const typename Traits<ST>::S *src,
                                          const typename Traits<ST>::S *srcm, const typename Traits<ST>::S *srcp,
                                          const uint8_t *fl, int c, int cf, int px, int pxy, int pxf, int pxyf, int G)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    const bool mv = (lm & ((XBC & 1) ? (L_MOVING | L_PRESSURE) : L_MOVING)) != 0;
    PresBC<float> pbc{};
    if ((XBC & 1) && (lm & L_PRESSURE)) pbc = pres_cell<ST, UNIF, float>(a.kf, cc, a.pbf, src, c, G);
    v[0] = Tr::ld(src + c);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const bool bq = (lm >> q) & 1u;
        const S *s = ex(q) > 0 ? srcm : (ex(q) < 0 ? srcp : src);
        const S *pa = bq ? src + (opp(q) * G + c) : s + (q * G + c - (ex(q) + ey(q) * px + ez(q) * pxy));
        float w = Tr::ld(pa);
        if (mv && bq) {
            const uint8_t nf = fl[cf - (ex(q) + ey(q) * pxf + ez(q) * pxyf)];
            if ((nf & F_KIND) == F_MOVING)
                w = vadd(w, UNIF ? a.kf.bbw[q] : __ldg(&cc->bbw[q]));
            else if ((XBC & 1) && (nf & F_KIND) == F_PRESSURE)
                w = pres_pull(q, pbc, w);
        }
        v[q] = w;
    }
}

// The 19 pulled values of one cell next to a wall (half-way bounce-back),
// from its link mask (MASK) or its neighbours' flags.
template <int ST, bool MASK, bool UNIF, int XBC>
__device__ __forceinline__ void pull_near(float (&v)[Q], const SweepArgs &a, const BlockGeom &b,
                                          const CollideConsts<float> *cc, const typename Traits<ST>::S *src,
                                          const typename Traits<ST>::S *srcm, const typename Traits<ST>::S *srcp,
                                          const uint8_t *fl, int c, int cf, int px, int pxy, int pxf, int pxyf, int G)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    if (MASK) {
        pull_mask<ST, UNIF, XBC>(v, __ldg(a.links + b.cell_base + cf), a, cc, src, srcm, srcp, fl, c, cf, px, pxy,
                                 pxf, pxyf, G);
    } else {
        PresBC<float> pbc{};
        if ((XBC & 1) && (__ldg(a.links + b.cell_base + cf) & L_PRESSURE))
            pbc = pres_cell<ST, UNIF, float>(a.kf, cc, a.pbf, src, c, G);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const uint8_t nf = fl[cf - (ex(q) + ey(q) * pxf + ez(q) * pxyf)];
            if (nf & F_KIND) {
                float w = Tr::ld(src + (opp(q) * G + c));
                if ((nf & F_KIND) == F_MOVING)
                    w = vadd(w, UNIF ? a.kf.bbw[q] : __ldg(&cc->bbw[q]));
                else if ((XBC & 1) && (nf & F_KIND) == F_PRESSURE)
                    w = pres_pull(q, pbc, w);
                v[q] = w;
            } else {
                const S *s = ex(q) > 0 ? srcm : (ex(q) < 0 ? srcp : src);
                v[q] = Tr::ld(s + (q * G + c - (ex(q) + ey(q) * px + ez(q) * pxy)));
            }
        }
    }
}

// curved walls of one near-wall cell (pressure-and-curved kernels only)
template <int ST>
__device__ __forceinline__ void pull_curved(float (&v)[Q], const SweepArgs &a, const BlockGeom &b,
                                            const typename Traits<ST>::S *src, int c, int cf, int G)
{
    using Tr = Traits<ST>;
    const uint32_t lm = __ldg(a.links + b.cell_base + cf);
    if (lm & L_CURVED)
        curved_links(v, lm, static_cast<const float *>(a.curv_q) + 18ll * __ldg(a.curv_idx + b.cell_base + cf),
                     [&](int p) { return Tr::ld(src + (p * G + c)); });
}

// the plain pull of one cell (no wall among its sources)
template <int ST>
__device__ __forceinline__ void pull_plain(float (&v)[Q], const typename Traits<ST>::S *src,
                                           const typename Traits<ST>::S *srcm, const typename Traits<ST>::S *srcp,
                                           int c, int px, int pxy, int G)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const S *s = ex(q) > 0 ? srcm : (ex(q) < 0 ? srcp : src);
        v[q] = Tr::ld(s + (q * G + c - (ex(q) + ey(q) * px + ez(q) * pxy)));
    }
}

template <int ST, int COLL, bool FORCE, int MINB, bool UNIF, bool MASK, int XBC>
__global__ void __launch_bounds__(256, MINB) sweep2_kernel(const __grid_constant__ SweepArgs a)
{
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    const CollideConsts<float> *__restrict__ consts = static_cast<const CollideConsts<float> *>(a.consts);

    for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const Tile tile = a.tiles[t];
        const BlockGeom &b = a.blocks[tile.block];
        const int nx = b.nx, ny = b.ny;
        int x, y, z;  // x: the first (even) cell of the pair
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
        // no lane leaves before the warp vote below (nx is even: x + 1 < nx too)
        const bool inside = x < nx && y < ny && z < b.nz;
        const int px = b.px;
        const int pxy = px * b.py;
        const int G = int(b.G);
        const CollideConsts<float> *cc = consts + b.inst;
        const CollKPtr<float> KP{cc};
        const CollKRef<float> KR{a.kf};
        const S *__restrict__ src = static_cast<const S *>(a.src) + b.pdf_base;
        // cell x pulls across the -x face when x = 0; cell x + 1 across the +x face when x + 1 = nx - 1
        const S *__restrict__ srcm0 = src + (x == 0 ? b.xm_off : 0ll);
        const S *__restrict__ srcp1 = src + (x + 2 == nx ? b.xp_off : 0ll);
        S *__restrict__ dst = static_cast<S *>(a.dst) + b.pdf_base;
        const uint8_t *__restrict__ fl = a.flags + b.cell_base;

        const int pxf = b.pxf, pxyf = b.pxf * b.py;
        const int c = (z + 1) * pxy + (y + 1) * px + x;
        const int cf = (z + 1) * pxyf + (y + 1) * pxf + x + OXF;
        F2 f[Q];
        // the plain pulls of the pair: every source lies inside the Block's
        // stored planes (ghost rows and planes in y and z; across x faces the
        // neighbour's column, or the same row's neighbour element at a wall)
        auto pull_pair = [&]() {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int a0 = q * G + c - (ey(q) * px + ez(q) * pxy);
                if (ex(q) == 0)
                    f[q] = Pair<ST>::ld2(src + a0);
                else if (ex(q) > 0)
                    f[q] = f2_pack(Tr::ld(srcm0 + (a0 - 1)), Tr::ld(src + a0));
                else
                    f[q] = f2_pack(Tr::ld(src + (a0 + 1)), Tr::ld(srcp1 + (a0 + 2)));
            }
        };
        // 16-bit storage without link masks (open Patches): the plain pulls are
        // issued before the flags arrive, so that they do not wait for them;
        // pairs next to a wall pull again below, solid ones drop them (the
        // 256^3 channel: 0.241 against 0.264 ms per sweep in F16S; FP32, bound
        // by bytes, ran 1% slower this way and keeps the flags first)
        constexpr bool SPEC = !MASK && ST != 0;
        if (SPEC && inside) pull_pair();
        const uint8_t fl0 = inside ? fl[cf] : uint8_t(F_NOSLIP), fl1 = inside ? fl[cf + 1] : uint8_t(F_NOSLIP);
        // MASK: both link masks (0 without a wall neighbour; cf is even) are
        // loaded beside the flags, so that the pulls wait for one round trip
        uint2 lmask = make_uint2(0u, 0u);
        if (MASK && inside) lmask = __ldg(reinterpret_cast<const uint2 *>(a.links + b.cell_base + cf));
        const bool solid0 = fl0 & F_KIND, solid1 = fl1 & F_KIND;
        const bool near0 = !solid0 && (fl0 & F_NEAR), near1 = !solid1 && (fl1 & F_NEAR);
        const bool take_near = MASK ? __any_sync(0xffffffffu, near0 || near1) : (near0 || near1);
        if (solid0 && solid1) continue;  // solid cells (and lanes outside the Block) are not updated
        if (!take_near) {
            if (!SPEC) pull_pair();
        } else if (MASK) {
            // one path for the whole warp: each cell's link mask (0 without a
            // wall neighbour) picks the pulled or the bounced PDF per direction,
            // so that lanes whose cells differ do not run both pulls
            float v0[Q], v1[Q];
            const uint32_t lm0 = near0 ? lmask.x : 0u;
            const uint32_t lm1 = near1 ? lmask.y : 0u;
            pull_mask<ST, UNIF, XBC>(v0, lm0, a, cc, src, srcm0, src, fl, c, cf, px, pxy, pxf, pxyf, G);
            pull_mask<ST, UNIF, XBC>(v1, lm1, a, cc, src, src, srcp1, fl, c + 1, cf + 1, px, pxy, pxf, pxyf, G);
            if (XBC & 2) {
                if (near0) pull_curved<ST>(v0, a, b, src, c, cf, G);
                if (near1) pull_curved<ST>(v1, a, b, src, c + 1, cf + 1, G);
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = f2_pack(v0[q], v1[q]);
        } else {
            float v0[Q], v1[Q];
            const S *srcp0 = src, *srcm1 = src;  // the inner faces of the pair stay in the Block
            if (near0) {
                pull_near<ST, MASK, UNIF, XBC>(v0, a, b, cc, src, srcm0, srcp0, fl, c, cf, px, pxy, pxf, pxyf, G);
                if (XBC & 2) pull_curved<ST>(v0, a, b, src, c, cf, G);
            } else {
                pull_plain<ST>(v0, src, srcm0, srcp0, c, px, pxy, G);
            }
            if (near1) {
                pull_near<ST, MASK, UNIF, XBC>(v1, a, b, cc, src, srcm1, srcp1, fl, c + 1, cf + 1, px, pxy, pxf, pxyf, G);
                if (XBC & 2) pull_curved<ST>(v1, a, b, src, c + 1, cf + 1, G);
            } else {
                pull_plain<ST>(v1, src, srcm1, srcp1, c + 1, px, pxy, G);
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = f2_pack(v0[q], v1[q]);
        }
        if (UNIF)
            collide_v<COLL, FORCE>(f, KR);
        else
            collide_v<COLL, FORCE>(f, KP);
        if (!solid0 && !solid1) {
#pragma unroll
            for (int q = 0; q < Q; ++q) Pair<ST>::st2(dst + (q * G + c), f[q]);
        } else {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                float lo, hi;
                f2_unpack(f[q], lo, hi);
                if (!solid0) Tr::st(dst + (q * G + c), lo);
                if (!solid1) Tr::st(dst + (q * G + c + 1), hi);
            }
        }
    }
}

template <int ST, int MINB, bool UNIF, bool MASK, int XBC>
void launch_sweep2_pres(const SweepArgs &a, dim3 grid, dim3 block, cudaStream_t s)
{
    if (a.collision == 0) {
        if (a.forced)
            sweep2_kernel<ST, 0, true, MINB, UNIF, MASK, XBC><<<grid, block, 0, s>>>(a);
        else
            sweep2_kernel<ST, 0, false, MINB, UNIF, MASK, XBC><<<grid, block, 0, s>>>(a);
    } else {
        if (a.forced)
            sweep2_kernel<ST, 1, true, MINB, UNIF, MASK, XBC><<<grid, block, 0, s>>>(a);
        else
            sweep2_kernel<ST, 1, false, MINB, UNIF, MASK, XBC><<<grid, block, 0, s>>>(a);
    }
}

// pressure boundaries and curved walls: separate instantiations (see launch_sweep_mask)
template <int ST, int MINB, bool UNIF, bool MASK>
void launch_sweep2_mask(const SweepArgs &a, dim3 grid, dim3 block, cudaStream_t s)
{
    switch (a.pres & 3) {
    case 0: launch_sweep2_pres<ST, MINB, UNIF, MASK, 0>(a, grid, block, s); break;
    case 1: launch_sweep2_pres<ST, MINB, UNIF, MASK, 1>(a, grid, block, s); break;
    case 2: launch_sweep2_pres<ST, MINB, UNIF, MASK, 2>(a, grid, block, s); break;
    default: launch_sweep2_pres<ST, MINB, UNIF, MASK, 3>(a, grid, block, s); break;
    }
}

template <int ST, int MINB>
void launch_sweep2_minb(const SweepArgs &a, dim3 grid, dim3 block, cudaStream_t s)
{
    if (a.unif) {
        if (a.mask)
            launch_sweep2_mask<ST, MINB, true, true>(a, grid, block, s);
        else
            launch_sweep2_mask<ST, MINB, true, false>(a, grid, block, s);
    } else {
        if (a.mask)
            launch_sweep2_mask<ST, MINB, false, true>(a, grid, block, s);
        else
            launch_sweep2_mask<ST, MINB, false, false>(a, grid, block, s);
    }
}

// Two cells per thread: block (tx, ty) threads cover 2 tx x ty cells.
template <int ST>
cudaError_t launch_sweep2_st(const SweepArgs &a, cudaStream_t s)
{
    if ((a.tx * a.ty) % 32 != 0 || a.tx * a.ty > 256 || (a.flat && (a.ty != 1 || a.tz != 1)))
        return cudaErrorInvalidConfiguration;
    dim3 block(a.tx, a.ty, 1);
    const unsigned gx = unsigned(a.grid > 0 ? a.grid : a.ntiles);
    if (gx == 0) return cudaSuccess;
    const dim3 grid(gx, unsigned(a.tz), 1);
    if (a.minb == 4)
        launch_sweep2_minb<ST, 4>(a, grid, block, s);
    else
        launch_sweep2_minb<ST, 3>(a, grid, block, s);
    return cudaGetLastError();
}

}  // namespace lbm
