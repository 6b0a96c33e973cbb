// TMA-staged D3Q19 sweep for Patches whose Blocks all have nx = TX cells
// (TX = 32, 64 or 128).
//
// The register sweep is latency-bound: every pulled PDF in flight holds a
// register, so the register file caps the bytes in flight per SM.  Here one
// producer warp streams, per z slice of a TY-row strip of a Block, 19 boxes
// (one per direction, shifted by -e_q) with cp.async.bulk.tensor into a ring
// of shared-memory stages, plus the x-halo columns from the neighbouring
// Blocks (direct reads across x faces, as in the register sweep) and the flag
// row; four consumer warps take two neighbouring cells per thread, read them
// from shared memory, apply bounce-back, collide both at once with packed
// FP32x2 arithmetic (collide.cuh; same rounding as the one-cell sweep) and
// store them with 64-bit coalesced global stores.
// Stages are handed over with mbarriers (full: transaction bytes landed;
// empty: all consumer warps have read the stage).  Every wait is bounded by
// a clock limit; a wait that expires writes an error word and the CTA leaves
// after waiting (again bounded) for its own copies in flight.
#pragma once

#include "device_common.cuh"
#include "lbm_internal.h"

namespace lbm {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of the given parity; false once `limit` SM clock
// cycles have passed without it completing.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            int c3, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

// Shared-memory layout of one stage: the 19 direction boxes (e_x = 0:
// TX x TY elements; e_x = +-1: (TX + A) x TY), 10 x-halo boxes (A x TY;
// slots 0..4 for the e_x = +1 directions 1,7,9,11,13 from the -x neighbour,
// 5..9 for e_x = -1 directions 2,8,10,12,14 from the +x neighbour) and the
// flag box (TX x TY bytes), each on a 128-byte boundary.
template <int ST, int TX>
struct TmaLayout {
    using S = typename Traits<ST>::S;
    static constexpr int E = int(sizeof(S));
    static constexpr int A = 16 / E;
    static constexpr int TY = 256 / TX;
    static constexpr int NCT = TX / 2 * TY;  // consumer threads (two cells each)
    static constexpr int NCW = NCT / 32;     // consumer warps
    static constexpr int THREADS = NCT + 32;
    static constexpr int BOXA = TX * TY * E;
    static constexpr int BOXB = (TX + A) * TY * E;
    static constexpr int HALO = A * TY * E;
    static constexpr int FLAG = TX * TY;
    __host__ __device__ static constexpr int r128(int v) { return (v + 127) / 128 * 128; }
    static constexpr int RA = r128(BOXA), RB = r128(BOXB), RH = r128(HALO), RF = r128(FLAG);
    __host__ __device__ static constexpr int box_off(int q)
    {
        int o = 0;
        for (int k = 0; k < q; ++k) o += ex(k) == 0 ? RA : RB;
        return o;
    }
    __host__ __device__ static constexpr int halo_slot(int q)
    {
        int k = 0;
        for (int j = 1; j < q; ++j)
            if (ex(j) == ex(q)) ++k;
        return ex(q) > 0 ? k : 5 + k;
    }
    static constexpr int HALO0 = box_off(Q);
    static constexpr int FLAGS = HALO0 + 10 * RH;
    static constexpr int STAGE = FLAGS + RF;
    static constexpr int STAGES = ST == 0 ? 3 : 5;
    static constexpr int SMEM = STAGES * STAGE + 2 * STAGES * 8 + 128;
    static constexpr int MINB = 3;  // resident CTAs the register budget allows
    static constexpr uint32_t BYTES_CORE = 9 * BOXA + 10 * BOXB + FLAG;
};

// Two neighbouring cells (x, x+1) of direction q from a staged box.
template <int ST, int TX, int q>
__device__ __forceinline__ F2 load_pair(const unsigned char *st, int ty, int x, bool hm, bool hp)
{
    using Ly = TmaLayout<ST, TX>;
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    constexpr int A = Ly::A;
    const S *box = reinterpret_cast<const S *>(st + Ly::box_off(q));
    float lo, hi;
    if (ex(q) == 0) {
        const S *p = box + ty * TX + x;  // even x: 4- or 8-byte aligned pair
        if (ST == 0) {
            const float2 v = *reinterpret_cast<const float2 *>(p);
            lo = v.x;
            hi = v.y;
        } else if (ST == 1) {
            const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(p));
            lo = v.x;
            hi = v.y;
        } else {
            const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
            lo = v.x;
            hi = v.y;
        }
    } else if (ex(q) > 0) {
        const S *p = box + ty * (TX + A) + x - 1 + A;
        lo = Tr::to_t(p[0]);
        hi = Tr::to_t(p[1]);
        if (x == 0 && hm)
            lo = Tr::to_t(reinterpret_cast<const S *>(st + Ly::HALO0 + Ly::halo_slot(q) * Ly::RH)[ty * A + A - 1]);
    } else {
        const S *p = box + ty * (TX + A) + x + 1;
        lo = Tr::to_t(p[0]);
        hi = Tr::to_t(p[1]);
        if (x == TX - 2 && hp)
            hi = Tr::to_t(reinterpret_cast<const S *>(st + Ly::HALO0 + Ly::halo_slot(q) * Ly::RH)[ty * A]);
    }
    return f2_pack(lo, hi);
}

template <int ST>
__device__ __forceinline__ void store_pair(typename Traits<ST>::S *p, F2 v, bool st_lo, bool st_hi)
{
    using Tr = Traits<ST>;
    float lo, hi;
    f2_unpack(v, lo, hi);
    if (st_lo && st_hi) {
        if (ST == 0)
            *reinterpret_cast<unsigned long long *>(p) = v.r;
        else if (ST == 1)
            *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(lo, hi);
        else
            *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(lo, hi);
    } else {
        if (st_lo) Tr::st(p, lo);
        if (st_hi) Tr::st(p + 1, hi);
    }
}

template <int q, int ST, int TX>
__device__ __forceinline__ void load_all(F2 (&f)[Q], const unsigned char *st, int ty, int x, bool hm,
                                         bool hp)
{
    f[q] = load_pair<ST, TX, q>(st, ty, x, hm, hp);
    if constexpr (q + 1 < Q) load_all<q + 1, ST, TX>(f, st, ty, x, hm, hp);
}

template <int ST, int COLL, bool FORCE, int TX, bool PRES>
__global__ void __launch_bounds__(TmaLayout<ST, TX>::THREADS, TmaLayout<ST, TX>::MINB)
    sweep_tma_kernel(const __grid_constant__ TmaSweepArgs ta, const __grid_constant__ TmaMaps maps)
{
    using Ly = TmaLayout<ST, TX>;
    using Tr = Traits<ST>;
    using S = typename Tr::S;
    constexpr int TY = Ly::TY, A = Ly::A, STAGES = Ly::STAGES;
    constexpr int NCW = Ly::NCW;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * Ly::STAGE);
    uint64_t *empty = full + STAGES;

    const int tid = int(threadIdx.x);
    const int warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        mbar_fence_init();
    }
    __syncthreads();

    const SweepArgs &a = ta.a;
    const long long lim = ta.wait_cycles;
    const int per_blk = ta.ngy * ta.nzc;

    if (warp == NCW) {
        // ------------------------------------------------------ producer
        const CUtensorMap *ma = &maps.box_a[ta.parity];
        const CUtensorMap *mb = &maps.box_b[ta.parity];
        const CUtensorMap *mh = &maps.halo[ta.parity];
        const CUtensorMap *mf = &maps.flags;
        int s = 0;
        uint32_t ph = 0;
        long long iter = 0;
        // stages whose copies may still be in flight, for the exit drain
        bool pending[STAGES];
        uint32_t pend_ph[STAGES];
        for (int k = 0; k < STAGES; ++k) pending[k] = false;
        bool ok = true;
        for (long long it = blockIdx.x; it < ta.nitems && ok; it += gridDim.x) {
            const int blk = int(it / per_blk);
            const int rem = int(it - (long long)blk * per_blk);
            const int zc = rem / ta.ngy, yg = rem - zc * ta.ngy;
            const BlockGeom &b = a.blocks[blk];
            const int y0 = yg * TY;
            const int z0 = zc * ta.zchunk, z1 = min(z0 + ta.zchunk, ta.nz);
            const int hm = b.xm_block, hp = b.xp_block;
            const uint32_t bytes =
                Ly::BYTES_CORE + (hm >= 0 ? 5u * Ly::HALO : 0u) + (hp >= 0 ? 5u * Ly::HALO : 0u);
            for (int z = z0; z < z1; ++z) {
                if (!mbar_wait(&empty[s], ph ^ 1u, lim)) {
                    if (lane == 0) atomicCAS(ta.err, 0, 2);
                    ok = false;
                    break;
                }
                unsigned char *st = smem + s * Ly::STAGE;
                if (lane == 0) mbar_arrive_expect_tx(&full[s], bytes);
                __syncwarp();
                const bool drop = iter == ta.drop_stage;
                if (!drop) {
                    if (lane < Q) {
                        const int q = lane;
                        const int exq = ex(q);
                        // e_x = +1 boxes start A cells left of the row (those
                        // read as zeros: lane 0 takes the neighbour's halo)
                        const int xs = exq > 0 ? -A : 0;
                        tma_load_4d(st + Ly::box_off(q), exq == 0 ? ma : mb, xs, y0 + 1 - ey(q),
                                    z + 1 - ez(q), blk * Q + q, &full[s]);
                    } else if (lane < Q + 10) {
                        // halo slot k: directions 1,7,9,11,13 (k < 5) / 2,8,10,12,14
                        const int k = lane - Q;
                        const int qq = k < 5 ? (k == 0 ? 1 : 5 + 2 * k) : (k == 5 ? 2 : 6 + 2 * (k - 5));
                        const int nbk = k < 5 ? hm : hp;
                        if (nbk >= 0)
                            tma_load_4d(st + Ly::HALO0 + k * Ly::RH, mh, k < 5 ? ta.nx - A : 0,
                                        y0 + 1 - ey(qq), z + 1 - ez(qq), nbk * Q + qq, &full[s]);
                    } else if (lane == Q + 10) {
                        tma_load_4d(st + Ly::FLAGS, mf, OXF, y0 + 1, z + 1, blk, &full[s]);
                    }
                }
                pending[s] = !drop;
                pend_ph[s] = ph;
                ++iter;
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
        // exit: every stage with copies issued must have landed before the
        // CTA's shared memory goes away (bounded wait)
        for (int k = 0; k < STAGES; ++k)
            if (pending[k] && !mbar_wait(&full[k], pend_ph[k], lim) && lane == 0) atomicCAS(ta.err, 0, 3);
        return;
    }

    // ------------------------------------------------------------ consumers
    const CollideConsts<float> *__restrict__ consts = static_cast<const CollideConsts<float> *>(a.consts);
    const int x = 2 * (tid % (TX / 2)), ty = tid / (TX / 2);
    const int px = ta.px, pxy = ta.px * ta.py;
    const int pxf = ta.pxf, pxyf = ta.pxf * ta.py;
    int s = 0;
    uint32_t ph = 0;
    for (long long it = blockIdx.x; it < ta.nitems; it += gridDim.x) {
        const int blk = int(it / per_blk);
        const int rem = int(it - (long long)blk * per_blk);
        const int zc = rem / ta.ngy, yg = rem - zc * ta.ngy;
        const BlockGeom &b = a.blocks[blk];
        const int y = yg * TY + ty;
        const int z0 = zc * ta.zchunk, z1 = min(z0 + ta.zchunk, ta.nz);
        const bool hm = b.xm_block >= 0, hp = b.xp_block >= 0;
        const int G = int(b.G);
        const CollKRef<float> K{ta.a.kf};  // one instance: constants are kernel parameters
        const S *__restrict__ src = static_cast<const S *>(a.src) + b.pdf_base;
        S *__restrict__ dst = static_cast<S *>(a.dst) + b.pdf_base;
        const uint8_t *__restrict__ fl = a.flags + b.cell_base;
        for (int z = z0; z < z1; ++z) {
            if (!mbar_wait(&full[s], ph, lim)) {
                if (lane == 0) atomicCAS(ta.err, 0, 1);
                return;
            }
            const unsigned char *st = smem + s * Ly::STAGE;
            const uint8_t fl0 = st[Ly::FLAGS + ty * TX + x], fl1 = st[Ly::FLAGS + ty * TX + x + 1];
            F2 f[Q];
            load_all<0, ST, TX>(f, st, ty, x, hm, hp);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (++s == STAGES) {
                s = 0;
                ph ^= 1u;
            }
            const bool solid0 = fl0 & F_KIND, solid1 = fl1 & F_KIND;
            if (solid0 && solid1) continue;  // solid cells are not updated
            const int c = (z + 1) * pxy + (y + 1) * px + x;
            if ((fl0 | fl1) & F_NEAR) {
                // half-way bounce-back, cell by cell, where the source is a wall or solid
                const int cf = (z + 1) * pxyf + (y + 1) * pxf + x + OXF;
                PresBC<float> pbc[2] = {};
                if (PRES) {
#pragma unroll
                    for (int k = 0; k < 2; ++k)
                        if (((k ? fl1 : fl0) & F_NEAR) && (__ldg(a.links + b.cell_base + cf + k) & L_PRESSURE))
                            pbc[k] = pres_cell<ST, true, float>(a.kf, nullptr, a.pbf, src, c + k, G);
                }
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    float v[2];
                    f2_unpack(f[q], v[0], v[1]);
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const uint8_t own = k ? fl1 : fl0;
                        if (!(own & F_NEAR)) continue;
                        const uint8_t nf = fl[cf + k - (ex(q) + ey(q) * pxf + ez(q) * pxyf)];
                        if (nf & F_KIND) {
                            float w = Tr::ld(src + (opp(q) * G + c + k));
                            if ((nf & F_KIND) == F_MOVING)
                                w = vadd(w, ta.a.kf.bbw[q]);
                            else if (PRES && (nf & F_KIND) == F_PRESSURE)
                                w = pres_pull(q, pbc[k], w);
                            v[k] = w;
                        }
                    }
                    f[q] = f2_pack(v[0], v[1]);
                }
            }
            collide_v<COLL, FORCE>(f, K);
#pragma unroll
            for (int q = 0; q < Q; ++q) store_pair<ST>(dst + (q * G + c), f[q], !solid0, !solid1);
        }
    }
}

template <int ST, int COLL, bool FORCE, int TX, bool PRES>
cudaError_t launch_tma_inst(const TmaSweepArgs &ta, const TmaMaps &maps, int grid, cudaStream_t s)
{
    constexpr int smem = TmaLayout<ST, TX>::SMEM;
    auto kern = sweep_tma_kernel<ST, COLL, FORCE, TX, PRES>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    kern<<<grid, TmaLayout<ST, TX>::THREADS, smem, s>>>(ta, maps);
    return cudaGetLastError();
}

template <int ST, int COLL, bool FORCE, int TX, bool PRES>
cudaError_t occupancy_tma_inst(int *n)
{
    constexpr int smem = TmaLayout<ST, TX>::SMEM;
    auto kern = sweep_tma_kernel<ST, COLL, FORCE, TX, PRES>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, TmaLayout<ST, TX>::THREADS, smem);
}

template <int ST, int COLL, bool FORCE, int TX, bool PRES>
cudaError_t tma_inst(const TmaSweepArgs &ta, const TmaMaps &maps, int grid, cudaStream_t s, int *occ)
{
    return occ ? occupancy_tma_inst<ST, COLL, FORCE, TX, PRES>(occ)
               : launch_tma_inst<ST, COLL, FORCE, TX, PRES>(ta, maps, grid, s);
}

// pressure boundaries are a separate instantiation: their near-wall setup
// would otherwise cost every TMA sweep registers
template <int ST, int TX, bool PRES>
cudaError_t tma_dispatch_pres(const TmaSweepArgs &ta, const TmaMaps &maps, int grid, cudaStream_t s, int *occ)
{
    if (ta.a.collision == 0)
        return ta.a.forced ? tma_inst<ST, 0, true, TX, PRES>(ta, maps, grid, s, occ)
                           : tma_inst<ST, 0, false, TX, PRES>(ta, maps, grid, s, occ);
    return ta.a.forced ? tma_inst<ST, 1, true, TX, PRES>(ta, maps, grid, s, occ)
                       : tma_inst<ST, 1, false, TX, PRES>(ta, maps, grid, s, occ);
}

template <int ST, int TX>
cudaError_t tma_dispatch(const TmaSweepArgs &ta, const TmaMaps &maps, int grid, cudaStream_t s, int *occ)
{
    return (ta.a.pres & 1) ? tma_dispatch_pres<ST, TX, true>(ta, maps, grid, s, occ)
                     : tma_dispatch_pres<ST, TX, false>(ta, maps, grid, s, occ);
}

template <int ST>
cudaError_t launch_sweep_tma_st(const TmaSweepArgs &ta, const TmaMaps &maps, int grid, cudaStream_t s,
                                int *occ)
{
    if (ta.nx == 32) return tma_dispatch<ST, 32>(ta, maps, grid, s, occ);
    if (ta.nx == 64) return tma_dispatch<ST, 64>(ta, maps, grid, s, occ);
    if (ta.nx == 128) return tma_dispatch<ST, 128>(ta, maps, grid, s, occ);
    return cudaErrorNotSupported;
}

}  // namespace lbm
