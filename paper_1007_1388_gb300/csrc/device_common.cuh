// Device-side helpers shared by the kernels of liblbm.so: storage formats
// and the per-cell collision.  Not shared with the oracle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "collide.cuh"
#include "sweep_types.h"

namespace lbm {

// Storage formats (enum values of include/lbm.h): S is the stored element,
// T the arithmetic type.  F16S/BF16S store g = s * f~ (s a power of two), so
// the kernels work in scaled units and only the moments are rescaled.
template <int ST> struct Traits;
template <> struct Traits<0> {
    using S = float;
    using T = float;
    static __device__ __forceinline__ T ld(const S *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(S *p, T v) { *p = v; }
    static __device__ __forceinline__ T to_t(S v) { return v; }
    static __device__ __forceinline__ S from_t(T v) { return v; }
};
template <> struct Traits<1> {
    using S = __half;
    using T = float;
    static __device__ __forceinline__ T ld(const S *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(S *p, T v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ T to_t(S v) { return __half2float(v); }
    static __device__ __forceinline__ S from_t(T v) { return __float2half_rn(v); }
};
template <> struct Traits<2> {
    using S = __nv_bfloat16;
    using T = float;
    static __device__ __forceinline__ T ld(const S *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(S *p, T v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ T to_t(S v) { return __bfloat162float(v); }
    static __device__ __forceinline__ S from_t(T v) { return __float2bfloat16_rn(v); }
};
template <> struct Traits<3> {
    using S = double;
    using T = double;
    static __device__ __forceinline__ T ld(const S *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(S *p, T v) { *p = v; }
    static __device__ __forceinline__ T to_t(S v) { return v; }
    static __device__ __forceinline__ S from_t(T v) { return v; }
};

// kernel-parameter copies of the collision constants (a single instance)
// pb = 2 s (rho_b - rho0) of the pressure boundaries in the arithmetic type
template <typename T>
__device__ __forceinline__ T param_pb(const SweepArgs &a);
template <>
__device__ __forceinline__ float param_pb<float>(const SweepArgs &a)
{
    return a.pbf;
}
template <>
__device__ __forceinline__ double param_pb<double>(const SweepArgs &a)
{
    return a.pbd;
}

template <typename T>
__device__ __forceinline__ const CollideConsts<T> &param_consts(const SweepArgs &a);
template <>
__device__ __forceinline__ const CollideConsts<float> &param_consts<float>(const SweepArgs &a)
{
    return a.kf;
}
template <>
__device__ __forceinline__ const CollideConsts<double> &param_consts<double>(const SweepArgs &a)
{
    return a.kd;
}

// ------------------------------------------------- pressure boundaries
// Anti-bounce-back with the velocity correction, in scaled units: the value
// pulled along e_q from a pressure node is
//   g_q = w_q [pb + 9 s rho0 (e_q.u_b)^2 - 3 s rho0 u_b.u_b] - g*_opp(q)(x),
// pb = 2 s (rho_b - rho0): twice the even part of the equilibrium (Eq. (2))
// at (rho_b, u_b) minus the population that left x towards the node.  u_b is
// the velocity of cell x's last collision, read back from its stored
// populations: u_b = (sum_j e_j g*_j) ufac - uoff (the Guo half-force
// removed from the post-collision momentum).  Every kernel goes through
// these two functions, so all sweep variants round it identically.
template <typename T>
struct PresBC {
    T P, ux, uy, uz, c9;  // P = pb - 3 s rho0 u_b.u_b, c9 = 9 s rho0
};

// one term of the momentum sum, in the order every caller uses (q = 1..18)
template <typename T>
__device__ __forceinline__ void pres_acc(int q, T g, T &jx, T &jy, T &jz)
{
    if (ex(q) > 0) jx = vadd(jx, g);
    if (ex(q) < 0) jx = vsub(jx, g);
    if (ey(q) > 0) jy = vadd(jy, g);
    if (ey(q) < 0) jy = vsub(jy, g);
    if (ez(q) > 0) jz = vadd(jz, g);
    if (ez(q) < 0) jz = vsub(jz, g);
}

template <typename T>
__device__ __forceinline__ PresBC<T> pres_finish(T jx, T jy, T jz, T pb, T ufac, T uox, T uoy, T uoz, T c45,
                                                 T nc15)
{
    PresBC<T> r;
    r.ux = vfma(jx, ufac, -uox);
    r.uy = vfma(jy, ufac, -uoy);
    r.uz = vfma(jz, ufac, -uoz);
    const T usq = vfma(r.ux, r.ux, vfma(r.uy, r.uy, vmul(r.uz, r.uz)));
    r.P = vfma(vadd(nc15, nc15), usq, pb);
    r.c9 = vadd(c45, c45);
    return r;
}

// From the stored populations of cell c: g*_q at src[q G + c], or, with SWAP
// (the in-place scheme after its local step), at src[opp(q) G + c].
template <int ST, typename T, bool SWAP = false>
__device__ __forceinline__ PresBC<T> pres_setup(const typename Traits<ST>::S *src, int c, int G, T pb, T ufac,
                                                T uox, T uoy, T uoz, T c45, T nc15)
{
    using Tr = Traits<ST>;
    T jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        // the in-place scheme writes this array in the same launch: coherent loads there
        const typename Tr::S *p = src + ((SWAP ? opp(q) : q) * G + c);
        pres_acc(q, SWAP ? Tr::to_t(*p) : Tr::ld(p), jx, jy, jz);
    }
    return pres_finish(jx, jy, jz, pb, ufac, uox, uoy, uoz, c45, nc15);
}

// From post-collision values still in registers, rounded through the storage
// format exactly as a later load would see them.
template <int ST, typename T>
__device__ __forceinline__ PresBC<T> pres_setup_regs(const T (&f)[Q], T pb, T ufac, T uox, T uoy, T uoz, T c45,
                                                     T nc15)
{
    using Tr = Traits<ST>;
    T jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int q = 1; q < Q; ++q) pres_acc(q, Tr::to_t(Tr::from_t(f[q])), jx, jy, jz);
    return pres_finish(jx, jy, jz, pb, ufac, uox, uoy, uoz, c45, nc15);
}

// g_q from the returning population g*_opp(q)(x); q is a constant after
// the callers' loops are unrolled
template <typename T>
__device__ __forceinline__ T pres_pull(int q, const PresBC<T> &p, T g_opp)
{
    // e_q.u_b up to its sign (it enters squared): the first nonzero
    // component of e_q taken positive, so q and opp(q) round alike
    const int a = ex(q), b = ey(q), c = ez(q);
    const int sg = a != 0 ? a : (b != 0 ? b : c);
    T eu;
    if (a != 0 && b != 0)
        eu = b * sg > 0 ? vadd(p.ux, p.uy) : vsub(p.ux, p.uy);
    else if (a != 0 && c != 0)
        eu = c * sg > 0 ? vadd(p.ux, p.uz) : vsub(p.ux, p.uz);
    else if (b != 0 && c != 0)
        eu = c * sg > 0 ? vadd(p.uy, p.uz) : vsub(p.uy, p.uz);
    else
        eu = a != 0 ? p.ux : (b != 0 ? p.uy : p.uz);
    return vsub(vmul(T(wq(q)), vfma(vmul(p.c9, eu), eu, p.P)), g_opp);
}

// ------------------------------------------------------- curved walls
// Linear interpolated bounce-back (Bouzidi, Firdaouss and Lallemand, 2001) on
// the pulled values f of a near-wall cell whose link mask has L_CURVED: the
// pull of direction p from a resting wall node at distance q along -e_p
// (table row `row`, q = 1/2 elsewhere) already holds the half-way value
// S_opp(p)(x); it becomes
//   q <  1/2: 2q S_opp(p)(x) + (1 - 2q) f_opp(p)   (f_opp(p) = S_opp(p)(x + e_p),
//             the pull from the fluid neighbour beyond; half-way if x + e_p is
//             not fluid)
//   q >= 1/2: S_opp(p)(x) / (2q) + (1 - 1/(2q)) S_p(x)
// Only wall pulls change, and f_opp(p) of the first case is a plain pull, so
// the order of the directions does not matter.  `srcp` reads S_p(x).
template <typename T, typename LoadOwn>
__device__ __forceinline__ void curved_links(T (&f)[Q], uint32_t lm, const T *row, LoadOwn srcp)
{
#pragma unroll
    for (int p = 1; p < Q; ++p) {
        if (!((lm >> p) & 1u)) continue;
        const T q = row[p - 1];
        if (q == T(0.5)) continue;
        const T bb = f[p];
        if (q < T(0.5)) {
            if ((lm >> opp(p)) & 1u) continue;
            const T q2 = vadd(q, q);
            f[p] = vfma(q2, bb, vmul(vsub(T(1), q2), f[opp(p)]));
        } else {
            const T h = T(1) / vadd(q, q);
            f[p] = vfma(h, bb, vmul(vsub(T(1), h), srcp(p)));
        }
    }
}

// the setup from the Patch's collision constants: kernel parameters for a
// single instance (UNIF), else the instance's table entry
template <int ST, bool UNIF, typename T, bool SWAP = false>
__device__ __forceinline__ PresBC<T> pres_cell(const CollideConsts<T> &kp, const CollideConsts<T> *kg, T pb,
                                               const typename Traits<ST>::S *src, int c, int G)
{
    if (UNIF)
        return pres_setup<ST, T, SWAP>(src, c, G, pb, kp.ufac, kp.uoff[0], kp.uoff[1], kp.uoff[2], kp.c45,
                                       kp.nc15);
    return pres_setup<ST, T, SWAP>(src, c, G, pb, __ldg(&kg->ufac), __ldg(&kg->uoff[0]), __ldg(&kg->uoff[1]),
                                   __ldg(&kg->uoff[2]), __ldg(&kg->c45), __ldg(&kg->nc15));
}

}  // namespace lbm
