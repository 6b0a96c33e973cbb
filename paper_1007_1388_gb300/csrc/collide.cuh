// The D3Q19 collision (Eq. (1) with the shifted equilibrium of Eq. (2), BGK or
// TRT, Guo forcing), written once over a "lane" type V with explicit
// arithmetic:
//   float  - one cell per thread, FP32, every operation rounded on its own
//            (__fadd_rn & co., so the compiler cannot contract differently);
//   F2     - two cells per thread in one 64-bit register pair, using the
//            packed FP32 instructions of sm_100+ (add/sub/mul/fma .f32x2);
//   double - one cell per thread, FP64 (the reference storage format).
// The float and F2 instantiations execute the same rounding sequence per
// cell, so the one-cell and two-cell sweeps give bitwise equal results.
//
// Algebra (scaled units g = s f~, see CollideConsts): with drho = sum g,
// u = (sum e g) ufac + uoff and A = drho - 1.5 rho0s u.u, the equilibrium of
// a direction pair (q, opp(q)) splits into an even part w B with
// B = A + 4.5 rho0s (e.u)^2, and an odd part w 3 rho0s (e.u).  The Guo source
// is folded in: omega (feq - g) + S = omega (feq + S/omega - g), which adds
// -3 a+ u.F to A, 9 a+ (e.u)(e.F) to B and 3 a- (e.F) to the odd part, with
// a+ = (1 - omega+/2)/omega+ and a- = (1 - omega-/2)/omega-.
//
// Every product that feeds an addition is an explicit fused multiply-add,
// with the relaxation rates folded into host-computed constants: the code
// generator fuses a packed multiply followed by a packed add into one FMA
// (a scalar __fmul_rn / __fadd_rn pair keeps two roundings), so a product
// left separate would round differently in the two lane types.  With no
// multiply-then-add pattern left there is nothing to fuse, and both lane
// types round identically.
#pragma once

#include <cuda_runtime.h>

#include "sweep_types.h"

namespace lbm {

// ------------------------------------------------------------ lane types
struct F2 {
    unsigned long long r;
};

__device__ __forceinline__ F2 f2_pack(float lo, float hi)
{
    F2 v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v.r) : "f"(lo), "f"(hi));
    return v;
}
__device__ __forceinline__ void f2_unpack(F2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v.r));
}

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }

__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ F2 vadd(F2 a, F2 b)
{
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 vsub(F2 a, F2 b)
{
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 vmul(F2 a, F2 b)
{
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c)
{
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return d;
}

// constant of the lane type: scalar, or the same value in both halves
template <typename V> struct Lane;
template <> struct Lane<float> {
    using S = float;
    static __device__ __forceinline__ float c(float v) { return v; }
};
template <> struct Lane<double> {
    using S = double;
    static __device__ __forceinline__ double c(double v) { return v; }
};
template <> struct Lane<F2> {
    using S = float;
    static __device__ __forceinline__ F2 c(float v) { return f2_pack(v, v); }
};


// Collision constants of an instance (see CollideConsts for their values),
// as the scalar type S of the lane: held in registers (CollK) or read from
// global memory at their point of use (CollKPtr, keeps them out of the
// register file of the one-cell sweep).  Index c: 0 axis, 1 diagonal pair.
template <typename S>
struct CollK {
    S zero, nc15, c45, ufac, uoff[3], k9F[3], nk3F[3], c0a, c0b;
    S obw[2], oc3[2], okF[2][3];
    S hwp, hwm, nwpw[2], nwmc3[2], nwmkF[2][3];
};

template <typename T>
struct CollKPtr {
    const CollideConsts<T> *__restrict__ p;
};

// Constants that are kernel parameters (one instance): read from the
// parameter (constant) bank at their point of use, no registers held.
template <typename T>
struct CollKRef {
    const CollideConsts<T> &p;
};

template <typename S, typename T>
__device__ __forceinline__ CollK<S> load_collk(const CollideConsts<T> *__restrict__ c)
{
    CollK<S> k;
    k.zero = S(__ldg(&c->zero));
    k.nc15 = S(__ldg(&c->nc15));
    k.c45 = S(__ldg(&c->c45));
    k.ufac = S(__ldg(&c->ufac));
    k.c0a = S(__ldg(&c->c0a));
    k.c0b = S(__ldg(&c->c0b));
    k.hwp = S(__ldg(&c->hwp));
    k.hwm = S(__ldg(&c->hwm));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        k.uoff[a] = S(__ldg(&c->uoff[a]));
        k.k9F[a] = S(__ldg(&c->k9F[a]));
        k.nk3F[a] = S(__ldg(&c->nk3F[a]));
    }
#pragma unroll
    for (int cl = 0; cl < 2; ++cl) {
        k.obw[cl] = S(__ldg(&c->obw[cl]));
        k.oc3[cl] = S(__ldg(&c->oc3[cl]));
        k.nwpw[cl] = S(__ldg(&c->nwpw[cl]));
        k.nwmc3[cl] = S(__ldg(&c->nwmc3[cl]));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            k.okF[cl][a] = S(__ldg(&c->okF[cl][a]));
            k.nwmkF[cl][a] = S(__ldg(&c->nwmkF[cl][a]));
        }
    }
    return k;
}

#define LBM_K0(name)                                                                                 \
    template <typename S>                                                                            \
    __device__ __forceinline__ S k_##name(const CollK<S> &k) { return k.name; }                      \
    template <typename T>                                                                            \
    __device__ __forceinline__ T k_##name(const CollKPtr<T> &k) { return __ldg(&k.p->name); }        \
    template <typename T>                                                                            \
    __device__ __forceinline__ T k_##name(const CollKRef<T> &k) { return k.p.name; }
#define LBM_K1(name)                                                                                 \
    template <typename S>                                                                            \
    __device__ __forceinline__ S k_##name(const CollK<S> &k, int i) { return k.name[i]; }            \
    template <typename T>                                                                            \
    __device__ __forceinline__ T k_##name(const CollKPtr<T> &k, int i) { return __ldg(&k.p->name[i]); } \
    template <typename T>                                                                            \
    __device__ __forceinline__ T k_##name(const CollKRef<T> &k, int i) { return k.p.name[i]; }
#define LBM_K2(name)                                                                                 \
    template <typename S>                                                                            \
    __device__ __forceinline__ S k_##name(const CollK<S> &k, int i, int j) { return k.name[i][j]; }  \
    template <typename T>                                                                            \
    __device__ __forceinline__ T k_##name(const CollKPtr<T> &k, int i, int j)                        \
    {                                                                                                \
        return __ldg(&k.p->name[i][j]);                                                              \
    }                                                                                                \
    template <typename T>                                                                            \
    __device__ __forceinline__ T k_##name(const CollKRef<T> &k, int i, int j) { return k.p.name[i][j]; }
LBM_K0(zero)
LBM_K0(nc15)
LBM_K0(c45)
LBM_K0(ufac)
LBM_K0(c0a)
LBM_K0(c0b)
LBM_K0(hwp)
LBM_K0(hwm)
LBM_K1(uoff)
LBM_K1(k9F)
LBM_K1(nk3F)
LBM_K1(obw)
LBM_K1(oc3)
LBM_K1(nwpw)
LBM_K1(nwmc3)
LBM_K2(okF)
LBM_K2(nwmkF)
#undef LBM_K0
#undef LBM_K1
#undef LBM_K2

// e.v for the representative (odd) direction q of a pair, from the three
// components: every e component is 0 or +-1, so this is 0 or 1 add/sub.
template <int q, typename V>
__device__ __forceinline__ V edot(V x, V y, V z)
{
    constexpr int a = ex(q), b = ey(q), c = ez(q);
    if (a != 0 && b != 0) return b > 0 ? vadd(x, y) : vsub(x, y);
    if (a != 0 && c != 0) return c > 0 ? vadd(x, z) : vsub(x, z);
    if (b != 0 && c != 0) return c > 0 ? vadd(y, z) : vsub(y, z);
    if (a != 0) return x;
    if (b != 0) return y;
    return z;
}

// One direction pair: q odd, its opposite q+1.
//   BGK: g'_q = (1 - w) g_q + omega w B + O,  g'_qb = (1 - w) g_qb + omega w B - O
//        with O = omega (odd part), omega = 1/tau;
//   TRT: dp = omega+ (g+ - w B), dm = omega- (g- - odd),
//        g'_q = g_q - dp - dm, g'_qb = g_qb - dp + dm.
template <int q, int COLL, bool FORCE, typename V, typename KT>
__device__ __forceinline__ void collide_pair(V (&f)[Q], const KT &K, V ux, V uy, V uz, V Ap)
{
    using L = Lane<V>;
    constexpr int cl = norm2(q) == 2 ? 1 : 0;
    const V eu = edot<q>(ux, uy, uz);
    const V t = FORCE ? vfma(L::c(k_c45(K)), eu, edot<q>(L::c(k_k9F(K, 0)), L::c(k_k9F(K, 1)), L::c(k_k9F(K, 2))))
                      : vmul(L::c(k_c45(K)), eu);
    const V B = vfma(t, eu, Ap);
    const V fa = f[q], fb = f[q + 1];
    if (COLL == 0) {
        const V oF = FORCE ? edot<q>(L::c(k_okF(K, cl, 0)), L::c(k_okF(K, cl, 1)), L::c(k_okF(K, cl, 2)))
                           : L::c(k_zero(K));
        const V O = vfma(L::c(k_oc3(K, cl)), eu, oF);
        const V nO = vsub(L::c(k_zero(K)), O);
        f[q] = vfma(L::c(k_obw(K, cl)), B, vfma(fa, L::c(k_c0b(K)), O));
        f[q + 1] = vfma(L::c(k_obw(K, cl)), B, vfma(fb, L::c(k_c0b(K)), nO));
    } else {
        const V dp = vfma(L::c(k_hwp(K)), vadd(fa, fb), vmul(L::c(k_nwpw(K, cl)), B));
        const V M = FORCE ? vfma(L::c(k_nwmc3(K, cl)), eu,
                                 edot<q>(L::c(k_nwmkF(K, cl, 0)), L::c(k_nwmkF(K, cl, 1)), L::c(k_nwmkF(K, cl, 2))))
                          : vmul(L::c(k_nwmc3(K, cl)), eu);
        const V dm = vfma(L::c(k_hwm(K)), vsub(fa, fb), M);
        f[q] = vsub(vsub(fa, dp), dm);
        f[q + 1] = vadd(vsub(fb, dp), dm);
    }
}

// Collides one cell (or two, for F2) in place: f holds the pulled,
// pre-collision PDFs in scaled units and receives the post-collision ones.
template <int COLL, bool FORCE, typename V, typename KT>
__device__ __forceinline__ void collide_v(V (&f)[Q], const KT &K)
{
    using L = Lane<V>;
    // moments, accumulated pair by pair (sum and difference of each pair are
    // used at once, so only the four accumulators stay live)
    V drho, jx, jy, jz;
    {
        const V s = vadd(f[1], f[2]), d = vsub(f[1], f[2]);  // (+1, 0, 0)
        drho = vadd(f[0], s);
        jx = d;
    }
    {
        const V s = vadd(f[3], f[4]), d = vsub(f[3], f[4]);  // (0, +1, 0)
        drho = vadd(drho, s);
        jy = d;
    }
    {
        const V s = vadd(f[5], f[6]), d = vsub(f[5], f[6]);  // (0, 0, +1)
        drho = vadd(drho, s);
        jz = d;
    }
    {
        const V s = vadd(f[7], f[8]), d = vsub(f[7], f[8]);  // (+1, +1, 0)
        drho = vadd(drho, s);
        jx = vadd(jx, d);
        jy = vadd(jy, d);
    }
    {
        const V s = vadd(f[9], f[10]), d = vsub(f[9], f[10]);  // (+1, -1, 0)
        drho = vadd(drho, s);
        jx = vadd(jx, d);
        jy = vsub(jy, d);
    }
    {
        const V s = vadd(f[11], f[12]), d = vsub(f[11], f[12]);  // (+1, 0, +1)
        drho = vadd(drho, s);
        jx = vadd(jx, d);
        jz = vadd(jz, d);
    }
    {
        const V s = vadd(f[13], f[14]), d = vsub(f[13], f[14]);  // (+1, 0, -1)
        drho = vadd(drho, s);
        jx = vadd(jx, d);
        jz = vsub(jz, d);
    }
    {
        const V s = vadd(f[15], f[16]), d = vsub(f[15], f[16]);  // (0, +1, +1)
        drho = vadd(drho, s);
        jy = vadd(jy, d);
        jz = vadd(jz, d);
    }
    {
        const V s = vadd(f[17], f[18]), d = vsub(f[17], f[18]);  // (0, +1, -1)
        drho = vadd(drho, s);
        jy = vadd(jy, d);
        jz = vsub(jz, d);
    }
    // u = j ufac + uoff (uoff = 0 without force; always an FMA, see above)
    const V ux = vfma(jx, L::c(k_ufac(K)), L::c(k_uoff(K, 0)));
    const V uy = vfma(jy, L::c(k_ufac(K)), L::c(k_uoff(K, 1)));
    const V uz = vfma(jz, L::c(k_ufac(K)), L::c(k_uoff(K, 2)));
    const V usq = vfma(ux, ux, vfma(uy, uy, vmul(uz, uz)));
    V Ap = vfma(L::c(k_nc15(K)), usq, drho);
    if (FORCE) {
        const V nuF = vfma(ux, L::c(k_nk3F(K, 0)), vfma(uy, L::c(k_nk3F(K, 1)), vmul(uz, L::c(k_nk3F(K, 2)))));
        Ap = vadd(Ap, nuF);
    }
    // rest direction, even part only: (1 - omega+) g0 + omega+ A/3
    f[0] = vfma(L::c(k_c0a(K)), Ap, vmul(f[0], L::c(k_c0b(K))));
    collide_pair<1, COLL, FORCE>(f, K, ux, uy, uz, Ap);
    collide_pair<3, COLL, FORCE>(f, K, ux, uy, uz, Ap);
    collide_pair<5, COLL, FORCE>(f, K, ux, uy, uz, Ap);
    collide_pair<7, COLL, FORCE>(f, K, ux, uy, uz, Ap);
    collide_pair<9, COLL, FORCE>(f, K, ux, uy, uz, Ap);
    collide_pair<11, COLL, FORCE>(f, K, ux, uy, uz, Ap);
    collide_pair<13, COLL, FORCE>(f, K, ux, uy, uz, Ap);
    collide_pair<15, COLL, FORCE>(f, K, ux, uy, uz, Ap);
    collide_pair<17, COLL, FORCE>(f, K, ux, uy, uz, Ap);
}

}  // namespace lbm
