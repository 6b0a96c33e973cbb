// Device-side helpers shared by the kernels of liblbm.so: storage formats
// and the per-cell collision.  Not shared with the oracle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.h"

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

// The collision constants one thread keeps in registers (loaded once per tile
// from the instance's CollideConsts).
template <typename T>
struct Coll {
    T rho0s, ufac, uoff[3];
    T omega_p, omega_m, cp, cm;
    T Fs[3];
};

template <typename T>
__device__ __forceinline__ Coll<T> load_coll(const CollideConsts<T> *__restrict__ c)
{
    Coll<T> r;
    r.rho0s = __ldg(&c->rho0s);
    r.ufac = __ldg(&c->ufac);
    r.omega_p = __ldg(&c->omega_p);
    r.omega_m = __ldg(&c->omega_m);
    r.cp = __ldg(&c->cp);
    r.cm = __ldg(&c->cm);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r.uoff[a] = __ldg(&c->uoff[a]);
        r.Fs[a] = __ldg(&c->Fs[a]);
    }
    return r;
}

// Moments of the pre-collision cell f (scaled units).
template <typename T, bool FORCE>
__device__ __forceinline__ void moments(const T (&f)[Q], const Coll<T> &P, T &drho, T &ux,
                                        T &uy, T &uz)
{
    // Sums written out per axis; unrolled loops fold e_q into +/- adds.
    T d = f[0], jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        d += f[q];
        if (ex(q) > 0) jx += f[q];
        if (ex(q) < 0) jx -= f[q];
        if (ey(q) > 0) jy += f[q];
        if (ey(q) < 0) jy -= f[q];
        if (ez(q) > 0) jz += f[q];
        if (ez(q) < 0) jz -= f[q];
    }
    drho = d;
    if (FORCE) {
        ux = fma(jx, P.ufac, P.uoff[0]);
        uy = fma(jy, P.ufac, P.uoff[1]);
        uz = fma(jz, P.ufac, P.uoff[2]);
    } else {
        ux = jx * P.ufac;
        uy = jy * P.ufac;
        uz = jz * P.ufac;
    }
}

// BGK (COLL = 0) or TRT (COLL = 1) collision with optional Guo forcing,
// Eq. (1) with the shifted equilibrium of Eq. (2).  Works on direction
// pairs (q, opp(q)): the even part of feq is shared, the odd part flips.
template <typename T, int COLL, bool FORCE>
__device__ __forceinline__ void collide(T (&f)[Q], const Coll<T> &P)
{
    T drho, ux, uy, uz;
    moments<T, FORCE>(f, P, drho, ux, uy, uz);
    const T usq = ux * ux + uy * uy + uz * uz;
    const T A = drho - T(1.5) * P.rho0s * usq;  // w-free, e-free part of feq
    const T c45 = T(4.5) * P.rho0s;
    const T c3 = T(3) * P.rho0s;
    T uF = T(0);
    if (FORCE) uF = ux * P.Fs[0] + uy * P.Fs[1] + uz * P.Fs[2];
    const T wp = P.omega_p;
    const T wm = P.omega_m;

    // rest direction: even part only
    {
        const T w0 = T(1.0 / 3.0);
        T feq0 = w0 * A;
        T d0 = feq0 - f[0];
        f[0] = fma(wp, d0, f[0]);
        if (FORCE) f[0] = fma(P.cp * w0, T(-3) * uF, f[0]);
    }
#pragma unroll
    for (int q = 1; q < Q; q += 2) {
        const int qb = q + 1;  // opposite of odd q
        const T w = T(wq(q));
        const T eu = T(ex(q)) * ux + T(ey(q)) * uy + T(ez(q)) * uz;
        const T even = w * fma(c45 * eu, eu, A);
        const T odd = (w * c3) * eu;
        T se = T(0), so = T(0);
        if (FORCE) {
            const T eF = T(ex(q)) * P.Fs[0] + T(ey(q)) * P.Fs[1] + T(ez(q)) * P.Fs[2];
            se = (P.cp * w) * fma(T(9) * eu, eF, T(-3) * uF);
            so = (P.cm * w * T(3)) * eF;
        }
        if (COLL == 0) {
            const T fa = f[q], fb = f[qb];
            T na = fma(wp, (even + odd) - fa, fa);
            T nb = fma(wp, (even - odd) - fb, fb);
            if (FORCE) {
                na += se + so;
                nb += se - so;
            }
            f[q] = na;
            f[qb] = nb;
        } else {
            const T fa = f[q], fb = f[qb];
            const T dp = wp * (T(0.5) * (fa + fb) - even);
            const T dm = wm * (T(0.5) * (fa - fb) - odd);
            T na = fa - dp - dm;
            T nb = fb - dp + dm;
            if (FORCE) {
                na += se + so;
                nb += se - so;
            }
            f[q] = na;
            f[qb] = nb;
        }
    }
}

// Fused ghost-layer write (the communication step folded into the work step):
// a cell on a y or z face of its Block also stores each PDF that leaves the
// Block through that face into the ghost cell of the neighbour that pulls it
// in the next step (5 PDFs per face cell, 1 per yz-edge cell).
template <typename Tr, typename T>
__device__ __forceinline__ void push_ghosts(typename Tr::S *__restrict__ dst, const BlockGeom &b,
                                            int y, int z, int c, int G, const T (&f)[Q])
{
    const int m = b.push_mask;
    const bool ylo = y == 0, yhi = y == b.ny - 1, zlo = z == 0, zhi = z == b.nz - 1;
    if (!m || !(ylo || yhi || zlo || zhi)) return;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int o = q * G + c;
        if (ey(q) < 0 && ylo && (m & 1)) Tr::st(dst + b.push_off[0] + o, f[q]);
        if (ey(q) > 0 && yhi && (m & 2)) Tr::st(dst + b.push_off[1] + o, f[q]);
        if (ez(q) < 0 && zlo && (m & 4)) Tr::st(dst + b.push_off[2] + o, f[q]);
        if (ez(q) > 0 && zhi && (m & 8)) Tr::st(dst + b.push_off[3] + o, f[q]);
        if (ey(q) < 0 && ez(q) < 0 && ylo && zlo && (m & 16)) Tr::st(dst + b.push_off[4] + o, f[q]);
        if (ey(q) > 0 && ez(q) < 0 && yhi && zlo && (m & 32)) Tr::st(dst + b.push_off[5] + o, f[q]);
        if (ey(q) < 0 && ez(q) > 0 && ylo && zhi && (m & 64)) Tr::st(dst + b.push_off[6] + o, f[q]);
        if (ey(q) > 0 && ez(q) > 0 && yhi && zhi && (m & 128)) Tr::st(dst + b.push_off[7] + o, f[q]);
    }
}

}  // namespace lbm
