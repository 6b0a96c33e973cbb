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

}  // namespace lbm
