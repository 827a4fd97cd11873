// device_util.cuh -- small device helpers shared by the 2D kernel translation units.
#pragma once

#include <cuda_runtime.h>

namespace iga2l {

// two-lane values: float2 uses Blackwell's packed FP32 FMA (one instruction, each half
// rounded as a scalar fmaf), double2 two scalar FMAs
template <typename T>
struct Vec2;
template <>
struct Vec2<float> { using type = float2; };
template <>
struct Vec2<double> { using type = double2; };

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <typename T2>
__device__ __forceinline__ T2 splat2(decltype(T2::x) v) { T2 r; r.x = v; r.y = v; return r; }

// Row e of an FP64 block inverse, held as the FP32 pair hi + lo, times the FP32 block
// residual r, by Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J.
// Sci. Comput. 26(6), 2005): every product split exactly into p + ep (TwoProduct by FMA),
// every running sum into t + es (TwoSum), the error terms gathered in c; the result is as
// accurate as the sum computed in about twice the FP32 precision and then rounded once.
// Two interleaved chains (even and odd f) halve the dependent adds.  Explicit _rn
// intrinsics keep the compiler from contracting the error-free transformations.
template <int SS>
__device__ __forceinline__ float dot2_row(const float *__restrict__ hi, const float *__restrict__ lo,
                                          const float *rv)
{
    float s0 = 0.f, s1 = 0.f, c0 = 0.f, c1 = 0.f;
#pragma unroll
    for (int f = 0; f < SS; ++f) {
        float &s = (f & 1) ? s1 : s0;
        float &c = (f & 1) ? c1 : c0;
        const float a = __ldg(&hi[f]), r = rv[f];
        const float p = __fmul_rn(a, r);
        const float ep = __fmaf_rn(a, r, -p);                  // a r = p + ep
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));   // s + p = t + es
        s = t;
        c = __fmaf_rn(__ldg(&lo[f]), r, __fadd_rn(c, __fadd_rn(ep, es)));
    }
    const float t = __fadd_rn(s0, s1);
    const float z = __fsub_rn(t, s0);
    const float e = __fadd_rn(__fsub_rn(s0, __fsub_rn(t, z)), __fsub_rn(s1, z));   // s0 + s1 = t + e
    return __fadd_rn(t, __fadd_rn(e, __fadd_rn(c0, c1)));
}

}  // namespace iga2l
