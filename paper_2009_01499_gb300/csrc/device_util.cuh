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
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Row e of an FP64 block inverse, held as the FP32 pair hi + lo, times the FP32 block
// residual r, by Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J.
// Sci. Comput. 26(6), 2005): every product split exactly into p + ep (TwoProduct by FMA),
// every running sum into t + es (TwoSum), the error terms gathered in c; the result is as
// accurate as the sum computed in about twice the FP32 precision and then rounded once.
// Four interleaved chains (f mod 4) quarter the dependent adds.  Explicit _rn intrinsics
// keep the compiler from contracting the error-free transformations.
__device__ __forceinline__ void two_sum(float a, float b, float &t, float &e)
{
    t = __fadd_rn(a, b);
    const float z = __fsub_rn(t, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, z)), __fsub_rn(b, z));   // a + b = t + e
}

// (element f of the row at hi[f * STRIDE], lo[f * STRIDE])
template <int SS, int STRIDE = 1>
__device__ __forceinline__ float dot2_row(const float *__restrict__ hi, const float *__restrict__ lo,
                                          const float *rv)
{
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int f = 0; f < SS; ++f) {
        const int k = f & 3;
        const float a = __ldg(&hi[f * STRIDE]), r = rv[f];
        const float p = __fmul_rn(a, r);
        const float ep = __fmaf_rn(a, r, -p);                  // a r = p + ep
        float t, es;
        two_sum(s[k], p, t, es);                               // s + p = t + es
        s[k] = t;
        c[k] = __fmaf_rn(__ldg(&lo[f * STRIDE]), r, __fadd_rn(c[k], __fadd_rn(ep, es)));
    }
    float t01, e01, t23, e23, t, e;
    two_sum(s[0], s[1], t01, e01);
    two_sum(s[2], s[3], t23, e23);
    two_sum(t01, t23, t, e);
    const float cc = __fadd_rn(__fadd_rn(c[0], c[1]), __fadd_rn(c[2], c[3]));
    return __fadd_rn(t, __fadd_rn(e, __fadd_rn(__fadd_rn(e01, e23), cc)));
}

}  // namespace iga2l
