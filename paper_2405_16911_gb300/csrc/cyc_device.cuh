// cyc_device.cuh -- device helpers shared by the projection kernels of libcyc.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cyc {

// exp(-j 2 pi theta / 2^64) with theta = phi * n mod 2^64 (Sec. 2: the phase term
// exp(-j 2 pi a~ n) at normalised cycle frequency a~ = phi / 2^64).  The product wraps
// exactly in u64, so the phase stays exact for any n; only its top 32 bits are used
// (error <= 2^-32 cycles), reduced to [-1/2, 1/2) cycles before the FP32 sine/cosine.
__device__ __forceinline__ float2 phase_rot(uint64_t phi, uint64_t n)
{
    uint64_t th = phi * n;
    int32_t hi = (int32_t)(th >> 32);
    float f = (float)hi * 2.3283064365386963e-10f;          // 2^-32
    float s, c;
    __sincosf(6.283185307179586f * f, &s, &c);
    return make_float2(c, -s);
}

// Lag product of Eq. (ACF-def) (conj = false: x[n+m] conj(x[n])) or Eq. (CCF-def)
// (conj = true: x[n+m] x[n]).  xm = x[n+m], x0 = x[n].
__device__ __forceinline__ float2 lag_product(float2 xm, float2 x0, bool conj)
{
    float yi = conj ? x0.y : -x0.y;
    return make_float2(xm.x * x0.x - xm.y * yi, xm.x * yi + xm.y * x0.x);
}

// Float-float accumulator: a value held as hi + lo, two FP32 numbers (about 48 significant
// bits).  This GPU's FP64 rate is a small fraction of its FP32 rate, so sums updated per
// element and per step are kept as FP32 pairs and updated with error-free transformations
// (Knuth's TwoSum: s + e == a + b exactly for s = fl(a + b)); FP64 is used only where a
// value leaves in FP64.  (hi, lo) += v with a relative error of about 2^-46.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float v)
{
    const float s = hi + v;
    const float bv = s - hi;
    const float e = (hi - (s - bv)) + (v - bv);
    const float t = lo + e;
    const float s2 = s + t;
    const float bt = s2 - s;
    lo = (s - (s2 - bt)) + (t - bt);
    hi = s2;
}

}  // namespace cyc
