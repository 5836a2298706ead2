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

// Forward DFT X[k] = sum_n x[n] exp(-j 2 pi k n / N) of NA length-N sequences (N a power of
// two) side by side in shared memory, natural order in and out, in the self-sorting
// (Stockham) form: radix-4 stages, and one radix-2 stage when log2 N is odd.  A stage of
// radix R combines the R length-p transforms at src[i + r N / R] (r < R), each twiddled by
// exp(-j 2 pi r k / (R p)) (k = i mod p), into dst[R i - (R - 1) k + q p] (q < R); the two
// buffers of a sequence alternate as source and destination, and on return src[a] points to
// its transform.  tw holds the twiddles by span, tw[h + m] = exp(-j pi m / h) for m < h
// (h = 1, 2, ..., N / 2), so a stage's twiddles are consecutive.  Every thread of the block
// calls it; it begins and ends with __syncthreads().
__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <int NA>
__device__ void fft_stockham(float2* (&src)[NA], float2* (&dst)[NA], int N, const float2* tw)
{
    for (int p = 1; p < N;) {
        __syncthreads();
        if (4 * p <= N) {
            for (int i = threadIdx.x; i < N / 4; i += blockDim.x) {
                const int k = i & (p - 1), j = 4 * i - 3 * k;
                const float2 w1 = tw[2 * p + k], w2 = tw[2 * p + 2 * k];
                float2 w3 = tw[3 * k < 2 * p ? 2 * p + 3 * k : 3 * k];   // exp(-j pi 3k / 2p)
                if (3 * k >= 2 * p) w3 = make_float2(-w3.x, -w3.y);
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const float2 b0 = src[a][i];
                    const float2 b1 = cmulf(src[a][i + N / 4], w1);
                    const float2 b2 = cmulf(src[a][i + N / 2], w2);
                    const float2 b3 = cmulf(src[a][i + 3 * (N / 4)], w3);
                    const float2 s02 = make_float2(b0.x + b2.x, b0.y + b2.y);
                    const float2 d02 = make_float2(b0.x - b2.x, b0.y - b2.y);
                    const float2 s13 = make_float2(b1.x + b3.x, b1.y + b3.y);
                    const float2 d13 = make_float2(b1.x - b3.x, b1.y - b3.y);
                    dst[a][j] = make_float2(s02.x + s13.x, s02.y + s13.y);
                    dst[a][j + p] = make_float2(d02.x + d13.y, d02.y - d13.x);        // d02 - j d13
                    dst[a][j + 2 * p] = make_float2(s02.x - s13.x, s02.y - s13.y);
                    dst[a][j + 3 * p] = make_float2(d02.x - d13.y, d02.y + d13.x);    // d02 + j d13
                }
            }
            p *= 4;
        } else {
            for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
                const int k = i & (p - 1), j = 2 * i - k;
                const float2 w = tw[p + k];
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const float2 u = src[a][i];
                    const float2 q = cmulf(src[a][i + N / 2], w);
                    dst[a][j] = make_float2(u.x + q.x, u.y + q.y);
                    dst[a][j + p] = make_float2(u.x - q.x, u.y - q.y);
                }
            }
            p *= 2;
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            float2* t = src[a];
            src[a] = dst[a];
            dst[a] = t;
        }
    }
    __syncthreads();
}

}  // namespace cyc
