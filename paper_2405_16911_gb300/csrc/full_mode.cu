// full_mode.cu -- the estimator on a uniform cycle-frequency grid a_k = -1/2 + k/A (the
// paper's Full mode, Sec. 4: every cycle frequency of [-1/2, 1/2) at resolution 1/A).
//
// For a_k on that grid the phase term depends on the absolute sample index n only through
// n mod A (A even):  exp(-j 2 pi a_k n) = (-1)^n exp(-j 2 pi k n / A), and (-1)^n = (-1)^r
// for r = n mod A.  So
//     sum_n P_c(n) exp(-j 2 pi a_k n) = sum_{r<A} (-1)^r F_c[r] exp(-j 2 pi k r / A),
//     F_c[r] = sum_{n = r mod A} P_c(n),
// an A-point DFT of the lag products folded modulo A.  A push only folds (O(samples x
// columns) work, bound by memory traffic instead of the O(samples x columns x A) projection);
// the DFT runs when the estimate is read.  F lives in the stream's sums array as
// float-float pairs (re hi, re lo, im hi, im lo: 16 bytes like a double2, about 48
// significant bits), [ncols][A] (a warp's residues are neighbours in memory for the fold
// and for the read), so reset, save and load work unchanged; the fold does no FP64
// arithmetic (this GPU's FP64 rate is a small fraction of its FP32 rate) and the read
// converts to FP64 before its FP64 DFT.
#include "cyc_device.cuh"
#include "cyc_impl.h"

namespace cyc {
namespace {

constexpr int FOLD_T = 256, FOLD_R = FOLD_T / 2;       // 128 residues x 2 halves of the terms

// Thread (r, h, l): the columns of lag l (both forms when F = 2) gain the pass terms i with
// (base + i) mod A == r, the first half of them (h = 0) or the second (h = 1).  One pair of
// sample reads x[i + m], y[i + D] serves both forms; consecutive threads take consecutive
// residues, so a warp's reads are consecutive, and four terms are loaded ahead.  FP32 runs
// of at most 64 terms, each added once to a float-float total; the second half's totals
// join the first's through shared memory (a fixed order), which then updates the fold.
// Two threads per (residue, lag) halve each thread's chain of dependent load rounds.
__global__ void __launch_bounds__(FOLD_T) fold_kernel(const float2* __restrict__ x, const float2* __restrict__ y,
                                                      int D, int64_t nc, int A, int base_mod,
                                                      const int32_t* __restrict__ col_lag,
                                                      const int8_t* __restrict__ col_conj, int ncols, int nF,
                                                      float4* __restrict__ F)
{
    __shared__ float4 half2[2][FOLD_R];                   // the second half's CONV and CONJ totals
    const int rl = threadIdx.x % FOLD_R, h = threadIdx.x / FOLD_R;
    const int r = blockIdx.x * FOLD_R + rl;
    const int c0 = blockIdx.y * nF;
    const bool live = r < A;
    const int m = col_lag[c0];
    float4 old[2];
    if (live && h == 0)
        for (int f = 0; f < nF; ++f) old[f] = F[(size_t)(c0 + f) * A + r];
    int64_t i = r - base_mod;
    if (i < 0) i += A;
    const int64_t K = (nc + A - 1) / A;                   // terms per residue, at most
    const int64_t Kh = (K + 1) / 2;
    i += h * Kh * (int64_t)A;
    const int64_t iend = h == 0 ? (i + Kh * (int64_t)A < nc ? i + Kh * (int64_t)A : nc) : nc;
    float4 V = make_float4(0.f, 0.f, 0.f, 0.f), J = V;        // CONV and CONJ totals, float-float
    while (live && i < iend) {
        float sr = 0.f, si = 0.f, tr = 0.f, ti = 0.f;
        int q = 0;
        for (; q < 64 && i + 3 * (int64_t)A < iend; q += 4, i += 4 * (int64_t)A) {
            float2 xm[4], y0[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                xm[k] = __ldg(&x[i + k * (int64_t)A + m]);
                y0[k] = __ldg(&y[i + k * (int64_t)A + D]);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float a = xm[k].x * y0[k].x, b = xm[k].y * y0[k].y;
                const float c = xm[k].y * y0[k].x, d = xm[k].x * y0[k].y;
                sr += a + b;  si += c - d;                   // x[n+m] conj(y[n])
                tr += a - b;  ti += c + d;                   // x[n+m] y[n]
            }
        }
        for (; q < 64 && i < iend; ++q, i += A) {
            const float2 xm = __ldg(&x[i + m]), y0 = __ldg(&y[i + D]);
            const float a = xm.x * y0.x, b = xm.y * y0.y, c = xm.y * y0.x, d = xm.x * y0.y;
            sr += a + b;  si += c - d;
            tr += a - b;  ti += c + d;
        }
        ff_add(V.x, V.y, sr);
        ff_add(V.z, V.w, si);
        ff_add(J.x, J.y, tr);
        ff_add(J.z, J.w, ti);
    }
    if (h == 1) {
        half2[0][rl] = V;
        half2[1][rl] = J;
    }
    __syncthreads();
    if (h == 1 || !live) return;
    const float4 V2 = half2[0][rl], J2 = half2[1][rl];
    ff_add(V.x, V.y, V2.x);
    ff_add(V.x, V.y, V2.y);
    ff_add(V.z, V.w, V2.z);
    ff_add(V.z, V.w, V2.w);
    ff_add(J.x, J.y, J2.x);
    ff_add(J.x, J.y, J2.y);
    ff_add(J.z, J.w, J2.z);
    ff_add(J.z, J.w, J2.w);
    for (int f = 0; f < nF; ++f) {
        const float4 t = col_conj[c0 + f] ? J : V;
        float4 o = old[f];
        ff_add(o.x, o.y, t.x);
        ff_add(o.x, o.y, t.y);
        ff_add(o.z, o.w, t.z);
        ff_add(o.z, o.w, t.w);
        F[(size_t)(c0 + f) * A + r] = o;
    }
}

// Block c: out[f][k][l] = (1/N) sum_r (-1)^r F_c[r] exp(-j 2 pi k r / A) for column
// c = l F + f, by an in-place radix-2 FFT in shared memory (FP64).
__global__ void dft_read_kernel(const float4* __restrict__ F, int A, int logA, int ncols, int nF, int L,
                                double inv_n, double2* __restrict__ out)
{
    extern __shared__ double2 v[];
    double2* tw = v + A;                                               // exp(-j 2 pi j / A), j < A/2
    const int c = blockIdx.x;
    for (int j = threadIdx.x; j < A / 2; j += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)j / (double)A, &sn, &cs);
        tw[j] = make_double2(cs, sn);
    }
    for (int r = threadIdx.x; r < A; r += blockDim.x) {
        const float4 ff = F[(size_t)c * A + r];
        const double2 q = make_double2((double)ff.x + (double)ff.y, (double)ff.z + (double)ff.w);
        const double s = (r & 1) ? -1.0 : 1.0;
        const unsigned rev = __brev((unsigned)r) >> (32 - logA);       // bit-reversed position
        v[rev] = make_double2(s * q.x, s * q.y);
    }
    __syncthreads();
    for (int len = 2; len <= A; len <<= 1) {
        const int half = len >> 1;
        for (int t = threadIdx.x; t < A / 2; t += blockDim.x) {
            const int grp = t / half, j = t % half;
            const int i0 = grp * len + j, i1 = i0 + half;
            const double2 z = tw[j * (A / len)];                             // exp(-j 2 pi j / len)
            const double2 b = v[i1];
            const double2 w = make_double2(b.x * z.x - b.y * z.y, b.x * z.y + b.y * z.x);
            const double2 a = v[i0];
            v[i0] = make_double2(a.x + w.x, a.y + w.y);
            v[i1] = make_double2(a.x - w.x, a.y - w.y);
        }
        __syncthreads();
    }
    const int f = c % nF, l = c / nF;
    for (int k = threadIdx.x; k < A; k += blockDim.x)
        out[((size_t)f * A + k) * L + l] = make_double2(v[k].x * inv_n, v[k].y * inv_n);
}

}  // namespace

bool full_supported(int A) { return A >= 2 && A <= 4096 && (A & (A - 1)) == 0; }

cudaError_t full_fold(const ProjArgs& a, int A, double2* F, cudaStream_t st)
{
    if (a.nc <= 0) return cudaSuccess;
    const int base_mod = (int)(a.nbase & (uint64_t)(A - 1));
    // columns c = l nF + f: both forms of a lag share one thread (nF = columns per lag)
    const int nF = a.nforms > 0 ? a.nforms : 1;
    dim3 grid((A + FOLD_R - 1) / FOLD_R, a.ncols / nF);
    fold_kernel<<<grid, FOLD_T, 0, st>>>(a.x, a.y ? a.y : a.x, a.D, a.nc, A, base_mod, a.col_lag, a.col_conj,
                                         a.ncols, nF, reinterpret_cast<float4*>(F));
    return cudaGetLastError();
}

cudaError_t full_read(const double2* F, int A, int ncols, int nF, int L, double inv_n, double2* out, cudaStream_t st)
{
    int logA = 0;
    while ((1 << logA) < A) ++logA;
    const size_t smem = (size_t)A * 3 / 2 * sizeof(double2);
    static bool attr_set[64] = {false};                   // the attribute is per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(dft_read_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             4096 * 3 / 2 * 16);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dft_read_kernel<<<ncols, 256, smem, st>>>(reinterpret_cast<const float4*>(F), A, logA, ncols, nF, L, inv_n, out);
    return cudaGetLastError();
}

}  // namespace cyc
