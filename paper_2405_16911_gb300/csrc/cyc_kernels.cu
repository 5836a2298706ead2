// cyc_kernels.cu -- FP64 running-sum update and normalised read-out of libcyc.
#include "cyc_impl.h"

namespace cyc {
namespace {

// sums[e] += sum_s part[s][e], e = (u, c) flattened.  The splits are added in FP32 (a few
// dozen terms, each already a sum over thousands of samples) and the total once in FP64:
// FP64 arithmetic is scarce on this GPU, so it is kept to one add per value and push.
// Each thread folds two neighbouring elements with one 16-byte load per split and keeps
// eight loads in flight.
__global__ void reduce_partials_kernel(const float2* __restrict__ part, int nsplit, int n_uc,
                                       double2* __restrict__ sums)
{
    int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= n_uc) return;
    if (e + 1 < n_uc && (n_uc & 1) == 0) {
        const float4* p = reinterpret_cast<const float4*>(part + e);
        const size_t stride = (size_t)n_uc / 2;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        int s = 0;
        for (; s + 8 <= nsplit; s += 8) {
            float4 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldg(p + (size_t)(s + k) * stride);
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                acc.x += v[k].x + v[k + 1].x;
                acc.y += v[k].y + v[k + 1].y;
                acc.z += v[k].z + v[k + 1].z;
                acc.w += v[k].w + v[k + 1].w;
            }
        }
        for (; s < nsplit; ++s) {
            float4 v = __ldg(p + (size_t)s * stride);
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
        double2 o0 = sums[e], o1 = sums[e + 1];
        sums[e] = make_double2(o0.x + (double)acc.x, o0.y + (double)acc.y);
        sums[e + 1] = make_double2(o1.x + (double)acc.z, o1.y + (double)acc.w);
        return;
    }
    for (int k = 0; k < 2 && e + k < n_uc; ++k) {
        float sr = 0.f, si = 0.f;
        for (int s = 0; s < nsplit; ++s) {
            float2 v = part[(size_t)s * n_uc + e + k];
            sr += v.x;
            si += v.y;
        }
        double2 o = sums[e + k];
        sums[e + k] = make_double2(o.x + (double)sr, o.y + (double)si);
    }
}

// out[f][a][l] = sums[amap[a]][l * F + f] * inv_n   (normalisation by N_eff, Sec. 4)
__global__ void read_sums_kernel(const double2* __restrict__ sums, const int32_t* __restrict__ amap,
                                 int F, int A, int L, int ncols, double inv_n, double2* __restrict__ out)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = (int64_t)F * A * L;
    if (e >= total) return;
    int l = (int)(e % L);
    int a = (int)((e / L) % A);
    int f = (int)(e / ((int64_t)A * L));
    double2 v = sums[(size_t)amap[a] * ncols + l * F + f];
    out[e] = make_double2(v.x * inv_n, v.y * inv_n);
}

}  // namespace

cudaError_t reduce_partials(const float2* part, int nsplit, int n_uc, double2* sums, cudaStream_t st)
{
    if (n_uc <= 0) return cudaSuccess;
    int pairs = (n_uc + 1) / 2;
    reduce_partials_kernel<<<(pairs + 255) / 256, 256, 0, st>>>(part, nsplit, n_uc, sums);
    return cudaGetLastError();
}

cudaError_t read_sums(const double2* sums, const int32_t* amap, int F, int A, int L, int ncols,
                      double inv_n, double2* out, cudaStream_t st)
{
    int64_t total = (int64_t)F * A * L;
    if (total <= 0) return cudaSuccess;
    read_sums_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(sums, amap, F, A, L, ncols, inv_n, out);
    return cudaGetLastError();
}

}  // namespace cyc
