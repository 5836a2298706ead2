// cyc_kernels.cu -- FP64 running-sum update and normalised read-out of libcyc.
#include "cyc_impl.h"

namespace cyc {
namespace {

// sums[e] += sum_s part[s][e], e = (u, c) flattened; FP32 partials widened to FP64.
__global__ void reduce_partials_kernel(const float2* __restrict__ part, int nsplit, int n_uc,
                                       double2* __restrict__ sums)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_uc) return;
    double sr = 0.0, si = 0.0;
    for (int s = 0; s < nsplit; ++s) {
        float2 v = part[(size_t)s * n_uc + e];
        sr += (double)v.x;
        si += (double)v.y;
    }
    double2 o = sums[e];
    o.x += sr;
    o.y += si;
    sums[e] = o;
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
    reduce_partials_kernel<<<(n_uc + 255) / 256, 256, 0, st>>>(part, nsplit, n_uc, sums);
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
