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

// One thread per (u, c) element: the pass's splits in order.  FP64 throughout (the hop
// sums and the window sums are differences of large running quantities).
__global__ void fold_hops_kernel(HopArgs h)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= h.n_uc) return;
    double2 pend = h.pend[e], wsum = h.wsum[e];
    double tr = 0.0, ti = 0.0;
    int64_t hk = h.hops0;
    for (int s = 0; s < h.nsplit; ++s) {
        const float2 v = h.part[(size_t)s * h.n_uc + e];
        pend.x += (double)v.x;
        pend.y += (double)v.y;
        tr += (double)v.x;
        ti += (double)v.y;
        if ((int64_t)(s + 1) * h.hop - h.off <= h.nc) {            // split s ends hop hk
            double2* slot = h.ring + (size_t)(hk % h.w) * h.n_uc + e;
            if (hk >= h.w) {
                const double2 old = *slot;
                wsum.x -= old.x;
                wsum.y -= old.y;
            }
            wsum.x += pend.x;
            wsum.y += pend.y;
            *slot = pend;
            if (hk >= h.w - 1) h.wout[(size_t)((hk - h.w + 1) % h.cap) * h.n_uc + e] = wsum;
            pend = make_double2(0.0, 0.0);
            ++hk;
        }
    }
    h.pend[e] = pend;
    h.wsum[e] = wsum;
    const double2 o = h.sums[e];
    h.sums[e] = make_double2(o.x + tr, o.y + ti);
}

// Block (a, i): window k0 + i, cycle frequency a; the rotation is formed once per block.
__global__ void read_windows_kernel(const double2* __restrict__ wout, int64_t cap, int64_t k0,
                                    const int32_t* __restrict__ amap, const uint64_t* __restrict__ phi, int F,
                                    int A, int L, int Au, int ncols, uint64_t base, int64_t hop, double inv_n,
                                    double2* __restrict__ out)
{
    __shared__ double2 rot;
    const int a = blockIdx.x;
    const int64_t i = blockIdx.y, k = k0 + i;
    const int u = amap[a];
    if (threadIdx.x == 0) {
        // the window's first reference sample carries phase phi * (base + k hop) mod 2^64 in the
        // running sums; the window-local phase removes it: v * exp(+j 2 pi that / 2^64) / N
        const uint64_t th = phi[u] * (base + (uint64_t)k * (uint64_t)hop);
        const double t = (double)(th >> 11) * 0x1.0p-53;               // cycles in [0, 1)
        double sn, cs;
        sincospi(2.0 * t, &sn, &cs);
        rot = make_double2(cs * inv_n, sn * inv_n);
    }
    __syncthreads();
    const double2* src = wout + (size_t)(k % cap) * (size_t)Au * ncols + (size_t)u * ncols;
    double2* dst = out + (size_t)i * F * A * L;
    for (int e = threadIdx.x; e < F * L; e += blockDim.x) {
        const int f = e % F, l = e / F;                                 // source column l F + f
        const double2 v = src[e];
        dst[((size_t)f * A + a) * L + l] = make_double2(v.x * rot.x - v.y * rot.y, v.x * rot.y + v.y * rot.x);
    }
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

namespace cyc {

cudaError_t fold_hops(const HopArgs& h, cudaStream_t st)
{
    if (h.n_uc <= 0 || h.nsplit <= 0) return cudaSuccess;
    fold_hops_kernel<<<(h.n_uc + 255) / 256, 256, 0, st>>>(h);
    return cudaGetLastError();
}

cudaError_t read_windows(const double2* wout, int64_t cap, int64_t k0, int64_t n, const int32_t* amap,
                         const uint64_t* phi, int F, int A, int L, int Au, int ncols, uint64_t base, int64_t hop,
                         double inv_n, double2* out, cudaStream_t st)
{
    if (n <= 0 || A <= 0) return cudaSuccess;
    for (int64_t i0 = 0; i0 < n; i0 += 65535) {
        const int64_t m = n - i0 < 65535 ? n - i0 : 65535;
        read_windows_kernel<<<dim3(A, (unsigned)m), 128, 0, st>>>(wout, cap, k0 + i0, amap, phi, F, A, L, Au, ncols,
                                                                  base, hop, inv_n, out + (size_t)i0 * F * A * L);
    }
    return cudaGetLastError();
}

}  // namespace cyc
