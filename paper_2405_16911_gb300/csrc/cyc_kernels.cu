// cyc_kernels.cu -- FP64 running-sum update and normalised read-out of libcyc.
#include "cyc_device.cuh"
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
                                 int F, int A, int L, int ncols, double inv_n, double2* __restrict__ out,
                                 const int* err_src, int* err_dst)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (err_dst && e == 0) *err_dst = *err_src;
    int64_t total = (int64_t)F * A * L;
    if (e >= total) return;
    int l = (int)(e % L);
    int a = (int)((e / L) % A);
    int f = (int)(e / ((int64_t)A * L));
    double2 v = sums[(size_t)amap[a] * ncols + l * F + f];
    out[e] = make_double2(v.x * inv_n, v.y * inv_n);
}

// One thread per (u, c) element: the pass's splits in order.  A hop's sum (its FP32 split
// partials, added in float-float) is rounded to FP32 once and that value is both kept in the
// ring and added to the float-float window sum, so dropping it later subtracts exactly what
// was added; a completed window's sum is stored rounded to FP32 until it is read (the
// partials carry FP32 rounding already).  No FP64 arithmetic per split: this GPU's FP64
// rate made an FP64 version of this kernel bound by its FP64 adds and conversions.  The
// pass total joins the FP64 running sums once, as in reduce_partials.  Splits [0, nend)
// each end a hop, hop hops0 + s.  When the pass ends at most w hops, every ring slot it
// touches is read (the hop that leaves the window) before it is written, and no slot twice,
// so a batch of HOP_B splits issues all its loads before the dependent updates; a longer
// pass (a chunk longer than the window) runs the splits one at a time.
constexpr int HOP_T = 256, HOP_B = 8;

__global__ void __launch_bounds__(HOP_T) fold_hops_kernel(HopArgs h)
{
    const int e = blockIdx.x * HOP_T + threadIdx.x;
    if (e >= h.n_uc) return;
    const size_t n = (size_t)h.n_uc;
    const int64_t ends = (h.nc + h.off) / h.hop;
    const int nend = ends < (int64_t)h.nsplit ? (int)ends : h.nsplit;
    const bool batched = nend <= h.w;
    // ring slot of the next hop and window-ring slot of the window it would complete, advanced
    // one hop at a time (no 64-bit division per hop)
    int slot = (int)(h.hops0 % h.w);
    const int64_t kw0 = h.hops0 - h.w + 1;
    int wslot = (int)(((kw0 % h.cap) + h.cap) % h.cap);
    int64_t hk = h.hops0;
    float4 P = h.pend[e], W = h.wsum[e];                  // float-float (re hi, re lo, im hi, im lo)
    float tr = 0.f, ti = 0.f;
    for (int s0 = 0; s0 < h.nsplit; s0 += HOP_B) {
        float2 v[HOP_B], old[HOP_B];
#pragma unroll
        for (int j = 0; j < HOP_B; ++j) {
            const int s = s0 + j;
            v[j] = s < h.nsplit ? h.part[(size_t)s * n + e] : make_float2(0.f, 0.f);
            int sj = slot + j;                                         // < 2 w when s < nend <= w
            if (sj >= h.w) sj -= h.w;
            old[j] = batched && s < nend && hk + j >= h.w ? h.ring[(size_t)sj * n + e] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < HOP_B; ++j) {
            const int s = s0 + j;
            if (s >= h.nsplit) break;
            ff_add(P.x, P.y, v[j].x);
            ff_add(P.z, P.w, v[j].y);
            tr += v[j].x;
            ti += v[j].y;
            if (s < nend) {                                            // split s ends hop hk
                float2* rs = h.ring + (size_t)slot * n + e;
                if (hk >= h.w) {
                    const float2 o = batched ? old[j] : *rs;
                    ff_add(W.x, W.y, -o.x);
                    ff_add(W.z, W.w, -o.y);
                }
                const float2 h32 = make_float2(P.x + P.y, P.z + P.w);
                ff_add(W.x, W.y, h32.x);
                ff_add(W.z, W.w, h32.y);
                *rs = h32;
                if (hk >= h.w - 1) h.wout[(size_t)wslot * n + e] = make_float2(W.x + W.y, W.z + W.w);
                P = make_float4(0.f, 0.f, 0.f, 0.f);
                ++hk;
                if (++slot == h.w) slot = 0;
                if (++wslot == h.cap) wslot = 0;
            }
        }
    }
    h.pend[e] = P;
    h.wsum[e] = W;
    const double2 o = h.sums[e];
    h.sums[e] = make_double2(o.x + (double)tr, o.y + (double)ti);
}

// Block (a-tile, i): window k0 + i for RW_A cycle frequencies.  RW_A threads form the
// rotations from the exact u64 phase (FP64 sine and cosine, rounded to FP32 once); the
// products are FP32 (the stored window sums are FP32) and leave as FP64.
constexpr int RW_T = 256, RW_A = 8, RW_U = 8;

__global__ void __launch_bounds__(RW_T) read_windows_kernel(const float2* __restrict__ wout, int64_t cap,
                                                            int64_t k0, const int32_t* __restrict__ amap,
                                                            const uint64_t* __restrict__ phi, int F, int A, int L,
                                                            int Au, int ncols, uint64_t base, int64_t hop,
                                                            double inv_n, double2* __restrict__ out)
{
    __shared__ float2 rot[RW_A];
    __shared__ int urow[RW_A];
    const int a0 = blockIdx.x * RW_A;
    const int64_t i = blockIdx.y, k = k0 + i;
    const int na = A - a0 < RW_A ? A - a0 : RW_A;
    const int FL = F * L;
    const int total = na * FL;
    if (threadIdx.x < na) {
        const int u = amap[a0 + threadIdx.x];
        urow[threadIdx.x] = u;
        // the window's first reference sample carries phase phi * (base + k hop) mod 2^64 in the
        // running sums; the window-local phase removes it: v * exp(+j 2 pi that / 2^64) / N
        const uint64_t th = phi[u] * (base + (uint64_t)k * (uint64_t)hop);
        const double t = (double)(th >> 11) * 0x1.0p-53;               // cycles in [0, 1)
        double sn, cs;
        sincospi(2.0 * t, &sn, &cs);
        rot[threadIdx.x] = make_float2((float)(cs * inv_n), (float)(sn * inv_n));
    }
    __syncthreads();
    const float2* src = wout + (size_t)(k % cap) * (size_t)Au * ncols;
    double2* dst = out + (size_t)i * F * A * L;
    for (int q0 = 0; q0 < total; q0 += RW_T * RW_U) {
        float2 v[RW_U];
#pragma unroll
        for (int j = 0; j < RW_U; ++j) {
            const int q = q0 + j * RW_T + threadIdx.x;
            v[j] = q < total ? src[(size_t)urow[q / FL] * ncols + q % FL] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < RW_U; ++j) {
            const int q = q0 + j * RW_T + threadIdx.x;
            if (q >= total) break;
            const int ar = q / FL, e = q % FL;
            const int f = e % F, l = e / F;                             // source column l F + f
            const float2 r = rot[ar];
            dst[((size_t)f * A + a0 + ar) * L + l] =
                make_double2((double)(v[j].x * r.x - v[j].y * r.y), (double)(v[j].x * r.y + v[j].y * r.x));
        }
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
                      double inv_n, double2* out, cudaStream_t st, const int* err_src, int* err_dst)
{
    int64_t total = (int64_t)F * A * L;
    if (total <= 0) return cudaSuccess;
    read_sums_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(sums, amap, F, A, L, ncols, inv_n, out,
                                                                      err_src, err_dst);
    return cudaGetLastError();
}

}  // namespace cyc

namespace cyc {

cudaError_t fold_hops(const HopArgs& h, cudaStream_t st)
{
    if (h.n_uc <= 0 || h.nsplit <= 0) return cudaSuccess;
    fold_hops_kernel<<<(h.n_uc + HOP_T - 1) / HOP_T, HOP_T, 0, st>>>(h);
    return cudaGetLastError();
}

cudaError_t read_windows(const float2* wout, int64_t cap, int64_t k0, int64_t n, const int32_t* amap,
                         const uint64_t* phi, int F, int A, int L, int Au, int ncols, uint64_t base, int64_t hop,
                         double inv_n, double2* out, cudaStream_t st)
{
    if (n <= 0 || A <= 0) return cudaSuccess;
    for (int64_t i0 = 0; i0 < n; i0 += 65535) {
        const int64_t m = n - i0 < 65535 ? n - i0 : 65535;
        read_windows_kernel<<<dim3((A + RW_A - 1) / RW_A, (unsigned)m), RW_T, 0, st>>>(
            wout, cap, k0 + i0, amap, phi, F, A, L, Au, ncols, base, hop, inv_n, out + (size_t)i0 * F * A * L);
    }
    return cudaGetLastError();
}

}  // namespace cyc
