// proj_small.cu -- FP32 a-projection for a handful of distinct cycle frequencies.
//
// When only a few a are distinct (Au <= 32), a 128-row GEMM tile would be almost empty.
// Here every thread keeps the complex sums of up to 16 cycle frequencies x CB columns in
// registers while it walks its own strided samples (x[n] and x[n+m] are read once per
// sample for all of them), and the block then folds its threads' sums with warp shuffles
// and shared memory into one FP32 partial per (split, a, column).  More than 16 distinct a
// take two groups of blocks.  Same arithmetic as the GEMM path: lag products of Eqs.
// (ACF-def)/(CCF-def), weights exp(-j 2 pi phi n / 2^64) from the exact u64 phase (Sec. 4
// Set mode, per-alpha projection).  A thread's samples are NT apart, so its weight for the
// next sample is the current one times exp(-j 2 pi phi NT / 2^64) (one complex product
// instead of a sine and cosine), restarted from the exact phase every RESEED samples.
#include "cyc_device.cuh"
#include "cyc_impl.h"

namespace cyc {
namespace {

constexpr int NT = 256;
constexpr int RESEED = 8;                 // samples between exact weights of a thread
constexpr int64_t MIN_SPLIT = 8 * NT;     // at least 8 samples per thread and split

template <int AU, int CB>
__global__ void __launch_bounds__(NT) proj_small_kernel(ProjArgs a, int ncb)
{
    __shared__ float red[NT / 32][2 * AU * CB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cb = blockIdx.x % ncb, ug = blockIdx.x / ncb;
    const int c0 = cb * CB, ua = ug * AU;                     // first column and cycle frequency
    int64_t n_beg = (int64_t)blockIdx.y * a.split_len - a.split_off;
    int64_t n_end = n_beg + a.split_len;
    if (n_beg < 0) n_beg = 0;
    if (n_end > a.nc) n_end = a.nc;

    // per-block constants in shared memory (read as broadcasts): registers stay for the sums
    __shared__ uint64_t phi[AU];
    __shared__ float2 step[AU];                               // exp(-j 2 pi phi NT / 2^64)
    __shared__ int lag[CB];
    __shared__ bool cj[CB], okc[CB];
    for (int u = tid; u < AU; u += NT) {
        phi[u] = ua + u < a.Au ? a.phi[ua + u] : 0ull;
        step[u] = phase_rot(phi[u], (uint64_t)NT);
    }
    for (int j = tid; j < CB; j += NT) {
        okc[j] = c0 + j < a.ncols;
        lag[j] = okc[j] ? a.col_lag[c0 + j] : 0;
        cj[j] = okc[j] && a.col_conj[c0 + j];
    }
    __syncthreads();
    float sr[AU][CB], si[AU][CB];
    float2 w[AU];
#pragma unroll
    for (int u = 0; u < AU; ++u) {
        w[u] = make_float2(1.f, 0.f);
#pragma unroll
        for (int j = 0; j < CB; ++j) { sr[u][j] = 0.f; si[u][j] = 0.f; }
    }

    const float2* yv = a.y ? a.y : a.x;          // reference input (y = x for the auto forms)
    int k = 0;
    for (int64_t n = n_beg + tid; n < n_end; n += NT, ++k) {
        const float2 y0 = __ldg(&yv[n + a.D]);
        float2 p[CB];
#pragma unroll
        for (int j = 0; j < CB; ++j)
            p[j] = okc[j] ? lag_product(__ldg(&a.x[n + lag[j]]), y0, cj[j]) : make_float2(0.f, 0.f);
        if (k % RESEED == 0) {
            const uint64_t nabs = a.nbase + (uint64_t)n;
#pragma unroll
            for (int u = 0; u < AU; ++u) w[u] = phase_rot(phi[u], nabs);
        } else {
#pragma unroll
            for (int u = 0; u < AU; ++u) {
                const float2 s = step[u];
                w[u] = make_float2(w[u].x * s.x - w[u].y * s.y, w[u].x * s.y + w[u].y * s.x);
            }
        }
#pragma unroll
        for (int u = 0; u < AU; ++u)
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                sr[u][j] = fmaf(w[u].x, p[j].x, fmaf(-w[u].y, p[j].y, sr[u][j]));
                si[u][j] = fmaf(w[u].x, p[j].y, fmaf(w[u].y, p[j].x, si[u][j]));
            }
    }
    // fold the block: warp shuffles, then the eight warps through shared memory
#pragma unroll
    for (int u = 0; u < AU; ++u)
#pragma unroll
        for (int j = 0; j < CB; ++j) {
            float vr = sr[u][j], vi = si[u][j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vr += __shfl_xor_sync(0xffffffffu, vr, o);
                vi += __shfl_xor_sync(0xffffffffu, vi, o);
            }
            if (lane == 0) {
                red[warp][2 * (u * CB + j)] = vr;
                red[warp][2 * (u * CB + j) + 1] = vi;
            }
        }
    __syncthreads();
    for (int e = tid; e < AU * CB; e += NT) {
        const int u = e / CB, j = e % CB;
        if (ua + u >= a.Au || !(c0 + j < a.ncols)) continue;
        float vr = 0.f, vi = 0.f;
#pragma unroll
        for (int w8 = 0; w8 < NT / 32; ++w8) {
            vr += red[w8][2 * e];
            vi += red[w8][2 * e + 1];
        }
        a.part[((size_t)blockIdx.y * a.Au + ua + u) * a.ncols + c0 + j] = make_float2(vr, vi);
    }
}

int au_class(int Au) { return Au <= 1 ? 1 : Au <= 2 ? 2 : Au <= 4 ? 4 : Au <= 8 ? 8 : 16; }
int groups_of(int Au) { return Au > 16 ? 2 : 1; }
int cb_of(int Au) { return 64 / au_class(Au) > 32 ? 32 : 64 / au_class(Au); }

template <int AU, int CB>
cudaError_t launch(const ProjArgs& a, cudaStream_t st)
{
    const int ncb = (a.ncols + CB - 1) / CB;
    dim3 grid(ncb * groups_of(a.Au), a.nsplit);
    proj_small_kernel<AU, CB><<<grid, NT, 0, st>>>(a, ncb);
    return cudaGetLastError();
}

}  // namespace

bool small_supported(int Au) { return Au >= 1 && Au <= 32; }

ProjPlan small_plan(int Au, int ncols, int64_t nc, int num_sms)
{
    const int blocks = (ncols + cb_of(Au) - 1) / cb_of(Au) * groups_of(Au);
    int want = (2 * num_sms + blocks - 1) / blocks;       // about two blocks per SM
    int64_t len = (nc + want - 1) / want;
    if (len < MIN_SPLIT) len = MIN_SPLIT;
    ProjPlan p;
    p.split_len = len;
    p.nsplit = (int)((nc + len - 1) / len);
    if (p.nsplit < 1) p.nsplit = 1;
    return p;
}

size_t small_max_partials(int Au, int ncols, int num_sms)
{
    const int blocks = (ncols + cb_of(Au) - 1) / cb_of(Au) * groups_of(Au);
    size_t want = (size_t)((2 * num_sms + blocks - 1) / blocks);
    return want * (size_t)Au * (size_t)ncols;
}

cudaError_t small_launch(const ProjArgs& a, cudaStream_t st)
{
    switch (au_class(a.Au)) {
    case 1: return launch<1, 32>(a, st);
    case 2: return launch<2, 32>(a, st);
    case 4: return launch<4, 16>(a, st);
    case 8: return launch<8, 8>(a, st);
    default: return launch<16, 4>(a, st);
    }
}

}  // namespace cyc
