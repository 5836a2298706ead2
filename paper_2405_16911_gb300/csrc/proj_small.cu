// proj_small.cu -- FP32 a-projection for a handful of distinct cycle frequencies.
//
// When only a few a are distinct (Au <= 32), a 128-row GEMM tile would be almost empty.
// Here every thread keeps the complex sums of up to 16 cycle frequencies x CB columns in
// registers while it walks its own strided samples (x[n] and x[n+m] are read once per
// sample for all of them, the next sample's loads issued before this sample's arithmetic),
// and the block then folds its threads' sums with warp shuffles and shared memory into one
// FP32 partial per (split, a, column).  More cycle frequencies than a block holds take
// several groups of blocks.  Same arithmetic as the GEMM path: lag products of Eqs.
// (ACF-def)/(CCF-def), weights exp(-j 2 pi phi n / 2^64) from the exact u64 phase (Sec. 4
// Set mode, per-alpha projection).  A thread's samples are NT apart, so its weight for the
// next sample is the current one times exp(-j 2 pi phi NT / 2^64) (one complex product
// instead of a sine and cosine), restarted from the exact phase every RESEED samples.
//
// The grid is one wave (splits x column groups <= the blocks the SMs hold at once).  For a
// running-sum pass the last block of a column group to finish adds the group's partials to
// the FP64 sums (the splits summed in FP32 in a fixed order, the total added once in FP64:
// the update of reduce_partials, without a second launch), and one block copies the view's
// carried tail for the next pass.
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
    __shared__ float2 fin[NT];
    __shared__ int last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cb = blockIdx.x % ncb, ug = blockIdx.x / ncb;
    const int c0 = cb * CB, ua = ug * AU;                     // first column and cycle frequency
    int64_t n_beg = (int64_t)blockIdx.y * a.split_len - a.split_off;
    int64_t n_end = n_beg + a.split_len;
    if (n_beg < 0) n_beg = 0;
    if (n_end > a.nc) n_end = a.nc;

    if (a.tail_keep > 0 && blockIdx.x == 0 && blockIdx.y == 0)
        for (int64_t i = tid; i < a.tail_keep; i += NT) {
            a.tail_x[i] = a.x[a.tail_from + i];
            if (a.tail_y) a.tail_y[i] = a.y[a.tail_from + i];
        }

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
    const float2 zero = make_float2(0.f, 0.f);
    // the block's columns in registers: lag offsets (a column past ncols reads lag 0's sample
    // and its sums are never written) and the CONJ flags as a bit mask
    int lg[CB];
    unsigned cjm = 0;
#pragma unroll
    for (int j = 0; j < CB; ++j) {
        lg[j] = lag[j];
        cjm |= cj[j] ? 1u << j : 0u;
    }
    int64_t n = n_beg + tid;
    const float2* xn = a.x + n;                  // x[n], y[n + D]: advanced by NT per sample
    const float2* yn = yv + n + a.D;
    float2 ny = zero, nx[CB];                    // the thread's next sample
#pragma unroll
    for (int j = 0; j < CB; ++j) nx[j] = zero;
    if (n < n_end) {
        ny = __ldg(yn);
#pragma unroll
        for (int j = 0; j < CB; ++j) nx[j] = __ldg(xn + lg[j]);
    }
    for (int k = 0; n < n_end; n += NT, ++k) {
        float2 p[CB];
#pragma unroll
        for (int j = 0; j < CB; ++j) p[j] = lag_product(nx[j], ny, (cjm >> j) & 1u);
        xn += NT;
        yn += NT;
        if (n + NT < n_end) {
            ny = __ldg(yn);
#pragma unroll
            for (int j = 0; j < CB; ++j) nx[j] = __ldg(xn + lg[j]);
        }
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
    const size_t stride = (size_t)a.Au * a.ncols;             // one split's partials
    for (int e = tid; e < AU * CB; e += NT) {
        const int u = e / CB, j = e % CB;
        if (ua + u >= a.Au || !(c0 + j < a.ncols)) continue;
        float vr = 0.f, vi = 0.f;
#pragma unroll
        for (int w8 = 0; w8 < NT / 32; ++w8) {
            vr += red[w8][2 * e];
            vi += red[w8][2 * e + 1];
        }
        a.part[blockIdx.y * stride + (size_t)(ua + u) * a.ncols + c0 + j] = make_float2(vr, vi);
    }
    if (!a.sums) return;
    // running sums: the column group's last block (arrival counter) adds its splits
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&a.cnt[blockIdx.x], 1) == (int)gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    constexpr int E = AU * CB, G = NT / E;                     // G threads per element
    static_assert(NT % E == 0, "block shape");
    const int e = tid % E, g = tid / E, u = e / CB, j = e % CB;
    const bool ok = ua + u < a.Au && c0 + j < a.ncols;
    const size_t idx = (size_t)(ua + u) * a.ncols + c0 + j;
    float2 v = zero;
    if (ok)
        for (int sp = g; sp < (int)gridDim.y; sp += G) {
            const float2 q = __ldcg(&a.part[sp * stride + idx]);
            v.x += q.x;
            v.y += q.y;
        }
    fin[tid] = v;
    __syncthreads();
    if (g == 0 && ok) {
        float vr = 0.f, vi = 0.f;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            vr += fin[q * E + e].x;
            vi += fin[q * E + e].y;
        }
        if (a.replace) {
            a.sums[idx] = make_double2((double)vr, (double)vi);
        } else {
            const double2 o = a.sums[idx];
            a.sums[idx] = make_double2(o.x + (double)vr, o.y + (double)vi);
        }
    }
    if (tid == 0) a.cnt[blockIdx.x] = 0;                       // ready for the next launch
}

// Block shapes (cycle frequencies x columns per block): 16 to 64 complex register sums per
// thread; 17..32 cycle frequencies take groups of 8
int au_class(int Au) { return Au <= 1 ? 1 : Au <= 2 ? 2 : Au <= 4 ? 4 : (Au <= 8 || Au > 16) ? 8 : 16; }
int cb_of_class(int cls) { return cls == 1 ? 16 : cls == 2 ? 16 : cls == 4 ? 8 : cls == 8 ? 8 : 4; }
int groups_of(int Au) { return (Au + au_class(Au) - 1) / au_class(Au); }

template <int AU, int CB>
int occupancy()
{
    static int bps[64] = {0};                                 // blocks per SM, per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!bps[dev]) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, proj_small_kernel<AU, CB>, NT, 0) != cudaSuccess) {
            cudaGetLastError();
            b = 1;
        }
        bps[dev] = b < 1 ? 1 : b;
    }
    return bps[dev];
}

int blocks_per_sm(int Au)
{
    switch (au_class(Au)) {
    case 1: return occupancy<1, 16>();
    case 2: return occupancy<2, 16>();
    case 4: return occupancy<4, 8>();
    case 8: return occupancy<8, 8>();
    default: return occupancy<16, 4>();
    }
}

int splits_per_wave(int Au, int ncols, int num_sms)
{
    const int want = num_sms * blocks_per_sm(Au) / small_groups(Au, ncols);
    return want < 1 ? 1 : want;
}

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

int small_groups(int Au, int ncols)
{
    const int cb = cb_of_class(au_class(Au));
    return (ncols + cb - 1) / cb * groups_of(Au);
}

ProjPlan small_plan(int Au, int ncols, int64_t nc, int num_sms)
{
    const int want = splits_per_wave(Au, ncols, num_sms);
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
    return (size_t)splits_per_wave(Au, ncols, num_sms) * (size_t)Au * (size_t)ncols;
}

cudaError_t small_launch(const ProjArgs& a, cudaStream_t st)
{
    if (a.sums && !a.cnt) return cudaErrorInvalidValue;
    switch (au_class(a.Au)) {
    case 1: return launch<1, 16>(a, st);
    case 2: return launch<2, 16>(a, st);
    case 4: return launch<4, 8>(a, st);
    case 8: return launch<8, 8>(a, st);
    default: return launch<16, 4>(a, st);
    }
}

}  // namespace cyc
