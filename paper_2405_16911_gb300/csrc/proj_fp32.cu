// proj_fp32.cu -- FP32 CUDA-core a-projection of the cyclic correlation estimator.
//
// For one contiguous view of the stream the kernel forms, per (cycle frequency u, column c):
//   part[s][u][c] = sum_{n in split s} exp(-j 2 pi phi_u (nbase + n) / 2^64) * P_c(n)
//   P_c(n) = x[n + m_c] * conj(y[n + D])   (CONV, Eq. (ACF-def) lag product)
//   P_c(n) = x[n + m_c] * y[n + D]         (CONJ, Eq. (CCF-def) lag product)
// with y = x for the auto forms and D = M^- for signed lags (Eq. (impl-corr)).
// i.e. the per-alpha projection of the lag products in Sec. 4 Set mode, written as a
// complex GEMM  W[u][n] x P[n][c]  over the samples n.  Both operands are produced in
// shared memory per K-tile (the lag products are never stored in HBM); the phase is
// reduced exactly as a u64 product phi * n mod 2^64, so n may run far past 2^30.
//
// Tile: 128 cycle frequencies x 128 columns per CTA, 16 samples per K-tile, 256 threads,
// 8 x 8 complex accumulators per thread, double-buffered operand tiles.  The register sums
// are added into the CTA's own partial every FLUSH samples and restarted, so no FP32 chain
// is longer than FLUSH terms (a sequential FP32 sum of 2^20 positive terms drifts by about
// 1e-4 of its value; one of 4096 terms by a few 1e-6).
#include "cyc_impl.h"
#include "cyc_device.cuh"

namespace cyc {
namespace {

constexpr int TA = 128;    // cycle frequencies per CTA
constexpr int TC = 128;    // columns per CTA
constexpr int TK = 16;     // samples per K-tile
constexpr int NT = 256;    // threads
constexpr int FLUSH = 4096; // samples per register-sum chain

struct Smem {
    float2 w[2][TK][TA];
    float2 p[2][TK][TC];
};

__device__ __forceinline__ void gen_tile(const ProjArgs& a, Smem& sm, int buf, int64_t n_tile,
                                         int64_t n_end, uint64_t phi_g, bool a_ok, int gen_a,
                                         int lag_g, bool conj_g, bool c_ok, int gen_c, int k0)
{
    // W: thread owns cycle frequency gen_a, samples k0, k0 + 2, ..., k0 + 14
#pragma unroll
    for (int j = 0; j < TK / 2; ++j) {
        int k = k0 + 2 * j;
        int64_t n = n_tile + k;
        float2 w = make_float2(0.f, 0.f);
        if (a_ok && n < n_end) w = phase_rot(phi_g, a.nbase + (uint64_t)n);
        sm.w[buf][k][gen_a] = w;
    }
    // P: thread owns column gen_c, same samples
#pragma unroll
    for (int j = 0; j < TK / 2; ++j) {
        int k = k0 + 2 * j;
        int64_t n = n_tile + k;
        float2 p = make_float2(0.f, 0.f);
        if (c_ok && n < n_end) {
            float2 xm = __ldg(&a.x[n + lag_g]);
            float2 y0 = __ldg(&(a.y ? a.y : a.x)[n + a.D]);
            p = lag_product(xm, y0, conj_g);
        }
        sm.p[buf][k][gen_c] = p;
    }
}

// Adds (or, for the first chain, writes) the thread's 8 x 8 sums into the partial tile.
__device__ __forceinline__ void flush_sums(float2* out, const ProjArgs& a, int u0, int c0, int tx, int ty,
                                          float (&acc_r)[8][8], float (&acc_i)[8][8], bool add)
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int u = u0 + 2 * ty + (i & 1) + 32 * (i >> 1);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int c = c0 + 2 * tx + (j & 1) + 32 * (j >> 1);
            if (u < a.Au && c < a.ncols) {
                float2* o = &out[(size_t)u * a.ncols + c];
                float2 v = make_float2(acc_r[i][j], acc_i[i][j]);
                if (add) {
                    const float2 q = *o;
                    v.x += q.x;
                    v.y += q.y;
                }
                *o = v;
            }
            acc_r[i][j] = 0.f;
            acc_i[i][j] = 0.f;
        }
    }
}

__global__ void __launch_bounds__(NT, 1) proj_fp32_kernel(ProjArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int u0 = blockIdx.x * TA;
    const int c0 = blockIdx.y * TC;
    const int split = blockIdx.z;
    int64_t n_beg = (int64_t)split * a.split_len - a.split_off;
    int64_t n_end = n_beg + a.split_len;
    if (n_beg < 0) n_beg = 0;
    if (n_end > a.nc) n_end = a.nc;

    // generator roles
    const int gen_a = tid & (TA - 1), gen_c = tid & (TC - 1), k0 = tid >> 7;
    const bool a_ok = u0 + gen_a < a.Au;
    const bool c_ok = c0 + gen_c < a.ncols;
    const uint64_t phi_g = a_ok ? a.phi[u0 + gen_a] : 0ull;
    const int lag_g = c_ok ? a.col_lag[c0 + gen_c] : 0;
    const bool conj_g = c_ok ? (a.col_conj[c0 + gen_c] != 0) : false;

    float acc_r[8][8], acc_i[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) { acc_r[i][j] = 0.f; acc_i[i][j] = 0.f; }

    float2* out = a.part + (size_t)split * a.Au * a.ncols;
    bool flushed = false;
    int buf = 0;
    if (n_beg < n_end) gen_tile(a, sm, 0, n_beg, n_end, phi_g, a_ok, gen_a, lag_g, conj_g, c_ok, gen_c, k0);
    __syncthreads();
    for (int64_t nt = n_beg; nt < n_end; nt += TK) {
        if (nt > n_beg && (nt - n_beg) % FLUSH == 0) {
            flush_sums(out, a, u0, c0, tx, ty, acc_r, acc_i, flushed);
            flushed = true;
        }
        if (nt + TK < n_end)
            gen_tile(a, sm, buf ^ 1, nt + TK, n_end, phi_g, a_ok, gen_a, lag_g, conj_g, c_ok, gen_c, k0);
#pragma unroll 4
        for (int k = 0; k < TK; ++k) {
            float4 w4[4], p4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                w4[j] = *reinterpret_cast<const float4*>(&sm.w[buf][k][2 * ty + 32 * j]);
                p4[j] = *reinterpret_cast<const float4*>(&sm.p[buf][k][2 * tx + 32 * j]);
            }
            float wr[8], wi[8], pr[8], pi[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                wr[2 * j] = w4[j].x; wi[2 * j] = w4[j].y; wr[2 * j + 1] = w4[j].z; wi[2 * j + 1] = w4[j].w;
                pr[2 * j] = p4[j].x; pi[2 * j] = p4[j].y; pr[2 * j + 1] = p4[j].z; pi[2 * j + 1] = p4[j].w;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    acc_r[i][j] = fmaf(wr[i], pr[j], acc_r[i][j]);
                    acc_r[i][j] = fmaf(-wi[i], pi[j], acc_r[i][j]);
                    acc_i[i][j] = fmaf(wr[i], pi[j], acc_i[i][j]);
                    acc_i[i][j] = fmaf(wi[i], pr[j], acc_i[i][j]);
                }
        }
        __syncthreads();
        buf ^= 1;
    }

    // partials: thread's rows are 2ty + {0,1} + 32 j, columns 2tx + {0,1} + 32 j
    flush_sums(out, a, u0, c0, tx, ty, acc_r, acc_i, flushed);
}

int tiles_of(int Au, int ncols) { return ((Au + TA - 1) / TA) * ((ncols + TC - 1) / TC); }

}  // namespace

ProjPlan fp32_plan(int Au, int ncols, int64_t nc, int num_sms)
{
    int tiles = tiles_of(Au, ncols);
    int smax = max_splits(tiles, num_sms, Au, ncols);
    if ((int64_t)smax > nc / 2048) smax = (int)(nc / 2048);
    const int want = wave_splits(tiles, num_sms, smax);     // one CTA per SM, whole waves
    int64_t len = (nc + want - 1) / want;
    if (len < 4 * TK) len = 4 * TK;
    len = (len + TK - 1) / TK * TK;
    ProjPlan p;
    p.split_len = len;
    p.nsplit = (int)((nc + len - 1) / len);
    if (p.nsplit < 1) p.nsplit = 1;
    return p;
}

size_t fp32_max_partials(int Au, int ncols, int num_sms)
{
    return (size_t)max_splits(tiles_of(Au, ncols), num_sms, Au, ncols) * (size_t)Au * (size_t)ncols;
}

cudaError_t fp32_launch(const ProjArgs& a, cudaStream_t st)
{
    static bool attr_set[64] = {false};                   // the attribute is per device
    size_t smem = sizeof(Smem);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(proj_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dim3 grid((a.Au + TA - 1) / TA, (a.ncols + TC - 1) / TC, a.nsplit);
    proj_fp32_kernel<<<grid, NT, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace cyc
