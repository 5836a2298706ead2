// proposer.cu -- learned cycle-frequency proposer: spectral features, a small 1-D conv net
// with hand-written forward, backward and Adam kernels, and top-K proposals with a
// full-grid fallback (declared in include/cyc.h).
//
// Features of a signal (Welch, 16 segments of 4096 samples, Hann window): the averaged
// periodograms of x, x^2 and of the lag products x[n+d] conj(x[n]), d in {0, 1, 2, 3, 4, 6,
// 8, 12, 16} (d = 0: |x|^2), as log10, shifted so that bin j is frequency -1/2 + j/4096,
// each channel standardised.  Cycle frequencies show up there as lines: the cyclic
// statistics are Fourier coefficients of the lag products (Sec. 2); x^2 carries the
// conjugate lines, the lag products the conventional ones -- at non-zero lags only for a
// constant-envelope signal such as GMSK (Sec. 3).
//
// Net: four circular convolutions (kernel 9, padding 4), 11 -> 64 -> 64 -> 64 -> 2 channels,
// ReLU after the first three, then the mean over groups of 8 bins: 2 x 512 logits, one per
// grid bin a = -1/2 + k/512 and form (CONV, CONJ).  Activations are stored in FP16, weights
// kept in FP32 (master copy for Adam) and FP16 (used by the kernels), all sums in FP32.
#include <cuda_fp16.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "cyc_device.cuh"
#include "cyc_impl.h"
#include "tc_ptx.cuh"

using namespace cyc;

namespace {

constexpr int NFFT = 4096, NSEG = 16, NBIN = 512, POOL = 8, KW = 9, NL = 4;
constexpr int NLAGC = 9, NIN = 2 + NLAGC, MAXD = 16;
__constant__ int c_lagch[NLAGC] = {0, 1, 2, 3, 4, 6, 8, 12, 16};
constexpr int CHS[NL + 1] = {NIN, 64, 64, 64, 2};

int pfail(int code, const char* fmt, ...)
{
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    record_error(buf);
    return code;
}

#define PCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return pfail(e_ == cudaErrorMemoryAllocation ? CYC_ENOMEM : CYC_ECUDA,          \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                   \
    } while (0)

// parameter offsets in the flat FP32 vector: W1 b1 W2 b2 W3 b3 W4 b4
struct Layout {
    int w[NL], b[NL], total;
    Layout()
    {
        int o = 0;
        for (int l = 0; l < NL; ++l) {
            w[l] = o;
            o += CHS[l + 1] * CHS[l] * KW;
            b[l] = o;
            o += CHS[l + 1];
        }
        total = o;
    }
};
const Layout LAY;

// ------------------------------------------------------------------------ features (FFT)
// The windowed DFT of one segment of one channel (shared memory, natural order):
// X[k] = sum_n y[n] w[n] exp(-j 2 pi k n / N), by the self-sorting radix-4 form
// (fft_stockham, twiddles by span from twiddles()).  Input and output are in natural order,
// so no bit-reversed (bank-conflicted) permutation is needed.  d0 and d1 alternate as source
// and destination; the result's buffer is returned.
__device__ float2* segment_dft(const float2* __restrict__ xs, int ch, int seg, float2* d0, float2* d1,
                               const float2* tw)
{
    const int tid = threadIdx.x;
    const int lag = ch >= 2 ? c_lagch[ch - 2] : 0;
    __syncthreads();
    for (int k = tid; k < NFFT; k += blockDim.x) {
        float2 v = xs[(size_t)seg * NFFT + k];
        float2 y;
        if (ch == 0) {
            y = v;
        } else if (ch == 1) {
            y = make_float2(v.x * v.x - v.y * v.y, 2.f * v.x * v.y);
        } else {
            const float2 u = xs[(size_t)seg * NFFT + k + lag];      // x[n+d] conj(x[n])
            y = make_float2(u.x * v.x + u.y * v.y, u.y * v.x - u.x * v.y);
        }
        // Hann: 1/2 - 1/2 cos(2 pi k / N), the cosine read from the twiddle table (tw[N/2 + k]
        // = exp(-j 2 pi k / N); cos(2 pi k / N) = -cos(2 pi (k - N/2) / N) in the upper half)
        const float c = k < NFFT / 2 ? tw[NFFT / 2 + k].x : -tw[k].x;
        float w = 0.5f - 0.5f * c;
        d0[k] = make_float2(y.x * w, y.y * w);
    }
    float2* src[1] = {d0};
    float2* dst[1] = {d1};
    cyc::fft_stockham<1>(src, dst, NFFT, tw);
    return src[0];
}

// tw[h + p] = exp(-j pi p / h) for the spans h = 1, 2, 4, ..., N/2 and p < h (tw[0] unused):
// the twiddles of one butterfly stage are consecutive, so a warp reads consecutive words (one
// table exp(-j 2 pi k / N) read at k = p N / 2h put a stage's twiddles N / 2h entries apart,
// in one shared-memory bank for the middle stages).
__device__ void twiddles(float2* tw)
{
    for (int m = threadIdx.x; m < NFFT; m += blockDim.x) {
        if (m == 0) {
            tw[0] = make_float2(1.f, 0.f);
            continue;
        }
        const int h = 1 << (31 - __clz(m));
        float s, c;
        sincospif(-(float)(m - h) / (float)h, &s, &c);
        tw[m] = make_float2(c, s);
    }
}

// acc (the segments' summed periodogram, natural bin order) -> log10 of the mean, shifted so
// that output bin j is FFT bin (j + N/2) mod N, standardised, FP16.  v: NFFT floats of scratch.
__device__ void finish_channel(const float* acc, float* v, __half* o)
{
    __shared__ float red[2][16];
    const int tid = threadIdx.x;
    float s1 = 0.f, s2 = 0.f;
    for (int j = tid; j < NFFT; j += blockDim.x) {
        float t = log10f(acc[(j + NFFT / 2) & (NFFT - 1)] / NSEG + 1e-12f);
        v[j] = t;
        s1 += t;
        s2 += t * t;
    }
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = s1;
        red[1][tid >> 5] = s2;
    }
    __syncthreads();
    float t1 = 0.f, t2 = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        t1 += red[0][w];
        t2 += red[1][w];
    }
    const float mu = t1 / NFFT;
    const float sd = fmaxf(sqrtf(fmaxf(t2 / NFFT - mu * mu, 0.f)), 1e-6f);
    for (int j = tid; j < NFFT; j += blockDim.x) o[j] = __float2half_rn((v[j] - mu) / sd);
}

// One CTA per (signal, channel): the 16 segments one after the other (many signals at once).
__global__ void __launch_bounds__(512) features_kernel(const float2* __restrict__ x, int64_t T, __half* __restrict__ out)
{
    extern __shared__ float fsm[];
    float2* d0 = reinterpret_cast<float2*>(fsm);         // 2 x 4096 complex (FFT ping-pong)
    float2* d1 = d0 + NFFT;
    float2* tw = d1 + NFFT;                               // 4096 twiddles (twiddles())
    float* acc = reinterpret_cast<float*>(tw + NFFT);     // 4096
    const int sig = blockIdx.x / NIN, ch = blockIdx.x % NIN, tid = threadIdx.x;
    const float2* xs = x + (size_t)sig * T;
    twiddles(tw);
    for (int k = tid; k < NFFT; k += blockDim.x) acc[k] = 0.f;
    for (int seg = 0; seg < NSEG; ++seg) {
        const float2* d = segment_dft(xs, ch, seg, d0, d1, tw);
        for (int k = tid; k < NFFT; k += blockDim.x) acc[k] += d[k].x * d[k].x + d[k].y * d[k].y;
    }
    __syncthreads();
    finish_channel(acc, reinterpret_cast<float*>(d0), out + ((size_t)sig * NIN + ch) * NFFT);
}

// One signal, latency first: one CTA per (channel, segment) writes its periodogram to
// pg [NIN][NSEG][NFFT]; the last CTA of a channel to finish (arrival counter cnt[ch], reset
// by that CTA) sums the channel's segments in order (the same sums, in the same order, as
// features_kernel) and finishes the channel.
__global__ void __launch_bounds__(512) periodogram_kernel(const float2* __restrict__ x, float* __restrict__ pg,
                                                          int* __restrict__ cnt, __half* __restrict__ out)
{
    extern __shared__ float fsm[];
    __shared__ int last;
    float2* d0 = reinterpret_cast<float2*>(fsm);
    float2* d1 = d0 + NFFT;
    float2* tw = d1 + NFFT;
    const int ch = blockIdx.x / NSEG, seg = blockIdx.x % NSEG;
    twiddles(tw);
    const float2* d = segment_dft(x, ch, seg, d0, d1, tw);
    float* o = pg + ((size_t)ch * NSEG + seg) * NFFT;
    for (int k = threadIdx.x; k < NFFT; k += blockDim.x) o[k] = d[k].x * d[k].x + d[k].y * d[k].y;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&cnt[ch], 1) == NSEG - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    float* acc = fsm;                                     // d0, d1 are free: [NFFT] sums, [NFFT] scratch
    for (int k4 = threadIdx.x; k4 < NFFT / 4; k4 += blockDim.x) {   // 4 bins per thread and load
        float4 q[NSEG];
#pragma unroll
        for (int sg = 0; sg < NSEG; ++sg)
            q[sg] = __ldcg(reinterpret_cast<const float4*>(pg + ((size_t)ch * NSEG + sg) * NFFT) + k4);
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int sg = 0; sg < NSEG; ++sg) {
            a.x += q[sg].x;
            a.y += q[sg].y;
            a.z += q[sg].z;
            a.w += q[sg].w;
        }
        reinterpret_cast<float4*>(acc)[k4] = a;
    }
    __syncthreads();
    finish_channel(acc, acc + NFFT, out + (size_t)ch * NFFT);
    if (threadIdx.x == 0) cnt[ch] = 0;                    // ready for the next signal
}

// ------------------------------------------------------------------------ convolution
// y[b][o][i] = bias[o] + sum_c sum_k W[o][c][k] x[b][c][(i + k - 4) mod N]  (+ ReLU, mask)
// Block: 32 output channels x 32 MP positions of one sample; 256 threads, 4 x MP outputs each
// (MP = 4 for training batches; MP = 1 for a single signal, four times as many CTAs).
template <typename TIn, typename TOut, int MP>
__global__ void __launch_bounds__(256) conv_kernel(const TIn* __restrict__ x, int cin, int cout,
                                                   const __half* __restrict__ w, const float* __restrict__ bias,
                                                   int relu, const __half* __restrict__ mask, TOut* __restrict__ y)
{
    constexpr int TI = 32 * MP, TCO = 32;
    extern __shared__ float csm[];
    float* xs = csm;                          // [cin][TI + 8]
    float* ws = csm + cin * (TI + 8);         // [TCO][cin][9]
    const int b = blockIdx.z, i0 = blockIdx.x * TI, o0 = blockIdx.y * TCO, tid = threadIdx.x;
    const TIn* xb = x + (size_t)b * cin * NFFT;
    for (int e = tid; e < cin * (TI + 8); e += 256) {
        const int c = e / (TI + 8), j = e % (TI + 8);
        const int src = (i0 + j - 4 + NFFT) & (NFFT - 1);
        xs[e] = (float)xb[(size_t)c * NFFT + src];
    }
    for (int e = tid; e < TCO * cin * KW; e += 256) {
        const int o = e / (cin * KW);
        ws[e] = o0 + o < cout ? __half2float(w[(size_t)(o0 + o) * cin * KW + e % (cin * KW)]) : 0.f;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    float acc[4][MP];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int m = 0; m < MP; ++m) acc[a][m] = 0.f;
    for (int c = 0; c < cin; ++c) {
        const float* xr = xs + c * (TI + 8);
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            float wv[4], xv[MP];
#pragma unroll
            for (int a = 0; a < 4; ++a) wv[a] = ws[((warp + 8 * a) * cin + c) * KW + k];
#pragma unroll
            for (int m = 0; m < MP; ++m) xv[m] = xr[lane + 32 * m + k];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int m = 0; m < MP; ++m) acc[a][m] = fmaf(wv[a], xv[m], acc[a][m]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int o = o0 + warp + 8 * a;
        if (o >= cout) continue;
        const float bv = bias ? bias[o] : 0.f;
#pragma unroll
        for (int m = 0; m < MP; ++m) {
            const int i = i0 + lane + 32 * m;
            float v = acc[a][m] + bv;
            if (relu) v = fmaxf(v, 0.f);
            const size_t idx = ((size_t)b * cout + o) * NFFT + i;
            if (mask && !(__half2float(mask[idx]) > 0.f)) v = 0.f;
            y[idx] = (TOut)v;
        }
    }
}

// The 64-output-channel layers on the tensor cores (tcgen05, one CTA, kind::f16, FP32 sums in
// TMEM): y[b][co][p] = act(bias[co] + sum_{t<9} sum_ci w[co][ci][t] x[b][ci][(p + t - 4) mod 4096])
// is a GEMM over k = (t, ci) with M = positions and N = 64 output channels.  The CTA stages
// 256 + 8 positions of every input channel transposed, [ci / 8][row][8 channels] (16-byte rows
// one after another), so the A operand of tap t is the same tile started t rows later; the
// weights arrive packed as [t][ci / 8][co][8 channels] (pack_conv_kernel) by one bulk copy.
// Per CTA 9 x (cin16 / 16) MMAs of 128 x 64 x 16 (cin padded to a multiple of 16 with zeros),
// then 8 warps read the 128 x 64 accumulator (lane = position; warps w and w + 4 take the
// two halves of the channels of lane quadrant w) and store.
constexpr int CT_POS = 128, CT_ROWS = CT_POS + 8, CT_T = 256;
constexpr uint32_t CT_XLBO = CT_ROWS * 16;                 // bytes between 8-channel groups of x
constexpr long long kConvWaitBudget = 2000000000ll;        // SM cycles per bounded wait

int conv_ch(int cin) { return (cin + 15) / 16 * 2; }        // 8-channel groups, padded to 16 channels
int conv_nco(int cout) { return cout > 16 ? 64 : 16; }      // MMA N: 64 output channels, or 16 (padded)
size_t conv_tc_smem(int cin, int nco)
{
    return (size_t)conv_ch(cin) * CT_XLBO + (size_t)KW * conv_ch(cin) * nco * 16 + 64;
}

// w [co][ci][t] (FP16) -> [t][ci / 8][co < nco][ci % 8], zero beyond cin and cout
__global__ void pack_conv_kernel(const __half* __restrict__ w, int cin, int ch, int cout, int nco,
                                 __half* __restrict__ out)
{
    const int total = KW * ch * nco * 8;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int j = e & 7, co = (e >> 3) % nco, tc_ = e / (nco * 8);
        const int c = tc_ % ch, t = tc_ / ch, ci = c * 8 + j;
        out[e] = ci < cin && co < cout ? w[((size_t)co * cin + ci) * KW + t] : __float2half(0.f);
    }
}

template <int NCO>
__device__ __forceinline__ void tmem_ld_half(uint32_t taddr, uint32_t (&r)[NCO / 2])
{
    if constexpr (NCO == 64) tc::tmem_ld32(taddr, r);
    else tc::tmem_ld8(taddr, r);
}

template <typename TOut, int NCO>
__global__ void __launch_bounds__(CT_T) conv_tc_kernel(const __half* __restrict__ x, int cin, int ch, int cout,
                                                         const __half* __restrict__ wpk,
                                                         const float* __restrict__ bias, int relu,
                                                         TOut* __restrict__ y, int* err)
{
    constexpr int TCOLS = NCO < 32 ? 32 : NCO;                 // TMEM columns allocated (at least 32)
    extern __shared__ __align__(1024) unsigned char ctsm[];
    unsigned char* xs = ctsm;                                               // [ch][CT_ROWS][8]
    unsigned char* ws = ctsm + ch * CT_XLBO;                                // [KW][ch][CT_CO][8]
    const uint32_t wbytes = (uint32_t)(KW * ch * NCO * 16);
    uint64_t* bar = reinterpret_cast<uint64_t*>(ws + wbytes);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
    int* okf = reinterpret_cast<int*>(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p0 = blockIdx.x * CT_POS, b = blockIdx.y;
    const __half* xb = x + (size_t)b * cin * NFFT;
    if (warp == 0) tc::tmem_alloc<TCOLS>(slot);
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        tc::mbar_arrive_expect_tx(bar, wbytes);
        tc::bulk_g2s(ws, wpk, wbytes, bar);
    }
    // the input tile: row r is position p0 - 4 + r (circular), 8 channels per 16-byte word
    for (int e = tid; e < CT_ROWS * ch; e += CT_T) {
        const int c = e / CT_ROWS, r = e - c * CT_ROWS;
        const int pos = (p0 - 4 + r) & (NFFT - 1);
        uint32_t v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c0 = c * 8 + 2 * j;
            const __half h0 = c0 < cin ? xb[(size_t)c0 * NFFT + pos] : __float2half(0.f);
            const __half h1 = c0 + 1 < cin ? xb[(size_t)(c0 + 1) * NFFT + pos] : __float2half(0.f);
            const __half2 hh = __halves2half2(h0, h1);
            v[j] = *reinterpret_cast<const uint32_t*>(&hh);
        }
        *reinterpret_cast<uint4*>(xs + c * CT_XLBO + r * 16) = make_uint4(v[0], v[1], v[2], v[3]);
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *slot;
    if (tid == 0) {
        int ok = tc::mbar_wait(bar, 0, kConvWaitBudget) ? 1 : 0;       // the weights have landed
        if (ok) {
            const uint32_t idesc = tc::idesc_f16(128, NCO, false);
            const uint32_t xa = tc::smem_u32(xs), wa = tc::smem_u32(ws);
            uint32_t acc = 0;
            for (int t = 0; t < KW; ++t)
                for (int c = 0; c < ch; c += 2) {
                    const uint64_t ad = tc::smem_desc(xa + c * CT_XLBO + (uint32_t)t * 16, CT_XLBO, 128);
                    const uint64_t bd = tc::smem_desc(wa + (uint32_t)((t * ch + c) * NCO) * 16, NCO * 16, 128);
                    tc::mma_f16(tmem, ad, bd, idesc, acc);
                    acc = 1;
                }
            tc::mma_commit(bar);
        } else {
            atomicExch(err, 1);
        }
        *okf = ok;
    }
    __syncthreads();
    bool ok = *okf != 0;
    if (ok && !tc::mbar_wait(bar, 1, kConvWaitBudget)) {                 // the accumulators are final
        atomicExch(err, 1);
        ok = false;
    }
    tc::tc_fence_after();
    if (ok) {
        const int q = warp & 3, hf = warp >> 2;
        const int p = p0 + 32 * q + lane;
        uint32_t r[NCO / 2];
        tmem_ld_half<NCO>(tmem + ((uint32_t)(32 * q) << 16) + hf * (NCO / 2), r);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < NCO / 2; ++j) {
            const int co = hf * (NCO / 2) + j;
            if (co >= cout) break;
            float v = __uint_as_float(r[j]) + (bias ? bias[co] : 0.f);
            if (relu) v = fmaxf(v, 0.f);
            y[((size_t)b * cout + co) * NFFT + p] = (TOut)v;
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc<TCOLS>(tmem);
}

// dW[o][c][k] += sum_b sum_i dz[b][o][i] h[b][c][(i + k - 4) mod N];  db[o] += sum dz[b][o][i]
// Block: 16 x 16 (o, c) pairs, a range of positions of one sample; atomics across blocks.
__global__ void __launch_bounds__(256) conv_wgrad_kernel(const __half* __restrict__ h, const float* __restrict__ dz,
                                                         int cin, int cout, float* __restrict__ dW,
                                                         float* __restrict__ db, int ichunk)
{
    constexpr int T = 16;
    __shared__ float hs[T][256 + 9];          // odd row length: conflict-free column walks
    __shared__ float ds[T][256];
    const int tid = threadIdx.x, oc = tid / T, cc = tid % T;
    const int o0 = blockIdx.x * T, c0 = blockIdx.y * T;
    const int b = blockIdx.z / ichunk, part = blockIdx.z % ichunk;
    const int span = NFFT / ichunk;
    float acc[KW] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float bacc = 0.f;
    for (int i0 = part * span; i0 < (part + 1) * span; i0 += 256) {
        __syncthreads();
        for (int e = tid; e < T * (256 + 8); e += 256) {
            const int c = e / (256 + 8), j = e % (256 + 8);   // 264 positions per row are used
            const int src = (i0 + j - 4 + NFFT) & (NFFT - 1);
            hs[c][j] = c0 + c < cin ? __half2float(h[((size_t)b * cin + c0 + c) * NFFT + src]) : 0.f;
        }
        for (int e = tid; e < T * 256; e += 256) {
            const int o = e / 256, j = e % 256;
            ds[o][j] = o0 + o < cout ? dz[((size_t)b * cout + o0 + o) * NFFT + i0 + j] : 0.f;
        }
        __syncthreads();
        float win[KW];
#pragma unroll
        for (int k = 0; k < KW - 1; ++k) win[k] = hs[cc][k];
        for (int j = 0; j < 256; ++j) {
            win[KW - 1] = hs[cc][j + KW - 1];
            const float dv = ds[oc][j];
#pragma unroll
            for (int k = 0; k < KW; ++k) acc[k] = fmaf(dv, win[k], acc[k]);
            bacc += dv;
#pragma unroll
            for (int k = 0; k < KW - 1; ++k) win[k] = win[k + 1];
        }
    }
    if (o0 + oc < cout && c0 + cc < cin) {
#pragma unroll
        for (int k = 0; k < KW; ++k) atomicAdd(&dW[((size_t)(o0 + oc) * cin + c0 + cc) * KW + k], acc[k]);
        if (c0 == 0 && cc == 0) atomicAdd(&db[o0 + oc], bacc);
    }
}

// W'[c][o][k] = W[o][c][8 - k]: the backward-data convolution as a forward one.
__global__ void flip_weights_kernel(const __half* __restrict__ w, int cin, int cout, __half* __restrict__ wt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cin * cout * KW) return;
    const int k = e % KW, o = (e / KW) % cout, c = e / (KW * cout);
    wt[e] = w[((size_t)o * cin + c) * KW + (KW - 1 - k)];
}

// logits[b][f][j] = mean over 8 bins of z[b][f][8j..8j+7]; BCE with logits, and
// dz[b][f][i] = dL/dlogit / 8 (mean over all B x 1024 entries).
__global__ void pool_loss_kernel(const float* __restrict__ z, const float* __restrict__ labels, int B, float pw,
                                 float* __restrict__ logits, float* __restrict__ dz, float* __restrict__ loss)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = B * 2 * NBIN;
    float lv = 0.f;
    if (e < n) {
        const float* zz = z + (size_t)e * POOL;
        float s = 0.f;
#pragma unroll
        for (int r = 0; r < POOL; ++r) s += zz[r];
        const float zl = s / POOL;
        if (logits) logits[e] = zl;
        if (labels) {
            const float y = labels[e];
            const float lsp = fmaxf(-zl, 0.f) + log1pf(expf(-fabsf(zl)));   // -log sigmoid(z)
            const float lsn = fmaxf(zl, 0.f) + log1pf(expf(-fabsf(zl)));    // -log(1 - sigmoid(z))
            lv = (pw * y * lsp + (1.f - y) * lsn) / n;
            const float sg = 1.f / (1.f + expf(-zl));
            const float g = (pw * y * (sg - 1.f) + (1.f - y) * sg) / n;
            if (dz)
                for (int r = 0; r < POOL; ++r) dz[(size_t)e * POOL + r] = g / POOL;
        }
    }
    if (loss) {
        for (int o = 16; o > 0; o >>= 1) lv += __shfl_xor_sync(0xffffffffu, lv, o);
        if ((threadIdx.x & 31) == 0 && lv != 0.f) atomicAdd(loss, lv);
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            int n, float lr, float b1, float b2, float c1, float c2, float eps)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void to_half_kernel(const float* __restrict__ p, int n, __half* __restrict__ h)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) h[e] = __float2half_rn(p[e]);
}

// Top-K per form by logit, as ranks: the rank of bin e is the number of bins whose logit is
// larger, or equal with a lower bin (NaN counts as -inf), so the ranks are a permutation in
// the order larger logit first, lower bin first among equal logits, and the bin of rank r < k
// is proposal r.  Confidence of a form: 1 - sigmoid of the logit of rank k (the best bin left
// out), i.e. how sure the net is that no line was left behind.  Block (form, part) ranks 64
// bins, 8 threads per bin.  With hres set (page-locked host memory laid out like idx:
// proposals at [f k + r], the confidences at [2 NBIN + f], the status word at [2 NBIN + 2])
// the results, and the status word *derr, are written there as well.
constexpr int TK_BLOCKS = 8, TK_BINS = NBIN / TK_BLOCKS, TK_LANES = NBIN / TK_BINS;
static_assert(TK_BINS * TK_LANES == NBIN && TK_LANES == 8, "top-k layout");

__global__ void __launch_bounds__(NBIN) topk_kernel(const float* __restrict__ logits, int k, int* __restrict__ idx,
                                                    float* __restrict__ conf, int* hres, const int* derr)
{
    __shared__ float val[NBIN];
    const int f = blockIdx.x / TK_BLOCKS, part = blockIdx.x % TK_BLOCKS, t = threadIdx.x;
    const float v = logits[f * NBIN + t];
    val[t] = isnan(v) ? -INFINITY : v;
    __syncthreads();
    const int e = part * TK_BINS + t / TK_LANES, q = t % TK_LANES;
    const float ve = val[e];
    int r = 0;
    for (int j = q; j < NBIN; j += TK_LANES) {
        const float vj = val[j];
        r += (vj > ve || (vj == ve && j < e)) ? 1 : 0;
    }
#pragma unroll
    for (int o = 1; o < TK_LANES; o <<= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (q == 0 && r < k) {
        idx[f * k + r] = e;
        if (hres) hres[f * k + r] = e;
    }
    const bool put_conf = k < NBIN ? (q == 0 && r == k) : (part == 0 && t == 0);
    if (put_conf) {
        const float cf = k < NBIN ? 1.f - 1.f / (1.f + expf(-ve)) : 1.f;
        conf[f] = cf;
        if (hres) hres[2 * NBIN + f] = __float_as_int(cf);
    }
    if (hres && blockIdx.x == 0 && t == 0) hres[2 * NBIN + 2] = *derr;
}

}  // namespace

struct cyc_net {
    int device = 0;
    float* p = nullptr;       // FP32 master parameters
    __half* ph = nullptr;     // FP16 copy used by the kernels
    float* g = nullptr;       // gradients
    float* m = nullptr;
    float* v = nullptr;
    __half* wt = nullptr;     // flipped weights of one layer (backward data)
    int step = 0;
    int cap = 0;              // batch capacity of the buffers below
    __half* h[NL] = {nullptr, nullptr, nullptr, nullptr};   // h[0] unused (features), h[1..3]
    float* z4 = nullptr;      // last conv output [B][2][4096]
    float* dz = nullptr;      // [B][64][4096]
    float* dh = nullptr;      // [B][64][4096]
    float* logits = nullptr;  // [B][2][512]
    float* loss = nullptr;
    float* labels = nullptr;
    __half* feats = nullptr;  // [1][NIN][4096] for cyc_propose
    float2* xbuf = nullptr;   // staging for a host signal
    int64_t xcap = 0;
    int* topi = nullptr;      // [2][NBIN] proposals, then (at 2 NBIN) the two confidences as floats
    float* conf = nullptr;
    float* pg = nullptr;      // [NIN][NSEG][NFFT] one signal's segment periodograms (cyc_propose)
    int* h_res = nullptr;     // page-locked copy of topi and conf
    int* h_res_dev = nullptr; // its device address (nullptr: copied into it instead)
    int* fcnt = nullptr;      // [NIN] arrival counters of periodogram_kernel
    __half* wpk[NL] = {nullptr, nullptr, nullptr, nullptr};   // conv weights packed for the tensor cores
    int* derr = nullptr;      // set by a tensor-core conv whose bounded wait gave up (in topi's buffer)

    void free_acts()
    {
        for (int l = 1; l < NL; ++l)
            if (h[l]) { cudaFree(h[l]); h[l] = nullptr; }
        void* ps[] = {z4, dz, dh, logits};
        for (void* q : ps)
            if (q) cudaFree(q);
        z4 = nullptr; dz = nullptr; dh = nullptr; logits = nullptr;
        cap = 0;
    }
};

namespace {

int ensure_batch(cyc_net* n, int B)
{
    if (B <= n->cap) return CYC_OK;
    n->free_acts();
    for (int l = 1; l < NL; ++l) PCK(cudaMalloc(&n->h[l], (size_t)B * 64 * NFFT * sizeof(__half)));
    PCK(cudaMalloc(&n->z4, (size_t)B * 2 * NFFT * sizeof(float)));
    PCK(cudaMalloc(&n->dz, (size_t)B * 64 * NFFT * sizeof(float)));
    PCK(cudaMalloc(&n->dh, (size_t)B * 64 * NFFT * sizeof(float)));
    PCK(cudaMalloc(&n->logits, (size_t)B * 2 * NBIN * sizeof(float)));
    n->cap = B;
    return CYC_OK;
}

size_t conv_smem(int cin, int ti) { return (size_t)cin * (ti + 8) * 4 + (size_t)32 * cin * KW * 4; }

// Batches of at most kSmallBatch signals take the narrow tiles (latency of one proposal).
constexpr int kSmallBatch = 2;

template <typename TI, typename TO, int MP>
cudaError_t conv_mp(const TI* x, int cin, int cout, const __half* w, const float* bias, int relu, const __half* mask,
                    TO* y, int B, cudaStream_t st)
{
    static bool set[64] = {false};                        // the attribute is per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(conv_kernel<TI, TO, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)conv_smem(64, 32 * MP));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) set[dev] = true;
    }
    dim3 grid(NFFT / (32 * MP), (cout + 31) / 32, B);
    conv_kernel<TI, TO, MP><<<grid, 256, conv_smem(cin, 32 * MP), st>>>(x, cin, cout, w, bias, relu, mask, y);
    return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t conv(const TI* x, int cin, int cout, const __half* w, const float* bias, int relu, const __half* mask,
                 TO* y, int B, cudaStream_t st)
{
    if (B <= kSmallBatch) return conv_mp<TI, TO, 1>(x, cin, cout, w, bias, relu, mask, y, B, st);
    return conv_mp<TI, TO, 4>(x, cin, cout, w, bias, relu, mask, y, B, st);
}

// the FP16 weights of the 64-channel layers in the tensor-core kernel's layout (after every
// change of n->ph)
cudaError_t pack_weights(cyc_net* n, cudaStream_t st)
{
    for (int l = 0; l < NL; ++l)
        pack_conv_kernel<<<64, 256, 0, st>>>(n->ph + LAY.w[l], CHS[l], conv_ch(CHS[l]), CHS[l + 1],
                                             conv_nco(CHS[l + 1]), n->wpk[l]);
    return cudaGetLastError();
}

// Layer l on the tensor cores: y = relu(conv) in FP16 for the hidden layers, the plain
// convolution in FP32 for the output layer.
cudaError_t conv_tc(const cyc_net* n, int l, const __half* x, void* y, int B, cudaStream_t st)
{
    static bool set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<__half, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)conv_tc_smem(64, 64));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_tc_kernel<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)conv_tc_smem(64, 16));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) set[dev] = true;
    }
    const int cin = CHS[l], cout = CHS[l + 1];
    const dim3 grid(NFFT / CT_POS, B);
    if (l < NL - 1)
        conv_tc_kernel<__half, 64><<<grid, CT_T, conv_tc_smem(cin, 64), st>>>(
            x, cin, conv_ch(cin), cout, n->wpk[l], n->p + LAY.b[l], 1, static_cast<__half*>(y), n->derr);
    else
        conv_tc_kernel<float, 16><<<grid, CT_T, conv_tc_smem(cin, 16), st>>>(
            x, cin, conv_ch(cin), cout, n->wpk[l], n->p + LAY.b[l], 0, static_cast<float*>(y), n->derr);
    return cudaGetLastError();
}

// After a synchronisation: did a tensor-core convolution give up waiting?
int net_status(cyc_net* n, int flag)
{
    if (!flag) return CYC_OK;
    cudaMemset(n->derr, 0, sizeof(int));
    return pfail(CYC_ETIMEDOUT, "a tensor-core convolution gave up waiting; the outputs are unreliable");
}

// forward of B feature sets; leaves h[1..3], z4 and (pooled) logits in the net's buffers
int net_forward(cyc_net* n, const __half* feats, int B, cudaStream_t st)
{
    int rc = ensure_batch(n, B);
    if (rc) return rc;
    const __half* in = feats;
    for (int l = 0; l < NL - 1; ++l) {                 // 11 -> 64 -> 64 -> 64
        PCK(conv_tc(n, l, in, n->h[l + 1], B, st));
        in = n->h[l + 1];
    }
    PCK(conv_tc(n, NL - 1, in, n->z4, B, st));       // 64 -> 2, FP32 out
    return CYC_OK;
}

// gradients into n->g (zeroed first) and the loss into n->loss
int net_backward(cyc_net* n, const __half* feats, const float* labels, int B, float pw, cudaStream_t st)
{
    PCK(cudaMemsetAsync(n->g, 0, LAY.total * sizeof(float), st));
    PCK(cudaMemsetAsync(n->loss, 0, sizeof(float), st));
    const int ne = B * 2 * NBIN;
    pool_loss_kernel<<<(ne + 255) / 256, 256, 0, st>>>(n->z4, labels, B, pw, n->logits, n->dz, n->loss);
    PCK(cudaGetLastError());
    for (int l = NL - 1; l >= 0; --l) {
        const int cin = CHS[l], cout = CHS[l + 1];
        const __half* hin = l == 0 ? feats : n->h[l];
        const int ich = 8;
        dim3 gw((cout + 15) / 16, (cin + 15) / 16, B * ich);
        conv_wgrad_kernel<<<gw, 256, 0, st>>>(hin, n->dz, cin, cout, n->g + LAY.w[l], n->g + LAY.b[l], ich);
        PCK(cudaGetLastError());
        if (l == 0) break;
        // dL/dh_l = conv of dz with the flipped, transposed weights; times the ReLU mask of h_l
        const int nw = cin * cout * KW;
        flip_weights_kernel<<<(nw + 255) / 256, 256, 0, st>>>(n->ph + LAY.w[l], cin, cout, n->wt);
        PCK(cudaGetLastError());
        PCK((conv<float, float>(n->dz, cout, cin, n->wt, nullptr, 0, n->h[l], n->dh, B, st)));
        float* t = n->dz;
        n->dz = n->dh;
        n->dh = t;
    }
    return CYC_OK;
}

}  // namespace

extern "C" {

int cyc_net_create(const float* params, uint64_t seed, int device, cyc_net** out)
{
    if (!out) return pfail(CYC_EINVAL, "cyc_net_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return pfail(CYC_ECUDA, "cyc_net_create: device %d is not available", device);
    }
    cudaSetDevice(device);
    cyc_net* n = new cyc_net();
    n->device = device;
    std::vector<float> host(LAY.total, 0.f);
    if (params) {
        memcpy(host.data(), params, LAY.total * sizeof(float));
    } else {
        // He-normal weights from splitmix64 + Box-Muller, zero biases
        uint64_t st = seed;
        auto next = [&st]() {
            uint64_t z = (st += 0x9E3779B97F4A7C15ull);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            return z ^ (z >> 31);
        };
        for (int l = 0; l < NL; ++l) {
            const int nw = CHS[l + 1] * CHS[l] * KW;
            const double sdev = sqrt(2.0 / (CHS[l] * KW));
            for (int i = 0; i < nw; ++i) {
                double u1 = ((next() >> 11) + 1) * (1.0 / 9007199254740992.0);
                double u2 = (next() >> 11) * (1.0 / 9007199254740992.0);
                host[LAY.w[l] + i] = (float)(sdev * sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2));
            }
        }
    }
    int rc = CYC_OK;
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == CYC_OK) rc = pfail(CYC_ECUDA, "cyc_net_create: %s", cudaGetErrorString(e));
    };
    chk(cudaMalloc(&n->p, LAY.total * sizeof(float)));
    chk(cudaMalloc(&n->ph, LAY.total * sizeof(__half)));
    chk(cudaMalloc(&n->g, LAY.total * sizeof(float)));
    chk(cudaMalloc(&n->m, LAY.total * sizeof(float)));
    chk(cudaMalloc(&n->v, LAY.total * sizeof(float)));
    chk(cudaMalloc(&n->wt, 64 * 64 * KW * sizeof(__half)));
    chk(cudaMalloc(&n->loss, sizeof(float)));
    chk(cudaMalloc(&n->feats, NIN * NFFT * sizeof(__half)));
    chk(cudaMalloc(&n->topi, (2 * NBIN + 4) * sizeof(int)));
    n->conf = reinterpret_cast<float*>(n->topi + 2 * NBIN);
    n->derr = n->topi + 2 * NBIN + 2;
    for (int l = 0; l < NL; ++l)
        chk(cudaMalloc(&n->wpk[l], (size_t)KW * conv_ch(CHS[l]) * conv_nco(CHS[l + 1]) * 8 * sizeof(__half)));
    chk(cudaMalloc(&n->pg, (size_t)NIN * NSEG * NFFT * sizeof(float)));
    chk(cudaMalloc(&n->fcnt, NIN * sizeof(int)));
    chk(cudaMallocHost(&n->h_res, (2 * NBIN + 4) * sizeof(int)));
    if (rc == CYC_OK && cudaHostGetDevicePointer((void**)&n->h_res_dev, n->h_res, 0) != cudaSuccess) {
        cudaGetLastError();
        n->h_res_dev = nullptr;
    }
    if (rc == CYC_OK) {
        chk(cudaMemcpy(n->p, host.data(), LAY.total * sizeof(float), cudaMemcpyHostToDevice));
        chk(cudaMemset(n->m, 0, LAY.total * sizeof(float)));
        chk(cudaMemset(n->v, 0, LAY.total * sizeof(float)));
        chk(cudaMemset(n->topi, 0, (2 * NBIN + 4) * sizeof(int)));
        chk(cudaMemset(n->fcnt, 0, NIN * sizeof(int)));
        to_half_kernel<<<(LAY.total + 255) / 256, 256>>>(n->p, LAY.total, n->ph);
        chk(pack_weights(n, 0));
        chk(cudaDeviceSynchronize());
    }
    if (rc != CYC_OK) {
        cyc_net_destroy(n);
        return rc;
    }
    *out = n;
    return CYC_OK;
}

int cyc_net_destroy(cyc_net* n)
{
    if (!n) return CYC_OK;
    cudaSetDevice(n->device);
    n->free_acts();
    void* ps[] = {n->p, n->ph, n->g, n->m, n->v, n->wt, n->loss, n->labels, n->feats, n->xbuf, n->topi, n->pg,
                  n->fcnt, n->wpk[0], n->wpk[1], n->wpk[2], n->wpk[3]};
    for (void* q : ps)
        if (q) cudaFree(q);
    if (n->h_res) cudaFreeHost(n->h_res);
    delete n;
    return CYC_OK;
}

int cyc_net_nparams(void) { return LAY.total; }

int cyc_net_get_params(cyc_net* n, float* out)
{
    if (!n || !out) return pfail(CYC_EINVAL, "cyc_net_get_params: NULL argument");
    cudaSetDevice(n->device);
    PCK(cudaMemcpy(out, n->p, LAY.total * sizeof(float), cudaMemcpyDeviceToHost));
    return CYC_OK;
}

int cyc_net_set_params(cyc_net* n, const float* params)
{
    if (!n || !params) return pfail(CYC_EINVAL, "cyc_net_set_params: NULL argument");
    cudaSetDevice(n->device);
    PCK(cudaMemcpy(n->p, params, LAY.total * sizeof(float), cudaMemcpyHostToDevice));
    to_half_kernel<<<(LAY.total + 255) / 256, 256>>>(n->p, LAY.total, n->ph);
    PCK(pack_weights(n, 0));
    PCK(cudaDeviceSynchronize());
    n->step = 0;
    PCK(cudaMemset(n->m, 0, LAY.total * sizeof(float)));
    PCK(cudaMemset(n->v, 0, LAY.total * sizeof(float)));
    return CYC_OK;
}

int cyc_features(const void* x, int64_t T, int nsig, void* feats)
{
    if (!x || !feats || nsig <= 0) return pfail(CYC_EINVAL, "cyc_features: bad argument");
    if (T < (int64_t)NSEG * NFFT + MAXD)
        return pfail(CYC_EINVAL, "cyc_features: signals need at least %d samples", NSEG * NFFT + MAXD);
    static bool set[64] = {false};                        // the attribute is per device
    const int smem = 2 * NFFT * 8 + NFFT * 8 + NFFT * 4;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !set[dev]) {
        PCK(cudaFuncSetAttribute(features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        if (dev >= 0 && dev < 64) set[dev] = true;
    }
    features_kernel<<<nsig * NIN, 512, smem>>>((const float2*)x, T, (__half*)feats);
    PCK(cudaGetLastError());
    PCK(cudaDeviceSynchronize());
    return CYC_OK;
}

int cyc_net_forward(cyc_net* n, const void* feats, int B, float* logits)
{
    if (!n || !feats || !logits || B <= 0) return pfail(CYC_EINVAL, "cyc_net_forward: bad argument");
    cudaSetDevice(n->device);
    int rc = net_forward(n, (const __half*)feats, B, 0);
    if (rc) return rc;
    const int ne = B * 2 * NBIN;
    pool_loss_kernel<<<(ne + 255) / 256, 256>>>(n->z4, nullptr, B, 1.f, logits, nullptr, nullptr);
    PCK(cudaGetLastError());
    PCK(cudaDeviceSynchronize());
    int flag = 0;
    PCK(cudaMemcpy(&flag, n->derr, sizeof(int), cudaMemcpyDeviceToHost));
    return net_status(n, flag);
}

int cyc_net_gradients(cyc_net* n, const void* feats, const float* labels, int B, float pos_weight, float* grads,
                      float* loss)
{
    if (!n || !feats || !labels || B <= 0) return pfail(CYC_EINVAL, "cyc_net_gradients: bad argument");
    cudaSetDevice(n->device);
    int rc = net_forward(n, (const __half*)feats, B, 0);
    if (rc) return rc;
    rc = net_backward(n, (const __half*)feats, labels, B, pos_weight, 0);
    if (rc) return rc;
    PCK(cudaDeviceSynchronize());
    int flag = 0;
    PCK(cudaMemcpy(&flag, n->derr, sizeof(int), cudaMemcpyDeviceToHost));
    if ((rc = net_status(n, flag))) return rc;
    if (grads) PCK(cudaMemcpy(grads, n->g, LAY.total * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss) PCK(cudaMemcpy(loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return CYC_OK;
}

int cyc_net_train_step(cyc_net* n, const void* feats, const float* labels, int B, float lr, float pos_weight,
                       float* loss)
{
    int rc = cyc_net_gradients(n, feats, labels, B, pos_weight, nullptr, loss);
    if (rc) return rc;
    n->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
    adam_kernel<<<(LAY.total + 255) / 256, 256>>>(n->p, n->g, n->m, n->v, LAY.total, lr, b1, b2, c1, c2, 1e-8f);
    to_half_kernel<<<(LAY.total + 255) / 256, 256>>>(n->p, LAY.total, n->ph);
    PCK(pack_weights(n, 0));
    PCK(cudaGetLastError());
    return CYC_OK;
}

int cyc_propose(cyc_net* n, const void* x, int64_t T, int on_device, int k, float tau, double* alphas_conv,
                double* alphas_conj, float* conf, int* used_fallback)
{
    if (!n || !x || k <= 0 || k > NBIN || !alphas_conv || !alphas_conj || !used_fallback)
        return pfail(CYC_EINVAL, "cyc_propose: bad argument");
    if (T < (int64_t)NSEG * NFFT + MAXD)
        return pfail(CYC_EINVAL, "cyc_propose: needs at least %d samples", NSEG * NFFT + MAXD);
    cudaSetDevice(n->device);
    const float2* xd = (const float2*)x;
    const int64_t use = (int64_t)NSEG * NFFT + MAXD;
    if (!on_device) {
        if (n->xcap < use) {
            if (n->xbuf) cudaFree(n->xbuf);
            PCK(cudaMalloc(&n->xbuf, use * sizeof(float2)));
            n->xcap = use;
        }
        PCK(cudaMemcpy(n->xbuf, x, use * sizeof(float2), cudaMemcpyHostToDevice));
        xd = n->xbuf;
    }
    // features of one signal: a CTA per (channel, segment); the last of each channel finishes it
    {
        static bool set[64] = {false};
        const int smem = 2 * NFFT * 8 + NFFT * 8;
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || !set[dev]) {
            PCK(cudaFuncSetAttribute(periodogram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            if (dev >= 0 && dev < 64) set[dev] = true;
        }
        periodogram_kernel<<<NIN * NSEG, 512, smem>>>(xd, n->pg, n->fcnt, n->feats);
        PCK(cudaGetLastError());
    }
    int rc = net_forward(n, n->feats, 1, 0);
    if (rc) return rc;
    pool_loss_kernel<<<(2 * NBIN + 255) / 256, 256>>>(n->z4, nullptr, 1, 1.f, n->logits, nullptr, nullptr);
    topk_kernel<<<2 * TK_BLOCKS, NBIN>>>(n->logits, k, n->topi, n->conf, n->h_res_dev, n->derr);
    PCK(cudaGetLastError());
    // one synchronisation: the proposals [2][k] and the confidences (stored after them), written
    // into page-locked memory by the top-k kernel itself (else copied there)
    if (!n->h_res_dev) {
        PCK(cudaMemcpyAsync(n->h_res, n->topi, 2 * k * sizeof(int), cudaMemcpyDeviceToHost, 0));
        PCK(cudaMemcpyAsync(n->h_res + 2 * NBIN, n->conf, 2 * sizeof(float) + sizeof(int), cudaMemcpyDeviceToHost, 0));
    }
    PCK(cudaStreamSynchronize(0));
    if ((rc = net_status(n, n->h_res[2 * NBIN + 2]))) return rc;
    const int* idx = n->h_res;
    float cf[2];
    memcpy(cf, n->h_res + 2 * NBIN, sizeof cf);
    for (int r = 0; r < k; ++r) {
        alphas_conv[r] = -0.5 + idx[r] / (double)NBIN;
        alphas_conj[r] = -0.5 + idx[k + r] / (double)NBIN;
    }
    const float c = fminf(cf[0], cf[1]);
    if (conf) *conf = c;
    *used_fallback = c < tau ? 1 : 0;
    return CYC_OK;
}

}  // extern "C"
