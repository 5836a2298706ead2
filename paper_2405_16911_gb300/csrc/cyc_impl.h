// cyc_impl.h -- internal declarations shared by the host API and the kernel files of libcyc.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cyc.h"

namespace cyc {

// One projection pass over a contiguous view of the stream (Sec. 4, Eq. (impl-corr)):
//   part[s][u][c] = sum over n in split s of  W(u, n) * P_c(n)
// with W(u, n) = exp(-j 2 pi phi_u (nbase + n) / 2^64) and P_c the lag product of column c
// (c = lag index * F + form index).  The caller folds the splits into the FP64 sums.
// Term n of a pass is x[n + col_lag] * c(y[n + D]) * exp(-j 2 pi phi (nbase + n) / 2^64):
// col_lag = m + M^- >= 0 and D = M^- for signed lags m >= -M^- (Eq. (impl-corr)); y = x
// (y == nullptr) for the cyclic ACF / CCF, a second input for the cross forms.
struct ProjArgs {
    const float2*   x;          // view x[0 .. nc + M)
    int64_t         nc;         // committed n in this pass (0 <= n < nc)
    uint64_t        nbase;      // absolute phase index of term n = 0, mod 2^64
    const uint64_t* phi;        // [Au] cycle frequencies as u64 fixed point (cycles * 2^64)
    int             Au;
    const int32_t*  col_lag;    // [ncols] lag of each column
    const int8_t*   col_conj;   // [ncols] 1: CONJ column (x[n+m] x[n]), 0: CONV (x[n+m] x*[n])
    int             ncols;
    int             nsplit;     // number of n-splits (partials)
    int64_t         split_len;  // samples per split
    float2*         part;       // [nsplit][Au][ncols]
    int*            err = nullptr;  // device status word: a bounded wait that gave up sets it
    int             M = 0;          // lag span M^- + M^+ (halo of every staged block of samples)
    int64_t         x_avail = 0;    // samples readable from x (and y) (allocation bound, even)
    const float2*   y = nullptr;    // second input, same indexing as x; nullptr: y = x
    int             D = 0;          // offset M^- of the reference sample y[n + D]
    int64_t         split_off = 0;  // split s covers [s * split_len - split_off, + split_len) within [0, nc)
    int             nforms = 0;     // columns per lag (c = l * nforms + f); 0 where unused
};

// One work item of the tensor-core projection: 128 cycle frequencies x 128 columns x an
// n-range of one stream.  Sample n of the stream is x[n & xmask] (xmask = ring capacity - 1,
// or all ones for a linear view with x_avail readable samples).  Result element (row r,
// tile column j) goes to out[r * out_stride + j] for u0 + r < Au and c0 + j < ncols.
struct TcItem {
    const float2*   x;
    uint64_t        xmask;
    int64_t         x_avail;
    uint64_t        nbase;      // absolute index of stream sample 0, mod 2^64
    int64_t         n_beg, n_end;
    const uint64_t* phi;
    const int32_t*  col_lag;
    const int8_t*   col_conj;
    float2*         out;
    int             out_stride;
    int             u0, Au, c0, ncols, M;
    const float2*   y;          // second input (linear views only) or nullptr: y = x
    int             D;          // offset of the reference sample y[n + D]
    int64_t         out_peer;   // pair lists: the odd CTA's rows u0 + 128 .. go to out + out_peer
    // Dual items (pair lists): a second stream with the same cycle frequencies, lags and
    // forms over a range of the same length.  The even CTA stages and forms the columns of
    // the first stream, the odd CTA those of the second; the weights follow the first
    // stream's sample index, so the second stream's sums are rotated by
    // exp(-j 2 pi a dphase / 2^64) before they are written to out2.
    const float2*   x2;         // nullptr: not a dual item
    uint64_t        xmask2;
    int64_t         n_beg2;
    float2*         out2;
    int64_t         out_peer2;  // the odd CTA's rows of the second stream go to out2 + out_peer2
    uint64_t        dphase;     // (nbase2 + n_beg2) - (nbase + n_beg) mod 2^64
};

// Launch geometry chosen by a kernel family for one pass.
struct ProjPlan {
    int     nsplit;
    int64_t split_len;
};

// Equal n-splits for `tiles` CTAs per split on `slots` co-resident CTAs: the one-wave count
// slots / tiles, or more splits over several waves when the last wave's idle SMs cost more
// (time ~ waves(s) / s at least 10 % smaller: per-CTA fixed costs eat smaller gains), at
// most smax.  Config 2's 64 tile-CTAs per
// split on 152 SMs: 2 splits (84 % of the SMs busy) become 7 (three waves, 0.43 against 0.5).
inline int wave_splits(int tiles, int slots, int smax)
{
    const int base = slots >= tiles ? slots / tiles : 1;
    int best = base;
    double cost = (double)(((int64_t)tiles * base + slots - 1) / slots) / base;
    for (int s = base + 1; s <= smax; ++s) {
        const double c = (double)(((int64_t)tiles * s + slots - 1) / slots) / s;
        if (c < cost * 0.90) {
            cost = c;
            best = s;
        }
    }
    return best;
}

// Splits a stream's partial buffer is sized for: the one-wave count, or up to 64 within
// 256 MiB of FP32 partials.
inline int max_splits(int tiles, int slots, int Au, int ncols)
{
    const int base = slots >= tiles ? slots / tiles : 1;
    const int64_t per = (int64_t)Au * ncols * 8;
    int64_t cap = per > 0 ? ((int64_t)256 << 20) / per : 64;
    if (cap > 64) cap = 64;
    return base > cap ? base : (int)cap;
}

// FP32 CUDA-core projection (proj_fp32.cu).
ProjPlan    fp32_plan(int Au, int ncols, int64_t nc, int num_sms);
cudaError_t fp32_launch(const ProjArgs& a, cudaStream_t st);
size_t      fp32_max_partials(int Au, int ncols, int num_sms);   // float2 elements

// FP32 projection for at most 16 distinct cycle frequencies: per-thread register sums and
// a warp-shuffle fold (proj_small.cu).
bool        small_supported(int Au);
ProjPlan    small_plan(int Au, int ncols, int64_t nc, int num_sms);
cudaError_t small_launch(const ProjArgs& a, cudaStream_t st);
size_t      small_max_partials(int Au, int ncols, int num_sms);

// Tensor-core projection, FP16 single pass or BF16 three-product split (proj_tc.cu).
bool        tc_supported(int ncols, int M);
// pair_ctas: CTAs that can run as resident two-CTA clusters (tc_pair_ctas), 0 for the
// one-CTA kernel; tc_launch(pair = true) then runs cta_group::2 pairs.
int         tc_pair_ctas(int precision);
ProjPlan    tc_plan(int Au, int ncols, int64_t nc, int num_sms, int pair_ctas);
cudaError_t tc_launch(const ProjArgs& a, int precision, bool pair, cudaStream_t st);
size_t      tc_max_partials(int Au, int ncols, int num_sms);
int         tc_tile_rows();     // cycle frequencies per work item
int         tc_tile_cols();     // columns per work item
// The uniform grid a_k = -1/2 + k/A (full_mode.cu): fold a pass's lag products modulo A into
// F ([A][ncols], FP64, accumulated), and at read time the A-point DFT of every column into
// out[f][k][l] / N.  A a power of two in [2, 4096].
bool        full_supported(int A);
cudaError_t full_fold(const ProjArgs& a, int A, double2* F, cudaStream_t st);
cudaError_t full_read(const double2* F, int A, int ncols, int nF, int L, double inv_n, double2* out, cudaStream_t st);

// Cyclic spectrum (spectrum.cu): S[rows][Q] = R[rows][L] x E[L][Q] in FP64, E[l][q] =
// w(m_l) exp(-j 2 pi (-1/2 + q/Q) m_l) built into E ([L][Q]) on the device (taper 0: w = 1,
// 1: Hann 0.5 + 0.5 cos(pi m / (mmax + 1))).  lags: device array [L].
cudaError_t spectrum(const double2* R, const int32_t* lags, int rows, int L, int Q, int taper, double mmax,
                     double2* E, double2* S, cudaStream_t st);

// Persistent launch over a device list of work items (taken with an atomic counter that
// the caller zeroes before the launch); `grid` CTAs, one per SM.  pair = true: `grid`
// (even) CTAs in two-CTA clusters, each item covering rows u0 .. u0 + 255 (the odd CTA's
// half written at out + out_peer).
cudaError_t tc_launch_items(const TcItem* items, const int* nitems, int* counter, int grid, int precision, bool pair,
                            int* err, cudaStream_t st);

// Sets the calling thread's message returned by cyc_last_error() (cyc_api.cu).
void record_error(const char* msg);

// Helpers (cyc_kernels.cu).
// sums[u][c] += sum_s part[s][u][c]  (FP64)
cudaError_t reduce_partials(const float2* part, int nsplit, int n_uc, double2* sums, cudaStream_t st);
// Windowed streams (cyc_create_window): fold the hop-aligned partials of one pass into the
// pending hop, the ring of the last w completed hops, the running window sum and the FP64
// running sums; every window that completes gets its raw (absolute-phase) sum written to
// slot k % cap of `wout` ([cap][n_uc]).  Split s ends a hop when s * hop + hop - off <= nc.
struct HopArgs {
    const float2* part;
    int           nsplit;
    int           n_uc;
    int64_t       off, nc, hop;
    int           w;                // hops per window
    int64_t       hops0;            // hops completed before this pass
    float2*       ring;             // [w][n_uc] hop sums (FP32)
    float4*       wsum;             // [n_uc] window sum, float-float (re hi, re lo, im hi, im lo)
    float4*       pend;             // [n_uc] hop in progress, float-float
    double2*      sums;             // [n_uc]
    float2*       wout;             // [cap][n_uc] completed window sums (FP32)
    int64_t       cap;
};
cudaError_t fold_hops(const HopArgs& h, cudaStream_t st);
// Windows k0 .. k0 + n - 1 of a windowed stream into out[i][f][a][l]: wout[k % cap][amap[a]]
// [l F + f] times exp(+j 2 pi phi_a (base + k hop) / 2^64) / N (the window-local phase of
// Eq. (impl-corr)).
cudaError_t read_windows(const float2* wout, int64_t cap, int64_t k0, int64_t n, const int32_t* amap,
                         const uint64_t* phi, int F, int A, int L, int Au, int ncols, uint64_t base, int64_t hop,
                         double inv_n, double2* out, cudaStream_t st);
// out[f][a][l] = sums[amap[a]][l * F + f] / n_eff
cudaError_t read_sums(const double2* sums, const int32_t* amap, int F, int A, int L, int ncols,
                      double inv_n, double2* out, cudaStream_t st);

}  // namespace cyc
