// cyc_impl.h -- internal declarations shared by the host API and the kernel files of libcyc.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "../../include/cyc.h"

namespace cyc {

// Bounded device waits give up after this many SM cycles unless the caller sets another
// budget (about one second at 2 GHz).
constexpr long long kDefaultWaitBudget = 2000000000ll;

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
    // tensor-core passes: phi in unit order (order_units) with np pairs, nself values of
    // {0, 1/2}, U units in all
    int             np = 0, nself = 0, U = 0;
    long long       budget = 0;     // SM cycles per bounded wait (0: kDefaultWaitBudget)
    int             withhold = 0;   // test only: the projection leaves one producer arrival out
    // register-sum path only: with `sums` set, the last block of each column group to finish
    // adds the splits' partials to the FP64 running sums (`cnt`: one arrival counter per
    // column group, zero between launches); with tail_keep > 0, x[tail_from, + tail_keep)
    // (and y's) are copied to tail_x (tail_y), the next view's carried head
    double2*        sums = nullptr;
    int*            cnt = nullptr;
    int             replace = 0;    // with sums: write the pass's totals (sums zeroed by a reset)
    int64_t         tail_from = 0, tail_keep = 0;
    float2*         tail_x = nullptr;
    float2*         tail_y = nullptr;
};

// One work item of the tensor-core projection: 128 units of cycle frequencies (up to 256
// distinct a) x 128 columns x an n-range of one stream, run by one pair of CTAs.  Sample n
// of the stream is x[n & xmask] (xmask = ring capacity - 1, or all ones for a linear view
// with x_avail readable samples).  The result for distinct cycle frequency d (row of the
// unit order) and tile column j goes to out[(d - d_lo) * out_stride + j] for c0 + j < ncols.
struct TcItem {
    const float2*   x;
    uint64_t        xmask;
    int64_t         x_avail;
    uint64_t        nbase;      // absolute index of stream sample 0, mod 2^64
    int64_t         n_beg, n_end;
    const uint64_t* phi;        // distinct cycle frequencies in unit order
    const int32_t*  col_lag;
    const int8_t*   col_conj;
    float2*         out;
    int             out_stride;
    int             u0;         // first unit of the tile (a multiple of 128)
    int             d_lo;       // distinct row of the tile's first output
    int             np, nself, U;
    int             c0, ncols, M;
    const float2*   y;          // second input (linear views only) or nullptr: y = x
    int             D;          // offset of the reference sample y[n + D]
};

// Unit order of the distinct cycle frequencies for the tensor-core projection: every a whose
// negative -a (mod 1) is also present forms a pair with it (rows 2k: the one seen first,
// 2k + 1: its negative), then the self-conjugate values 0 and 1/2 (one unit of real weight
// rows), then the rest, one unit each.  A pair costs the same tensor work as one complex
// cycle frequency, because exp(+j 2 pi a n) is the conjugate of exp(-j 2 pi a n) (see
// proj_tc.cu).  phi_u is reordered in place and amap remapped; the result is a pure function
// of the distinct list, so equal lists give equal orders.
struct UnitLayout {
    int np = 0, nself = 0, ns = 0, U = 0;
};

inline UnitLayout order_units(std::vector<uint64_t>& phi_u, std::vector<int32_t>& amap)
{
    const int Au = (int)phi_u.size();
    std::vector<int> where(Au, -1);
    std::vector<std::pair<uint64_t, int>> sorted(Au);
    for (int i = 0; i < Au; ++i) sorted[i] = {phi_u[i], i};
    std::sort(sorted.begin(), sorted.end());
    auto find = [&](uint64_t v) -> int {
        auto itv = std::lower_bound(sorted.begin(), sorted.end(), std::make_pair(v, -1));
        return (itv != sorted.end() && itv->first == v) ? itv->second : -1;
    };
    std::vector<int> pairs, selfs, singles;
    std::vector<char> used(Au, 0);
    for (int i = 0; i < Au; ++i) {
        if (used[i]) continue;
        const uint64_t v = phi_u[i];
        if (v == 0 || v == (1ull << 63)) {
            selfs.push_back(i);
            used[i] = 1;
            continue;
        }
        const int j = find(~v + 1ull);
        if (j >= 0 && !used[j]) {
            pairs.push_back(i);
            pairs.push_back(j);
            used[i] = used[j] = 1;
        } else {
            singles.push_back(i);
            used[i] = 1;
        }
    }
    std::vector<int> order;
    order.reserve(Au);
    order.insert(order.end(), pairs.begin(), pairs.end());
    order.insert(order.end(), selfs.begin(), selfs.end());
    order.insert(order.end(), singles.begin(), singles.end());
    std::vector<uint64_t> nphi(Au);
    for (int k = 0; k < Au; ++k) {
        nphi[k] = phi_u[order[k]];
        where[order[k]] = k;
    }
    phi_u.swap(nphi);
    for (auto& a : amap) a = where[a];
    UnitLayout L;
    L.np = (int)pairs.size() / 2;
    L.nself = (int)selfs.size();
    L.ns = (int)singles.size();
    L.U = L.np + (L.nself > 0 ? 1 : 0) + L.ns;
    return L;
}

// Distinct row (in unit order) of output h (0, 1) of unit k, or -1: a pair gives rows 2k
// and 2k + 1, the real unit rows 2 np .. 2 np + nself - 1, a single unit one row.
__host__ __device__ inline int unit_row(int k, int h, int np, int nself, int U)
{
    if (k < 0 || k >= U) return -1;
    if (k < np) return 2 * k + h;
    const int nr = nself > 0 ? 1 : 0;
    if (k < np + nr) return h < nself ? 2 * np + h : -1;
    return h == 0 ? 2 * np + nself + (k - np - nr) : -1;
}

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
int         small_groups(int Au, int ncols);   // column groups (blocks per split) of the grid
cudaError_t small_launch(const ProjArgs& a, cudaStream_t st);
size_t      small_max_partials(int Au, int ncols, int num_sms);

// Tensor-core projection, FP16 single pass or BF16 three-product split (proj_tc.cu), on
// pairs of CTAs (two-CTA clusters issuing cta_group::2 MMAs).
bool        tc_supported(int ncols, int M);
// CTAs that can run as resident two-CTA clusters (0: cluster launches unavailable, and the
// tensor-core precisions with them).
int         tc_pair_ctas(int precision);
ProjPlan    tc_plan(int U, int Au, int ncols, int64_t nc, int num_sms, int pair_ctas);
cudaError_t tc_launch(const ProjArgs& a, int precision, cudaStream_t st);
size_t      tc_max_partials(int U, int Au, int ncols, int num_sms);
int         tc_pair_units();    // units per work item (128)
int         tc_tile_rows();     // rows of an item's partial tile (2 outputs per unit: 256)
int         tc_tile_cols();     // columns per work item (128)
// The uniform grid a_k = -1/2 + k/A (full_mode.cu): fold a pass's lag products modulo A into
// the fold ([ncols][A] float-float, accumulated), and at read time the A-point DFT of every
// column into out[f][k][l] / N.  A a power of two in [2, 4096].
//
// One pass of a Full-mode stream.  Its view is the carried tail followed by one or more
// chunks, each in a buffer of its own (a chunk may be the caller's device memory, 8-byte
// aligned): source s covers view samples [start[s], start[s + 1]).  Fold sample v is view
// sample off + v.  Term i < nc adds x[v + m] c_f(y[v + D]) (v = i, m the shifted lag) to
// residue (i + base_mod) mod A.  The same launch copies the view's last `keep` samples to nx
// (and ny for two inputs) for the next pass.  The view stays below 2^30 samples.
constexpr int kFoldSrc = 17;         // the tail and up to 16 chunks
struct FoldArgs {
    int nsrc = 0;
    int32_t start[kFoldSrc + 1] = {};
    const float2* sx[kFoldSrc] = {};
    const float2* sy[kFoldSrc] = {}; // == sx for one input
    int64_t off = 0;
    int64_t nc = 0;
    int D = 0;                       // M^-
    int A = 0;
    uint32_t base_mod = 0;
    const int32_t* sl = nullptr;     // [L] shifted lags m + M^-, ascending
    const int32_t* perm = nullptr;   // [L] the lag index of each sorted position
    int L = 0, F = 0;
    int fV = -1, fJ = -1;            // form index of x conj(y) and of x y (-1: not kept)
    int xl = 0;                      // full_row_samples(sl, L)
    bool consecutive = false;        // full_lags_consecutive(sl, L)
    float4* fold = nullptr;          // [L F][A]
    float2* nx = nullptr;
    float2* ny = nullptr;            // null for one input
    int64_t keep = 0;
};
// Windowed Full mode: windows k0 .. k0 + nwin - 1, window k0 + w reading view samples
// vbase0 + w hop + n (n < N, plus the lags); each lag's N-point FFT per form, divided by N,
// goes to ring slot (k mod cap) as [ncols][N] FP32.
struct FullWinArgs {
    int64_t k0 = 0, hop = 0, vbase0 = 0, cap = 0;
    int N = 0, logN = 0, ncols = 0;
    const int32_t* col_lag = nullptr;    // [ncols] shifted lag of column l F + f
    const float2* tw = nullptr;          // [N] FFT twiddles by span: [h + p] = exp(-j pi p / h), FP32
    float2* ring = nullptr;              // [cap][ncols][N]
};
cudaError_t full_windows(const FoldArgs& a, const FullWinArgs& w, int nwin, cudaStream_t st);
// out [n][F][N][L] FP64 from ring slots k0 .. k0 + n - 1
cudaError_t full_read_windows(const float2* ring, int64_t cap, int64_t k0, int64_t n, int N, int F, int L,
                              double2* out, cudaStream_t st);
bool        full_supported(int A);
int         full_row_samples(const int32_t* sorted_shifted_lags, int L);   // x samples per staged row
bool        full_lags_consecutive(const int32_t* sorted_shifted_lags, int L);  // each 16-lag tile m, m + 1, ...
cudaError_t full_fold(const FoldArgs& f, cudaStream_t st);
cudaError_t full_read(const double2* F, int A, int ncols, int nF, int L, double inv_n, double2* out, cudaStream_t st);

// Cyclic spectrum (spectrum.cu): S[rows][Q] = R[rows][L] x E[L][Q] in FP64, E[l][q] =
// w(m_l) exp(-j 2 pi (-1/2 + q/Q) m_l) built into E ([L][Q]) on the device (taper 0: w = 1,
// 1: Hann 0.5 + 0.5 cos(pi m / (mmax + 1))).  lags: device array [L].
cudaError_t spectrum(const double2* R, const int32_t* lags, int rows, int L, int Q, int taper, double mmax,
                     double2* E, double2* S, cudaStream_t st);

// Cycle-frequency detection (detect.cu): per form and cycle frequency of R [F][A][L] (FP64),
// the statistic s = max over lags |R|^2 (0 for form conv_f where dc[a]), the median of s over
// the offsets +-2 .. +-win (circular), and flags (bit 0 detected: s > kappa * median and a
// local maximum; bit 1 local maximum), ratio = s / median (may be null), count of detections.
// Scratch s [F][A].  win in [2, 32].
bool        detect_supported(int win);
cudaError_t detect(const double2* R, int F, int A, int L, const uint8_t* dc, int conv_f, int win, double kappa,
                   double* s, uint8_t* flags, float* ratio, int* count, cudaStream_t st);

// Persistent launch over a device list of work items (taken with an atomic counter that
// the caller zeroes before the launch); `grid` (even) CTAs in two-CTA clusters, one per SM.
cudaError_t tc_launch_items(const TcItem* items, const int* nitems, int* counter, int grid, int precision, int* err,
                            long long budget, cudaStream_t st);

// Device allocation of the stream and server set-up paths.  Test hook: with the environment
// variable CYC_TEST_FAIL_ALLOC=k at the start of a cyc_create_* or cyc_server_open call, the
// k-th allocation of that call fails as if the device were out of memory (nothing is
// allocated), so that the tests can check that a failed admission leaves nothing behind.
void        test_alloc_arm();       // reads the hook at the start of a set-up call
cudaError_t dev_malloc(void** p, size_t bytes);

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
// With err_dst set, the launch also copies the status word *err_src there (a page-locked
// host word, so that a host read needs no copy besides the one into `out`).
cudaError_t read_sums(const double2* sums, const int32_t* amap, int F, int A, int L, int ncols,
                      double inv_n, double2* out, cudaStream_t st, const int* err_src = nullptr,
                      int* err_dst = nullptr);

}  // namespace cyc
