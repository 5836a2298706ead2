// cyc_api.cu -- host side of libcyc: stream state, ingest with the carried tail, the
// projection passes, FP64 running sums, read-out, save/load.  Declared in include/cyc.h.
#include <math.h>
#include <stdlib.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <set>

#include "cyc_impl.h"

using namespace cyc;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? CYC_ENOMEM : CYC_ECUDA,         \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// Makes the handle's device current for the duration of an entry point.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

constexpr int64_t kDefaultChunk = 1 << 20;
constexpr int64_t kMaxChunk = 1ll << 28;
constexpr int32_t kMaxLag = 1 << 20;
constexpr int kStagePad = 256;      // zeroed samples after every staging buffer
constexpr int kWinSplits = 64;      // hop-aligned partials per pass of a windowed tensor-core stream
constexpr size_t kWinPartBytes = 64u << 20;   // FP32 windowed streams: partials of a pass, at most
constexpr uint32_t kBlobVersion = 3;       // 3: tensor-core streams keep their sums in unit order

// a (cycles/sample) -> round(a * 2^64) mod 2^64, exactly.  a = m * 2^e with m the 53-bit
// integer significand, so a * 2^64 = m * 2^(e+64): a left shift (bits beyond 2^64 are
// whole cycles and drop out) or a rounded right shift, then two's-complement negation
// for a < 0.  (a - floor(a) would not do: for negative a it rounds.)  The result is off
// from a by at most 2^-65 cycles/sample, and only when a has bits below 2^-64.
uint64_t alpha_to_phi(double a)
{
    if (a == 0.0) return 0;
    int ex = 0;
    double fr = frexp(fabs(a), &ex);                  // |a| = fr * 2^ex, fr in [0.5, 1)
    uint64_t m = (uint64_t)ldexp(fr, 53);             // exact, < 2^53
    int sh = ex - 53 + 64;
    uint64_t phi;
    if (sh >= 64) phi = 0;
    else if (sh >= 0) phi = m << sh;
    else if (sh < -54) phi = 0;
    else phi = (m + (1ull << (-sh - 1))) >> (-sh);
    return a < 0 ? (~phi + 1ull) : phi;
}

uint64_t fnv1a(uint64_t h, const void* p, size_t n)
{
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    return h;
}

struct BlobHeader {
    char     magic[8];
    uint32_t version;
    int32_t  F, L, A, Au;
    int32_t  conj_flag;
    int64_t  n0, T, n_eff, held;
    uint64_t fingerprint;
};

}  // namespace

void cyc::record_error(const char* msg) { g_err = msg; }

namespace {
thread_local int g_alloc_fail_at = 0, g_alloc_count = 0;
}

void cyc::test_alloc_arm()
{
    const char* ev = getenv("CYC_TEST_FAIL_ALLOC");
    g_alloc_fail_at = ev ? atoi(ev) : 0;
    g_alloc_count = 0;
}

cudaError_t cyc::dev_malloc(void** p, size_t bytes)
{
    if (g_alloc_fail_at > 0 && ++g_alloc_count == g_alloc_fail_at) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

struct cyc_stream {
    int device = 0;
    cudaStream_t st = nullptr;
    int num_sms = 1;
    int pair_ctas = 0;              // > 0: tensor-core passes run as two-CTA pairs
    int precision = CYC_P_FP32;
    int conj_flag = 0;
    int F = 0;
    int forms[2] = {0, 0};
    std::vector<int32_t> lags;
    int L = 0;
    int32_t M = 0;                  // lag span M^- + M^+: samples carried from push to push
    int32_t Mneg = 0;               // M^- = max(0, -min lag): window offset of Eq. (impl-corr)
    bool cross = false;             // two inputs (cyc_create_xy / cyc_push_xy)
    // uniform grid a_k = -1/2 + k/A (cyc_create_full): sums holds the lag products folded mod A
    bool full = false;
    int32_t* d_fsl = nullptr;       // Full mode: shifted lags in ascending order
    int32_t* d_fperm = nullptr;     // Full mode: the lag index of each sorted position
    int fxl = 0;                    // Full mode: x samples per staged row of the fold
    bool fcons = false;             // Full mode: each 16-lag tile of sorted lags is consecutive
    // Full mode: pushes not folded yet (one launch folds them all): x, y and length; host
    // chunks and misaligned device chunks are copied into stage[cur] after the tail first
    struct Pend { const float2* x; const float2* y; int64_t c; };
    std::vector<Pend> fpend;
    int64_t fpend_total = 0;
    bool fpend_host = false;        // a host copy on the copy stream feeds the pending fold
    float2* d_ftw = nullptr;        // windowed Full mode: FFT twiddles by span, [h + p] = exp(-j pi p / h)
    int64_t carry = 0;              // samples carried from pass to pass (M; A + M - 1 for Full windows)
    // windowed output (cyc_create_window): window k covers committed n in [k hop, k hop + N)
    bool win = false;
    int64_t win_len = 0, hop = 0, win_cap = 0;
    int win_w = 0;                  // hops per window
    int win_splits = 0;             // hop-aligned partials per pass (one pass covers win_splits - 1 hops)
    int64_t hops = 0;               // hops completed
    int64_t win_made = 0, win_read = 0;
    float2* w_ring = nullptr;       // [win_w][Au][ncols] the last win_w completed hops (FP32)
    float4* w_sum = nullptr;        // [Au][ncols] sum of those (float-float: re hi, re lo, im hi, im lo)
    float4* w_pend = nullptr;       // [Au][ncols] the hop in progress (float-float)
    float2* w_out = nullptr;        // [win_cap][Au][ncols] raw sums of completed, unread windows (FP32)
    // cyclic spectra (cyc_read_spectrum), allocated on first use
    int32_t* d_lags = nullptr;      // the signed lags [L]
    double2* sp_E = nullptr;        // DFT matrix [L][sp_Q]
    double2* sp_S = nullptr;        // spectrum [F][A][sp_Q] for host outputs
    int sp_Q = 0;
    // cycle-frequency detection (cyc_detect), allocated on first use
    double* dt_s = nullptr;         // statistic [F][A]
    uint8_t* dt_flags = nullptr;    // [F][A] for host outputs
    float* dt_ratio = nullptr;      // [F][A] for host outputs
    uint8_t* dt_dc = nullptr;       // [A] 1 where the conventional a = 0 entry is left out
    int* dt_count = nullptr;
    std::vector<double> alphas;
    int A = 0;
    std::vector<uint64_t> phi_u;
    std::vector<int32_t> amap;
    int Au = 0;
    UnitLayout units;               // tensor-core streams: phi_u in unit order (order_units)
    int ncols = 0;
    long long wait_budget = 0;      // SM cycles per bounded device wait (0: the default)
    int withhold = 0;               // test only (CYC_TEST_WITHHOLD_ARRIVAL=1 at creation)
    int64_t n0 = 0, T = 0, n_eff = 0, held = 0, max_chunk = kDefaultChunk;
    uint64_t fingerprint = 0;
    // device state
    float2* stage[2] = {nullptr, nullptr};
    float2* stage_y[2] = {nullptr, nullptr};   // second input, same layout (cross streams)
    int cur = 0;
    double2* sums = nullptr;
    uint64_t* d_phi = nullptr;
    int32_t* d_amap = nullptr;
    int32_t* d_col_lag = nullptr;
    int8_t* d_col_conj = nullptr;
    float2* part = nullptr;
    size_t part_elems = 0;
    double2* d_out = nullptr;
    int* d_err = nullptr;       // set by a kernel whose bounded wait gave up
    int* h_err = nullptr;       // page-locked copy, read after a stream synchronisation
    int* h_err_dev = nullptr;   // its address on the device (a read kernel writes it directly)
    void* h_stage = nullptr;    // page-locked landing buffer of cyc_read into host memory (first use)
    void* h_stage_dev = nullptr;   // its address on the device (nullptr: copied into it instead)
    int* d_cnt = nullptr;       // register-sum passes: arrival counter per column group
    bool zero_sums = false;     // a reset's zeroing of the sums is still to be done (see cyc_reset)
    // host pushes: chunks are copied on a stream of their own, so that the copy of one pass
    // overlaps the projection of the previous one (created at the first host push)
    cudaStream_t xst = nullptr;
    cudaEvent_t ev_copied = nullptr;        // the current pass's chunk has landed
    cudaEvent_t ev_read[2] = {nullptr, nullptr};   // the last pass that viewed stage[b] is done
    // profiling
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending, ev_free;
    double prof_ms = 0.0;
    int64_t prof_launches = 0, kernel_launches = 0;

    void free_events()
    {
        for (auto& e : ev_pending) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
        for (auto& e : ev_free) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
        ev_pending.clear();
        ev_free.clear();
    }

    void free_all()
    {
        free_events();
        if (xst) { cudaStreamSynchronize(xst); cudaStreamDestroy(xst); xst = nullptr; }
        if (ev_copied) { cudaEventDestroy(ev_copied); ev_copied = nullptr; }
        for (auto& e : ev_read)
            if (e) { cudaEventDestroy(e); e = nullptr; }
        void* ps[] = {stage[0], stage[1], stage_y[0], stage_y[1], sums, d_phi, d_amap, d_col_lag, d_col_conj,
                      part, d_out, d_err, w_ring, w_sum, w_pend, w_out, d_lags, sp_E, sp_S,
                      dt_s, dt_flags, dt_ratio, dt_dc, dt_count, d_fsl, d_fperm, d_ftw, d_cnt};
        for (void* p : ps)
            if (p) cudaFree(p);
        if (h_err) cudaFreeHost(h_err);
        if (h_stage) cudaFreeHost(h_stage);
        h_stage = nullptr;
        h_stage_dev = nullptr;
        h_err_dev = nullptr;
        d_cnt = nullptr;
        stage[0] = stage[1] = stage_y[0] = stage_y[1] = nullptr;
        sums = nullptr; d_phi = nullptr; d_amap = nullptr; d_col_lag = nullptr;
        d_col_conj = nullptr; part = nullptr; d_out = nullptr; d_err = nullptr; h_err = nullptr;
        w_ring = w_out = nullptr;
        w_sum = w_pend = nullptr;
        d_lags = nullptr;
        sp_E = sp_S = nullptr;
        sp_Q = 0;
        dt_s = nullptr; dt_flags = nullptr; dt_ratio = nullptr; dt_dc = nullptr; dt_count = nullptr;
        d_fsl = d_fperm = nullptr;
        d_ftw = nullptr;
    }
};

namespace {

int check_params(const cyc_params* p)
{
    if (!p) return fail(CYC_EINVAL, "cyc_create_ex: params is NULL");
    if (!p->lags || p->nlags <= 0) return fail(CYC_EINVAL, "lag list is empty");
    if (!p->alphas || p->nalphas <= 0) return fail(CYC_EINVAL, "cycle-frequency list is empty");
    int32_t lo = 0, hi = 0;
    for (int i = 0; i < p->nlags; ++i) {
        if (p->lags[i] < -kMaxLag || p->lags[i] > kMaxLag)
            return fail(CYC_EINVAL, "lag %d (%d) is outside [-%d, %d]", i, p->lags[i], kMaxLag, kMaxLag);
        lo = p->lags[i] < lo ? p->lags[i] : lo;
        hi = p->lags[i] > hi ? p->lags[i] : hi;
    }
    if ((int64_t)hi - lo > kMaxLag) return fail(CYC_EINVAL, "the lags span more than %d samples", kMaxLag);
    for (int i = 0; i < p->nalphas; ++i)
        if (!isfinite(p->alphas[i])) return fail(CYC_EINVAL, "cycle frequency %d is not finite", i);
    if (p->conj_flag < 1 || p->conj_flag > 3) return fail(CYC_EINVAL, "conj_flag must be 1, 2 or 3");
    if (p->precision < CYC_P_FP32 || p->precision > CYC_P_BF16X3)
        return fail(CYC_EINVAL, "unknown precision %d", p->precision);
    if (p->max_chunk < 0 || p->max_chunk > kMaxChunk)
        return fail(CYC_EINVAL, "max_chunk must be in [0, 2^28]");
    if ((int64_t)p->nlags * 2 > (1 << 24) || (int64_t)p->nalphas > (1 << 24))
        return fail(CYC_EINVAL, "too many lags or cycle frequencies");
    return CYC_OK;
}

int alloc_state(cyc_stream* s)
{
    s->carry = s->full && s->win ? (int64_t)s->A + s->M - 1 : s->M;
    size_t stage_n = (size_t)(s->carry + s->max_chunk + kStagePad);
    for (int b = 0; b < 2; ++b) {
        CK(dev_malloc((void**)&s->stage[b], stage_n * sizeof(float2)));
        CK(cudaMemset(s->stage[b], 0, stage_n * sizeof(float2)));
        if (s->cross) {
            CK(dev_malloc((void**)&s->stage_y[b], stage_n * sizeof(float2)));
            CK(cudaMemset(s->stage_y[b], 0, stage_n * sizeof(float2)));
        }
    }
    CK(dev_malloc((void**)&s->sums, (size_t)s->Au * s->ncols * sizeof(double2)));
    CK(cudaMemset(s->sums, 0, (size_t)s->Au * s->ncols * sizeof(double2)));
    CK(dev_malloc((void**)&s->d_phi, s->Au * sizeof(uint64_t)));
    CK(cudaMemcpy(s->d_phi, s->phi_u.data(), s->Au * sizeof(uint64_t), cudaMemcpyHostToDevice));
    CK(dev_malloc((void**)&s->d_amap, s->A * sizeof(int32_t)));
    CK(cudaMemcpy(s->d_amap, s->amap.data(), s->A * sizeof(int32_t), cudaMemcpyHostToDevice));
    std::vector<int32_t> cl(s->ncols);
    std::vector<int8_t> cc(s->ncols);
    // column c = lag index * F + form index: both forms of a lag are neighbours
    for (int f = 0; f < s->F; ++f)
        for (int l = 0; l < s->L; ++l) {
            cl[l * s->F + f] = s->lags[l] + s->Mneg;        // shifted lag m + M^- >= 0
            cc[l * s->F + f] = s->forms[f] == CYC_CONJ ? 1 : 0;
        }
    CK(dev_malloc((void**)&s->d_col_lag, s->ncols * sizeof(int32_t)));
    CK(cudaMemcpy(s->d_col_lag, cl.data(), s->ncols * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(dev_malloc((void**)&s->d_col_conj, s->ncols * sizeof(int8_t)));
    CK(cudaMemcpy(s->d_col_conj, cc.data(), s->ncols * sizeof(int8_t), cudaMemcpyHostToDevice));
    if (s->full) {                    // the fold takes the lags in ascending order, 16 per tile
        std::vector<int32_t> perm(s->L), sl(s->L);
        for (int l = 0; l < s->L; ++l) perm[l] = l;
        std::stable_sort(perm.begin(), perm.end(), [&](int32_t u, int32_t v) { return s->lags[u] < s->lags[v]; });
        for (int p = 0; p < s->L; ++p) sl[p] = s->lags[perm[p]] + s->Mneg;
        s->fxl = full_row_samples(sl.data(), s->L);
        s->fcons = full_lags_consecutive(sl.data(), s->L);
        CK(dev_malloc((void**)&s->d_fsl, s->L * sizeof(int32_t)));
        CK(cudaMemcpy(s->d_fsl, sl.data(), s->L * sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(dev_malloc((void**)&s->d_fperm, s->L * sizeof(int32_t)));
        CK(cudaMemcpy(s->d_fperm, perm.data(), s->L * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    if (s->precision != CYC_P_FP32)
        s->part_elems = tc_max_partials(s->units.U, s->Au, s->ncols, s->num_sms);
    else if (small_supported(s->Au)) {
        s->part_elems = small_max_partials(s->Au, s->ncols, s->num_sms);
        const int ng = small_groups(s->Au, s->ncols);
        CK(dev_malloc((void**)&s->d_cnt, ng * sizeof(int)));
        CK(cudaMemset(s->d_cnt, 0, ng * sizeof(int)));
    }
    else
        s->part_elems = fp32_max_partials(s->Au, s->ncols, s->num_sms);
    if (s->win && !s->full) {
        // FP32 streams: as many hop partials per pass as 64 MB holds (short hops then cost few
        // launches); tensor-core streams: kWinSplits
        const size_t nuc = (size_t)s->Au * s->ncols;
        size_t ws = kWinSplits;
        if (s->precision == CYC_P_FP32) {
            ws = kWinPartBytes / (nuc * sizeof(float2));
            ws = ws < (size_t)kWinSplits ? (size_t)kWinSplits : ws > 65535 ? 65535 : ws;
        }
        s->win_splits = (int)ws;
        if (s->part_elems < ws * nuc) s->part_elems = ws * nuc;
    }
    CK(dev_malloc((void**)&s->part, s->part_elems * sizeof(float2)));
    if (s->win && s->full) {          // Full-mode windows: the ring of spectra and the twiddles
        CK(dev_malloc((void**)&s->w_out, (size_t)s->win_cap * s->ncols * s->A * sizeof(float2)));
        // the FFT's twiddles by butterfly span: tw[h + p] = exp(-j pi p / h) = exp(-j 2 pi
        // (p A / 2h) / A) for h = 1, 2, ..., A/2 and p < h (tw[0] unused)
        std::vector<float2> tw(s->A);
        tw[0] = make_float2(1.f, 0.f);
        for (int h = 1; h < s->A; h <<= 1)
            for (int q = 0; q < h; ++q) {
                const double ang = -2.0 * M_PI * (double)(q * (s->A / (2 * h))) / (double)s->A;
                tw[h + q] = make_float2((float)cos(ang), (float)sin(ang));
            }
        CK(dev_malloc((void**)&s->d_ftw, tw.size() * sizeof(float2)));
        CK(cudaMemcpy(s->d_ftw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    } else if (s->win) {
        const size_t nuc = (size_t)s->Au * s->ncols;
        CK(dev_malloc((void**)&s->w_ring, (size_t)s->win_w * nuc * sizeof(float2)));
        CK(dev_malloc((void**)&s->w_sum, nuc * sizeof(float4)));
        CK(dev_malloc((void**)&s->w_pend, nuc * sizeof(float4)));
        CK(dev_malloc((void**)&s->w_out, (size_t)s->win_cap * nuc * sizeof(float2)));
        CK(cudaMemset(s->w_sum, 0, nuc * sizeof(float4)));
        CK(cudaMemset(s->w_pend, 0, nuc * sizeof(float4)));
    }
    CK(dev_malloc((void**)&s->d_out, (size_t)s->F * s->A * s->L * sizeof(double2)));
    CK(dev_malloc((void**)&s->d_err, sizeof(int)));
    CK(cudaMemset(s->d_err, 0, sizeof(int)));
    CK(cudaMallocHost(&s->h_err, sizeof(int)));
    *s->h_err = 0;
    if (cudaHostGetDevicePointer((void**)&s->h_err_dev, s->h_err, 0) != cudaSuccess) {
        cudaGetLastError();
        s->h_err_dev = nullptr;
    }
    return CYC_OK;
}

// One device pass over view = stage[cur][0 .. held + c): nc committed terms.  The view's
// samples [tail_from, + keep) are the next view's head: *tail_done says whether the pass
// copied them (the register-sum kernel does) or the caller must.
int project(cyc_stream* s, int64_t nc, int64_t tail_from, int64_t keep, bool* tail_done)
{
    *tail_done = false;
    ProjArgs a;
    a.x = s->stage[s->cur];
    a.nc = nc;
    a.nbase = (uint64_t)s->n0 + (uint64_t)s->n_eff + (uint64_t)s->Mneg;   // index of y[M^-]
    a.phi = s->d_phi;
    a.Au = s->Au;
    a.col_lag = s->d_col_lag;
    a.col_conj = s->d_col_conj;
    a.ncols = s->ncols;
    a.part = s->part;
    a.err = s->d_err;
    a.M = s->M;
    a.x_avail = (s->M + s->max_chunk + kStagePad) & ~(int64_t)1;
    a.y = s->cross ? s->stage_y[s->cur] : nullptr;
    a.D = s->Mneg;
    a.nforms = s->F;
    a.np = s->units.np;
    a.nself = s->units.nself;
    a.U = s->units.U;
    a.budget = s->wait_budget;
    a.withhold = s->withhold;
    // FP32 with a handful of distinct cycle frequencies: register sums + warp shuffles
    const bool small = s->precision == CYC_P_FP32 && small_supported(s->Au);
    ProjPlan pl = s->precision != CYC_P_FP32 ? tc_plan(s->units.U, s->Au, s->ncols, nc, s->num_sms, s->pair_ctas)
                  : small                    ? small_plan(s->Au, s->ncols, nc, s->num_sms)
                                             : fp32_plan(s->Au, s->ncols, nc, s->num_sms);
    if (s->win) {                     // one split per hop (the first and last may be partial)
        a.split_off = s->n_eff % s->hop;
        pl.split_len = s->hop;
        pl.nsplit = (int)((nc + a.split_off + s->hop - 1) / s->hop);
    }
    a.nsplit = pl.nsplit;
    a.split_len = pl.split_len;
    if ((size_t)pl.nsplit * s->Au * s->ncols > s->part_elems)
        return fail(CYC_ECUDA, "internal: partial buffer too small (%d splits)", pl.nsplit);
    if (small) {                      // one launch: the FP64 update and the tail copy included
        if (!s->win) {
            a.sums = s->sums;
            a.cnt = s->d_cnt;
            a.replace = s->zero_sums ? 1 : 0;   // a reset's zeroing folded into this update
            s->zero_sums = false;
        }
        if (keep > 0) {
            a.tail_from = tail_from;
            a.tail_keep = keep;
            a.tail_x = s->stage[s->cur ^ 1];
            a.tail_y = s->cross ? s->stage_y[s->cur ^ 1] : nullptr;
            *tail_done = true;
        }
    }
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (s->prof) {
        if (!s->ev_free.empty()) {
            ev = s->ev_free.back();
            s->ev_free.pop_back();
        } else {
            CK(cudaEventCreate(&ev.first));
            CK(cudaEventCreate(&ev.second));
        }
        CK(cudaEventRecord(ev.first, s->st));
    }
    CK(s->precision != CYC_P_FP32 ? tc_launch(a, s->precision, s->st)
       : small                    ? small_launch(a, s->st)
                                  : fp32_launch(a, s->st));
    if (s->prof) {
        CK(cudaEventRecord(ev.second, s->st));
        s->ev_pending.push_back(ev);
    }
    s->prof_launches++;
    if (s->win) {
        HopArgs h;
        h.part = s->part;
        h.nsplit = pl.nsplit;
        h.n_uc = s->Au * s->ncols;
        h.off = a.split_off;
        h.nc = nc;
        h.hop = s->hop;
        h.w = s->win_w;
        h.hops0 = s->hops;
        h.ring = s->w_ring;
        h.wsum = s->w_sum;
        h.pend = s->w_pend;
        h.sums = s->sums;
        h.wout = s->w_out;
        h.cap = s->win_cap;
        CK(fold_hops(h, s->st));
        const int64_t done = (s->n_eff + nc) / s->hop;           // hops complete after this pass
        s->hops = done;
        s->win_made = done >= s->win_w ? done - s->win_w + 1 : 0;
        s->kernel_launches++;
    } else if (!a.sums) {
        CK(reduce_partials(s->part, pl.nsplit, s->Au * s->ncols, s->sums, s->st));
        s->kernel_launches++;
    }
    s->kernel_launches++;
    return CYC_OK;
}

// Windows complete after T samples: window k needs samples up to k hop + win_len + M - 1.
int64_t windows_made(const cyc_stream* s, int64_t T)
{
    return T - s->M >= s->win_len ? (T - s->M - s->win_len) / s->hop + 1 : 0;
}

// Fold the pending pushes of a Full-mode stream in one launch: the view is the carried tail
// stage[cur][0, held) followed by the pending chunks; the same launch writes the view's last
// `keep` samples to stage[cur ^ 1] as the next tail.
int full_flush(cyc_stream* s)
{
    if (s->fpend.empty()) return CYC_OK;
    const int64_t c = s->fpend_total;
    const int64_t held_f = s->T < s->M ? s->T : s->M;       // the tail the running sums view
    int64_t nc = held_f + c - s->M;
    if (nc < 0) nc = 0;
    const int64_t T2 = s->T + c;
    const int64_t keep = T2 < s->carry ? T2 : s->carry;
    FoldArgs f;
    f.nsrc = 1 + (int)s->fpend.size();
    f.start[0] = 0;
    f.sx[0] = s->stage[s->cur];
    f.sy[0] = s->cross ? s->stage_y[s->cur] : f.sx[0];
    int64_t pos = s->held;
    for (size_t k = 0; k < s->fpend.size(); ++k) {
        f.start[k + 1] = (int32_t)pos;
        f.sx[k + 1] = s->fpend[k].x;
        f.sy[k + 1] = s->cross ? s->fpend[k].y : s->fpend[k].x;
        pos += s->fpend[k].c;
    }
    f.start[f.nsrc] = (int32_t)pos;
    f.off = s->held - held_f;
    f.nc = nc;
    f.D = s->Mneg;
    f.A = s->Au;
    f.base_mod = (uint32_t)(((uint64_t)s->n0 + (uint64_t)s->n_eff + (uint64_t)s->Mneg) & (uint64_t)(s->Au - 1));
    f.sl = s->d_fsl;
    f.perm = s->d_fperm;
    f.L = s->L;
    f.F = s->F;
    for (int k = 0; k < s->F; ++k) {
        if (s->forms[k] == CYC_CONV) f.fV = k;
        if (s->forms[k] == CYC_CONJ) f.fJ = k;
    }
    f.xl = s->fxl;
    f.consecutive = s->fcons;
    f.fold = reinterpret_cast<float4*>(s->sums);
    f.nx = s->stage[s->cur ^ 1];
    f.ny = s->cross ? s->stage_y[s->cur ^ 1] : nullptr;
    f.keep = keep;
    s->fpend.clear();
    s->fpend_total = 0;
    if (s->fpend_host) {
        CK(cudaStreamWaitEvent(s->st, s->ev_copied, 0));
        s->fpend_host = false;
    }
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (s->prof && nc > 0) {
        if (!s->ev_free.empty()) {
            ev = s->ev_free.back();
            s->ev_free.pop_back();
        } else {
            CK(cudaEventCreate(&ev.first));
            CK(cudaEventCreate(&ev.second));
        }
        CK(cudaEventRecord(ev.first, s->st));
    }
    CK(full_fold(f, s->st));
    if (ev.first) {
        CK(cudaEventRecord(ev.second, s->st));
        s->ev_pending.push_back(ev);
        s->prof_launches++;
    }
    if (nc > 0 || keep > 0) s->kernel_launches += 1;
    if (s->win) {                     // Full-mode windows completed by this pass, from the same view
        const int64_t made2 = windows_made(s, T2);
        if (made2 > s->win_made) {
            FullWinArgs w;
            w.k0 = s->win_made;
            w.hop = s->hop;
            w.vbase0 = w.k0 * s->hop - (s->T - s->held);        // view sample of window k0's first y
            w.cap = s->win_cap;
            w.N = s->A;
            while ((1 << w.logN) < w.N) ++w.logN;
            w.ncols = s->ncols;
            w.col_lag = s->d_col_lag;
            w.tw = s->d_ftw;
            w.ring = s->w_out;
            CK(full_windows(f, w, (int)(made2 - s->win_made), s->st));
            s->kernel_launches += 1;
            s->win_made = made2;
        }
    }
    if (s->xst) CK(cudaEventRecord(s->ev_read[s->cur], s->st));     // this view is free again
    s->n_eff += nc;
    s->T = T2;
    s->cur ^= 1;
    s->held = keep;
    return CYC_OK;
}

// Queue a Full-mode push: 8-byte aligned device chunks are read where they are; host chunks
// and misaligned device chunks are copied into stage[cur] behind the tail and the chunks
// already queued (host chunks on the copy stream).  The pending chunks are folded in one
// launch when the next would not fit (16 chunks, max_chunk samples) and before anything
// reads the stream's state.
int full_push(cyc_stream* s, const float2* src, const float2* ysrc, int64_t nsamples, bool on_device)
{
    int64_t left = nsamples;
    while (left > 0) {
        int64_t c = left < s->max_chunk ? left : s->max_chunk;
        if ((int)s->fpend.size() + 1 >= kFoldSrc || s->fpend_total + c > s->max_chunk) {
            int rc = full_flush(s);
            if (rc) return rc;
        }
        const bool direct = on_device && ((uintptr_t)src & 7) == 0 && (!s->cross || ((uintptr_t)ysrc & 7) == 0);
        if (direct) {
            s->fpend.push_back({src, ysrc, c});
        } else {
            float2* dx = s->stage[s->cur] + s->held + s->fpend_total;
            float2* dy = s->cross ? s->stage_y[s->cur] + s->held + s->fpend_total : nullptr;
            cudaStream_t cs = on_device ? s->st : s->xst;
            if (!on_device) CK(cudaStreamWaitEvent(cs, s->ev_read[s->cur], 0));
            CK(cudaMemcpyAsync(dx, src, (size_t)c * sizeof(float2), cudaMemcpyDefault, cs));
            if (s->cross) CK(cudaMemcpyAsync(dy, ysrc, (size_t)c * sizeof(float2), cudaMemcpyDefault, cs));
            if (!on_device) {
                CK(cudaEventRecord(s->ev_copied, cs));
                s->fpend_host = true;
            }
            s->fpend.push_back({dx, dy, c});
        }
        s->fpend_total += c;
        src += c;
        if (ysrc) ysrc += c;
        left -= c;
    }
    return CYC_OK;
}

// Project the samples pending in the view of a (Set-mode) stream: one pass over
// stage[cur][0, held + pending), then the view's last `keep` samples become the next view's
// head.
int set_flush(cyc_stream* s)
{
    const int64_t c = s->fpend_total;
    if (c <= 0) return CYC_OK;
    float2* view = s->stage[s->cur];
    if (s->fpend_host) {
        CK(cudaStreamWaitEvent(s->st, s->ev_copied, 0));
        s->fpend_host = false;
    }
    const int64_t nview = s->held + c;
    int64_t nc = nview - s->M;
    if (nc < 0) nc = 0;
    const int64_t T2 = s->T + c;
    const int64_t keep = T2 < s->M ? T2 : s->M;
    s->fpend_total = 0;
    bool tail_done = false;
    if (nc > 0) {
        int rc = project(s, nc, nview - keep, keep, &tail_done);
        if (rc) return rc;
    }
    if (keep > 0 && !tail_done) {
        CK(cudaMemcpyAsync(s->stage[s->cur ^ 1], view + nview - keep, (size_t)keep * sizeof(float2),
                           cudaMemcpyDeviceToDevice, s->st));
        if (s->cross)
            CK(cudaMemcpyAsync(s->stage_y[s->cur ^ 1], s->stage_y[s->cur] + nview - keep,
                               (size_t)keep * sizeof(float2), cudaMemcpyDeviceToDevice, s->st));
    }
    s->n_eff += nc;
    s->T = T2;
    if (s->xst) CK(cudaEventRecord(s->ev_read[s->cur], s->st));     // this view is free again
    s->cur ^= 1;
    s->held = keep;
    return CYC_OK;
}

// Run the pending pushes of a stream (Full mode: fold them; Set mode: project them) before
// anything reads or replaces its state.
int settle(cyc_stream* s)
{
    const bool pending = s->full ? !s->fpend.empty() : s->fpend_total != 0;
    if (!pending && !s->zero_sums) return CYC_OK;
    DeviceGuard g(s->device);
    if (!g.ok) return fail(CYC_ECUDA, "cudaSetDevice failed");
    if (pending) {
        const int rc = s->full ? full_flush(s) : set_flush(s);
        if (rc) return rc;
    }
    if (s->zero_sums) {               // a reset that no pass has folded in yet
        CK(cudaMemsetAsync(s->sums, 0, (size_t)s->Au * s->ncols * sizeof(double2), s->st));
        s->zero_sums = false;
    }
    return CYC_OK;
}

// After a stream synchronisation: did a kernel's bounded wait give up?  The status word has
// landed in h_err; report and clear it.
int check_status(cyc_stream* s)
{
    const int flag = *s->h_err;
    if (flag) {
        *s->h_err = 0;
        CK(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->st));
        CK(cudaStreamSynchronize(s->st));
        return fail(CYC_ETIMEDOUT, "a projection kernel gave up waiting (code %d); the sums are unreliable", flag);
    }
    return CYC_OK;
}

// Queues the copy of the kernels' status word, synchronises the stream and reports it.
int sync_and_check(cyc_stream* s)
{
    CK(cudaMemcpyAsync(s->h_err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return check_status(s);
}

bool is_device_ptr(const void* p, int device, bool* wrong_device)
{
    cudaPointerAttributes at;
    *wrong_device = false;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        if (at.device != device) *wrong_device = true;
        return true;
    }
    return false;
}

// Device outputs are written as double2 (16-byte stores).
bool misaligned16(const void* p) { return ((uintptr_t)p & 15) != 0; }

}  // namespace

extern "C" {

int cyc_create(const int32_t* lags, int nlags, const double* alphas, int nalphas, int conj_flag,
               cyc_stream** out)
{
    cyc_params p;
    memset(&p, 0, sizeof p);
    p.lags = lags;
    p.nlags = nlags;
    p.alphas = alphas;
    p.nalphas = nalphas;
    p.conj_flag = conj_flag;
    p.precision = CYC_P_FP32;
    return cyc_create_ex(&p, out);
}

static int create_impl(const cyc_params* p, bool cross, int64_t win_len, int64_t hop, int64_t win_cap,
                       cyc_stream** out, bool full = false)
{
    if (!out) return fail(CYC_EINVAL, "cyc_create_ex: out is NULL");
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        return fail(CYC_ECUDA, "no CUDA device is available");
    }
    if (p->device < 0 || p->device >= ndev) return fail(CYC_EINVAL, "device %d out of range", p->device);

    cyc_stream* s = new (std::nothrow) cyc_stream();
    if (!s) return fail(CYC_ENOMEM, "host allocation failed");
    s->device = p->device;
    s->st = (cudaStream_t)p->cuda_stream;
    s->precision = p->precision;
    s->conj_flag = p->conj_flag;
    if (p->conj_flag & CYC_CONV) s->forms[s->F++] = CYC_CONV;
    if (p->conj_flag & CYC_CONJ) s->forms[s->F++] = CYC_CONJ;
    s->lags.assign(p->lags, p->lags + p->nlags);
    s->L = p->nlags;
    s->cross = cross;
    s->full = full;
    if (win_len > 0) {
        s->win = true;
        s->win_len = win_len;
        s->hop = hop;
        s->win_w = (int)(win_len / hop);
        s->win_cap = win_cap;
    }
    int32_t lo = 0, hi = 0;
    for (int32_t m : s->lags) {
        lo = m < lo ? m : lo;
        hi = m > hi ? m : hi;
    }
    s->Mneg = -lo;
    s->M = hi - lo;
    s->alphas.assign(p->alphas, p->alphas + p->nalphas);
    s->A = p->nalphas;
    std::map<uint64_t, int> uniq;
    s->amap.resize(s->A);
    for (int i = 0; i < s->A; ++i) {
        uint64_t ph = alpha_to_phi(s->alphas[i]);
        auto it = uniq.find(ph);
        if (it == uniq.end()) {
            it = uniq.emplace(ph, (int)s->phi_u.size()).first;
            s->phi_u.push_back(ph);
        }
        s->amap[i] = it->second;
    }
    s->Au = (int)s->phi_u.size();
    if (s->precision != CYC_P_FP32) s->units = order_units(s->phi_u, s->amap);
    s->ncols = s->F * s->L;
    s->n0 = p->n0;
    s->max_chunk = p->max_chunk > 0 ? p->max_chunk : kDefaultChunk;
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, s->lags.data(), s->lags.size() * sizeof(int32_t));
    h = fnv1a(h, s->phi_u.data(), s->phi_u.size() * sizeof(uint64_t));
    h = fnv1a(h, s->amap.data(), s->amap.size() * sizeof(int32_t));
    h = fnv1a(h, &s->conj_flag, sizeof s->conj_flag);
    h = fnv1a(h, &s->n0, sizeof s->n0);
    const int32_t xy = s->cross ? 1 : 0;
    h = fnv1a(h, &xy, sizeof xy);
    h = fnv1a(h, &s->win_len, sizeof s->win_len);
    const int32_t fm = s->full ? 1 : 0;
    h = fnv1a(h, &fm, sizeof fm);
    h = fnv1a(h, &s->hop, sizeof s->hop);
    s->fingerprint = h;

    if (s->precision != CYC_P_FP32 && !tc_supported(s->ncols, s->M)) {
        delete s;
        return fail(CYC_ENOTSUP, "the tensor-core projection supports lag spans up to 2560 (span %d); use CYC_P_FP32",
                    s->M);
    }
    DeviceGuard g(s->device);
    if (!g.ok) { delete s; return fail(CYC_ECUDA, "cudaSetDevice(%d) failed", p->device); }
    if (cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
        delete s;
        return fail(CYC_ECUDA, "cannot query the SM count");
    }
    if (s->precision != CYC_P_FP32) {
        s->pair_ctas = tc_pair_ctas(s->precision);
        if (s->pair_ctas < 2) {
            delete s;
            return fail(CYC_ENOTSUP, "the tensor-core projection needs two-CTA clusters, which this device cannot "
                                     "hold; use CYC_P_FP32");
        }
        const char* ev = getenv("CYC_TEST_WITHHOLD_ARRIVAL");
        s->withhold = (ev && ev[0] == '1') ? 1 : 0;
    }
    test_alloc_arm();
    rc = alloc_state(s);
    if (rc) {
        s->free_all();
        delete s;
        return rc;
    }
    *out = s;
    return CYC_OK;
}

int cyc_create_ex(const cyc_params* p, cyc_stream** out) { return create_impl(p, false, 0, 0, 0, out); }

int cyc_create_xy(const cyc_params* p, cyc_stream** out) { return create_impl(p, true, 0, 0, 0, out); }

int cyc_create_full(const cyc_params* p, int32_t A, int cross, cyc_stream** out)
{
    if (out) *out = nullptr;
    if (!p) return fail(CYC_EINVAL, "cyc_create_full: params is NULL");
    if (!full_supported(A)) return fail(CYC_EINVAL, "cyc_create_full: A must be a power of two in [2, 4096]");
    if (p->precision != CYC_P_FP32) return fail(CYC_EINVAL, "cyc_create_full: the folded grid runs in FP32/FP64 only");
    std::vector<double> grid(A);
    for (int k = 0; k < A; ++k) grid[k] = -0.5 + (double)k / (double)A;          // exact in binary
    cyc_params q = *p;
    q.alphas = grid.data();
    q.nalphas = A;
    return create_impl(&q, cross != 0, 0, 0, 0, out, true);
}

int cyc_create_full_window(const cyc_params* p, int32_t A, int64_t hop, int64_t capacity, int cross,
                           cyc_stream** out)
{
    if (out) *out = nullptr;
    if (!p) return fail(CYC_EINVAL, "cyc_create_full_window: params is NULL");
    if (!full_supported(A)) return fail(CYC_EINVAL, "cyc_create_full_window: A must be a power of two in [2, 4096]");
    if (p->precision != CYC_P_FP32) return fail(CYC_EINVAL, "cyc_create_full_window: FP32 only");
    if (hop < 1 || hop > ((int64_t)1 << 30)) return fail(CYC_EINVAL, "cyc_create_full_window: hop must be in [1, 2^30]");
    if (capacity < 1 || capacity > (1 << 20))
        return fail(CYC_EINVAL, "cyc_create_full_window: capacity must be in [1, 2^20]");
    if ((double)capacity * A * p->nlags * ((p->conj_flag & 1) + ((p->conj_flag >> 1) & 1)) * 8.0 > 64e9)
        return fail(CYC_EINVAL, "cyc_create_full_window: the ring would exceed 64 GB");
    std::vector<double> grid(A);
    for (int k = 0; k < A; ++k) grid[k] = -0.5 + (double)k / (double)A;          // exact in binary
    cyc_params q = *p;
    q.alphas = grid.data();
    q.nalphas = A;
    return create_impl(&q, cross != 0, A, hop, capacity, out, true);
}

int cyc_create_window(const cyc_params* p, int64_t win_len, int64_t hop, int64_t capacity, int cross,
                      cyc_stream** out)
{
    if (out) *out = nullptr;
    if (hop < 1 || win_len < hop || win_len % hop != 0 || win_len / hop > (1 << 16))
        return fail(CYC_EINVAL, "cyc_create_window: need hop >= 1, win_len a multiple of hop, win_len / hop <= 65536");
    if (hop < 16 && p && p->precision != CYC_P_FP32)
        return fail(CYC_EINVAL, "cyc_create_window: hops below 16 samples need CYC_P_FP32");
    if (capacity < 1 || capacity > (1 << 20)) return fail(CYC_EINVAL, "cyc_create_window: capacity must be in [1, 2^20]");
    return create_impl(p, cross != 0, win_len, hop, capacity, out);
}

static int push_impl(cyc_stream* s, const void* xchunk, const void* ychunk, int64_t nsamples, int on_device,
                     const char* who)
{
    if (nsamples < 0) return fail(CYC_EINVAL, "%s: nsamples < 0", who);
    if (nsamples == 0) return CYC_OK;
    if (s->win) {                     // room for every window this push completes?
        const int64_t made2 = windows_made(s, s->T + s->fpend_total + nsamples);
        if (made2 - s->win_read > s->win_cap)
            return fail(CYC_EAGAIN, "%s: the push would complete %lld windows with room for %lld; read windows first",
                        who, (long long)(made2 - s->win_made), (long long)(s->win_cap - (s->win_made - s->win_read)));
    }
    if (!xchunk || (s->cross && !ychunk)) return fail(CYC_EINVAL, "%s: chunk is NULL", who);
    DeviceGuard g(s->device);
    if (!g.ok) return fail(CYC_ECUDA, "cudaSetDevice failed");
    if (on_device) {
        bool wrong = false;
        if (!is_device_ptr(xchunk, s->device, &wrong) || wrong ||
            (s->cross && (!is_device_ptr(ychunk, s->device, &wrong) || wrong)))
            return fail(CYC_EINVAL, "%s: on_device set but a chunk is not memory of device %d", who, s->device);
    }
    const float2* src = (const float2*)xchunk;
    const float2* ysrc = (const float2*)ychunk;
    if (!on_device && !s->xst) {
        CK(cudaStreamCreateWithFlags(&s->xst, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&s->ev_copied, cudaEventDisableTiming));
        // both staging buffers are free once the work queued so far is done
        for (auto& e : s->ev_read) {
            CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            CK(cudaEventRecord(e, s->st));
        }
    }
    if (s->full) return full_push(s, src, ysrc, nsamples, on_device != 0);
    // a1: the view is [carried tail (held samples) | pending samples], for both inputs.  Each
    // push is copied in behind what is pending (a host chunk through the copy stream, once
    // the pass that last viewed this buffer is done); the projection runs when the view
    // holds a full pass (max_chunk samples, or win_splits - 1 hops for windowed streams) and
    // before anything reads the stream, so that short pushes share one launch.
    const int64_t pass = s->win ? std::min<int64_t>(s->max_chunk, (int64_t)(s->win_splits - 1) * s->hop) : s->max_chunk;
    int64_t left = nsamples;
    while (left > 0) {
        const int64_t c = std::min<int64_t>(left, pass - s->fpend_total);
        const int64_t at = s->held + s->fpend_total;
        cudaStream_t cs = on_device ? s->st : s->xst;
        if (!on_device) CK(cudaStreamWaitEvent(cs, s->ev_read[s->cur], 0));
        CK(cudaMemcpyAsync(s->stage[s->cur] + at, src, (size_t)c * sizeof(float2), cudaMemcpyDefault, cs));
        if (s->cross)
            CK(cudaMemcpyAsync(s->stage_y[s->cur] + at, ysrc, (size_t)c * sizeof(float2), cudaMemcpyDefault, cs));
        if (!on_device) {
            CK(cudaEventRecord(s->ev_copied, cs));
            s->fpend_host = true;
        }
        s->fpend_total += c;
        src += c;
        if (ysrc) ysrc += c;
        left -= c;
        if (s->fpend_total == pass) {
            int rc = set_flush(s);
            if (rc) return rc;
        }
    }
    return CYC_OK;
}

int cyc_push(cyc_stream* s, const void* chunk, int64_t nsamples, int on_device)
{
    if (!s) return fail(CYC_EINVAL, "cyc_push: handle is NULL");
    if (s->cross) return fail(CYC_EINVAL, "cyc_push: the stream has two inputs; use cyc_push_xy");
    return push_impl(s, chunk, nullptr, nsamples, on_device, "cyc_push");
}

int cyc_push_xy(cyc_stream* s, const void* x_chunk, const void* y_chunk, int64_t nsamples, int on_device)
{
    if (!s) return fail(CYC_EINVAL, "cyc_push_xy: handle is NULL");
    if (!s->cross) return fail(CYC_EINVAL, "cyc_push_xy: the stream has one input; use cyc_push");
    return push_impl(s, x_chunk, y_chunk, nsamples, on_device, "cyc_push_xy");
}

int cyc_sync(cyc_stream* s)
{
    if (!s) return fail(CYC_EINVAL, "cyc_sync: handle is NULL");
    if (int rc0 = settle(s)) return rc0;
    DeviceGuard g(s->device);
    return sync_and_check(s);
}

int cyc_read(cyc_stream* s, double* out, int64_t* n_eff)
{
    if (!s) return fail(CYC_EINVAL, "cyc_read: handle is NULL");
    if (int rc0 = settle(s)) return rc0;
    if (n_eff) *n_eff = s->n_eff;
    if (s->n_eff == 0) return fail(CYC_ENODATA, "cyc_read: N_eff is 0 (fewer than max(lags) + 1 samples)");
    if (!out) return fail(CYC_EINVAL, "cyc_read: out is NULL");
    DeviceGuard g(s->device);
    bool wrong = false;
    bool dev = is_device_ptr(out, s->device, &wrong);
    if (wrong) return fail(CYC_EINVAL, "cyc_read: out is memory of another device");
    if (dev && misaligned16(out)) return fail(CYC_EINVAL, "cyc_read: device out must be 16-byte aligned");
    // host memory: the result lands in a page-locked buffer of the handle's (up to 64 MB, made
    // at the first host read) and is copied from there.  Set-mode streams have the read
    // kernel write it, and the status word beside it, straight into page-locked memory (one
    // launch, one synchronisation); Full-mode streams, or without a device address for the
    // buffer, queue its copy beside the status word's; without the buffer the copy goes
    // straight to `out`.
    const size_t bytes = (size_t)s->F * s->A * s->L * sizeof(double2);
    if (!dev && !s->h_stage && bytes <= ((size_t)64 << 20)) {
        if (cudaMallocHost(&s->h_stage, bytes) != cudaSuccess) {
            cudaGetLastError();
            s->h_stage = nullptr;
        } else if (cudaHostGetDevicePointer(&s->h_stage_dev, s->h_stage, 0) != cudaSuccess) {
            cudaGetLastError();
            s->h_stage_dev = nullptr;
        }
    }
    const bool direct = !dev && !s->full && s->h_stage_dev && s->h_err_dev;
    double2* dst = dev ? (double2*)out : direct ? (double2*)s->h_stage_dev : s->d_out;
    if (s->full)
        CK(full_read(s->sums, s->Au, s->ncols, s->F, s->L, 1.0 / (double)s->n_eff, dst, s->st));
    else
        CK(read_sums(s->sums, s->d_amap, s->F, s->A, s->L, s->ncols, 1.0 / (double)s->n_eff, dst, s->st,
                     direct ? s->d_err : nullptr, direct ? s->h_err_dev : nullptr));
    s->kernel_launches++;
    if (dev) return sync_and_check(s);
    int rc;
    if (direct) {
        CK(cudaStreamSynchronize(s->st));
        rc = check_status(s);
    } else {
        CK(cudaMemcpyAsync(s->h_stage ? s->h_stage : (void*)out, s->d_out, bytes, cudaMemcpyDeviceToHost, s->st));
        rc = sync_and_check(s);
    }
    if (rc == CYC_OK && s->h_stage) memcpy(out, s->h_stage, bytes);
    return rc;
}

int cyc_read_spectrum(cyc_stream* s, int32_t Q, int32_t taper, double* out)
{
    if (!s) return fail(CYC_EINVAL, "cyc_read_spectrum: handle is NULL");
    if (int rc0 = settle(s)) return rc0;
    if (Q < 1 || Q > (1 << 16)) return fail(CYC_EINVAL, "cyc_read_spectrum: Q must be in [1, 65536]");
    if (taper != 0 && taper != 1) return fail(CYC_EINVAL, "cyc_read_spectrum: taper must be 0 or 1");
    if (s->n_eff == 0) return fail(CYC_ENODATA, "cyc_read_spectrum: N_eff is 0");
    if (!out) return fail(CYC_EINVAL, "cyc_read_spectrum: out is NULL");
    DeviceGuard g(s->device);
    bool wrong = false;
    const bool dev = is_device_ptr(out, s->device, &wrong);
    if (wrong) return fail(CYC_EINVAL, "cyc_read_spectrum: out is memory of another device");
    if (dev && misaligned16(out)) return fail(CYC_EINVAL, "cyc_read_spectrum: device out must be 16-byte aligned");
    if (!s->d_lags) {
        CK(dev_malloc((void**)&s->d_lags, (size_t)s->L * sizeof(int32_t)));
        CK(cudaMemcpy(s->d_lags, s->lags.data(), (size_t)s->L * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    if (Q > s->sp_Q) {
        CK(cudaStreamSynchronize(s->st));
        if (s->sp_E) cudaFree(s->sp_E);
        if (s->sp_S) cudaFree(s->sp_S);
        s->sp_E = s->sp_S = nullptr;
        s->sp_Q = 0;
        CK(cudaMalloc(&s->sp_E, (size_t)s->L * Q * sizeof(double2)));
        CK(cudaMalloc(&s->sp_S, (size_t)s->F * s->A * Q * sizeof(double2)));
        s->sp_Q = Q;
    }
    const double inv_n = 1.0 / (double)s->n_eff;
    if (s->full)
        CK(full_read(s->sums, s->Au, s->ncols, s->F, s->L, inv_n, s->d_out, s->st));
    else
        CK(read_sums(s->sums, s->d_amap, s->F, s->A, s->L, s->ncols, inv_n, s->d_out, s->st));
    double mmax = 0.0;
    for (int32_t m : s->lags) mmax = std::max(mmax, (double)(m < 0 ? -m : m));
    double2* dst = dev ? (double2*)out : s->sp_S;
    CK(spectrum(s->d_out, s->d_lags, s->F * s->A, s->L, Q, taper, mmax, s->sp_E, dst, s->st));
    s->kernel_launches += 3;
    if (!dev)
        CK(cudaMemcpyAsync(out, s->sp_S, (size_t)s->F * s->A * Q * sizeof(double2), cudaMemcpyDeviceToHost, s->st));
    return sync_and_check(s);
}

int cyc_detect(cyc_stream* s, double kappa, int32_t win, uint8_t* flags, float* ratio, int32_t* ndetected)
{
    if (!s) return fail(CYC_EINVAL, "cyc_detect: handle is NULL");
    if (int rc0 = settle(s)) return rc0;
    if (ndetected) *ndetected = 0;
    if (!flags) return fail(CYC_EINVAL, "cyc_detect: flags is NULL");
    if (!(kappa > 0.0) || !isfinite(kappa)) return fail(CYC_EINVAL, "cyc_detect: kappa must be positive and finite");
    if (!detect_supported(win)) return fail(CYC_EINVAL, "cyc_detect: win must be in [2, 32]");
    if (s->n_eff == 0) return fail(CYC_ENODATA, "cyc_detect: N_eff is 0");
    DeviceGuard g(s->device);
    bool wrong = false;
    const bool fdev = is_device_ptr(flags, s->device, &wrong);
    if (wrong) return fail(CYC_EINVAL, "cyc_detect: flags is memory of another device");
    const bool rdev = ratio && is_device_ptr(ratio, s->device, &wrong);
    if (wrong) return fail(CYC_EINVAL, "cyc_detect: ratio is memory of another device");
    if (rdev && ((uintptr_t)ratio & 3) != 0) return fail(CYC_EINVAL, "cyc_detect: device ratio must be 4-byte aligned");
    const size_t nfa = (size_t)s->F * s->A;
    if (!s->dt_s) {
        CK(dev_malloc((void**)&s->dt_s, nfa * sizeof(double)));
        CK(dev_malloc((void**)&s->dt_flags, nfa));
        CK(dev_malloc((void**)&s->dt_ratio, nfa * sizeof(float)));
        CK(dev_malloc((void**)&s->dt_count, sizeof(int)));
        CK(dev_malloc((void**)&s->dt_dc, (size_t)s->A));
        std::vector<uint8_t> dc(s->A);
        for (int i = 0; i < s->A; ++i) dc[i] = (!s->cross && alpha_to_phi(s->alphas[i]) == 0) ? 1 : 0;
        CK(cudaMemcpy(s->dt_dc, dc.data(), (size_t)s->A, cudaMemcpyHostToDevice));
    }
    const double inv_n = 1.0 / (double)s->n_eff;
    if (s->full)
        CK(full_read(s->sums, s->Au, s->ncols, s->F, s->L, inv_n, s->d_out, s->st));
    else
        CK(read_sums(s->sums, s->d_amap, s->F, s->A, s->L, s->ncols, inv_n, s->d_out, s->st));
    const int conv_f = s->forms[0] == CYC_CONV ? 0 : -1;
    uint8_t* fl = fdev ? flags : s->dt_flags;
    float* ra = ratio ? (rdev ? ratio : s->dt_ratio) : nullptr;
    CK(detect(s->d_out, s->F, s->A, s->L, s->dt_dc, conv_f, win, kappa, s->dt_s, fl, ra, s->dt_count, s->st));
    s->kernel_launches += 3;
    if (!fdev) CK(cudaMemcpyAsync(flags, s->dt_flags, nfa, cudaMemcpyDeviceToHost, s->st));
    if (ratio && !rdev) CK(cudaMemcpyAsync(ratio, s->dt_ratio, nfa * sizeof(float), cudaMemcpyDeviceToHost, s->st));
    int count = 0;
    CK(cudaMemcpyAsync(&count, s->dt_count, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    const int rc = sync_and_check(s);
    if (ndetected) *ndetected = count;
    return rc;
}

int cyc_read_windows(cyc_stream* s, double* out, int64_t max_win, int64_t* nwin, int64_t* first_k)
{
    if (!s) return fail(CYC_EINVAL, "cyc_read_windows: handle is NULL");
    if (int rc0 = settle(s)) return rc0;
    if (!s->win) return fail(CYC_EINVAL, "cyc_read_windows: not a windowed stream (cyc_create_window)");
    if (nwin) *nwin = 0;
    if (first_k) *first_k = s->win_read;
    int64_t n = s->win_made - s->win_read;
    if (n > max_win) n = max_win;
    if (n <= 0) return CYC_OK;
    if (!out) return fail(CYC_EINVAL, "cyc_read_windows: out is NULL");
    DeviceGuard g(s->device);
    bool wrong = false;
    const bool dev = is_device_ptr(out, s->device, &wrong);
    if (wrong) return fail(CYC_EINVAL, "cyc_read_windows: out is memory of another device");
    if (dev && misaligned16(out)) return fail(CYC_EINVAL, "cyc_read_windows: device out must be 16-byte aligned");
    const int64_t per = (int64_t)s->F * s->A * s->L;
    const uint64_t base = (uint64_t)s->n0 + (uint64_t)s->Mneg;
    const double inv_n = 1.0 / (double)s->win_len;
    if (s->full) {                    // Full-mode windows: spectra in the ring, transposed to [F][A][L]
        if (dev) {
            CK(full_read_windows(s->w_out, s->win_cap, s->win_read, n, s->A, s->F, s->L, (double2*)out, s->st));
            s->kernel_launches += 1;
        } else {
            for (int64_t i = 0; i < n; ++i) {
                CK(full_read_windows(s->w_out, s->win_cap, s->win_read + i, 1, s->A, s->F, s->L, s->d_out, s->st));
                CK(cudaMemcpyAsync((double2*)out + i * per, s->d_out, (size_t)per * sizeof(double2),
                                   cudaMemcpyDeviceToHost, s->st));
            }
            s->kernel_launches += n;
        }
    } else if (dev) {
        CK(read_windows(s->w_out, s->win_cap, s->win_read, n, s->d_amap, s->d_phi, s->F, s->A, s->L, s->Au, s->ncols,
                        base, s->hop, inv_n, (double2*)out, s->st));
        s->kernel_launches += 1;
    } else {
        for (int64_t i = 0; i < n; ++i) {            // one window at a time through the read buffer
            CK(read_windows(s->w_out, s->win_cap, s->win_read + i, 1, s->d_amap, s->d_phi, s->F, s->A, s->L, s->Au,
                            s->ncols, base, s->hop, inv_n, s->d_out, s->st));
            CK(cudaMemcpyAsync((double2*)out + i * per, s->d_out, (size_t)per * sizeof(double2),
                               cudaMemcpyDeviceToHost, s->st));
        }
        s->kernel_launches += n;
    }
    s->win_read += n;
    if (nwin) *nwin = n;
    return sync_and_check(s);
}

int cyc_reset(cyc_stream* s)
{
    if (!s) return fail(CYC_EINVAL, "cyc_reset: handle is NULL");
    if (int rc0 = settle(s)) return rc0;
    DeviceGuard g(s->device);
    // FP32 streams on the register-sum path (no windows, no Full mode) leave the zeroing to
    // their next pass, which writes its totals instead of adding them (or to settle(), if
    // anything reads the sums first); the others zero the sums here
    if (s->precision == CYC_P_FP32 && small_supported(s->Au) && !s->win && !s->full)
        s->zero_sums = true;
    else
        CK(cudaMemsetAsync(s->sums, 0, (size_t)s->Au * s->ncols * sizeof(double2), s->st));
    if (s->win && !s->full) {
        CK(cudaMemsetAsync(s->w_sum, 0, (size_t)s->Au * s->ncols * sizeof(float4), s->st));
        CK(cudaMemsetAsync(s->w_pend, 0, (size_t)s->Au * s->ncols * sizeof(float4), s->st));
    }
    if (s->win) s->hops = s->win_made = s->win_read = 0;
    s->T = s->n_eff = s->held = 0;
    return CYC_OK;
}

int cyc_destroy(cyc_stream* s)
{
    if (!s) return CYC_OK;
    {
        DeviceGuard g(s->device);
        cudaStreamSynchronize(s->st);
        s->free_all();
    }
    delete s;
    return CYC_OK;
}

int cyc_save(cyc_stream* s, void* buf, size_t* len)
{
    if (!s || !len) return fail(CYC_EINVAL, "cyc_save: NULL argument");
    if (int rc0 = settle(s)) return rc0;
    if (s->win) return fail(CYC_ENOTSUP, "cyc_save: windowed streams keep no blob");
    size_t sums_b = (size_t)s->Au * s->ncols * sizeof(double2);
    const size_t held_b = (size_t)s->held * sizeof(float2) * (s->cross ? 2 : 1);
    size_t need = sizeof(BlobHeader) + held_b + sums_b;
    if (!buf) { *len = need; return CYC_OK; }
    if (*len < need) { *len = need; return fail(CYC_EINVAL, "cyc_save: buffer too small (%zu < %zu)", *len, need); }
    DeviceGuard g(s->device);
    BlobHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "CYCSTAT1", 8);
    h.version = kBlobVersion;
    h.F = s->F; h.L = s->L; h.A = s->A; h.Au = s->Au;
    h.conj_flag = s->conj_flag;
    h.n0 = s->n0; h.T = s->T; h.n_eff = s->n_eff; h.held = s->held;
    h.fingerprint = s->fingerprint;
    unsigned char* b = (unsigned char*)buf;
    memcpy(b, &h, sizeof h);
    CK(cudaStreamSynchronize(s->st));
    if (s->held) {
        CK(cudaMemcpy(b + sizeof h, s->stage[s->cur], (size_t)s->held * sizeof(float2), cudaMemcpyDeviceToHost));
        if (s->cross)
            CK(cudaMemcpy(b + sizeof h + (size_t)s->held * sizeof(float2), s->stage_y[s->cur],
                          (size_t)s->held * sizeof(float2), cudaMemcpyDeviceToHost));
    }
    CK(cudaMemcpy(b + sizeof h + held_b, s->sums, sums_b, cudaMemcpyDeviceToHost));
    *len = need;
    return CYC_OK;
}

int cyc_load(cyc_stream* s, const void* buf, size_t len)
{
    if (!s || !buf) return fail(CYC_EINVAL, "cyc_load: NULL argument");
    if (int rc0 = settle(s)) return rc0;
    if (s->win) return fail(CYC_ENOTSUP, "cyc_load: windowed streams keep no blob");
    BlobHeader h;
    if (len < sizeof h) return fail(CYC_EINVAL, "cyc_load: blob too short");
    memcpy(&h, buf, sizeof h);
    if (memcmp(h.magic, "CYCSTAT1", 8) || h.version != kBlobVersion)
        return fail(CYC_EINVAL, "cyc_load: not a libcyc state blob of version %u", kBlobVersion);
    if (h.fingerprint != s->fingerprint || h.F != s->F || h.L != s->L || h.A != s->A || h.Au != s->Au ||
        h.conj_flag != s->conj_flag || h.n0 != s->n0)
        return fail(CYC_EINVAL, "cyc_load: blob was saved by a stream with other lags, cycle frequencies, forms, "
                                "inputs or n0");
    if (h.held < 0 || h.held > s->M || h.T < 0 || h.n_eff < 0 || h.held > h.T)
        return fail(CYC_EINVAL, "cyc_load: inconsistent counters in blob");
    size_t sums_b = (size_t)s->Au * s->ncols * sizeof(double2);
    const size_t held_b = (size_t)h.held * sizeof(float2) * (s->cross ? 2 : 1);
    size_t need = sizeof h + held_b + sums_b;
    if (len < need) return fail(CYC_EINVAL, "cyc_load: blob truncated (%zu < %zu)", len, need);
    DeviceGuard g(s->device);
    const unsigned char* b = (const unsigned char*)buf;
    CK(cudaStreamSynchronize(s->st));
    if (h.held) {
        CK(cudaMemcpy(s->stage[s->cur], b + sizeof h, (size_t)h.held * sizeof(float2), cudaMemcpyHostToDevice));
        if (s->cross)
            CK(cudaMemcpy(s->stage_y[s->cur], b + sizeof h + (size_t)h.held * sizeof(float2),
                          (size_t)h.held * sizeof(float2), cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(s->sums, b + sizeof h + held_b, sums_b, cudaMemcpyHostToDevice));
    s->T = h.T;
    s->n_eff = h.n_eff;
    s->held = h.held;
    return CYC_OK;
}

int cyc_info(cyc_stream* s, int* forms, int* nunique, int64_t* total, int64_t* n_eff)
{
    if (!s) return fail(CYC_EINVAL, "cyc_info: handle is NULL");
    if (int rc0 = settle(s)) return rc0;
    if (forms) *forms = s->F;
    if (nunique) *nunique = s->Au;
    if (total) *total = s->T;
    if (n_eff) *n_eff = s->n_eff;
    return CYC_OK;
}

int cyc_phase_increment(double a, uint64_t* phi)
{
    if (!phi || !isfinite(a)) return fail(CYC_EINVAL, "cyc_phase_increment: a must be finite, phi non-NULL");
    *phi = alpha_to_phi(a);
    return CYC_OK;
}

int cyc_sums(cyc_stream* s, double** sums, int64_t* nvalues, int64_t* n_eff)
{
    if (!s || !sums) return fail(CYC_EINVAL, "cyc_sums: NULL argument");
    if (int rc0 = settle(s)) return rc0;
    if (s->win) return fail(CYC_ENOTSUP, "cyc_sums: windowed streams keep their windows apart from the sums");
    if (s->full) return fail(CYC_ENOTSUP, "cyc_sums: Full-mode streams keep float-float folds, not FP64 sums");
    DeviceGuard g(s->device);
    CK(cudaStreamSynchronize(s->st));
    *sums = (double*)s->sums;
    if (nvalues) *nvalues = (int64_t)s->Au * s->ncols;
    if (n_eff) *n_eff = s->n_eff;
    return CYC_OK;
}

int cyc_set_n_eff(cyc_stream* s, int64_t n_eff)
{
    if (!s) return fail(CYC_EINVAL, "cyc_set_n_eff: handle is NULL");
    if (int rc0 = settle(s)) return rc0;
    if (n_eff < 0) return fail(CYC_EINVAL, "cyc_set_n_eff: n_eff < 0");
    if (s->win) return fail(CYC_ENOTSUP, "cyc_set_n_eff: not for windowed streams");
    s->n_eff = n_eff;
    return CYC_OK;
}

int cyc_set_wait_budget(cyc_stream* s, int64_t cycles)
{
    if (!s) return fail(CYC_EINVAL, "cyc_set_wait_budget: handle is NULL");
    if (cycles < 0 || cycles > ((int64_t)1 << 40)) return fail(CYC_EINVAL, "cyc_set_wait_budget: cycles must be in [0, 2^40]");
    s->wait_budget = cycles;
    return CYC_OK;
}

int cyc_profile(cyc_stream* s, int enable)
{
    if (!s) return fail(CYC_EINVAL, "cyc_profile: handle is NULL");
    s->prof = enable != 0;
    return CYC_OK;
}

int cyc_profile_read(cyc_stream* s, double* proj_ms, int64_t* proj_launches, int64_t* kernels)
{
    if (!s) return fail(CYC_EINVAL, "cyc_profile_read: handle is NULL");
    if (int rc0 = settle(s)) return rc0;
    DeviceGuard g(s->device);
    CK(cudaStreamSynchronize(s->st));
    for (auto& e : s->ev_pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e.first, e.second));
        s->prof_ms += ms;
        s->ev_free.push_back(e);
    }
    s->ev_pending.clear();
    if (proj_ms) *proj_ms = s->prof_ms;
    if (proj_launches) *proj_launches = s->prof_launches;
    if (kernels) *kernels = s->kernel_launches;
    s->prof_ms = 0.0;
    s->prof_launches = 0;
    s->kernel_launches = 0;
    return CYC_OK;
}

const char* cyc_strerror(int code)
{
    switch (code) {
    case CYC_OK: return "success";
    case CYC_EINVAL: return "invalid argument";
    case CYC_ENOMEM: return "out of memory";
    case CYC_ECUDA: return "CUDA error";
    case CYC_EAGAIN: return "not admitted, try again";
    case CYC_ETIMEDOUT: return "bounded device wait timed out";
    case CYC_ENODATA: return "no data (N_eff == 0)";
    case CYC_ENOTSUP: return "not supported";
    default: return "unknown status";
    }
}

const char* cyc_last_error(void) { return g_err.c_str(); }

}  // extern "C"
