// cyc_server.cu -- continuous-batching server over many streams (declared in include/cyc.h).
//
// Each stream keeps its samples in a device ring (power-of-two capacity), its FP64 sums and
// its tables on the device.  cyc_server_submit copies a chunk into the ring on a copy stream
// and returns once it has landed.  The engine thread forms batches: for every open stream
// with new samples, the committed range [n_sched, T - M) becomes work items of 128 units of
// cycle frequencies (a and -a share a unit: up to 256 distinct values) x 128 columns x at
// most item_samples terms (tile-major, so the items of one stream tile are consecutive and
// share one fold).  A batch is launched as
//     H2D copy of the item and fold lists  ->  CUDA graph [zero the item counter ->
//     persistent tensor-core kernel over the items -> FP64 fold of the item partials]
// with two batches in flight, so chunks that arrive while one batch runs join the next.
// When a batch's event completes, the engine advances each stream's committed count and
// reports every chunk whose samples are fully used.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>
#include <time.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "cyc_impl.h"

using namespace cyc;

namespace {

int sfail(int code, const char* fmt, ...)
{
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    record_error(buf);
    return code;
}

#define SCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return sfail(e_ == cudaErrorMemoryAllocation ? CYC_ENOMEM : CYC_ECUDA,          \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                   \
    } while (0)

double now_s()
{
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// sums[(d_lo+r)*ncols + c0+j] += sum over the item partials of one stream tile (FP32 adds
// over the items, one FP64 add per value); rows r < nrows of the tile exist.
struct Fold {
    double2* sums;
    int      d_lo, nrows, c0, ncols;
    int64_t  slot0;      // first partial tile (units of one tile of float2)
    int      nslots;
};

// A block task is FOLD_Q x blockDim.x consecutive elements of one fold's tile: the fold is
// found once per task and the element's row and column with 32-bit arithmetic (64-bit
// division per element cost more than the fold's memory traffic).
constexpr int FOLD_Q = 8;

__global__ void fold_kernel(const Fold* __restrict__ folds, const int* __restrict__ nfolds,
                            const float2* __restrict__ slots, int tm, int tn)
{
    const int TILE = tm * tn;
    const int per = FOLD_Q * (int)blockDim.x;
    const int tasks = (TILE + per - 1) / per;             // tasks per fold
    const int ntask = *nfolds * tasks;
    for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
        const int fi = t / tasks, ti = t - fi * tasks;
        const Fold f = folds[fi];
#pragma unroll
        for (int q = 0; q < FOLD_Q; ++q) {
            const int le = ti * per + q * (int)blockDim.x + (int)threadIdx.x;
            if (le >= TILE) break;
            const int r = le / tn, j = le - r * tn;
            if (r >= f.nrows || f.c0 + j >= f.ncols) continue;
            float sr = 0.f, si = 0.f;
            for (int k = 0; k < f.nslots; ++k) {
                const float2 v = slots[(size_t)(f.slot0 + k) * TILE + le];
                sr += v.x;
                si += v.y;
            }
            double2* d = f.sums + (size_t)(f.d_lo + r) * f.ncols + f.c0 + j;
            const double2 o = *d;
            *d = make_double2(o.x + (double)sr, o.y + (double)si);
        }
    }
}

struct Rec {
    int64_t  end;        // stream sample count after this chunk
    uint64_t tag;
    int64_t  n;
    double   t_submit;
};

struct SrvStream {
    std::mutex mu;                    // submit / close of this stream
    std::atomic<bool> open{false};
    std::atomic<bool> closing{false};
    int F = 0, L = 0, A = 0, Au = 0, ncols = 0;
    UnitLayout units;                 // phi in unit order (order_units)
    int32_t M = 0;
    int64_t n0 = 0;
    float2* ring = nullptr;
    uint64_t cap = 0;
    double2* sums = nullptr;
    uint64_t* d_phi = nullptr;
    int32_t* d_amap = nullptr;
    int32_t* d_col_lag = nullptr;
    int8_t* d_col_conj = nullptr;
    double2* d_out = nullptr;
    size_t bytes = 0;
    std::atomic<int64_t> T{0};        // samples on the device
    std::atomic<int64_t> n_done{0};   // committed terms folded into the sums
    std::atomic<int64_t> n_sched{0};  // committed terms handed to batches (written by the engine)
    std::deque<Rec> recs;             // submitted, not yet finished (under mu)

    void release()
    {
        void* ps[] = {ring, sums, d_phi, d_amap, d_col_lag, d_col_conj, d_out};
        for (void* p : ps)
            if (p) cudaFree(p);
        ring = nullptr; sums = nullptr; d_phi = nullptr; d_amap = nullptr; d_col_lag = nullptr;
        d_col_conj = nullptr; d_out = nullptr;
    }
};

struct Batch {
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int buf = 0;
    std::vector<std::pair<int, int64_t>> marks;   // (sid, committed count reached)
    int nitems = 0;
};

}  // namespace

struct cyc_server {
    cyc_server_params p;
    int num_sms = 1;
    int grid = 2;               // CTAs of the persistent launch (two-CTA pairs)
    cudaStream_t cst = nullptr, xst = nullptr;
    std::vector<std::unique_ptr<SrvStream>> streams;
    std::mutex admin;
    uint64_t used = 0;
    // batch buffers (two in flight)
    TcItem* h_items[2] = {nullptr, nullptr};
    TcItem* d_items[2] = {nullptr, nullptr};
    Fold* h_folds[2] = {nullptr, nullptr};
    Fold* d_folds[2] = {nullptr, nullptr};
    int* h_counts[2] = {nullptr, nullptr};        // [nitems, nfolds]
    int* d_counts[2] = {nullptr, nullptr};
    int* d_counter = nullptr;
    int* d_err = nullptr;
    float2* slots = nullptr;
    int64_t nslot_cap = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // engine
    std::thread engine;
    std::atomic<bool> stop{false};
    std::mutex cv_mu;
    std::condition_variable cv;
    std::mutex form_mu;               // held while a batch is formed (close waits on it)
    std::deque<Batch> inflight;
    std::vector<Batch> spare;
    int next_buf = 0;
    int rr = 0;
    std::atomic<int> engine_error{0};
    // completions
    std::mutex done_mu;
    std::condition_variable done_cv;
    std::deque<cyc_done> done_q;
    std::atomic<int64_t> outstanding{0};
    // stats
    std::atomic<int64_t> n_batches{0}, n_items{0};
    std::atomic<double> busy_ms{0.0};

    int form_and_launch();
    void complete(Batch& b);
    void run();
};

namespace {

uint64_t next_pow2(uint64_t v)
{
    uint64_t c = 1;
    while (c < v) c <<= 1;
    return c;
}

}  // namespace

// Builds one batch from the streams with new samples; returns the number of items (0: none).
int cyc_server::form_and_launch()
{
    const int b = next_buf;
    TcItem* items = h_items[b];
    Fold* folds = h_folds[b];
    int ni = 0, nf = 0;
    int64_t ns = 0;
    std::vector<std::pair<int, int64_t>> marks;
    const int nstreams = (int)streams.size();
    const int UP = tc_pair_units(), TR = tc_tile_rows(), BNc = tc_tile_cols();
    const int64_t IS = p.item_samples;
    const int64_t TILE = (int64_t)TR * BNc;

    // one stream: as many of its pieces as the batch has room for (false: no room at all).
    // Items and their partial slots are tile-major: slot(ip, ic, pc) = base + (ip tcn + ic) np + pc
    auto single = [&](int sid) -> bool {
        SrvStream& s = *streams[sid];
        const int64_t upto = s.T.load() - s.M, n_sched = s.n_sched.load();
        if (upto <= n_sched) return true;
        const int ta = (s.units.U + UP - 1) / UP, tcn = (s.ncols + BNc - 1) / BNc;
        int64_t span = upto - n_sched;
        const int pieces = (int)((span + IS - 1) / IS);
        const int room_items = (p.max_items - ni) / (ta * tcn);
        const int64_t room_slots = (nslot_cap - ns) / (ta * tcn);
        const int room_folds = (p.max_items - nf) / (ta * tcn);
        int fit = (int)std::min<int64_t>(pieces, std::min<int64_t>(room_items, room_slots));
        if (room_folds <= 0) fit = 0;
        if (fit <= 0) return false;
        if (fit < pieces) span = (int64_t)fit * IS;
        const int64_t base = ns;
        ns += (int64_t)ta * tcn * fit;
        for (int ip = 0; ip < ta; ++ip) {
            const int u0 = ip * UP;
            const int d_lo = unit_row(u0, 0, s.units.np, s.units.nself, s.units.U);
            const int d_hi = ip + 1 < ta ? unit_row(u0 + UP, 0, s.units.np, s.units.nself, s.units.U) : s.Au;
            for (int ic = 0; ic < tcn; ++ic) {
                const int64_t slot0 = base + (int64_t)(ip * tcn + ic) * fit;
                Fold& f = folds[nf++];
                f.sums = s.sums;
                f.d_lo = d_lo;
                f.nrows = d_hi - d_lo;
                f.c0 = ic * BNc;
                f.ncols = s.ncols;
                f.slot0 = slot0;
                f.nslots = fit;
                for (int pc = 0; pc < fit; ++pc) {
                    TcItem& it = items[ni++];
                    it.x = s.ring;
                    it.xmask = s.cap - 1;
                    it.x_avail = INT64_MAX;
                    it.nbase = (uint64_t)s.n0;
                    it.n_beg = n_sched + pc * IS;
                    it.n_end = it.n_beg + std::min<int64_t>(IS, span - pc * IS);
                    it.phi = s.d_phi;
                    it.col_lag = s.d_col_lag;
                    it.col_conj = s.d_col_conj;
                    it.out = slots + (slot0 + pc) * TILE;
                    it.out_stride = BNc;
                    it.u0 = u0;
                    it.d_lo = d_lo;
                    it.np = s.units.np;
                    it.nself = s.units.nself;
                    it.U = s.units.U;
                    it.c0 = ic * BNc;
                    it.ncols = s.ncols;
                    it.M = s.M;
                    it.y = nullptr;
                    it.D = 0;
                }
            }
        }
        s.n_sched.store(n_sched + span);
        marks.emplace_back(sid, n_sched + span);
        return true;
    };

    for (int k = 0; k < nstreams; ++k) {
        const int sid = (rr + k) % nstreams;
        SrvStream& s = *streams[sid];
        if (!s.open.load(std::memory_order_acquire) || s.closing.load()) continue;
        if (s.T.load() - s.M <= s.n_sched.load()) continue;
        if (!single(sid)) break;
    }
    rr = (rr + 1) % (nstreams > 0 ? nstreams : 1);
    if (ni == 0) return 0;
    h_counts[b][0] = ni;
    h_counts[b][1] = nf;
    Batch bt;
    if (!spare.empty()) {
        bt = spare.back();
        spare.pop_back();
    } else {
        if (cudaEventCreate(&bt.ev0) != cudaSuccess || cudaEventCreate(&bt.ev1) != cudaSuccess) return -1;
    }
    bt.buf = b;
    bt.marks = std::move(marks);
    bt.nitems = ni;
    if (cudaMemcpyAsync(d_items[b], items, sizeof(TcItem) * ni, cudaMemcpyHostToDevice, cst) != cudaSuccess ||
        cudaMemcpyAsync(d_folds[b], folds, sizeof(Fold) * nf, cudaMemcpyHostToDevice, cst) != cudaSuccess ||
        cudaMemcpyAsync(d_counts[b], h_counts[b], 2 * sizeof(int), cudaMemcpyHostToDevice, cst) != cudaSuccess ||
        cudaEventRecord(bt.ev0, cst) != cudaSuccess || cudaGraphLaunch(graph[b], cst) != cudaSuccess ||
        cudaEventRecord(bt.ev1, cst) != cudaSuccess)
        return -1;
    inflight.push_back(std::move(bt));
    next_buf ^= 1;
    n_batches++;
    n_items += ni;
    return ni;
}

void cyc_server::complete(Batch& bt)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, bt.ev0, bt.ev1) == cudaSuccess) busy_ms.store(busy_ms.load() + ms);
    const double t = now_s();
    int err = 0;
    cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    std::vector<cyc_done> fin;
    for (auto& mk : bt.marks) {
        SrvStream& s = *streams[mk.first];
        s.n_done.store(mk.second);
        std::lock_guard<std::mutex> lk(s.mu);
        while (!s.recs.empty() && s.recs.front().end - s.M <= mk.second) {
            const Rec& r = s.recs.front();
            cyc_done d;
            d.sid = mk.first;
            d.status = err ? CYC_ETIMEDOUT : 0;
            d.tag = r.tag;
            d.nsamples = r.n;
            d.submit_s = r.t_submit;
            d.done_s = t;
            fin.push_back(d);
            s.recs.pop_front();
        }
    }
    if (err) engine_error.store(err);
    if (!fin.empty()) {
        std::lock_guard<std::mutex> lk(done_mu);
        for (auto& d : fin) done_q.push_back(d);
        outstanding -= (int64_t)fin.size();
    }
    done_cv.notify_all();
    bt.marks.clear();
    spare.push_back(bt);
}

void cyc_server::run()
{
    cudaSetDevice(p.device);
    while (!stop.load()) {
        bool progressed = false;
        while (!inflight.empty()) {
            cudaError_t q = cudaEventQuery(inflight.front().ev1);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) {
                engine_error.store(-1);
                cudaGetLastError();
            }
            complete(inflight.front());
            inflight.pop_front();
            progressed = true;
        }
        if (inflight.size() < 2) {
            std::lock_guard<std::mutex> lk(form_mu);
            int r = form_and_launch();
            if (r < 0) engine_error.store(-1);
            if (r > 0) progressed = true;
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(cv_mu);
            cv.wait_for(lk, std::chrono::microseconds(inflight.empty() ? 2000 : 20));
        }
    }
    for (auto& bt : inflight) {
        cudaEventSynchronize(bt.ev1);
        complete(bt);
    }
    inflight.clear();
}

namespace {

int capture_graph(cyc_server* s, int b)
{
    cudaGraph_t g = nullptr;
    SCK(cudaStreamBeginCapture(s->cst, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(s->d_counter, 0, sizeof(int), s->cst);
    tc_launch_items(s->d_items[b], s->d_counts[b], s->d_counter, s->grid, s->p.precision, s->d_err, 0, s->cst);
    fold_kernel<<<s->num_sms * 4, 256, 0, s->cst>>>(s->d_folds[b], s->d_counts[b] + 1, s->slots, tc_tile_rows(),
                                                    tc_tile_cols());
    cudaError_t e = cudaStreamEndCapture(s->cst, &g);
    if (e != cudaSuccess) return sfail(CYC_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&s->graph[b], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return sfail(CYC_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    return CYC_OK;
}

void destroy_server(cyc_server* s)
{
    if (s->engine.joinable()) {
        s->stop.store(true);
        s->cv.notify_all();
        s->engine.join();
    }
    if (s->cst) cudaStreamSynchronize(s->cst);
    for (auto& st : s->streams)
        if (st) st->release();
    for (auto& bt : s->spare) {
        cudaEventDestroy(bt.ev0);
        cudaEventDestroy(bt.ev1);
    }
    for (int b = 0; b < 2; ++b) {
        if (s->graph[b]) cudaGraphExecDestroy(s->graph[b]);
        if (s->h_items[b]) cudaFreeHost(s->h_items[b]);
        if (s->h_folds[b]) cudaFreeHost(s->h_folds[b]);
        if (s->h_counts[b]) cudaFreeHost(s->h_counts[b]);
        if (s->d_items[b]) cudaFree(s->d_items[b]);
        if (s->d_folds[b]) cudaFree(s->d_folds[b]);
        if (s->d_counts[b]) cudaFree(s->d_counts[b]);
    }
    if (s->d_counter) cudaFree(s->d_counter);
    if (s->d_err) cudaFree(s->d_err);
    if (s->slots) cudaFree(s->slots);
    if (s->cst) cudaStreamDestroy(s->cst);
    if (s->xst) cudaStreamDestroy(s->xst);
    delete s;
}

}  // namespace

extern "C" {

int cyc_server_create(const cyc_server_params* pp, cyc_server** out)
{
    if (!pp || !out) return sfail(CYC_EINVAL, "cyc_server_create: NULL argument");
    *out = nullptr;
    cyc_server_params p = *pp;
    if (p.max_streams <= 0) p.max_streams = 256;
    if (p.max_items <= 0) p.max_items = 1024;
    if (p.item_samples <= 0) p.item_samples = 65536;
    if (p.ring_samples <= 0) p.ring_samples = 1 << 22;
    if (p.precision != CYC_P_FP16 && p.precision != CYC_P_BF16X3)
        return sfail(CYC_EINVAL, "cyc_server_create: precision must be CYC_P_FP16 or CYC_P_BF16X3");
    if (p.max_streams > 65536 || p.max_items > (1 << 20) || p.ring_samples > (1ll << 32) || p.item_samples > (1ll << 30))
        return sfail(CYC_EINVAL, "cyc_server_create: parameter out of range");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || p.device < 0 || p.device >= ndev) {
        cudaGetLastError();
        return sfail(CYC_ECUDA, "cyc_server_create: device %d is not available", p.device);
    }
    DevGuard g(p.device);
    cyc_server* s = new (std::nothrow) cyc_server();
    if (!s) return sfail(CYC_ENOMEM, "cyc_server_create: host allocation failed");
    s->p = p;
    int rc = CYC_OK;
    auto chk = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && rc == CYC_OK)
            rc = sfail(e == cudaErrorMemoryAllocation ? CYC_ENOMEM : CYC_ECUDA, "cyc_server_create: %s: %s", what,
                       cudaGetErrorString(e));
    };
    chk(cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, p.device), "SM count");
    if (p.mem_budget == 0) {
        size_t fr = 0, tot = 0;
        chk(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
        s->p.mem_budget = fr / 2;
    }
    chk(cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking), "compute stream");
    chk(cudaStreamCreateWithFlags(&s->xst, cudaStreamNonBlocking), "copy stream");
    const int64_t tile = (int64_t)tc_tile_rows() * tc_tile_cols();
    {
        const int pc = tc_pair_ctas(p.precision);
        if (pc < 2 && rc == CYC_OK)
            rc = sfail(CYC_ENOTSUP, "cyc_server_create: the device cannot hold the two-CTA clusters the server runs on");
        s->grid = (pc < s->num_sms ? pc : s->num_sms) & ~1;
        if (s->grid < 2) s->grid = 2;
    }
    s->nslot_cap = (int64_t)p.max_items;                 // one partial tile per item
    for (int b = 0; b < 2 && rc == CYC_OK; ++b) {
        chk(cudaMallocHost(&s->h_items[b], sizeof(TcItem) * p.max_items), "pinned items");
        chk(cudaMallocHost(&s->h_folds[b], sizeof(Fold) * p.max_items), "pinned folds");
        chk(cudaMallocHost(&s->h_counts[b], 2 * sizeof(int)), "pinned counts");
        chk(cudaMalloc(&s->d_items[b], sizeof(TcItem) * p.max_items), "items");
        chk(cudaMalloc(&s->d_folds[b], sizeof(Fold) * p.max_items), "folds");
        chk(cudaMalloc(&s->d_counts[b], 2 * sizeof(int)), "counts");
        if (rc == CYC_OK) chk(cudaMemset(s->d_counts[b], 0, 2 * sizeof(int)), "counts");
    }
    if (rc == CYC_OK) chk(cudaMalloc(&s->d_counter, sizeof(int)), "counter");
    if (rc == CYC_OK) chk(cudaMalloc(&s->d_err, sizeof(int)), "status");
    if (rc == CYC_OK) chk(cudaMemset(s->d_err, 0, sizeof(int)), "status");
    if (rc == CYC_OK) chk(cudaMalloc(&s->slots, sizeof(float2) * tile * s->nslot_cap), "partial tiles");
    if (rc == CYC_OK) {
        // an empty launch fixes the kernel's shared-memory attribute before capture
        chk(cudaMemset(s->d_counter, 0, sizeof(int)), "counter");
        chk(tc_launch_items(s->d_items[0], s->d_counts[0], s->d_counter, 2, p.precision, s->d_err, 0, s->cst),
            "warm-up");
        chk(cudaStreamSynchronize(s->cst), "warm-up");
    }
    for (int b = 0; b < 2 && rc == CYC_OK; ++b) rc = capture_graph(s, b);
    if (rc == CYC_OK) {
        s->streams.resize(p.max_streams);
        for (auto& st : s->streams) st.reset(new SrvStream());
        s->engine = std::thread([s] { s->run(); });
    }
    if (rc != CYC_OK) {
        destroy_server(s);
        return rc;
    }
    *out = s;
    return CYC_OK;
}

int cyc_server_destroy(cyc_server* srv)
{
    if (!srv) return CYC_OK;
    DevGuard g(srv->p.device);
    destroy_server(srv);
    return CYC_OK;
}

int cyc_server_open(cyc_server* srv, const int32_t* lags, int nlags, const double* alphas, int nalphas,
                    int conj_flag, int64_t n0, int* sid)
{
    if (!srv || !lags || !alphas || !sid) return sfail(CYC_EINVAL, "cyc_server_open: NULL argument");
    if (nlags <= 0 || nalphas <= 0) return sfail(CYC_EINVAL, "cyc_server_open: empty lag or cycle-frequency list");
    if (conj_flag < 1 || conj_flag > 3) return sfail(CYC_EINVAL, "cyc_server_open: conj_flag must be 1, 2 or 3");
    int32_t M = 0;
    for (int i = 0; i < nlags; ++i) {
        if (lags[i] < 0) return sfail(CYC_EINVAL, "cyc_server_open: lag %d is negative", i);
        M = lags[i] > M ? lags[i] : M;
    }
    for (int i = 0; i < nalphas; ++i)
        if (!isfinite(alphas[i])) return sfail(CYC_EINVAL, "cyc_server_open: cycle frequency %d is not finite", i);
    const int F = (conj_flag & CYC_CONV ? 1 : 0) + (conj_flag & CYC_CONJ ? 1 : 0);
    if (!tc_supported(nlags * F, M)) return sfail(CYC_ENOTSUP, "cyc_server_open: max lag %d exceeds 2560", M);
    // distinct cycle frequencies, lag-major columns
    std::map<uint64_t, int> uniq;
    std::vector<uint64_t> phi_u;
    std::vector<int32_t> amap(nalphas);
    for (int i = 0; i < nalphas; ++i) {
        uint64_t ph = 0;
        cyc_phase_increment(alphas[i], &ph);
        auto it = uniq.find(ph);
        if (it == uniq.end()) {
            it = uniq.emplace(ph, (int)phi_u.size()).first;
            phi_u.push_back(ph);
        }
        amap[i] = it->second;
    }
    const int Au = (int)phi_u.size(), ncols = nlags * F;
    const UnitLayout units = order_units(phi_u, amap);
    const int forms[2] = {conj_flag & CYC_CONV ? CYC_CONV : CYC_CONJ, CYC_CONJ};
    std::vector<int32_t> cl(ncols);
    std::vector<int8_t> cc(ncols);
    for (int l = 0; l < nlags; ++l)
        for (int f = 0; f < F; ++f) {
            cl[l * F + f] = lags[l];
            cc[l * F + f] = forms[f] == CYC_CONJ ? 1 : 0;
        }
    const uint64_t cap = next_pow2((uint64_t)std::max<int64_t>(srv->p.ring_samples, 4 * 4096 + 2 * (int64_t)M));
    const size_t bytes = cap * sizeof(float2) + (size_t)Au * ncols * sizeof(double2) + Au * sizeof(uint64_t) +
                         nalphas * sizeof(int32_t) + ncols * 5 + (size_t)F * nalphas * nlags * sizeof(double2);
    DevGuard g(srv->p.device);
    std::lock_guard<std::mutex> lk(srv->admin);
    test_alloc_arm();
    int slot = -1;
    for (int i = 0; i < (int)srv->streams.size(); ++i)
        if (!srv->streams[i]->open && !srv->streams[i]->closing.load()) {
            slot = i;
            break;
        }
    if (slot < 0) return sfail(CYC_EAGAIN, "cyc_server_open: all %d stream slots are in use", (int)srv->streams.size());
    if (srv->used + bytes > srv->p.mem_budget)
        return sfail(CYC_EAGAIN, "cyc_server_open: %zu more bytes would exceed the budget (%llu of %llu held)", bytes,
                     (unsigned long long)srv->used, (unsigned long long)srv->p.mem_budget);
    SrvStream& s = *srv->streams[slot];
    s.F = F; s.L = nlags; s.A = nalphas; s.Au = Au; s.ncols = ncols; s.M = M; s.n0 = n0;
    s.cap = cap;
    s.units = units;
    auto fail_free = [&](cudaError_t e, const char* what) {
        s.release();
        return sfail(e == cudaErrorMemoryAllocation ? CYC_EAGAIN : CYC_ECUDA, "cyc_server_open: %s: %s", what,
                     cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = dev_malloc((void**)&s.ring, cap * sizeof(float2))) != cudaSuccess) return fail_free(e, "ring");
    if ((e = dev_malloc((void**)&s.sums, (size_t)Au * ncols * sizeof(double2))) != cudaSuccess) return fail_free(e, "sums");
    if ((e = dev_malloc((void**)&s.d_phi, Au * sizeof(uint64_t))) != cudaSuccess) return fail_free(e, "tables");
    if ((e = dev_malloc((void**)&s.d_amap, nalphas * sizeof(int32_t))) != cudaSuccess) return fail_free(e, "tables");
    if ((e = dev_malloc((void**)&s.d_col_lag, ncols * sizeof(int32_t))) != cudaSuccess) return fail_free(e, "tables");
    if ((e = dev_malloc((void**)&s.d_col_conj, ncols * sizeof(int8_t))) != cudaSuccess) return fail_free(e, "tables");
    if ((e = dev_malloc((void**)&s.d_out, (size_t)F * nalphas * nlags * sizeof(double2))) != cudaSuccess)
        return fail_free(e, "read buffer");
    if ((e = cudaMemset(s.sums, 0, (size_t)Au * ncols * sizeof(double2))) != cudaSuccess ||
        (e = cudaMemcpy(s.d_phi, phi_u.data(), Au * sizeof(uint64_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(s.d_amap, amap.data(), nalphas * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(s.d_col_lag, cl.data(), ncols * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(s.d_col_conj, cc.data(), ncols * sizeof(int8_t), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail_free(e, "initialisation");
    s.bytes = bytes;
    s.T.store(0);
    s.n_done.store(0);
    s.n_sched.store(0);
    {
        std::lock_guard<std::mutex> lk2(s.mu);
        s.recs.clear();
    }
    srv->used += bytes;
    s.open.store(true, std::memory_order_release);
    *sid = slot;
    return CYC_OK;
}

int cyc_server_submit(cyc_server* srv, int sid, const void* chunk, int64_t nsamples, uint64_t tag)
{
    if (!srv || sid < 0 || sid >= (int)srv->streams.size()) return sfail(CYC_EINVAL, "cyc_server_submit: bad server or stream id");
    SrvStream& s = *srv->streams[sid];
    if (!s.open || s.closing.load()) return sfail(CYC_EINVAL, "cyc_server_submit: stream %d is not open", sid);
    if (nsamples < 0 || (nsamples > 0 && !chunk)) return sfail(CYC_EINVAL, "cyc_server_submit: bad chunk");
    if (nsamples == 0) return CYC_OK;
    if (nsamples > (int64_t)s.cap - 2 * s.M - 16)
        return sfail(CYC_EINVAL, "cyc_server_submit: chunk of %lld samples exceeds the stream ring", (long long)nsamples);
    if (srv->engine_error.load()) return sfail(CYC_ECUDA, "cyc_server_submit: the server engine has failed");
    DevGuard g(srv->p.device);
    std::lock_guard<std::mutex> lk(s.mu);
    const int64_t T = s.T.load();
    // the ring keeps every sample from the first uncommitted term on
    if (T + nsamples - s.n_done.load() > (int64_t)s.cap)
        return sfail(CYC_EAGAIN, "cyc_server_submit: ring of stream %d is full, retry", sid);
    const uint64_t pos = (uint64_t)T & (s.cap - 1);
    const uint64_t first = std::min<uint64_t>((uint64_t)nsamples, s.cap - pos);
    const float2* src = (const float2*)chunk;
    SCK(cudaMemcpyAsync(s.ring + pos, src, first * sizeof(float2), cudaMemcpyDefault, srv->xst));
    if (first < (uint64_t)nsamples)
        SCK(cudaMemcpyAsync(s.ring, src + first, (nsamples - first) * sizeof(float2), cudaMemcpyDefault, srv->xst));
    SCK(cudaStreamSynchronize(srv->xst));
    s.recs.push_back(Rec{T + nsamples, tag, nsamples, now_s()});
    srv->outstanding++;
    s.T.store(T + nsamples);
    srv->cv.notify_one();
    return CYC_OK;
}

int cyc_server_poll(cyc_server* srv, cyc_done* done, int max, int* ndone)
{
    if (!srv || !ndone || (max > 0 && !done)) return sfail(CYC_EINVAL, "cyc_server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(srv->done_mu);
    int n = 0;
    while (n < max && !srv->done_q.empty()) {
        done[n++] = srv->done_q.front();
        srv->done_q.pop_front();
    }
    *ndone = n;
    return srv->engine_error.load() ? sfail(CYC_ECUDA, "cyc_server_poll: the server engine has failed") : CYC_OK;
}

int cyc_server_drain(cyc_server* srv, double timeout_s)
{
    if (!srv) return sfail(CYC_EINVAL, "cyc_server_drain: NULL server");
    const double t_end = now_s() + timeout_s;
    std::unique_lock<std::mutex> lk(srv->done_mu);
    while (srv->outstanding.load() > 0) {
        // chunks shorter than the lag span finish only with a later chunk: they count as done
        // once everything submitted so far is in the sums
        bool all_in = true;
        for (auto& st : srv->streams)
            if (st->open.load() && st->n_done.load() < st->T.load() - st->M) all_in = false;
        if (all_in) break;
        if (srv->engine_error.load()) return sfail(CYC_ECUDA, "cyc_server_drain: the server engine has failed");
        if (now_s() > t_end) return sfail(CYC_ETIMEDOUT, "cyc_server_drain: timed out");
        srv->done_cv.wait_for(lk, std::chrono::milliseconds(1));
    }
    return CYC_OK;
}

int cyc_server_read(cyc_server* srv, int sid, double* out, int64_t* n_eff)
{
    if (!srv || sid < 0 || sid >= (int)srv->streams.size() || !out) return sfail(CYC_EINVAL, "cyc_server_read: bad argument");
    SrvStream& s = *srv->streams[sid];
    if (!s.open) return sfail(CYC_EINVAL, "cyc_server_read: stream %d is not open", sid);
    const double t_end = now_s() + 60.0;
    const int64_t want = std::max<int64_t>(0, s.T.load() - s.M);
    while (s.n_done.load() < want) {
        if (srv->engine_error.load()) return sfail(CYC_ECUDA, "cyc_server_read: the server engine has failed");
        if (now_s() > t_end) return sfail(CYC_ETIMEDOUT, "cyc_server_read: stream %d did not finish", sid);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    if (n_eff) *n_eff = want;
    if (want == 0) return sfail(CYC_ENODATA, "cyc_server_read: N_eff is 0");
    DevGuard g(srv->p.device);
    cudaPointerAttributes at;
    bool dev = cudaPointerGetAttributes(&at, out) == cudaSuccess &&
               (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev && ((uintptr_t)out & 15) != 0) return sfail(CYC_EINVAL, "cyc_server_read: device out must be 16-byte aligned");
    double2* dst = dev ? (double2*)out : s.d_out;
    // the sums were last written by a batch on the compute stream
    SCK(read_sums(s.sums, s.d_amap, s.F, s.A, s.L, s.ncols, 1.0 / (double)want, dst, srv->cst));
    if (!dev)
        SCK(cudaMemcpyAsync(out, s.d_out, (size_t)s.F * s.A * s.L * sizeof(double2), cudaMemcpyDeviceToHost, srv->cst));
    SCK(cudaStreamSynchronize(srv->cst));
    return CYC_OK;
}

int cyc_server_close(cyc_server* srv, int sid)
{
    if (!srv || sid < 0 || sid >= (int)srv->streams.size()) return sfail(CYC_EINVAL, "cyc_server_close: bad argument");
    SrvStream& s = *srv->streams[sid];
    if (!s.open) return sfail(CYC_EINVAL, "cyc_server_close: stream %d is not open", sid);
    s.closing.store(true);
    { std::lock_guard<std::mutex> lk(srv->form_mu); }   // no batch formation is using the stream now
    // wait for the batches that still read this stream (the engine forms no new ones)
    const double t_end = now_s() + 60.0;
    for (;;) {
        if (s.n_done.load() >= s.n_sched.load()) break;
        if (now_s() > t_end) return sfail(CYC_ETIMEDOUT, "cyc_server_close: stream %d did not finish", sid);
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    DevGuard g(srv->p.device);
    cudaStreamSynchronize(srv->cst);
    {
        std::lock_guard<std::mutex> lk(s.mu);
        int64_t dropped = (int64_t)s.recs.size();
        s.recs.clear();
        srv->outstanding -= dropped;
    }
    std::lock_guard<std::mutex> lk(srv->admin);
    s.open.store(false);
    s.release();
    srv->used -= s.bytes;
    s.bytes = 0;
    s.closing.store(false);
    return CYC_OK;
}

int cyc_server_stats(cyc_server* srv, int64_t* batches, int64_t* items, double* busy_ms, uint64_t* bytes_held)
{
    if (!srv) return sfail(CYC_EINVAL, "cyc_server_stats: NULL server");
    if (batches) *batches = srv->n_batches.load();
    if (items) *items = srv->n_items.load();
    if (busy_ms) *busy_ms = srv->busy_ms.load();
    if (bytes_held) *bytes_held = srv->used;
    return CYC_OK;
}

}  // extern "C"
