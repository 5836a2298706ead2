// cyc_static.cu -- cyc_estimate_static: a one-shot estimate that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need an estimate:
// a real-time signal-processing callback that must not call cudaMalloc/cudaFree (they can
// synchronise the whole device and take unbounded time), or a plug-in inside a host
// application whose own memory pool has already reserved the GPU's memory.  For them this
// entry point runs the FP32 projection kernel with all of its scratch (the cycle-frequency
// and column tables and the FP32 partial sums) in one file-scope device array of fixed
// size, and folds the partials straight into the caller's output buffer in FP64.
//
// The array belongs to this file's module.  CUDA loads modules lazily by default, so the
// array (kScratchBytes, about 8.1 MiB) and the kernels are brought onto a device by the
// first call on that device, which also looks up the array's device address; from then on
// the array stays resident until the process exits.  A caller whose host application
// reserves the device memory must therefore make one call (any valid size) before that, or
// run with CUDA_MODULE_LOADING=EAGER so that the module loads with the context.  The tables
// a call needs are written into the array by kernels that carry them as launch parameters,
// so a call only queues work and never waits for the stream.
// Every call shares the array and it keeps the previous call's contents; everything a call
// reads from it is written by that same call first.  Two calls whose GPU work overlaps
// (calls on different CUDA streams) race on the array and give wrong results; calls on one
// stream are ordered and safe.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>

#include "cyc_impl.h"

using namespace cyc;

namespace {

constexpr int kMaxAlphas = 4096;                 // cycle frequencies per call
constexpr int kMaxCols = 2048;                   // lags x forms per call
constexpr size_t kMaxPartials = (size_t)1 << 20; // FP32 complex partial sums (8 MiB)
constexpr int64_t kPassSamples = (int64_t)1 << 20;
constexpr int kMaxDevices = 64;

// byte layout of the scratch array
constexpr size_t kOffPhi = 0;                                        // uint64_t[kMaxAlphas]
constexpr size_t kOffLag = kOffPhi + kMaxAlphas * sizeof(uint64_t);  // int32_t[kMaxCols]
constexpr size_t kOffConj = kOffLag + kMaxCols * sizeof(int32_t);    // int8_t[kMaxCols]
constexpr size_t kOffPart = (kOffConj + kMaxCols + 255) / 256 * 256; // float2[kMaxPartials]
constexpr size_t kScratchBytes = kOffPart + kMaxPartials * sizeof(float2);

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Device address of g_static_scratch per device (host code cannot use the symbol itself).
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices];

// Errors go to the same thread-local message that cyc_last_error() returns.
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

// out[f][a][l] = (first ? 0 : out) + sum_s part[s][a][l*F + f], then times `scale`.
__global__ void static_fold_kernel(const float2* __restrict__ part, int nsplit, int A, int L, int F,
                                   int first, double scale, double2* __restrict__ out)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = (int64_t)F * A * L;
    if (e >= total) return;
    int l = (int)(e % L);
    int a = (int)((e / L) % A);
    int f = (int)(e / ((int64_t)A * L));
    int ncols = L * F;
    size_t idx = (size_t)a * ncols + (size_t)l * F + f;
    double sr = 0.0, si = 0.0;
    for (int s = 0; s < nsplit; ++s) {
        float2 v = part[(size_t)s * A * ncols + idx];
        sr += (double)v.x;
        si += (double)v.y;
    }
    double2 o = first ? make_double2(0.0, 0.0) : out[e];
    out[e] = make_double2((o.x + sr) * scale, (o.y + si) * scale);
}

// A slice of the tables, passed by value as the launch's parameters (a few KB), copied into
// the scratch array: no host-to-device copy from pageable memory, which could make the
// call wait for the stream.
constexpr int kTableBytes = 3968;
struct TableSlice {
    unsigned char* dst;
    uint32_t       nbytes;
    uint32_t       pad;
    unsigned char  data[kTableBytes];
};

__global__ void table_kernel(TableSlice t)
{
    for (uint32_t i = threadIdx.x; i < t.nbytes; i += blockDim.x) t.dst[i] = t.data[i];
}

uint64_t phase_step(double a)
{
    uint64_t phi = 0;
    cyc_phase_increment(a, &phi);
    return phi;
}

// Device or managed memory of device `dev` (managed memory reports the device it was
// allocated on).
bool on_device(const void* p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" int cyc_estimate_static(const void* x, int64_t T, const int32_t* lags, int nlags,
                                   const double* alphas, int nalphas, int conj_flag, int64_t n0,
                                   double* out, int64_t* n_eff, void* cuda_stream)
{
    // ---- arguments and limits (nothing is queued on a failure) ----
    if (!x || !out || !lags || !alphas) return sfail(CYC_EINVAL, "cyc_estimate_static: NULL pointer argument");
    if (T < 0) return sfail(CYC_EINVAL, "cyc_estimate_static: T < 0");
    if (nlags <= 0 || nalphas <= 0) return sfail(CYC_EINVAL, "cyc_estimate_static: empty lag or cycle-frequency list");
    if (conj_flag < 1 || conj_flag > 3) return sfail(CYC_EINVAL, "cyc_estimate_static: conj_flag must be 1, 2 or 3");
    const int F = (conj_flag & CYC_CONV ? 1 : 0) + (conj_flag & CYC_CONJ ? 1 : 0);
    if (nalphas > kMaxAlphas)
        return sfail(CYC_EINVAL, "cyc_estimate_static: %d cycle frequencies exceed the limit of %d", nalphas, kMaxAlphas);
    if ((int64_t)nlags * F > kMaxCols)
        return sfail(CYC_EINVAL, "cyc_estimate_static: %d lags x %d forms exceed the limit of %d columns", nlags, F,
                     kMaxCols);
    if ((size_t)nalphas * nlags * F > kMaxPartials)
        return sfail(CYC_EINVAL, "cyc_estimate_static: %d cycle frequencies x %d columns exceed the %zu partial sums "
                     "of the static scratch", nalphas, nlags * F, kMaxPartials);
    int32_t M = 0;
    for (int i = 0; i < nlags; ++i) {
        if (lags[i] < 0) return sfail(CYC_EINVAL, "cyc_estimate_static: lag %d is negative", i);
        if (lags[i] > M) M = lags[i];
    }
    for (int i = 0; i < nalphas; ++i)
        if (!isfinite(alphas[i])) return sfail(CYC_EINVAL, "cyc_estimate_static: cycle frequency %d is not finite", i);
    const int64_t nc = T - M;
    if (n_eff) *n_eff = nc > 0 ? nc : 0;
    if (nc <= 0) return sfail(CYC_ENODATA, "cyc_estimate_static: N_eff is 0 (T <= max lag)");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return sfail(CYC_ECUDA, "cyc_estimate_static: no usable current CUDA device");
    }
    if (!on_device(x, dev) || !on_device(out, dev))
        return sfail(CYC_EINVAL, "cyc_estimate_static: x and out must be memory of the current device %d", dev);
    if (((uintptr_t)x & 7) != 0 || ((uintptr_t)out & 15) != 0)
        return sfail(CYC_EINVAL, "cyc_estimate_static: x must be 8-byte and out 16-byte aligned");

    // ---- once per device: the device address of the scratch array ----
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p)
                return sfail(CYC_ECUDA, "cyc_estimate_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            g_scratch_addr[dev] = p;
        }
        base = (unsigned char*)g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // ---- tables: built on the stack, written into the scratch array in stream order by
    // kernels that carry them as launch parameters ----
    const int ncols = nlags * F;
    unsigned char tab[kOffConj + kMaxCols];
    uint64_t* phi = (uint64_t*)(tab + kOffPhi);
    int32_t* col_lag = (int32_t*)(tab + kOffLag);
    int8_t* col_conj = (int8_t*)(tab + kOffConj);
    for (int i = 0; i < nalphas; ++i) phi[i] = phase_step(alphas[i]);
    const int forms[2] = {conj_flag & CYC_CONV ? CYC_CONV : CYC_CONJ, CYC_CONJ};
    for (int l = 0; l < nlags; ++l)
        for (int f = 0; f < F; ++f) {
            col_lag[l * F + f] = lags[l];
            col_conj[l * F + f] = forms[f] == CYC_CONJ ? 1 : 0;
        }
    cudaError_t e;
    const size_t spans[3][2] = {{kOffPhi, (size_t)nalphas * sizeof(uint64_t)},
                                {kOffLag, (size_t)ncols * sizeof(int32_t)},
                                {kOffConj, (size_t)ncols}};
    for (const auto& sp : spans)
        for (size_t o = 0; o < sp[1]; o += kTableBytes) {
            TableSlice t;
            t.dst = base + sp[0] + o;
            t.nbytes = (uint32_t)(sp[1] - o < (size_t)kTableBytes ? sp[1] - o : (size_t)kTableBytes);
            t.pad = 0;
            memcpy(t.data, tab + sp[0] + o, t.nbytes);
            table_kernel<<<1, 256, 0, st>>>(t);
            if ((e = cudaGetLastError()) != cudaSuccess)
                return sfail(CYC_ECUDA, "cyc_estimate_static: table launch failed: %s", cudaGetErrorString(e));
        }

    int num_sms = 1;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    const int max_split = (int)(kMaxPartials / ((size_t)nalphas * ncols));

    // ---- passes of at most kPassSamples committed terms, folded into `out` in FP64 ----
    const float2* xv = (const float2*)x;
    for (int64_t p0 = 0; p0 < nc; p0 += kPassSamples) {
        int64_t np = nc - p0 < kPassSamples ? nc - p0 : kPassSamples;
        ProjPlan pl = fp32_plan(nalphas, ncols, np, num_sms);
        if (pl.nsplit > max_split) {
            pl.nsplit = max_split;
            pl.split_len = ((np + max_split - 1) / max_split + 15) / 16 * 16;
            pl.nsplit = (int)((np + pl.split_len - 1) / pl.split_len);
        }
        ProjArgs a;
        a.x = xv + p0;
        a.nc = np;
        a.nbase = (uint64_t)n0 + (uint64_t)p0;
        a.phi = (const uint64_t*)(base + kOffPhi);
        a.Au = nalphas;
        a.col_lag = (const int32_t*)(base + kOffLag);
        a.col_conj = (const int8_t*)(base + kOffConj);
        a.ncols = ncols;
        a.nsplit = pl.nsplit;
        a.split_len = pl.split_len;
        a.part = (float2*)(base + kOffPart);
        if ((e = fp32_launch(a, st)) != cudaSuccess)
            return sfail(CYC_ECUDA, "cyc_estimate_static: projection launch failed: %s", cudaGetErrorString(e));
        const bool last = p0 + np >= nc;
        int64_t total = (int64_t)F * nalphas * nlags;
        static_fold_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            a.part, pl.nsplit, nalphas, nlags, F, p0 == 0 ? 1 : 0, last ? 1.0 / (double)nc : 1.0, (double2*)out);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return sfail(CYC_ECUDA, "cyc_estimate_static: fold launch failed: %s", cudaGetErrorString(e));
    }
    return CYC_OK;
}
