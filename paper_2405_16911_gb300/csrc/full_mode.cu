// full_mode.cu -- the estimator on a uniform cycle-frequency grid a_k = -1/2 + k/A (the
// paper's Full mode, Sec. 4: every cycle frequency of [-1/2, 1/2) at resolution 1/A).
//
// For a_k on that grid the phase term depends on the absolute sample index n only through
// n mod A (A even):  exp(-j 2 pi a_k n) = (-1)^n exp(-j 2 pi k n / A), and (-1)^n = (-1)^r
// for r = n mod A.  So
//     sum_n P_c(n) exp(-j 2 pi a_k n) = sum_{r<A} (-1)^r F_c[r] exp(-j 2 pi k r / A),
//     F_c[r] = sum_{n = r mod A} P_c(n),
// an A-point DFT of the lag products folded modulo A.  A push only folds (O(samples x
// columns) work instead of the O(samples x columns x A) projection); the DFT runs when the
// estimate is read.  F lives in the stream's sums array as
// float-float pairs (re hi, re lo, im hi, im lo: 16 bytes like a double2, about 48
// significant bits), [ncols][A] (a warp's residues are neighbours in memory for the fold
// and for the read), so reset, save and load work unchanged; the fold does no FP64
// arithmetic (this GPU's FP64 rate is a small fraction of its FP32 rate) and the read
// converts to FP64 before its FP64 DFT.
#include "cyc_device.cuh"
#include "cyc_impl.h"

namespace cyc {
namespace {

constexpr int FJ = 64;                  // offsets j per tile
constexpr int FLT = 16;                 // lags per tile
constexpr int FOW = 2;                  // warps per row group: offsets 32 ow .. 32 ow + 31
constexpr int FQG = 8;                  // row groups (rows q = g mod 8 of each batch)
constexpr int FWARPS = FOW * FQG;
constexpr int FT = 32 * FWARPS;         // threads per CTA
constexpr int FNBUF = 4;                // staged slots in flight per row group
constexpr int FR = FOW;                 // rows per slot: one per warp of the group
constexpr int FRUN = 256;               // rows between additions to the float-float tile
constexpr int FPAIRS = 16;              // (lag, offset) pairs per thread: 4 lags x 4 offsets
constexpr int FSLOTS = FPAIRS * FOW * 32;   // the tile's (lag, offset) pairs
// shared memory beside the row groups' rings: the tree reduction of the row groups' sums
// (FQG / 2 groups of FSLOTS float4) and the tile's fold entries (2 forms x FSLOTS float4)
constexpr size_t kRedBytes = (size_t)(FQG / 2) * FSLOTS * sizeof(float4) + (size_t)2 * FSLOTS * sizeof(float4);
constexpr size_t kFoldSmem = 224 * 1024;
constexpr int kXlMax = 184;             // widest staged x window: the rings fit beside the tree

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 8-byte asynchronous global -> shared copy; bytes = 0 stores zeros and reads nothing
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Two FP32 fused multiply-adds in one instruction: (a.x b.x + c.x, a.y b.y + c.y), each
// rounded as fmaf would round it.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// The pass's source table, copied to shared memory (indexed at run time).
struct SrcTab {
    int n;
    int start[kFoldSrc + 1];
    const float2* x[kFoldSrc];
    const float2* y[kFoldSrc];
};

// The source holding view sample v, searched forward from s (a lower bound).
__device__ __forceinline__ int src_from(const SrcTab& t, int v, int s)
{
    while (s + 1 < t.n && t.start[s + 1] <= v) ++s;
    return s;
}

__device__ __forceinline__ void ff_add2(float4& t, float re, float im)
{
    ff_add(t.x, t.y, re);
    ff_add(t.z, t.w, im);
}

// Slot of a (lag, offset) pair of the tile: pair (k, i) of lane (t_l, t_o) in warp ow is lag
// 4 t_l + k and offset 32 ow + 4 t_o + i (lane = 8 t_l + t_o); slots run lane-fastest, so
// that a warp touching one pair of each of its lanes touches 32 neighbouring slots.
__device__ __forceinline__ int slot_of(int pr, int ow, int lane) { return (pr * FOW + ow) * 32 + lane; }
__device__ __forceinline__ void slot_pair(int s, int& lag, int& off)
{
    const int lane = s & 31, ow = (s >> 5) % FOW, pr = s / (32 * FOW);
    lag = 4 * (lane >> 3) + (pr >> 2);
    off = 32 * ow + 4 * (lane & 7) + (pr & 3);
}

// Stage row q of a tile: x samples [vx, vx + xl) of the view (none when X is false) and y
// samples [vy, vy + 64), zero where not live.  One warp per row, 8-byte asynchronous copies,
// a plain loop where the row lies inside one source.  cx, cy: the warp's source cursors
// (rows are staged in increasing order).
template <bool X>
__device__ __forceinline__ void stage_row(const FoldArgs& a, const SrcTab& t, uint32_t dst, int lane, int xl,
                                          int nview, int row0, bool live, int mlo, int& cx, int& cy)
{
    const float2* zero = t.x[0];
    if (X) {
        const int vx = row0 + mlo + (int)a.off;
        cx = src_from(t, vx, cx);
        if (live && vx + xl <= t.start[cx + 1]) {
            const float2* src = t.x[cx] + (vx - t.start[cx]);
            for (int cc = lane; cc < xl; cc += 32) cp_async8(dst + (uint32_t)cc * 8u, src + cc, 8u);
        } else {
            for (int cc = lane; cc < xl; cc += 32) {
                const int v = vx + cc;
                const bool ok = live && v < nview;
                const int s = ok ? src_from(t, v, cx) : 0;
                cp_async8(dst + (uint32_t)cc * 8u, ok ? t.x[s] + (v - t.start[s]) : zero, ok ? 8u : 0u);
            }
        }
    }
    const int vy = row0 + (int)a.off + a.D;
    const uint32_t dy = dst + (uint32_t)xl * 8u;
    cy = src_from(t, vy, cy);
    if (live && row0 + FJ <= (int)a.nc && vy + FJ <= t.start[cy + 1]) {
        const float2* src = t.y[cy] + (vy - t.start[cy]);
        for (int jj = lane; jj < FJ; jj += 32) cp_async8(dy + (uint32_t)jj * 8u, src + jj, 8u);
    } else {
        for (int jj = lane; jj < FJ; jj += 32) {
            const bool ok = live && row0 + jj < (int)a.nc;
            const int s = ok ? src_from(t, vy + jj, cy) : 0;
            cp_async8(dy + (uint32_t)jj * 8u, ok ? t.y[s] + (vy + jj - t.start[s]) : zero, ok ? 8u : 0u);
        }
    }
}

// One pass of a Full-mode stream.  Term i of the pass (i < nc) adds
//     x[i + m] conj(y[i + D])  and  x[i + m] y[i + D]
// to the fold entries of residue (i + base_mod) mod A, for every lag m (shifted, m + M^- >= 0).
// With the four real sums  P_A = sum xr yr,  P_B = sum xi yi,  P_C = sum xi yr,  P_D = sum xr yi
// both forms follow:  x conj(y) = (P_A + P_B, P_C - P_D),  x y = (P_A - P_B, P_C + P_D); the
// pairs (P_A, P_C) and (P_D, P_B) are x times (yr, yr) and (yi, yi), two paired FMAs per term.
//
// Tile (blockIdx.x, blockIdx.y): the 64 offsets j0 .. j0 + 63 and the 16 lags at sorted
// positions 16 blockIdx.y .. + 15, which own their fold entries: the CTA copies them into
// shared memory and writes them back once at the end (A < 64: the 64 / A offsets of a residue
// hold separate entries, added together in a fixed order at the write-back).  Row q of the
// tile holds the terms i = j0 + j + q S (S = max(A, 64): each offset keeps its residue from
// row to row).  Row group g (two warps, ow = 0, 1: offsets 32 ow .. 32 ow + 31) takes the rows
// q = g mod 8 and runs its own pipeline: FNBUF slots of FR rows in shared memory, each warp
// staging one row per slot with 8-byte asynchronous copies (the x samples of the tile's lags
// and the 64 y samples, zero where i >= nc so that partial rows add nothing), the pair
// meeting at a named barrier of its own.  Each lane takes 4 lags x 4 offsets.  MODE 0 (every
// tile's lags consecutive): the lane's 16 terms need 8 x and 4 y samples, six 16-byte
// shared-memory reads (lanes of equal t_o + t_l read the same x); MODE 1: a window from the
// tile's smallest lag, 16 x samples per lane; MODE 2 (a tile's lags spread wider than the
// window that fits): the x samples come from global memory (cached), only y is staged.  Every FRUN rows the row groups' FP32 sums are added in a fixed
// tree through shared memory and each pair's total, one FP32 run, is added to its
// float-float entry.  The grid also copies the next pass's tail (the view's last `keep`
// samples) to its buffer, so a pass is one launch.  View indices fit in 32 bits (the host
// keeps a pass's view below 2^30 samples).
template <int MODE>
__global__ void __launch_bounds__(FT, 1) fold_kernel(FoldArgs a)
{
    constexpr bool XG = MODE == 2;                           // x read from global memory
    extern __shared__ __align__(16) float2 sm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = wid / FOW, ow = wid % FOW;
    const int t_l = lane >> 3, t_o = lane & 7;
    __shared__ SrcTab tab;
    if (threadIdx.x == 0) tab.n = a.nsrc;
    if (threadIdx.x <= kFoldSrc) tab.start[threadIdx.x] = a.start[threadIdx.x];
    if (threadIdx.x < kFoldSrc) {
        tab.x[threadIdx.x] = a.sx[threadIdx.x];
        tab.y[threadIdx.x] = a.sy[threadIdx.x];
    }
    __syncthreads();
    const int nview = tab.start[tab.n];
    const int ncta = gridDim.x * gridDim.y, cta = blockIdx.y * gridDim.x + blockIdx.x;
    // the next pass's tail, one sample per CTA and thread round: loaded now, stored at the end
    const int keep = (int)a.keep;
    const int t0 = (int)threadIdx.x * ncta + cta;
    float2 tx0 = make_float2(0.f, 0.f), ty0 = tx0;
    if (t0 < keep) {
        const int v = nview - keep + t0, s = src_from(tab, v, 0);
        tx0 = tab.x[s][v - tab.start[s]];
        if (a.ny) ty0 = tab.y[s][v - tab.start[s]];
    }
    const int j0 = blockIdx.x * FJ;
    const int nc = (int)a.nc;
    const int A = a.A;
    const int S = A >= FJ ? A : FJ;
    const int p0 = blockIdx.y * FLT;
    __shared__ int lagidx[FLT], segv[FLT];
    if (nc > j0) {
        if (threadIdx.x < FLT) {
            const int p = p0 + threadIdx.x;
            lagidx[threadIdx.x] = p < a.L ? a.perm[p] : -1;
            segv[threadIdx.x] = p < a.L ? a.sl[p] : 0;
        }
        __syncthreads();
        const int mlo = segv[0];
        const int xl = XG ? 0 : a.xl;
        const int rl = xl + FJ;                              // staged samples per row: x, then y
        const int rows = (nc - j0 + S - 1) / S;
        const int nbg = ((rows + FQG - 1) / FQG + FR - 1) / FR;   // slots each row group runs
        float2* gsm = sm + (size_t)g * FNBUF * FR * rl;                    // the group's ring
        float4* red = reinterpret_cast<float4*>(sm + (size_t)FQG * FNBUF * FR * rl);   // [FQG / 2][FSLOTS]
        float4* fsm = red + (FQG / 2) * FSLOTS;                            // [2][FSLOTS] the tile's fold
        const uint32_t gbase = smem_addr(gsm);
        const int bar = 1 + g;                               // named barrier of the row group

        // group slot bg holds rows q = g + FQG (FR bg + r); warp ow stages r = ow (FR = FOW)
        int cur_x = 0, cur_y = 0;
        auto stage = [&](int bg, int sl_) {
            const int q = g + FQG * (FR * bg + ow);
            stage_row<!XG>(a, tab, gbase + (uint32_t)((sl_ * FR + ow) * rl) * 8u, lane, xl, nview, j0 + q * S,
                           q < rows, mlo, cur_x, cur_y);
        };
#pragma unroll 1
        for (int bg = 0; bg < FNBUF - 1; ++bg) {
            if (bg < nbg) stage(bg, bg);
            cp_async_commit();
        }
        for (int t = threadIdx.x; t < 2 * FSLOTS; t += FT) {            // the tile's fold entries
            const int form = t / FSLOTS, sl = t % FSLOTS;
            int kk, e;
            slot_pair(sl, kk, e);
            const int l = lagidx[kk], f = form == 0 ? a.fV : a.fJ;
            const bool ok = l >= 0 && f >= 0 && (A >= FJ || e < A);
            const float4* src = ok ? a.fold + (size_t)(l * a.F + f) * A +
                                         ((uint32_t)(j0 + e + a.base_mod) & (uint32_t)(A - 1))
                                   : (const float4*)a.fold;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(fsm + t)), "l"(src),
                         "r"(ok ? 16u : 0u) : "memory");
        }
        cp_async_commit();

        int d[4];                                            // x offsets of the lane's four lags
#pragma unroll
        for (int k = 0; k < 4; ++k)
            d[k] = lagidx[4 * t_l + k] < 0 ? (XG ? -(1 << 30) : 0)
                   : XG ? segv[4 * t_l + k] + (int)a.off : segv[4 * t_l + k] - mlo;
        const int obase = 32 * ow + 4 * t_o;                 // the lane's first offset
        float2 pac[FPAIRS], pdb[FPAIRS];                     // (P_A, P_C), (P_D, P_B); pair 4 k + i
#pragma unroll
        for (int pr = 0; pr < FPAIRS; ++pr) pac[pr] = pdb[pr] = make_float2(0.f, 0.f);

        int slot = 0, run = 0;
#pragma unroll 1
        for (int bg = 0; bg < nbg; ++bg) {
            // copy groups: slots 0 .. FNBUF - 2, the fold entries, then one slot per iteration;
            // slot bg has landed once at most FNBUF - 1 (bg < FNBUF - 1) or FNBUF - 2 newer
            // groups are pending
            if (bg < FNBUF - 1)
                cp_async_wait<FNBUF - 1>();
            else
                cp_async_wait<FNBUF - 2>();
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(32 * FOW) : "memory");
            {
                const int bn = bg + FNBUF - 1;
                if (bn < nbg) stage(bn, slot == 0 ? FNBUF - 1 : slot - 1);
                cp_async_commit();
            }
            const float2* buf = gsm + (size_t)slot * FR * rl;
#pragma unroll 1
            for (int r = 0; r < FR; ++r) {
                const float2* xr = buf + r * rl;
                const float4* yq = reinterpret_cast<const float4*>(xr + xl + obase);
                const float4 ya = yq[0], yb = yq[1];
                const float2 yv[4] = {make_float2(ya.x, ya.y), make_float2(ya.z, ya.w), make_float2(yb.x, yb.y),
                                      make_float2(yb.z, yb.w)};
                float2 xv[4][4];
                if (MODE == 0) {
                    const float4* xq = reinterpret_cast<const float4*>(xr + obase + 4 * t_l);
                    float2 xs[8];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float4 u = xq[c];
                        xs[2 * c] = make_float2(u.x, u.y);
                        xs[2 * c + 1] = make_float2(u.z, u.w);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k)
#pragma unroll
                        for (int i = 0; i < 4; ++i) xv[k][i] = xs[k + i];
                } else if (MODE == 1) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
#pragma unroll
                        for (int i = 0; i < 4; ++i) xv[k][i] = xr[obase + d[k] + i];
                } else {
                    const int row0 = j0 + (g + FQG * (FR * bg + r)) * S;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int v = row0 + obase + i + d[k];     // d[k] < 0: no such lag
                            if (v >= 0 && v < nview) {
                                const int sv = src_from(tab, v, 0);
                                xv[k][i] = tab.x[sv][v - tab.start[sv]];
                            } else {
                                xv[k][i] = make_float2(0.f, 0.f);
                            }
                        }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 yr2 = make_float2(yv[i].x, yv[i].x), yi2 = make_float2(yv[i].y, yv[i].y);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        pac[4 * k + i] = ffma2(xv[k][i], yr2, pac[4 * k + i]);
                        pdb[4 * k + i] = ffma2(xv[k][i], yi2, pdb[4 * k + i]);
                    }
                }
            }
            slot = slot == FNBUF - 1 ? 0 : slot + 1;
            run += FR * FQG;
            if (run == FRUN || bg + 1 == nbg) {
                run = 0;
                if (bg < FNBUF - 1) cp_async_wait<0>();      // the fold entries (early flush only)
                // the row groups' sums, added in a fixed tree: groups [h, 2h) hand theirs to [0, h)
#pragma unroll 1
                for (int h = FQG / 2; h >= 1; h >>= 1) {
                    __syncthreads();
                    if (g >= h && g < 2 * h)
#pragma unroll
                        for (int pr = 0; pr < FPAIRS; ++pr)
                            red[(g - h) * FSLOTS + slot_of(pr, ow, lane)] =
                                make_float4(pac[pr].x, pac[pr].y, pdb[pr].x, pdb[pr].y);
                    __syncthreads();
                    if (g < h)
#pragma unroll
                        for (int pr = 0; pr < FPAIRS; ++pr) {
                            const float4 u = red[g * FSLOTS + slot_of(pr, ow, lane)];
                            pac[pr].x += u.x; pac[pr].y += u.y; pdb[pr].x += u.z; pdb[pr].y += u.w;
                        }
                }
                __syncthreads();
                if (g == 0)
#pragma unroll
                    for (int pr = 0; pr < FPAIRS; ++pr)
                        red[slot_of(pr, ow, lane)] = make_float4(pac[pr].x, pac[pr].y, pdb[pr].x, pdb[pr].y);
#pragma unroll
                for (int pr = 0; pr < FPAIRS; ++pr) pac[pr] = pdb[pr] = make_float2(0.f, 0.f);
                __syncthreads();
                for (int sl = threadIdx.x; sl < FSLOTS; sl += FT) {
                    const float4 u = red[sl];                     // (P_A, P_C, P_D, P_B)
                    float4 tv = fsm[sl], tj = fsm[FSLOTS + sl];
                    ff_add2(tv, u.x + u.w, u.y - u.z);
                    ff_add2(tj, u.x - u.w, u.y + u.z);
                    fsm[sl] = tv;
                    fsm[FSLOTS + sl] = tj;
                }
            }
        }
        cp_async_wait<0>();
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * FSLOTS; t += FT) {           // write the tile's fold back
            const int form = t / FSLOTS, sl = t % FSLOTS;
            int kk, e;
            slot_pair(sl, kk, e);
            const int l = lagidx[kk], f = form == 0 ? a.fV : a.fJ;
            if (l < 0 || f < 0 || (A < FJ && e >= A)) continue;   // A < 64: added in by the residue's first offset
            float4 v = fsm[t];
            if (A < FJ)                                   // the residue's other offsets, in order
                for (int e2 = e + A; e2 < FJ; e2 += A) {
                    const int pr = 4 * (kk & 3) + (e2 & 3);
                    const float4 u = fsm[form * FSLOTS + slot_of(pr, e2 >> 5, 8 * (kk >> 2) + ((e2 & 31) >> 2))];
                    ff_add(v.x, v.y, u.x);
                    ff_add(v.x, v.y, u.y);
                    ff_add(v.z, v.w, u.z);
                    ff_add(v.z, v.w, u.w);
                }
            a.fold[(size_t)(l * a.F + f) * A + ((uint32_t)(j0 + e + a.base_mod) & (uint32_t)(A - 1))] = v;
        }
    }
    if (t0 < keep) {
        a.nx[t0] = tx0;
        if (a.ny) a.ny[t0] = ty0;
    }
    for (int t = t0 + FT * ncta; t < keep; t += FT * ncta) {          // tails longer than the grid
        const int v = nview - keep + t, sv = src_from(tab, v, 0);
        a.nx[t] = tab.x[sv][v - tab.start[sv]];
        if (a.ny) a.ny[t] = tab.y[sv][v - tab.start[sv]];
    }
}

// Windowed Full mode.  Block (l, w): window k = k0 + w of lag l, whose reference samples
// are view samples base + n, n < N (base = vbase0 + w hop), for both forms: the products
// P(n) = x[base + n + m] c_f(y[base + n + D]) (m the shifted lag) times (-1)^n go in natural
// order into shared memory, the self-sorting radix-4 FFT (fft_stockham, FP32, both forms
// side by side) gives sum_n P(n) exp(-j 2 pi (-1/2 + kk/N) n) in natural order, and the
// spectrum divided by N goes to ring slot (k mod cap) as [column][kk].  No bit-reversed
// permutation, and a stage's twiddles are consecutive (none that share a bank).
__global__ void __launch_bounds__(256) window_fft_kernel(FoldArgs a, FullWinArgs w)
{
    extern __shared__ __align__(16) float2 fw[];             // V, J twice ([4][N]), twiddles [N]
    __shared__ SrcTab tab;
    if (threadIdx.x == 0) tab.n = a.nsrc;
    if (threadIdx.x <= kFoldSrc) tab.start[threadIdx.x] = a.start[threadIdx.x];
    if (threadIdx.x < kFoldSrc) {
        tab.x[threadIdx.x] = a.sx[threadIdx.x];
        tab.y[threadIdx.x] = a.sy[threadIdx.x];
    }
    const int N = w.N, l = blockIdx.x;
    float2* Vs = fw;
    float2* Js = fw + N;
    float2* Vd = fw + 2 * N;
    float2* Jd = fw + 3 * N;
    float2* tw = fw + 4 * N;
    for (int j = threadIdx.x; j < N; j += blockDim.x) tw[j] = w.tw[j];
    __syncthreads();
    const int m = w.col_lag[l * a.F];                         // shifted lag of lag index l
    const int base = (int)(w.vbase0 + (int64_t)blockIdx.y * w.hop);
    int cx = 0, cy = 0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const int vx = base + n + m, vy = base + n + a.D;
        cx = src_from(tab, vx, cx);
        cy = src_from(tab, vy, cy);
        const float2 xm = tab.x[cx][vx - tab.start[cx]];
        const float2 y = tab.y[cy][vy - tab.start[cy]];
        const float sg = (n & 1) ? -1.f : 1.f;
        const float ar = xm.x * y.x, bi = xm.y * y.y, cr = xm.y * y.x, di = xm.x * y.y;
        Vs[n] = make_float2(sg * (ar + bi), sg * (cr - di));   // x conj(y)
        Js[n] = make_float2(sg * (ar - bi), sg * (cr + di));   // x y
    }
    float2* src[2] = {Vs, Js};
    float2* dst[2] = {Vd, Jd};
    fft_stockham<2>(src, dst, N, tw);
    Vs = src[0];
    Js = src[1];
    const int64_t slot = (w.k0 + blockIdx.y) % w.cap;
    const float inv = 1.f / (float)N;                          // a power of two: exact
    float2* rV = a.fV >= 0 ? w.ring + ((size_t)slot * w.ncols + l * a.F + a.fV) * N : nullptr;
    float2* rJ = a.fJ >= 0 ? w.ring + ((size_t)slot * w.ncols + l * a.F + a.fJ) * N : nullptr;
    for (int kk = threadIdx.x; kk < N; kk += blockDim.x) {
        if (rV) rV[kk] = make_float2(Vs[kk].x * inv, Vs[kk].y * inv);
        if (rJ) rJ[kk] = make_float2(Js[kk].x * inv, Js[kk].y * inv);
    }
}

// out[i][f][kk][l] (FP64) = ring slot ((k0 + i) mod cap) [l F + f][kk]: 32 x 32 tiles of (kk,
// l) transposed through shared memory.  Grid (ceil(N / 32) x ceil(L / 32), F, n).
__global__ void window_read_kernel(const float2* __restrict__ ring, int64_t cap, int64_t k0, int N, int F, int L,
                                   double2* __restrict__ out)
{
    __shared__ float2 t[32][33];
    const int ntl = (L + 31) / 32;
    const int kt = blockIdx.x / ntl, lt = blockIdx.x % ntl, f = blockIdx.y, i = blockIdx.z;
    const int64_t slot = (k0 + i) % cap;
    const int ncols = F * L;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {       // r: lag within the tile
        const int l = lt * 32 + r, kk = kt * 32 + threadIdx.x;
        t[r][threadIdx.x] = l < L && kk < N ? ring[((size_t)slot * ncols + l * F + f) * N + kk] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {       // r: kk within the tile
        const int kk = kt * 32 + r, l = lt * 32 + threadIdx.x;
        if (l < L && kk < N) {
            const float2 v = t[threadIdx.x][r];
            out[(((size_t)i * F + f) * N + kk) * L + l] = make_double2(v.x, v.y);
        }
    }
}

// Block c: out[f][k][l] = (1/N) sum_r (-1)^r F_c[r] exp(-j 2 pi k r / A) for column
// c = l F + f, by an in-place radix-2 FFT in shared memory (FP64).
__global__ void dft_read_kernel(const float4* __restrict__ F, int A, int logA, int ncols, int nF, int L,
                                double inv_n, double2* __restrict__ out)
{
    extern __shared__ double2 v[];
    double2* tw = v + A;                                               // exp(-j 2 pi j / A), j < A/2
    const int c = blockIdx.x;
    for (int j = threadIdx.x; j < A / 2; j += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)j / (double)A, &sn, &cs);
        tw[j] = make_double2(cs, sn);
    }
    for (int r = threadIdx.x; r < A; r += blockDim.x) {
        const float4 ff = F[(size_t)c * A + r];
        const double2 q = make_double2((double)ff.x + (double)ff.y, (double)ff.z + (double)ff.w);
        const double s = (r & 1) ? -1.0 : 1.0;
        const unsigned rev = __brev((unsigned)r) >> (32 - logA);       // bit-reversed position
        v[rev] = make_double2(s * q.x, s * q.y);
    }
    __syncthreads();
    for (int len = 2; len <= A; len <<= 1) {
        const int half = len >> 1;
        for (int t = threadIdx.x; t < A / 2; t += blockDim.x) {
            const int grp = t / half, j = t % half;
            const int i0 = grp * len + j, i1 = i0 + half;
            const double2 z = tw[j * (A / len)];                             // exp(-j 2 pi j / len)
            const double2 b = v[i1];
            const double2 w = make_double2(b.x * z.x - b.y * z.y, b.x * z.y + b.y * z.x);
            const double2 a = v[i0];
            v[i0] = make_double2(a.x + w.x, a.y + w.y);
            v[i1] = make_double2(a.x - w.x, a.y - w.y);
        }
        __syncthreads();
    }
    const int f = c % nF, l = c / nF;
    for (int k = threadIdx.x; k < A; k += blockDim.x)
        out[((size_t)f * A + k) * L + l] = make_double2(v[k].x * inv_n, v[k].y * inv_n);
}

}  // namespace

bool full_supported(int A) { return A >= 2 && A <= 4096 && (A & (A - 1)) == 0; }

bool full_lags_consecutive(const int32_t* sl, int L)
{
    for (int p = 1; p < L; ++p)
        if (p % FLT != 0 && sl[p] != sl[p - 1] + 1) return false;
    return true;
}

int full_row_samples(const int32_t* sl, int L)
{
    int span = 0;
    for (int p0 = 0; p0 < L; p0 += FLT) {
        const int p1 = p0 + FLT - 1 < L - 1 ? p0 + FLT - 1 : L - 1;
        span = sl[p1] - sl[p0] > span ? sl[p1] - sl[p0] : span;
    }
    return (span + FJ + 3) & ~3;          // even: rows stay 16-byte aligned
}

namespace {

template <int MODE>
cudaError_t launch_fold(const FoldArgs& f, dim3 grid, size_t smem, cudaStream_t st)
{
    static bool attr_set[64] = {false};                   // the attribute is per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(fold_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kFoldSmem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    fold_kernel<MODE><<<grid, FT, smem, st>>>(f);
    return cudaGetLastError();
}

}  // namespace

cudaError_t full_fold(const FoldArgs& f, cudaStream_t st)
{
    if (f.nc <= 0 && f.keep <= 0) return cudaSuccess;
    if (f.nsrc < 1 || f.nsrc > kFoldSrc) return cudaErrorInvalidValue;
    const int mode = f.xl > kXlMax ? 2 : f.consecutive ? 0 : 1;
    const int rl = (mode == 2 ? 0 : f.xl) + FJ;
    const size_t smem = (size_t)FQG * FNBUF * FR * rl * sizeof(float2) + kRedBytes;
    if (smem > kFoldSmem) return cudaErrorInvalidValue;
    const dim3 grid(f.A >= FJ ? f.A / FJ : 1, (f.L + FLT - 1) / FLT);
    if (grid.y > 65535) return cudaErrorInvalidValue;      // more than 2^20 lags
    return mode == 0 ? launch_fold<0>(f, grid, smem, st)
         : mode == 1 ? launch_fold<1>(f, grid, smem, st)
                     : launch_fold<2>(f, grid, smem, st);
}

cudaError_t full_windows(const FoldArgs& a, const FullWinArgs& w, int nwin, cudaStream_t st)
{
    if (nwin <= 0) return cudaSuccess;
    if (a.nsrc < 1 || a.nsrc > kFoldSrc || w.N < 2 || w.N > 4096) return cudaErrorInvalidValue;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(window_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(4096 * 5 * sizeof(float2)));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    const size_t smem = (size_t)w.N * 5 * sizeof(float2);
    for (int i0 = 0; i0 < nwin; i0 += 65535) {             // grid.y holds 65535 windows
        FullWinArgs wi = w;
        wi.k0 = w.k0 + i0;
        wi.vbase0 = w.vbase0 + (int64_t)i0 * w.hop;
        window_fft_kernel<<<dim3(a.L, nwin - i0 < 65535 ? nwin - i0 : 65535), 256, smem, st>>>(a, wi);
    }
    return cudaGetLastError();
}

cudaError_t full_read_windows(const float2* ring, int64_t cap, int64_t k0, int64_t n, int N, int F, int L,
                              double2* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    for (int64_t i0 = 0; i0 < n; i0 += 65535) {             // grid.z holds 65535 windows
        const int64_t m = n - i0 < 65535 ? n - i0 : 65535;
        const dim3 grid(((N + 31) / 32) * ((L + 31) / 32), F, (unsigned)m);
        window_read_kernel<<<grid, dim3(32, 8), 0, st>>>(ring, cap, k0 + i0, N, F, L, out + (size_t)i0 * F * N * L);
    }
    return cudaGetLastError();
}

cudaError_t full_read(const double2* F, int A, int ncols, int nF, int L, double inv_n, double2* out, cudaStream_t st)
{
    int logA = 0;
    while ((1 << logA) < A) ++logA;
    const size_t smem = (size_t)A * 3 / 2 * sizeof(double2);
    static bool attr_set[64] = {false};                   // the attribute is per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(dft_read_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             4096 * 3 / 2 * 16);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    dft_read_kernel<<<ncols, 256, smem, st>>>(reinterpret_cast<const float4*>(F), A, logA, ncols, nF, L, inv_n, out);
    return cudaGetLastError();
}

}  // namespace cyc
