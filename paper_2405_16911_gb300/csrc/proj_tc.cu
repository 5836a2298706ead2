// proj_tc.cu -- tensor-core a-projection (tcgen05, sm_103a): FP16 single pass and the
// BF16 three-product split, FP32 accumulation in tensor memory (TMEM).
//
// A work item is 128 cycle frequencies (MMA M) x 256 columns (MMA N) x a range of committed
// n.  The complex GEMM  S[u][c] = sum_n W[u][n] P_c(n)  (Sec. 4 Set mode: the per-alpha
// projection of the lag products; W = exp(-j 2 pi a n), P = x[n+m] x*[n] or x[n+m] x[n],
// Eqs. (ACF-def), (CCF-def)) runs as two real GEMMs over K = (re, im) of 8 samples per
// K = 16 step:
//     D_r += [Wr | -Wi] . [Pr ; Pi]        D_i += [Wi | Wr] . [Pr ; Pi]
// D_r and D_i live in TMEM columns [0, 256) and [256, 512).  The weights carry the absolute
// sample index, so an item accumulates in TMEM without any per-tile rotation.  The tensor
// core's FP32 accumulation drifts with the length of the chain (on the mean-power entry,
// about 2e-3 of its value over 2^19 samples), so an item longer than Cfg::SUBN samples (4096
// for BF16x3, 65536 for FP16) runs as consecutive sub-items, each a fresh TMEM chain: the
// first writes the item's FP32 partial tile, the later ones add to it.
// Operands go through a ring of shared-memory stages (one 8-sample group each), K-major,
// no swizzle, 8-row x 16-byte core matrices:
//   P block: row r (column), chunk k (0: Pr, 1: Pi) at (r/8)*256 + k*128 + (r%8)*16
//   W block: row r (cycle freq), chunk k (0: Wi, 1: Wr, 2: -Wi) at (r/8)*384 + k*128 + (r%8)*16
// so that [Wr | -Wi] starts at chunk 1 and [Wi | Wr] at chunk 0, both with LBO = 128.
// The samples x[n .. n + XB + M) of each block are staged in shared memory by TMA bulk
// copies (a ring of two slots), so that the lag-product warps read shared memory only.
// BF16x3: v = hi + lo, hi = bf16(v), lo = bf16(v - hi); products hi.hi, hi.lo, lo.hi.
//
// Items with at most 128 columns ("narrow", e.g. 64 lags x 2 forms) issue N = 128 MMAs: each
// P thread forms one column (B row = tile column) and the epilogue reads 128 D columns.
//
// Warp roles (576 threads).  Two producer sets; set k produces the groups G = k mod 2 of
// the CTA's running group counter G, so one set's latencies hide behind the other's work:
//   set k, warps 8k+0..3  P warps: thread t forms tile columns 2t, 2t+1 (with lag-major
//                         columns both forms of one lag) -> B rows t and t + 128
//   set k, warps 8k+4..7  W warps: thread t forms the weights of cycle-frequency row t;
//                         set 0's are also the epilogue (TMEM lane quadrant = warp % 4)
//   warp 16  TMEM allocation; lane 0 issues every tcgen05.mma and commit
//   warp 17  lane 0: the TMA sample loader
// Items may start at any sample; the staged block then starts one sample earlier (bulk
// copies need 16-byte alignment) and readers skip it.  The linear view needs x_avail even.
// Barriers: full[s] (8 producer warps -> MMA), empty[s] (tcgen05.commit -> producers),
// xfull/xempty for the sample slots, done (last MMA of an item -> epilogue).  Every wait is
// bounded; a wait that gives up sets the caller's status word and the CTA winds down.
//
// Two launch modes share the code: one item per CTA derived from the grid (cyc_push), and a
// persistent list of items taken with an atomic counter (the multi-stream server).
//
// CTA pairs (grid mode): a cluster of two CTAs on two SMs takes two neighbouring 128-row
// cycle-frequency tiles over the same columns and samples and issues cta_group::2 MMAs with
// M = 256.  Each CTA forms the weights of its own 128 rows (A) and half of the B rows: the
// even CTA B rows [0, N/2), the odd one [N/2, N) -- so each SM forms half the lag products
// and its tensor core reads half of B from its own shared memory.  Producers of both CTAs
// arrive on the even CTA's full[s]; the even CTA's MMA thread signals empty[s] and done in
// both CTAs through a multicast commit.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cyc_device.cuh"
#include "cyc_impl.h"
#include "tc_ptx.cuh"

namespace cyc {
namespace {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int GS = 8;                    // samples per group (one K = 16 step)
constexpr int NSET = 2;                  // producer sets
constexpr int P_WARPS = 4, W_WARPS = 4, SET_WARPS = P_WARPS + W_WARPS;
constexpr int MMA_WARP = NSET * SET_WARPS;
constexpr int LOAD_WARP = MMA_WARP + 1;
constexpr int NTHREADS = (LOAD_WARP + 1) * 32;
constexpr int P_BYTES = 8192, W_BYTES = 6144;
constexpr uint32_t P_LBO = 128, P_SBO = 256, W_LBO = 128, W_SBO = 384;
constexpr int XSLOT = 3072;              // samples per staging slot (block + halo)
constexpr int MAX_LAG = 2560;            // leaves blocks of at least 512 samples
constexpr uint32_t TM_DR = 0, TM_DI = 256;
constexpr long long WAIT_BUDGET = 2000000000ll;   // SM cycles (about one second)

// Waits and arrivals on the stage barriers: cluster scope when the pair shares them.
template <bool PAIR>
__device__ __forceinline__ bool bwait(void* bar, uint32_t parity)
{
    if constexpr (PAIR) return tc::mbar_wait_cluster(bar, parity, WAIT_BUDGET);
    else return tc::mbar_wait(bar, parity, WAIT_BUDGET);
}

template <bool PAIR>
__device__ __forceinline__ void full_arrive(void* bar)
{
    if constexpr (PAIR) tc::mbar_arrive_remote(bar, 0);     // the even CTA's barrier
    else tc::mbar_arrive(bar);
}

template <int PREC>
struct Cfg;
template <>
struct Cfg<CYC_P_FP16> {
    static constexpr int NLEV = 1, NPASS = 1, NSTAGE = 10;
    static constexpr bool BF = false;
    static constexpr int SUBN = 1 << 16;     // samples per TMEM chain (drift ~4e-4 against 1e-2)
};
template <>
struct Cfg<CYC_P_BF16X3> {
    static constexpr int NLEV = 2, NPASS = 3, NSTAGE = 6;
    static constexpr bool BF = true;
    static constexpr int SUBN = 1 << 12;     // samples per TMEM chain (drift ~1.6e-5 against 1e-4)
};

template <int PREC>
__host__ __device__ constexpr int stage_bytes() { return Cfg<PREC>::NLEV * (P_BYTES + W_BYTES); }
template <int PREC>
__host__ __device__ constexpr int xslots_off() { return Cfg<PREC>::NSTAGE * stage_bytes<PREC>(); }
template <int PREC>
__host__ __device__ constexpr int smem_bytes() { return xslots_off<PREC>() + 2 * XSLOT * 8 + 1024; }

// ---- packing: 8 floats -> 16 bytes of FP16 / BF16 (+ BF16 remainders) --------------------
__device__ __forceinline__ uint32_t pack_h2(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ uint32_t pack_b2(float a, float b, uint32_t* lo)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    float2 hf = __bfloat1622float2(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    *lo = *reinterpret_cast<uint32_t*>(&l);
    return *reinterpret_cast<uint32_t*>(&h);
}

template <bool BF>
__device__ __forceinline__ void pack8(const float (&v)[8], uint32_t (&hi)[4], uint32_t (&lo)[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if constexpr (BF) hi[k] = pack_b2(v[2 * k], v[2 * k + 1], &lo[k]);
        else hi[k] = pack_h2(v[2 * k], v[2 * k + 1]);
    }
}

__device__ __forceinline__ void st16(unsigned char* p, const uint32_t (&v)[4])
{
    *reinterpret_cast<uint4*>(p) = make_uint4(v[0], v[1], v[2], v[3]);
}

struct Bars {
    uint64_t full[16];
    uint64_t empty[16];
    uint64_t xfull[2];
    uint64_t xempty[2];
    uint64_t done;
    uint32_t tmem;
    int item;
    int abort;
    int add;                                    // this sub-item adds to the partial tile
    int cmd;                                    // loop control: -1 stop, -2 next sub-item, >= 0 item
    int64_t sub_end;                            // n_end of the whole item
    TcItem it;
};

// Columns c, c + 1 of one partial-tile row (only those below cmax exist), written or added.
__device__ __forceinline__ void put2(float2* out, int c, float4 v, bool vec, int cmax, bool add)
{
    if (vec && c + 1 < cmax) {
        float4* o = reinterpret_cast<float4*>(&out[c]);
        if (add) {
            const float4 q = *o;
            v.x += q.x; v.y += q.y; v.z += q.z; v.w += q.w;
        }
        *o = v;
        return;
    }
    if (c < cmax) {
        float2 w = make_float2(v.x, v.y);
        if (add) { w.x += out[c].x; w.y += out[c].y; }
        out[c] = w;
    }
    if (c + 1 < cmax) {
        float2 w = make_float2(v.z, v.w);
        if (add) { w.x += out[c + 1].x; w.y += out[c + 1].y; }
        out[c + 1] = w;
    }
}

// Epilogue warp (TMEM lane quadrant q): its 32 rows of the item's D tile into the FP32
// partial tile.  Wide items: D columns r, r + 128 <-> tile columns 2r, 2r + 1; narrow items:
// D column r <-> tile column r.  live = false writes zeros.
__device__ __forceinline__ void drain_tile(uint32_t tmem, int q, int lane, const TcItem& it, bool narrow,
                                           bool live, bool add)
{
    const int row = q * 32 + lane;
    const bool vec = (it.out_stride & 1) == 0;
    const int cmax = it.ncols - it.c0;
    float2* out = it.out + (size_t)row * it.out_stride;
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    const bool mine = it.u0 + row < it.Au;
    if (it.x2 != nullptr) {
        // dual item: D columns [0, 128) are the first stream's tile columns, [128, 256) the
        // second stream's, rotated onto its own sample index
        const float2 rot = mine ? phase_rot(it.phi[it.u0 + row], it.dphase) : make_float2(1.f, 0.f);
        float2* out2 = it.out2 + (size_t)row * it.out_stride;
        for (int cb = 0; cb < 16; ++cb) {
            uint32_t dr0[8], di0[8], dr1[8], di1[8];
            tc::tmem_ld8(lane_addr + TM_DR + cb * 8, dr0);
            tc::tmem_ld8(lane_addr + TM_DI + cb * 8, di0);
            tc::tmem_ld8(lane_addr + TM_DR + 128 + cb * 8, dr1);
            tc::tmem_ld8(lane_addr + TM_DI + 128 + cb * 8, di1);
            tc::tmem_ld_wait();
            if (!mine) continue;
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                float4 v = live ? make_float4(__uint_as_float(dr0[j]), __uint_as_float(di0[j]),
                                              __uint_as_float(dr0[j + 1]), __uint_as_float(di0[j + 1]))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
                put2(out, cb * 8 + j, v, vec, cmax, add);
                const float ar = __uint_as_float(dr1[j]), ai = __uint_as_float(di1[j]);
                const float br = __uint_as_float(dr1[j + 1]), bi = __uint_as_float(di1[j + 1]);
                v = live ? make_float4(ar * rot.x - ai * rot.y, ar * rot.y + ai * rot.x,
                                       br * rot.x - bi * rot.y, br * rot.y + bi * rot.x)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
                put2(out2, cb * 8 + j, v, vec, cmax, add);
            }
        }
        return;
    }
    for (int cb = 0; cb < 16; ++cb) {
        uint32_t dr0[8], di0[8], dr1[8], di1[8];
        tc::tmem_ld8(lane_addr + TM_DR + cb * 8, dr0);
        tc::tmem_ld8(lane_addr + TM_DI + cb * 8, di0);
        if (!narrow) {
            tc::tmem_ld8(lane_addr + TM_DR + 128 + cb * 8, dr1);
            tc::tmem_ld8(lane_addr + TM_DI + 128 + cb * 8, di1);
        }
        tc::tmem_ld_wait();
        if (!mine) continue;
        if (narrow) {
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                const float4 v = live ? make_float4(__uint_as_float(dr0[j]), __uint_as_float(di0[j]),
                                                    __uint_as_float(dr0[j + 1]), __uint_as_float(di0[j + 1]))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                put2(out, cb * 8 + j, v, vec, cmax, add);
            }
            continue;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 v = live ? make_float4(__uint_as_float(dr0[j]), __uint_as_float(di0[j]),
                                                __uint_as_float(dr1[j]), __uint_as_float(di1[j]))
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            put2(out, 2 * (cb * 8 + j), v, vec, cmax, add);
        }
    }
}

__device__ __forceinline__ void give_up(int* err, Bars* b, int code)
{
    b->abort = 1;
    if (err) atomicCAS(err, 0, code);
}

// The item of CTA (bx, by, bz) for a single cyc_push pass.
__device__ __forceinline__ TcItem grid_item(const ProjArgs& a, int bx, int by, int bz)
{
    TcItem it;
    it.x = a.x;
    it.xmask = ~0ull;
    it.x_avail = a.x_avail;
    it.nbase = a.nbase;
    const int64_t b = (int64_t)bz * a.split_len - a.split_off;
    it.n_beg = b > 0 ? b : 0;
    it.n_end = b + a.split_len < a.nc ? b + a.split_len : a.nc;
    it.phi = a.phi;
    it.col_lag = a.col_lag;
    it.col_conj = a.col_conj;
    it.u0 = bx * BM;
    it.c0 = by * BN;
    it.Au = a.Au;
    it.ncols = a.ncols;
    it.M = a.M;
    it.out = a.part + ((size_t)bz * a.Au + (size_t)it.u0) * a.ncols + it.c0;
    it.out_stride = a.ncols;
    it.y = a.y;
    it.D = a.D;
    it.out_peer = 0;
    it.x2 = nullptr;
    it.xmask2 = 0;
    it.n_beg2 = 0;
    it.out2 = nullptr;
    it.out_peer2 = 0;
    it.dphase = 0;
    return it;
}

template <int PREC, bool LIST, bool PAIR>
__global__ void __launch_bounds__(NTHREADS, 1)
proj_tc_kernel(ProjArgs pa, const TcItem* __restrict__ items, const int* __restrict__ nitems, int* counter, int* err)
{
    using C = Cfg<PREC>;
    extern __shared__ __align__(1024) unsigned char smem[];
    Bars* bars = reinterpret_cast<Bars*>(smem + xslots_off<PREC>() + 2 * XSLOT * 8);
    float2* xs = reinterpret_cast<float2*>(smem + xslots_off<PREC>());
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (!LIST) err = pa.err;
    const uint32_t crank = PAIR ? tc::cluster_rank() : 0u;

    if (tid == 0) {
        for (int s = 0; s < C::NSTAGE; ++s) {
            tc::mbar_init(&bars->full[s], PAIR ? 2 * SET_WARPS : SET_WARPS);
            tc::mbar_init(&bars->empty[s], 1);
        }
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(&bars->xfull[k], 1);
            tc::mbar_init(&bars->xempty[k], NSET * P_WARPS);
        }
        tc::mbar_init(&bars->done, 1);
        bars->abort = 0;
        bars->add = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) {
        if constexpr (PAIR) tc::tmem_alloc_pair<512>(&bars->tmem);
        else tc::tmem_alloc<512>(&bars->tmem);
    }
    tc::tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) tc::cluster_sync();        // the other CTA's barriers exist before any arrival
    tc::tc_fence_after();
    const uint32_t tmem = bars->tmem;

    const int pset = warp < MMA_WARP ? warp / SET_WARPS : 0;
    const int role = warp % SET_WARPS;              // 0-1 P, 2-5 W
    uint32_t G = 0;                                 // groups this CTA has run (all items)
    uint32_t Bk = 0;                                // sample blocks this CTA has staged
    uint32_t nit = 0;                               // items this CTA has run
    int lastb = -1;                                 // loader: last block issued (running count)

    for (;;) {
        // ---- next (sub-)item (thread 0 fetches; everybody reads it after the barrier) ----
        // cmd: -1 stop, -2 the next sub-item of the current item, >= 0 a new item.  CTA pairs
        // on an item list follow the even CTA's cmd, handed over through distributed shared
        // memory, so that both always run the same items and the same number of iterations.
        if (tid == 0 && (!(PAIR && LIST) || crank == 0)) {
            int cmd = -1;
            if (!bars->abort) {
                if (nit > 0 && bars->it.n_end < bars->sub_end) {
                    cmd = -2;
                } else if (LIST) {
                    cmd = atomicAdd(counter, 1);
                    if (cmd >= *nitems) cmd = -1;
                } else if (nit == 0) {
                    cmd = 0;
                }
            }
            if constexpr (PAIR && LIST) tc::st_remote_s32(&bars->cmd, 1, cmd);
            bars->cmd = cmd;
        }
        if constexpr (PAIR && LIST) tc::cluster_sync();
        if (tid == 0) {
            const int cmd = bars->cmd;
            int idx = -1;
            if (cmd == -2) {
                // the next sub-item of the current item: a fresh TMEM chain that adds
                idx = bars->item;
                bars->it.n_beg2 += bars->it.n_end - bars->it.n_beg;     // dual items advance in step
                bars->it.n_beg = bars->it.n_end;
                bars->add = 1;
            } else if (cmd >= 0) {
                idx = cmd;
                bars->add = 0;
                if constexpr (LIST) {
                    bars->it = items[cmd];
                    if (PAIR && crank == 1) {                  // the odd CTA's 128 rows
                        bars->it.u0 += BM;
                        bars->it.out += bars->it.out_peer;
                        if (bars->it.out2) bars->it.out2 += bars->it.out_peer2;
                    }
                } else {
                    bars->it = grid_item(pa, blockIdx.x, blockIdx.y, blockIdx.z);
                }
                bars->sub_end = bars->it.n_end;
            }
            if (idx >= 0) {
                const int64_t e = bars->it.n_beg + C::SUBN;
                bars->it.n_end = e < bars->sub_end ? e : bars->sub_end;
            }
            bars->item = idx;
        }
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
        if (bars->item < 0) break;
        const TcItem& it = bars->it;
        const int64_t n_beg = it.n_beg, n_end = it.n_end;
        const int64_t span = n_end - n_beg;
        const int ngroups = span > 0 ? (int)((span + GS - 1) / GS) : 0;
        const int mpad = (it.M + 1) & ~1;
        // a slot holds x[block start - xoff .. + XB + M] and, for a second input, y[block
        // start + D - yoff .. + XB] from YOFF on (both copies start at an even sample)
        const bool cross = it.y != nullptr;
        const int XB = cross ? ((XSLOT - mpad - 4) / 2) & ~(GS - 1)
                             : (XSLOT - mpad - 2) & ~(GS - 1);  // samples per staged block
        const int YOFF = XB + mpad + 2;
        const int D = it.D;
        const int yoff = (int)((n_beg + D) & 1);
        const int nblocks = (ngroups * GS + XB - 1) / XB;
        // dual items: each CTA of the pair stages and forms the columns of its own stream
        const bool dual = PAIR && LIST && it.x2 != nullptr;
        const bool second = dual && crank == 1;
        const float2* xsrc = second ? it.x2 : it.x;
        const uint64_t xmsk = second ? it.xmask2 : it.xmask;
        const int64_t nsrc = second ? it.n_beg2 : n_beg;    // this CTA's first sample of the range
        const int xoff = (int)(nsrc & 1);     // bulk copies start at an even sample (16-byte aligned)
        const bool narrow = !dual && it.ncols - it.c0 <= BN / 2;   // N = 128 MMAs, one column per P thread

        if (warp < MMA_WARP && role < P_WARPS) {
            // -------------------------------------------------------- P warps (lag products)
            const int t = (warp - pset * SET_WARPS) * 32 + lane;     // 0..127
            const int c0 = it.c0, ncols = it.ncols;
            // wide items: columns 2t, 2t+1 -> B rows t, t+128; narrow items: column t -> row t.
            // CTA pairs hold B rows [N/2 rank, N/2 (rank + 1)): wide, thread t forms column
            // 2t + rank (its B row t); narrow, threads t < 64 form column 64 rank + t.
            // dual items: thread t forms column t of this CTA's stream (its B row t)
            const int jA = dual ? t
                         : PAIR ? (narrow ? (t < 64 ? 64 * (int)crank + t : ncols) : 2 * t + (int)crank)
                                : (narrow ? t : 2 * t);
            const int jB = 2 * t + 1;
            const bool okA = c0 + jA < ncols, okB = !PAIR && !narrow && c0 + jB < ncols;
            const int mA = okA ? it.col_lag[c0 + jA] : 0, mB = okB ? it.col_lag[c0 + jB] : 0;
            const bool cjA = okA && it.col_conj[c0 + jA], cjB = okB && it.col_conj[c0 + jB];
            const bool same_lag = okB && mA == mB;
            const uint32_t offA = (t / 8) * P_SBO + (t % 8) * 16;             // B row t
            const uint32_t offB = ((t + 128) / 8) * P_SBO + (t % 8) * 16;     // B row t + 128
            bool run = true;
            for (int b = 0; b < nblocks && run; ++b) {
                const uint32_t bg = Bk + b;
                if (!tc::mbar_wait(&bars->xfull[bg & 1], (bg >> 1) & 1, WAIT_BUDGET)) {
                    give_up(err, bars, 4);
                    break;
                }
                const float2* xsl = xs + (bg & 1) * XSLOT;
                const int g_lo = b * (XB / GS), g_hi = min(ngroups, (b + 1) * (XB / GS));
                for (int g = g_lo; g < g_hi; ++g) {
                    const uint32_t Gg = G + g;
                    if ((int)(Gg % NSET) != pset) continue;
                    const int s = Gg % C::NSTAGE;
                    if (Gg >= (uint32_t)C::NSTAGE && !bwait<PAIR>(&bars->empty[s], ((Gg / C::NSTAGE) - 1) & 1)) {
                        give_up(err, bars, 1);
                        run = false;
                        break;
                    }
                    const float2* xb = xsl + xoff + (g * GS - b * XB);
                    const float2* yb = cross ? xsl + YOFF + yoff + (g * GS - b * XB) : xb + D;
                    const int64_t n = n_beg + (int64_t)g * GS;
                    float prA[8], piA[8], prB[8], piB[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float2 pA = make_float2(0.f, 0.f), pB = make_float2(0.f, 0.f);
                        if (n + i < n_end) {
                            float2 x0 = yb[i];                  // reference sample y[n + D]
                            float2 xa = okA ? xb[i + mA] : make_float2(0.f, 0.f);
                            float2 xv = same_lag ? xa : (okB ? xb[i + mB] : make_float2(0.f, 0.f));
                            if (okA) pA = lag_product(xa, x0, cjA);
                            if (okB) pB = lag_product(xv, x0, cjB);
                        }
                        prA[i] = pA.x; piA[i] = pA.y; prB[i] = pB.x; piB[i] = pB.y;
                    }
                    unsigned char* st = smem + s * stage_bytes<PREC>();
                    unsigned char* sl = st + P_BYTES + W_BYTES;             // lo level
                    uint32_t h[4], l[4];
                    pack8<C::BF>(prA, h, l);
                    st16(st + offA, h);
                    if (C::BF) st16(sl + offA, l);
                    pack8<C::BF>(piA, h, l);
                    st16(st + offA + P_LBO, h);
                    if (C::BF) st16(sl + offA + P_LBO, l);
                    if (!PAIR && !narrow) {
                        pack8<C::BF>(prB, h, l);
                        st16(st + offB, h);
                        if (C::BF) st16(sl + offB, l);
                        pack8<C::BF>(piB, h, l);
                        st16(st + offB + P_LBO, h);
                        if (C::BF) st16(sl + offB + P_LBO, l);
                    }
                    tc::fence_async_smem();
                    __syncwarp();
                    if (lane == 0) full_arrive<PAIR>(&bars->full[s]);
                }
                __syncwarp();
                if (run && lane == 0) tc::mbar_arrive(&bars->xempty[bg & 1]);
            }
        } else if (warp < MMA_WARP) {
            // -------------------------------------------------------- W warps (weights)
            const int row = (warp - pset * SET_WARPS - P_WARPS) * 32 + lane;   // 0..127
            const bool ok = it.u0 + row < it.Au;
            const uint64_t phi = ok ? it.phi[it.u0 + row] : 0ull;
            const uint64_t nb = it.nbase + (uint64_t)n_beg;
            const uint32_t offW = (row / 8) * W_SBO + (row % 8) * 16;
            // R_i = exp(-j 2 pi phi i / 2^64): the weights of a group are its anchor W_0 (from
            // the exact u64 phase) times R_i, one sine/cosine pair per group instead of eight
            float rr[8], ri[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float2 r = phase_rot(phi, (uint64_t)i);
                rr[i] = r.x;
                ri[i] = r.y;
            }
            for (int g = 0; g < ngroups; ++g) {
                const uint32_t Gg = G + g;
                if ((int)(Gg % NSET) != pset) continue;
                const int s = Gg % C::NSTAGE;
                if (Gg >= (uint32_t)C::NSTAGE && !bwait<PAIR>(&bars->empty[s], ((Gg / C::NSTAGE) - 1) & 1)) {
                    give_up(err, bars, 1);
                    break;
                }
                float wr[8], wi[8];
                if (ok) {
                    const float2 w0 = phase_rot(phi, nb + (uint64_t)g * GS);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        wr[i] = w0.x * rr[i] - w0.y * ri[i];
                        wi[i] = w0.x * ri[i] + w0.y * rr[i];
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) { wr[i] = 0.f; wi[i] = 0.f; }
                }
                uint32_t rh[4], rl[4], ih[4], il[4], nh[4], nl[4];
                pack8<C::BF>(wr, rh, rl);
                pack8<C::BF>(wi, ih, il);
#pragma unroll
                for (int k = 0; k < 4; ++k) {           // -Wi: round-to-nearest is odd-symmetric
                    nh[k] = ih[k] ^ 0x80008000u;
                    nl[k] = il[k] ^ 0x80008000u;
                }
                unsigned char* st = smem + s * stage_bytes<PREC>() + P_BYTES;
                st16(st + offW + 0 * W_LBO, ih);
                st16(st + offW + 1 * W_LBO, rh);
                st16(st + offW + 2 * W_LBO, nh);
                if (C::BF) {
                    unsigned char* sl = st + P_BYTES + W_BYTES;
                    st16(sl + offW + 0 * W_LBO, il);
                    st16(sl + offW + 1 * W_LBO, rl);
                    st16(sl + offW + 2 * W_LBO, nl);
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) full_arrive<PAIR>(&bars->full[s]);
            }
        } else if (warp == LOAD_WARP && lane == 0) {
            // -------------------------------------------------------- sample loader (TMA)
            for (int b = 0; b < nblocks; ++b) {
                const uint32_t bg = Bk + b;
                const int slot = bg & 1;
                if (bg >= 2 && !tc::mbar_wait(&bars->xempty[slot], ((bg >> 1) - 1) & 1, WAIT_BUDGET)) {
                    give_up(err, bars, 5);
                    break;
                }
                const int64_t ns = nsrc + (int64_t)b * XB - xoff;    // even
                int64_t cnt = ((int64_t)XB + mpad + xoff + 1) & ~(int64_t)1;
                if (cnt > it.x_avail - ns) cnt = it.x_avail - ns;
                int64_t ys = 0, ycnt = 0;
                if (cross) {
                    ys = n_beg + (int64_t)b * XB + D - yoff;          // even
                    ycnt = ((int64_t)XB + yoff + 1) & ~(int64_t)1;
                    if (ycnt > it.x_avail - ys) ycnt = it.x_avail - ys;
                }
                tc::mbar_arrive_expect_tx(&bars->xfull[slot], (uint32_t)((cnt + ycnt) * 8));
                if (cross) tc::bulk_g2s(xs + slot * XSLOT + YOFF, it.y + ys, (uint32_t)(ycnt * 8), &bars->xfull[slot]);
                const uint64_t pos = (uint64_t)ns & xmsk;
                const uint64_t room = xmsk - pos + 1;           // samples before the ring wraps
                if (xmsk == ~0ull || (uint64_t)cnt <= room) {
                    tc::bulk_g2s(xs + slot * XSLOT, xsrc + pos, (uint32_t)(cnt * 8), &bars->xfull[slot]);
                } else {
                    tc::bulk_g2s(xs + slot * XSLOT, xsrc + pos, (uint32_t)(room * 8), &bars->xfull[slot]);
                    tc::bulk_g2s(xs + slot * XSLOT + room, xsrc, (uint32_t)((cnt - room) * 8), &bars->xfull[slot]);
                }
                lastb = (int)bg;
            }
        } else if (warp == MMA_WARP && lane == 0 && crank == 0) {
            // -------------------------------------------------------- MMA issuer
            const uint32_t idesc = tc::idesc_f16(PAIR ? 2 * BM : BM, narrow ? BN / 2 : BN, C::BF);
            const uint32_t pbase = tc::smem_u32(smem);
            for (int g = 0; g < ngroups; ++g) {
                const uint32_t Gg = G + g;
                const int s = Gg % C::NSTAGE;
                if (!bwait<PAIR>(&bars->full[s], (Gg / C::NSTAGE) & 1)) {
                    give_up(err, bars, 2);
                    break;
                }
                tc::tc_fence_after();
                const uint32_t sb = pbase + s * stage_bytes<PREC>();
#pragma unroll
                for (int p = 0; p < C::NPASS; ++p) {
                    const int la = (p == 2) ? 1 : 0, lb = (p == 1) ? 1 : 0;
                    const uint32_t pb = sb + lb * (P_BYTES + W_BYTES);
                    const uint32_t wb = sb + la * (P_BYTES + W_BYTES) + P_BYTES;
                    const uint64_t bdesc = tc::smem_desc(pb, P_LBO, P_SBO);
                    const uint64_t ar = tc::smem_desc(wb + 1 * W_LBO, W_LBO, W_SBO);
                    const uint64_t ai = tc::smem_desc(wb + 0 * W_LBO, W_LBO, W_SBO);
                    const uint32_t acc = (g > 0 || p > 0) ? 1u : 0u;
                    if constexpr (PAIR) {
                        tc::mma_f16_pair(tmem + TM_DR, ar, bdesc, idesc, acc);
                        tc::mma_f16_pair(tmem + TM_DI, ai, bdesc, idesc, acc);
                    } else {
                        tc::mma_f16(tmem + TM_DR, ar, bdesc, idesc, acc);
                        tc::mma_f16(tmem + TM_DI, ai, bdesc, idesc, acc);
                    }
                }
                if constexpr (PAIR) tc::mma_commit_pair(&bars->empty[s], 3);
                else tc::mma_commit(&bars->empty[s]);
            }
            if constexpr (PAIR) tc::mma_commit_pair(&bars->done, 3);
            else tc::mma_commit(&bars->done);
        }

        // ------------------------------------------------------------ epilogue (set 0 W warps)
        if (warp >= P_WARPS && warp < SET_WARPS) {
            const bool got = bwait<PAIR>(&bars->done, nit & 1);
            if (!got) give_up(err, bars, 3);
            tc::tc_fence_after();
            const bool live = got && ngroups > 0 && !bars->abort;
            drain_tile(tmem, warp & 3, lane, it, narrow, live, bars->add != 0);
        }
        G += ngroups;
        Bk += nblocks;
        ++nit;
        // everybody is done with this item's descriptor before thread 0 replaces it
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
    }

    // no sample copy may still be landing when the CTA exits
    if (warp == LOAD_WARP && lane == 0)
        for (int b = lastb > 0 ? lastb - 1 : 0; b <= lastb; ++b)
            if (b >= 0) tc::mbar_wait(&bars->xfull[b & 1], (b >> 1) & 1, WAIT_BUDGET);
    tc::tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) tc::cluster_sync();        // no MMA of the pair still reads this CTA
    if (warp == MMA_WARP) {
        tc::tc_fence_after();
        if constexpr (PAIR) tc::tmem_dealloc_pair<512>(tmem);
        else tc::tmem_dealloc<512>(tmem);
    }
}

int tiles_of(int Au, int ncols) { return ((Au + BM - 1) / BM) * ((ncols + BN - 1) / BN); }

template <int PREC, bool LIST, bool PAIR>
cudaError_t set_smem()
{
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(proj_tc_kernel<PREC, LIST, PAIR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<PREC>());
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

template <int PREC>
cudaError_t launch_grid(const ProjArgs& a, bool pair, cudaStream_t st)
{
    int gx = (a.Au + BM - 1) / BM;
    const dim3 block(NTHREADS);
    if (pair) {
        cudaError_t e = set_smem<PREC, false, true>();
        if (e != cudaSuccess) return e;
        gx = (gx + 1) & ~1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(gx, (a.ncols + BN - 1) / BN, a.nsplit);
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem_bytes<PREC>();
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, proj_tc_kernel<PREC, false, true>, a, (const TcItem*)nullptr,
                                  (const int*)nullptr, (int*)nullptr, (int*)nullptr);
    }
    cudaError_t e = set_smem<PREC, false, false>();
    if (e != cudaSuccess) return e;
    dim3 grid(gx, (a.ncols + BN - 1) / BN, a.nsplit);
    proj_tc_kernel<PREC, false, false><<<grid, block, smem_bytes<PREC>(), st>>>(a, nullptr, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_list(const TcItem* items, const int* nitems, int* counter, int grid, bool pair, int* err,
                        cudaStream_t st)
{
    ProjArgs none;
    none.x = nullptr; none.nc = 0; none.nbase = 0; none.phi = nullptr; none.Au = 0; none.col_lag = nullptr;
    none.col_conj = nullptr; none.ncols = 0; none.nsplit = 0; none.split_len = 0; none.part = nullptr;
    if (pair) {
        cudaError_t e = set_smem<PREC, true, true>();
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((grid + 1) & ~1);
        cfg.blockDim = dim3(NTHREADS);
        cfg.dynamicSmemBytes = smem_bytes<PREC>();
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, proj_tc_kernel<PREC, true, true>, none, items, nitems, counter, err);
    }
    cudaError_t e = set_smem<PREC, true, false>();
    if (e != cudaSuccess) return e;
    proj_tc_kernel<PREC, true, false><<<grid, NTHREADS, smem_bytes<PREC>(), st>>>(none, items, nitems, counter, err);
    return cudaGetLastError();
}

// CTA pairs that can be resident at once (0: cluster launches unavailable).
template <int PREC>
int pair_slots()
{
    if (set_smem<PREC, false, true>() != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = smem_bytes<PREC>();
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, proj_tc_kernel<PREC, false, true>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace

bool tc_supported(int ncols, int M) { return ncols > 0 && M >= 0 && M <= MAX_LAG; }

int tc_tile_rows() { return BM; }
int tc_tile_cols() { return BN; }

int tc_pair_ctas(int precision)
{
    const int n = precision == CYC_P_FP16 ? pair_slots<CYC_P_FP16>()
                : precision == CYC_P_BF16X3 ? pair_slots<CYC_P_BF16X3>() : 0;
    return 2 * n;
}

ProjPlan tc_plan(int Au, int ncols, int64_t nc, int num_sms, int pair_ctas)
{
    int tiles = tiles_of(Au, ncols);
    int slots = num_sms;
    if (pair_ctas > 0) {            // x tiles rounded up to whole pairs
        const int tx = (Au + BM - 1) / BM;
        tiles = ((tx + 1) & ~1) * ((ncols + BN - 1) / BN);
        slots = pair_ctas < num_sms ? pair_ctas : num_sms;
    }
    // splits of at least 2048 samples, within what the partial buffer holds
    int smax = max_splits(tiles_of(Au, ncols), num_sms, Au, ncols);
    if ((int64_t)smax > nc / 2048) smax = (int)(nc / 2048);
    const int want = wave_splits(tiles, slots, smax);
    int64_t len = (nc + want - 1) / want;
    if (len < 256) len = 256;
    len = (len + GS - 1) / GS * GS;
    ProjPlan p;
    p.split_len = len;
    p.nsplit = (int)((nc + len - 1) / len);
    if (p.nsplit < 1) p.nsplit = 1;
    return p;
}

size_t tc_max_partials(int Au, int ncols, int num_sms)
{
    return (size_t)max_splits(tiles_of(Au, ncols), num_sms, Au, ncols) * (size_t)Au * (size_t)ncols;
}

cudaError_t tc_launch(const ProjArgs& a, int precision, bool pair, cudaStream_t st)
{
    if (precision == CYC_P_FP16) return launch_grid<CYC_P_FP16>(a, pair, st);
    if (precision == CYC_P_BF16X3) return launch_grid<CYC_P_BF16X3>(a, pair, st);
    return cudaErrorInvalidValue;
}

cudaError_t tc_launch_items(const TcItem* items, const int* nitems, int* counter, int grid, int precision,
                            bool pair, int* err, cudaStream_t st)
{
    if (precision == CYC_P_FP16) return launch_list<CYC_P_FP16>(items, nitems, counter, grid, pair, err, st);
    if (precision == CYC_P_BF16X3) return launch_list<CYC_P_BF16X3>(items, nitems, counter, grid, pair, err, st);
    return cudaErrorInvalidValue;
}

}  // namespace cyc
