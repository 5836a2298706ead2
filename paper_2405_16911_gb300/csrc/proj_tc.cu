// proj_tc.cu -- tensor-core a-projection (tcgen05, sm_103a): FP16 single pass and the
// BF16 three-product split, FP32 accumulation in tensor memory (TMEM).
//
// The projection (Sec. 4 Set mode: the per-alpha correlation of the lag products;
// Eqs. (ACF-def), (CCF-def)) is  S_a[c] = sum_n W_a(n) P_c(n)  with W_a(n) = exp(-j 2 pi a n)
// and P_c the lag product of column c.  Writing W = Wr + j Wi and P = Pr + j Pi, the four
// real sums  Trr = sum Wr Pr,  Tii = sum Wi Pi,  Tri = sum Wr Pi,  Tir = sum Wi Pr  give both
//     S_a  = (Trr - Tii) + j (Tri + Tir)          (weights W_a)
//     S_-a = (Trr + Tii) + j (Tri - Tir)          (weights conj(W_a) = W_-a)
// so a cycle frequency and its negative cost one real GEMM of two weight rows (Wr, Wi) by
// two lag-product rows (Pr, Pi): 2 real multiply-adds per complex term instead of the 4 of
// a complex GEMM.  The distinct cycle frequencies are ordered into *units* of two weight
// rows (see order_units in cyc_impl.h):
//   pair    (a, -a)            rows Wr(a), Wi(a)      -> S_a and S_-a
//   real    (0 and/or 1/2)     rows W(0), W(1/2)      -> each row's own (Tr, Ti); W is real
//   single  a without partner  rows Wr(a), Wi(a)      -> S_a only
// A uniform grid -1/2 + k/A (A even) is A/2 - 1 pairs and one real unit: no row is idle.
//
// Work item: 256 units (512 weight rows) x 128 complex columns x a range of committed n, on a
// pair of CTAs (a cluster of two issuing cta_group::2 MMAs with M = 256, N = 256, K = 16
// samples).  The units form two sub-tiles of 128; CTA r holds the weight rows of units
// u0 + 128 q + 64 r .. + 63 of sub-tile q (A operands A_0, A_1: 128 rows each, its TMEM lanes)
// and forms the lag products of tile columns 64 r .. 64 r + 63 (B operand: B rows 128 r ..
// 128 r + 127 of the pair's 256).  Every stage issues D_q += A_q B for both sub-tiles, so one
// stage of lag products serves 512 weight rows, and each CTA's TMEM holds two accumulators
// (D_0, D_1) of its 128 rows times all 256 real columns.
//
// Shared-memory operands per stage (16 samples), K-major, no swizzle, 8-row x 16-byte core
// matrices, row r and sample chunk k (0: samples 0-7, 1: 8-15) at (r/8)*256 + k*128 + (r%8)*16:
//   A_q: rows 2i / 2i + 1 = the two weight rows of unit i of the sub-tile
//   B: for slot s < 32 (tile column 64 r + 2 s): Pr at row s, Pi at row 32 + s;
//      for slot s >= 32 (tile column 64 r + 2 (s - 32) + 1): Pr at 64 + s - 32, Pi at 96 + s - 32
// so every store of a warp covers 32 consecutive B rows (no bank conflicts).  A stage holds
// per level [A_0 | A_1 | B]; BF16x3 (v = hi + lo, hi = bf16(v), lo = bf16(v - hi)) issues
// hi.hi, hi.lo and lo.hi, the hi level first.
//
// The tensor core's FP32 accumulation drifts with the length of the chain, so an item runs as
// chains of at most Cfg::SUBN samples, each a fresh accumulator; the first chain writes the
// item's FP32 partial tile and later ones add to it.
//
// Warp roles (704 threads):
//   set k = 0, 1 (stages G with G mod 2 = k, so one set's latency hides behind the other's):
//     warps 8k + 0..3   P warps: warp 8k + p, lane t forms slot 32 (p & 1) + t for the samples
//                       8 (p >> 1) .. + 7 of the stage
//     warps 8k + 4..7   W warps: thread i forms both weight rows of unit i % 64 of sub-tile
//                       i / 64 (one rotation gives the real and the imaginary part)
//   warps 16..19        epilogue (TMEM lane quadrant = warp % 4)
//   warp 20             TMEM allocation; lane 0 of the even CTA issues every MMA and commit
//   warp 21             lane 0: TMA loader of the sample blocks (ring of two slots)
// A set's eight warps meet at a named barrier after writing a stage, and one thread per CTA
// then arrives on the even CTA's full barrier: two arrivals per stage (one arrival per warp,
// 12 or more per stage, serialised on the barrier and cost more than a stage of MMAs).
// Barriers: full[s] (one arrival per CTA of the pair -> the even CTA's MMA thread),
// empty[s] (MMA commit -> producers of both CTAs), xfull / xempty (sample slots), done
// (last MMA of a chain -> epilogues of both CTAs), tfree (epilogues of both CTAs -> MMA).
//
// Every wait is bounded by a cycle budget given at launch.  A wait that gives up sets the
// caller's status word and an abort flag in shared memory of both CTAs; every other wait
// polls the flag and fails at once, so one lost arrival ends the whole pair within one
// budget.  Before the CTAs exit, issued sample copies and MMAs are waited for (bounded,
// ignoring the flag), and the pair deallocates its TMEM after a cluster barrier.
//
// Two launch modes share the code: one item per CTA pair derived from the grid (cyc_push),
// and a persistent list of items taken with an atomic counter (the multi-stream server),
// where the even CTA fetches and hands the item index to the odd one through distributed
// shared memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cyc_device.cuh"
#include "cyc_impl.h"
#include "tc_ptx.cuh"

namespace cyc {
namespace {

constexpr int ROWS = 128;                // weight rows per CTA and sub-tile (64 units)
constexpr int CTA_UNITS = 64;
constexpr int SUB_UNITS = 128;           // units of a sub-tile (both CTAs)
constexpr int NSUB = 2;                  // sub-tiles per item
constexpr int ITEM_UNITS = NSUB * SUB_UNITS;
constexpr int TILE_CC = 128;             // complex columns per item
constexpr int GS = 16;                   // samples per stage (one K = 16 step)
constexpr int NSET = 2;
constexpr int P_WARPS = 4, W_WARPS = 4, SET_WARPS = P_WARPS + W_WARPS;
constexpr int EPI_WARP = NSET * SET_WARPS;
constexpr int MMA_WARP = EPI_WARP + 4;
constexpr int LOAD_WARP = MMA_WARP + 1;
constexpr int NTHREADS = (LOAD_WARP + 1) * 32;
constexpr int OPB = 4096;                // one operand block of one level: 128 rows x 16 samples x 2 B
constexpr int LEVEL_BYTES = (NSUB + 1) * OPB;   // [A_0 | A_1 | B]
constexpr uint32_t LBO = 128, SBO = 256;
constexpr int XSLOT = 3072;              // samples per staging slot (block + halo)
constexpr int MAX_LAG = 2560;            // leaves blocks of at least 240 samples
constexpr int TM_COLS = 256;             // one accumulator
constexpr int FULL_ARRIVALS = 2;         // one per CTA and stage (after the set's named barrier)
constexpr int TFREE_ARRIVALS = 2 * 4;    // epilogue warps of both CTAs

template <int PREC>
struct Cfg;
template <>
struct Cfg<CYC_P_FP16> {
    static constexpr int NLEV = 1, NPASS = 1, NSTAGE = 12;
    static constexpr bool BF = false;
    static constexpr int SUBN = 1 << 16;     // samples per TMEM chain (drift ~4e-4 against 1e-2)
};
template <>
struct Cfg<CYC_P_BF16X3> {
    static constexpr int NLEV = 2, NPASS = 3, NSTAGE = 6;
    static constexpr bool BF = true;
    static constexpr int SUBN = 1 << 13;     // samples per TMEM chain (drift ~1e-5 against 1e-4)
};

template <int PREC>
__host__ __device__ constexpr int stage_bytes() { return Cfg<PREC>::NLEV * LEVEL_BYTES; }
template <int PREC>
__host__ __device__ constexpr int xslots_off() { return Cfg<PREC>::NSTAGE * stage_bytes<PREC>(); }
template <int PREC>
__host__ __device__ constexpr int smem_bytes() { return xslots_off<PREC>() + 2 * XSLOT * 8 + 1024; }
static_assert(smem_bytes<CYC_P_BF16X3>() <= 227 * 1024 && smem_bytes<CYC_P_FP16>() <= 227 * 1024, "shared memory");

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
__device__ __forceinline__ void pack8(const float* v, uint32_t (&hi)[4], uint32_t (&lo)[4])
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

__device__ __forceinline__ uint32_t op_off(int row, int chunk)
{
    return (uint32_t)((row >> 3) * SBO + chunk * LBO + (row & 7) * 16);
}

// Named barrier `id` (1 + producer set) over the set's warps: every warp of a set passes it
// once per stage of the set, whatever happened, so it can never wait for a warp that left.
__device__ __forceinline__ void set_sync(int id)
{
    asm volatile("bar.sync %0, %1;" :: "r"(id), "n"(SET_WARPS * 32) : "memory");
}

struct Bars {
    uint64_t full[12];
    uint64_t empty[12];
    uint64_t xfull[2];
    uint64_t xempty[2];
    uint64_t done;
    uint64_t tfree;
    uint64_t fin;
    uint32_t tmem;
    int item;
    int cmd;                                    // loop control: -1 stop, >= 0 item
    volatile int abort;
    TcItem it;
};
static_assert(sizeof(Bars) <= 1024, "barrier block");

// Eight partial-tile columns c0 .. c0 + 7 of one row (only those below cmax exist), written
// or added; the old values are all loaded before any store.
__device__ __forceinline__ void put8(float2* out, int c0, const float (&v)[16], bool vec, int cmax, bool add)
{
    if (vec && c0 + 7 < cmax) {
        float4* o = reinterpret_cast<float4*>(out + c0);
        float4 q[4];
        if (add) {
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = o[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 w = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
            if (add) { w.x += q[k].x; w.y += q[k].y; w.z += q[k].z; w.w += q[k].w; }
            o[k] = w;
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (c0 + k < cmax) {
            float2 w = make_float2(v[2 * k], v[2 * k + 1]);
            if (add) { w.x += out[c0 + k].x; w.y += out[c0 + k].y; }
            out[c0 + k] = w;
        }
    }
}

// Epilogue warp (TMEM lane quadrant q) of CTA `rank`: its 32 weight rows of sub-tile `sub`
// (accumulator `tbuf`) into the item's partial tile.  Lanes 2i and 2i + 1 hold the two rows
// of one unit and swap their values by a shuffle.  live = false writes zeros.
__device__ __forceinline__ void drain_tile(uint32_t tbuf, int q, int lane, const TcItem& it, int rank, int sub,
                                           bool live, bool add)
{
    const int rho = q * 32 + lane;
    const int unit = it.u0 + sub * SUB_UNITS + rank * CTA_UNITS + (rho >> 1), h = rho & 1;
    const int d = unit_row(unit, h, it.np, it.nself, it.U);
    const int kind = unit >= it.U ? -1 : unit < it.np ? 0 : unit < it.np + (it.nself > 0 ? 1 : 0) ? 1 : 2;
    const bool vec = (it.out_stride & 1) == 0;
    const int cmax = it.ncols - it.c0;
    float2* out = d >= 0 ? it.out + (size_t)(d - it.d_lo) * it.out_stride : nullptr;
    const uint32_t lane_addr = tbuf + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
#pragma unroll 1
        for (int s0 = 0; s0 < 32; s0 += 4) {
            uint32_t pr0[4], pi0[4], pr1[4], pi1[4];
            if (live) {
                const uint32_t col = lane_addr + (uint32_t)(128 * r + s0);
                tc::tmem_ld4(col, pr0);
                tc::tmem_ld4(col + 32, pi0);
                tc::tmem_ld4(col + 64, pr1);
                tc::tmem_ld4(col + 96, pi1);
                tc::tmem_ld_wait();
            }
            float o[16];                        // tile columns 64 r + 2 s0 + 2 i + qq
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int qq = 0; qq < 2; ++qq) {
                    const float own_r = live ? __uint_as_float(qq ? pr1[i] : pr0[i]) : 0.f;
                    const float own_i = live ? __uint_as_float(qq ? pi1[i] : pi0[i]) : 0.f;
                    const float oth_r = __shfl_xor_sync(0xffffffffu, own_r, 1);
                    const float oth_i = __shfl_xor_sync(0xffffffffu, own_i, 1);
                    const float trr = h ? oth_r : own_r, tri = h ? oth_i : own_i;
                    const float tir = h ? own_r : oth_r, tii = h ? own_i : oth_i;
                    float vr = own_r, vi = own_i;          // real unit: the row's own sums
                    if (kind == 0 || kind == 2) {
                        vr = h ? trr + tii : trr - tii;
                        vi = h ? tri - tir : tri + tir;
                    }
                    o[4 * i + 2 * qq] = vr;
                    o[4 * i + 2 * qq + 1] = vi;
                }
            }
            if (out) put8(out, 64 * r + 2 * s0, o, vec, cmax, add);
        }
    }
}

struct Ctl {
    int*      err;
    long long budget;        // SM cycles per wait
    int       withhold;      // test only: one producer arrival of CTA (0, 0, 0) is left out
};

__device__ __forceinline__ void give_up(const Ctl& ctl, Bars* b, int code, uint32_t crank)
{
    b->abort = 1;
    tc::st_remote_s32((void*)&b->abort, crank ^ 1u, 1);      // the partner CTA of the pair
    if (ctl.err) atomicCAS(ctl.err, 0, code);
}

// The item of CTA pair (px, by, bz) for a single cyc_push pass.
__device__ __forceinline__ TcItem grid_item(const ProjArgs& a, int px, int by, int bz)
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
    it.np = a.np;
    it.nself = a.nself;
    it.U = a.U;
    it.u0 = px * ITEM_UNITS;
    it.d_lo = unit_row(it.u0, 0, a.np, a.nself, a.U);
    if (it.d_lo < 0) it.d_lo = 0;
    it.c0 = by * TILE_CC;
    it.ncols = a.ncols;
    it.M = a.M;
    it.out = a.part + ((size_t)bz * a.Au + (size_t)it.d_lo) * a.ncols + it.c0;
    it.out_stride = a.ncols;
    it.y = a.y;
    it.D = a.D;
    return it;
}

// Weights of one unit for the W warps: its two rows (real and imaginary part of
// exp(-j 2 pi phi n / 2^64) for pairs and singles; W(0) = 1 and W(1/2) = (-1)^n, exactly, for
// the real unit).
struct UnitW {
    uint64_t phi;
    bool     live[2];
    bool     real;            // the real unit: row h holds W of realphi[h]
    uint64_t realphi[2];
};

__device__ __forceinline__ UnitW unit_weights(const TcItem& it, int unit)
{
    UnitW u;
    u.phi = 0;
    u.real = false;
    u.live[0] = u.live[1] = unit < it.U;
    u.realphi[0] = u.realphi[1] = 0;
    const int nr = it.nself > 0 ? 1 : 0;
    if (unit >= it.U) return u;
    if (unit < it.np) {
        u.phi = it.phi[2 * unit];
    } else if (unit < it.np + nr) {
        u.real = true;
        u.live[1] = it.nself > 1;
        u.realphi[0] = it.phi[2 * it.np];
        u.realphi[1] = it.nself > 1 ? it.phi[2 * it.np + 1] : 0;
    } else {
        u.phi = it.phi[2 * it.np + it.nself + (unit - it.np - nr)];
    }
    return u;
}

template <int PREC, bool LIST>
__global__ void __launch_bounds__(NTHREADS, 1)
proj_tc_kernel(ProjArgs pa, const TcItem* __restrict__ items, const int* __restrict__ nitems, int* counter, Ctl ctl)
{
    using C = Cfg<PREC>;
    constexpr int CG = C::SUBN / GS;                 // stages per chain
    extern __shared__ __align__(1024) unsigned char smem[];
    Bars* bars = reinterpret_cast<Bars*>(smem + xslots_off<PREC>() + 2 * XSLOT * 8);
    float2* xs = reinterpret_cast<float2*>(smem + xslots_off<PREC>());
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t crank = tc::cluster_rank();
    const long long budget = ctl.budget;
    const volatile int* ab = &bars->abort;

    if (tid == 0) {
        for (int s = 0; s < C::NSTAGE; ++s) {
            tc::mbar_init(&bars->full[s], FULL_ARRIVALS);
            tc::mbar_init(&bars->empty[s], 1);
        }
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(&bars->xfull[k], 1);
            tc::mbar_init(&bars->xempty[k], NSET * P_WARPS);
        }
        tc::mbar_init(&bars->done, 1);
        tc::mbar_init(&bars->tfree, TFREE_ARRIVALS);
        tc::mbar_init(&bars->fin, 1);
        bars->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) tc::tmem_alloc_pair<NSUB * TM_COLS>(&bars->tmem);
    tc::tc_fence_before();
    __syncthreads();
    tc::cluster_sync();                              // the other CTA's barriers exist before any arrival
    tc::tc_fence_after();
    const uint32_t tmem = bars->tmem;

    const int pset = warp < EPI_WARP ? warp / SET_WARPS : 0;
    const int role = warp % SET_WARPS;               // 0-3 P, 4-7 W
    uint32_t G = 0;                                  // stages this CTA has run (all items)
    uint32_t Bk = 0;                                 // sample blocks this CTA has staged
    uint32_t J = 0;                                  // accumulator chains this CTA has run
    uint32_t nit = 0;                                // items this CTA has run
    int lastb = -1;                                  // loader: last block issued (running count)
    bool mma_issued = false;

    for (;;) {
        // ---- next item (cmd -1: stop).  Pairs on an item list follow the even CTA's cmd,
        // handed over through distributed shared memory, so that both always run the same
        // items; in grid mode both CTAs of a pair derive the same item from the grid.
        if (tid == 0 && (!LIST || crank == 0)) {
            int cmd = -1;
            if (LIST) {
                if (!bars->abort) {
                    cmd = atomicAdd(counter, 1);
                    if (cmd >= *nitems) cmd = -1;
                }
                tc::st_remote_s32(&bars->cmd, 1, cmd);
            } else if (nit == 0) {
                cmd = 0;
            }
            bars->cmd = cmd;
        }
        if constexpr (LIST) tc::cluster_sync();
        if (tid == 0) {
            const int cmd = bars->cmd;
            if (cmd >= 0) {
                if constexpr (LIST) bars->it = items[cmd];
                else bars->it = grid_item(pa, blockIdx.x >> 1, blockIdx.y, blockIdx.z);
            }
            bars->item = cmd;
        }
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
        if (bars->item < 0) break;
        const TcItem& it = bars->it;
        const int64_t n_beg = it.n_beg, n_end = it.n_end;
        const int64_t span = n_end - n_beg;
        const int ngroups = span > 0 ? (int)((span + GS - 1) / GS) : 0;
        const int nchains = (ngroups + CG - 1) / CG;
        const int mpad = (it.M + 1) & ~1;
        // a slot holds x[block start - xoff .. + XB + M] and, for a second input, y[block
        // start + D - yoff .. + XB] from YOFF on (both copies start at an even sample)
        const bool cross = it.y != nullptr;
        const int XB = cross ? ((XSLOT - mpad - 4) / 2) & ~(GS - 1)
                             : (XSLOT - mpad - 2) & ~(GS - 1);  // samples per staged block
        const int YOFF = XB + mpad + 2;
        const int D = it.D;
        const int yoff = (int)((n_beg + D) & 1);
        const int xoff = (int)(n_beg & 1);    // bulk copies start at an even sample (16-byte aligned)
        const int nblocks = (ngroups * GS + XB - 1) / XB;

        if (warp < EPI_WARP && role < P_WARPS) {
            // -------------------------------------------------------- P warps (lag products)
            // slot 32 sg + t: tile column 64 r + 2 t + sg, B rows (Pr, Pi) = (64 sg + t, 64 sg + 32 + t)
            const int sg = role & 1, hk = role >> 1;                 // samples 8 hk .. 8 hk + 7
            const int t = lane;
            const int cA = it.c0 + 64 * (int)crank + 2 * t + sg;
            const bool okA = cA < it.ncols;
            const int mA = okA ? it.col_lag[cA] : 0;
            const bool cjA = okA && it.col_conj[cA];
            const uint32_t oR = NSUB * OPB + op_off(64 * sg + t, hk);
            const uint32_t oI = NSUB * OPB + op_off(64 * sg + 32 + t, hk);
            bool bad = false;
            for (int b = 0; b < nblocks; ++b) {
                const uint32_t bg = Bk + b;
                if (!bad && !tc::mbar_wait_ab<false>(&bars->xfull[bg & 1], (bg >> 1) & 1, budget, ab)) {
                    give_up(ctl, bars, 4, crank);
                    bad = true;
                }
                const float2* xsl = xs + (bg & 1) * XSLOT;
                const int g_lo = b * (XB / GS), g_hi = min(ngroups, (b + 1) * (XB / GS));
                for (int g = g_lo; g < g_hi; ++g) {
                    const uint32_t Gg = G + g;
                    if ((int)(Gg % NSET) != pset) continue;
                    const int s = Gg % C::NSTAGE;
                    if (!bad && Gg >= (uint32_t)C::NSTAGE &&
                        !tc::mbar_wait_ab<true>(&bars->empty[s], ((Gg / C::NSTAGE) - 1) & 1, budget, ab)) {
                        give_up(ctl, bars, 1, crank);
                        bad = true;
                    }
                    if (!bad) {
                        const int o = g * GS - b * XB + 8 * hk;
                        const float2* xb = xsl + xoff + o;
                        const float2* yb = cross ? xsl + YOFF + yoff + o : xb + D;
                        const int64_t left = n_end - (n_beg + (int64_t)g * GS + 8 * hk);
                        const int lim = okA ? (left < 8 ? (int)left : 8) : 0;   // samples of this chunk in range
                        float pr[8], pi[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float2 xv = xb[i + mA], y0 = yb[i];          // x[n + m], y[n + D]
                            const float yi = cjA ? y0.y : -y0.y;
                            const bool in = i < lim;
                            pr[i] = in ? xv.x * y0.x - xv.y * yi : 0.f;
                            pi[i] = in ? xv.x * yi + xv.y * y0.x : 0.f;
                        }
                        unsigned char* st = smem + s * stage_bytes<PREC>();     // hi level
                        uint32_t hv[4], lv[4];
                        pack8<C::BF>(pr, hv, lv);
                        st16(st + oR, hv);
                        if (C::BF) st16(st + LEVEL_BYTES + oR, lv);
                        pack8<C::BF>(pi, hv, lv);
                        st16(st + oI, hv);
                        if (C::BF) st16(st + LEVEL_BYTES + oI, lv);
                        tc::fence_async_smem();
                    }
                    set_sync(1 + pset);
                }
                __syncwarp();
                if (!bad && lane == 0) tc::mbar_arrive(&bars->xempty[bg & 1]);
            }
        } else if (warp < EPI_WARP) {
            // -------------------------------------------------------- W warps (weights)
            const int wt = (role - P_WARPS) * 32 + lane;                 // 0..127
            const int sub = wt >> 6, ui = wt & 63;
            const UnitW uw = unit_weights(it, it.u0 + sub * SUB_UNITS + (int)crank * CTA_UNITS + ui);
            const uint64_t nb = it.nbase + (uint64_t)n_beg;
            // row 2 ui: Wr, row 2 ui + 1: Wi
            const uint32_t ob = (uint32_t)sub * OPB;
            const uint32_t oR0 = ob + op_off(2 * ui, 0), oR1 = ob + op_off(2 * ui, 1);
            const uint32_t oI0 = ob + op_off(2 * ui + 1, 0), oI1 = ob + op_off(2 * ui + 1, 1);
            // W(n0 + i) = W0 R_i with R_i = exp(-j 2 pi phi i / 2^64) and W0 the stage's anchor
            // (exact u64 phase): one sine/cosine pair per stage and unit.  The real unit's rows
            // are W(0) = 1 and W(1/2) = (-1)^n, formed exactly.
            float rr[GS], ri[GS];
#pragma unroll
            for (int i = 0; i < GS; ++i) {
                const float2 r = phase_rot(uw.phi, (uint64_t)i);
                rr[i] = r.x;
                ri[i] = r.y;
            }
            const bool arriver = role == P_WARPS && lane == 0;
            bool bad = false;
            for (int g = 0; g < ngroups; ++g) {
                const uint32_t Gg = G + g;
                if ((int)(Gg % NSET) != pset) continue;
                const int s = Gg % C::NSTAGE;
                if (!bad && Gg >= (uint32_t)C::NSTAGE &&
                    !tc::mbar_wait_ab<true>(&bars->empty[s], ((Gg / C::NSTAGE) - 1) & 1, budget, ab)) {
                    give_up(ctl, bars, 1, crank);
                    bad = true;
                }
                if (!bad) {
                    const uint64_t n = nb + (uint64_t)g * GS;
                    unsigned char* st = smem + s * stage_bytes<PREC>();     // hi level
                    uint32_t hv[4], lv[4];
                    if (!uw.real) {
                        const float2 w0 = uw.live[0] ? phase_rot(uw.phi, n) : make_float2(0.f, 0.f);
#pragma unroll
                        for (int half = 0; half < 2; ++half) {
                            float re[8], im[8];
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                re[k] = w0.x * rr[8 * half + k] - w0.y * ri[8 * half + k];
                                im[k] = w0.x * ri[8 * half + k] + w0.y * rr[8 * half + k];
                            }
                            const uint32_t orr = half ? oR1 : oR0, oii = half ? oI1 : oI0;
                            pack8<C::BF>(re, hv, lv);
                            st16(st + orr, hv);
                            if (C::BF) st16(st + LEVEL_BYTES + orr, lv);
                            pack8<C::BF>(im, hv, lv);
                            st16(st + oii, hv);
                            if (C::BF) st16(st + LEVEL_BYTES + oii, lv);
                        }
                    } else {
                        // W(0) = 1, W(1/2) = (-1)^n: exact in every format, the lo level is zero
                        const bool odd = (n & 1) != 0;        // GS is even: sample i has parity odd ^ (i & 1)
                        const uint32_t one = C::BF ? 0x3F80u : 0x3C00u, sgn = 0x8000u;
                        uint32_t r0[4], r1[4], zero[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t a = one | (odd ? sgn : 0u), b = one | (odd ? 0u : sgn);
                            const uint32_t alt = a | (b << 16);           // samples 2k, 2k + 1
                            const uint32_t flat = one | (one << 16);
                            r0[k] = uw.realphi[0] ? alt : flat;
                            r1[k] = uw.live[1] ? (uw.realphi[1] ? alt : flat) : 0u;
                        }
                        st16(st + oR0, r0);
                        st16(st + oR1, r0);
                        st16(st + oI0, r1);
                        st16(st + oI1, r1);
                        if (C::BF) {
                            st16(st + LEVEL_BYTES + oR0, zero);
                            st16(st + LEVEL_BYTES + oR1, zero);
                            st16(st + LEVEL_BYTES + oI0, zero);
                            st16(st + LEVEL_BYTES + oI1, zero);
                        }
                    }
                    tc::fence_async_smem();
                }
                set_sync(1 + pset);
                const bool hold = ctl.withhold && !LIST && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 &&
                                  Gg == 0;
                if (arriver && !hold && !*ab) tc::mbar_arrive_remote(&bars->full[s], 0);
            }
        } else if (warp < MMA_WARP) {
            // -------------------------------------------------------- epilogue
            const int q = warp & 3;
            if (nchains == 0)
                for (int sub = 0; sub < NSUB; ++sub) drain_tile(0, q, lane, it, (int)crank, sub, false, false);
            for (int j = 0; j < nchains; ++j) {
                const uint32_t Jg = J + j;
                if (!tc::mbar_wait_ab<true>(&bars->done, Jg & 1, budget, ab)) {
                    give_up(ctl, bars, 3, crank);
                    break;
                }
                tc::tc_fence_after();
                for (int sub = 0; sub < NSUB; ++sub)
                    drain_tile(tmem + sub * TM_COLS, q, lane, it, (int)crank, sub, true, j > 0);
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive_remote(&bars->tfree, 0);
            }
        } else if (warp == LOAD_WARP && lane == 0) {
            // -------------------------------------------------------- sample loader (TMA)
            for (int b = 0; b < nblocks; ++b) {
                const uint32_t bg = Bk + b;
                const int slot = bg & 1;
                if (bg >= 2 && !tc::mbar_wait_ab<false>(&bars->xempty[slot], ((bg >> 1) - 1) & 1, budget, ab)) {
                    give_up(ctl, bars, 5, crank);
                    break;
                }
                const int64_t ns = n_beg + (int64_t)b * XB - xoff;        // even
                int64_t cnt = ((int64_t)XB + mpad + xoff + 1) & ~(int64_t)1;
                if (cnt > it.x_avail - ns) cnt = it.x_avail - ns;
                int64_t ys = 0, ycnt = 0;
                if (cross) {
                    ys = n_beg + (int64_t)b * XB + D - yoff;              // even
                    ycnt = ((int64_t)XB + yoff + 1) & ~(int64_t)1;
                    if (ycnt > it.x_avail - ys) ycnt = it.x_avail - ys;
                }
                tc::mbar_arrive_expect_tx(&bars->xfull[slot], (uint32_t)((cnt + ycnt) * 8));
                if (cross) tc::bulk_g2s(xs + slot * XSLOT + YOFF, it.y + ys, (uint32_t)(ycnt * 8), &bars->xfull[slot]);
                const uint64_t pos = (uint64_t)ns & it.xmask;
                const uint64_t room = it.xmask - pos + 1;        // samples before the ring wraps
                if (it.xmask == ~0ull || (uint64_t)cnt <= room) {
                    tc::bulk_g2s(xs + slot * XSLOT, it.x + pos, (uint32_t)(cnt * 8), &bars->xfull[slot]);
                } else {
                    tc::bulk_g2s(xs + slot * XSLOT, it.x + pos, (uint32_t)(room * 8), &bars->xfull[slot]);
                    tc::bulk_g2s(xs + slot * XSLOT + room, it.x, (uint32_t)((cnt - room) * 8), &bars->xfull[slot]);
                }
                lastb = (int)bg;
            }
        } else if (warp == MMA_WARP && lane == 0 && crank == 0) {
            // -------------------------------------------------------- MMA issuer
            const uint32_t idesc = tc::idesc_f16(2 * ROWS, 2 * TILE_CC, C::BF);
            const uint32_t pbase = tc::smem_u32(smem);
            bool stop = false;
            for (int j = 0; j < nchains && !stop; ++j) {
                const uint32_t Jg = J + j;
                if (Jg >= 1 && !tc::mbar_wait_ab<true>(&bars->tfree, (Jg - 1) & 1, budget, ab)) {
                    give_up(ctl, bars, 6, crank);
                    break;
                }
                tc::tc_fence_after();
                const int g0 = j * CG, g1 = min(ngroups, g0 + CG);
                for (int g = g0; g < g1; ++g) {
                    const uint32_t Gg = G + g;
                    const int s = Gg % C::NSTAGE;
                    if (!tc::mbar_wait_ab<true>(&bars->full[s], (Gg / C::NSTAGE) & 1, budget, ab)) {
                        give_up(ctl, bars, 2, crank);
                        stop = true;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t sb = pbase + s * stage_bytes<PREC>();
#pragma unroll
                    for (int p = 0; p < C::NPASS; ++p) {
                        const int la = (p == 2) ? 1 : 0, lb = (p == 1) ? 1 : 0;
                        const uint64_t bdesc = tc::smem_desc(sb + lb * LEVEL_BYTES + NSUB * OPB, LBO, SBO);
#pragma unroll
                        for (int sub = 0; sub < NSUB; ++sub) {
                            const uint64_t adesc = tc::smem_desc(sb + la * LEVEL_BYTES + sub * OPB, LBO, SBO);
                            tc::mma_f16_pair(tmem + sub * TM_COLS, adesc, bdesc, idesc, (g > g0 || p > 0) ? 1u : 0u);
                        }
                    }
                    mma_issued = true;
                    tc::mma_commit_pair(&bars->empty[s], 3);
                }
                if (!stop) tc::mma_commit_pair(&bars->done, 3);
            }
        }
        G += ngroups;
        Bk += nblocks;
        J += nchains;
        ++nit;
        // everybody is done with this item's descriptor before thread 0 replaces it
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
    }

    // no sample copy may still be landing and no MMA still running when the CTAs exit
    // (these waits ignore the abort flag: the copies and MMAs complete on their own)
    if (warp == LOAD_WARP && lane == 0)
        for (int b = lastb > 0 ? lastb - 1 : 0; b <= lastb; ++b)
            if (b >= 0) tc::mbar_wait(&bars->xfull[b & 1], (b >> 1) & 1, budget);
    if (warp == MMA_WARP && lane == 0 && crank == 0 && mma_issued) {
        tc::mma_commit_pair(&bars->fin, 1);
        tc::mbar_wait(&bars->fin, 0, budget);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::cluster_sync();                              // no MMA of the pair still uses this CTA
    if (warp == MMA_WARP) {
        tc::tc_fence_after();
        tc::tmem_dealloc_pair<NSUB * TM_COLS>(tmem);
    }
}

template <int PREC, bool LIST>
cudaError_t set_smem()
{
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(proj_tc_kernel<PREC, LIST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes<PREC>());
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

template <int PREC, bool LIST>
cudaError_t launch_pairs(dim3 grid, const ProjArgs& a, const TcItem* items, const int* nitems, int* counter,
                         const Ctl& ctl, cudaStream_t st)
{
    cudaError_t e = set_smem<PREC, LIST>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
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
    return cudaLaunchKernelEx(&cfg, proj_tc_kernel<PREC, LIST>, a, items, nitems, counter, ctl);
}

// CTA pairs that can be resident at once (0: cluster launches unavailable).
template <int PREC>
int pair_slots()
{
    if (set_smem<PREC, false>() != cudaSuccess) return 0;
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
    if (cudaOccupancyMaxActiveClusters(&n, proj_tc_kernel<PREC, false>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ProjArgs empty_args()
{
    ProjArgs none;
    none.x = nullptr; none.nc = 0; none.nbase = 0; none.phi = nullptr; none.Au = 0; none.col_lag = nullptr;
    none.col_conj = nullptr; none.ncols = 0; none.nsplit = 0; none.split_len = 0; none.part = nullptr;
    return none;
}

}  // namespace

bool tc_supported(int ncols, int M) { return ncols > 0 && M >= 0 && M <= MAX_LAG; }

int tc_pair_units() { return ITEM_UNITS; }
int tc_tile_cols() { return TILE_CC; }
int tc_tile_rows() { return 2 * ITEM_UNITS; }

int tc_pair_ctas(int precision)
{
    const int n = precision == CYC_P_FP16 ? pair_slots<CYC_P_FP16>()
                : precision == CYC_P_BF16X3 ? pair_slots<CYC_P_BF16X3>() : 0;
    return 2 * n;
}

// CTAs per split: two per (unit tile, column tile).
static int tc_ctas(int U, int ncols)
{
    return 2 * ((U + ITEM_UNITS - 1) / ITEM_UNITS) * ((ncols + TILE_CC - 1) / TILE_CC);
}

ProjPlan tc_plan(int U, int Au, int ncols, int64_t nc, int num_sms, int pair_ctas)
{
    const int tiles = tc_ctas(U, ncols);
    const int slots = pair_ctas < num_sms ? pair_ctas : num_sms;
    // splits of at least 2048 samples, within what the partial buffer holds
    int smax = max_splits(tiles, num_sms, Au, ncols);
    if ((int64_t)smax > nc / 2048) smax = (int)(nc / 2048);
    const int want = wave_splits(tiles, slots > 0 ? slots : 1, smax);
    int64_t len = (nc + want - 1) / want;
    if (len < 256) len = 256;
    len = (len + GS - 1) / GS * GS;
    ProjPlan p;
    p.split_len = len;
    p.nsplit = (int)((nc + len - 1) / len);
    if (p.nsplit < 1) p.nsplit = 1;
    return p;
}

size_t tc_max_partials(int U, int Au, int ncols, int num_sms)
{
    return (size_t)max_splits(tc_ctas(U, ncols), num_sms, Au, ncols) * (size_t)Au * (size_t)ncols;
}

cudaError_t tc_launch(const ProjArgs& a, int precision, cudaStream_t st)
{
    const dim3 grid(2 * ((a.U + ITEM_UNITS - 1) / ITEM_UNITS), (a.ncols + TILE_CC - 1) / TILE_CC, a.nsplit);
    const Ctl ctl{a.err, a.budget > 0 ? a.budget : kDefaultWaitBudget, a.withhold};
    if (precision == CYC_P_FP16)
        return launch_pairs<CYC_P_FP16, false>(grid, a, nullptr, nullptr, nullptr, ctl, st);
    if (precision == CYC_P_BF16X3)
        return launch_pairs<CYC_P_BF16X3, false>(grid, a, nullptr, nullptr, nullptr, ctl, st);
    return cudaErrorInvalidValue;
}

cudaError_t tc_launch_items(const TcItem* items, const int* nitems, int* counter, int grid, int precision, int* err,
                            long long budget, cudaStream_t st)
{
    const Ctl ctl{err, budget > 0 ? budget : kDefaultWaitBudget, 0};
    const dim3 g((grid + 1) & ~1);
    if (precision == CYC_P_FP16)
        return launch_pairs<CYC_P_FP16, true>(g, empty_args(), items, nitems, counter, ctl, st);
    if (precision == CYC_P_BF16X3)
        return launch_pairs<CYC_P_BF16X3, true>(g, empty_args(), items, nitems, counter, ctl, st);
    return cudaErrorInvalidValue;
}

}  // namespace cyc
