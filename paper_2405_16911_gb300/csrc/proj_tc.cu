// proj_tc.cu -- tensor-core a-projection (tcgen05, sm_103a): FP16 single pass and the
// BF16 three-product split, FP32 accumulation in tensor memory.
//
// Per CTA: 128 cycle frequencies (MMA M) x 256 columns (MMA N) x one n-split.  The complex
// GEMM  S[u][c] = sum_n W[u][n] P_c(n)  (Sec. 4 Set mode: the per-alpha projection of the
// lag products; W = exp(-j 2 pi a n), P = x[n+m] x*[n] or x[n+m] x[n], Eqs. (ACF-def),
// (CCF-def)) is run as two real GEMMs over K = (re, im) of 8 samples per K=16 step:
//     D_r += [Wr | -Wi] . [Pr ; Pi]        D_i += [Wi | Wr] . [Pr ; Pi]
// D_r and D_i live in TMEM columns [0, 256) and [256, 512).  The phase is folded into W
// with the absolute sample index, so the whole n-range accumulates in TMEM without any
// per-tile rotation; the epilogue writes one FP32 partial per CTA.
//
// Warp roles (544 threads): two producer sets, set k producing the groups g = k mod 2, so
// that one set's load and sine latencies hide behind the other's work.  In set k:
//   warps 8k+0..3  P producers: thread t forms the lag products of tile columns 2t and 2t+1
//                  (with lag-major columns, both forms of one lag) -> B-operand rows t, t+128
//   warps 8k+4..7  W producers: thread t forms W for cycle frequency row t; those of set 0
//                  are afterwards the epilogue (TMEM lane quadrant = warp % 4 = row / 32)
//   warp 16        TMEM allocation; lane 0 issues every tcgen05.mma and commit
//   warp 17        lane 0 streams the samples into shared memory: blocks of XB samples plus
//                  the M-sample halo, by TMA bulk copy into a ring of two slots ("xfull":
//                  transaction-counted, "xempty": released by the eight P warps)
// Operands go through an NSTAGE ring of shared-memory stages (one 8-sample group each),
// guarded by "full" (producers -> MMA) and "empty" (tcgen05.commit -> producers) mbarriers.
// Operand layout: K-major, no swizzle, 8-row x 16-byte core matrices.
//   P block: row r (column), chunk k (0: Pr, 1: Pi) at (r/8)*256 + k*128 + (r%8)*16
//   W block: row r (cycle freq), chunk k (0: Wi, 1: Wr, 2: -Wi) at (r/8)*384 + k*128 + (r%8)*16
// so that [Wr | -Wi] starts at chunk 1 and [Wi | Wr] at chunk 0, both with LBO = 128.
// BF16x3 keeps a hi and a lo copy of each block: v = hi + lo, hi = bf16(v), lo = bf16(v - hi),
// and issues hi.hi, hi.lo, lo.hi.
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
constexpr int MMA_WARP = 8 * NSET;
constexpr int LOAD_WARP = MMA_WARP + 1;
constexpr int NTHREADS = (LOAD_WARP + 1) * 32;
constexpr int XSLOT = 3072;              // samples per staging slot (block + halo)
constexpr int MAX_LAG = 2560;            // leaves blocks of at least 512 samples
constexpr int P_BYTES = 8192, W_BYTES = 6144;
constexpr uint32_t P_LBO = 128, P_SBO = 256, W_LBO = 128, W_SBO = 384;
constexpr long long WAIT_BUDGET = 2000000000ll;   // SM cycles (about one second)

template <int PREC>
struct Cfg;
template <>
struct Cfg<CYC_P_FP16> {
    static constexpr int NLEV = 1, NPASS = 1, NSTAGE = 10;
    static constexpr bool BF = false;
};
template <>
struct Cfg<CYC_P_BF16X3> {
    static constexpr int NLEV = 2, NPASS = 3, NSTAGE = 6;
    static constexpr bool BF = true;
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
__device__ __forceinline__ void pack8(const float (&v)[8], uint4& hi, uint4& lo)
{
    if constexpr (BF) {
        hi.x = pack_b2(v[0], v[1], &lo.x);
        hi.y = pack_b2(v[2], v[3], &lo.y);
        hi.z = pack_b2(v[4], v[5], &lo.z);
        hi.w = pack_b2(v[6], v[7], &lo.w);
    } else {
        hi = make_uint4(pack_h2(v[0], v[1]), pack_h2(v[2], v[3]), pack_h2(v[4], v[5]), pack_h2(v[6], v[7]));
    }
}

__device__ __forceinline__ uint4 neg8(uint4 v)
{
    const uint32_t s = 0x80008000u;
    return make_uint4(v.x ^ s, v.y ^ s, v.z ^ s, v.w ^ s);
}

__device__ __forceinline__ void st16(unsigned char* p, uint4 v) { *reinterpret_cast<uint4*>(p) = v; }

struct Bars {
    uint64_t full[16];
    uint64_t empty[16];
    uint64_t xfull[2];
    uint64_t xempty[2];
    uint64_t done;
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ void flag_error(const ProjArgs& a, Bars* b, int code)
{
    b->abort = 1;
    if (a.err) atomicCAS(a.err, 0, code);
}

template <int PREC>
__global__ void __launch_bounds__(NTHREADS, 1) proj_tc_kernel(ProjArgs a)
{
    using C = Cfg<PREC>;
    extern __shared__ __align__(1024) unsigned char smem[];
    Bars* bars = reinterpret_cast<Bars*>(smem + xslots_off<PREC>() + 2 * XSLOT * 8);
    float2* xs = reinterpret_cast<float2*>(smem + xslots_off<PREC>());     // two slots of XSLOT samples
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int u0 = blockIdx.x * BM;
    const int c0 = blockIdx.y * BN;
    const int64_t n_beg = (int64_t)blockIdx.z * a.split_len;
    int64_t n_end = n_beg + a.split_len;
    if (n_end > a.nc) n_end = a.nc;
    const int ngroups = n_end > n_beg ? (int)((n_end - n_beg + GS - 1) / GS) : 0;
    const int mpad = (a.M + 1) & ~1;
    const int XB = (XSLOT - mpad) & ~(GS - 1);            // samples per staged block
    const int nblocks = (ngroups * GS + XB - 1) / XB;

    if (tid == 0) {
        for (int s = 0; s < C::NSTAGE; ++s) {
            tc::mbar_init(&bars->full[s], 8);      // one arrival per producer warp
            tc::mbar_init(&bars->empty[s], 1);     // one tcgen05.commit
        }
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(&bars->xfull[k], 1);     // loader's arrive.expect_tx (+ bytes)
            tc::mbar_init(&bars->xempty[k], 4 * NSET);
        }
        tc::mbar_init(&bars->done, 1);
        bars->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) tc::tmem_alloc<512>(&bars->tmem);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = bars->tmem;

    const int pset = warp < MMA_WARP ? warp / 8 : 0;       // producer set
    const int role = warp % 8;                              // 0-3 P, 4-7 W
    if (warp < MMA_WARP && role < 4) {
        // ------------------------------------------------------------ P producers
        const int t = tid - pset * 256;                     // 0..127
        const int jA = 2 * t, jB = 2 * t + 1;               // tile-local columns
        const bool okA = c0 + jA < a.ncols, okB = c0 + jB < a.ncols;
        const int mA = okA ? a.col_lag[c0 + jA] : 0, mB = okB ? a.col_lag[c0 + jB] : 0;
        const bool cjA = okA && a.col_conj[c0 + jA], cjB = okB && a.col_conj[c0 + jB];
        const uint32_t offA = (t / 8) * P_SBO + (t % 8) * 16;               // B-operand row t
        const uint32_t offB = ((t + 128) / 8) * P_SBO + (t % 8) * 16;       // row t + 128
        const bool same_lag = okB && mA == mB;
        int cur_b = -1;
        for (int g = pset; g < ngroups; g += NSET) {
            const int s = g % C::NSTAGE;
            if (g >= C::NSTAGE && !tc::mbar_wait(&bars->empty[s], ((g / C::NSTAGE) - 1) & 1, WAIT_BUDGET)) {
                flag_error(a, bars, 1);
                break;
            }
            const int b = (g * GS) / XB;
            if (b != cur_b) {
                __syncwarp();
                if (cur_b >= 0 && lane == 0) tc::mbar_arrive(&bars->xempty[cur_b & 1]);
                if (!tc::mbar_wait(&bars->xfull[b & 1], (b >> 1) & 1, WAIT_BUDGET)) {
                    flag_error(a, bars, 4);
                    break;
                }
                cur_b = b;
            }
            const float2* xb = xs + (b & 1) * XSLOT + (g * GS - b * XB);   // sample n_beg + 8g
            float prA[8], piA[8], prB[8], piB[8];
            const int64_t n = n_beg + (int64_t)g * GS;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float2 pA = make_float2(0.f, 0.f), pB = make_float2(0.f, 0.f);
                if (n + i < n_end) {
                    float2 x0 = xb[i];
                    float2 xa = okA ? xb[i + mA] : make_float2(0.f, 0.f);
                    float2 xv = same_lag ? xa : (okB ? xb[i + mB] : make_float2(0.f, 0.f));
                    if (okA) pA = lag_product(xa, x0, cjA);
                    if (okB) pB = lag_product(xv, x0, cjB);
                }
                prA[i] = pA.x; piA[i] = pA.y; prB[i] = pB.x; piB[i] = pB.y;
            }
            unsigned char* st = smem + s * stage_bytes<PREC>();
            uint4 h, l;
            pack8<C::BF>(prA, h, l);
            st16(st + offA, h);
            if (C::BF) st16(st + P_BYTES + W_BYTES + offA, l);
            pack8<C::BF>(piA, h, l);
            st16(st + offA + P_LBO, h);
            if (C::BF) st16(st + P_BYTES + W_BYTES + offA + P_LBO, l);
            pack8<C::BF>(prB, h, l);
            st16(st + offB, h);
            if (C::BF) st16(st + P_BYTES + W_BYTES + offB, l);
            pack8<C::BF>(piB, h, l);
            st16(st + offB + P_LBO, h);
            if (C::BF) st16(st + P_BYTES + W_BYTES + offB + P_LBO, l);
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bars->full[s]);
        }
    } else if (warp < MMA_WARP) {
        // ------------------------------------------------------------ W producers
        const int t = tid - pset * 256 - 128;               // row 0..127
        const bool ok = u0 + t < a.Au;
        const uint64_t phi = ok ? a.phi[u0 + t] : 0ull;
        const uint32_t offW = (t / 8) * W_SBO + (t % 8) * 16;
        for (int g = pset; g < ngroups; g += NSET) {
            const int s = g % C::NSTAGE;
            if (g >= C::NSTAGE && !tc::mbar_wait(&bars->empty[s], ((g / C::NSTAGE) - 1) & 1, WAIT_BUDGET)) {
                flag_error(a, bars, 1);
                break;
            }
            float wr[8], wi[8];
            if (ok) {
                // each weight straight from the exact u64 phase phi * n mod 2^64
                const uint64_t n = a.nbase + (uint64_t)(n_beg + (int64_t)g * GS);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float2 w = phase_rot(phi, n + (uint64_t)i);
                    wr[i] = w.x;
                    wi[i] = w.y;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) { wr[i] = 0.f; wi[i] = 0.f; }
            }
            unsigned char* st = smem + s * stage_bytes<PREC>() + P_BYTES;
            uint4 rh, rl, ih, il;
            pack8<C::BF>(wr, rh, rl);
            pack8<C::BF>(wi, ih, il);
            st16(st + offW + 0 * W_LBO, ih);
            st16(st + offW + 1 * W_LBO, rh);
            st16(st + offW + 2 * W_LBO, neg8(ih));
            if (C::BF) {
                unsigned char* sl = st + P_BYTES + W_BYTES;
                st16(sl + offW + 0 * W_LBO, il);
                st16(sl + offW + 1 * W_LBO, rl);
                st16(sl + offW + 2 * W_LBO, neg8(il));
            }
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bars->full[s]);
        }
    } else if (warp == LOAD_WARP && lane == 0) {
        // ------------------------------------------------------------ sample loader (TMA)
        int last = -1;
        for (int b = 0; b < nblocks; ++b) {
            const int slot = b & 1;
            if (b >= 2 && !tc::mbar_wait(&bars->xempty[slot], ((b >> 1) - 1) & 1, WAIT_BUDGET)) {
                flag_error(a, bars, 5);
                break;
            }
            const int64_t ns = n_beg + (int64_t)b * XB;
            int64_t cnt = (int64_t)XB + mpad;
            if (cnt > a.x_avail - ns) cnt = a.x_avail - ns;
            cnt &= ~(int64_t)1;
            tc::mbar_arrive_expect_tx(&bars->xfull[slot], (uint32_t)(cnt * 8));
            tc::bulk_g2s(xs + slot * XSLOT, a.x + ns, (uint32_t)(cnt * 8), &bars->xfull[slot]);
            last = b;
        }
        // no copy may still be landing when the CTA exits
        for (int b = last > 0 ? last - 1 : 0; b <= last; ++b)
            if (b >= 0) tc::mbar_wait(&bars->xfull[b & 1], (b >> 1) & 1, WAIT_BUDGET);
    } else if (warp == MMA_WARP && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        constexpr uint32_t idesc = tc::idesc_f16(BM, BN, C::BF);
        const uint32_t base = tc::smem_u32(smem);
        for (int g = 0; g < ngroups; ++g) {
            const int s = g % C::NSTAGE;
            if (!tc::mbar_wait(&bars->full[s], (g / C::NSTAGE) & 1, WAIT_BUDGET)) {
                flag_error(a, bars, 2);
                break;
            }
            tc::tc_fence_after();
            const uint32_t sb = base + s * stage_bytes<PREC>();
#pragma unroll
            for (int p = 0; p < C::NPASS; ++p) {
                const int la = (p == 2) ? 1 : 0, lb = (p == 1) ? 1 : 0;
                const uint32_t pb = sb + lb * (P_BYTES + W_BYTES);
                const uint32_t wb = sb + la * (P_BYTES + W_BYTES) + P_BYTES;
                const uint64_t bdesc = tc::smem_desc(pb, P_LBO, P_SBO);
                const uint64_t ar = tc::smem_desc(wb + 1 * W_LBO, W_LBO, W_SBO);
                const uint64_t ai = tc::smem_desc(wb + 0 * W_LBO, W_LBO, W_SBO);
                const uint32_t acc = (g > 0 || p > 0) ? 1u : 0u;
                tc::mma_f16(tmem, ar, bdesc, idesc, acc);
                tc::mma_f16(tmem + 256, ai, bdesc, idesc, acc);
            }
            tc::mma_commit(&bars->empty[s]);
        }
        tc::mma_commit(&bars->done);
    }

    // ---------------------------------------------------------------- epilogue (warps 4-7)
    if (warp >= 4 && warp < 8) {
        const bool got = tc::mbar_wait(&bars->done, 0, WAIT_BUDGET);
        if (!got) flag_error(a, bars, 3);
        tc::tc_fence_after();
        const int q = warp & 3;                  // TMEM lane quadrant
        const int row = q * 32 + lane;
        const int u = u0 + row;
        float2* out = a.part + ((size_t)blockIdx.z * a.Au + (size_t)(u < a.Au ? u : 0)) * a.ncols;
        const bool vec = (a.ncols & 1) == 0;     // rows start 16-byte aligned
        for (int cb = 0; cb < 8; ++cb) {
            uint32_t dr0[16], di0[16], dr1[16], di1[16];
            const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
            tc::tmem_ld16(lane_addr + cb * 16, dr0);
            tc::tmem_ld16(lane_addr + 256 + cb * 16, di0);
            tc::tmem_ld16(lane_addr + 128 + cb * 16, dr1);
            tc::tmem_ld16(lane_addr + 384 + cb * 16, di1);
            tc::tmem_ld_wait();
            if (u >= a.Au) continue;
            const bool live = got && ngroups > 0;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int r = cb * 16 + j;               // B-operand rows r, r + 128 <-> columns 2r, 2r+1
                const int c = c0 + 2 * r;
                float4 v = live ? make_float4(__uint_as_float(dr0[j]), __uint_as_float(di0[j]),
                                              __uint_as_float(dr1[j]), __uint_as_float(di1[j]))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
                if (vec && c + 1 < a.ncols) {
                    *reinterpret_cast<float4*>(&out[c]) = v;
                } else {
                    if (c < a.ncols) out[c] = make_float2(v.x, v.y);
                    if (c + 1 < a.ncols) out[c + 1] = make_float2(v.z, v.w);
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc::tc_fence_after();
        tc::tmem_dealloc<512>(tmem);
    }
}

int tiles_of(int Au, int ncols) { return ((Au + BM - 1) / BM) * ((ncols + BN - 1) / BN); }

template <int PREC>
cudaError_t launch(const ProjArgs& a, cudaStream_t st)
{
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(proj_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem_bytes<PREC>());
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    dim3 grid((a.Au + BM - 1) / BM, (a.ncols + BN - 1) / BN, a.nsplit);
    proj_tc_kernel<PREC><<<grid, NTHREADS, smem_bytes<PREC>(), st>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool tc_supported(int ncols, int M) { return ncols > 0 && M >= 0 && M <= MAX_LAG; }

ProjPlan tc_plan(int Au, int ncols, int64_t nc, int num_sms)
{
    int tiles = tiles_of(Au, ncols);
    int want = num_sms >= tiles ? num_sms / tiles : 1;
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
    int tiles = tiles_of(Au, ncols);
    size_t want = num_sms >= tiles ? (size_t)(num_sms / tiles) : 1;
    return want * (size_t)Au * (size_t)ncols;
}

cudaError_t tc_launch(const ProjArgs& a, int precision, cudaStream_t st)
{
    if (precision == CYC_P_FP16) return launch<CYC_P_FP16>(a, st);
    if (precision == CYC_P_BF16X3) return launch<CYC_P_BF16X3>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace cyc
