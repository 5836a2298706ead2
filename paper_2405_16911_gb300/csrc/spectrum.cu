// spectrum.cu -- cyclic spectra from a stream's cyclic correlation estimate (the cyclic
// correlogram; the paper lists cyclic spectra as its next step, Sec. 6):
//     S[f][a][q] = sum_l w(m_l) R[f][a][l] exp(-j 2 pi f_q m_l),   f_q = -1/2 + q/Q,
// w = 1 (rectangular) or the Hann lag window 0.5 + 0.5 cos(pi m / (Mmax + 1)).  In FP64: a
// [F A] x [L] by [L] x [Q] complex product with the DFT matrix E[l][q] built on the device.
#include "cyc_impl.h"

namespace cyc {
namespace {

__global__ void dft_matrix_kernel(const int32_t* __restrict__ lags, int L, int Q, int taper, double mmax,
                                  double2* __restrict__ E)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)L * Q) return;
    const int l = (int)(e / Q), q = (int)(e % Q);
    const int m = lags[l];
    const double w = taper ? 0.5 + 0.5 * cospi((double)m / (mmax + 1.0)) : 1.0;
    // f_q m mod 1 exactly: f_q = (2q - Q) / (2Q), so f_q m = (2q - Q) m / (2Q)
    const int64_t num = (int64_t)(2 * q - Q) * m;
    const int64_t den = 2 * (int64_t)Q;
    int64_t r = num % den;
    if (r < 0) r += den;
    double sn, cs;
    sincospi(-2.0 * (double)r / (double)den, &sn, &cs);
    E[e] = make_double2(w * cs, w * sn);
}

// S[rows][Q] = R[rows][L] x E[L][Q], complex FP64; block = 32 output columns x 32 rows,
// 256 threads (4 rows each), K tiles of 16 through shared memory.
__global__ void __launch_bounds__(256) zgemm_kernel(const double2* __restrict__ R, const double2* __restrict__ E,
                                                    int rows, int K, int Q, double2* __restrict__ S)
{
    __shared__ double2 Rs[32][17];
    __shared__ double2 Es[16][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int row0 = blockIdx.y * 32, col0 = blockIdx.x * 32;
    double2 acc[4];
    for (int i = 0; i < 4; ++i) acc[i] = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int t = threadIdx.x; t < 32 * 16; t += 256) {
            const int r = t / 16, kk = t % 16;
            Rs[r][kk] = (row0 + r < rows && k0 + kk < K) ? R[(size_t)(row0 + r) * K + k0 + kk] : make_double2(0.0, 0.0);
            const int kk2 = t / 32, c = t % 32;
            Es[kk2][c] = (k0 + kk2 < K && col0 + c < Q) ? E[(size_t)(k0 + kk2) * Q + col0 + c] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            const double2 e = Es[kk][tx];
            for (int i = 0; i < 4; ++i) {
                const double2 r = Rs[ty + 8 * i][kk];
                acc[i].x = fma(r.x, e.x, fma(-r.y, e.y, acc[i].x));
                acc[i].y = fma(r.x, e.y, fma(r.y, e.x, acc[i].y));
            }
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty + 8 * i, c = col0 + tx;
        if (r < rows && c < Q) S[(size_t)r * Q + c] = acc[i];
    }
}

}  // namespace

cudaError_t spectrum(const double2* R, const int32_t* lags, int rows, int L, int Q, int taper, double mmax,
                     double2* E, double2* S, cudaStream_t st)
{
    const int64_t ne = (int64_t)L * Q;
    dft_matrix_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(lags, L, Q, taper, mmax, E);
    dim3 grid((Q + 31) / 32, (rows + 31) / 32);
    zgemm_kernel<<<grid, 256, 0, st>>>(R, E, rows, L, Q, S);
    return cudaGetLastError();
}

}  // namespace cyc
