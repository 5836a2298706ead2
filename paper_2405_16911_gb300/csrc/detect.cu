// detect.cu -- cycle-frequency detection on a stream's estimate (cyc_detect, include/cyc.h).
//
// The paper names the estimation of cycle frequencies as its next step (Sec. 6).  The rule is
// a constant-false-alarm test per form over the stream's cycle-frequency list read as a
// circular grid: the statistic s(a) = max over lags |R^a(m)|^2 (zero for the conventional
// form at a = 0 mod 1 of a one-input stream: that entry is the mean power), the noise level
// nu(a) = the median of s over the offsets +-2 .. +-win (the mean of the two middle values;
// the immediate neighbours are left out, they share the line's leakage), and a detection
// where s(a) > kappa nu(a) and s(a) is at least both of its neighbours.  Two small kernels:
// the statistic per (form, a) from the FP64 estimate, then the test per (form, a), each
// thread sorting its 2 (win - 1) neighbours' values.
#include "cyc_impl.h"

namespace cyc {
namespace {

constexpr int MAX_WIN = 32;

// s[f][a] = max_l |R[f][a][l]|^2; zero where f is the conventional form and dc[a] is set.
__global__ void statistic_kernel(const double2* __restrict__ R, int F, int A, int L, const uint8_t* __restrict__ dc,
                                 int conv_f, double* __restrict__ s)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= F * A) return;
    const int f = e / A, a = e - f * A;
    double m = 0.0;
    if (!(f == conv_f && dc[a])) {
        const double2* r = R + (size_t)e * L;
        for (int l = 0; l < L; ++l) {
            const double2 v = r[l];
            const double p = v.x * v.x + v.y * v.y;
            m = p > m ? p : m;
        }
    }
    s[e] = m;
}

// flags[f][a]: bit 0 detected, bit 1 local maximum; ratio[f][a] = s / max(nu, tiny).
__global__ void cfar_kernel(const double* __restrict__ s, int F, int A, int win, double kappa,
                            uint8_t* __restrict__ flags, float* __restrict__ ratio, int* __restrict__ count)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= F * A) return;
    const int f = e / A, a = e - f * A;
    const double* sf = s + (size_t)f * A;
    double v[2 * (MAX_WIN - 1)];
    int n = 0;
    for (int d = -win; d <= win; ++d) {
        if (d >= -1 && d <= 1) continue;
        const int j = ((a + d) % A + A) % A;
        // insertion into the sorted prefix v[0 .. n)
        const double x = sf[j];
        int i = n++;
        while (i > 0 && v[i - 1] > x) {
            v[i] = v[i - 1];
            --i;
        }
        v[i] = x;
    }
    const double nu = 0.5 * (v[n / 2 - 1] + v[n / 2]);
    const double sa = sf[a];
    const double r = sa / (nu > 1e-300 ? nu : 1e-300);
    const bool lm = sa >= sf[(a + A - 1) % A] && sa >= sf[(a + 1) % A];
    const bool det = lm && r > kappa;
    flags[e] = (uint8_t)((det ? 1 : 0) | (lm ? 2 : 0));
    if (ratio) ratio[e] = (float)r;
    if (det) atomicAdd(count, 1);
}

}  // namespace

bool detect_supported(int win) { return win >= 2 && win <= MAX_WIN; }

cudaError_t detect(const double2* R, int F, int A, int L, const uint8_t* dc, int conv_f, int win, double kappa,
                   double* s, uint8_t* flags, float* ratio, int* count, cudaStream_t st)
{
    const int n = F * A, bs = 128;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    statistic_kernel<<<(n + bs - 1) / bs, bs, 0, st>>>(R, F, A, L, dc, conv_f, s);
    cfar_kernel<<<(n + bs - 1) / bs, bs, 0, st>>>(s, F, A, win, kappa, flags, ratio, count);
    return cudaGetLastError();
}

}  // namespace cyc
