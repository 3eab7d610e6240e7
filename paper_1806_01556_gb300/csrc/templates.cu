// Template bank generation (FIR coefficients of the FT convolution, Sec. 2.1).
//
// The paper gives 85 filters of 421 taps but not their definition. The library reads them as
// the Fourier response of a linearly drifting tone, indexed by mean frequency:
//     A_z(q) = integral_0^1 exp(2 pi i (-(q + z/2) tau + z tau^2 / 2)) d tau.
// Two kernels, both in double precision:
//   1. fdas_quad_taps: one thread per (template, tap). It evaluates A_z(q) by composite
//      16-point Gauss-Legendre quadrature, with enough panels that each panel spans less than
//      one cycle of the integrand. It writes the taps (double2) temporarily into the first
//      n_tap*16 bytes of the template's own output row.
//   2. fdas_dft_taps: one CTA per template. It copies its taps to shared memory, then writes
//      T[m] = conj(sum_q a[q] exp(-2 pi i m q / F)) as complex64 over the same row. The extra
//      CTA (blockIdx.x == n_temp) writes the float twiddle table exp(-2 pi i k / F) used by the
//      convolution kernel.
#include <cmath>

#include "fdas_internal.cuh"

namespace fdas {
namespace {

constexpr int kGlNodes = 16;

struct GaussLegendre {
    double x[kGlNodes];  // nodes on (-1, 1)
    double w[kGlNodes];  // weights, summing to 2
};

// Nodes and weights of the n-point Gauss-Legendre rule: Newton iteration on the Legendre
// polynomial P_n from the usual cosine initial guess; w = 2 / ((1 - x^2) P_n'(x)^2).
GaussLegendre gauss_legendre_16() {
    GaussLegendre g;
    const int n = kGlNodes;
    for (int i = 0; i < n; ++i) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        g.x[i] = x;
        g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return g;
}

__global__ void fdas_quad_taps(GaussLegendre gl, int n_temp, int n_tap, int z_min, int z_step, int n_panel,
                               int fft_len, double2 *rows) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n_temp * n_tap) return;
    const int t = gid / n_tap;
    const int qi = gid - t * n_tap;
    const int h = (n_tap - 1) / 2;
    const double q = (double)(qi - h);
    const double z = (double)(z_min + t * z_step);
    double re = 0.0, im = 0.0;
    if (z == 0.0) {
        re = (qi == h) ? 1.0 : 0.0;  // A_0(q) is the unit impulse
    } else {
        const double inv_p = 1.0 / n_panel;
        const double lin = -(q + 0.5 * z);
        for (int p = 0; p < n_panel; ++p) {
            const double left = p * inv_p;
#pragma unroll
            for (int k = 0; k < kGlNodes; ++k) {
                const double tau = left + (gl.x[k] + 1.0) * 0.5 * inv_p;
                double cyc = fma(0.5 * z * tau, tau, lin * tau);
                cyc -= floor(cyc);
                double s, c;
                sincospi(2.0 * cyc, &s, &c);
                const double wk = gl.w[k] * 0.5 * inv_p;
                re = fma(wk, c, re);
                im = fma(wk, s, im);
            }
        }
    }
    // The template's output row starts at t * fft_len complex64 = t * fft_len / 2 double2.
    rows[(size_t)t * (fft_len / 2) + qi] = make_double2(re, im);
}

__global__ void fdas_dft_taps(int n_temp, int n_tap, int fft_len, double2 *rows_d, float2 *rows_f) {
    extern __shared__ double2 sm[];
    double2 *tw = sm;             // fft_len entries: exp(-2 pi i k / F)
    double2 *taps = sm + fft_len;  // n_tap entries
    const int t = blockIdx.x;
    for (int k = threadIdx.x; k < fft_len; k += blockDim.x) {
        double s, c;
        sincospi(2.0 * k / fft_len, &s, &c);
        tw[k] = make_double2(c, -s);
    }
    if (t == n_temp) {  // twiddle row for the convolution kernel
        __syncthreads();
        for (int k = threadIdx.x; k < fft_len; k += blockDim.x)
            rows_f[(size_t)n_temp * fft_len + k] = make_float2((float)tw[k].x, (float)tw[k].y);
        return;
    }
    for (int qi = threadIdx.x; qi < n_tap; qi += blockDim.x) taps[qi] = rows_d[(size_t)t * (fft_len / 2) + qi];
    __syncthreads();  // every tap is in shared memory before the row is overwritten below
    const int h = (n_tap - 1) / 2;
    const int mask = fft_len - 1;
    for (int m = threadIdx.x; m < fft_len; m += blockDim.x) {
        double re = 0.0, im = 0.0;
        int idx = (int)(((long long)m * (fft_len - h)) & mask);  // m * (-h) mod F
        for (int qi = 0; qi < n_tap; ++qi) {
            const double2 a = taps[qi];
            const double2 w = tw[idx];
            re = fma(a.x, w.x, fma(-a.y, w.y, re));
            im = fma(a.x, w.y, fma(a.y, w.x, im));
            idx = (idx + m) & mask;
        }
        rows_f[(size_t)t * fft_len + m] = make_float2((float)re, (float)-im);  // conjugate
    }
}

}  // namespace

cudaError_t launch_templates(const fdas_params &p, void *d_tmpl, cudaStream_t s) {
    static const GaussLegendre gl = gauss_legendre_16();
    const int h = (p.n_tap - 1) / 2;
    const int zmax = std::abs(p.z_min);
    // Phase rate of the integrand is at most |q| + |z|/2 cycles per unit tau; keep panels under a cycle.
    const int n_panel = 16 + h + (zmax + 1) / 2;
    const int total = p.n_temp * p.n_tap;
    fdas_quad_taps<<<(total + 127) / 128, 128, 0, s>>>(gl, p.n_temp, p.n_tap, p.z_min, p.z_step, n_panel, p.fft_len,
                                                       static_cast<double2 *>(d_tmpl));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)(p.fft_len + p.n_tap) * sizeof(double2);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(fdas_dft_taps, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fdas_dft_taps<<<p.n_temp + 1, 512, smem, s>>>(p.n_temp, p.n_tap, p.fft_len, static_cast<double2 *>(d_tmpl),
                                                  static_cast<float2 *>(d_tmpl));
    return cudaGetLastError();
}

}  // namespace fdas
