// chi^2 / extreme-value significance fit of IG^k_max (section "Theory" of
// arXiv 1811.00631), in FP64 on the device.
//
// A single null tuple gives 2 IG ~ chi^2_df; the maximum over T effective
// tests has CDF F_df(2 g)^T.  T is the maximum-likelihood estimate over the
// irrelevant variables, T = -n / sum ln F_df(2 IG_i); p_i = 1 - F^T and
// IG_lim = F^{-1}((1 - alpha)^(1/T)) / 2.
//
// F_df(x) = P(df/2, x/2), the regularised lower incomplete gamma function,
// evaluated with the power series (Abramowitz & Stegun 6.5.29) below a + 1
// and with the Legendre continued fraction for the upper tail (A&S 6.5.31),
// summed by the modified Lentz method, above it.
#include <math.h>

#include "mdfs_internal.cuh"

namespace mdfs {

__device__ double gamma_p_series(double a, double x) {
    // P(a, x) = x^a e^-x / Gamma(a + 1) * sum_n x^n / ((a+1)...(a+n))
    double term = 1.0, sum = 1.0, ap = a;
    for (int n = 0; n < 2000; ++n) {
        ap += 1.0;
        term *= x / ap;
        sum += term;
        if (fabs(term) < fabs(sum) * 1e-17) break;
    }
    return exp(a * log(x) - x - lgamma(a + 1.0)) * sum;
}

__device__ double gamma_q_fraction(double a, double x) {
    // Q(a, x) = x^a e^-x / Gamma(a) * 1 / (x + 1 - a - 1 (1 - a) / (x + 3 - a - 2 (2 - a) / (...)))
    const double tiny = 1e-300;
    double b = x + 1.0 - a;
    double c = 1.0 / tiny;
    double d = 1.0 / b;
    double h = d;
    for (int i = 1; i < 2000; ++i) {
        const double an = -i * (i - a);
        b += 2.0;
        d = an * d + b;
        if (fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        const double del = d * c;
        h *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    return exp(a * log(x) - x - lgamma(a)) * h;
}

__device__ double chi2_cdf(double x, int df) {
    if (!(x > 0.0)) return 0.0;
    const double a = 0.5 * df, z = 0.5 * x;
    if (z < a + 1.0) return gamma_p_series(a, z);
    return 1.0 - gamma_q_fraction(a, z);
}

__global__ void __launch_bounds__(256) ig_lim_kernel(const float* __restrict__ ig, int M, int df,
                                                     const uint8_t* __restrict__ mask, double alpha,
                                                     double* __restrict__ p_values, double* __restrict__ res) {
    __shared__ double s_sum[8];
    __shared__ int s_n[8];
    __shared__ double s_T;
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double sum = 0.0;
    int n = 0;
    for (int i = tid; i < M; i += blockDim.x) {
        if (mask && !mask[i]) continue;
        const double u = chi2_cdf(2.0 * (double)ig[i], df);
        if (u > 0.0) {
            sum += log(u);
            ++n;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    if (lane == 0) {
        s_sum[warp] = sum;
        s_n[warp] = n;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        int nn = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t += s_sum[w];
            nn += s_n[w];
        }
        s_ok = (nn > 0 && t < 0.0);
        s_T = s_ok ? -(double)nn / t : 0.0;
        res[2] = (double)nn;
        res[1] = s_T;
    }
    __syncthreads();
    if (!s_ok) return;
    const double T = s_T;
    for (int i = tid; i < M; i += blockDim.x) {
        const double u = chi2_cdf(2.0 * (double)ig[i], df);
        p_values[i] = u > 0.0 ? -expm1(T * log(u)) : 1.0;
    }
    if (tid == 0) {
        const double target = pow(1.0 - alpha, 1.0 / T);
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 1100 && chi2_cdf(hi, df) < target; ++it) hi *= 2.0;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (chi2_cdf(mid, df) < target) lo = mid;
            else hi = mid;
        }
        res[0] = 0.25 * (lo + hi);
    }
}

cudaError_t launch_ig_lim(const float* ig, int M, int df, const uint8_t* mask, double alpha, double* p_values,
                          double* res, cudaStream_t st) {
    ig_lim_kernel<<<1, 256, 0, st>>>(ig, M, df, mask, alpha, p_values, res);
    return cudaGetLastError();
}

}  // namespace mdfs
