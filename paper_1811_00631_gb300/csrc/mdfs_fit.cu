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
#include <climits>
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

// Pass 1, one thread per variable: u_i = F_df(2 IG_i), written where the
// p-values will go (pass 3 turns them into p-values in place).
__global__ void __launch_bounds__(256) fit_cdf_kernel(const float* __restrict__ ig, int M, int df,
                                                      double* __restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) u[i] = chi2_cdf(2.0 * (double)ig[i], df);
}

// Pass 2, one CTA of 256 threads: T by maximum likelihood, then IG_lim.
// The sum of ln u_i runs in a fixed order (strided by thread, then a fixed
// reduction tree), so T is the same on every call.  IG_lim solves
// F_df(x) = (1 - alpha)^(1/T): the smallest power of two at or above the root
// comes from 256 points 2^0 .. 2^255 evaluated at once, then 12 rounds of
// 256-way multisection shrink the bracket [lo, hi] (F(lo) < target <= F(hi))
// by 257 each, far below the FP64 spacing of the root.
__global__ void __launch_bounds__(256) fit_t_kernel(const double* __restrict__ u, int M, int df,
                                                    const uint8_t* __restrict__ mask, double alpha,
                                                    double* __restrict__ res) {
    __shared__ double s_sum[8];
    __shared__ int s_n[8];
    __shared__ double s_T, s_lo, s_hi;
    __shared__ int s_ok, s_first;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double sum = 0.0;
    int n = 0;
    for (int i = tid; i < M; i += blockDim.x) {
        if (mask && !mask[i]) continue;
        const double ui = u[i];
        if (ui > 0.0) {
            sum += log(ui);
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
        s_first = INT_MAX;
    }
    __syncthreads();
    if (!s_ok) return;
    const double target = pow(1.0 - alpha, 1.0 / s_T);
    // bracket: the first 2^t (t = 0 .. 255) whose CDF reaches the target
    if (chi2_cdf(ldexp(1.0, tid), df) >= target) atomicMin(&s_first, tid);
    __syncthreads();
    if (tid == 0) {
        if (s_first == INT_MAX) {  // beyond 2^255: report that bound
            s_lo = s_hi = ldexp(1.0, (int)blockDim.x - 1);
        } else {
            s_hi = ldexp(1.0, s_first);
            s_lo = s_first > 0 ? ldexp(1.0, s_first - 1) : 0.0;
        }
    }
    __syncthreads();
    for (int round = 0; round < 12; ++round) {
        const double lo = s_lo, hi = s_hi;
        const double x = lo + (hi - lo) * ((double)(tid + 1) / (double)(blockDim.x + 1));
        const bool reached = chi2_cdf(x, df) >= target;
        __syncthreads();  // every thread has read the bracket
        if (tid == 0) s_first = INT_MAX;
        __syncthreads();
        if (reached) atomicMin(&s_first, tid);
        __syncthreads();
        const int first = s_first;
        if (first == tid) s_hi = x;                                        // first point at or above
        if (first == tid + 1) s_lo = x;                                    // the point before it
        if (first == INT_MAX && tid == (int)blockDim.x - 1) s_lo = x;      // every point below
        __syncthreads();
    }
    if (tid == 0) res[0] = 0.25 * (s_lo + s_hi);
}

// Pass 3, one thread per variable: p_i = 1 - u_i^T (as -expm1(T ln u_i),
// accurate for small p), 1 where u_i = 0.  Nothing is written if the fit failed.
__global__ void __launch_bounds__(256) fit_p_kernel(int M, const double* __restrict__ res, double* __restrict__ p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const double T = res[1];
    if (!(res[2] > 0.0) || !(T > 0.0)) return;
    const double ui = p[i];
    p[i] = ui > 0.0 ? -expm1(T * log(ui)) : 1.0;
}

cudaError_t launch_ig_lim_cdf(const float* ig, int M, int df, double* p_values, cudaStream_t st) {
    fit_cdf_kernel<<<(M + 255) / 256, 256, 0, st>>>(ig, M, df, p_values);
    return cudaGetLastError();
}

cudaError_t launch_ig_lim_fit(const double* p_values, int M, int df, const uint8_t* mask, double alpha, double* res,
                              cudaStream_t st) {
    fit_t_kernel<<<1, 256, 0, st>>>(p_values, M, df, mask, alpha, res);
    return cudaGetLastError();
}

cudaError_t launch_ig_lim_p(int M, const double* res, double* p_values, cudaStream_t st) {
    fit_p_kernel<<<(M + 255) / 256, 256, 0, st>>>(M, res, p_values);
    return cudaGetLastError();
}

}  // namespace mdfs
