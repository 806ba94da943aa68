// Input preparation on the device: the Matern covariance of Eq. 2 (Section III-D) written
// straight into the lower tile layout, and the per-tile sums of squares behind the
// precision criterion of Section IV-C.  Both are HBM-bound (8 bytes written or read per
// element).
#include "tc_internal.h"

// Device-only unless a host test harness asks for both sides.
#ifndef MATERN_FN
#define MATERN_FN __device__
#endif

namespace tc {

// ---------------------------------------------------------------- K_nu for any nu > 0
// Eq. 2 for a smoothness that is not a half integer needs the modified Bessel function of the
// second kind.  With nu = mu + m, |mu| <= 1/2, K_mu and K_{mu+1} come from
//   x <= 2: Temme's power series (N. M. Temme, J. Comput. Phys. 19 (1975) 324-337);
//   x >  2: Temme's normalising sum  sum_k C_k U_k = (2x)^-(mu+1/2)  over the confluent
//           functions U_k = U(mu+1/2+k, 2mu+1, 2x), whose ratios are the minimal solution of
//           their three-term recurrence, taken by Miller's backward recurrence (Gautschi,
//           SIAM Rev. 9 (1967) 24-82);
// and K_{mu+j+1} = K_{mu+j-1} + 2(mu+j)/x K_{mu+j} (stable upwards) reaches nu.

// g1 = (1/Gamma(1-mu) - 1/Gamma(1+mu)) / (2mu) and g2 = (1/Gamma(1-mu) + 1/Gamma(1+mu)) / 2
// for |mu| <= 1/2, from the odd and even parts of the Taylor series of 1/Gamma(1+z) at 0
// (Abramowitz & Stegun 6.1.34 lists it as the series of 1/Gamma(z), shifted by one power).
// Twenty-two terms leave a tail below 1e-18 at |z| = 1/2, and mu -> 0 needs no limit.
MATERN_FN inline void temme_gammas(double mu, double &g1, double &g2) {
    const double m2 = mu * mu;
    g1 = -(5.7721566490153286e-1 + m2 * (-4.2002635034095236e-2 + m2 * (-4.2197734555544337e-2 +
           m2 * (7.2189432466630995e-3 + m2 * (-2.1524167411495097e-4 + m2 * (-2.0134854780788239e-5 +
           m2 * (1.1330272319816959e-6 + m2 * (6.1160951044814158e-9 + m2 * (-1.1812745704870201e-9 +
           m2 * (7.7822634399050713e-12 + m2 * 5.1003702874544760e-13))))))))));
    g2 = 1.0 + m2 * (-6.5587807152025388e-1 + m2 * (1.6653861138229149e-1 + m2 * (-9.6219715278769736e-3 +
         m2 * (-1.1651675918590651e-3 + m2 * (1.2805028238811619e-4 + m2 * (-1.2504934821426707e-6 +
         m2 * (-2.0563384169776071e-7 + m2 * (5.0020076444692229e-9 + m2 * (1.0434267116911005e-10 +
         m2 * -3.6968056186422057e-12)))))))));
}

// K_mu(x), K_{mu+1}(x) for |mu| <= 1/2, 0 < x <= 2.  With c_k = (x^2/4)^k / k!:
//   K_mu = sum c_k f_k,  K_{mu+1} = (2/x) sum c_k (p_k - k f_k),
//   f_k = (k f_{k-1} + p_{k-1} + q_{k-1}) / (k^2 - mu^2),  p_k = p_{k-1}/(k-mu),  q_k = q_{k-1}/(k+mu),
//   p_0 = (x/2)^-mu Gamma(1+mu) / 2,  q_0 = (x/2)^mu Gamma(1-mu) / 2,
//   f_0 = (mu pi / sin(mu pi)) (cosh(s) g1 + sinh(s)/s ln(2/x) g2),  s = mu ln(2/x).
// The terms fall at least like 1/(k!)^2; at x = 2 fifteen reach the double rounding unit.
MATERN_FN inline void bessel_k_series(double mu, double x, double g1, double g2, double &k0, double &k1) {
    const double lg = log(2.0 / x);
    const double s = mu * lg;
    const double fac = (mu == 0.0) ? 1.0 : (3.141592653589793 * mu) / sin(3.141592653589793 * mu);
    const double shs = (s == 0.0) ? 1.0 : sinh(s) / s;
    double f = fac * (cosh(s) * g1 + shs * lg * g2);
    const double e = exp(s);
    double p = 0.5 * e / (g2 - mu * g1);       // 1/Gamma(1+mu) = g2 - mu g1
    double q = 0.5 / (e * (g2 + mu * g1));     // 1/Gamma(1-mu) = g2 + mu g1
    const double y = 0.25 * x * x;
    double c = 1.0, s0 = f, s1 = p;
    for (int k = 1; k <= 60; ++k) {
        const double dk = (double)k;
        f = (dk * f + p + q) / (dk * dk - mu * mu);
        p /= dk - mu;
        q /= dk + mu;
        c *= y / dk;
        const double t0 = c * f, t1 = c * (p - dk * f);
        s0 += t0;
        s1 += t1;
        if (fabs(t0) < 1e-17 * fabs(s0) && fabs(t1) < 1e-17 * fabs(s1)) break;
    }
    k0 = s0;
    k1 = s1 * (2.0 / x);
}

// e^x K_mu(x), e^x K_{mu+1}(x) for |mu| <= 1/2, x > 2.  U_k satisfies
//   U_{k-1} - 2(k+x) U_k + a_k U_{k+1} = 0,  a_k = (k+1/2)^2 - mu^2,
// so r_k = U_k / U_{k-1} = 1 / (2(k+x) - a_k r_{k+1}), started at r_{K+1} = 0.  The sum
// S = sum C_k U_k / U_0 with C_k / C_{k-1} = a_{k-1} / k is nested alongside,
//   T_{k-1} = 1 + (a_{k-1}/k) r_k T_k,  S = T_0,
// and then e^x K_mu = sqrt(pi / 2x) / S,  K_{mu+1} / K_mu = (mu + 1/2 + x + (mu^2 - 1/4) r_1) / x.
// K = 6 + 150/x terms keep the truncation below the rounding unit for every x > 2.
MATERN_FN inline void bessel_k_ratio(double mu, double x, double &k0, double &k1) {
    const int K = 6 + (int)ceil(150.0 / x);
    const double m2 = mu * mu;
    double r = 0.0, T = 1.0;
    for (int k = K; k >= 1; --k) {
        const double dk = (double)k;
        const double ak = (dk + 0.5) * (dk + 0.5) - m2;
        const double am = (dk - 0.5) * (dk - 0.5) - m2;
        r = 1.0 / (2.0 * (dk + x) - ak * r);
        T = 1.0 + (am / dk) * r * T;
    }
    k0 = sqrt(3.141592653589793 / (2.0 * x)) / T;
    k1 = k0 * (mu + 0.5 + x + (m2 - 0.25) * r) / x;
}

// Per-call constants of the Matern correlation for smoothness nu: m = floor(nu + 1/2),
// mu = nu - m, Temme's g1, g2 and pre = 2^(1-nu) / Gamma(nu), with
// Gamma(nu) = Gamma(1+mu) (mu+1) ... (mu+m-1), or Gamma(1+mu)/mu when m = 0.
struct MaternNu {
    double nu, mu, g1, g2, pre;
    int m;
};

MATERN_FN inline MaternNu matern_nu(double nu) {
    MaternNu c;
    c.nu = nu;
    c.m = (int)floor(nu + 0.5);
    c.mu = nu - c.m;
    temme_gammas(c.mu, c.g1, c.g2);
    double gam = 1.0 / (c.g2 - c.mu * c.g1);
    if (c.m == 0) gam /= c.mu;
    for (int j = 1; j < c.m; ++j) gam *= c.mu + j;
    c.pre = exp2(1.0 - nu) / gam;
    return c;
}

// 2^(1-nu)/Gamma(nu) x^nu K_nu(x), the Matern correlation of Eq. 2 at x = h/a >= 0 (1 at 0).
// Below x <= 2 with nu ln(2/x) > 600 the value is 1 to far below the rounding unit (the
// deviation is O(x^2) for nu > 1 and O(x^(2 nu)) otherwise), and K_nu would overflow; above
// x = 1450, x^nu e^-x underflows for every nu <= 16.
MATERN_FN inline double matern_corr(const MaternNu &c, double x) {
    if (x == 0.0) return 1.0;
    if (x > 1450.0) return 0.0;
    const bool small = x <= 2.0;
    if (small && c.nu * log(2.0 / x) > 600.0) return 1.0;
    double k0, k1;
    if (small) bessel_k_series(c.mu, x, c.g1, c.g2, k0, k1);
    else bessel_k_ratio(c.mu, x, k0, k1);
    double kn = k0;
    if (c.m > 0) {
        for (int j = 1; j < c.m; ++j) {
            const double k2 = k0 + (2.0 * (c.mu + j) / x) * k1;
            k0 = k1;
            k1 = k2;
        }
        kn = k1;
    }
    if (small) return c.pre * (pow(x, c.nu) * kn);
    const double h = exp(-0.5 * x);               // e^-x in two halves: x^nu e^-x/2 stays finite
    return c.pre * ((pow(x, c.nu) * h) * (kn * h));
}

// One CTA row (blockIdx.y) per tile; the x-dimension strides over the tile's b*b
// elements in column-major order so consecutive threads write consecutive rows.
// The arithmetic is spelled with explicit round-to-nearest intrinsics so that no
// multiply-add is contracted: h and x = h/a are then bit-identical to a plain IEEE
// evaluation, and only exp() may differ (by its last bit) from another library.
__global__ void __launch_bounds__(256)
k_matern(double *A, int64_t n, int b, const double *__restrict__ pts, double sigma2, double a,
         int nu2, double nu, double nugget) {
    const int t = blockIdx.y;
    const MaternNu cn = matern_nu(nu2 ? 1.0 : nu);  // only read on the general path (nu2 == 0)
    // tile (i, j) from the packed index t = i(i+1)/2 + j
    int i = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((int64_t)i * (i + 1) / 2 > t) --i;
    while ((int64_t)(i + 1) * (i + 2) / 2 <= t) ++i;
    const int j = t - i * (i + 1) / 2;
    double *T = A + (int64_t)t * b * b;
    const int64_t bb = (int64_t)b * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bb; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % b), c = (int)(e / b);
        const int64_t gi = (int64_t)i * b + r, gj = (int64_t)j * b + c;
        double v;
        if (gi >= n || gj >= n) {
            v = (gi == gj) ? 1.0 : 0.0;
        } else {
            const double dx = __dsub_rn(pts[2 * gi], pts[2 * gj]);
            const double dy = __dsub_rn(pts[2 * gi + 1], pts[2 * gj + 1]);
            const double h = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
            const double x = __ddiv_rn(h, a);
            const double ex = nu2 ? exp(-x) : 0.0;
            double f;
            if (nu2 == 1) f = ex;                                               // nu = 1/2
            else if (nu2 == 3) f = __dmul_rn(__dadd_rn(1.0, x), ex);           // nu = 3/2
            else if (nu2 == 5) f = __dmul_rn(__dadd_rn(__dadd_rn(1.0, x), __ddiv_rn(__dmul_rn(x, x), 3.0)), ex);  // 5/2
            else f = matern_corr(cn, x);                                       // any other nu
            v = __dmul_rn(sigma2, f);
            if (gi == gj) v = __dadd_rn(v, nugget);
        }
        T[e] = v;
    }
}

// Sum of squares of the valid (row, column < n) elements of every tile; one CTA per tile,
// fixed reduction order.
// Sum of squares of tile t0 + blockIdx.x (global packed index; the tile itself at
// A + blockIdx.x b^2), padding excluded.
__global__ void __launch_bounds__(256) k_tile_sumsq(const double *A, int b, int64_t n, double *out, int t0) {
    __shared__ double red[256];
    const int t = t0 + (int)blockIdx.x;
    int i = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((int64_t)i * (i + 1) / 2 > t) --i;
    while ((int64_t)(i + 1) * (i + 2) / 2 <= t) ++i;
    const int j = t - i * (i + 1) / 2;
    const double *T = A + (int64_t)blockIdx.x * b * b;
    const int64_t bb = (int64_t)b * b;
    const int nvr = (int)((n - (int64_t)i * b) < b ? (n - (int64_t)i * b) : b);
    const int nvc = (int)((n - (int64_t)j * b) < b ? (n - (int64_t)j * b) : b);
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < bb; e += 256) {
        const int r = (int)(e % b), c = (int)(e / b);
        if (r < nvr && c < nvc) {
            const double v = T[e];
            s = fma(v, v, s);
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[t] = red[0];
}

void launch_matern(double *A, int64_t n, int b, int nt, const double *pts, double sigma2, double a,
                   int nu2, double nu, double nugget, cudaStream_t s) {
    const int T = nt * (nt + 1) / 2;
    int gx = (int)(((int64_t)b * b + 255) / 256);
    if (gx > 64) gx = 64;
    k_matern<<<dim3(gx, T), 256, 0, s>>>(A, n, b, pts, sigma2, a, nu2, nu, nugget);
}

void launch_tile_sumsq(const double *A, int nt, int b, int64_t n, double *out, cudaStream_t s) {
    const int T = nt * (nt + 1) / 2;
    k_tile_sumsq<<<T, 256, 0, s>>>(A, b, n, out, 0);
}
void launch_tile_sumsq_range(const double *A_first, int t0, int count, int b, int64_t n, double *out, cudaStream_t s) {
    if (count > 0) k_tile_sumsq<<<count, 256, 0, s>>>(A_first, b, n, out, t0);
}

}  // namespace tc
