// Input preparation on the device: the Matern covariance of Eq. 2 (Section III-D) written
// straight into the lower tile layout, and the per-tile sums of squares behind the
// precision criterion of Section IV-C.  Both are HBM-bound (8 bytes written or read per
// element).
#include "tc_internal.h"

namespace tc {

// One CTA row (blockIdx.y) per tile; the x-dimension strides over the tile's b*b
// elements in column-major order so consecutive threads write consecutive rows.
// The arithmetic is spelled with explicit round-to-nearest intrinsics so that no
// multiply-add is contracted: h and x = h/a are then bit-identical to a plain IEEE
// evaluation, and only exp() may differ (by its last bit) from another library.
__global__ void __launch_bounds__(256)
k_matern(double *A, int64_t n, int b, const double *__restrict__ pts, double sigma2, double a,
         int nu2, double nugget) {
    const int t = blockIdx.y;
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
            const double ex = exp(-x);
            double f;
            if (nu2 == 1) f = ex;                                               // nu = 1/2
            else if (nu2 == 3) f = __dmul_rn(__dadd_rn(1.0, x), ex);           // nu = 3/2
            else f = __dmul_rn(__dadd_rn(__dadd_rn(1.0, x), __ddiv_rn(__dmul_rn(x, x), 3.0)), ex);  // 5/2
            v = __dmul_rn(sigma2, f);
            if (gi == gj) v = __dadd_rn(v, nugget);
        }
        T[e] = v;
    }
}

// Sum of squares of the valid (row, column < n) elements of every tile; one CTA per tile,
// fixed reduction order.
__global__ void __launch_bounds__(256) k_tile_sumsq(const double *A, int b, int64_t n, double *out) {
    __shared__ double red[256];
    const int t = blockIdx.x;
    int i = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((int64_t)i * (i + 1) / 2 > t) --i;
    while ((int64_t)(i + 1) * (i + 2) / 2 <= t) ++i;
    const int j = t - i * (i + 1) / 2;
    const double *T = A + (int64_t)t * b * b;
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
                   int nu2, double nugget, cudaStream_t s) {
    const int T = nt * (nt + 1) / 2;
    int gx = (int)(((int64_t)b * b + 255) / 256);
    if (gx > 64) gx = 64;
    k_matern<<<dim3(gx, T), 256, 0, s>>>(A, n, b, pts, sigma2, a, nu2, nugget);
}

void launch_tile_sumsq(const double *A, int nt, int b, int64_t n, double *out, cudaStream_t s) {
    const int T = nt * (nt + 1) / 2;
    k_tile_sumsq<<<T, 256, 0, s>>>(A, b, n, out);
}

}  // namespace tc
