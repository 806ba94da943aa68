// FP64 kernels of the tile Cholesky: SYRK/GEMM updates (Algorithm 1's inner n-loop,
// Section III-A), the diagonal POTRF, the panel TRSM, and the substitution / residual
// kernels of the solve.  GB300's FP64 pipe issues about two DFMA per clock per SM
// (~1.05 TFLOP/s for the chip), so these kernels are DFMA-bound by a wide margin: the
// 64 x 64 register-blocked tile below keeps the pipe saturated from one CTA per SM.
#include "tc_internal.h"

#include <cmath>

namespace tc {

// Right-hand-side kernels are compiled for 1, 4 and 16 columns: GB300 issues a DFMA for every
// unrolled column even when its predicate is off, and FP64 is its scarce pipe.
#define NQ_DISPATCH(nrhs, kern, grid, block, smem, stream, ...)                             \
    do {                                                                                  \
        if ((nrhs) <= 1) kern<1><<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);      \
        else if ((nrhs) <= 4) kern<4><<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__); \
        else kern<16><<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                \
    } while (0)


// acc (rows tx + 16 i, columns ty + 16 j of a 64 x 64 block) += X[:, k0:k1] Y[:, k0:k1]^T.
// X and Y point at the block's first row/column; column l of each is at l * ld.
__device__ __forceinline__ void dgemm_block(double (&acc)[4][4], const double *__restrict__ X,
                                            const double *__restrict__ Y, int ld, int k0, int k1,
                                            double (*Xs)[64], double (*Ys)[64]) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int k = k0; k < k1; k += 16) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + 256 * e, l = idx >> 6, r = idx & 63;
            const bool ok = (k + l) < k1;
            Xs[l][r] = ok ? X[(int64_t)(k + l) * ld + r] : 0.0;
            Ys[l][r] = ok ? Y[(int64_t)(k + l) * ld + r] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < 16; ++l) {
            double a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Xs[l][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Ys[l][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ bool failed(const int *status) {
    return status && *(volatile const int *)status != 0;
}

// ----------------------------------------------------------------------------- updates
__global__ void __launch_bounds__(256, 2)
k_dgemm_update(const DJob *__restrict__ jobs, const DItem *__restrict__ items, int ld,
               double *__restrict__ partials, const int *status) {
    __shared__ double Xs[16][64], Ys[16][64];
    const DItem it = items[blockIdx.x];
    const DJob jb = jobs[it.job];
    if (failed(status) || failed(jb.status)) return;
    const int i0 = it.bi * 64, j0 = it.bj * 64;
    double acc[4][4] = {};
    dgemm_block(acc, jb.X + i0, jb.Y + j0, ld, it.k0, it.k1, Xs, Ys);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    if (it.part < 0) {
        double *C = jb.C + (int64_t)j0 * ld + i0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) C[(int64_t)(ty + 16 * j) * ld + tx + 16 * i] -= acc[i][j];
    } else {
        double *P = partials + (int64_t)it.part * 4096;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) P[(ty + 16 * j) * 64 + tx + 16 * i] = acc[i][j];
    }
}

__global__ void __launch_bounds__(256)
k_dgemm_reduce(const DRed *__restrict__ reds, int ld, const double *__restrict__ partials,
               const int *status) {
    if (failed(status)) return;
    const DRed r = reds[blockIdx.x];
    for (int e = 0; e < 16; ++e) {
        const int idx = threadIdx.x + 256 * e, rr = idx & 63, cc = idx >> 6;
        double s = 0.0;
        for (int p = 0; p < r.nparts; ++p) s += partials[(int64_t)(r.part0 + p) * 4096 + cc * 64 + rr];
        r.C[(int64_t)cc * ld + rr] -= s;
    }
}

// ------------------------------------------------------------------------------- POTRF
// Factor the 64 x 64 lower block at D in place (right-looking in shared memory).  A
// non-positive pivot records the 1-based global column in *status and stops.  Each step
// touches only the trailing triangle (threads: row r = tid % 64, columns c = j+1+tid/64 step 4)
// and scales the column by the pivot's reciprocal: GB300 retires about 2 FP64 operations per
// clock per SM, so every skipped multiply-add and division counts.
__device__ __forceinline__ void potrf64_body(double *D, int ld, int col0, int *status) {
    __shared__ double S[64][65];
    __shared__ int fail;
    __shared__ double rp;
    const int tid = threadIdx.x, r = tid & 63, cg = tid >> 6;
    for (int idx = tid; idx < 4096; idx += 256) {
        const int rr = idx & 63, c = idx >> 6;
        S[rr][c] = (rr >= c) ? D[(int64_t)c * ld + rr] : 0.0;
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < 64; ++j) {
        if (tid == 0) {
            const double d = S[j][j];
            if (!(d > 0.0)) {
                fail = j + 1;
            } else {
                const double sd = sqrt(d);
                S[j][j] = sd;
                rp = 1.0 / sd;
            }
        }
        __syncthreads();
        if (fail) break;
        if (tid > j && tid < 64) S[tid][j] *= rp;
        __syncthreads();
        const double lrj = S[r][j];
        for (int c = j + 1 + cg; c < 64; c += 4)
            if (r >= c) S[r][c] = fma(-lrj, S[c][j], S[r][c]);
        __syncthreads();
    }
    if (fail) {
        if (tid == 0) atomicCAS(status, 0, col0 + fail);
        return;
    }
    for (int idx = tid; idx < 4096; idx += 256) {
        const int rr = idx & 63, c = idx >> 6;
        if (rr >= c) D[(int64_t)c * ld + rr] = S[rr][c];
    }
}
__global__ void __launch_bounds__(256) k_potrf_block(double *D, int ld, int col0, int *status) {
    if (failed(status)) return;
    potrf64_body(D, ld, col0, status);
}

// Right-side solve of a strip of ROWS rows held in shared memory: X L^T = S in place, L the
// 64 x 64 lower block in Ls, rinv[j] = 1 / L[j][j].  Column j: X[r][j] = S[r][j] / L[j][j], then
// S[r][c] -= X[r][j] L[c][j] for c > j (threads: row tid % ROWS, columns step 256 / ROWS).
template <int ROWS>
__device__ __forceinline__ void strip_solve(double (*Ss)[65], double (*Ls)[65], const double *rinv) {
    const int tid = threadIdx.x, r = tid % ROWS, cg = tid / ROWS;
    constexpr int CS = 256 / ROWS;
    for (int j = 0; j < 64; ++j) {
        if (tid < ROWS) Ss[tid][j] *= rinv[j];
        __syncthreads();
        const double xrj = Ss[r][j];
        for (int c = j + 1 + cg; c < 64; c += CS) Ss[r][c] = fma(-xrj, Ls[c][j], Ss[r][c]);
        __syncthreads();
    }
}

// POTRF panel: rows below the factored 64-block within the diagonal tile, 16-row strips
// (the solve is bound by one SM's FP64 rate, so more, smaller strips finish sooner).
constexpr int PANEL_ROWS = 16;
__device__ __forceinline__ void panel_body(double *Pb, const double *L, int ld) {
    __shared__ double Ls[64][65], Ss[PANEL_ROWS][65], rinv[64];
    const int tid = threadIdx.x;
    for (int idx = tid; idx < 4096; idx += 256) {
        const int r = idx & 63, c = idx >> 6;
        Ls[r][c] = (r >= c) ? L[(int64_t)c * ld + r] : 0.0;
    }
    for (int idx = tid; idx < PANEL_ROWS * 64; idx += 256) {
        const int r = idx % PANEL_ROWS, c = idx / PANEL_ROWS;
        Ss[r][c] = Pb[(int64_t)c * ld + r];
    }
    __syncthreads();
    if (tid < 64) rinv[tid] = 1.0 / Ls[tid][tid];
    __syncthreads();
    strip_solve<PANEL_ROWS>(Ss, Ls, rinv);
    for (int idx = tid; idx < PANEL_ROWS * 64; idx += 256) {
        const int r = idx % PANEL_ROWS, c = idx / PANEL_ROWS;
        Pb[(int64_t)c * ld + r] = Ss[r][c];
    }
}
__global__ void __launch_bounds__(256) k_trsm_rows(double *P, const double *L, int ld, const int *status) {
    if (failed(status)) return;
    panel_body(P + blockIdx.x * PANEL_ROWS, L, ld);
}

// Column TRSM (Algorithm 1: A_mk = A_mk L_kk^{-T}): one CTA per 64-row strip of a tile,
// left-looking over the 64-column blocks of L_kk.
__global__ void __launch_bounds__(256, 2)
k_trsm_strips(const TStrip *__restrict__ strips, int ld, int b, const int *status) {
    if (failed(status) || failed(strips[blockIdx.x].status)) return;
    extern __shared__ double smem[];
    double(*Xs)[64] = reinterpret_cast<double(*)[64]>(smem);
    double(*Ys)[64] = reinterpret_cast<double(*)[64]>(smem + 16 * 64);
    double(*Ls)[65] = reinterpret_cast<double(*)[65]>(smem + 32 * 64);
    double(*Ss)[65] = reinterpret_cast<double(*)[65]>(smem + 32 * 64 + 64 * 65);
    double *rinv = smem + 32 * 64 + 2 * 64 * 65;
    const TStrip st = strips[blockIdx.x];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double *X = st.C + st.r0;
    for (int jb = 0; jb < b / 64; ++jb) {
        double acc[4][4] = {};
        dgemm_block(acc, X, st.L + jb * 64, ld, 0, jb * 64, Xs, Ys);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                Ss[tx + 16 * i][ty + 16 * j] = X[(int64_t)(jb * 64 + ty + 16 * j) * ld + tx + 16 * i] - acc[i][j];
        for (int idx = tid; idx < 4096; idx += 256) {
            const int r = idx & 63, c = idx >> 6;
            Ls[r][c] = (r >= c) ? st.L[(int64_t)(jb * 64 + c) * ld + jb * 64 + r] : 0.0;
        }
        __syncthreads();
        if (tid < 64) rinv[tid] = 1.0 / Ls[tid][tid];
        __syncthreads();
        strip_solve<64>(Ss, Ls, rinv);
        for (int idx = tid; idx < 4096; idx += 256) {
            const int r = idx & 63, c = idx >> 6;
            X[(int64_t)(jb * 64 + c) * ld + r] = Ss[r][c];
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------- tile bookkeeping
__device__ __forceinline__ double *diag_tile(double *W, int t, int b) {
    return W + ((int64_t)t * (t + 1) / 2 + t) * (int64_t)b * b;
}

// log|A| = 2 sum log L_ii over the n valid diagonal entries, fixed summation order.
__global__ void __launch_bounds__(1024) k_logdet(const double *W, int b, int64_t n, double *out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int64_t g = threadIdx.x; g < n; g += 1024) {
        const int t = (int)(g / b), r = (int)(g % b);
        const double *D = W + ((int64_t)t * (t + 1) / 2 + t) * (int64_t)b * b;
        s += log(D[(int64_t)r * b + r]);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = 2.0 * red[0];
}

// Padding of the last tile row: rows/columns >= n become those of the identity.
__global__ void k_fix_padding(double *W, int nt, int b, int64_t n) {
    const int j = blockIdx.y;                       // tile column in the last tile row
    const int i = nt - 1;
    const int nv = (int)(n - (int64_t)i * b);      // valid rows of the last tile row
    double *T = W + ((int64_t)i * (i + 1) / 2 + j) * (int64_t)b * b;
    const int64_t bb = (int64_t)b * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bb; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % b), c = (int)(e / b);
        if (j < i) {
            if (r >= nv) T[e] = 0.0;
        } else if (r >= nv || c >= nv) {
            T[e] = (r == c) ? 1.0 : 0.0;
        }
    }
}

// Export clean-up: strictly upper parts of diagonal tiles and all padding become 0.
__global__ void k_zero_upper_diag(double *W, int nt, int b, int64_t n) {
    const int t = blockIdx.y;
    const int64_t bb = (int64_t)b * b;
    const int nv_last = (int)(n - (int64_t)(nt - 1) * b);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bb; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % b), c = (int)(e / b);
        if (t < nt) {  // diagonal tile t
            double *D = W + ((int64_t)t * (t + 1) / 2 + t) * bb;
            const bool pad = (t == nt - 1) && (r >= nv_last || c >= nv_last);
            if (c > r || pad) D[e] = 0.0;
        } else {       // off-diagonal tile (nt-1, j) of the last tile row, j = t - nt
            const int j = t - nt, i = nt - 1;
            double *T = W + ((int64_t)i * (i + 1) / 2 + j) * bb;
            if (r >= nv_last) T[e] = 0.0;
        }
    }
}

// Sum the four per-part accumulators of each row in a fixed order and subtract them from
// R[q * ldr + g0 + r] (rows r of a 64-row chunk, RHS q < nrhs).
template <int NQ>
__device__ __forceinline__ void part_reduce_sub(double (*red)[17], const double (&acc)[NQ], int nrhs,
                                                double *R, int64_t ldr, int64_t g0) {
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    for (int p = 0; p < 4; ++p) {
        __syncthreads();
        if (part == p)
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) red[rr][q] = (p == 0) ? acc[q] : red[rr][q] + acc[q];
    }
    __syncthreads();
    for (int e = tid; e < 64 * nrhs; e += 256) {
        const int r = e % 64, q = e / 64;
        R[q * ldr + g0 + r] -= red[r][q];
    }
}

// -------------------------------------------------------------------------------- solves
// One warp solves the 64 x 64 triangle held in S (S[r][c] = L[r][c], r >= c) against the 64
// values in blk: forward (L x = blk) or backward (L^T x = blk).  Each lane owns rows lane and
// lane + 32; the solved value travels by shuffle, so the 64 steps need no block barrier, and
// the pivots' reciprocals are formed up front (x * (1/d): one extra rounding, off the chain).
__device__ __forceinline__ void warp_tri64(double (*S)[65], double *blk, bool forward) {
    const int lane = threadIdx.x & 31;
    double x0 = blk[lane], x1 = blk[lane + 32];
    const double r0 = 1.0 / S[lane][lane], r1 = 1.0 / S[lane + 32][lane + 32];
    if (forward) {
        for (int j = 0; j < 32; ++j) {
            if (lane == j) x0 *= r0;
            const double xj = __shfl_sync(0xffffffffu, x0, j);
            if (lane > j) x0 = fma(-S[lane][j], xj, x0);
            x1 = fma(-S[lane + 32][j], xj, x1);
        }
        for (int j = 0; j < 32; ++j) {
            if (lane == j) x1 *= r1;
            const double xj = __shfl_sync(0xffffffffu, x1, j);
            if (lane > j) x1 = fma(-S[lane + 32][32 + j], xj, x1);
        }
    } else {
        for (int j = 31; j >= 0; --j) {
            if (lane == j) x1 *= r1;
            const double xj = __shfl_sync(0xffffffffu, x1, j);
            if (lane < j) x1 = fma(-S[32 + j][lane + 32], xj, x1);
            x0 = fma(-S[32 + j][lane], xj, x0);
        }
        for (int j = 31; j >= 0; --j) {
            if (lane == j) x0 *= r0;
            const double xj = __shfl_sync(0xffffffffu, x0, j);
            if (lane < j) x0 = fma(-S[j][lane], xj, x0);
        }
    }
    blk[lane] = x0;
    blk[lane + 32] = x1;
}

// Forward substitution with one diagonal tile, one right-hand side r (in place): per 64-row
// block, the product with the solved part (256 threads, 4 partial sums per row, fixed order)
// and the warp solve of the diagonal block.
// T: the right-hand side's storage type (double, or float for the FP32 correction solves of a
// refined batched solve); the arithmetic is FP64 either way.
template <typename T>
__device__ __forceinline__ void fwd_diag_body(const double *L, int ld, int b, T *r) {
    __shared__ double red[4][64];
    __shared__ double blk[64];
    __shared__ double S[64][65];
    T *z = r;                            // solved in place (block barriers order the accesses)
    const int tid = threadIdx.x;
    const int rr = tid & 63, part = tid >> 6;
    for (int jb = 0; jb < b / 64; ++jb) {
        double acc = 0.0;
        for (int l = part; l < jb * 64; l += 4) acc = fma(L[(int64_t)l * ld + jb * 64 + rr], (double)z[l], acc);
        red[part][rr] = acc;
        for (int idx = tid; idx < 4096; idx += 256) {
            const int lr = idx & 63, lc = idx >> 6;
            S[lr][lc] = (lr >= lc) ? L[(int64_t)(jb * 64 + lc) * ld + jb * 64 + lr] : 0.0;
        }
        __syncthreads();
        if (tid < 64) blk[tid] = (double)z[jb * 64 + tid] - (red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid]);
        __syncthreads();
        if (tid < 32) warp_tri64(S, blk, true);
        __syncthreads();
        if (tid < 64) z[jb * 64 + tid] = (T)blk[tid];
        __syncthreads();
    }
}

// Back substitution with one diagonal tile: L_jj^T x = z, one right-hand side (in place).
template <typename T>
__device__ __forceinline__ void bwd_diag_body(const double *L, int ld, int b, T *x) {
    __shared__ double S[64][65];
    __shared__ double red[4][64];
    __shared__ double blk[64];
    const int tid = threadIdx.x;
    const int rr = tid & 63, part = tid >> 6;
    for (int jb = b / 64 - 1; jb >= 0; --jb) {
        // acc[r] = sum_{l >= (jb+1)*64} L[l][jb*64 + r] x[l]: rows of the tile's column block,
        // read along l (column-major L: contiguous in l for a fixed column)
        double acc = 0.0;
        const double *Lc = L + (int64_t)(jb * 64 + rr) * ld;
        for (int l = (jb + 1) * 64 + part; l < b; l += 4) acc = fma(Lc[l], (double)x[l], acc);
        red[part][rr] = acc;
        for (int idx = tid; idx < 4096; idx += 256) {
            const int lr = idx & 63, lc = idx >> 6;
            S[lr][lc] = (lr >= lc) ? L[(int64_t)(jb * 64 + lc) * ld + jb * 64 + lr] : 0.0;
        }
        __syncthreads();
        if (tid < 64) blk[tid] = (double)x[jb * 64 + tid] - (red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid]);
        __syncthreads();
        if (tid < 32) warp_tri64(S, blk, false);
        __syncthreads();
        if (tid < 64) x[jb * 64 + tid] = (T)blk[tid];
        __syncthreads();
    }
}

// Inside a diagonal tile, after a sub-block solve: R[r] -= sum_c L[c ld + r] Z[c] for the
// `rows` rows below the sub-block (one CTA per 64 rows, four partial sums per row).
template <int NQ>
__global__ void __launch_bounds__(256)
k_gemv_below(const double *L, int ld, int cols, const double *Z, double *R, int64_t ldr, int nrhs) {
    __shared__ double red[64][17];
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6, r0 = blockIdx.x * 64;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int c = part; c < cols; c += 4) {
        const double l = L[(int64_t)c * ld + r0 + rr];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (q < nrhs) acc[q] = fma(l, Z[q * ldr + c], acc[q]);
    }
    part_reduce_sub(red, acc, nrhs, R, ldr, r0);
}

// The back-substitution counterpart: R[i] -= sum_c L[i ld + c] X[c] for the rows above the
// sub-block (L points at the sub-block's first row, column 0; a warp per output row, lanes
// along c, so each row of L^T is read contiguously).
template <int NQ>
__global__ void __launch_bounds__(256)
k_gemv_above(const double *L, int ld, int cols, const double *X, double *R, int64_t ldr, int nrhs) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = blockIdx.x * 64 + warp; i < blockIdx.x * 64 + 64; i += 8) {
        double acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
        for (int c = lane; c < cols; c += 32) {
            const double l = L[(int64_t)i * ld + c];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) acc[q] = fma(l, X[q * ldr + c], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double v = acc[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && q < nrhs) R[q * ldr + i] -= v;
        }
    }
}

// Forward substitution with the s x s lower triangle at L (leading dimension ld): L z = r for
// each RHS column (one CTA each).
__global__ void __launch_bounds__(256) k_fwd_diag(const double *L, int ld, int b, double *R, int64_t ldr) {
    fwd_diag_body(L, ld, b, R + blockIdx.x * ldr);
}

// r_i -= L_ij z_j for every tile row i > j; one CTA per 64-row chunk of a tile row.
template <int NQ>
__global__ void __launch_bounds__(256)
k_fwd_update(const double *W, int b, int j, double *R, int64_t ldr, int nrhs) {
    __shared__ double zs[128][16];
    __shared__ double red[64][17];
    const int chunks = b / 64;
    const int i = j + 1 + blockIdx.x / chunks, r0 = (blockIdx.x % chunks) * 64;
    const double *L = W + ((int64_t)i * (i + 1) / 2 + j) * (int64_t)b * b;
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int c0 = 0; c0 < b; c0 += 128) {
        __syncthreads();
        for (int e = tid; e < 128 * nrhs; e += 256) {
            const int c = e % 128, q = e / 128;
            zs[c][q] = R[q * ldr + (int64_t)j * b + c0 + c];
        }
        __syncthreads();
        for (int c = part; c < 128; c += 4) {
            const double l = L[(int64_t)(c0 + c) * b + r0 + rr];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) acc[q] = fma(l, zs[c][q], acc[q]);
        }
    }
    part_reduce_sub(red, acc, nrhs, R, ldr, (int64_t)i * b + r0);
}

// Back substitution with the s x s lower triangle at L: L^T x = z for each RHS column.
__global__ void __launch_bounds__(256) k_bwd_diag(const double *L, int ld, int b, double *R, int64_t ldr) {
    bwd_diag_body(L, ld, b, R + blockIdx.x * ldr);
}

// z_i -= L_ji^T x_j for every tile row i < j; one CTA per 64-row chunk of tile row i.
template <int NQ>
__global__ void __launch_bounds__(256)
k_bwd_update(const double *W, int b, int j, double *R, int64_t ldr, int nrhs) {
    __shared__ double xs[64][16];
    __shared__ double S[64][65];
    const int chunks = b / 64;
    const int i = blockIdx.x / chunks, r0 = (blockIdx.x % chunks) * 64;
    const double *L = W + ((int64_t)j * (j + 1) / 2 + i) * (int64_t)b * b;   // tile (j, i)
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int c0 = 0; c0 < b; c0 += 64) {
        __syncthreads();
        for (int idx = tid; idx < 4096; idx += 256) {
            const int c = idx & 63, r = idx >> 6;
            S[r][c] = L[(int64_t)(r0 + r) * b + c0 + c];      // (L_ji^T)[r][c] = L_ji[c][r]
        }
        for (int e = tid; e < 64 * nrhs; e += 256) {
            const int c = e % 64, q = e / 64;
            xs[c][q] = R[q * ldr + (int64_t)j * b + c0 + c];
        }
        __syncthreads();
        for (int c = part; c < 64; c += 4) {
            const double l = S[rr][c];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) acc[q] = fma(l, xs[c][q], acc[q]);
        }
    }
    part_reduce_sub(reinterpret_cast<double(*)[17]>(&S[0][0]), acc, nrhs, R, ldr, (int64_t)i * b + r0);
}

// R = B - A X (absmode 0) or R = |A| X (absmode 1, B unused) for the symmetric A held as
// lower tiles; rows and columns >= n (padding) contribute nothing and R's padding is 0.
template <int NQ>
__global__ void __launch_bounds__(256)
k_symv_resid(const double *A, int nt, int b, int64_t n, const double *X, int64_t ldx,
             const double *B, int64_t ldb, double *R, int64_t ldr, int nrhs, int absmode) {
    __shared__ double xs[64][16];
    __shared__ double S[64][65];
    const int chunks = b / 64;
    const int i = blockIdx.x / chunks, r0 = (blockIdx.x % chunks) * 64;
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    const int64_t bb = (int64_t)b * b;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int j = 0; j < nt; ++j) {
        const bool lower = j <= i;
        const double *T = lower ? A + ((int64_t)i * (i + 1) / 2 + j) * bb : A + ((int64_t)j * (j + 1) / 2 + i) * bb;
        for (int c0 = 0; c0 < b; c0 += 64) {
            __syncthreads();
            for (int idx = tid; idx < 4096; idx += 256) {
                const int lo = idx & 63, hi = idx >> 6;
                double v;
                int64_t gr, gc;
                if (lower) {   // S[r][c] = A_ij[r0 + r][c0 + c], coalesced along r
                    v = T[(int64_t)(c0 + hi) * b + r0 + lo];
                    gr = (int64_t)i * b + r0 + lo; gc = (int64_t)j * b + c0 + hi;
                    if (gr >= n || gc >= n) v = 0.0;
                    S[lo][hi] = absmode ? fabs(v) : v;
                } else {       // S[r][c] = A_ji[c0 + c][r0 + r], coalesced along c
                    v = T[(int64_t)(r0 + hi) * b + c0 + lo];
                    gr = (int64_t)i * b + r0 + hi; gc = (int64_t)j * b + c0 + lo;
                    if (gr >= n || gc >= n) v = 0.0;
                    S[hi][lo] = absmode ? fabs(v) : v;
                }
            }
            for (int e = tid; e < 64 * nrhs; e += 256) {
                const int c = e % 64, q = e / 64;
                const int64_t g = (int64_t)j * b + c0 + c;
                xs[c][q] = (g < n) ? X[q * ldx + g] : 0.0;
            }
            __syncthreads();
            for (int c = part; c < 64; c += 4) {
                const double l = S[rr][c];
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (q < nrhs) acc[q] = fma(l, xs[c][q], acc[q]);
            }
        }
    }
    double(*red)[17] = reinterpret_cast<double(*)[17]>(&S[0][0]);
    for (int p = 0; p < 4; ++p) {
        __syncthreads();
        if (part == p)
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) red[rr][q] = (p == 0) ? acc[q] : red[rr][q] + acc[q];
    }
    __syncthreads();
    for (int e = tid; e < 64 * nrhs; e += 256) {
        const int r = e % 64, q = e / 64;
        const int64_t g = (int64_t)i * b + r0 + r;
        double out = 0.0;
        if (g < n) out = absmode ? red[r][q] : B[q * ldb + g] - red[r][q];
        R[q * ldr + g] = out;
    }
}

// One right-hand side: R = B - A x (ABS false) or R = |A| x (ABS true; x = ones when X is
// null), A symmetric and held as lower tiles (column-major, the diagonal tiles full).  One
// CTA per 64 rows [r0, r0 + 64) of tile row i; every element of its 64 x n row panel is
// loaded once, straight from global memory into registers, for one multiply-add.
//   * tiles A_ij, j <= i: columns of the stored tile.  Warp w takes the columns c = w (mod 8),
//     each lane two adjacent rows (one 16-byte load per column; a warp reads 512 contiguous
//     bytes), with two accumulators per row so that consecutive columns do not chain.
//   * tiles right of the diagonal, A_ij = A_ji^T (j > i): row r of A_ij is column r of the
//     stored A_ji, contiguous in memory.  Warp w takes the rows r0 + 8w ... r0 + 8w + 7, its
//     lanes two adjacent columns per 64, with x's pair loaded once for the eight rows.
// Partial sums meet in a fixed order (lanes by shuffle, warps in shared memory), so the
// result does not depend on scheduling.  Rows and columns >= n (padding) contribute nothing
// and R's padding is 0.  The multiply-adds, not the bytes, bound it: a GB300 SM retires two
// FP64 multiply-adds per clock, n^2 per call.
template <bool ABS>
__global__ void __launch_bounds__(256)
k_symv1(const double *__restrict__ A, int nt, int b, int64_t n, const double *__restrict__ X,
        const double *__restrict__ B, double *__restrict__ R) {
    __shared__ double red[8][64];
    __shared__ double tr[64];
    const int chunks = b / 64;
    const int i = blockIdx.x / chunks, r0 = (blockIdx.x % chunks) * 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t bb = (int64_t)b * b;
    // tiles left of and on the diagonal
    double a0 = 0.0, a1 = 0.0, e0 = 0.0, e1 = 0.0;
    for (int j = 0; j <= i; ++j) {
        const double *T = A + ((int64_t)i * (i + 1) / 2 + j) * bb + r0 + 2 * lane;
        const double *x = X ? X + (int64_t)j * b : nullptr;
        const int cmax = (int)min((int64_t)b, n - (int64_t)j * b);
        int c = warp;
#pragma unroll 2
        for (; c + 8 < cmax; c += 16) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(T + (int64_t)c * b));
            const double2 w = __ldg(reinterpret_cast<const double2 *>(T + (int64_t)(c + 8) * b));
            const double xv = x ? __ldg(x + c) : 1.0, xw = x ? __ldg(x + c + 8) : 1.0;
            a0 = fma(ABS ? fabs(v.x) : v.x, xv, a0);
            a1 = fma(ABS ? fabs(v.y) : v.y, xv, a1);
            e0 = fma(ABS ? fabs(w.x) : w.x, xw, e0);
            e1 = fma(ABS ? fabs(w.y) : w.y, xw, e1);
        }
        if (c < cmax) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(T + (int64_t)c * b));
            const double xv = x ? __ldg(x + c) : 1.0;
            a0 = fma(ABS ? fabs(v.x) : v.x, xv, a0);
            a1 = fma(ABS ? fabs(v.y) : v.y, xv, a1);
        }
    }
    red[warp][2 * lane] = a0 + e0;
    red[warp][2 * lane + 1] = a1 + e1;
    // tiles right of the diagonal, through the stored tiles (j, i)
    double acc[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) acc[p] = 0.0;
    for (int j = i + 1; j < nt; ++j) {
        const double *T = A + ((int64_t)j * (j + 1) / 2 + i) * bb + (int64_t)(r0 + 8 * warp) * b + 2 * lane;
        const double *x = X ? X + (int64_t)j * b + 2 * lane : nullptr;
        const int cmax = (int)min((int64_t)b, n - (int64_t)j * b);
        for (int m = 0; m < b; m += 64) {
            double2 xv = x ? __ldg(reinterpret_cast<const double2 *>(x + m)) : make_double2(1.0, 1.0);
            const int c = m + 2 * lane;
            if (c >= cmax) xv.x = 0.0;
            if (c + 1 >= cmax) xv.y = 0.0;
            const bool lo = c < cmax, hi = c + 1 < cmax;
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                double2 v = __ldg(reinterpret_cast<const double2 *>(T + (int64_t)p * b + m));
                if (!lo) v.x = 0.0;
                if (!hi) v.y = 0.0;
                acc[p] = fma(ABS ? fabs(v.x) : v.x, xv.x, acc[p]);
                acc[p] = fma(ABS ? fabs(v.y) : v.y, xv.y, acc[p]);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        double v = acc[p];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) tr[8 * warp + p] = v;
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        const int r = threadIdx.x;
        double s = tr[r];
#pragma unroll
        for (int w = 0; w < 8; ++w) s += red[w][r];
        const int64_t g = (int64_t)i * b + r0 + r;
        double out = 0.0;
        if (g < n) out = ABS ? s : B[g] - s;
        R[g] = out;
    }
}

// out[c] = max_r |V[c*ld + r]|, r < n (out must start at 0; max of non-negative doubles is
// monotone in their bit patterns, so atomicMax on the bits is exact and order-free).
__global__ void k_colmax_abs(const double *V, int64_t ld, int64_t n, double *out) {
    const int c = blockIdx.y;
    double m = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(V[c * ld + r]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long *>(out + c), (unsigned long long)__double_as_longlong(m));
}

__global__ void k_axpy_cols(double *X, int64_t ldx, const double *D, int64_t ldd, int64_t n) {
    const int c = blockIdx.y;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        X[c * ldx + r] += D[c * ldd + r];
}

__global__ void __launch_bounds__(1024) k_dot_self(const double *v, int64_t n, double *out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) s = fma(v[i], v[i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}


// Batched POTRF step: one CTA per matrix entry (same 64-block position in each).
__global__ void __launch_bounds__(256) k_potrf_blocks(const PEntry *__restrict__ e, int ld) {
    const PEntry E = e[blockIdx.x];
    if (failed(E.status)) return;
    potrf64_body(E.D, ld, E.col0, E.status);
}

// Batched POTRF panel: rows below each entry's factored 64-block (grid.y = entry).
__global__ void __launch_bounds__(256) k_trsm_rows_batched(const PEntry *__restrict__ e, int ld) {
    const PEntry E = e[blockIdx.y];
    if (failed(E.status) || (int)blockIdx.x * PANEL_ROWS >= E.rows) return;
    panel_body(E.D + 64 + blockIdx.x * PANEL_ROWS, E.D, ld);
}

void launch_potrf_blocks(const PEntry *e, int n, int ld, cudaStream_t s) {
    if (n > 0) k_potrf_blocks<<<n, 256, 0, s>>>(e, ld);
}
void launch_trsm_rows_batched(const PEntry *e, int n, int max_rows, int ld, cudaStream_t s) {
    if (n > 0 && max_rows > 0) k_trsm_rows_batched<<<dim3(max_rows / PANEL_ROWS, n), 256, 0, s>>>(e, ld);
}


// log|A_i| = 2 sum log L_ii for every matrix of a batch (one CTA each, fixed order)
__global__ void __launch_bounds__(256) k_logdet_batched(const LEntry *__restrict__ e, int b, double *out) {
    __shared__ double red[256];
    const LEntry E = e[blockIdx.x];
    double s = 0.0;
    for (int64_t g = threadIdx.x; g < E.n; g += 256) {
        const int t = (int)(g / b), r = (int)(g % b);
        const double *D = E.W + ((int64_t)t * (t + 1) / 2 + t) * (int64_t)b * b;
        s += log(D[(int64_t)r * b + r]);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = 2.0 * red[0];
}

// identity padding of the last tile row of every ragged matrix (grid.z = matrix)
__global__ void k_fix_padding_batched(const LEntry *__restrict__ e, int b) {
    const LEntry E = e[blockIdx.z];
    const int j = blockIdx.y, i = E.nt - 1;
    if (j > i || E.n % b == 0) return;
    const int nv = (int)(E.n - (int64_t)i * b);
    double *T = E.W + ((int64_t)i * (i + 1) / 2 + j) * (int64_t)b * b;
    const int64_t bb = (int64_t)b * b;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < bb; x += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(x % b), c = (int)(x / b);
        if (j < i) {
            if (r >= nv) T[x] = 0.0;
        } else if (r >= nv || c >= nv) {
            T[x] = (r == c) ? 1.0 : 0.0;
        }
    }
}

void launch_logdet_batched(const LEntry *e, int count, int b, double *out, cudaStream_t s) {
    if (count > 0) k_logdet_batched<<<count, 256, 0, s>>>(e, b, out);
}
void launch_fix_padding_batched(const LEntry *e, int count, int ntmax, int b, cudaStream_t s) {
    if (count > 0) k_fix_padding_batched<<<dim3(16, ntmax, count), 256, 0, s>>>(e, b);
}


// ------------------------------------------------------------ grouped (batched) solves
__global__ void __launch_bounds__(256) k_fwd_diag_g(const SDiag *__restrict__ e, double *R, int b) {
    const SDiag E = e[blockIdx.y];
    fwd_diag_body(E.L, b, b, R + E.off + blockIdx.x * E.ldr);
}

template <int NQ>
__global__ void __launch_bounds__(256) k_fwd_update_g(const SUpd *__restrict__ u, double *R, int b, int nrhs) {
    const SUpd U = u[blockIdx.x];
    __shared__ double zs[128][16];
    __shared__ double red[64][17];
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int c0 = 0; c0 < b; c0 += 128) {
        __syncthreads();
        for (int e = tid; e < 128 * nrhs; e += 256) {
            const int c = e % 128, q = e / 128;
            zs[c][q] = R[U.src + q * U.ldr + c0 + c];
        }
        __syncthreads();
        for (int c = part; c < 128; c += 4) {
            const double l = U.L[(int64_t)(c0 + c) * b + U.r0 + rr];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) acc[q] = fma(l, zs[c][q], acc[q]);
        }
    }
    part_reduce_sub(red, acc, nrhs, R + U.dst, U.ldr, 0);
}

__global__ void __launch_bounds__(256) k_bwd_diag_g(const SDiag *__restrict__ e, double *R, int b) {
    const SDiag E = e[blockIdx.y];
    bwd_diag_body(E.L, b, b, R + E.off + blockIdx.x * E.ldr);
}

template <int NQ>
__global__ void __launch_bounds__(256) k_bwd_update_g(const SUpd *__restrict__ u, double *R, int b, int nrhs) {
    const SUpd U = u[blockIdx.x];
    __shared__ double xs[64][16];
    __shared__ double S[64][65];
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int c0 = 0; c0 < b; c0 += 64) {
        __syncthreads();
        for (int idx = tid; idx < 4096; idx += 256) {
            const int c = idx & 63, r = idx >> 6;
            S[r][c] = U.L[(int64_t)(U.r0 + r) * b + c0 + c];
        }
        for (int e = tid; e < 64 * nrhs; e += 256) {
            const int c = e % 64, q = e / 64;
            xs[c][q] = R[U.src + q * U.ldr + c0 + c];
        }
        __syncthreads();
        for (int c = part; c < 64; c += 4) {
            const double l = S[rr][c];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) acc[q] = fma(l, xs[c][q], acc[q]);
        }
    }
    part_reduce_sub(reinterpret_cast<double(*)[17]>(&S[0][0]), acc, nrhs, R + U.dst, U.ldr, 0);
}

// FP32 forms of the grouped substitution (the correction solves of a refined batched solve): the
// factor tiles are read in FP64 and rounded to FP32 on load, products and sums run on the FP32
// pipe (GB300 retires 64x more FP32 than FP64 operations per clock); the diagonal blocks keep
// FP64 arithmetic on the FP32 vectors.  Iterative refinement with FP64 residuals takes the
// result to FP64 accuracy: a correction needs only a few correct digits.
template <int NQ>
__device__ __forceinline__ void part_reduce_sub_f(float (*red)[17], const float (&acc)[NQ], int nrhs, float *R,
                                                  int64_t ldr) {
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    for (int p = 0; p < 4; ++p) {
        __syncthreads();
        if (part == p)
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) red[rr][q] = (p == 0) ? acc[q] : red[rr][q] + acc[q];
    }
    __syncthreads();
    for (int e = tid; e < 64 * nrhs; e += 256) {
        const int r = e % 64, q = e / 64;
        R[q * ldr + r] -= red[r][q];
    }
}
__global__ void __launch_bounds__(256) k_fwd_diag_gf(const SDiag *__restrict__ e, float *R, int b) {
    const SDiag E = e[blockIdx.y];
    fwd_diag_body(E.L, b, b, R + E.off + blockIdx.x * E.ldr);
}
__global__ void __launch_bounds__(256) k_bwd_diag_gf(const SDiag *__restrict__ e, float *R, int b) {
    const SDiag E = e[blockIdx.y];
    bwd_diag_body(E.L, b, b, R + E.off + blockIdx.x * E.ldr);
}
template <int NQ>
__global__ void __launch_bounds__(256) k_fwd_update_gf(const SUpd *__restrict__ u, float *R, int b, int nrhs) {
    const SUpd U = u[blockIdx.x];
    __shared__ float zs[128][17];
    __shared__ float red[64][17];
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    float acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.f;
    for (int c0 = 0; c0 < b; c0 += 128) {
        __syncthreads();
        for (int e = tid; e < 128 * nrhs; e += 256) {
            const int c = e % 128, q = e / 128;
            zs[c][q] = R[U.src + q * U.ldr + c0 + c];
        }
        __syncthreads();
        for (int c = part; c < 128; c += 4) {
            const float l = (float)U.L[(int64_t)(c0 + c) * b + U.r0 + rr];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) acc[q] = fmaf(l, zs[c][q], acc[q]);
        }
    }
    part_reduce_sub_f(red, acc, nrhs, R + U.dst, U.ldr);
}
template <int NQ>
__global__ void __launch_bounds__(256) k_bwd_update_gf(const SUpd *__restrict__ u, float *R, int b, int nrhs) {
    const SUpd U = u[blockIdx.x];
    __shared__ float xs[64][17];
    __shared__ float S[64][65];
    __shared__ float red[64][17];
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    float acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.f;
    for (int c0 = 0; c0 < b; c0 += 64) {
        __syncthreads();
        for (int idx = tid; idx < 4096; idx += 256) {
            const int c = idx & 63, r = idx >> 6;
            S[r][c] = (float)U.L[(int64_t)(U.r0 + r) * b + c0 + c];
        }
        for (int e = tid; e < 64 * nrhs; e += 256) {
            const int c = e % 64, q = e / 64;
            xs[c][q] = R[U.src + q * U.ldr + c0 + c];
        }
        __syncthreads();
        for (int c = part; c < 64; c += 4) {
            const float l = S[rr][c];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) acc[q] = fmaf(l, xs[c][q], acc[q]);
        }
    }
    part_reduce_sub_f(red, acc, nrhs, R + U.dst, U.ldr);
}
__global__ void k_to_f32(const double *__restrict__ x, float *__restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}
__global__ void k_add_f32(double *__restrict__ x, const float *__restrict__ d, int64_t n, int assign) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = assign ? (double)d[i] : x[i] + (double)d[i];
}

template <int NQ>
__global__ void __launch_bounds__(256)
k_symv_g(const SRes *__restrict__ rs, int b, const double *X, const double *B, double *R, int nrhs, int absmode) {
    const SRes Q = rs[blockIdx.x];
    __shared__ double xs[64][16];
    __shared__ double S[64][65];
    const int i = Q.i, r0 = Q.r0;
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    const int64_t bb = (int64_t)b * b;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int j = 0; j < Q.nt; ++j) {
        const bool lower = j <= i;
        const double *T = lower ? Q.A + ((int64_t)i * (i + 1) / 2 + j) * bb : Q.A + ((int64_t)j * (j + 1) / 2 + i) * bb;
        for (int c0 = 0; c0 < b; c0 += 64) {
            __syncthreads();
            for (int idx = tid; idx < 4096; idx += 256) {
                const int lo = idx & 63, hi = idx >> 6;
                double v;
                int64_t gr, gc;
                if (lower) {
                    v = T[(int64_t)(c0 + hi) * b + r0 + lo];
                    gr = (int64_t)i * b + r0 + lo; gc = (int64_t)j * b + c0 + hi;
                    if (gr >= Q.n || gc >= Q.n) v = 0.0;
                    S[lo][hi] = absmode ? fabs(v) : v;
                } else {
                    v = T[(int64_t)(r0 + hi) * b + c0 + lo];
                    gr = (int64_t)i * b + r0 + hi; gc = (int64_t)j * b + c0 + lo;
                    if (gr >= Q.n || gc >= Q.n) v = 0.0;
                    S[hi][lo] = absmode ? fabs(v) : v;
                }
            }
            for (int e = tid; e < 64 * nrhs; e += 256) {
                const int c = e % 64, q = e / 64;
                const int64_t g = (int64_t)j * b + c0 + c;
                xs[c][q] = (g < Q.n) ? (X ? X[Q.xo + q * Q.ldr + g] : 1.0) : 0.0;
            }
            __syncthreads();
            for (int c = part; c < 64; c += 4) {
                const double l = S[rr][c];
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (q < nrhs) acc[q] = fma(l, xs[c][q], acc[q]);
            }
        }
    }
    double(*red)[17] = reinterpret_cast<double(*)[17]>(&S[0][0]);
    for (int p = 0; p < 4; ++p) {
        __syncthreads();
        if (part == p)
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) red[rr][q] = (p == 0) ? acc[q] : red[rr][q] + acc[q];
    }
    __syncthreads();
    for (int e = tid; e < 64 * nrhs; e += 256) {
        const int r = e % 64, q = e / 64;
        const int64_t g = (int64_t)i * b + r0 + r;
        double out = 0.0;
        if (g < Q.n) out = absmode ? red[r][q] : B[Q.bo + q * Q.ldr + g] - red[r][q];
        R[Q.ro + q * Q.ldr + g] = out;
    }
}

__global__ void k_colmax_g(const SMax *__restrict__ m, const double *V, int nrhs, double *out) {
    const SMax M = m[blockIdx.y];
    for (int c = 0; c < nrhs; ++c) {
        double mx = 0.0;
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < M.n; r += (int64_t)gridDim.x * blockDim.x)
            mx = fmax(mx, fabs(V[M.off + c * M.ldr + r]));
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0)
            atomicMax(reinterpret_cast<unsigned long long *>(out + M.out + c), (unsigned long long)__double_as_longlong(mx));
    }
}

__global__ void k_axpy_flat(double *X, const double *D, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        X[e] += D[e];
}

// one CTA per matrix: out[M.out] = u . v over its n entries (fixed order)
__global__ void __launch_bounds__(256) k_dots_g(const SMax *__restrict__ m, const double *u, const double *v, double *out) {
    const SMax M = m[blockIdx.x];
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < M.n; r += 256) s = fma(u[M.off + r], v[M.off + r], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[M.out] = red[0];
}

void launch_fwd_diag_g(const SDiag *e, int ne, double *R, int b, int nrhs, cudaStream_t s) {
    if (ne > 0) k_fwd_diag_g<<<dim3(nrhs, ne), 256, 0, s>>>(e, R, b);
}
void launch_fwd_update_g(const SUpd *u, int nu, double *R, int b, int nrhs, cudaStream_t s) {
    if (nu > 0) NQ_DISPATCH(nrhs, k_fwd_update_g, nu, 256, 0, s, u, R, b, nrhs);
}
void launch_bwd_diag_g(const SDiag *e, int ne, double *R, int b, int nrhs, cudaStream_t s) {
    if (ne > 0) k_bwd_diag_g<<<dim3(nrhs, ne), 256, 0, s>>>(e, R, b);
}
void launch_bwd_update_g(const SUpd *u, int nu, double *R, int b, int nrhs, cudaStream_t s) {
    if (nu > 0) NQ_DISPATCH(nrhs, k_bwd_update_g, nu, 256, 0, s, u, R, b, nrhs);
}
void launch_fwd_diag_gf(const SDiag *e, int ne, float *R, int b, int nrhs, cudaStream_t s) {
    if (ne > 0) k_fwd_diag_gf<<<dim3(nrhs, ne), 256, 0, s>>>(e, R, b);
}
void launch_fwd_update_gf(const SUpd *u, int nu, float *R, int b, int nrhs, cudaStream_t s) {
    if (nu > 0) NQ_DISPATCH(nrhs, k_fwd_update_gf, nu, 256, 0, s, u, R, b, nrhs);
}
void launch_bwd_diag_gf(const SDiag *e, int ne, float *R, int b, int nrhs, cudaStream_t s) {
    if (ne > 0) k_bwd_diag_gf<<<dim3(nrhs, ne), 256, 0, s>>>(e, R, b);
}
void launch_bwd_update_gf(const SUpd *u, int nu, float *R, int b, int nrhs, cudaStream_t s) {
    if (nu > 0) NQ_DISPATCH(nrhs, k_bwd_update_gf, nu, 256, 0, s, u, R, b, nrhs);
}
void launch_to_f32(const double *x, float *y, int64_t n, cudaStream_t s) {
    if (n > 0) k_to_f32<<<608, 256, 0, s>>>(x, y, n);
}
void launch_add_f32(double *x, const float *d, int64_t n, int assign, cudaStream_t s) {
    if (n > 0) k_add_f32<<<608, 256, 0, s>>>(x, d, n, assign);
}
void launch_symv_g(const SRes *r, int nr, int b, const double *X, const double *B, double *R, int nrhs, int absmode,
                   cudaStream_t s) {
    if (nr > 0) NQ_DISPATCH(nrhs, k_symv_g, nr, 256, 0, s, r, b, X, B, R, nrhs, absmode);
}
void launch_colmax_g(const SMax *m, int nm, const double *V, int nrhs, double *out, cudaStream_t s) {
    if (nm > 0) k_colmax_g<<<dim3(8, nm), 256, 0, s>>>(m, V, nrhs, out);
}
void launch_axpy_flat(double *X, const double *D, int64_t count, cudaStream_t s) {
    k_axpy_flat<<<1024, 256, 0, s>>>(X, D, count);
}
void launch_dots_g(const SMax *m, int nm, const double *u, const double *v, double *out, cudaStream_t s) {
    if (nm > 0) k_dots_g<<<nm, 256, 0, s>>>(m, u, v, out);
}

// ---------------------------------------------------------------------------- launchers

void launch_dgemm_update(const DJob *jobs, const DItem *items, int nitems, int ld, double *partials,
                         const int *status, cudaStream_t s) {
    if (nitems > 0) k_dgemm_update<<<nitems, 256, 0, s>>>(jobs, items, ld, partials, status);
}
void launch_dgemm_reduce(const DRed *reds, int nreds, int ld, const double *partials, const int *status,
                         cudaStream_t s) {
    if (nreds > 0) k_dgemm_reduce<<<nreds, 256, 0, s>>>(reds, ld, partials, status);
}
void launch_potrf_block(double *D, int ld, int col0, int *status, cudaStream_t s) {
    k_potrf_block<<<1, 256, 0, s>>>(D, ld, col0, status);
}
void launch_trsm_rows(double *P, const double *L, int ld, int rows, const int *status, cudaStream_t s) {
    if (rows > 0) k_trsm_rows<<<rows / PANEL_ROWS, 256, 0, s>>>(P, L, ld, status);
}
void launch_trsm_strips(const TStrip *strips, int nstrips, int ld, int b, const int *status, cudaStream_t s) {
    const size_t smem = (32 * 64 + 2 * 64 * 65 + 64) * sizeof(double);
    static std::atomic<unsigned long long> attr{0};
    if (attrs_pending(attr)) {
        cudaFuncSetAttribute(k_trsm_strips, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        mark_attrs_set(attr);
    }
    if (nstrips > 0) k_trsm_strips<<<nstrips, 256, smem, s>>>(strips, ld, b, status);
}
void launch_logdet(const double *W, int nt, int b, int64_t n, double *out, cudaStream_t s) {
    (void)nt;
    k_logdet<<<1, 1024, 0, s>>>(W, b, n, out);
}
void launch_fix_padding(double *W, int nt, int b, int64_t n, cudaStream_t s) {
    if (n % b == 0) return;
    k_fix_padding<<<dim3(64, nt), 256, 0, s>>>(W, nt, b, n);
}
void launch_zero_upper_diag(double *W, int nt, int b, int64_t n, cudaStream_t s) {
    k_zero_upper_diag<<<dim3(64, (n % b) ? 2 * nt - 1 : nt), 256, 0, s>>>(W, nt, b, n);
}
// A diagonal tile's substitution in sub-blocks of DIAG_SUB rows: a one-CTA triangular solve
// per sub-block, then a many-CTA product with the rest of its columns (the one-CTA part,
// bound by a single SM's FP64 rate, shrinks from b^2/2 to b DIAG_SUB/2 multiply-adds).
constexpr int DIAG_SUB = 256;
void launch_fwd_diag(const double *Ljj, int b, double *R, int64_t ldr, int nrhs, cudaStream_t s) {
    const int S = (b % DIAG_SUB) ? b : DIAG_SUB;     // tiles not a multiple of it: one block
    for (int sb = 0; sb < b / S; ++sb) {
        k_fwd_diag<<<nrhs, 256, 0, s>>>(Ljj + (int64_t)sb * S * b + sb * S, b, S, R + sb * S, ldr);
        const int rows = b - (sb + 1) * S;
        if (rows > 0)
            NQ_DISPATCH(nrhs, k_gemv_below, rows / 64, 256, 0, s, Ljj + (int64_t)sb * S * b + (sb + 1) * S, b, S,
                        R + sb * S, R + (sb + 1) * S, ldr, nrhs);
    }
}
void launch_fwd_update(const double *W, int nt, int b, int j, double *R, int64_t ldr, int nrhs, cudaStream_t s) {
    const int ntiles = nt - 1 - j;
    if (ntiles > 0) NQ_DISPATCH(nrhs, k_fwd_update, ntiles * (b / 64), 256, 0, s, W, b, j, R, ldr, nrhs);
}
void launch_bwd_diag(const double *Ljj, int b, double *R, int64_t ldr, int nrhs, cudaStream_t s) {
    const int S = (b % DIAG_SUB) ? b : DIAG_SUB;     // tiles not a multiple of it: one block
    for (int sb = b / S - 1; sb >= 0; --sb) {
        k_bwd_diag<<<nrhs, 256, 0, s>>>(Ljj + (int64_t)sb * S * b + sb * S, b, S, R + sb * S, ldr);
        if (sb > 0)
            NQ_DISPATCH(nrhs, k_gemv_above, sb * S / 64, 256, 0, s, Ljj + sb * S, b, S, R + sb * S, R, ldr, nrhs);
    }
}
void launch_bwd_update(const double *W, int nt, int b, int j, double *R, int64_t ldr, int nrhs, cudaStream_t s) {
    (void)nt;
    if (j > 0) NQ_DISPATCH(nrhs, k_bwd_update, j * (b / 64), 256, 0, s, W, b, j, R, ldr, nrhs);
}
void launch_symv_resid(const double *A, int nt, int b, int64_t n, const double *X, int64_t ldx,
                       const double *B, int64_t ldb, double *R, int64_t ldr, int nrhs, int absmode,
                       cudaStream_t s) {
    const auto al16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    if (nrhs == 1 && al16(A) && al16(X) && b % 64 == 0) {      // 16-byte loads of A and x
        if (absmode)
            k_symv1<true><<<nt * (b / 64), 256, 0, s>>>(A, nt, b, n, X, nullptr, R);
        else
            k_symv1<false><<<nt * (b / 64), 256, 0, s>>>(A, nt, b, n, X, B, R);
        return;
    }
    NQ_DISPATCH(nrhs, k_symv_resid, nt * (b / 64), 256, 0, s, A, nt, b, n, X, ldx, B, ldb, R, ldr, nrhs, absmode);
}
void launch_colmax_abs(const double *V, int64_t ld, int64_t n, int ncols, double *out, cudaStream_t s) {
    k_colmax_abs<<<dim3(64, ncols), 256, 0, s>>>(V, ld, n, out);
}
void launch_axpy_cols(double *X, int64_t ldx, const double *D, int64_t ldd, int64_t n, int ncols, cudaStream_t s) {
    k_axpy_cols<<<dim3(64, ncols), 256, 0, s>>>(X, ldx, D, ldd, n);
}
__global__ void __launch_bounds__(1024) k_dot(const double *u, const double *v, int64_t n, double *out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) s = fma(u[i], v[i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

void launch_dot(const double *u, const double *v, int64_t n, double *out, cudaStream_t s) {
    k_dot<<<1, 1024, 0, s>>>(u, v, n, out);
}

void launch_dot_self(const double *v, int64_t n, double *out, cudaStream_t s) {
    k_dot_self<<<1, 1024, 0, s>>>(v, n, out);
}

// ------------------------------------------------------------- tile-pointer variants
// Used by the out-of-core executor, whose tiles live in cache slots at arbitrary
// addresses: the job comes by value and the grid is the 64 x 64 block grid.
__global__ void __launch_bounds__(256, 2) k_dgemm_tile(const DJob job, int ld) {
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (job.lower && bi < bj) return;
    __shared__ double Xs[16][64], Ys[16][64];
    double acc[4][4] = {};
    dgemm_block(acc, job.X + bi * 64, job.Y + bj * 64, ld, 0, job.K, Xs, Ys);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double *C = job.C + (int64_t)bj * 64 * ld + bi * 64;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) C[(int64_t)(ty + 16 * j) * ld + tx + 16 * i] -= acc[i][j];
}

// TRSM of up to TG_MAX tiles at C[0..] with the same L_kk at L (one CTA per 64-row strip;
// grid b/64 x tiles).
struct TGroup {
    double *C[TG_MAX];
};
__global__ void __launch_bounds__(256, 2)
k_trsm_tile(const __grid_constant__ TGroup g, const double *L, int ld, int b, const int *status) {
    if (failed(status)) return;
    double *C = g.C[blockIdx.y];
    extern __shared__ double smem[];
    double(*Xs)[64] = reinterpret_cast<double(*)[64]>(smem);
    double(*Ys)[64] = reinterpret_cast<double(*)[64]>(smem + 16 * 64);
    double(*Ls)[65] = reinterpret_cast<double(*)[65]>(smem + 32 * 64);
    double(*Ss)[65] = reinterpret_cast<double(*)[65]>(smem + 32 * 64 + 64 * 65);
    double *rinv = smem + 32 * 64 + 2 * 64 * 65;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double *X = C + blockIdx.x * 64;
    for (int jb = 0; jb < b / 64; ++jb) {
        double acc[4][4] = {};
        dgemm_block(acc, X, L + jb * 64, ld, 0, jb * 64, Xs, Ys);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                Ss[tx + 16 * i][ty + 16 * j] = X[(int64_t)(jb * 64 + ty + 16 * j) * ld + tx + 16 * i] - acc[i][j];
        for (int idx = tid; idx < 4096; idx += 256) {
            const int r = idx & 63, c = idx >> 6;
            Ls[r][c] = (r >= c) ? L[(int64_t)(jb * 64 + c) * ld + jb * 64 + r] : 0.0;
        }
        __syncthreads();
        if (tid < 64) rinv[tid] = 1.0 / Ls[tid][tid];
        __syncthreads();
        strip_solve<64>(Ss, Ls, rinv);
        for (int idx = tid; idx < 4096; idx += 256) {
            const int r = idx & 63, c = idx >> 6;
            X[(int64_t)(jb * 64 + c) * ld + r] = Ss[r][c];
        }
        __syncthreads();
    }
}

// Y = L^{-1} for a lower-triangular b x b tile L (column-major, ld = b), by forward
// substitution L y_c = e_c column by column.  CTA x owns columns 4x .. 4x+3 and
// b-4-4x .. b-1-4x: a long and a short group, so every CTA carries about the same work
// (column c costs (b - c)^2 / 2 multiply-adds).  For each group, and each 64-row block from
// the group's first nonzero row on, the product with the already solved rows (kept in shared
// memory) is followed by the 64 x 64 diagonal solve.
constexpr int TRINV_COLS = 4;
__device__ __forceinline__ void trinv_body(const double *__restrict__ L, int b, double *__restrict__ Y) {
    extern __shared__ double tsm[];
    double *Ys = tsm;                               // b x 4: the group's columns, row-major by row
    double(*Ld)[65] = reinterpret_cast<double(*)[65]>(tsm + (size_t)b * TRINV_COLS);
    double(*Acc)[TRINV_COLS] = reinterpret_cast<double(*)[TRINV_COLS]>(tsm + (size_t)b * TRINV_COLS + 64 * 65);
    const int tid = threadIdx.x;
    const int r = tid & 63, cg = tid >> 6;          // row in block, column of the group
    for (int grp = 0; grp < 2; ++grp) {
        const int c0 = grp == 0 ? (int)blockIdx.x * TRINV_COLS : b - TRINV_COLS - (int)blockIdx.x * TRINV_COLS;
        const int ib0 = c0 / 64;
        __syncthreads();                            // the previous group's output is written
        for (int i = tid; i < ib0 * 64 * TRINV_COLS; i += 256) Ys[i] = 0.0;
        for (int ib = ib0; ib < b / 64; ++ib) {
            const int row = ib * 64 + r;
            double a = (row == c0 + cg) ? 1.0 : 0.0;
            for (int l = ib0 * 64; l < ib * 64; ++l) a = fma(-L[(int64_t)l * b + row], Ys[l * TRINV_COLS + cg], a);
            Acc[r][cg] = a;
            for (int i = tid; i < 4096; i += 256) {
                const int rr = i & 63, cc = i >> 6;
                Ld[rr][cc] = (rr >= cc) ? L[(int64_t)(ib * 64 + cc) * b + ib * 64 + rr] : 0.0;
            }
            __syncthreads();
            for (int j = 0; j < 64; ++j) {
                if (tid < TRINV_COLS) Acc[j][tid] = Acc[j][tid] / Ld[j][j];
                __syncthreads();
                {
                    const int rr = tid / TRINV_COLS, cc = tid % TRINV_COLS;    // 64 x 4 = 256 threads
                    if (rr > j) Acc[rr][cc] = fma(-Ld[rr][j], Acc[j][cc], Acc[rr][cc]);
                }
                __syncthreads();
            }
            Ys[(ib * 64 + tid / TRINV_COLS) * TRINV_COLS + tid % TRINV_COLS] = Acc[tid / TRINV_COLS][tid % TRINV_COLS];
            __syncthreads();
        }
        for (int i = tid; i < b * TRINV_COLS; i += 256) {
            const int rr = i % b, cc = i / b;
            Y[(int64_t)(c0 + cc) * b + rr] = Ys[rr * TRINV_COLS + cc];
        }
    }
}
__global__ void __launch_bounds__(256) k_trinv(const double *__restrict__ L, int b, double *__restrict__ Y) {
    trinv_body(L, b, Y);
}
// the same for several tiles at once (grid.y = entry): the diagonal tiles of a batch's column
__global__ void __launch_bounds__(256) k_trinv_batched(const TEntry *__restrict__ e, int b) {
    const TEntry E = e[blockIdx.y];
    trinv_body(E.L, b, E.Y);
}

// sum of log of the nv leading diagonal entries of one tile, fixed order, into *out
__global__ void __launch_bounds__(256) k_logdiag_tile(const double *D, int b, int nv, double *out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int r = threadIdx.x; r < nv; r += 256) s += log(D[(int64_t)r * b + r]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// padding of one tile of the last tile row: rows >= nv zero (off-diagonal), identity
// outside the nv x nv block (diagonal)
__global__ void k_fix_padding_tile(double *T, int b, int nv, int diag) {
    const int64_t bb = (int64_t)b * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bb; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % b), c = (int)(e / b);
        if (!diag) {
            if (r >= nv) T[e] = 0.0;
        } else if (r >= nv || c >= nv) {
            T[e] = (r == c) ? 1.0 : 0.0;
        }
    }
}

// r_i -= L_ij z_j for one tile L_ij (ptr), rows of tile row i; grid = b/64 chunks
template <int NQ>
__global__ void __launch_bounds__(256)
k_fwd_update_tile(const double *L, int b, int i, int j, double *R, int64_t ldr, int nrhs) {
    __shared__ double zs[128][16];
    __shared__ double red[64][17];
    const int r0 = blockIdx.x * 64;
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int c0 = 0; c0 < b; c0 += 128) {
        __syncthreads();
        for (int e = tid; e < 128 * nrhs; e += 256) {
            const int c = e % 128, q = e / 128;
            zs[c][q] = R[q * ldr + (int64_t)j * b + c0 + c];
        }
        __syncthreads();
        for (int c = part; c < 128; c += 4) {
            const double l = L[(int64_t)(c0 + c) * b + r0 + rr];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) acc[q] = fma(l, zs[c][q], acc[q]);
        }
    }
    part_reduce_sub(red, acc, nrhs, R, ldr, (int64_t)i * b + r0);
}

// z_i -= L_ji^T x_j for one tile L_ji (ptr); grid = b/64 chunks of tile row i
template <int NQ>
__global__ void __launch_bounds__(256)
k_bwd_update_tile(const double *L, int b, int i, int j, double *R, int64_t ldr, int nrhs) {
    __shared__ double xs[64][16];
    __shared__ double S[64][65];
    const int r0 = blockIdx.x * 64;
    const int tid = threadIdx.x, rr = tid & 63, part = tid >> 6;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int c0 = 0; c0 < b; c0 += 64) {
        __syncthreads();
        for (int idx = tid; idx < 4096; idx += 256) {
            const int c = idx & 63, r = idx >> 6;
            S[r][c] = L[(int64_t)(r0 + r) * b + c0 + c];
        }
        for (int e = tid; e < 64 * nrhs; e += 256) {
            const int c = e % 64, q = e / 64;
            xs[c][q] = R[q * ldr + (int64_t)j * b + c0 + c];
        }
        __syncthreads();
        for (int c = part; c < 64; c += 4) {
            const double l = S[rr][c];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nrhs) acc[q] = fma(l, xs[c][q], acc[q]);
        }
    }
    part_reduce_sub(reinterpret_cast<double(*)[17]>(&S[0][0]), acc, nrhs, R, ldr, (int64_t)i * b + r0);
}

void launch_dgemm_tile(const DJob &job, int ld, cudaStream_t s) {
    k_dgemm_tile<<<dim3(job.M / 64, job.N / 64), 256, 0, s>>>(job, ld);
}
static size_t trsm_tile_smem() {
    const size_t smem = (32 * 64 + 2 * 64 * 65 + 64) * sizeof(double);
    static std::atomic<unsigned long long> attr{0};
    if (attrs_pending(attr)) {
        cudaFuncSetAttribute(k_trsm_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        mark_attrs_set(attr);
    }
    return smem;
}
void launch_trsm_tile(double *C, const double *L, int ld, int b, const int *status, cudaStream_t s) {
    launch_trsm_group(&C, 1, L, ld, b, status, s);
}
void launch_trsm_group(double *const *C, int ntiles, const double *L, int ld, int b, const int *status,
                       cudaStream_t s) {
    if (ntiles <= 0) return;
    const size_t smem = trsm_tile_smem();
    TGroup g{};
    for (int t = 0; t < ntiles; ++t) g.C[t] = C[t];
    k_trsm_tile<<<dim3(b / 64, ntiles), 256, smem, s>>>(g, L, ld, b, status);
}
void launch_trinv(const double *L, int b, double *Y, cudaStream_t s) {
    const size_t smem = ((size_t)b * TRINV_COLS + 64 * 65 + 64 * TRINV_COLS) * sizeof(double);
    static std::atomic<unsigned long long> attr{0};
    if (attrs_pending(attr)) {     // sized for the largest tile it serves (b <= 2048)
        cudaFuncSetAttribute(k_trinv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(((size_t)2048 * TRINV_COLS + 64 * 65 + 64 * TRINV_COLS) * sizeof(double)));
        mark_attrs_set(attr);
    }
    k_trinv<<<b / (2 * TRINV_COLS), 256, smem, s>>>(L, b, Y);
}
void launch_trinv_batched(const TEntry *e, int n, int b, cudaStream_t s) {
    if (n <= 0) return;
    const size_t smem = ((size_t)b * TRINV_COLS + 64 * 65 + 64 * TRINV_COLS) * sizeof(double);
    static std::atomic<unsigned long long> attr{0};
    if (attrs_pending(attr)) {     // sized for the largest tile it serves (b <= 2048)
        cudaFuncSetAttribute(k_trinv_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(((size_t)2048 * TRINV_COLS + 64 * 65 + 64 * TRINV_COLS) * sizeof(double)));
        mark_attrs_set(attr);
    }
    k_trinv_batched<<<dim3(b / (2 * TRINV_COLS), n), 256, smem, s>>>(e, b);
}
void launch_logdiag_tile(const double *D, int b, int nv, double *out, cudaStream_t s) {
    k_logdiag_tile<<<1, 256, 0, s>>>(D, b, nv, out);
}
void launch_fix_padding_tile(double *T, int b, int nv, int diag, cudaStream_t s) {
    k_fix_padding_tile<<<64, 256, 0, s>>>(T, b, nv, diag);
}
void launch_fwd_update_tile(const double *L, int b, int i, int j, double *R, int64_t ldr, int nrhs, cudaStream_t s) {
    NQ_DISPATCH(nrhs, k_fwd_update_tile, b / 64, 256, 0, s, L, b, i, j, R, ldr, nrhs);
}
void launch_bwd_update_tile(const double *L, int b, int i, int j, double *R, int64_t ldr, int nrhs, cudaStream_t s) {
    NQ_DISPATCH(nrhs, k_bwd_update_tile, b / 64, 256, 0, s, L, b, i, j, R, ldr, nrhs);
}

}  // namespace tc
