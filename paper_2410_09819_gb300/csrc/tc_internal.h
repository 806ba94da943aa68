// Internal declarations shared by the tile_chol translation units (not part of the ABI).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace tc {

constexpr int BLK = 64;         // FP64 kernels work on 64 x 64 blocks
constexpr int NSM = 152;        // GB300 streaming multiprocessors

__host__ __device__ __forceinline__ int64_t tidx(int64_t i, int64_t j) { return i * (i + 1) / 2 + j; }

// C -= X Y^T on a (M x N) block grid; X is M x K and Y is N x K, all column-major with
// leading dimension ld (the tile size): the layout of a tile row of the factor.
struct DJob {
    double *C;
    const double *X;
    const double *Y;
    int K, M, N, lower;
    const int *status;   // info word of the matrix (skip when non-zero), or nullptr
};

// One CTA of the FP64 update: 64 x 64 output block (bi, bj) of job `job`, contraction
// range [k0, k1).  part < 0: subtract straight into C, else write the block to
// partial buffer `part` (split-K; a reduce launch subtracts the partials in order).
struct DItem {
    int job;
    uint16_t bi, bj;
    int k0, k1;
    int part;
};

// Reduce: C_block -= sum_{p < nparts} partial[part0 + p]; C_block is the 64 x 64 block
// at C (leading dimension ld).
struct DRed {
    double *C;
    int part0, nparts;
};

// A 64-row strip of one TRSM tile: solve X L^T = C in place for rows [r0, r0 + 64).
struct TStrip {
    double *C;          // tile (m, k) of the factor
    const double *L;    // L_kk
    const int *status;  // info word of the matrix
    int r0;
};

// One diagonal tile's blocked POTRF step (batched over matrices): the 64-block at D,
// its panel below (rows) and the matrix's info word; col0 = global column of the block.
struct PEntry {
    double *D;
    int *status;
    int col0, rows;
};

// Grouped (batched) substitution tasks.  Offsets are element offsets into one RHS buffer
// holding every matrix's padded right-hand sides (column stride ldr of that matrix).
struct SDiag {          // diagonal block solve: L_jj, rows of block j
    const double *L;
    int64_t off, ldr;
};
struct SUpd {           // off-diagonal update of a 64-row chunk: dst -= op(L) src
    const double *L;    // tile (i, j) for forward, (j, i) for back substitution
    int64_t src, dst, ldr;
    int r0;             // chunk's first row inside the destination tile row
};
struct TEntry {         // triangular inverse of one diagonal tile: Y = L^{-1} (b x b, column-major)
    const double *L;
    double *Y;
};
void launch_trinv_batched(const TEntry *e, int n, int b, cudaStream_t s);
struct SRes {           // residual / |A| x of one 64-row chunk of one matrix
    const double *A;    // the matrix's tiles
    int64_t n;
    int nt, i, r0;
    int64_t xo, bo, ro, ldr;
};
struct SMax {           // column maxima of one matrix's block of a buffer
    int64_t off, ldr, n;
    int out;            // output index of column 0
};

// A matrix of a batch for the batched log-determinant / padding kernels.
struct LEntry {
    double *W;          // first tile of this matrix in the concatenated tile array
    int64_t n;
    int nt;
};

// Tensor-core update of one 128 x 256 block (bm, bn) of output tile (m, k) (k_mxp.cu).
struct QItem {
    double *C;          // output tile (m, k)
    int xoff, yoff;     // global packed index of tiles (m, 0) and (k, 0): sources are +n
    uint16_t bm, bn;
};

// Operand copy of packed tile `tile` in precision q (1 TF32 pair, 2 FP16, 3 FP8) into
// slot `slot` of that precision's pool.
struct CopyJob {
    int tile;
    int q;
    int slot;
};

// ------------------------------------------------------------------ launchers (k_fp64.cu)
void launch_dgemm_update(const DJob *jobs, const DItem *items, int nitems, int ld,
                         double *partials, const int *status, cudaStream_t s);
void launch_dgemm_reduce(const DRed *reds, int nreds, int ld, const double *partials,
                         const int *status, cudaStream_t s);
void launch_potrf_block(double *D, int ld, int col0, int *status, cudaStream_t s);
void launch_trsm_rows(double *P, const double *L, int ld, int rows, const int *status, cudaStream_t s);
void launch_potrf_blocks(const PEntry *e, int n, int ld, cudaStream_t s);
void launch_trsm_rows_batched(const PEntry *e, int n, int max_rows, int ld, cudaStream_t s);
void launch_trsm_strips(const TStrip *strips, int nstrips, int ld, int b, const int *status, cudaStream_t s);
void launch_logdet(const double *W, int nt, int b, int64_t n, double *out, cudaStream_t s);
void launch_fix_padding(double *W, int nt, int b, int64_t n, cudaStream_t s);
void launch_zero_upper_diag(double *W, int nt, int b, int64_t n, cudaStream_t s);
void launch_logdet_batched(const LEntry *e, int count, int b, double *out, cudaStream_t s);
void launch_fix_padding_batched(const LEntry *e, int count, int ntmax, int b, cudaStream_t s);

// tile-pointer variants (out-of-core executor)
void launch_dgemm_tile(const DJob &job, int ld, cudaStream_t s);
void launch_trsm_tile(double *C, const double *L, int ld, int b, const int *status, cudaStream_t s);
constexpr int TG_MAX = 16;   // tiles per grouped TRSM launch

// Function attributes (dynamic shared-memory opt-in) are per device.  attrs_pending() stays
// true for the current device until mark_attrs_set() records it (one bit per device ordinal),
// so a host thread never launches before the attributes are in place: two threads may both
// set them once, which is harmless.
inline unsigned long long device_bit() {
    int dev = 0;
    cudaGetDevice(&dev);
    return 1ull << (dev & 63);
}
inline bool attrs_pending(const std::atomic<unsigned long long> &mask) {
    return !(mask.load(std::memory_order_acquire) & device_bit());
}
inline void mark_attrs_set(std::atomic<unsigned long long> &mask) {
    mask.fetch_or(device_bit(), std::memory_order_release);
}
void launch_trinv(const double *L, int b, double *Y, cudaStream_t s);   // Y = L^{-1}, b x b
void launch_trsm_group(double *const *C, int ntiles, const double *L, int ld, int b, const int *status,
                       cudaStream_t s);
void launch_logdiag_tile(const double *D, int b, int nv, double *out, cudaStream_t s);
void launch_fix_padding_tile(double *T, int b, int nv, int diag, cudaStream_t s);
void launch_fwd_update_tile(const double *L, int b, int i, int j, double *R, int64_t ldr, int nrhs, cudaStream_t s);
void launch_bwd_update_tile(const double *L, int b, int i, int j, double *R, int64_t ldr, int nrhs, cudaStream_t s);

// solves (column-major right-hand sides, leading dimension ldr, nrhs <= 16 per launch)
void launch_fwd_diag(const double *Ljj, int b, double *R, int64_t ldr, int nrhs, cudaStream_t s);
void launch_fwd_update(const double *W, int nt, int b, int j, double *R, int64_t ldr, int nrhs, cudaStream_t s);
void launch_bwd_diag(const double *Ljj, int b, double *R, int64_t ldr, int nrhs, cudaStream_t s);
void launch_bwd_update(const double *W, int nt, int b, int j, double *R, int64_t ldr, int nrhs, cudaStream_t s);
void launch_symv_resid(const double *A, int nt, int b, int64_t n, const double *X, int64_t ldx,
                       const double *B, int64_t ldb, double *R, int64_t ldr, int nrhs, int absmode,
                       cudaStream_t s);
void launch_colmax_abs(const double *V, int64_t ld, int64_t n, int ncols, double *out, cudaStream_t s);
void launch_axpy_cols(double *X, int64_t ldx, const double *D, int64_t ldd, int64_t n, int ncols, cudaStream_t s);
void launch_dot_self(const double *v, int64_t n, double *out, cudaStream_t s);
void launch_dot(const double *u, const double *v, int64_t n, double *out, cudaStream_t s);
void launch_fwd_diag_g(const SDiag *e, int ne, double *R, int b, int nrhs, cudaStream_t s);
// FP32 forms (correction solves of a refined batched solve; factor tiles read in FP64)
void launch_fwd_diag_gf(const SDiag *e, int ne, float *R, int b, int nrhs, cudaStream_t s);
void launch_fwd_update_gf(const SUpd *u, int nu, float *R, int b, int nrhs, cudaStream_t s);
void launch_bwd_diag_gf(const SDiag *e, int ne, float *R, int b, int nrhs, cudaStream_t s);
void launch_bwd_update_gf(const SUpd *u, int nu, float *R, int b, int nrhs, cudaStream_t s);
void launch_to_f32(const double *x, float *y, int64_t n, cudaStream_t s);
void launch_add_f32(double *x, const float *d, int64_t n, int assign, cudaStream_t s);   // x (+)= d
void launch_fwd_update_g(const SUpd *u, int nu, double *R, int b, int nrhs, cudaStream_t s);
void launch_bwd_diag_g(const SDiag *e, int ne, double *R, int b, int nrhs, cudaStream_t s);
void launch_bwd_update_g(const SUpd *u, int nu, double *R, int b, int nrhs, cudaStream_t s);
void launch_symv_g(const SRes *r, int nr, int b, const double *X, const double *B, double *R, int nrhs, int absmode,
                   cudaStream_t s);
void launch_colmax_g(const SMax *m, int nm, const double *V, int nrhs, double *out, cudaStream_t s);
void launch_axpy_flat(double *X, const double *D, int64_t count, cudaStream_t s);
void launch_dots_g(const SMax *m, int nm, const double *u, const double *v, double *out, cudaStream_t s);

// ------------------------------------------------------------------ launchers (k_gen.cu)
void launch_matern(double *A, int64_t n, int b, int nt, const double *pts, double sigma2,
                   double a, int nu2, double nu, double nugget, cudaStream_t s);
void launch_tile_sumsq(const double *A, int nt, int b, int64_t n, double *out, cudaStream_t s);
// tiles t0 .. t0+count-1 of the packed layout, the first of them at A_first
void launch_tile_sumsq_range(const double *A_first, int t0, int count, int b, int64_t n, double *out, cudaStream_t s);

// Emulated-FP64 update of one 128 x Z_BN block of an FP64 or FP32 output tile (k_ozaki.cu).
struct ZItem {
    double *C;
    int xoff, yoff;
    uint16_t bm, bn;
    int ct = -1;        // global index of the output tile (plane counts relative to its scale)
};

// One grouped out-of-core update launch: tiles C[t] -= sum_{n<k} X_{t,n} Y_n^T, the operands
// given by digit-pool slot (ZG_MAX tiles and ZK_MAX sources at most per launch).
constexpr int ZG_MAX = 16, ZK_MAX = 256;
// CTAs (x dimension) per listed tile for the per-tile conversion kernels (grid-stride loops):
// about two full waves of 256-thread CTAs over the 152 SMs whatever the number of tiles, at
// least 64 per tile
inline int tile_ctas(int ntiles) {
    const int c = ntiles > 0 ? 2432 / ntiles : 64;
    return c < 64 ? 64 : (c > 1024 ? 1024 : c);
}
constexpr int Z_BN = 16;     // columns of one emulated-update work item (rows: 128)
constexpr int Z64_BN = 64;   // columns of a work item of the mixed-precision update kernel (k_ozaki64.cu)
// 3D maps over the digit-plane pool (K bytes, rows of a plane, plane index) for k_zgemm64:
// x[d-1] boxes of d X planes (128 rows), y[d-1] boxes of d Y planes (64 rows)
struct Z64Maps {
    CUtensorMap x[2];
    CUtensorMap y[5];
};
// Digit planes of the correction product R L^{-T} of the refined TRSM.  Truncation is
// relative to each operand's largest entry, so a product's relative error is amplified by
// A ~ K max|C| max|L^{-1}| / |X| (cancellation; A ~ 200 on Matern tiles).  X0 = C L^{-T} and
// the residual R = C - X0 L^T keep all 14 planes (R ~ 2^-54 A |C|); the correction's own
// truncation then adds ~2^-28 A |R| ~ 2^-82 A^2 |X|, far below FP64 rounding.  (X0 on 7
// planes as well gave 2^-56 A^2 = 6.6e-13 backward error: measured, and rejected.)
constexpr int ZREF_PLANES = 7;
// Digit planes of the TRSM product L_mk = C_mk L_kk^{-T} for a tile stored in precision p
// (FP64, FP32, FP16, FP8): truncation 16^-planes of the tile scale, amplified by A ~ 2^8,
// stays below the rounding to the stored format (2^-32 < 2^-24, 2^-16 < 2^-11, 2^-8 < 2^-4).
constexpr int ZTRSM_PLANES[4] = {14, 10, 6, 4};
constexpr int QG_MAX = 16, QK_MAX = 256;
struct ZGroup {
    int ntiles = 0, k = 0;
    int assign = 0;             // 0: C -= sum X Y^T;  1: C = sum X Y^T
    double *C[ZG_MAX];
    int lower[ZG_MAX] = {};
    int xs[ZG_MAX][ZK_MAX];
    int ys[ZK_MAX];
};
// The same for the FP16 / FP8 tensor-core updates (operand copies by cache slot).
struct QGroup {
    int ntiles = 0, k = 0;
    double *C[QG_MAX];
    int xs[QG_MAX][QK_MAX];
    int ys[QK_MAX];
};
void launch_copy_slot(const double *pool, int b, int slot, int q, const double *amaxS, __half *p16, uint8_t *p8,
                      int *e16, int *e8, cudaStream_t s);
void launch_round_slot(double *T, int b, int p, const double *amaxL, int *e_out, cudaStream_t s);
void launch_pack_compact(const double *T, int b, int p, const int *e, void *dst, cudaStream_t s);
void launch_unpack_compact(const void *src, int b, int p, const int *e, double *T, cudaStream_t s);
void launch_qgemm_group(int kind, const CUtensorMap &mx, const CUtensorMap &my, const QGroup &g, const int *exps,
                        int b, int *err, cudaStream_t s, unsigned long long limit_ns = 0, int stall = 0);

// ------------------------------------------------------------------ launchers (k_ozaki.cu)
size_t zgemm_smem_bytes();
void launch_digits(const double *W, int b, const int *tiles, int ntiles, const double *amax, uint8_t *pool, int *exps,
                   cudaStream_t s, const double *alt = nullptr);
void launch_lower_only(double *T, int b, cudaStream_t s);
void launch_add_tiles(double *W, int b, const int *tiles, int ntiles, const double *src, cudaStream_t s);
void launch_add_tile(double *dst, const double *src, int b, cudaStream_t s);     // dst += src, one b x b tile
// planes: digit planes of the output precision (14 FP64, 10 FP32, fewer for TRSM products);
// src_planes_tab: per digit slot, the leading planes that can be non-zero (nullptr: all);
// limit_ns: bound of each pipeline wait (0: 4 s), after which *err is set and the call ends;
// stall != 0: the failure-detection test hook (the MMA issuer waits on a barrier nothing arrives at).
// Plane counts of a mixed-precision update launch (k_zgemm's SKIP form): per source, the X / Y
// planes its stored formats can have non-zero (src_planes_tab), and a pair budget relative to
// the output tile's scale: su = rref - floor((e_out - e_x - e_y - 4 margin) / 4), within
// [1, 14], e_out the digit exponent of the output tile's input amax (out_amax[it.ct]).  The
// launch adds the plane pairs it multiplies to *pair_count.
struct ZPlanes {
    const uint8_t *src_planes_tab = nullptr;
    const double *out_amax = nullptr;
    int rref = 14, margin = 2;
    unsigned long long *pair_count = nullptr;
};
void launch_zgemm(const CUtensorMap &mx, const CUtensorMap &my, const ZItem *items, int nitems, const int *exps, int k,
                  int b, int *err, cudaStream_t s, int planes = 14, int assign = 0,
                  const ZPlanes *mixed = nullptr, unsigned long long limit_ns = 0, int stall = 0);
void launch_zgemm_group(const CUtensorMap &mx, const CUtensorMap &my, const ZGroup &g, const int *exps, int b,
                        int *err, cudaStream_t s, int planes = 14, unsigned long long limit_ns = 0, int stall = 0);
void launch_digits_src(const double *src, int b, int transpose, int dst, const double *amax, uint8_t *pool, int *exps,
                       cudaStream_t s);
void launch_amax_ptr(const double *src, int64_t count, double *out, cudaStream_t s);
void launch_set_identity(double *T, int b, cudaStream_t s);
int make_digit_map(CUtensorMap *map, void *pool, int64_t rows, int b, int box_rows);

// ------------------------------------------------------------------ launchers (k_mxp.cu)
int make_pool_map(CUtensorMap *map, void *pool, int64_t nslots, int b, int esize, int box_rows);
int make_pool_map_k(CUtensorMap *map, void *pool, int64_t nslots, int b, int esize, int box_rows, int box_k_bytes);
// 3D map over nplanes byte planes of b x b (row-major, K innermost): box 128 bytes x box_rows x depth
int make_plane_map3(CUtensorMap *map, void *pool, int64_t nplanes, int b, int box_rows, int depth);
int make_zgemm64_maps(Z64Maps *m, void *pool, int64_t nplanes, int b);
// Mixed-precision digit-plane updates over 128 x Z64_BN items (k_ozaki64.cu); mixed.rref is the
// reference plane count of the outputs (14 FP64, 10 FP32)
void launch_zgemm64(const Z64Maps &maps, const ZItem *items, int nitems, const int *exps, int k, int b, int *err,
                    cudaStream_t s, const ZPlanes &mixed, int assign, unsigned long long limit_ns, int stall);
size_t qgemm_smem_bytes();
void launch_qgemm(int kind, const CUtensorMap &a0, const CUtensorMap &a1, const CUtensorMap &b0,
                  const CUtensorMap &b1, const QItem *items, int nitems, const int *slot, const int *exps,
                  int k, int b, int *err, cudaStream_t s, unsigned long long limit_ns = 0, int stall = 0);
void launch_tile_amax(const double *W, int b, const int *tiles, int ntiles, double *amax, cudaStream_t s,
                      const double *alt = nullptr);
void launch_store_round(double *W, int b, const int *tiles, int ntiles, const uint8_t *prec, const double *amaxL,
                        double *amaxS, cudaStream_t s);
void launch_make_copies(const double *W, int b, const CopyJob *jobs, int njobs, const double *amaxS, float *hi,
                        float *lo, __half *p16, uint8_t *p8, int *e16, int *e8, cudaStream_t s);

}  // namespace tc
