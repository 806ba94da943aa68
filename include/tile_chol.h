/*
 * tile_chol -- mixed-precision left-looking tile Cholesky for one GB300 (sm_103a).
 *
 * C ABI.  Every entry point returns an int status: TC_OK (0), a negative TC_ERR_*
 * code, or a positive value: the 1-based global column at which the factorization met
 * a pivot that was not positive (the matrix is not numerically SPD; LAPACK's "info"
 * convention -- the paper does not define failure).  No exception or abort crosses
 * this boundary; after TC_ERR_CUDA the message is available from tc_last_error().
 *
 * Problem (arXiv 2410.09819, Section III-A): A = L L^T for a symmetric positive
 * definite n x n matrix A, by the left-looking tile algorithm of Algorithm 1, with a
 * per-tile precision map (Section IV-C) and out-of-core tile caching (Section IV-B,
 * Algorithms 2 and 3) when the matrix does not fit the device.
 *
 * Tile layout ("lower tile-major"), used for every matrix argument named *_tiles:
 *   b = tile size (a multiple of 64, 64 <= b <= 4096), Nt = ceil(n / b),
 *   T = Nt (Nt + 1) / 2 tiles;
 *   tile (i, j), i >= j, starts at element (i (i + 1) / 2 + j) * b * b;
 *   inside a tile, element (r, c) is at c * b + r (column-major, leading dimension b).
 *   Only lower tiles are stored.  Diagonal tiles hold the full b x b symmetric block.
 *   When n is not a multiple of b, the rows and columns of the last tile row/column
 *   beyond n are padding: the library ignores what the caller stores there and treats
 *   the padded matrix as diag(A, I), which leaves L and log|A| unchanged.
 *
 * Memory: a pointer argument may be host or device memory unless stated otherwise;
 * the library asks the CUDA runtime which it is.  Host buffers are best page-locked
 * (cudaHostAlloc); pageable memory works but copies slower.  The caller keeps
 * ownership of every buffer it passes.  The handle owns its device workspace (the
 * factor, the per-precision operand copies, the out-of-core tile cache) and its
 * streams; it is released by tc_destroy().
 *
 * Streams and threads: all device work of a handle runs on the stream given in
 * tc_config.stream (or one the handle creates), plus internal copy streams that
 * synchronise with it through events.  Calls return after the work they start has
 * completed unless stated otherwise.  A handle must not be used by two host threads
 * at once.
 */
#ifndef TILE_CHOL_H
#define TILE_CHOL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Tile precision codes used in precision maps (Section IV-C, Fig. 4). */
enum { TC_FP64 = 0, TC_FP32 = 1, TC_FP16 = 2, TC_FP8 = 3 };

/* Status codes. */
enum {
    TC_OK = 0,
    TC_ERR_ARG = -1,        /* an argument is out of range or NULL where not allowed */
    TC_ERR_STATE = -2,      /* call order: e.g. solve before a successful factor */
    TC_ERR_CUDA = -100,     /* a CUDA call failed; see tc_last_error() */
    TC_ERR_OOM = -101,      /* device memory (or the configured cache cap) too small */
    TC_ERR_TIMEOUT = -102,  /* a bounded device-side wait gave up */
    TC_ERR_HOSTMEM = -103,  /* page-locked host memory could not be allocated */
    TC_ERR_UNSUPPORTED = -104 /* a configuration this build does not provide */
};

typedef struct tc_handle_s *tc_handle;

/* Handle configuration.  Fill with tc_config_default() and override fields. */
typedef struct {
    int device;                 /* CUDA device ordinal (default 0) */
    void *stream;               /* cudaStream_t to run on; NULL: the handle makes one */
    int ooc;                    /* tile_chol_factor_ooc scheduling policy (Section III-C):
                                   0 V3 (default): accumulators resident through their
                                     updates, operand tiles cached (LRU), L_kk pinned until
                                     its column's TRSMs are done;
                                   1 V2: as V3 without the L_kk pin;
                                   2 V1: accumulators resident, no operand reuse;
                                   3 async: no reuse at all; every update step loads its
                                     accumulator and copies it back;
                                   4 sync: as async with every copy on the compute stream
                                     (no copy / compute overlap).
                                   Other values: TC_ERR_ARG. */
    int64_t device_cap_bytes;   /* tile_chol_factor_ooc: device tile-cache cap in bytes;
                                   0: free device memory minus 4 GiB */
    int prefetch_depth;         /* reserved: tile_chol_factor_ooc enqueues its whole static
                                   schedule, so copies run ahead as far as free slots allow */
    int lookahead;              /* reserved */
    int fp64_mode;              /* how SYRK/GEMM updates of FP64 (and FP32) output tiles run:
                                   0: FP64 tiles on the FP64 pipe (DFMA), FP32 tiles as
                                      3 x TF32 tensor-core products;
                                   1: both on the FP8 tensor cores through exact base-16
                                      digit planes of every final tile (14 planes for FP64
                                      outputs: normwise FP64 accuracy; 10 for FP32 outputs:
                                      below 2^-40 of the tile scale); needs 14 b^2 extra
                                      bytes per lower tile and a tile size multiple of 128;
                                   2: as 1, and the TRSMs of a one-matrix factorization
                                      (in core or out of core) run on the emulated engine as
                                      products with L_kk^{-1} (from FP64 substitution):
                                      low-precision tiles as L_mk = C_mk L_kk^{-T}, whose
                                      error kappa(L_kk) u is far below their accuracy
                                      level; FP64 tiles with one refinement step,
                                      X0 = C L^{-T}, L_mk = X0 + (C - X0 L^T) L^{-T}, which
                                      keeps the backward error at substitution's level */
    int ooc_eviction;           /* tile_chol_factor_ooc eviction rule: 0 least recently used
                                   (default); 1 Belady's MIN: the static schedule's whole
                                   request sequence is known before the first copy, so the
                                   unpinned tile whose next use lies farthest ahead leaves
                                   (the offline optimum for the copy count).  Other values:
                                   TC_ERR_ARG. */
    int fp32_updates;           /* with fp64_mode >= 1, how FP32 output tiles are updated:
                                   0 (default): 10 digit planes on the FP8 tensor cores
                                   (truncation below 2^-40 of the tile scale, FP64 sums);
                                   1: 3 x TF32 tensor-core products with FP32 accumulation
                                   (as with fp64_mode 0: FP32-level arithmetic, the
                                   paper's FP32 tiles).  Other values: TC_ERR_ARG. */
    int wait_limit_us;          /* bound, in microseconds, of every wait inside the
                                   tensor-core update kernels (a pipeline stage that does not
                                   arrive in time); 0 (default): 4 s.  When a wait runs out the
                                   kernel stops issuing, lets its own copies and MMAs finish,
                                   releases its tensor memory and returns; the call then
                                   returns TC_ERR_TIMEOUT and the handle stays usable.
                                   Negative: TC_ERR_ARG. */
    int wait_test;              /* failure-detection test hook, 0 for normal use.  Non-zero: the
                                   MMA issuer of every tensor-core update kernel first waits
                                   on a barrier that no thread arrives at, so each launch runs
                                   into its wait bound (pair it with a short wait_limit_us) and
                                   the call returns TC_ERR_TIMEOUT.  Nothing faults or hangs:
                                   the kernels take their normal teardown. */
    int reserved[3];
} tc_config;

/* Per-call statistics (any field a call does not produce is left 0). */
typedef struct {
    double t_ms;                /* wall time of the call, device-synchronised */
    double flops;               /* n^3/3, the algorithmic count of the factorization */
    double update_flops[4];     /* SYRK/GEMM flops executed per output precision */
    double trsm_flops, potrf_flops;
    int64_t tiles[4];           /* lower off-diagonal + diagonal tiles per precision */
    int64_t h2d_bytes, d2h_bytes;           /* out-of-core host<->device traffic */
    int64_t cache_hits, cache_misses, evictions;
    int64_t kernel_launches;    /* kernels this call launched */
    int refine_iters;           /* solve: refinement steps taken */
    double berr;                /* solve: final normwise backward error (max over RHS) */
    int info;                   /* same as the return value for factor calls */
    int ooc;                    /* 1 if the call ran out-of-core */
    /* device time (CUDA events on the launching stream) spent in the SYRK/GEMM update
       launches of each output precision, in the POTRF and TRSM launches, and in the
       down-cast / operand-copy launches of the factorization */
    double t_update_ms[4];
    double t_potrf_ms, t_trsm_ms, t_convert_ms;
    int64_t update_launches[4];
    /* tensor-core work the updates of each output precision executed (in-core factor): on
       digit planes (FP64 / FP32 outputs), 2 x rows x cols x K per plane pair multiplied, the
       planes that a stored tile cannot have non-zero skipped; TF32 x 3: three passes; FP16 /
       FP8: equal to update_flops.  0 for the FP64 pipe (fp64_mode 0). */
    double tensor_flops[4];
} tc_stats;

/* Defaults: device 0, own stream, cap 0 (auto), prefetch 2, lookahead 1. */
void tc_config_default(tc_config *cfg);

/* Create a handle on cfg->device.  cfg may be NULL (defaults).  *out is set on TC_OK.
 * TC_ERR_ARG: fp64_mode outside 0..2, fp32_updates outside 0..1 or wait_limit_us < 0.  (Out of core, FP32
 * output tiles always take the digit-plane path.) */
int tc_create(tc_handle *out, const tc_config *cfg);

/* Release every device and host resource of the handle (NULL is allowed). */
void tc_destroy(tc_handle h);

/* Message of the last failing call of this handle ("" if none).  Owned by the handle. */
const char *tc_last_error(tc_handle h);

/* Change the handle's cfg.wait_limit_us (bound of each wait in the tensor-core update
 * kernels, microseconds; 0: the 4 s default) and cfg.wait_test (the failure-detection test
 * hook, 0 for normal use) for its later calls, so that a caller can shorten the waits for a
 * watchdog, or test the timeout path, and then restore them on the same handle.  The paper
 * has no counterpart (it does not discuss failure detection).  TC_ERR_ARG for a NULL handle
 * or a negative limit. */
int tc_set_wait_limit(tc_handle h, int wait_limit_us, int wait_test);

/*
 * Synthetic covariance, Eq. 2 (Section III-D): writes the lower tiles of
 *   Sigma_ij = sigma2 / (2^(nu-1) Gamma(nu)) (h/a)^nu K_nu(h/a) + nugget [i == j],
 * h = |s_i - s_j|, x = h/a.  nu in {0.5, 1.5, 2.5} takes the closed forms e^-x, (1+x)e^-x,
 * (1+x+x^2/3)e^-x; any other nu in (0, 16] evaluates K_nu on the device (Temme's series for
 * x <= 2, Temme's normalising sum with Miller's backward recurrence above, then the upward
 * recurrence in nu; relative error a few units of 1e-15).  points: n x 2 row-major doubles
 * (x_i, y_i).  A_tiles: output, T b*b doubles in the tile layout above (padding set to
 * identity).
 * Errors: TC_ERR_ARG for n < 1, b not in [64, 4096] or not a multiple of 64, more than
 * 65535 lower tiles (Nt > 361), a <= 0, sigma2 <= 0 or nu outside (0, 16].
 */
int tc_matern_tiles(tc_handle h, int64_t n, int b, const double *points,
                    double sigma2, double range_a, double nu, double nugget,
                    double *A_tiles);

/*
 * Per-tile precision map, Section IV-C: tile (i, j), i > j, gets the lowest format p
 * in the allowed set with  Nt ||A_ij||_F / ||A||_F < eps_high / u_p,  where u_p is the
 * unit roundoff of p (FP32 2^-24, FP16 2^-11, FP8 E4M3 2^-4) and ||A||_F is taken over
 * the full symmetric matrix; otherwise FP64.  Diagonal tiles and tiles with
 * 1 <= i - j <= band stay FP64.  prec_set 1..4 allows {64}, {64,32}, {64,32,16},
 * {64,32,16,8} (Fig. 4).  Norms are FP64, computed on the device from A_tiles.
 * map_out: host or device, Nt*Nt bytes, row-major, entries TC_FP* (upper part 0).
 * norms_out: optional (NULL allowed), Nt*Nt doubles (tile Frobenius norms, lower part)
 * followed by one double ||A||_F.
 */
int tile_chol_precision_map(tc_handle h, int64_t n, int b, const double *A_tiles,
                            double eps_high, int band, int prec_set,
                            uint8_t *map_out, double *norms_out);

/*
 * Factor A = L L^T (Algorithm 1, left-looking, per-tile precision).
 * A_tiles: the caller's matrix in the tile layout, host or device; it is read, never
 *   written, and must stay valid (unchanged) until the handle's next factor or
 *   destroy, because tile_chol_solve's refinement reads it.
 * map: NULL for all-FP64, else Nt*Nt bytes (host or device) as produced by
 *   tile_chol_precision_map; the diagonal is treated as FP64 whatever it holds.
 *   Each update C_mk -= sum_{n<k} L_mn L_kn^T runs in the precision of its output
 *   tile p(m, k): operand tiles stored wider are rounded to it (RNE, fresh power-of-two
 *   scale for FP16/FP8), narrower ones are widened exactly.  FP16 and FP8 (E4M3)
 *   updates run on the tensor cores with FP32 accumulation.  FP64 and FP32 updates
 *   follow cfg.fp64_mode: with 0, FP64 on the DFMA pipe and FP32 as three TF32
 *   tensor-core products (hi*hi + hi*lo + lo*hi); with 1 or 2, both as exact products of
 *   base-16 digit planes on the E4M3 tensor cores (14 planes for FP64 outputs, 10 for
 *   FP32, or TF32 x 3 with cfg.fp32_updates = 1) with FP64 sums.  POTRF is FP64; the
 *   TRSM is FP64 substitution (modes 0, 1) or, in mode 2, products with L_kk^{-1} on the
 *   emulated engine (see fp64_mode).  Each final L_mk is then stored in p(m, k).
 * Runs in device memory: the handle holds a working copy of the factor (and, when
 *   A_tiles is host memory, a device copy of A); TC_ERR_OOM when that does not fit (use
 *   tile_chol_factor_ooc).
 * Returns TC_OK, a positive column (not SPD), or an error.  stats may be NULL.
 */
int tile_chol_factor(tc_handle h, int64_t n, int b, const double *A_tiles,
                     const uint8_t *map, tc_stats *stats);

/*
 * tile_chol_precision_map (Section IV-C) followed by tile_chol_factor (Algorithm 1) with
 * that map, on one device copy of A: a host A_tiles is copied once into the handle's device
 * copy (which the factor and tile_chol_solve's refinement then read), instead of once for
 * the map's tile norms and again for the factor.  A device A_tiles is used in place and
 * must stay valid as for tile_chol_factor.  The map and the factor are the ones the two
 * separate calls give.
 * map_out: host or device, Nt*Nt bytes (written, as tile_chol_precision_map).
 * stats: the factorization's, as tile_chol_factor (NULL allowed).
 * Returns as tile_chol_factor; TC_ERR_ARG for a NULL A_tiles or map_out, eps_high <= 0,
 * band < 0 or prec_set outside 1..4; TC_ERR_OOM when the device copy does not fit.
 */
int tile_chol_factor_mapped(tc_handle h, int64_t n, int b, const double *A_tiles,
                            double eps_high, int band, int prec_set, uint8_t *map_out,
                            tc_stats *stats);

/*
 * Out-of-core factorization (Sections III-C and IV-B, Algorithms 2 and 3): A_tiles is HOST
 * memory (best page-locked) holding A in the tile layout; on return it holds the factor L
 * (in place, as the paper's write-back does; upper triangles of diagonal tiles are left as
 * they were, or zeroed by fp64_mode 2; padding rows/columns as those of the identity).  The
 * device keeps a cache of at most cfg.device_cap_bytes of tiles (with fp64_mode >= 1 each
 * slot also holds the tile's 14 digit planes, and with a mixed map its FP16 / E4M3 operand
 * copies and a compact stage, so fewer tiles fit): a tile an update needs is reused when
 * cached, else copied in, evicting per cfg.ooc_eviction (least recently used, or Belady's
 * MIN) a tile that no pending task pins; under the default policy (cfg.ooc = V3) the
 * accumulator tile stays resident through its updates and L_kk until every TRSM of column
 * k is done.  The accumulators of a column are processed a group at a time.  Copies run on
 * their own streams, overlapped with the kernels.
 * map: NULL or all-FP64 with any fp64_mode; a mixed map needs fp64_mode >= 1
 * (TC_ERR_UNSUPPORTED otherwise).  Final low-precision tiles are written back both as FP64
 * (into A_tiles) and as a compact copy at their precision into a page-locked store the
 * handle owns (TC_ERR_HOSTMEM if it cannot be allocated); later loads of such a tile move
 * only the compact copy.
 * stats reports host<->device bytes, cache hits/misses/evictions.  Afterwards
 * tile_chol_solve / tile_chol_loglik stream the factor from A_tiles (no refinement: A is
 * gone) and tile_chol_logdet is available.  A_tiles must stay valid until then.
 * Returns TC_OK, a positive column (not SPD), or an error (TC_ERR_OOM: cache below 4
 * tiles or too small for the schedule).
 */
int tile_chol_factor_ooc(tc_handle h, int64_t n, int b, double *A_tiles, const uint8_t *map, tc_stats *stats);

/*
 * Solve A X = B with the last factor: forward (L Z = B) and back (L^T X = Z)
 * substitution in FP64, then up to max_refine steps of iterative refinement
 * R = B - A X (FP64, with the caller's A), X += solve(R), stopping once the normwise
 * backward error max_c ||R_c||_inf / (||A||_inf ||X_c||_inf + ||B_c||_inf) <= target_berr.
 * B, X: n x nrhs column-major with leading dimensions ldb, ldx >= n; host or device;
 * X may equal B.  Requires a successful tile_chol_factor (else TC_ERR_STATE).
 */
int tile_chol_solve(tc_handle h, int nrhs, const double *B, int64_t ldb,
                    double *X, int64_t ldx, int max_refine, double target_berr,
                    tc_stats *stats);

/* log|A| = 2 sum_i log L_ii of the last factor (needed by Eq. 1). */
int tile_chol_logdet(tc_handle h, double *logdet_out);

/*
 * Gaussian log-likelihood of Eq. 1 for the last factor:
 *   l = -n/2 log(2 pi) - 1/2 log|A| - 1/2 ||L^{-1} y||^2.
 * y: n doubles, host or device.  y == NULL evaluates Eq. 1 at y = 0 (the form used by
 * the KL divergence of Eq. 3).
 */
int tile_chol_loglik(tc_handle h, const double *y, double *loglik_out);

/*
 * Eq. 1 with the quadratic form taken from a refined solve: y^T Sigma^{-1} y = y^T x where
 * A x = y is solved as tile_chol_solve does (up to max_refine FP64 refinement steps until the
 * normwise backward error is <= target_berr), so a mixed-precision factor still gives the
 * quadratic term to FP64 accuracy; log|A| comes from the factor.  y: n doubles, host or
 * device.  berr_out (optional): the solve's final backward error.
 */
int tile_chol_loglik_refined(tc_handle h, const double *y, int max_refine, double target_berr,
                             double *loglik_out, double *berr_out);

/*
 * Eq. 1 with the quadratic form y^T Sigma^{-1} y = y^T x from a solution the caller already
 * has (x from tile_chol_solve of the same right-hand side y on the current factor: the
 * likelihood of Section III-D needs one solve, and this evaluates it without a second one);
 * log|A| comes from the factor.  y, x: n doubles each, host or device.  Returns TC_ERR_STATE
 * without a successful factorization, TC_ERR_ARG for null pointers.
 */
int tile_chol_loglik_solved(tc_handle h, const double *y, const double *x, double *loglik_out);

/*
 * Copy the last factor out as FP64 values of the stored tiles (tile layout; upper
 * triangles of diagonal tiles and padding are written as 0).  L_tiles: host or device.
 */
int tile_chol_get_factor(tc_handle h, double *L_tiles);

/*
 * Batched factorization of many independent SPD matrices sharing one tile size b (the
 * geospatial batched workload: uneven n, one map each).  Every column step of the
 * left-looking algorithm is one grouped launch over all matrices that have that column,
 * and the whole launch sequence is captured once into a CUDA graph and replayed while
 * the batch (count, n[], b, the A pointers and the maps) repeats.
 *   n[count]:        orders (each >= 1; ceil(n/b) <= 65535).
 *   A_tiles[count]:  pointers, each host or device memory, each in the tile layout of its n.
 *                    Read only; must stay valid until the handle's next factor or destroy.
 *   maps:            NULL (all FP64) or count pointers, each NULL or Nt_i*Nt_i bytes.
 *   info_out[count], logdet_out[count]: optional outputs per matrix (0 / log|A_i|).
 * Returns TC_OK, the info of the first failing matrix (> 0), or an error.  tile_chol_logdet
 * afterwards reports the first matrix; the *_batched solve/likelihood cover all of them.
 */
int tile_chol_factor_batched(tc_handle h, int count, const int64_t *n, int b, const double *const *A_tiles,
                             const uint8_t *const *maps, int *info_out, double *logdet_out, tc_stats *stats);

/*
 * Solve A_i X_i = B_i for every matrix of the last batched factorization, with up to
 * max_refine refinement steps (FP64 residuals with the caller's A_i, every matrix refined
 * together) until every normwise backward error is <= target_berr.  1 <= nrhs <= 16.
 * B[i], X[i]: n_i x nrhs column-major with leading dimension n_i, host or device.
 * berr_out[count] (optional): final backward errors.  Each substitution step is one grouped
 * launch over all matrices.
 */
int tile_chol_solve_batched(tc_handle h, int nrhs, const double *const *B, double *const *X, int max_refine,
                            double target_berr, double *berr_out, tc_stats *stats);

/* Copy the factor of matrix `index` of the last batched factorization out, as
 * tile_chol_get_factor does for a single one (tile layout of its n; upper triangles of
 * diagonal tiles and padding written as 0).  L_tiles: host or device.  TC_ERR_ARG for an
 * index outside the batch, TC_ERR_STATE without a successful in-core factorization. */
int tile_chol_get_factor_batched(tc_handle h, int index, double *L_tiles);

/* Eq. 1 for every matrix of the last batched factorization; y NULL: at y = 0; else y[i]
 * (n_i doubles, host or device).  loglik_out[count]. */
int tile_chol_loglik_batched(tc_handle h, const double *const *y, double *loglik_out);

/*
 * Precision map without any allocation (the paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code held to a fixed memory
 * budget or to a custom allocator that owns all device memory, real-time loops that cannot
 * afford an allocation's latency or failure).  Same map as tile_chol_precision_map, for the
 * current CUDA device, without a handle:
 *   A_tiles: device memory of the current device, the tile layout above (read only).
 *   map_out: device memory of the current device, Nt*Nt bytes, row-major (written, upper
 *            part TC_FP64 = 0).
 *   stream:  cudaStream_t to run on (NULL: the legacy default stream).  The call only
 *            enqueues work; it does not wait for it.
 * The per-tile sums of squares go to a fixed scratch array inside the library (263 KB,
 * held on every GPU that loads the library until the process exits), so the size is
 * limited to Nt = ceil(n / b) <= 256 tiles per column; larger problems get TC_ERR_ARG.
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The first call on a
 * device (and the first after a device reset) looks up the scratch array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All calls on a
 * device share the one scratch array, so calls whose GPU work overlaps (different streams,
 * no ordering) race and must be serialised by the caller.
 * Returns TC_OK; TC_ERR_ARG for sizes or arguments out of range and for buffers that are
 * not device memory of the current device; TC_ERR_CUDA when a launch fails, and, without
 * launching anything or clearing it, when the CUDA runtime already holds an error from
 * earlier work (cudaPeekAtLastError).
 */
int tile_chol_precision_map_noalloc(int64_t n, int b, const double *A_tiles, double eps_high, int band,
                                    int prec_set, uint8_t *map_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TILE_CHOL_H */
