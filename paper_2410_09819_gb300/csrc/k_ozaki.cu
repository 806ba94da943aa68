// FP64 tile updates emulated on the FP8 tensor cores (GB300's FP64 pipe delivers only
// ~1.25 TFLOP/s; its E4M3 tensor cores ~3.5 PFLOP/s).
//
// Splitting (the error-free slicing of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 2012, with a per-tile exponent):
// every final FP64 tile X with e = the smallest integer such that max|X| <= 2^e is written
// as X = 2^e sum_{s=1..S} 16^-s D_s + R with S = 14 integer "digit planes" D_s
// (D_1 in [-16, 16], the others in [-8, 8], |R| <= 2^(e-57)), each stored in E4M3, which
// holds these integers exactly.  Then
//     X Y^T = 2^(ex+ey) sum_{d=2..15} 16^-d G_d,   G_d = sum_{s+t=d} D_s(X) D_t(Y)^T,
// dropping the pairs with s + t > 15 (below 2^-54 of the product's scale).  Each G_d over one
// source tile (K <= 4096) is an integer below 2^24 in magnitude, so the tensor cores'
// FP32 accumulation is exact; the drain recombines the 14 groups with int64 Horner steps
// (exact) and adds 2^(ex+ey) (H1 16^-8 + H2 16^-15) to an FP64 running sum per element.
// The result is the FP64 update up to FP64-level rounding relative to the tiles' scale
// (a normwise bound, which is what the factorization's backward error needs).
#include "tc_internal.h"
#include "zgemm_common.h"

#include <cuda.h>
#include <cuda_fp8.h>

#include <cstring>

namespace tc {

constexpr int ZS = 14;                 // digit planes per tile
constexpr int ZBM = 128, ZBN = Z_BN;   // work item: 128 rows x 16 columns
constexpr int ZKB = 128;               // K bytes (= E4M3 elements) per stage
// Pipeline (shared memory: ZXS x ZXP x 16 KB + ZYS x 28 KB <= 227 KB).  The single MMA-issuing
// thread is the limit on GB300: a tcgen05.mma of N <= 128 occupies the tensor pipe for only ~69
// cycles, while each mbarrier wait in the issue stream leaves it idle for ~200-300 cycles, so X
// planes travel in stages of ZXP = 2 (one wait, one fence and one commit per two planes; +15-22 %
// over one plane per stage, measured for plane budgets 2..14).  Compile-time knobs for sweeps.
#ifndef ZGEMM_XS
#define ZGEMM_XS 5
#endif
#ifndef ZGEMM_YS
#define ZGEMM_YS 2
#endif
#ifndef ZGEMM_XP
#define ZGEMM_XP 2
#endif
constexpr int ZXS = ZGEMM_XS;          // X stages of ZXP planes
constexpr int ZYS = ZGEMM_YS;          // Y-set stages
constexpr int ZX_BYTES = ZBM * ZKB;    // 16 KB: one X plane block
constexpr int ZXP = ZGEMM_XP;          // X planes per stage
constexpr int ZXSTAGE = ZXP * ZX_BYTES;
constexpr int ZY_BYTES = ZBN * ZKB;    // 2 KB: one Y plane block
constexpr int ZYSET = ZS * ZY_BYTES;   // 28 KB: all Y planes of a K block
constexpr int ZTHREADS = 192;          // producer, MMA, 4 drain warps
constexpr unsigned long long ZLIMIT_NS = 4000000000ull;   // default bound of a pipeline wait
constexpr unsigned long long ZDRAIN_NS = 2000000000ull;   // bound of the teardown waits

// ------------------------------------------------------------------- digit planes
// Digits of one element in integer arithmetic (GB300 runs FP64 at 2 operations per clock per
// SM, so a floating-point x16 / rint / subtract chain would make this kernel ALU-bound):
// q = x 2^(56 - e) rounded to the nearest integer from the bit pattern (|q| <= 2^56 since
// |x| <= 2^e), then balanced base-16 digits from the least significant end: d_s in [-8, 8]
// for s >= 2, d_1 = what remains, in [-16, 16].  x 2^-e = sum_s d_s 16^-s + R 2^-e with
// |R| <= 2^(e - 57), the splitting the emulated products assume.
__device__ __forceinline__ long long fixed56(double x, int e) {
    const long long bits = __double_as_longlong(x);
    int ex = (int)((bits >> 52) & 0x7FF);
    long long m = bits & 0xFFFFFFFFFFFFFLL;
    if (ex == 0) ex = 1;                       // subnormal (or zero): no hidden bit
    else m |= 1LL << 52;                       // |x| = m 2^(ex - 1075)
    const int sh = ex - 1019 - e;              // x 2^(56 - e) = m 2^sh, sh <= 4
    long long q;
    if (sh >= 0) q = m << sh;
    else if (sh > -63) q = (m + (1LL << (-sh - 1))) >> (-sh);
    else q = 0;
    return bits < 0 ? -q : q;
}
// Four adjacent elements (columns 4j .. 4j+3 of a row): one 32-bit store per plane.
__device__ __forceinline__ uint32_t e4m3_digit(int d) {
    return (uint32_t)(uint8_t)__nv_cvt_float_to_fp8((float)d, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ void put_digits4(const long long (&q0)[4], uint8_t *P, int64_t o, int64_t bb) {
    long long q[4] = {q0[0], q0[1], q0[2], q0[3]};
#pragma unroll
    for (int s = ZS - 1; s >= 1; --s) {
        uint32_t w = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int r = (int)(q[u] & 15);
            if (r > 8) r -= 16;
            q[u] = (q[u] - r) >> 4;
            w |= e4m3_digit(r) << (8 * u);
        }
        *reinterpret_cast<uint32_t *>(P + (int64_t)s * bb + o) = w;
    }
    uint32_t w = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) w |= e4m3_digit((int)q[u]) << (8 * u);
    *reinterpret_cast<uint32_t *>(P + o) = w;
}

// exps[t] = smallest e with amax[t] <= 2^e; planes of tile t at pool + (t*ZS + s) b^2,
// each row-major (K-major) b x b.  The values come from tile t of W, or (alt != nullptr)
// from the blockIdx.y-th tile of the contiguous buffer alt.
__global__ void __launch_bounds__(256)
k_digits(const double *W, int b, const int *tiles, const double *amax, uint8_t *pool, int *exps, const double *alt) {
    __shared__ double S[32][33];
    const int t = tiles[blockIdx.y];
    const double *T = alt ? alt + (int64_t)blockIdx.y * b * b : W + (int64_t)t * b * b;
    const double am = amax[t];
    int e = 0;
    if (am > 0.0) {
        int ex;
        const double f = frexp(am, &ex);
        e = (f == 0.5) ? ex - 1 : ex;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) exps[t] = e;
    const int nbc = b / 32;
    const int64_t bb = (int64_t)b * b;
    uint8_t *P = pool + (int64_t)t * ZS * bb;
    for (int blk = blockIdx.x; blk < nbc * nbc; blk += gridDim.x) {
        const int r0 = (blk % nbc) * 32, c0 = (blk / nbc) * 32;
        __syncthreads();
        for (int idx = threadIdx.x; idx < 1024; idx += 256) {
            const int r = idx & 31, c = idx >> 5;
            S[r][c] = T[(int64_t)(c0 + c) * b + r0 + r];
        }
        __syncthreads();
        {   // 256 threads x 4 adjacent columns = the 32 x 32 block
            const int c = (threadIdx.x & 7) * 4, r = threadIdx.x >> 3;
            const long long q[4] = {fixed56(S[r][c], e), fixed56(S[r][c + 1], e), fixed56(S[r][c + 2], e),
                                    fixed56(S[r][c + 3], e)};
            put_digits4(q, P, (int64_t)(r0 + r) * b + c0 + c, bb);
        }
    }
}

// --------------------------------------------------------------------- update kernel
// Work items: one 128 x ZBN block (bm, bn) of one output tile.  The kernel is persistent:
// CTA c takes items c, c + gridDim.x, ...; every role walks the same item sequence.

// In-core form: item i is items[i]; its sources are the consecutive digit slots
// it.xoff + n and it.yoff + n.
struct ZArgs {
    const ZItem *items;
    int nitems;
    const int *exps;
    const uint8_t *planes;          // leading planes each digit slot can have non-zero (SKIP form)
    const double *oamax;            // SKIP form: input amax of every output tile, or nullptr
    int rref, margin;               // SKIP form: pair budget relative to the output's scale
    unsigned long long *pair_count; // SKIP form: plane pairs multiplied (added at the end)
    int k, b;
    int *err;
    int assign;         // 0: C -= sum X Y^T;  1: C = sum X Y^T
    unsigned long long limit_ns;    // bound of each pipeline wait
    int stall;                      // test hook: wait first on a barrier nothing arrives at
    __device__ int count() const { return nitems; }
    __device__ bool tile(int i, ZItem &it) const {
        it = items[i];
        return true;
    }
    __device__ int xsrc(const ZItem &it, int n) const { return it.xoff + n; }
    __device__ int ysrc(const ZItem &it, int n) const { return it.yoff + n; }
};

// Out-of-core form: up to ZG_MAX output tiles of one tile column, whose sources sit in
// arbitrary cache slots; the slot lists travel in the launch parameters.  Item i of the
// ntiles x (b/ZBM) x (b/ZBN) blocks; blocks entirely above the diagonal of a `lower` tile
// carry no work.
struct ZGroupArgs {
    double *C[ZG_MAX];
    uint16_t xs[ZG_MAX][ZK_MAX];   // X_n of tile g: digit slot xs[g][n]
    uint16_t ys[ZK_MAX];           // Y_n (shared by the group): digit slot ys[n]
    const int *exps;
    const uint8_t *planes;
    const double *oamax;
    int rref, margin;
    unsigned long long *pair_count;
    int k, b, ntiles;
    int *err;
    int assign;
    uint32_t lower;                // bit g: tile g is a diagonal tile
    unsigned long long limit_ns;
    int stall;
    __device__ int count() const { return ntiles * (b / ZBM) * (b / ZBN); }
    __device__ bool tile(int i, ZItem &it) const {
        const int nbm = b / ZBM, per = nbm * (b / ZBN);
        const int g = i / per, r = i % per;
        it.C = C[g];
        it.xoff = g;
        it.yoff = 0;
        it.bm = (uint16_t)(r % nbm);
        it.bn = (uint16_t)(r / nbm);
        return !(((lower >> g) & 1u) && it.bm * ZBM + ZBM - 1 < it.bn * ZBN);
    }
    __device__ int xsrc(const ZItem &it, int n) const { return xs[it.xoff][n]; }
    __device__ int ysrc(const ZItem &, int n) const { return ys[n]; }
};

// Order of the X planes within a K block: plane s meets 14 - s partner planes, so its MMA
// work falls from 14 units (s = 0) to 1 (s = 13); alternating long and short planes
// (0, SU-1, 1, SU-2, ...) keeps the work per 16 KB stage even, and the TMA ring never has to
// deliver the short planes' stages back to back.
template <int SU>
__device__ __forceinline__ int plane_order(int i) { return (i & 1) ? SU - 1 - (i >> 1) : (i >> 1); }
__device__ __forceinline__ int plane_order_n(int i, int S) { return (i & 1) ? S - 1 - (i >> 1) : (i >> 1); }

// Plane counts (SKIP form, mixed-precision updates): a source tile stored in FP8 (E4M3 with a
// power-of-two scale 2^e8) holds multiples of 2^(e8 - 9) below 2^(e8 + 9), so relative to its
// digit exponent at most 18 bits are set and digit planes 6..14 are zero; FP16 (scale 2^e16)
// holds multiples of 2^(e16 - 24) below 2^(e16 + 16): planes 11..14 are zero.  planes[slot]
// gives the leading planes that can be non-zero; the kernel multiplies only those, which
// changes no bit of the result (the skipped products are exact zeros).

// Plane counts of one source (SKIP form): SU_n, the budget of plane pairs s + t < SU_n, and the
// X / Y planes multiplied.  With out-of-scale truncation (oamax set), a pair whose scale
// 2^(e_x + e_y) lies d binary orders below the output tile's input scale 2^e_out drops
// floor((d - 4 margin) / 4) planes from the reference count rref: the terms it drops stay below
// 16^-margin of what the reference count drops for a pair at the output's own scale, and a pair
// above the output's scale keeps more planes (up to SU).  SU_n is rounded up to an even count
// and the plane counts to {5, 10, 14} (clipped to SU_n): the counts the issue code is unrolled
// for.  Rounding up only adds terms.
struct ZShape {
    int sx, sy, su;
};
template <int SU, class Args>
__device__ __forceinline__ ZShape z_shape(const Args &a, int eo, int xt, int yt) {
    int su = a.rref;
    if (a.oamax) {
        const int d = eo - a.exps[xt] - a.exps[yt] - 4 * a.margin;
        const int j = d >= 0 ? d / 4 : -((3 - d) / 4);        // floor(d / 4)
        su = a.rref - j;
    }
    su = su < 1 ? 1 : (su > SU ? SU : su);
    su = (su + 1) & ~1;
    if (su > SU) su = SU;
    const int px = a.planes[xt], py = a.planes[yt];
    int sx = px <= 5 ? 5 : (px <= 10 ? 10 : 14), sy = py <= 5 ? 5 : (py <= 10 ? 10 : 14);
    sx = sx < su ? sx : su;
    sy = sy < su ? sy : su;
    return {sx, sy, su};
}
__device__ __forceinline__ int z_pairs(const ZShape &z) {
    int p = 0;
    for (int s = 0; s < z.sx; ++s) p += z.sy < z.su - s ? z.sy : z.su - s;
    return p;
}

// Order of the X planes of one K block (producer and MMA issuer agree on it): interleaved
// long / short planes, except in the first K block of a source whose Y partners stop short of
// SU (SY < SU), which runs in ascending order so that every group is started by its own first
// MMA (see the SKIP note at k_zgemm).
__device__ __forceinline__ int plane_at(int i, int sx, int sy, int su, int kb) {
    return (sy < su && kb == 0) ? i : plane_order_n(i, sx);
}

// The MMAs of one K block for a source with SX X planes and SY Y planes (compile-time, fully
// unrolled: the single issuing thread must keep the tensor pipe fed).  Pairs (s, t) with
// s < SX, t < SY, s + t < SU; plane s multiplies its partners t = 0 .. min(SY, SU - s) - 1 in
// one MMA whose column block t lands on accumulator group s + t.  Returns false if a stage did
// not arrive within the wait bound.
template <int SU, int SX, int SY>
__device__ __forceinline__ bool z_issue_kblock(int kb, uint64_t xdesc_base, uint64_t yd, uint32_t dbase,
                                               uint64_t *xfull, uint64_t *xempty, int &xst, int &xph,
                                               volatile int *abort_flag, unsigned long long lim) {
    constexpr uint32_t idesc0 = (1u << 4) | ((uint32_t)(ZBM >> 4) << 24);
    const bool asc = SY < SU && kb == 0;
#pragma unroll
    for (int i0 = 0; i0 < SX; i0 += ZXP) {
        if (!z_wait(xfull + xst, xph, abort_flag, lim)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t xsd = xdesc_base + (uint64_t)((xst * ZXSTAGE) >> 4);
#pragma unroll
        for (int h = 0; h < ZXP; ++h)
            if (i0 + h < SX) {
                const int i = i0 + h;
                const int s = asc ? i : ((i & 1) ? SX - 1 - (i >> 1) : (i >> 1));
                const int np = SY < SU - s ? SY : SU - s;
                const uint64_t xd = xsd + (uint64_t)((h * ZX_BYTES) >> 4);
                const uint32_t idesc = idesc0 | ((uint32_t)((np * ZBN) >> 3) << 17);
                const uint32_t d = dbase + (uint32_t)(s * ZBN);
                if (kb > 0) {
                    z_mma4(d, xd, yd, idesc, 1u);
                } else if (s == 0) {
                    z_mma4(d, xd, yd, idesc, 0u);                   // starts groups 0 .. np-1
                } else if (asc && np == SY) {
                    // groups s .. s+np-2 are running; group s+np-1 starts here (K step 0)
                    if (np > 1) z_mma(d, xd, yd, idesc0 | ((uint32_t)(((np - 1) * ZBN) >> 3) << 17), 1u);
                    z_mma(d + (uint32_t)((np - 1) * ZBN), xd, yd + (uint64_t)(((np - 1) * ZY_BYTES) >> 4),
                          idesc0 | ((uint32_t)(ZBN >> 3) << 17), 0u);
                    z_mma3(d, xd, yd, idesc);
                } else {
                    z_mma4(d, xd, yd, idesc, 1u);                   // all its groups are running
                }
            }
        z_commit(xempty + xst);
        if (++xst == ZXS) { xst = 0; xph ^= 1; }
    }
    return true;
}

// Persistent update kernel: C -= sum_{n<k} X_n Y_n^T for 128 x ZBN output blocks, X_n the
// tiles (m, n) and Y_n the tiles (k, n), through their first SU digit planes (SU = 14 for
// FP64 outputs; SU = 10, i.e. pairs with s + t <= 11 and a truncation below 2^-40 of the tile
// scale, for FP32 outputs: with 8 planes the truncation, which is relative to the operand
// tile's largest entry, cost 50x in the factor's backward error at eps_high = 1e-9).
//   warp 0  TMA producer: per source and 128-byte K block, the SU Y planes of the block's ZBN
//           columns (back to back, one stage of the Y ring) and the SU X planes (two per stage
//           of the X ring), in the interleaved plane order;
//   warp 1  MMA issuer: per X plane s, one tcgen05.mma per 32-byte K step with N = ZBN (SU - s)
//           multiplies it by all its partners Y_0 .. Y_{SU-1-s} at once (the four K steps in one
//           asm block); column block t lands on accumulator group s + t, so the grouping by
//           weight comes from the TMEM address;
//   warps 2-5 drain: the SU group sums of a source leave TMEM (exact FP32 integers), are
//           recombined by int64 Horner steps and added, scaled by 2^(e_x + e_y), to FP64
//           running sums; C is written once per item.
// The accumulators are double-buffered in TMEM (2 x SU x ZBN <= 512 columns), so the drain
// of source q overlaps the MMAs of source q + 1, and the item stream never stops between
// items (no per-item prologue).
//
// SKIP (mixed-precision updates): a source multiplies only the SX X planes and SY Y planes its
// stored formats can have non-zero (pairs s < SX, t < SY, s + t < SU).  Plane 0 then starts
// groups 0 .. SY-1 only, so in the first K block the planes run in ascending order and plane
// s >= 1 starts the one group it reaches first (s + SY - 1) with a separate MMA for K step 0;
// every group the source writes is thus initialised by its own first MMA, and the drain reads
// only those (the others hold an earlier source's sums).
//
// Failure handling: every pipeline wait gives up after args.limit_ns (or when another role
// set the abort flag), and the CTA then sets *err and stops issuing.  Before the TMEM is
// released and the CTA exits, the MMA issuer waits for all of its issued MMAs and the
// producer for all of its issued copies; those waits ignore the abort flag (the operations
// depend on nothing outside the CTA, so they end) and are bounded by ZDRAIN_NS.
template <int SU, bool SKIP, class Args>
__global__ void __launch_bounds__(ZTHREADS, 1)
k_zgemm(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
        const __grid_constant__ Args args) {
    static_assert(SU <= ZS, "at most 14 digit planes");
    extern __shared__ __align__(1024) uint8_t zsmem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(zsmem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *xbuf = smem;                             // ZXS x 16 KB
    uint8_t *ybuf = smem + ZXS * ZXSTAGE;             // ZYS x (SU x ZBN rows x 128 B)
    uint64_t *xfull = reinterpret_cast<uint64_t *>(ybuf + ZYS * ZYSET);
    uint64_t *xempty = xfull + ZXS;
    uint64_t *yfull = xempty + ZXS;
    uint64_t *yempty = yfull + ZYS;
    uint64_t *accf = yempty + ZYS;                    // [2]
    uint64_t *acce = accf + 2;                        // [2]
    uint64_t *done = acce + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    volatile int *never = abort_flag + 1;             // nothing sets it: waits that must not be cut short
    const unsigned long long lim = args.limit_ns;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = args.k, b = args.b;
    const int kblocks = b / ZKB;
    const int nitems = args.count();
    if ((int)blockIdx.x >= nitems) return;             // whole CTA, before any barrier
    if (threadIdx.x == 0) {
        for (int s = 0; s < ZXS; ++s) {
            z_init(xfull + s, 1);
            z_init(xempty + s, 1);
        }
        for (int s = 0; s < ZYS; ++s) {
            z_init(yfull + s, 1);
            z_init(yempty + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            z_init(accf + a, 1);
            z_init(acce + a, 4);
        }
        z_init(done, 1);
        *abort_flag = 0;
        *never = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(z_smem(tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        // --------------------------------------------------------------- TMA producer
        if (lane == 0) {
            int xst = 0, xph = 1, yst = 0, yph = 1, issued_x = 0, issued_y = 0;   // empty slots: phase 1 passes
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                ZItem it;
                if (!args.tile(item, it)) continue;
                const int eo = (SKIP && args.oamax) ? z_digit_exp(args.oamax[it.ct]) : 0;
                for (int n = 0; n < k && ok; ++n) {
                    const int xt = args.xsrc(it, n), yt = args.ysrc(it, n);
                    const ZShape zs = SKIP ? z_shape<SU>(args, eo, xt, yt) : ZShape{SU, SU, SU};
                    const int sx = zs.sx, sy = zs.sy;
                    for (int kb = 0; kb < kblocks && ok; ++kb) {
                        if (!z_wait(yempty + yst, yph, abort_flag, lim)) { ok = false; break; }
                        z_expect(yfull + yst, sy * ZY_BYTES);
                        for (int t = 0; t < sy; ++t)
                            z_tma(ybuf + yst * ZYSET + t * ZY_BYTES, &mapY, kb * ZKB, (yt * ZS + t) * b + it.bn * ZBN,
                                  yfull + yst);
                        ++issued_y;
                        if (++yst == ZYS) { yst = 0; yph ^= 1; }
                        for (int i0 = 0; i0 < sx; i0 += ZXP) {
                            if (!z_wait(xempty + xst, xph, abort_flag, lim)) { ok = false; break; }
                            const int cnt = sx - i0 < ZXP ? sx - i0 : ZXP;
                            z_expect(xfull + xst, (uint32_t)(cnt * ZX_BYTES));
                            for (int h = 0; h < cnt; ++h) {
                                const int s = SKIP ? plane_at(i0 + h, sx, sy, zs.su, kb) : plane_order<SU>(i0 + h);
                                z_tma(xbuf + xst * ZXSTAGE + h * ZX_BYTES, &mapX, kb * ZKB, (xt * ZS + s) * b + it.bm * ZBM,
                                      xfull + xst);
                            }
                            ++issued_x;
                            if (++xst == ZXS) { xst = 0; xph ^= 1; }
                        }
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(args.err, 1);
            }
            // Every copy lands before the shared memory goes away, whichever role gave up and
            // whenever: only the last ZXS (ZYS) copies of a ring can still be in flight (each
            // earlier one was consumed before its stage was refilled), and each is the latest
            // phase of its stage's full barrier.  Without an abort they end as soon as those
            // copies land.
            for (int q = issued_x - ZXS < 0 ? 0 : issued_x - ZXS; q < issued_x; ++q)
                if (!z_wait(xfull + q % ZXS, (q / ZXS) & 1, never, ZDRAIN_NS)) atomicExch(args.err, 3);
            for (int q = issued_y - ZYS < 0 ? 0 : issued_y - ZYS; q < issued_y; ++q)
                if (!z_wait(yfull + q % ZYS, (q / ZYS) & 1, never, ZDRAIN_NS)) atomicExch(args.err, 3);
        }
    } else if (warp == 1) {
        // --------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            // kind::f8f6f4, D F32, A/B E4M3, K-major, M = 128; N set per instruction
            const uint32_t idesc0 = (1u << 4) | ((uint32_t)(ZBM >> 4) << 24);
            // shared-memory descriptors advance by 2 per 32-byte K step (address field in
            // 16-byte units); stage indices and phases run as counters (no division)
            const uint64_t xdesc_base = z_desc(z_smem(xbuf)), ydesc_base = z_desc(z_smem(ybuf));
            int xst = 0, xph = 0, yst = 0, yph = 0, q = 0;   // q: sources issued so far (all items)
            unsigned long long pairs_done = 0;
            bool ok = true;
            // test hook: `done` completes only after the final commit below, so this wait runs
            // into the bound and takes the abort path
            if (args.stall && !z_wait(done, 0, abort_flag, lim)) ok = false;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                ZItem it;
                if (!args.tile(item, it)) continue;
                const int eo = (SKIP && args.oamax) ? z_digit_exp(args.oamax[it.ct]) : 0;
                for (int n = 0; n < k && ok; ++n, ++q) {
                    const int a = q & 1;
                    if (!z_wait(acce + a, ((q >> 1) & 1) ^ 1, abort_flag, lim)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dbase = tmem + (uint32_t)(a * SU * ZBN);
                    const ZShape zs = SKIP ? z_shape<SU>(args, eo, args.xsrc(it, n), args.ysrc(it, n)) : ZShape{SU, SU, SU};
                    if (SKIP) pairs_done += (unsigned long long)z_pairs(zs);
                    for (int kb = 0; kb < kblocks && ok; ++kb) {
                        if (!z_wait(yfull + yst, yph, abort_flag, lim)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint64_t yd = ydesc_base + (uint64_t)((yst * ZYSET) >> 4);
                        if constexpr (!SKIP) {
                            // planes in stages of ZXP: one wait, one fence and one commit per stage
#pragma unroll
                            for (int i0 = 0; i0 < SU; i0 += ZXP) {
                                if (!z_wait(xfull + xst, xph, abort_flag, lim)) {
                                    ok = false;
                                    break;
                                }
                                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                                const uint64_t xsd = xdesc_base + (uint64_t)((xst * ZXSTAGE) >> 4);
#pragma unroll
                                for (int h = 0; h < ZXP; ++h)
                                    if (i0 + h < SU) {
                                        const int s = plane_order<SU>(i0 + h);
                                        const uint64_t xd = xsd + (uint64_t)((h * ZX_BYTES) >> 4);
                                        const uint32_t idesc = idesc0 | ((uint32_t)(((SU - s) * ZBN) >> 3) << 17);
                                        const uint32_t d = dbase + (uint32_t)(s * ZBN);
                                        // plane 0 comes first in every K block and covers all groups,
                                        // so it alone starts the accumulators of a source tile
                                        z_mma4(d, xd, yd, idesc, (kb > 0 || i0 + h > 0) ? 1u : 0u);
                                    }
                                z_commit(xempty + xst);
                                if (++xst == ZXS) { xst = 0; xph ^= 1; }
                            }
                        } else {
                            // dispatch on the source's plane budget and plane counts (z_shape's values)
                            bool r = false;
                            switch (zs.su * 256 + zs.sx * 16 + zs.sy) {
                            case 3669: r = z_issue_kblock<14, 5, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3674: r = z_issue_kblock<14, 5, 10>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3678: r = z_issue_kblock<14, 5, 14>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3749: r = z_issue_kblock<14, 10, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3754: r = z_issue_kblock<14, 10, 10>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3758: r = z_issue_kblock<14, 10, 14>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3813: r = z_issue_kblock<14, 14, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3818: r = z_issue_kblock<14, 14, 10>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3822: r = z_issue_kblock<14, 14, 14>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3157: r = z_issue_kblock<12, 5, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3162: r = z_issue_kblock<12, 5, 10>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3164: r = z_issue_kblock<12, 5, 12>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3237: r = z_issue_kblock<12, 10, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3242: r = z_issue_kblock<12, 10, 10>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3244: r = z_issue_kblock<12, 10, 12>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3269: r = z_issue_kblock<12, 12, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3274: r = z_issue_kblock<12, 12, 10>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 3276: r = z_issue_kblock<12, 12, 12>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 2645: r = z_issue_kblock<10, 5, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 2650: r = z_issue_kblock<10, 5, 10>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 2725: r = z_issue_kblock<10, 10, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 2730: r = z_issue_kblock<10, 10, 10>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 2133: r = z_issue_kblock<8, 5, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 2136: r = z_issue_kblock<8, 5, 8>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 2181: r = z_issue_kblock<8, 8, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 2184: r = z_issue_kblock<8, 8, 8>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 1621: r = z_issue_kblock<6, 5, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 1622: r = z_issue_kblock<6, 5, 6>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 1637: r = z_issue_kblock<6, 6, 5>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 1638: r = z_issue_kblock<6, 6, 6>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 1092: r = z_issue_kblock<4, 4, 4>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            case 546: r = z_issue_kblock<2, 2, 2>(kb, xdesc_base, yd, dbase, xfull, xempty, xst, xph, abort_flag, lim); break;
                            default: atomicExch(args.err, 2); break;   // not produced by z_shape
                            }
                            if (!r) ok = false;
                        }
                        if (!ok) break;
                        z_commit(yempty + yst);
                        if (++yst == ZYS) { yst = 0; yph ^= 1; }
                    }
                    if (ok) z_commit(accf + a);
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(args.err, 1);
            }
            if (SKIP && args.pair_count && pairs_done) atomicAdd(args.pair_count, pairs_done);
            // every issued MMA completes before the TMEM is released and the CTA exits
            z_commit(done);
            if (!z_wait(done, 0, never, ZDRAIN_NS)) atomicExch(args.err, 3);
        }
    } else {
        // --------------------------------------------------------------- drain + epilogue
        const int quarter = warp & 3;
        bool ok = true;
        int q = 0;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            ZItem it;
            if (!args.tile(item, it)) continue;
            const int eo = (SKIP && args.oamax) ? z_digit_exp(args.oamax[it.ct]) : 0;
            double run[ZBN];
#pragma unroll
            for (int j = 0; j < ZBN; ++j) run[j] = 0.0;
            for (int n = 0; n < k; ++n, ++q) {
                const int a = q & 1;
                if (!z_wait(accf + a, (q >> 1) & 1, abort_flag, lim)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int xt = args.xsrc(it, n), yt = args.ysrc(it, n);
                const int E = args.exps[xt] + args.exps[yt];
                // groups this source wrote (SKIP: the others hold an earlier source's sums)
                int G = SU;
                if constexpr (SKIP) {
                    const ZShape zs = z_shape<SU>(args, eo, xt, yt);
                    G = zs.sx + zs.sy - 1 < zs.su ? zs.sx + zs.sy - 1 : zs.su;
                }
                // hi holds groups 0 .. min(SU, 7) - 1, lo the rest (weights 16^-(g+2))
                const double s_hi = ldexp(1.0, E - 4 * ((SU < 7 ? SU : 7) + 1)), s_lo = ldexp(1.0, E - 4 * (SU + 1));
                const uint32_t lanebase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * SU * ZBN);
                long long hi[ZBN], lo[ZBN];
#pragma unroll
                for (int j = 0; j < ZBN; ++j) hi[j] = lo[j] = 0;
                for (int g = 0; g < G; ++g) {
                    float v[16];
                    z_ld16(lanebase + (uint32_t)(g * ZBN), v);
                    // group sums are exact integers below 2^24 in magnitude: a 32-bit
                    // conversion (a 64-bit one would run on the FP64 pipe)
                    if (g < 7) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) hi[j] = hi[j] * 16 + (long long)__float2int_rn(v[j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) lo[j] = lo[j] * 16 + (long long)__float2int_rn(v[j]);
                    }
                }
                // the accumulator buffer is free for source q + 2 once every lane has read it
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) z_arrive(acce + a);
                // groups G .. SU-1 are zero: the Horner steps they would take are shifts
                constexpr int NH = SU < 7 ? SU : 7;            // groups of hi
                if (G < SU) {
                    const long long m_hi = 1LL << (G < NH ? 4 * (NH - G) : 0);
                    const long long m_lo = 1LL << (G > NH ? 4 * (SU - G) : 0);
#pragma unroll
                    for (int j = 0; j < ZBN; ++j) {
                        hi[j] *= m_hi;
                        lo[j] *= m_lo;
                    }
                }
                if (G > NH) {
#pragma unroll
                    for (int j = 0; j < ZBN; ++j) run[j] = fma((double)lo[j], s_lo, fma((double)hi[j], s_hi, run[j]));
                } else {                                        // no lo groups: lo == 0
#pragma unroll
                    for (int j = 0; j < ZBN; ++j) run[j] = fma((double)hi[j], s_hi, run[j]);
                }
            }
            if (!ok) break;
            const int row = it.bm * ZBM + quarter * 32 + lane;
#pragma unroll
            for (int j = 0; j < ZBN; ++j) {
                double *c = it.C + (int64_t)(it.bn * ZBN + j) * b + row;
                *c = args.assign ? run[j] : *c - run[j];
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(args.err, 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}


// Digit planes of one b x b matrix at src (column-major; row-major when transpose != 0)
// into slot dst of the pool, exponent from *amax.
__global__ void __launch_bounds__(256)
k_digits_src(const double *src, int b, int transpose, int dst, const double *amax, uint8_t *pool, int *exps) {
    __shared__ double S[32][33];
    const double am = *amax;
    int e = 0;
    if (am > 0.0) {
        int ex;
        const double f = frexp(am, &ex);
        e = (f == 0.5) ? ex - 1 : ex;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) exps[dst] = e;
    const int nbc = b / 32;
    const int64_t bb = (int64_t)b * b;
    uint8_t *P = pool + (int64_t)dst * ZS * bb;
    for (int blk = blockIdx.x; blk < nbc * nbc; blk += gridDim.x) {
        const int r0 = (blk % nbc) * 32, c0 = (blk / nbc) * 32;
        __syncthreads();
        for (int idx = threadIdx.x; idx < 1024; idx += 256) {
            const int r = idx & 31, c = idx >> 5;
            S[r][c] = transpose ? src[(int64_t)(r0 + r) * b + c0 + c] : src[(int64_t)(c0 + c) * b + r0 + r];
        }
        __syncthreads();
        {   // 256 threads x 4 adjacent columns = the 32 x 32 block
            const int c = (threadIdx.x & 7) * 4, r = threadIdx.x >> 3;
            const long long q[4] = {fixed56(S[r][c], e), fixed56(S[r][c + 1], e), fixed56(S[r][c + 2], e),
                                    fixed56(S[r][c + 3], e)};
            put_digits4(q, P, (int64_t)(r0 + r) * b + c0 + c, bb);
        }
    }
}

// max |src[e]| as the largest sign-cleared bit pattern (non-negative doubles order like their
// bit patterns; integer maxima keep this off the FP64 pipe)
__global__ void k_amax_ptr(const double *src, int64_t count, double *out) {
    unsigned long long m = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(src[e]) & 0x7FFFFFFFFFFFFFFFull);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned long long *>(out), m);
}

// zero the strictly upper part of a column-major b x b tile (a factored diagonal tile as L_kk)
__global__ void k_lower_only(double *T, int b) {
    const int64_t bb = (int64_t)b * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bb; e += (int64_t)gridDim.x * blockDim.x)
        if (e % b < e / b) T[e] = 0.0;
}

// tile tiles[y] of W += the y-th tile of src
__global__ void k_add_tiles(double *W, int b, const int *tiles, const double *src) {
    const int64_t bb = (int64_t)b * b;
    double *T = W + (int64_t)tiles[blockIdx.y] * bb;
    const double *S = src + (int64_t)blockIdx.y * bb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bb; e += (int64_t)gridDim.x * blockDim.x)
        T[e] += S[e];
}

__global__ void k_set_identity(double *T, int b) {
    const int64_t bb = (int64_t)b * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bb; e += (int64_t)gridDim.x * blockDim.x)
        T[e] = (e % b == e / b) ? 1.0 : 0.0;
}

void launch_digits_src(const double *src, int b, int transpose, int dst, const double *amax, uint8_t *pool, int *exps,
                       cudaStream_t s) {
    const int blocks = (b / 32) * (b / 32);          // one 32 x 32 block per CTA pass, 4 CTAs per SM
    k_digits_src<<<blocks < 608 ? blocks : 608, 256, 0, s>>>(src, b, transpose, dst, amax, pool, exps);
}
void launch_amax_ptr(const double *src, int64_t count, double *out, cudaStream_t s) {
    const int64_t want = (count + 4095) / 4096;
    k_amax_ptr<<<want < 608 ? (int)want : 608, 256, 0, s>>>(src, count, out);
}
void launch_set_identity(double *T, int b, cudaStream_t s) { k_set_identity<<<64, 256, 0, s>>>(T, b); }

// ------------------------------------------------------------------------- host side
// map over the digit pool: rows = tiles * 14 * b, b bytes each; box 128 bytes x box_rows
int make_digit_map(CUtensorMap *map, void *pool, int64_t rows, int b, int box_rows) {
    return make_pool_map(map, pool, rows / b, b, 1, box_rows);
}

size_t zgemm_smem_bytes() { return (size_t)ZXS * ZXSTAGE + ZYS * ZYSET + 1024 + 256; }

static int sm_count() {            // per device, cached
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int> &c = cache[dev & 63];
    int n = c.load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        c.store(n, std::memory_order_relaxed);
    }
    return n;
}

void launch_digits(const double *W, int b, const int *tiles, int ntiles, const double *amax, uint8_t *pool, int *exps,
                   cudaStream_t s, const double *alt) {
    if (ntiles > 0) k_digits<<<dim3(tile_ctas(ntiles), ntiles), 256, 0, s>>>(W, b, tiles, amax, pool, exps, alt);
}
void launch_lower_only(double *T, int b, cudaStream_t s) { k_lower_only<<<64, 256, 0, s>>>(T, b); }
__global__ void k_add_tile(double *dst, const double *src, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] += src[e];
}
void launch_add_tile(double *dst, const double *src, int b, cudaStream_t s) {
    k_add_tile<<<608, 256, 0, s>>>(dst, src, (int64_t)b * b);
}
void launch_add_tiles(double *W, int b, const int *tiles, int ntiles, const double *src, cudaStream_t s) {
    if (ntiles > 0) k_add_tiles<<<dim3(64, ntiles), 256, 0, s>>>(W, b, tiles, src);
}

template <int SU, bool SKIP, class Args>
static void set_zgemm_smem(size_t smem) {
    cudaFuncSetAttribute(k_zgemm<SU, SKIP, Args>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

void launch_zgemm(const CUtensorMap &mx, const CUtensorMap &my, const ZItem *items, int nitems, const int *exps, int k,
                  int b, int *err, cudaStream_t s, int planes, int assign, const ZPlanes *mixed,
                  unsigned long long limit_ns, int stall) {
    if (nitems <= 0 || k <= 0) return;
    static std::atomic<unsigned long long> attr{0};
    const size_t smem = zgemm_smem_bytes();
    if (attrs_pending(attr)) {
        set_zgemm_smem<14, false, ZArgs>(smem);
        set_zgemm_smem<10, false, ZArgs>(smem);
        set_zgemm_smem<7, false, ZArgs>(smem);
        set_zgemm_smem<6, false, ZArgs>(smem);
        set_zgemm_smem<4, false, ZArgs>(smem);
        set_zgemm_smem<14, true, ZArgs>(smem);
        mark_attrs_set(attr);
    }
    const bool skip = mixed && mixed->src_planes_tab && (planes == 14 || planes == 10);
    ZArgs a{items, nitems, exps, skip ? mixed->src_planes_tab : nullptr, skip ? mixed->out_amax : nullptr,
            skip ? mixed->rref : planes, skip ? mixed->margin : 0, skip ? mixed->pair_count : nullptr,
            k, b, err, assign, limit_ns ? limit_ns : ZLIMIT_NS, stall};
    const int grid = nitems < sm_count() ? nitems : sm_count();      // persistent: one CTA per SM
    // mixed precision: FP64 and FP32 outputs share the 14-group form (rref 14 / 10 planes)
    if (skip) k_zgemm<14, true><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
    else if (planes == 10) k_zgemm<10, false><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
    else if (planes == 7) k_zgemm<7, false><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
    else if (planes == 6) k_zgemm<6, false><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
    else if (planes == 4) k_zgemm<4, false><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
    else k_zgemm<14, false><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
}

void launch_zgemm_group(const CUtensorMap &mx, const CUtensorMap &my, const ZGroup &g, const int *exps, int b,
                        int *err, cudaStream_t s, int planes, unsigned long long limit_ns, int stall) {
    if (g.ntiles <= 0 || g.k <= 0) return;
    static std::atomic<unsigned long long> attr{0};
    const size_t smem = zgemm_smem_bytes();
    if (attrs_pending(attr)) {
        set_zgemm_smem<14, false, ZGroupArgs>(smem);
        set_zgemm_smem<10, false, ZGroupArgs>(smem);
        set_zgemm_smem<7, false, ZGroupArgs>(smem);
        set_zgemm_smem<6, false, ZGroupArgs>(smem);
        set_zgemm_smem<4, false, ZGroupArgs>(smem);
        mark_attrs_set(attr);
    }
    ZGroupArgs a;
    memset(&a, 0, sizeof a);
    for (int t = 0; t < g.ntiles; ++t) {
        a.C[t] = g.C[t];
        if (g.lower[t]) a.lower |= 1u << t;
        for (int n = 0; n < g.k; ++n) a.xs[t][n] = (uint16_t)g.xs[t][n];
    }
    for (int n = 0; n < g.k; ++n) a.ys[n] = (uint16_t)g.ys[n];
    a.exps = exps;
    a.planes = nullptr;              // cache slots: every operand form keeps all 14 planes
    a.oamax = nullptr;
    a.rref = planes;
    a.pair_count = nullptr;
    a.k = g.k;
    a.b = b;
    a.ntiles = g.ntiles;
    a.err = err;
    a.assign = g.assign;
    a.limit_ns = limit_ns ? limit_ns : ZLIMIT_NS;
    a.stall = stall;
    const int items = g.ntiles * (b / ZBM) * (b / ZBN);
    const int grid = items < sm_count() ? items : sm_count();        // persistent: one CTA per SM
    if (planes == 10) k_zgemm<10, false><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
    else if (planes == 7) k_zgemm<7, false><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
    else if (planes == 6) k_zgemm<6, false><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
    else if (planes == 4) k_zgemm<4, false><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
    else k_zgemm<14, false><<<grid, ZTHREADS, smem, s>>>(mx, my, a);
}

}  // namespace tc
