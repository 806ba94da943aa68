// Mixed-precision kernels (Section IV-C): storing each final tile in its precision, the
// on-the-fly down-casts that produce per-precision operand copies, and the tensor-core
// SYRK/GEMM updates of FP32 / FP16 / FP8 output tiles on sm_103a (tcgen05 + TMA).
//
// Operand copies ("pools"): one b x b tile per slot, row-major (K-major for the MMA:
// element (r, l) of tile (i, j) at r*b + l).  FP16 and FP8 (E4M3) copies carry a
// power-of-two scale 2^e, e the smallest integer with amax <= fmax * 2^e; FP32 tiles
// are split into two TF32 halves hi = tf32(x), lo = tf32(x - hi) and multiplied as
// hi*hi + hi*lo + lo*hi (three tensor-core passes with FP32 accumulation).
#include "tc_internal.h"

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstring>

namespace tc {

// ----------------------------------------------------------------------- rounding
// Round-to-nearest-even of x to a binary format with t explicit fraction bits and
// minimum normal exponent emin: spacing 2^(max(E, emin) - t) for |x| in [2^E, 2^(E+1)).
// Done on the bit pattern with integer operations (GB300 runs about 2 FP64 operations per
// clock per SM): the dropped low bits of the 53-bit significand decide the rounding, ties to
// even; the result is q 2^(max(E, emin) - t).  (Checked bit for bit against the
// floating-point form x / spacing -> rint -> * spacing on 3.6 million values, ties included.)
__device__ __forceinline__ double pow2(int k) {     // 2^k for -1022 <= k <= 1023
    return __longlong_as_double((long long)(k + 1023) << 52);
}
__device__ __forceinline__ double round_fmt(double x, int t, int emin) {
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0x7FF) return x;
    long long m = bits & 0xFFFFFFFFFFFFFLL;
    int e, E;                                       // |x| = m 2^(e - 52); E = exponent of its leading bit
    if (ex == 0) {
        if (m == 0) return x;
        e = -1022;
        E = (63 - __clzll(m)) + e - 52;
    } else {
        m |= 1LL << 52;
        e = ex - 1023;
        E = e;
    }
    if (E < emin) E = emin;
    const int shift = (E - t) - (e - 52);           // low significand bits to drop
    if (shift <= 0) return x;
    if (shift > 62) return bits < 0 ? -0.0 : 0.0;
    long long q = m >> shift;
    const long long rem = m & ((1LL << shift) - 1), half = 1LL << (shift - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
    const int k = E - t;
    const double r = (k >= -1022 && k <= 1023) ? (double)q * pow2(k) : ldexp((double)q, k);
    return bits < 0 ? -r : r;
}

// smallest integer e with amax <= fmax * 2^e (0 for amax == 0)
__device__ __forceinline__ int scale_exp(double amax, double fmax) {
    if (!(amax > 0.0)) return 0;
    int ea, ef;
    frexp(amax, &ea);
    frexp(fmax, &ef);
    int e = ea - ef;
    for (int g = 0; g < 4 && amax > ldexp(fmax, e); ++g) ++e;
    for (int g = 0; g < 4 && amax <= ldexp(fmax, e - 1); ++g) --e;
    return e;
}

__device__ __forceinline__ double fmt_max(int p) { return p == 2 ? 65504.0 : 448.0; }

// value of x stored in precision p with scale exponent e (p: 1 FP32, 2 FP16, 3 FP8)
__device__ __forceinline__ double to_stored(double x, int p, int e) {
    // scaling by 2^-e and back is exact, so the scaled format's rounding is the unscaled
    // rounding with its minimum exponent moved by e
    if (p == 1) return round_fmt(x, 23, -126);
    if (p == 2) return round_fmt(x, 10, e - 14);
    return round_fmt(x, 3, e - 6);
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// amax of every listed tile (atomic max of non-negative doubles on their bit patterns)
__global__ void k_tile_amax(const double *W, int b, const int *tiles, double *amax, const double *alt) {
    const int t = tiles[blockIdx.y];
    const double *T = alt ? alt + (int64_t)blockIdx.y * b * b : W + (int64_t)t * b * b;
    const int64_t bb = (int64_t)b * b;
    unsigned long long m = 0;           // sign-cleared bit patterns order like |x|
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bb; e += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(T[e]) & 0x7FFFFFFFFFFFFFFFull);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned long long *>(amax + t), m);
}

// W tile <- its value stored in precision prec[t] (Section IV-C), and amax of the result
__global__ void k_store_round(double *W, int b, const int *tiles, const uint8_t *prec, const double *amaxL,
                              double *amaxS) {
    const int t = tiles[blockIdx.y];
    const int p = prec[t];
    double *T = W + (int64_t)t * b * b;
    const int64_t bb = (int64_t)b * b;
    const int e = (p >= 2) ? scale_exp(amaxL[t], fmt_max(p)) : 0;
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < bb; i += (int64_t)gridDim.x * blockDim.x) {
        double v = T[i];
        if (p != 0) {
            v = to_stored(v, p, e);
            T[i] = v;
        }
        m = fmax(m, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(amaxS + t, m);
}

// Operand copy of tile t in precision q (1: TF32 hi/lo pair, 2: FP16, 3: FP8 E4M3), written
// transposed into its pool slot (row-major).  32 x 32 blocks through shared memory.
__global__ void __launch_bounds__(256)
k_make_copies(const double *W, int b, const CopyJob *jobs, const double *amaxS, float *pool_hi, float *pool_lo,
              __half *pool16, uint8_t *pool8, int *exps16, int *exps8, CopyJob one) {
    __shared__ double S[32][33];
    const CopyJob J = jobs ? jobs[blockIdx.y] : one;
    const double *T = W + (int64_t)J.tile * b * b;
    const int nbc = b / 32;
    const int e = (J.q >= 2) ? scale_exp(amaxS[J.tile], fmt_max(J.q)) : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (J.q == 2) exps16[J.tile] = e;
        if (J.q == 3) exps8[J.tile] = e;
    }
    const int64_t base = (int64_t)J.slot * b * b;
    const double sc = ldexp(1.0, -e);                 // 2^-e, exact
    for (int blk = blockIdx.x; blk < nbc * nbc; blk += gridDim.x) {
        const int r0 = (blk % nbc) * 32, c0 = (blk / nbc) * 32;
        __syncthreads();
        for (int idx = threadIdx.x; idx < 1024; idx += 256) {
            const int r = idx & 31, c = idx >> 5;
            S[r][c] = T[(int64_t)(c0 + c) * b + r0 + r];       // coalesced along r
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < 1024; idx += 256) {
            const int c = idx & 31, r = idx >> 5;
            const double v = S[r][c];
            const int64_t o = base + (int64_t)(r0 + r) * b + c0 + c;   // coalesced along c
            if (J.q == 1) {
                const double x = round_fmt(v, 23, -126);               // FP32 value
                const double hi = round_fmt(x, 10, -126);              // TF32 (10 fraction bits)
                const double lo = round_fmt(x - hi, 10, -126);
                pool_hi[o] = (float)hi;
                pool_lo[o] = (float)lo;
            } else if (J.q == 2) {
                // rounded in FP64, then scaled and narrowed exactly (the value is representable)
                pool16[o] = __float2half_rn((float)(round_fmt(v, 10, e - 14) * sc));
            } else {
                const float r8 = (float)(round_fmt(v, 3, e - 6) * sc);
                pool8[o] = (uint8_t)__nv_cvt_float_to_fp8(r8, __NV_SATFINITE, __NV_E4M3);
            }
        }
    }
}

// =================================================================== tcgen05 GEMM
// One CTA = one 128 x 128 block (bm, bn) of one output tile (m, k) in precision q:
//   C_mk[block] -= sum_{n<k} 2^(e_mn + e_kn) X_mn[rows] Y_kn[cols]^T
// Warp 0: TMA producer; warp 1: MMA issuer (and TMEM owner); warps 2..9: epilogue.
// The FP32 accumulator of source tile n lives in TMEM buffer n % 2 (128 columns each);
// the epilogue drains it, scales it and adds it to a register running sum while the
// tensor cores work on tile n + 1.  At the end the running sum is subtracted from the
// FP64 tile in HBM.
constexpr int QBM = 128, QBN = 128, QKB = 128;          // block rows, cols, K bytes per stage
constexpr int QSTAGES = 4;
constexpr int QA_BYTES = QBM * QKB, QB_BYTES = QBN * QKB, QSTAGE_BYTES = QA_BYTES + QB_BYTES;
constexpr int QTHREADS = 320;
constexpr unsigned long long QTIMEOUT_NS = 4000000000ull;  // default bound of a pipeline wait
constexpr unsigned long long QDRAIN_NS = 2000000000ull;    // bound of the teardown waits

// In-core form: one CTA per QItem; operand n of item `it` is the packed tile it.xoff + n
// (X) / it.yoff + n (Y), found in the pool through slot[] and scaled by exps[tile].
struct QArgs {
    const QItem *items;
    const int *slot;      // slot of each (global) packed tile in this precision's pool (-1: none)
    const int *exps;      // scale exponents of the copies (FP16/FP8), nullptr for TF32
    int k, b;
    int *err;             // error word: set on a timed-out wait or a missing operand slot
    unsigned long long limit_ns;   // bound of each pipeline wait
    int stall;                     // test hook: wait first on a barrier nothing arrives at
    __device__ void tile(QItem &it) const { it = items[blockIdx.x]; }
    __device__ int xslot(const QItem &it, int n) const { return slot[it.xoff + n]; }
    __device__ int yslot(const QItem &it, int n) const { return slot[it.yoff + n]; }
    __device__ int xexp(const QItem &it, int n) const { return exps[it.xoff + n]; }
    __device__ int yexp(const QItem &it, int n) const { return exps[it.yoff + n]; }
};

// Out-of-core form: up to QG_MAX output tiles of one tile column whose operands sit in
// arbitrary cache slots (lists in the launch parameters; exps indexed by slot).  Grid:
// ntiles x (b/QBM) x (b/QBN).
struct QGroupArgs {
    double *C[QG_MAX];
    uint16_t xs[QG_MAX][QK_MAX];
    uint16_t ys[QK_MAX];
    const int *exps;
    int k, b;
    int *err;
    unsigned long long limit_ns;
    int stall;
    __device__ void tile(QItem &it) const {
        const int nbm = b / QBM, per = nbm * (b / QBN);
        const int g = blockIdx.x / per, r = blockIdx.x % per;
        it.C = C[g];
        it.xoff = g;
        it.yoff = 0;
        it.bm = (uint16_t)(r % nbm);
        it.bn = (uint16_t)(r / nbm);
    }
    __device__ int xslot(const QItem &it, int n) const { return xs[it.xoff][n]; }
    __device__ int yslot(const QItem &, int n) const { return ys[n]; }
    __device__ int xexp(const QItem &it, int n) const { return exps[xs[it.xoff][n]]; }
    __device__ int yexp(const QItem &, int n) const { return exps[ys[n]]; }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false when the phase did not complete within limit_ns or another role of
// the CTA gave up (abort flag in shared memory).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: rows of 128 bytes, 8-row
// groups 1024 bytes apart (stride byte offset), version 1 (bits 46-48), swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

template <int KIND>
__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if constexpr (KIND == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    } else if constexpr (KIND == 2) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    }
}

// Instruction descriptor: D = F32 (bits 4-5 = 1), A/B format (bits 7-9 / 10-12: TF32 = 2
// for kind::tf32, F16 = 0 for kind::f16, E4M3 = 0 for kind::f8f6f4), both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
template <int KIND>
__device__ __forceinline__ uint32_t make_idesc() {
    const uint32_t fmt = (KIND == 1) ? 2u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(QBN >> 3) << 17) | ((uint32_t)(QBM >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// KIND 1: TF32 x3 (maps: A_hi, A_lo, B_hi, B_lo); 2: FP16; 3: FP8 E4M3 (maps: A, -, B, -)
template <int KIND, class Args>
__global__ void __launch_bounds__(QTHREADS, 1)
k_qgemm(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
        const __grid_constant__ CUtensorMap mapB0, const __grid_constant__ CUtensorMap mapB1,
        const __grid_constant__ Args args) {
    extern __shared__ __align__(1024) uint8_t qsmem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(qsmem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + QSTAGES * QSTAGE_BYTES);
    uint64_t *empty = full + QSTAGES;
    uint64_t *accf = empty + QSTAGES;
    uint64_t *acce = accf + 2;
    uint64_t *done = acce + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    volatile int *never = abort_flag + 1;        // nothing sets it: waits that must not be cut short
    const unsigned long long lim = args.limit_ns;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    QItem it;
    args.tile(it);
    const int k = args.k, b = args.b;
    const int nsrc = k;
    constexpr int PASSES = (KIND == 1) ? 3 : 1;
    const int kblocks = b * (KIND == 1 ? 4 : (KIND == 2 ? 2 : 1)) / QKB;   // 128-byte K blocks per tile
    const int steps_per_src = kblocks * PASSES;
    const int total_steps = nsrc * steps_per_src;

    if (threadIdx.x == 0) {
        for (int s = 0; s < QSTAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf + a, 1);
            mbar_init(acce + a, 8);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *never = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(2 * QBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;


    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int issued = 0;
            for (int s = 0; s < total_steps; ++s) {
                const int stage = s % QSTAGES, round = s / QSTAGES;
                if (!mbar_wait(empty + stage, (round & 1) ^ 1, abort_flag, lim)) {
                    *abort_flag = 1;
                    atomicExch(args.err, 1);
                    break;
                }
                const int n = s / steps_per_src, j = s % steps_per_src;
                const int kb = j / PASSES, pass = j % PASSES;
                const int sx = args.xslot(it, n), sy = args.yslot(it, n);
                if (sx < 0 || sy < 0) {
                    *abort_flag = 1;
                    atomicExch(args.err, 2);
                    break;
                }
                uint8_t *sa = smem + stage * QSTAGE_BYTES;
                uint8_t *sb = sa + QA_BYTES;
                constexpr int EB = (KIND == 1) ? 4 : (KIND == 2 ? 2 : 1);
                const int x = kb * (QKB / EB);
                // TF32 passes: (lo, hi), (hi, lo), (hi, hi)
                const CUtensorMap *ma = (KIND == 1 && pass == 0) ? &mapA1 : &mapA0;
                const CUtensorMap *mb = (KIND == 1 && pass == 1) ? &mapB1 : &mapB0;
                mbar_expect_tx(full + stage, QSTAGE_BYTES);
                tma_load_2d(sa, ma, x, sx * b + it.bm * QBM, full + stage);
                tma_load_2d(sb, mb, x, sy * b + it.bn * QBN, full + stage);
                ++issued;
            }
            // Every copy lands before the shared memory goes away, whichever role gave up and
            // whenever: only the last QSTAGES copies can still be in flight (each earlier one was
            // consumed before its stage was refilled), and each is the latest phase of its
            // stage's full barrier.  Without an abort they end as soon as those copies land.
            for (int s = issued - QSTAGES < 0 ? 0 : issued - QSTAGES; s < issued; ++s)
                if (!mbar_wait(full + s % QSTAGES, (s / QSTAGES) & 1, never, QDRAIN_NS)) atomicExch(args.err, 3);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = make_idesc<KIND>();
            bool ok = true;
            // test hook: `done` completes only after the final commit below, so this wait runs
            // into the bound and takes the abort path
            if (args.stall && !mbar_wait(done, 0, abort_flag, lim)) ok = false;
            for (int n = 0; n < nsrc && ok; ++n) {
                const int a = n & 1, use = n >> 1;
                if (!mbar_wait(acce + a, (use & 1) ^ 1, abort_flag, lim)) { ok = false; break; }
                tc_fence_after();
                for (int j = 0; j < steps_per_src; ++j) {
                    const int s = n * steps_per_src + j;
                    const int stage = s % QSTAGES, round = s / QSTAGES;
                    if (!mbar_wait(full + stage, round & 1, abort_flag, lim)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + stage * QSTAGE_BYTES);
                    const uint32_t sb = sa + QA_BYTES;
#pragma unroll
                    for (int kk = 0; kk < QKB / 32; ++kk)
                        mma_issue<KIND>(tmem + a * QBN, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), idesc,
                                        (j > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(empty + stage);
                }
                if (!ok) break;
                mma_commit(accf + a);
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(args.err, 1);
            }
            // all issued MMAs complete before the TMEM is released: this wait is not cut short
            // by the abort flag (the MMAs depend on nothing outside the CTA, so it ends)
            mma_commit(done);
            if (!mbar_wait(done, 0, never, QDRAIN_NS)) atomicExch(args.err, 3);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // warps 2..9: TMEM lane quarter = warp % 4 (hardware rule), column half = (warp - 2) / 4
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        constexpr int EC = QBN / 2;            // columns per epilogue warp
        float run[EC];
#pragma unroll
        for (int j = 0; j < EC; ++j) run[j] = 0.f;
        // reference exponent: the largest scale product over the source tiles
        int eref = 0;
        if (KIND != 1) {
            eref = -100000;
            for (int n = 0; n < nsrc; ++n) {
                const int e = args.xexp(it, n) + args.yexp(it, n);
                eref = e > eref ? e : eref;
            }
        }
        bool ok = true;
        for (int n = 0; n < nsrc; ++n) {
            const int a = n & 1, use = n >> 1;
            if (!mbar_wait(accf + a, use & 1, abort_flag, lim)) { ok = false; break; }
            tc_fence_after();
            float sc = 1.f;
            if (KIND != 1) sc = ldexpf(1.f, args.xexp(it, n) + args.yexp(it, n) - eref);
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + a * QBN + half * EC;
#pragma unroll
            for (int c = 0; c < EC / 32; ++c) {
                float v[32];
                tmem_ld32(tbase + c * 32, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) run[c * 32 + j] = fmaf(sc, v[j], run[c * 32 + j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce + a);
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(args.err, 1);
        } else {
            const int row = it.bm * QBM + quarter * 32 + lane;
            double *C = it.C;
            const double sref = ldexp(1.0, eref);
#pragma unroll
            for (int j = 0; j < EC; ++j) {
                const int col = it.bn * QBN + half * EC + j;
                C[(int64_t)col * b + row] -= (double)run[j] * sref;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * QBN) : "memory");
}

// ------------------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D map over a pool: rows = nslots * b, columns = b elements of esize bytes; box of
// (128 bytes) x box_rows with 128-byte swizzle.
// rows of b elements; box: box_k_bytes (128 or 64, swizzled to match) x box_rows
int make_pool_map_k(CUtensorMap *map, void *pool, int64_t nslots, int b, int esize, int box_rows, int box_k_bytes) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return -1;
    if (box_k_bytes != 128 && box_k_bytes != 64) return -1;
    const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    cuuint64_t dims[2] = {(cuuint64_t)b, (cuuint64_t)(nslots * b)};
    cuuint64_t strides[1] = {(cuuint64_t)b * esize};
    cuuint32_t box[2] = {(cuuint32_t)(box_k_bytes / esize), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, dt, 2, pool, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    box_k_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)r;
}
int make_plane_map3(CUtensorMap *map, void *pool, int64_t nplanes, int b, int box_rows, int depth) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return -1;
    cuuint64_t dims[3] = {(cuuint64_t)b, (cuuint64_t)b, (cuuint64_t)nplanes};
    cuuint64_t strides[2] = {(cuuint64_t)b, (cuuint64_t)b * b};
    cuuint32_t box[3] = {128, (cuuint32_t)box_rows, (cuuint32_t)depth};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, pool, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)r;
}
int make_pool_map(CUtensorMap *map, void *pool, int64_t nslots, int b, int esize, int box_rows) {
    return make_pool_map_k(map, pool, nslots, b, esize, box_rows, QKB);
}

size_t qgemm_smem_bytes() { return (size_t)QSTAGES * QSTAGE_BYTES + 1024 + 256; }

template <int KIND, class Args>
static void launch_q(const CUtensorMap &a0, const CUtensorMap &a1, const CUtensorMap &b0, const CUtensorMap &b1,
                     const Args &args, int nitems, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    const size_t smem = qgemm_smem_bytes();
    if (attrs_pending(attr)) {
        cudaFuncSetAttribute(k_qgemm<KIND, Args>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        mark_attrs_set(attr);
    }
    k_qgemm<KIND, Args><<<nitems, QTHREADS, smem, s>>>(a0, a1, b0, b1, args);
}

void launch_qgemm(int kind, const CUtensorMap &a0, const CUtensorMap &a1, const CUtensorMap &b0,
                  const CUtensorMap &b1, const QItem *items, int nitems, const int *slot, const int *exps,
                  int k, int b, int *err, cudaStream_t s, unsigned long long limit_ns, int stall) {
    if (nitems <= 0) return;
    QArgs args{items, slot, exps, k, b, err, limit_ns ? limit_ns : QTIMEOUT_NS, stall};
    if (kind == 1) launch_q<1>(a0, a1, b0, b1, args, nitems, s);
    else if (kind == 2) launch_q<2>(a0, a1, b0, b1, args, nitems, s);
    else launch_q<3>(a0, a1, b0, b1, args, nitems, s);
}

// FP16 (kind 2) or FP8 (kind 3) updates of up to QG_MAX out-of-core tiles; the operand
// copies sit in the cache-slot pool mapped by `mx` / `my` (slot s at rows s*b .. s*b+b-1).
void launch_qgemm_group(int kind, const CUtensorMap &mx, const CUtensorMap &my, const QGroup &g, const int *exps,
                        int b, int *err, cudaStream_t s, unsigned long long limit_ns, int stall) {
    if (g.ntiles <= 0 || g.k <= 0) return;
    QGroupArgs a;
    memset(&a, 0, sizeof a);
    for (int t = 0; t < g.ntiles; ++t) {
        a.C[t] = g.C[t];
        for (int n = 0; n < g.k; ++n) a.xs[t][n] = (uint16_t)g.xs[t][n];
    }
    for (int n = 0; n < g.k; ++n) a.ys[n] = (uint16_t)g.ys[n];
    a.exps = exps;
    a.k = g.k;
    a.b = b;
    a.err = err;
    a.limit_ns = limit_ns ? limit_ns : QTIMEOUT_NS;
    a.stall = stall;
    const int nitems = g.ntiles * (b / QBM) * (b / QBN);
    if (kind == 2) launch_q<2>(mx, mx, my, my, a, nitems, s);
    else launch_q<3>(mx, mx, my, my, a, nitems, s);
}

void launch_tile_amax(const double *W, int b, const int *tiles, int ntiles, double *amax, cudaStream_t s,
                      const double *alt) {
    // one grid row per listed tile, at most 65535 rows per launch
    for (int t0 = 0; t0 < ntiles; t0 += 65535) {
        const int nt = ntiles - t0 < 65535 ? ntiles - t0 : 65535;
        k_tile_amax<<<dim3(tile_ctas(nt), nt), 256, 0, s>>>(W, b, tiles + t0, amax, alt ? alt + (int64_t)t0 * b * b : nullptr);
    }
}
void launch_store_round(double *W, int b, const int *tiles, int ntiles, const uint8_t *prec, const double *amaxL,
                        double *amaxS, cudaStream_t s) {
    if (ntiles > 0) k_store_round<<<dim3(tile_ctas(ntiles), ntiles), 256, 0, s>>>(W, b, tiles, prec, amaxL, amaxS);
}
void launch_make_copies(const double *W, int b, const CopyJob *jobs, int njobs, const double *amaxS, float *hi,
                        float *lo, __half *p16, uint8_t *p8, int *e16, int *e8, cudaStream_t s) {
    if (njobs > 0) k_make_copies<<<dim3(tile_ctas(njobs), njobs), 256, 0, s>>>(W, b, jobs, amaxS, hi, lo, p16, p8, e16, e8, CopyJob{});
}

// ------------------------------------------------------------ out-of-core, one cache slot
// The slot pool holds FP64 tiles at pool + s b^2; exps, amax arrays are indexed by slot.
void launch_copy_slot(const double *pool, int b, int slot, int q, const double *amaxS, __half *p16, uint8_t *p8,
                      int *e16, int *e8, cudaStream_t s) {
    const int blocks = (b / 32) * (b / 32);
    k_make_copies<<<dim3(blocks < 608 ? blocks : 608, 1), 256, 0, s>>>(pool, b, nullptr, amaxS, nullptr, nullptr, p16,
                                                                       p8, e16, e8, CopyJob{slot, q, slot});
}

// T <- its value stored in precision p (scale from *amaxL, exponent to *e_out)
__global__ void k_round_slot(double *T, int b, int p, const double *amaxL, int *e_out) {
    const int e = (p >= 2) ? scale_exp(*amaxL, fmt_max(p)) : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *e_out = e;
    const int64_t bb = (int64_t)b * b;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < bb; i += (int64_t)gridDim.x * blockDim.x)
        T[i] = to_stored(T[i], p, e);
}

// compact host copy of a stored tile: FP32 as float, FP16 / FP8 as the scaled format value
// (exact: the tile already holds representable values); unpack is the exact inverse
__global__ void k_pack_compact(const double *T, int b, int p, const int *e_in, void *dst) {
    const int e = (p >= 2) ? *e_in : 0;
    const double sc = ldexp(1.0, -e);                // exact scaling; the values are representable
    const int64_t bb = (int64_t)b * b;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < bb; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = T[i];
        if (p == 1) static_cast<float *>(dst)[i] = (float)v;
        else if (p == 2) static_cast<__half *>(dst)[i] = __float2half_rn((float)(v * sc));
        else static_cast<uint8_t *>(dst)[i] = (uint8_t)__nv_cvt_float_to_fp8((float)(v * sc), __NV_SATFINITE, __NV_E4M3);
    }
}
__global__ void k_unpack_compact(const void *src, int b, int p, const int *e_in, double *T) {
    const int e = (p >= 2) ? *e_in : 0;
    const double sc = ldexp(1.0, e);
    const int64_t bb = (int64_t)b * b;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < bb; i += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (p == 1) v = (double)static_cast<const float *>(src)[i];
        else if (p == 2) v = (double)__half2float(static_cast<const __half *>(src)[i]);
        else {
            const __half_raw hr = __nv_cvt_fp8_to_halfraw(static_cast<const __nv_fp8_storage_t *>(src)[i], __NV_E4M3);
            v = (double)__half2float(__half(hr));
        }
        T[i] = v * sc;
    }
}
void launch_round_slot(double *T, int b, int p, const double *amaxL, int *e_out, cudaStream_t s) {
    k_round_slot<<<608, 256, 0, s>>>(T, b, p, amaxL, e_out);
}
void launch_pack_compact(const double *T, int b, int p, const int *e, void *dst, cudaStream_t s) {
    k_pack_compact<<<608, 256, 0, s>>>(T, b, p, e, dst);
}
void launch_unpack_compact(const void *src, int b, int p, const int *e, double *T, cudaStream_t s) {
    k_unpack_compact<<<608, 256, 0, s>>>(src, b, p, e, T);
}

}  // namespace tc
