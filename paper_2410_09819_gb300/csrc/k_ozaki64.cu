// Mixed-precision FP64 / FP32 tile updates emulated on the FP8 tensor cores, with 128 x 64
// output blocks (the digit-plane method of k_ozaki.cu: X Y^T = 2^(ex+ey) sum_d 16^-d G_d,
// G_d = sum_{s+t=d} D_s(X) D_t(Y)^T, exact FP32 group sums in TMEM, exact int64 recombination).
//
// Why a second kernel: in a mixed-precision factorization every source carries its own plane
// budget (the stored formats bound its planes, its scale against the output's bounds the pairs
// worth multiplying), 57 pairs per FP64-output product and 37 per FP32-output product on
// average at n = 131072 against the FP64 path's 105.  With 128 x 16 blocks an X plane then
// meets few partners: its MMA has N = 16 x partners, mostly at or below 128, where one
// tcgen05.mma (kind::f8f6f4, M = 128, K = 32) still occupies the tensor pipe ~69 cycles, and
// the issuing thread's fixed cost per stage (a barrier wait of ~200-300 cycles, fence, commit)
// is spread over little MMA work (measured on GB300).  Here an X plane's MMA spans 64 columns
// per partner (N = 64 x partners <= 256), and one pipeline unit carries a whole K block of two
// X planes together with the Y planes they meet, so one wait and one commit cover 8 MMAs.
//
// Accumulator passes: the groups 0 .. G-1 a source writes (G = min(su, sx + sy - 1)) are split
// into P = ceil(G / 4) passes of consecutive groups, the smaller first; a pass [g0, g1) holds
// its groups in one of two TMEM buffers of 4 x 64 columns (double-buffered across passes) and
// multiplies the pairs with g0 <= s + t < g1.  Within a pass the X planes slo .. shi that have
// partners run in chunks of two consecutive planes; chunk [sa, sb] meets the consecutive Y
// planes max(0, g0 - sb) .. min(sy, g1 - sa) - 1 (five at most).  A unit = (pass, K block,
// chunk): those Y planes (8 KB each) and the chunk's X planes (16 KB each), contiguous in a
// ring of 8 KB slots, loaded by two 3D TMA copies, guarded by one barrier pair; units are
// released in FIFO order, each right after its own MMAs.
#include "tc_internal.h"
#include "zgemm_common.h"

#include <cuda.h>

#include <atomic>
#include <cstring>

namespace tc {
namespace z64 {

constexpr int ZS = 14;                 // digit planes per tile
constexpr int BM = 128, BN = Z64_BN;   // work item: 128 rows x 64 columns
constexpr int KB = 128;                // K bytes per unit (4 MMAs of K = 32)
constexpr int GP = 4;                  // accumulator groups per pass
constexpr int BUF = GP * BN;           // TMEM columns of one accumulator buffer (two buffers)
constexpr int SLOT = 8192;             // ring slot: one Y plane block (64 rows x 128 B)
constexpr int XPL = 2 * SLOT;          // one X plane block (128 rows x 128 B)
#ifndef ZGEMM64_RING
#define ZGEMM64_RING 27
#endif
constexpr int RING = ZGEMM64_RING;     // slots
constexpr int SETS = 32;               // units in flight at most
constexpr int YMAX = GP + 1;           // Y planes of a unit at most
constexpr int DRAIN_WARPS = 8;         // two per TMEM lane quarter, 32 columns each
constexpr int THREADS = 64 + 32 * DRAIN_WARPS;
constexpr unsigned long long LIMIT_NS = 4000000000ull;   // default bound of a pipeline wait
constexpr unsigned long long DRAIN_NS = 2000000000ull;   // bound of the teardown waits
static_assert(BUF * 2 <= 512, "two accumulator buffers fit TMEM");
// FIFO placement: a unit that does not fit before the ring's end starts at slot 0, so the ring
// must hold the largest unit after the largest gap
static_assert(RING >= 2 * (YMAX + 2 * 2) - 1, "a unit after the largest end-of-ring gap fits");

struct Args {
    const ZItem *items;
    int nitems;
    const int *exps;
    const uint8_t *planes;          // leading planes each digit slot can have non-zero, or null (all 14)
    const double *oamax;            // input amax of every output tile, or null (rref planes for every source)
    int rref, margin;               // pair budget relative to the output's scale
    unsigned long long *pair_count; // plane pairs multiplied (added at the end)
    int k, b;
    int *err;
    int assign;                     // 0: C -= sum X Y^T;  1: C = sum X Y^T
    unsigned long long limit_ns;    // bound of each pipeline wait
    int stall;                      // test hook: wait first on a barrier nothing arrives at
};

// Plane counts of one source: su, the budget of plane pairs s + t < su (from the scales: a pair
// whose scale 2^(e_x + e_y) lies d binary orders below the output tile's input scale 2^e_out
// keeps floor((d - 4 margin) / 4) planes fewer than rref, within [1, 14]), and the X / Y planes
// its stored formats can have non-zero (the skipped products are exact zeros).
struct Shape {
    int sx, sy, su;
};
// Without output scales (oamax null) every source runs on rref planes; without a plane table
// (planes null) every operand may use all 14.
__device__ __forceinline__ Shape shape(const Args &a, int eo, int xt, int yt) {
    int su = a.rref;
    if (a.oamax) {
        const int d = eo - a.exps[xt] - a.exps[yt] - 4 * a.margin;
        const int j = d >= 0 ? d / 4 : -((3 - d) / 4);        // floor(d / 4)
        su = a.rref - j;
    }
    su = su < 1 ? 1 : (su > ZS ? ZS : su);
    int sx = a.planes ? a.planes[xt] : ZS, sy = a.planes ? a.planes[yt] : ZS;
    sx = sx < su ? sx : su;
    sy = sy < su ? sy : su;
    return {sx, sy, su};
}
__device__ __forceinline__ int pairs(const Shape &z) {
    int p = 0;
    for (int s = 0; s < z.sx; ++s) p += z.sy < z.su - s ? z.sy : z.su - s;
    return p;
}
__device__ __forceinline__ int groups(const Shape &z) { return z.su < z.sx + z.sy - 1 ? z.su : z.sx + z.sy - 1; }
__device__ __forceinline__ int npass(int G) { return (G + GP - 1) / GP; }

// Pass p of P over groups [0, G): [g0, g1), sizes as even as possible, the smaller first; the X
// planes slo .. shi with a partner in it.
struct Pass {
    int g0, g1, slo, shi;
};
__device__ __forceinline__ Pass pass(int p, int P, int G, int sx, int sy) {
    const int base = G / P, big = P - G % P;               // passes big .. P-1 hold base + 1 groups
    Pass r;
    r.g0 = p * base + (p > big ? p - big : 0);
    r.g1 = r.g0 + base + (p >= big ? 1 : 0);
    r.slo = r.g0 - sy + 1 > 0 ? r.g0 - sy + 1 : 0;
    r.shi = (sx < r.g1 ? sx : r.g1) - 1;
    return r;
}
// The chunk of X planes [sa, sa + nx - 1] starting at sa, and the Y planes [ylo, ylo + ny) it meets.
struct Chunk {
    int sa, nx, ylo, ny;
};
__device__ __forceinline__ Chunk chunk(const Pass &ps, int sa, int sy) {
    Chunk c;
    c.sa = sa;
    c.nx = ps.shi - sa >= 1 ? 2 : 1;
    const int sb = sa + c.nx - 1;
    c.ylo = ps.g0 - sb > 0 ? ps.g0 - sb : 0;
    const int yhi = sy < ps.g1 - sa ? sy : ps.g1 - sa;
    c.ny = yhi - c.ylo;
    return c;
}

// Persistent kernel: C -= sum_{n<k} X_n Y_n^T (C = ... when assign) for 128 x 64 output blocks of
// FP64- or FP32-output tiles of a mixed-precision map.
//   warp 0  TMA producer: per item, source, pass, K block and chunk one unit;
//   warp 1  MMA issuer: per unit one barrier wait, per X plane of the chunk one asm block of 4
//           MMAs (the K steps) with N = 64 x partners into the groups s + t0 .. of the pass's
//           buffer, one commit;
//   warps 2-9 drain: per pass, the groups leave TMEM (exact FP32 integers), are recombined by
//           int64 Horner steps and added, scaled by 2^(e_x + e_y) 16^-(g1 + 1), to FP64 running
//           sums; C is written once per item.
// Group initialisation: in the first K block of a pass the X planes run in ascending order;
// plane slo starts the groups it covers, and each later plane s covers [max(s, g0), s + t1(s)),
// reaching at most one group past those already started: when t1(s) = sy that group s + sy - 1
// is new, and for K step 0 a separate MMA of the one partner t = sy - 1 starts it.
// Failure handling as in k_zgemm: bounded pipeline waits that set *err and stop the CTA; before
// the TMEM is released the MMA issuer waits for its issued MMAs and the producer for its issued
// copies (waits that ignore the abort flag, bounded by DRAIN_NS).
template <class A>
__global__ void __maxnreg__(168)   // 320 threads: 3 warps on some SMSP x 32 x 168 <= 16K registers
k_zgemm64(const __grid_constant__ Z64Maps maps, const __grid_constant__ A args) {
    extern __shared__ __align__(1024) uint8_t zsmem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(zsmem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *ring = smem;                             // RING x 8 KB
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + RING * SLOT);   // [SETS]
    uint64_t *empty = full + SETS;                    // [SETS]
    uint64_t *accf = empty + SETS;                    // [2]
    uint64_t *acce = accf + 2;                        // [2]
    uint64_t *done = acce + 2;
    long long *uend = reinterpret_cast<long long *>(done + 1);   // [SETS] producer: end slot of each unit
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(uend + SETS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    volatile int *never = abort_flag + 1;             // nothing sets it: waits that must not be cut short
    const unsigned long long lim = args.limit_ns;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = args.k, b = args.b;
    const int kblocks = b / KB;
    const int nitems = args.nitems;
    if ((int)blockIdx.x >= nitems) return;             // whole CTA, before any barrier
    if (threadIdx.x == 0) {
        for (int u = 0; u < SETS; ++u) {
            z_init(full + u, 1);
            z_init(empty + u, 1);
        }
        for (int a = 0; a < 2; ++a) {
            z_init(accf + a, 1);
            z_init(acce + a, DRAIN_WARPS);
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
            // ring state: pos = slot of the next unit, head / tail = slots allocated / released
            // so far (gaps at the ring's end included), nset / nrel = units allocated / released
            int pos = 0, nset = 0, nrel = 0;
            long long head = 0, tail = 0;
            bool ok = true;
            // place a unit of sz slots: wait (in FIFO order) for the MMAs of the oldest units to
            // release what it needs; false if a wait ran into its bound
            auto alloc = [&](int sz, int &slot, int &set) -> bool {
                int sp = pos;
                long long start = head;
                if (sp + sz > RING) {
                    start += RING - sp;
                    sp = 0;
                }
                while (nrel < nset && (start + sz - tail > RING || nset - nrel >= SETS)) {
                    if (!z_wait(empty + (nrel & (SETS - 1)), (uint32_t)((nrel / SETS) & 1), abort_flag, lim))
                        return false;
                    tail = uend[nrel & (SETS - 1)];
                    ++nrel;
                }
                slot = sp;
                set = nset & (SETS - 1);
                uend[set] = start + sz;
                head = start + sz;
                pos = sp + sz == RING ? 0 : sp + sz;
                ++nset;
                return true;
            };
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const ZItem it = args.items[item];
                const int eo = args.oamax ? z_digit_exp(args.oamax[it.ct]) : 0;
                for (int n = 0; n < k && ok; ++n) {
                    const int xt = it.xoff + n, yt = it.yoff + n;
                    const Shape zs = shape(args, eo, xt, yt);
                    const int G = groups(zs), P = npass(G);
                    for (int p = 0; p < P && ok; ++p) {
                        const Pass ps = pass(p, P, G, zs.sx, zs.sy);
                        for (int kb = 0; kb < kblocks && ok; ++kb)
                            for (int sa = ps.slo; sa <= ps.shi && ok; sa += 2) {
                                const Chunk c = chunk(ps, sa, zs.sy);
                                int slot, set;
                                if (!alloc(c.ny + 2 * c.nx, slot, set)) { ok = false; break; }
                                z_expect(full + set, (uint32_t)(c.ny * SLOT + c.nx * XPL));
                                z_tma3(ring + slot * SLOT, &maps.y[c.ny - 1], kb * KB, it.bn * BN, yt * ZS + c.ylo, full + set);
                                z_tma3(ring + (slot + c.ny) * SLOT, &maps.x[c.nx - 1], kb * KB, it.bm * BM, xt * ZS + c.sa,
                                       full + set);
                            }
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(args.err, 1);
            }
            // Every copy lands before the shared memory goes away: only the last SETS units can
            // still have copies in flight (an older unit's barrier was re-armed only after the
            // MMAs had consumed it), each the latest phase of its full barrier.
            for (int j = nset - SETS < 0 ? 0 : nset - SETS; j < nset; ++j)
                if (!z_wait(full + (j & (SETS - 1)), (uint32_t)((j / SETS) & 1), never, DRAIN_NS)) atomicExch(args.err, 3);
        }
    } else if (warp == 1) {
        // --------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            // kind::f8f6f4, D F32, A/B E4M3, K-major, M = 128; N set per instruction
            const uint32_t idesc0 = (1u << 4) | ((uint32_t)(BM >> 4) << 24);
            const uint64_t rdesc = z_desc(z_smem(ring));
            int pos = 0, set = 0, q = 0;                 // q: passes issued so far (all items)
            unsigned long long pairs_done = 0;
            bool ok = true;
            // test hook: `done` completes only after the final commit below, so this wait runs
            // into the bound and takes the abort path
            if (args.stall && !z_wait(done, 0, abort_flag, lim)) ok = false;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const ZItem it = args.items[item];
                const int eo = args.oamax ? z_digit_exp(args.oamax[it.ct]) : 0;
                for (int n = 0; n < k && ok; ++n) {
                    const Shape zs = shape(args, eo, it.xoff + n, it.yoff + n);
                    const int G = groups(zs), P = npass(G);
                    pairs_done += (unsigned long long)pairs(zs);
                    for (int p = 0; p < P && ok; ++p, ++q) {
                        const Pass ps = pass(p, P, G, zs.sx, zs.sy);
                        const int a = q & 1;
                        if (!z_wait(acce + a, ((q >> 1) & 1) ^ 1, abort_flag, lim)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t dbase = tmem + (uint32_t)(a * BUF);
                        for (int kb = 0; kb < kblocks && ok; ++kb)
                            for (int sa = ps.slo; sa <= ps.shi; sa += 2) {
                                const Chunk c = chunk(ps, sa, zs.sy);
                                const int sz = c.ny + 2 * c.nx;
                                if (pos + sz > RING) pos = 0;       // the producer's placement
                                const int slot = pos;
                                pos = pos + sz == RING ? 0 : pos + sz;
                                const int u = set++;
                                if (!z_wait(full + (u & (SETS - 1)), (uint32_t)((u / SETS) & 1), abort_flag, lim)) {
                                    ok = false;
                                    break;
                                }
                                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                                const uint64_t ud = rdesc + (uint64_t)((slot * SLOT) >> 4);
#pragma unroll
                                for (int h = 0; h < 2; ++h)
                                    if (h < c.nx) {
                                        const int s = c.sa + h;
                                        const int t0 = ps.g0 - s > 0 ? ps.g0 - s : 0;
                                        const int t1 = zs.sy < ps.g1 - s ? zs.sy : ps.g1 - s;
                                        const int np = t1 - t0;
                                        // A: X plane h of the unit; B: its Y planes t0 - ylo ..;
                                        // D: groups s + t0 - g0 .. of the pass's buffer
                                        const uint64_t xd = ud + (uint64_t)(((c.ny * SLOT) + h * XPL) >> 4);
                                        const uint64_t bd = ud + (uint64_t)(((t0 - c.ylo) * SLOT) >> 4);
                                        const uint32_t d = dbase + (uint32_t)((s + t0 - ps.g0) * BN);
                                        const uint32_t idesc = idesc0 | ((uint32_t)((np * BN) >> 3) << 17);
                                        if (kb > 0) {
                                            z_mma4(d, xd, bd, idesc, 1u);
                                        } else if (s == ps.slo) {
                                            z_mma4(d, xd, bd, idesc, 0u);           // starts its groups
                                        } else if (t1 == zs.sy) {
                                            // groups s+t0 .. s+sy-2 are running; group s+sy-1 starts here
                                            if (np > 1) z_mma(d, xd, bd, idesc0 | ((uint32_t)(((np - 1) * BN) >> 3) << 17), 1u);
                                            z_mma(d + (uint32_t)((np - 1) * BN), xd, bd + (uint64_t)(((np - 1) * SLOT) >> 4),
                                                  idesc0 | ((uint32_t)(BN >> 3) << 17), 0u);
                                            z_mma3(d, xd, bd, idesc);
                                        } else {
                                            z_mma4(d, xd, bd, idesc, 1u);           // all its groups are running
                                        }
                                    }
                                z_commit(empty + (u & (SETS - 1)));
                            }
                        if (ok) z_commit(accf + a);
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(args.err, 1);
            }
            if (args.pair_count && pairs_done) atomicAdd(args.pair_count, pairs_done);
            // every issued MMA completes before the TMEM is released and the CTA exits
            z_commit(done);
            if (!z_wait(done, 0, never, DRAIN_NS)) atomicExch(args.err, 3);
        }
    } else {
        // --------------------------------------------------------------- drain + epilogue
        const int quarter = warp & 3, half = (warp - 2) >> 2;    // TMEM lanes 32 quarter.., columns 32 half..
        bool ok = true;
        int q = 0;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const ZItem it = args.items[item];
            const int eo = args.oamax ? z_digit_exp(args.oamax[it.ct]) : 0;
            double run[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) run[j] = 0.0;
            for (int n = 0; n < k && ok; ++n) {
                const int xt = it.xoff + n, yt = it.yoff + n;
                const int E = args.exps[xt] + args.exps[yt];
                const Shape zs = shape(args, eo, xt, yt);
                const int G = groups(zs), P = npass(G);
                for (int p = 0; p < P; ++p, ++q) {
                    const Pass ps = pass(p, P, G, zs.sx, zs.sy);
                    const int a = q & 1;
                    if (!z_wait(accf + a, (q >> 1) & 1, abort_flag, lim)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // groups g0 .. g1-1 (weights 16^-(g+2)): Horner over the pass, then one scale
                    const int ng = ps.g1 - ps.g0;
                    const double sc = ldexp(1.0, E - 4 * (ps.g1 + 1));
                    const uint32_t lanebase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * BUF + half * 32);
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        long long h[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) h[j] = 0;
#pragma unroll 1
                        for (int g = 0; g < ng; ++g) {
                            float v[16];
                            z_ld16(lanebase + (uint32_t)(g * BN + c * 16), v);
                            // group sums are exact integers below 2^24 in magnitude: a 32-bit
                            // conversion (a 64-bit one would run on the FP64 pipe)
#pragma unroll
                            for (int j = 0; j < 16; ++j) h[j] = h[j] * 16 + (long long)__float2int_rn(v[j]);
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) run[c * 16 + j] = fma((double)h[j], sc, run[c * 16 + j]);
                    }
                    // the accumulator buffer is free for pass q + 2 once every drain warp has read it
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) z_arrive(acce + a);
                }
            }
            if (!ok) break;
            const int row = it.bm * BM + quarter * 32 + lane;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                double *cp = it.C + (int64_t)(it.bn * BN + half * 32 + j) * b + row;
                *cp = args.assign ? run[j] : *cp - run[j];
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

// the slot ring, the 1024-byte alignment of its base, the barriers, unit ends, TMEM holder and flags
constexpr size_t SMEM = (size_t)RING * SLOT + 1024 + (2 * SETS + 5) * 8 + SETS * 8 + 16;
static_assert(SMEM <= 232448, "dynamic shared memory of k_zgemm64 above the 227 KB a CTA may use");

}  // namespace z64

static int sm_count64() {            // per device, cached
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

int make_zgemm64_maps(Z64Maps *m, void *pool, int64_t nplanes, int b) {
    for (int d = 1; d <= 2; ++d)
        if (make_plane_map3(&m->x[d - 1], pool, nplanes, b, z64::BM, d)) return -1;
    for (int d = 1; d <= 5; ++d)
        if (make_plane_map3(&m->y[d - 1], pool, nplanes, b, z64::BN, d)) return -1;
    return 0;
}

void launch_zgemm64(const Z64Maps &maps, const ZItem *items, int nitems, const int *exps, int k, int b, int *err,
                    cudaStream_t s, const ZPlanes &mixed, int assign, unsigned long long limit_ns, int stall) {
    if (nitems <= 0 || k <= 0) return;
    static std::atomic<unsigned long long> attr{0};
    if (attrs_pending(attr)) {
        cudaFuncSetAttribute(z64::k_zgemm64<z64::Args>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)z64::SMEM);
        mark_attrs_set(attr);
    }
    z64::Args a{items, nitems, exps, mixed.src_planes_tab, mixed.out_amax, mixed.rref, mixed.margin, mixed.pair_count,
                k, b, err, assign, limit_ns ? limit_ns : z64::LIMIT_NS, stall};
    const int grid = nitems < sm_count64() ? nitems : sm_count64();  // persistent: one CTA per SM
    z64::k_zgemm64<z64::Args><<<grid, z64::THREADS, z64::SMEM, s>>>(maps, a);
}

}  // namespace tc
