// Out-of-core factorization (Sections III-C and IV-B, Algorithms 2 and 3): the matrix stays
// in (page-locked) host memory and a bounded pool of device tile slots caches tiles.
//
// The whole left-looking task order is known before the first launch (static schedule),
// so the host thread walks it once and enqueues everything asynchronously:
//   * load_tile (Algorithm 3): a cached tile is reused (hit); a miss takes a free slot or
//     evicts the least-recently-used unpinned one, and copies the tile in on the H2D stream;
//   * the accumulator tile (m, k) stays resident while its updates run (V1), and the
//     diagonal tile L_kk stays pinned until every TRSM of column k is done (V3);
//   * each final tile is copied back to its place in the host matrix on the D2H stream
//     (Algorithm 2), overwriting A with L.
// Stream order plus events replace the paper's Ready table and busy-waits: a copy into a
// slot waits for the last kernel that read the evicted tile and for that tile's write-back;
// a kernel waits for the copies of its operands; a re-load of a written-back tile waits for
// its write-back.  Nothing on the host blocks until the end of the call.
//
// The accumulators of a tile column are taken G at a time (the same left-looking order,
// grouped so that one TRSM launch, and with tensor-core updates one update launch per
// precision, covers G tiles and fills the GPU).  With emulated FP64 updates every slot also
// holds the tile's 14 digit planes, made on the device when a final tile is first used as an
// operand after it arrived (or after it was factored).
//
// Mixed precision (Section IV-C with Section III-C): a final tile of precision p < FP64 is
// rounded to its stored value, written back to the host matrix as FP64 (the result) and as a
// compact copy at p's width (4, 2 or 1 bytes per element) into a page-locked host store;
// every later load of it moves only the compact copy and widens it on the device -- the
// host-link traffic of re-loads shrinks with the precision, the paper's point.  Updates run
// in the output tile's precision: FP64 and FP32 outputs on digit planes (14 / 10 planes),
// FP16 and FP8 outputs on scaled FP16 / E4M3 operand copies made per slot on first use.
#include "tc_handle.h"

#include <algorithm>
#include <cmath>
#include <cstring>

using namespace tc;

namespace {

enum OpForm { OP_Z14 = 0, OP_Z10, OP_Q16, OP_Q8, OP_N };

// Scheduling policies of Section III-C (tc_config.ooc): V3 the default; V2 without the
// diagonal pin; V1 without operand reuse; async without accumulator residency (every update
// step loads its accumulator and copies it back); sync as async with every copy on the
// compute stream (no overlap).
enum OocPolicy { OOC_V3 = 0, OOC_V2 = 1, OOC_V1 = 2, OOC_ASYNC = 3, OOC_SYNC = 4 };

inline int elem_bytes(int p) { return p == TC_FP32 ? 4 : p == TC_FP16 ? 2 : p == TC_FP8 ? 1 : 8; }

struct TileCache {
    tc_handle h;
    double *pool = nullptr;      // FP64 tile per slot
    uint8_t *dpool = nullptr;    // digit planes, 14 b^2 bytes per slot
    __half *p16 = nullptr;       // mixed: scaled FP16 operand copy per slot
    uint8_t *p8 = nullptr;       // mixed: scaled E4M3 operand copy per slot
    uint8_t *stage = nullptr;    // mixed: compact copy in flight, 4 b^2 bytes per slot
    int *exps = nullptr;         // per-slot digit exponent
    int *e16 = nullptr, *e8 = nullptr;   // per-slot operand-copy exponents
    double *amax = nullptr;      // per-slot max |a| of the (stored) tile
    double *amaxL = nullptr;     // per-slot max |a| before rounding to the stored precision
    int *tile_e = nullptr;       // per-tile storage scale exponent (FP16 / FP8 tiles)
    CUtensorMap mx, my, m16, m8;
    std::vector<char> has_amax, dig, c16, c8;
    // host side
    double *host = nullptr;      // the matrix in host memory (tile layout), in/out
    uint8_t *hcompact = nullptr; // compact copies of final low-precision tiles
    std::vector<int64_t> hoff;   // their offsets (-1: FP64 tile)
    std::vector<uint8_t> prec;   // stored precision of each tile (mixed)
    std::vector<char> final_;    // tile has been factored and written back
    int nslots = 0, b = 0;
    int64_t bb = 0;
    size_t tile_bytes = 0;
    cudaStream_t cs, h2d, d2h;
    std::vector<int> slot_tile, pins, where;
    std::vector<int> prev_tile;        // tile a free slot held before it was dropped (-1: none)
    std::vector<uint64_t> last;
    std::vector<cudaEvent_t> ready, used;
    std::vector<cudaEvent_t> tile_wb;
    std::vector<char> wb_pending;
    uint64_t clock = 0;
    int64_t hits = 0, misses = 0, evictions = 0, h2d_bytes = 0, d2h_bytes = 0, conversions = 0;
    // Belady's MIN (optional): for request i, the index of the next request of the same tile
    const std::vector<int64_t> *future = nullptr;
    int64_t req = 0;
    std::vector<int64_t> next_use;

    double *ptr(int s) const { return pool + (int64_t)s * bb; }
    uint8_t *stg(int s) const { return stage + (int64_t)s * 4 * bb; }
    bool compact(int t) const { return !prec.empty() && prec[t] != TC_FP64; }

    cudaEvent_t wb_event(int t) {
        if (!tile_wb[t]) cudaEventCreateWithFlags(&tile_wb[t], cudaEventDisableTiming);
        return tile_wb[t];
    }

    // Algorithm 3: slot holding tile t (copied in on a miss when `load`: as FP64, or for a
    // final low-precision tile as its compact copy, widened on the compute stream); -1 if
    // every slot is pinned (cache too small for the schedule).
    int acquire(int t, bool load) {
        const int64_t nxt = (future && req < (int64_t)future->size()) ? (*future)[req] : 0;
        ++req;
        if (where[t] >= 0) {
            const int s = where[t];
            ++hits;
            last[s] = ++clock;
            if (future) next_use[s] = nxt;
            cudaStreamWaitEvent(cs, ready[s], 0);
            return s;
        }
        ++misses;
        int v = -1;
        for (int s = 0; s < nslots && v < 0; ++s)
            if (slot_tile[s] < 0) v = s;
        if (v < 0 && future) {
            int64_t best = -1;
            for (int s = 0; s < nslots; ++s)
                if (pins[s] == 0 && next_use[s] > best) {
                    best = next_use[s];
                    v = s;
                }
        } else if (v < 0) {
            uint64_t best = ~0ull;
            for (int s = 0; s < nslots; ++s)
                if (pins[s] == 0 && last[s] < best) {
                    best = last[s];
                    v = s;
                }
        }
        if (v < 0) return -1;
        // the tile the slot held last (evicted now, or dropped earlier): its write-back reads
        // the slot, so the copy into it waits for that write-back
        const int old = slot_tile[v] >= 0 ? slot_tile[v] : prev_tile[v];
        if (slot_tile[v] >= 0) {
            ++evictions;
            where[old] = -1;
        }
        if (old >= 0 && wb_pending[old]) cudaStreamWaitEvent(h2d, tile_wb[old], 0);
        cudaStreamWaitEvent(h2d, used[v], 0);                                  // last kernel that read the slot
        const bool packed = load && final_[t] && compact(t);
        if (load) {
            if (wb_pending[t]) cudaStreamWaitEvent(h2d, tile_wb[t], 0);        // host copy must be final
            if (packed) {
                const size_t nb = (size_t)bb * elem_bytes(prec[t]);
                cudaMemcpyAsync(stg(v), hcompact + hoff[t], nb, cudaMemcpyHostToDevice, h2d);
                h2d_bytes += (int64_t)nb;
            } else {
                cudaMemcpyAsync(ptr(v), host + (int64_t)t * bb, tile_bytes, cudaMemcpyHostToDevice, h2d);
                h2d_bytes += (int64_t)tile_bytes;
            }
        }
        cudaEventRecord(ready[v], h2d);
        if (!dig.empty()) dig[v] = 0;
        if (!c16.empty()) c16[v] = c8[v] = 0;
        if (!has_amax.empty()) has_amax[v] = 0;
        slot_tile[v] = t;
        where[t] = v;
        last[v] = ++clock;
        if (future) next_use[v] = nxt;
        cudaStreamWaitEvent(cs, ready[v], 0);
        if (packed) launch_unpack_compact(stg(v), b, prec[t], tile_e + t, ptr(v), cs);
        return v;
    }

    void touched(int s) { cudaEventRecord(used[s], cs); }

    // the operand form `f` of the final tile in slot s, made on first use
    void make_form(int s, int f) {
        char &have = (f <= OP_Z10) ? dig[s] : (f == OP_Q16 ? c16[s] : c8[s]);
        if (have) return;
        const int sp = span_begin(h, CAT_CONVERT);
        if (!has_amax[s]) {
            cudaMemsetAsync(amax + s, 0, sizeof(double), cs);
            launch_amax_ptr(ptr(s), bb, amax + s, cs);
            has_amax[s] = 1;
        }
        if (f <= OP_Z10) launch_digits_src(ptr(s), b, 0, s, amax + s, dpool, exps, cs);
        else launch_copy_slot(pool, b, s, f == OP_Q16 ? TC_FP16 : TC_FP8, amax, p16, p8, e16, e8, cs);
        span_end(h, sp);
        have = 1;
        ++conversions;
    }

    // digit planes of the b x b matrix at src into digit slot d (d may be the extra slot)
    void planes_of(const double *src, int d, int transpose = 0) {
        cudaMemsetAsync(amax + d, 0, sizeof(double), cs);
        launch_amax_ptr(src, bb, amax + d, cs);
        launch_digits_src(src, b, transpose, d, amax + d, dpool, exps, cs);
    }

    int acquire_op(int t, int f) {
        const int s = acquire(t, true);
        if (s >= 0) make_form(s, f);
        return s;
    }

    // drop slot s from the cache (policies without reuse); its next use re-loads the tile
    void forget(int s) {
        if (s < 0 || pins[s] != 0 || slot_tile[s] < 0) return;
        where[slot_tile[s]] = -1;
        prev_tile[s] = slot_tile[s];
        slot_tile[s] = -1;
    }

    // Algorithm 2's memcpy_GPU_to_CPU: final tile back to the host matrix (and, for a
    // low-precision tile, rounded to its stored value first and its compact copy saved);
    // `partial`: an accumulator that is not final yet (async policies), copied back as is
    void write_back(int t, int s, bool partial = false) {
        if (partial) {
            cudaEventRecord(used[s], cs);
            cudaStreamWaitEvent(d2h, used[s], 0);
            cudaMemcpyAsync(host + (int64_t)t * bb, ptr(s), tile_bytes, cudaMemcpyDeviceToHost, d2h);
            d2h_bytes += (int64_t)tile_bytes;
            cudaEventRecord(wb_event(t), d2h);
            wb_pending[t] = 1;
            return;
        }
        const int p = prec.empty() ? (int)TC_FP64 : (int)prec[t];
        if (p != TC_FP64) {
            const int sp = span_begin(h, CAT_CONVERT);
            cudaMemsetAsync(amaxL + s, 0, sizeof(double), cs);
            launch_amax_ptr(ptr(s), bb, amaxL + s, cs);
            launch_round_slot(ptr(s), b, p, amaxL + s, tile_e + t, cs);
            launch_pack_compact(ptr(s), b, p, tile_e + t, stg(s), cs);
            span_end(h, sp);
        }
        cudaEventRecord(used[s], cs);
        cudaStreamWaitEvent(d2h, used[s], 0);
        cudaMemcpyAsync(host + (int64_t)t * bb, ptr(s), tile_bytes, cudaMemcpyDeviceToHost, d2h);
        d2h_bytes += (int64_t)tile_bytes;
        if (p != TC_FP64) {
            const size_t nb = (size_t)bb * elem_bytes(p);
            cudaMemcpyAsync(hcompact + hoff[t], stg(s), nb, cudaMemcpyDeviceToHost, d2h);
            d2h_bytes += (int64_t)nb;
        }
        cudaEventRecord(wb_event(t), d2h);
        wb_pending[t] = 1;
        final_[t] = 1;
    }

    void destroy() {
        for (auto *v : {&ready, &used, &tile_wb})
            for (cudaEvent_t e : *v)
                if (e) cudaEventDestroy(e);
    }
};

int ooc_streams(tc_handle h) {
    if (!h->s_h2d) CK(cudaStreamCreateWithFlags(&h->s_h2d, cudaStreamNonBlocking));
    if (!h->s_d2h) CK(cudaStreamCreateWithFlags(&h->s_d2h, cudaStreamNonBlocking));
    return TC_OK;
}

// Bytes of one cache slot: the FP64 tile, with emulated updates its 14 digit planes, and in
// mixed precision the FP16 and E4M3 operand copies and a 4-byte-per-element compact stage.
int64_t slot_bytes(int64_t bb, bool digits, bool mixed) {
    return 8 * bb + (digits ? 14 * bb + 16 : 0) + (mixed ? 7 * bb + 24 : 0);
}

int init_cache(tc_handle h, TileCache &C, double *host, int nt, int b, bool digits, const uint8_t *map = nullptr) {
    const int64_t T = tidx(nt, 0);
    const bool mixed = map != nullptr;
    C.h = h;
    C.host = host;
    C.b = b;
    C.bb = (int64_t)b * b;
    C.tile_bytes = (size_t)C.bb * sizeof(double);
    int64_t cap = h->cfg.device_cap_bytes;
    if (cap <= 0) {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        cap = (int64_t)fr - ((int64_t)4 << 30);
    }
    int64_t ns = cap / slot_bytes(C.bb, digits, mixed);
    ns = std::min<int64_t>(ns, T + 2);
    if (ns < 4) return set_err(h, TC_ERR_OOM, "device tile cache below 4 tiles");
    if (digits && ns > 65535) ns = 65535;          // operand slots travel as 16-bit indices
    C.nslots = (int)ns;
    int rc = ensure(h, h->W, (size_t)ns * C.tile_bytes);
    if (rc) return rc;
    C.pool = static_cast<double *>(h->W.p);
    if (digits) {
        // one digit slot beyond the cache (index ns) holds the planes of L_kk^{-1}
        const int64_t nd = ns + 1;
        if ((rc = ensure(h, h->dpool, (size_t)nd * 14 * C.bb))) return rc;
        if ((rc = ensure(h, h->ztab, (size_t)nd * (2 * sizeof(double) + 3 * sizeof(int)) + (size_t)T * sizeof(int))))
            return rc;
        C.dpool = static_cast<uint8_t *>(h->dpool.p);
        C.amax = static_cast<double *>(h->ztab.p);
        C.amaxL = C.amax + nd;
        C.exps = reinterpret_cast<int *>(C.amaxL + nd);
        C.e16 = C.exps + nd;
        C.e8 = C.e16 + nd;
        C.tile_e = C.e8 + nd;
        if (make_digit_map(&C.mx, C.dpool, nd * 14 * b, b, 128) || make_digit_map(&C.my, C.dpool, nd * 14 * b, b, Z_BN))
            return set_err(h, TC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the digit-plane cache");
        C.dig.assign(ns, 0);
        C.has_amax.assign(ns, 0);
    }
    C.final_.assign(T, 0);
    if (mixed) {
        if ((rc = ensure(h, h->pool16, (size_t)ns * 2 * C.bb)) || (rc = ensure(h, h->pool8, (size_t)ns * C.bb)) ||
            (rc = ensure(h, h->pool_hi, (size_t)ns * 4 * C.bb)))
            return rc;
        C.p16 = static_cast<__half *>(h->pool16.p);
        C.p8 = static_cast<uint8_t *>(h->pool8.p);
        C.stage = static_cast<uint8_t *>(h->pool_hi.p);
        if (make_pool_map(&C.m16, C.p16, ns, b, 2, 128) || make_pool_map(&C.m8, C.p8, ns, b, 1, 128))
            return set_err(h, TC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the operand-copy cache");
        C.c16.assign(ns, 0);
        C.c8.assign(ns, 0);
        // compact host store: one region per low-precision tile, in tile order
        C.prec.assign(T, TC_FP64);
        C.hoff.assign(T, -1);
        int64_t off = 0;
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < i; ++j) {
                const int64_t t = tidx(i, j);
                C.prec[t] = map[(size_t)i * nt + j];
                if (C.prec[t] != TC_FP64) {
                    C.hoff[t] = off;
                    off += (C.bb * elem_bytes(C.prec[t]) + 255) / 256 * 256;
                }
            }
        if ((size_t)off > h->hcompact_bytes) {
            if (h->hcompact) cudaFreeHost(h->hcompact);
            h->hcompact = nullptr;
            h->hcompact_bytes = 0;
            cudaError_t e = cudaHostAlloc(&h->hcompact, (size_t)off, cudaHostAllocDefault);
            if (e != cudaSuccess) {
                cudaGetLastError();
                h->hcompact = nullptr;
                return set_err(h, TC_ERR_HOSTMEM, "page-locked host store for compact tiles could not be allocated");
            }
            h->hcompact_bytes = (size_t)off;
        }
        C.hcompact = static_cast<uint8_t *>(h->hcompact);
    }
    if ((rc = ooc_streams(h))) return rc;
    C.cs = h->s;
    C.h2d = h->s_h2d;
    C.d2h = h->s_d2h;
    if (h->cfg.ooc == OOC_SYNC) C.h2d = C.d2h = h->s;      // no copy / compute overlap
    C.slot_tile.assign(ns, -1);
    C.prev_tile.assign(ns, -1);
    C.pins.assign(ns, 0);
    C.last.assign(ns, 0);
    C.where.assign(T, -1);
    C.tile_wb.assign(T, nullptr);
    C.wb_pending.assign(T, 0);
    C.ready.resize(ns);
    C.used.resize(ns);
    for (int s = 0; s < ns; ++s) {
        CK(cudaEventCreateWithFlags(&C.ready[s], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&C.used[s], cudaEventDisableTiming));
    }
    return TC_OK;
}

#define ACQ(var, tile, load)                                                                 \
    const int var = C.acquire((tile), (load));                                               \
    if (var < 0) {                                                                           \
        C.destroy();                                                                         \
        return set_err(h, TC_ERR_OOM, "device tile cache too small for the schedule");       \
    }
#define ACQ_OP(var, tile, form)                                                              \
    const int var = C.acquire_op((tile), (form));                                            \
    if (var < 0) {                                                                           \
        C.destroy();                                                                         \
        return set_err(h, TC_ERR_OOM, "device tile cache too small for the schedule");       \
    }

// Accumulators per group and operand tiles per tensor-core update launch for a cache of
// `nslots` slots: the group fills the GPU's 152 SMs (TRSM: b/64 strips per tile) while its
// accumulators hold at most an eighth of the cache, and the pinned set of one launch (the
// diagonal tile, G accumulators, kc (G + 1) operands) fits in the cache.
struct OocShape {
    int group, chunk;
};
OocShape ooc_shape(int nslots, int b, bool zmode) {
    const int strips = b / 64;
    int G = std::max(1, std::min(std::min(TG_MAX, (2 * 152 + strips - 1) / strips), nslots / 8));
    if (zmode) {
        G = std::min(G, ZG_MAX);
        G = std::max(1, std::min(G, (nslots - 3) / 2));
        const int kc = std::max(1, std::min(ZK_MAX, (nslots - 2 - G) / (G + 1)));
        return {G, kc};
    }
    G = std::max(1, std::min(G, nslots - 3));
    return {G, 0};
}

// The tile requests (acquisitions) of the factorization loop below, in order, for Belady's
// MIN: the sequence depends on the schedule (policy, group, chunk) but not on what the cache
// holds.  It must follow the loop's acquisition order; the tests hold the library's
// counters equal to the schedule simulator's under MIN.
std::vector<int64_t> ooc_future(int nt, const OocShape &S, bool zmode, int policy) {
    const bool pin_diag = policy == OOC_V3, keep_acc = policy <= OOC_V1;
    std::vector<int> seq;
    for (int k = 0; k < nt; ++k)
        for (int g0 = k; g0 < nt; g0 += S.group) {
            const int g1 = std::min(nt, g0 + S.group);
            auto accs = [&] {
                for (int m = g0; m < g1; ++m) seq.push_back((int)tidx(m, k));
            };
            if (keep_acc) accs();
            if (zmode) {
                for (int n0 = 0; n0 < k; n0 += S.chunk) {
                    const int kc = std::min(S.chunk, k - n0);
                    if (!keep_acc) accs();
                    for (int nn = n0; nn < n0 + kc; ++nn) seq.push_back((int)tidx(k, nn));
                    for (int m = g0; m < g1; ++m)
                        for (int nn = n0; nn < n0 + kc; ++nn) seq.push_back((int)tidx(m, nn));
                }
            } else {
                for (int m = g0; m < g1; ++m)
                    for (int nn = 0; nn < k; ++nn) {
                        if (!keep_acc) seq.push_back((int)tidx(m, k));
                        seq.push_back((int)tidx(m, nn));
                        seq.push_back((int)tidx(k, nn));
                    }
            }
            if (!keep_acc) accs();
            if (g0 != k && !pin_diag) seq.push_back((int)tidx(k, k));
        }
    std::vector<int64_t> future(seq.size());
    std::vector<int64_t> seen(tidx(nt, 0), (int64_t)seq.size() + 1);
    for (int64_t i = (int64_t)seq.size() - 1; i >= 0; --i) {
        future[i] = seen[seq[i]];
        seen[seq[i]] = i;
    }
    return future;
}

}  // namespace

extern "C" int tile_chol_factor_ooc(tc_handle h, int64_t n, int b, double *A_tiles, const uint8_t *map,
                                    tc_stats *stats) {
    int rc = check_nb(h, n, b);
    if (rc) return rc;
    if (!A_tiles) return set_err(h, TC_ERR_ARG, "A_tiles must not be NULL");
    if (on_device(A_tiles)) return set_err(h, TC_ERR_ARG, "out-of-core factorization needs A_tiles in host memory");
    const int nt = (int)((n + b - 1) / b);
    std::vector<uint8_t> pm((size_t)nt * nt, TC_FP64);
    bool mixed = false;
    if (map) {
        if (on_device(map)) CK(cudaMemcpy(pm.data(), map, pm.size(), cudaMemcpyDeviceToHost));
        else memcpy(pm.data(), map, pm.size());
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j <= i; ++j) {
                uint8_t &v = pm[(size_t)i * nt + j];
                if (i == j) v = TC_FP64;
                if (v > TC_FP8) return set_err(h, TC_ERR_ARG, "precision map entries must be 0..3");
                mixed |= (v != TC_FP64);
            }
    }
    const bool zmode = h->cfg.fp64_mode >= 1;
    const int policy = h->cfg.ooc;
    if (policy < OOC_V3 || policy > OOC_SYNC) return set_err(h, TC_ERR_ARG, "tc_config.ooc must be 0..4 (V3, V2, V1, async, sync)");
    if (h->cfg.ooc_eviction < 0 || h->cfg.ooc_eviction > 1)
        return set_err(h, TC_ERR_ARG, "tc_config.ooc_eviction must be 0 (LRU) or 1 (Belady MIN)");
    const bool keep_ops = policy <= OOC_V2, pin_diag = policy == OOC_V3, keep_acc = policy <= OOC_V1;
    if (mixed && !zmode)
        return set_err(h, TC_ERR_UNSUPPORTED, "out-of-core mixed precision runs on the tensor-core engine (fp64_mode >= 1)");
    if (zmode && b % 128)
        return set_err(h, TC_ERR_UNSUPPORTED, "emulated FP64 updates need a tile size that is a multiple of 128");
    CK(cudaSetDevice(h->device));
    const double t0 = now_ms();
    const int64_t launches0 = h->launches;
    h->factored = false;
    h->ooc = false;
    h->n = n;
    h->b = b;
    h->nt = nt;
    h->map = pm;
    h->mixed = mixed;
    h->A_dev = nullptr;
    spans_reset(h);
    for (int p = 0; p < 4; ++p) h->upd_launches[p] = 0;
    if (h->graph) {                      // the slot pool may move: no replay of an old graph
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        h->graph_key.clear();
    }
    TileCache C;
    if ((rc = init_cache(h, C, A_tiles, nt, b, zmode, mixed ? pm.data() : nullptr))) return rc;
    if ((rc = ensure(h, h->logdiag, (size_t)nt * sizeof(double)))) return rc;
    double *logdiag = static_cast<double *>(h->logdiag.p);
    int *status = static_cast<int *>(h->status.p);
    CK(cudaMemsetAsync(status, 0, 2 * sizeof(int), h->s));
    const int nv_last = (int)(n - (int64_t)(nt - 1) * b);
    double upd_flops[4] = {0, 0, 0, 0};
    int64_t tiles_p[4] = {0, 0, 0, 0};
    const OocShape S = ooc_shape(C.nslots, b, zmode);
    std::vector<int64_t> future;
    if (h->cfg.ooc_eviction == 1) {
        future = ooc_future(nt, S, zmode, policy);
        C.future = &future;
        C.next_use.assign(C.nslots, 0);
    }
    // fp64_mode 2: TRSM as products with L_kk^{-1} on the emulated engine (FP64 tiles refined
    // once with the exact residual), L_kk^{-1} at invbuf, X0 of group tile i at invbuf + (1+i) b^2
    const bool inv_trsm = zmode && h->cfg.fp64_mode == 2;
    const int vslot = C.nslots;          // extra digit slot: planes of L_kk^{-1}
    double *inv = nullptr;
    if (inv_trsm) {
        if ((rc = ensure(h, h->invbuf, (size_t)(1 + S.group) * C.bb * sizeof(double)))) return rc;
        inv = static_cast<double *>(h->invbuf.p);
    }
    // output precision -> operand form and update category
    auto form_of = [&](int m, int k) {
        const int p = (m == k) ? (int)TC_FP64 : (int)pm[(size_t)m * nt + k];
        return p == TC_FP64 ? OP_Z14 : p == TC_FP32 ? OP_Z10 : p == TC_FP16 ? OP_Q16 : OP_Q8;
    };
    static const int cat_of[OP_N] = {CAT_UPD64, CAT_UPD32, CAT_UPD16, CAT_UPD8};
    static const int prec_of[OP_N] = {TC_FP64, TC_FP32, TC_FP16, TC_FP8};

    for (int k = 0; k < nt; ++k) {
        int diag_slot = -1;
        for (int g0 = k; g0 < nt; g0 += S.group) {
            const int g1 = std::min(nt, g0 + S.group);
            int sc[ZG_MAX];
            // V1-V3: the accumulators stay resident (and pinned) through their updates
#define ACQ_ACCS()                                                                            \
    for (int m = g0; m < g1; ++m) {                                                           \
        ACQ(s_acc, (int)tidx(m, k), true);                                                    \
        sc[m - g0] = s_acc;                                                                   \
        ++C.pins[s_acc];                                                                      \
        if (m == nt - 1 && nv_last != b) {                                                    \
            launch_fix_padding_tile(C.ptr(s_acc), b, nv_last, m == k, h->s);                  \
            CK_LAUNCH();                                                                      \
        }                                                                                     \
    }
            // async / sync: every update step copies its accumulators back and lets them go
#define RELEASE_ACCS()                                                                        \
    for (int m = g0; m < g1; ++m) {                                                           \
        C.write_back((int)tidx(m, k), sc[m - g0], true);                                      \
        --C.pins[sc[m - g0]];                                                                 \
        C.forget(sc[m - g0]);                                                                 \
    }
            if (keep_acc) ACQ_ACCS();
            if (zmode) {
                bool present[OP_N] = {false, false, false, false};
                for (int m = g0; m < g1; ++m) present[form_of(m, k)] = true;
                for (int n0 = 0; n0 < k; n0 += S.chunk) {
                    const int kc = std::min(S.chunk, k - n0);
                    int ys[ZK_MAX], xs[ZG_MAX][ZK_MAX];
                    if (!keep_acc) ACQ_ACCS();
                    for (int nn = n0; nn < n0 + kc; ++nn) {
                        ACQ(sy, (int)tidx(k, nn), true);
                        for (int f = 0; f < OP_N; ++f)
                            if (present[f]) C.make_form(sy, f);
                        ys[nn - n0] = sy;
                        ++C.pins[sy];
                    }
                    for (int m = g0; m < g1; ++m)
                        for (int nn = n0; nn < n0 + kc; ++nn) {
                            ACQ_OP(sx, (int)tidx(m, nn), form_of(m, k));
                            xs[m - g0][nn - n0] = sx;
                            ++C.pins[sx];
                        }
                    for (int f = 0; f < OP_N; ++f) {
                        if (!present[f]) continue;
                        ZGroup zg;
                        QGroup qg;
                        int cnt = 0;
                        for (int m = g0; m < g1; ++m) {
                            if (form_of(m, k) != f) continue;
                            double *Cp = C.ptr(sc[m - g0]);
                            if (f <= OP_Z10) {
                                zg.C[cnt] = Cp;
                                zg.lower[cnt] = (m == k);
                                for (int q = 0; q < kc; ++q) zg.xs[cnt][q] = xs[m - g0][q];
                            } else {
                                qg.C[cnt] = Cp;
                                for (int q = 0; q < kc; ++q) qg.xs[cnt][q] = xs[m - g0][q];
                            }
                            upd_flops[prec_of[f]] += (m == k ? 1.0 : 2.0) * kc * (double)b * b * b;
                            ++cnt;
                        }
                        const int spz = span_begin(h, cat_of[f]);   // operands are resident from here
                        if (f <= OP_Z10) {
                            zg.ntiles = cnt;
                            zg.k = kc;
                            for (int q = 0; q < kc; ++q) zg.ys[q] = ys[q];
                            launch_zgemm_group(C.mx, C.my, zg, C.exps, b, status + 1, h->s, f == OP_Z14 ? 14 : 10, wait_limit_ns(h), wait_test(h));
                        } else {
                            qg.ntiles = cnt;
                            qg.k = kc;
                            for (int q = 0; q < kc; ++q) qg.ys[q] = ys[q];
                            launch_qgemm_group(f == OP_Q16 ? 2 : 3, f == OP_Q16 ? C.m16 : C.m8,
                                               f == OP_Q16 ? C.m16 : C.m8, qg, f == OP_Q16 ? C.e16 : C.e8, b,
                                               status + 1, h->s, wait_limit_ns(h), wait_test(h));
                        }
                        span_end(h, spz);
                        CK_LAUNCH();
                        ++h->upd_launches[prec_of[f]];
                    }
                    for (int m = g0; m < g1; ++m)
                        for (int q = 0; q < kc; ++q) {
                            C.touched(xs[m - g0][q]);
                            --C.pins[xs[m - g0][q]];
                        }
                    for (int q = 0; q < kc; ++q) {
                        C.touched(ys[q]);
                        --C.pins[ys[q]];
                    }
                    if (!keep_ops) {                 // V1 / async / sync: no operand table
                        for (int m = g0; m < g1; ++m)
                            for (int q = 0; q < kc; ++q) C.forget(xs[m - g0][q]);
                        for (int q = 0; q < kc; ++q) C.forget(ys[q]);
                    }
                    if (!keep_acc) RELEASE_ACCS();
                }
            } else {
                for (int m = g0; m < g1; ++m)
                    for (int nn = 0; nn < k; ++nn) {
                        int sa = keep_acc ? sc[m - g0] : -1;
                        if (!keep_acc) {
                            ACQ(s1, (int)tidx(m, k), true);
                            sa = s1;
                            ++C.pins[sa];
                            if (m == nt - 1 && nv_last != b) {
                                launch_fix_padding_tile(C.ptr(sa), b, nv_last, m == k, h->s);
                                CK_LAUNCH();
                            }
                        }
                        ACQ(sx, (int)tidx(m, nn), true);
                        ++C.pins[sx];
                        ACQ(sy, (int)tidx(k, nn), true);
                        const int spd = span_begin(h, CAT_UPD64);   // operands are resident from here
                        launch_dgemm_tile({C.ptr(sa), C.ptr(sx), C.ptr(sy), b, b, b, m == k ? 1 : 0, nullptr}, b, h->s);
                        span_end(h, spd);
                        CK_LAUNCH();
                        ++h->upd_launches[TC_FP64];
                        upd_flops[TC_FP64] += (m == k ? 1.0 : 2.0) * (double)b * b * b;
                        C.touched(sx);
                        C.touched(sy);
                        --C.pins[sx];
                        if (!keep_ops) {
                            C.forget(sx);
                            C.forget(sy);
                        }
                        if (!keep_acc) {
                            C.write_back((int)tidx(m, k), sa, true);
                            --C.pins[sa];
                            C.forget(sa);
                        }
                    }
            }
            if (!keep_acc) ACQ_ACCS();               // the accumulators once more, for POTRF / TRSM
            if (g0 != k && !pin_diag) {              // V2 and below: L_kk may have left the cache
                ACQ(sd, (int)tidx(k, k), true);
                diag_slot = sd;
                ++C.pins[sd];
                if (inv_trsm && k + 1 < nt) {
                    C.planes_of(C.ptr(sd), sd, 0);
                    C.dig[sd] = C.has_amax[sd] = 0;
                }
            }
            if (g0 == k) {
                double *D = C.ptr(sc[0]);
                const int spp = span_begin(h, CAT_POTRF);
                for (int jb = 0; jb < b / 64; ++jb) {
                    launch_potrf_block(D + (int64_t)jb * 64 * b + jb * 64, b, k * b + jb * 64, status, h->s);
                    CK_LAUNCH();
                    if (jb + 1 < b / 64) {
                        const int rows = b - (jb + 1) * 64;
                        launch_trsm_rows(D + (int64_t)jb * 64 * b + (jb + 1) * 64, D + (int64_t)jb * 64 * b + jb * 64,
                                         b, rows, status, h->s);
                        CK_LAUNCH();
                        const double *Pn = D + (int64_t)jb * 64 * b + (jb + 1) * 64;
                        launch_dgemm_tile({D + (int64_t)(jb + 1) * 64 * b + (jb + 1) * 64, Pn, Pn, 64, rows, rows, 1, nullptr},
                                          b, h->s);
                        CK_LAUNCH();
                    }
                }
                launch_logdiag_tile(D, b, k == nt - 1 ? nv_last : b, logdiag + k, h->s);
                CK_LAUNCH();
                span_end(h, spp);
                diag_slot = sc[0];               // V3: pinned until the column's TRSMs are done
                if (inv_trsm && k + 1 < nt) {
                    const int spi = span_begin(h, CAT_TRSM);
                    launch_lower_only(D, b, h->s);
                    if (b <= 2048) {
                        launch_trinv(D, b, inv, h->s);
                        C.planes_of(inv, vslot, 0);
                    } else {
                        launch_set_identity(inv, b, h->s);
                        launch_trsm_tile(inv, D, b, b, nullptr, h->s);   // L_kk^{-T}
                        C.planes_of(inv, vslot, 1);
                    }
                    C.planes_of(D, diag_slot, 0);    // L_kk (a diagonal tile is never an update operand)
                    C.dig[diag_slot] = 0;
                    C.has_amax[diag_slot] = 0;
                    span_end(h, spi);
                    CK_LAUNCH();
                }
            }
            double *off[ZG_MAX];
            int noff = 0;
            for (int m = std::max(g0, k + 1); m < g1; ++m) off[noff++] = C.ptr(sc[m - g0]);
            if (noff && inv_trsm) {
                const int spt = span_begin(h, CAT_TRSM);
                int so[ZG_MAX], ref[ZG_MAX], nref = 0;
                for (int m = std::max(g0, k + 1); m < g1; ++m) so[m - std::max(g0, k + 1)] = sc[m - g0];
                // X0 = C L^{-T} (FP64 tiles into the scratch X0, refined below; the others final,
                // on as many planes as their stored precision needs)
                ZGroup z1[4];
                for (int p = 0; p < 4; ++p) {
                    z1[p].k = 1;
                    z1[p].assign = 1;
                    z1[p].ys[0] = vslot;
                }
                for (int i = 0; i < noff; ++i) {
                    const int m = std::max(g0, k + 1) + i;
                    const int p = pm[(size_t)m * nt + k];
                    const bool refine = p == TC_FP64;
                    C.planes_of(C.ptr(so[i]), so[i]);
                    ZGroup &z = z1[p];
                    z.C[z.ntiles] = refine ? inv + (int64_t)(1 + i) * C.bb : C.ptr(so[i]);
                    z.xs[z.ntiles][0] = so[i];
                    ++z.ntiles;
                    if (refine) ref[nref++] = i;
                }
                for (int p = 0; p < 4; ++p)
                    launch_zgemm_group(C.mx, C.my, z1[p], C.exps, b, status + 1, h->s, ZTRSM_PLANES[p], wait_limit_ns(h), wait_test(h));
                if (nref) {
                    ZGroup z2, z3;
                    z2.ntiles = z3.ntiles = nref;
                    z2.k = z3.k = 1;
                    z2.assign = 0;
                    z3.assign = 1;
                    z2.ys[0] = diag_slot;
                    z3.ys[0] = vslot;
                    for (int r = 0; r < nref; ++r) {
                        const int i = ref[r];
                        C.planes_of(inv + (int64_t)(1 + i) * C.bb, so[i]);
                        z2.C[r] = z3.C[r] = C.ptr(so[i]);
                        z2.xs[r][0] = z3.xs[r][0] = so[i];
                    }
                    launch_zgemm_group(C.mx, C.my, z2, C.exps, b, status + 1, h->s, 14, wait_limit_ns(h), wait_test(h));  // R = C - X0 L^T
                    for (int r = 0; r < nref; ++r) C.planes_of(C.ptr(so[ref[r]]), so[ref[r]]);
                    launch_zgemm_group(C.mx, C.my, z3, C.exps, b, status + 1, h->s, ZREF_PLANES, wait_limit_ns(h), wait_test(h));  // R L^{-T}
                    for (int r = 0; r < nref; ++r)
                        launch_add_tile(C.ptr(so[ref[r]]), inv + (int64_t)(1 + ref[r]) * C.bb, b, h->s);
                }
                for (int i = 0; i < noff; ++i) C.dig[so[i]] = C.has_amax[so[i]] = 0;
                span_end(h, spt);
                CK_LAUNCH();
                C.touched(diag_slot);
            } else if (noff) {
                const int spt = span_begin(h, CAT_TRSM);
                launch_trsm_group(off, noff, C.ptr(diag_slot), b, b, status, h->s);
                span_end(h, spt);
                CK_LAUNCH();
                C.touched(diag_slot);
            }
            for (int m = g0; m < g1; ++m) {
                const int t = (int)tidx(m, k);
                C.write_back(t, sc[m - g0]);
                ++tiles_p[m == k ? (int)TC_FP64 : (int)pm[(size_t)m * nt + k]];
                if (m != k) --C.pins[sc[m - g0]];
            }
            if (!pin_diag) {                         // V3 alone keeps L_kk pinned for the column
                --C.pins[diag_slot];
                if (!keep_ops) C.forget(diag_slot);
            }
            if (!keep_ops)
                for (int m = std::max(g0, k + 1); m < g1; ++m) C.forget(sc[m - g0]);
        }
        if (pin_diag) --C.pins[diag_slot];
    }
#undef ACQ_ACCS
#undef RELEASE_ACCS
    std::vector<double> ld(nt);
    int st2[2] = {0, 0};
    CK(cudaMemcpyAsync(ld.data(), logdiag, nt * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(st2, status, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    CK(cudaStreamSynchronize(h->s_d2h));
    CK(cudaStreamSynchronize(h->s_h2d));
    C.destroy();
    if (st2[1]) return set_err(h, TC_ERR_TIMEOUT, "a tensor-core update timed out waiting on its pipeline");
    const int info = st2[0];
    double logdet = 0.0;
    for (int k = 0; k < nt; ++k) logdet += ld[k];
    h->logdet = 2.0 * logdet;
    h->factored = (info == 0);
    h->ooc = true;
    h->host_factor = A_tiles;
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->t_ms = now_ms() - t0;
        stats->flops = (double)n * n * n / 3.0;
        for (int p = 0; p < 4; ++p) {
            stats->update_flops[p] = upd_flops[p];
            stats->tiles[p] = tiles_p[p];
            stats->update_launches[p] = h->upd_launches[p];
        }
        stats->trsm_flops = (double)nt * (nt - 1) / 2.0 * b * (double)b * b;
        stats->potrf_flops = nt * (double)b * b * b / 3.0;
        stats->h2d_bytes = C.h2d_bytes;
        stats->d2h_bytes = C.d2h_bytes;
        stats->cache_hits = C.hits;
        stats->cache_misses = C.misses;
        stats->evictions = C.evictions;
        stats->kernel_launches = h->launches - launches0;
        stats->info = info;
        stats->ooc = 1;
        double ms[CAT_N];
        span_totals(h, ms);
        for (int p = 0; p < 4; ++p) stats->t_update_ms[p] = ms[CAT_UPD64 + p];
        stats->t_potrf_ms = ms[CAT_POTRF];
        stats->t_trsm_ms = ms[CAT_TRSM];
        stats->t_convert_ms = ms[CAT_CONVERT];
    }
    if (info) set_err(h, info, "matrix is not positive definite (see the returned column)");
    return info;
}

namespace tc {

// Forward (and back) substitution with the factor in host memory: tiles stream through the
// slot pool one tile column at a time (forward) and one tile row at a time (back).
int ooc_subst(tc_handle h, double *R, int64_t ldr, int nrhs, bool back, int64_t *h2d_bytes) {
    const int nt = h->nt, b = h->b;
    TileCache C;
    int rc = init_cache(h, C, h->host_factor, nt, b, false);
    if (rc) return rc;
    for (int c0 = 0; c0 < nrhs; c0 += 16) {
        const int nc = std::min(16, nrhs - c0);
        double *Rc = R + (int64_t)c0 * ldr;
        for (int j = 0; j < nt; ++j) {
            ACQ(sd, (int)tidx(j, j), true);
            launch_fwd_diag(C.ptr(sd), b, Rc + (int64_t)j * b, ldr, nc, h->s);
            CK_LAUNCH();
            C.touched(sd);
            for (int i = j + 1; i < nt; ++i) {
                ACQ(si, (int)tidx(i, j), true);
                launch_fwd_update_tile(C.ptr(si), b, i, j, Rc, ldr, nc, h->s);
                CK_LAUNCH();
                C.touched(si);
            }
        }
        if (!back) continue;
        for (int j = nt - 1; j >= 0; --j) {
            ACQ(sd, (int)tidx(j, j), true);
            launch_bwd_diag(C.ptr(sd), b, Rc + (int64_t)j * b, ldr, nc, h->s);
            CK_LAUNCH();
            C.touched(sd);
            for (int i = 0; i < j; ++i) {
                ACQ(si, (int)tidx(j, i), true);
                launch_bwd_update_tile(C.ptr(si), b, i, j, Rc, ldr, nc, h->s);
                CK_LAUNCH();
                C.touched(si);
            }
        }
    }
    CK(cudaStreamSynchronize(h->s));
    CK(cudaStreamSynchronize(h->s_h2d));
    if (h2d_bytes) *h2d_bytes += C.h2d_bytes;
    C.destroy();
    return TC_OK;
}

}  // namespace tc
