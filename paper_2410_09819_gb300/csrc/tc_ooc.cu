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
#include "tc_handle.h"

#include <algorithm>
#include <cmath>
#include <cstring>

using namespace tc;

namespace {

struct TileCache {
    tc_handle h;
    double *pool = nullptr;
    double *host = nullptr;      // the matrix in host memory (tile layout), in/out
    int nslots = 0;
    int64_t bb = 0;
    size_t tile_bytes = 0;
    cudaStream_t cs, h2d, d2h;
    std::vector<int> slot_tile, pins, where;
    std::vector<uint64_t> last;
    std::vector<cudaEvent_t> ready, used;
    std::vector<cudaEvent_t> tile_wb;
    std::vector<char> wb_pending;
    uint64_t clock = 0;
    int64_t hits = 0, misses = 0, evictions = 0, h2d_bytes = 0, d2h_bytes = 0;
    std::string err;

    double *ptr(int s) const { return pool + (int64_t)s * bb; }

    cudaEvent_t wb_event(int t) {
        if (!tile_wb[t]) cudaEventCreateWithFlags(&tile_wb[t], cudaEventDisableTiming);
        return tile_wb[t];
    }

    // Algorithm 3: slot holding tile t (copied in on a miss when `load`); -1 if every slot
    // is pinned (cache too small for the schedule).
    int acquire(int t, bool load) {
        if (where[t] >= 0) {
            const int s = where[t];
            ++hits;
            last[s] = ++clock;
            cudaStreamWaitEvent(cs, ready[s], 0);
            return s;
        }
        ++misses;
        int v = -1;
        for (int s = 0; s < nslots && v < 0; ++s)
            if (slot_tile[s] < 0) v = s;
        if (v < 0) {
            uint64_t best = ~0ull;
            for (int s = 0; s < nslots; ++s)
                if (pins[s] == 0 && last[s] < best) {
                    best = last[s];
                    v = s;
                }
        }
        if (v < 0) return -1;
        if (slot_tile[v] >= 0) {
            const int old = slot_tile[v];
            ++evictions;
            where[old] = -1;
            if (wb_pending[old]) cudaStreamWaitEvent(h2d, tile_wb[old], 0);   // its write-back reads the slot
        }
        cudaStreamWaitEvent(h2d, used[v], 0);                                  // last kernel that read the slot
        if (load) {
            if (wb_pending[t]) cudaStreamWaitEvent(h2d, tile_wb[t], 0);        // host copy must be final
            cudaMemcpyAsync(ptr(v), host + (int64_t)t * bb, tile_bytes, cudaMemcpyHostToDevice, h2d);
            h2d_bytes += (int64_t)tile_bytes;
        }
        cudaEventRecord(ready[v], h2d);
        slot_tile[v] = t;
        where[t] = v;
        last[v] = ++clock;
        cudaStreamWaitEvent(cs, ready[v], 0);
        return v;
    }

    void touched(int s) { cudaEventRecord(used[s], cs); }

    // Algorithm 2's memcpy_GPU_to_CPU: final tile back to the host matrix
    void write_back(int t, int s) {
        cudaEventRecord(used[s], cs);
        cudaStreamWaitEvent(d2h, used[s], 0);
        cudaMemcpyAsync(host + (int64_t)t * bb, ptr(s), tile_bytes, cudaMemcpyDeviceToHost, d2h);
        cudaEventRecord(wb_event(t), d2h);
        wb_pending[t] = 1;
        d2h_bytes += (int64_t)tile_bytes;
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

int init_cache(tc_handle h, TileCache &C, double *host, int nt, int b) {
    const int64_t T = tidx(nt, 0);
    C.h = h;
    C.host = host;
    C.bb = (int64_t)b * b;
    C.tile_bytes = (size_t)C.bb * sizeof(double);
    int64_t cap = h->cfg.device_cap_bytes;
    if (cap <= 0) {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        cap = (int64_t)fr - ((int64_t)4 << 30);
    }
    int64_t ns = cap / (int64_t)C.tile_bytes;
    ns = std::min<int64_t>(ns, T + 2);
    if (ns < 4) return set_err(h, TC_ERR_OOM, "device tile cache below 4 tiles");
    C.nslots = (int)ns;
    int rc = ensure(h, h->W, (size_t)ns * C.tile_bytes);
    if (rc) return rc;
    C.pool = static_cast<double *>(h->W.p);
    if ((rc = ooc_streams(h))) return rc;
    C.cs = h->s;
    C.h2d = h->s_h2d;
    C.d2h = h->s_d2h;
    C.slot_tile.assign(ns, -1);
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

}  // namespace

extern "C" int tile_chol_factor_ooc(tc_handle h, int64_t n, int b, double *A_tiles, const uint8_t *map,
                                    tc_stats *stats) {
    int rc = check_nb(h, n, b);
    if (rc) return rc;
    if (!A_tiles) return set_err(h, TC_ERR_ARG, "A_tiles must not be NULL");
    if (on_device(A_tiles)) return set_err(h, TC_ERR_ARG, "out-of-core factorization needs A_tiles in host memory");
    const int nt = (int)((n + b - 1) / b);
    if (map) {
        std::vector<uint8_t> m((size_t)nt * nt);
        if (on_device(map)) CK(cudaMemcpy(m.data(), map, m.size(), cudaMemcpyDeviceToHost));
        else memcpy(m.data(), map, m.size());
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < i; ++j)
                if (m[(size_t)i * nt + j] != TC_FP64)
                    return set_err(h, TC_ERR_UNSUPPORTED, "out-of-core runs take an all-FP64 map in this build");
    }
    CK(cudaSetDevice(h->device));
    const double t0 = now_ms();
    const int64_t launches0 = h->launches;
    h->factored = false;
    h->ooc = false;
    h->n = n;
    h->b = b;
    h->nt = nt;
    h->map.assign((size_t)nt * nt, TC_FP64);
    h->mixed = false;
    h->A_dev = nullptr;
    spans_reset(h);
    for (int p = 0; p < 4; ++p) h->upd_launches[p] = 0;

    TileCache C;
    if ((rc = init_cache(h, C, A_tiles, nt, b))) return rc;
    if ((rc = ensure(h, h->logdiag, (size_t)nt * sizeof(double)))) return rc;
    double *logdiag = static_cast<double *>(h->logdiag.p);
    int *status = static_cast<int *>(h->status.p);
    CK(cudaMemsetAsync(status, 0, 2 * sizeof(int), h->s));
    const int nv_last = (int)(n - (int64_t)(nt - 1) * b);
    double upd_flops = 0.0;

    for (int k = 0; k < nt; ++k) {
        int diag_slot = -1;
        for (int m = k; m < nt; ++m) {
            const int t = (int)tidx(m, k);
            ACQ(sc, t, true);                // V1: the accumulator stays resident for its updates
            ++C.pins[sc];
            if (m == nt - 1 && nv_last != b) {
                launch_fix_padding_tile(C.ptr(sc), b, nv_last, m == k, h->s);
                CK_LAUNCH();
            }
            const int sp = k > 0 ? span_begin(h, CAT_UPD64) : -1;
            for (int nn = 0; nn < k; ++nn) {
                ACQ(sx, (int)tidx(m, nn), true);
                ++C.pins[sx];
                ACQ(sy, (int)tidx(k, nn), true);
                launch_dgemm_tile({C.ptr(sc), C.ptr(sx), C.ptr(sy), b, b, b, m == k ? 1 : 0}, b, h->s);
                CK_LAUNCH();
                ++h->upd_launches[TC_FP64];
                upd_flops += (m == k ? 1.0 : 2.0) * (double)b * b * b;
                C.touched(sx);
                C.touched(sy);
                --C.pins[sx];
            }
            span_end(h, sp);
            double *D = C.ptr(sc);
            if (m == k) {
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
                        launch_dgemm_tile({D + (int64_t)(jb + 1) * 64 * b + (jb + 1) * 64, Pn, Pn, 64, rows, rows, 1},
                                          b, h->s);
                        CK_LAUNCH();
                    }
                }
                launch_logdiag_tile(D, b, k == nt - 1 ? nv_last : b, logdiag + k, h->s);
                CK_LAUNCH();
                span_end(h, spp);
                diag_slot = sc;              // V3: pinned until the column's TRSMs are done
            } else {
                const int spt = span_begin(h, CAT_TRSM);
                launch_trsm_tile(D, C.ptr(diag_slot), b, b, status, h->s);
                span_end(h, spt);
                CK_LAUNCH();
                C.touched(diag_slot);
            }
            C.write_back(t, sc);
            if (m != k) --C.pins[sc];
        }
        --C.pins[diag_slot];
    }
    std::vector<double> ld(nt);
    int st2[2] = {0, 0};
    CK(cudaMemcpyAsync(ld.data(), logdiag, nt * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(st2, status, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    CK(cudaStreamSynchronize(h->s_d2h));
    CK(cudaStreamSynchronize(h->s_h2d));
    C.destroy();
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
        stats->update_flops[TC_FP64] = upd_flops;
        stats->trsm_flops = (double)nt * (nt - 1) / 2.0 * b * (double)b * b;
        stats->potrf_flops = nt * (double)b * b * b / 3.0;
        stats->tiles[TC_FP64] = tidx(nt, 0);
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
        stats->t_update_ms[0] = ms[CAT_UPD64];
        stats->update_launches[0] = h->upd_launches[0];
        stats->t_potrf_ms = ms[CAT_POTRF];
        stats->t_trsm_ms = ms[CAT_TRSM];
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
    int rc = init_cache(h, C, h->host_factor, nt, b);
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
