// C ABI of tile_chol (include/tile_chol.h): handle, argument checks, the host-side
// static scheduler of Algorithm 1 and the solve / log-likelihood drivers.
//
// Scheduling (Section III-B): the whole left-looking task order is fixed before the
// first launch.  For every tile column k the scheduler emits, in this order,
//   1. the SYRK/GEMM updates of column k (one grouped launch per precision; FP64 ones
//      are split along K when the column has too few output blocks to fill 152 SMs),
//   2. POTRF of the diagonal tile (blocked: 64-wide panels),
//   3. the TRSMs of the tiles below it (one CTA per 64-row strip),
// and uploads the tables once.  Stream order replaces the paper's Ready table: a launch
// starts only after everything it reads has been written by earlier launches.
#include "tc_handle.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace tc;

namespace {

// ------------------------------------------------------------------ static schedule
struct ColPlan {
    int it0 = 0, nit = 0;        // FP64 update items
    int red0 = 0, nred = 0;      // split-K reductions
    int st0 = 0, nst = 0;        // TRSM strips
    std::vector<std::pair<int, int>> potrf_items;  // (first item, count) per 64-panel (trailing update)
};

struct Plan {
    std::vector<DJob> jobs;
    std::vector<DItem> items;
    std::vector<DRed> reds;
    std::vector<TStrip> strips;
    std::vector<ColPlan> cols;
    int max_parts = 0;
    double update_flops[4] = {0, 0, 0, 0};
    double trsm_flops = 0, potrf_flops = 0;
};

constexpr int kTargetItems = 8 * 2 * NSM;   // >= 8 waves of 2 CTAs per SM before splitting K

// Emit the items of one job: every 64 x 64 output block (lower ones only for a diagonal
// SYRK), split along K into `splits` ranges when asked (the reduction then subtracts the
// partial blocks from C in a fixed order, so results do not depend on timing).
void emit_job_items(Plan &P, int job, int ld, int splits, int &part_next) {
    const DJob J = P.jobs[job];
    const int mb = J.M / 64, nb = J.N / 64;
    for (int bj = 0; bj < nb; ++bj)
        for (int bi = J.lower ? bj : 0; bi < mb; ++bi) {
            if (splits <= 1) {
                P.items.push_back({job, (uint16_t)bi, (uint16_t)bj, 0, J.K, -1});
                continue;
            }
            const int part0 = part_next;
            const int chunk = ((J.K + splits - 1) / splits + 15) / 16 * 16;
            int np = 0;
            for (int k0 = 0; k0 < J.K; k0 += chunk, ++np)
                P.items.push_back({job, (uint16_t)bi, (uint16_t)bj, k0, std::min(J.K, k0 + chunk), part_next++});
            P.reds.push_back({J.C + (int64_t)bj * 64 * ld + bi * 64, part0, np});
        }
}

Plan build_plan(double *W, int nt, int b, const std::vector<uint8_t> &map, bool mixed) {
    Plan P;
    P.cols.resize(nt);
    const int64_t bb = (int64_t)b * b;
    auto T = [&](int i, int j) { return W + tidx(i, j) * bb; };
    for (int k = 0; k < nt; ++k) {
        ColPlan &C = P.cols[k];
        // 1. updates of column k (FP64 output tiles here; low-precision ones elsewhere)
        C.it0 = (int)P.items.size();
        C.red0 = (int)P.reds.size();
        if (k > 0) {
            const int K = k * b;
            std::vector<int> jobs_here;
            int base = 0;
            for (int m = k; m < nt; ++m) {
                const bool fp64 = (m == k) || !mixed || map[(size_t)m * nt + k] == TC_FP64;
                if (!fp64) continue;
                jobs_here.push_back((int)P.jobs.size());
                P.jobs.push_back({T(m, k), T(m, 0), T(k, 0), K, b, b, m == k ? 1 : 0});
                base += (m == k) ? (b / 64) * (b / 64 + 1) / 2 : (b / 64) * (b / 64);
                P.update_flops[TC_FP64] += (m == k ? 1.0 : 2.0) * (double)b * b * K;
            }
            int splits = 1;
            if (base > 0 && base < kTargetItems) splits = std::min((kTargetItems + base - 1) / base, std::max(1, K / 256));
            int part_next = 0;
            for (int jj : jobs_here) emit_job_items(P, jj, b, splits, part_next);
            P.max_parts = std::max(P.max_parts, part_next);
        }
        C.nit = (int)P.items.size() - C.it0;
        C.nred = (int)P.reds.size() - C.red0;
        // 2. POTRF trailing updates of the diagonal tile, panel by panel
        double *D = T(k, k);
        for (int jb = 0; jb + 1 < b / 64; ++jb) {
            const int M = b - (jb + 1) * 64;
            const int job = (int)P.jobs.size();
            const double *Pn = D + (int64_t)jb * 64 * b + (jb + 1) * 64;
            P.jobs.push_back({D + (int64_t)(jb + 1) * 64 * b + (jb + 1) * 64, Pn, Pn, 64, M, M, 1});
            const int i0 = (int)P.items.size();
            int dummy = 0;
            emit_job_items(P, job, b, 1, dummy);
            C.potrf_items.push_back({i0, (int)P.items.size() - i0});
        }
        P.potrf_flops += (double)b * b * b / 3.0;
        // 3. TRSM strips of the tiles below the diagonal
        C.st0 = (int)P.strips.size();
        for (int m = k + 1; m < nt; ++m)
            for (int r0 = 0; r0 < b; r0 += 64) P.strips.push_back({T(m, k), D, r0});
        C.nst = (int)P.strips.size() - C.st0;
        P.trsm_flops += (double)(nt - 1 - k) * b * b * b;
    }
    return P;
}

size_t align_up(size_t x) { return (x + 255) / 256 * 256; }


// ----------------------------------------------------------- mixed-precision schedule
// Which low-precision operand copies each final tile needs (Section IV-C: an update runs
// in the precision of the tile it writes, so tile (i, j) is needed in p(i, k') for every
// output (i, k'), j < k' < i, that reads it as X, and in p(m, i) for every output (m, i),
// m > i, that reads it as Y), the pool slot of each copy, and per column the tensor-core
// work items, the tiles to store in their precision and the copies to make.
struct MxpPlan {
    std::vector<int> slot[3];          // [q-1][packed tile] -> slot, -1 if not needed
    int64_t nslots[3] = {0, 0, 0};
    std::vector<uint8_t> prec;         // precision of every packed tile (diagonal FP64)
    std::vector<int> tiles;            // per column: off-diagonal tiles to store / copy
    std::vector<CopyJob> copies;
    std::vector<QItem> qitems;
    struct Col { int t0, nt, c0, nc, q0[3], nq[3]; };
    std::vector<Col> cols;
    double flops[4] = {0, 0, 0, 0};
};

MxpPlan build_mxp(int nt, int b, const std::vector<uint8_t> &map) {
    MxpPlan M;
    const int64_t T = tidx(nt, 0);
    auto P = [&](int i, int j) { return (int)map[(size_t)i * nt + j]; };
    for (int q = 0; q < 3; ++q) M.slot[q].assign(T, -1);
    M.prec.assign(T, 0);
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < i; ++j) {
            M.prec[tidx(i, j)] = (uint8_t)P(i, j);
            unsigned mask = 0;
            for (int kk = j + 1; kk < i; ++kk) mask |= 1u << P(i, kk);
            for (int m = i + 1; m < nt; ++m) mask |= 1u << P(m, i);
            for (int q = 1; q <= 3; ++q)
                if (mask & (1u << q)) M.slot[q - 1][tidx(i, j)] = (int)M.nslots[q - 1]++;
        }
    M.cols.resize(nt);
    const int nbk = b / 128;
    for (int k = 0; k < nt; ++k) {
        MxpPlan::Col &C = M.cols[k];
        for (int q = 1; q <= 3; ++q) {
            C.q0[q - 1] = (int)M.qitems.size();
            if (k > 0)
                for (int m = k + 1; m < nt; ++m) {
                    if (P(m, k) != q) continue;
                    for (int bn = 0; bn < nbk; ++bn)
                        for (int bm = 0; bm < nbk; ++bm) M.qitems.push_back({m, (uint16_t)bm, (uint16_t)bn});
                    M.flops[q] += 2.0 * b * (double)b * k * b;
                }
            C.nq[q - 1] = (int)M.qitems.size() - C.q0[q - 1];
        }
        C.t0 = (int)M.tiles.size();
        C.c0 = (int)M.copies.size();
        for (int m = k + 1; m < nt; ++m) {
            const int t = (int)tidx(m, k);
            M.tiles.push_back(t);
            for (int q = 1; q <= 3; ++q)
                if (M.slot[q - 1][t] >= 0) M.copies.push_back({t, q, M.slot[q - 1][t]});
        }
        C.nt = (int)M.tiles.size() - C.t0;
        C.nc = (int)M.copies.size() - C.c0;
    }
    return M;
}

struct MxpDev {
    const int *slot[3];
    int *exps16, *exps8;
    const uint8_t *prec;
    double *amaxL, *amaxS;
    const int *tiles;
    const CopyJob *copies;
    const QItem *qitems;
};

int setup_mxp(tc_handle h, const MxpPlan &M, MxpDev &D) {
    const int b = h->b;
    const int64_t T = tidx(h->nt, 0);
    const size_t bb = (size_t)b * b;
    int rc;
    if (M.nslots[0]) {
        if ((rc = ensure(h, h->pool_hi, M.nslots[0] * bb * 4)) || (rc = ensure(h, h->pool_lo, M.nslots[0] * bb * 4)))
            return rc;
    }
    if (M.nslots[1] && (rc = ensure(h, h->pool16, M.nslots[1] * bb * 2))) return rc;
    if (M.nslots[2] && (rc = ensure(h, h->pool8, M.nslots[2] * bb * 1))) return rc;
    // one table buffer: slots (3T ints), exps16, exps8 (T ints each), amaxL, amaxS (T doubles),
    // prec (T bytes), tiles, copies, qitems
    const size_t o_slot = 0, o_e16 = align_up(o_slot + 3 * T * 4), o_e8 = align_up(o_e16 + T * 4);
    const size_t o_aL = align_up(o_e8 + T * 4), o_aS = align_up(o_aL + T * 8), o_prec = align_up(o_aS + T * 8);
    const size_t o_tiles = align_up(o_prec + T), o_cp = align_up(o_tiles + M.tiles.size() * 4);
    const size_t o_q = align_up(o_cp + M.copies.size() * sizeof(CopyJob));
    const size_t total = align_up(o_q + M.qitems.size() * sizeof(QItem));
    if ((rc = ensure(h, h->mxtab, total))) return rc;
    std::vector<char> host(total, 0);
    for (int q = 0; q < 3; ++q) memcpy(host.data() + o_slot + (size_t)q * T * 4, M.slot[q].data(), T * 4);
    memcpy(host.data() + o_prec, M.prec.data(), T);
    if (!M.tiles.empty()) memcpy(host.data() + o_tiles, M.tiles.data(), M.tiles.size() * 4);
    if (!M.copies.empty()) memcpy(host.data() + o_cp, M.copies.data(), M.copies.size() * sizeof(CopyJob));
    if (!M.qitems.empty()) memcpy(host.data() + o_q, M.qitems.data(), M.qitems.size() * sizeof(QItem));
    CK(cudaMemcpyAsync(h->mxtab.p, host.data(), total, cudaMemcpyHostToDevice, h->s));
    char *base = static_cast<char *>(h->mxtab.p);
    for (int q = 0; q < 3; ++q) D.slot[q] = reinterpret_cast<const int *>(base + o_slot + (size_t)q * T * 4);
    D.exps16 = reinterpret_cast<int *>(base + o_e16);
    D.exps8 = reinterpret_cast<int *>(base + o_e8);
    D.amaxL = reinterpret_cast<double *>(base + o_aL);
    D.amaxS = reinterpret_cast<double *>(base + o_aS);
    D.prec = reinterpret_cast<const uint8_t *>(base + o_prec);
    D.tiles = reinterpret_cast<const int *>(base + o_tiles);
    D.copies = reinterpret_cast<const CopyJob *>(base + o_cp);
    D.qitems = reinterpret_cast<const QItem *>(base + o_q);
    // tensor maps over the pools (128 x 128-byte boxes, 128-byte swizzle)
    if (M.nslots[0] && (make_pool_map(&h->map_hi, h->pool_hi.p, M.nslots[0], b, 4, 128) ||
                        make_pool_map(&h->map_lo, h->pool_lo.p, M.nslots[0], b, 4, 128)))
        return set_err(h, TC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the TF32 pools");
    if (M.nslots[1] && make_pool_map(&h->map16, h->pool16.p, M.nslots[1], b, 2, 128))
        return set_err(h, TC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the FP16 pool");
    if (M.nslots[2] && make_pool_map(&h->map8, h->pool8.p, M.nslots[2], b, 1, 128))
        return set_err(h, TC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the FP8 pool");
    return TC_OK;
}

// Low-precision updates of column k (before its POTRF) and the stores / operand copies of
// its final tiles (after its TRSMs).
int mxp_updates(tc_handle h, const MxpPlan &M, const MxpDev &D, int k) {
    const MxpPlan::Col &C = M.cols[k];
    int *err = static_cast<int *>(h->status.p) + 1;
    double *W = static_cast<double *>(h->W.p);
    for (int q = 1; q <= 3; ++q) {
        if (!C.nq[q - 1]) continue;
        const CUtensorMap &a0 = q == 1 ? h->map_hi : q == 2 ? h->map16 : h->map8;
        const CUtensorMap &a1 = q == 1 ? h->map_lo : a0;
        const int sp = span_begin(h, CAT_UPD64 + q);
        launch_qgemm(q, a0, a1, a0, a1, W, D.qitems + C.q0[q - 1], C.nq[q - 1], D.slot[q - 1],
                     q == 2 ? D.exps16 : q == 3 ? D.exps8 : nullptr, k, h->b, h->nt, err, h->s);
        span_end(h, sp);
        CK_LAUNCH();
        ++h->upd_launches[q];
    }
    return TC_OK;
}

int mxp_convert(tc_handle h, const MxpPlan &M, const MxpDev &D, int k) {
    const MxpPlan::Col &C = M.cols[k];
    if (!C.nt) return TC_OK;
    double *W = static_cast<double *>(h->W.p);
    const int sp = span_begin(h, CAT_CONVERT);
    launch_tile_amax(W, h->b, D.tiles + C.t0, C.nt, D.amaxL, h->s);
    CK_LAUNCH();
    launch_store_round(W, h->b, D.tiles + C.t0, C.nt, D.prec, D.amaxL, D.amaxS, h->s);
    CK_LAUNCH();
    if (C.nc) {
        launch_make_copies(W, h->b, D.copies + C.c0, C.nc, D.amaxS, static_cast<float *>(h->pool_hi.p),
                           static_cast<float *>(h->pool_lo.p), static_cast<__half *>(h->pool16.p),
                           static_cast<uint8_t *>(h->pool8.p), D.exps16, D.exps8, h->s);
        CK_LAUNCH();
    }
    span_end(h, sp);
    return TC_OK;
}

int run_factor(tc_handle h, const Plan &P, const MxpPlan *M) {
    const int nt = h->nt, b = h->b;
    // upload tables
    const size_t sj = P.jobs.size() * sizeof(DJob), si = P.items.size() * sizeof(DItem);
    const size_t sr = P.reds.size() * sizeof(DRed), ss = P.strips.size() * sizeof(TStrip);
    const size_t oj = 0, oi = align_up(oj + sj), orr = align_up(oi + si), os = align_up(orr + sr);
    const size_t total = align_up(os + ss);
    int rc = ensure(h, h->tables, total);
    if (rc) return rc;
    std::vector<char> host(total);
    if (sj) memcpy(host.data() + oj, P.jobs.data(), sj);
    if (si) memcpy(host.data() + oi, P.items.data(), si);
    if (sr) memcpy(host.data() + orr, P.reds.data(), sr);
    if (ss) memcpy(host.data() + os, P.strips.data(), ss);
    CK(cudaMemcpyAsync(h->tables.p, host.data(), total, cudaMemcpyHostToDevice, h->s));
    char *base = static_cast<char *>(h->tables.p);
    const DJob *djobs = reinterpret_cast<const DJob *>(base + oj);
    const DItem *ditems = reinterpret_cast<const DItem *>(base + oi);
    const DRed *dreds = reinterpret_cast<const DRed *>(base + orr);
    const TStrip *dstrips = reinterpret_cast<const TStrip *>(base + os);
    rc = ensure(h, h->partials, (size_t)std::max(1, P.max_parts) * 4096 * sizeof(double));
    if (rc) return rc;
    double *parts = static_cast<double *>(h->partials.p);
    int *status = static_cast<int *>(h->status.p);
    double *W = static_cast<double *>(h->W.p);
    const int64_t bb = (int64_t)b * b;
    MxpDev D{};
    if (M) {
        rc = setup_mxp(h, *M, D);
        if (rc) return rc;
        const int64_t T = tidx(nt, 0);
        CK(cudaMemsetAsync(D.amaxL, 0, T * sizeof(double), h->s));
        CK(cudaMemsetAsync(D.amaxS, 0, T * sizeof(double), h->s));
        CK(cudaMemsetAsync(D.exps16, 0, T * sizeof(int), h->s));
        CK(cudaMemsetAsync(D.exps8, 0, T * sizeof(int), h->s));
    }

    for (int k = 0; k < nt; ++k) {
        const ColPlan &C = P.cols[k];
        if (C.nit) {
            const int sp = span_begin(h, CAT_UPD64);
            launch_dgemm_update(djobs, ditems + C.it0, C.nit, b, parts, status, h->s);
            span_end(h, sp);
            CK_LAUNCH();
            ++h->upd_launches[TC_FP64];
        }
        if (C.nred) {
            launch_dgemm_reduce(dreds + C.red0, C.nred, b, parts, status, h->s);
            CK_LAUNCH();
        }
        if (M && (rc = mxp_updates(h, *M, D, k))) return rc;
        double *Dk = W + tidx(k, k) * bb;
        const int sp_potrf = span_begin(h, CAT_POTRF);
        for (int jb = 0; jb < b / 64; ++jb) {
            launch_potrf_block(Dk + (int64_t)jb * 64 * b + jb * 64, b, k * b + jb * 64, status, h->s);
            CK_LAUNCH();
            if (jb + 1 < b / 64) {
                const int rows = b - (jb + 1) * 64;
                launch_trsm_rows(Dk + (int64_t)jb * 64 * b + (jb + 1) * 64, Dk + (int64_t)jb * 64 * b + jb * 64, b,
                                 rows, status, h->s);
                CK_LAUNCH();
                const auto &pi = C.potrf_items[jb];
                launch_dgemm_update(djobs, ditems + pi.first, pi.second, b, parts, status, h->s);
                CK_LAUNCH();
            }
        }
        span_end(h, sp_potrf);
        if (C.nst) {
            const int sp = span_begin(h, CAT_TRSM);
            launch_trsm_strips(dstrips + C.st0, C.nst, b, b, status, h->s);
            span_end(h, sp);
            CK_LAUNCH();
        }
        if (M && (rc = mxp_convert(h, *M, D, k))) return rc;
    }
    return TC_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void tc_config_default(tc_config *cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->device = 0;
    cfg->stream = nullptr;
    cfg->ooc = 0;
    cfg->device_cap_bytes = 0;
    cfg->prefetch_depth = 2;
    cfg->lookahead = 1;
}

int tc_create(tc_handle *out, const tc_config *cfg) {
    if (!out) return TC_ERR_ARG;
    *out = nullptr;
    tc_handle h = new tc_handle_s();
    if (cfg) h->cfg = *cfg;
    else tc_config_default(&h->cfg);
    h->device = h->cfg.device;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || h->device < 0 || h->device >= ndev) {
        cudaGetLastError();
        delete h;
        return TC_ERR_CUDA;
    }
    if (cudaSetDevice(h->device) != cudaSuccess) {
        delete h;
        return TC_ERR_CUDA;
    }
    if (h->cfg.stream) {
        h->s = static_cast<cudaStream_t>(h->cfg.stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return TC_ERR_CUDA;
        }
        h->own_stream = true;
    }
    if (ensure(h, h->status, 256) || ensure(h, h->scratch, 4096 * sizeof(double))) {
        tc_destroy(h);
        return TC_ERR_OOM;
    }
    *out = h;
    return TC_OK;
}

void tc_destroy(tc_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->s) cudaStreamSynchronize(h->s);
    for (DevBuf *d : {&h->W, &h->Acopy, &h->status, &h->scratch, &h->tables, &h->partials, &h->vec, &h->sumsq,
                      &h->pool_hi, &h->pool_lo, &h->pool16, &h->pool8, &h->mxtab, &h->logdiag})
        release(*d);
    if (h->s_h2d) cudaStreamDestroy(h->s_h2d);
    if (h->s_d2h) cudaStreamDestroy(h->s_d2h);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    if (h->own_stream && h->s) cudaStreamDestroy(h->s);
    delete h;
}

const char *tc_last_error(tc_handle h) { return h ? h->err.c_str() : "null handle"; }

int tc_matern_tiles(tc_handle h, int64_t n, int b, const double *points, double sigma2, double range_a,
                    double nu, double nugget, double *A_tiles) {
    int rc = check_nb(h, n, b);
    if (rc) return rc;
    if (!points || !A_tiles) return set_err(h, TC_ERR_ARG, "points and A_tiles must not be NULL");
    if (!(range_a > 0) || !(sigma2 > 0)) return set_err(h, TC_ERR_ARG, "range and variance must be positive");
    int nu2 = 0;
    if (nu == 0.5) nu2 = 1;
    else if (nu == 1.5) nu2 = 3;
    else if (nu == 2.5) nu2 = 5;
    else return set_err(h, TC_ERR_ARG, "smoothness must be 0.5, 1.5 or 2.5");
    CK(cudaSetDevice(h->device));
    const int nt = (int)((n + b - 1) / b);
    const double *dpts = points;
    DevBuf tmp_pts, tmp_out;
    if (!on_device(points)) {
        rc = ensure(h, tmp_pts, (size_t)n * 2 * sizeof(double));
        if (rc) return rc;
        CK(cudaMemcpyAsync(tmp_pts.p, points, (size_t)n * 2 * sizeof(double), cudaMemcpyHostToDevice, h->s));
        dpts = static_cast<const double *>(tmp_pts.p);
    }
    const size_t bytes = (size_t)nt * (nt + 1) / 2 * b * b * sizeof(double);
    double *dout = A_tiles;
    const bool out_dev = on_device(A_tiles);
    if (!out_dev) {
        rc = ensure(h, tmp_out, bytes);
        if (rc) { release(tmp_pts); return rc; }
        dout = static_cast<double *>(tmp_out.p);
    }
    launch_matern(dout, n, b, nt, dpts, sigma2, range_a, nu2, nugget, h->s);
    CK_LAUNCH();
    if (!out_dev) CK(cudaMemcpyAsync(A_tiles, dout, bytes, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    release(tmp_pts);
    release(tmp_out);
    return TC_OK;
}

int tile_chol_precision_map(tc_handle h, int64_t n, int b, const double *A_tiles, double eps_high, int band,
                            int prec_set, uint8_t *map_out, double *norms_out) {
    int rc = check_nb(h, n, b);
    if (rc) return rc;
    if (!A_tiles || !map_out) return set_err(h, TC_ERR_ARG, "A_tiles and map_out must not be NULL");
    if (!(eps_high > 0) || band < 0 || prec_set < 1 || prec_set > 4)
        return set_err(h, TC_ERR_ARG, "eps_high > 0, band >= 0 and prec_set in 1..4 are required");
    CK(cudaSetDevice(h->device));
    const int nt = (int)((n + b - 1) / b);
    const int64_t T = (int64_t)nt * (nt + 1) / 2;
    const double *dA = A_tiles;
    DevBuf tmp;
    if (!on_device(A_tiles)) {
        const size_t bytes = (size_t)T * b * b * sizeof(double);
        rc = ensure(h, tmp, bytes);
        if (rc) return rc;
        CK(cudaMemcpyAsync(tmp.p, A_tiles, bytes, cudaMemcpyHostToDevice, h->s));
        dA = static_cast<const double *>(tmp.p);
    }
    rc = ensure(h, h->sumsq, (size_t)T * sizeof(double));
    if (rc) { release(tmp); return rc; }
    launch_tile_sumsq(dA, nt, b, n, static_cast<double *>(h->sumsq.p), h->s);
    CK_LAUNCH();
    std::vector<double> ss(T);
    CK(cudaMemcpyAsync(ss.data(), h->sumsq.p, T * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    release(tmp);
    // ||A||_F over the full symmetric matrix: off-diagonal tiles count twice
    double tot = 0.0;
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j <= i; ++j) tot += (i == j ? 1.0 : 2.0) * ss[tidx(i, j)];
    const double normA = std::sqrt(tot);
    const double u[4] = {std::ldexp(1.0, -53), std::ldexp(1.0, -24), std::ldexp(1.0, -11), std::ldexp(1.0, -4)};
    std::vector<uint8_t> pm((size_t)nt * nt, 0);
    std::vector<double> norms((size_t)nt * nt + 1, 0.0);
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j <= i; ++j) {
            const double nij = std::sqrt(ss[tidx(i, j)]);
            norms[(size_t)i * nt + j] = nij;
            if (i == j || i - j <= band) continue;
            const double ratio = (double)nt * nij / normA;
            // lowest allowed precision first: FP8, FP16, FP32
            for (int p = TC_FP8; p >= TC_FP32; --p) {
                if (p > prec_set - 1) continue;
                if (ratio < eps_high / u[p]) {
                    pm[(size_t)i * nt + j] = (uint8_t)p;
                    break;
                }
            }
        }
    norms[(size_t)nt * nt] = normA;
    if (on_device(map_out)) {
        CK(cudaMemcpy(map_out, pm.data(), pm.size(), cudaMemcpyHostToDevice));
    } else {
        memcpy(map_out, pm.data(), pm.size());
    }
    if (norms_out) {
        if (on_device(norms_out)) CK(cudaMemcpy(norms_out, norms.data(), norms.size() * sizeof(double), cudaMemcpyHostToDevice));
        else memcpy(norms_out, norms.data(), norms.size() * sizeof(double));
    }
    return TC_OK;
}

int tile_chol_factor(tc_handle h, int64_t n, int b, const double *A_tiles, const uint8_t *map, tc_stats *stats) {
    int rc = check_nb(h, n, b);
    if (rc) return rc;
    if (!A_tiles) return set_err(h, TC_ERR_ARG, "A_tiles must not be NULL");
    CK(cudaSetDevice(h->device));
    const double t0 = now_ms();
    const int64_t launches0 = h->launches;
    h->factored = false;
    h->ooc = false;
    h->normA_inf = -1.0;
    const int nt = (int)((n + b - 1) / b);
    const int64_t T = (int64_t)nt * (nt + 1) / 2;
    const size_t bytes = (size_t)T * b * b * sizeof(double);
    h->n = n;
    h->b = b;
    h->nt = nt;
    // precision map (host copy)
    h->map.assign((size_t)nt * nt, TC_FP64);
    if (map) {
        if (on_device(map)) CK(cudaMemcpy(h->map.data(), map, h->map.size(), cudaMemcpyDeviceToHost));
        else memcpy(h->map.data(), map, h->map.size());
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < nt; ++j) {
                uint8_t &v = h->map[(size_t)i * nt + j];
                if (j >= i) v = TC_FP64;
                if (v > TC_FP8) return set_err(h, TC_ERR_ARG, "precision map entries must be 0..3");
            }
    }
    h->mixed = false;
    for (uint8_t v : h->map) h->mixed |= (v != TC_FP64);
    if (h->mixed && b % 128) return set_err(h, TC_ERR_UNSUPPORTED, "mixed precision needs a tile size that is a multiple of 128");
    if (h->cfg.ooc == 1) return set_err(h, TC_ERR_UNSUPPORTED, "out-of-core mode is not available in this build");

    rc = ensure(h, h->W, bytes);
    if (rc) return rc;
    // the caller's A stays readable for refinement: reference it on the device or copy it
    if (on_device(A_tiles)) {
        h->A_dev = A_tiles;
    } else {
        rc = ensure(h, h->Acopy, bytes);
        if (rc) return rc;
        CK(cudaMemcpyAsync(h->Acopy.p, A_tiles, bytes, cudaMemcpyHostToDevice, h->s));
        h->A_dev = static_cast<const double *>(h->Acopy.p);
    }
    double *W = static_cast<double *>(h->W.p);
    CK(cudaMemcpyAsync(W, h->A_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
    launch_fix_padding(W, nt, b, n, h->s);
    CK_LAUNCH();
    CK(cudaMemsetAsync(h->status.p, 0, 2 * sizeof(int), h->s));

    spans_reset(h);
    for (int p = 0; p < 4; ++p) h->upd_launches[p] = 0;
    Plan P = build_plan(W, nt, b, h->map, h->mixed);
    MxpPlan M;
    if (h->mixed) {
        M = build_mxp(nt, b, h->map);
        for (int p = 1; p < 4; ++p) P.update_flops[p] = M.flops[p];
    }
    rc = run_factor(h, P, h->mixed ? &M : nullptr);
    if (rc) return rc;
    double *sc = static_cast<double *>(h->scratch.p);
    launch_logdet(W, nt, b, n, sc, h->s);
    CK_LAUNCH();
    int st2[2] = {0, 0};
    CK(cudaMemcpyAsync(st2, h->status.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->s));
    double ld = 0.0;
    CK(cudaMemcpyAsync(&ld, sc, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    const int info = st2[0];
    if (st2[1]) {
        h->factored = false;
        return set_err(h, TC_ERR_TIMEOUT, st2[1] == 2 ? "tensor-core update found no operand copy (internal)"
                                                        : "a tensor-core update timed out waiting on its pipeline");
    }
    h->logdet = ld;
    h->factored = (info == 0);
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->t_ms = now_ms() - t0;
        stats->flops = (double)n * n * n / 3.0;
        for (int p = 0; p < 4; ++p) stats->update_flops[p] = P.update_flops[p];
        stats->trsm_flops = P.trsm_flops;
        stats->potrf_flops = P.potrf_flops;
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j <= i; ++j) stats->tiles[h->map[(size_t)i * nt + j]]++;
        stats->kernel_launches = h->launches - launches0;
        stats->info = info;
        double ms[CAT_N];
        span_totals(h, ms);
        for (int p = 0; p < 4; ++p) {
            stats->t_update_ms[p] = ms[CAT_UPD64 + p];
            stats->update_launches[p] = h->upd_launches[p];
        }
        stats->t_potrf_ms = ms[CAT_POTRF];
        stats->t_trsm_ms = ms[CAT_TRSM];
        stats->t_convert_ms = ms[CAT_CONVERT];
    }
    if (info) set_err(h, info, "matrix is not positive definite (see the returned column)");
    return info;
}

int tile_chol_logdet(tc_handle h, double *logdet_out) {
    if (!h || !logdet_out) return TC_ERR_ARG;
    if (!h->factored) return set_err(h, TC_ERR_STATE, "no successful factorization");
    *logdet_out = h->logdet;
    return TC_OK;
}

// Forward (and optionally back) substitution on the padded column-major buffer R
// (leading dimension ldr = nt*b), nrhs <= 16 per pass.
static int subst(tc_handle h, double *R, int64_t ldr, int nrhs, bool back) {
    if (h->ooc) return ooc_subst(h, R, ldr, nrhs, back, nullptr);
    const int nt = h->nt, b = h->b;
    const double *W = static_cast<const double *>(h->W.p);
    const int64_t bb = (int64_t)b * b;
    for (int c0 = 0; c0 < nrhs; c0 += 16) {
        const int nc = std::min(16, nrhs - c0);
        double *Rc = R + (int64_t)c0 * ldr;
        for (int j = 0; j < nt; ++j) {
            launch_fwd_diag(W + tidx(j, j) * bb, b, Rc + (int64_t)j * b, ldr, nc, h->s);
            CK_LAUNCH();
            launch_fwd_update(W, nt, b, j, Rc, ldr, nc, h->s);
            if (j + 1 < nt) CK_LAUNCH();
        }
        if (!back) continue;
        for (int j = nt - 1; j >= 0; --j) {
            launch_bwd_diag(W + tidx(j, j) * bb, b, Rc + (int64_t)j * b, ldr, nc, h->s);
            CK_LAUNCH();
            launch_bwd_update(W, nt, b, j, Rc, ldr, nc, h->s);
            if (j > 0) CK_LAUNCH();
        }
    }
    return TC_OK;
}

int tile_chol_solve(tc_handle h, int nrhs, const double *B, int64_t ldb, double *X, int64_t ldx, int max_refine,
                    double target_berr, tc_stats *stats) {
    if (!h) return TC_ERR_ARG;
    if (!h->factored) return set_err(h, TC_ERR_STATE, "no successful factorization");
    if (nrhs < 1 || !B || !X || ldb < h->n || ldx < h->n || max_refine < 0)
        return set_err(h, TC_ERR_ARG, "bad solve arguments");
    CK(cudaSetDevice(h->device));
    const double t0 = now_ms();
    const int64_t launches0 = h->launches;
    const int nt = h->nt, b = h->b;
    const int64_t n = h->n, ldr = (int64_t)nt * b;
    // workspace: Bd (padded copy of B), Xd, Rd  (each ldr x nrhs)
    const size_t colbytes = (size_t)ldr * nrhs * sizeof(double);
    int rc = ensure(h, h->vec, 3 * colbytes);
    if (rc) return rc;
    double *Bd = static_cast<double *>(h->vec.p);
    double *Xd = Bd + (size_t)ldr * nrhs;
    double *Rd = Xd + (size_t)ldr * nrhs;
    CK(cudaMemsetAsync(Bd, 0, colbytes, h->s));
    CK(cudaMemcpy2DAsync(Bd, ldr * sizeof(double), B, ldb * sizeof(double), n * sizeof(double), nrhs,
                         cudaMemcpyDefault, h->s));
    CK(cudaMemcpyAsync(Xd, Bd, colbytes, cudaMemcpyDeviceToDevice, h->s));
    rc = subst(h, Xd, ldr, nrhs, true);
    if (rc) return rc;
    double *sc = static_cast<double *>(h->scratch.p);
    // ||A||_inf (once per factor): max row sum of |A| = max of |A| * ones
    if (h->ooc) max_refine = 0;      // A was overwritten by the out-of-core factor: no residuals
    if (h->normA_inf < 0 && max_refine > 0) {
        CK(cudaMemsetAsync(Rd, 0, (size_t)ldr * sizeof(double), h->s));
        // ones vector in Rd[ldr .. 2 ldr) is not needed: use a dedicated column of Rd
        std::vector<double> ones((size_t)ldr, 0.0);
        for (int64_t i = 0; i < n; ++i) ones[i] = 1.0;
        CK(cudaMemcpyAsync(Rd, ones.data(), (size_t)ldr * sizeof(double), cudaMemcpyHostToDevice, h->s));
        double *rowsum = Rd + (nrhs > 1 ? ldr : 0);
        DevBuf tmp;
        if (nrhs == 1) {
            rc = ensure(h, tmp, (size_t)ldr * sizeof(double));
            if (rc) return rc;
            rowsum = static_cast<double *>(tmp.p);
        }
        launch_symv_resid(h->A_dev, nt, b, n, Rd, ldr, nullptr, 0, rowsum, ldr, 1, 1, h->s);
        CK_LAUNCH();
        CK(cudaMemsetAsync(sc, 0, sizeof(double), h->s));
        launch_colmax_abs(rowsum, ldr, n, 1, sc, h->s);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(&h->normA_inf, sc, sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        release(tmp);
    }
    int it = 0;
    double berr = -1.0;
    for (;; ++it) {
        if (max_refine == 0) break;
        // R = B - A X and the normwise backward error per column
        for (int c0 = 0; c0 < nrhs; c0 += 16) {
            const int nc = std::min(16, nrhs - c0);
            launch_symv_resid(h->A_dev, nt, b, n, Xd + (int64_t)c0 * ldr, ldr, Bd + (int64_t)c0 * ldr, ldr,
                              Rd + (int64_t)c0 * ldr, ldr, nc, 0, h->s);
            CK_LAUNCH();
        }
        CK(cudaMemsetAsync(sc, 0, 3 * nrhs * sizeof(double), h->s));
        launch_colmax_abs(Rd, ldr, n, nrhs, sc, h->s);
        CK_LAUNCH();
        launch_colmax_abs(Xd, ldr, n, nrhs, sc + nrhs, h->s);
        CK_LAUNCH();
        launch_colmax_abs(Bd, ldr, n, nrhs, sc + 2 * nrhs, h->s);
        CK_LAUNCH();
        std::vector<double> mx(3 * nrhs);
        CK(cudaMemcpyAsync(mx.data(), sc, 3 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        berr = 0.0;
        for (int c = 0; c < nrhs; ++c) {
            const double den = h->normA_inf * mx[nrhs + c] + mx[2 * nrhs + c];
            berr = std::max(berr, den > 0 ? mx[c] / den : 0.0);
        }
        if (berr <= target_berr || it >= max_refine) break;
        rc = subst(h, Rd, ldr, nrhs, true);
        if (rc) return rc;
        launch_axpy_cols(Xd, ldr, Rd, ldr, n, nrhs, h->s);
        CK_LAUNCH();
    }
    CK(cudaMemcpy2DAsync(X, ldx * sizeof(double), Xd, ldr * sizeof(double), n * sizeof(double), nrhs,
                         cudaMemcpyDefault, h->s));
    CK(cudaStreamSynchronize(h->s));
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->t_ms = now_ms() - t0;
        stats->refine_iters = it;
        stats->berr = berr;
        stats->kernel_launches = h->launches - launches0;
    }
    return TC_OK;
}

int tile_chol_loglik(tc_handle h, const double *y, double *loglik_out) {
    if (!h || !loglik_out) return TC_ERR_ARG;
    if (!h->factored) return set_err(h, TC_ERR_STATE, "no successful factorization");
    CK(cudaSetDevice(h->device));
    const double two_pi = 6.283185307179586476925286766559;
    double quad = 0.0;
    if (y) {
        const int64_t ldr = (int64_t)h->nt * h->b;
        int rc = ensure(h, h->vec, (size_t)ldr * sizeof(double) * 3);
        if (rc) return rc;
        double *z = static_cast<double *>(h->vec.p);
        CK(cudaMemsetAsync(z, 0, (size_t)ldr * sizeof(double), h->s));
        CK(cudaMemcpyAsync(z, y, (size_t)h->n * sizeof(double), cudaMemcpyDefault, h->s));
        rc = subst(h, z, ldr, 1, false);
        if (rc) return rc;
        double *sc = static_cast<double *>(h->scratch.p);
        launch_dot_self(z, h->n, sc, h->s);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(&quad, sc, sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
    }
    *loglik_out = -0.5 * (double)h->n * std::log(two_pi) - 0.5 * h->logdet - 0.5 * quad;
    return TC_OK;
}

int tile_chol_get_factor(tc_handle h, double *L_tiles) {
    if (!h || !L_tiles) return TC_ERR_ARG;
    if (!h->factored) return set_err(h, TC_ERR_STATE, "no successful factorization");
    CK(cudaSetDevice(h->device));
    const int nt = h->nt, b = h->b;
    const size_t bytes = (size_t)nt * (nt + 1) / 2 * b * b * sizeof(double);
    double *dst = L_tiles;
    DevBuf tmp;
    const bool dev = on_device(L_tiles);
    if (!dev) {
        int rc = ensure(h, tmp, bytes);
        if (rc) return rc;
        dst = static_cast<double *>(tmp.p);
    }
    CK(cudaMemcpyAsync(dst, h->ooc ? static_cast<const void *>(h->host_factor) : h->W.p, bytes, cudaMemcpyDefault,
                       h->s));
    launch_zero_upper_diag(dst, nt, b, h->n, h->s);
    CK_LAUNCH();
    if (!dev) CK(cudaMemcpyAsync(L_tiles, dst, bytes, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    release(tmp);
    return TC_OK;
}

}  // extern "C"
