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
// The plan covers a list of matrices sharing one tile size (a single factorization is a
// list of one): column step k groups the work of column k of every matrix that has one,
// so each launch below serves the whole batch.
struct PotrfStep {
    int pe0 = 0, npe = 0;        // PEntry range (one per matrix)
    int it0 = 0, nit = 0;        // trailing-update items
    int rows = 0;                // panel rows below the 64-block
};

struct ColPlan {
    int z0 = 0, nz = 0;          // emulated-FP64 update items
    int y0 = 0, ny = 0;          // emulated FP32-output update items (10 digit planes)
    int v0 = 0, nv = 0;          // TRSM as an emulated product with L_kk^{-1} (assign mode)
    int ti0 = 0, nti = 0;        //   ... the diagonal tiles inverted for it (tinv / dinv entries)
    int nvp[4] = {0, 0, 0, 0};   //   ... of which per output precision (items in that order)
    int dg0 = 0, ndg = 0;        // tiles whose digit planes are made after the column's TRSMs
    int it0 = 0, nit = 0;        // FP64 update items
    int red0 = 0, nred = 0;      // split-K reductions
    int st0 = 0, nst = 0;        // TRSM strips
    std::vector<PotrfStep> potrf;
};

struct Plan {
    std::vector<DJob> jobs;
    std::vector<DItem> items;
    std::vector<DRed> reds;
    std::vector<TStrip> strips;
    std::vector<PEntry> pentries;
    std::vector<LEntry> lentries;
    std::vector<ZItem> zitems, zitems32, zinv, zinvc, zref;
    std::vector<TEntry> tinv;    // L_kk^{-1} of every matrix's diagonal tile, per column
    std::vector<int> dinv;       //   ... the digit slot each inverse goes to (the diagonal tile's)
    bool inv_trsm = false, inv_refine = false;
    // columns of the update work items (zitems, zitems32): 128 x Z64_BN blocks for the
    // mixed-precision kernel when any matrix has a mixed map, else 128 x Z_BN
    int zwidth = Z_BN;
    std::vector<int> dtiles;
    std::vector<ColPlan> cols;
    int64_t Ttot = 0;
    int max_parts = 0, ntmax = 0;
    double update_flops[4] = {0, 0, 0, 0};
    double tensor_flops[4] = {0, 0, 0, 0};   // executed tensor-core work of the updates
    double trsm_flops = 0, potrf_flops = 0;
};

// Leading digit planes a final tile (i, j) can have non-zero: its stored format bounds them
// (E4M3 with a power-of-two scale: 5; FP16 with a scale: 10; FP32, FP64: all 14).
inline int stored_planes(const MatDesc &M, int i, int j) {
    if (!M.mixed || i == j) return 14;
    const int p = M.map[(size_t)i * M.nt + j];
    return p == TC_FP8 ? 5 : p == TC_FP16 ? 10 : 14;
}
// Order of the 128 x Z_BN work items of one output tile for the persistent emulated-update
// kernel.  Its 152 CTAs take items c, c + 152, ..., so each run of 152 consecutive items runs
// at once, and every item walks all its sources: an X slab (row block bm) is read by the
// items of its bm in the same run, a Y slab (column block bn) by those of its bn.  Runs of
// kItemRowBlocks row blocks x ~152/kItemRowBlocks column blocks keep both sets small (each
// slab is fetched from DRAM once per run that uses it: about (nbn / 38 + nbm / 4) times per
// tile instead of nbn * nbm / 152 times for X with row-block-fastest runs).
constexpr int kItemRowBlocks = 4;
template <class F>
void for_tile_items(int b, bool lower_only, F &&emit, int width = Z_BN) {
    const int nbm = b / 128, nbn = b / width;
    for (int bm0 = 0; bm0 < nbm; bm0 += kItemRowBlocks)
        for (int bn = 0; bn < nbn; ++bn)
            for (int bm = bm0; bm < std::min(nbm, bm0 + kItemRowBlocks); ++bm)
                if (!lower_only || bm * 128 + 127 >= bn * width) emit(bm, bn);
}

// Plane pairs (s, t), s < sx, t < sy, s + t < su, that one emulated product multiplies.
inline int plane_pairs(int sx, int sy, int su) {
    sx = std::min(sx, su);
    sy = std::min(sy, su);
    int n = 0;
    for (int s = 0; s < sx; ++s) n += std::min(sy, su - s);
    return n;
}

constexpr int kTargetItems = 8 * 2 * NSM;   // >= 8 waves of 2 CTAs per SM before splitting K
// Mixed-precision digit-plane updates: a source pair 4 (m + j) binary orders below the output
// tile's scale keeps j planes fewer than the reference count, m = kPlaneMargin; the terms it
// drops then stay below 16^-m of those a pair at the output's own scale drops.
constexpr int kPlaneMargin = 2;

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

Plan build_plan(tc_handle h, double *W, int *status) {
    Plan P;
    const int b = h->b;
    const int64_t bb = (int64_t)b * b;
    for (const MatDesc &M : h->mats) {
        P.ntmax = std::max(P.ntmax, M.nt);
        P.Ttot = std::max<int64_t>(P.Ttot, M.tile0 + tidx(M.nt, 0));
    }
    P.cols.resize(P.ntmax);
    const bool zmode = h->cfg.fp64_mode >= 1;
    for (const MatDesc &M : h->mats)
        if (M.mixed && zmode) P.zwidth = Z64_BN;
    const int zw = P.zwidth;
    // explicit-inverse TRSM (fp64_mode 2, single matrix: one scratch).  Mixed precision takes
    // L_mk = C_mk L_kk^{-T} as it is (its error, kappa(L_kk) u, is far below the accuracy level
    // of a mixed-precision factorization); an all-FP64 factorization adds one refinement step
    // with the residual C_mk - X0 L_kk^T, which brings the backward error back to the level of
    // substitution (the explicit inverse alone loses a factor ~kappa(L_kk)).
    // a batch uses the inverse-based TRSM when its maps are mixed (products at each stored
    // precision's plane count, no refinement step); an all-FP64 batch keeps the FP64 strips
    P.inv_trsm = h->cfg.fp64_mode == 2 && (h->mats.size() == 1 || (zw == Z64_BN && b <= 2048));
    P.inv_refine = P.inv_trsm && h->mats.size() == 1 && !h->mats[0].mixed;
    // L_kk^{-1} at invbuf, X0 of tile (k + i, k) at invbuf + i b^2 (sized by factor_matrices)
    double *inv_scratch = static_cast<double *>(h->invbuf.p);
    auto T = [&](const MatDesc &M, int i, int j) { return W + (M.tile0 + tidx(i, j)) * bb; };
    const int nmat = (int)h->mats.size();
    for (int mi = 0; mi < nmat; ++mi) {
        const MatDesc &M = h->mats[mi];
        P.lentries.push_back({W + M.tile0 * bb, M.n, M.nt});
    }
    for (int k = 0; k < P.ntmax; ++k) {
        ColPlan &C = P.cols[k];
        // 1. updates of column k (FP64 output tiles here; low-precision ones in build_mxp)
        C.it0 = (int)P.items.size();
        C.red0 = (int)P.reds.size();
        C.z0 = (int)P.zitems.size();
        C.y0 = (int)P.zitems32.size();
        if (k > 0) {
            const int K = k * b;
            std::vector<int> jobs_here;
            int base = 0;
            for (int mi = 0; mi < nmat; ++mi) {
                const MatDesc &M = h->mats[mi];
                if (M.nt <= k) continue;
                for (int m = k; m < M.nt; ++m) {
                    const bool fp64 = (m == k) || !M.mixed || M.map[(size_t)m * M.nt + k] == TC_FP64;
                    if (!fp64 && zmode && h->cfg.fp32_updates == 0 && M.map[(size_t)m * M.nt + k] == TC_FP32) {
                        // FP32 output: 10 digit planes of each operand, FP64 running sums
                        double *Cp = T(M, m, k);
                        const int xo = (int)(M.tile0 + tidx(m, 0)), yo = (int)(M.tile0 + tidx(k, 0));
                        const int ct = (int)(M.tile0 + tidx(m, k));
                        for_tile_items(b, false, [&](int bm, int bn) {
                            P.zitems32.push_back({Cp, xo, yo, (uint16_t)bm, (uint16_t)bn, ct});
                        }, zw);
                        P.update_flops[TC_FP32] += 2.0 * (double)b * b * K;
                        for (int nn = 0; nn < k; ++nn)
                            P.tensor_flops[TC_FP32] += 2.0 * (double)b * b * b *
                                                       plane_pairs(stored_planes(M, m, nn), stored_planes(M, k, nn), 10);
                        continue;
                    }
                    if (!fp64) continue;
                    if (zmode) {
                        // emulated FP64: 128 x 16 blocks (the diagonal SYRK keeps blocks reaching the lower part)
                        double *Cp = T(M, m, k);
                        const int xo = (int)(M.tile0 + tidx(m, 0)), yo = (int)(M.tile0 + tidx(k, 0));
                        int items = 0;
                        const int ct = (int)(M.tile0 + tidx(m, k));
                        for_tile_items(b, m == k, [&](int bm, int bn) {
                            P.zitems.push_back({Cp, xo, yo, (uint16_t)bm, (uint16_t)bn, ct});
                            ++items;
                        }, zw);
                        P.update_flops[TC_FP64] += (m == k ? 1.0 : 2.0) * (double)b * b * K;
                        for (int nn = 0; nn < k; ++nn)
                            P.tensor_flops[TC_FP64] += 2.0 * 128.0 * zw * b * items *
                                                       plane_pairs(stored_planes(M, m, nn), stored_planes(M, k, nn), 14);
                        continue;
                    }
                    jobs_here.push_back((int)P.jobs.size());
                    P.jobs.push_back({T(M, m, k), T(M, m, 0), T(M, k, 0), K, b, b, m == k ? 1 : 0, status + 2 + mi});
                    base += (m == k) ? (b / 64) * (b / 64 + 1) / 2 : (b / 64) * (b / 64);
                    P.update_flops[TC_FP64] += (m == k ? 1.0 : 2.0) * (double)b * b * K;
                }
            }
            int splits = 1;
            if (base > 0 && base < kTargetItems)
                splits = std::min((kTargetItems + base - 1) / base, std::max(1, K / 256));
            int part_next = 0;
            for (int jj : jobs_here) emit_job_items(P, jj, b, splits, part_next);
            P.max_parts = std::max(P.max_parts, part_next);
        }
        C.nit = (int)P.items.size() - C.it0;
        C.nred = (int)P.reds.size() - C.red0;
        C.nz = (int)P.zitems.size() - C.z0;
        C.ny = (int)P.zitems32.size() - C.y0;
        // digit planes of the final tiles of this column (operands of later emulated updates)
        C.dg0 = (int)P.dtiles.size();
        if (zmode)
            for (const MatDesc &M : h->mats)
                if (M.nt > k)
                    for (int m = k + 1; m < M.nt; ++m) P.dtiles.push_back((int)(M.tile0 + tidx(m, k)));
        C.ndg = (int)P.dtiles.size() - C.dg0;
        // TRSM of a mixed-precision column as C_mk L_kk^{-T} on the emulated engine (one matrix)
        C.v0 = (int)P.zinv.size();
        C.ti0 = (int)P.tinv.size();
        if (P.inv_trsm) {
            // digit slots: C_mk (and later X0, R) in the tile's own slot, L_kk^{-1} in the slot of
            // the diagonal tile (k, k), L_kk in that of (k+1, k+1) (diagonal tiles are never
            // update operands, and (k+1, k+1) is not factored yet).  Inverse e of the column
            // (one per matrix with tiles below its diagonal tile) at invbuf + e b^2.
            for (int mi = 0; mi < nmat; ++mi) {
                const MatDesc &M = h->mats[mi];
                if (M.nt <= k + 1) continue;
                const int e = (int)P.tinv.size() - C.ti0;
                P.tinv.push_back({T(M, k, k), inv_scratch + (int64_t)e * bb});
                P.dinv.push_back((int)(M.tile0 + tidx(k, k)));
            }
            // tiles in precision order: one product launch per output precision
            for (int p = 0; p < 4; ++p)
            for (int mi = 0; mi < nmat; ++mi) {
            const MatDesc &M = h->mats[mi];
            const int sinv = (int)(M.tile0 + tidx(k, k)), sl = (int)(M.tile0 + tidx(k + 1, k + 1));
            for (int m = k + 1; m < M.nt; ++m) {
                if ((M.mixed ? (int)M.map[(size_t)m * M.nt + k] : TC_FP64) != p) continue;
                const size_t before = P.zinv.size();
                double *Cp = T(M, m, k);
                double *Cs = P.inv_refine ? inv_scratch + (int64_t)(m - k) * bb : nullptr;
                const int sx = (int)(M.tile0 + tidx(m, k));
                // mixed maps: the products run on the 128 x 64 kernel (fixed plane counts)
                for_tile_items(b, false, [&](int bm, int bn) {
                    P.zinv.push_back({Cp, sx, sinv, (uint16_t)bm, (uint16_t)bn});
                    if (P.inv_refine) {
                        P.zinvc.push_back({Cs, sx, sinv, (uint16_t)bm, (uint16_t)bn});
                        P.zref.push_back({Cp, sx, sl, (uint16_t)bm, (uint16_t)bn});
                    }
                }, P.inv_refine ? Z_BN : zw);
                C.nvp[p] += (int)(P.zinv.size() - before);
            }
            }
        }
        C.nv = (int)P.zinv.size() - C.v0;
        C.nti = (int)P.tinv.size() - C.ti0;
        // 2. blocked POTRF of the diagonal tiles: per 64-panel, the block, its panel and the
        //    trailing update, each one launch over all matrices
        for (int jb = 0; jb < b / 64; ++jb) {
            PotrfStep ps;
            ps.rows = b - (jb + 1) * 64;
            ps.pe0 = (int)P.pentries.size();
            for (int mi = 0; mi < nmat; ++mi) {
                const MatDesc &M = h->mats[mi];
                if (M.nt <= k) continue;
                double *D = T(M, k, k);
                P.pentries.push_back({D + (int64_t)jb * 64 * b + jb * 64, status + 2 + mi, k * b + jb * 64, ps.rows});
            }
            ps.npe = (int)P.pentries.size() - ps.pe0;
            ps.it0 = (int)P.items.size();
            if (ps.rows > 0)
                for (int mi = 0; mi < nmat; ++mi) {
                    const MatDesc &M = h->mats[mi];
                    if (M.nt <= k) continue;
                    double *D = T(M, k, k);
                    const double *Pn = D + (int64_t)jb * 64 * b + (jb + 1) * 64;
                    const int job = (int)P.jobs.size();
                    P.jobs.push_back({D + (int64_t)(jb + 1) * 64 * b + (jb + 1) * 64, Pn, Pn, 64, ps.rows, ps.rows, 1,
                                      status + 2 + mi});
                    int dummy = 0;
                    emit_job_items(P, job, b, 1, dummy);
                }
            ps.nit = (int)P.items.size() - ps.it0;
            C.potrf.push_back(ps);
        }
        // 3. TRSM strips of the tiles below the diagonal
        C.st0 = (int)P.strips.size();
        for (int mi = 0; mi < nmat; ++mi) {
            const MatDesc &M = h->mats[mi];
            if (M.nt <= k) continue;
            P.potrf_flops += (double)b * b * b / 3.0;
            for (int m = k + 1; m < M.nt; ++m) {
                if (!P.inv_trsm)
                    for (int r0 = 0; r0 < b; r0 += 64) P.strips.push_back({T(M, m, k), T(M, k, k), status + 2 + mi, r0});
                P.trsm_flops += (double)b * b * b;
            }
        }
        C.nst = (int)P.strips.size() - C.st0;
    }
    return P;
}

size_t align_up(size_t x) { return (x + 255) / 256 * 256; }

// ----------------------------------------------------------- mixed-precision schedule
// Which low-precision operand copies each final tile needs (Section IV-C: an update runs
// in the precision of the tile it writes, so tile (i, j) is needed in p(i, k') for every
// output (i, k'), j < k' < i, that reads it as X, and in p(m, i) for every output (m, i),
// m > i, that reads it as Y), the pool slot of each copy, and per column step the
// tensor-core work items, the tiles to store in their precision and the copies to make.
// Tile indices are global: matrix tile0 + packed index.
struct MxpPlan {
    std::vector<int> slot[3];          // [q-1][global tile] -> slot, -1 if not needed
    int64_t nslots[3] = {0, 0, 0};
    std::vector<uint8_t> prec;         // precision of every tile (diagonal FP64)
    std::vector<int> tiles;            // per column step: off-diagonal tiles to store / copy
    std::vector<CopyJob> copies;
    std::vector<QItem> qitems;
    struct Col { int t0, nt, c0, nc, q0[3], nq[3]; };
    std::vector<Col> cols;
    int64_t T = 0;
    double flops[4] = {0, 0, 0, 0};
};

MxpPlan build_mxp(tc_handle h, double *W) {
    MxpPlan X;
    // FP32 outputs on digit planes (fp64_mode >= 1 and fp32_updates 0), else as TF32 x 3
    const bool zmode = h->cfg.fp64_mode >= 1 && h->cfg.fp32_updates == 0;
    const int b = h->b;
    const int64_t bb = (int64_t)b * b;
    int ntmax = 0;
    for (const MatDesc &M : h->mats) {
        X.T = std::max<int64_t>(X.T, M.tile0 + tidx(M.nt, 0));
        ntmax = std::max(ntmax, M.nt);
    }
    for (int q = 0; q < 3; ++q) X.slot[q].assign(X.T, -1);
    X.prec.assign(X.T, 0);
    for (const MatDesc &M : h->mats) {
        if (!M.mixed) continue;
        const int nt = M.nt;
        auto P = [&](int i, int j) { return (int)M.map[(size_t)i * nt + j]; };
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < i; ++j) {
                const int64_t g = M.tile0 + tidx(i, j);
                X.prec[g] = (uint8_t)P(i, j);
                unsigned mask = 0;
                for (int kk = j + 1; kk < i; ++kk) mask |= 1u << P(i, kk);
                for (int m = i + 1; m < nt; ++m) mask |= 1u << P(m, i);
                if (zmode) mask &= ~(1u << TC_FP32);
                for (int q = 1; q <= 3; ++q)
                    if (mask & (1u << q)) X.slot[q - 1][g] = (int)X.nslots[q - 1]++;
            }
    }
    X.cols.resize(ntmax);
    const int nbk = b / 128;
    for (int k = 0; k < ntmax; ++k) {
        MxpPlan::Col &C = X.cols[k];
        for (int q = 1; q <= 3; ++q) {
            C.q0[q - 1] = (int)X.qitems.size();
            if (k > 0 && !(zmode && q == TC_FP32))
                for (const MatDesc &M : h->mats) {
                    if (!M.mixed || M.nt <= k) continue;
                    for (int m = k + 1; m < M.nt; ++m) {
                        if ((int)M.map[(size_t)m * M.nt + k] != q) continue;
                        double *Cp = W + (M.tile0 + tidx(m, k)) * bb;
                        const int xo = (int)(M.tile0 + tidx(m, 0)), yo = (int)(M.tile0 + tidx(k, 0));
                        for (int bn = 0; bn < nbk; ++bn)
                            for (int bm = 0; bm < nbk; ++bm) X.qitems.push_back({Cp, xo, yo, (uint16_t)bm, (uint16_t)bn});
                        X.flops[q] += 2.0 * b * (double)b * k * b;
                    }
                }
            C.nq[q - 1] = (int)X.qitems.size() - C.q0[q - 1];
        }
        C.t0 = (int)X.tiles.size();
        C.c0 = (int)X.copies.size();
        for (const MatDesc &M : h->mats) {
            if (!M.mixed || M.nt <= k) continue;
            for (int m = k + 1; m < M.nt; ++m) {
                const int g = (int)(M.tile0 + tidx(m, k));
                X.tiles.push_back(g);
                for (int q = 1; q <= 3; ++q)
                    if (X.slot[q - 1][g] >= 0) X.copies.push_back({g, q, X.slot[q - 1][g]});
            }
        }
        C.nt = (int)X.tiles.size() - C.t0;
        C.nc = (int)X.copies.size() - C.c0;
    }
    return X;
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
    const int64_t T = M.T;
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
    CK(cudaMemcpy(h->mxtab.p, host.data(), total, cudaMemcpyHostToDevice));
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

// Low-precision updates of column step k (before its POTRF).
int mxp_updates(tc_handle h, const MxpPlan &M, const MxpDev &D, int k, bool spans) {
    const MxpPlan::Col &C = M.cols[k];
    int *err = static_cast<int *>(h->status.p) + 1;
    for (int q = 1; q <= 3; ++q) {
        if (!C.nq[q - 1]) continue;
        const CUtensorMap &a0 = q == 1 ? h->map_hi : q == 2 ? h->map16 : h->map8;
        const CUtensorMap &a1 = q == 1 ? h->map_lo : a0;
        const int sp = spans ? span_begin(h, CAT_UPD64 + q) : -1;
        launch_qgemm(q, a0, a1, a0, a1, D.qitems + C.q0[q - 1], C.nq[q - 1], D.slot[q - 1],
                     q == 2 ? D.exps16 : q == 3 ? D.exps8 : nullptr, k, h->b, err, h->s, wait_limit_ns(h), wait_test(h));
        span_end(h, sp);
        CK_LAUNCH();
        ++h->upd_launches[q];
    }
    return TC_OK;
}

// Stores and operand copies of the final tiles of column step k (after its TRSMs).
int mxp_convert(tc_handle h, const MxpPlan &M, const MxpDev &D, int k, bool spans) {
    const MxpPlan::Col &C = M.cols[k];
    if (!C.nt) return TC_OK;
    double *W = static_cast<double *>(h->W.p);
    const int sp = spans ? span_begin(h, CAT_CONVERT) : -1;
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

// Device copies of the plan's tables (uploaded before any launch so that the launch
// sequence itself can be captured into a CUDA graph).
struct PlanDev {
    const DJob *jobs;
    const DItem *items;
    const DRed *reds;
    const TStrip *strips;
    const PEntry *pentries;
    const LEntry *lentries;
    const TEntry *tinv = nullptr;       // inverse-based TRSM: the diagonal tiles to invert, per column
    const int *dinv = nullptr;          //   ... and the digit slots of their inverses
    const ZItem *zitems = nullptr, *zitems32 = nullptr, *zinv = nullptr, *zinvc = nullptr, *zref = nullptr;
    double *zamax2 = nullptr;
    double *zamax3 = nullptr;    // refinement: amax of L_kk, X0 and R (3 x Ttot)
    const int *dtiles = nullptr;
    const uint8_t *zplanes = nullptr;   // leading non-zero digit planes per tile (mixed maps), else null
    double *oamax = nullptr;            // mixed: input amax of every tile (plane budgets of the updates)
    const int *alltiles = nullptr;      // mixed: 0 .. Ttot-1 (the tile list of that amax)
    unsigned long long *pairs = nullptr;   // mixed: plane pairs multiplied, FP64 / FP32 outputs
    int *zexps = nullptr;
    double *zamax = nullptr;
    MxpDev mx{};
    bool mixed = false;
};

int prepare_factor(tc_handle h, const Plan &P, const MxpPlan *M, PlanDev &D) {
    const size_t sj = P.jobs.size() * sizeof(DJob), si = P.items.size() * sizeof(DItem);
    const size_t sr = P.reds.size() * sizeof(DRed), ss = P.strips.size() * sizeof(TStrip);
    const size_t sp = P.pentries.size() * sizeof(PEntry), sl = P.lentries.size() * sizeof(LEntry);
    const size_t oj = 0, oi = align_up(oj + sj), orr = align_up(oi + si), os = align_up(orr + sr);
    const size_t st = P.tinv.size() * sizeof(TEntry), sdv = P.dinv.size() * sizeof(int);
    const size_t op = align_up(os + ss), ol = align_up(op + sp), ot = align_up(ol + sl), odv = align_up(ot + st);
    const size_t total = align_up(odv + sdv);
    int rc = ensure(h, h->tables, total);
    if (rc) return rc;
    std::vector<char> host(total);
    if (sj) memcpy(host.data() + oj, P.jobs.data(), sj);
    if (si) memcpy(host.data() + oi, P.items.data(), si);
    if (sr) memcpy(host.data() + orr, P.reds.data(), sr);
    if (ss) memcpy(host.data() + os, P.strips.data(), ss);
    if (sp) memcpy(host.data() + op, P.pentries.data(), sp);
    if (sl) memcpy(host.data() + ol, P.lentries.data(), sl);
    if (st) memcpy(host.data() + ot, P.tinv.data(), st);
    if (sdv) memcpy(host.data() + odv, P.dinv.data(), sdv);
    CK(cudaMemcpy(h->tables.p, host.data(), total, cudaMemcpyHostToDevice));
    char *base = static_cast<char *>(h->tables.p);
    D.jobs = reinterpret_cast<const DJob *>(base + oj);
    D.items = reinterpret_cast<const DItem *>(base + oi);
    D.reds = reinterpret_cast<const DRed *>(base + orr);
    D.strips = reinterpret_cast<const TStrip *>(base + os);
    D.pentries = reinterpret_cast<const PEntry *>(base + op);
    D.lentries = reinterpret_cast<const LEntry *>(base + ol);
    D.tinv = reinterpret_cast<const TEntry *>(base + ot);
    D.dinv = reinterpret_cast<const int *>(base + odv);
    if ((rc = ensure(h, h->partials, (size_t)std::max(1, P.max_parts) * 4096 * sizeof(double)))) return rc;
    h->pairs_dev = nullptr;
    if (!P.zitems.empty() || !P.zitems32.empty() || !P.zinv.empty() || !P.dtiles.empty()) {
        // digit planes (14 per tile), exponents, amax, the Z items and the digit tile lists
        const int64_t Tt = P.Ttot;
        const size_t bb = (size_t)h->b * h->b;
        if ((rc = ensure(h, h->dpool, (size_t)Tt * 14 * bb))) return rc;
        const size_t oz = 0, oy = align_up(P.zitems.size() * sizeof(ZItem));
        const size_t ov = align_up(oy + P.zitems32.size() * sizeof(ZItem));
        const size_t ovc = align_up(ov + P.zinv.size() * sizeof(ZItem));
        const size_t ovr = align_up(ovc + P.zinvc.size() * sizeof(ZItem));
        const size_t od = align_up(ovr + P.zref.size() * sizeof(ZItem)), oe = align_up(od + P.dtiles.size() * 4);
        const size_t oa = align_up(oe + Tt * 4), oa2 = align_up(oa + Tt * 8), oa3 = align_up(oa2 + Tt * 8);
        const size_t opl = align_up(oa3 + (P.inv_refine ? 3 * Tt * 8 : 0));
        const size_t ooa = align_up(opl + Tt), oall = align_up(ooa + Tt * 8), opc = align_up(oall + Tt * 4);
        const size_t zt = align_up(opc + 2 * sizeof(unsigned long long));
        if ((rc = ensure(h, h->ztab, zt))) return rc;
        std::vector<char> zh(zt, 0);
        if (!P.zitems.empty()) memcpy(zh.data() + oz, P.zitems.data(), P.zitems.size() * sizeof(ZItem));
        if (!P.zitems32.empty()) memcpy(zh.data() + oy, P.zitems32.data(), P.zitems32.size() * sizeof(ZItem));
        if (!P.zinv.empty()) memcpy(zh.data() + ov, P.zinv.data(), P.zinv.size() * sizeof(ZItem));
        if (!P.zinvc.empty()) memcpy(zh.data() + ovc, P.zinvc.data(), P.zinvc.size() * sizeof(ZItem));
        if (!P.zref.empty()) memcpy(zh.data() + ovr, P.zref.data(), P.zref.size() * sizeof(ZItem));
        if (!P.dtiles.empty()) memcpy(zh.data() + od, P.dtiles.data(), P.dtiles.size() * 4);
        // digit planes a stored tile can have non-zero: E4M3 with its power-of-two scale 2^e holds
        // multiples of 2^(e-9) below 2^(e+9) (18 bits: planes 1..5), FP16 multiples of 2^(e-24)
        // below 2^(e+16) (40 bits: planes 1..10); FP32 and FP64 use all 14
        bool any_mixed = false;
        for (const MatDesc &Md : h->mats) any_mixed |= Md.mixed;
        if (any_mixed) {
            int *all = reinterpret_cast<int *>(zh.data() + oall);
            for (int64_t t = 0; t < Tt; ++t) all[t] = (int)t;
            uint8_t *pl = reinterpret_cast<uint8_t *>(zh.data() + opl);
            memset(pl, 14, Tt);
            for (const MatDesc &Md : h->mats) {
                if (!Md.mixed) continue;
                for (int i = 0; i < Md.nt; ++i)
                    for (int j = 0; j < i; ++j) {
                        const int p = Md.map[(size_t)i * Md.nt + j];
                        pl[Md.tile0 + tidx(i, j)] = (uint8_t)(p == TC_FP8 ? 5 : p == TC_FP16 ? 10 : 14);
                    }
            }
        }
        CK(cudaMemcpy(h->ztab.p, zh.data(), zt, cudaMemcpyHostToDevice));
        char *zb = static_cast<char *>(h->ztab.p);
        D.zitems = reinterpret_cast<const ZItem *>(zb + oz);
        D.zitems32 = reinterpret_cast<const ZItem *>(zb + oy);
        D.zinv = reinterpret_cast<const ZItem *>(zb + ov);
        D.zinvc = reinterpret_cast<const ZItem *>(zb + ovc);
        D.zref = reinterpret_cast<const ZItem *>(zb + ovr);
        if (P.inv_refine) D.zamax3 = reinterpret_cast<double *>(zb + oa3);
        D.zamax2 = reinterpret_cast<double *>(zb + oa2);
        D.dtiles = reinterpret_cast<const int *>(zb + od);
        D.zexps = reinterpret_cast<int *>(zb + oe);
        D.zamax = reinterpret_cast<double *>(zb + oa);
        D.zplanes = any_mixed ? reinterpret_cast<const uint8_t *>(zb + opl) : nullptr;
        if (any_mixed) {
            D.oamax = reinterpret_cast<double *>(zb + ooa);
            D.alltiles = reinterpret_cast<const int *>(zb + oall);
            D.pairs = reinterpret_cast<unsigned long long *>(zb + opc);
        }
        h->pairs_dev = D.pairs;
        if (make_digit_map(&h->map_zx, h->dpool.p, Tt * 14 * h->b, h->b, 128) ||
            make_digit_map(&h->map_zy, h->dpool.p, Tt * 14 * h->b, h->b, Z_BN))
            return set_err(h, TC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the digit planes");
        if (P.zwidth == Z64_BN && make_zgemm64_maps(&h->maps64, h->dpool.p, Tt * 14, h->b))
            return set_err(h, TC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the digit planes (3D maps)");
    }
    D.mixed = M != nullptr;
    if (M && (rc = setup_mxp(h, *M, D.mx))) return rc;
    return TC_OK;
}

// The launch sequence of one factorization (capturable: device-side copies, memsets and
// kernels only).  A_dev of every matrix is copied into W first.
int execute_factor(tc_handle h, const Plan &P, const MxpPlan *M, const PlanDev &D, bool spans) {
    const int b = h->b;
    const int64_t bb = (int64_t)b * b;
    int *status = static_cast<int *>(h->status.p);
    double *W = static_cast<double *>(h->W.p);
    double *parts = static_cast<double *>(h->partials.p);
    const int nmat = (int)h->mats.size();
    for (const MatDesc &Md : h->mats)
        CK(cudaMemcpyAsync(W + Md.tile0 * bb, Md.A_dev, (size_t)tidx(Md.nt, 0) * bb * sizeof(double),
                           cudaMemcpyDeviceToDevice, h->s));
    launch_fix_padding_batched(D.lentries, nmat, P.ntmax, b, h->s);
    CK_LAUNCH();
    CK(cudaMemsetAsync(status, 0, (2 + nmat) * sizeof(int), h->s));
    if (D.zamax) CK(cudaMemsetAsync(D.zamax, 0, P.Ttot * sizeof(double), h->s));
    if (D.zamax2) CK(cudaMemsetAsync(D.zamax2, 0, P.Ttot * sizeof(double), h->s));
    if (D.zamax3) CK(cudaMemsetAsync(D.zamax3, 0, 3 * P.Ttot * sizeof(double), h->s));
    if (D.oamax) {
        // scale of every output tile before its updates: the reference of its plane budgets
        CK(cudaMemsetAsync(D.oamax, 0, P.Ttot * sizeof(double), h->s));
        CK(cudaMemsetAsync(D.pairs, 0, 2 * sizeof(unsigned long long), h->s));
        launch_tile_amax(W, b, D.alltiles, (int)P.Ttot, D.oamax, h->s);
        CK_LAUNCH();
    }
    // mixed-precision digit-plane updates: per-source plane budgets relative to the output
    // tile's input scale (FP64 outputs: 14 reference planes; FP32 outputs: 10), margin 2 planes
    ZPlanes zp64, zp32;
    zp64.src_planes_tab = zp32.src_planes_tab = D.zplanes;
    zp64.out_amax = zp32.out_amax = D.oamax;
    zp64.rref = 14;
    zp32.rref = 10;
    zp64.margin = zp32.margin = kPlaneMargin;
    zp64.pair_count = D.pairs;
    zp32.pair_count = D.pairs ? D.pairs + 1 : nullptr;
    if (M) {
        CK(cudaMemsetAsync(D.mx.amaxL, 0, M->T * sizeof(double), h->s));
        CK(cudaMemsetAsync(D.mx.amaxS, 0, M->T * sizeof(double), h->s));
        CK(cudaMemsetAsync(D.mx.exps16, 0, M->T * sizeof(int), h->s));
        CK(cudaMemsetAsync(D.mx.exps8, 0, M->T * sizeof(int), h->s));
    }
    for (int k = 0; k < P.ntmax; ++k) {
        const ColPlan &C = P.cols[k];
        if (C.nit) {
            const int sp = spans ? span_begin(h, CAT_UPD64) : -1;
            launch_dgemm_update(D.jobs, D.items + C.it0, C.nit, b, parts, nullptr, h->s);
            span_end(h, sp);
            CK_LAUNCH();
            ++h->upd_launches[TC_FP64];
        }
        if (C.nred) {
            launch_dgemm_reduce(D.reds + C.red0, C.nred, b, parts, nullptr, h->s);
            CK_LAUNCH();
        }
        if (C.nz) {
            const int sp = spans ? span_begin(h, CAT_UPD64) : -1;
            if (P.zwidth == Z64_BN)
                launch_zgemm64(h->maps64, D.zitems + C.z0, C.nz, D.zexps, k, b, status + 1, h->s, zp64, 0,
                               wait_limit_ns(h), wait_test(h));
            else
                launch_zgemm(h->map_zx, h->map_zy, D.zitems + C.z0, C.nz, D.zexps, k, b, status + 1, h->s, 14, 0,
                             D.zplanes ? &zp64 : nullptr, wait_limit_ns(h), wait_test(h));
            span_end(h, sp);
            CK_LAUNCH();
            ++h->upd_launches[TC_FP64];
        }
        if (C.ny) {
            const int sp = spans ? span_begin(h, CAT_UPD32) : -1;
            if (P.zwidth == Z64_BN)
                launch_zgemm64(h->maps64, D.zitems32 + C.y0, C.ny, D.zexps, k, b, status + 1, h->s, zp32, 0,
                               wait_limit_ns(h), wait_test(h));
            else
                launch_zgemm(h->map_zx, h->map_zy, D.zitems32 + C.y0, C.ny, D.zexps, k, b, status + 1, h->s, 10, 0,
                             D.zplanes ? &zp32 : nullptr, wait_limit_ns(h), wait_test(h));
            span_end(h, sp);
            CK_LAUNCH();
            ++h->upd_launches[TC_FP32];
        }
        if (M) {
            const int rc = mxp_updates(h, *M, D.mx, k, spans);
            if (rc) return rc;
        }
        const int sp_potrf = spans ? span_begin(h, CAT_POTRF) : -1;
        for (const PotrfStep &ps : C.potrf) {
            launch_potrf_blocks(D.pentries + ps.pe0, ps.npe, b, h->s);
            CK_LAUNCH();
            if (ps.rows > 0) {
                launch_trsm_rows_batched(D.pentries + ps.pe0, ps.npe, ps.rows, b, h->s);
                CK_LAUNCH();
                launch_dgemm_update(D.jobs, D.items + ps.it0, ps.nit, b, parts, nullptr, h->s);
                CK_LAUNCH();
            }
        }
        span_end(h, sp_potrf);
        if (C.nv) {
            // L_mk = C_mk L_kk^{-T}: L_kk^{-1} by column-parallel substitution (FP64), then digit
            // planes of L_kk^{-1} and of every C_mk, and one emulated product per tile (three,
            // with the refinement step, for an all-FP64 factorization)
            const int sp = spans ? span_begin(h, CAT_TRSM) : -1;
            const MatDesc &Md = h->mats[0];
            double *inv = static_cast<double *>(h->invbuf.p);
            uint8_t *pool = static_cast<uint8_t *>(h->dpool.p);
            if (b <= 2048) {
                // inverse e of the column at inv + e b^2 (one per matrix), then its amax and
                // digit planes into the diagonal tile's slot
                launch_trinv_batched(D.tinv + C.ti0, C.nti, b, h->s);
                CK_LAUNCH();
                launch_tile_amax(W, b, D.dinv + C.ti0, C.nti, D.zamax2, h->s, inv);
                CK_LAUNCH();
                launch_digits(W, b, D.dinv + C.ti0, C.nti, D.zamax2, pool, D.zexps, h->s, inv);
                CK_LAUNCH();
            } else {                       // one matrix: its shared-memory column panel would not fit
                const int gkk = (int)(Md.tile0 + tidx(k, k));
                const double *Lkk0 = W + (Md.tile0 + tidx(k, k)) * bb;
                launch_set_identity(inv, b, h->s);
                CK_LAUNCH();
                launch_trsm_tile(inv, Lkk0, b, b, nullptr, h->s);     // inv = L_kk^{-T}
                CK_LAUNCH();
                launch_amax_ptr(inv, bb, D.zamax2 + gkk, h->s);
                CK_LAUNCH();
                launch_digits_src(inv, b, 1, gkk, D.zamax2 + gkk, pool, D.zexps, h->s);
                CK_LAUNCH();
            }
            launch_tile_amax(W, b, D.dtiles + C.dg0, C.ndg, D.zamax2, h->s);
            CK_LAUNCH();
            launch_digits(W, b, D.dtiles + C.dg0, C.ndg, D.zamax2, pool, D.zexps, h->s);
            CK_LAUNCH();
            if (!P.inv_refine) {
                // the product's truncation stays below the rounding to each stored precision
                int off = C.v0;
                for (int p = 0; p < 4; ++p) {
                    if (P.zwidth == Z64_BN) {
                        ZPlanes fixed;                  // every source on the precision's plane count
                        fixed.src_planes_tab = nullptr;
                        fixed.out_amax = nullptr;
                        fixed.rref = ZTRSM_PLANES[p];
                        fixed.margin = 0;
                        fixed.pair_count = nullptr;
                        launch_zgemm64(h->maps64, D.zinv + off, C.nvp[p], D.zexps, 1, b, status + 1, h->s, fixed, 1,
                                       wait_limit_ns(h), wait_test(h));
                    } else {
                        launch_zgemm(h->map_zx, h->map_zy, D.zinv + off, C.nvp[p], D.zexps, 1, b, status + 1, h->s,
                                     ZTRSM_PLANES[p], 1, nullptr, wait_limit_ns(h), wait_test(h));
                    }
                    CK_LAUNCH();
                    off += C.nvp[p];
                }
            } else {
                // X0 = C L_kk^{-T};  R = C - X0 L_kk^T;  L_mk = X0 + R L_kk^{-T}  (C is overwritten by R)
                const int Tt = (int)P.Ttot, gl = (int)(Md.tile0 + tidx(k + 1, k + 1));
                double *Lkk = W + (Md.tile0 + tidx(k, k)) * bb, *X0 = inv + bb;
                double *am_l = D.zamax3, *am_x = D.zamax3 + Tt, *am_r = D.zamax3 + 2 * Tt;
                launch_lower_only(Lkk, b, h->s);
                CK_LAUNCH();
                launch_amax_ptr(Lkk, bb, am_l + gl, h->s);
                CK_LAUNCH();
                launch_digits_src(Lkk, b, 0, gl, am_l + gl, pool, D.zexps, h->s);
                CK_LAUNCH();
                launch_zgemm(h->map_zx, h->map_zy, D.zinvc + C.v0, C.nv, D.zexps, 1, b, status + 1, h->s, 14, 1, nullptr,
                             wait_limit_ns(h), wait_test(h));
                CK_LAUNCH();
                launch_tile_amax(W, b, D.dtiles + C.dg0, C.ndg, am_x, h->s, X0);
                CK_LAUNCH();
                launch_digits(W, b, D.dtiles + C.dg0, C.ndg, am_x, pool, D.zexps, h->s, X0);
                CK_LAUNCH();
                launch_zgemm(h->map_zx, h->map_zy, D.zref + C.v0, C.nv, D.zexps, 1, b, status + 1, h->s, 14, 0, nullptr,
                             wait_limit_ns(h), wait_test(h));
                CK_LAUNCH();
                launch_tile_amax(W, b, D.dtiles + C.dg0, C.ndg, am_r, h->s);
                CK_LAUNCH();
                launch_digits(W, b, D.dtiles + C.dg0, C.ndg, am_r, pool, D.zexps, h->s);
                CK_LAUNCH();
                launch_zgemm(h->map_zx, h->map_zy, D.zinv + C.v0, C.nv, D.zexps, 1, b, status + 1, h->s, ZREF_PLANES, 1,
                             nullptr, wait_limit_ns(h), wait_test(h));
                CK_LAUNCH();
                launch_add_tiles(W, b, D.dtiles + C.dg0, C.ndg, X0, h->s);
                CK_LAUNCH();
            }
            span_end(h, sp);
        }
        if (C.nst) {
            const int sp = spans ? span_begin(h, CAT_TRSM) : -1;
            launch_trsm_strips(D.strips + C.st0, C.nst, b, b, nullptr, h->s);
            span_end(h, sp);
            CK_LAUNCH();
        }
        if (M) {
            const int rc = mxp_convert(h, *M, D.mx, k, spans);
            if (rc) return rc;
        }
        if (C.ndg) {
            const int sp = spans ? span_begin(h, CAT_CONVERT) : -1;
            launch_tile_amax(W, b, D.dtiles + C.dg0, C.ndg, D.zamax, h->s);
            CK_LAUNCH();
            launch_digits(W, b, D.dtiles + C.dg0, C.ndg, D.zamax, static_cast<uint8_t *>(h->dpool.p), D.zexps, h->s);
            span_end(h, sp);
            CK_LAUNCH();
        }
    }
    double *sc = static_cast<double *>(h->scratch.p);
    launch_logdet_batched(D.lentries, nmat, b, sc, h->s);
    CK_LAUNCH();
    return TC_OK;
}

// Results of the last execute: info words and log-determinants of every matrix.
int collect_results(tc_handle h, int *first_bad, int *err_word) {
    const int nmat = (int)h->mats.size();
    std::vector<int> st(2 + nmat);
    h->logdets.assign(nmat, 0.0);
    CK(cudaMemcpyAsync(st.data(), h->status.p, st.size() * sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(h->logdets.data(), h->scratch.p, nmat * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    h->pairs_exec[0] = h->pairs_exec[1] = 0;
    if (h->pairs_dev) CK(cudaMemcpyAsync(h->pairs_exec, h->pairs_dev, sizeof h->pairs_exec, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    h->infos.assign(st.begin() + 2, st.end());
    *err_word = st[1];
    *first_bad = 0;
    for (int i = 0; i < nmat && !*first_bad; ++i) *first_bad = h->infos[i];
    return TC_OK;
}

void fill_stats(tc_handle h, const Plan &P, const MxpPlan *M, tc_stats *stats, double t0, int64_t launches0,
                int info) {
    memset(stats, 0, sizeof *stats);
    stats->t_ms = now_ms() - t0;
    for (const MatDesc &Md : h->mats) {
        stats->flops += (double)Md.n * Md.n * Md.n / 3.0;
        for (int i = 0; i < Md.nt; ++i)
            for (int j = 0; j <= i; ++j) stats->tiles[i == j ? 0 : Md.map[(size_t)i * Md.nt + j]]++;
    }
    stats->update_flops[0] = P.update_flops[0];
    if (M)
        for (int p = 1; p < 4; ++p) stats->update_flops[p] = M->flops[p];
    stats->update_flops[1] += P.update_flops[1];
    for (int p = 0; p < 4; ++p) stats->tensor_flops[p] = P.tensor_flops[p];
    if (h->pairs_dev) {
        // mixed precision: the plane pairs the update kernels counted as they issued them
        const double per_pair = 2.0 * 128.0 * P.zwidth * h->b;
        stats->tensor_flops[TC_FP64] = per_pair * (double)h->pairs_exec[0];
        stats->tensor_flops[TC_FP32] = per_pair * (double)h->pairs_exec[1];
    }
    if (M) {
        stats->tensor_flops[TC_FP32] += 3.0 * M->flops[TC_FP32];     // TF32 x 3 (when FP32 runs there)
        stats->tensor_flops[TC_FP16] += M->flops[TC_FP16];
        stats->tensor_flops[TC_FP8] += M->flops[TC_FP8];
    }
    stats->trsm_flops = P.trsm_flops;
    stats->potrf_flops = P.potrf_flops;
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

// Plan + prepare + execute the matrices in h->mats (W already sized).  With use_graph the
// launch sequence is captured once into a CUDA graph and replayed while the batch repeats.
int factor_matrices(tc_handle h, tc_stats *stats, bool use_graph, const std::vector<int64_t> *key) {
    const double t0 = now_ms();
    const int64_t launches0 = h->launches;
    spans_reset(h);
    for (int p = 0; p < 4; ++p) h->upd_launches[p] = 0;
    bool mixed = false;
    for (const MatDesc &Md : h->mats) mixed |= Md.mixed;
    int *status = static_cast<int *>(h->status.p);
    double *W = static_cast<double *>(h->W.p);
    int rc = ensure(h, h->status, (2 + h->mats.size()) * sizeof(int));
    if (rc) return rc;
    status = static_cast<int *>(h->status.p);
    if ((rc = ensure(h, h->scratch, std::max<size_t>(4096, h->mats.size()) * sizeof(double)))) return rc;
    if (h->cfg.fp64_mode == 2 && (h->mats.size() == 1 || mixed)) {
        // L_kk^{-1} of every matrix of a column (and, for one all-FP64 matrix, X0 of each tile)
        const size_t bb = (size_t)h->b * h->b;
        const size_t tiles = h->mats.size() > 1 ? h->mats.size() : (mixed ? 1 : 1 + (size_t)h->mats[0].nt);
        if ((rc = ensure(h, h->invbuf, tiles * bb * sizeof(double)))) return rc;
    }
    Plan P = build_plan(h, W, status);
    MxpPlan M;
    if (mixed) M = build_mxp(h, W);
    const MxpPlan *Mp = mixed ? &M : nullptr;
    // a captured graph holds device pointers and reads the uploaded tables: it replays only
    // while no buffer moved and no other factorization re-uploaded its tables
    if (!use_graph && h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        h->graph_key.clear();
    }
    const bool replay = use_graph && h->graph && key && *key == h->graph_key && h->graph_gen == h->buf_gen;
    if (!replay) {
        PlanDev D;
        if ((rc = prepare_factor(h, P, Mp, D))) return rc;
        if (use_graph) {
            if (h->graph) {
                cudaGraphExecDestroy(h->graph);
                h->graph = nullptr;
                h->graph_key.clear();
            }
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
            rc = execute_factor(h, P, Mp, D, false);
            cudaError_t e = cudaStreamEndCapture(h->s, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture", __LINE__);
            e = cudaGraphInstantiate(&h->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate", __LINE__);
            h->graph_key = *key;
            h->graph_gen = h->buf_gen;
        } else {
            if ((rc = execute_factor(h, P, Mp, D, true))) return rc;
        }
    }
    if (use_graph) CK(cudaGraphLaunch(h->graph, h->s));
    int bad = 0, err = 0;
    if ((rc = collect_results(h, &bad, &err))) return rc;
    if (err) {
        h->factored = false;
        return set_err(h, TC_ERR_TIMEOUT, err == 2 ? "tensor-core update found no operand copy (internal)"
                                                     : "a tensor-core update timed out waiting on its pipeline");
    }
    if (stats) fill_stats(h, P, Mp, stats, t0, launches0, bad);
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
    if (h->cfg.fp64_mode < 0 || h->cfg.fp64_mode > 2 || h->cfg.fp32_updates < 0 || h->cfg.fp32_updates > 1 ||
        h->cfg.wait_limit_us < 0) {
        delete h;
        return TC_ERR_ARG;
    }
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
                      &h->pool_hi, &h->pool_lo, &h->pool16, &h->pool8, &h->mxtab, &h->logdiag, &h->dpool, &h->ztab,
                      &h->invbuf, &h->stab})
        release(*d);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    release(h->bstage);
    if (h->hcompact) cudaFreeHost(h->hcompact);
    if (h->s_h2d) cudaStreamDestroy(h->s_h2d);
    if (h->s_d2h) cudaStreamDestroy(h->s_d2h);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    if (h->own_stream && h->s) cudaStreamDestroy(h->s);
    delete h;
}

const char *tc_last_error(tc_handle h) { return h ? h->err.c_str() : "null handle"; }

int tc_set_wait_limit(tc_handle h, int wait_limit_us, int wait_test) {
    if (!h) return TC_ERR_ARG;
    if (wait_limit_us < 0) return set_err(h, TC_ERR_ARG, "wait_limit_us must be >= 0");
    h->cfg.wait_limit_us = wait_limit_us;
    h->cfg.wait_test = wait_test;
    return TC_OK;
}

int tc_matern_tiles(tc_handle h, int64_t n, int b, const double *points, double sigma2, double range_a,
                    double nu, double nugget, double *A_tiles) {
    int rc = check_nb(h, n, b);
    if (rc) return rc;
    if (!points || !A_tiles) return set_err(h, TC_ERR_ARG, "points and A_tiles must not be NULL");
    if (!(range_a > 0) || !(sigma2 > 0)) return set_err(h, TC_ERR_ARG, "range and variance must be positive");
    int nu2 = 0;                                  // 0: the Bessel form for any other nu
    if (nu == 0.5) nu2 = 1;
    else if (nu == 1.5) nu2 = 3;
    else if (nu == 2.5) nu2 = 5;
    else if (!(nu > 0.0 && nu <= 16.0)) return set_err(h, TC_ERR_ARG, "smoothness must lie in (0, 16]");
    const int nt = (int)((n + b - 1) / b);
    if ((int64_t)nt * (nt + 1) / 2 > 65535)           // one grid row per lower tile
        return set_err(h, TC_ERR_ARG, "the generator takes at most 65535 lower tiles (Nt <= 361)");
    CK(cudaSetDevice(h->device));
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
    launch_matern(dout, n, b, nt, dpts, sigma2, range_a, nu2, nu, nugget, h->s);
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
    rc = ensure(h, h->sumsq, (size_t)T * sizeof(double));
    if (rc) return rc;
    double *ssd = static_cast<double *>(h->sumsq.p);
    DevBuf tmp;
    if (on_device(A_tiles)) {
        launch_tile_sumsq(A_tiles, nt, b, n, ssd, h->s);
        CK_LAUNCH();
    } else {
        // a host matrix streams through a bounded staging buffer (about 1 GiB of tiles), so the
        // map needs no device copy of A beside what the handle already holds
        const size_t tile_bytes = (size_t)b * b * sizeof(double);
        const int64_t per = std::max<int64_t>(1, std::min<int64_t>(T, ((int64_t)1 << 30) / (int64_t)tile_bytes));
        rc = ensure(h, tmp, (size_t)per * tile_bytes);
        if (rc) return rc;
        for (int64_t t0 = 0; t0 < T; t0 += per) {
            const int64_t cnt = std::min<int64_t>(per, T - t0);
            CK(cudaMemcpyAsync(tmp.p, A_tiles + t0 * (int64_t)b * b, (size_t)cnt * tile_bytes, cudaMemcpyHostToDevice,
                               h->s));
            launch_tile_sumsq_range(static_cast<const double *>(tmp.p), (int)t0, (int)cnt, b, n, ssd, h->s);
            CK_LAUNCH();
        }
    }
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
    h->factored = false;
    h->ooc = false;
    const int nt = (int)((n + b - 1) / b);
    const int64_t T = tidx(nt, 0);
    const size_t bytes = (size_t)T * b * b * sizeof(double);
    MatDesc M;
    M.n = n;
    M.nt = nt;
    M.tile0 = 0;
    M.map.assign((size_t)nt * nt, TC_FP64);
    if (map) {
        if (on_device(map)) CK(cudaMemcpy(M.map.data(), map, M.map.size(), cudaMemcpyDeviceToHost));
        else memcpy(M.map.data(), map, M.map.size());
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < nt; ++j) {
                uint8_t &v = M.map[(size_t)i * nt + j];
                if (j >= i) v = TC_FP64;
                if (v > TC_FP8) return set_err(h, TC_ERR_ARG, "precision map entries must be 0..3");
            }
    }
    for (uint8_t v : M.map) M.mixed |= (v != TC_FP64);
    if (M.mixed && b % 128) return set_err(h, TC_ERR_UNSUPPORTED, "mixed precision needs a tile size that is a multiple of 128");
    if (h->cfg.fp64_mode >= 1 && b % 128)
        return set_err(h, TC_ERR_UNSUPPORTED, "emulated FP64 updates need a tile size that is a multiple of 128");
    if ((rc = ensure(h, h->W, bytes))) return rc;
    // the caller's A stays readable for refinement: reference it on the device or copy it
    if (on_device(A_tiles)) {
        M.A_dev = A_tiles;
    } else {
        if ((rc = ensure(h, h->Acopy, bytes))) return rc;
        CK(cudaMemcpyAsync(h->Acopy.p, A_tiles, bytes, cudaMemcpyHostToDevice, h->s));
        M.A_dev = static_cast<const double *>(h->Acopy.p);
    }
    h->mats.assign(1, M);
    h->n = n;
    h->b = b;
    h->nt = nt;
    h->map = M.map;
    h->mixed = M.mixed;
    h->A_dev = M.A_dev;
    h->normA_inf = -1.0;
    h->normA_infs.assign(1, -1.0);
    if ((rc = factor_matrices(h, stats, false, nullptr))) return rc;
    const int info = h->infos[0];
    h->logdet = h->logdets[0];
    h->factored = (info == 0);
    if (info) set_err(h, info, "matrix is not positive definite (see the returned column)");
    return info;
}

// The precision map of Section IV-C and the factorization of Algorithm 1 on one device copy of
// A: a host matrix crosses the link once (into the handle's copy, which the factor then
// references), not once for the map's norms and again for the factor.
int tile_chol_factor_mapped(tc_handle h, int64_t n, int b, const double *A_tiles, double eps_high, int band,
                            int prec_set, uint8_t *map_out, tc_stats *stats) {
    int rc = check_nb(h, n, b);
    if (rc) return rc;
    if (!A_tiles || !map_out) return set_err(h, TC_ERR_ARG, "A_tiles and map_out must not be NULL");
    if (!(eps_high > 0) || band < 0 || prec_set < 1 || prec_set > 4)
        return set_err(h, TC_ERR_ARG, "eps_high > 0, band >= 0 and prec_set in 1..4 are required");
    CK(cudaSetDevice(h->device));
    const double *Ad = A_tiles;
    if (!on_device(A_tiles)) {
        const int nt = (int)((n + b - 1) / b);
        const size_t bytes = (size_t)tidx(nt, 0) * b * b * sizeof(double);
        h->factored = false;                       // the handle's copy of A is replaced
        if ((rc = ensure(h, h->Acopy, bytes))) return rc;
        CK(cudaMemcpyAsync(h->Acopy.p, A_tiles, bytes, cudaMemcpyHostToDevice, h->s));
        Ad = static_cast<const double *>(h->Acopy.p);
    }
    if ((rc = tile_chol_precision_map(h, n, b, Ad, eps_high, band, prec_set, map_out, nullptr))) return rc;
    return tile_chol_factor(h, n, b, Ad, map_out, stats);
}

int tile_chol_logdet(tc_handle h, double *logdet_out) {
    if (!h || !logdet_out) return TC_ERR_ARG;
    if (!h->factored) return set_err(h, TC_ERR_STATE, "no successful factorization");
    *logdet_out = h->logdet;
    return TC_OK;
}

// Forward (and optionally back) substitution with the factor tiles at W (nt tile rows) on
// the padded column-major buffer R (leading dimension ldr = nt*b), nrhs <= 16 per pass.
static int subst_w(tc_handle h, const double *W, int nt, double *R, int64_t ldr, int nrhs, bool back) {
    const int b = h->b;
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

static int subst(tc_handle h, double *R, int64_t ldr, int nrhs, bool back) {
    if (h->ooc) return ooc_subst(h, R, ldr, nrhs, back, nullptr);
    return subst_w(h, static_cast<const double *>(h->W.p), h->nt, R, ldr, nrhs, back);
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

int tile_chol_loglik_refined(tc_handle h, const double *y, int max_refine, double target_berr, double *loglik_out,
                             double *berr_out) {
    if (!h || !y || !loglik_out) return TC_ERR_ARG;
    if (!h->factored) return set_err(h, TC_ERR_STATE, "no successful factorization");
    CK(cudaSetDevice(h->device));
    const int64_t n = h->n;
    DevBuf xy;
    int rc = ensure(h, xy, (size_t)2 * n * sizeof(double));
    if (rc) return rc;
    double *x = static_cast<double *>(xy.p), *yd = x + n;
    CK(cudaMemcpyAsync(yd, y, n * sizeof(double), cudaMemcpyDefault, h->s));
    tc_stats st;
    if ((rc = tile_chol_solve(h, 1, yd, n, x, n, max_refine, target_berr, &st))) {
        release(xy);
        return rc;
    }
    double *sc = static_cast<double *>(h->scratch.p);
    launch_dot(yd, x, n, sc, h->s);
    CK_LAUNCH();
    double quad = 0.0;
    CK(cudaMemcpyAsync(&quad, sc, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    release(xy);
    const double two_pi = 6.283185307179586476925286766559;
    *loglik_out = -0.5 * (double)n * std::log(two_pi) - 0.5 * h->logdet - 0.5 * quad;
    if (berr_out) *berr_out = st.berr;
    return TC_OK;
}

int tile_chol_loglik_solved(tc_handle h, const double *y, const double *x, double *loglik_out) {
    if (!h || !y || !x || !loglik_out) return TC_ERR_ARG;
    if (!h->factored) return set_err(h, TC_ERR_STATE, "no successful factorization");
    CK(cudaSetDevice(h->device));
    const int64_t n = h->n;
    const double *yd = y, *xd = x;
    DevBuf tmp;
    if (!on_device(y) || !on_device(x)) {
        const int rc = ensure(h, tmp, (size_t)2 * n * sizeof(double));
        if (rc) return rc;
        double *t = static_cast<double *>(tmp.p);
        if (!on_device(y)) {
            CK(cudaMemcpyAsync(t, y, n * sizeof(double), cudaMemcpyDefault, h->s));
            yd = t;
        }
        if (!on_device(x)) {
            CK(cudaMemcpyAsync(t + n, x, n * sizeof(double), cudaMemcpyDefault, h->s));
            xd = t + n;
        }
    }
    double *sc = static_cast<double *>(h->scratch.p);
    launch_dot(yd, xd, n, sc, h->s);
    CK_LAUNCH();
    double quad = 0.0;
    CK(cudaMemcpyAsync(&quad, sc, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    release(tmp);
    const double two_pi = 6.283185307179586476925286766559;
    *loglik_out = -0.5 * (double)n * std::log(two_pi) - 0.5 * h->logdet - 0.5 * quad;
    return TC_OK;
}

static int copy_factor(tc_handle h, const double *src, int64_t n, int nt, double *L_tiles);

int tile_chol_get_factor(tc_handle h, double *L_tiles) {
    if (!h || !L_tiles) return TC_ERR_ARG;
    if (!h->factored) return set_err(h, TC_ERR_STATE, "no successful factorization");
    CK(cudaSetDevice(h->device));
    return copy_factor(h, h->ooc ? h->host_factor : static_cast<const double *>(h->W.p), h->n, h->nt, L_tiles);
}

int tile_chol_get_factor_batched(tc_handle h, int index, double *L_tiles) {
    if (!h || !L_tiles) return TC_ERR_ARG;
    if (!h->factored || h->ooc) return set_err(h, TC_ERR_STATE, "no successful in-core factorization");
    if (index < 0 || index >= (int)h->mats.size()) return set_err(h, TC_ERR_ARG, "index outside the last batch");
    CK(cudaSetDevice(h->device));
    const MatDesc &M = h->mats[index];
    return copy_factor(h, static_cast<const double *>(h->W.p) + M.tile0 * (int64_t)h->b * h->b, M.n, M.nt, L_tiles);
}

// The factor tiles at src (device, or the out-of-core host factor) into L_tiles (host or
// device), with upper triangles of diagonal tiles and padding written as 0.
static int copy_factor(tc_handle h, const double *src, int64_t n, int nt, double *L_tiles) {
    const int b = h->b;
    const size_t bytes = (size_t)nt * (nt + 1) / 2 * b * b * sizeof(double);
    double *dst = L_tiles;
    DevBuf tmp;
    const bool dev = on_device(L_tiles);
    if (!dev) {
        int rc = ensure(h, tmp, bytes);
        if (rc) return rc;
        dst = static_cast<double *>(tmp.p);
    }
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->s));
    launch_zero_upper_diag(dst, nt, b, n, h->s);
    CK_LAUNCH();
    if (!dev) CK(cudaMemcpyAsync(L_tiles, dst, bytes, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    release(tmp);
    return TC_OK;
}

// ----------------------------------------------------------------------- batched
int tile_chol_factor_batched(tc_handle h, int count, const int64_t *n, int b, const double *const *A_tiles,
                             const uint8_t *const *maps, int *info_out, double *logdet_out, tc_stats *stats) {
    if (!h) return TC_ERR_ARG;
    if (count < 1 || !n || !A_tiles) return set_err(h, TC_ERR_ARG, "count >= 1, n and A_tiles are required");
    for (int i = 0; i < count; ++i) {
        int rc = check_nb(h, n[i], b);
        if (rc) return rc;
        if (!A_tiles[i]) return set_err(h, TC_ERR_ARG, "A_tiles entries must not be NULL");
    }
    CK(cudaSetDevice(h->device));
    h->factored = false;
    h->ooc = false;
    const int64_t bb = (int64_t)b * b;
    std::vector<MatDesc> mats(count);
    int64_t T = 0, Thost = 0;
    for (int i = 0; i < count; ++i) {
        MatDesc &M = mats[i];
        M.n = n[i];
        M.nt = (int)((n[i] + b - 1) / b);
        M.tile0 = T;
        T += tidx(M.nt, 0);
        M.map.assign((size_t)M.nt * M.nt, TC_FP64);
        if (maps && maps[i]) {
            if (on_device(maps[i])) CK(cudaMemcpy(M.map.data(), maps[i], M.map.size(), cudaMemcpyDeviceToHost));
            else memcpy(M.map.data(), maps[i], M.map.size());
            for (int r = 0; r < M.nt; ++r)
                for (int c = 0; c < M.nt; ++c) {
                    uint8_t &v = M.map[(size_t)r * M.nt + c];
                    if (c >= r) v = TC_FP64;
                    if (v > TC_FP8) return set_err(h, TC_ERR_ARG, "precision map entries must be 0..3");
                }
        }
        for (uint8_t v : M.map) M.mixed |= (v != TC_FP64);
        if (M.mixed && b % 128) return set_err(h, TC_ERR_UNSUPPORTED, "mixed precision needs a tile size that is a multiple of 128");
        if (!on_device(A_tiles[i])) Thost += tidx(M.nt, 0);
    }
    int rc = ensure(h, h->W, (size_t)T * bb * sizeof(double));
    if (rc) return rc;
    // inputs in host memory are staged on the device (outside the captured graph)
    if (Thost && (rc = ensure(h, h->bstage, (size_t)Thost * bb * sizeof(double)))) return rc;
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
        const size_t bytes = (size_t)tidx(mats[i].nt, 0) * bb * sizeof(double);
        if (on_device(A_tiles[i])) {
            mats[i].A_dev = A_tiles[i];
        } else {
            double *dst = static_cast<double *>(h->bstage.p) + off * bb;
            CK(cudaMemcpyAsync(dst, A_tiles[i], bytes, cudaMemcpyHostToDevice, h->s));
            mats[i].A_dev = dst;
            off += tidx(mats[i].nt, 0);
        }
    }
    // graph key: everything the captured launch sequence depends on
    std::vector<int64_t> key = {count, b, (int64_t)(uintptr_t)h->W.p, (int64_t)(uintptr_t)h->status.p};
    uint64_t mh = 1469598103934665603ull;
    for (int i = 0; i < count; ++i) {
        key.push_back(n[i]);
        key.push_back((int64_t)(uintptr_t)mats[i].A_dev);
        for (uint8_t v : mats[i].map) mh = (mh ^ v) * 1099511628211ull;
    }
    key.push_back((int64_t)mh);
    h->mats = std::move(mats);
    h->b = b;
    h->n = h->mats[0].n;
    h->nt = h->mats[0].nt;
    h->map = h->mats[0].map;
    h->mixed = h->mats[0].mixed;
    h->A_dev = h->mats[0].A_dev;
    h->normA_inf = -1.0;
    h->normA_infs.assign(count, -1.0);
    if ((rc = factor_matrices(h, stats, true, &key))) return rc;
    int first_bad = 0;
    for (int i = 0; i < count; ++i) {
        if (info_out) info_out[i] = h->infos[i];
        if (logdet_out) logdet_out[i] = h->logdets[i];
        if (!first_bad && h->infos[i]) first_bad = i + 1;
    }
    h->logdet = h->logdets[0];
    h->factored = (first_bad == 0);
    if (first_bad) {
        char buf[128];
        snprintf(buf, sizeof buf, "matrix %d of the batch is not positive definite (see info_out)", first_bad - 1);
        set_err(h, TC_ERR_ARG, buf);
        return h->infos[first_bad - 1];
    }
    return TC_OK;
}

// Grouped substitution plan over every matrix of the last batched factorization: per tile
// column step one launch for all diagonal blocks and one for all off-diagonal updates.
struct BatchSolvePlan {
    std::vector<int64_t> off;            // RHS block of matrix i in a buffer (elements)
    int64_t total = 0;
    std::vector<SDiag> diag;             // forward steps, then backward steps
    std::vector<SUpd> upd;
    std::vector<std::pair<int, int>> fd, fu, bd, bu;   // (first, count) per step
    std::vector<SRes> res;
    std::vector<SMax> mx;
};

static BatchSolvePlan plan_batch_solve(tc_handle h, int nrhs) {
    BatchSolvePlan S;
    const int count = (int)h->mats.size(), b = h->b;
    const int64_t bb = (int64_t)b * b;
    const double *W = static_cast<const double *>(h->W.p);
    S.off.assign(count + 1, 0);
    int ntmax = 0;
    for (int i = 0; i < count; ++i) {
        S.off[i + 1] = S.off[i] + (int64_t)h->mats[i].nt * b * nrhs;
        ntmax = std::max(ntmax, h->mats[i].nt);
    }
    S.total = S.off[count];
    auto tile = [&](const MatDesc &M, int r, int c) { return W + (M.tile0 + tidx(r, c)) * bb; };
    for (int j = 0; j < ntmax; ++j) {
        const int d0 = (int)S.diag.size(), u0 = (int)S.upd.size();
        for (int i = 0; i < count; ++i) {
            const MatDesc &M = h->mats[i];
            if (M.nt <= j) continue;
            const int64_t ldr = (int64_t)M.nt * b;
            S.diag.push_back({tile(M, j, j), S.off[i] + (int64_t)j * b, ldr});
            for (int r = j + 1; r < M.nt; ++r)
                for (int r0 = 0; r0 < b; r0 += 64)
                    S.upd.push_back({tile(M, r, j), S.off[i] + (int64_t)j * b, S.off[i] + (int64_t)r * b + r0, ldr, r0});
        }
        S.fd.push_back({d0, (int)S.diag.size() - d0});
        S.fu.push_back({u0, (int)S.upd.size() - u0});
    }
    for (int j = ntmax - 1; j >= 0; --j) {
        const int d0 = (int)S.diag.size(), u0 = (int)S.upd.size();
        for (int i = 0; i < count; ++i) {
            const MatDesc &M = h->mats[i];
            if (M.nt <= j) continue;
            const int64_t ldr = (int64_t)M.nt * b;
            S.diag.push_back({tile(M, j, j), S.off[i] + (int64_t)j * b, ldr});
            for (int r = 0; r < j; ++r)
                for (int r0 = 0; r0 < b; r0 += 64)
                    S.upd.push_back({tile(M, j, r), S.off[i] + (int64_t)j * b, S.off[i] + (int64_t)r * b + r0, ldr, r0});
        }
        S.bd.push_back({d0, (int)S.diag.size() - d0});
        S.bu.push_back({u0, (int)S.upd.size() - u0});
    }
    for (int i = 0; i < count; ++i) {
        const MatDesc &M = h->mats[i];
        const int64_t ldr = (int64_t)M.nt * b;
        for (int r = 0; r < M.nt; ++r)
            for (int r0 = 0; r0 < b; r0 += 64)
                S.res.push_back({M.A_dev, M.n, M.nt, r, r0, S.off[i], S.off[i], S.off[i], ldr});
        S.mx.push_back({S.off[i], ldr, M.n, i * nrhs});
    }
    return S;
}

struct BatchSolveDev {
    const SDiag *diag;
    const SUpd *upd;
    const SRes *res;
    const SMax *mx;
};

static int upload_batch_solve(tc_handle h, const BatchSolvePlan &S, BatchSolveDev &D) {
    const size_t od = 0, ou = align_up(S.diag.size() * sizeof(SDiag)), orr = align_up(ou + S.upd.size() * sizeof(SUpd));
    const size_t om = align_up(orr + S.res.size() * sizeof(SRes)), total = align_up(om + S.mx.size() * sizeof(SMax));
    int rc = ensure(h, h->stab, total);
    if (rc) return rc;
    std::vector<char> host(total, 0);
    if (!S.diag.empty()) memcpy(host.data() + od, S.diag.data(), S.diag.size() * sizeof(SDiag));
    if (!S.upd.empty()) memcpy(host.data() + ou, S.upd.data(), S.upd.size() * sizeof(SUpd));
    if (!S.res.empty()) memcpy(host.data() + orr, S.res.data(), S.res.size() * sizeof(SRes));
    if (!S.mx.empty()) memcpy(host.data() + om, S.mx.data(), S.mx.size() * sizeof(SMax));
    CK(cudaMemcpy(h->stab.p, host.data(), total, cudaMemcpyHostToDevice));
    char *base = static_cast<char *>(h->stab.p);
    D.diag = reinterpret_cast<const SDiag *>(base + od);
    D.upd = reinterpret_cast<const SUpd *>(base + ou);
    D.res = reinterpret_cast<const SRes *>(base + orr);
    D.mx = reinterpret_cast<const SMax *>(base + om);
    return TC_OK;
}

// The same sweeps in FP32 (Rf: FP32 vectors of the RHS layout): the correction solves of a
// refined solve, whose FP64 residuals carry the accuracy.
static int batch_subst_f32(tc_handle h, const BatchSolvePlan &S, const BatchSolveDev &D, float *R, int nrhs) {
    const int b = h->b;
    for (size_t j = 0; j < S.fd.size(); ++j) {
        launch_fwd_diag_gf(D.diag + S.fd[j].first, S.fd[j].second, R, b, nrhs, h->s);
        CK_LAUNCH();
        if (S.fu[j].second) {
            launch_fwd_update_gf(D.upd + S.fu[j].first, S.fu[j].second, R, b, nrhs, h->s);
            CK_LAUNCH();
        }
    }
    for (size_t j = 0; j < S.bd.size(); ++j) {
        launch_bwd_diag_gf(D.diag + S.bd[j].first, S.bd[j].second, R, b, nrhs, h->s);
        CK_LAUNCH();
        if (S.bu[j].second) {
            launch_bwd_update_gf(D.upd + S.bu[j].first, S.bu[j].second, R, b, nrhs, h->s);
            CK_LAUNCH();
        }
    }
    return TC_OK;
}

static int batch_subst(tc_handle h, const BatchSolvePlan &S, const BatchSolveDev &D, double *R, int nrhs, bool back) {
    const int b = h->b;
    for (size_t j = 0; j < S.fd.size(); ++j) {
        launch_fwd_diag_g(D.diag + S.fd[j].first, S.fd[j].second, R, b, nrhs, h->s);
        CK_LAUNCH();
        if (S.fu[j].second) {
            launch_fwd_update_g(D.upd + S.fu[j].first, S.fu[j].second, R, b, nrhs, h->s);
            CK_LAUNCH();
        }
    }
    if (!back) return TC_OK;
    for (size_t j = 0; j < S.bd.size(); ++j) {
        launch_bwd_diag_g(D.diag + S.bd[j].first, S.bd[j].second, R, b, nrhs, h->s);
        CK_LAUNCH();
        if (S.bu[j].second) {
            launch_bwd_update_g(D.upd + S.bu[j].first, S.bu[j].second, R, b, nrhs, h->s);
            CK_LAUNCH();
        }
    }
    return TC_OK;
}

int tile_chol_solve_batched(tc_handle h, int nrhs, const double *const *B, double *const *X, int max_refine,
                            double target_berr, double *berr_out, tc_stats *stats) {
    if (!h) return TC_ERR_ARG;
    if (!h->factored || h->ooc) return set_err(h, TC_ERR_STATE, "no successful in-core factorization");
    if (nrhs < 1 || nrhs > 16 || !B || !X || max_refine < 0)
        return set_err(h, TC_ERR_ARG, "bad batched solve arguments (1 <= nrhs <= 16)");
    CK(cudaSetDevice(h->device));
    const double t0 = now_ms();
    const int64_t launches0 = h->launches;
    const int count = (int)h->mats.size(), b = h->b;
    BatchSolvePlan S = plan_batch_solve(h, nrhs);
    BatchSolveDev D{};
    int rc = upload_batch_solve(h, S, D);
    if (rc) return rc;
    // refined solves run their substitutions in FP32 (Rf) and their residuals in FP64
    const bool f32 = max_refine > 0;
    if ((rc = ensure(h, h->vec, (size_t)3 * S.total * sizeof(double) + (f32 ? (size_t)S.total * sizeof(float) : 0))))
        return rc;
    if ((rc = ensure(h, h->scratch, std::max<size_t>(4096, (size_t)(3 * nrhs + 1) * count) * sizeof(double)))) return rc;
    double *Bd = static_cast<double *>(h->vec.p), *Xd = Bd + S.total, *Rd = Xd + S.total;
    float *Rf = reinterpret_cast<float *>(Rd + S.total);
    double *sc = static_cast<double *>(h->scratch.p);
    CK(cudaMemsetAsync(Bd, 0, S.total * sizeof(double), h->s));
    for (int i = 0; i < count; ++i) {
        const MatDesc &M = h->mats[i];
        CK(cudaMemcpy2DAsync(Bd + S.off[i], (size_t)M.nt * b * sizeof(double), B[i], M.n * sizeof(double),
                             M.n * sizeof(double), nrhs, cudaMemcpyDefault, h->s));
    }
    if (f32) {
        launch_to_f32(Bd, Rf, S.total, h->s);
        CK_LAUNCH();
        if ((rc = batch_subst_f32(h, S, D, Rf, nrhs))) return rc;
        launch_add_f32(Xd, Rf, S.total, 1, h->s);
        CK_LAUNCH();
    } else {
        CK(cudaMemcpyAsync(Xd, Bd, S.total * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
        if ((rc = batch_subst(h, S, D, Xd, nrhs, true))) return rc;
    }
    // ||A_i||_inf once per factorization: max row sum of |A_i| (X = nullptr reads ones)
    if (max_refine > 0 && h->normA_infs[0] < 0) {
        CK(cudaMemsetAsync(sc, 0, (size_t)count * nrhs * sizeof(double), h->s));
        launch_symv_g(D.res, (int)S.res.size(), b, nullptr, nullptr, Rd, 1, 1, h->s);
        CK_LAUNCH();
        launch_colmax_g(D.mx, count, Rd, 1, sc, h->s);
        CK_LAUNCH();
        std::vector<double> nm((size_t)count * nrhs);
        CK(cudaMemcpyAsync(nm.data(), sc, nm.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        for (int i = 0; i < count; ++i) h->normA_infs[i] = nm[(size_t)i * nrhs];
    }
    std::vector<double> berr(count, -1.0);
    int it = 0;
    for (; max_refine > 0; ++it) {
        launch_symv_g(D.res, (int)S.res.size(), b, Xd, Bd, Rd, nrhs, 0, h->s);
        CK_LAUNCH();
        CK(cudaMemsetAsync(sc, 0, (size_t)3 * nrhs * count * sizeof(double), h->s));
        launch_colmax_g(D.mx, count, Rd, nrhs, sc, h->s);
        CK_LAUNCH();
        launch_colmax_g(D.mx, count, Xd, nrhs, sc + (size_t)nrhs * count, h->s);
        CK_LAUNCH();
        launch_colmax_g(D.mx, count, Bd, nrhs, sc + (size_t)2 * nrhs * count, h->s);
        CK_LAUNCH();
        std::vector<double> mx((size_t)3 * nrhs * count);
        CK(cudaMemcpyAsync(mx.data(), sc, mx.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        double worst = 0.0;
        for (int i = 0; i < count; ++i) {
            double e = 0.0;
            for (int c = 0; c < nrhs; ++c) {
                const size_t k0 = (size_t)i * nrhs + c;
                const double den = h->normA_infs[i] * mx[(size_t)nrhs * count + k0] + mx[(size_t)2 * nrhs * count + k0];
                e = std::max(e, den > 0 ? mx[k0] / den : 0.0);
            }
            berr[i] = e;
            worst = std::max(worst, e);
        }
        if (worst <= target_berr || it >= max_refine) break;
        // one refinement step for every matrix (already-accurate ones stay accurate)
        launch_to_f32(Rd, Rf, S.total, h->s);
        CK_LAUNCH();
        if ((rc = batch_subst_f32(h, S, D, Rf, nrhs))) return rc;
        launch_add_f32(Xd, Rf, S.total, 0, h->s);
        CK_LAUNCH();
    }
    for (int i = 0; i < count; ++i) {
        const MatDesc &M = h->mats[i];
        CK(cudaMemcpy2DAsync(X[i], M.n * sizeof(double), Xd + S.off[i], (size_t)M.nt * b * sizeof(double),
                             M.n * sizeof(double), nrhs, cudaMemcpyDefault, h->s));
    }
    CK(cudaStreamSynchronize(h->s));
    double worst = 0.0;
    for (int i = 0; i < count; ++i) {
        if (berr_out) berr_out[i] = berr[i];
        worst = std::max(worst, berr[i]);
    }
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->t_ms = now_ms() - t0;
        stats->refine_iters = it;
        stats->berr = max_refine > 0 ? worst : -1.0;
        stats->kernel_launches = h->launches - launches0;
    }
    return TC_OK;
}

int tile_chol_loglik_batched(tc_handle h, const double *const *y, double *loglik_out) {
    if (!h || !loglik_out) return TC_ERR_ARG;
    if (!h->factored || h->ooc) return set_err(h, TC_ERR_STATE, "no successful in-core factorization");
    CK(cudaSetDevice(h->device));
    const int count = (int)h->mats.size(), b = h->b;
    std::vector<double> quad(count, 0.0);
    if (y) {
        BatchSolvePlan S = plan_batch_solve(h, 1);
        BatchSolveDev D{};
        int rc = upload_batch_solve(h, S, D);
        if (rc) return rc;
        if ((rc = ensure(h, h->vec, (size_t)S.total * sizeof(double)))) return rc;
        if ((rc = ensure(h, h->scratch, std::max<size_t>(4096, (size_t)count) * sizeof(double)))) return rc;
        double *z = static_cast<double *>(h->vec.p), *sc = static_cast<double *>(h->scratch.p);
        CK(cudaMemsetAsync(z, 0, S.total * sizeof(double), h->s));
        for (int i = 0; i < count; ++i) {
            if (!y[i]) return set_err(h, TC_ERR_ARG, "y entries must not be NULL");
            CK(cudaMemcpyAsync(z + S.off[i], y[i], h->mats[i].n * sizeof(double), cudaMemcpyDefault, h->s));
        }
        if ((rc = batch_subst(h, S, D, z, 1, false))) return rc;
        launch_dots_g(D.mx, count, z, z, sc, h->s);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(quad.data(), sc, count * sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
    }
    const double two_pi = 6.283185307179586476925286766559;
    (void)b;
    for (int i = 0; i < count; ++i)
        loglik_out[i] = -0.5 * (double)h->mats[i].n * std::log(two_pi) - 0.5 * h->logdets[i] - 0.5 * quad[i];
    return TC_OK;
}

}  // extern "C"
