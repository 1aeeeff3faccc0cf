// supernodal.cpp -- host plan of the non-uniform supernodal tiling (Sec. 5.4).
//
// For the patterns the selector sends to the sparse end, the paper replaces the uniform
// n_b grid by dense cells fitted to supernodes.  This file builds that layout from the
// symbolic factor the analysis already holds (same ordering, same elimination tree):
//   * fundamental supernodes: column j+1 continues j's supernode when it is j's etree
//     parent, j is its only child and the column counts nest (c_j = c_{j+1} + 1);
//   * relaxed amalgamation along contiguous child -> parent links (Sec. 5.4 cites the
//     Ashcraft-Grimes heuristic with standard thresholds), merged width capped at the
//     largest device tile (kMaxNb), wider fundamental supernodes cut into panels of
//     kMaxNb columns;
//   * one packed row list per supernode (its own columns, then the rows below) and a
//     dense column-major panel per supernode in one arena;
//   * cells (J, I): the run of supernode I's rows owned by row supernode J (I's diagonal
//     block is the cell (I, I));
//   * the left-looking task list of Sec. 5.4: for each supernode J in order, every
//     UPDATE L_KJ -= L_KI L_JI^T from the supernodes I < J with a cell (J, I), then the
//     FACTOR (POTRF) of J's diagonal cell, then the TRSM of each cell below it.
// Plans analysed for the supernodal route execute this layout on the GPU (replay.cu).
#include <algorithm>
#include <functional>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <vector>

#include "plan.hpp"

using std::int32_t;
using std::int64_t;
using std::vector;

namespace {

// Amalgamation thresholds (Sec. 5.4 names Ashcraft-Grimes relaxation with standard,
// untuned defaults without listing them; these are the defaults common to supernodal
// codes): a merge that keeps the width <= 4 is always taken; up to 16, 48 and beyond,
// it is taken while the explicit zeros stay below 80 %, 10 % and 5 % of the stored
// lower trapezoid.
constexpr int64_t kRelaxW[3] = {4, 16, 48};
constexpr double kRelaxZ[3] = {0.8, 0.1, 0.05};

bool relax_ok(int64_t w, double zfrac) {
    if (w <= kRelaxW[0]) return true;
    if (w <= kRelaxW[1]) return zfrac < kRelaxZ[0];
    if (w <= kRelaxW[2]) return zfrac < kRelaxZ[1];
    return zfrac < kRelaxZ[2];
}

}  // namespace

const stc::SnPlan& stc_plan::supernodal() const {
    std::lock_guard<std::mutex> g(sn_mu);
    if (sn) return *sn;
    auto S = std::make_unique<stc::SnPlan>();
    const int64_t N = n;
    const int64_t W = stc::kMaxNb;
    vector<int64_t> cnt(N), nchild(N, 0);
    for (int64_t j = 0; j < N; ++j) {
        cnt[j] = Lp[j + 1] - Lp[j];
        if (parent[j] >= 0) nchild[parent[j]]++;
    }
    // fundamental supernodes: first columns
    vector<int64_t> fs;
    for (int64_t j = 0; j < N; ++j) {
        const bool cont = j > 0 && parent[j - 1] == j && cnt[j - 1] == cnt[j] + 1 && nchild[j] == 1;
        if (!cont) fs.push_back(j);
    }
    fs.push_back(N);
    // relaxed amalgamation: the current group [gf, gl) absorbs the next fundamental
    // supernode s = [sf, sl) when s holds the etree parent of the group's last column.
    // The merged rows are the group's columns followed by s's rows (the etree paths of
    // the group's columns all pass through s, so their rows below s are s's rows).
    vector<int64_t> rf;
    {
        auto nnz_of = [&](int64_t a, int64_t b) {
            double t = 0;
            for (int64_t j = a; j < b; ++j) t += double(cnt[j]);
            return t;
        };
        int64_t gf = fs[0], gl = fs[1];
        double gnnz = nnz_of(gf, gl);
        for (size_t k = 1; k + 1 < fs.size(); ++k) {
            const int64_t sf = fs[k], sl = fs[k + 1];
            const double snnz = nnz_of(sf, sl);
            const int64_t p = parent[gl - 1];
            bool merge = false;
            if (p >= sf && p < sl && sl - gf <= W) {
                const double w = double(sl - gf);
                const double below = double(cnt[sf] - (sl - sf));
                const double stored = w * (w + 1) / 2 + w * below;
                merge = relax_ok(sl - gf, (stored - gnnz - snnz) / stored);
            }
            if (merge) {
                gl = sl;
                gnnz += snnz;
            } else {
                rf.push_back(gf);
                gf = sf;
                gl = sl;
                gnnz = snnz;
            }
        }
        rf.push_back(gf);
        rf.push_back(N);
    }
    // panels of at most W columns
    for (size_t k = 0; k + 1 < rf.size(); ++k)
        for (int64_t a = rf[k]; a < rf[k + 1]; a += W) S->first.push_back((int32_t)a);
    S->first.push_back((int32_t)N);
    const int32_t nsn = (int32_t)S->first.size() - 1;
    vector<int32_t> snof(N);
    for (int32_t s = 0; s < nsn; ++s)
        for (int64_t j = S->first[s]; j < S->first[s + 1]; ++j) snof[j] = s;
    // row lists and panels: rows of [a, b) are a..b-1, then the structure of column b-1
    // below its diagonal
    S->rptr.assign(nsn + 1, 0);
    S->off.assign(nsn, 0);
    for (int32_t s = 0; s < nsn; ++s) {
        const int64_t a = S->first[s], b = S->first[s + 1], w = b - a;
        for (int64_t j = a; j < b; ++j) S->rows.push_back((int32_t)j);
        for (int64_t q = Lp[b - 1] + 1; q < Lp[b]; ++q) S->rows.push_back(Li[q]);
        S->rptr[s + 1] = (int64_t)S->rows.size();
        const int64_t m = S->rptr[s + 1] - S->rptr[s];
        S->off[s] = S->arena;
        S->arena += (m * w + 3) / 4 * 4;  // 32-byte aligned panels
        double nz = 0;
        for (int64_t j = a; j < b; ++j) nz += double(cnt[j]);
        const int64_t trap = w * (w + 1) / 2 + w * (m - w);
        S->stored += trap;
        S->zeros += trap - (int64_t)nz;
    }
    // cells, by column supernode (rows ascending), and by row supernode
    S->cptr.assign(nsn + 1, 0);
    vector<vector<int32_t>> byrow(nsn);
    for (int32_t s = 0; s < nsn; ++s) {
        const int64_t r0 = S->rptr[s], m = S->rptr[s + 1] - r0;
        const int32_t w = S->first[s + 1] - S->first[s];
        S->cells.insert(S->cells.end(), {s, s, 0, w});
        for (int64_t r = w; r < m;) {
            const int32_t J = snof[S->rows[r0 + r]];
            int64_t e = r + 1;
            while (e < m && snof[S->rows[r0 + e]] == J) ++e;
            byrow[J].push_back((int32_t)(S->cells.size() / 4));
            S->cells.insert(S->cells.end(), {s, J, (int32_t)r, (int32_t)e});
            r = e;
        }
        S->cptr[s + 1] = (int32_t)(S->cells.size() / 4);
    }
    // left-looking task list
    auto cell_of = [&](int32_t I, int32_t J) {  // cell (J, I) of column supernode I
        int32_t lo = S->cptr[I], hi = S->cptr[I + 1];
        while (lo < hi) {
            const int32_t mid = (lo + hi) / 2;
            if (S->cells[4 * mid + 1] < J) lo = mid + 1; else hi = mid;
        }
        return (lo < S->cptr[I + 1] && S->cells[4 * lo + 1] == J) ? lo : -1;
    };
    for (int32_t J = 0; J < nsn; ++J) {
        for (int32_t cJI : byrow[J]) {
            const int32_t I = S->cells[4 * cJI];
            for (int32_t cKI = cJI; cKI < S->cptr[I + 1]; ++cKI) {
                const int32_t K = S->cells[4 * cKI + 1];
                const int32_t cKJ = cell_of(J, K);
                if (cKJ < 0) throw std::logic_error("supernodal update without a target cell");
                S->tasks.insert(S->tasks.end(), {stc::SN_UPDATE, cKJ, cKI, cJI});
            }
        }
        S->tasks.insert(S->tasks.end(), {stc::SN_FACTOR, S->cptr[J], -1, -1});
        for (int32_t c = S->cptr[J] + 1; c < S->cptr[J + 1]; ++c)
            S->tasks.insert(S->tasks.end(), {stc::SN_TRSM, c, -1, -1});
    }
    build_device_form(*S, snof, byrow, cell_of);
    sn = std::move(S);
    return *sn;
}

void stc_plan::build_device_form(stc::SnPlan& S, const vector<int32_t>& snof,
                                 const vector<vector<int32_t>>& byrow,
                                 const std::function<int32_t(int32_t, int32_t)>& cell_of) const {
    const int32_t nsn = (int32_t)S.first.size() - 1;
    const int32_t ncell = (int32_t)(S.cells.size() / 4);
    auto nrows = [&](int32_t s) { return (int32_t)(S.rptr[s + 1] - S.rptr[s]); };
    auto width = [&](int32_t s) { return S.first[s + 1] - S.first[s]; };
    auto cell_rows = [&](int32_t c) {  // global row indices of cell c
        const int32_t I = S.cells[4 * c];
        return S.rows.data() + S.rptr[I] + S.cells[4 * c + 2];
    };
    auto height = [&](int32_t c) { return S.cells[4 * c + 3] - S.cells[4 * c + 2]; };
    S.dcells.resize(ncell);
    for (int32_t c = 0; c < ncell; ++c) {
        const int32_t I = S.cells[4 * c], h = height(c);
        stc::SnDevCell& d = S.dcells[c];
        d.off = S.off[I] + S.cells[4 * c + 2];
        d.ld = nrows(I);
        d.h = h;
        d.w = width(I);
        d.I = I;
        d.J = S.cells[4 * c + 1];
        d.nslices = (I == d.J) ? 1 : (h + stc::kSnSliceH - 1) / stc::kSnSliceH;
    }
    // column map of a source cell (J,I): its rows as columns of J (one per cell)
    vector<int32_t> cmap_of(ncell, -1);
    auto cmap = [&](int32_t c) {
        if (cmap_of[c] < 0) {
            const int32_t J = S.cells[4 * c + 1];
            cmap_of[c] = (int32_t)S.maps.size();
            const int32_t* r = cell_rows(c);
            for (int32_t i = 0; i < height(c); ++i) S.maps.push_back((int16_t)(r[i] - S.first[J]));
        }
        return cmap_of[c];
    };
    for (int32_t J = 0; J < nsn; ++J) {
        const int32_t dJ = S.cptr[J];
        // diagonal cell: every (J,I) SYRK-like update, then POTRF
        stc::SnDevTask t{};
        t.kind = stc::SN_T_DIAG; t.cell = dJ; t.diag = dJ; t.rs0 = 0; t.rs1 = width(J); t.slice = 0;
        t.ubeg = (int32_t)S.dupds.size();
        for (int32_t cJI : byrow[J]) {
            stc::SnDevUpd u{};
            u.a = cJI; u.b = cJI; u.ar0 = 0; u.ar1 = height(cJI);
            u.cmap = cmap(cJI);
            u.rmap = u.cmap;
            u.klen = width(S.cells[4 * cJI]);
            S.dupds.push_back(u);
        }
        t.uend = (int32_t)S.dupds.size();
        S.dtasks.push_back(t);
        // off-diagonal cells (K,J): row slices, GEMM-like updates from every I with cells
        // (K,I) and (J,I), then TRSM
        for (int32_t cKJ = S.cptr[J] + 1; cKJ < S.cptr[J + 1]; ++cKJ) {
            const int32_t K = S.cells[4 * cKJ + 1], h = height(cKJ);
            const int32_t* tr = cell_rows(cKJ);
            // per source I: the cell (K,I), its row map into (K,J), and (J,I)
            struct Src { int32_t cKI, cJI, rmap, klen; };
            vector<Src> srcs;
            for (int32_t cJI : byrow[J]) {
                const int32_t I = S.cells[4 * cJI];
                const int32_t cKI = cell_of(I, K);
                if (cKI < 0) continue;
                Src x{cKI, cJI, (int32_t)S.maps.size(), width(I)};
                const int32_t* r = cell_rows(cKI);
                for (int32_t i = 0, q = 0; i < height(cKI); ++i) {
                    while (q < h && tr[q] < r[i]) ++q;
                    if (q >= h || tr[q] != r[i]) throw std::logic_error("supernodal row map: not a subset");
                    S.maps.push_back((int16_t)q);
                }
                srcs.push_back(x);
            }
            const int32_t nsl = S.dcells[cKJ].nslices;
            for (int32_t sl = 0; sl < nsl; ++sl) {
                stc::SnDevTask o{};
                o.kind = stc::SN_T_OFF; o.cell = cKJ; o.diag = dJ; o.slice = sl;
                o.rs0 = sl * stc::kSnSliceH; o.rs1 = std::min(h, o.rs0 + stc::kSnSliceH);
                o.ubeg = (int32_t)S.dupds.size();
                for (const Src& x : srcs) {
                    const int16_t* m = S.maps.data() + x.rmap;
                    const int32_t hk = height(x.cKI);
                    const int32_t a0 = (int32_t)(std::lower_bound(m, m + hk, (int16_t)o.rs0) - m);
                    const int32_t a1 = (int32_t)(std::lower_bound(m, m + hk, (int16_t)o.rs1) - m);
                    if (a0 >= a1) continue;
                    stc::SnDevUpd u{};
                    u.a = x.cKI; u.b = x.cJI; u.ar0 = a0; u.ar1 = a1;
                    u.rmap = x.rmap; u.cmap = cmap(x.cJI); u.klen = x.klen;
                    S.dupds.push_back(u);
                }
                o.uend = (int32_t)S.dupds.size();
                S.dtasks.push_back(o);
            }
        }
    }
    // per-cell column maps (every off-diagonal cell (J, I) is a source of J's diagonal
    // task, so each has one), the cells owned by each row supernode, and the FMAs the
    // device form executes: updates (lower half on a diagonal target), POTRF, TRSM
    S.cell_cmap = cmap_of;
    S.rptr_cells.assign(nsn + 1, 0);
    for (int32_t J = 0; J < nsn; ++J) {
        S.rptr_cells[J + 1] = S.rptr_cells[J] + (int32_t)byrow[J].size();
        S.row_cells.insert(S.row_cells.end(), byrow[J].begin(), byrow[J].end());
    }
    double fma = 0.0;
    for (const stc::SnDevTask& t : S.dtasks) {
        const double w = S.dcells[t.cell].w;
        for (int32_t u = t.ubeg; u < t.uend; ++u) {
            const stc::SnDevUpd& x = S.dupds[u];
            const double ra = x.ar1 - x.ar0, hb = S.dcells[x.b].h;
            fma += (t.kind == stc::SN_T_DIAG ? ra * (ra + 1) / 2 : ra * hb) * x.klen;
        }
        fma += t.kind == stc::SN_T_DIAG ? w * (w + 1) * (w + 2) / 6 : double(t.rs1 - t.rs0) * w * (w + 1) / 2;
    }
    S.fma_exec = fma;
    // selected inverse tasks: supernodes in reverse order, for each its off-diagonal cells
    // (row slices as in the factorization) with one contribution per cell (K', J) of J,
    // then its diagonal cell with its own cells as contributions
    S.cell_rowoff.resize(ncell);
    for (int32_t c = 0; c < ncell; ++c) S.cell_rowoff[c] = (int32_t)(S.rptr[S.cells[4 * c]] + S.cells[4 * c + 2]);
    for (int32_t J = nsn - 1; J >= 0; --J) {
        const int32_t c0 = S.cptr[J], c1 = S.cptr[J + 1];
        for (int32_t T = c0 + 1; T < c1; ++T) {
            const int32_t K = S.cells[4 * T + 1];
            for (int32_t sl = 0; sl < S.dcells[T].nslices; ++sl) {
                stc::SnSTask t{};
                t.kind = stc::SN_S_OFF; t.cell = T; t.diag = c0;
                t.rs0 = sl * stc::kSnSliceH; t.rs1 = std::min(height(T), t.rs0 + stc::kSnSliceH);
                t.cbeg = (int32_t)S.scons.size();
                for (int32_t c2 = c0 + 1; c2 < c1; ++c2) {
                    const int32_t K2 = S.cells[4 * c2 + 1];
                    stc::SnSCon q{};
                    q.lcell = c2;
                    if (K2 == K) { q.mode = stc::SN_SC_SAME; q.scell = S.cptr[K]; }
                    else if (K2 < K) { q.mode = stc::SN_SC_LOWER; q.scell = cell_of(K2, K); }
                    else { q.mode = stc::SN_SC_UPPER; q.scell = cell_of(K, K2); }
                    if (q.scell < 0) throw std::logic_error("selected inverse: source cell missing");
                    S.scons.push_back(q);
                }
                t.cend = (int32_t)S.scons.size();
                S.stasks.push_back(t);
            }
        }
        stc::SnSTask d{};
        d.kind = stc::SN_S_DIAG; d.cell = c0; d.diag = c0; d.rs0 = 0; d.rs1 = width(J);
        d.cbeg = (int32_t)S.scons.size();
        for (int32_t c2 = c0 + 1; c2 < c1; ++c2) {
            stc::SnSCon q{};
            q.lcell = c2; q.scell = c2; q.mode = stc::SN_SC_OWN;
            S.scons.push_back(q);
        }
        d.cend = (int32_t)S.scons.size();
        S.stasks.push_back(d);
    }
    // value and CSC maps into the arena
    vector<int64_t> iperm(n);
    for (int64_t k = 0; k < n; ++k) iperm[perm[k]] = k;
    auto arena_off = [&](int64_t r, int64_t c) -> int64_t {  // r >= c, permuted
        const int32_t s = snof[c];
        const int32_t* b = S.rows.data() + S.rptr[s];
        const int32_t* e = S.rows.data() + S.rptr[s + 1];
        const int32_t* x = std::lower_bound(b, e, (int32_t)r);
        if (x == e || *x != r) throw std::logic_error("entry outside the supernodal panels");
        return S.off[s] + (x - b) + (c - S.first[s]) * (int64_t)(e - b);
    };
    S.value_map.resize(nnzA);
    for (int64_t p = 0; p < nnzA; ++p) {
        const int64_t a = iperm[arow[p]], b = iperm[acol[p]];
        S.value_map[p] = arena_off(std::max(a, b), std::min(a, b));
    }
    // a column's structure is an ascending subset of its supernode's rows: one merge walk
    S.csc_map.resize(Lp[n]);
    for (int32_t s = 0; s < nsn; ++s) {
        const int32_t* R = S.rows.data() + S.rptr[s];
        const int64_t m = nrows(s);
        for (int64_t j = S.first[s]; j < S.first[s + 1]; ++j) {
            int64_t x = 0;
            for (int64_t q = Lp[j]; q < Lp[j + 1]; ++q) {
                while (x < m && R[x] < Li[q]) ++x;
                if (x >= m || R[x] != Li[q]) throw std::logic_error("entry outside the supernodal panels");
                S.csc_map[q] = S.off[s] + x + (j - S.first[s]) * m;
            }
        }
    }
}
