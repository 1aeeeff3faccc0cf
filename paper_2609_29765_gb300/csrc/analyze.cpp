// analyze.cpp -- host-side symbolic analysis (once per sparsity pattern).
//
// Follows arxiv 2609.29765:
//   Sec. 3     ordering (geometric nested dissection / RCM / natural / given) and the
//              symbolic Cholesky factorization of the permuted pattern;
//   Sec. 4     uniform n_b tile grid over L, active-column sets aind, contiguous and
//              full-width predicates, banded half-width kd_t of diagonal tiles;
//   Sec. 5.1   routing features phi, rho, sigma and the selector;
//   Sec. 5.2   per-tile metadata pass, Algorithm 1 task list, per-task scatter maps;
//   Sec. 5.3   the task DAG the device executor replays (counters instead of P).
//
// The elimination tree uses Liu's ancestor algorithm with path compression and the
// structure of L is built row by row from row subtrees (Liu 1990 / Gilbert-Ng-Peyton
// 1994, the pipeline cited in Sec. 5.4).
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <numeric>
#include <limits>
#include <thread>

#include "plan.hpp"

using std::int16_t;
using std::int32_t;
using std::int64_t;
using std::vector;

namespace {

constexpr int kMaxNb = 128;

// Runs f(chunk, worker) for every chunk in [0, nchunks) on up to `threads` threads
// (worker in [0, threads)); chunks are handed out in increasing order.  Every caller
// writes each output element from exactly one chunk, so results do not depend on the
// thread count (nor on how many threads could be started).  An exception in a worker is
// rethrown here after all workers joined.
template <class F>
void parallel_chunks(int threads, int64_t nchunks, F&& f) {
    const int nt = int(std::max<int64_t>(1, std::min<int64_t>(threads, nchunks)));
    if (nt == 1) {
        for (int64_t c = 0; c < nchunks; ++c) f(c, 0);
        return;
    }
    std::atomic<int64_t> next{0};
    std::atomic<bool> failed{false};
    std::exception_ptr err;
    std::mutex emu;
    auto work = [&](int w) {
        try {
            for (int64_t c; !failed.load(std::memory_order_relaxed) && (c = next.fetch_add(1)) < nchunks;)
                f(c, w);
        } catch (...) {
            std::lock_guard<std::mutex> g(emu);
            if (!err) err = std::current_exception();
            failed = true;
        }
    };
    vector<std::thread> pool;
    try {
        pool.reserve(nt - 1);
        for (int w = 1; w < nt; ++w) pool.emplace_back(work, w);
    } catch (...) {
        // no more threads to be had: the ones started and this thread share the chunks
    }
    work(0);
    for (auto& th : pool) th.join();
    if (err) std::rethrow_exception(err);
}

int validate_pattern(int64_t n, const int64_t* Ap, const int64_t* Ai) {
    if (n <= 0 || !Ap || !Ai) return STC_ERR_INVALID_ARG;
    if (n > INT32_MAX - 1) return STC_ERR_UNSUPPORTED;
    if (Ap[0] != 0) return STC_ERR_INVALID_PATTERN;
    for (int64_t j = 0; j < n; ++j) {
        if (Ap[j + 1] < Ap[j]) return STC_ERR_INVALID_PATTERN;
        if (Ap[j + 1] == Ap[j] || Ai[Ap[j]] != j) return STC_ERR_INVALID_PATTERN;  // diagonal first
        for (int64_t p = Ap[j] + 1; p < Ap[j + 1]; ++p)
            if (Ai[p] <= Ai[p - 1] || Ai[p] >= n) return STC_ERR_INVALID_PATTERN;
    }
    return STC_OK;
}

// ---------------------------------------------------------------------------
// Geometric nested dissection on integral lattice coordinates.  A box holding at
// most `leaf` nodes is emitted whole; otherwise its longest axis (extent hi-lo+1,
// ties -> lowest axis) is cut by the plane floor((lo+hi)/2): the two half-boxes are
// ordered first (lower half, then upper half), the plane's nodes last.  Leaves and
// planes are emitted in x-fastest lexicographic order.  Rows with a NaN coordinate
// (set-aside dense rows) follow at the end in input order.
// ---------------------------------------------------------------------------
struct Lattice {
    vector<int64_t> x, y, z;
    int64_t c(int64_t v, int a) const { return a == 0 ? x[v] : (a == 1 ? y[v] : z[v]); }
    bool lex_less(int64_t u, int64_t v) const {
        if (z[u] != z[v]) return z[u] < z[v];
        if (y[u] != y[v]) return y[u] < y[v];
        return x[u] < x[v];
    }
};

void nd_split(const Lattice& g, int64_t* first, int64_t* last, std::array<int64_t, 3> lo,
              std::array<int64_t, 3> hi, int64_t leaf, vector<int64_t>& out) {
    const int64_t cnt = last - first;
    if (cnt == 0) return;
    auto lex = [&](int64_t u, int64_t v) { return g.lex_less(u, v); };
    if (cnt <= leaf) {
        std::sort(first, last, lex);
        out.insert(out.end(), first, last);
        return;
    }
    int ax = 0;
    for (int a = 1; a < 3; ++a)
        if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
    const int64_t s = lo[ax] + hi[ax];
    const int64_t mid = s >= 0 ? s / 2 : -((-s + 1) / 2);
    int64_t* m1 = std::partition(first, last, [&](int64_t v) { return g.c(v, ax) < mid; });
    int64_t* m2 = std::partition(m1, last, [&](int64_t v) { return g.c(v, ax) == mid; });
    // [first,m1) lower half, [m1,m2) plane, [m2,last) upper half
    auto lhi = hi; lhi[ax] = mid - 1;
    auto rlo = lo; rlo[ax] = mid + 1;
    nd_split(g, first, m1, lo, lhi, leaf, out);
    nd_split(g, m2, last, rlo, hi, leaf, out);
    std::sort(m1, m2, lex);
    out.insert(out.end(), m1, m2);
}

int order_nd(int64_t n, const double* coords, int64_t leaf, vector<int64_t>& perm) {
    if (!coords) return STC_ERR_INVALID_ARG;
    Lattice g;
    g.x.assign(n, 0); g.y.assign(n, 0); g.z.assign(n, 0);
    vector<int64_t> nodes, aside;
    std::array<int64_t, 3> lo{0, 0, 0}, hi{-1, -1, -1};
    for (int64_t i = 0; i < n; ++i) {
        const double* c = coords + 3 * i;
        if (std::isnan(c[0]) || std::isnan(c[1]) || std::isnan(c[2])) { aside.push_back(i); continue; }
        int64_t v[3];
        for (int a = 0; a < 3; ++a) {
            if (std::floor(c[a]) != c[a] || std::fabs(c[a]) > 1e15) return STC_ERR_UNSUPPORTED;
            v[a] = (int64_t)c[a];
        }
        g.x[i] = v[0]; g.y[i] = v[1]; g.z[i] = v[2];
        for (int a = 0; a < 3; ++a) {
            if (nodes.empty() || v[a] < lo[a]) lo[a] = v[a];
            if (nodes.empty() || v[a] > hi[a]) hi[a] = v[a];
        }
        nodes.push_back(i);
    }
    perm.clear();
    perm.reserve(n);
    nd_split(g, nodes.data(), nodes.data() + nodes.size(), lo, hi, leaf, perm);
    perm.insert(perm.end(), aside.begin(), aside.end());
    return (int64_t)perm.size() == n ? STC_OK : STC_ERR_INVALID_PATTERN;
}

// Full symmetric adjacency (no diagonal) of a lower CSC pattern.
void adjacency(int64_t n, const int64_t* Ap, const int64_t* Ai, vector<int64_t>& xadj,
               vector<int64_t>& adj) {
    xadj.assign(n + 1, 0);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t p = Ap[j] + 1; p < Ap[j + 1]; ++p) { xadj[j + 1]++; xadj[Ai[p] + 1]++; }
    for (int64_t j = 0; j < n; ++j) xadj[j + 1] += xadj[j];
    adj.assign(xadj[n], 0);
    vector<int64_t> f(xadj.begin(), xadj.end() - 1);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t p = Ap[j] + 1; p < Ap[j + 1]; ++p) { adj[f[j]++] = Ai[p]; adj[f[Ai[p]]++] = j; }
}

// Reverse Cuthill-McKee with a George-Liu pseudo-peripheral start per component.
void order_rcm(int64_t n, const int64_t* Ap, const int64_t* Ai, vector<int64_t>& perm) {
    vector<int64_t> xadj, adj;
    adjacency(n, Ap, Ai, xadj, adj);
    auto deg = [&](int64_t v) { return xadj[v + 1] - xadj[v]; };
    vector<int64_t> level(n, -1), order;
    order.reserve(n);
    vector<char> done(n, 0);
    vector<int64_t> bfs;
    auto bfs_levels = [&](int64_t root, vector<int64_t>& visit) {
        visit.clear();
        visit.push_back(root);
        level[root] = 0;
        for (size_t h = 0; h < visit.size(); ++h) {
            int64_t v = visit[h];
            for (int64_t p = xadj[v]; p < xadj[v + 1]; ++p)
                if (level[adj[p]] < 0) { level[adj[p]] = level[v] + 1; visit.push_back(adj[p]); }
        }
        int64_t ecc = level[visit.back()];
        for (int64_t v : visit) level[v] = -1;
        return ecc;
    };
    for (int64_t s = 0; s < n; ++s) {
        if (done[s]) continue;
        // component members, then a minimum-degree start
        vector<int64_t> comp;
        bfs_levels(s, comp);
        int64_t root = comp[0];
        for (int64_t v : comp)
            if (deg(v) < deg(root) || (deg(v) == deg(root) && v < root)) root = v;
        int64_t ecc = bfs_levels(root, bfs);
        for (int it = 0; it < 8; ++it) {  // pseudo-peripheral node search
            // min-degree node of the last level
            for (int64_t v : bfs) level[v] = -1;
            vector<int64_t> vis2;
            level[root] = 0;
            vis2.push_back(root);
            for (size_t h = 0; h < vis2.size(); ++h) {
                int64_t v = vis2[h];
                for (int64_t p = xadj[v]; p < xadj[v + 1]; ++p)
                    if (level[adj[p]] < 0) { level[adj[p]] = level[v] + 1; vis2.push_back(adj[p]); }
            }
            int64_t lastlev = level[vis2.back()], cand = -1;
            for (int64_t v : vis2)
                if (level[v] == lastlev && (cand < 0 || deg(v) < deg(cand))) cand = v;
            for (int64_t v : vis2) level[v] = -1;
            int64_t e2 = bfs_levels(cand, bfs);
            if (e2 <= ecc) break;
            ecc = e2;
            root = cand;
        }
        // Cuthill-McKee BFS, neighbours by ascending degree (ties: index)
        size_t head = order.size();
        order.push_back(root);
        done[root] = 1;
        vector<int64_t> nb;
        for (size_t h = head; h < order.size(); ++h) {
            int64_t v = order[h];
            nb.clear();
            for (int64_t p = xadj[v]; p < xadj[v + 1]; ++p)
                if (!done[adj[p]]) { done[adj[p]] = 1; nb.push_back(adj[p]); }
            std::sort(nb.begin(), nb.end(), [&](int64_t a, int64_t b) {
                return deg(a) != deg(b) ? deg(a) < deg(b) : a < b;
            });
            order.insert(order.end(), nb.begin(), nb.end());
        }
    }
    perm.assign(order.rbegin(), order.rend());
}

// Strict lower part of A_p = P A P^T as row lists: row r holds columns c < r.
void permuted_rows(int64_t n, const int64_t* Ap, const int64_t* Ai, const vector<int64_t>& iperm,
                   vector<int64_t>& rp, vector<int32_t>& rc, int threads) {
    // columns in chunks, walked twice (count, then write at offsets prefix-summed in chunk
    // order, so each row lists its columns in the order of a serial column sweep)
    const int64_t nch = std::max<int64_t>(1, std::min<int64_t>(int64_t(threads) * 8, n / 2048));
    const int64_t mem_cap = std::max<int64_t>(1, (int64_t(1) << 30) / (8 * n));
    const int nw = int(std::min<int64_t>(std::min<int64_t>(threads, nch), mem_cap));
    vector<vector<std::pair<int32_t, int64_t>>> touch(nch);
    vector<vector<int64_t>> acc(nw);
    auto walk = [&](int64_t c, int w, bool fill) {
        vector<int64_t>& ct = acc[w];
        if (ct.empty()) ct.assign(n, 0);
        vector<std::pair<int32_t, int64_t>>& tl = touch[c];
        if (fill)
            for (const auto& e : tl) ct[e.first] = e.second;
        for (int64_t j = c * n / nch; j < (c + 1) * n / nch; ++j)
            for (int64_t p = Ap[j] + 1; p < Ap[j + 1]; ++p) {
                const int64_t a = iperm[Ai[p]], b = iperm[j], r = std::max(a, b);
                if (fill) rc[ct[r]++] = (int32_t)std::min(a, b);
                else if (ct[r]++ == 0) tl.push_back({(int32_t)r, 0});
            }
        for (auto& e : tl) {
            if (!fill) e.second = ct[e.first];
            ct[e.first] = 0;
        }
    };
    parallel_chunks(nw, nch, [&](int64_t c, int w) { walk(c, w, false); });
    rp.assign(n + 1, 0);
    for (const auto& tl : touch)
        for (const auto& e : tl) rp[e.first + 1] += e.second;
    for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
    vector<int64_t> next(rp.begin(), rp.end() - 1);
    for (auto& tl : touch)
        for (auto& e : tl) {
            const int64_t start = next[e.first];
            next[e.first] += e.second;
            e.second = start;
        }
    rc.assign(rp[n], 0);
    parallel_chunks(nw, nch, [&](int64_t c, int w) { walk(c, w, true); });
}

// Liu's elimination tree and the structure of L from row subtrees.  The structure of row
// i of L is the row subtree of i: the etree paths from the columns of row i of A up to i.
// Rows are walked in chunks of consecutive rows, twice: once to count each chunk's
// entries per column, once to write them, at offsets that put every column's rows in
// ascending order (the chunks' counts are prefix-summed in chunk order).
void symbolic(int64_t n, const vector<int64_t>& rp, const vector<int32_t>& rc,
              vector<int64_t>& parent, vector<int64_t>& Lp, stc::RowIndexVec& Li, int threads) {
    parent.assign(n, -1);
    {
        vector<int64_t> anc(n, -1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                int64_t j = rc[p];
                while (j != -1 && j < i) {
                    int64_t nxt = anc[j];
                    anc[j] = i;
                    if (nxt == -1) parent[j] = i;
                    j = nxt;
                }
            }
    }
    const int64_t nch = std::max<int64_t>(1, std::min<int64_t>(int64_t(threads) * 8, n / 512));
    // each worker holds 12 n bytes of scratch: at most ~1 GiB in total
    const int64_t mem_cap = std::max<int64_t>(1, (int64_t(1) << 30) / (12 * n));
    const int nw = int(std::min<int64_t>(std::min<int64_t>(threads, nch), mem_cap));
    // per chunk: (column, entries of the chunk's rows in it), then (column, first slot)
    vector<vector<std::pair<int32_t, int64_t>>> touch(nch);
    vector<vector<int32_t>> mark(nw);
    vector<vector<int64_t>> acc(nw);
    auto walk = [&](int64_t c, int w, bool fill) {
        vector<int32_t>& mk = mark[w];
        vector<int64_t>& ct = acc[w];
        if (mk.empty()) { mk.assign(n, -1); ct.assign(n, 0); }
        const int64_t i0 = c * n / nch, i1 = (c + 1) * n / nch;
        vector<std::pair<int32_t, int64_t>>& tl = touch[c];
        if (fill)
            for (const auto& e : tl) ct[e.first] = e.second;
        for (int64_t i = i0; i < i1; ++i) {
            mk[i] = (int32_t)i;  // row ids differ between chunks: no reset within a walk
            if (fill) Li[Lp[i]] = (int32_t)i;  // the diagonal heads column i
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
                for (int64_t j = rc[p]; mk[j] != i; j = parent[j]) {
                    mk[j] = (int32_t)i;
                    if (fill) Li[ct[j]++] = (int32_t)i;
                    else if (ct[j]++ == 0) tl.push_back({(int32_t)j, 0});
                }
        }
        for (auto& e : tl) {
            if (!fill) e.second = ct[e.first];
            ct[e.first] = 0;
        }
    };
    parallel_chunks(nw, nch, [&](int64_t c, int w) { walk(c, w, false); });
    vector<int64_t> cnt(n, 1);  // the diagonal
    for (const auto& tl : touch)
        for (const auto& e : tl) cnt[e.first] += e.second;
    Lp.assign(n + 1, 0);
    for (int64_t j = 0; j < n; ++j) Lp[j + 1] = Lp[j] + cnt[j];
    for (int64_t j = 0; j < n; ++j) cnt[j] = Lp[j] + 1;  // next free slot below the diagonal
    for (auto& tl : touch)
        for (auto& e : tl) {
            const int64_t start = cnt[e.first];
            cnt[e.first] += e.second;
            e.second = start;
        }
    Li.clear();
    Li.resize(Lp[n]);  // uninitialised: the second walk writes every entry
    for (auto& mk : mark) std::fill(mk.begin(), mk.end(), -1);  // the second walk marks again
    parallel_chunks(nw, nch, [&](int64_t c, int w) { walk(c, w, true); });
}

}  // namespace

// ---------------------------------------------------------------------------
int stc_plan::tile_id(int64_t I, int64_t J) const {
    if (J < 0 || J >= nt || I < J || I >= nt) return -1;
    int lo = colstart[J], hi = colstart[J + 1];
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (tiles[mid].I == I) return mid;
        if (tiles[mid].I < I) lo = mid + 1; else hi = mid;
    }
    return -1;
}

namespace {

// stored index of logical column lc in tile t (-1 if not stored)
int stored_col(const stc_plan& P, const stc::DTile& t, int lc) {
    if (t.c0 >= 0) return (lc >= t.c0 && lc < t.c0 + t.sw) ? lc - t.c0 : -1;
    const int16_t* a = P.saind.data() + t.aoff;
    const int16_t* e = std::lower_bound(a, a + t.sw, (int16_t)lc);
    return (e != a + t.sw && *e == lc) ? int(e - a) : -1;
}

int64_t tile_entry_offset(const stc_plan& P, const stc::DTile& T, int lr, int lc) {
    const int64_t nb = P.nb;
    if (T.kind == stc::TILE_DIAG_DENSE) return T.off + lr + (int64_t)lc * nb;
    if (T.kind == stc::TILE_DIAG_BAND) {
        if (lr - lc > T.kd) return -1;
        return T.off + (T.kd + lc - lr) + (int64_t)lr * (T.kd + 1);
    }
    int s = stored_col(P, T, lc);
    if (s < 0) return -1;
    return T.off + lr + (int64_t)s * nb;
}

int64_t entry_offset(const stc_plan& P, int64_t r, int64_t c) {  // r >= c, permuted
    const int64_t nb = P.nb;
    int t = P.tile_id(r / nb, c / nb);
    if (t < 0) return -1;
    return tile_entry_offset(P, P.tiles[t], int(r % nb), int(c % nb));
}

// The tiles of one block column, with offsets into the column's own lists; build_tiles
// merges the columns in order.
struct ColTiles {
    vector<stc::DTile> tiles;   // aoff / xoff relative to this column's saind / cext
    vector<int64_t> size;       // stored doubles of each tile
    vector<int32_t> nact;
    vector<int64_t> aoff;       // offset of each tile's active columns in `aind`
    vector<int16_t> aind, saind, cext;
    vector<int8_t> contig, full;
};

struct TileScratch {            // per worker
    struct Acc { uint64_t m[2]; int r0, r1, kd; int32_t ext; };
    vector<int32_t> slot;
    vector<int64_t> touched;
    vector<int16_t> clo, chi;   // per tile of the column: row extent of each column
    vector<Acc> acc;
    vector<int16_t> cols;
};

void build_block_column(const stc_plan& P, int64_t J, bool dense, TileScratch& S, ColTiles& out) {
    const int64_t n = P.n, nb = P.nb;
    if (S.slot.empty()) S.slot.assign(P.nt, -1);
    S.touched.clear();
    S.acc.clear();
    S.clo.clear();
    S.chi.clear();
    const int64_t c0 = J * nb, c1 = std::min(n, (J + 1) * nb);
    for (int64_t j = c0; j < c1; ++j)
        for (int64_t q = P.Lp[j]; q < P.Lp[j + 1]; ++q) {
            int64_t i = P.Li[q], I = i / nb;
            if (S.slot[I] < 0) {
                S.slot[I] = (int32_t)S.acc.size();
                S.acc.push_back(TileScratch::Acc{{0, 0}, INT_MAX, -1, -1, (int32_t)S.clo.size()});
                S.clo.resize(S.clo.size() + nb, (int16_t)nb);
                S.chi.resize(S.chi.size() + nb, 0);
                S.touched.push_back(I);
            }
            TileScratch::Acc& a = S.acc[S.slot[I]];
            int lr = int(i - I * nb), lc = int(j - c0);
            a.m[lc >> 6] |= 1ull << (lc & 63);
            a.r0 = std::min(a.r0, lr);
            a.r1 = std::max(a.r1, lr + 1);
            S.clo[a.ext + lc] = (int16_t)std::min<int>(S.clo[a.ext + lc], lr);
            S.chi[a.ext + lc] = (int16_t)std::max<int>(S.chi[a.ext + lc], lr + 1);
            if (I == J) a.kd = std::max(a.kd, lr - lc);
        }
    std::sort(S.touched.begin(), S.touched.end());
    for (int64_t I : S.touched) {
        const TileScratch::Acc& a = S.acc[S.slot[I]];
        S.slot[I] = -1;
        stc::DTile t{};
        t.I = (int32_t)I; t.J = (int32_t)J;
        vector<int16_t>& cols = S.cols;
        cols.clear();
        for (int c = 0; c < nb; ++c)
            if (a.m[c >> 6] >> (c & 63) & 1) cols.push_back((int16_t)c);
        const int cnt = (int)cols.size();
        const bool contiguous = cols.back() - cols.front() + 1 == cnt;
        out.nact.push_back(cnt);
        out.aoff.push_back((int64_t)out.aind.size());
        out.aind.insert(out.aind.end(), cols.begin(), cols.end());
        out.contig.push_back(contiguous);
        out.full.push_back(cnt == nb);
        t.pd_slot = -1;
        t.aoff = -1;
        t.xoff = -1;
        int64_t size;
        if (I == J) {
            t.sw = int(c1 - c0);
            t.c0 = 0;
            t.r0 = 0; t.r1 = int(nb);
            if (dense) {
                t.kind = stc::TILE_DIAG_DENSE;
                t.kd = int(nb - 1);
                size = nb * nb;
            } else {
                t.kind = stc::TILE_DIAG_BAND;
                t.kd = std::max(a.kd, 0);
                size = (int64_t)(t.kd + 1) * nb;
            }
            t.pd_slot = (int32_t)J;
        } else {
            t.kind = stc::TILE_OFF;
            t.kd = -1;
            if (dense) {
                t.sw = int(nb); t.c0 = 0; t.r0 = 0; t.r1 = int(nb);
            } else {
                t.sw = cnt;
                t.r0 = a.r0; t.r1 = a.r1;
                if (contiguous) {
                    t.c0 = cols.front();
                } else {
                    t.c0 = -1;
                    t.aoff = (int32_t)out.saind.size();
                    out.saind.insert(out.saind.end(), cols.begin(), cols.end());
                }
            }
            size = (int64_t)t.sw * nb;
            // row extents of each kExtW stored columns (dense route: all n_b columns)
            t.xoff = (int32_t)(out.cext.size() / 2);
            for (int s0 = 0; s0 < t.sw; s0 += stc::kExtW) {
                int lo = int(nb), hi = 0;
                for (int s = s0; s < std::min(t.sw, s0 + stc::kExtW); ++s) {
                    const int lc = dense ? s : cols[s];
                    lo = std::min<int>(lo, S.clo[a.ext + lc]);
                    hi = std::max<int>(hi, S.chi[a.ext + lc]);
                }
                out.cext.push_back((int16_t)lo);
                out.cext.push_back((int16_t)hi);
            }
        }
        t.nfinal = 1;
        out.tiles.push_back(t);
        out.size.push_back(size);
    }
}

// Tile map of L (Sec. 4): block columns are built in parallel, then laid out in order
// (block-column-major, I ascending, 32-byte aligned tiles).
int build_tiles(stc_plan& P, int threads) {
    const int64_t nt = P.nt;
    const bool dense = P.route_exec == STC_ROUTE_DENSE;
    P.colstart.assign(nt + 1, 0);
    P.diag_tile.assign(nt, -1);
    vector<ColTiles> col(nt);
    const int nw = int(std::max<int64_t>(1, std::min<int64_t>(threads, nt)));
    vector<TileScratch> scratch(nw);
    const int64_t per = std::max<int64_t>(1, nt / (int64_t(nw) * 16));  // block columns per chunk
    parallel_chunks(nw, (nt + per - 1) / per, [&](int64_t c, int w) {
        for (int64_t J = c * per; J < std::min(nt, (c + 1) * per); ++J)
            build_block_column(P, J, dense, scratch[w], col[J]);
    });
    scratch.clear();
    int64_t off = 0;
    for (int64_t J = 0; J < nt; ++J) {
        ColTiles& C = col[J];
        P.colstart[J] = (int32_t)P.tiles.size();
        const int32_t sbase = (int32_t)P.saind.size(), xbase = (int32_t)(P.cext.size() / 2);
        const int64_t abase = (int64_t)P.aind_struct.size();
        for (size_t k = 0; k < C.tiles.size(); ++k) {
            stc::DTile t = C.tiles[k];
            if (t.aoff >= 0) t.aoff += sbase;
            if (t.xoff >= 0) t.xoff += xbase;
            if (t.I == t.J) P.diag_tile[J] = (int32_t)P.tiles.size();
            t.off = off;
            off += (C.size[k] + 3) / 4 * 4;  // 32-byte aligned tiles
            P.stored_entries += C.size[k];
            P.aoff_struct.push_back(abase + C.aoff[k]);
            P.tiles.push_back(t);
        }
        P.nact.insert(P.nact.end(), C.nact.begin(), C.nact.end());
        P.aind_struct.insert(P.aind_struct.end(), C.aind.begin(), C.aind.end());
        P.contig.insert(P.contig.end(), C.contig.begin(), C.contig.end());
        P.full.insert(P.full.end(), C.full.begin(), C.full.end());
        P.saind.insert(P.saind.end(), C.saind.begin(), C.saind.end());
        P.cext.insert(P.cext.end(), C.cext.begin(), C.cext.end());
        C = ColTiles();  // release the column's lists
    }
    P.colstart[nt] = (int32_t)P.tiles.size();
    P.partial_off = off;
    P.npartials = nt;
    P.factor_doubles = (off + nt + 31) / 32 * 32;  // 256-byte aligned item stride
    // off-diagonal tiles per block row (ascending n), for Algorithm 1 and the solve
    P.rowstart.assign(nt + 1, 0);
    for (const auto& t : P.tiles)
        if (t.I != t.J) P.rowstart[t.I + 1]++;
    for (int64_t k = 0; k < nt; ++k) P.rowstart[k + 1] += P.rowstart[k];
    P.rowtiles.assign(P.rowstart[nt], 0);
    vector<int32_t> f(P.rowstart.begin(), P.rowstart.end() - 1);
    for (int32_t t = 0; t < (int32_t)P.tiles.size(); ++t)
        if (P.tiles[t].I != P.tiles[t].J) P.rowtiles[f[P.tiles[t].I]++] = t;
    return STC_OK;
}

void build_alg1(stc_plan& P) {
    const int64_t nt = P.nt;
    auto emit = [&](int64_t c, int64_t m, int64_t k, int64_t nn) {
        P.alg1.push_back(c); P.alg1.push_back(m); P.alg1.push_back(k); P.alg1.push_back(nn);
    };
    for (int64_t k = 0; k < nt; ++k) {
        for (int32_t a = P.rowstart[k]; a < P.rowstart[k + 1]; ++a) {
            emit(2, -1, k, P.tiles[P.rowtiles[a]].J);
            P.n_syrk++;
        }
        emit(1, -1, k, -1);
        P.n_potrf++;
        for (int32_t t = P.colstart[k]; t < P.colstart[k + 1]; ++t) {
            const int64_t m = P.tiles[t].I;
            if (m == k) continue;
            int32_t a = P.rowstart[k], b = P.rowstart[m];
            while (a < P.rowstart[k + 1] && b < P.rowstart[m + 1]) {
                int32_t na = P.tiles[P.rowtiles[a]].J, nbb = P.tiles[P.rowtiles[b]].J;
                if (na == nbb) { emit(4, m, k, na); P.n_gemm++; ++a; ++b; }
                else if (na < nbb) ++a;
                else ++b;
            }
            emit(3, m, k, -1);
            P.n_trsm++;
        }
    }
}

// logical columns stored in tile t
void stored_cols(const stc_plan& P, const stc::DTile& t, vector<int>& out) {
    out.resize(t.sw);
    for (int s = 0; s < t.sw; ++s) out[s] = t.c0 >= 0 ? t.c0 + s : P.saind[t.aoff + s];
}

}  // namespace

// Kernel geometry the cost model mirrors: inner-dimension chunk of the tile products
// and panel width of the TRSM.
constexpr int kChunk = stc::kExtW;
constexpr int kPanel = stc::kPanelW;

stc::TaskSet* stc_plan::taskset(int32_t slices, bool bl_order, bool fwd) {
    std::lock_guard<std::mutex> g(mu);
    auto it = tasksets.find(taskset_key(slices, bl_order, fwd));
    if (it != tasksets.end()) return it->second.get();
    auto ts = std::make_unique<stc::TaskSet>();
    const int64_t NT = nt;
    const int NB = (int)nb;
    // a device task holds at most 64 rows of an off-diagonal or SYRK tile
    const int32_t eff = std::max<int32_t>(slices, (NB + 63) / 64);
    ts->slices = eff;
    int h = (NB + eff - 1) / eff;
    h = (h + 7) / 8 * 8;
    if (h > 64) h = 64;
    // at most kMaxSlices slices per tile (one completion bit per slice and panel)
    if ((NB + h - 1) / h > stc::kMaxSlices) h = ((NB + stc::kMaxSlices - 1) / stc::kMaxSlices + 7) / 8 * 8;
    ts->slice_h = h;
    // tasks in Algorithm-1 (topological) order first, with the model inputs of each:
    // the source tiles its updates wait for (in order) and the final dependency
    struct Meta {
        std::vector<int32_t> srcs;   // per update: tiles it waits for (1 or 2)
        std::vector<double> ucost;   // per update FMAs
        std::vector<int8_t> nsrc;
        int32_t final_tile = -1;     // tile awaited before the final op (-1: none)
        double fcost = 0;
        bool trsm = false;           // TASK_OFF: the final op (TRSM) follows L_kk group by group
        int npub = 0;                // >0: the task publishes its tile in npub steps
    };
    vector<stc::DTask> tasks;
    vector<Meta> meta;
    vector<vector<int32_t>> producers(tiles.size());
    ts->nfinal.assign(tiles.size(), 0);
    // executed FMAs of the chunked products, with the same extent skipping as the kernel
    auto ext = [&](const stc::DTile& T, int s0, int s1, int& lo, int& hi) {
        if (T.xoff < 0) { lo = 0; hi = NB; return; }
        lo = NB; hi = 0;
        for (int q = s0 / stc::kExtW; q <= s1 / stc::kExtW; ++q) {
            lo = std::min<int>(lo, cext[2 * (T.xoff + q)]);
            hi = std::max<int>(hi, cext[2 * (T.xoff + q) + 1]);
        }
    };
    auto inner_range = [&](const vector<int16_t>& im, const stc::DUpd& u, int k0, int K, bool b, int& s0,
                           int& s1) {
        if (u.kmap < 0) {
            s0 = (b ? u.kb0 : u.ka0) + k0;
            s1 = s0 + K - 1;
        } else {
            s0 = im[2 * (u.kmap + k0) + (b ? 1 : 0)];
            s1 = im[2 * (u.kmap + k0 + K - 1) + (b ? 1 : 0)];
        }
    };
    auto syrk_cost = [&](const vector<int16_t>& im, const stc::DUpd& u, int r0, int d0, int rb) {  // rows [d0,rb), cols [r0,rb)
        const stc::DTile& A = tiles[u.a];
        double c = 0.0;
        for (int k0 = 0; k0 < u.klen; k0 += kChunk) {
            const int K = std::min(kChunk, u.klen - k0);
            int s0, s1, lo, hi;
            inner_range(im, u, k0, K, false, s0, s1);
            ext(A, s0, s1, lo, hi);
            const int e0 = std::max(d0, lo), e1 = std::min(rb, hi);
            if (e0 >= e1) continue;
            const double rows = e1 - e0, rect = std::max(0, std::min(d0, e1) - std::max(r0, lo));
            c += (rows * rect + rows * (rows + 1) / 2) * K;
        }
        return c;
    };
    auto gemm_cost = [&](const vector<int16_t>& im, const stc::DUpd& u, const stc::DTile& O) {
        const stc::DTile& A = tiles[u.a];
        const stc::DTile& B = tiles[u.b];
        double c = 0.0;
        for (int k0 = 0; k0 < u.klen; k0 += kChunk) {
            const int K = std::min(kChunk, u.klen - k0);
            int s0, s1, alo, ahi, blo, bhi;
            inner_range(im, u, k0, K, false, s0, s1);
            ext(A, s0, s1, alo, ahi);
            inner_range(im, u, k0, K, true, s0, s1);
            ext(B, s0, s1, blo, bhi);
            const int e0 = std::max(u.ra0, alo), e1 = std::min(u.ra1, ahi);
            int c0 = u.oc0, c1 = u.oc1;
            if (O.c0 >= 0) { c0 = std::max(c0, blo - O.c0); c1 = std::min(c1, bhi - O.c0); }
            if (e0 < e1 && c0 < c1) c += double(e1 - e0) * (c1 - c0) * K;
        }
        return c;
    };
    auto trsm_cost = [&](const stc::DTile& O, int tr0, int tr1) {
        double c = 0.0;
        for (int p = 0; p < O.sw; p += kPanel) {
            const int pw = std::min(kPanel, O.sw - p);
            for (int k0 = 0; k0 < p; k0 += kChunk) {
                int lo, hi;
                ext(O, k0, std::min(p, k0 + kChunk) - 1, lo, hi);
                const int x0 = std::max(tr0, lo), x1 = std::min(tr1, hi);
                if (x0 < x1) c += double(x1 - x0) * pw * std::min(kChunk, p - k0);
            }
            int lo, hi;
            ext(O, p, p + pw - 1, lo, hi);
            const int y0 = std::max(tr0, lo), y1 = std::min(tr1, hi);
            if (y0 < y1) c += double(y1 - y0) * pw * (pw + 1) / 2;
        }
        return c;
    };
    // completion bit of column group g of row slice s of a diagonal tile
    constexpr int DG = stc::kDiagGroupW;
    auto dbit = [](int g, int s) { return (int32_t)(1u << (g * stc::kMaxDiagSlices + s)); };
    // modelled cost of one more slice of a diagonal tile: with two slices per off-diagonal
    // tile (the choice for wide batches, whose replay is bound by the SMs' FP64 throughput)
    // an extra slice's staging and synchronisation weigh more than a shorter chain; with
    // more slices (few items, the chain bounds) they weigh little.  Measured on the
    // n = 200,000 band: 64 value sets 739 ms with four slices of (k,k), 720 ms with three;
    // one value set 270 ms with four, 287 ms with three.
    const double kSliceSync = eff <= 2 ? 150000.0 : 3000.0;
    auto potrf_cost = [&](const stc::DTile& D) {
        double w = D.sw, kd = std::min<double>(D.kd, w - 1);
        return (D.kind == stc::TILE_DIAG_BAND) ? w * (kd + 1) * (kd + 1) / 2 : w * w * w / 6;
    };
    // tasks of each block column are built independently (in parallel), then laid out in
    // block-column order with their update and map offsets shifted
    struct Local {
        vector<stc::DTask> tasks;
        vector<Meta> meta;
        vector<stc::DUpd> upds;
        vector<int16_t> imap;
    };
    vector<Local> loc(NT);
    auto build_col = [&](int64_t k, Local& Lk) {
        vector<int> ca, cb;
        const int32_t dk = diag_tile[k];
        const stc::DTile& D = tiles[dk];
        const bool has_syrk = rowstart[k + 1] > rowstart[k];
        const int G = (D.sw + DG - 1) / DG;  // column groups of the diagonal tile
        if (eff == 1 || !has_syrk) {
            // TASK_DIAG: every SYRK from (k,n), n < k, then POTRF
            stc::DTask t{};
            Meta mt;
            t.kind = stc::TASK_DIAG; t.tile = dk; t.diag = dk;
            t.ubeg = (int32_t)Lk.upds.size();
            for (int32_t a = rowstart[k]; a < rowstart[k + 1]; ++a) {
                const int32_t at = rowtiles[a];
                const stc::DTile& A = tiles[at];
                stc::DUpd u{};
                u.a = at; u.b = at; u.kmap = -1; u.klen = A.sw; u.ka0 = 0; u.kb0 = 0;
                u.ra0 = A.r0; u.ra1 = A.r1; u.oc0 = A.r0; u.oc1 = A.r1;
                Lk.upds.push_back(u);
                mt.srcs.push_back(at); mt.nsrc.push_back(1); mt.ucost.push_back(syrk_cost(Lk.imap, u, A.r0, A.r0, A.r1));
            }
            t.uend = (int32_t)Lk.upds.size();
            t.rs0 = 0; t.rs1 = NB; t.tr0 = 0; t.tr1 = NB;
            mt.fcost = potrf_cost(D);
            mt.npub = G;
            Lk.tasks.push_back(t);
            Lk.meta.push_back(mt);
            for (int g = 0; g < G; ++g) ts->nfinal[dk] |= dbit(g, 0);
        } else {
            // TASK_SYRK row slices of (k,k): each applies every SYRK into its rows, then
            // factors them against the columns the earlier slices publish (a row-partitioned
            // POTRF), so the factorization of (k,k) is spread over the slices' CTAs.  Cuts lie
            // on kDiagGroupW-row boundaries, slices hold at most 64 rows, and the cut set
            // minimises the largest slice's modelled work (its SYRK products plus its rows'
            // share of the POTRF), plus a synchronisation cost per extra slice.
            vector<double> wb(G, 0.0);
            for (int b = 0; b < G; ++b) {
                const int r0 = b * DG, r1 = std::min(D.sw, r0 + DG);
                for (int32_t a = rowstart[k]; a < rowstart[k + 1]; ++a) {
                    const stc::DTile& A = tiles[rowtiles[a]];
                    const int ra = std::max(r0, A.r0), rb = std::min(r1, A.r1);
                    if (ra >= rb) continue;
                    stc::DUpd u{};
                    u.a = rowtiles[a]; u.b = u.a; u.kmap = -1; u.klen = A.sw;
                    wb[b] += syrk_cost(Lk.imap, u, A.r0, ra, rb);
                }
                for (int r = r0; r < r1; ++r) {
                    const double m = std::min(r, D.kd);
                    wb[b] += m * (m + 1) / 2;
                }
            }
            unsigned best_mask = 0;
            double best = std::numeric_limits<double>::infinity();
            for (unsigned mask = 0; mask < (1u << std::max(0, G - 1)); ++mask) {
                // bit b - 1 of mask: a cut before group b
                int runs = 0, len = 0;
                double cur = 0.0, worst = 0.0;
                bool ok = true;
                for (int b = 0; b < G && ok; ++b) {
                    if (b > 0 && (mask >> (b - 1) & 1u)) {
                        worst = std::max(worst, cur);
                        cur = 0.0;
                        len = 0;
                        ++runs;
                    }
                    cur += wb[b];
                    ok = ++len * DG <= 64;
                }
                ++runs;
                worst = std::max(worst, cur);
                if (!ok || runs > stc::kMaxDiagSlices) continue;
                const double obj = worst + kSliceSync * (runs - 1);
                if (obj < best) { best = obj; best_mask = mask; }
            }
            vector<int> cuts{0};
            for (int b = 1; b < G; ++b)
                if (best_mask >> (b - 1) & 1u) cuts.push_back(b * DG);
            cuts.push_back(D.sw);
            const int kd = D.kd;
            for (size_t s = 0; s + 1 < cuts.size(); ++s) {
                const int rs0 = cuts[s], rs1 = cuts[s + 1], R = rs1 - rs0;
                stc::DTask t{};
                Meta mt;
                t.kind = stc::TASK_SYRK; t.tile = dk; t.diag = dk; t.slice = (int32_t)s;
                t.rs0 = rs0; t.rs1 = rs1; t.tr0 = rs0; t.tr1 = rs1;
                t.ubeg = (int32_t)Lk.upds.size();
                for (int32_t a = rowstart[k]; a < rowstart[k + 1]; ++a) {
                    const int32_t at = rowtiles[a];
                    const stc::DTile& A = tiles[at];
                    const int ra = std::max(rs0, A.r0), rb = std::min(rs1, A.r1);
                    if (ra >= rb) continue;
                    stc::DUpd u{};
                    u.a = at; u.b = at; u.kmap = -1; u.klen = A.sw; u.ka0 = 0; u.kb0 = 0;
                    u.ra0 = ra; u.ra1 = rb; u.oc0 = A.r0; u.oc1 = rb;
                    Lk.upds.push_back(u);
                    mt.srcs.push_back(at); mt.nsrc.push_back(1);
                    mt.ucost.push_back(syrk_cost(Lk.imap, u, A.r0, ra, rb));
                }
                t.uend = (int32_t)Lk.upds.size();
                // the factorization of the rows, as the kernel executes it: per group of the
                // earlier slices' columns (skipped where it lies outside the band of every
                // row of the slice) a TRSM of the rows and the rank-kDiagGroupW update of
                // their later columns; then the POTRF of the slice's own diagonal block
                double fc = 0.0;
                int npub = 0;
                for (int g0 = 0; g0 < rs0; g0 += DG) {
                    if (g0 + DG <= rs0 - kd) continue;
                    fc += double(R) * DG * (DG - 1) / 2 + double(R) * (rs0 - g0 - DG) * DG +
                          double(R) * (R + 1) / 2 * DG;
                    ts->nfinal[dk] |= dbit(g0 / DG, (int)s);
                    ++npub;
                }
                {
                    const int64_t kdd = std::min(kd, R - 1);
                    for (int64_t j = 0; j < R; ++j) {
                        const double m = double(std::min<int64_t>(kdd, R - 1 - j));
                        fc += m * (m + 1) / 2 + m;
                    }
                }
                for (int g = rs0 / DG; g < (rs1 + DG - 1) / DG; ++g) {
                    ts->nfinal[dk] |= dbit(g, (int)s);
                    ++npub;
                }
                mt.fcost = fc;
                mt.npub = npub;
                if (s > 0) {  // follows the earlier slices' published groups
                    mt.final_tile = dk;
                    mt.trsm = true;
                }
                Lk.tasks.push_back(t);
                Lk.meta.push_back(mt);
            }
        }
        // OFF(m,k) row slices: GEMM from every n in N(k) & N(m), n < k, then TRSM
        for (int32_t o = colstart[k]; o < colstart[k + 1]; ++o) {
            const stc::DTile& O = tiles[o];
            if (O.I == O.J) continue;
            const int64_t m = O.I;
            for (int rs0 = 0; rs0 < NB; rs0 += h) {
                const int rs1 = std::min(NB, rs0 + h);
                const int tr0 = std::max(rs0, O.r0), tr1 = std::min(rs1, O.r1);
                if (tr0 >= tr1) continue;
                stc::DTask s{};
                Meta ms;
                s.kind = stc::TASK_OFF; s.tile = o; s.diag = dk; s.slice = rs0 / h;
                s.rs0 = rs0; s.rs1 = rs1; s.tr0 = tr0; s.tr1 = tr1;
                s.ubeg = (int32_t)Lk.upds.size();
                int32_t a = rowstart[k], b = rowstart[m];
                while (a < rowstart[k + 1] && b < rowstart[m + 1]) {
                    const int32_t kt = rowtiles[a], mtile = rowtiles[b];
                    const int32_t na = tiles[kt].J, nm = tiles[mtile].J;
                    if (na < nm) { ++a; continue; }
                    if (nm < na) { ++b; continue; }
                    ++a; ++b;
                    const stc::DTile& A = tiles[mtile];  // (m,n)
                    const stc::DTile& B = tiles[kt];     // (k,n)
                    stc::DUpd u{};
                    u.a = mtile; u.b = kt;
                    u.ra0 = std::max(tr0, A.r0); u.ra1 = std::min(tr1, A.r1);
                    size_t imap_mark = Lk.imap.size();
                    if (A.c0 >= 0 && B.c0 >= 0) {
                        const int lo = std::max(A.c0, B.c0), hi = std::min(A.c0 + A.sw, B.c0 + B.sw);
                        u.kmap = -1; u.klen = std::max(0, hi - lo);
                        u.ka0 = lo - A.c0; u.kb0 = lo - B.c0;
                    } else {
                        stored_cols(*this, A, ca);
                        stored_cols(*this, B, cb);
                        u.kmap = (int32_t)(Lk.imap.size() / 2);
                        int x = 0, y = 0, len = 0;
                        while (x < (int)ca.size() && y < (int)cb.size()) {
                            if (ca[x] == cb[y]) {
                                Lk.imap.push_back((int16_t)x); Lk.imap.push_back((int16_t)y);
                                ++len; ++x; ++y;
                            } else if (ca[x] < cb[y]) ++x; else ++y;
                        }
                        u.klen = len; u.ka0 = 0; u.kb0 = 0;
                    }
                    if (O.c0 >= 0) {
                        const int lo = std::max(O.c0, B.r0), hi = std::min(O.c0 + O.sw, B.r1);
                        u.oc0 = lo - O.c0; u.oc1 = hi - O.c0;
                    } else {
                        u.oc0 = 0; u.oc1 = O.sw;
                    }
                    if (u.klen <= 0 || u.ra0 >= u.ra1 || u.oc0 >= u.oc1) {
                        Lk.imap.resize(imap_mark);
                        continue;
                    }
                    Lk.upds.push_back(u);
                    ms.srcs.push_back(mtile); ms.srcs.push_back(kt); ms.nsrc.push_back(2);
                    ms.ucost.push_back(gemm_cost(Lk.imap, u, O));
                }
                s.uend = (int32_t)Lk.upds.size();
                ms.final_tile = dk;
                ms.fcost = trsm_cost(O, tr0, tr1);
                ms.trsm = true;
                ms.npub = (O.sw + kPanel - 1) / kPanel;
                                Lk.tasks.push_back(s);
                Lk.meta.push_back(ms);
                for (int q = 0; q * kPanel < O.sw; ++q)
                    ts->nfinal[o] |= (int32_t)(1u << (q * stc::kMaxSlices + s.slice));
            }
        }
    };
    {
        int nth = opt.host_threads;
        if (nth <= 0) nth = int(std::min<unsigned>(32, std::max<unsigned>(1, std::thread::hardware_concurrency())));
        const int64_t per = std::max<int64_t>(1, NT / (int64_t(nth) * 16));
        parallel_chunks(nth, (NT + per - 1) / per, [&](int64_t c, int) {
            for (int64_t k = c * per; k < std::min<int64_t>(NT, (c + 1) * per); ++k) build_col(k, loc[k]);
        });
    }
    {
        size_t nt_ = 0, nu = 0, nm = 0;
        for (const Local& Lk : loc) {
            nt_ += Lk.tasks.size();
            nu += Lk.upds.size();
            nm += Lk.imap.size();
        }
        tasks.reserve(nt_);
        meta.reserve(nt_);
        ts->upds.reserve(nu);
        ts->imap.reserve(nm);
    }
    for (int64_t k = 0; k < NT; ++k) {
        Local& Lk = loc[k];
        const int32_t ubase = (int32_t)ts->upds.size(), mbase = (int32_t)(ts->imap.size() / 2);
        for (stc::DUpd& u : Lk.upds)
            if (u.kmap >= 0) u.kmap += mbase;
        for (size_t i = 0; i < Lk.tasks.size(); ++i) {
            stc::DTask t = Lk.tasks[i];
            t.ubeg += ubase;
            t.uend += ubase;
            producers[t.tile].push_back((int32_t)tasks.size());
            tasks.push_back(t);
            meta.push_back(std::move(Lk.meta[i]));
        }
        ts->upds.insert(ts->upds.end(), Lk.upds.begin(), Lk.upds.end());
        ts->imap.insert(ts->imap.end(), Lk.imap.begin(), Lk.imap.end());
        Lk = Local();
    }
    // TASK_FWD (fused forward substitution): one per block, after every factorization
    // task; they produce nothing another factorization task reads
    const size_t nfact = tasks.size();
    if (fwd)
        for (int64_t k = 0; k < NT; ++k) {
            stc::DTask f{};
            f.kind = stc::TASK_FWD; f.tile = diag_tile[k]; f.diag = diag_tile[k];
            f.rs0 = 0; f.rs1 = NB; f.tr0 = 0; f.tr1 = NB;
            tasks.push_back(f);
            meta.emplace_back();
        }
    // Queue order: earliest start on unbounded workers.  Tiles are published in steps
    // (an off-diagonal slice per TRSM panel, a diagonal tile per kDiagGroupW factored
    // columns), so a consumer can start on a tile's first published part ("avail") and
    // finishes its use of it a fraction of its own work after the tile is final ("fin").
    // A task starts when its first input is available and runs its updates in order;
    // the key is raised to exceed every dependency's key, so the order stays
    // topological (a waited-for task is always taken from the queue earlier).
    const double kSync = 3000.0;  // per-task overhead, FMA-equivalents
    const double kInf = std::numeric_limits<double>::infinity();
    const size_t T = tasks.size();
    vector<double> key(T, 0.0), fin(T, 0.0), tile_fin(tiles.size(), 0.0), tile_key(tiles.size(), 0.0);
    vector<double> tile_avail(tiles.size(), kInf);
    auto avail = [&](int32_t tl) { return tile_avail[tl] < kInf ? tile_avail[tl] : tile_fin[tl]; };
    for (size_t i = 0; i < nfact; ++i) {
        const Meta& mt = meta[i];
        double kdep = 0.0;
        for (int32_t s : mt.srcs) kdep = std::max(kdep, tile_key[s]);
        if (mt.final_tile >= 0) kdep = std::max(kdep, tile_key[mt.final_tile]);
        double first;
        if (!mt.srcs.empty()) {
            first = avail(mt.srcs[0]);
            if (mt.nsrc[0] == 2) first = std::max(first, avail(mt.srcs[1]));
        } else if (mt.final_tile >= 0) {
            first = mt.trsm ? avail(mt.final_tile) : tile_fin[mt.final_tile];  // POTRF: after its SYRKs
        } else {
            first = 0.0;
        }
        double t = first;
        size_t q = 0;
        for (size_t u = 0; u < mt.ucost.size(); ++u) {
            double rs = avail(mt.srcs[q]), re = tile_fin[mt.srcs[q]];
            if (mt.nsrc[u] == 2) {
                rs = std::max(rs, avail(mt.srcs[q + 1]));
                re = std::max(re, tile_fin[mt.srcs[q + 1]]);
            }
            q += mt.nsrc[u];
            t = std::max(std::max(t, rs) + mt.ucost[u], re + mt.ucost[u] / 4);
        }
        double tf = t;  // start of the final operation
        if (mt.final_tile >= 0 && mt.trsm) {
            tf = std::max(t, avail(mt.final_tile));
            t = std::max(tf + mt.fcost, tile_fin[mt.final_tile] + mt.fcost / 4);
        } else if (mt.final_tile >= 0) {
            tf = std::max(t, tile_fin[mt.final_tile]);
            t = tf + mt.fcost;
        } else {
            t += mt.fcost;
        }
        t += kSync;
        fin[i] = t;
        key[i] = std::max(first, kdep + 1e-6);
        {
            // algorithmic count: a row slice's share of POTRF(k) is sum_r m (m+1) / 2 over its
            // rows r, m = min(r, kd) (its fcost is what the kernel executes)
            double fa = mt.fcost;
            if (tasks[i].kind == stc::TASK_SYRK) {
                const stc::DTile& Dt = tiles[tasks[i].tile];
                fa = 0.0;
                for (int r = tasks[i].rs0; r < tasks[i].rs1; ++r) {
                    const double m = std::min(r, Dt.kd);
                    fa += m * (m + 1) / 2;
                }
            }
            ts->fma += std::accumulate(mt.ucost.begin(), mt.ucost.end(), 0.0) + fa;
        }
        {
            // the POTRF cost of the model is the banded-Cholesky estimate w (kd+1)^2 / 2;
            // the kernel updates, after column j, the min(kd, w-1-j) rows below it
            double fc = mt.fcost;
            if (tasks[i].kind == stc::TASK_DIAG) {
                const stc::DTile& Dt = tiles[tasks[i].tile];
                const int64_t kdd = std::min<int64_t>(Dt.kd, Dt.sw - 1);
                fc = 0.0;
                for (int64_t j = 0; j < Dt.sw; ++j) {
                    const double m = double(std::min<int64_t>(kdd, Dt.sw - 1 - j));
                    fc += m * (m + 1) / 2 + m;
                }
            }
            ts->fma_exec += std::accumulate(mt.ucost.begin(), mt.ucost.end(), 0.0) + fc;
        }
        const int32_t o = tasks[i].tile;
        if (mt.npub > 0) tile_avail[o] = std::min(tile_avail[o], tf + (t - tf) / mt.npub);
        tile_fin[o] = std::max(tile_fin[o], fin[i]);
        tile_key[o] = std::max(tile_key[o], key[i]);
    }
    if (bl_order) {
        // Priority by bottom level: the longest modelled path from a task to the end of its
        // item's DAG.  Predecessors rank strictly above their successors (every task costs
        // at least kSync), so the descending order is topological.  Measured: better for a
        // single factorization of a wide DAG (the 64^3 FEM pattern), worse for batches.
        vector<double> cost(T), bl(T);
        for (size_t i = 0; i < T; ++i)
            cost[i] = bl[i] = std::accumulate(meta[i].ucost.begin(), meta[i].ucost.end(), 0.0) + meta[i].fcost + kSync;
        for (size_t ii = nfact; ii-- > 0;) {
            auto pull = [&](int32_t tile) {
                // producers built before ii (a row slice of (k,k) reads only the slices
                // of its own tile that precede it)
                for (int32_t d : producers[tile])
                    if ((size_t)d < ii) bl[d] = std::max(bl[d], cost[d] + bl[ii]);
            };
            for (int32_t s2 : meta[ii].srcs) pull(s2);
            if (meta[ii].final_tile >= 0) pull(meta[ii].final_tile);
        }
        for (size_t i = 0; i < T; ++i) key[i] = -bl[i];
    }
    if (fwd) {
        // TASK_FWD k after the tasks of every tile it reads ((k,k), the tiles of block row k)
        // and after FWD k-1; and no earlier than the tasks of (k+2,k+2), so that a CTA that
        // takes it finds its inputs final instead of waiting for them
        vector<double> tkey(tiles.size(), -std::numeric_limits<double>::infinity());
        for (size_t i = 0; i < nfact; ++i) tkey[tasks[i].tile] = std::max(tkey[tasks[i].tile], key[i]);
        double prev = -std::numeric_limits<double>::infinity();
        for (int64_t k = 0; k < NT; ++k) {
            double kk = std::max(prev, std::max(tkey[diag_tile[k]], tkey[diag_tile[std::min<int64_t>(NT - 1, k + 2)]]));
            for (int32_t a = rowstart[k]; a < rowstart[k + 1]; ++a) kk = std::max(kk, tkey[rowtiles[a]]);
            kk += 1e-6 * (std::abs(kk) + 1.0);
            key[nfact + k] = kk;
            prev = kk;
        }
    }
    vector<int32_t> order(T);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    if (fwd) {
        // Forward substitution of block k hosted by a factorization task that usually starts
        // by waiting (slice 0 of a diagonal tile, or an unsliced one), so that it fills the
        // host's wait instead of taking a CTA slot of its own: the second such task, in queue
        // order, after every task of (k,k) and of the tiles of block row k and after the host
        // of block k-1.  The host runs it first (DTask.own_wait = diagonal tile of k, plus 1).
        // A block with no host left keeps its own TASK_FWD.
        vector<int32_t> pos(T);
        for (size_t q = 0; q < T; ++q) pos[order[q]] = (int32_t)q;
        vector<int32_t> dep(NT, -1);
        for (size_t i = 0; i < nfact; ++i) {
            const int64_t row = tiles[tasks[i].tile].I;  // block row of the task's tile
            dep[row] = std::max(dep[row], pos[i]);
        }
        int32_t prev = -1;
        std::vector<char> drop(T, 0);
        auto eligible = [&](int32_t q) {
            const stc::DTask& h = tasks[order[q]];
            return h.kind == stc::TASK_DIAG || (h.kind == stc::TASK_SYRK && h.slice == 0);
        };
        for (int64_t k = 0; k < NT; ++k) {
            // the second eligible position after the block's inputs, or the first free eligible
            // task after it and after the previous block's host
            int32_t from = -1, seen = 0, host = -1;
            for (int32_t q = dep[k] + 1; q < (int32_t)T; ++q)
                if (eligible(q) && ++seen == 2) { from = q; break; }
            if (from >= 0)
                for (int32_t q = std::max(from, prev + 1); q < (int32_t)T; ++q)
                    if (eligible(q) && tasks[order[q]].own_wait == 0) { host = q; break; }
            if (host < 0) break;  // this block and the later ones keep their TASK_FWD
            tasks[order[host]].own_wait = diag_tile[k] + 1;
            drop[nfact + k] = 1;
            prev = host;
        }
        // the blocks without a host last, in block order (after every host)
        vector<int32_t> kept;
        kept.reserve(T);
        for (int32_t i : order)
            if ((size_t)i < nfact) kept.push_back(i);
        double klast = kept.empty() ? 0.0 : key[kept.back()];
        for (int64_t k = 0; k < NT; ++k)
            if (!drop[nfact + k]) {
                key[nfact + k] = klast += 1.0;
                kept.push_back((int32_t)(nfact + k));
            }
        order.swap(kept);
        // Value scatter of block column k inside the launch, hosted by a task that usually
        // waits at its start (slice 1 of a diagonal tile waits for slice 0's first groups):
        // the second such position before the first task of column k (or the nearest free
        // one before it).  Every task of column k waits for the column's fill flag, so a
        // host must come earlier in the queue.  Columns without a host get a TASK_FILL at
        // the head of the queue; when fewer than half the columns find a host the set
        // keeps the separate scatter kernel.
        const size_t Q = order.size();
        vector<int32_t> firstq(NT, (int32_t)Q);
        for (size_t q = 0; q < Q; ++q) {
            const int64_t col = tiles[tasks[order[q]].tile].J;
            firstq[col] = std::min<int32_t>(firstq[col], (int32_t)q);
        }
        auto fhost = [&](int32_t q) {
            const stc::DTask& h = tasks[order[q]];
            return h.kind == stc::TASK_SYRK && h.slice == 1;
        };
        vector<int32_t> host(NT, -1);
        int64_t nhost = 0;
        for (int64_t k = 0; k < NT; ++k) {
            int32_t from = -1, seen = 0;
            for (int32_t q = firstq[k] - 1; q >= 0; --q)
                if (fhost(q) && ++seen == 2) { from = q; break; }
            for (int32_t q = from; q >= 0; --q)
                if (fhost(q) && tasks[order[q]].fill == 0) {
                    tasks[order[q]].fill = (int32_t)k + 1;
                    host[k] = q;
                    ++nhost;
                    break;
                }
        }
        if (2 * nhost < NT) {
            for (int64_t k = 0; k < NT; ++k)
                if (host[k] >= 0) tasks[order[host[k]]].fill = 0;
        } else {
            ts->fill_inside = true;
            vector<int32_t> head;
            for (int64_t k = 0; k < NT; ++k)
                if (host[k] < 0) {
                    stc::DTask f{};
                    f.kind = stc::TASK_FILL; f.tile = diag_tile[k]; f.diag = diag_tile[k];
                    tasks.push_back(f);
                    key.push_back(-1.0);
                    head.push_back((int32_t)(tasks.size() - 1));
                }
            head.insert(head.end(), order.begin(), order.end());
            order.swap(head);
        }
    }
    ts->tasks.reserve(order.size());
    ts->qkey.reserve(order.size());
    for (int32_t i : order) {
        ts->tasks.push_back(tasks[i]);
        ts->qkey.push_back(key[i]);
    }
    ts->period = T ? key[order.back()] / double(std::max<int64_t>(1, NT)) : 0.0;
    const double makespan = T ? *std::max_element(fin.begin(), fin.end()) : 0.0;
    ts->par = makespan > 0.0 ? ts->fma / makespan : 1.0;
    stc::TaskSet* raw = ts.get();
    tasksets[taskset_key(slices, bl_order, fwd)] = std::move(ts);
    return raw;
}

// ---------------------------------------------------------------------------
// Public entry points (host side).
// ---------------------------------------------------------------------------
extern "C" const char* stc_strerror(int code) {
    switch (code) {
        case STC_OK: return "success";
        case STC_ERR_INVALID_ARG: return "invalid argument";
        case STC_ERR_INVALID_PATTERN: return "invalid pattern (not lower CSC with sorted rows and a diagonal)";
        case STC_ERR_OUT_OF_MEMORY: return "out of memory";
        case STC_ERR_CUDA: return "CUDA runtime error";
        case STC_ERR_TIMEOUT: return "device dependency wait exceeded its limit";
        case STC_ERR_UNSUPPORTED: return "unsupported option or size";
        case STC_ERR_BUFFER_TOO_SMALL: return "buffer too small";
        default: return "unknown error";
    }
}

extern "C" void stc_options_default(stc_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->nb = 128;
    o->force_route = STC_ROUTE_AUTO;
    o->ordering = STC_ORDER_AUTO;
    o->nd_leaf = 64;
}

static int analyze_impl(int64_t n, const int64_t* Ap, const int64_t* Ai, const double* coords,
                        const stc_options* opt_in, stc_plan** out) {
    auto t0 = std::chrono::steady_clock::now();
    if (!out) return STC_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = validate_pattern(n, Ap, Ai);
    if (rc) return rc;
    stc_options opt;
    stc_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.nb == 0) opt.nb = 128;
    if (opt.nd_leaf <= 0) opt.nd_leaf = 64;
    if (opt.nb < 8 || opt.nb > kMaxNb || opt.nb % 8) return STC_ERR_UNSUPPORTED;
    if (opt.force_route != STC_ROUTE_AUTO && opt.force_route != STC_ROUTE_DENSE &&
        opt.force_route != STC_ROUTE_SEMISPARSE && opt.force_route != STC_ROUTE_SUPERNODAL)
        return STC_ERR_INVALID_ARG;
    if (opt.row_slices != 0 && opt.row_slices != 1 && opt.row_slices != 2 && opt.row_slices != 4 &&
        opt.row_slices != 8)
        return STC_ERR_INVALID_ARG;
    if (opt.replay_ctas < 0) return STC_ERR_INVALID_ARG;
    if (opt.gate_rho_dense == 0) opt.gate_rho_dense = 0.90;
    if (opt.gate_phi_fill == 0) opt.gate_phi_fill = 2.0;
    if (opt.gate_rho_semi == 0) opt.gate_rho_semi = 0.15;
    if (opt.gate_sigma_skew == 0) opt.gate_sigma_skew = 20.0;

    int threads = opt.host_threads;
    if (threads <= 0) threads = int(std::min<unsigned>(32, std::max<unsigned>(1, std::thread::hardware_concurrency())));
    threads = std::min(threads, 256);

    auto P = std::make_unique<stc_plan>();
    P->n = n; P->nb = opt.nb; P->nt = (n + opt.nb - 1) / opt.nb; P->nnzA = Ap[n];
    P->opt = opt;
    P->opt.perm = nullptr;

    // ---- ordering (Sec. 3) ----
    int ord = opt.ordering;
    if (ord == STC_ORDER_GIVEN) {
        if (!opt.perm) return STC_ERR_INVALID_ARG;
        P->perm.assign(opt.perm, opt.perm + n);
        vector<char> seen(n, 0);
        for (int64_t v : P->perm) {
            if (v < 0 || v >= n || seen[v]) return STC_ERR_INVALID_ARG;
            seen[v] = 1;
        }
    } else if (ord == STC_ORDER_NATURAL) {
        P->perm.resize(n);
        std::iota(P->perm.begin(), P->perm.end(), 0);
    } else if (ord == STC_ORDER_ND || (ord == STC_ORDER_AUTO && coords)) {
        rc = order_nd(n, coords, opt.nd_leaf, P->perm);
        if (rc) return rc;
        ord = STC_ORDER_ND;
    } else if (ord == STC_ORDER_RCM || ord == STC_ORDER_AUTO) {
        order_rcm(n, Ap, Ai, P->perm);
        ord = STC_ORDER_RCM;
    } else {
        return STC_ERR_INVALID_ARG;
    }
    vector<int64_t> iperm(n);
    for (int64_t k = 0; k < n; ++k) iperm[P->perm[k]] = k;

    // ---- symbolic factorization ----
    vector<int64_t> rp;
    vector<int32_t> rcv;
    permuted_rows(n, Ap, Ai, iperm, rp, rcv, threads);
    symbolic(n, rp, rcv, P->parent, P->Lp, P->Li, threads);
    if (ord == STC_ORDER_AUTO) ord = STC_ORDER_RCM;
    // AUTO without coordinates: keep the natural order when RCM does not reduce the fill
    if (opt.ordering == STC_ORDER_AUTO && !coords) {
        vector<int64_t> idp(n), par2, Lp2;
        stc::RowIndexVec Li2;
        std::iota(idp.begin(), idp.end(), 0);
        permuted_rows(n, Ap, Ai, idp, rp, rcv, threads);
        symbolic(n, rp, rcv, par2, Lp2, Li2, threads);
        if (Lp2[n] <= P->Lp[n]) {
            P->perm = idp; iperm = idp; P->parent.swap(par2); P->Lp.swap(Lp2); P->Li.swap(Li2);
            ord = STC_ORDER_NATURAL;
        }
    }
    P->ordering = ord;
    rp.clear(); rp.shrink_to_fit(); rcv.clear(); rcv.shrink_to_fit();
    for (int64_t j = 0; j < n; ++j) {
        double c = double(P->Lp[j + 1] - P->Lp[j]);
        P->flops_alg += c * c;
    }

    // ---- features and selector (Sec. 5.1): computed on the structural tile map ----
    P->route_exec = STC_ROUTE_SEMISPARSE;
    rc = build_tiles(*P, threads);  // structural pass (semisparse storage)
    if (rc) return rc;
    {
        double sum = 0; int64_t cnt = 0;
        for (size_t t = 0; t < P->tiles.size(); ++t)
            if (P->tiles[t].I != P->tiles[t].J) { sum += double(P->nact[t]) / double(P->nb); cnt++; }
        P->rho = cnt ? sum / cnt : 1.0;
        P->phi = double(P->Lp[n]) / double(P->nnzA);
        double mx = 0;
        for (int64_t j = 0; j < n; ++j) mx = std::max(mx, double(P->Lp[j + 1] - P->Lp[j]));
        P->sigma = mx / (double(P->Lp[n]) / double(n));
        int sel;
        if (P->rho >= opt.gate_rho_dense) sel = STC_ROUTE_DENSE;
        else if (P->phi > opt.gate_phi_fill) sel = STC_ROUTE_SUPERNODAL;
        else if (P->rho >= opt.gate_rho_semi || P->sigma >= opt.gate_sigma_skew) sel = STC_ROUTE_SEMISPARSE;
        else sel = STC_ROUTE_SUPERNODAL;
        P->route_selected = sel;
        P->route_exec = opt.force_route != STC_ROUTE_AUTO ? opt.force_route : sel;
    }
    if (P->route_exec == STC_ROUTE_DENSE) {  // rebuild storage as full tiles
        P->tiles.clear(); P->nact.clear(); P->aoff_struct.clear(); P->aind_struct.clear();
        P->contig.clear(); P->full.clear(); P->saind.clear(); P->stored_entries = 0;
        rc = build_tiles(*P, threads);
        if (rc) return rc;
    }
    build_alg1(*P);

    // ---- value map (a1), padding identity, CSC map of L ----
    // columns of A (and of L below) in chunks of kColChunk, each chunk's entries written once
    constexpr int64_t kColChunk = 2048;
    const int64_t ncc = (n + kColChunk - 1) / kColChunk;
    std::atomic<bool> unmapped{false};
    P->value_map.resize(P->nnzA);
    P->vdiag.resize(P->nnzA);
    P->arow.resize(P->nnzA);
    P->acol.resize(P->nnzA);
    parallel_chunks(threads, ncc, [&](int64_t c, int) {
        for (int64_t j = c * kColChunk; j < std::min(n, (c + 1) * kColChunk); ++j)
            for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) {
                int64_t a = iperm[Ai[p]], b = iperm[j];
                int64_t off = entry_offset(*P, std::max(a, b), std::min(a, b));
                if (off < 0) unmapped = true;
                P->value_map[p] = off;
                P->vdiag[p] = Ai[p] == j;
                P->arow[p] = (int32_t)Ai[p];
                P->acol[p] = (int32_t)j;
            }
    });
    if (unmapped) return STC_ERR_INVALID_PATTERN;
    {
        const stc::DTile& D = P->tiles[P->diag_tile[P->nt - 1]];
        for (int64_t r = D.sw; r < P->nb; ++r)
            P->pad_diag.push_back(D.kind == stc::TILE_DIAG_BAND ? D.off + D.kd + r * (D.kd + 1)
                                                                 : D.off + r + r * P->nb);
    }
    // rows of a column ascend, so its tiles are met in order: a cursor replaces the lookup
    P->csc_map.resize(P->Lp[n]);
    parallel_chunks(threads, P->nt, [&](int64_t J, int) {
        const int32_t tend = P->colstart[J + 1];
        for (int64_t j = J * P->nb; j < std::min(n, (J + 1) * P->nb); ++j) {
            int32_t t = P->colstart[J];
            for (int64_t q = P->Lp[j]; q < P->Lp[j + 1]; ++q) {
                const int64_t r = P->Li[q], I = r / P->nb;
                while (t < tend && P->tiles[t].I < I) ++t;
                int64_t off = -1;
                if (t < tend && P->tiles[t].I == I)
                    off = tile_entry_offset(*P, P->tiles[t], int(r - I * P->nb), int(j - J * P->nb));
                if (off < 0) unmapped = true;
                P->csc_map[q] = off;
            }
        }
    });
    if (unmapped) return STC_ERR_INVALID_PATTERN;
    // ---- selected inverse: stored-index lookup, tasks in reverse block-column order ----
    P->sinv.assign(P->tiles.size() * (size_t)P->nb, (int16_t)-1);
    for (size_t t = 0; t < P->tiles.size(); ++t) {
        const stc::DTile& T = P->tiles[t];
        int16_t* row = P->sinv.data() + t * P->nb;
        if (T.I == T.J) {
            for (int c = 0; c < T.sw; ++c) row[c] = (int16_t)c;
        } else {
            for (int s2 = 0; s2 < T.sw; ++s2) row[T.c0 >= 0 ? T.c0 + s2 : P->saind[T.aoff + s2]] = (int16_t)s2;
        }
    }
    for (int64_t k = P->nt - 1; k >= 0; --k) {
        const int32_t dk = P->diag_tile[k];
        for (int32_t o = P->colstart[k]; o < P->colstart[k + 1]; ++o) {
            const stc::DTile& O = P->tiles[o];
            if (O.I == O.J) continue;
            stc::DSTask t{};
            t.kind = stc::TASK_SOFF; t.tile = o; t.diag = dk; t.r0 = O.r0; t.r1 = O.r1;
            t.cbeg = (int32_t)P->scons.size();
            for (int32_t q = P->colstart[k]; q < P->colstart[k + 1]; ++q) {
                const stc::DTile& Jt = P->tiles[q];
                if (Jt.I == Jt.J) continue;
                const int64_t j = Jt.I, m = O.I;
                stc::DSCon c{};
                c.ltile = q;
                if (j == m) { c.stile = P->diag_tile[m]; c.mode = stc::SCON_DIAG; }
                else if (m > j) { c.stile = P->tile_id(m, j); c.mode = stc::SCON_MJ; }
                else { c.stile = P->tile_id(j, m); c.mode = stc::SCON_JM; }
                if (c.stile < 0) continue;  // structurally zero block: no contribution
                P->scons.push_back(c);
            }
            t.cend = (int32_t)P->scons.size();
            P->stasks.push_back(t);
        }
        stc::DSTask d{};
        d.kind = stc::TASK_SDIAG; d.tile = dk; d.diag = dk; d.r0 = 0; d.r1 = (int32_t)P->nb;
        d.cbeg = (int32_t)P->scons.size();
        for (int32_t q = P->colstart[k]; q < P->colstart[k + 1]; ++q) {
            if (P->tiles[q].I == P->tiles[q].J) continue;
            stc::DSCon c{};
            c.ltile = q; c.stile = q; c.mode = stc::SCON_OWN;
            P->scons.push_back(c);
        }
        d.cend = (int32_t)P->scons.size();
        P->stasks.push_back(d);
    }
    stc::TaskSet* ts = P->taskset(1);
    P->flops_tile = 2.0 * ts->fma_exec;
    if (P->route_exec == STC_ROUTE_SUPERNODAL) {  // Sec. 5.4 layout, built now: it sizes the factor
        const stc::SnPlan& S = P->supernodal();
        P->flops_tile = 2.0 * S.fma_exec;
    }
    P->analyze_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = P.release();
    return STC_OK;
}

extern "C" int stc_analyze(int64_t n, const int64_t* colptr, const int64_t* rowind,
                           const double* coords, const stc_options* opt, stc_plan** plan_out) {
    try {
        return analyze_impl(n, colptr, rowind, coords, opt, plan_out);
    } catch (const std::bad_alloc&) {
        return STC_ERR_OUT_OF_MEMORY;
    } catch (...) {
        return STC_ERR_INVALID_ARG;
    }
}

static int plan_info_impl(const stc_plan* P, stc_plan_info* o);
extern "C" int stc_plan_info_get(const stc_plan* P, stc_plan_info* o) {
    try {
        return plan_info_impl(P, o);
    } catch (const std::bad_alloc&) {
        return STC_ERR_OUT_OF_MEMORY;
    } catch (...) {
        return STC_ERR_INVALID_ARG;
    }
}
static int plan_info_impl(const stc_plan* P, stc_plan_info* o) {
    if (!P || !o) return STC_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->n = P->n; o->nb = P->nb; o->nt = P->nt; o->ntiles = (int64_t)P->tiles.size();
    o->nnzA = P->nnzA; o->nnzL = P->Lp[P->n];
    o->stored_entries = P->route_exec == STC_ROUTE_SUPERNODAL ? P->supernodal().stored : P->stored_entries;
    o->factor_doubles = P->item_doubles();
    o->route_selected = P->route_selected; o->route_executed = P->route_exec;
    o->ordering = P->ordering;
    o->phi = P->phi; o->rho = P->rho; o->sigma = P->sigma;
    o->ntasks_alg1 = (int64_t)P->alg1.size() / 4;
    o->n_potrf = P->n_potrf; o->n_syrk = P->n_syrk; o->n_trsm = P->n_trsm; o->n_gemm = P->n_gemm;
    o->flops_alg = P->flops_alg; o->flops_tile = P->flops_tile;
    o->analyze_seconds = P->analyze_seconds;
    return STC_OK;
}

static int plan_export_impl(const stc_plan* P, int what, void* buf, size_t* bytes) {
    if (!P || !bytes) return STC_ERR_INVALID_ARG;
    vector<int64_t> tmp;
    const void* src = nullptr;
    size_t sz = 0;
    switch (what) {
        case STC_EXPORT_PERM: src = P->perm.data(); sz = P->perm.size() * 8; break;
        case STC_EXPORT_ETREE: src = P->parent.data(); sz = P->parent.size() * 8; break;
        case STC_EXPORT_LP: src = P->Lp.data(); sz = P->Lp.size() * 8; break;
        case STC_EXPORT_LI:
            tmp.assign(P->Li.begin(), P->Li.end()); src = tmp.data(); sz = tmp.size() * 8; break;
        case STC_EXPORT_TILES:
            for (size_t t = 0; t < P->tiles.size(); ++t) {
                const auto& T = P->tiles[t];
                int64_t f[9] = {T.I, T.J, P->nact[t], P->aoff_struct[t], P->contig[t], P->full[t],
                                T.I == T.J ? (int64_t)0 : (int64_t)-1, 0, 0};
                if (T.I == T.J) {  // structural kd (storage kd may be n_b-1 on the dense route)
                    int64_t kd = 0, r0 = P->nb, r1 = 0;
                    const int64_t c0 = T.J * P->nb, c1 = std::min(P->n, c0 + P->nb);
                    for (int64_t j = c0; j < c1; ++j)
                        for (int64_t q = P->Lp[j]; q < P->Lp[j + 1] && P->Li[q] < c1; ++q) {
                            kd = std::max<int64_t>(kd, P->Li[q] - j);
                            r0 = std::min<int64_t>(r0, P->Li[q] - c0);
                            r1 = std::max<int64_t>(r1, P->Li[q] - c0 + 1);
                        }
                    f[6] = kd; f[7] = r0; f[8] = r1;
                } else {
                    int64_t r0 = P->nb, r1 = 0;  // structural row extent
                    const int64_t c0 = T.J * P->nb, c1 = std::min(P->n, c0 + P->nb);
                    const int64_t lo = (int64_t)T.I * P->nb, hi = lo + P->nb;
                    for (int64_t j = c0; j < c1; ++j) {
                        const int32_t* b = P->Li.data() + P->Lp[j];
                        const int32_t* e = P->Li.data() + P->Lp[j + 1];
                        const int32_t* x = std::lower_bound(b, e, (int32_t)lo);
                        if (x != e && *x < hi) {
                            r0 = std::min<int64_t>(r0, *x - lo);
                            const int32_t* y = std::lower_bound(x, e, (int32_t)hi);
                            r1 = std::max<int64_t>(r1, *(y - 1) - lo + 1);
                        }
                    }
                    f[7] = r0; f[8] = r1;
                }
                tmp.insert(tmp.end(), f, f + 9);
            }
            src = tmp.data(); sz = tmp.size() * 8;
            break;
        case STC_EXPORT_AIND:
            tmp.assign(P->aind_struct.begin(), P->aind_struct.end()); src = tmp.data(); sz = tmp.size() * 8;
            break;
        case STC_EXPORT_TASKS: src = P->alg1.data(); sz = P->alg1.size() * 8; break;
        case STC_EXPORT_VALUE_MAP: src = P->value_map.data(); sz = P->value_map.size() * 8; break;
        case STC_EXPORT_TILE_OFFSETS:
            for (const auto& T : P->tiles) tmp.push_back(T.off);
            src = tmp.data(); sz = tmp.size() * 8;
            break;
        case STC_EXPORT_CHUNK_EXTENTS: {
            const int groups = stc::kMaxNb / stc::kExtW;
            tmp.assign(P->tiles.size() * groups * 2, -1);
            for (size_t t = 0; t < P->tiles.size(); ++t) {
                const auto& T = P->tiles[t];
                if (T.xoff < 0) continue;
                for (int q = 0; q * stc::kExtW < T.sw; ++q) {
                    tmp[(t * groups + q) * 2] = P->cext[2 * (T.xoff + q)];
                    tmp[(t * groups + q) * 2 + 1] = P->cext[2 * (T.xoff + q) + 1];
                }
            }
            src = tmp.data(); sz = tmp.size() * 8;
            break;
        }
        case STC_EXPORT_SN_NODES:
        case STC_EXPORT_SN_ROWS:
        case STC_EXPORT_SN_CELLS:
        case STC_EXPORT_SN_TASKS:
        case STC_EXPORT_SN_DEV_CELLS:
        case STC_EXPORT_SN_DEV_TASKS:
        case STC_EXPORT_SN_DEV_UPDS:
        case STC_EXPORT_SN_DEV_MAPS:
        case STC_EXPORT_SN_VALUE_MAP:
        case STC_EXPORT_SN_CSC_MAP:
        case STC_EXPORT_SN_SEL_TASKS:
        case STC_EXPORT_SN_SEL_CONS:
        case STC_EXPORT_SN_CELL_ROWOFF: {
            const stc::SnPlan& S = P->supernodal();
            const int64_t nsn = (int64_t)S.first.size() - 1;
            if (what == STC_EXPORT_SN_NODES) {
                for (int64_t s = 0; s < nsn; ++s) {
                    const int64_t f[4] = {S.first[s], S.first[s + 1] - S.first[s], S.rptr[s + 1] - S.rptr[s], S.off[s]};
                    tmp.insert(tmp.end(), f, f + 4);
                }
            } else if (what == STC_EXPORT_SN_ROWS) {
                tmp.assign(S.rows.begin(), S.rows.end());
            } else if (what == STC_EXPORT_SN_CELLS) {
                tmp.assign(S.cells.begin(), S.cells.end());
            } else if (what == STC_EXPORT_SN_TASKS) {
                tmp.assign(S.tasks.begin(), S.tasks.end());
            } else if (what == STC_EXPORT_SN_DEV_CELLS) {
                for (const stc::SnDevCell& c : S.dcells) {
                    const int64_t f[7] = {c.off, c.ld, c.h, c.w, c.I, c.J, c.nslices};
                    tmp.insert(tmp.end(), f, f + 7);
                }
            } else if (what == STC_EXPORT_SN_DEV_TASKS) {
                for (const stc::SnDevTask& t : S.dtasks) {
                    const int64_t f[8] = {t.kind, t.cell, t.diag, t.ubeg, t.uend, t.rs0, t.rs1, t.slice};
                    tmp.insert(tmp.end(), f, f + 8);
                }
            } else if (what == STC_EXPORT_SN_DEV_UPDS) {
                for (const stc::SnDevUpd& u : S.dupds) {
                    const int64_t f[7] = {u.a, u.b, u.ar0, u.ar1, u.rmap, u.cmap, u.klen};
                    tmp.insert(tmp.end(), f, f + 7);
                }
            } else if (what == STC_EXPORT_SN_DEV_MAPS) {
                tmp.assign(S.maps.begin(), S.maps.end());
            } else if (what == STC_EXPORT_SN_VALUE_MAP) {
                tmp.assign(S.value_map.begin(), S.value_map.end());
            } else if (what == STC_EXPORT_SN_SEL_TASKS) {
                for (const stc::SnSTask& t : S.stasks) {
                    const int64_t f[7] = {t.kind, t.cell, t.diag, t.cbeg, t.cend, t.rs0, t.rs1};
                    tmp.insert(tmp.end(), f, f + 7);
                }
            } else if (what == STC_EXPORT_SN_SEL_CONS) {
                for (const stc::SnSCon& c : S.scons) {
                    const int64_t f[3] = {c.lcell, c.scell, c.mode};
                    tmp.insert(tmp.end(), f, f + 3);
                }
            } else if (what == STC_EXPORT_SN_CELL_ROWOFF) {
                tmp.assign(S.cell_rowoff.begin(), S.cell_rowoff.end());
            } else {
                tmp.assign(S.csc_map.begin(), S.csc_map.end());
            }
            src = tmp.data(); sz = tmp.size() * 8;
            break;
        }
        default: return STC_ERR_INVALID_ARG;
    }
    if (!buf) { *bytes = sz; return STC_OK; }
    if (*bytes < sz) { *bytes = sz; return STC_ERR_BUFFER_TOO_SMALL; }
    if (sz) std::memcpy(buf, src, sz);
    *bytes = sz;
    return STC_OK;
}

static int taskset_export_impl(const stc_plan* P, int32_t slices, int bl_order, int what, void* buf,
                               size_t* bytes) {
    if (!P || !bytes) return STC_ERR_INVALID_ARG;
    if (slices != 1 && slices != 2 && slices != 4 && slices != 8) return STC_ERR_INVALID_ARG;
    // task sets are built on demand under the plan's lock, as on the first factorization
    const stc::TaskSet* ts = const_cast<stc_plan*>(P)->taskset(slices, (bl_order & 1) != 0, (bl_order & 2) != 0);
    vector<int64_t> tmp;
    switch (what) {
        case STC_TASKSET_TASKS:
            for (const stc::DTask& t : ts->tasks) {
                const int64_t f[13] = {t.kind, t.tile, t.diag, t.ubeg, t.uend, t.rs0, t.rs1,
                                       t.tr0, t.tr1, t.own_wait, t.slice, ts->slice_h, t.fill};
                tmp.insert(tmp.end(), f, f + 13);
            }
            break;
        case STC_TASKSET_UPDS:
            for (const stc::DUpd& u : ts->upds) {
                const int64_t f[10] = {u.a, u.b, u.kmap, u.klen, u.ka0, u.kb0, u.ra0, u.ra1, u.oc0, u.oc1};
                tmp.insert(tmp.end(), f, f + 10);
            }
            break;
        case STC_TASKSET_IMAP: tmp.assign(ts->imap.begin(), ts->imap.end()); break;
        case STC_TASKSET_TILES:
            for (size_t t = 0; t < P->tiles.size(); ++t) {
                const stc::DTile& T = P->tiles[t];
                const int64_t f[13] = {T.off, T.I, T.J, T.kind, T.sw, T.c0, T.aoff, T.kd, T.r0, T.r1,
                                       ts->nfinal[t], T.pd_slot, T.xoff};
                tmp.insert(tmp.end(), f, f + 13);
            }
            break;
        case STC_TASKSET_SAIND: tmp.assign(P->saind.begin(), P->saind.end()); break;
        case STC_TASKSET_CEXT: tmp.assign(P->cext.begin(), P->cext.end()); break;
        case STC_TASKSET_CSC_MAP: tmp.assign(P->csc_map.begin(), P->csc_map.end()); break;
        case STC_TASKSET_PAD_DIAG: tmp.assign(P->pad_diag.begin(), P->pad_diag.end()); break;
        default: return STC_ERR_INVALID_ARG;
    }
    const size_t sz = tmp.size() * 8;
    if (!buf) { *bytes = sz; return STC_OK; }
    if (*bytes < sz) { *bytes = sz; return STC_ERR_BUFFER_TOO_SMALL; }
    if (sz) std::memcpy(buf, tmp.data(), sz);
    *bytes = sz;
    return STC_OK;
}

extern "C" int stc_plan_export_taskset(const stc_plan* P, int32_t slices, int bl_order, int what, void* buf,
                                       size_t* bytes) {
    try {
        return taskset_export_impl(P, slices, bl_order, what, buf, bytes);
    } catch (const std::bad_alloc&) {
        return STC_ERR_OUT_OF_MEMORY;
    } catch (...) {
        return STC_ERR_INVALID_PATTERN;
    }
}

extern "C" int stc_plan_export(const stc_plan* P, int what, void* buf, size_t* bytes) {
    try {
        return plan_export_impl(P, what, buf, bytes);
    } catch (const std::bad_alloc&) {
        return STC_ERR_OUT_OF_MEMORY;
    } catch (...) {
        return STC_ERR_INVALID_PATTERN;
    }
}
