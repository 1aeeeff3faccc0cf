// plan_io.cpp -- saving and loading an analysed plan.
//
// The analysis is the artefact that the repeated factorizations reuse (Sec. 6.6: analyze
// once, factorize many times); saving it lets another process, or a later run, skip
// stc_analyze.  The blob holds every host array of the plan; task sets, the supernodal
// layout and the device copies are rebuilt on first use, as after stc_analyze.
//
// Layout (native little-endian; x86-64 and AArch64 agree):
//   "STCPLAN1" | u32 version | u32 0 | u64 payload bytes | u64 FNV-1a 64 of the payload |
//   payload: scalars, then each array as (u64 element count, raw elements)
// Loading checks the magic, version, size, checksum and the array lengths against the
// plan's dimensions, so a truncated or corrupted blob is refused rather than used.
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "plan.hpp"

using std::int32_t;
using std::int64_t;
using std::uint64_t;
using std::vector;

namespace {

constexpr char kMagic[8] = {'S', 'T', 'C', 'P', 'L', 'A', 'N', '1'};
constexpr uint32_t kVersion = 2;
constexpr size_t kHeader = 8 + 4 + 4 + 8 + 8;

uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct Writer {
    vector<unsigned char> out;
    void raw(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        out.insert(out.end(), c, c + n);
    }
    template <class T> void put(const T& v) { raw(&v, sizeof(T)); }
    template <class T, class A> void vec(const vector<T, A>& v) {
        put<uint64_t>(v.size());
        if (!v.empty()) raw(v.data(), v.size() * sizeof(T));
    }
};

struct Sizer {  // the Writer's byte count without the copy
    size_t bytes = 0;
    template <class T> void put(const T&) { bytes += sizeof(T); }
    template <class T, class A> void vec(const vector<T, A>& v) { bytes += 8 + v.size() * sizeof(T); }
};

struct Reader {
    const unsigned char* p;
    size_t left;
    bool ok = true;
    bool raw(void* dst, size_t n) {
        if (!ok || n > left) return ok = false;
        if (n) std::memcpy(dst, p, n);
        p += n;
        left -= n;
        return true;
    }
    template <class T> bool get(T& v) { return raw(&v, sizeof(T)); }
    template <class T, class A> bool vec(vector<T, A>& v) {
        uint64_t cnt = 0;
        if (!get(cnt)) return false;
        if (cnt > left / sizeof(T)) return ok = false;
        v.resize(cnt);
        return raw(v.data(), cnt * sizeof(T));
    }
};

// Every array of the plan, in one fixed order shared by both directions (PL is
// `const stc_plan` when saving).
template <class IO, class PL>
void fields(IO& io, PL& P) {
    io.vec(P.perm); io.vec(P.parent); io.vec(P.Lp); io.vec(P.Li);
    io.vec(P.tiles); io.vec(P.nact); io.vec(P.aoff_struct); io.vec(P.aind_struct);
    io.vec(P.contig); io.vec(P.full); io.vec(P.saind); io.vec(P.cext);
    io.vec(P.colstart); io.vec(P.diag_tile); io.vec(P.rowstart); io.vec(P.rowtiles);
    io.vec(P.alg1); io.vec(P.value_map); io.vec(P.pad_diag); io.vec(P.csc_map);
    io.vec(P.sinv); io.vec(P.stasks); io.vec(P.scons); io.vec(P.vdiag);
    io.vec(P.arow); io.vec(P.acol);
}

template <class IO, class PL>
void scalars(IO& io, PL& P) {
    io.put(P.n); io.put(P.nb); io.put(P.nt); io.put(P.nnzA);
    io.put(P.opt);
    io.put(P.route_selected); io.put(P.route_exec); io.put(P.ordering);
    io.put(P.phi); io.put(P.rho); io.put(P.sigma); io.put(P.analyze_seconds);
    io.put(P.stored_entries); io.put(P.factor_doubles); io.put(P.npartials); io.put(P.partial_off);
    io.put(P.n_potrf); io.put(P.n_syrk); io.put(P.n_trsm); io.put(P.n_gemm);
    io.put(P.flops_alg); io.put(P.flops_tile);
}

struct GetAdapter {  // Reader with the Writer's put/vec names
    Reader& r;
    template <class T> void put(T& v) { r.get(v); }
    template <class T, class A> void vec(vector<T, A>& v) { r.vec(v); }
};

// A loaded plan is handed to kernels that index its arrays without further checks, so
// every length, index and offset is checked against the plan's dimensions: each tile's
// whole footprint (from its kind, stored width and band) lies inside the tile area, the
// partials fit the item stride, every stored-column index, extent, map entry and tile id
// is in range, perm is a permutation and the etree and L's structure are well formed.
// The checksum only catches damage in transit; this catches a blob that is intact but
// inconsistent (edited, or written by a build with another layout).
bool in(int64_t v, int64_t lo, int64_t hi) { return v >= lo && v < hi; }

bool consistent(const stc_plan& P) {
    const int64_t n = P.n, nt = P.nt, nb = P.nb;
    const size_t nT = P.tiles.size();
    if (n <= 0 || nb < 8 || nb > stc::kMaxNb || nb % 8 || nt != (n + nb - 1) / nb) return false;
    if (P.nnzA < n || P.npartials != nt || P.partial_off < 0 || P.partial_off + P.npartials > P.factor_doubles)
        return false;
    if ((int64_t)P.perm.size() != n || (int64_t)P.parent.size() != n) return false;
    {
        vector<char> seen(n, 0);
        for (int64_t v : P.perm) {
            if (!in(v, 0, n) || seen[v]) return false;
            seen[v] = 1;
        }
    }
    for (int64_t j = 0; j < n; ++j)
        if (P.parent[j] != -1 && !in(P.parent[j], j + 1, n)) return false;
    if ((int64_t)P.Lp.size() != n + 1 || P.Lp[0] != 0 || (int64_t)P.Li.size() != P.Lp[n]) return false;
    for (int64_t j = 0; j < n; ++j) {
        if (P.Lp[j + 1] <= P.Lp[j] || P.Li[P.Lp[j]] != j) return false;  // diagonal first
        for (int64_t q = P.Lp[j] + 1; q < P.Lp[j + 1]; ++q)
            if (!in(P.Li[q], P.Li[q - 1] + 1, n)) return false;
    }
    if (P.nact.size() != nT || P.aoff_struct.size() != nT || P.contig.size() != nT || P.full.size() != nT)
        return false;
    for (size_t t = 0; t < nT; ++t)
        if (P.nact[t] < 0 || P.nact[t] > nb || P.aoff_struct[t] < 0 ||
            (size_t)P.aoff_struct[t] + (size_t)P.nact[t] > P.aind_struct.size())
            return false;
    if ((int64_t)P.colstart.size() != nt + 1 || (int64_t)P.diag_tile.size() != nt) return false;
    if ((int64_t)P.rowstart.size() != nt + 1 || P.colstart[0] != 0 || P.colstart[nt] != (int32_t)nT) return false;
    if (P.rowstart[0] != 0 || (size_t)P.rowstart[nt] != P.rowtiles.size()) return false;
    for (int64_t k = 0; k < nt; ++k)
        if (P.colstart[k + 1] < P.colstart[k] || P.rowstart[k + 1] < P.rowstart[k]) return false;
    if ((int64_t)P.value_map.size() != P.nnzA || (int64_t)P.vdiag.size() != P.nnzA ||
        (int64_t)P.arow.size() != P.nnzA || (int64_t)P.acol.size() != P.nnzA)
        return false;
    for (int64_t e = 0; e < P.nnzA; ++e)
        if (!in(P.arow[e], 0, n) || !in(P.acol[e], 0, n) || (P.vdiag[e] != 0 && P.vdiag[e] != 1)) return false;
    if ((int64_t)P.csc_map.size() != P.Lp[n] || P.sinv.size() != nT * (size_t)nb) return false;
    for (int16_t v : P.sinv)
        if (!in(v, -1, nb)) return false;
    for (int16_t v : P.saind)
        if (!in(v, 0, nb)) return false;
    for (int16_t v : P.cext)
        if (!in(v, 0, nb + 1)) return false;
    if (P.route_exec != STC_ROUTE_DENSE && P.route_exec != STC_ROUTE_SEMISPARSE &&
        P.route_exec != STC_ROUTE_SUPERNODAL)
        return false;
    for (const stc::DTile& T : P.tiles) {
        if (!in(T.I, 0, nt) || !in(T.J, 0, nt) || T.I < T.J) return false;
        if (T.sw < 0 || T.sw > nb || T.r0 < 0 || T.r1 > nb || T.r0 > T.r1) return false;
        int64_t size;
        if (T.kind == stc::TILE_OFF) {
            if (T.I == T.J || T.pd_slot != -1) return false;
            size = nb * (int64_t)T.sw;
            if (T.c0 >= 0 ? T.c0 + (int64_t)T.sw > nb : (T.aoff < 0 || (size_t)T.aoff + (size_t)T.sw > P.saind.size()))
                return false;
            if (T.xoff >= 0 && 2 * ((size_t)T.xoff + ((size_t)T.sw + stc::kExtW - 1) / stc::kExtW) > P.cext.size())
                return false;
        } else if (T.kind == stc::TILE_DIAG_DENSE || T.kind == stc::TILE_DIAG_BAND) {
            if (T.I != T.J || !in(T.pd_slot, 0, P.npartials) || T.xoff >= 0) return false;
            if (!in(T.kd, 0, nb)) return false;
            size = T.kind == stc::TILE_DIAG_DENSE ? nb * nb : nb * (int64_t)(T.kd + 1);
        } else {
            return false;
        }
        if (T.off < 0 || T.off + size > P.partial_off) return false;
    }
    for (int32_t t : P.rowtiles)
        if (!in(t, 0, (int64_t)nT)) return false;
    for (int32_t t : P.diag_tile)
        if (!in(t, 0, (int64_t)nT) || P.tiles[t].kind == stc::TILE_OFF) return false;
    for (const stc::DSTask& t : P.stasks)
        if (!in(t.tile, 0, (int64_t)nT) || !in(t.diag, 0, (int64_t)nT) || t.cbeg < 0 || t.cend < t.cbeg ||
            (size_t)t.cend > P.scons.size() || t.r0 < 0 || t.r1 > nb || t.r0 > t.r1)
            return false;
    for (const stc::DSCon& c : P.scons)
        if (!in(c.ltile, 0, (int64_t)nT) || !in(c.stile, 0, (int64_t)nT) || !in(c.mode, 0, 4)) return false;
    for (int64_t v : P.pad_diag)
        if (!in(v, 0, P.partial_off)) return false;
    for (int64_t v : P.value_map)
        if (!in(v, 0, P.partial_off)) return false;
    for (int64_t v : P.csc_map)
        if (!in(v, 0, P.partial_off)) return false;
    return true;
}

}  // namespace

extern "C" int stc_plan_save(const stc_plan* plan, void* buf, size_t* bytes) {
    if (!plan || !bytes) return STC_ERR_INVALID_ARG;
    try {
        const stc_plan& P = *plan;  // its options hold no perm pointer after analysis
        Sizer z;
        scalars(z, P);
        fields(z, P);
        const size_t total = kHeader + z.bytes;
        if (!buf) {
            *bytes = total;
            return STC_OK;
        }
        if (*bytes < total) {
            *bytes = total;
            return STC_ERR_BUFFER_TOO_SMALL;
        }
        Writer w;
        w.out.reserve(z.bytes);
        scalars(w, P);
        fields(w, P);
        unsigned char* o = static_cast<unsigned char*>(buf);
        const uint32_t ver = kVersion, zero = 0;
        const uint64_t len = w.out.size(), sum = fnv1a(w.out.data(), w.out.size());
        std::memcpy(o, kMagic, 8);
        std::memcpy(o + 8, &ver, 4);
        std::memcpy(o + 12, &zero, 4);
        std::memcpy(o + 16, &len, 8);
        std::memcpy(o + 24, &sum, 8);
        if (len) std::memcpy(o + kHeader, w.out.data(), len);
        *bytes = total;
        return STC_OK;
    } catch (const std::bad_alloc&) {
        return STC_ERR_OUT_OF_MEMORY;
    } catch (...) {
        return STC_ERR_INVALID_ARG;
    }
}

extern "C" int stc_plan_load(const void* buf, size_t bytes, stc_plan** plan_out) {
    if (!buf || !plan_out) return STC_ERR_INVALID_ARG;
    *plan_out = nullptr;
    try {
        const unsigned char* b = static_cast<const unsigned char*>(buf);
        if (bytes < kHeader || std::memcmp(b, kMagic, 8) != 0) return STC_ERR_INVALID_PATTERN;
        uint32_t ver = 0;
        uint64_t len = 0, sum = 0;
        std::memcpy(&ver, b + 8, 4);
        std::memcpy(&len, b + 16, 8);
        std::memcpy(&sum, b + 24, 8);
        if (ver != kVersion) return STC_ERR_UNSUPPORTED;
        if (len != bytes - kHeader || fnv1a(b + kHeader, len) != sum) return STC_ERR_INVALID_PATTERN;
        auto P = std::make_unique<stc_plan>();
        Reader r{b + kHeader, len};
        GetAdapter g{r};
        scalars(g, *P);
        fields(g, *P);
        if (!r.ok || r.left != 0 || !consistent(*P)) return STC_ERR_INVALID_PATTERN;
        P->opt.perm = nullptr;
        *plan_out = P.release();
        return STC_OK;
    } catch (const std::bad_alloc&) {
        return STC_ERR_OUT_OF_MEMORY;
    } catch (...) {
        return STC_ERR_INVALID_PATTERN;
    }
}
