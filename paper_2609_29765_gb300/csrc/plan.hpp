// plan.hpp -- internal plan structures shared by the host analysis (analyze.cpp)
// and the CUDA kernels (replay.cu).  Not part of the public ABI (include/stc.h).
#pragma once
#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <type_traits>
#include <utility>
#include <vector>

#include "stc.h"

namespace stc {

// Allocator that leaves elements uninitialised on a value-less resize: for large index
// arrays that are written in full, in parallel, right after they are sized.
template <class T>
struct UninitAlloc : std::allocator<T> {
    template <class U> struct rebind { using other = UninitAlloc<U>; };
    UninitAlloc() = default;
    template <class U> UninitAlloc(const UninitAlloc<U>&) noexcept {}
    template <class U> void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
        ::new (static_cast<void*>(p)) U;
    }
    template <class U, class... A> void construct(U* p, A&&... a) {
        ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
    }
};
using RowIndexVec = std::vector<int32_t, UninitAlloc<int32_t>>;

// ---------------------------------------------------------------------------
// Device-side descriptors (plain old data, uploaded as arrays).
// ---------------------------------------------------------------------------
enum : int32_t { TILE_OFF = 0, TILE_DIAG_DENSE = 1, TILE_DIAG_BAND = 2 };

// One stored tile of the factor (Sec. 4).  Off-diagonal tiles are column-major
// n_b x sw (stored columns at full height, zeros included, Sec. 4.1).  Dense diagonal
// tiles are column-major n_b x n_b holding L's lower triangle.  Banded diagonal tiles
// hold L^T in LAPACK upper-band packed form, (kd+1) x n_b column-major, entry
// L[r][c] (r >= c, r - c <= kd) at (kd + c - r) + r*(kd+1)  (Sec. 4.3).
struct DTile {
    int64_t off;      // offset (doubles) of the tile in one item's factor
    int32_t I, J;     // tile coordinates (row block, column block)
    int32_t kind;     // TILE_*
    int32_t sw;       // stored columns (off-diagonal) / logical width (diagonal)
    int32_t c0;       // first logical column if the stored set is contiguous, else -1
    int32_t aoff;     // offset of the stored-column list in the saind array
    int32_t kd;       // banded half-width (TILE_DIAG_BAND), n_b-1 otherwise
    int32_t r0, r1;   // structural row extent [r0, r1) inside the tile
    int32_t nfinal;   // value of the tile's completion counter once it is final
    int32_t pd_slot;  // diagonal tiles: index of the logdet partial; else -1
    int32_t xoff;     // off-diagonal tiles: first (lo, hi) pair in the chunk-extent array; else -1
};

// Structural row extent of each group of kExtW consecutive stored columns of an
// off-diagonal tile: rows outside [lo, hi) are zero in all of those columns, so a
// product over those columns can skip them (empty group: lo = n_b, hi = 0).
constexpr int kExtW = 16;
constexpr int kMaxNb = 128;  // largest tile size n_b
// Panel width of the blocked TRSM; a factored diagonal tile is published to its TRSMs
// this many columns at a time.
constexpr int kPanelW = 32;
// Completion word of an off-diagonal tile: bit q * kMaxSlices + s is set once row slice
// s has finished TRSM panel q (columns [q kPanelW, (q+1) kPanelW) of its rows are final),
// so a consumer can wait for exactly the rows and columns it reads.
constexpr int kMaxSlices = 8;
static_assert((kMaxNb / kPanelW) * kMaxSlices <= 32, "completion word holds every (panel, slice) bit");
// Completion word of a diagonal tile: its rows are factored in up to kMaxDiagSlices row
// slices (cut on multiples of kDiagGroupW rows); bit g * kMaxDiagSlices + s is set once
// slice s has made final the columns [g kDiagGroupW, (g+1) kDiagGroupW) of its rows.  The
// tile's nfinal holds every bit that will be set (a banded tile skips groups that lie
// wholly outside the band of a slice's rows).
constexpr int kDiagGroupW = 16;
constexpr int kMaxDiagSlices = 4;
static_assert((kMaxNb / kDiagGroupW) * kMaxDiagSlices <= 32, "completion word holds every (group, slice) bit");

enum : int32_t { TASK_DIAG = 0, TASK_OFF = 1, TASK_SYRK = 2, TASK_FWD = 3, TASK_FILL = 4 };

// One device task, the cases of Algorithm 1 grouped by output tile (row slice):
//   TASK_DIAG  every SYRK into (k,k), then POTRF(k)                 (unsliced)
//   TASK_SYRK  every SYRK into rows [rs0,rs1) of (k,k), then the factorization of those
//              rows: solved against the columns [0, rs0) that the earlier slices
//              publish group by group, then the Cholesky factor of the slice's own
//              diagonal block (a row-partitioned POTRF(k))          (row slice)
//   TASK_OFF   every GEMM into rows [rs0,rs1) of (m,k), then the TRSM of those rows
//   TASK_FWD   forward substitution of block row k (tile = diag = (k,k)): y_k from the
//              right-hand sides, L_kn y_n and L_kk, once they are final (only in the task
//              sets of the fused factorization + solve, for blocks no waiting diagonal task
//              hosts; see own_wait)
//   TASK_FILL  value scatter of block column k (tile = (k,k)): the column's range of the
//              factor from the values through the fill map (fused task sets that fill
//              inside the launch, for columns no waiting task hosts; see fill)
struct DTask {
    int32_t kind;
    int32_t tile;        // output tile
    int32_t diag;        // tile (k,k)
    int32_t ubeg, uend;  // range in the update array
    int32_t rs0, rs1;    // row slice of the output tile
    int32_t tr0, tr1;    // rows of the slice the TRSM touches (slice cut to r-extent)
    int32_t own_wait;    // fused task sets: on a TASK_DIAG or slice-0 TASK_SYRK, 1 + the
                         // diagonal tile of the block whose forward substitution it runs
                         // first (0: none)
    int32_t slice;       // TASK_OFF, TASK_SYRK: index of the row slice in its tile
    int32_t fill;        // fused task sets that fill inside the launch: on a slice-1
                         // TASK_SYRK, 1 + the block column whose value scatter it runs
                         // first (0: none)
};

// One SYRK (a == b) or GEMM source of a task: out -= A(rows, inner) * B(cols, inner)^T.
struct DUpd {
    int32_t a, b;        // operand tiles: (m,n) and (k,n); SYRK: both (k,n)
    int32_t kmap;        // offset of (sa, sb) int16 pairs in imap, or -1 if contiguous
    int32_t klen;        // inner length
    int32_t ka0, kb0;    // contiguous inner: first stored column in a / in b
    int32_t ra0, ra1;    // output rows touched (local rows of the output tile)
    int32_t oc0, oc1;    // output stored columns touched (GEMM); SYRK: unused
    int32_t pad[2];
};

// Selected inverse (Takahashi recurrence on the tile map), walked in reverse order.
//   TASK_SOFF  Sigma_mk = -(sum_j Sigma_(m,j) L_jk) L_kk^{-1} on the stored columns of (m,k)
//   TASK_SDIAG Sigma_kk from Z = sum_j Sigma_jk^T L_jk and the element recurrence inside
//              the diagonal tile
enum : int32_t { TASK_SOFF = 0, TASK_SDIAG = 1 };
enum : int32_t { SCON_MJ = 0, SCON_JM = 1, SCON_DIAG = 2, SCON_OWN = 3 };

struct DSTask {
    int32_t kind;
    int32_t tile;        // output tile (m,k) or (k,k)
    int32_t diag;        // tile (k,k)
    int32_t cbeg, cend;  // contributions
    int32_t r0, r1;      // output rows computed (row extent)
    int32_t pad;
};

// One contribution to a selected-inverse task.
//   SCON_MJ:   Sigma tile (m,j), m > j, times L_jk      SCON_JM: Sigma tile (j,m)^T times L_jk
//   SCON_DIAG: symmetric Sigma tile (m,m) times L_mk   SCON_OWN: Sigma_jk^T L_jk (diagonal task)
struct DSCon {
    int32_t ltile;       // L tile (j,k)
    int32_t stile;       // Sigma tile read
    int32_t mode;
    int32_t pad;
};

struct DevPlanArrays {          // device pointers of one plan's metadata
    DTile* tiles = nullptr;
    int16_t* saind = nullptr;   // stored-column -> logical-column lists
    int16_t* cext = nullptr;    // per-tile chunk row extents, (lo, hi) pairs
    DTask* tasks = nullptr;     // in queue (ASAP) order
    DUpd* upds = nullptr;
    int16_t* imap = nullptr;    // inner-dimension (sa, sb) pairs
    int64_t* value_map = nullptr;
    int64_t* pad_diag = nullptr;   // offsets set to 1.0 (padding of the ragged tile)
    int64_t* csc_map = nullptr;    // nnzL: offset of each structural L entry
    int32_t* fill_src = nullptr;   // per factor double: the A entry stored there, -1 (zero)
                                   // or -2 (padding diagonal, 1.0)
    int32_t* perm = nullptr;
    int32_t* srow_beg = nullptr;   // solve: per block row, tiles (k,n) n<k: [beg,end)
    int32_t* srow_tiles = nullptr;
    int32_t* scol_beg = nullptr;   // solve: per block column, tiles (m,k) m>k
    int32_t* scol_tiles = nullptr;
    int32_t* diag_tile = nullptr;  // per block: tile id of (k,k)
    int16_t* sinv = nullptr;       // per tile, per logical column: stored index or -1
    DSTask* stasks = nullptr;      // selected-inverse tasks
    DSCon* scons = nullptr;
    int8_t* vdiag = nullptr;       // per A entry: 1 on the diagonal
    int32_t* arow = nullptr;       // per A entry: original row, column
    int32_t* acol = nullptr;
    int device = -1;
    int32_t ntasks = 0;
};

// Host-side task list for one row-slice count.
struct TaskSet {
    int32_t slices = 1;
    std::vector<DTask> tasks;
    std::vector<DUpd> upds;
    std::vector<int16_t> imap;
    int32_t slice_h = 0;          // rows per slice of an off-diagonal tile
    bool fill_inside = false;     // fused set: the value scatter runs inside the launch
    std::vector<int32_t> nfinal;  // per tile completion target (count, or bit mask)
    std::vector<double> qkey;     // modelled start of each task (queue order)
    double period = 0.0;          // modelled time per block column
    double par = 0.0;             // modelled average parallelism (work / makespan)
    double fma = 0.0;             // modelled FMAs (queue-order cost model)
    double fma_exec = 0.0;        // FMAs the kernels execute (exact POTRF count)
    // device copies
    DTask* d_tasks = nullptr;
    DUpd* d_upds = nullptr;
    int16_t* d_imap = nullptr;
    DTile* d_tiles = nullptr;     // tiles with this set's nfinal
    int device = -1;
};

// Non-uniform supernodal tiling (Sec. 5.4), host plan.  Supernode s owns the columns
// [first[s], first[s+1]) and the rows rows[rptr[s] .. rptr[s+1]) (its own columns first,
// ascending); its panel is a dense column-major rows x width block at arena offset off[s].
// A cell (I, J, r0, r1) is the run [r0, r1) of column supernode I's rows owned by row
// supernode J; cells of I are cells[cptr[I] .. cptr[I+1]), the diagonal cell first.
enum : int32_t { SN_FACTOR = 0, SN_TRSM = 1, SN_UPDATE = 2 };
enum : int32_t { SN_T_DIAG = 0, SN_T_OFF = 1 };
constexpr int kSnSliceH = 64;
struct SnDevCell {
    int64_t off;     // arena offset of the cell's first row (column 0 of its supernode)
    int32_t ld;      // rows of the column supernode's panel (leading dimension)
    int32_t h, w;    // rows of the cell, columns of its supernode
    int32_t I, J;    // column supernode, row supernode
    int32_t nslices; // device tasks that write it
};
struct SnDevTask {
    int32_t kind;    // SN_T_DIAG or SN_T_OFF
    int32_t cell;    // target cell
    int32_t diag;    // diagonal cell of the target's column supernode
    int32_t ubeg, uend;
    int32_t rs0, rs1;  // rows of the target cell written
    int32_t slice;
};
struct SnDevUpd {
    int32_t a, b;      // source cells (K,I) and (J,I); a == b for a diagonal target
    int32_t ar0, ar1;  // rows of a used
    int32_t rmap;      // offset in maps: target row of each row of a (from row 0 of a)
    int32_t cmap;      // offset in maps: target column of each row of b
    int32_t klen;      // inner length (columns of supernode I)
    int32_t pad;
};
// Selected inverse on the supernodal layout (Takahashi's recurrence walked over the
// supernodes in reverse): an off-diagonal task computes rows [rs0, rs1) of
// Sigma(K,J) = -(sum over J's cells (K',J) of Sigma(rows of (K,J), rows of (K',J))
// L(K',J)) L_JJ^{-1}; the Sigma block comes from the diagonal cell of K (K' = K), from
// the cell (K,K') of supernode K' (K' < K) or transposed from the cell (K',K) of K
// (K' > K), rows located by searching the source cell's row list.  A diagonal task forms
// Z = sum over J's cells of Sigma(K',J)^T L(K',J) and runs the element recurrence inside
// the diagonal block.
enum : int32_t { SN_S_OFF = 0, SN_S_DIAG = 1 };
enum : int32_t { SN_SC_SAME = 0, SN_SC_LOWER = 1, SN_SC_UPPER = 2, SN_SC_OWN = 3 };
struct SnSTask {
    int32_t kind;      // SN_S_OFF or SN_S_DIAG
    int32_t cell;      // target cell
    int32_t diag;      // diagonal cell of J
    int32_t cbeg, cend;
    int32_t rs0, rs1;  // rows of the target cell written
    int32_t pad;
};
struct SnSCon {
    int32_t lcell;     // L cell (K',J)
    int32_t scell;     // Sigma cell read
    int32_t mode;      // SN_SC_*
    int32_t pad;
};
struct SnPlan {
    std::vector<int32_t> first;
    std::vector<int64_t> rptr;
    std::vector<int32_t> rows;
    std::vector<int64_t> off;
    int64_t arena = 0;           // doubles per item
    std::vector<int32_t> cells;  // 4 per cell: I, J, r0, r1
    std::vector<int32_t> cptr;
    // 4 per task: SN_FACTOR (kind, diagonal cell, -1, -1); SN_TRSM (kind, cell, -1, -1);
    // SN_UPDATE (kind, target cell (K,J), source cells (K,I) and (J,I))
    std::vector<int32_t> tasks;
    int64_t stored = 0;          // lower-trapezoid entries of all panels
    int64_t zeros = 0;           // of which structurally zero (relaxation)

    // Device form (the executor's input; the same shape as the tile route's tasks): one
    // task per diagonal cell (its updates, then POTRF) and per row slice of <= kSnSliceH
    // rows of an off-diagonal cell (its updates, then the TRSM against the diagonal
    // cell), in left-looking order.  An update subtracts A B^T, A = rows [ar0, ar1) of
    // cell a, B = all rows of cell b, inner dimension the klen columns of their column
    // supernode, from the target at rows rmap[i] (cell-local) and columns cmap[j]
    // (columns of the target's column supernode); a diagonal task keeps the lower part.
    std::vector<SnDevCell> dcells;
    std::vector<SnDevTask> dtasks;
    std::vector<SnDevUpd> dupds;
    std::vector<int16_t> maps;
    std::vector<int64_t> value_map;  // per A entry: arena offset (permuted lower entry)
    std::vector<int64_t> csc_map;    // per structural L entry: arena offset
    std::vector<int32_t> cell_cmap;  // per cell: offset in maps of its rows as columns of
                                     // its row supernode (-1 for diagonal cells)
    std::vector<int32_t> rptr_cells, row_cells;  // per row supernode J: cells (J, I), I < J
    double fma_exec = 0.0;           // FMAs of the device form (updates, POTRF, TRSM)
    std::vector<SnSTask> stasks;     // selected inverse, reverse supernode order
    std::vector<SnSCon> scons;
    std::vector<int32_t> cell_rowoff;  // per cell: offset in rows of its first row
    int32_t nsn() const { return (int32_t)first.size() - 1; }
    // item layout of the supernodal route: the arena, then one logdet partial per supernode
    int64_t poff() const { return (arena + 31) / 32 * 32; }
    int64_t item_doubles() const { return (poff() + nsn() + 31) / 32 * 32; }
};

// Device copies of a supernodal plan (uploaded on first use per device).
struct SnDev {
    SnDevCell* cells = nullptr;
    SnDevTask* tasks = nullptr;
    SnDevUpd* upds = nullptr;
    int16_t* maps = nullptr;
    int32_t* first = nullptr;       // nsn + 1
    int32_t* cell_cmap = nullptr;
    int32_t* cptr = nullptr;        // nsn + 1: cells of column supernode I (diagonal first)
    int32_t* rptr_cells = nullptr;  // nsn + 1
    int32_t* row_cells = nullptr;
    int64_t* value_map = nullptr;
    int64_t* csc_map = nullptr;
    int32_t* fill_src = nullptr;    // per arena double: the A entry stored there or -1
    SnSTask* stasks = nullptr;
    SnSCon* scons = nullptr;
    int32_t* rows = nullptr;        // the supernodes' row lists (permuted indices)
    int32_t* cell_rowoff = nullptr;
    int device = -1;
};

}  // namespace stc

// The opaque plan of the public ABI.
struct stc_plan {
    // pattern / options
    int64_t n = 0, nb = 0, nt = 0, nnzA = 0;
    stc_options opt{};
    int32_t route_selected = STC_ROUTE_SEMISPARSE, route_exec = STC_ROUTE_SEMISPARSE;
    int32_t ordering = STC_ORDER_NATURAL;
    double phi = 0, rho = 0, sigma = 0;
    double analyze_seconds = 0;
    std::vector<int64_t> perm;     // perm[k] = original index of pivot k
    std::vector<int64_t> parent;   // elimination tree of the permuted matrix
    std::vector<int64_t> Lp;       // symbolic structure of L (permuted), CSC
    stc::RowIndexVec Li;
    // tiles (block-column-major: J ascending, I ascending)
    std::vector<stc::DTile> tiles;
    std::vector<int32_t> nact;         // |A| (structural active columns)
    std::vector<int64_t> aoff_struct;  // offset into aind_struct
    std::vector<int16_t> aind_struct;  // structural active columns (exported)
    std::vector<int8_t> contig, full;
    std::vector<int16_t> saind;        // stored-column lists (indexed tiles only)
    std::vector<int16_t> cext;         // (lo, hi) row extent per kExtW stored columns
    std::vector<int32_t> colstart;     // tiles of block column J: [colstart[J], colstart[J+1])
    std::vector<int32_t> diag_tile;    // per block
    std::vector<int32_t> rowstart, rowtiles;  // per block row k: off-diagonal tiles (k,n), n asc
    int64_t stored_entries = 0;
    int64_t factor_doubles = 0;        // item stride (doubles)
    int64_t npartials = 0;             // logdet partials per item (= nt)
    int64_t partial_off = 0;           // offset (doubles) of the partials in an item
    std::vector<int64_t> alg1;         // Algorithm 1 tasks, 4 per task
    int64_t n_potrf = 0, n_syrk = 0, n_trsm = 0, n_gemm = 0;
    double flops_alg = 0, flops_tile = 0;
    std::vector<int64_t> value_map;    // nnzA
    std::vector<int64_t> pad_diag;
    std::vector<int64_t> csc_map;      // nnzL
    std::vector<int16_t> sinv;         // ntiles x nb
    std::vector<stc::DSTask> stasks;   // selected inverse, reverse block-column order
    std::vector<stc::DSCon> scons;
    std::vector<int8_t> vdiag;         // nnzA
    std::vector<int32_t> arow, acol;   // nnzA (original indices)
    // task sets by slice count, device arrays
    std::map<int32_t, std::unique_ptr<stc::TaskSet>> tasksets;
    stc::DevPlanArrays dev;
    std::mutex mu;

    // supernodal layout, built on first use from the symbolic factor (at analysis when the
    // plan executes on the supernodal route)
    mutable std::unique_ptr<stc::SnPlan> sn;
    mutable std::mutex sn_mu;
    stc::SnDev sndev;
    // library-owned workspace and selected-inverse scratch, for calls that pass none
    // (allocated on first such call, grown as needed, freed with the plan)
    void* own_ws = nullptr;
    size_t own_ws_bytes = 0;
    void* own_sig = nullptr;
    size_t own_sig_bytes = 0;
    std::mutex own_mu;
    // item stride, logdet partials offset and count of the route the plan executes
    int64_t item_doubles() const { return route_exec == STC_ROUTE_SUPERNODAL ? supernodal().item_doubles() : factor_doubles; }
    int64_t logdet_off() const { return route_exec == STC_ROUTE_SUPERNODAL ? supernodal().poff() : partial_off; }
    int64_t nlogdet() const { return route_exec == STC_ROUTE_SUPERNODAL ? supernodal().nsn() : npartials; }
    const stc::SnPlan& supernodal() const;
    void build_device_form(stc::SnPlan& S, const std::vector<int32_t>& snof,
                           const std::vector<std::vector<int32_t>>& byrow,
                           const std::function<int32_t(int32_t, int32_t)>& cell_of) const;

    int tile_id(int64_t I, int64_t J) const;  // -1 if not active
    // built on demand (host); bl_order: queue by bottom level (longest path to the end of
    // the item's DAG) instead of modelled earliest start
    // fwd: with one TASK_FWD per block (the fused factorization + forward substitution)
    stc::TaskSet* taskset(int32_t slices, bool bl_order = false, bool fwd = false);
    static int32_t taskset_key(int32_t slices, bool bl_order, bool fwd = false) {
        return (slices * 2 + (bl_order ? 1 : 0)) * 2 + (fwd ? 1 : 0);
    }
};
