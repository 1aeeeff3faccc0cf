/*
 * stc.h -- C ABI of the GB300 structure-adaptive tile Cholesky (numeric phase).
 *
 * Method: arxiv 2609.29765, "Dense Matrices Are Alike; Sparse Matrices Are Sparse in
 * Their Own Way: A Structure-Adaptive Tile Cholesky Factorization".
 *
 *   analyze   -- once per sparsity pattern, on the host (Sec. 3 ordering and symbolic
 *                factorization; Sec. 5.1 selector; Sec. 5.2 per-tile metadata, task list
 *                of Algorithm 1 and per-task scatter maps).  The interface splits a
 *                once-per-pattern analyze from a repeated factorize (Sec. 6.6).
 *   factorize -- per call, on the GPU: replay of the POTRF / SYRK / TRSM / GEMM tile
 *                tasks (Algorithm 1 executed as in Algorithm 2, with device-side
 *                dependency counters in place of the progress matrix P, Sec. 5.3) on
 *                dense tiles and on active-column tiles (Sec. 4).
 *   logdet, solve -- consume the factor where it sits (Sec. 5.4 log-determinant reuse;
 *                Sec. 6.7 solves).
 *   logdet_backward / quad_backward -- adjoints; no counterpart in the paper (it leaves
 *                selected inversion to separate work, Sec. 6.2): Takahashi selected
 *                inverse on the same tile map.
 *
 * Conventions (every entry point):
 *   - Return value: STC_OK (0) or a negative STC_ERR_* code; nothing is thrown.
 *   - Patterns are the LOWER triangle with the diagonal, CSC, int64, rows strictly
 *     ascending in each column, in the caller's original ordering.
 *   - A plan (stc_plan) is opaque, owned by the library, freed by stc_plan_destroy.
 *     It keeps a device copy of its metadata, created on first device use on the
 *     current CUDA device (that first call synchronizes the device; make it before
 *     any stream capture, or call stc_plan_upload first).
 *   - All d_* buffers are DEVICE pointers owned by the caller; all h_* / unprefixed
 *     array arguments of analyze/export are HOST pointers owned by the caller.
 *   - Device calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = legacy default stream).  Numerical failure is not an error return: it is
 *     reported per batch item in d_info (0 = success, j+1 = first non-positive pivot at
 *     global permuted column j); the item's logdet is then NaN.
 *   - Batched buffers are item-major: item b of d_values starts at b*nnzA, item b of a
 *     factor at b*stc_factor_bytes(plan,1) bytes.
 */
#ifndef STC_H
#define STC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define STC_OK 0
#define STC_ERR_INVALID_ARG (-1)     /* null pointer, bad size, bad option        */
#define STC_ERR_INVALID_PATTERN (-2) /* not lower CSC / unsorted / missing diag   */
#define STC_ERR_OUT_OF_MEMORY (-3)   /* host or device allocation failed          */
#define STC_ERR_CUDA (-4)            /* a CUDA runtime call failed                */
#define STC_ERR_TIMEOUT (-5)         /* a device dependency wait hit its limit    */
#define STC_ERR_UNSUPPORTED (-6)     /* option or size outside what is built      */
#define STC_ERR_BUFFER_TOO_SMALL (-7)

/* A short English description of a return code (STC_OK or STC_ERR_*); a static string,
 * never NULL ("unknown error" for any other value).  Host only; no counterpart in the
 * paper. */
const char* stc_strerror(int code);

/* ---- routes (Sec. 5.1) ------------------------------------------------- */
#define STC_ROUTE_AUTO (-1)
#define STC_ROUTE_DENSE 0       /* every active tile stored as a full n_b x n_b block  */
#define STC_ROUTE_SEMISPARSE 1  /* active-column tiles + banded-packed diagonal tiles */
#define STC_ROUTE_SUPERNODAL 2  /* non-uniform supernodal panels (Sec. 5.4)           */

/* ---- orderings (Sec. 3) ------------------------------------------------ */
#define STC_ORDER_AUTO 0     /* ND when coordinates are given, else best of RCM/natural */
#define STC_ORDER_NATURAL 1
#define STC_ORDER_GIVEN 2    /* stc_options.perm */
#define STC_ORDER_ND 3       /* geometric nested dissection on lattice coordinates    */
#define STC_ORDER_RCM 4      /* reverse Cuthill-McKee                                  */

typedef struct stc_options {
    int32_t nb;           /* tile size n_b; 0 = 128.  Built range 8..128, multiple of 8 */
    int32_t force_route;  /* STC_ROUTE_AUTO, _DENSE, _SEMISPARSE or _SUPERNODAL        */
    int32_t ordering;     /* STC_ORDER_*                                               */
    int32_t nd_leaf;      /* ND leaf size; 0 = 64                                      */
    const int64_t* perm;  /* host [n], for STC_ORDER_GIVEN: perm[k] = original index of
                             the k-th pivot (copied during analyze)                    */
    int32_t row_slices;   /* rows of an off-diagonal tile split into this many device
                             tasks (1,2,4,8); 0 = chosen per call from the batch size  */
    int32_t host_threads; /* host threads stc_analyze may use; 0 = all hardware threads
                             (at most 32).  The plan does not depend on this count.   */
    int64_t spin_limit;   /* polls before a device dependency wait gives up with
                             STC_ERR_TIMEOUT; 0 = default (about 10 s)                 */
    double gate_rho_dense;   /* selector gates (Table 5); 0 = default 0.90 */
    double gate_phi_fill;    /* 0 = default 2.0  */
    double gate_rho_semi;    /* 0 = default 0.15 */
    double gate_sigma_skew;  /* 0 = default 20   */
    int32_t replay_ctas;     /* CTAs of the persistent device kernels (factorize, solve,
                                selected inverse); 0 = chosen from the batch and the SM
                                count.  1 = serial replay: one CTA executes the task queue
                                strictly in queue order, the reference schedule that a
                                parallel run must reproduce bit for bit (race check).   */
    int32_t reserved1;
} stc_options;

typedef struct stc_plan stc_plan;

typedef struct stc_plan_info {
    int64_t n, nb, nt;          /* order, tile size, N_T = ceil(n/nb)                 */
    int64_t ntiles;             /* active tiles (diagonal included)                   */
    int64_t nnzA;               /* stored lower entries of A                          */
    int64_t nnzL;               /* structural non-zeros of L (diagonal included)      */
    int64_t stored_entries;     /* doubles stored for L (tiles, or the lower trapezoids
                                   of the supernodal panels), per item               */
    int64_t factor_doubles;     /* per-item factor footprint incl. logdet partials    */
    int32_t route_selected;     /* selector's choice (STC_ROUTE_*)                    */
    int32_t route_executed;     /* route the plan runs (dense, semisparse, supernodal) */
    int32_t ordering;           /* ordering used (STC_ORDER_*)                        */
    int32_t reserved0;
    double phi, rho, sigma;     /* routing features (Sec. 5.1)                        */
    int64_t ntasks_alg1;        /* Algorithm 1 tasks                                  */
    int64_t n_potrf, n_syrk, n_trsm, n_gemm;
    double flops_alg;           /* sum_j c_j^2 (c_j = column count of L)              */
    double flops_tile;          /* flops the device kernels execute (tile routes: row
                                   slice = 1; supernodal: updates, POTRF and TRSM)   */
    double analyze_seconds;     /* host wall time of stc_analyze                      */
} stc_plan_info;

/* what stc_plan_export returns (all int64 unless noted) */
#define STC_EXPORT_PERM 0       /* [n]                                               */
#define STC_EXPORT_ETREE 1      /* [n] parent of each permuted column, -1 for roots  */
#define STC_EXPORT_LP 2         /* [n+1] column pointers of L's structure            */
#define STC_EXPORT_LI 3         /* [nnzL] row indices of L's structure               */
#define STC_EXPORT_TILES 4      /* [ntiles][9]: I, J, |A|, aind offset, contiguous,
                                   full, kd (diag) or -1, row extent r0, r1           */
#define STC_EXPORT_AIND 5       /* concatenated active-column lists                  */
#define STC_EXPORT_TASKS 6      /* [ntasks][4]: Algorithm 1 (case, m, k, n), -1 = unused */
#define STC_EXPORT_VALUE_MAP 7  /* [nnzA] offset (doubles) of each A entry in a factor */
#define STC_EXPORT_TILE_OFFSETS 8 /* [ntiles] offset (doubles) of each tile's storage */
#define STC_EXPORT_CHUNK_EXTENTS 9 /* [ntiles][8][2]: for each group of 16 stored columns
                                     of an off-diagonal tile, the first and one past the
                                     last local row holding a structural entry of L in
                                     those columns (n_b, 0 if none); (-1, -1) for groups
                                     past the stored width and for diagonal tiles.  The
                                     tile products skip rows outside these extents (the
                                     paper computes on full-height columns, Sec. 4.1). */
/* The non-uniform supernodal tiling of Sec. 5.4 (host plan; built on first request from
 * the plan's ordering and symbolic factor; the numeric phase still runs on the tile
 * routes).  Fundamental supernodes, relaxed by amalgamation along contiguous etree
 * links (width <= 4 always; <= 16 / <= 48 / wider while explicit zeros stay below
 * 80 % / 10 % / 5 % of the panel's lower trapezoid; merged width <= 128), wider
 * supernodes cut into 128-column panels. */
#define STC_EXPORT_SN_NODES 10  /* [nsn][4]: first column, width, rows, panel offset in a
                                   per-item arena (doubles; rows x width column-major) */
#define STC_EXPORT_SN_ROWS 11   /* concatenated row lists (permuted indices): each
                                   supernode's own columns, then the rows below, ascending */
#define STC_EXPORT_SN_CELLS 12  /* [ncells][4]: column supernode I, row supernode J, and
                                   the run [r0, r1) of I's row list that J owns; the
                                   diagonal cell (I, I, 0, width) first for each I       */
#define STC_EXPORT_SN_TASKS 13  /* [ntasks][4], left-looking order (for each supernode J:
                                   its updates, its factor, its TRSMs):
                                   (0, diagonal cell of J, -1, -1)  FACTOR (POTRF)
                                   (1, cell (K,J), -1, -1)          TRSM against J's factor
                                   (2, cell (K,J), cell (K,I), cell (J,I))
                                                                    UPDATE L_KJ -= L_KI L_JI^T,
                                   rows and columns placed by sorted-subset scatter    */
/* The same plan in device form (the input of a supernodal executor, shaped like the
 * tile route's tasks): one task per diagonal cell (all its updates, then POTRF) and per
 * row slice of <= 64 rows of an off-diagonal cell (all its updates, then the TRSM
 * against the diagonal cell), in left-looking order.  Cell c's entry (i, k) lies at
 * arena offset off + i + k * ld.  An update subtracts A B^T, A = rows [ar0, ar1) of cell
 * a, B = all rows of cell b (inner dimension: the klen columns of their supernode), at
 * target rows maps[rmap + i] (cell-local, i counted from row 0 of a) and target columns
 * maps[cmap + j]; a diagonal task keeps the lower part. */
#define STC_EXPORT_SN_DEV_CELLS 14  /* [ncells][7]: off, ld, h, w, I, J, row slices        */
#define STC_EXPORT_SN_DEV_TASKS 15  /* [ntasks][8]: kind (0 diagonal, 1 off-diagonal slice),
                                       cell, diagonal cell, update range [ubeg, uend),
                                       rows [rs0, rs1), slice                             */
#define STC_EXPORT_SN_DEV_UPDS 16   /* [nupds][7]: a, b, ar0, ar1, rmap, cmap, klen       */
#define STC_EXPORT_SN_DEV_MAPS 17   /* the row / column position maps (int16 widened)     */
#define STC_EXPORT_SN_VALUE_MAP 18  /* [nnzA] arena offset of each entry of A             */
#define STC_EXPORT_SN_CSC_MAP 19    /* [nnzL] arena offset of each structural entry of L  */
/* The supernodal selected inverse (Takahashi's recurrence over the supernodes, in
 * reverse): an off-diagonal task computes rows [rs0, rs1) of Sigma(K,J) = -(sum over J's
 * cells (K',J) of Sigma(rows of (K,J), rows of (K',J)) L(K',J)) L_JJ^{-1}, reading Sigma
 * from the diagonal cell of K (mode 0, K' = K), from the cell (K,K') of supernode K'
 * (mode 1, K' < K) or transposed from the cell (K',K) of K (mode 2, K' > K); a diagonal
 * task sums Sigma(K',J)^T L(K',J) over J's cells (mode 3) and runs the element recurrence
 * in the diagonal block. */
#define STC_EXPORT_SN_SEL_TASKS 20  /* [ntasks][7]: kind (0 off-diagonal, 1 diagonal), cell,
                                       diagonal cell, contributions [cbeg, cend), rows
                                       [rs0, rs1)                                       */
#define STC_EXPORT_SN_SEL_CONS 21   /* [ncons][3]: L cell (K',J), Sigma cell read, mode     */
#define STC_EXPORT_SN_CELL_ROWOFF 22 /* [ncells] offset in STC_EXPORT_SN_ROWS of each cell's
                                       first row                                        */

/* Fill *opt with defaults (nb 128, auto route, auto ordering, ND leaf 64; selector gates
 * of Table 5: rho_dense 0.90, phi 2.0, rho_semi 0.15, sigma 20). */
void stc_options_default(stc_options* opt);

/* Symbolic analysis (host only; no GPU needed): the once-per-pattern analyze of Sec. 6.6
 * -- ordering and symbolic factorization (Sec. 3), features and selector (Sec. 5.1),
 * per-tile metadata, Algorithm 1's task list and the scatter maps (Sec. 5.2), and on the
 * supernodal route the supernodal layout (Sec. 5.4).
 *   n, colptr[n+1], rowind[nnz]: lower CSC pattern of A (original order).
 *   coords: optional host [n][3] lattice coordinates for geometric ND (integral values;
 *           rows with a NaN coordinate are set-aside dense rows, ordered last); NULL ok.
 *   opt: NULL = defaults.  *plan_out receives a new plan.
 * Errors: STC_ERR_INVALID_ARG, STC_ERR_INVALID_PATTERN, STC_ERR_UNSUPPORTED (nb outside
 * 8..128 or not a multiple of 8; ND without integral coordinates), STC_ERR_OUT_OF_MEMORY. */
int stc_analyze(int64_t n, const int64_t* colptr, const int64_t* rowind,
                const double* coords, const stc_options* opt, stc_plan** plan_out);

/* The plan's summary (the quantities the paper reports per matrix: features and route,
 * Sec. 5.1 and Table 1; nnz(L) and stored entries, App. C; task counts and flops).
 * Named stc_plan_info_get because stc_plan_info names its struct.  *out written. */
int stc_plan_info_get(const stc_plan* plan, stc_plan_info* out);

/* Copy one symbolic array (STC_EXPORT_*: the ordering and etree of Sec. 3, the tile map
 * and active-column lists of Sec. 4.1, kd of Sec. 4.3, Algorithm 1's tasks, the
 * supernodal layout of Sec. 5.4) into host memory, for bit-exact checks.  Call with
 * buf == NULL to read the size in bytes into *bytes; STC_ERR_BUFFER_TOO_SMALL if *bytes
 * is short. */
int stc_plan_export(const stc_plan* plan, int what, void* buf, size_t* bytes);

/* Copy one array of the device task list that stc_factorize replays (Algorithm 1's tasks
 * grouped per output tile, Sec. 5.2-5.3) with `slices` row slices per off-diagonal tile
 * (1, 2, 4 or 8; bit 0 of bl_order: queued by bottom level, as for one or two value
 * sets; bit 1: the set of stc_factorize_solve, with its forward-substitution tasks), so
 * that host-side checks can execute it.  Every entry is widened to int64.  The set is
 * built on first request, as on the first factorization that uses it. */
#define STC_TASKSET_TASKS 0     /* [ntasks][13] in queue order: kind (0 DIAG = SYRKs + POTRF,
                                   1 OFF = GEMMs + TRSM of a row slice, 2 SYRK = SYRKs into
                                   a row slice of (k,k) + the factorization of its rows,
                                   3 FWD = forward substitution of block row k, 4 FILL =
                                   value upload of block column k),
                                   output tile, diagonal tile, update range [ubeg, uend),
                                   row slice [rs0, rs1), TRSM rows [tr0, tr1), hosted
                                   forward step (1 + its diagonal tile; 0: none), slice
                                   index, slice height of the off-diagonal tiles, hosted
                                   value upload (1 + its block column; 0: none)           */
#define STC_TASKSET_UPDS 1      /* [nupds][10]: a, b (operand tiles), kmap (pair offset in
                                   the imap, -1 = contiguous inner range), klen, ka0, kb0
                                   (first stored column of a / b when contiguous), ra0, ra1
                                   (output rows), oc0, oc1 (output stored columns; SYRK
                                   slice: oc0 = first column)                               */
#define STC_TASKSET_IMAP 2      /* [npairs][2]: stored column of a and of b per inner index */
#define STC_TASKSET_TILES 3     /* [ntiles][13]: offset, I, J, kind (0 off-diagonal, 1 dense
                                   diagonal, 2 banded diagonal), stored width, first
                                   logical column if contiguous else -1, offset in the
                                   stored-column list, storage kd, row extent r0, r1,
                                   completion word once final (off-diagonal: bit
                                   q*8 + s per TRSM panel q of row slice s; diagonal: bit
                                   g*4 + s per 16-column group g of row slice s), logdet
                                   slot, extent-pair offset                              */
#define STC_TASKSET_SAIND 4     /* stored-column lists of indexed tiles                      */
#define STC_TASKSET_CEXT 5      /* (lo, hi) row extent per 16 stored columns                 */
#define STC_TASKSET_CSC_MAP 6   /* [nnzL] factor offset of each structural entry of L        */
#define STC_TASKSET_PAD_DIAG 7  /* factor offsets set to 1.0 (padding of the ragged tile)    */
int stc_plan_export_taskset(const stc_plan* plan, int32_t slices, int bl_order, int what, void* buf,
                            size_t* bytes);

/* Upload the plan's device metadata (tile or supernodal descriptors, task list, value
 * and CSC maps: the per-task offsets resolved at analysis, Sec. 5.2) to the current CUDA
 * device now (synchronous), and load the library's device module there.  Optional:
 * every device call does it on first use. */
int stc_plan_upload(stc_plan* plan);

/* Free a plan, its device copies and its own workspace (no-op on NULL). */
void stc_plan_destroy(stc_plan* plan);

/* Save / load an analysed plan (the analysis is what the repeated factorizations reuse,
 * Sec. 6.6; a saved plan lets a later process skip stc_analyze).
 * stc_plan_save writes a self-contained host blob (magic, version, size, FNV-1a
 * checksum, then every host array of the plan, native little-endian); buf == NULL reads
 * the size into *bytes; STC_ERR_BUFFER_TOO_SMALL if *bytes is short.  stc_plan_load
 * builds a new plan from such a blob (the caller keeps the buffer and destroys the plan
 * with stc_plan_destroy); task sets and device copies are rebuilt on first use.  A
 * truncated, corrupted or inconsistent blob gives STC_ERR_INVALID_PATTERN, another
 * format version STC_ERR_UNSUPPORTED, and no plan. */
int stc_plan_save(const stc_plan* plan, void* buf, size_t* bytes);
int stc_plan_load(const void* buf, size_t bytes, stc_plan** plan_out);

/* Bytes of caller-owned device memory (Sec. 3: the factor is allocated once from the
 * symbolic analysis, every tile's offset resolved in advance):
 *   factor    -- the factor of `batch` items in the route's storage (tiles, or supernodal
 *                panels), then one logdet partial per diagonal tile / supernode; item
 *                stride = the value at batch 1
 *   workspace -- dependency counters, queue head and status word used by factorize,
 *                solve, selinv and logdet_backward (contents need not be initialised).
 *
 * Workspace convention (factorize, factorize_scattered, solve, selinv, logdet_backward):
 * d_work == NULL uses a workspace owned by the plan instead, allocated on the first such
 * call and grown when a larger one is needed (that call synchronizes the device, so
 * make it before any stream capture); it is freed with the plan, every call on the plan
 * shares it, and calls that overlap on the GPU race on it.  Its status word is read with
 * stc_plan_sync_status.  The paper's interface passes no workspace (Sec. 6.6); a caller
 * that owns its memory passes d_work to keep calls on several streams independent. */
size_t stc_factor_bytes(const stc_plan* plan, int64_t batch);
size_t stc_workspace_bytes(const stc_plan* plan, int64_t batch);

/* Numeric factorization (Sec. 6.6's repeated factorize; Algorithm 1's tasks executed as
 * in Algorithm 2, Sec. 5.3, with per-tile counters in place of the progress matrix P;
 * on the supernodal route the left-looking supernodal tasks of Sec. 5.4) of `batch`
 * value sets of the plan's pattern by one persistent kernel walking the task DAG.
 *   d_values [batch][nnzA] FP64 in the original CSC order of the analyzed pattern;
 *   d_factor stc_factor_bytes(plan,batch) bytes (written); d_work
 *   stc_workspace_bytes(plan,batch) bytes, or NULL (see above); d_info [batch] int32
 *   (written).
 * A wait that exceeds spin_limit sets the workspace status to STC_ERR_TIMEOUT and the
 * kernel finishes (results then undefined); read it with stc_sync_status. */
int stc_factorize(const stc_plan* plan, const double* d_values, int64_t batch,
                  void* d_factor, void* d_work, int32_t* d_info, void* stream);

/* The two halves of stc_factorize, for callers that time or overlap them separately:
 *   stc_scatter_values      -- the value upload of Sec. 6.7 (A's entries placed into the
 *                              factor storage allocated in Sec. 3): zero the factor,
 *                              copy d_values through the plan's value map, set the
 *                              padding diagonal of a ragged last tile to 1;
 *   stc_factorize_scattered -- Algorithm 2's task replay (Sec. 5.3; Sec. 5.4 on the
 *                              supernodal route) on a factor that stc_scatter_values
 *                              filled (same arguments as stc_factorize). */
int stc_scatter_values(const stc_plan* plan, const double* d_values, int64_t batch,
                       void* d_factor, void* stream);
int stc_factorize_scattered(const stc_plan* plan, int64_t batch, void* d_factor, void* d_work,
                            int32_t* d_info, void* stream);

/* Mixed batches: several plans (patterns of different sizes), each with its own batch of
 * value sets, factorized by ONE persistent kernel launch whose queue merges the plans'
 * task lists in earliest-start order (up to STC_GROUP_MAX_PLANS plans).  No counterpart
 * in the paper beyond its motivation: INLA factorizes many matrices per fit (Sec. 1, 2),
 * and Algorithm 2's executor takes any ready task, whichever matrix it belongs to.
 * Plans of every executable route mix freely (a group holding a supernodal plan runs the
 * kernel variant that also executes supernodal tasks).
 *   stc_group_create: host + device set-up (synchronous; uploads the plans and the merged
 *     queue); plans must outlive the group; batch[p] in 1 .. 2^28-1.
 *   stc_factorize_group: d_values[p], d_factor[p], d_info[p] are host arrays of device
 *     pointers laid out as for stc_factorize with batch[p]; d_work:
 *     stc_group_workspace_bytes(group) bytes.  logdet / solve then run per plan. */
#define STC_GROUP_MAX_PLANS 8
typedef struct stc_group stc_group;
int stc_group_create(int32_t nplans, const stc_plan* const* plans, const int64_t* batch,
                     stc_group** group_out);
size_t stc_group_workspace_bytes(const stc_group* group);
int stc_factorize_group(stc_group* group, const double* const* d_values, void* const* d_factor,
                        int32_t* const* d_info, void* d_work, void* stream);
void stc_group_destroy(stc_group* group);

/* The same in one call: a group of the nplans plans (batch[p] value sets each) is
 * created, run on `stream` and destroyed; its workspace comes from the stream-ordered
 * allocator (cudaMallocAsync) and is released before returning.  Synchronous: returns
 * after the factorization has finished, with its status (STC_OK, STC_ERR_TIMEOUT, or an
 * error of group creation or of CUDA).  Buffers as for stc_factorize_group. */
int stc_factorize_mixed(int32_t nplans, const stc_plan* const* plans, const double* const* d_values,
                        const int64_t* batch, void* const* d_factor, int32_t* const* d_info, void* stream);

/* Synchronize `stream` and return the device status word of d_work: STC_OK or
 * STC_ERR_TIMEOUT (a dependency wait gave up), or STC_ERR_CUDA.  The failure reporting
 * that replaces a hung spin-wait on P (Sec. 5.3 waits without a limit). */
int stc_sync_status(const void* d_work, void* stream);
/* The same for the plan's own workspace (calls made with d_work == NULL);
 * STC_ERR_INVALID_ARG if no call has used it yet. */
int stc_plan_sync_status(const stc_plan* plan, void* stream);

/* logdet(A_b) = 2 sum_j log L_jj for every item b, from the factor where it sits (Sec.
 * 5.4: the log-determinant is reused from the factorization; Sec. 6.7 returns it from
 * the device factor): the factorization leaves sum log L_jj of each diagonal tile or
 * supernode in the item's partials, summed here in a fixed order.  d_factor from
 * stc_factorize; d_logdet [batch] FP64 (written; NaN for an item whose info != 0). */
int stc_logdet(const stc_plan* plan, const void* d_factor, int64_t batch,
               double* d_logdet, void* stream);

/* x = A^{-1} b = P^T L^{-T} L^{-1} P b for `nrhs` right-hand sides per item (Sec. 6.7:
 * the solves consume the factor where it sits on the device): forward substitution over
 * block rows (or supernodes), then backward, one persistent kernel over every (item,
 * rhs) chain with per-block completion flags.  d_b, d_x [batch][nrhs][n] FP64 (original
 * ordering; d_x written, may not alias d_b); d_work stc_workspace_bytes(plan,
 * batch*nrhs) bytes or NULL (see above). */
int stc_solve(const stc_plan* plan, const void* d_factor, int64_t batch, int64_t nrhs,
              const double* d_b, double* d_x, void* d_work, void* stream);

/* Factorization and solve in one call: stc_factorize followed by stc_solve's result,
 * with the forward substitution L y = P b (Sec. 6.7: the solves consume the factor where
 * it sits on the device) run inside the factorization's persistent launch, one task per
 * (item, block row) queued behind the factorization wavefront, so only the backward
 * substitution runs after it.  Same arguments as stc_factorize and stc_solve: d_values
 * [batch][nnzA]; d_b, d_x [batch][nrhs][n] FP64 (original ordering; d_x written, may not
 * alias d_b); d_factor and d_info written as by stc_factorize (the factor is the same to
 * the bit); d_work stc_factorize_solve_workspace_bytes(plan, batch, nrhs) bytes or NULL
 * (see above).  Status as for stc_factorize (stc_sync_status on d_work).  On the
 * supernodal route it runs the two calls one after the other.  d_values and d_b (here, in
 * stc_factorize_forward, stc_factorize and stc_scatter_values) may also point to pinned
 * host memory that the device can address (cudaHostAlloc'ed memory under unified
 * addressing): the kernels then read the inputs in place, the upload overlapping the
 * factorization, with no separate copy (on a GB300 with NVLink-C2C: the same step time
 * as with inputs in HBM); pageable host memory is not supported. */
size_t stc_factorize_solve_workspace_bytes(const stc_plan* plan, int64_t batch, int64_t nrhs);
int stc_factorize_solve(const stc_plan* plan, const double* d_values, int64_t batch, int64_t nrhs,
                        const double* d_b, void* d_factor, double* d_x, void* d_work, int32_t* d_info,
                        void* stream);
/* Its two halves, for callers that time or overlap them separately (tile routes only; a
 * supernodal plan gives STC_ERR_UNSUPPORTED; d_work is required):
 *   stc_factorize_forward -- the value upload of Sec. 6.7 (d_values as for stc_factorize;
 *                            where the plan's task set has enough waiting tasks to host it,
 *                            each block column's values are placed inside the same launch,
 *                            ahead of that column's tasks; else by stc_scatter_values
 *                            first), the factorization and the forward substitution (d_b as
 *                            above); y stays in d_work;
 *   stc_solve_backward    -- the backward substitution L^T z = y, x = P^T z, from the y
 *                            that stc_factorize_forward left in the same d_work (same
 *                            batch and nrhs). */
int stc_factorize_forward(const stc_plan* plan, const double* d_values, int64_t batch, int64_t nrhs,
                          const double* d_b, void* d_factor, void* d_work, int32_t* d_info, void* stream);
int stc_solve_backward(const stc_plan* plan, const void* d_factor, int64_t batch, int64_t nrhs,
                       double* d_x, void* d_work, void* stream);
/* 1 if stc_factorize_forward of `batch` value sets places the values inside its launch
 * (no separate scatter kernel), 0 if it runs stc_scatter_values first (and on the
 * supernodal route); a negative STC_ERR_* on error.  Builds the task set on first use. */
int stc_factorize_forward_fills(const stc_plan* plan, int64_t batch);

/* Copy L's values out of the factor storage into CSC order (STC_EXPORT_LP / LI layout),
 * the "factor returned" form of Sec. 6.7 (Table 6 reports the factor kept on the device
 * and returned to the caller): d_factor from stc_factorize; d_Lx [batch][nnzL] FP64
 * (written). */
int stc_factor_to_csc(const stc_plan* plan, const void* d_factor, int64_t batch,
                      double* d_Lx, void* stream);

/* Selected inverse Sigma = (P A P^T)^{-1} on every stored entry of the tile storage
 * (no counterpart in the paper, which leaves selected inversion to separate work,
 * Sec. 6.2: Takahashi's recurrence on the same tile map, walked in reverse block-column
 * order by one persistent kernel).  Sigma is exact on the structural entries of L;
 * stored entries the symbolic factor proves zero hold unspecified finite values.
 *   d_factor: a factor from stc_factorize; d_sigma: stc_factor_bytes(plan,batch) bytes
 *   (written, same layout as the factor, must not alias it); d_work:
 *   stc_workspace_bytes(plan,batch) bytes or NULL (see above).
 * On the supernodal route the same recurrence runs over the supernodes (the task form
 * of stc_plan_export's SN_SEL_TASKS / SN_SEL_CONS), in the supernodal layout. */
int stc_selinv(const stc_plan* plan, const void* d_factor, int64_t batch, void* d_sigma,
               void* d_work, void* stream);

/* Adjoint of logdet (no counterpart in the paper: the gradient d logdet / dA = A^{-1}
 * needs the selected inversion Sec. 6.2 leaves to separate work): d_gvalues[b][e] (+)=
 * gout[b] * d logdet(A_b) / d a_e for every stored lower entry e of A (original CSC
 * order), i.e. (2 - delta_ij) (A^{-1})_ij, A symmetric parametrised by its lower
 * triangle.  d_gout [batch] or NULL (= 1); accumulate != 0 adds to d_gvalues.  Runs
 * stc_selinv into d_sigma first (scratch of stc_factor_bytes(plan,batch) bytes, or NULL
 * for one owned by the plan, grown and shared like the plan's workspace); d_work as for
 * stc_selinv. */
int stc_logdet_backward(const stc_plan* plan, const void* d_factor, int64_t batch,
                        const double* d_gout, double* d_gvalues, int accumulate, void* d_sigma,
                        void* d_work, void* stream);

/* Symmetric outer-product adjoint, for quadratic forms and solves (no counterpart in the
 * paper; the adjoint of x^T A x and of x = A^{-1} b with respect to A's lower values):
 *   d_gvalues[b][e] (+)= scale[b] * (2 - delta_ij)/2 * (u_i v_j + u_j v_i),  e = (i, j)
 * with u, v [batch][n] in the original ordering; scale [batch] or NULL (= 1).
 * u = v = x gives d(x^T A x)/d a_e; u = A^{-1} b, v = A^{-1} g, scale = -1 gives the
 * adjoint of the solve x = A^{-1} b for an upstream gradient g on x. */
/* d(x^T A x)/d a_e = gout[b] (2 - delta_ij) x_i x_j for every stored A entry e = (i, j)
 * (stc_sym_outer_backward with u = v = x, scale = gout): x [batch][n] in the original
 * ordering; gout [batch] or NULL (= 1); d_gvalues [batch][nnzA], added to when
 * accumulate != 0. */
int stc_quad_backward(const stc_plan* plan, int64_t batch, const double* d_x, const double* d_gout,
                      double* d_gvalues, int accumulate, void* stream);
int stc_sym_outer_backward(const stc_plan* plan, int64_t batch, const double* d_u,
                           const double* d_v, const double* d_scale, double* d_gvalues,
                           int accumulate, void* stream);

/* out[b] = x_b^T A_b x_b from the lower CSC values (d_values [batch][nnzA], d_x [batch][n]);
 * the Gaussian quadratic form beside logdet in an INLA objective (Sec. 1), no
 * counterpart in the paper's interface. */
int stc_quad_form(const stc_plan* plan, int64_t batch, const double* d_values,
                  const double* d_x, double* d_out, void* stream);

/* FP64 throughput probe (no counterpart in the paper): runs independent DFMA chains on
 * every SM for `iters` iterations, synchronously on the legacy stream, and writes the
 * measured GFLOP/s to *gflops.  d_scratch: device buffer of scratch_doubles >= 256
 * doubles (results are written there so the work is not optimised away). */
int stc_fp64_peak_probe(double* d_scratch, int64_t scratch_doubles, int64_t iters, double* gflops);

/* Factorization that allocates nothing and takes no workspace argument.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot obtain
 * device memory at the moment they factorize -- for example a service that reserves
 * all GPU memory through its own allocator at start-up and forbids later cudaMalloc,
 * a real-time loop that must not risk the device-wide synchronisation a cudaMalloc can
 * cause, or a plug-in host that hands a library only its input and output buffers.
 *
 * It runs the same value scatter and the same persistent task-DAG kernel as
 * stc_factorize, but the kernel's scratch (queue head, status word and per-tile
 * dependency counters) lives in a fixed device array inside libstc.so, of
 * STC_NOALLOC_SCRATCH_BYTES bytes, held by every GPU that loads the library until the
 * process exits.  Needed: 64 + 4 * batch * ntiles bytes (ntiles from stc_plan_info);
 * a larger request returns STC_ERR_UNSUPPORTED without launching anything.
 *   d_values [batch][nnzA] input; d_factor (stc_factor_bytes(plan,batch) bytes) and
 *   d_info [batch] outputs as for stc_factorize; d_status: optional device int32 that
 *   receives STC_OK or STC_ERR_TIMEOUT when the kernel ends (NULL = not reported).
 * Preconditions: stc_plan_upload(plan) was called on the current device (otherwise
 * STC_ERR_INVALID_ARG: uploading would allocate).  stc_plan_upload also loads the
 * library's device module on that device and looks up the array's device address
 * (cudaGetSymbolAddress), so the array is placed there at that moment: call it before
 * reserving the rest of the GPU's memory and before any stream capture.  Every call on a
 * device shares the one array and clears the part it uses on `stream` before its kernel
 * starts; calls whose kernels overlap on the GPU (different streams, or several threads)
 * race on it and give undefined results, so serialise them.  It replays the unsliced
 * task list with every item of a task in lockstep (no per-batch choice of row slices or
 * queue order), so its speed can differ from stc_factorize's; its results are the same
 * to rounding.  Tile routes only (a supernodal plan gives STC_ERR_UNSUPPORTED). */
#define STC_NOALLOC_SCRATCH_BYTES (4u << 20)
int stc_factorize_noalloc(const stc_plan* plan, const double* d_values, int64_t batch,
                          void* d_factor, int32_t* d_info, int32_t* d_status, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* STC_H */
