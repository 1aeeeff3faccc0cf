// replay.cu -- numeric phase on the GPU (sm_103a): value scatter, the persistent
// task-DAG replay of the tile Cholesky, log-determinant, triangular solves and the
// factor export.  arxiv 2609.29765, Algorithm 1 (task list), Algorithm 2 (executor),
// Sec. 4 (active-column and banded tiles), Sec. 5.3 (progress matrix -> counters).
//
// GB300 notes that shape this file:
//  * FP64 runs at ~2 DFMA/clk/SM (measured 1.21 TFLOP/s DFMA, 1.06 TFLOP/s for
//    mma.sync.m8n8k4.f64), so every tile kernel is DFMA-bound; tiles live in shared
//    memory, the inner loops are 4x4 register micro-tiles of DFMA, and the tensor-core
//    DMMA path is not used (it is slower on this part).
//  * One persistent kernel per call walks the whole DAG of every batch item: CTAs take
//    task slots from a global counter in a topological (earliest-start) order and wait
//    on per-tile completion counters (the paper's progress matrix P and per-cell
//    update counters), so the hundreds of thousands of small tile tasks of a batch cost
//    one launch.  Every wait is bounded: past the limit it records STC_ERR_TIMEOUT in
//    the workspace status word and the kernel drains without further waiting.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <functional>
#include <queue>
#include <climits>
#include <cstdio>
#include <cstring>
#include <stdexcept>

#include "plan.hpp"

namespace stc {
namespace {

constexpr int kThreads = 256;
constexpr int kNbMax = 128;
constexpr int kLdc = kNbMax + 1;   // shared-memory leading dimension of the tile buffer
constexpr int kKc = 32;            // inner-dimension chunk staged per step
constexpr int kPb = kPanelW;       // panel width of the blocked TRSM
constexpr int kStage = kKc * (kNbMax + 9);          // doubles per staging buffer (odd ld)
constexpr int kCbuf = kLdc * kNbMax + 16;           // tile buffer (+ overrun pad)
constexpr int kSmemDoubles = kCbuf + 2 * kStage + kNbMax;
constexpr size_t kSmemBytes = kSmemDoubles * sizeof(double) + 64;
constexpr long long kDefaultSpin = 40000000LL;

// Replay-kernel geometry, sized for two resident CTAs per SM (so one CTA's dependency
// waits and latency-bound phases overlap the other's DFMA work): off-diagonal and SYRK
// tasks hold at most kRRows rows, diagonal tiles are held as a packed lower triangle,
// and the inner dimension is staged 16 columns at a time.
constexpr int kRRows = 64;
constexpr int kRLd = kRRows + 1;
constexpr int kRKc = 16;
static_assert(kRKc == kExtW, "chunk extents are kept per staged inner chunk");
constexpr int kRStLd = kNbMax + 8;
constexpr int kRStage = kRKc * kRStLd;
constexpr int kRPacked = kNbMax * (kNbMax + 1) / 2;
constexpr int kRCbuf = (kRLd * kNbMax > kRPacked ? kRLd * kNbMax : kRPacked) + 16;
constexpr size_t kRSmemBytes = (size_t)(kRCbuf + 2 * kRStage + kNbMax) * sizeof(double);

// packed lower triangle of an nb x nb tile, column-major: (r, c), r >= c
__host__ __device__ __forceinline__ int pk(int nb, int r, int c) { return c * nb - (c * (c + 1)) / 2 + r; }

struct WorkHeader {          // start of the caller's workspace
    unsigned long long head; // next task slot
    int status;              // STC_OK or STC_ERR_TIMEOUT
    int pad[13];
};
static_assert(sizeof(WorkHeader) == 64, "header size");

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait (thread 0) until *cnt >= target.  Returns false on timeout / earlier error.
__device__ bool wait_counter(const int* cnt, int target, long long limit, int* status) {
    if (ld_acquire(cnt) >= target) return true;
    for (long long it = 0;; ++it) {
        if (ld_acquire(cnt) >= target) return true;
        if (*(volatile int*)status != STC_OK) return false;
        if (it >= limit) {
            atomicCAS(status, STC_OK, STC_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(it < 64 ? 32 : 256);
    }
}

// Wait (thread 0) until every bit of need is set in *cnt (an off-diagonal tile's
// completion word).  Returns false on timeout / earlier error.
__device__ bool wait_bits(const int* cnt, unsigned need, long long limit, int* status) {
    if (((unsigned)ld_acquire(cnt) & need) == need) return true;
    for (long long it = 0;; ++it) {
        if (((unsigned)ld_acquire(cnt) & need) == need) return true;
        if (*(volatile int*)status != STC_OK) return false;
        if (it >= limit) {
            atomicCAS(status, STC_OK, STC_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(it < 64 ? 32 : 256);
    }
}
__device__ __forceinline__ void red_release_or(int* p, unsigned v) {
    asm volatile("red.release.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Completion bits of an off-diagonal tile covering rows [lo, hi) (slices of h rows) and
// stored columns [s0, s1].
__device__ __forceinline__ unsigned off_need(int lo, int hi, int s0, int s1, int h) {
    if (lo >= hi) return 0u;
    const int a = lo / h, b = (hi - 1) / h;
    const unsigned sl = ((2u << b) - 1u) & ~((1u << a) - 1u);
    unsigned m = 0u;
    for (int q = s0 / kPanelW; q <= s1 / kPanelW; ++q) m |= sl << (q * kMaxSlices);
    return m;
}

// Record the first failing pivot (global column + 1) of an item; 0 = none yet.
__device__ void record_info(int* info, int v) {
    int old = *(volatile int*)info;
    while (old == 0 || old > v) {
        int prev = atomicCAS(info, old, v);
        if (prev == old) break;
        old = prev;
    }
}

// L_kk[r][c] (r >= c) from a diagonal tile in global memory (zero outside the band).
__device__ __forceinline__ double diag_at(const double* T, const DTile& d, int nb, int r, int c) {
    if (d.kind == TILE_DIAG_DENSE) return __ldcg(T + r + (size_t)c * nb);
    if (r - c > d.kd) return 0.0;
    return __ldcg(T + (d.kd + c - r) + (size_t)r * (d.kd + 1));
}

__device__ __forceinline__ int logical_col(const DTile& t, const int16_t* saind, int s) {
    return t.c0 >= 0 ? t.c0 + s : saind[t.aoff + s];
}

// Visit every (r, c), r < R, c < NC, with consecutive threads on consecutive rows: the
// rows of a column go to a power-of-two group of threads (bit operations only, no
// integer division), the groups take columns in turn.  f must not synchronise.
template <class Fn>
__device__ __forceinline__ void for_rc(int R, int NC, Fn f) {
    const int rp = R <= 1 ? 1 : min(kThreads / 2, 1 << (32 - __clz(R - 1)));
    const int sh = 31 - __clz(rp);
    const int r0 = threadIdx.x & (rp - 1);
    for (int c = threadIdx.x >> sh; c < NC; c += kThreads >> sh)
        for (int r = r0; r < R; r += rp) f(r, c);
}

// ---------------------------------------------------------------------------
// C(r,c) -= sum_k A(r,k) B(c,k), r < R, c < Cn; A(r,k) = A[r + k*lda],
// B(c,k) = B[c + k*ldb], C(r,c) = C[r + c*ldc].  TR x TC register micro-tiles, the
// micro-tiles of the region spread over the CTA.  LOWER: only micro-tiles touching
// r >= c (rows and columns index the same range) are computed, and only r >= c is
// written.  A/B rows up to the next multiple of 4 must be readable (pad).
// ---------------------------------------------------------------------------
template <bool LOWER, int TR, int TC, bool PACKED>
__device__ void mma_tiles(double* __restrict__ C, int ldc, int R, int Cn,
                          const double* __restrict__ A, int lda,
                          const double* __restrict__ B, int ldb, int K, int pnb, int pr0, int pc0,
                          int tid0 = 0, int nthr = kThreads) {
    const int MR = (R + TR - 1) / TR, MC = (Cn + TC - 1) / TC;
    const int count = LOWER ? MR * (MR + 1) / 2 : MR * MC;
    for (int mt = (int)threadIdx.x - tid0; mt < count; mt += nthr) {
        int ri, cj;
        if (LOWER) {
            // mt -> (ri, cj), cj <= ri, row-major over the lower triangle
            int r = (int)((sqrtf(8.0f * mt + 1.0f) - 1.0f) * 0.5f);
            while (r * (r + 1) / 2 > mt) --r;
            while ((r + 1) * (r + 2) / 2 <= mt) ++r;
            ri = r;
            cj = mt - r * (r + 1) / 2;
        } else {
            ri = mt % MR;
            cj = mt / MR;
        }
        const int r0 = ri * TR, c0 = cj * TC;
        // the accumulators start from C, so the update needs no separate subtraction
        double acc[TR][TC];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TC; ++j) {
                const int r = r0 + i, c = c0 + j;
                acc[i][j] = 0.0;
                if (r < R && c < Cn && (!LOWER || r >= c))
                    acc[i][j] = PACKED ? C[pk(pnb, pr0 + r, pc0 + c)] : C[r + c * ldc];
            }
        const double* a = A + r0;
        const double* b = B + c0;
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
            double av[TR], bv[TC];
#pragma unroll
            for (int i = 0; i < TR; ++i) av[i] = a[i];
#pragma unroll
            for (int j = 0; j < TC; ++j) bv[j] = b[j];
#pragma unroll
            for (int i = 0; i < TR; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j) acc[i][j] = fma(-av[i], bv[j], acc[i][j]);
            a += lda;
            b += ldb;
        }
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TC; ++j) {
                const int r = r0 + i, c = c0 + j;
                if (r < R && c < Cn && (!LOWER || r >= c)) {
                    if (PACKED) C[pk(pnb, pr0 + r, pc0 + c)] = acc[i][j];
                    else C[r + c * ldc] = acc[i][j];
                }
            }
    }
}

// 4x4 micro-tiles when they keep at least 3/4 of the CTA busy, else 2x2 (four times as
// many micro-tiles, so narrow row slices still occupy every warp).
template <bool LOWER>
__device__ __forceinline__ void mma_sub(double* C, int ldc, int R, int Cn, const double* A, int lda,
                                        const double* B, int ldb, int K) {
    const int m4 = (R + 3) >> 2, n4 = (Cn + 3) >> 2;
    const int c44 = LOWER ? m4 * (m4 + 1) / 2 : m4 * n4;
    if (c44 >= (kThreads * 3) / 4)
        mma_tiles<LOWER, 4, 4, false>(C, ldc, R, Cn, A, lda, B, ldb, K, 0, 0, 0);
    else
        mma_tiles<LOWER, 2, 2, false>(C, ldc, R, Cn, A, lda, B, ldb, K, 0, 0, 0);
}

// Same into a packed lower triangle P (pk layout, tile width pnb); the region starts at
// (pr0, pc0) of the tile.
template <bool LOWER>
__device__ __forceinline__ void mma_sub_packed(double* P, int pnb, int pr0, int pc0, int R, int Cn,
                                               const double* A, int lda, const double* B, int ldb, int K,
                                               int tid0 = 0, int nthr = kThreads) {
    if ((int)threadIdx.x < tid0 || (int)threadIdx.x >= tid0 + nthr) return;
    const int m4 = (R + 3) >> 2, n4 = (Cn + 3) >> 2;
    const int c44 = LOWER ? m4 * (m4 + 1) / 2 : m4 * n4;
    if (c44 >= (nthr * 3) / 4)
        mma_tiles<LOWER, 4, 4, true>(P, 0, R, Cn, A, lda, B, ldb, K, pnb, pr0, pc0, tid0, nthr);
    else
        mma_tiles<LOWER, 2, 2, true>(P, 0, R, Cn, A, lda, B, ldb, K, pnb, pr0, pc0, tid0, nthr);
}

// Forward substitution of a row block against a panel: X(r, 0:pw) <- X(r, 0:pw) D^{-T},
// D lower pw x pw in shared memory (D(i,j) = D[i + j*ldd]), reciprocal diagonal dinv[].
// TPR threads share a row: each keeps the columns j = q (mod TPR) in registers, the
// owner of column j finishes x_j and broadcasts it by shuffle, and every thread then
// removes x_j's contribution from its later columns (right-looking).
template <int TPR, bool BACK>
__device__ void trsm_rows_t(double* X, int ldx, int R, int pw, const double* D, int ldd,
                            const double* dinv) {
    constexpr int NJ = kPb / TPR;
    const int q = threadIdx.x % TPR;
    const int lane = threadIdx.x & 31;
    const int base = lane - q;
    for (int rr = threadIdx.x / TPR; rr < ((R + (kThreads / TPR) - 1) / (kThreads / TPR)) * (kThreads / TPR);
         rr += kThreads / TPR) {
        const bool live = rr < R;
        double b[NJ];
#pragma unroll
        for (int s = 0; s < NJ; ++s) {
            const int k = s * TPR + q;
            b[s] = (live && k < pw) ? X[rr + k * ldx] : 0.0;
        }
#pragma unroll
        for (int jj = 0; jj < kPb; ++jj) {
            const int j = BACK ? kPb - 1 - jj : jj;
            if (j < pw) {
                const double xj = __shfl_sync(0xffffffffu, b[j / TPR] * dinv[j], base + (j % TPR));
                if (q == j % TPR) b[j / TPR] = xj;
#pragma unroll
                for (int s = 0; s < NJ; ++s) {
                    // s and j are compile-time here: register groups whose columns all lie on
                    // the finished side of j issue no instruction (a masked DFMA still takes a
                    // slot of the FP64 pipe)
                    if (BACK ? s * TPR >= j : s * TPR + TPR - 1 <= j) continue;
                    const int k = s * TPR + q;
                    if (!BACK && k > j && k < pw) b[s] = fma(-xj, D[k + j * ldd], b[s]);
                    if (BACK && k < j) b[s] = fma(-xj, D[j + k * ldd], b[s]);
                }
            }
        }
        if (live) {
#pragma unroll
            for (int s = 0; s < NJ; ++s) {
                const int k = s * TPR + q;
                if (k < pw) X[rr + k * ldx] = b[s];
            }
        }
    }
}

// Forward (X D^{-T}) or backward (X D^{-1}) substitution of a row block against a
// lower pw x pw panel block D, choosing 2, 4 or 8 threads per row from the row count.
template <bool BACK>
__device__ __forceinline__ void trsm_rows_dir(double* X, int ldx, int R, int pw, const double* D, int ldd,
                                              const double* dinv) {
    if (R <= kThreads / 8) trsm_rows_t<8, BACK>(X, ldx, R, pw, D, ldd, dinv);
    else if (R <= kThreads / 4) trsm_rows_t<4, BACK>(X, ldx, R, pw, D, ldd, dinv);
    else trsm_rows_t<2, BACK>(X, ldx, R, pw, D, ldd, dinv);
}

__device__ __forceinline__ void trsm_rows(double* X, int ldx, int R, int pw, const double* D, int ldd,
                                          const double* dinv) {
    trsm_rows_dir<false>(X, ldx, R, pw, D, ldd, dinv);
}

struct SnArgs {
    const SnDevCell* cells;
    const SnDevTask* tasks;
    const SnDevUpd* upds;
    const int16_t* maps;
    const int32_t* first;    // first column of each supernode
    double* factor;          // item 0
    long long fstride;       // doubles per item
    long long poff;          // offset of the logdet partials (one per supernode)
    int* counters;           // [batch][ncells]
    int ncells;
    int* info;
    WorkHeader* hdr;
    int ntasks;
    long long batch;
    long long spin;
};

// One supernodal task; defined with the supernodal route below.
__device__ __forceinline__ void sn_task(const SnArgs& a, int ti, long long item, double* C, double* S0, double* S1,
                                        double* sv, int* s_rm, int* s_cm, int& s_ok);

struct ReplayArgs {        // one job: a plan and a batch of value sets
    const DTile* tiles;
    const int16_t* saind;
    const int16_t* cext;     // chunk row extents of the off-diagonal tiles
    const DTask* tasks;
    const DUpd* upds;
    const int16_t* imap;
    double* factor;          // item 0
    long long fstride;       // doubles per item
    long long poff;          // offset of the logdet partials in an item
    int* counters;           // [batch][ntiles]
    int ntiles;
    int* info;               // [batch]
    WorkHeader* hdr;
    int ntasks;
    long long batch;
    int nb;
    int slice_h;             // rows per row slice of an off-diagonal tile
    long long spin;
    int sn;                  // != 0: a supernodal plan, executed from the launch's snj[job]
    // TASK_FWD (fused factorization + forward substitution; null otherwise)
    const double* rhs;       // [batch][nrhs][n]
    double* y;               // [batch * nrhs][nt * nb]: forward results, read by the backward solve
    int* sdone;              // [batch * nrhs][2 nt]: the solve's step flags (forward half set here)
    const int32_t* perm;     // permuted position -> original index
    const int32_t* rowstart; // per block row k: its off-diagonal tiles (k,n) in rowtiles
    const int32_t* rowtiles;
    long long n;
    int nrhs;
    int nt;
    // value scatter inside the launch (fused sets with fill_inside; null otherwise)
    const double* vals;      // [batch][nnzA]
    long long nnz;
    const int32_t* fill_src; // per factor double: the A entry stored there, -1 (zero), -2 (1.0)
    int* fillflag;           // [batch][nt]: block column k of the item filled
    const int32_t* colstart; // per block column: its first tile (the diagonal), tiles in order
};

// One launch of the replay kernel: up to kMaxJobs jobs (plans) in one persistent grid.
// Queue entry of a slot: job << 60 | task << 28 | item; without a queue (one job) the
// slot is task * batch + item (all items of a task in lockstep).
constexpr int kMaxJobs = 8;
struct ReplayLaunch {
    ReplayArgs job[kMaxJobs];
    SnArgs snj[kMaxJobs];    // the supernodal jobs' arguments (mixed-route groups)
    int njobs;
    const uint64_t* queue;
    long long total;
    WorkHeader* hdr;
};
__host__ __device__ __forceinline__ uint64_t qpack(int job, int task, long long item) {
    return (uint64_t)job << 60 | (uint64_t)(uint32_t)task << 28 | (uint64_t)item;
}

// Load rows [rs0, rs0+R) of stored columns [0, sw) of an off-diagonal tile into C.
__device__ void load_off(double* C, int ldc, const double* T, int nb, int rs0, int R, int sw) {
    for_rc(R, sw, [&](int r, int c) { C[r + c * ldc] = __ldcg(T + rs0 + r + (size_t)c * nb); });
}
__device__ void store_off(const double* C, int ldc, double* T, int nb, int rs0, int R, int sw) {
    for_rc(R, sw, [&](int r, int c) { __stcg(T + rs0 + r + (size_t)c * nb, C[r + c * ldc]); });
}

// Rows [r0, r1) of a diagonal tile, read in storage order (coalesced: a warp per stored
// column of a dense tile, a warp per row of a banded one, up to eight loads in flight per
// lane): fn(r, c, L[r][c]) for every stored entry with r >= c (entries of a banded tile
// outside the band are not visited).
template <class Fn>
__device__ void read_diag_rows(const double* T, const DTile& d, int nb, int r0, int r1, Fn fn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kW = kThreads / 32;
    if (d.kind == TILE_DIAG_DENSE) {
        for (int c = warp; c < nb; c += 2 * kW) {
            double v[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int cc = c + h * kW, r = r0 + lane + 32 * u;
                    v[h][u] = (cc < nb && r < r1) ? __ldcg(T + r + (size_t)cc * nb) : 0.0;
                }
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int cc = c + h * kW, r = r0 + lane + 32 * u;
                    if (cc < nb && r < r1 && r >= cc) fn(r, cc, v[h][u]);
                }
        }
    } else {
        const int w = d.kd + 1;  // storage (q, r): L[r][r - kd + q] at q + r w
        for (int r = r0 + warp; r < r1; r += 2 * kW) {
            double v[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int rr = r + h * kW, q = lane + 32 * u;
                    v[h][u] = (rr < r1 && q < w) ? __ldcg(T + q + (size_t)rr * w) : 0.0;
                }
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int rr = r + h * kW, q = lane + 32 * u, c = rr - d.kd + q;
                    if (rr < r1 && q < w && c >= 0) fn(rr, c, v[h][u]);
                }
        }
    }
}

// Entries L[r][c], r in [r0, r1), c in [c0, min(c1, r + 1)), written to a diagonal tile's
// storage in storage order (a warp per stored column / per row): T <- get(r, c); banded
// tiles only inside the band.
template <class Get>
__device__ void write_diag_rows(double* T, const DTile& d, int nb, int r0, int r1, int c0, int c1, Get get) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kW = kThreads / 32;
    if (d.kind == TILE_DIAG_DENSE) {
        for (int c = c0 + warp; c < c1; c += kW)
            for (int r = max(r0, c) + lane; r < r1; r += 32) __stcg(T + r + (size_t)c * nb, get(r, c));
    } else {
        const int w = d.kd + 1;
        for (int r = r0 + warp; r < r1; r += kW) {
            // row r holds columns [r - kd, r]: the part inside [c0, c1)
            const int ca = max(max(c0, r - d.kd), 0), cb = min(c1, r + 1);
            for (int c = ca + lane; c < cb; c += 32) __stcg(T + (d.kd + c - r) + (size_t)r * w, get(r, c));
        }
    }
}

// Diagonal tile -> packed lower triangle in shared memory (zero outside a band).
__device__ void load_diag_packed(double* P, const double* T, const DTile& d, int nb) {
    if (d.kind == TILE_DIAG_BAND && d.kd < nb - 1) {
        for (int i = threadIdx.x; i < nb * (nb + 1) / 2; i += kThreads) P[i] = 0.0;
        __syncthreads();
    }
    read_diag_rows(T, d, nb, 0, nb, [&](int r, int c, double v) { P[pk(nb, r, c)] = v; });
}
// Columns [c0, c1) of the packed triangle back into the diagonal tile's storage (dense:
// with the zero upper part; banded: the entries inside the band).
__device__ void store_diag_cols(const double* P, double* T, const DTile& d, int nb, int c0, int c1) {
    if (d.kind == TILE_DIAG_DENSE) {
        for_rc(nb, c1 - c0, [&](int r, int cc) {
            const int c = c0 + cc;
            __stcg(T + r + (size_t)c * nb, r >= c ? P[pk(nb, r, c)] : 0.0);
        });
    } else {
        write_diag_rows(T, d, nb, c0, min(nb, c1 + d.kd), c0, c1, [&](int r, int c) { return P[pk(nb, r, c)]; });
    }
}

// Full lower triangle (and zero upper) of a diagonal tile into C.
__device__ void load_diag(double* C, const double* T, const DTile& d, int nb) {
    for_rc(nb, nb, [&](int r, int c) { C[r + c * kLdc] = r >= c ? diag_at(T, d, nb, r, c) : 0.0; });
}
__device__ void store_diag(const double* C, double* T, const DTile& d, int nb) {
    if (d.kind == TILE_DIAG_DENSE) {
        for_rc(nb, nb, [&](int r, int c) { __stcg(T + r + (size_t)c * nb, r >= c ? C[r + c * kLdc] : 0.0); });
    } else {
        const int w = d.kd + 1;
        for_rc(w, nb, [&](int q, int r) {  // storage (q, r): L[r][r - kd + q]
            const int c = r - d.kd + q;
            if (c >= 0) __stcg(T + q + (size_t)r * w, C[r + c * kLdc]);
        });
    }
}

// Stage a (R x K) chunk of stored columns of tile T into S (S[r + k*ld]); rows beyond R
// up to a multiple of 4 are zeroed.
__device__ void stage_cols(double* S, int ld, const double* T, int nb, int row0, int R,
                           const DUpd& u, const int16_t* imap, bool use_b, int k0, int K) {
    const int Rp = ((R + 3) & ~3) + 4;
    for_rc(Rp, K, [&](int r, int k) {
        double v = 0.0;
        if (r < R) {
            int s;
            if (u.kmap < 0) s = (use_b ? u.kb0 : u.ka0) + k0 + k;
            else s = imap[2 * (u.kmap + k0 + k) + (use_b ? 1 : 0)];
            v = __ldcg(T + row0 + r + (size_t)s * nb);
        }
        S[r + k * ld] = v;
    });
}

// Union [lo, hi) of the structural row extents of stored columns [s0, s1] of tile T
// (rows outside are zero in every one of those columns); [0, nb) without extents.
__device__ __forceinline__ void col_ext(const int16_t* __restrict__ cext, const DTile& T, int nb, int s0, int s1,
                                        int& lo, int& hi) {
    if (T.xoff < 0) { lo = 0; hi = nb; return; }
    lo = nb; hi = 0;
    for (int q = s0 / kExtW; q <= s1 / kExtW; ++q) {
        lo = min(lo, (int)cext[2 * (T.xoff + q)]);
        hi = max(hi, (int)cext[2 * (T.xoff + q) + 1]);
    }
}

// Stored columns of the A (or B) operand covered by inner positions [k0, k0+K) of u.
__device__ __forceinline__ void inner_cols(const DUpd& u, const int16_t* imap, bool b, int k0, int K,
                                           int& s0, int& s1) {
    if (u.kmap < 0) {
        s0 = (b ? u.kb0 : u.ka0) + k0;
        s1 = s0 + K - 1;
    } else {
        s0 = imap[2 * (u.kmap + k0) + (b ? 1 : 0)];
        s1 = imap[2 * (u.kmap + k0 + K - 1) + (b ? 1 : 0)];
    }
}

// B rows for a GEMM: rows = logical columns of the output tile's stored columns oc0.. .
__device__ void stage_rows_gather(double* S, int ld, const double* T, int nb, const DTile& O,
                                  const int16_t* saind, int oc0, int Cn, const DUpd& u,
                                  const int16_t* imap, int k0, int K) {
    const int Cp = ((Cn + 3) & ~3) + 4;
    for_rc(Cp, K, [&](int c, int k) {
        double v = 0.0;
        if (c < Cn) {
            const int row = logical_col(O, saind, oc0 + c);
            const int s = u.kmap < 0 ? u.kb0 + k0 + k : imap[2 * (u.kmap + k0 + k) + 1];
            v = __ldcg(T + row + (size_t)s * nb);
        }
        S[c + k * ld] = v;
    });
}

// POTRF of a diagonal tile held as a packed lower triangle (see potrf_packed below).
template <int PP>
struct PotrfShared {
    double blk[PP][PP];    // L of the current panel's diagonal block, blk[row][col]
    double inv[PP];        // 1 / L_jj of the panel
    int bad;
};

// All threads: rows [p+pw, rend) of panel p solved against the diagonal block; the solved
// rows also go to S (row i at S[i - p - pw], column l at stride kRStLd), zero-padded.
template <int PP>
__device__ void potrf_rows_below(double* P, int nb, int p, int pw, int rend, double* S,
                                 const PotrfShared<PP>& sh) {
    const int R2 = rend - p - pw;
    const int R2p = ((max(R2, 0) + 3) & ~3) + 4;
    for (int rr = threadIdx.x; rr < R2p; rr += kThreads) {
        const int i = p + pw + rr;
        double x[PP];
        if (rr < R2) {
#pragma unroll
            for (int l = 0; l < PP; ++l) x[l] = l < pw ? P[pk(nb, i, p + l)] : 0.0;
#pragma unroll
            for (int j = 0; j < PP; ++j) {
                if (j < pw) {
                    double sacc = x[j];
#pragma unroll
                    for (int l = 0; l < j; ++l) sacc = fma(-x[l], sh.blk[j][l], sacc);
                    x[j] = sacc * sh.inv[j];
                }
            }
#pragma unroll
            for (int l = 0; l < PP; ++l)
                if (l < pw) P[pk(nb, i, p + l)] = x[l];
        } else {
#pragma unroll
            for (int l = 0; l < PP; ++l) x[l] = 0.0;
        }
#pragma unroll
        for (int l = 0; l < PP; ++l) S[rr + l * kRStLd] = x[l];
    }
}

// Warp 0 only: the 8x8 diagonal block at (p, p), first reduced by the rank-kw update
// from the solved rows of the previous panel (S rows 0..rv-1, columns at stride ld; rows
// from rv on are outside the previous panel's band and zero there), then factored.  Each lane holds two entries of one row, (r, c0) and (r, c0 + 1) with
// r = lane / 4 and c0 = 2 (lane % 4), so a pivot costs one reciprocal square root and
// two fused multiply-adds per lane instead of one per later column.
__device__ void potrf_diag8(double* P, int nb, int p, int pw, const double* S, int ld, int kw, int rv,
                            PotrfShared<8>& sh) {
    const int lane = threadIdx.x & 31;
    const int r = lane >> 2, c0 = 2 * (lane & 3);
    double x[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int c = c0 + e;
        double v = 0.0;
        if (r < pw && c <= r) {
            v = P[pk(nb, p + r, p + c)];
            if (r < rv)
                for (int m = 0; m < kw; ++m) v = fma(-S[r + m * ld], S[c + m * ld], v);
        }
        x[e] = v;
    }
    int badl = -1;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < pw) {
            const int src = 4 * j + (j >> 1);
            const double d = __shfl_sync(0xffffffffu, x[j & 1], src);
            if (!(d > 0.0) && badl < 0) badl = p + j;  // the first non-positive pivot
            const double inv = rsqrt(d);
            if ((lane & 3) == (j >> 1) && r >= j) x[j & 1] = (r == j) ? d * inv : x[j & 1] * inv;
            // L(r, j) and L(c, j) of this lane's entries, then the rank-1 update
            const double lr = __shfl_sync(0xffffffffu, x[j & 1], 4 * r + (j >> 1));
            const double l0 = __shfl_sync(0xffffffffu, x[j & 1], 4 * c0 + (j >> 1));
            const double l1 = __shfl_sync(0xffffffffu, x[j & 1], 4 * (c0 + 1) + (j >> 1));
            if (c0 > j && r >= c0) x[0] = fma(-lr, l0, x[0]);
            if (c0 + 1 > j && r >= c0 + 1) x[1] = fma(-lr, l1, x[1]);
            if (lane == 0) sh.inv[j] = inv;
        }
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int c = c0 + e;
        const bool in = r < pw && c <= r;
        sh.blk[r][c] = in ? x[e] : 0.0;
        if (in) P[pk(nb, p + r, p + c)] = x[e];
    }
    if (lane == 0 && badl >= 0 && sh.bad < 0) sh.bad = badl;
}

// Blocked right-looking Cholesky of the w x w leading block of the packed lower
// triangle P (pk layout, tile width nb) in shared memory, panels of 8 with a one-panel
// look-ahead: warp 0 applies the previous panel's rank-8 update to the next 8x8
// diagonal block and factors it, while warps 1-7 update everything below that block
// (the rest of the next panel's columns and the trailing triangle) in one pass; then
// the rows below the new block are solved against it, one row per thread, and copied to
// the staging buffer S for the next step.  Rows more than kd below the diagonal are
// structurally zero and skipped.  *bad receives the first non-positive pivot column (or
// -1); *logsum = sum_j log L_jj, one log per diagonal entry reduced in a fixed order.
// pub(c) is called by every thread (after a barrier) each time columns [c - pubw, c) have
// become final, for c < w a multiple of pubw (a multiple of 8).  *bad and *logsum are
// valid in thread 0 only.
template <class Pub>
__device__ void potrf_packed(double* P, int nb, int w, int kd, double* S, int* bad, double* logsum, int pubw,
                             Pub pub) {
    __shared__ PotrfShared<8> sh;
    if (threadIdx.x == 0) sh.bad = -1;
    __syncthreads();
    {
        const int pw = min(8, w);
        if (threadIdx.x < 32) potrf_diag8(P, nb, 0, pw, S, kRStLd, 0, 0, sh);
        __syncthreads();
        potrf_rows_below<8>(P, nb, 0, pw, min(w, pw + kd), S, sh);
        __syncthreads();
    }
    for (int p = 0; p < w; p += 8) {
        const int pw = min(8, w - p);
        const int rend = min(w, p + pw + kd);
        const int pn = p + pw;
        if (pn >= w) break;
        const int pwn = min(8, w - pn);
        const int R3 = rend - pn - pwn;  // rows below the next diagonal block
        if (threadIdx.x < 32) {
            potrf_diag8(P, nb, pn, pwn, S, kRStLd, pw, rend - pn, sh);
        } else if (R3 > 0) {
            mma_sub_packed<false>(P, nb, pn + pwn, pn, R3, pwn, S + pwn, kRStLd, S, kRStLd, pw, 32, kThreads - 32);
            mma_sub_packed<true>(P, nb, pn + pwn, pn + pwn, R3, R3, S + pwn, kRStLd, S + pwn, kRStLd, pw,
                                 32, kThreads - 32);
        }
        __syncthreads();
        potrf_rows_below<8>(P, nb, pn, pwn, min(w, pn + pwn + kd), S, sh);
        __syncthreads();
        if (pn + pwn < w && (pn + pwn) % pubw == 0) pub(pn + pwn);
    }
    __shared__ double s_red[kThreads / 32];
    double lg = 0.0;
    for (int j = threadIdx.x; j < w; j += kThreads) lg += log(P[pk(nb, j, j)]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lg += __shfl_down_sync(0xffffffffu, lg, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = lg;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) t += s_red[q];
        *bad = sh.bad;
        *logsum = t;
    }
    __syncthreads();
}

// Completion bits of a diagonal tile: the column groups covering [c0, c1) of row slice s
// (c0 a multiple of kDiagGroupW), every group of a set of slices, and every slice's bits
// of the groups [0, g].
__device__ __forceinline__ unsigned diag_bits(int c0, int c1, int s) {
    unsigned m = 0u;
    for (int g = c0 / kDiagGroupW; g * kDiagGroupW < c1; ++g) m |= 1u << (g * kMaxDiagSlices + s);
    return m;
}
__device__ __forceinline__ unsigned slice_bits(unsigned slices) {
    unsigned m = 0u;
    for (int g = 0; g < kMaxNb / kDiagGroupW; ++g) m |= slices << (g * kMaxDiagSlices);
    return m;
}
__device__ __forceinline__ unsigned diag_prefix(int g) {
    const int nbits = (g + 1) * kMaxDiagSlices;
    return nbits >= 32 ? ~0u : (1u << nbits) - 1u;
}

// Sum of v over the CTA in a fixed order (per-thread values, then warps, then warp sums).
__device__ double cta_sum_fixed(double v) {
    __shared__ double s_part[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += s_part[q];
    __syncthreads();
    return t;
}

// Factorization of rows [a0, b0) of a diagonal tile (the second half of TASK_SYRK, after
// its SYRKs; POTRF(k) of Algorithm 1 partitioned by rows).  C holds the rows,
// C[(r - a0) + c * kRLd] for columns [0, b0).  Columns [0, a0) belong to the earlier
// slices: group by group (kDiagGroupW columns) the rows [g0, a0) of L that they published
// are staged, this slice's rows are solved against the group's diagonal block and
// published, and the rank-kDiagGroupW update from them is applied to their later columns;
// a group wholly outside the band of these rows is zero in them and skipped.  The slice's
// own diagonal block is then factored (potrf_packed) and published group by group.  The
// last slice writes the tile's logdet partial from every L_jj.  s_ok turns 0 when a wait
// fails (timeout or an earlier error).
__device__ void slice_factor(const ReplayArgs& a, const DTask& t, const DTile& O, double* F, int* cnt,
                             long long item, double* C, double* S0, double* S1, double* sv, int& s_ok) {
    const int nb = a.nb, a0 = t.rs0, b0 = t.rs1, R = b0 - a0, sl = t.slice;
    double* T = F + O.off;
    const unsigned nf = (unsigned)O.nfinal;
    const unsigned below = (1u << sl) - 1u;  // the slices before this one, in a group's bits
    for (int g0 = 0; g0 < a0; g0 += kDiagGroupW) {
        if (g0 + kDiagGroupW <= a0 - O.kd) continue;
        const int g = g0 / kDiagGroupW;
        if (threadIdx.x == 0)
            s_ok = wait_bits(cnt + t.tile, nf & (below << (g * kMaxDiagSlices)), a.spin, &a.hdr->status);
        __syncthreads();
        if (!s_ok) return;
        // rows [g0, a0) of the group's columns into S0 (row r - g0, column c - g0): zero above
        // the diagonal, outside the band and on the padding rows the products read
        const int Rs = a0 - g0, Rsp = ((Rs + 3) & ~3) + 4;
        if (O.kind == TILE_DIAG_BAND) {
            // consecutive threads along a stored row
            for (int idx = threadIdx.x; idx < Rsp * kDiagGroupW; idx += kThreads) {
                const int r = idx / kDiagGroupW, c = idx % kDiagGroupW;
                S0[r + c * kRStLd] = (r < Rs && r >= c) ? diag_at(T, O, nb, g0 + r, g0 + c) : 0.0;
            }
        } else {
            for_rc(Rsp, kDiagGroupW, [&](int r, int c) {
                S0[r + c * kRStLd] = (r < Rs && r >= c) ? diag_at(T, O, nb, g0 + r, g0 + c) : 0.0;
            });
        }
        __syncthreads();
        if (threadIdx.x < kDiagGroupW) sv[threadIdx.x] = 1.0 / S0[threadIdx.x * (kRStLd + 1)];
        __syncthreads();
        double* X = C + g0 * kRLd;
        trsm_rows(X, kRLd, R, kDiagGroupW, S0, kRStLd, sv);
        __syncthreads();
        write_diag_rows(T, O, nb, a0, b0, g0, g0 + kDiagGroupW, [&](int r, int c) { return C[(r - a0) + c * kRLd]; });
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) red_release_or(cnt + t.tile, 1u << (g * kMaxDiagSlices + sl));
        // later columns of the rows: [g0 + kDiagGroupW, a0) against the staged rows, the
        // slice's own triangle [a0, b0) against the rows themselves
        const int cn = a0 - g0 - kDiagGroupW;
        if (cn > 0)
            mma_sub<false>(X + kDiagGroupW * kRLd, kRLd, R, cn, X, kRLd, S0 + kDiagGroupW, kRStLd, kDiagGroupW);
        mma_sub<true>(C + a0 * kRLd, kRLd, R, R, X, kRLd, X, kRLd, kDiagGroupW);
        __syncthreads();
    }
    // the slice's own diagonal block, as a packed triangle in S0 (R (R+1) / 2 <= kRStage)
    double* P = S0;
    for (int idx = threadIdx.x; idx < R * R; idx += kThreads) {
        const int i = idx % R, j = idx / R;
        if (i >= j) P[pk(R, i, j)] = C[i + (a0 + j) * kRLd];
    }
    __syncthreads();
    int bad = -1, done = 0;
    double ls;
    auto own = [&](int r, int c) { return P[pk(R, r - a0, c - a0)]; };
    potrf_packed(P, R, R, min(O.kd, R - 1), S1, &bad, &ls, kDiagGroupW, [&](int c1) {
        write_diag_rows(T, O, nb, a0 + done, b0, a0 + done, a0 + c1, own);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) red_release_or(cnt + t.tile, diag_bits(a0 + done, a0 + c1, sl));
        done = c1;
    });
    write_diag_rows(T, O, nb, a0 + done, b0, a0 + done, b0, own);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bad >= 0) record_info(a.info + item, O.J * nb + a0 + bad + 1);
        red_release_or(cnt + t.tile, diag_bits(a0 + done, b0, sl));
    }
    if (b0 == O.sw) {
        // the last slice: logdet partial of the tile once every earlier slice is final
        if (threadIdx.x == 0 && sl > 0)
            s_ok = wait_bits(cnt + t.tile, nf & slice_bits(below), a.spin, &a.hdr->status);
        __syncthreads();
        if (!s_ok) return;
        double lg = 0.0;
        for (int j = threadIdx.x; j < O.sw; j += kThreads)
            lg += log(j < a0 ? diag_at(T, O, nb, j, j) : P[pk(R, j - a0, j - a0)]);
        lg = cta_sum_fixed(lg);
        if (threadIdx.x == 0) F[a.poff + O.pd_slot] = bad >= 0 ? __longlong_as_double(0x7ff8000000000000LL) : lg;
    }
}

// a1 inside the factorization launch (TASK_FILL, or a slice-1 TASK_SYRK hosting it): the
// value scatter of block column k for one item, every double of the column's tiles (they
// are contiguous in the factor, up to the logdet partials) from the values through the
// fill map, eight entries per thread in flight (the last column also zeroes the item's
// tail after the partials); then the column's fill flag is set.
__device__ void fill_col(const ReplayArgs& a, int k, long long item, double* F) {
    const long long b = a.tiles[a.colstart[k]].off;
    const long long e = k + 1 < a.nt ? a.tiles[a.colstart[k + 1]].off : a.poff;
    const double* v = a.vals + item * a.nnz;
    constexpr int U = 8;
    for (long long f0 = b + threadIdx.x; f0 < e; f0 += (long long)kThreads * U) {
        int src[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long f = f0 + (long long)u * kThreads;
            src[u] = f < e ? __ldg(a.fill_src + f) : -1;
        }
        double x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = src[u] >= 0 ? __ldg(v + src[u]) : (src[u] == -2 ? 1.0 : 0.0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long f = f0 + (long long)u * kThreads;
            if (f < e) __stcg(F + f, x[u]);
        }
    }
    if (k == a.nt - 1)  // the item's tail after the logdet partials (which the diagonal tasks write)
        for (long long f = a.poff + a.nt + threadIdx.x; f < a.fstride; f += kThreads) __stcg(F + f, 0.0);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) red_release_add(a.fillflag + item * a.nt + k, 1);
}

// a10 inside the factorization launch (TASK_FWD): forward substitution of block row k for
// every right-hand side of one item, y_k = L_kk^{-1} (b_k - sum_n L_kn y_n), once L_kk, the
// tiles L_kn of block row k and the y_n are final.  The products take a row per thread
// (threads kThreads / nb apart share a row, over stored columns taken in turn, four
// accumulators, partial sums added in a fixed order).  The substitution runs on the unit
// triangle M = L_kk diag(L_kk)^{-1} (scaled in place in the packed copy in C), so a column
// step is one FMA per later row: the owner of row j publishes u_j, the warps that own rows
// meet at a named barrier, and every later row takes its term; y = diag(L_kk)^{-1} u.  y_k
// goes to the solve's y array and its step flag is set to the panel count, as the solve's
// own forward step would leave it, so that the backward solve can follow.  A step whose
// waits fail still sets its flags (with the status word set, later steps stop early).
__device__ void fwd_task(const ReplayArgs& a, int dtile, long long item, double* F, int* cnt, double* C,
                         double* S0, double* S1, double* sv, int& s_ok) {
    const int nb = a.nb, nt = a.nt, np = (nb + 31) / 32;
    const DTile O = a.tiles[dtile];
    const int k = O.J, sw = O.sw, kd = min(O.kd, nb - 1);
    if (threadIdx.x == 0) {
        bool ok = s_ok && wait_bits(cnt + dtile, (unsigned)O.nfinal, a.spin, &a.hdr->status);
        for (int q = a.rowstart[k]; ok && q < a.rowstart[k + 1]; ++q) {
            const int tt = a.rowtiles[q];
            ok = wait_bits(cnt + tt, (unsigned)a.tiles[tt].nfinal, a.spin, &a.hdr->status);
            for (int r = 0; ok && r < a.nrhs; ++r)
                ok = wait_counter(a.sdone + (item * a.nrhs + r) * 2LL * nt + a.tiles[tt].J, np, a.spin,
                                  &a.hdr->status);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (s_ok) {
        load_diag_packed(C, F + O.off, O, nb);
        __syncthreads();
        for (int j = threadIdx.x; j < sw; j += kThreads) sv[j] = 1.0 / C[pk(nb, j, j)];
        __syncthreads();
        {
            // M = L diag(L)^{-1} below the diagonal, a warp per column
            const int lane = threadIdx.x & 31;
            for (int j = threadIdx.x >> 5; j < sw; j += kThreads / 32)
                for (int i = j + 1 + lane; i < min(sw, j + kd + 1); i += 32) C[pk(nb, i, j)] *= sv[j];
        }
        __syncthreads();
        const int G = kThreads / nb, row = threadIdx.x % nb, part = threadIdx.x / nb;
        const int nrow = (sw + 31) & ~31;  // threads of the warps that own rows
        double* vb = S1;        // the block's right-hand side after the products
        double* us = S1 + nb;   // u = diag(L) y
        for (int r = 0; r < a.nrhs; ++r) {
            const long long ch = item * a.nrhs + r;
            const double* ych = a.y + ch * (long long)nt * nb;
            if (part < G) {
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                for (int q = a.rowstart[k]; q < a.rowstart[k + 1]; ++q) {
                    const DTile T = a.tiles[a.rowtiles[q]];
                    if (row < T.r0 || row >= T.r1) continue;
                    const double* Tc = F + T.off + row;
                    const double* yn = ych + (long long)T.J * nb;
                    int c = part;
                    for (; c + 3 * G < T.sw; c += 4 * G) {
                        s0 = fma(__ldcg(Tc + (size_t)c * nb), __ldcg(yn + logical_col(T, a.saind, c)), s0);
                        s1 = fma(__ldcg(Tc + (size_t)(c + G) * nb), __ldcg(yn + logical_col(T, a.saind, c + G)), s1);
                        s2 = fma(__ldcg(Tc + (size_t)(c + 2 * G) * nb), __ldcg(yn + logical_col(T, a.saind, c + 2 * G)),
                                 s2);
                        s3 = fma(__ldcg(Tc + (size_t)(c + 3 * G) * nb), __ldcg(yn + logical_col(T, a.saind, c + 3 * G)),
                                 s3);
                    }
                    for (; c < T.sw; c += G)
                        s0 = fma(__ldcg(Tc + (size_t)c * nb), __ldcg(yn + logical_col(T, a.saind, c)), s0);
                }
                S0[part * nb + row] = (s0 + s1) + (s2 + s3);
            }
            __syncthreads();
            if (threadIdx.x < nb) {
                const long long g = (long long)k * nb + threadIdx.x;
                double s2 = 0.0;
                for (int p2 = 0; p2 < G; ++p2) s2 += S0[p2 * nb + threadIdx.x];
                vb[threadIdx.x] = (g < a.n ? a.rhs[ch * a.n + a.perm[g]] : 0.0) - s2;
            }
            __syncthreads();
            if ((int)threadIdx.x < nrow) {
                const int i = threadIdx.x;
                double ur = i < sw ? vb[i] : 0.0;
                for (int j = 0; j < sw; ++j) {
                    if (i == j) us[j] = ur;
                    asm volatile("bar.sync 1, %0;" ::"r"(nrow) : "memory");
                    if (i > j && i < sw && i - j <= kd) ur = fma(-C[pk(nb, i, j)], us[j], ur);
                }
            }
            __syncthreads();
            double* yk = a.y + ch * (long long)nt * nb + (long long)k * nb;
            for (int i = threadIdx.x; i < nb; i += kThreads) __stcg(yk + i, i < sw ? us[i] * sv[i] : 0.0);
            __syncthreads();
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        for (int r = 0; r < a.nrhs; ++r) red_release_add(a.sdone + (item * a.nrhs + r) * 2LL * nt + k, np);
}

// WITH_SN: the launch may hold supernodal jobs (a mixed-route group); their tasks run
// through sn_task.  The tile-only instantiation is the one every single-plan factorization
// of a tile route uses.
template <bool WITH_SN>
__global__ void __launch_bounds__(kThreads, 2) replay_kernel_t(const __grid_constant__ ReplayLaunch Lc) {
    extern __shared__ double smem[];
    double* C = smem;              // row-slice buffer (ld kRLd) or packed diagonal tile
    double* S0 = C + kRCbuf;       // staging, kRKc columns of ld kRStLd
    double* S1 = S0 + kRStage;
    double* sv = S1 + kRStage;     // kNbMax doubles
    __shared__ long long s_slot;
    __shared__ int s_ok;
    const long long total = Lc.total;
    for (;;) {
        if (threadIdx.x == 0) s_slot = (long long)atomicAdd(&Lc.hdr->head, 1ULL);
        __syncthreads();
        const long long slot = s_slot;
        __syncthreads();
        if (slot >= total) break;
        int ti, jb;
        long long item;
        if (Lc.queue) {
            const uint64_t e = Lc.queue[slot];
            jb = (int)(e >> 60);
            ti = (int)((e >> 28) & 0xffffffffULL);
            item = (long long)(e & ((1ULL << 28) - 1));
        } else {
            jb = 0;
            ti = (int)(slot / Lc.job[0].batch);
            item = slot % Lc.job[0].batch;
        }
        if constexpr (WITH_SN) {
            if (Lc.job[jb].sn) {
                __shared__ int s_rm[kNbMax], s_cm[kNbMax];
                sn_task(Lc.snj[jb], ti, item, C, S0, S1, sv, s_rm, s_cm, s_ok);
                continue;
            }
        }
        const ReplayArgs& a = Lc.job[jb];
        const int nb = a.nb;
        const DTask t = a.tasks[ti];
        double* F = a.factor + item * a.fstride;
        int* cnt = a.counters + item * a.ntiles;
        const DTile O = a.tiles[t.tile];
        if (threadIdx.x == 0) s_ok = (*(volatile int*)&a.hdr->status == STC_OK);
        __syncthreads();
        if (a.vals) {
            // value scatter inside the launch: a hosted or explicit column fill first, and
            // no work on a column before its values are in place
            if (t.fill > 0 || t.kind == TASK_FILL) {
                fill_col(a, t.kind == TASK_FILL ? O.J : t.fill - 1, item, F);
                if (t.kind == TASK_FILL) continue;
            }
            if (threadIdx.x == 0 && s_ok)
                s_ok = wait_counter(a.fillflag + item * a.nt + O.J, 1, a.spin, &a.hdr->status);
            __syncthreads();
        }
        if (t.own_wait > 0 && a.y) {
            // fused task sets: a forward-substitution step hosted by this task, run first
            fwd_task(a, t.own_wait - 1, item, F, cnt, C, S0, S1, sv, s_ok);
            __syncthreads();
        }
        if (t.kind == TASK_DIAG) {
            // SYRKs + POTRF on the whole diagonal tile, held as a packed triangle
            if (s_ok) {
                load_diag_packed(C, F + O.off, O, nb);
                __syncthreads();
                for (int ui = t.ubeg; ui < t.uend && s_ok; ++ui) {
                    const DUpd u = a.upds[ui];
                    const DTile A = a.tiles[u.a];
                    unsigned got = 0u;
                    for (int k0 = 0; k0 < u.klen; k0 += kRKc) {
                        const int K = min(kRKc, u.klen - k0);
                        int s0, s1, lo, hi;
                        inner_cols(u, a.imap, false, k0, K, s0, s1);
                        col_ext(a.cext, A, nb, s0, s1, lo, hi);
                        const int e0 = max(u.ra0, lo), e1 = min(u.ra1, hi);
                        if (e0 >= e1) continue;  // the chunk is zero on these rows
                        const unsigned need = off_need(e0, e1, s0, s1, a.slice_h);
                        if (need & ~got) {  // wait for exactly the rows and columns read
                            if (threadIdx.x == 0) s_ok = wait_bits(cnt + u.a, need, a.spin, &a.hdr->status);
                            __syncthreads();
                            if (!s_ok) break;
                            got |= need;
                        }
                        stage_cols(S0, kRStLd, F + A.off, nb, e0, e1 - e0, u, a.imap, false, k0, K);
                        __syncthreads();
                        mma_sub_packed<true>(C, nb, e0, e0, e1 - e0, e1 - e0, S0, kRStLd, S0, kRStLd, K);
                        __syncthreads();
                    }
                }
                if (s_ok) {
                    // columns are published kDiagGroupW at a time as they become final (one
                    // slice holds every row), so the TRSMs of this block column can start
                    // before the whole tile is factored
                    int bad, done = 0;
                    double ls;
                    potrf_packed(C, nb, O.sw, min(O.kd, nb - 1), S0, &bad, &ls, kDiagGroupW, [&](int c1) {
                        store_diag_cols(C, F + O.off, O, nb, done, c1);
                        __threadfence();
                        __syncthreads();
                        if (threadIdx.x == 0) red_release_or(cnt + t.tile, diag_bits(done, c1, 0));
                        done = c1;
                    });
                    if (threadIdx.x == 0) {
                        if (bad >= 0) record_info(a.info + item, O.J * nb + bad + 1);
                        F[a.poff + O.pd_slot] = bad >= 0 ? __longlong_as_double(0x7ff8000000000000LL) : ls;
                    }
                    store_diag_cols(C, F + O.off, O, nb, done, nb);
                    __threadfence();
                    __syncthreads();
                    if (threadIdx.x == 0) red_release_or(cnt + t.tile, diag_bits(done, O.sw, 0));
                }
            }
        } else if (t.kind == TASK_FWD) {
            fwd_task(a, t.tile, item, F, cnt, C, S0, S1, sv, s_ok);
        } else if (t.kind == TASK_SYRK) {
            // rows [rs0, rs1) of (k,k): every SYRK update, lower part only, then their
            // factorization
            const int R = t.rs1 - t.rs0;
            if (s_ok) {
                const double* T = F + O.off;
                for_rc(R, t.rs1, [&](int r, int c) { C[r + c * kRLd] = 0.0; });
                __syncthreads();
                read_diag_rows(T, O, nb, t.rs0, t.rs1, [&](int r, int c, double v) { C[(r - t.rs0) + c * kRLd] = v; });
                __syncthreads();
                for (int ui = t.ubeg; ui < t.uend && s_ok; ++ui) {
                    const DUpd u = a.upds[ui];
                    const DTile A = a.tiles[u.a];
                    unsigned got = 0u;
                    // output rows [d0, rb), columns [r0, rb) (rectangle left of d0, then triangle)
                    const int r0 = u.oc0, d0 = u.ra0, rb = u.ra1;
                    for (int k0 = 0; k0 < u.klen; k0 += kRKc) {
                        const int K = min(kRKc, u.klen - k0);
                        int s0, s1, lo, hi;
                        inner_cols(u, a.imap, false, k0, K, s0, s1);
                        col_ext(a.cext, A, nb, s0, s1, lo, hi);
                        const int q0 = max(r0, lo), e0 = max(d0, lo), e1 = min(rb, hi);
                        if (e0 >= e1) continue;  // the chunk is zero on these rows
                        const unsigned need = off_need(q0, e1, s0, s1, a.slice_h);
                        if (need & ~got) {
                            if (threadIdx.x == 0) s_ok = wait_bits(cnt + u.a, need, a.spin, &a.hdr->status);
                            __syncthreads();
                            if (!s_ok) break;
                            got |= need;
                        }
                        stage_cols(S0, kRStLd, F + A.off, nb, q0, e1 - q0, u, a.imap, false, k0, K);
                        __syncthreads();
                        const int ch = min(d0, e1);
                        if (ch > q0)
                            mma_sub<false>(C + (e0 - t.rs0) + q0 * kRLd, kRLd, e1 - e0, ch - q0,
                                           S0 + (e0 - q0), kRStLd, S0, kRStLd, K);
                        mma_sub<true>(C + (e0 - t.rs0) + e0 * kRLd, kRLd, e1 - e0, e1 - e0,
                                      S0 + (e0 - q0), kRStLd, S0 + (e0 - q0), kRStLd, K);
                        __syncthreads();
                    }
                }
                if (s_ok) slice_factor(a, t, O, F, cnt, item, C, S0, S1, sv, s_ok);
            }
        } else {
            const int R = t.rs1 - t.rs0;
            const int sw = O.sw;
            if (s_ok) {
                load_off(C, kRLd, F + O.off, nb, t.rs0, R, sw);
                __syncthreads();
                for (int ui = t.ubeg; ui < t.uend && s_ok; ++ui) {
                    const DUpd u = a.upds[ui];
                    const DTile A = a.tiles[u.a];
                    const DTile B = a.tiles[u.b];
                    unsigned got_a = 0u, got_b = 0u;
                    for (int k0 = 0; k0 < u.klen; k0 += kRKc) {
                        const int K = min(kRKc, u.klen - k0);
                        int sa0, sa1, sb0, sb1, alo, ahi, blo, bhi;
                        inner_cols(u, a.imap, false, k0, K, sa0, sa1);
                        col_ext(a.cext, A, nb, sa0, sa1, alo, ahi);
                        inner_cols(u, a.imap, true, k0, K, sb0, sb1);
                        col_ext(a.cext, B, nb, sb0, sb1, blo, bhi);
                        // rows of A and (contiguous output) columns of B that are nonzero here
                        const int e0 = max(u.ra0, alo), e1 = min(u.ra1, ahi);
                        int c0 = u.oc0, c1 = u.oc1;
                        if (O.c0 >= 0) { c0 = max(c0, blo - O.c0); c1 = min(c1, bhi - O.c0); }
                        if (e0 >= e1 || c0 >= c1) continue;
                        // rows of B read: the logical columns of output columns [c0, c1)
                        const unsigned need_a = off_need(e0, e1, sa0, sa1, a.slice_h);
                        const unsigned need_b =
                            off_need(max(blo, logical_col(O, a.saind, c0)), min(bhi, logical_col(O, a.saind, c1 - 1) + 1),
                                     sb0, sb1, a.slice_h);
                        if ((need_a & ~got_a) | (need_b & ~got_b)) {
                            if (threadIdx.x == 0)
                                s_ok = wait_bits(cnt + u.a, need_a, a.spin, &a.hdr->status) &&
                                       wait_bits(cnt + u.b, need_b, a.spin, &a.hdr->status);
                            __syncthreads();
                            if (!s_ok) break;
                            got_a |= need_a;
                            got_b |= need_b;
                        }
                        stage_cols(S0, kRStLd, F + A.off, nb, e0, e1 - e0, u, a.imap, false, k0, K);
                        stage_rows_gather(S1, kRStLd, F + B.off, nb, O, a.saind, c0, c1 - c0, u, a.imap, k0, K);
                        __syncthreads();
                        mma_sub<false>(C + (e0 - t.rs0) + c0 * kRLd, kRLd, e1 - e0, c1 - c0, S0, kRStLd,
                                       S1, kRStLd, K);
                        __syncthreads();
                    }
                }
                // TRSM of rows [tr0, tr1) against L_kk restricted to the stored columns
                // L_kk arrives kDiagGroupW columns at a time (per row slice of (k,k))
                const DTile D = a.tiles[t.diag];
                if (s_ok) {
                    // rows of X outside a column group's extent are zero there and stay zero
                    const double* DT = F + D.off;
                    // right-looking by panels of kPb columns: solve panel p as soon as L_kk's
                    // columns up to it are final, publish it, then update the later panels with
                    // it, so the work left after the last columns of L_kk arrive is small
                    for (int p = 0; p < sw; p += kPb) {
                        const int pw = min(kPb, sw - p);
                        if (threadIdx.x == 0) {
                            const int gl = logical_col(O, a.saind, p + pw - 1) / kDiagGroupW;
                            s_ok = wait_bits(cnt + t.diag, (unsigned)D.nfinal & diag_prefix(gl), a.spin,
                                             &a.hdr->status);
                        }
                        __syncthreads();
                        if (!s_ok) break;
                        int lo, hi;
                        col_ext(a.cext, O, nb, p, p + pw - 1, lo, hi);
                        const int y0 = max(t.tr0, lo), y1 = min(t.tr1, hi);
                        if (y0 < y1) {
                            // diagonal block of the panel and its reciprocal diagonal
                            // (consecutive threads along a stored row of a banded L_kk, down a
                            // column of a dense one; leading dimension kPb + 1)
                            const bool band = D.kind == TILE_DIAG_BAND;
                            for (int idx = threadIdx.x; idx < kPb * kPb; idx += kThreads) {
                                const int i = band ? idx / kPb : idx & (kPb - 1);
                                const int j = band ? idx & (kPb - 1) : idx / kPb;
                                double v = 0.0;
                                if (i < pw && j < pw && i >= j)
                                    v = diag_at(DT, D, nb, logical_col(O, a.saind, p + i),
                                                logical_col(O, a.saind, p + j));
                                S0[i + j * (kPb + 1)] = v;
                            }
                            __syncthreads();
                            if (threadIdx.x < pw) sv[threadIdx.x] = 1.0 / S0[threadIdx.x * (kPb + 2)];
                            __syncthreads();
                            trsm_rows(C + (y0 - t.rs0) + p * kRLd, kRLd, y1 - y0, pw, S0, kPb + 1, sv);
                            __syncthreads();
                        }
                        // columns [p, p + pw) of this slice are final: publish them
                        store_off(C + p * kRLd, kRLd, F + O.off + (size_t)p * nb, nb, t.rs0, R, pw);
                        __threadfence();
                        __syncthreads();
                        if (threadIdx.x == 0)
                            red_release_or(cnt + t.tile, 1u << ((p / kPanelW) * kMaxSlices + t.slice));
                        // X(:, pn:sw) -= X(:, p:p+pw) L_kk(later columns, panel p)^T
                        const int pn = p + pw, Cn = sw - pn;
                        if (Cn <= 0 || y0 >= y1) continue;
                        for (int k0 = p; k0 < pn; k0 += kRKc) {
                            const int K = min(kRKc, pn - k0);
                            col_ext(a.cext, O, nb, k0, k0 + K - 1, lo, hi);
                            const int x0 = max(t.tr0, lo), x1 = min(t.tr1, hi);
                            if (x0 >= x1) continue;
                            const int Cp = ((Cn + 3) & ~3) + 4;
                            if (D.kind == TILE_DIAG_BAND) {
                                // along stored rows of L_kk: consecutive threads on consecutive k
                                for (int idx = threadIdx.x; idx < Cp * K; idx += kThreads) {
                                    const int c = idx / K, k = idx - c * K;
                                    S1[c + k * kRStLd] = c < Cn ? diag_at(DT, D, nb, logical_col(O, a.saind, pn + c),
                                                                          logical_col(O, a.saind, k0 + k))
                                                                : 0.0;
                                }
                            } else {
                                for_rc(Cp, K, [&](int c, int k) {
                                    double v = 0.0;
                                    if (c < Cn)
                                        v = diag_at(DT, D, nb, logical_col(O, a.saind, pn + c),
                                                    logical_col(O, a.saind, k0 + k));
                                    S1[c + k * kRStLd] = v;
                                });
                            }
                            __syncthreads();
                            double* X = C + (x0 - t.rs0);
                            mma_sub<false>(X + pn * kRLd, kRLd, x1 - x0, Cn, X + k0 * kRLd, kRLd, S1, kRStLd, K);
                            __syncthreads();
                        }
                    }
                }
            }
        }
        // every task has published its tile's parts itself (completion bits)
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// a1: value scatter, in gather form: every double of every item's factor written once, in order:
// F[b][f] = values[b][src[f]] (src >= 0), 1 (src == -2, padding diagonal) or 0.  Replaces
// the zero-fill plus scattered writes by one coalesced pass over the factor; the source
// map is read once for the whole batch.
__global__ void fill_kernel(const double* __restrict__ vals, long long nnz, long long batch,
                            const int32_t* __restrict__ src, double* __restrict__ F, long long fstride) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long f = tid; f < fstride; f += stride) {
        const int e = __ldg(src + f);
        const double c = e == -2 ? 1.0 : 0.0;
        if (e >= 0) {
            for (long long b = 0; b < batch; ++b) __stcs(F + b * fstride + f, __ldg(vals + b * nnz + e));
        } else {
            for (long long b = 0; b < batch; ++b) __stcs(F + b * fstride + f, c);
        }
    }
}

// a9: logdet = 2 * sum of the per-diagonal-tile partials, fixed order (one warp/item).
__global__ void logdet_kernel(const double* __restrict__ F, long long fstride, long long poff,
                              int np, long long batch, double* __restrict__ out) {
    const long long item = blockIdx.x * (long long)(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (item >= batch) return;
    const double* p = F + item * fstride + poff;
    double s = 0.0;
    for (int i = lane; i < np; i += 32) s += p[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[item] = 2.0 * s;
}

__global__ void to_csc_kernel(const double* __restrict__ F, long long fstride, long long batch,
                              const int64_t* __restrict__ map, long long nnzl, double* __restrict__ out) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = tid; q < nnzl; q += stride) {
        const int64_t m = __ldg(map + q);
        for (long long b = 0; b < batch; ++b) out[b * nnzl + q] = F[b * fstride + m];
    }
}


// ---------------------------------------------------------------------------
// a10: solve.  One persistent kernel over every (item, rhs) chain.  Task k < nt is
// the forward block row k:  y_k = L_kk^{-1} (P b)_k - sum_{n<k} L_kn y_n ;  task nt+i is
// the backward block column k = nt-1-i:  z_k = L_kk^{-T} (y_k - sum_{m>k} L_mk^T z_m),
// written in place of y_k and scattered to x = P^T z.  The diagonal tile is staged in
// shared memory; warp 0 runs the substitution with four rows per lane.
// ---------------------------------------------------------------------------
struct SolveArgs {
    const DTile* tiles;
    const int16_t* saind;
    const int32_t* rowstart;   // per block row: off-diagonal tiles (k,n), n ascending
    const int32_t* rowtiles;
    const int32_t* colstart;   // per block column: tiles (m,k), diagonal first
    const int32_t* diag;
    const int32_t* perm;
    const double* factor;
    long long fstride;
    const double* b;           // [chains][n]
    double* x;                 // [chains][n]
    double* y;                 // workspace [chains][nt*nb]
    int* done;                 // workspace [chains][2*nt]
    WorkHeader* hdr;
    long long chains;          // batch * nrhs
    long long nrhs;
    int nt, nb;
    long long n;
    long long spin;
    int ti0;                   // first step: 0 (forward + backward) or nt (backward only)
};

constexpr int kSolveWarps = kThreads / 32;
constexpr int kSolvePre = kNbMax / 2;  // tile entries per thread held across a wait (forward)
static_assert(kNbMax <= 128 && kThreads == 256, "the solve's register prefetch covers 128 x 128 tiles");
// diagonal tile (>= (nb + 1) nb and (kd + 1) nb doubles) + four 32 x 33 panel triangles
constexpr size_t kSolveSmem = ((size_t)kLdc * kNbMax + 4 * 32 * 33) * sizeof(double);

// Diagonal-block substitution with the unit lower triangular M = L diag(L)^{-1} (Ls
// holds M, its columns scaled beforehand, off the dependency chain), panels of 32: warp 0
// solves the panel's 32x32 triangle with its rows (forward) or columns (backward) in
// registers, one lane per row/column, values broadcast by shuffle, so a step of the chain
// is one shuffle and one FMA; the rows below (forward) or above (backward) the panel are
// then updated with one thread per row.  Forward: v <- M^{-1} v (the caller scales by
// diag(L)^{-1} afterwards); backward: v <- M^{-T} v (the caller scales before).
template <bool BACK>
__device__ void diag_solve(double* v, const double* Ls, const DTile& D, int nb, int w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kd = min(D.kd, nb - 1);
    const int np = (w + 31) / 32;
    for (int qi = 0; qi < np; ++qi) {
        const int p = BACK ? (np - 1 - qi) * 32 : qi * 32;
        const int pw = min(32, w - p);
        if (warp == 0) {
            double Lr[32];
            double vi = 0.0;
            if (lane < pw) {
#pragma unroll
                for (int l = 0; l < 32; ++l) {
                    // forward: row p+lane, columns p+l < row; backward: column p+lane, rows p+l > it
                    const int r = BACK ? p + l : p + lane, c = BACK ? p + lane : p + l;
                    Lr[l] = (l < pw && r > c) ? Ls[r + c * kLdc] : 0.0;
                }
                vi = v[p + lane];
            } else {
#pragma unroll
                for (int l = 0; l < 32; ++l) Lr[l] = 0.0;
            }
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const int j = BACK ? 31 - jj : jj;
                if (j < pw) {
                    const double yj = __shfl_sync(0xffffffffu, vi, j);
                    if (!BACK && lane > j) vi = fma(-Lr[j], yj, vi);
                    if (BACK && lane < j) vi = fma(-Lr[j], yj, vi);
                }
            }
            if (lane < pw) v[p + lane] = vi;
        }
        __syncthreads();
        if (!BACK) {
            const int rend = min(w, p + pw + kd);
            for (int r = p + pw + threadIdx.x; r < rend; r += kThreads) {
                double s0 = v[r], s1 = 0.0;
                for (int l = 0; l < pw; l += 2) {
                    s0 = fma(-Ls[r + (p + l) * kLdc], v[p + l], s0);
                    if (l + 1 < pw) s1 = fma(-Ls[r + (p + l + 1) * kLdc], v[p + l + 1], s1);
                }
                v[r] = s0 + s1;
            }
        } else {
            const int cbeg = max(0, p - kd);
            for (int c = cbeg + threadIdx.x; c < p; c += kThreads) {
                double s0 = v[c], s1 = 0.0;
                for (int l = 0; l < pw; l += 2) {
                    s0 = fma(-Ls[p + l + c * kLdc], v[p + l], s0);
                    if (l + 1 < pw) s1 = fma(-Ls[p + l + 1 + c * kLdc], v[p + l + 1], s1);
                }
                v[c] = s0 + s1;
            }
        }
        __syncthreads();
    }
}

// ---- one-dimensional TMA (cp.async.bulk) into shared memory, completion on an mbarrier
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// src and dst 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Bounded wait for the mbarrier phase `parity` to complete; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit) {
    for (long long it = 0; it <= limit; ++it) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// L_kk[r][c] (r >= c) from a diagonal tile staged in shared memory: a banded tile in its
// storage layout (entry at kd + c + r kd: consecutive rows and consecutive columns both
// land in distinct banks), a dense tile column-major with leading dimension nb + 1.
struct DiagView {
    const double* d;
    int kd, ld;
    bool band;
    __device__ __forceinline__ double at(int r, int c) const {
        if (band) return (r - c > kd) ? 0.0 : d[kd + c + r * kd];
        return d[r + c * ld];
    }
};

// v <- L^{-1} v (forward) or v <- L^{-T} v (backward) for a diagonal tile held in shared
// memory, panels of 32.  Inside a panel warp 0 solves with the unit triangle
// M = L diag(L)^{-1} of the panel's 32 x 32 diagonal block, prepared in Mp by
// prepare_panels (so a step of the dependency chain is one shuffle and one FMA); the
// panel's final entries are stored to ypub and published (one count on *done per panel,
// in the order the panels are solved: first to last forward, last to first backward);
// the rows below (forward) or columns above (backward) are then updated by one thread
// each with the true L.
// Strict lower part of M = L diag(L)^{-1} on the 32 x 32 diagonal block of every panel,
// panel q at Mp + q kMpStride, entry (i, l) at i + 33 l (zero elsewhere), and 1 / L_jj in
// dinv: off the dependency chain of the solve (it needs only the diagonal tile).
constexpr int kMpStride = 32 * 33;
__device__ void prepare_panels(double* Mp, double* dinv, const DiagView& L, int nb) {
    for (int c = threadIdx.x; c < nb; c += kThreads) dinv[c] = 1.0 / L.at(c, c);
    __syncthreads();
    const int np = (nb + 31) / 32;
    for (int idx = threadIdx.x; idx < np * 1024; idx += kThreads) {
        const int q = idx >> 10, i = idx & 31, l = (idx >> 5) & 31;
        const int p = q * 32, pw = min(32, nb - p);
        Mp[q * kMpStride + i + 33 * l] = (i < pw && l < i) ? L.at(p + i, p + l) * dinv[p + l] : 0.0;
    }
}

template <bool BACK>
__device__ void diag_solve_tile(double* v, const DiagView& L, int nb, const double* dinv, const double* Mp,
                                double* ypub, int* done) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int np = (nb + 31) / 32;
    if (BACK) {
        for (int c = threadIdx.x; c < nb; c += kThreads) v[c] *= dinv[c];
        __syncthreads();
    }
    for (int qi = 0; qi < np; ++qi) {
        const int p = BACK ? (np - 1 - qi) * 32 : qi * 32;
        const int pw = min(32, nb - p);
        if (warp == 0) {
            double Lr[32];
            double vi = 0.0;
#pragma unroll
            for (int l = 0; l < 32; ++l) {
                // forward: row p+lane, columns p+l < row; backward: column p+lane, rows p+l > it
                const double* M = Mp + (p / 32) * kMpStride;
                Lr[l] = BACK ? M[l + lane * 33] : M[lane + l * 33];
            }
            if (lane < pw) vi = v[p + lane];
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const int j = BACK ? 31 - jj : jj;
                if (j < pw) {
                    const double wj = __shfl_sync(0xffffffffu, vi, j);
                    if (BACK ? lane < j : lane > j) vi = fma(-Lr[j], wj, vi);
                }
            }
            // the panel's entries are final: store and publish them (one count per panel)
            const double val = BACK ? vi : vi * dinv[p + lane];
            if (lane < pw) {
                v[p + lane] = val;
                __stcg(ypub + p + lane, val);
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) red_release_add(done, 1);
        }
        __syncthreads();
        if (!BACK) {
            const int rend = min(nb, p + pw + L.kd);
            for (int r = p + pw + threadIdx.x; r < rend; r += kThreads) {
                double s0 = v[r], s1 = 0.0;
                int l = 0;
                for (; l + 1 < pw; l += 2) {
                    s0 = fma(-L.at(r, p + l), v[p + l], s0);
                    s1 = fma(-L.at(r, p + l + 1), v[p + l + 1], s1);
                }
                if (l < pw) s0 = fma(-L.at(r, p + l), v[p + l], s0);
                v[r] = s0 + s1;
            }
        } else {
            for (int c = max(0, p - L.kd) + threadIdx.x; c < p; c += kThreads) {
                double s0 = 0.0, s1 = 0.0;
                int l = 0;
                for (; l + 1 < pw; l += 2) {
                    s0 = fma(L.at(p + l, c), v[p + l], s0);
                    s1 = fma(L.at(p + l + 1, c), v[p + l + 1], s1);
                }
                if (l < pw) s0 = fma(L.at(p + l, c), v[p + l], s0);
                v[c] = fma(-(s0 + s1), dinv[c], v[c]);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads, 1) solve_kernel(SolveArgs a) {
    extern __shared__ __align__(16) double smem[];
    double* Dsm = smem;                            // diagonal tile (banded: storage layout, by TMA;
                                                   // dense: column-major, ld nb + 1)
    double* Mp = smem + kLdc * kNbMax;             // unit panel triangles (prepare_panels)
    __shared__ double acc[kSolveWarps * kNbMax];   // per-warp partial sums
    __shared__ double v[kNbMax];                   // block right-hand side / solution
    __shared__ double ysm[kNbMax];                 // the y (or z) block an off-diagonal tile multiplies
    __shared__ double sdinv[kNbMax];               // 1 / L_jj of the diagonal tile
    __shared__ __align__(8) unsigned long long bar;
    __shared__ long long s_slot;
    __shared__ int s_ok;
    const long long total = (2LL * a.nt - a.ti0) * a.chains;
    const int nb = a.nb, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int np = (nb + 31) / 32;                 // panels of a block: its completion count
    __shared__ int s_pb[kNbMax / 32 + 1];          // stored-column start of each panel (forward)
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0;
    for (;;) {
        if (threadIdx.x == 0) s_slot = (long long)atomicAdd(&a.hdr->head, 1ULL);
        __syncthreads();
        const long long slot = s_slot;
        __syncthreads();
        if (slot >= total) break;
        const int ti = (int)(slot / a.chains) + a.ti0;
        const long long ch = slot % a.chains;
        const long long item = ch / a.nrhs;
        const double* F = a.factor + item * a.fstride;
        double* y = a.y + ch * (long long)a.nt * nb;
        int* done = a.done + ch * 2LL * a.nt;
        const bool fwd = ti < a.nt;
        const int k = fwd ? ti : a.nt - 1 - (ti - a.nt);
        const DTile D = a.tiles[a.diag[k]];
        const bool band = D.kind == TILE_DIAG_BAND;
        const DiagView Lv{Dsm, band ? D.kd : min(D.kd, nb - 1), band ? 0 : nb + 1, band};
        if (threadIdx.x == 0) {
            s_ok = (*(volatile int*)&a.hdr->status == STC_OK);
            if (band) {
                // the banded tile is contiguous: bulk copies into shared memory, issued before
                // any wait (the previous step's readers have passed the barriers above)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const unsigned bytes = (unsigned)((D.kd + 1) * nb * sizeof(double));
                mbar_expect_tx(&bar, bytes);
                for (unsigned o = 0; o < bytes; o += 32768u)
                    tma_load_1d((char*)Dsm + o, (const char*)(F + D.off) + o, min(32768u, bytes - o), &bar);
            }
            if (s_ok && !fwd) s_ok = wait_counter(done + k, np, a.spin, &a.hdr->status);
        }
        __syncthreads();
        bool solved = false;
        if (s_ok) {
            for (int i = threadIdx.x; i < kSolveWarps * nb; i += kThreads) acc[i] = 0.0;
            if (!band)
                for_rc(nb, nb, [&](int r, int c) {
                    if (r >= c) Dsm[r + c * (nb + 1)] = __ldcg(F + D.off + r + (size_t)c * nb);
                });
            for (int r = threadIdx.x; r < nb; r += kThreads) {
                const long long g = (long long)k * nb + r;
                v[r] = fwd ? (g < a.n ? a.b[ch * a.n + a.perm[g]] : 0.0) : __ldcg(y + g);
            }
        }
        // the diagonal tile: wait for its bulk copy (issued whatever the status, so always
        // awaited before the buffer is reused or the kernel ends), then prepare the panel
        // triangles of the solve, all before the waits on the other chains' blocks
        if (band) {
            if (!mbar_wait(&bar, parity, a.spin)) {
                if (threadIdx.x == 0) atomicCAS(&a.hdr->status, STC_OK, STC_ERR_TIMEOUT);
                mbar_wait(&bar, parity, a.spin);
                s_ok = 0;
            }
            parity ^= 1u;
        }
        __syncthreads();
        if (s_ok) {
            prepare_panels(Mp, sdinv, Lv, nb);
            __syncthreads();
            if (fwd) {
                // acc -= L_kn y_n over the off-diagonal tiles of block row k (oldest n first),
                // 32 columns of y_n at a time as y_n's panels are published: each thread owns
                // one row and, in every panel, a residue class of the tile's stored columns
                // (s_pb: the stored-column range of each panel), with four accumulators; the
                // tile's entries are loaded to registers before the first wait
                const int G = min(kThreads / nb, kSolveWarps), gr = threadIdx.x % nb, gq = threadIdx.x / nb;
                constexpr int kPer = kSolvePre / 4;  // stored columns per thread and panel
                for (int q = a.rowstart[k]; q < a.rowstart[k + 1]; ++q) {
                    const DTile T = a.tiles[a.rowtiles[q]];
                    const bool act = gq < G && gr >= T.r0 && gr < T.r1;
                    if (threadIdx.x <= np) s_pb[threadIdx.x] = T.sw;
                    __syncthreads();
                    for (int c = threadIdx.x; c < T.sw; c += kThreads) {
                        const int qc = logical_col(T, a.saind, c) >> 5;
                        const int qp = c > 0 ? logical_col(T, a.saind, c - 1) >> 5 : -1;
                        for (int z = qp + 1; z <= qc; ++z) s_pb[z] = c;
                    }
                    __syncthreads();
                    const double* base = F + T.off + gr;
                    double pre[4][kPer];
#pragma unroll
                    for (int z = 0; z < 4; ++z)
#pragma unroll
                        for (int j = 0; j < kPer; ++j) {
                            const int c = (z < np ? s_pb[z] : T.sw) + gq + j * G;
                            pre[z][j] = (act && z < np && c < s_pb[z + 1]) ? __ldcg(base + (size_t)c * nb) : 0.0;
                        }
                    const double* yn = y + (long long)T.J * nb;
                    double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
#pragma unroll
                    for (int z = 0; z < 4; ++z) {
                        if (z >= np) break;
                        const int b0 = s_pb[z], b1 = s_pb[z + 1];
                        if (b0 >= b1) continue;  // no stored column in this panel of y_n
                        if (threadIdx.x == 0) s_ok = wait_counter(done + T.J, z + 1, a.spin, &a.hdr->status);
                        __syncthreads();
                        if (!s_ok) break;
                        for (int c = b0 + threadIdx.x; c < b1; c += kThreads) ysm[c] = __ldcg(yn + logical_col(T, a.saind, c));
                        __syncthreads();
                        if (act) {
#pragma unroll
                            for (int j = 0; j < kPer; j += 4) {
                                const int c = b0 + gq + j * G;
                                if (c < b1) p0 = fma(-pre[z][j], ysm[c], p0);
                                if (c + G < b1) p1 = fma(-pre[z][j + 1], ysm[c + G], p1);
                                if (c + 2 * G < b1) p2 = fma(-pre[z][j + 2], ysm[c + 2 * G], p2);
                                if (c + 3 * G < b1) p3 = fma(-pre[z][j + 3], ysm[c + 3 * G], p3);
                            }
                        }
                    }
                    if (!s_ok) break;
                    if (act) acc[gq * nb + gr] += (p0 + p1) + (p2 + p3);
                    __syncthreads();
                }
            } else {
                // acc -= L_mk^T z_m over the tiles below the diagonal in block column k (oldest
                // m first), 32 rows of z_m at a time as z_m's panels are published (last panel
                // first): each warp owns 16 stored columns (c = 32 g + 4 warp + j), lane l the
                // rows l + 32 i; the 16 partial sums of a lane are reduced over the warp by a
                // reduce-scatter butterfly (16 shuffles and adds per lane, after which lane
                // pair 2v, 2v+1 holds column v's total)
                for (int q = a.colstart[k + 1] - 1; q >= a.colstart[k]; --q) {
                    const DTile T = a.tiles[q];
                    if (T.I == T.J) continue;
                    double pre[4][4][4];
#pragma unroll
                    for (int g = 0; g < 4; ++g)
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int c = 32 * g + warp * 4 + j, r = lane + 32 * i;
                                pre[g][j][i] = (c < T.sw && r >= T.r0 && r < T.r1)
                                                   ? __ldcg(F + T.off + (size_t)c * nb + r) : 0.0;
                            }
                    const double* zm = y + (long long)T.I * nb;
                    double d[16];
#pragma unroll
                    for (int v2 = 0; v2 < 16; ++v2) d[v2] = 0.0;
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) {
                        const int i = 3 - ii;
                        // rows [32 i, 32 i + 32) of z_m: published once np - i panels are
                        if (i >= np || 32 * i >= T.r1 || 32 * i + 32 <= T.r0) continue;
                        if (threadIdx.x == 0) s_ok = wait_counter(done + a.nt + T.I, np - i, a.spin, &a.hdr->status);
                        __syncthreads();
                        if (!s_ok) break;
                        const int r = lane + 32 * i;
                        const double zr = (r >= T.r0 && r < T.r1) ? __ldcg(zm + r) : 0.0;
#pragma unroll
                        for (int g = 0; g < 4; ++g)
#pragma unroll
                            for (int j = 0; j < 4; ++j) d[4 * g + j] = fma(pre[g][j][i], zr, d[4 * g + j]);
                    }
                    if (!s_ok) break;
#pragma unroll
                    for (int st = 0; st < 4; ++st) {
                        const int h = 8 >> st, m = 16 >> st;
                        const bool up = (lane & m) != 0;
#pragma unroll
                        for (int t = 0; t < h; ++t) {
                            const double send = up ? d[t] : d[t + h];
                            const double keep = up ? d[t + h] : d[t];
                            d[t] = keep + __shfl_xor_sync(0xffffffffu, send, m);
                        }
                    }
                    d[0] += __shfl_xor_sync(0xffffffffu, d[0], 1);
                    if ((lane & 1) == 0) {
                        const int vi = lane >> 1;
                        const int c = 32 * (vi >> 2) + warp * 4 + (vi & 3);
                        if (c < T.sw) acc[warp * nb + logical_col(T, a.saind, c)] -= d[0];
                    }
                    __syncthreads();
                }
            }
            for (int r = threadIdx.x; r < nb; r += kThreads) {
                double sacc = 0.0;
                for (int w2 = 0; w2 < kSolveWarps; ++w2) sacc += acc[w2 * nb + r];
                v[r] += sacc;
            }
        }
        __syncthreads();
        if (s_ok) {
            int* dk = done + (fwd ? k : a.nt + k);
            if (fwd) diag_solve_tile<false>(v, Lv, nb, sdinv, Mp, y + (long long)k * nb, dk);
            else diag_solve_tile<true>(v, Lv, nb, sdinv, Mp, y + (long long)k * nb, dk);
            solved = true;
            if (!fwd)
                for (int i = threadIdx.x; i < nb; i += kThreads) {
                    const long long g = (long long)k * nb + i;
                    if (g < a.n) a.x[ch * a.n + a.perm[g]] = v[i];
                }
        }
        // a step that did not solve (a failed wait) still completes its count, so that
        // no later wait depends on it
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0 && !solved) red_release_add(done + (fwd ? k : a.nt + k), np);
    }
}

// ---------------------------------------------------------------------------
// Supernodal route (Sec. 5.4): the same persistent executor over non-uniform cells.
// Each supernode owns a dense column-major panel (its rows x its columns, at most 128
// columns); a cell is the run of the panel's rows owned by one row supernode (at most
// 128 rows).  A device task is a diagonal cell (its SYRK-like updates, then POTRF) or a
// row slice of <= 64 rows of an off-diagonal cell (its GEMM-like updates, then the TRSM
// against the diagonal cell).  An update subtracts A B^T, A = rows [ar0, ar1) of the
// source cell (K,I), B = the source cell (J,I), inner dimension the dense columns of I,
// and scatters the product into the target through sorted-subset row and column maps
// (each row of A lands on one target row, each row of B on one target column).  A
// cell's completion counter counts its finished slices.
// ---------------------------------------------------------------------------

// C(rm[r], cm[c]) -= sum_k A(r,k) B(c,k) for r < R, c < Cn: the tile product of
// mma_tiles with the result scattered through row and column maps (shared memory, each
// map injective).  PACKED: C is a packed lower triangle of width pnb; LOWER: only
// r >= c (rm and cm ascending, so the mapped entry is in the lower triangle).
template <bool LOWER, int TR, int TC, bool PACKED>
__device__ void mma_scatter_tiles(double* __restrict__ C, int ldc, int R, int Cn, const double* __restrict__ A,
                                  int lda, const double* __restrict__ B, int ldb, int K, const int* rm,
                                  const int* cm, int pnb) {
    const int MR = (R + TR - 1) / TR, MC = (Cn + TC - 1) / TC;
    const int count = LOWER ? MR * (MR + 1) / 2 : MR * MC;
    for (int mt = threadIdx.x; mt < count; mt += kThreads) {
        int ri, cj;
        if (LOWER) {
            int r = (int)((sqrtf(8.0f * mt + 1.0f) - 1.0f) * 0.5f);
            while (r * (r + 1) / 2 > mt) --r;
            while ((r + 1) * (r + 2) / 2 <= mt) ++r;
            ri = r;
            cj = mt - r * (r + 1) / 2;
        } else {
            ri = mt % MR;
            cj = mt / MR;
        }
        const int r0 = ri * TR, c0 = cj * TC;
        int ci[TR][TC];
        double acc[TR][TC];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TC; ++j) {
                const int r = r0 + i, c = c0 + j;
                const bool live = r < R && c < Cn && (!LOWER || r >= c);
                ci[i][j] = live ? (PACKED ? pk(pnb, rm[r], cm[c]) : rm[r] + cm[c] * ldc) : -1;
                acc[i][j] = live ? C[ci[i][j]] : 0.0;
            }
        const double* a = A + r0;
        const double* b = B + c0;
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
            double av[TR], bv[TC];
#pragma unroll
            for (int i = 0; i < TR; ++i) av[i] = a[i];
#pragma unroll
            for (int j = 0; j < TC; ++j) bv[j] = b[j];
#pragma unroll
            for (int i = 0; i < TR; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j) acc[i][j] = fma(-av[i], bv[j], acc[i][j]);
            a += lda;
            b += ldb;
        }
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TC; ++j)
                if (ci[i][j] >= 0) C[ci[i][j]] = acc[i][j];
    }
}

template <bool LOWER, bool PACKED>
__device__ __forceinline__ void mma_scatter(double* C, int ldc, int R, int Cn, const double* A, int lda,
                                            const double* B, int ldb, int K, const int* rm, const int* cm,
                                            int pnb) {
    const int m4 = (R + 3) >> 2, n4 = (Cn + 3) >> 2;
    const int c44 = LOWER ? m4 * (m4 + 1) / 2 : m4 * n4;
    if (c44 >= (kThreads * 3) / 4)
        mma_scatter_tiles<LOWER, 4, 4, PACKED>(C, ldc, R, Cn, A, lda, B, ldb, K, rm, cm, pnb);
    else
        mma_scatter_tiles<LOWER, 2, 2, PACKED>(C, ldc, R, Cn, A, lda, B, ldb, K, rm, cm, pnb);
}

// Rows [r0, r0 + R) and inner columns [k0, k0 + K) of a cell into S[r + k * ld], zero
// rows up to the next multiple of 4 (+4), as the micro-tiles read them.
__device__ __forceinline__ void sn_stage(double* S, int ld, const double* F, const SnDevCell& c, int r0, int R,
                                         int k0, int K) {
    const int Rp = ((R + 3) & ~3) + 4;
    const double* base = F + c.off + r0 + (size_t)k0 * c.ld;
    for_rc(Rp, K, [&](int r, int k) { S[r + k * ld] = r < R ? __ldcg(base + r + (size_t)k * c.ld) : 0.0; });
}

// One supernodal task (a diagonal cell or a row slice of an off-diagonal cell) of item
// `item`, executed by the whole CTA: its updates, then POTRF or TRSM, then publication.
// C, S0, S1, sv: the replay kernel's shared buffers; s_rm, s_cm: kNbMax ints of shared
// memory; s_ok: the CTA's shared status flag.
__device__ __forceinline__ void sn_task(const SnArgs& a, int ti, long long item, double* C, double* S0, double* S1,
                                        double* sv, int* s_rm, int* s_cm, int& s_ok) {
    const SnDevTask t = a.tasks[ti];
    const SnDevCell O = a.cells[t.cell];
    double* F = a.factor + item * a.fstride;
    int* cnt = a.counters + item * a.ncells;
    if (threadIdx.x == 0) s_ok = (*(volatile int*)&a.hdr->status == STC_OK);
    __syncthreads();
    if (t.kind == SN_T_DIAG) {
        const int w = O.w;
        if (s_ok) {
            // lower triangle of the diagonal cell -> packed triangle of width w
            for_rc(w, w, [&](int r, int c) {
                if (r >= c) C[pk(w, r, c)] = __ldcg(F + O.off + r + (size_t)c * O.ld);
            });
            __syncthreads();
            for (int ui = t.ubeg; ui < t.uend && s_ok; ++ui) {
                const SnDevUpd u = a.upds[ui];
                const SnDevCell A = a.cells[u.a];
                if (threadIdx.x == 0) s_ok = wait_counter(cnt + u.a, A.nslices, a.spin, &a.hdr->status);
                for (int i = threadIdx.x; i < A.h; i += kThreads) s_rm[i] = a.maps[u.rmap + i];
                __syncthreads();
                if (!s_ok) break;
                for (int k0 = 0; k0 < u.klen; k0 += kRKc) {
                    const int K = min(kRKc, u.klen - k0);
                    sn_stage(S0, kRStLd, F, A, 0, A.h, k0, K);
                    __syncthreads();
                    mma_scatter<true, true>(C, 0, A.h, A.h, S0, kRStLd, S0, kRStLd, K, s_rm, s_rm, w);
                    __syncthreads();
                }
            }
            if (s_ok) {
                int bad;
                double ls;
                potrf_packed(C, w, w, w - 1, S0, &bad, &ls, kPb, [](int) {});
                for_rc(w, w, [&](int r, int c) {
                    if (r >= c) __stcg(F + O.off + r + (size_t)c * O.ld, C[pk(w, r, c)]);
                });
                if (threadIdx.x == 0) {
                    if (bad >= 0) record_info(a.info + item, a.first[O.I] + bad + 1);
                    F[a.poff + O.I] = bad >= 0 ? __longlong_as_double(0x7ff8000000000000LL) : ls;
                }
            }
        }
    } else {
        const int R = t.rs1 - t.rs0, w = O.w;
        if (s_ok) {
            for_rc(R, w, [&](int r, int c) { C[r + c * kRLd] = __ldcg(F + O.off + t.rs0 + r + (size_t)c * O.ld); });
            __syncthreads();
            for (int ui = t.ubeg; ui < t.uend && s_ok; ++ui) {
                const SnDevUpd u = a.upds[ui];
                const SnDevCell A = a.cells[u.a];
                const SnDevCell B = a.cells[u.b];
                const int Ra = u.ar1 - u.ar0;
                if (threadIdx.x == 0)
                    s_ok = wait_counter(cnt + u.a, A.nslices, a.spin, &a.hdr->status) &&
                           wait_counter(cnt + u.b, B.nslices, a.spin, &a.hdr->status);
                for (int i = threadIdx.x; i < Ra; i += kThreads) s_rm[i] = a.maps[u.rmap + u.ar0 + i] - t.rs0;
                for (int j = threadIdx.x; j < B.h; j += kThreads) s_cm[j] = a.maps[u.cmap + j];
                __syncthreads();
                if (!s_ok) break;
                for (int k0 = 0; k0 < u.klen; k0 += kRKc) {
                    const int K = min(kRKc, u.klen - k0);
                    sn_stage(S0, kRStLd, F, A, u.ar0, Ra, k0, K);
                    sn_stage(S1, kRStLd, F, B, 0, B.h, k0, K);
                    __syncthreads();
                    mma_scatter<false, false>(C, kRLd, Ra, B.h, S0, kRStLd, S1, kRStLd, K, s_rm, s_cm, 0);
                    __syncthreads();
                }
            }
            if (s_ok) {
                const SnDevCell D = a.cells[t.diag];
                if (threadIdx.x == 0) s_ok = wait_counter(cnt + t.diag, 1, a.spin, &a.hdr->status);
                __syncthreads();
                if (s_ok) {
                    // X <- X L_JJ^{-T}, right-looking by panels of kPb columns
                    const double* DT = F + D.off;
                    for (int p = 0; p < w; p += kPb) {
                        const int pw = min(kPb, w - p);
                        for (int idx = threadIdx.x; idx < kPb * kPb; idx += kThreads) {
                            const int i = idx & (kPb - 1), j = idx / kPb;
                            S0[i + j * (kPb + 1)] =
                                (i < pw && j < pw && i >= j) ? __ldcg(DT + p + i + (size_t)(p + j) * D.ld) : 0.0;
                        }
                        __syncthreads();
                        if (threadIdx.x < pw) sv[threadIdx.x] = 1.0 / S0[threadIdx.x * (kPb + 2)];
                        __syncthreads();
                        trsm_rows(C + p * kRLd, kRLd, R, pw, S0, kPb + 1, sv);
                        __syncthreads();
                        const int pn = p + pw, Cn = w - pn;
                        if (Cn <= 0) continue;
                        for (int k0 = p; k0 < pn; k0 += kRKc) {
                            const int K = min(kRKc, pn - k0);
                            const int Cp = ((Cn + 3) & ~3) + 4;
                            for_rc(Cp, K, [&](int c, int k) {
                                S1[c + k * kRStLd] = c < Cn ? __ldcg(DT + pn + c + (size_t)(k0 + k) * D.ld) : 0.0;
                            });
                            __syncthreads();
                            mma_sub<false>(C + pn * kRLd, kRLd, R, Cn, C + k0 * kRLd, kRLd, S1, kRStLd, K);
                            __syncthreads();
                        }
                    }
                    for_rc(R, w, [&](int r, int c) { __stcg(F + O.off + t.rs0 + r + (size_t)c * O.ld, C[r + c * kRLd]); });
                }
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) red_release_add(cnt + t.cell, 1);
}

__global__ void __launch_bounds__(kThreads, 2) sn_replay_kernel(const __grid_constant__ SnArgs a) {
    extern __shared__ double smem[];
    double* C = smem;              // row-slice buffer (ld kRLd) or packed diagonal cell
    double* S0 = C + kRCbuf;       // staging, kRKc columns of ld kRStLd
    double* S1 = S0 + kRStage;
    double* sv = S1 + kRStage;     // kNbMax doubles
    __shared__ int s_rm[kNbMax], s_cm[kNbMax];
    __shared__ long long s_slot;
    __shared__ int s_ok;
    const long long total = (long long)a.ntasks * a.batch;
    for (;;) {
        if (threadIdx.x == 0) s_slot = (long long)atomicAdd(&a.hdr->head, 1ULL);
        __syncthreads();
        const long long slot = s_slot;
        __syncthreads();
        if (slot >= total) break;
        sn_task(a, (int)(slot / a.batch), slot % a.batch, C, S0, S1, sv, s_rm, s_cm, s_ok);
    }
}

// Supernodal solve.  One persistent kernel over every (item, rhs) chain; step J < nsn is
// the forward block of supernode J:  y_J = L_JJ^{-1} ((P b)_J - sum_I L_(J,I) y_I) over
// the cells (J, I) that row supernode J owns; step nsn + i is the backward block of
// J = nsn-1-i:  z_J = L_JJ^{-T} (y_J - sum_K L_(K,J)^T z_K) over the cells below J's
// diagonal; z is scattered to x = P^T z.
struct SnSolveArgs {
    const SnDevCell* cells;
    const int16_t* maps;
    const int32_t* cell_cmap;
    const int32_t* first;
    const int32_t* cptr;       // cells of column supernode J: [cptr[J], cptr[J+1]), diagonal first
    const int32_t* rptr_cells; // cells owned by row supernode J
    const int32_t* row_cells;
    const int32_t* perm;
    const double* factor;
    long long fstride;
    const double* b;           // [chains][n]
    double* x;                 // [chains][n]
    double* y;                 // workspace [chains][n]
    int* done;                 // workspace [chains][2*nsn]
    WorkHeader* hdr;
    long long chains, nrhs;
    int nsn;
    long long n, spin;
};

__global__ void __launch_bounds__(kThreads, 1) sn_solve_kernel(SnSolveArgs a) {
    extern __shared__ double smem[];
    double* Ls = smem;                              // diagonal block, L(r,c) at r + c*kLdc
    __shared__ double v[kNbMax], ys[kNbMax], sdinv[kNbMax];
    __shared__ double part[kThreads];
    __shared__ long long s_slot;
    __shared__ int s_ok;
    const long long total = 2LL * a.nsn * a.chains;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_slot = (long long)atomicAdd(&a.hdr->head, 1ULL);
        __syncthreads();
        const long long slot = s_slot;
        __syncthreads();
        if (slot >= total) break;
        const int ti = (int)(slot / a.chains);
        const long long ch = slot % a.chains;
        const long long item = ch / a.nrhs;
        const double* F = a.factor + item * a.fstride;
        double* y = a.y + ch * a.n;
        int* done = a.done + ch * 2LL * a.nsn;
        const bool fwd = ti < a.nsn;
        const int J = fwd ? ti : a.nsn - 1 - (ti - a.nsn);
        const SnDevCell D = a.cells[a.cptr[J]];
        const int w = D.w, c0 = a.first[J];
        if (threadIdx.x == 0) {
            s_ok = (*(volatile int*)&a.hdr->status == STC_OK);
            if (s_ok && !fwd) s_ok = wait_counter(done + J, 1, a.spin, &a.hdr->status);
        }
        __syncthreads();
        if (s_ok) {
            // diagonal block, scaled to the unit lower triangle M = L diag(L)^{-1}
            for_rc(kNbMax, kNbMax, [&](int r, int c) { Ls[r + c * kLdc] = 0.0; });
            __syncthreads();
            for_rc(w, w, [&](int r, int c) {
                if (r >= c) Ls[r + c * kLdc] = __ldcg(F + D.off + r + (size_t)c * D.ld);
            });
            __syncthreads();
            for (int c = threadIdx.x; c < w; c += kThreads) sdinv[c] = 1.0 / Ls[c * (kLdc + 1)];
            for (int r = threadIdx.x; r < kNbMax; r += kThreads) {
                v[r] = 0.0;
                if (r < w) v[r] = fwd ? a.b[ch * a.n + a.perm[c0 + r]] : __ldcg(y + c0 + r);
            }
            __syncthreads();
            for_rc(w, w, [&](int r, int c) { if (r > c) Ls[r + c * kLdc] *= sdinv[c]; });
            __syncthreads();
            if (fwd) {
                // v[map[i]] -= sum_k L_(J,I)[i][k] y_I[k], cells in ascending I
                for (int q = a.rptr_cells[J]; q < a.rptr_cells[J + 1] && s_ok; ++q) {
                    const int cid = a.row_cells[q];
                    const SnDevCell T = a.cells[cid];
                    if (threadIdx.x == 0) s_ok = wait_counter(done + T.I, 1, a.spin, &a.hdr->status);
                    __syncthreads();
                    if (!s_ok) break;
                    const int cI = a.first[T.I];
                    for (int k = threadIdx.x; k < T.w; k += kThreads) ys[k] = __ldcg(y + cI + k);
                    __syncthreads();
                    // two threads per row (T.h <= 128), halves of the inner range
                    const int i = threadIdx.x >> 1, hf = threadIdx.x & 1;
                    double s0 = 0.0, s1 = 0.0;
                    if (i < T.h) {
                        const double* Lr = F + T.off + i;
                        int k = hf;
                        for (; k + 2 < T.w; k += 4) {
                            s0 = fma(__ldcg(Lr + (size_t)k * T.ld), ys[k], s0);
                            s1 = fma(__ldcg(Lr + (size_t)(k + 2) * T.ld), ys[k + 2], s1);
                        }
                        if (k < T.w) s0 = fma(__ldcg(Lr + (size_t)k * T.ld), ys[k], s0);
                    }
                    double sacc = s0 + s1;
                    sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
                    if (i < T.h && hf == 0) v[a.maps[a.cell_cmap[cid] + i]] -= sacc;
                    __syncthreads();
                }
            } else {
                // v[k] -= sum_i L_(K,J)[i][k] z_K[map[i]], cells below the diagonal, last first
                for (int q = a.cptr[J + 1] - 1; q > a.cptr[J] && s_ok; --q) {
                    const SnDevCell T = a.cells[q];
                    if (threadIdx.x == 0) s_ok = wait_counter(done + a.nsn + T.J, 1, a.spin, &a.hdr->status);
                    __syncthreads();
                    if (!s_ok) break;
                    const int cK = a.first[T.J];
                    const int16_t* m = a.maps + a.cell_cmap[q];
                    for (int i = threadIdx.x; i < T.h; i += kThreads) ys[i] = __ldcg(y + cK + m[i]);
                    __syncthreads();
                    for (int k = warp; k < T.w; k += kThreads / 32) {
                        const double* Lc = F + T.off + (size_t)k * T.ld;
                        double d = 0.0;
                        for (int i = lane; i < T.h; i += 32) d = fma(__ldcg(Lc + i), ys[i], d);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
                        if (lane == 0) part[k] = d;
                    }
                    __syncthreads();
                    for (int k = threadIdx.x; k < T.w; k += kThreads) v[k] -= part[k];
                    __syncthreads();
                }
            }
            if (s_ok) {
                DTile Dt{};
                Dt.kd = w - 1;
                if (fwd) {
                    diag_solve<false>(v, Ls, Dt, kNbMax, w);
                    for (int i = threadIdx.x; i < w; i += kThreads) v[i] *= sdinv[i];
                    __syncthreads();
                } else {
                    for (int i = threadIdx.x; i < w; i += kThreads) v[i] *= sdinv[i];
                    __syncthreads();
                    diag_solve<true>(v, Ls, Dt, kNbMax, w);
                }
                for (int i = threadIdx.x; i < w; i += kThreads) {
                    __stcg(y + c0 + i, v[i]);
                    if (!fwd) a.x[ch * a.n + a.perm[c0 + i]] = v[i];
                }
            }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) red_release_add(done + (fwd ? J : a.nsn + J), 1);
    }
}

// DFMA throughput probe: 8 independent FMA chains per thread.
__global__ void fp64_probe_kernel(double* out, long long iters, double a, double b) {
    double c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) c[i] = threadIdx.x * 1e-3 + i;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = fma(c[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += c[i];
    out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

// ---------------------------------------------------------------------------
// a12: selected inverse Sigma = A_p^{-1} on the stored tiles (Takahashi recurrence,
// Takahashi 1973; not in the paper, which leaves selected inversion to separate work),
// one persistent kernel walking block columns in reverse order with per-tile counters.
// Off-diagonal tile:  Sigma_mk = -(sum_j Sigma_(m,j) L_jk) L_kk^{-1}  (stored columns of
// (m,k); entries the symbolic factor proves zero are never read by structural outputs).
// Diagonal tile: Z = sum_j Sigma_jk^T L_jk, then column c = w-1..0 of the tile:
//   Sigma_rc = (-Z_rc - sum_{i>c} L_ic Sigma_ri) / L_cc          (r > c)
//   Sigma_cc = 1/L_cc^2 + (-Z_cc - sum_{i>c} L_ic Sigma_ic) / L_cc
// ---------------------------------------------------------------------------
struct SelinvArgs {
    const DTile* tiles;
    const int16_t* saind;
    const int16_t* sinv;     // [ntiles][nb]
    const DSTask* tasks;
    const DSCon* cons;
    const double* factor;
    double* sigma;
    long long fstride;
    int* counters;           // [batch][ntiles]
    int ntiles;
    WorkHeader* hdr;
    int ntasks;
    long long batch;
    int nb;
    long long spin;
};

__device__ __forceinline__ double sym_at(const double* T, const DTile& d, int nb, int r, int c) {
    return r >= c ? diag_at(T, d, nb, r, c) : diag_at(T, d, nb, c, r);
}

// S[r + k*ld] = get(r, k) for r < R, zero for R <= r < Rp, k < K; consecutive threads on
// consecutive r (RFAST) or consecutive k -- whichever is contiguous in the source -- with
// four loads in flight per thread.
template <bool RFAST, class Get>
__device__ void stage_gather(double* S, int ld, int R, int Rp, int K, Get get) {
    const int n = Rp * K;
    for (int b = threadIdx.x; b < n; b += 4 * kThreads) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = b + u * kThreads;
            const int r = RFAST ? j % Rp : j / K, k = RFAST ? j / Rp : j % K;
            v[u] = (j < n && r < R) ? get(r, k) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = b + u * kThreads;
            const int r = RFAST ? j % Rp : j / K, k = RFAST ? j / Rp : j % K;
            if (j < n) S[r + k * ld] = v[u];
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1) selinv_kernel(SelinvArgs a) {
    extern __shared__ double smem[];
    double* C = smem;
    double* S0 = C + kCbuf;
    double* S1 = S0 + kStage;
    double* sv = S1 + kStage;
    __shared__ long long s_slot;
    __shared__ int s_ok;
    const long long total = (long long)a.ntasks * a.batch;
    const int nb = a.nb;
    constexpr int LDS = kNbMax + 9;  // odd: column-wise staging stores hit distinct banks
    __shared__ int16_t s_idx[2][kNbMax];  // stored-column indices of a contribution's tiles
    for (;;) {
        if (threadIdx.x == 0) s_slot = (long long)atomicAdd(&a.hdr->head, 1ULL);
        __syncthreads();
        const long long slot = s_slot;
        __syncthreads();
        if (slot >= total) break;
        const int ti = (int)(slot / a.batch);
        const long long item = slot % a.batch;
        const DSTask t = a.tasks[ti];
        const double* Lf = a.factor + item * a.fstride;
        double* Sg = a.sigma + item * a.fstride;
        int* cnt = a.counters + item * a.ntiles;
        const DTile O = a.tiles[t.tile];
        const DTile D = a.tiles[t.diag];
        if (threadIdx.x == 0) s_ok = (*(volatile int*)&a.hdr->status == STC_OK);
        __syncthreads();
        if (t.kind == TASK_SOFF && s_ok) {
            const int R = t.r1 - t.r0, sw = O.sw;
            for_rc(R, sw, [&](int r, int c) { C[r + c * kLdc] = 0.0; });
            __syncthreads();
            for (int ci = t.cbeg; ci < t.cend; ++ci) {
                const DSCon cn = a.cons[ci];
                const DTile Lt = a.tiles[cn.ltile];
                const DTile St = a.tiles[cn.stile];
                if (threadIdx.x == 0) s_ok = wait_counter(cnt + cn.stile, 1, a.spin, &a.hdr->status);
                __syncthreads();
                if (!s_ok) break;
                const double* LT = Lf + Lt.off;
                const double* ST = Sg + St.off;
                const int16_t* si_S = a.sinv + (size_t)cn.stile * nb;
                const int16_t* si_L = a.sinv + (size_t)cn.ltile * nb;
                // stored-column indices used by every chunk: Sigma's for the inner rows i
                // (MJ) or the output rows (JM), L's for the output's stored columns
                for (int q = threadIdx.x; q < nb; q += kThreads) {
                    s_idx[0][q] = si_S[q];
                    s_idx[1][q] = q < sw ? si_L[logical_col(O, a.saind, q)] : (int16_t)-1;
                }
                __syncthreads();
                for (int i0 = Lt.r0; i0 < Lt.r1; i0 += kKc) {
                    const int K = min(kKc, Lt.r1 - i0);
                    const int Rp = ((R + 3) & ~3) + 4, Cp = ((sw + 3) & ~3) + 4;
                    if (cn.mode == SCON_MJ) {  // Sigma(m, j): output rows contiguous
                        stage_gather<true>(S0, LDS, R, Rp, K, [&](int r, int kk) {
                            const int sidx = s_idx[0][i0 + kk];
                            return sidx >= 0 ? __ldcg(ST + t.r0 + r + (size_t)sidx * nb) : 0.0;
                        });
                    } else if (cn.mode == SCON_JM) {  // Sigma(j, m)^T: inner rows contiguous
                        stage_gather<false>(S0, LDS, R, Rp, K, [&](int r, int kk) {
                            const int sidx = s_idx[0][t.r0 + r];
                            return sidx >= 0 ? __ldcg(ST + i0 + kk + (size_t)sidx * nb) : 0.0;
                        });
                    } else {
                        stage_gather<true>(S0, LDS, R, Rp, K,
                                           [&](int r, int kk) { return sym_at(ST, St, nb, t.r0 + r, i0 + kk); });
                    }
                    // L(j, k) rows i0.. of the output's stored columns: rows contiguous
                    stage_gather<false>(S1, LDS, sw, Cp, K, [&](int c, int kk) {
                        const int sl = s_idx[1][c];
                        return sl >= 0 ? __ldcg(LT + (i0 + kk) + (size_t)sl * nb) : 0.0;
                    });
                    __syncthreads();
                    mma_sub<false>(C, kLdc, R, sw, S0, LDS, S1, LDS, K);  // C = -sum Sigma L
                    __syncthreads();
                }
            }
            if (s_ok) {
                // X L_g = C on the stored columns, panels from the right (backward)
                const double* DT = Lf + D.off;
                for (int p = ((sw - 1) / kPb) * kPb; p >= 0; p -= kPb) {
                    const int pw = min(kPb, sw - p);
                    for (int k0 = p + pw; k0 < sw; k0 += kKc) {
                        const int K = min(kKc, sw - k0);
                        const int Cp = ((pw + 3) & ~3) + 4;
                        for_rc(Cp, K, [&](int c, int kk) {
                            double v = 0.0;
                            if (c < pw)
                                v = diag_at(DT, D, nb, logical_col(O, a.saind, k0 + kk), logical_col(O, a.saind, p + c));
                            S1[c + kk * LDS] = v;
                        });
                        __syncthreads();
                        mma_sub<false>(C + p * kLdc, kLdc, R, pw, C + k0 * kLdc, kLdc, S1, LDS, K);
                        __syncthreads();
                    }
                    const bool band = D.kind == TILE_DIAG_BAND;
                    for (int idx = threadIdx.x; idx < kPb * kPb; idx += kThreads) {
                        const int i = band ? idx / kPb : idx & (kPb - 1);
                        const int j = band ? idx & (kPb - 1) : idx / kPb;
                        double v = 0.0;
                        if (i < pw && j < pw && i >= j)
                            v = diag_at(DT, D, nb, logical_col(O, a.saind, p + i), logical_col(O, a.saind, p + j));
                        S0[i + j * (kPb + 1)] = v;
                    }
                    __syncthreads();
                    if (threadIdx.x < pw) sv[threadIdx.x] = 1.0 / S0[threadIdx.x * (kPb + 2)];
                    __syncthreads();
                    trsm_rows_dir<true>(C + p * kLdc, kLdc, R, pw, S0, kPb + 1, sv);
                    __syncthreads();
                }
                double* T = Sg + O.off;
                for_rc(R, sw, [&](int r, int c) { __stcg(T + t.r0 + r + (size_t)c * nb, C[r + c * kLdc]); });
            }
        } else if (t.kind == TASK_SDIAG && s_ok) {
            const int w = O.sw;
            const int kd = min(O.kd, nb - 1);
            for_rc(nb, nb, [&](int r, int c) { C[r + c * kLdc] = 0.0; });
            __syncthreads();
            for (int ci = t.cbeg; ci < t.cend; ++ci) {
                const DSCon cn = a.cons[ci];
                const DTile Tt = a.tiles[cn.ltile];
                if (threadIdx.x == 0) s_ok = wait_counter(cnt + cn.stile, 1, a.spin, &a.hdr->status);
                __syncthreads();
                if (!s_ok) break;
                const double* LT = Lf + Tt.off;
                const double* ST = Sg + Tt.off;
                const bool contig = Tt.c0 >= 0;
                const int M = contig ? Tt.sw : w;   // rows/cols of the Z block
                const int16_t* si = a.sinv + (size_t)cn.ltile * nb;
                for (int q = threadIdx.x; q < nb; q += kThreads) s_idx[0][q] = contig ? (int16_t)q : si[q];
                __syncthreads();
                for (int i0 = Tt.r0; i0 < Tt.r1; i0 += kKc) {
                    const int K = min(kKc, Tt.r1 - i0);
                    const int Mp = ((M + 3) & ~3) + 4;
                    // rows i0.. of the stored columns: contiguous along the inner index
                    stage_gather<false>(S0, LDS, M, Mp, K, [&](int r, int kk) {
                        const int sidx = s_idx[0][r];
                        return sidx >= 0 ? __ldcg(ST + (i0 + kk) + (size_t)sidx * nb) : 0.0;
                    });
                    stage_gather<false>(S1, LDS, M, Mp, K, [&](int r, int kk) {
                        const int sidx = s_idx[0][r];
                        return sidx >= 0 ? __ldcg(LT + (i0 + kk) + (size_t)sidx * nb) : 0.0;
                    });
                    __syncthreads();
                    double* Cz = contig ? C + Tt.c0 * (1 + kLdc) : C;
                    mma_sub<true>(Cz, kLdc, M, M, S0, LDS, S1, LDS, K);  // C = -Z (lower)
                    __syncthreads();
                }
            }
            if (s_ok) {
                // packed lower triangle of L_kk in the staging area: (r, c) at c*nb - c(c-1)/2 + r - c
                double* Lp = S0;
                const double* DT = Lf + D.off;
                read_diag_rows(DT, D, nb, 0, nb,
                               [&](int r, int c, double v) { Lp[c * nb - c * (c - 1) / 2 + (r - c)] = v; });
                __syncthreads();
                for (int c = w - 1; c >= 0; --c) {
                    const double* Lc = Lp + c * nb - c * (c - 1) / 2 - c;  // Lc[i] = L[i][c]
                    const double inv = 1.0 / Lc[c];
                    const int iend = min(w, c + kd + 1);
                    for (int r = c + 1 + threadIdx.x; r < iend; r += kThreads) {
                        double s0 = C[r + c * kLdc], s1 = 0.0;
                        int i = c + 1;
                        for (; i + 1 < iend; i += 2) {
                            s0 = fma(-Lc[i], i >= r ? C[i + r * kLdc] : C[r + i * kLdc], s0);
                            s1 = fma(-Lc[i + 1], i + 1 >= r ? C[i + 1 + r * kLdc] : C[r + (i + 1) * kLdc], s1);
                        }
                        if (i < iend) s0 = fma(-Lc[i], i >= r ? C[i + r * kLdc] : C[r + i * kLdc], s0);
                        C[r + c * kLdc] = (s0 + s1) * inv;
                    }
                    __syncthreads();
                    if (threadIdx.x < 32) {
                        double sacc = 0.0;
                        for (int i = c + 1 + threadIdx.x; i < iend; i += 32) sacc = fma(Lc[i], C[i + c * kLdc], sacc);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
                        if (threadIdx.x == 0) C[c + c * kLdc] = inv * inv + (C[c + c * kLdc] - sacc) * inv;
                    }
                    __syncthreads();
                }
                store_diag(C, Sg + O.off, O, nb);
            }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) red_release_add(cnt + t.tile, 1);
    }
}

// ---------------------------------------------------------------------------
// Selected inverse on the supernodal layout (Takahashi's recurrence over the supernodes,
// walked in reverse; not in the paper, which leaves selected inversion to separate work).
// Off-diagonal task, rows [rs0, rs1) of cell (K,J):
//   Sigma(K,J) = -(sum over J's cells (K',J) of Sigma(rows_K, rows_K') L(K',J)) L_JJ^{-1}
// with Sigma(rows_K, rows_K') read from the diagonal cell of K (K' = K), from the cell
// (K,K') of supernode K' (K' < K) or transposed from the cell (K',K) of K (K' > K), each
// row located by a search of the source cell's row list.  Diagonal task: C = -Z,
// Z = sum over J's cells of Sigma(K',J)^T L(K',J), then the element recurrence inside the
// diagonal block (as for a diagonal tile).
// ---------------------------------------------------------------------------
struct SnSelinvArgs {
    const SnDevCell* cells;
    const SnSTask* tasks;
    const SnSCon* cons;
    const int32_t* rows;       // the supernodes' row lists
    const int32_t* rowoff;     // per cell: offset of its first row in rows
    const int32_t* first;      // first column of each supernode
    const double* factor;
    double* sigma;
    long long fstride;
    int* counters;             // [batch][ncells]
    int ncells;
    WorkHeader* hdr;
    int ntasks;
    long long batch;
    long long spin;
};

__global__ void __launch_bounds__(kThreads, 1) sn_selinv_kernel(SnSelinvArgs a) {
    extern __shared__ double smem[];
    double* C = smem;
    double* S0 = C + kCbuf;
    double* S1 = S0 + kStage;
    double* sv = S1 + kStage;
    __shared__ long long s_slot;
    __shared__ int s_ok;
    __shared__ int ia[kNbMax], ja[kNbMax], srow[kNbMax];
    constexpr int LDS = kNbMax + 9;
    const long long total = (long long)a.ntasks * a.batch;
    for (;;) {
        if (threadIdx.x == 0) s_slot = (long long)atomicAdd(&a.hdr->head, 1ULL);
        __syncthreads();
        const long long slot = s_slot;
        __syncthreads();
        if (slot >= total) break;
        const int ti = (int)(slot / a.batch);
        const long long item = slot % a.batch;
        const SnSTask t = a.tasks[ti];
        const double* Lf = a.factor + item * a.fstride;
        double* Sg = a.sigma + item * a.fstride;
        int* cnt = a.counters + item * a.ncells;
        const SnDevCell O = a.cells[t.cell];
        const SnDevCell D = a.cells[t.diag];
        const int w = D.w;
        const double* DL = Lf + D.off;  // L_JJ(r, c) = DL[r + c * D.ld], r >= c
        if (threadIdx.x == 0) s_ok = (*(volatile int*)&a.hdr->status == STC_OK);
        __syncthreads();
        if (t.kind == SN_S_OFF && s_ok) {
            const int R = t.rs1 - t.rs0;
            const int K = O.J;
            for_rc(R, w, [&](int r, int c) { C[r + c * kLdc] = 0.0; });
            __syncthreads();
            for (int ci = t.cbeg; ci < t.cend; ++ci) {
                const SnSCon q = a.cons[ci];
                const SnDevCell Lc = a.cells[q.lcell];
                const SnDevCell Sc = a.cells[q.scell];
                const int Kp = Lc.J, h = Lc.h;
                if (threadIdx.x == 0) s_ok = wait_counter(cnt + q.scell, Sc.nslices, a.spin, &a.hdr->status);
                // row lists: the source cell's (for the searches) and the index maps of the
                // gathered block G(i, j) = Sigma(row i of the target slice, row j of (K',J))
                for (int i = threadIdx.x; i < Sc.h; i += kThreads) srow[i] = a.rows[a.rowoff[q.scell] + i];
                __syncthreads();
                if (!s_ok) break;
                const int* rt = a.rows + a.rowoff[t.cell] + t.rs0;
                const int* rp = a.rows + a.rowoff[q.lcell];
                auto find = [&](int r) {  // position of global row r in the source cell's rows
                    int lo = 0, hi = Sc.h;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (srow[mid] < r) lo = mid + 1; else hi = mid;
                    }
                    return lo;
                };
                for (int i = threadIdx.x; i < R; i += kThreads)
                    ia[i] = q.mode == SN_SC_LOWER ? find(rt[i]) : rt[i] - a.first[K];
                for (int j = threadIdx.x; j < h; j += kThreads)
                    ja[j] = q.mode == SN_SC_UPPER ? find(rp[j]) : rp[j] - a.first[q.mode == SN_SC_SAME ? K : Kp];
                __syncthreads();
                const double* ST = Sg + Sc.off;
                const double* LT = Lf + Lc.off;
                for (int j0 = 0; j0 < h; j0 += kKc) {
                    const int Kc = min(kKc, h - j0);
                    const int Rp = ((R + 3) & ~3) + 4, Cp = ((w + 3) & ~3) + 4;
                    stage_gather<true>(S0, LDS, R, Rp, Kc, [&](int r, int k) {
                        const int x = ia[r], y = ja[j0 + k];
                        if (q.mode == SN_SC_SAME)
                            return __ldcg(ST + max(x, y) + (size_t)min(x, y) * Sc.ld);
                        if (q.mode == SN_SC_LOWER) return __ldcg(ST + x + (size_t)y * Sc.ld);
                        return __ldcg(ST + y + (size_t)x * Sc.ld);
                    });
                    // L(K',J) rows j0.. (contiguous along the inner index)
                    stage_gather<false>(S1, LDS, w, Cp, Kc,
                                        [&](int c, int k) { return __ldcg(LT + (j0 + k) + (size_t)c * Lc.ld); });
                    __syncthreads();
                    mma_sub<false>(C, kLdc, R, w, S0, LDS, S1, LDS, Kc);  // C = -sum G L
                    __syncthreads();
                }
            }
            if (s_ok) {
                // X L_JJ = C, panels from the right (backward)
                for (int p = ((w - 1) / kPb) * kPb; p >= 0; p -= kPb) {
                    const int pw = min(kPb, w - p);
                    for (int k0 = p + pw; k0 < w; k0 += kKc) {
                        const int Kc = min(kKc, w - k0);
                        const int Cp = ((pw + 3) & ~3) + 4;
                        for_rc(Cp, Kc, [&](int c, int kk) {
                            S1[c + kk * LDS] = c < pw ? __ldcg(DL + (k0 + kk) + (size_t)(p + c) * D.ld) : 0.0;
                        });
                        __syncthreads();
                        mma_sub<false>(C + p * kLdc, kLdc, R, pw, C + k0 * kLdc, kLdc, S1, LDS, Kc);
                        __syncthreads();
                    }
                    for (int idx = threadIdx.x; idx < kPb * kPb; idx += kThreads) {
                        const int i = idx & (kPb - 1), j = idx / kPb;
                        S0[i + j * (kPb + 1)] =
                            (i < pw && j < pw && i >= j) ? __ldcg(DL + (p + i) + (size_t)(p + j) * D.ld) : 0.0;
                    }
                    __syncthreads();
                    if (threadIdx.x < pw) sv[threadIdx.x] = 1.0 / S0[threadIdx.x * (kPb + 2)];
                    __syncthreads();
                    trsm_rows_dir<true>(C + p * kLdc, kLdc, R, pw, S0, kPb + 1, sv);
                    __syncthreads();
                }
                double* T = Sg + O.off + t.rs0;
                for_rc(R, w, [&](int r, int c) { __stcg(T + r + (size_t)c * O.ld, C[r + c * kLdc]); });
            }
        } else if (t.kind == SN_S_DIAG && s_ok) {
            for_rc(w, w, [&](int r, int c) { C[r + c * kLdc] = 0.0; });
            __syncthreads();
            for (int ci = t.cbeg; ci < t.cend; ++ci) {
                const SnSCon q = a.cons[ci];
                const SnDevCell Lc = a.cells[q.lcell];
                if (threadIdx.x == 0) s_ok = wait_counter(cnt + q.scell, Lc.nslices, a.spin, &a.hdr->status);
                __syncthreads();
                if (!s_ok) break;
                const double* ST = Sg + Lc.off;
                const double* LT = Lf + Lc.off;
                for (int i0 = 0; i0 < Lc.h; i0 += kKc) {
                    const int Kc = min(kKc, Lc.h - i0);
                    const int Mp = ((w + 3) & ~3) + 4;
                    stage_gather<false>(S0, LDS, w, Mp, Kc,
                                        [&](int r, int k) { return __ldcg(ST + (i0 + k) + (size_t)r * Lc.ld); });
                    stage_gather<false>(S1, LDS, w, Mp, Kc,
                                        [&](int r, int k) { return __ldcg(LT + (i0 + k) + (size_t)r * Lc.ld); });
                    __syncthreads();
                    mma_sub<true>(C, kLdc, w, w, S0, LDS, S1, LDS, Kc);  // C = -Z (lower)
                    __syncthreads();
                }
            }
            if (s_ok) {
                // packed lower triangle of L_JJ: (r, c) at c*w - c(c-1)/2 + r - c
                double* Lp = S0;
                for_rc(w, w, [&](int r, int c) {
                    if (r >= c) Lp[c * w - c * (c - 1) / 2 + (r - c)] = __ldcg(DL + r + (size_t)c * D.ld);
                });
                __syncthreads();
                for (int c = w - 1; c >= 0; --c) {
                    const double* Lcol = Lp + c * w - c * (c - 1) / 2 - c;  // Lcol[i] = L[i][c]
                    const double inv = 1.0 / Lcol[c];
                    for (int r = c + 1 + threadIdx.x; r < w; r += kThreads) {
                        double s0 = C[r + c * kLdc], s1 = 0.0;
                        int i = c + 1;
                        for (; i + 1 < w; i += 2) {
                            s0 = fma(-Lcol[i], i >= r ? C[i + r * kLdc] : C[r + i * kLdc], s0);
                            s1 = fma(-Lcol[i + 1], i + 1 >= r ? C[i + 1 + r * kLdc] : C[r + (i + 1) * kLdc], s1);
                        }
                        if (i < w) s0 = fma(-Lcol[i], i >= r ? C[i + r * kLdc] : C[r + i * kLdc], s0);
                        C[r + c * kLdc] = (s0 + s1) * inv;
                    }
                    __syncthreads();
                    if (threadIdx.x < 32) {
                        double sacc = 0.0;
                        for (int i = c + 1 + threadIdx.x; i < w; i += 32) sacc = fma(Lcol[i], C[i + c * kLdc], sacc);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
                        if (threadIdx.x == 0) C[c + c * kLdc] = inv * inv + (C[c + c * kLdc] - sacc) * inv;
                    }
                    __syncthreads();
                }
                double* T = Sg + D.off;
                for_rc(w, w, [&](int r, int c) {
                    if (r >= c) __stcg(T + r + (size_t)c * D.ld, C[r + c * kLdc]);
                });
            }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) red_release_add(cnt + t.cell, 1);
    }
}

// d logdet / d a_e = gout_b (2 - delta_e) Sigma_e, gathered through the value map.
__global__ void grad_gather_kernel(const double* __restrict__ Sg, long long fstride, long long batch,
                                   const int64_t* __restrict__ map, const int8_t* __restrict__ vdiag, long long nnz,
                                   const double* __restrict__ gout, double* __restrict__ g, int accumulate) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = tid; e < nnz; e += stride) {
        const int64_t m = __ldg(map + e);
        const double w = vdiag[e] ? 1.0 : 2.0;
        for (long long b = 0; b < batch; ++b) {
            double v = w * Sg[b * fstride + m] * (gout ? gout[b] : 1.0);
            if (accumulate) v += g[b * nnz + e];
            g[b * nnz + e] = v;
        }
    }
}

// g_e = scale_b (2 - delta_e)/2 (u_i v_j + u_j v_i) for A entry e = (i, j).
__global__ void outer_grad_kernel(const int32_t* __restrict__ arow, const int32_t* __restrict__ acol,
                                  const int8_t* __restrict__ vdiag, long long nnz, long long batch,
                                  const double* __restrict__ u, const double* __restrict__ v, long long n,
                                  const double* __restrict__ scale, double* __restrict__ g, int accumulate) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = tid; e < nnz; e += stride) {
        const long long i = arow[e], j = acol[e];
        const double w = vdiag[e] ? 0.5 : 1.0;
        for (long long b = 0; b < batch; ++b) {
            const double* ub = u + b * n;
            const double* vb = v + b * n;
            double val = w * (ub[i] * vb[j] + ub[j] * vb[i]) * (scale ? scale[b] : 1.0);
            if (accumulate) val += g[b * nnz + e];
            g[b * nnz + e] = val;
        }
    }
}

// out_b = x_b^T A_b x_b = sum_e (2 - delta_e) a_e x_i x_j  (one block per item, fixed order)
__global__ void quad_form_kernel(const int32_t* __restrict__ arow, const int32_t* __restrict__ acol,
                                 const int8_t* __restrict__ vdiag, long long nnz, const double* __restrict__ vals,
                                 const double* __restrict__ x, long long n, double* __restrict__ out) {
    __shared__ double red[kThreads / 32];
    const long long b = blockIdx.x;
    const double* xb = x + b * n;
    const double* ab = vals + b * nnz;
    double s = 0.0;
    for (long long e = threadIdx.x; e < nnz; e += blockDim.x)
        s += (vdiag[e] ? 1.0 : 2.0) * ab[e] * xb[arow[e]] * xb[acol[e]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
        out[b] = t;
    }
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
struct DevInfo {
    int sms = 0;
    bool attr_set = false;
};
DevInfo g_dev[64];
std::mutex g_dev_mu;

int device_info(int* dev, int* sms) {
    if (cudaGetDevice(dev) != cudaSuccess) return STC_ERR_CUDA;
    if (*dev < 0 || *dev >= 64) return STC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(g_dev_mu);
    DevInfo& d = g_dev[*dev];
    if (!d.attr_set) {
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, *dev) != cudaSuccess) return STC_ERR_CUDA;
        if (cudaFuncSetAttribute(replay_kernel_t<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRSmemBytes) != cudaSuccess)
            return STC_ERR_CUDA;
        if (cudaFuncSetAttribute(replay_kernel_t<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRSmemBytes) != cudaSuccess)
            return STC_ERR_CUDA;
        if (cudaFuncSetAttribute(selinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess)
            return STC_ERR_CUDA;
        if (cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSolveSmem) != cudaSuccess)
            return STC_ERR_CUDA;
        if (cudaFuncSetAttribute(sn_replay_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRSmemBytes) !=
            cudaSuccess)
            return STC_ERR_CUDA;
        if (cudaFuncSetAttribute(sn_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSolveSmem) !=
            cudaSuccess)
            return STC_ERR_CUDA;
        if (cudaFuncSetAttribute(sn_selinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
            cudaSuccess)
            return STC_ERR_CUDA;
        d.attr_set = true;
    }
    *sms = d.sms;
    return STC_OK;
}

template <class T>
int upload(T** dst, const std::vector<T>& src) {
    *dst = nullptr;
    if (src.empty()) return STC_OK;
    if (cudaMalloc((void**)dst, src.size() * sizeof(T)) != cudaSuccess) return STC_ERR_OUT_OF_MEMORY;
    if (cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return STC_ERR_CUDA;
    return STC_OK;
}

void free_dev(stc_plan* P) {
    DevPlanArrays& d = P->dev;
    void* ptrs[] = {d.saind, d.cext, d.value_map, d.pad_diag, d.csc_map, d.fill_src, d.perm, d.srow_beg,
                    d.srow_tiles, d.scol_beg, d.diag_tile, d.sinv, d.stasks, d.scons, d.vdiag,
                    d.arow, d.acol};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    d = DevPlanArrays{};
    SnDev& q = P->sndev;
    void* sptrs[] = {q.cells, q.tasks, q.upds, q.maps, q.first, q.cell_cmap, q.cptr, q.rptr_cells, q.row_cells,
                     q.value_map, q.csc_map, q.fill_src, q.stasks, q.scons, q.rows, q.cell_rowoff};
    for (void* p : sptrs)
        if (p) cudaFree(p);
    q = SnDev{};
    {
        std::lock_guard<std::mutex> g(P->own_mu);
        if (P->own_ws) cudaFree(P->own_ws);
        if (P->own_sig) cudaFree(P->own_sig);
        P->own_ws = P->own_sig = nullptr;
        P->own_ws_bytes = P->own_sig_bytes = 0;
    }
    for (auto& kv : P->tasksets) {
        TaskSet* ts = kv.second.get();
        if (ts->d_tasks) cudaFree(ts->d_tasks);
        if (ts->d_upds) cudaFree(ts->d_upds);
        if (ts->d_imap) cudaFree(ts->d_imap);
        if (ts->d_tiles) cudaFree(ts->d_tiles);
        ts->d_tasks = nullptr; ts->d_upds = nullptr; ts->d_imap = nullptr; ts->d_tiles = nullptr;
        ts->device = -1;
    }
}

// Host allocation failures while a task set or a device copy is prepared come back as
// STC_ERR_OUT_OF_MEMORY instead of unwinding through the C ABI.
template <class F>
int no_throw(F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return STC_ERR_OUT_OF_MEMORY;
    } catch (const std::length_error&) {
        return STC_ERR_OUT_OF_MEMORY;
    } catch (...) {
        return STC_ERR_INVALID_ARG;
    }
}

// The plan's device task list for `slices` row slices (built on the host on first use).
int get_taskset(stc_plan* P, int32_t slices, bool bl_order, TaskSet** out, bool fwd = false) {
    *out = nullptr;
    return no_throw([&] {
        *out = P->taskset(slices, bl_order, fwd);
        return STC_OK;
    });
}

// Device copies of the plan's arrays on the current device (synchronous on first use).
int ensure_plan_impl(stc_plan* P, int dev);
int ensure_plan(stc_plan* P, int dev) {
    return no_throw([&] { return ensure_plan_impl(P, dev); });
}
int ensure_plan_impl(stc_plan* P, int dev) {
    std::lock_guard<std::mutex> g(P->mu);
    if (P->dev.device == dev) return STC_OK;
    if (P->dev.device >= 0) free_dev(P);
    DevPlanArrays& d = P->dev;
    int rc;
    std::vector<int32_t> perm32(P->perm.begin(), P->perm.end());
    if ((rc = upload(&d.saind, P->saind))) return rc;
    if ((rc = upload(&d.cext, P->cext))) return rc;
    if ((rc = upload(&d.value_map, P->value_map))) return rc;
    if ((rc = upload(&d.pad_diag, P->pad_diag))) return rc;
    {
        std::vector<int32_t> src((size_t)P->factor_doubles, -1);
        for (int64_t e = 0; e < P->nnzA; ++e) src[P->value_map[e]] = (int32_t)e;
        for (int64_t f : P->pad_diag) src[f] = -2;
        if ((rc = upload(&d.fill_src, src))) return rc;
    }
    if ((rc = upload(&d.csc_map, P->csc_map))) return rc;
    if ((rc = upload(&d.perm, perm32))) return rc;
    if ((rc = upload(&d.srow_beg, P->rowstart))) return rc;
    if ((rc = upload(&d.srow_tiles, P->rowtiles))) return rc;
    if ((rc = upload(&d.scol_beg, P->colstart))) return rc;
    if ((rc = upload(&d.diag_tile, P->diag_tile))) return rc;
    if ((rc = upload(&d.sinv, P->sinv))) return rc;
    if ((rc = upload(&d.stasks, P->stasks))) return rc;
    if ((rc = upload(&d.scons, P->scons))) return rc;
    if ((rc = upload(&d.vdiag, P->vdiag))) return rc;
    if ((rc = upload(&d.arow, P->arow))) return rc;
    if ((rc = upload(&d.acol, P->acol))) return rc;
    d.device = dev;
    return STC_OK;
}

int ensure_taskset_impl(stc_plan* P, TaskSet* ts, int dev);
int ensure_taskset(stc_plan* P, TaskSet* ts, int dev) {
    return no_throw([&] { return ensure_taskset_impl(P, ts, dev); });
}
int ensure_taskset_impl(stc_plan* P, TaskSet* ts, int dev) {
    std::lock_guard<std::mutex> g(P->mu);
    if (ts->device == dev) return STC_OK;
    std::vector<DTile> tiles = P->tiles;
    for (size_t t = 0; t < tiles.size(); ++t) tiles[t].nfinal = ts->nfinal[t];
    int rc;
    if ((rc = upload(&ts->d_tiles, tiles))) return rc;
    if ((rc = upload(&ts->d_tasks, ts->tasks))) return rc;
    if ((rc = upload(&ts->d_upds, ts->upds))) return rc;
    std::vector<int16_t> im = ts->imap;
    if (im.empty()) im.push_back(0);
    if ((rc = upload(&ts->d_imap, im))) return rc;
    ts->device = dev;
    return STC_OK;
}

// Device copies of the supernodal layout (synchronous on first use per device).
int ensure_sn_impl(stc_plan* P, int dev) {
    const SnPlan& S = P->supernodal();
    std::lock_guard<std::mutex> g(P->mu);
    SnDev& d = P->sndev;
    if (d.device == dev) return STC_OK;
    if (d.device >= 0) return STC_ERR_UNSUPPORTED;  // one device per plan's supernodal copy
    int rc;
    std::vector<int32_t> cptr(S.cptr.begin(), S.cptr.end());
    std::vector<int16_t> maps = S.maps;
    if (maps.empty()) maps.push_back(0);
    std::vector<int32_t> rc_list = S.row_cells;
    if (rc_list.empty()) rc_list.push_back(0);
    if ((rc = upload(&d.cells, S.dcells))) return rc;
    if ((rc = upload(&d.tasks, S.dtasks))) return rc;
    if ((rc = upload(&d.upds, S.dupds))) return rc;
    if ((rc = upload(&d.maps, maps))) return rc;
    if ((rc = upload(&d.first, S.first))) return rc;
    if ((rc = upload(&d.cell_cmap, S.cell_cmap))) return rc;
    if ((rc = upload(&d.cptr, cptr))) return rc;
    if ((rc = upload(&d.rptr_cells, S.rptr_cells))) return rc;
    if ((rc = upload(&d.row_cells, rc_list))) return rc;
    if ((rc = upload(&d.value_map, S.value_map))) return rc;
    if ((rc = upload(&d.csc_map, S.csc_map))) return rc;
    {
        std::vector<int32_t> src((size_t)S.item_doubles(), -1);
        for (int64_t e = 0; e < P->nnzA; ++e) src[S.value_map[e]] = (int32_t)e;
        if ((rc = upload(&d.fill_src, src))) return rc;
    }
    std::vector<SnSCon> scons = S.scons;
    if (scons.empty()) scons.push_back(SnSCon{});
    if ((rc = upload(&d.stasks, S.stasks))) return rc;
    if ((rc = upload(&d.scons, scons))) return rc;
    if ((rc = upload(&d.rows, S.rows))) return rc;
    if ((rc = upload(&d.cell_rowoff, S.cell_rowoff))) return rc;
    d.device = dev;
    return STC_OK;
}
int ensure_sn(stc_plan* P, int dev) {
    return no_throw([&] { return ensure_sn_impl(P, dev); });
}

// The plan's own workspace (sigma = false) or selected-inverse scratch (sigma = true) of
// at least `bytes`, for callers that pass a NULL buffer.  Growing it frees the old buffer
// (cudaFree waits for the device) and allocates a new one, so the first call of a size
// synchronizes; calls that use it must not overlap on the GPU.
int own_buffer(stc_plan* P, bool sigma, size_t bytes, void** out) {
    std::lock_guard<std::mutex> g(P->own_mu);
    void*& ptr = sigma ? P->own_sig : P->own_ws;
    size_t& have = sigma ? P->own_sig_bytes : P->own_ws_bytes;
    if (have < bytes) {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        have = 0;
        if (cudaMalloc(&ptr, std::max<size_t>(bytes, 256)) != cudaSuccess) {
            ptr = nullptr;
            return STC_ERR_OUT_OF_MEMORY;
        }
        have = std::max<size_t>(bytes, 256);
    }
    *out = ptr;
    return STC_OK;
}

// Two CTAs per SM hide one CTA's waits behind the other's arithmetic when many items
// are in flight; with few items every task is on the critical path and gets an SM alone.
long long batch_total(const ReplayLaunch& L) {
    long long b = 0;
    for (int j = 0; j < L.njobs; ++j) b += L.job[j].batch;
    return b;
}
long long default_ctas(int sms, long long batch) { return batch >= 16 ? 2LL * sms : (long long)sms; }
// Grid of a persistent kernel: the plan's replay_ctas option when set (1 = serial replay
// in queue order, the race check's reference schedule), else `dflt`; never more CTAs
// than slots.
int grid_of(const stc_plan* P, long long dflt, long long slots) {
    const long long g = P->opt.replay_ctas > 0 ? (long long)P->opt.replay_ctas : dflt;
    return (int)std::max<long long>(1, std::min<long long>(g, slots));
}

void fill_job(ReplayArgs& a, const stc_plan* P, const TaskSet* ts, void* d_factor, int* counters, int32_t* d_info,
              int64_t batch, WorkHeader* hdr) {
    a.tiles = ts->d_tiles; a.saind = P->dev.saind; a.cext = P->dev.cext; a.tasks = ts->d_tasks; a.upds = ts->d_upds;
    a.imap = ts->d_imap; a.factor = (double*)d_factor; a.fstride = P->factor_doubles;
    a.poff = P->partial_off; a.hdr = hdr; a.counters = counters;
    a.ntiles = (int)P->tiles.size(); a.info = d_info; a.ntasks = (int)ts->tasks.size();
    a.batch = batch; a.nb = (int)P->nb; a.slice_h = ts->slice_h;
    a.spin = P->opt.spin_limit > 0 ? P->opt.spin_limit : kDefaultSpin;
}

bool is_sn(const stc_plan* P) { return P->route_exec == STC_ROUTE_SUPERNODAL; }
// completion counters per item: one per tile, or one per supernodal cell
size_t counters_per_item(const stc_plan* P) { return is_sn(P) ? P->supernodal().dcells.size() : P->tiles.size(); }
size_t factorize_ws(const stc_plan* P, int64_t batch) {
    return sizeof(WorkHeader) + (size_t)batch * counters_per_item(P) * sizeof(int);
}
// solve: a done flag per (chain, forward/backward step) and a y vector per chain
size_t solve_flags(const stc_plan* P, int64_t chains) {
    const size_t steps = is_sn(P) ? (size_t)P->supernodal().nsn() : (size_t)P->nt;
    return ((size_t)chains * 2 * steps * sizeof(int) + 255) / 256 * 256;
}
size_t solve_ws(const stc_plan* P, int64_t chains) {
    const size_t ylen = is_sn(P) ? (size_t)P->n : (size_t)(P->nt * P->nb);
    return sizeof(WorkHeader) + solve_flags(P, chains) + (size_t)chains * ylen * sizeof(double);
}

int32_t pick_slices_impl(stc_plan* P, int64_t batch, int sms) {
    if (P->opt.row_slices > 0) return P->opt.row_slices;
    // Split heavy tiles so the chain POTRF -> TRSM -> SYRK of consecutive block columns
    // is spread over several SMs (the per-SM FP64 rate is low), but no further than the
    // batch needs: thinner slices cost efficiency inside each task.
    if (P->nb < 48) return 1;
    // independent work in flight: the batch times the modelled parallelism of one item's
    // task DAG (work over critical path); thresholds measured on the n = 200,000 band
    // (2 slices at 64 items, 4 at 32, 8 at 16 and fewer), the spatio-temporal and FEM
    // patterns (parallelism in the hundreds: unsliced)
    const double width = (double)batch * P->taskset(2)->par;
    const int s = width >= 0.6 * sms ? 2 : width >= 0.3 * sms ? 4 : 8;
    return P->nb < 96 ? std::max(1, s / 2) : s;
}

// The task set a factorization of `batch` value sets replays (slice count from the batch,
// bottom-level order for one or two value sets).
int pick_taskset(stc_plan* P, int64_t batch, int sms, bool bl_order, TaskSet** out, bool fwd = false) {
    *out = nullptr;
    return no_throw([&] {
        *out = P->taskset(pick_slices_impl(P, batch, sms), bl_order, fwd);
        return STC_OK;
    });
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Arguments of a supernodal job (the plan's device copies must be resident).
void fill_sn(SnArgs& a, const stc_plan* P, void* d_factor, int* counters, int32_t* d_info, int64_t batch,
             WorkHeader* hdr) {
    const SnPlan& Sp = P->supernodal();
    a.cells = P->sndev.cells; a.tasks = P->sndev.tasks; a.upds = P->sndev.upds; a.maps = P->sndev.maps;
    a.first = P->sndev.first; a.factor = (double*)d_factor; a.fstride = Sp.item_doubles(); a.poff = Sp.poff();
    a.hdr = hdr; a.counters = counters; a.ncells = (int)Sp.dcells.size(); a.info = d_info;
    a.ntasks = (int)Sp.dtasks.size(); a.batch = batch;
    a.spin = P->opt.spin_limit > 0 ? P->opt.spin_limit : kDefaultSpin;
}

// Supernodal factorization: the persistent kernel over (task, item) slots, every item of
// a task in lockstep (the left-looking task order is topological).
int sn_factorize_scattered(stc_plan* P, int64_t batch, void* d_factor, void* d_work, int32_t* d_info, void* stream,
                           int dev, int sms) {
    int rc;
    if ((rc = ensure_sn(P, dev))) return rc;
    cudaStream_t st = S(stream);
    if (cudaMemsetAsync(d_work, 0, factorize_ws(P, batch), st) != cudaSuccess) return STC_ERR_CUDA;
    if (cudaMemsetAsync(d_info, 0, (size_t)batch * sizeof(int32_t), st) != cudaSuccess) return STC_ERR_CUDA;
    SnArgs a{};
    fill_sn(a, P, d_factor, (int*)((char*)d_work + sizeof(WorkHeader)), d_info, batch, (WorkHeader*)d_work);
    const long long total = (long long)a.ntasks * batch;
    const int grid = grid_of(P, default_ctas(sms, batch), total);
    sn_replay_kernel<<<grid, kThreads, kRSmemBytes, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

int sn_solve(stc_plan* P, const void* d_factor, int64_t batch, int64_t nrhs, const double* d_b, double* d_x,
             void* d_work, void* stream, int dev, int sms) {
    int rc;
    if ((rc = ensure_sn(P, dev))) return rc;
    const SnPlan& Sp = P->supernodal();
    const long long chains = batch * nrhs;
    cudaStream_t st = S(stream);
    const size_t flags = solve_flags(P, chains);
    if (cudaMemsetAsync(d_work, 0, sizeof(WorkHeader) + flags, st) != cudaSuccess) return STC_ERR_CUDA;
    SnSolveArgs a{};
    a.cells = P->sndev.cells; a.maps = P->sndev.maps; a.cell_cmap = P->sndev.cell_cmap; a.first = P->sndev.first;
    a.cptr = P->sndev.cptr; a.rptr_cells = P->sndev.rptr_cells; a.row_cells = P->sndev.row_cells;
    a.perm = P->dev.perm; a.factor = (const double*)d_factor; a.fstride = Sp.item_doubles();
    a.b = d_b; a.x = d_x; a.hdr = (WorkHeader*)d_work;
    a.done = (int*)((char*)d_work + sizeof(WorkHeader));
    a.y = (double*)((char*)d_work + sizeof(WorkHeader) + flags);
    a.chains = chains; a.nrhs = nrhs; a.nsn = Sp.nsn(); a.n = P->n;
    a.spin = P->opt.spin_limit > 0 ? P->opt.spin_limit : kDefaultSpin;
    const long long total = 2LL * a.nsn * chains;
    const int grid = grid_of(P, sms, total);
    sn_solve_kernel<<<grid, kThreads, kSolveSmem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

// Supernodal selected inverse: the persistent kernel over (task, item) slots.
int sn_selinv(stc_plan* P, const void* d_factor, int64_t batch, void* d_sigma, void* d_work, void* stream, int dev,
              int sms) {
    int rc;
    if ((rc = ensure_sn(P, dev))) return rc;
    const SnPlan& Sp = P->supernodal();
    cudaStream_t st = S(stream);
    if (cudaMemsetAsync(d_sigma, 0, stc_factor_bytes(P, batch), st) != cudaSuccess) return STC_ERR_CUDA;
    if (cudaMemsetAsync(d_work, 0, factorize_ws(P, batch), st) != cudaSuccess) return STC_ERR_CUDA;
    SnSelinvArgs a{};
    a.cells = P->sndev.cells; a.tasks = P->sndev.stasks; a.cons = P->sndev.scons; a.rows = P->sndev.rows;
    a.rowoff = P->sndev.cell_rowoff; a.first = P->sndev.first; a.factor = (const double*)d_factor;
    a.sigma = (double*)d_sigma; a.fstride = Sp.item_doubles(); a.hdr = (WorkHeader*)d_work;
    a.counters = (int*)((char*)d_work + sizeof(WorkHeader)); a.ncells = (int)Sp.dcells.size();
    a.ntasks = (int)Sp.stasks.size(); a.batch = batch;
    a.spin = P->opt.spin_limit > 0 ? P->opt.spin_limit : kDefaultSpin;
    const long long total = (long long)a.ntasks * batch;
    const int grid = grid_of(P, sms, total);
    sn_selinv_kernel<<<grid, kThreads, kSmemBytes, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

}  // namespace
}  // namespace stc

// ---------------------------------------------------------------------------
// Allocation-free factorization: the replay kernel's scratch (WorkHeader + per-tile
// counters) comes from this fixed array instead of a caller workspace.  Host code
// must not pass `g_noalloc_scratch` itself to a kernel (on the host that name is only
// a stand-in for the device object); the device address is looked up once per device.
// ---------------------------------------------------------------------------
namespace stc {
namespace {
static __device__ __align__(256) unsigned char g_noalloc_scratch[STC_NOALLOC_SCRATCH_BYTES];

struct NoallocSlot {
    void* ptr = nullptr;
    bool ready = false;
};
NoallocSlot g_noalloc[64];
std::mutex g_noalloc_mu;

int noalloc_scratch(int dev, void** out) {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    NoallocSlot& s = g_noalloc[dev];
    if (!s.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return STC_ERR_CUDA;
        s.ptr = p;
        s.ready = true;
    }
    *out = s.ptr;
    return STC_OK;
}
}  // namespace
}  // namespace stc

using namespace stc;

extern "C" int stc_plan_upload(stc_plan* P) {
    if (!P) return STC_ERR_INVALID_ARG;
    int dev, sms;
    int rc = device_info(&dev, &sms);
    if (rc) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    TaskSet* ts = nullptr;
    if ((rc = get_taskset(P, 1, false, &ts))) return rc;
    if ((rc = ensure_taskset(P, ts, dev))) return rc;
    if (is_sn(P) && (rc = ensure_sn(P, dev))) return rc;
    // resolve the allocation-free entry point's scratch array now, so that the module
    // holding it is loaded on this device before the caller reserves the rest of its memory
    void* scratch = nullptr;
    return noalloc_scratch(dev, &scratch);
}

extern "C" void stc_plan_destroy(stc_plan* P) {
    if (!P) return;
    if (P->dev.device >= 0 || !P->tasksets.empty()) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (P->dev.device >= 0 && P->dev.device != cur) cudaSetDevice(P->dev.device);
        free_dev(P);
        if (cur >= 0) cudaSetDevice(cur);
    }
    delete P;
}

extern "C" size_t stc_factor_bytes(const stc_plan* P, int64_t batch) {
    if (!P || batch < 0) return 0;
    return (size_t)batch * (size_t)P->item_doubles() * sizeof(double);
}

extern "C" size_t stc_workspace_bytes(const stc_plan* P, int64_t batch) {
    if (!P || batch < 0) return 0;
    return std::max(factorize_ws(P, batch), solve_ws(P, batch));
}

extern "C" int stc_scatter_values(const stc_plan* Pc, const double* d_values, int64_t batch, void* d_factor,
                                  void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_values || !d_factor || batch <= 0) return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    if (is_sn(P) && (rc = ensure_sn(P, dev))) return rc;
    cudaStream_t st = S(stream);
    const long long fd = P->item_doubles();
    const int blocks = (int)std::max<long long>(1, std::min<long long>((long long)sms * 16, (fd + 255) / 256));
    fill_kernel<<<blocks, 256, 0, st>>>(d_values, P->nnzA, batch, is_sn(P) ? P->sndev.fill_src : P->dev.fill_src,
                                        (double*)d_factor, fd);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

extern "C" int stc_factorize_scattered(const stc_plan* Pc, int64_t batch, void* d_factor, void* d_work,
                                       int32_t* d_info, void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_factor || !d_info || batch <= 0) return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    if (!d_work && (rc = own_buffer(P, false, stc_workspace_bytes(P, batch), &d_work))) return rc;
    if (is_sn(P)) return sn_factorize_scattered(P, batch, d_factor, d_work, d_info, stream, dev, sms);
    // one or two value sets: the item's own DAG width decides, so the critical path goes first
    TaskSet* ts = nullptr;
    if ((rc = pick_taskset(P, batch, sms, batch <= 2, &ts))) return rc;
    if ((rc = ensure_taskset(P, ts, dev))) return rc;
    cudaStream_t st = S(stream);
    if (cudaMemsetAsync(d_work, 0, factorize_ws(P, batch), st) != cudaSuccess) return STC_ERR_CUDA;
    if (cudaMemsetAsync(d_info, 0, (size_t)batch * sizeof(int32_t), st) != cudaSuccess) return STC_ERR_CUDA;
    ReplayLaunch Lc{};
    fill_job(Lc.job[0], P, ts, d_factor, (int*)((char*)d_work + sizeof(WorkHeader)), d_info, batch,
             (WorkHeader*)d_work);
    Lc.njobs = 1;
    Lc.queue = nullptr;
    Lc.hdr = (WorkHeader*)d_work;
    Lc.total = (long long)ts->tasks.size() * batch;
    const int grid = grid_of(P, default_ctas(sms, batch_total(Lc)), Lc.total);
    replay_kernel_t<false><<<grid, kThreads, kRSmemBytes, st>>>(Lc);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

extern "C" int stc_factorize(const stc_plan* P, const double* d_values, int64_t batch, void* d_factor,
                             void* d_work, int32_t* d_info, void* stream) {
    if (!P || !d_values || !d_factor || !d_info || batch <= 0) return STC_ERR_INVALID_ARG;
    int rc = stc_scatter_values(P, d_values, batch, d_factor, stream);
    if (rc) return rc;
    return stc_factorize_scattered(P, batch, d_factor, d_work, d_info, stream);
}

extern "C" int stc_sync_status(const void* d_work, void* stream) {
    if (!d_work) return STC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return STC_ERR_CUDA;
    WorkHeader h;
    if (cudaMemcpy(&h, d_work, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return STC_ERR_CUDA;
    return h.status;
}

extern "C" int stc_plan_sync_status(const stc_plan* Pc, void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P) return STC_ERR_INVALID_ARG;
    void* w;
    {
        std::lock_guard<std::mutex> g(P->own_mu);
        w = P->own_ws;
    }
    if (!w) return STC_ERR_INVALID_ARG;  // no call has used the plan's own workspace yet
    return stc_sync_status(w, stream);
}

extern "C" int stc_logdet(const stc_plan* P, const void* d_factor, int64_t batch, double* d_logdet,
                          void* stream) {
    if (!P || !d_factor || !d_logdet || batch <= 0) return STC_ERR_INVALID_ARG;
    const int wpb = 8;
    const long long blocks = (batch + wpb - 1) / wpb;
    int64_t stride, poff, np;
    if (no_throw([&] {
            stride = P->item_doubles();
            poff = P->logdet_off();
            np = P->nlogdet();
            return STC_OK;
        }))
        return STC_ERR_OUT_OF_MEMORY;
    logdet_kernel<<<(unsigned)blocks, 32 * wpb, 0, S(stream)>>>((const double*)d_factor, stride, poff, (int)np, batch,
                                                                d_logdet);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

extern "C" int stc_factor_to_csc(const stc_plan* Pc, const void* d_factor, int64_t batch, double* d_Lx,
                                 void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_factor || !d_Lx || batch <= 0) return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    if (is_sn(P) && (rc = ensure_sn(P, dev))) return rc;
    const long long nnzl = P->Lp[P->n];
    const int blocks = std::max(1, std::min<int>(sms * 8, (int)((nnzl + 255) / 256)));
    to_csc_kernel<<<blocks, 256, 0, S(stream)>>>((const double*)d_factor, P->item_doubles(), batch,
                                                 is_sn(P) ? P->sndev.csc_map : P->dev.csc_map, nnzl, d_Lx);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

extern "C" int stc_solve(const stc_plan* Pc, const void* d_factor, int64_t batch, int64_t nrhs, const double* d_b,
                         double* d_x, void* d_work, void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_factor || !d_b || !d_x || batch <= 0 || nrhs <= 0 || d_b == d_x)
        return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    if (!d_work && (rc = own_buffer(P, false, stc_workspace_bytes(P, batch * nrhs), &d_work))) return rc;
    if (is_sn(P)) return sn_solve(P, d_factor, batch, nrhs, d_b, d_x, d_work, stream, dev, sms);
    TaskSet* ts = nullptr;
    if ((rc = get_taskset(P, 1, false, &ts))) return rc;
    if ((rc = ensure_taskset(P, ts, dev))) return rc;
    const long long chains = batch * nrhs;
    cudaStream_t st = S(stream);
    const size_t flags = solve_flags(P, chains);
    if (cudaMemsetAsync(d_work, 0, sizeof(WorkHeader) + flags, st) != cudaSuccess) return STC_ERR_CUDA;
    SolveArgs a{};
    a.tiles = ts->d_tiles; a.saind = P->dev.saind; a.rowstart = P->dev.srow_beg; a.rowtiles = P->dev.srow_tiles;
    a.colstart = P->dev.scol_beg; a.diag = P->dev.diag_tile; a.perm = P->dev.perm;
    a.factor = (const double*)d_factor; a.fstride = P->factor_doubles; a.b = d_b; a.x = d_x;
    a.hdr = (WorkHeader*)d_work;
    a.done = (int*)((char*)d_work + sizeof(WorkHeader));
    a.y = (double*)((char*)d_work + sizeof(WorkHeader) + flags);
    a.chains = chains; a.nrhs = nrhs; a.nt = (int)P->nt; a.nb = (int)P->nb; a.n = P->n;
    a.spin = P->opt.spin_limit > 0 ? P->opt.spin_limit : kDefaultSpin;
    const long long total = 2LL * P->nt * chains;
    const int grid = grid_of(P, sms, total);
    solve_kernel<<<grid, kThreads, kSolveSmem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

// Fused factorization + solve: [header | completion counters | fill flags (one per item
// and block column)], then (256-byte aligned) the solve's step flags and y vectors.
size_t fused_solve_off(const stc_plan* P, int64_t batch) {
    return (factorize_ws(P, batch) + (size_t)batch * P->nt * sizeof(int) + 255) / 256 * 256;
}

extern "C" size_t stc_factorize_solve_workspace_bytes(const stc_plan* P, int64_t batch, int64_t nrhs) {
    if (!P || batch < 0 || nrhs < 0) return 0;
    if (is_sn(P)) return std::max(factorize_ws(P, batch), solve_ws(P, batch * nrhs));
    return fused_solve_off(P, batch) + solve_ws(P, batch * nrhs) - sizeof(WorkHeader);
}

extern "C" int stc_factorize_forward(const stc_plan* Pc, const double* d_values, int64_t batch, int64_t nrhs,
                                     const double* d_b, void* d_factor, void* d_work, int32_t* d_info,
                                     void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_values || !d_factor || !d_info || !d_b || !d_work || batch <= 0 || nrhs <= 0)
        return STC_ERR_INVALID_ARG;
    if (is_sn(P)) return STC_ERR_UNSUPPORTED;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    TaskSet* ts = nullptr;
    if ((rc = pick_taskset(P, batch, sms, batch <= 2, &ts, true))) return rc;
    if ((rc = ensure_taskset(P, ts, dev))) return rc;
    // the value scatter: inside the launch (hosted by waiting tasks) or, for task sets
    // with too few hosts, the scatter kernel first
    if (!ts->fill_inside && (rc = stc_scatter_values(P, d_values, batch, d_factor, stream))) return rc;
    const long long chains = batch * nrhs;
    cudaStream_t st = S(stream);
    const size_t off = fused_solve_off(P, batch), flags = solve_flags(P, chains);
    if (cudaMemsetAsync(d_work, 0, off + flags, st) != cudaSuccess) return STC_ERR_CUDA;
    if (cudaMemsetAsync(d_info, 0, (size_t)batch * sizeof(int32_t), st) != cudaSuccess) return STC_ERR_CUDA;
    WorkHeader* hdr = (WorkHeader*)d_work;
    ReplayLaunch Lc{};
    fill_job(Lc.job[0], P, ts, d_factor, (int*)((char*)d_work + sizeof(WorkHeader)), d_info, batch, hdr);
    ReplayArgs& j = Lc.job[0];
    j.rhs = d_b;
    j.sdone = (int*)((char*)d_work + off);
    j.y = (double*)((char*)d_work + off + flags);
    j.perm = P->dev.perm; j.rowstart = P->dev.srow_beg; j.rowtiles = P->dev.srow_tiles;
    j.n = P->n; j.nrhs = (int)nrhs; j.nt = (int)P->nt;
    if (ts->fill_inside) {
        j.vals = d_values; j.nnz = P->nnzA; j.fill_src = P->dev.fill_src;
        j.fillflag = (int*)((char*)d_work + factorize_ws(P, batch));
        j.colstart = P->dev.scol_beg;
    }
    Lc.njobs = 1;
    Lc.queue = nullptr;
    Lc.hdr = hdr;
    Lc.total = (long long)ts->tasks.size() * batch;
    replay_kernel_t<false><<<grid_of(P, default_ctas(sms, batch_total(Lc)), Lc.total), kThreads, kRSmemBytes, st>>>(Lc);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

extern "C" int stc_factorize_forward_fills(const stc_plan* Pc, int64_t batch) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || batch <= 0) return STC_ERR_INVALID_ARG;
    if (is_sn(P)) return 0;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    TaskSet* ts = nullptr;
    if ((rc = pick_taskset(P, batch, sms, batch <= 2, &ts, true))) return rc;
    return ts->fill_inside ? 1 : 0;
}

extern "C" int stc_solve_backward(const stc_plan* Pc, const void* d_factor, int64_t batch, int64_t nrhs,
                                  double* d_x, void* d_work, void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_factor || !d_x || !d_work || batch <= 0 || nrhs <= 0) return STC_ERR_INVALID_ARG;
    if (is_sn(P)) return STC_ERR_UNSUPPORTED;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    TaskSet* ts = nullptr;
    if ((rc = pick_taskset(P, batch, sms, batch <= 2, &ts, true))) return rc;
    if ((rc = ensure_taskset(P, ts, dev))) return rc;
    const long long chains = batch * nrhs;
    cudaStream_t st = S(stream);
    const size_t off = fused_solve_off(P, batch), flags = solve_flags(P, chains);
    WorkHeader* hdr = (WorkHeader*)d_work;
    // the solve kernel's backward steps; its slot counter restarted, the status word keeps
    // the factorization's outcome
    if (cudaMemsetAsync(&hdr->head, 0, sizeof(hdr->head), st) != cudaSuccess) return STC_ERR_CUDA;
    SolveArgs a{};
    a.tiles = ts->d_tiles; a.saind = P->dev.saind; a.rowstart = P->dev.srow_beg; a.rowtiles = P->dev.srow_tiles;
    a.colstart = P->dev.scol_beg; a.diag = P->dev.diag_tile; a.perm = P->dev.perm;
    a.factor = (const double*)d_factor; a.fstride = P->factor_doubles; a.b = nullptr; a.x = d_x;
    a.hdr = hdr;
    a.done = (int*)((char*)d_work + off);
    a.y = (double*)((char*)d_work + off + flags);
    a.chains = chains; a.nrhs = nrhs; a.nt = (int)P->nt; a.nb = (int)P->nb; a.n = P->n;
    a.spin = P->opt.spin_limit > 0 ? P->opt.spin_limit : kDefaultSpin;
    a.ti0 = (int)P->nt;
    const long long total = P->nt * chains;
    solve_kernel<<<grid_of(P, sms, total), kThreads, kSolveSmem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

extern "C" int stc_factorize_solve(const stc_plan* Pc, const double* d_values, int64_t batch, int64_t nrhs,
                                   const double* d_b, void* d_factor, double* d_x, void* d_work, int32_t* d_info,
                                   void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_values || !d_factor || !d_info || !d_b || !d_x || batch <= 0 || nrhs <= 0 || d_b == d_x)
        return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    if (!d_work && (rc = own_buffer(P, false, stc_factorize_solve_workspace_bytes(P, batch, nrhs), &d_work)))
        return rc;
    if (is_sn(P)) {
        // supernodal route: the factorization, then the solve, on the same stream
        if ((rc = stc_factorize(P, d_values, batch, d_factor, d_work, d_info, stream))) return rc;
        return stc_solve(P, d_factor, batch, nrhs, d_b, d_x, d_work, stream);
    }
    if ((rc = stc_factorize_forward(P, d_values, batch, nrhs, d_b, d_factor, d_work, d_info, stream))) return rc;
    return stc_solve_backward(P, d_factor, batch, nrhs, d_x, d_work, stream);
}

extern "C" int stc_fp64_peak_probe(double* d_scratch, int64_t scratch_doubles, int64_t iters, double* gflops) {
    if (!d_scratch || !gflops || scratch_doubles < 256 || iters <= 0) return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    const long long blocks = std::min<long long>((long long)sms * 4, scratch_doubles / 256);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return STC_ERR_CUDA;
    fp64_probe_kernel<<<(unsigned)blocks, 256>>>(d_scratch, iters, 1.0000001, 1e-9);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0);
        fp64_probe_kernel<<<(unsigned)blocks, 256>>>(d_scratch, iters, 1.0000001, 1e-9);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = STC_ERR_CUDA; break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (cudaGetLastError() != cudaSuccess) return STC_ERR_CUDA;
    *gflops = 2.0 * 8.0 * (double)iters * (double)blocks * 256.0 / (best * 1e-3) / 1e9;
    return STC_OK;
}

extern "C" int stc_selinv(const stc_plan* Pc, const void* d_factor, int64_t batch, void* d_sigma, void* d_work,
                          void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_factor || !d_sigma || batch <= 0 || d_factor == d_sigma) return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    if (!d_work && (rc = own_buffer(P, false, stc_workspace_bytes(P, batch), &d_work))) return rc;
    if (is_sn(P)) return sn_selinv(P, d_factor, batch, d_sigma, d_work, stream, dev, sms);
    TaskSet* ts = nullptr;
    if ((rc = get_taskset(P, 1, false, &ts))) return rc;
    if ((rc = ensure_taskset(P, ts, dev))) return rc;
    cudaStream_t st = S(stream);
    if (cudaMemsetAsync(d_sigma, 0, stc_factor_bytes(P, batch), st) != cudaSuccess) return STC_ERR_CUDA;
    if (cudaMemsetAsync(d_work, 0, factorize_ws(P, batch), st) != cudaSuccess) return STC_ERR_CUDA;
    SelinvArgs a{};
    a.tiles = ts->d_tiles; a.saind = P->dev.saind; a.sinv = P->dev.sinv; a.tasks = P->dev.stasks;
    a.cons = P->dev.scons; a.factor = (const double*)d_factor; a.sigma = (double*)d_sigma;
    a.fstride = P->factor_doubles; a.hdr = (WorkHeader*)d_work;
    a.counters = (int*)((char*)d_work + sizeof(WorkHeader)); a.ntiles = (int)P->tiles.size();
    a.ntasks = (int)P->stasks.size(); a.batch = batch; a.nb = (int)P->nb;
    a.spin = P->opt.spin_limit > 0 ? P->opt.spin_limit : kDefaultSpin;
    const long long total = (long long)a.ntasks * batch;
    const int grid = grid_of(P, sms, total);
    selinv_kernel<<<grid, kThreads, kSmemBytes, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

extern "C" int stc_logdet_backward(const stc_plan* Pc, const void* d_factor, int64_t batch, const double* d_gout,
                                   double* d_gvalues, int accumulate, void* d_sigma, void* d_work, void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_gvalues || batch <= 0) return STC_ERR_INVALID_ARG;
    int rc;
    if (!d_sigma) {
        int dev, sms;
        if ((rc = device_info(&dev, &sms))) return rc;
        if ((rc = ensure_plan(P, dev))) return rc;
        if ((rc = own_buffer(P, true, stc_factor_bytes(P, batch), &d_sigma))) return rc;
    }
    if ((rc = stc_selinv(P, d_factor, batch, d_sigma, d_work, stream))) return rc;
    int sms = g_dev[P->dev.device].sms;
    const int blocks = std::max(1, std::min<int>(sms * 8, (int)((P->nnzA + 255) / 256)));
    grad_gather_kernel<<<blocks, 256, 0, S(stream)>>>((const double*)d_sigma, P->item_doubles(), batch,
                                                       is_sn(P) ? P->sndev.value_map : P->dev.value_map, P->dev.vdiag,
                                                       P->nnzA, d_gout, d_gvalues, accumulate);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

extern "C" int stc_sym_outer_backward(const stc_plan* Pc, int64_t batch, const double* d_u, const double* d_v,
                                      const double* d_scale, double* d_gvalues, int accumulate, void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_u || !d_v || !d_gvalues || batch <= 0) return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    const int blocks = std::max(1, std::min<int>(sms * 8, (int)((P->nnzA + 255) / 256)));
    outer_grad_kernel<<<blocks, 256, 0, S(stream)>>>(P->dev.arow, P->dev.acol, P->dev.vdiag, P->nnzA, batch, d_u, d_v,
                                                      P->n, d_scale, d_gvalues, accumulate);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

extern "C" int stc_quad_form(const stc_plan* Pc, int64_t batch, const double* d_values, const double* d_x,
                             double* d_out, void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_values || !d_x || !d_out || batch <= 0) return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if ((rc = ensure_plan(P, dev))) return rc;
    quad_form_kernel<<<(unsigned)batch, kThreads, 0, S(stream)>>>(P->dev.arow, P->dev.acol, P->dev.vdiag, P->nnzA,
                                                                  d_values, d_x, P->n, d_out);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Mixed batches of several plans in one launch.
// ---------------------------------------------------------------------------
struct stc_group {
    std::vector<stc_plan*> plans;
    std::vector<int64_t> batch;
    std::vector<TaskSet*> ts;
    std::vector<size_t> cnt_off;  // byte offset of each job's counters in the workspace
    size_t ws_bytes = 0;
    uint64_t* d_queue = nullptr;
    long long total = 0;
    int device = -1;
    bool has_sn = false;      // a supernodal plan among the jobs (the mixed-route kernel runs)
};

extern "C" int stc_group_create(int32_t nplans, const stc_plan* const* plans, const int64_t* batch,
                                stc_group** out) {
    if (!out) return STC_ERR_INVALID_ARG;
    *out = nullptr;
    if (nplans < 1 || nplans > kMaxJobs || !plans || !batch) return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    auto g = std::make_unique<stc_group>();
    g->device = dev;
    int64_t btot = 0;
    for (int p = 0; p < nplans; ++p) {
        if (!plans[p] || batch[p] <= 0 || batch[p] >= (1LL << 28)) return STC_ERR_INVALID_ARG;
        btot += batch[p];
    }
    size_t off = sizeof(WorkHeader);
    for (int p = 0; p < nplans; ++p) {
        stc_plan* P = const_cast<stc_plan*>(plans[p]);
        if ((rc = ensure_plan(P, dev))) return rc;
        TaskSet* ts = nullptr;
        if (is_sn(P)) {
            if ((rc = ensure_sn(P, dev))) return rc;
            g->has_sn = true;
        } else {
            if ((rc = pick_taskset(P, btot, sms, false, &ts))) return rc;
            if ((rc = ensure_taskset(P, ts, dev))) return rc;
        }
        g->plans.push_back(P);
        g->batch.push_back(batch[p]);
        g->ts.push_back(ts);
        g->cnt_off.push_back(off);
        off += ((size_t)batch[p] * counters_per_item(P) * sizeof(int) + 255) / 256 * 256;
    }
    g->ws_bytes = off;
    // queue keys: the tile plans' modelled earliest starts; a supernodal plan's tasks (in
    // their left-looking order) spread evenly over the longest tile plan's span
    double span = 0.0;
    for (int p = 0; p < nplans; ++p)
        if (g->ts[p] && !g->ts[p]->qkey.empty()) span = std::max(span, g->ts[p]->qkey.back());
    if (!(span > 0.0)) span = 1.0;
    auto ntasks = [&](int p) { return g->ts[p] ? g->ts[p]->tasks.size() : g->plans[p]->supernodal().dtasks.size(); };
    auto key = [&](int p, size_t t) {
        return g->ts[p] ? g->ts[p]->qkey[t] : span * double(t + 1) / double(ntasks(p));
    };
    // merged queue: plans' task lists in earliest-start order, each task expanded to its
    // plan's batch items in lockstep
    std::vector<uint64_t> q;
    size_t nslots = 0;
    for (int p = 0; p < nplans; ++p) nslots += ntasks(p) * (size_t)batch[p];
    q.reserve(nslots);
    typedef std::pair<double, int> E;
    std::priority_queue<E, std::vector<E>, std::greater<E>> h;
    std::vector<size_t> pos(nplans, 0);
    for (int p = 0; p < nplans; ++p)
        if (ntasks(p) > 0) h.push(E(key(p, 0), p));
    while (!h.empty()) {
        const int p = h.top().second;
        h.pop();
        const size_t t = pos[p];
        for (int64_t b = 0; b < batch[p]; ++b) q.push_back(qpack(p, (int)t, b));
        if (++pos[p] < ntasks(p)) h.push(E(key(p, pos[p]), p));
    }
    g->total = (long long)q.size();
    if (cudaMalloc((void**)&g->d_queue, std::max<size_t>(1, q.size()) * sizeof(uint64_t)) != cudaSuccess)
        return STC_ERR_OUT_OF_MEMORY;
    if (!q.empty() && cudaMemcpy(g->d_queue, q.data(), q.size() * sizeof(uint64_t), cudaMemcpyHostToDevice) !=
                          cudaSuccess) {
        cudaFree(g->d_queue);
        return STC_ERR_CUDA;
    }
    *out = g.release();
    return STC_OK;
}

extern "C" size_t stc_group_workspace_bytes(const stc_group* g) { return g ? g->ws_bytes : 0; }

extern "C" int stc_factorize_group(stc_group* g, const double* const* d_values, void* const* d_factor,
                                   int32_t* const* d_info, void* d_work, void* stream) {
    if (!g || !d_values || !d_factor || !d_info || !d_work) return STC_ERR_INVALID_ARG;
    const int np = (int)g->plans.size();
    for (int p = 0; p < np; ++p)
        if (!d_values[p] || !d_factor[p] || !d_info[p]) return STC_ERR_INVALID_ARG;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    if (dev != g->device) return STC_ERR_INVALID_ARG;
    cudaStream_t st = S(stream);
    for (int p = 0; p < np; ++p)
        if ((rc = stc_scatter_values(g->plans[p], d_values[p], g->batch[p], d_factor[p], stream))) return rc;
    if (cudaMemsetAsync(d_work, 0, g->ws_bytes, st) != cudaSuccess) return STC_ERR_CUDA;
    ReplayLaunch Lc{};
    for (int p = 0; p < np; ++p) {
        if (cudaMemsetAsync(d_info[p], 0, (size_t)g->batch[p] * sizeof(int32_t), st) != cudaSuccess)
            return STC_ERR_CUDA;
        int* counters = (int*)((char*)d_work + g->cnt_off[p]);
        if (g->ts[p]) {
            fill_job(Lc.job[p], g->plans[p], g->ts[p], d_factor[p], counters, d_info[p], g->batch[p],
                     (WorkHeader*)d_work);
        } else {
            fill_sn(Lc.snj[p], g->plans[p], d_factor[p], counters, d_info[p], g->batch[p], (WorkHeader*)d_work);
            Lc.job[p].sn = 1;
            Lc.job[p].batch = g->batch[p];
        }
    }
    Lc.njobs = np;
    Lc.queue = g->d_queue;
    Lc.hdr = (WorkHeader*)d_work;
    Lc.total = g->total;
    const int grid = grid_of(g->plans[0], default_ctas(sms, batch_total(Lc)), Lc.total);
    if (g->has_sn)
        replay_kernel_t<true><<<grid, kThreads, kRSmemBytes, st>>>(Lc);
    else
        replay_kernel_t<false><<<grid, kThreads, kRSmemBytes, st>>>(Lc);
    return cudaGetLastError() == cudaSuccess ? STC_OK : STC_ERR_CUDA;
}

extern "C" void stc_group_destroy(stc_group* g) {
    if (!g) return;
    if (g->d_queue) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (g->device >= 0 && g->device != cur) cudaSetDevice(g->device);
        cudaFree(g->d_queue);
        if (cur >= 0) cudaSetDevice(cur);
    }
    delete g;
}

extern "C" int stc_factorize_noalloc(const stc_plan* Pc, const double* d_values, int64_t batch, void* d_factor,
                                     int32_t* d_info, int32_t* d_status, void* stream) {
    stc_plan* P = const_cast<stc_plan*>(Pc);
    if (!P || !d_values || !d_factor || !d_info || batch <= 0) return STC_ERR_INVALID_ARG;
    if (is_sn(P)) return STC_ERR_UNSUPPORTED;  // tile routes only
    const size_t need = factorize_ws(P, batch);
    if (need > (size_t)STC_NOALLOC_SCRATCH_BYTES) return STC_ERR_UNSUPPORTED;
    int dev, sms, rc;
    if ((rc = device_info(&dev, &sms))) return rc;
    // the plan and its one-slice task set must already be resident (uploading allocates)
    TaskSet* ts = nullptr;
    {
        std::lock_guard<std::mutex> g(P->mu);
        auto it = P->tasksets.find(stc_plan::taskset_key(1, false));
        if (it != P->tasksets.end()) ts = it->second.get();
        if (P->dev.device != dev || !ts || ts->device != dev) return STC_ERR_INVALID_ARG;
    }
    void* scratch = nullptr;
    if ((rc = noalloc_scratch(dev, &scratch))) return rc;
    cudaStream_t st = S(stream);
    if ((rc = stc_scatter_values(P, d_values, batch, d_factor, stream))) return rc;
    if (cudaMemsetAsync(scratch, 0, need, st) != cudaSuccess) return STC_ERR_CUDA;
    if (cudaMemsetAsync(d_info, 0, (size_t)batch * sizeof(int32_t), st) != cudaSuccess) return STC_ERR_CUDA;
    ReplayLaunch Lc{};
    fill_job(Lc.job[0], P, ts, d_factor, (int*)((char*)scratch + sizeof(WorkHeader)), d_info, batch,
             (WorkHeader*)scratch);
    Lc.njobs = 1;
    Lc.queue = nullptr;
    Lc.hdr = (WorkHeader*)scratch;
    Lc.total = (long long)ts->tasks.size() * batch;
    const int grid = grid_of(P, default_ctas(sms, batch_total(Lc)), Lc.total);
    replay_kernel_t<false><<<grid, kThreads, kRSmemBytes, st>>>(Lc);
    if (cudaGetLastError() != cudaSuccess) return STC_ERR_CUDA;
    if (d_status && cudaMemcpyAsync(d_status, &Lc.hdr->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
                        cudaSuccess)
        return STC_ERR_CUDA;
    return STC_OK;
}
