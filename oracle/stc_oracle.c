/*
 * stc_oracle.c -- plain, slow, FP64 CPU oracle for the structure-adaptive tile
 * Cholesky (arxiv 2609.29765, "sTiles").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg may use it.  It shares no code, header, table or helper with the
 * CUDA path (paper_2609_29765_gb300/csrc).
 *
 * Every routine is the textbook definition written out, in the order the paper
 * (or the textbook it cites) states it, with no blocking, fusion or reordering:
 *
 *   orc_nd_lattice     geometric nested dissection on lattice coordinates
 *                      (Sec. 3 runs ND among its candidate orderings; the exact
 *                      bisection rule is this project's reading, see header of
 *                      the function).
 *   orc_permute_lower  A_p = P A P^T on the lower-triangular CSC pattern.
 *   orc_symbolic       elimination tree (parent[j] = min{i>j : L_ij != 0}) and the
 *                      column structure of L by merging children's structures
 *                      (Sec. 5.4 symbolic phase: etree + column counts).
 *   orc_numeric        left-looking column Cholesky (Sec. 5.2 left-looking sweep,
 *                      at column granularity):  x = A_p[j:,j];
 *                      x -= L[j:,k] L_jk for each k<j with L_jk != 0, ascending;
 *                      L_jj = sqrt(x_0), L[j+1:,j] = x[1:]/L_jj.
 *   orc_logdet         2 * sum_j log L_jj  (log-determinant reused from the factor,
 *                      Sec. 5.4 and Sec. 6.7).
 *   orc_solve          x = P^T L^-T L^-1 P b  (solves consume the factor, Sec. 6.7).
 *   orc_selinv         Takahashi recurrence for Sigma = A_p^{-1} on pattern(L):
 *                      Sigma_ij = delta_ij/L_jj^2 - (1/L_jj) sum_{k in struct(L_:j),k>j}
 *                                 L_kj Sigma_ik,   j = n-1..0.
 *                      (The paper leaves selected inversion to separate work,
 *                      Sec. 6.2; this is the textbook recurrence, Takahashi 1973.)
 *   orc_grad_logdet    d logdet / d a_ij = (2 - delta_ij) Sigma_ij on the lower CSC
 *                      entries of the ORIGINAL matrix.
 *   orc_tile_map       uniform n_b grid over L (Sec. 4): active tiles, active-column
 *                      sets aind (Sec. 4.1), contiguous / full-width predicates and
 *                      the banded half-width kd_t of each diagonal tile (Sec. 5.2,
 *                      per-tile metadata), plus each tile's structural row extent.
 *   orc_task_list      Algorithm 1 (left-looking tile Cholesky task collection).
 *
 * Conventions: all indices are int64; perm[k] = original index of the k-th pivot,
 * so (A_p)_{ij} = A_{perm[i],perm[j]}.  CSC arrays hold the lower triangle with
 * the diagonal, rows sorted ascending within each column.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;

/* ------------------------------------------------------------------------- */
/* small growable int64 vector                                               */
/* ------------------------------------------------------------------------- */
typedef struct { i64* v; i64 n, cap; } vec64;

static int vpush(vec64* a, i64 x) {
    if (a->n == a->cap) {
        i64 nc = a->cap ? 2 * a->cap : 64;
        i64* nv = (i64*)realloc(a->v, (size_t)nc * sizeof(i64));
        if (!nv) return -1;
        a->v = nv; a->cap = nc;
    }
    a->v[a->n++] = x;
    return 0;
}

static int cmp_i64(const void* a, const void* b) {
    i64 x = *(const i64*)a, y = *(const i64*)b;
    return (x > y) - (x < y);
}

/* binary search for row r in sorted Li[lo..hi); returns position or -1 */
static i64 find_row(const i64* Li, i64 lo, i64 hi, i64 r) {
    while (lo < hi) {
        i64 mid = lo + (hi - lo) / 2;
        if (Li[mid] == r) return mid;
        if (Li[mid] < r) lo = mid + 1; else hi = mid;
    }
    return -1;
}

/* ------------------------------------------------------------------------- */
/* Geometric nested dissection on lattice coordinates.                        */
/*                                                                           */
/* Reading of the ordering step (the paper names ND among its candidates but  */
/* fixes no rule): the box [lo,hi] (inclusive, per axis) starts as the        */
/* bounding box of all lattice nodes.  A box holding at most leaf_max nodes is */
/* a leaf.  Otherwise the longest axis (extent hi-lo+1; ties to the lowest    */
/* axis index) is cut at mid = floor((lo+hi)/2): nodes with coordinate < mid  */
/* form the left box [lo,mid-1], > mid the right box [mid+1,hi], == mid the   */
/* separator.  Order: left, right, separator.  Leaf and separator nodes are   */
/* emitted in lexicographic order with x fastest (sort key (z,y,x)).  Rows    */
/* whose coordinates are NaN (dense / border rows set aside before ordering, */
/* Sec. 3) are appended last in input order.                                  */
/* ------------------------------------------------------------------------- */
static const i64* g_xyz; /* comparator context */

static int cmp_lex(const void* a, const void* b) {
    i64 u = *(const i64*)a, v = *(const i64*)b;
    for (int ax = 2; ax >= 0; --ax) {
        i64 cu = g_xyz[3 * u + ax], cv = g_xyz[3 * v + ax];
        if (cu != cv) return (cu > cv) - (cu < cv);
    }
    return 0;
}

static i64 nd_rec(const i64* xyz, i64* nodes, i64 cnt, i64 lo[3], i64 hi[3],
                  i64 leaf_max, i64* out, i64 pos) {
    if (cnt == 0) return pos;
    if (cnt <= leaf_max) {
        g_xyz = xyz;
        qsort(nodes, (size_t)cnt, sizeof(i64), cmp_lex);
        for (i64 t = 0; t < cnt; ++t) out[pos++] = nodes[t];
        return pos;
    }
    int ax = 0;
    for (int a = 1; a < 3; ++a)
        if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
    i64 mid = (lo[ax] + hi[ax]);
    mid = (mid >= 0) ? mid / 2 : -((-mid + 1) / 2);
    i64* left = (i64*)malloc((size_t)cnt * sizeof(i64));
    i64* right = (i64*)malloc((size_t)cnt * sizeof(i64));
    i64* sep = (i64*)malloc((size_t)cnt * sizeof(i64));
    i64 nl = 0, nr = 0, ns = 0;
    for (i64 t = 0; t < cnt; ++t) {
        i64 c = xyz[3 * nodes[t] + ax];
        if (c < mid) left[nl++] = nodes[t];
        else if (c > mid) right[nr++] = nodes[t];
        else sep[ns++] = nodes[t];
    }
    i64 llo[3], lhi[3], rlo[3], rhi[3];
    for (int a = 0; a < 3; ++a) { llo[a] = rlo[a] = lo[a]; lhi[a] = rhi[a] = hi[a]; }
    lhi[ax] = mid - 1;
    rlo[ax] = mid + 1;
    pos = nd_rec(xyz, left, nl, llo, lhi, leaf_max, out, pos);
    pos = nd_rec(xyz, right, nr, rlo, rhi, leaf_max, out, pos);
    g_xyz = xyz;
    qsort(sep, (size_t)ns, sizeof(i64), cmp_lex);
    for (i64 t = 0; t < ns; ++t) out[pos++] = sep[t];
    free(left); free(right); free(sep);
    return pos;
}

/* coords: [n][3] doubles, integral lattice coordinates, NaN = set aside.
 * Returns 0, or -1 on non-integral coordinates / allocation failure. */
int orc_nd_lattice(i64 n, const double* coords, i64 leaf_max, i64* perm) {
    i64* xyz = (i64*)calloc((size_t)(3 * (n > 0 ? n : 1)), sizeof(i64));
    i64* nodes = (i64*)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    char* aside = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!xyz || !nodes || !aside) return -1;
    i64 cnt = 0, lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
    for (i64 i = 0; i < n; ++i) {
        const double* c = coords + 3 * i;
        if (isnan(c[0]) || isnan(c[1]) || isnan(c[2])) { aside[i] = 1; continue; }
        for (int a = 0; a < 3; ++a) {
            double r = floor(c[a]);
            if (r != c[a]) { free(xyz); free(nodes); free(aside); return -1; }
            xyz[3 * i + a] = (i64)r;
            if (cnt == 0 || xyz[3 * i + a] < lo[a]) lo[a] = xyz[3 * i + a];
            if (cnt == 0 || xyz[3 * i + a] > hi[a]) hi[a] = xyz[3 * i + a];
        }
        nodes[cnt++] = i;
    }
    i64 pos = nd_rec(xyz, nodes, cnt, lo, hi, leaf_max, perm, 0);
    for (i64 i = 0; i < n; ++i)
        if (aside[i]) perm[pos++] = i;
    free(xyz); free(nodes); free(aside);
    return pos == n ? 0 : -1;
}

/* ------------------------------------------------------------------------- */
/* A_p = P A P^T on lower CSC.  emap[e] = position in (Bp,Bi) of A's entry e. */
/* ------------------------------------------------------------------------- */
int orc_permute_lower(i64 n, const i64* Ap, const i64* Ai, const i64* perm,
                      i64* Bp, i64* Bi, i64* emap) {
    i64 nnz = Ap[n];
    i64* iperm = (i64*)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    i64* key = (i64*)malloc((size_t)(nnz > 0 ? nnz : 1) * 2 * sizeof(i64));
    if (!iperm || !key) return -1;
    for (i64 k = 0; k < n; ++k) iperm[perm[k]] = k;
    for (i64 j = 0; j <= n; ++j) Bp[j] = 0;
    for (i64 j = 0; j < n; ++j)
        for (i64 p = Ap[j]; p < Ap[j + 1]; ++p) {
            i64 a = iperm[Ai[p]], b = iperm[j];
            i64 r = a > b ? a : b, c = a > b ? b : a;
            key[2 * p] = r; key[2 * p + 1] = c;
            Bp[c + 1]++;
        }
    for (i64 j = 0; j < n; ++j) Bp[j + 1] += Bp[j];
    i64* fill = (i64*)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    for (i64 j = 0; j < n; ++j) fill[j] = Bp[j];
    for (i64 p = 0; p < nnz; ++p) {
        i64 c = key[2 * p + 1];
        Bi[fill[c]] = key[2 * p];
        emap[p] = fill[c];
        fill[c]++;
    }
    /* insertion sort of each column by row, carrying the entry map */
    i64* inv = (i64*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(i64));
    for (i64 p = 0; p < nnz; ++p) inv[emap[p]] = p;
    for (i64 j = 0; j < n; ++j)
        for (i64 q = Bp[j] + 1; q < Bp[j + 1]; ++q) {
            i64 r = Bi[q], e = inv[q], t = q;
            while (t > Bp[j] && Bi[t - 1] > r) { Bi[t] = Bi[t - 1]; inv[t] = inv[t - 1]; --t; }
            Bi[t] = r; inv[t] = e;
        }
    for (i64 q = 0; q < nnz; ++q) emap[inv[q]] = q;
    free(iperm); free(key); free(fill); free(inv);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Symbolic factorization: etree + column structure of L.                    */
/* struct(L_:j) = {i >= j : A_ij != 0}  U  (U_{c: parent[c]=j} struct(L_:c)\{c}) */
/* parent[j] = smallest row of struct(L_:j) above j, or -1 for a root.        */
/* ------------------------------------------------------------------------- */
typedef struct {
    i64 n;
    i64* parent;
    i64* Lp;
    i64* Li;
} orc_sym;

orc_sym* orc_symbolic(i64 n, const i64* Ap, const i64* Ai) {
    orc_sym* s = (orc_sym*)calloc(1, sizeof(orc_sym));
    s->n = n;
    s->parent = (i64*)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    s->Lp = (i64*)malloc((size_t)(n + 1) * sizeof(i64));
    i64* child_head = (i64*)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    i64* child_next = (i64*)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    i64* mark = (i64*)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    vec64 rows = {0, 0, 0}, col = {0, 0, 0};
    for (i64 j = 0; j < n; ++j) { child_head[j] = -1; mark[j] = -1; }
    s->Lp[0] = 0;
    for (i64 j = 0; j < n; ++j) {
        col.n = 0;
        mark[j] = j;
        vpush(&col, j); /* the diagonal is always structurally present */
        for (i64 p = Ap[j]; p < Ap[j + 1]; ++p) {
            i64 i = Ai[p];
            if (i > j && mark[i] != j) { mark[i] = j; vpush(&col, i); }
        }
        for (i64 c = child_head[j]; c != -1; c = child_next[c])
            for (i64 q = s->Lp[c]; q < s->Lp[c + 1]; ++q) {
                i64 i = rows.v[q];
                if (i > j && mark[i] != j) { mark[i] = j; vpush(&col, i); }
            }
        qsort(col.v, (size_t)col.n, sizeof(i64), cmp_i64);
        for (i64 t = 0; t < col.n; ++t) vpush(&rows, col.v[t]);
        s->Lp[j + 1] = rows.n;
        s->parent[j] = col.n > 1 ? col.v[1] : -1;
        if (s->parent[j] >= 0) {
            child_next[j] = child_head[s->parent[j]];
            child_head[s->parent[j]] = j;
        }
    }
    s->Li = rows.v ? rows.v : (i64*)malloc(sizeof(i64));
    free(col.v); free(child_head); free(child_next); free(mark);
    return s;
}

i64 orc_sym_nnz(const orc_sym* s) { return s->Lp[s->n]; }

void orc_sym_get(const orc_sym* s, i64* parent, i64* Lp, i64* Li) {
    memcpy(parent, s->parent, (size_t)s->n * sizeof(i64));
    memcpy(Lp, s->Lp, (size_t)(s->n + 1) * sizeof(i64));
    memcpy(Li, s->Li, (size_t)s->Lp[s->n] * sizeof(i64));
}

void orc_sym_free(orc_sym* s) {
    if (!s) return;
    free(s->parent); free(s->Lp); free(s->Li); free(s);
}

/* ------------------------------------------------------------------------- */
/* Numeric left-looking column Cholesky on the structure of L.               */
/* Bx: values of A_p in (Bp,Bi) layout.  Lx: output, Lp/Li layout.           */
/* Returns 0, or j+1 for the first column whose pivot is not positive.       */
/* ------------------------------------------------------------------------- */
i64 orc_numeric(const orc_sym* s, const i64* Bp, const i64* Bi, const double* Bx, double* Lx) {
    i64 n = s->n;
    const i64 *Lp = s->Lp, *Li = s->Li;
    /* row lists: for each row j, the columns k<j with L_jk structurally nonzero,
       ascending (built by sweeping k ascending) */
    i64* rcount = (i64*)calloc((size_t)(n + 1), sizeof(i64));
    for (i64 k = 0; k < n; ++k)
        for (i64 q = Lp[k] + 1; q < Lp[k + 1]; ++q) rcount[Li[q] + 1]++;
    for (i64 j = 0; j < n; ++j) rcount[j + 1] += rcount[j];
    i64* rcol = (i64*)malloc((size_t)(rcount[n] > 0 ? rcount[n] : 1) * sizeof(i64));
    i64* rfill = (i64*)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    for (i64 j = 0; j < n; ++j) rfill[j] = rcount[j];
    for (i64 k = 0; k < n; ++k)
        for (i64 q = Lp[k] + 1; q < Lp[k + 1]; ++q) rcol[rfill[Li[q]]++] = k;
    double* x = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    i64 info = 0;
    for (i64 j = 0; j < n && info == 0; ++j) {
        /* x <- A_p[j:, j] */
        for (i64 p = Bp[j]; p < Bp[j + 1]; ++p)
            if (Bi[p] >= j) x[Bi[p]] += Bx[p];
        /* x -= L[j:, k] * L_jk for every k < j with L_jk != 0, ascending k */
        for (i64 t = rcount[j]; t < rcount[j + 1]; ++t) {
            i64 k = rcol[t];
            i64 pj = find_row(Li, Lp[k], Lp[k + 1], j);
            double ljk = Lx[pj];
            for (i64 q = pj; q < Lp[k + 1]; ++q) x[Li[q]] -= Lx[q] * ljk;
        }
        double d = x[j];
        if (!(d > 0.0)) { info = j + 1; break; }
        double ljj = sqrt(d);
        Lx[Lp[j]] = ljj;
        for (i64 q = Lp[j] + 1; q < Lp[j + 1]; ++q) Lx[q] = x[Li[q]] / ljj;
        for (i64 q = Lp[j]; q < Lp[j + 1]; ++q) x[Li[q]] = 0.0;
    }
    free(rcount); free(rcol); free(rfill); free(x);
    return info;
}

double orc_logdet(const orc_sym* s, const double* Lx) {
    double acc = 0.0;
    for (i64 j = 0; j < s->n; ++j) acc += log(Lx[s->Lp[j]]);
    return 2.0 * acc;
}

/* x = P^T L^-T L^-1 P b ;  (P b)[i] = b[perm[i]] */
void orc_solve(const orc_sym* s, const double* Lx, const i64* perm, const double* b, double* xout) {
    i64 n = s->n;
    const i64 *Lp = s->Lp, *Li = s->Li;
    double* y = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (i64 i = 0; i < n; ++i) y[i] = b[perm[i]];
    /* forward: L y = P b (column-oriented) */
    for (i64 j = 0; j < n; ++j) {
        y[j] /= Lx[Lp[j]];
        for (i64 q = Lp[j] + 1; q < Lp[j + 1]; ++q) y[Li[q]] -= Lx[q] * y[j];
    }
    /* backward: L^T z = y */
    for (i64 j = n - 1; j >= 0; --j) {
        double acc = y[j];
        for (i64 q = Lp[j] + 1; q < Lp[j + 1]; ++q) acc -= Lx[q] * y[Li[q]];
        y[j] = acc / Lx[Lp[j]];
    }
    for (i64 i = 0; i < n; ++i) xout[perm[i]] = y[i];
    free(y);
}

/* ------------------------------------------------------------------------- */
/* Takahashi selected inverse on pattern(L).  Sx has the layout of Lx.        */
/* ------------------------------------------------------------------------- */
static double sig_at(const orc_sym* s, const double* Sx, i64 a, i64 b) {
    i64 r = a > b ? a : b, c = a > b ? b : a;
    i64 p = find_row(s->Li, s->Lp[c], s->Lp[c + 1], r);
    return p >= 0 ? Sx[p] : NAN; /* closure guarantees p >= 0 */
}

void orc_selinv(const orc_sym* s, const double* Lx, double* Sx) {
    i64 n = s->n;
    const i64 *Lp = s->Lp, *Li = s->Li;
    for (i64 j = n - 1; j >= 0; --j) {
        double ljj = Lx[Lp[j]];
        /* off-diagonal entries of column j, rows i > j (descending order not
           needed: every Sigma_ik used has min(i,k) > j, i.e. a later column) */
        for (i64 q = Lp[j] + 1; q < Lp[j + 1]; ++q) {
            i64 i = Li[q];
            double acc = 0.0;
            for (i64 t = Lp[j] + 1; t < Lp[j + 1]; ++t)
                acc += Lx[t] * sig_at(s, Sx, i, Li[t]);
            Sx[q] = -acc / ljj;
        }
        double acc = 0.0;
        for (i64 t = Lp[j] + 1; t < Lp[j + 1]; ++t) acc += Lx[t] * Sx[t];
        Sx[Lp[j]] = 1.0 / (ljj * ljj) - acc / ljj;
    }
}

/* d logdet(A) / d a_ij for every stored lower entry (i,j) of the ORIGINAL A:
 * (2 - delta_ij) * (A^{-1})_ij, with (A^{-1})_ij = Sigma_{iperm[i], iperm[j]}. */
void orc_grad_logdet(const orc_sym* s, const double* Sx, i64 n, const i64* Ap, const i64* Ai,
                     const i64* perm, double* g) {
    i64* iperm = (i64*)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    for (i64 k = 0; k < n; ++k) iperm[perm[k]] = k;
    for (i64 j = 0; j < n; ++j)
        for (i64 p = Ap[j]; p < Ap[j + 1]; ++p) {
            i64 i = Ai[p];
            double v = sig_at(s, Sx, iperm[i], iperm[j]);
            g[p] = (i == j ? 1.0 : 2.0) * v;
        }
    free(iperm);
}

/* ------------------------------------------------------------------------- */
/* Tile map on the uniform n_b grid (Sec. 4 and the per-tile metadata of       */
/* Sec. 5.2).  Tiles are listed in block-column-major order (J asc, I asc).   */
/* For each tile: I, J, |A|, offset into aind, contiguous flag, full flag,    */
/* kd (diagonal tiles; -1 otherwise) and the structural row extent [r0,r1).   */
/* Diagonal tiles: the active set is the whole logical width (the diagonal of */
/* an SPD matrix is non-zero, Sec. 4.3); the ragged last tile has logical     */
/* width n - (N_T-1) n_b.                                                     */
/* ------------------------------------------------------------------------- */
typedef struct {
    i64 nt, ntiles, naind;
    i64 *tI, *tJ, *nact, *aoff, *contig, *full, *kd, *r0, *r1;
    i64* aind;
} orc_tiles;

orc_tiles* orc_tile_map(const orc_sym* s, i64 nb) {
    i64 n = s->n;
    i64 nt = (n + nb - 1) / nb;
    orc_tiles* T = (orc_tiles*)calloc(1, sizeof(orc_tiles));
    T->nt = nt;
    vec64 tI = {0}, tJ = {0}, nact = {0}, aoff = {0}, contig = {0}, full = {0}, kd = {0},
          r0 = {0}, r1 = {0}, aind = {0};
    /* colhit[I*nb + c] = 1 when column c of block column J has a structural entry in row block I */
    char* colhit = (char*)malloc((size_t)nt * (size_t)nb);
    i64* rmin = (i64*)malloc((size_t)nt * sizeof(i64));
    i64* rmax = (i64*)malloc((size_t)nt * sizeof(i64));
    i64* kdv = (i64*)malloc((size_t)nt * sizeof(i64));
    for (i64 J = 0; J < nt; ++J) {
        memset(colhit, 0, (size_t)nt * (size_t)nb);
        for (i64 I = 0; I < nt; ++I) { rmin[I] = nb; rmax[I] = -1; kdv[I] = -1; }
        i64 c0 = J * nb, c1 = (J + 1) * nb < n ? (J + 1) * nb : n;
        for (i64 j = c0; j < c1; ++j)
            for (i64 q = s->Lp[j]; q < s->Lp[j + 1]; ++q) {
                i64 i = s->Li[q];
                i64 I = i / nb, lr = i - I * nb, lc = j - c0;
                colhit[I * nb + lc] = 1;
                if (lr < rmin[I]) rmin[I] = lr;
                if (lr > rmax[I]) rmax[I] = lr;
                if (I == J && lr - lc > kdv[I]) kdv[I] = lr - lc;
            }
        for (i64 I = J; I < nt; ++I) {
            i64 cnt = 0, first = -1, last = -1;
            for (i64 c = 0; c < nb; ++c)
                if (colhit[I * nb + c]) { if (first < 0) first = c; last = c; cnt++; }
            if (cnt == 0) continue;
            vpush(&tI, I); vpush(&tJ, J); vpush(&nact, cnt); vpush(&aoff, aind.n);
            for (i64 c = 0; c < nb; ++c)
                if (colhit[I * nb + c]) vpush(&aind, c);
            vpush(&contig, (last - first + 1) == cnt);
            vpush(&full, cnt == nb);
            vpush(&kd, I == J ? kdv[I] : -1);
            vpush(&r0, rmin[I]); vpush(&r1, rmax[I] + 1);
        }
    }
    free(colhit); free(rmin); free(rmax); free(kdv);
    T->ntiles = tI.n; T->naind = aind.n;
    T->tI = tI.v; T->tJ = tJ.v; T->nact = nact.v; T->aoff = aoff.v; T->contig = contig.v;
    T->full = full.v; T->kd = kd.v; T->r0 = r0.v; T->r1 = r1.v; T->aind = aind.v;
    return T;
}

void orc_tiles_sizes(const orc_tiles* T, i64* out3) { out3[0] = T->nt; out3[1] = T->ntiles; out3[2] = T->naind; }

/* fields: [ntiles][9] = I, J, nact, aoff, contig, full, kd, r0, r1 ; aind[naind] */
void orc_tiles_get(const orc_tiles* T, i64* fields, i64* aind) {
    for (i64 t = 0; t < T->ntiles; ++t) {
        i64* f = fields + 9 * t;
        f[0] = T->tI[t]; f[1] = T->tJ[t]; f[2] = T->nact[t]; f[3] = T->aoff[t];
        f[4] = T->contig[t]; f[5] = T->full[t]; f[6] = T->kd[t]; f[7] = T->r0[t]; f[8] = T->r1[t];
    }
    if (T->naind) memcpy(aind, T->aind, (size_t)T->naind * sizeof(i64));
}

void orc_tiles_free(orc_tiles* T) {
    if (!T) return;
    free(T->tI); free(T->tJ); free(T->nact); free(T->aoff); free(T->contig); free(T->full);
    free(T->kd); free(T->r0); free(T->r1); free(T->aind); free(T);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1: left-looking tile Cholesky task collection.                   */
/* N(k) = { i != k : tile (i,k) or tile (k,i) active }, iterated ascending.   */
/* Emits (case, m, k, n) with -1 for an unused slot:                          */
/*   for k: (2,-,k,n) for n in N(k), n<k; (1,-,k,-);                          */
/*          for m in N(k), m>k: (4,m,k,n) for n in N(k) & N(m), n<k; (3,m,k,-)*/
/* Returns the number of tasks; writes them when out != NULL.                 */
/* ------------------------------------------------------------------------- */
i64 orc_task_list(const orc_tiles* T, i64* out) {
    i64 nt = T->nt;
    /* lower neighbours of each block: rowlist[k] = { n < k : tile (k,n) active },
       below-diagonal neighbours: collist[k] = { m > k : tile (m,k) active },
       both ascending (tiles are listed J asc, I asc) */
    i64* rc = (i64*)calloc((size_t)(nt + 1), sizeof(i64));
    i64* cc = (i64*)calloc((size_t)(nt + 1), sizeof(i64));
    for (i64 t = 0; t < T->ntiles; ++t)
        if (T->tI[t] != T->tJ[t]) { rc[T->tI[t] + 1]++; cc[T->tJ[t] + 1]++; }
    for (i64 k = 0; k < nt; ++k) { rc[k + 1] += rc[k]; cc[k + 1] += cc[k]; }
    i64 noff = rc[nt] > 0 ? rc[nt] : 1;
    i64* rl = (i64*)malloc((size_t)noff * sizeof(i64));
    i64* cl = (i64*)malloc((size_t)noff * sizeof(i64));
    i64* rf = (i64*)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(i64));
    i64* cf = (i64*)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(i64));
    for (i64 k = 0; k < nt; ++k) { rf[k] = rc[k]; cf[k] = cc[k]; }
    for (i64 t = 0; t < T->ntiles; ++t)
        if (T->tI[t] != T->tJ[t]) { rl[rf[T->tI[t]]++] = T->tJ[t]; cl[cf[T->tJ[t]]++] = T->tI[t]; }
    i64 cnt = 0;
#define EMIT(cs, m, k, nn) do { if (out) { out[4*cnt]=(cs); out[4*cnt+1]=(m); out[4*cnt+2]=(k); out[4*cnt+3]=(nn);} cnt++; } while (0)
    for (i64 k = 0; k < nt; ++k) {
        for (i64 a = rc[k]; a < rc[k + 1]; ++a) EMIT(2, -1, k, rl[a]);
        EMIT(1, -1, k, -1);
        for (i64 b = cc[k]; b < cc[k + 1]; ++b) {
            i64 m = cl[b];
            /* n in N(k) and N(m), n < k: merge of the two ascending lower lists */
            i64 a = rc[k], e = rc[m];
            while (a < rc[k + 1] && e < rc[m + 1]) {
                if (rl[a] == rl[e]) { EMIT(4, m, k, rl[a]); ++a; ++e; }
                else if (rl[a] < rl[e]) ++a;
                else ++e;
            }
            EMIT(3, m, k, -1);
        }
    }
#undef EMIT
    free(rc); free(cc); free(rl); free(cl); free(rf); free(cf);
    return cnt;
}
