/*
 * spx_oracle.c -- plain, slow, obviously correct CPU reference for the
 * supernodal sparse factorization of Lacoste et al., "Taking advantage of
 * hybrid systems for sparse direct solvers via task-based runtimes"
 * (Sec. III, "Supernodal factorization").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or table with the CUDA library.
 *
 * Everything here is FP64 and works column by column, in the order the
 * textbook definitions state; there is no blocking, no supernode and no
 * reordering beyond what each definition says.
 *
 * Conventions: 0-based indices; a matrix is CSC with int64 column pointers
 * and int32 row indices; a permutation `perm` maps new -> old
 * (the k-th unknown of the reordered system is old unknown perm[k]).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Nested dissection on a regular grid (Sec. III: the first step is a nested
 * dissection of the connectivity graph, whose separators become the nodes of
 * the elimination tree).  The paper uses Scotch; its rules are not given, so
 * this follows the geometric reading: split the box across its longest axis
 * (ties to the lowest axis, x < y < z) at plane lo + floor(len/2); order the
 * lower half, then the upper half, then the separator plane; boxes of at most
 * 8 grid nodes and separator planes are ordered lexicographically with x
 * fastest; the dof of one node are consecutive.                             */
/* ------------------------------------------------------------------------ */

static void ora_emit_box(int nx, int ny, int dof, const int lo[3],
                         const int hi[3], int64_t *perm, int64_t *pos)
{
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x) {
                int64_t node = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
                for (int d = 0; d < dof; ++d) perm[(*pos)++] = node * dof + d;
            }
}

static void ora_nd_box(int nx, int ny, int dof, const int lo[3], const int hi[3],
                       int64_t *perm, int64_t *pos)
{
    int len[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    if (len[0] <= 0 || len[1] <= 0 || len[2] <= 0) return;
    int64_t vol = (int64_t)len[0] * len[1] * len[2];
    if (vol <= 8) {
        ora_emit_box(nx, ny, dof, lo, hi, perm, pos);
        return;
    }
    int ax = 0;
    if (len[1] > len[ax]) ax = 1;
    if (len[2] > len[ax]) ax = 2;
    int cut = lo[ax] + len[ax] / 2;
    int lo_a[3], hi_a[3], lo_b[3], hi_b[3], lo_s[3], hi_s[3];
    for (int d = 0; d < 3; ++d) {
        lo_a[d] = lo_b[d] = lo_s[d] = lo[d];
        hi_a[d] = hi_b[d] = hi_s[d] = hi[d];
    }
    hi_a[ax] = cut;          /* lower half  [lo, cut)   */
    lo_b[ax] = cut + 1;      /* upper half  [cut+1, hi) */
    lo_s[ax] = cut;          /* separator   [cut, cut+1) */
    hi_s[ax] = cut + 1;
    ora_nd_box(nx, ny, dof, lo_a, hi_a, perm, pos);
    ora_nd_box(nx, ny, dof, lo_b, hi_b, perm, pos);
    ora_emit_box(nx, ny, dof, lo_s, hi_s, perm, pos);
}

int ora_nd_grid(int nx, int ny, int nz, int dof, int64_t *perm)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || dof <= 0) return -1;
    int lo[3] = {0, 0, 0}, hi[3] = {nx, ny, nz};
    int64_t pos = 0;
    ora_nd_box(nx, ny, dof, lo, hi, perm, &pos);
    return pos == (int64_t)nx * ny * nz * dof ? 0 : -2;
}

/* ------------------------------------------------------------------------ */
/* Nested dissection on a general graph (same section).  Reading used here:
 * level-structure bisection.  Subsets of at most 64 vertices, and graphs
 * whose level structure has fewer than 3 levels, are emitted in ascending
 * vertex order.  A disconnected subset is split into its connected
 * components, taken in order of their smallest vertex.  A connected subset
 * is rooted at a pseudo-peripheral vertex: start at its smallest vertex;
 * repeatedly move to the vertex of the last BFS level with the fewest
 * neighbours inside the subset (ties: smallest index) while that makes the
 * level structure deeper.  With m levels, level floor(m/2) is the
 * separator; levels below it are ordered first, levels above it second,
 * the separator (ascending) last.  `adjp/adji` is the graph without
 * self-loops, symmetric.                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    const int64_t *adjp;
    const int32_t *adji;
    int32_t *label;   /* label of the subset a vertex currently belongs to */
    int32_t *level;   /* BFS level scratch */
    int32_t next_label;
    int64_t *perm;
    int64_t pos;
} ora_graph_ctx;

static int ora_cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* BFS from root inside subset `lab`; fills order[] (BFS order), level[] of
 * visited vertices, returns the number of visited vertices and sets *nlev. */
static int64_t ora_bfs(ora_graph_ctx *g, int32_t lab, int32_t root, int32_t *order,
                       int32_t *nlev)
{
    int64_t head = 0, tail = 0;
    order[tail++] = root;
    g->level[root] = 0;
    int32_t maxlev = 0;
    /* visited marker: level >= 0 for this BFS; caller resets to -1 */
    while (head < tail) {
        int32_t v = order[head++];
        for (int64_t p = g->adjp[v]; p < g->adjp[v + 1]; ++p) {
            int32_t w = g->adji[p];
            if (g->label[w] != lab || g->level[w] >= 0) continue;
            g->level[w] = g->level[v] + 1;
            if (g->level[w] > maxlev) maxlev = g->level[w];
            order[tail++] = w;
        }
    }
    *nlev = maxlev + 1;
    return tail;
}

static void ora_nd_subset(ora_graph_ctx *g, int32_t *verts, int64_t nv);

static void ora_emit_sorted(ora_graph_ctx *g, int32_t *verts, int64_t nv)
{
    qsort(verts, (size_t)nv, sizeof(int32_t), ora_cmp_i32);
    for (int64_t i = 0; i < nv; ++i) g->perm[g->pos++] = verts[i];
}

static void ora_nd_subset(ora_graph_ctx *g, int32_t *verts, int64_t nv)
{
    if (nv <= 0) return;
    if (nv <= 64) {
        ora_emit_sorted(g, verts, nv);
        return;
    }
    int32_t lab = g->next_label++;
    for (int64_t i = 0; i < nv; ++i) {
        g->label[verts[i]] = lab;
        g->level[verts[i]] = -1;
    }
    qsort(verts, (size_t)nv, sizeof(int32_t), ora_cmp_i32);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    int32_t nlev = 0;
    int64_t seen = ora_bfs(g, lab, verts[0], order, &nlev);
    if (seen < nv) {
        /* Disconnected: split into components, ordered by smallest vertex. */
        int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
        int32_t *comp_lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
        int64_t ncomp = 0;
        /* collect components one by one using fresh BFS runs */
        int64_t done = 0;
        for (int64_t i = 0; i < nv; ++i) g->level[verts[i]] = -1;
        int64_t *starts = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv + 1));
        for (int64_t i = 0; i < nv; ++i) {
            int32_t v = verts[i];
            if (g->level[v] >= 0) continue;
            int32_t nl;
            int64_t c = ora_bfs(g, lab, v, comp + done, &nl);
            starts[ncomp++] = done;
            done += c;
        }
        starts[ncomp] = done;
        (void)comp_lab;
        for (int64_t c = 0; c < ncomp; ++c) {
            int64_t cn = starts[c + 1] - starts[c];
            int32_t *cv = (int32_t *)malloc(sizeof(int32_t) * (size_t)cn);
            memcpy(cv, comp + starts[c], sizeof(int32_t) * (size_t)cn);
            ora_nd_subset(g, cv, cn);
            free(cv);
        }
        free(starts);
        free(comp_lab);
        free(comp);
        free(order);
        return;
    }
    /* Pseudo-peripheral root. */
    int32_t root = verts[0];
    for (;;) {
        int32_t best = -1, bestdeg = 0;
        for (int64_t i = 0; i < nv; ++i) {
            int32_t v = order[i];
            if (g->level[v] != nlev - 1) continue;
            int32_t deg = 0;
            for (int64_t p = g->adjp[v]; p < g->adjp[v + 1]; ++p)
                if (g->label[g->adji[p]] == lab) ++deg;
            if (best < 0 || deg < bestdeg || (deg == bestdeg && v < best)) {
                best = v;
                bestdeg = deg;
            }
        }
        for (int64_t i = 0; i < nv; ++i) g->level[verts[i]] = -1;
        int32_t nl2 = 0;
        ora_bfs(g, lab, best, order, &nl2);
        if (nl2 > nlev) {
            root = best;
            nlev = nl2;
            continue;
        }
        /* keep the previous root's level structure */
        for (int64_t i = 0; i < nv; ++i) g->level[verts[i]] = -1;
        ora_bfs(g, lab, root, order, &nlev);
        break;
    }
    if (nlev < 3) {
        free(order);
        ora_emit_sorted(g, verts, nv);
        return;
    }
    int32_t mid = nlev / 2;
    int64_t na = 0, nb = 0, ns = 0;
    for (int64_t i = 0; i < nv; ++i) {
        int32_t l = g->level[verts[i]];
        if (l < mid) ++na; else if (l > mid) ++nb; else ++ns;
    }
    int32_t *va = (int32_t *)malloc(sizeof(int32_t) * (size_t)(na + 1));
    int32_t *vb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nb + 1));
    int32_t *vs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns + 1));
    na = nb = ns = 0;
    for (int64_t i = 0; i < nv; ++i) {
        int32_t v = verts[i], l = g->level[v];
        if (l < mid) va[na++] = v; else if (l > mid) vb[nb++] = v; else vs[ns++] = v;
    }
    free(order);
    ora_nd_subset(g, va, na);
    ora_nd_subset(g, vb, nb);
    ora_emit_sorted(g, vs, ns);
    free(va);
    free(vb);
    free(vs);
}

int ora_nd_graph(int64_t n, const int64_t *adjp, const int32_t *adji, int64_t *perm)
{
    if (n < 0) return -1;
    ora_graph_ctx g;
    g.adjp = adjp;
    g.adji = adji;
    g.label = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    g.level = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    g.next_label = 1;
    g.perm = perm;
    g.pos = 0;
    int32_t *all = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < n; ++i) {
        all[i] = (int32_t)i;
        g.label[i] = 0;
        g.level[i] = -1;
    }
    ora_nd_subset(&g, all, n);
    free(all);
    free(g.label);
    free(g.level);
    return g.pos == n ? 0 : -2;
}

/* ------------------------------------------------------------------------ */
/* Elimination tree (Sec. III, citing Liu): parent(j) = min{ i > j : L(i,j)
 * != 0 }.  Computed here with Liu's ancestor algorithm on the pattern of the
 * (already permuted, symmetric) matrix; the symbolic routine below derives
 * the same tree a second, independent way.                                  */
/* ------------------------------------------------------------------------ */

int ora_etree(int64_t n, const int64_t *Ap, const int32_t *Ai, int64_t *parent)
{
    int64_t *anc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t k = 0; k < n; ++k) {
        parent[k] = -1;
        anc[k] = -1;
        /* entries A(i,k) with i < k: row k of the lower triangle */
        for (int64_t p = Ap[k]; p < Ap[k + 1]; ++p) {
            int64_t i = Ai[p];
            while (i >= 0 && i < k) {
                int64_t up = anc[i];
                anc[i] = k;          /* path compression towards k */
                if (up < 0) parent[i] = k;
                i = up;
            }
        }
    }
    free(anc);
    return 0;
}

/* Column counts c_j = |struct(L(:,j))| (diagonal included) by row subtrees:
 * the nonzeros of row i of L are the nodes met walking the elimination tree
 * up from every k with A(i,k) != 0, k < i, until i or a node already
 * visited for row i.                                                        */
int ora_colcounts(int64_t n, const int64_t *Ap, const int32_t *Ai, const int64_t *parent,
                  int64_t *count)
{
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t j = 0; j < n; ++j) {
        count[j] = 1;
        mark[j] = -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        mark[i] = i;
        for (int64_t p = Ap[i]; p < Ap[i + 1]; ++p) {
            int64_t k = Ai[p];   /* symmetric pattern: column i holds row k */
            if (k >= i) continue;
            while (k >= 0 && mark[k] != i) {
                mark[k] = i;
                count[k] += 1;   /* L(i,k) != 0 */
                k = parent[k];
            }
        }
    }
    free(mark);
    return 0;
}

/* Symbolic factorization (Sec. III: predict the nonzero pattern of the
 * factor).  Column by column: struct(L(:,j)) = {j} U struct(A(j+1:n, j))
 * U the union over children c (parent(c) = j) of struct(L(:,c)) minus c;
 * parent(j) = the smallest row of struct(L(:,j)) other than j.  Lp must be
 * preallocated from column counts; Li receives sorted row indices.  Returns
 * -(j+1) if column j does not fit its count.                               */
int ora_symbolic(int64_t n, const int64_t *Ap, const int32_t *Ai, const int64_t *Lp,
                 int32_t *Li, int64_t *parent)
{
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *child_head = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *child_next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int rc = 0;
    for (int64_t j = 0; j < n; ++j) {
        mark[j] = -1;
        child_head[j] = -1;
        child_next[j] = -1;
    }
    for (int64_t j = 0; j < n && rc == 0; ++j) {
        int64_t len = 0;
        mark[j] = j;
        buf[len++] = (int32_t)j;
        for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) {
            int64_t i = Ai[p];
            if (i > j && mark[i] != j) {
                mark[i] = j;
                buf[len++] = (int32_t)i;
            }
        }
        for (int64_t c = child_head[j]; c >= 0; c = child_next[c]) {
            for (int64_t p = Lp[c]; p < Lp[c + 1]; ++p) {
                int64_t i = Li[p];
                if (i > j && mark[i] != j) {
                    mark[i] = j;
                    buf[len++] = (int32_t)i;
                }
            }
        }
        if (len != Lp[j + 1] - Lp[j]) {
            rc = (int)-(j + 1);
            break;
        }
        qsort(buf, (size_t)len, sizeof(int32_t), ora_cmp_i32);
        memcpy(Li + Lp[j], buf, sizeof(int32_t) * (size_t)len);
        parent[j] = len > 1 ? buf[1] : -1;
        if (parent[j] >= 0) {
            child_next[j] = child_head[parent[j]];
            child_head[parent[j]] = j;
        }
    }
    free(buf);
    free(child_next);
    free(child_head);
    free(mark);
    return rc;
}

/* Row lists of the pattern: for every row i, the columns k < i with
 * L(i,k) != 0 in ascending k (the "row subtree").                           */
static void ora_row_lists(int64_t n, const int64_t *Lp, const int32_t *Li, int64_t **Rp_out,
                          int32_t **Rk_out)
{
    int64_t *Rp = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    for (int64_t k = 0; k < n; ++k)
        for (int64_t p = Lp[k] + 1; p < Lp[k + 1]; ++p) Rp[Li[p] + 1] += 1;
    for (int64_t i = 0; i < n; ++i) Rp[i + 1] += Rp[i];
    int32_t *Rk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(Rp[n] + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < n; ++i) fill[i] = Rp[i];
    for (int64_t k = 0; k < n; ++k)          /* ascending k => sorted lists */
        for (int64_t p = Lp[k] + 1; p < Lp[k + 1]; ++p) Rk[fill[Li[p]]++] = (int32_t)k;
    free(fill);
    *Rp_out = Rp;
    *Rk_out = Rk;
}

/* ------------------------------------------------------------------------ */
/* Numerical Cholesky, left-looking, one column at a time (Sec. III: the
 * factorization computes L with P A P^T = L L^T; the left-looking variant
 * gathers every update into the column being computed).  For column j:
 *   w = A(j:n, j);  for every k < j with L(j,k) != 0, in ascending k:
 *   w(i) -= L(i,k) * L(j,k) for i >= j;  L(j,j) = sqrt(w(j));
 *   L(i,j) = w(i) / L(j,j).
 * Returns 0, or -(j+1) if the pivot of column j is not positive.  Lp/Li is
 * the symbolic pattern (sorted, diagonal first).  Ap/Ai/Ax is the permuted
 * matrix; only its lower triangle is read.                                  */
/* ------------------------------------------------------------------------ */

int ora_cholesky(int64_t n, const int64_t *Ap, const int32_t *Ai, const double *Ax,
                 const int64_t *Lp, const int32_t *Li, double *Lx)
{
    int64_t *Rp;
    int32_t *Rk;
    ora_row_lists(n, Lp, Li, &Rp, &Rk);
    double *w = (double *)calloc((size_t)(n + 1), sizeof(double));
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int rc = 0;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p)
            if (Ai[p] >= j) w[Ai[p]] += Ax[p];
        for (int64_t r = Rp[j]; r < Rp[j + 1]; ++r) {
            int64_t k = Rk[r];
            int64_t p = next[k];           /* position of row j in column k */
            double ljk = Lx[p];
            for (int64_t q = p; q < Lp[k + 1]; ++q) w[Li[q]] -= Lx[q] * ljk;
            next[k] = p + 1;
        }
        double d = w[j];
        if (!(d > 0.0)) {
            rc = (int)-(j + 1);
            break;
        }
        double ljj = sqrt(d);
        Lx[Lp[j]] = ljj;
        w[j] = 0.0;
        for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) {
            Lx[p] = w[Li[p]] / ljj;
            w[Li[p]] = 0.0;
        }
        next[j] = Lp[j] + 1;
    }
    free(next);
    free(w);
    free(Rk);
    free(Rp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Numerical LU with static pivoting on the symmetric pattern of A + A^T
 * (Sec. III: PaStiX factors non-symmetric matrices on the pattern of
 * A + A^T and does no dynamic pivoting).  Left-looking column j:
 *   x = A(:, j);  for every k < j with U(k,j) != 0, ascending:
 *     U(k,j) = x(k);  x(i) -= L(i,k) * U(k,j) for i > k;
 *   U(j,j) = x(j), replaced by sign(x(j)) * tau when |x(j)| < tau
 *   (sign +1 for 0);  L(i,j) = x(i) / U(j,j) for i > j.
 * L is unit lower (the stored diagonal slot holds U(j,j)); U is returned
 * transposed in the pattern of L: Ut[p] = U(j, Li[p]) for p in column j.
 * The static-pivot threshold tau is a reading (the paper gives none):
 * tau = sqrt(eps) * ||A||_inf.  *nrepl receives the replacement count.       */
/* ------------------------------------------------------------------------ */

int ora_lu(int64_t n, const int64_t *Ap, const int32_t *Ai, const double *Ax, const int64_t *Lp,
           const int32_t *Li, double tau, double *Lx, double *Ut, int64_t *nrepl)
{
    int64_t *Rp;
    int32_t *Rk;
    ora_row_lists(n, Lp, Li, &Rp, &Rk);
    double *x = (double *)calloc((size_t)(n + 1), sizeof(double));
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    *nrepl = 0;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) x[Ai[p]] += Ax[p];
        for (int64_t r = Rp[j]; r < Rp[j + 1]; ++r) {
            int64_t k = Rk[r];
            int64_t p = next[k];           /* position of row j in column k */
            double ukj = x[k];
            Ut[p] = ukj;                   /* U(k,j) sits at L(j,k)'s slot */
            x[k] = 0.0;
            for (int64_t q = Lp[k] + 1; q < Lp[k + 1]; ++q) x[Li[q]] -= Lx[q] * ukj;
            next[k] = p + 1;
        }
        double piv = x[j];
        if (fabs(piv) < tau) {
            piv = (piv < 0.0) ? -tau : tau;
            *nrepl += 1;
        }
        Ut[Lp[j]] = piv;
        Lx[Lp[j]] = 1.0;
        x[j] = 0.0;
        for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) {
            Lx[p] = x[Li[p]] / piv;
            x[Li[p]] = 0.0;
        }
        next[j] = Lp[j] + 1;
    }
    free(next);
    free(x);
    free(Rk);
    free(Rp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Selected inverse of A = L L^T on the pattern of L (the Takahashi
 * recurrence; the gradient of log det A is A^{-T} on A's pattern).  From
 * Z = A^{-1} = L^{-T} L^{-1}, L^T Z is lower triangular with diagonal
 * 1 / L(j,j); reading its entries (j, i), i >= j, gives, for the rows S of
 * column j below the diagonal, processed for j = n-1 down to 0:
 *   Z(i, j) = -(1 / L(j,j)) sum_{k in S} L(k, j) Z(k, i)      (i in S)
 *   Z(j, j) = 1 / L(j,j)^2 - (1 / L(j,j)) sum_{k in S} L(k, j) Z(k, j)
 * Every Z(k, i) with k, i in S lies in the pattern of L (columns of S are
 * ancestors of j and S is a clique in the filled graph) and belongs to a
 * column > j, already final.  Zx is returned on the pattern of L (lower
 * entries, same positions as Lx).  Returns 0, or -1 if a needed entry is
 * missing from the pattern.                                                 */
/* ------------------------------------------------------------------------ */

static int64_t ora_find(const int64_t *Lp, const int32_t *Li, int64_t col, int64_t row)
{
    int64_t lo = Lp[col], hi = Lp[col + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (Li[mid] == row) return mid;
        if (Li[mid] < row) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

int ora_selinv(int64_t n, const int64_t *Lp, const int32_t *Li, const double *Lx, double *Zx)
{
    for (int64_t j = n - 1; j >= 0; --j) {
        const int64_t p0 = Lp[j], p1 = Lp[j + 1];   /* p0: the diagonal */
        const double d = Lx[p0];
        /* off-diagonal entries first; they only read columns > j */
        for (int64_t pi = p0 + 1; pi < p1; ++pi) {
            const int64_t i = Li[pi];
            double s = 0.0;
            for (int64_t pk = p0 + 1; pk < p1; ++pk) {
                const int64_t k = Li[pk];
                const int64_t c = k < i ? k : i, r = k < i ? i : k;
                const int64_t q = ora_find(Lp, Li, c, r);
                if (q < 0) return -1;
                s += Lx[pk] * Zx[q];
            }
            Zx[pi] = -s / d;
        }
        double s = 0.0;
        for (int64_t pk = p0 + 1; pk < p1; ++pk) s += Lx[pk] * Zx[pk];
        Zx[p0] = 1.0 / (d * d) - s / d;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Numerical LDL^T with static pivoting (the L D L^T variant of the
 * factorization, Sec. V-B: the update becomes C = C - L D L^T).  Left-looking
 * column j, on the lower pattern:
 *   w = A(j:n, j);  for every k < j with L(j,k) != 0, in ascending k:
 *   w(i) -= L(i,k) * d_k * L(j,k) for i >= j;
 *   d_j = w(j), replaced by sign(d_j) * tau when |d_j| < tau (+tau for 0)
 *   and counted; L(i,j) = w(i) / d_j for i > j.
 * L is unit lower; the stored diagonal slot of Lx holds d_j.  With tau = 0 a
 * zero pivot returns -(j+1).  Ap/Ai/Ax is the permuted matrix; only its
 * lower triangle is read.                                                   */
/* ------------------------------------------------------------------------ */

int ora_ldlt(int64_t n, const int64_t *Ap, const int32_t *Ai, const double *Ax, const int64_t *Lp,
             const int32_t *Li, double tau, double *Lx, int64_t *nrepl)
{
    int64_t *Rp;
    int32_t *Rk;
    ora_row_lists(n, Lp, Li, &Rp, &Rk);
    double *w = (double *)calloc((size_t)(n + 1), sizeof(double));
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int rc = 0;
    *nrepl = 0;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p)
            if (Ai[p] >= j) w[Ai[p]] += Ax[p];
        for (int64_t r = Rp[j]; r < Rp[j + 1]; ++r) {
            int64_t k = Rk[r];
            int64_t p = next[k];           /* position of row j in column k */
            double f = Lx[Lp[k]] * Lx[p];  /* d_k L(j,k) */
            for (int64_t q = p; q < Lp[k + 1]; ++q) w[Li[q]] -= Lx[q] * f;
            next[k] = p + 1;
        }
        double d = w[j];
        if (tau > 0.0) {
            if (fabs(d) < tau) {
                d = d < 0.0 ? -tau : tau;
                (*nrepl)++;
            }
        } else if (d == 0.0) {
            rc = (int)-(j + 1);
            break;
        }
        Lx[Lp[j]] = d;
        w[j] = 0.0;
        for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) {
            Lx[p] = w[Li[p]] / d;
            w[Li[p]] = 0.0;
        }
        next[j] = Lp[j] + 1;
    }
    free(next);
    free(w);
    free(Rk);
    free(Rp);
    return rc;
}

/* L D L^T x = b: forward substitution with the unit L, division by D,
 * backward substitution with L^T; in place, permuted numbering.            */
int ora_solve_ldlt(int64_t n, const int64_t *Lp, const int32_t *Li, const double *Lx, int64_t nrhs,
                   double *X, int64_t ldx)
{
    for (int64_t c = 0; c < nrhs; ++c) {
        double *x = X + c * ldx;
        for (int64_t j = 0; j < n; ++j)
            for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) x[Li[p]] -= Lx[p] * x[j];
        for (int64_t j = 0; j < n; ++j) x[j] /= Lx[Lp[j]];
        for (int64_t j = n - 1; j >= 0; --j) {
            double s = x[j];
            for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) s -= Lx[p] * x[Li[p]];
            x[j] = s;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Triangular solves on the factors (forward then backward substitution), in
 * the permuted numbering, nrhs columns of leading dimension ldb, in place. */
/* ------------------------------------------------------------------------ */

int ora_solve_cholesky(int64_t n, const int64_t *Lp, const int32_t *Li, const double *Lx,
                       int64_t nrhs, double *B, int64_t ldb)
{
    for (int64_t c = 0; c < nrhs; ++c) {
        double *x = B + c * ldb;
        for (int64_t j = 0; j < n; ++j) {          /* L y = b */
            x[j] /= Lx[Lp[j]];
            for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) x[Li[p]] -= Lx[p] * x[j];
        }
        for (int64_t j = n - 1; j >= 0; --j) {     /* L^T x = y */
            double s = x[j];
            for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) s -= Lx[p] * x[Li[p]];
            x[j] = s / Lx[Lp[j]];
        }
    }
    return 0;
}

int ora_solve_lu(int64_t n, const int64_t *Lp, const int32_t *Li, const double *Lx,
                 const double *Ut, int64_t nrhs, double *B, int64_t ldb)
{
    for (int64_t c = 0; c < nrhs; ++c) {
        double *x = B + c * ldb;
        for (int64_t j = 0; j < n; ++j)            /* L y = b, unit diagonal */
            for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) x[Li[p]] -= Lx[p] * x[j];
        for (int64_t j = n - 1; j >= 0; --j) {     /* U x = y; row j of U = Ut col j */
            double s = x[j];
            for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) s -= Ut[p] * x[Li[p]];
            x[j] = s / Ut[Lp[j]];
        }
    }
    return 0;
}

/* y = A x for a CSC matrix (used for residuals in the tests). */
int ora_spmv(int64_t n, const int64_t *Ap, const int32_t *Ai, const double *Ax, const double *x,
             double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) y[Ai[p]] += Ax[p] * x[j];
    return 0;
}
