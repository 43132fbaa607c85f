// analyze.cpp -- host analysis of libspx (Sec. III of Lacoste et al.):
// nested-dissection ordering, elimination tree, supernode partition with its
// block-symbolic structure, amalgamation (Sec. V: up to 12% extra fill),
// vertical splitting of wide supernodes, the panel elimination tree and its
// levels, the (source, target) update tasks with their row maps, and the
// assembly / residual maps.  Runs on the host only and needs no GPU.
#include "spx_plan.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <numeric>
#include <queue>
#include <string>
#include <tuple>

namespace spx {

// ---------------------------------------------------------------------------
// Geometric nested dissection (Sec. III ordering step).  Reading of the rule
// (the paper delegates to Scotch): cut the box across its longest axis, ties
// to x then y then z, at plane lo + len/2; lower part, upper part, then the
// separator plane; boxes of at most 8 nodes and the planes themselves are
// listed with x fastest; the dof of a node stay together.
// ---------------------------------------------------------------------------
void order_grid(int nx, int ny, int nz, int dof, std::vector<int64_t> &perm)
{
    perm.clear();
    perm.reserve((size_t)nx * ny * nz * dof);
    struct Box { int lo[3], hi[3]; bool emit_only; };
    auto emit = [&](const Box &b) {
        for (int z = b.lo[2]; z < b.hi[2]; ++z)
            for (int y = b.lo[1]; y < b.hi[1]; ++y)
                for (int x = b.lo[0]; x < b.hi[0]; ++x) {
                    int64_t node = x + (int64_t)nx * (y + (int64_t)ny * z);
                    for (int d = 0; d < dof; ++d) perm.push_back(node * dof + d);
                }
    };
    // Explicit stack; a box is pushed as (separator emit, upper, lower) so the
    // pops come out lower, upper, separator.
    std::vector<Box> stack;
    stack.push_back(Box{{0, 0, 0}, {nx, ny, nz}, false});
    while (!stack.empty()) {
        Box b = stack.back();
        stack.pop_back();
        int len[3] = {b.hi[0] - b.lo[0], b.hi[1] - b.lo[1], b.hi[2] - b.lo[2]};
        if (len[0] <= 0 || len[1] <= 0 || len[2] <= 0) continue;
        if (b.emit_only || (int64_t)len[0] * len[1] * len[2] <= 8) {
            emit(b);
            continue;
        }
        int ax = (len[1] > len[0]) ? 1 : 0;
        if (len[2] > len[ax]) ax = 2;
        int cut = b.lo[ax] + len[ax] / 2;
        Box lower = b, upper = b, sep = b;
        lower.hi[ax] = cut;
        upper.lo[ax] = cut + 1;
        sep.lo[ax] = cut;
        sep.hi[ax] = cut + 1;
        sep.emit_only = true;
        stack.push_back(sep);
        stack.push_back(upper);
        stack.push_back(lower);
    }
}

// ---------------------------------------------------------------------------
// Level-structure nested dissection of a general graph (same step).  Reading:
// sets of <= 64 vertices and level structures of < 3 levels are listed in
// ascending order; a disconnected set is handled component by component in
// order of smallest vertex; a connected set is rooted at a pseudo-peripheral
// vertex found from its smallest vertex by moving to the least-connected
// (then smallest) vertex of the deepest level while the structure deepens;
// the middle level floor(m/2) separates the lower and upper levels, which are
// ordered before it.
// ---------------------------------------------------------------------------
namespace {

struct GraphND {
    const std::vector<int64_t> &adjp;
    const std::vector<int32_t> &adji;
    std::vector<int32_t> owner;   // set id of each vertex
    std::vector<int32_t> dist;    // BFS distance, -1 = unvisited
    std::vector<int64_t> &out;
    int32_t fresh = 1;

    GraphND(const std::vector<int64_t> &p, const std::vector<int32_t> &i, int64_t n,
            std::vector<int64_t> &o)
        : adjp(p), adji(i), owner(n, 0), dist(n, -1), out(o) {}

    // BFS restricted to set `id`; returns visit order, depth via *depth.
    std::vector<int32_t> bfs(int32_t id, int32_t root, int32_t *depth)
    {
        std::vector<int32_t> order;
        order.push_back(root);
        dist[root] = 0;
        int32_t deepest = 0;
        for (size_t h = 0; h < order.size(); ++h) {
            int32_t v = order[h];
            for (int64_t p = adjp[v]; p < adjp[v + 1]; ++p) {
                int32_t w = adji[p];
                if (owner[w] != id || dist[w] != -1) continue;
                dist[w] = dist[v] + 1;
                deepest = std::max(deepest, dist[w]);
                order.push_back(w);
            }
        }
        *depth = deepest + 1;
        return order;
    }

    void reset(const std::vector<int32_t> &vs)
    {
        for (int32_t v : vs) dist[v] = -1;
    }

    void list_sorted(std::vector<int32_t> vs)
    {
        std::sort(vs.begin(), vs.end());
        for (int32_t v : vs) out.push_back(v);
    }

    void run(std::vector<int32_t> vs)
    {
        if (vs.empty()) return;
        if (vs.size() <= 64) {
            list_sorted(std::move(vs));
            return;
        }
        std::sort(vs.begin(), vs.end());
        int32_t id = fresh++;
        for (int32_t v : vs) {
            owner[v] = id;
            dist[v] = -1;
        }
        int32_t depth = 0;
        std::vector<int32_t> order = bfs(id, vs[0], &depth);
        if (order.size() < vs.size()) {
            reset(vs);
            std::vector<std::vector<int32_t>> comps;
            for (int32_t v : vs) {
                if (dist[v] != -1) continue;
                int32_t d;
                comps.push_back(bfs(id, v, &d));
            }
            for (auto &c : comps) run(std::move(c));
            return;
        }
        int32_t root = vs[0];
        while (true) {
            int32_t cand = -1, cand_deg = 0;
            for (int32_t v : order) {
                if (dist[v] != depth - 1) continue;
                int32_t deg = 0;
                for (int64_t p = adjp[v]; p < adjp[v + 1]; ++p) deg += (owner[adji[p]] == id);
                if (cand < 0 || deg < cand_deg || (deg == cand_deg && v < cand)) {
                    cand = v;
                    cand_deg = deg;
                }
            }
            reset(vs);
            int32_t d2 = 0;
            order = bfs(id, cand, &d2);
            if (d2 > depth) {
                root = cand;
                depth = d2;
                continue;
            }
            reset(vs);
            order = bfs(id, root, &depth);
            break;
        }
        if (depth < 3) {
            list_sorted(std::move(vs));
            return;
        }
        int32_t mid = depth / 2;
        std::vector<int32_t> lo, hi, sep;
        for (int32_t v : vs) {
            if (dist[v] < mid) lo.push_back(v);
            else if (dist[v] > mid) hi.push_back(v);
            else sep.push_back(v);
        }
        run(std::move(lo));
        run(std::move(hi));
        list_sorted(std::move(sep));
    }
};

}  // namespace

void order_graph(int64_t n, const std::vector<int64_t> &adjp, const std::vector<int32_t> &adji,
                 std::vector<int64_t> &perm)
{
    perm.clear();
    perm.reserve(n);
    GraphND g(adjp, adji, n, perm);
    std::vector<int32_t> all(n);
    std::iota(all.begin(), all.end(), 0);
    g.run(std::move(all));
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
namespace {

// Symmetric adjacency (no diagonal) of A + A^T in the original numbering.
void build_adjacency(int64_t n, const int64_t *colptr, const int32_t *rowind,
                     std::vector<int64_t> &adjp, std::vector<int32_t> &adji)
{
    std::vector<int64_t> deg(n + 1, 0);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            int64_t i = rowind[p];
            if (i == j) continue;
            deg[i + 1]++;
            deg[j + 1]++;
        }
    for (int64_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
    std::vector<int32_t> tmp(deg[n]);
    std::vector<int64_t> fill(deg.begin(), deg.end() - 1);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            int64_t i = rowind[p];
            if (i == j) continue;
            tmp[fill[i]++] = (int32_t)j;
            tmp[fill[j]++] = (int32_t)i;
        }
    // sort and deduplicate each list
    adjp.assign(n + 1, 0);
    adji.clear();
    adji.reserve(tmp.size());
    for (int64_t v = 0; v < n; ++v) {
        auto b = tmp.begin() + deg[v], e = tmp.begin() + deg[v + 1];
        std::sort(b, e);
        auto last = std::unique(b, e);
        adji.insert(adji.end(), b, last);
        adjp[v + 1] = (int64_t)adji.size();
    }
}

// Adjacency of the permuted graph: column j lists iperm of neighbours.
void permute_adjacency(int64_t n, const std::vector<int64_t> &adjp,
                       const std::vector<int32_t> &adji, const std::vector<int64_t> &perm,
                       const std::vector<int64_t> &iperm, std::vector<int64_t> &padjp,
                       std::vector<int32_t> &padji)
{
    padjp.assign(n + 1, 0);
    padji.resize(adji.size());
    for (int64_t j = 0; j < n; ++j) padjp[j + 1] = padjp[j] + (adjp[perm[j] + 1] - adjp[perm[j]]);
    for (int64_t j = 0; j < n; ++j) {
        int64_t o = perm[j], q = padjp[j];
        for (int64_t p = adjp[o]; p < adjp[o + 1]; ++p) padji[q++] = (int32_t)iperm[adji[p]];
        std::sort(padji.begin() + padjp[j], padji.begin() + padjp[j + 1]);
    }
}

// Elimination tree by Liu's ancestor method on the permuted adjacency.
void elimination_tree(int64_t n, const std::vector<int64_t> &padjp,
                      const std::vector<int32_t> &padji, std::vector<int64_t> &parent)
{
    parent.assign(n, -1);
    std::vector<int64_t> root_of(n, -1);   // virtual forest with path compression
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t p = padjp[j]; p < padjp[j + 1]; ++p) {
            int64_t i = padji[p];
            if (i >= j) break;  // sorted: only the entries above the diagonal of column j
            while (true) {
                int64_t a = root_of[i];
                if (a == j) break;
                root_of[i] = j;
                if (a < 0) {
                    parent[i] = j;
                    break;
                }
                i = a;
            }
        }
    }
}

// Postorder of a forest whose children are visited in ascending order.
std::vector<int64_t> postorder(int64_t n, const std::vector<int64_t> &parent)
{
    std::vector<int64_t> head(n, -1), next(n, -1);
    for (int64_t j = n - 1; j >= 0; --j) {
        if (parent[j] < 0) continue;
        next[j] = head[parent[j]];
        head[parent[j]] = j;
    }
    std::vector<int64_t> post;
    post.reserve(n);
    std::vector<int64_t> stack;
    for (int64_t r = 0; r < n; ++r) {
        if (parent[r] >= 0) continue;
        stack.push_back(r);
        while (!stack.empty()) {
            int64_t v = stack.back();
            if (head[v] >= 0) {
                int64_t c = head[v];
                head[v] = next[c];
                stack.push_back(c);
            } else {
                stack.pop_back();
                post.push_back(v);
            }
        }
    }
    return post;
}

inline double stored_entries(double w, double h) { return w * h - w * (w - 1.0) / 2.0; }

}  // namespace

// ---------------------------------------------------------------------------
// The analysis.
// ---------------------------------------------------------------------------
std::string analyze(int64_t n, const int64_t *colptr, const int32_t *rowind, int method,
                    const AnalyzeOptions &opt, Plan &P)
{
    auto t0 = std::chrono::steady_clock::now();
    if (n <= 0) return "n must be positive";
    if (n >= (int64_t)INT32_MAX) return "n must be below 2^31";
    if (colptr[0] != 0) return "colptr[0] must be 0";
    for (int64_t j = 0; j < n; ++j)
        if (colptr[j + 1] < colptr[j]) return "colptr must be non-decreasing";
    const int64_t nnz = colptr[n];
    for (int64_t p = 0; p < nnz; ++p)
        if (rowind[p] < 0 || rowind[p] >= n) return "row index out of range";
    {
        std::vector<int32_t> col;
        for (int64_t j = 0; j < n; ++j) {
            col.assign(rowind + colptr[j], rowind + colptr[j + 1]);
            std::sort(col.begin(), col.end());
            if (std::adjacent_find(col.begin(), col.end()) != col.end())
                return "duplicate entry in column " + std::to_string(j);
        }
    }
    if (opt.max_width < 1) return "max_width must be positive";

    P = Plan();
    P.n = n;
    P.method = method;
    P.lower_only = opt.lower_only;
    P.nnz_a = nnz;

    std::vector<int64_t> adjp;
    std::vector<int32_t> adji;
    build_adjacency(n, colptr, rowind, adjp, adji);

    // ---- ordering ----------------------------------------------------------
    int ordering = opt.ordering;
    if (ordering == 0) ordering = (opt.grid[0] > 0 && opt.grid[1] > 0) ? 1 : 2;
    std::vector<int64_t> perm;
    if (ordering == 1) {
        int nz = opt.grid[2] > 0 ? opt.grid[2] : 1;
        int dof = opt.dof > 0 ? opt.dof : 1;
        if ((int64_t)opt.grid[0] * opt.grid[1] * nz * dof != n) return "grid * dof does not match n";
        order_grid(opt.grid[0], opt.grid[1], nz, dof, perm);
    } else if (ordering == 2) {
        order_graph(n, adjp, adji, perm);
    } else if (ordering == 3) {
        if (!opt.perm) return "ordering GIVEN needs opt->perm";
        perm.assign(opt.perm, opt.perm + n);
    } else if (ordering == 4) {
        perm.resize(n);
        std::iota(perm.begin(), perm.end(), 0);
    } else {
        return "unknown ordering";
    }
    {
        std::vector<char> seen(n, 0);
        if ((int64_t)perm.size() != n) return "permutation has the wrong length";
        for (int64_t v : perm) {
            if (v < 0 || v >= n || seen[v]) return "permutation is not a permutation";
            seen[v] = 1;
        }
    }
    std::vector<int64_t> iperm(n);
    for (int64_t k = 0; k < n; ++k) iperm[perm[k]] = k;

    std::vector<int64_t> padjp;
    std::vector<int32_t> padji;
    permute_adjacency(n, adjp, adji, perm, iperm, padjp, padji);
    std::vector<int64_t> parent;
    elimination_tree(n, padjp, padji, parent);

    // ---- postorder (identity for nested-dissection orders) ----------------
    {
        std::vector<int64_t> post = postorder(n, parent);
        bool identity = true;
        for (int64_t k = 0; k < n && identity; ++k) identity = (post[k] == k);
        if (!identity) {
            std::vector<int64_t> perm2(n);
            for (int64_t k = 0; k < n; ++k) perm2[k] = perm[post[k]];
            perm.swap(perm2);
            for (int64_t k = 0; k < n; ++k) iperm[perm[k]] = k;
            permute_adjacency(n, adjp, adji, perm, iperm, padjp, padji);
            elimination_tree(n, padjp, padji, parent);
        }
    }

    // ---- fundamental supernodes with their row structure -------------------
    // Column j extends the supernode of column j-1 when j is the only child of
    // j-1's parent chain (parent(j-1) = j, one child) and column j of A below
    // the diagonal adds no row to the structure; otherwise a new supernode
    // starts with struct = {j} + rows of A below j + the rows of its child
    // supernodes beyond their last column.
    std::vector<int32_t> nchild(n, 0);
    for (int64_t j = 0; j < n; ++j)
        if (parent[j] >= 0) nchild[parent[j]]++;
    std::vector<int64_t> sfirst;             // first column per supernode
    std::vector<int64_t> srowp{0};           // row offsets
    std::vector<int32_t> srows;              // rows (sorted after finalize)
    std::vector<int64_t> mark(n, -1);
    std::vector<std::vector<int32_t>> child_sn(n);   // supernodes whose last column's parent is j
    int64_t cur = -1;
    auto finalize = [&](int64_t s, int64_t lastcol) {
        std::sort(srows.begin() + srowp[s], srows.end());
        srowp.push_back((int64_t)srows.size());
        int64_t p = parent[lastcol];
        if (p >= 0) child_sn[p].push_back((int32_t)s);
    };
    for (int64_t j = 0; j < n; ++j) {
        bool extend = false;
        if (cur >= 0 && parent[j - 1] == j && nchild[j] == 1) {
            extend = true;
            for (int64_t p = padjp[j]; p < padjp[j + 1]; ++p) {
                int64_t i = padji[p];
                if (i > j && mark[i] != cur) {
                    extend = false;
                    break;
                }
            }
        }
        if (extend) continue;
        if (cur >= 0) finalize(cur, j - 1);
        cur = (int64_t)sfirst.size();
        sfirst.push_back(j);
        mark[j] = cur;
        srows.push_back((int32_t)j);
        for (int64_t p = padjp[j]; p < padjp[j + 1]; ++p) {
            int64_t i = padji[p];
            if (i > j && mark[i] != cur) {
                mark[i] = cur;
                srows.push_back((int32_t)i);
            }
        }
        for (int32_t c : child_sn[j]) {
            int64_t clast = sfirst[c + 1] - 1;
            for (int64_t p = srowp[c]; p < srowp[c + 1]; ++p) {
                int64_t i = srows[p];
                if (i > clast && mark[i] != cur) {
                    mark[i] = cur;
                    srows.push_back((int32_t)i);
                }
            }
        }
        std::vector<int32_t>().swap(child_sn[j]);
    }
    finalize(cur, n - 1);
    const int64_t ns = (int64_t)sfirst.size();
    sfirst.push_back(n);
    P.nsuper = ns;

    // exact counts: column j of supernode s has h_s - (j - first_s) entries
    {
        double fl = 0.0;
        int64_t nnzl = 0;
        for (int64_t s = 0; s < ns; ++s) {
            int64_t h = srowp[s + 1] - srowp[s];
            for (int64_t j = sfirst[s]; j < sfirst[s + 1]; ++j) {
                double c = (double)(h - (j - sfirst[s]));
                nnzl += (int64_t)c;
                fl += (method == 0) ? c * c : 2.0 * (c - 1.0) * (c - 1.0) + (c - 1.0);
            }
        }
        P.nnz_l = nnzl;
        P.flops_exact = fl;
    }

    // ---- amalgamation (Sec. V: allow up to 12% extra fill) -----------------
    // A supernode may merge into the next one in column order when that one is
    // its parent; the merged structure is its own columns followed by the
    // parent's rows.  Merges are taken smallest added fill first while the
    // total of explicit zeros stays within amalg_ratio * nnz(L).
    std::vector<int64_t> s_parent(ns, -1);
    {
        std::vector<int64_t> col2sn(n);
        for (int64_t s = 0; s < ns; ++s)
            for (int64_t j = sfirst[s]; j < sfirst[s + 1]; ++j) col2sn[j] = s;
        for (int64_t s = 0; s < ns; ++s) {
            int64_t p = parent[sfirst[s + 1] - 1];
            s_parent[s] = p >= 0 ? col2sn[p] : -1;
        }
    }
    std::vector<int64_t> a_first(ns), a_w(ns), a_h(ns), prev(ns), next(ns), uf(ns), ver(ns, 0);
    std::vector<char> alive(ns, 1);
    for (int64_t s = 0; s < ns; ++s) {
        a_first[s] = sfirst[s];
        a_w[s] = sfirst[s + 1] - sfirst[s];
        a_h[s] = srowp[s + 1] - srowp[s];
        prev[s] = s - 1;
        next[s] = (s + 1 < ns) ? s + 1 : -1;
        uf[s] = s;
    }
    std::function<int64_t(int64_t)> find = [&](int64_t x) {
        int64_t r = x;
        while (uf[r] != r) r = uf[r];
        while (uf[x] != r) {
            int64_t t = uf[x];
            uf[x] = r;
            x = t;
        }
        return r;
    };
    // node x (alive, identified by its top supernode) can merge into next(x)
    auto merge_cost = [&](int64_t x, double *extra) -> bool {
        int64_t y = next[x];
        if (y < 0 || s_parent[x] < 0 || find(s_parent[x]) != y) return false;
        double w = (double)(a_w[x] + a_w[y]);
        double h = (double)(a_w[x] + a_h[y]);
        *extra = stored_entries(w, h) - stored_entries((double)a_w[x], (double)a_h[x]) -
                 stored_entries((double)a_w[y], (double)a_h[y]);
        return true;
    };
    double budget = std::max(0.0, opt.amalg_ratio) * (double)P.nnz_l;
    double used = 0.0;
    {
        typedef std::tuple<double, int64_t, int64_t, int64_t> Cand;  // extra, x, ver x, ver next
        std::priority_queue<Cand, std::vector<Cand>, std::greater<Cand>> heap;
        auto push = [&](int64_t x) {
            double e;
            if (x >= 0 && alive[x] && merge_cost(x, &e)) heap.emplace(e, x, ver[x], ver[next[x]]);
        };
        for (int64_t s = 0; s < ns; ++s) push(s);
        while (!heap.empty()) {
            auto [e, x, vx, vy] = heap.top();
            heap.pop();
            if (!alive[x] || ver[x] != vx || next[x] < 0 || ver[next[x]] != vy) continue;
            double e2;
            if (!merge_cost(x, &e2) || e2 != e) continue;
            if (used + e > budget) break;
            used += e;
            int64_t y = next[x];
            // x joins y: y keeps its identity (top), grows downward
            a_first[y] = a_first[x];
            a_h[y] = a_w[x] + a_h[y];
            a_w[y] = a_w[x] + a_w[y];
            alive[x] = 0;
            uf[x] = y;
            prev[y] = prev[x];
            if (prev[x] >= 0) next[prev[x]] = y;
            ver[y]++;
            push(y);
            if (prev[y] >= 0) {
                ver[prev[y]]++;
                push(prev[y]);
            }
        }
    }
    // s_parent of merged nodes: the parent of the top supernode
    // ---- splitting into panels (Sec. III: wide supernodes are split) ------
    const int maxw = opt.max_width;
    std::vector<int64_t> pfcol;
    std::vector<int32_t> pw, ph;
    std::vector<int64_t> prow{0};
    std::vector<int32_t> rows;
    int64_t nnz_stored = 0;
    double flops_stored = 0.0;
    for (int64_t y = 0; y < ns; ++y) {
        if (!alive[y]) continue;
        int64_t f = a_first[y], w = a_w[y];
        int64_t lastcol = f + w - 1;
        // rows below the supernode: rows of the top supernode beyond its columns
        std::vector<int32_t> below;
        for (int64_t p = srowp[y]; p < srowp[y + 1]; ++p)
            if (srows[p] > lastcol) below.push_back(srows[p]);
        for (int64_t c0 = f; c0 <= lastcol; c0 += maxw) {
            int64_t width = std::min<int64_t>(maxw, lastcol + 1 - c0);
            pfcol.push_back(c0);
            pw.push_back((int32_t)width);
            int64_t h = (lastcol + 1 - c0) + (int64_t)below.size();
            if (h >= (int64_t)INT32_MAX) return "panel too tall";
            ph.push_back((int32_t)h);
            for (int64_t r = c0; r <= lastcol; ++r) rows.push_back((int32_t)r);
            rows.insert(rows.end(), below.begin(), below.end());
            prow.push_back((int64_t)rows.size());
            nnz_stored += (int64_t)stored_entries((double)width, (double)h);
            for (int64_t j = 0; j < width; ++j) {
                double c = (double)(h - j);
                flops_stored += (method == 0) ? c * c : 2.0 * (c - 1.0) * (c - 1.0) + (c - 1.0);
            }
        }
    }
    const int32_t np = (int32_t)pfcol.size();
    P.npanels = np;
    P.nnz_stored = nnz_stored;
    P.flops_stored = flops_stored;
    std::vector<int32_t> col2panel(n);
    for (int32_t p = 0; p < np; ++p)
        for (int64_t j = pfcol[p]; j < pfcol[p] + pw[p]; ++j) col2panel[j] = p;

    std::vector<int64_t> pval(np + 1, 0);
    for (int32_t p = 0; p < np; ++p) pval[p + 1] = pval[p] + (int64_t)ph[p] * pw[p];

    // ---- panel tree and levels ---------------------------------------------
    std::vector<int32_t> pparent(np, -1), plevel(np, 0);
    for (int32_t p = 0; p < np; ++p)
        if (ph[p] > pw[p]) pparent[p] = col2panel[rows[prow[p] + pw[p]]];
    for (int32_t p = 0; p < np; ++p)
        if (pparent[p] >= 0) plevel[pparent[p]] = std::max(plevel[pparent[p]], plevel[p] + 1);
    int32_t nlev = 0;
    for (int32_t p = 0; p < np; ++p) nlev = std::max(nlev, plevel[p] + 1);
    std::vector<int32_t> level_ptr(nlev + 1, 0), level_panels(np);
    for (int32_t p = 0; p < np; ++p) level_ptr[plevel[p] + 1]++;
    for (int32_t l = 0; l < nlev; ++l) level_ptr[l + 1] += level_ptr[l];
    {
        std::vector<int32_t> fill(level_ptr.begin(), level_ptr.end() - 1);
        for (int32_t p = 0; p < np; ++p) level_panels[fill[plevel[p]]++] = p;
    }

    // position of global row r inside panel t's row list
    auto pos_in = [&](int32_t t, int32_t r) -> int64_t {
        int64_t lastcol = (int64_t)rows[prow[t] + ph[t] - 1];
        (void)lastcol;
        int64_t off = (int64_t)r - pfcol[t];
        int64_t w = pw[t];
        // columns of the diagonal block and the rest of the supernode are consecutive
        int64_t b = prow[t], e = prow[t + 1];
        if (off >= 0 && off < (e - b) && rows[b + off] == r) return off;
        (void)w;
        auto it = std::lower_bound(rows.begin() + b, rows.begin() + e, r);
        if (it == rows.begin() + e || *it != r) return -1;
        return (int64_t)(it - (rows.begin() + b));
    };

    // ---- update tasks (one per couple of panels) ---------------------------
    std::vector<Task> tasks;
    std::vector<int32_t> level_task_ptr(nlev + 1, 0);
    std::vector<int32_t> relmap;
    double upd = 0.0, upd_elems = 0.0;
    for (int32_t l = 0; l < nlev; ++l) {
        for (int32_t q = level_ptr[l]; q < level_ptr[l + 1]; ++q) {
            int32_t k = level_panels[q];
            int32_t h = ph[k], w = pw[k];
            int64_t b = prow[k];
            int32_t i = w;
            while (i < h) {
                int32_t t = col2panel[rows[b + i]];
                int32_t r1 = i;
                int64_t tend = pfcol[t] + pw[t];
                while (r1 < h && rows[b + r1] < tend) ++r1;
                Task tk;
                tk.src = k;
                tk.tgt = t;
                tk.r0 = i;
                tk.r1 = r1;
                tk.relmap_off = (int64_t)relmap.size();
                for (int32_t r = i; r < h; ++r) {
                    int64_t pp = pos_in(t, rows[b + r]);
                    if (pp < 0) return "internal error: source row missing from its target panel";
                    relmap.push_back((int32_t)pp);
                }
                double M = (double)(h - i), N = (double)(r1 - i), K = (double)w;
                upd += (method == 0) ? (2.0 * (M - N) * N * K + N * (N + 1.0) * K)
                                     : (2.0 * M * N * K + 2.0 * (M - N) * N * K);
                // operands read once, updated target entries read and written once
                upd_elems += (method == 0)
                                 ? (M + N) * K + 2.0 * ((M - N) * N + N * (N + 1.0) / 2.0)
                                 : (M + N) * K + (M - N + N) * K + 2.0 * (M * N + (M - N) * N);
                tasks.push_back(tk);
                i = r1;
            }
        }
        level_task_ptr[l + 1] = (int32_t)tasks.size();
    }
    P.update_flops = upd;
    P.update_elems = upd_elems;
    for (int32_t p = 0; p < np; ++p) {
        const double w = pw[p], off = (double)ph[p] - pw[p];
        for (int32_t j = 0; j < pw[p]; ++j) {
            const double c = w - j;
            P.diag_flops += (method == 0) ? c * c : 2.0 * (c - 1.0) * (c - 1.0) + (c - 1.0);
        }
        P.trsm_flops += (method == 0 ? 1.0 : 2.0) * off * w * w;
        P.diag_elems += 2.0 * w * w;
        P.trsm_elems += (method == 0 ? 1.0 : 2.0) * (2.0 * off * w + w * w);
    }

    // ---- assembly map --------------------------------------------------------
    std::vector<int64_t> amap(nnz, -1);
    for (int64_t j = 0; j < n; ++j) {
        int64_t pj = iperm[j];
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            int64_t pi = iperm[rowind[p]];
            int64_t row = pi, col = pj;
            bool upper = pi < pj;
            if (opt.lower_only) {
                // one stored entry stands for (i, j) and (j, i): keep it below the diagonal
                if (rowind[p] < j) return "lower_only input holds an upper-triangle entry";
                row = std::max(pi, pj);
                col = std::min(pi, pj);
                upper = false;
            } else if (upper && method == 0) {
                continue;  // the lower mirror carries the value
            }
            int32_t panel;
            bool to_u = false;
            if (upper) {
                // U(pi, pj): inside pj's diagonal block -> L panel, else U^T panel of pi
                int32_t pc = col2panel[pj];
                if (pi >= pfcol[pc]) {
                    panel = pc;
                } else {
                    panel = col2panel[pi];
                    row = pj;
                    col = pi;
                    to_u = true;
                }
            } else {
                panel = col2panel[col];
            }
            int64_t r = pos_in(panel, (int32_t)row);
            if (r < 0) return "internal error: matrix entry outside the symbolic structure";
            int64_t off = pval[panel] + (col - pfcol[panel]) * ph[panel] + r;
            amap[p] = to_u ? (-2 - off) : off;
        }
    }

    // ---- residual map: full matrix by rows, original numbering -------------
    {
        std::vector<int64_t> cnt(n + 1, 0);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
                cnt[rowind[p] + 1]++;
                if (opt.lower_only && rowind[p] != j) cnt[j + 1]++;
            }
        for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
        P.csr_ptr = cnt;
        P.csr_col.resize(cnt[n]);
        P.csr_src.resize(cnt[n]);
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
                int64_t i = rowind[p];
                P.csr_col[fill[i]] = (int32_t)j;
                P.csr_src[fill[i]++] = p;
                if (opt.lower_only && i != j) {
                    P.csr_col[fill[j]] = (int32_t)i;
                    P.csr_src[fill[j]++] = p;
                }
            }
    }

    P.perm = std::move(perm);
    P.iperm = std::move(iperm);
    P.pfcol = std::move(pfcol);
    P.pw = std::move(pw);
    P.ph = std::move(ph);
    P.prow = std::move(prow);
    P.rows = std::move(rows);
    P.pval = std::move(pval);
    P.pparent = std::move(pparent);
    P.plevel = std::move(plevel);
    P.col2panel = std::move(col2panel);
    P.nlevels = nlev;
    P.level_ptr = std::move(level_ptr);
    P.level_panels = std::move(level_panels);
    P.tasks = std::move(tasks);
    P.level_task_ptr = std::move(level_task_ptr);
    P.relmap = std::move(relmap);
    P.amap = std::move(amap);
    P.analyze_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return std::string();
}

}  // namespace spx
