// spx_plan.h -- host-side result of the analysis (ordering, elimination
// tree, supernodes, panels, update tasks, maps).  Internal to libspx.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace spx {

// One (source panel, target panel) update task (Sec. III: "one update task
// per couple of panels").  Rows [r0, r1) of the source face the target's
// columns (the N side); rows [r0, h_src) are updated (the M side).
struct Task {
    int32_t src;
    int32_t tgt;
    int32_t r0;
    int32_t r1;
    int64_t relmap_off;  // relmap[relmap_off + (i - r0)] = target row of source row i
};

struct Plan {
    int64_t n = 0;
    int method = 0;             // spx_method
    int lower_only = 0;
    int64_t nnz_a = 0;

    std::vector<int64_t> perm;  // new -> old
    std::vector<int64_t> iperm; // old -> new

    // exact symbolic statistics (before amalgamation)
    int64_t nsuper = 0;
    int64_t nnz_l = 0;
    double flops_exact = 0.0;

    // panels after amalgamation and splitting, in column order
    int32_t npanels = 0;
    std::vector<int64_t> pfcol;   // first column
    std::vector<int32_t> pw;      // width
    std::vector<int32_t> ph;      // height (rows incl. diagonal block)
    std::vector<int64_t> prow;    // offsets into rows, npanels + 1
    std::vector<int32_t> rows;    // permuted row indices, sorted per panel
    std::vector<int64_t> pval;    // value offsets (column-major h x w), npanels + 1
    std::vector<int32_t> pparent; // panel elimination tree
    std::vector<int32_t> plevel;
    std::vector<int32_t> col2panel;

    int32_t nlevels = 0;
    std::vector<int32_t> level_ptr;     // nlevels + 1, into level_panels
    std::vector<int32_t> level_panels;  // panels by level, ascending index within a level

    std::vector<Task> tasks;            // grouped by level of the source
    std::vector<int32_t> level_task_ptr;// nlevels + 1
    std::vector<int32_t> relmap;

    // assembly: for each input entry, >= 0: offset in the L panels;
    // <= -2: offset (-2 - v) in the U^T panels (LU); -1: not stored.
    std::vector<int64_t> amap;

    // full matrix by rows in the ORIGINAL numbering, for residuals:
    // row i holds entries (csr_col[e], value input[csr_src[e]]).
    std::vector<int64_t> csr_ptr;
    std::vector<int32_t> csr_col;
    std::vector<int64_t> csr_src;

    int64_t nnz_stored = 0;
    double flops_stored = 0.0;
    double update_flops = 0.0;
    // algorithmic work per kernel class (flops; element traffic, x element size = bytes)
    double diag_flops = 0.0, trsm_flops = 0.0;
    double diag_elems = 0.0, trsm_elems = 0.0, update_elems = 0.0;
    double analyze_ms = 0.0;
};

struct AnalyzeOptions {
    int ordering = 0;
    int grid[3] = {0, 0, 0};
    int dof = 1;
    int max_width = 128;
    double amalg_ratio = 0.12;
    const int64_t *perm = nullptr;
    int lower_only = 0;
};

// Returns an empty string on success, else an error message.
std::string analyze(int64_t n, const int64_t *colptr, const int32_t *rowind, int method,
                    const AnalyzeOptions &opt, Plan &plan);

// Orderings (exposed for tests through the plan's permutation).
void order_grid(int nx, int ny, int nz, int dof, std::vector<int64_t> &perm);
void order_graph(int64_t n, const std::vector<int64_t> &adjp, const std::vector<int32_t> &adji,
                 std::vector<int64_t> &perm);

}  // namespace spx
