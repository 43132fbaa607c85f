// batch_kernel.cuh -- device layout of the batched static-pivot LU.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace spx {

// Update task of one source panel: rows [r0, h) of the source are updated
// against its facing rows [r0, r1); relmap[relmap_off + i - r0] is the row of
// source row i inside the target panel.
struct BTask {
    int32_t tgt, r0, r1, relmap_off;
};

// One analysed pattern (shared by every system with that pattern).  All
// indices are local to the class; the pointers are into device arrays.
struct BClass {
    int32_t n, npanels, nlevels, nnz;
    int64_t nstored;              // stored elements of L (and of U^T)
    const int32_t *pfcol, *pw, *ph, *prow;
    const int64_t *pval;
    const int32_t *rows;
    const int32_t *task_ptr;      // npanels + 1, tasks grouped by source panel
    const BTask *tasks;
    const int32_t *relmap;
    const int64_t *amap;          // input entry -> >= 0: L offset; <= -2: U^T offset (-2 - v); -1: none
    const int32_t *csr_ptr, *csr_col, *csr_src;   // A by rows, original numbering
    const int32_t *perm, *iperm;  // new -> old, old -> new
    const int32_t *level_ptr, *level_panels;
};

struct BSys {
    int32_t cls, n;
    int64_t voff;                 // first input value
    int64_t foff;                 // first element of the system's L and U^T storage
    int64_t xoff;                 // first entry of its right-hand side / solution
};

struct BatchArgs {
    const BClass *cls;
    const BSys *sys;
    const int32_t *order;         // processing order (largest first)
    int32_t nsys;
    int32_t leaf_width;           // panels at most this wide are processed one per warp
    int32_t max_iter;             // refinement corrections after the first solve
    int32_t do_solve;
    double tol;                   // target backward error
    double tau_opt;               // < 0: sqrt(2^-52) ||A||_inf per system
    unsigned *queue;              // next position in `order` (zeroed before each launch)
    const double *vals;
    const double *B;
    double *X;
    void *L, *U;                  // T storage
    int32_t *iters, *converged, *nrepl;
    double *berr;
    int64_t *bad_col;             // first zero pivot per system (-1: none)
    unsigned *summary;            // [0]: systems not converged, [1]: systems with a zero pivot
};

constexpr int kBatchThreads = 256;
constexpr int kBatchMaxWidth = 64;    // widest panel of a batched system
constexpr int kBatchLeafMax = 16;     // widest panel one warp may take

size_t batch_smem_bytes(int elem_bytes, int n_max);
int batch_max_ctas_per_sm(int elem_bytes, int n_max, int rows_per_thread);
void launch_batch(const BatchArgs &a, int elem_bytes, int rows_per_thread, int grid, int n_max,
                  cudaStream_t s);

}  // namespace spx
