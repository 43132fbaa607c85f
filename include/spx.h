/*
 * spx.h -- C ABI of the GB300-native supernodal sparse direct solver.
 *
 * The operations follow the problem statement of Lacoste et al., "Taking
 * advantage of hybrid systems for sparse direct solvers via task-based
 * runtimes": solve A x = b by a supernodal Cholesky (L L^T) or static-pivot
 * LU factorization (Sec. III).  The analysis orders the unknowns by nested
 * dissection, builds the elimination tree and the block-symbolic structure of
 * the factor; the numerical factorization then processes, for every panel
 * (supernode), the factorization of its diagonal block, the triangular solve
 * of its off-diagonal blocks, and the updates of the facing panels (Sec. III,
 * the three steps of the 1D task), all on the GPU.
 *
 * Conventions for every call:
 *  - Indices are 0-based.  Matrices are CSC: colptr (int64, n+1 entries),
 *    rowind (int32, colptr[n] entries, sorted or not), values (double).
 *  - The caller owns every buffer it passes in and keeps ownership; the
 *    library copies what it needs.  A handle owns all host and device memory
 *    it allocates, released by spx_free.
 *  - Dense right-hand sides and solutions are column-major with a leading
 *    dimension >= n.
 *  - A call never aborts; it returns a status.  spx_last_error gives a
 *    message for the last failing call on a handle.  Calls on one handle are
 *    not thread-safe; different handles are independent.
 *  - `cuda_stream` is a cudaStream_t (NULL: the legacy default stream); all
 *    device work of a call is ordered on it, and a call returns after that
 *    work has completed.
 */
#ifndef SPX_H
#define SPX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spx_handle_s *spx_handle;

typedef enum {
    SPX_OK = 0,
    SPX_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad index) */
    SPX_ERR_ALLOC = 2,          /* host or device allocation failed */
    SPX_ERR_CUDA = 3,           /* a CUDA call failed, or no usable sm_103 device */
    SPX_ERR_NOT_SPD = 4,        /* Cholesky met a non-positive pivot (column in spx_info) */
    SPX_ERR_ZERO_PIVOT = 5,     /* LU met a zero pivot with static pivoting disabled */
    SPX_ERR_TIMEOUT = 6,        /* a bounded device wait expired */
    SPX_ERR_NOT_CONVERGED = 7,  /* refinement did not reach the requested backward error */
    SPX_ERR_STATE = 8           /* call out of order (e.g. solve before factorize) */
} spx_status;

/* SPX_LLT: Cholesky (SPD).  SPX_LU: static-pivot LU on the pattern of
 * A + A^T.  SPX_LDLT: symmetric indefinite L D L^T with static pivoting, unit
 * L; its updates compute C = C - L D L^T (Sec. V-B) from a stored D L^T
 * operand; panels at most 64 wide (max_width is clamped to 64). */
typedef enum { SPX_LLT = 0, SPX_LU = 1, SPX_LDLT = 2 } spx_method;

/* Arithmetic of the bulk panel updates.  SPX_FP64 stores and updates the
 * factor in double precision.  The other modes store the factor in single
 * precision and run the updates on the tensor cores (TF32 / BF16 operands
 * with FP32 accumulation; FP32 = three-pass split TF32), while the
 * diagonal-block factorizations, residuals and corrections stay in FP64. */
typedef enum { SPX_FP64 = 0, SPX_FP32 = 1, SPX_TF32 = 2, SPX_BF16 = 3 } spx_precision;

typedef enum {
    SPX_ORDER_AUTO = 0,     /* grid rule when grid[] is set, else graph rule */
    SPX_ORDER_GRID = 1,     /* geometric nested dissection of grid[0]*grid[1]*grid[2]*dof */
    SPX_ORDER_GRAPH = 2,    /* level-structure nested dissection of the graph of A + A^T */
    SPX_ORDER_GIVEN = 3,    /* use opt->perm */
    SPX_ORDER_NATURAL = 4   /* identity */
} spx_ordering;

typedef struct {
    int32_t ordering;       /* spx_ordering */
    int32_t grid[3];        /* nx, ny, nz for the grid rule (nz = 1 in 2-D) */
    int32_t dof;            /* unknowns per grid node (consecutive), >= 1 */
    int32_t max_width;      /* supernodes wider than this are split into panels (Sec. III); 0 = default 128 */
    double amalg_ratio;     /* amalgamation may add this fraction of nnz(L) as explicit zeros (Sec. V: 12%); <0 = default 0.12 */
    const int64_t *perm;    /* SPX_ORDER_GIVEN: new -> old permutation of length n (copied) */
    int32_t lower_only;     /* 1: the CSC holds only the lower triangle of a symmetric matrix (LLT only) */
    int32_t queue_panels;   /* levels of the panel tree run as one persistent launch over a device-side
                               task queue (Cholesky, LDL^T; panels at most 64 wide): > 0 = the top levels
                               holding at most this many panels; < 0 = none (every level launched on its
                               own); 0 = default: the whole tree for an FP64 factor, none for the
                               single-precision factors (the policy that measured fastest) */
    double pivot_tau;       /* LU static-pivot threshold; < 0 = sqrt(2^-52) * ||A||_inf at factorize */
    int32_t deterministic;  /* 1: bit-reproducible factors -- the updates of a level run in rounds, one
                               task per target panel per round in task order, so that every target
                               entry receives its contributions in a fixed order (every level launched
                               on its own; more launches); 0 (default): concurrent updates with atomic
                               reductions in whatever order they land */
    int32_t reserved1;
} spx_options;

/* Fill *opt with the defaults above. */
void spx_default_options(spx_options *opt);

typedef struct {
    int32_t max_iter;       /* plain iterative-refinement steps before GMRES-IR (default 10) */
    int32_t gmres_restart;  /* FGMRES restart length (default 30) */
    int32_t gmres_max_iter; /* total FGMRES iterations (default 200) */
    int32_t mode;           /* 0: no refinement; 1: plain refinement; 2: plain, then FGMRES on stall (default) */
    double tol;             /* target backward error (default 1e-12) */
} spx_refine;

void spx_default_refine(spx_refine *r);

typedef struct {
    int32_t iters;          /* plain refinement steps taken */
    int32_t gmres_iters;    /* FGMRES iterations taken */
    int32_t converged;      /* 1 if every column met tol (or no refinement was asked) */
    int32_t reserved0;
    double backward_error;  /* max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) */
} spx_solve_info;

typedef struct {
    int64_t n;
    int64_t nnz_a;          /* entries of the input CSC */
    int64_t nnz_l;          /* exact entries of L (diagonal included) from the symbolic factorization */
    int64_t nnz_stored;     /* lower entries kept in the panels after amalgamation */
    int64_t factor_bytes;   /* device bytes of the panel storage (L, or L and U) */
    int64_t nsupernodes;    /* fundamental supernodes */
    int64_t npanels;        /* panels after amalgamation and splitting */
    int64_t nlevels;        /* levels of the panel elimination tree */
    int64_t nupdates;       /* (source panel, target panel) update tasks */
    int64_t bad_col;        /* permuted column of the first failed pivot, or -1 */
    int64_t npivot_repl;    /* LU: static pivot replacements in the last factorization */
    int32_t method;         /* spx_method */
    int32_t precision;      /* spx_precision of the last factorization */
    double flops;           /* exact-pattern factorization flops: sum c_j^2 (LLT) or sum 2(c_j-1)^2+(c_j-1) (LU) */
    double flops_stored;    /* the same count on the amalgamated panel structure */
    double update_flops;    /* flops of the panel updates on the stored structure */
    int64_t launches_factor;/* kernels one spx_factorize launches */
    int64_t launches_solve; /* kernels the last spx_solve launched */
    double analyze_ms;      /* host time of spx_analyze */
    double factor_ms;       /* device time of the last spx_factorize (assembly included) */
    double solve_ms;        /* device time of the last spx_solve */
    int64_t npivot_neg;     /* LDL^T: negative pivots of the last factorization (the inertia, when
                               no pivot was replaced) */
    int64_t noalloc_timeout;/* 1 if the last spx_solve_noalloc whose work has completed had a sweep
                               wait give up (its X is then undefined), else 0 */
} spx_info;

/* Host-only analysis (Sec. III: ordering, elimination tree, symbolic
 * factorization, amalgamation (Sec. V, 12% extra fill) and splitting of wide
 * supernodes).  `colptr`/`rowind` are host arrays, copied; the pattern
 * used is that of A + A^T.  `opt` may be NULL (defaults).  Needs no GPU. */
spx_status spx_analyze(int64_t n, const int64_t *colptr, const int32_t *rowind, spx_method method,
                       const spx_options *opt, spx_handle *out);

/* Numerical factorization on the device (Sec. III: per panel, diagonal-block
 * factorization, panel TRSM, updates of the facing panels; Sec. V-B: the
 * update computes A_i A_j^T and subtracts it directly at the positions of the
 * target panel's block structure).  `values` are the CSC values in the order
 * of the analysed pattern, host or device memory (`values_on_device`).  May
 * be called again with new values.  Returns SPX_ERR_NOT_SPD (Cholesky in FP64)
 * or SPX_ERR_ZERO_PIVOT (LU / LDL^T without a replacement threshold) at a pivot
 * failure (spx_info.bad_col), and SPX_ERR_TIMEOUT when one of the bounded
 * device waits ran out: a tensor-core pipeline wait, a task-queue counter
 * (spx_set_wait_limit), or the hand-off between the two warps of a diagonal
 * block; the factor is then undefined and the handle stays usable. */
spx_status spx_factorize(spx_handle h, const double *values, int values_on_device,
                         spx_precision precision, void *cuda_stream);

/* Solve A X = B for nrhs columns.  B and X are host or device arrays
 * (`on_device`), column-major with leading dimensions ldb, ldx >= n; X may
 * equal B.  `refine` NULL: no refinement for FP64 factors, the defaults for
 * lower-precision factors.  `info` may be NULL.  Each forward or backward
 * sweep is one launch walking a device-side work queue whose waits are
 * bounded; SPX_ERR_TIMEOUT if one ran out (here or in an earlier
 * spx_solve_noalloc on the handle). */
spx_status spx_solve(spx_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X,
                     int64_t ldx, int on_device, const spx_refine *refine, spx_solve_info *info,
                     void *cuda_stream);

/* Statistics of the analysis and of the last factorization/solve. */
spx_status spx_get_info(spx_handle h, spx_info *info);

/* Bounded device waits of the triangular sweeps (spx_solve,
 * spx_solve_noalloc): a wait on a work-queue counter gives up after `polls`
 * polls of about 256 ns and the call returns SPX_ERR_TIMEOUT (spx_solve) or
 * records it (spx_solve_noalloc, see spx_info.noalloc_timeout); the
 * solution is then undefined and the handle stays usable.  polls = 0
 * restores the default, 2^22 (about a second), which only a stalled device
 * exhausts.  SPX_ERR_ARG for polls outside [0, 2^32). */
spx_status spx_set_wait_limit(spx_handle h, int64_t polls);

/* Copy the final permutation (new -> old, length n) to host memory. */
spx_status spx_get_perm(spx_handle h, int64_t *perm);

/* Copy the numerical factor to host arrays laid out on a caller-given CSC
 * pattern in the permuted numbering (Lp: n+1, Li: sorted rows, diagonal
 * first).  Lx receives L (LU: unit diagonal stored as 1); Ut, for LU only,
 * receives U transposed on the same pattern (Ut[p] = U(j, Li[p]) for p in
 * column j; may be NULL for LLT).  Every pattern entry must lie inside the
 * panel structure (SPX_ERR_ARG otherwise).  Values are converted to double. */
spx_status spx_get_factor(spx_handle h, const int64_t *Lp, const int32_t *Li, double *Lx,
                          double *Ut);

/* Copy the panel structure (host arrays of info.npanels entries; any may be
 * NULL): first column, width, height (rows of the panel including its
 * diagonal block), level in the panel elimination tree (leaves 0) and parent
 * panel (-1 for a root).  Panels are numbered in column order. */
spx_status spx_get_panels(spx_handle h, int64_t *first_col, int32_t *width, int32_t *height,
                          int32_t *level, int32_t *parent);

/* Allocation-free solve.  (The paper has no counterpart; this entry point
 * exists for callers that cannot allocate device memory when they solve:
 * a real-time loop, where a cudaMalloc would synchronize the device and
 * stall it, and hosts whose device memory belongs to another allocator that
 * must see every byte.)  It runs one forward
 * and one backward sweep through the factor of the last spx_factorize --
 * spx_solve without refinement -- and allocates nothing: no cudaMalloc,
 * cudaFree, graph or library call that allocates.
 *   B, X : device arrays, column-major, leading dimensions ldb, ldx >= n;
 *          X must not overlap B.
 *   The sweep vectors live in one file-scope device buffer of 16 MiB that
 *   every GPU loading the library holds until the process exits; the call
 *   needs 4 * n * nrhs elements of the factor's type (8 bytes for an FP64
 *   factor, 4 otherwise) plus 4 * npanels + 3 32-bit words (the sweep
 *   counters and the error word), and returns SPX_ERR_ARG when that exceeds
 *   16 MiB.
 *   The sweeps wait on device-side counters with a bounded wait
 *   (spx_set_wait_limit); the call's own error word, kept in the same
 *   buffer and zeroed at the start of each call, is copied to host memory
 *   the handle owns at the end of the call's work: once the caller has
 *   synchronized cuda_stream, spx_get_info's noalloc_timeout is 1 if a wait
 *   ran out (X is then undefined; only a stalled device or a tiny wait
 *   limit causes it) and 0 otherwise.
 *   All calls share that buffer and it keeps the previous call's contents:
 *   calls whose GPU work overlaps (other streams, other handles, other
 *   threads) race and must be ordered by the caller.
 *   The work is enqueued on cuda_stream and the call returns without
 *   waiting for it.  The current device must be the one the handle
 *   factorized on.  spx_factorize looks up the buffer's device address
 *   (cudaGetSymbolAddress, once per device), which also loads the module
 *   that holds the buffer, so this call only reads the cached address. */
spx_status spx_solve_noalloc(spx_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X,
                             int64_t ldx, void *cuda_stream);

/* ---- Differentiation: log-determinant, selected inverse, adjoints -------
 *
 * For a solve x = A^{-1} b with loss gradient g = dL/dx, the adjoint reuses
 * the stored factor: lambda = A^{-T} g (spx_solve on g; A is symmetric for
 * a Cholesky factor), dL/db = lambda and dL/dA = -lambda x^T, needed only on
 * A's pattern (spx_solve_grad).  For log det A = 2 sum_j log L(j,j)
 * (spx_logdet), d log det A / dA = A^{-T}, again only on A's pattern: the
 * selected inverse Z = (P A P^T)^{-1} on the structure of L (Takahashi's
 * recurrence, by panels from the root down, gathering the entries it needs
 * through the same row maps as the updates of Sec. V-B) gives it
 * (spx_selected_inverse, spx_logdet_grad).  Gradients are with respect to
 * the stored CSC values, each entry independent, in the analysed pattern's
 * order. */

/* log det A of the last Cholesky factorization (FP64 sum; an FP32 factor
 * gives an FP32-accurate value). */
spx_status spx_logdet(spx_handle h, double *logdet);

/* Selected inverse of the last Cholesky factorization, kept on the device;
 * needs an SPX_FP64 factor and panels at most 64 wide (max_width <= 64). */
spx_status spx_selected_inverse(spx_handle h, void *cuda_stream);

/* Entries of the selected inverse on a caller-given lower pattern of the
 * permuted matrix (Lp, Li as for spx_get_factor), into host Zx. */
spx_status spx_get_selected_inverse(spx_handle h, const int64_t *Lp, const int32_t *Li, double *Zx);

/* grad[e] = (A^{-1})_{ji} for every stored entry e = (i, j) of A (nnz
 * doubles, host or device per on_device); computes the selected inverse
 * first if needed. */
spx_status spx_logdet_grad(spx_handle h, double *grad, int on_device, void *cuda_stream);

/* grad[e] = -sum_r Lam(i, r) X(j, r) for every stored entry e = (i, j) of A:
 * the adjoint of X = A^{-1} B with respect to A's values, given Lam =
 * A^{-T} dL/dX.  Lam, X: n x nrhs column-major (ldl, ldx >= n); grad: nnz
 * doubles; all host or all device per on_device. */
spx_status spx_solve_grad(spx_handle h, int32_t nrhs, const double *Lam, int64_t ldl, const double *X,
                          int64_t ldx, double *grad, int on_device, void *cuda_stream);

/* Message for the last failing call on h (or on handle creation when h is
 * NULL).  The string stays valid until the next call on h. */
const char *spx_last_error(spx_handle h);

/* Kernel classes of the factorization, for spx_kernel_stats. */
enum {
    SPX_K_ASSEMBLE = 0,   /* zeroing and scattering A into the panels, ||A||_inf */
    SPX_K_DIAG = 1,       /* diagonal-block POTRF / GETRF */
    SPX_K_TRSM = 2,       /* panel triangular solves */
    SPX_K_UPDATE = 3,     /* supernodal updates with fused scatter, CUDA cores */
    SPX_K_UPDATE_TC = 4,  /* supernodal updates with fused scatter, tensor cores (tcgen05) */
    SPX_K_QUEUE = 5,      /* the upper levels' persistent task-queue launch (all three steps) */
    SPX_K_CLASSES = 6
};

typedef struct {
    double ms[SPX_K_CLASSES];       /* device time per class in the last profiled factorization */
    int64_t launches[SPX_K_CLASSES];/* kernel launches per class */
    double flops[SPX_K_CLASSES];    /* algorithmic flops per class on the stored structure */
    double bytes[SPX_K_CLASSES];    /* algorithmic bytes per class (operands read once, targets read and written once) */
} spx_kernel_stats;

/* on = 1: the next factorizations run launch by launch (no graph) with CUDA
 * events around every kernel class of every level, on the library's stream,
 * and spx_get_kernel_stats reports the accumulated per-class device time.
 * The work of the levels in the task queue is counted in SPX_K_QUEUE. */
spx_status spx_set_profiling(spx_handle h, int on);
spx_status spx_get_kernel_stats(spx_handle h, spx_kernel_stats *out);

/* Roofline model of the factorization's work on the analysed structure:
 * for every task of each kernel class (a panel's diagonal block, a panel's
 * TRSM, an update task, the assembly), the time it takes at the better of
 * its two bounds, max(flops / compute peak, bytes / bandwidth), with the
 * algorithmic flops and bytes spx_get_kernel_stats uses, summed per class
 * into model_ms[SPX_K_CLASSES] (milliseconds).  Update tasks go to the engine
 * spx_factorize would use in `precision`.  peaks[4]: HBM GB/s, FP64 GFLOP/s
 * (the diagonal blocks always), FP32 CUDA-core GFLOP/s, tensor-core GFLOP/s
 * of the mode's operand type.  Sum over the classes / measured factorization
 * time = the fraction of the roofline model the factorization reaches. */
spx_status spx_roofline_model(spx_handle h, spx_precision precision, const double *peaks,
                              double *model_ms);

/* Release a handle and everything it owns.  NULL-safe. */
void spx_free(spx_handle h);

/* ---- Subtree-to-rank distribution with fan-in (Sec. VI) ------------------
 *
 * The paper's future work distributes the elimination tree's bottom
 * subtrees over GPUs and accumulates their contributions to the top
 * separators before those are factored (fan-in).  spx_partition maps whole
 * subtrees of the panel tree to nranks ranks, balancing their flops within
 * 5% where the tree allows; the panels above them (the top) belong to rank
 * 0.  Every update task then stays inside one rank's subtrees or goes from
 * them into the top, so one sum over the ranks of their top panels is the
 * whole exchange.  A distributed factorization, one handle per rank on the
 * same pattern:
 *   every rank r: spx_partition, spx_factorize_part(h, values, ..., r) --
 *                 rank r's subtrees factored, their updates subtracted into
 *                 its copy of the top panels, which holds A's values on rank
 *                 0 and zeros on the other ranks;
 *                 spx_part_get(h, -1, 0, buf): its top panel values;
 *   sum the buffers onto rank 0 (e.g. an NCCL or gloo reduce);
 *   rank 0:       spx_part_set(h, -1, 0, sum); spx_factorize_part(h, NULL, ..., -1)
 *                 factors the top.  For a solve on rank 0, copy each other
 *                 rank's part in (spx_part_get / spx_part_set with inverses).
 * Cholesky and LDL^T, panels at most 64 wide; every part runs on the
 * device-side task queue.  Calls return after their device work completed. */

/* Partition for nranks ranks.  panel_owner (host int32[npanels], or NULL):
 * the rank owning each panel, -1 for the top.  part_values, part_inverses
 * (host int64[nranks + 1], or NULL): elements of the factor's type in the
 * packed values and inverse blocks of each part (index nranks: the top).
 * SPX_ERR_ARG for LU, panels wider than 64, or nranks outside [1, 4096]. */
spx_status spx_partition(spx_handle h, int32_t nranks, int32_t *panel_owner, int64_t *part_values,
                         int64_t *part_inverses);

/* part = r in [0, nranks): factor rank r's subtrees (values as for
 * spx_factorize); part = -1: factor the top panels of this handle (after
 * its own part and spx_part_set of the summed top values; `values` is not
 * read).  After the top the handle reports a complete factor: a solve needs
 * every other rank's part copied in first. */
spx_status spx_factorize_part(spx_handle h, const double *values, int values_on_device,
                              spx_precision precision, int32_t part, void *cuda_stream);

/* Copy the panel values (and, with_inverses = 1, then the inverted diagonal
 * blocks) of part `part` (-1: the top) between the handle's factor and a
 * packed device buffer `buf` of the factor's type (sizes from spx_partition). */
spx_status spx_part_get(spx_handle h, int32_t part, int32_t with_inverses, void *buf, void *cuda_stream);
spx_status spx_part_set(spx_handle h, int32_t part, int32_t with_inverses, const void *buf,
                        void *cuda_stream);

/* ---- The supernodal update on its own (the kernel study of Sec. V-B) ------
 *
 * C = C - A B^T, where A (m x k) holds the rows of a source panel, B is its
 * first nb_rows rows (the rows facing the target's columns, as in the
 * Cholesky update) and C is a target panel (ldc x nc, column-major) whose
 * rows are cut into blocks.  Row i of A lands on row rowmap[i] of C and row
 * j of B on column colmap[j]; each block of A lies inside one block of C, so
 * the product is subtracted directly at those positions with no temporary
 * buffer (Sec. V-B).  A plan describes this single (source, target) task
 * exactly as the analysis describes one of the factorization's tasks;
 * spx_update_stage stores A the way the factorization stores a panel
 * (column-major, plus for the tensor cores the rounded K-major operand copy
 * the panel TRSM writes); spx_update_run launches the factorization's own
 * update kernels over the task's tiles -- update_kernel on the CUDA cores or
 * update_tc_kernel on the tcgen05 tensor cores -- with the factorization's
 * tile rules.  Entries are subtracted with atomic adds.
 *
 *   precision : SPX_FP64: A, W and C are double.  Otherwise they are float
 *               (the mixed factor's storage) and the products use the mode's
 *               arithmetic: SPX_FP32 = FP32 on the CUDA cores or split TF32
 *               (hi*hi + hi*lo + lo*hi) on the tensor cores; SPX_TF32 / SPX_BF16
 *               = TF32 / BF16 operands; FP32 accumulation throughout.
 *   engine    : 0 = the factorization's choice (tensor cores for the single-
 *               precision modes when k >= 32, except LDL^T in SPX_FP32; CUDA
 *               cores otherwise); 1 = CUDA cores; 2 = tensor cores (SPX_ERR_ARG
 *               for SPX_FP64 and for LDL^T in SPX_FP32).
 *   ldlt      : 1 = the LDL^T update C = C - L (D L^T)^T (Sec. V-B): A holds
 *               rows of L and W (spx_update_stage) the same rows of D L^T; B is
 *               the first nb_rows rows of W.
 *   lower     : 1 = only entries with source row index i >= facing row index j
 *               (the diagonal-block region of a Cholesky target).
 *   rowmap    : host int32[m], entries in [0, ldc); colmap: host int32[nb_rows],
 *               entries in [0, nc); both copied.  SPX_ERR_ARG otherwise.
 * The plan owns its device copies; the caller owns A, W and C. */
typedef struct spx_update_s *spx_update_plan;

spx_status spx_update_create(int64_t m, int64_t nb_rows, int64_t k, int64_t ldc, int64_t nc,
                             const int32_t *rowmap, const int32_t *colmap, int lower,
                             spx_precision precision, int engine, int ldlt, spx_update_plan *out);

/* Stage the source panel: A (and W for LDL^T) are device arrays, column-
 * major m x k with leading dimension lda >= m, of the plan's element type.
 * Returns after the staging has completed on cuda_stream. */
spx_status spx_update_stage(spx_update_plan u, const void *A, const void *W, int64_t lda,
                            void *cuda_stream);

/* C -= A B^T on the device array C (ldc x nc, the plan's element type).
 * wait = 0: enqueue on cuda_stream and return (repeated calls accumulate);
 * wait = 1: also wait for completion and report SPX_ERR_TIMEOUT if a bounded
 * wait of the tensor-core pipeline expired. */
spx_status spx_update_run(spx_update_plan u, void *C, int wait, void *cuda_stream);

/* Engine in use (1 CUDA cores, 2 tensor cores) and output tiles per run. */
spx_status spx_update_get_info(spx_update_plan u, int32_t *engine, int64_t *tiles);

/* Message for the last failing call on u (or on plan creation when u is NULL). */
const char *spx_update_last_error(spx_update_plan u);

/* Release a plan.  NULL-safe. */
void spx_update_free(spx_update_plan u);

/* ---- Batched static-pivot LU of many small independent systems ----------
 *
 * The factorization of Sec. III (static pivoting, panels, updates with the
 * scatter fused as in Sec. V-B) applied to a batch of unrelated systems, for
 * workloads of thousands of small systems where one system cannot fill the
 * GPU.  Each system has its own CSC pattern, values and one right-hand side;
 * systems with identical patterns (and grid) share one analysis.  One
 * persistent kernel, captured in a CUDA graph, factorizes every system and
 * solves it with FP64 iterative refinement: each CTA takes whole systems
 * from a device queue, largest first, so no CTA waits on another.
 *
 * Batched arrays are concatenations over the systems in order:
 *   colptr : n_s + 1 entries per system, each starting at 0 (int64);
 *   rowind, values : colptr_s[n_s] entries per system;
 *   B, X   : n_s entries per system (one right-hand side each). */
typedef struct spx_batch_s *spx_batch;

typedef struct {
    int32_t nsys;           /* systems */
    int32_t nclasses;       /* distinct patterns analysed */
    int64_t n_total;        /* sum of n */
    int64_t n_max;          /* largest n */
    int64_t nnz_total;      /* sum of nnz(A) */
    int64_t nnz_l_total;    /* sum of exact nnz(L) (diagonal included) */
    int64_t factor_elems;   /* stored elements of L plus U^T over all systems */
    double flops;           /* exact-pattern LU flops over all systems: sum 2(c_j-1)^2+(c_j-1) */
    int32_t precision;      /* spx_precision of the last run */
    int32_t ctas_per_sm;    /* launch configuration in use ... */
    int32_t leaf_width;     /* panels at most this wide go one per warp (0: none) */
    int32_t rows_per_thread;/* rows of the update tile per thread (1, 2 or 4) */
    double tuned_ms;        /* run time of the configuration spx_batch_tune chose (0: not tuned) */
    double analyze_ms;      /* host time of spx_batch_analyze */
    double run_ms;          /* device time of the last spx_batch_run (the persistent launch) */
    int64_t max_pivot_repl; /* largest number of static pivot replacements in one system */
    int32_t not_converged;  /* systems of the last run that missed the target */
    int32_t max_iters;      /* most refinement steps one system took */
    double max_backward_error;  /* largest final backward error over the systems */
} spx_batch_info;

/* Host-only analysis of a batch.  n: host int64[nsys]; colptr, rowind: host
 * concatenations as above (copied).  grid: NULL, or host int32[3 * nsys]
 * (nx, ny, nz per system) for the grid ordering rule.  opt: NULL or options
 * (ordering, dof, amalg_ratio, pivot_tau, max_width <= 64; perm and
 * lower_only are not allowed).  Every system is analysed for LU on the
 * pattern of A + A^T. */
spx_status spx_batch_analyze(int32_t nsys, const int64_t *n, const int64_t *colptr,
                             const int32_t *rowind, const int32_t *grid, const spx_options *opt,
                             spx_batch *out);

/* Factorize every system and solve it, in one persistent launch.
 *   values : concatenated CSC values; B, X: concatenated right-hand sides and
 *            solutions; host memory (on_device = 0: copied in and out inside
 *            the call) or device memory (on_device = 1).  B == NULL:
 *            factorize only (X untouched).
 *   precision : SPX_FP64 or SPX_FP32, the arithmetic of the stored factor,
 *            the panel updates and the sweeps; residuals b - A x and the
 *            corrections x += d are FP64.
 *   refine : NULL or mode 0: one solve; else up to max_iter corrections per
 *            system, stopping at backward error <= tol.
 * Returns SPX_ERR_ZERO_PIVOT if a system met a zero pivot with pivot_tau = 0,
 * SPX_ERR_NOT_CONVERGED if refinement was asked and a system missed tol;
 * spx_batch_system_info tells which. */
spx_status spx_batch_run(spx_batch b, const double *values, const double *B, double *X,
                         int on_device, spx_precision precision, const spx_refine *refine,
                         void *cuda_stream);

/* Autotuner: runs spx_batch_run on these arguments for candidate launch
 * configurations -- panels per warp up to width 0/4/8/16 (the leaf-versus-
 * top schedule), 1/2/4 update rows per thread (the update tile), CTAs per SM
 * -- times each with CUDA events and keeps the fastest for later runs.  X
 * holds a valid result afterwards. */
spx_status spx_batch_tune(spx_batch b, const double *values, const double *B, double *X,
                          int on_device, spx_precision precision, const spx_refine *refine,
                          void *cuda_stream);

/* Set the launch configuration by hand (0 keeps the current value of
 * ctas_per_sm / rows_per_thread; leaf_width 0 disables the per-warp mode). */
spx_status spx_batch_set_config(spx_batch b, int32_t ctas_per_sm, int32_t leaf_width,
                                int32_t rows_per_thread);

spx_status spx_batch_get_info(spx_batch b, spx_batch_info *info);

/* Per-system results of the last run, host arrays of nsys entries (any may
 * be NULL): refinement steps, final backward error, 1 if it met tol, static
 * pivot replacements, permuted column of the first zero pivot (-1: none). */
spx_status spx_batch_system_info(spx_batch b, int32_t *iters, double *berr, int32_t *converged,
                                 int32_t *npivot_repl, int64_t *bad_col);

/* Ordering (new -> old) of system s, host int64[n_s]. */
spx_status spx_batch_get_perm(spx_batch b, int32_t s, int64_t *perm);

/* Factor of system s on a caller-given lower pattern (Lp, Li; CSC of the
 * permuted matrix, as spx_get_factor): Lx (unit diagonal) and Ut = U^T. */
spx_status spx_batch_get_factor(spx_batch b, int32_t s, const int64_t *Lp, const int32_t *Li,
                                double *Lx, double *Ut);

const char *spx_batch_last_error(spx_batch b);

/* Release a batch handle.  NULL-safe. */
void spx_batch_free(spx_batch b);

#ifdef __cplusplus
}
#endif

#endif /* SPX_H */
