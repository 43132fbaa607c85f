// kernels.cuh -- device-side data layout and kernel launchers of libspx.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace spx {

// Structure of the panels on the device (uploaded once after the analysis).
struct DevPlan {
    int64_t n;
    int32_t npanels;
    const int64_t *pfcol;   // first column per panel
    const int32_t *pw;      // width
    const int32_t *ph;      // height (rows incl. diagonal block); leading dimension
    const int64_t *prow;    // row-list offsets
    const int32_t *rows;    // permuted row indices
    const int64_t *pval;    // value offsets
    const int64_t *pinv;    // offsets of the inverted diagonal blocks (w x w, column-major)
    const int32_t *relmap;  // target row of each updated source row, per task
};

struct DevTask {
    int32_t src, tgt, r0, r1;
    int64_t relmap_off;
};

// A tile of one update task: rows [m0, m0+64) x columns [n0, n0+64) in the
// source panel's local row numbering, or (narrow tiles, for tasks facing at
// most 16 rows) rows [m0, m0+256) x columns [n0, n0+16).
struct UpdTile {
    int32_t task, m0, n0, pad;
};

// A 128 x 128 tensor-core tile of one update task: source rows [m0, m0+128)
// against facing rows [n0, n0+128).
struct TcTile {
    int32_t task, m0, n0, pad;
};

// A chunk of rows [r0, r0+64) of one panel for the TRSM / solve kernels.
struct RowChunk {
    int32_t panel, r0;
};

constexpr int kMaxWidth = 160;      // widest panel the diagonal-block kernels keep in shared memory
constexpr int kUpdTile = 64;
constexpr int kUpdNarrowN = 16;   // tasks facing at most this many rows take 256 x 16 tiles
constexpr int kTrsmRows = 64;

// TRSM variants on the off-diagonal rows X of a panel (diagonal block D):
enum TrsmMode : int {
    TRSM_LLT = 0,        // X <- X L^{-T}, L = lower(D)            (Cholesky)
    TRSM_LU_L = 1,       // X <- X U^{-1}, U = upper(D)            (LU, L panel)
    TRSM_LU_U = 2,       // X <- X L^{-T}, L = unit lower(D)       (LU, U^T panel)
    TRSM_RIGHT_LINV = 3, // X <- X L^{-1}, L = lower(D)            (selected inversion)
    TRSM_LDLT = 4        // W = X l^{-T} (unit l) to Wout, X <- W D^{-1}   (LDL^T)
};

// The largest shared-memory carveout, for the solve-sweep kernels (their
// occupancy is set by shared memory; the factorization kernels are faster
// with the default split).
template <typename F>
inline bool set_max_carveout(F *kernel)
{
    cudaFuncSetAttribute(reinterpret_cast<const void *>(kernel), cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    return true;
}

// ---- factorization -------------------------------------------------------
template <typename T>
void launch_assemble(int64_t nnz, const double *vals, const int64_t *amap, T *L, T *U,
                     cudaStream_t s);

// ranges[3 r ..]: (storage offset, length, packed offset); mode 0 pack, 1 unpack, 2 zero
template <typename T>
void launch_pack_ranges(const int64_t *ranges, int nr, T *store, T *buf, int mode, cudaStream_t s);

template <typename T>
void launch_potrf(const DevPlan &p, const int32_t *panels, int count, int wmax, int threads, T *L, T *Dinv,
                  const double *replace_tau, int64_t *err_col, unsigned long long *nrepl,
                  cudaStream_t s);

template <typename T>
void launch_getrf(const DevPlan &p, const int32_t *panels, int count, int wmax, int threads, T *L, T *Dinv,
                  const double *tau, int64_t *err_col, unsigned long long *nrepl, cudaStream_t s);

// opc (may be null): K-major operand copy for the tensor-core updates, rows
// at prow[panel] + r with kpad elements each.  op_kind 0: TF32-rounded FP32;
// 1: BF16; 2: split TF32, hi = tf32(x) in opc and lo = tf32(x - hi) in opc_lo.
// op_kind 3 / 4 (LDL^T): TF32 / BF16 copies of L in opc and of D L^T in
// opc_lo.  Wout: the D L^T rows in the factor's type (TRSM_LDLT only).
template <typename T>
void launch_trsm(const DevPlan &p, const RowChunk *chunks, int count, int wmax, const T *Dinv,
                 T *X, int mode, void *opc, void *opc_lo, int kpad, int op_kind, cudaStream_t s,
                 T *Wout = nullptr);

// Chain-link look-ahead step: chunk 0 of panel ch.panel's TRSM and the
// update of the next panel's diagonal block by it (task `task`).
template <typename T>
void launch_lead(const DevPlan &p, RowChunk ch, const DevTask *tasks, int32_t task, const T *Dinv, T *L,
                 void *opc, void *opc_lo, int kpad, int op_kind, cudaStream_t s);


// LDL^T diagonal blocks, panels at most 64 wide (factor.cu): l with d on the
// diagonal, l^{-1} with 1/d on its diagonal at Dinv; static pivoting with
// threshold *tau; negative pivots counted in *nneg.
template <typename T>
void launch_ldlt_diag(const DevPlan &p, const int32_t *panels, int count, int wmax, T *L, T *Dinv,
                      const double *tau, int64_t *err_col, unsigned long long *nrepl,
                      unsigned long long *nneg, cudaStream_t s);

// Tensor-core update (update_tc.cu).  tmap / tmap_lo: CUtensorMaps over the
// operand copies (make_operand_map; tmap_lo is used for kind 2 only); err
// receives 1 if a bounded wait expired.
size_t tc_smem_bytes(int kind);
int make_operand_map(void *tmap_out, void *base, int64_t rows, int kpad, int bf16);
void launch_update_tc(const void *tmap, const void *tmap_lo, int kind, const DevPlan &p,
                      const DevTask *tasks, const TcTile *tiles, int count, float *C, int lower,
                      int *err, cudaStream_t s);

template <typename T>
void launch_update(const DevPlan &p, const DevTask *tasks, const UpdTile *tiles, int count,
                   const T *Aop, const T *Bop, T *C, int lower, int from_r1, cudaStream_t s, int narrow = 0);

// Operand copy of a column-major m x k panel A (ld lda; W: the D L^T rows
// for op_kinds 3 / 4, same layout) into rows [0, m) of opc / opc_lo, kpad
// elements per row, zero past k (kernel study; the factorization's TRSM
// writes the same copy, operand.cuh).
template <typename T>
void launch_stage_operand(int64_t m, int k, const T *A, const T *W, int64_t lda, void *opc, void *opc_lo,
                          int kpad, int op_kind, cudaStream_t s);

// ---- persistent task queue of the upper levels (fqueue.cu) ----------------
// Items: a panel's diagonal block, a 64-row TRSM chunk, an update tile on the
// tensor cores or on the CUDA cores (64 x 64, or 256 x 16 for tasks facing
// at most 16 rows), listed so that every item's inputs come from earlier items.
enum FqKind : int32_t { FQ_DIAG = 0, FQ_TRSM = 1, FQ_TC = 2, FQ_UPD64 = 3, FQ_UPD16 = 4 };
struct FqItem {
    int32_t kind;
    int32_t idx;   // panel (DIAG), chunk (TRSM), tile (TC: tensor-core tile list; UPD: CUDA-core tile list)
};
struct FactorQueue {
    const FqItem *items;
    int32_t nitems;
    const int32_t *need;       // per panel: update tiles of the queue that target it
    const int32_t *pchunk;     // per panel: index of its first TRSM chunk in the chunk list
    int32_t *cnt;              // per panel: finished update tiles into it
    int32_t *diag_done;        // per panel: 1 once its diagonal block is factored
    int32_t *chunk_done;       // per chunk: 1 once its TRSM is done
    int32_t *head;             // next item to hand out
    int32_t *err;              // 1 when a counter wait gave up, 2 when a tensor-core pipeline wait did
    uint32_t spin_limit;       // polls of ~256 ns before a counter wait gives up
};
// The counters cnt, diag_done, chunk_done, head and err are zeroed before
// each launch.  T: factor storage; ldlt: LDL^T diagonal blocks and the
// D L^T operand W; tc_kind: operand kind of the tensor-core tiles (-1: none).
template <typename T>
void launch_factor_queue(const DevPlan &p, const FactorQueue &q, const DevTask *tasks, const RowChunk *chunks,
                         const UpdTile *tiles, const TcTile *tctiles, T *L, T *Dinv, T *W, const double *tau,
                         int64_t *err_col, unsigned long long *nrepl, unsigned long long *nneg, int ldlt,
                         int tc_kind, const void *tmap, const void *tmap_lo, void *opc, void *opc_lo, int kpad,
                         int op_kind, cudaStream_t s);
// Resident CTAs of the queue kernel on the current device (its grid size).
template <typename T>
int factor_queue_grid(int ldlt, int tc_kind);

// ---- solves ----------------------------------------------------------------
// Vectors in the permuted numbering are of the factor's type T, column-major
// n x nrhs.  Forward: Z_p = D_p^{-1} Y_p, then Y(rows below) -= L_off Z_p.
// Backward: T_p += L_off^T X(rows below) (split over row chunks), then
// X_p = D_p^{-T} (Z_p - T_p)  (LU: U_p^{-1} (Z_p - T_p) with the U^T panel).
// Each direction is one launch over a work queue (sweep.cu).
template <typename T>
void launch_permute_in(int64_t n, int nrhs, const double *B, int64_t ldb, const int64_t *perm,
                       T *Y, cudaStream_t s);
template <typename T>
void launch_permute_out(int64_t n, int nrhs, const T *Y, const int64_t *perm, double *X,
                        int64_t ldx, cudaStream_t s);
// Device-resident work queue of one sweep direction (sweep.cu).  items[]:
// >= 0 a row chunk (index into the chunk list), < 0 panel -(item + 1), in
// an order where every item's inputs come from earlier items.  cnt, flag
// and head are zeroed before each sweep; err is set when a wait runs out.
struct SweepQueue {
    const int32_t *items;
    int32_t nitems;
    const int32_t *tptr, *tgt;   // per chunk: the distinct panels owning its rows
    const int32_t *need;         // per panel: counts its panel item waits for
    const int32_t *merge;        // per panel: its first chunk when the panel item takes it along, else -1
    int32_t *cnt, *flag, *head;
    int32_t *err;
    int32_t mat_elems, matb_elems, vec_elems;   // shared-memory staging, elements of T (matb_elems 0: no chunks taken along)
    uint32_t spin_limit;                        // polls of ~256 ns before a wait gives up
};
constexpr uint32_t kDefaultSpinLimit = 1u << 22;   // about a second
template <typename T>
void launch_fwd_queue(const DevPlan &p, const SweepQueue &q, const RowChunk *chunks, const T *Dinv,
                      int unit, const T *L, T *Y, T *Z, int nrhs, cudaStream_t s);
template <typename T>
void launch_bwd_queue(const DevPlan &p, const SweepQueue &q, const RowChunk *chunks, const T *Dinv,
                      int lu, const T *Lop, const T *Z, T *Tacc, T *X, int nrhs, cudaStream_t s);

// ---- FGMRES vector kernels (FP64, n x nrhs column blocks, ld n) ----------
void launch_spmv_cols(int64_t n, int nrhs, const int64_t *rp, const int32_t *ci, const int64_t *src,
                      const double *vals, const double *X, double *Y, cudaStream_t s);
// out[v * nrhs + c] = <V_v(:, c), w(:, c)> for v < nv (out zeroed inside)
void launch_dots(int64_t n, int nrhs, int nv, const double *V, const double *w, double *out,
                 cudaStream_t s);
// w(:, c) += sign * sum_v coef[v * nrhs + c] V_v(:, c)
void launch_combine(int64_t n, int nrhs, int nv, const double *V, const double *coef, double sign,
                    double *w, cudaStream_t s);
// v(:, c) = w(:, c) * sc[c]
void launch_scale_cols(int64_t n, int nrhs, const double *w, const double *sc, double *v, cudaStream_t s);

// ---- residuals and norms ---------------------------------------------------
// R = B - A X for nrhs columns (A by rows, original numbering); per column
// stores max|r|, max|x|, max|b| into norms[3*c + {0,1,2}] (bit patterns of
// non-negative doubles, combined with atomicMax).
void launch_residual(int64_t n, int nrhs, const int64_t *rp, const int32_t *ci,
                     const int64_t *src, const double *vals, const double *X, int64_t ldx,
                     const double *B, int64_t ldb, double *R, unsigned long long *norms,
                     cudaStream_t s);
void launch_row_abs_sum_max(int64_t n, const int64_t *rp, const int64_t *src, const double *vals,
                            unsigned long long *out, cudaStream_t s);
void launch_axpy_cols(int64_t n, int nrhs, const double *D, double *X, int64_t ldx,
                      cudaStream_t s);

// ---- selected inversion, log-determinant, adjoints (selinv.cu) ----------
// row_task[prow[p] + r]: the update task of panel p whose facing rows hold
// row r (r >= width of p)
void launch_selinv_off(const DevPlan &p, const RowChunk *chunks, int count, int nsplit,
                       const int32_t *row_task, const DevTask *tasks, const double *Lh, double *Z,
                       cudaStream_t s);
void launch_selinv_diag(const DevPlan &p, const int32_t *panels, int count, int nsplit, int wmax,
                        const double *Dinv, const double *Lh, double *Z, cudaStream_t s);
template <typename T>
void launch_logdet(const DevPlan &p, const T *L, double *out, cudaStream_t s);
void launch_gather(int64_t nnz, const int64_t *zmap, const double *Z, double *grad, cudaStream_t s);
void launch_solve_grad(int64_t n, int nrhs, const int64_t *rp, const int32_t *ci, const int64_t *src,
                       const double *Lam, int64_t ldl, const double *X, int64_t ldx, double *grad,
                       cudaStream_t s);

}  // namespace spx
