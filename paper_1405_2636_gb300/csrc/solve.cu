// solve.cu -- triangular solves on the panel factor, residuals and norms.
// Forward substitution walks the levels of the panel tree upward, backward
// substitution walks them downward; every level is one diagonal-block launch
// and one off-diagonal launch.  Right-hand sides are column-major n x nrhs in
// the permuted numbering, always double; the factor may be float.
#include "kernels.cuh"

namespace spx {

constexpr int kRhsChunk = 16;
constexpr int kDiagRows = 32;   // rows of D^{-1} one CTA of the diagonal products handles

template <typename T>
__global__ void permute_in_kernel(int64_t n, int nrhs, const double *__restrict__ B, int64_t ldb,
                                  const int64_t *__restrict__ perm, T *__restrict__ Y)
{
    const int64_t total = n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, k = e - c * n;
        Y[e] = (T)B[perm[k] + c * ldb];
    }
}

template <typename T>
__global__ void permute_out_kernel(int64_t n, int nrhs, const T *__restrict__ Y,
                                   const int64_t *__restrict__ perm, double *__restrict__ X,
                                   int64_t ldx)
{
    const int64_t total = n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, k = e - c * n;
        X[perm[k] + c * ldx] = (double)Y[e];
    }
}

static unsigned grid_for(int64_t total)
{
    int64_t b = (total + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <typename T>
void launch_permute_in(int64_t n, int nrhs, const double *B, int64_t ldb, const int64_t *perm,
                       T *Y, cudaStream_t s)
{
    permute_in_kernel<T><<<grid_for(n * nrhs), 256, 0, s>>>(n, nrhs, B, ldb, perm, Y);
}

template <typename T>
void launch_permute_out(int64_t n, int nrhs, const T *Y, const int64_t *perm, double *X,
                        int64_t ldx, cudaStream_t s)
{
    permute_out_kernel<T><<<grid_for(n * nrhs), 256, 0, s>>>(n, nrhs, Y, perm, X, ldx);
}

// ---------------------------------------------------------------------------
// Forward, diagonal block: Z_p = Linv_p Y_p, rows [32 y, 32 y + 32) of the
// panel per CTA (grid.y).  LU: Linv is unit (the diagonal slot holds U^{-1}).
// The 32 rows of Linv are staged in shared memory first (coalesced bulk
// loads), so the products never wait on one global load at a time.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) fwd_diag_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                       const T *__restrict__ Dinv, int unit,
                                                       const T *__restrict__ Y, T *__restrict__ Z,
                                                       int nrhs)
{
    extern __shared__ unsigned char smraw[];
    pdl_trigger();
    const int pid = panels[blockIdx.x];
    const int w = p.pw[pid];
    const int i0 = blockIdx.y * kDiagRows;
    if (i0 >= w) return;
    T *ys = reinterpret_cast<T *>(smraw);        // ys[c * w + k]
    T *ms = ys + (size_t)w * kRhsChunk;           // ms[k * 33 + li] = Linv(i0 + li, k)
    const T *Mi = Dinv + p.pinv[pid];
    const int64_t f = p.pfcol[pid], n = p.n;
    const int tid = threadIdx.x;
    const int li = tid & 31, cg = tid >> 5;     // row within the block, column group of 8
    const int i = i0 + li;
    const int nrow = min(kDiagRows, w - i0);
    const int kend = min(w, i0 + kDiagRows);     // Linv(i, k) = 0 for k > i
    for (int e = tid; e < kend * kDiagRows; e += blockDim.x) {
        const int r = e & 31, k = e >> 5;
        ms[k * 33 + r] = r < nrow ? Mi[(i0 + r) + (int64_t)k * w] : (T)0;
    }
    pdl_wait();   // Y comes from the previous level's kernels
    for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
        const int nc = min(kRhsChunk, nrhs - c0);
        for (int e = tid; e < kend * nc; e += blockDim.x) {
            const int k = e % kend, c = e / kend;
            ys[c * w + k] = Y[f + k + (int64_t)(c0 + c) * n];
        }
        __syncthreads();
        if (li < nrow) {
            for (int c = cg; c < nc; c += 8) {
                const T *yc = ys + c * w;
                T a0 = unit ? yc[i] : (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
                const int kl = unit ? i : i + 1;
                int k = 0;
                for (; k + 3 < kl; k += 4) {
                    a0 += ms[k * 33 + li] * yc[k];
                    a1 += ms[(k + 1) * 33 + li] * yc[k + 1];
                    a2 += ms[(k + 2) * 33 + li] * yc[k + 2];
                    a3 += ms[(k + 3) * 33 + li] * yc[k + 3];
                }
                for (; k < kl; ++k) a0 += ms[k * 33 + li] * yc[k];
                Z[f + i + (int64_t)(c0 + c) * n] = (a0 + a1) + (a2 + a3);
            }
        }
        __syncthreads();
    }
}

// Forward, off-diagonal rows of one chunk: Y[rows(i)] -= L(i, :) Z_p, with
// the 64 x w block of L staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) fwd_off_kernel(DevPlan p, const RowChunk *__restrict__ chunks,
                                                      const T *__restrict__ L,
                                                      const T *__restrict__ Z, T *__restrict__ Y,
                                                      int nrhs)
{
    extern __shared__ unsigned char smraw[];
    pdl_trigger();
    const RowChunk ch = chunks[blockIdx.x];
    const int pid = ch.panel;
    const int w = p.pw[pid], h = p.ph[pid];
    T *zp = reinterpret_cast<T *>(smraw);        // zp[c * w + k]
    T *lsm = zp + (size_t)w * kRhsChunk;          // lsm[k * 64 + r]
    const T *Pn = L + p.pval[pid];
    const int64_t f = p.pfcol[pid], n = p.n;
    const int32_t *rows = p.rows + p.prow[pid];
    const int tid = threadIdx.x;
    const int r = tid & 63, g = tid >> 6;   // 64 rows x 4 column groups
    const int i = ch.r0 + r;
    const int nr = min(64, h - ch.r0);
    for (int e = tid; e < w * 64; e += blockDim.x) {
        const int rr = e & 63, k = e >> 6;
        lsm[e] = rr < nr ? Pn[ch.r0 + rr + (int64_t)k * h] : (T)0;
    }
    pdl_wait();   // Z from the diagonal kernel just before
    for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
        const int nc = min(kRhsChunk, nrhs - c0);
        for (int e = tid; e < w * nc; e += blockDim.x) {
            const int k = e % w, c = e / w;
            zp[c * w + k] = Z[f + k + (int64_t)(c0 + c) * n];
        }
        __syncthreads();
        if (r < nr) {
            T acc[4] = {(T)0, (T)0, (T)0, (T)0};
            for (int k = 0; k < w; ++k) {
                const T l = lsm[k * 64 + r];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = g + 4 * q;
                    if (c < nc) acc[q] += l * zp[c * w + k];
                }
            }
            const int64_t gi = rows[i];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = g + 4 * q;
                if (c < nc) atomicAdd(Y + gi + (int64_t)(c0 + c) * n, -acc[q]);
            }
        }
        __syncthreads();
    }
}

// Backward, off-diagonal rows of one chunk: Tacc_p += Lop(chunk, :)^T X[rows(chunk)].
template <typename T>
__global__ void __launch_bounds__(256) bwd_off_kernel(DevPlan p, const RowChunk *__restrict__ chunks,
                                                      const T *__restrict__ Lop,
                                                      const T *__restrict__ X,
                                                      T *__restrict__ Tacc, int nrhs)
{
    extern __shared__ unsigned char smraw[];
    pdl_trigger();
    T *ls = reinterpret_cast<T *>(smraw);            // ls[k * 65 + r]
    const RowChunk ch = chunks[blockIdx.x];
    const int pid = ch.panel;
    const int w = p.pw[pid], h = p.ph[pid];
    T *xs = ls + (size_t)w * 65;                      // xs[c * 64 + r]
    const T *Pn = Lop + p.pval[pid];
    const int64_t f = p.pfcol[pid], n = p.n;
    const int32_t *rows = p.rows + p.prow[pid];
    const int tid = threadIdx.x;
    const int nr = min(64, h - ch.r0);
    for (int e = tid; e < w * 64; e += blockDim.x) {
        const int r = e & 63, k = e >> 6;
        ls[k * 65 + r] = r < nr ? Pn[ch.r0 + r + (int64_t)k * h] : (T)0;
    }
    pdl_wait();   // X of the rows below comes from earlier levels
    for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
        const int nc = min(kRhsChunk, nrhs - c0);
        for (int e = tid; e < 64 * nc; e += blockDim.x) {
            const int r = e & 63, c = e >> 6;
            xs[c * 64 + r] = (r < nr) ? X[rows[ch.r0 + r] + (int64_t)(c0 + c) * n] : (T)0;
        }
        __syncthreads();
        for (int e = tid; e < w * nc; e += blockDim.x) {
            const int k = e % w, c = e / w;
            T acc = (T)0;
#pragma unroll 8
            for (int r = 0; r < 64; ++r) acc += ls[k * 65 + r] * xs[c * 64 + r];
            atomicAdd(Tacc + f + k + (int64_t)(c0 + c) * n, acc);
        }
        __syncthreads();
    }
}

// Backward, diagonal block: X_p = M (Z_p - Tacc_p) with M = Linv^T (Cholesky)
// or U^{-1} (LU), rows [32 y, 32 y + 32) per CTA.  LDL^T (lu == 2):
// X_p = l^{-T} (D^{-1} Z_p - Tacc_p), the unit l^{-1} below the diagonal of
// Dinv and 1/d on it.
template <typename T>
__global__ void __launch_bounds__(256) bwd_diag_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                       const T *__restrict__ Dinv, int lu,
                                                       const T *__restrict__ Z,
                                                       const T *__restrict__ Tacc,
                                                       T *__restrict__ X, int nrhs)
{
    extern __shared__ unsigned char smraw[];
    pdl_trigger();
    T *ys = reinterpret_cast<T *>(smraw);          // ys[c * w + k]
    const int pid = panels[blockIdx.x];
    const int w = p.pw[pid];
    const int i0 = blockIdx.y * kDiagRows;
    if (i0 >= w) return;
    T *ms = ys + (size_t)w * kRhsChunk;            // ms[li * (w + 1) + k] = M(i0 + li, k)
    const T *Mi = Dinv + p.pinv[pid];
    const int64_t f = p.pfcol[pid], n = p.n;
    const int tid = threadIdx.x;
    const int li = tid & 31, cg = tid >> 5;
    const int i = i0 + li;
    const int nrow = min(kDiagRows, w - i0);
    // M(i, k) for k >= i: Cholesky Linv(k, i) = Mi[k + i w]; LU Uinv(i, k) = Mi[i + k w]
    for (int e = tid; e < nrow * w; e += blockDim.x) {
        int a, k;
        if (lu == 1) { a = e % nrow; k = e / nrow; } else { k = e % w; a = e / w; }
        const int ii = i0 + a;
        T v = (T)0;
        if (k >= ii) v = lu == 1 ? Mi[ii + k * w] : (lu == 2 && k == ii ? (T)1 : Mi[k + ii * w]);
        ms[a * (w + 1) + k] = v;
    }
    pdl_wait();   // Z, Tacc and X from earlier kernels
    for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
        const int nc = min(kRhsChunk, nrhs - c0);
        for (int e = tid; e < w * nc; e += blockDim.x) {
            const int k = e % w, c = e / w;
            const int64_t g = f + k + (int64_t)(c0 + c) * n;
            ys[c * w + k] = (lu == 2 ? Z[g] * Mi[k + k * w] : Z[g]) - Tacc[g];
        }
        __syncthreads();
        if (li < nrow) {
            for (int c = cg; c < nc; c += 8) {
                const T *yc = ys + c * w;
                const T *mr = ms + li * (w + 1);
                T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
                int k = i;
                for (; k + 3 < w; k += 4) {
                    a0 += mr[k] * yc[k];
                    a1 += mr[k + 1] * yc[k + 1];
                    a2 += mr[k + 2] * yc[k + 2];
                    a3 += mr[k + 3] * yc[k + 3];
                }
                for (; k < w; ++k) a0 += mr[k] * yc[k];
                X[f + i + (int64_t)(c0 + c) * n] = (a0 + a1) + (a2 + a3);
            }
        }
        __syncthreads();
    }
}

template <typename T>
void launch_fwd_diag(const DevPlan &p, const int32_t *panels, int count, int wmax, const T *Dinv,
                     int unit, const T *Y, T *Z, int nrhs, cudaStream_t s)
{
    if (count <= 0) return;
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(fwd_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(T) * ((size_t)kMaxWidth * kRhsChunk + (size_t)kMaxWidth * 33)));
        once = true;
    }
    dim3 grid(count, (wmax + kDiagRows - 1) / kDiagRows);
    const size_t smem = sizeof(T) * ((size_t)wmax * kRhsChunk + (size_t)wmax * 33);
    static const bool carveout_once = set_max_carveout(fwd_diag_kernel<T>);
    (void)carveout_once;
    launch_pdl(sizeof(T) == 4, fwd_diag_kernel<T>, grid, dim3(256), smem, s, p, panels, Dinv, unit, Y, Z, nrhs);
}

template <typename T>
void launch_fwd_off(const DevPlan &p, const RowChunk *chunks, int count, int wmax, const T *L,
                    const T *Z, T *Y, int nrhs, cudaStream_t s)
{
    if (count <= 0) return;
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(fwd_off_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(T) * ((size_t)kMaxWidth * kRhsChunk + (size_t)kMaxWidth * 64)));
        once = true;
    }
    const size_t smem = sizeof(T) * ((size_t)wmax * kRhsChunk + (size_t)wmax * 64);
    static const bool carveout_once = set_max_carveout(fwd_off_kernel<T>);
    (void)carveout_once;
    launch_pdl(sizeof(T) == 4, fwd_off_kernel<T>, dim3(count), dim3(256), smem, s, p, chunks, L, Z, Y, nrhs);
}

template <typename T>
void launch_bwd_off(const DevPlan &p, const RowChunk *chunks, int count, int wmax, const T *Lop,
                    const T *X, T *Tacc, int nrhs, cudaStream_t s)
{
    if (count <= 0) return;
    static bool once = false;
    const size_t most = sizeof(T) * ((size_t)kMaxWidth * 65 + 64 * kRhsChunk);
    if (!once) {
        cudaFuncSetAttribute(bwd_off_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        once = true;
    }
    const size_t smem = sizeof(T) * ((size_t)wmax * 65 + 64 * kRhsChunk);
    static const bool carveout_once = set_max_carveout(bwd_off_kernel<T>);
    (void)carveout_once;
    launch_pdl(sizeof(T) == 4, bwd_off_kernel<T>, dim3(count), dim3(256), smem, s, p, chunks, Lop, X, Tacc, nrhs);
}

template <typename T>
void launch_bwd_diag(const DevPlan &p, const int32_t *panels, int count, int wmax, const T *Dinv,
                     int lu, const T *Z, const T *Tacc, T *X, int nrhs, cudaStream_t s)
{
    if (count <= 0) return;
    static bool once = false;
    const size_t most = sizeof(T) * ((size_t)kMaxWidth * kRhsChunk + kDiagRows * (kMaxWidth + 1));
    if (!once) {
        cudaFuncSetAttribute(bwd_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        once = true;
    }
    dim3 grid(count, (wmax + kDiagRows - 1) / kDiagRows);
    const size_t smem = sizeof(T) * ((size_t)wmax * kRhsChunk + kDiagRows * (wmax + 1));
    static const bool carveout_once = set_max_carveout(bwd_diag_kernel<T>);
    (void)carveout_once;
    launch_pdl(sizeof(T) == 4, bwd_diag_kernel<T>, grid, dim3(256), smem, s, p, panels, Dinv, lu, Z, Tacc, X, nrhs);
}

// ---------------------------------------------------------------------------
// Residual R = B - A X (A by rows in the original numbering) with the
// per-column infinity norms of r, x and b.
// ---------------------------------------------------------------------------
// NaN compares as +inf so that a broken solution can never look converged.
__device__ __forceinline__ double nan_to_inf(double v) { return v != v ? INFINITY : v; }

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *a, double v)
{
    atomicMax(a, (unsigned long long)__double_as_longlong(nan_to_inf(v)));
}

__global__ void __launch_bounds__(256) residual_kernel(int64_t n, int nrhs,
                                                       const int64_t *__restrict__ rp,
                                                       const int32_t *__restrict__ ci,
                                                       const int64_t *__restrict__ src,
                                                       const double *__restrict__ vals,
                                                       const double *__restrict__ X, int64_t ldx,
                                                       const double *__restrict__ B, int64_t ldb,
                                                       double *__restrict__ R,
                                                       unsigned long long *norms)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < nrhs; ++c) {
        double r = 0.0, ax = 0.0, ab = 0.0;
        if (i < n) {
            double s = 0.0;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += vals[src[e]] * X[ci[e] + c * ldx];
            const double b = B[i + c * ldb];
            r = b - s;
            R[i + c * n] = r;
            r = nan_to_inf(fabs(r));
            ax = nan_to_inf(fabs(X[i + c * ldx]));
            ab = nan_to_inf(fabs(b));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
            ax = fmax(ax, __shfl_down_sync(0xffffffffu, ax, o));
            ab = fmax(ab, __shfl_down_sync(0xffffffffu, ab, o));
        }
        if (lane == 0) {
            atomic_max_nonneg(norms + 3 * c + 0, r);
            atomic_max_nonneg(norms + 3 * c + 1, ax);
            atomic_max_nonneg(norms + 3 * c + 2, ab);
        }
    }
}

void launch_residual(int64_t n, int nrhs, const int64_t *rp, const int32_t *ci, const int64_t *src,
                     const double *vals, const double *X, int64_t ldx, const double *B, int64_t ldb,
                     double *R, unsigned long long *norms, cudaStream_t s)
{
    residual_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, nrhs, rp, ci, src, vals, X, ldx,
                                                                B, ldb, R, norms);
}

__global__ void row_abs_sum_kernel(int64_t n, const int64_t *__restrict__ rp,
                                   const int64_t *__restrict__ src, const double *__restrict__ vals,
                                   unsigned long long *out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += fabs(vals[src[e]]);
    s = nan_to_inf(s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, s);
}

void launch_row_abs_sum_max(int64_t n, const int64_t *rp, const int64_t *src, const double *vals,
                            unsigned long long *out, cudaStream_t s)
{
    row_abs_sum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, rp, src, vals, out);
}

__global__ void axpy_cols_kernel(int64_t n, int nrhs, const double *__restrict__ D,
                                 double *__restrict__ X, int64_t ldx)
{
    const int64_t total = n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        X[i + c * ldx] += D[e];
    }
}

void launch_axpy_cols(int64_t n, int nrhs, const double *D, double *X, int64_t ldx, cudaStream_t s)
{
    axpy_cols_kernel<<<grid_for(n * nrhs), 256, 0, s>>>(n, nrhs, D, X, ldx);
}

// ---------------------------------------------------------------------------
// Vector kernels of the FGMRES refinement (n x nrhs column blocks, FP64).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) spmv_cols_kernel(int64_t n, int nrhs, const int64_t *__restrict__ rp,
                                                        const int32_t *__restrict__ ci,
                                                        const int64_t *__restrict__ src,
                                                        const double *__restrict__ vals,
                                                        const double *__restrict__ X,
                                                        double *__restrict__ Y)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < nrhs; ++c) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += vals[src[e]] * X[ci[e] + c * n];
        Y[i + c * n] = s;
    }
}

// out[v * nrhs + c] += sum_r V_v[r, c] * w[r, c] for v < nv (V_v = V + v * n * nrhs)
__global__ void __launch_bounds__(256) dots_kernel(int64_t n, int nrhs, int nv, const double *__restrict__ V,
                                                   const double *__restrict__ w, double *out)
{
    const int c = blockIdx.y;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int v = 0; v < nv; ++v) {
        const double *Vv = V + (int64_t)v * n * nrhs + c * n;
        const double *wc = w + c * n;
        double s = 0.0;
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) s += Vv[r] * wc[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        __shared__ double part[8];
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += part[q];
            atomicAdd(out + v * nrhs + c, t);
        }
        __syncthreads();
    }
}

// w[r, c] += sign * sum_v coef[v * nrhs + c] * V_v[r, c]
__global__ void __launch_bounds__(256) combine_kernel(int64_t n, int nrhs, int nv, const double *__restrict__ V,
                                                      const double *__restrict__ coef, double sign,
                                                      double *__restrict__ w)
{
    const int64_t total = n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        double s = 0.0;
        for (int v = 0; v < nv; ++v) s += coef[v * nrhs + c] * V[(int64_t)v * total + e];
        w[e] += sign * s;
    }
}

// v[r, c] = w[r, c] * s[c]
__global__ void scale_cols_kernel(int64_t n, int nrhs, const double *__restrict__ w,
                                  const double *__restrict__ sc, double *__restrict__ v)
{
    const int64_t total = n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x)
        v[e] = w[e] * sc[e / n];
}

void launch_spmv_cols(int64_t n, int nrhs, const int64_t *rp, const int32_t *ci, const int64_t *src,
                      const double *vals, const double *X, double *Y, cudaStream_t s)
{
    spmv_cols_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, nrhs, rp, ci, src, vals, X, Y);
}

void launch_dots(int64_t n, int nrhs, int nv, const double *V, const double *w, double *out,
                 cudaStream_t s)
{
    int64_t bx = (n + 255) / 256;
    if (bx > 64) bx = 64;
    dim3 grid((unsigned)bx, (unsigned)nrhs);
    cudaMemsetAsync(out, 0, sizeof(double) * nv * nrhs, s);
    dots_kernel<<<grid, 256, 0, s>>>(n, nrhs, nv, V, w, out);
}

void launch_combine(int64_t n, int nrhs, int nv, const double *V, const double *coef, double sign,
                    double *w, cudaStream_t s)
{
    combine_kernel<<<grid_for(n * nrhs), 256, 0, s>>>(n, nrhs, nv, V, coef, sign, w);
}

void launch_scale_cols(int64_t n, int nrhs, const double *w, const double *sc, double *v, cudaStream_t s)
{
    scale_cols_kernel<<<grid_for(n * nrhs), 256, 0, s>>>(n, nrhs, w, sc, v);
}

template void launch_permute_in<double>(int64_t, int, const double *, int64_t, const int64_t *, double *, cudaStream_t);
template void launch_permute_out<double>(int64_t, int, const double *, const int64_t *, double *, int64_t, cudaStream_t);
template void launch_fwd_diag<double>(const DevPlan &, const int32_t *, int, int, const double *, int, const double *, double *, int, cudaStream_t);
template void launch_fwd_off<double>(const DevPlan &, const RowChunk *, int, int, const double *, const double *, double *, int, cudaStream_t);
template void launch_bwd_off<double>(const DevPlan &, const RowChunk *, int, int, const double *, const double *, double *, int, cudaStream_t);
template void launch_bwd_diag<double>(const DevPlan &, const int32_t *, int, int, const double *, int, const double *, const double *, double *, int, cudaStream_t);
template void launch_permute_in<float>(int64_t, int, const double *, int64_t, const int64_t *, float *, cudaStream_t);
template void launch_permute_out<float>(int64_t, int, const float *, const int64_t *, double *, int64_t, cudaStream_t);
template void launch_fwd_diag<float>(const DevPlan &, const int32_t *, int, int, const float *, int, const float *, float *, int, cudaStream_t);
template void launch_fwd_off<float>(const DevPlan &, const RowChunk *, int, int, const float *, const float *, float *, int, cudaStream_t);
template void launch_bwd_off<float>(const DevPlan &, const RowChunk *, int, int, const float *, const float *, float *, int, cudaStream_t);
template void launch_bwd_diag<float>(const DevPlan &, const int32_t *, int, int, const float *, int, const float *, const float *, float *, int, cudaStream_t);


}  // namespace spx
