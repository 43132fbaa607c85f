// solve.cu -- triangular solves on the panel factor, residuals and norms.
// Forward substitution walks the levels of the panel tree upward, backward
// substitution walks them downward; every level is one diagonal-block launch
// and one off-diagonal launch.  Right-hand sides are column-major n x nrhs in
// the permuted numbering, always double; the factor may be float.
#include "kernels.cuh"

namespace spx {

constexpr int kRhsChunk = 16;

__global__ void permute_in_kernel(int64_t n, int nrhs, const double *__restrict__ B, int64_t ldb,
                                  const int64_t *__restrict__ perm, double *__restrict__ Y)
{
    const int64_t total = n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, k = e - c * n;
        Y[e] = B[perm[k] + c * ldb];
    }
}

__global__ void permute_out_kernel(int64_t n, int nrhs, const double *__restrict__ Y,
                                   const int64_t *__restrict__ perm, double *__restrict__ X,
                                   int64_t ldx)
{
    const int64_t total = n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, k = e - c * n;
        X[perm[k] + c * ldx] = Y[e];
    }
}

static unsigned grid_for(int64_t total)
{
    int64_t b = (total + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (unsigned)b;
}

void launch_permute_in(int64_t n, int nrhs, const double *B, int64_t ldb, const int64_t *perm,
                       double *Y, cudaStream_t s)
{
    permute_in_kernel<<<grid_for(n * nrhs), 256, 0, s>>>(n, nrhs, B, ldb, perm, Y);
}

void launch_permute_out(int64_t n, int nrhs, const double *Y, const int64_t *perm, double *X,
                        int64_t ldx, cudaStream_t s)
{
    permute_out_kernel<<<grid_for(n * nrhs), 256, 0, s>>>(n, nrhs, Y, perm, X, ldx);
}

// ---------------------------------------------------------------------------
// Forward, diagonal block: y_p <- D_lower^{-1} y_p (unit: LU's L).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) fwd_diag_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                       const T *__restrict__ L, int unit,
                                                       double *__restrict__ Y, int nrhs)
{
    __shared__ double ys[kMaxWidth * kRhsChunk];
    const int pid = panels[blockIdx.x];
    const int w = p.pw[pid], h = p.ph[pid];
    const T *D = L + p.pval[pid];
    const int64_t f = p.pfcol[pid], n = p.n;
    const int tid = threadIdx.x;
    for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
        const int nc = min(kRhsChunk, nrhs - c0);
        for (int e = tid; e < w * nc; e += blockDim.x) {
            const int k = e % w, c = e / w;
            ys[c * w + k] = Y[f + k + (int64_t)(c0 + c) * n];
        }
        __syncthreads();
        for (int j = 0; j < w; ++j) {
            if (!unit && tid < nc) ys[tid * w + j] /= (double)D[j + (int64_t)j * h];
            __syncthreads();
            const int rest = w - j - 1;
            for (int e = tid; e < rest * nc; e += blockDim.x) {
                const int i = j + 1 + e % rest, c = e / rest;
                ys[c * w + i] -= (double)D[i + (int64_t)j * h] * ys[c * w + j];
            }
            __syncthreads();
        }
        for (int e = tid; e < w * nc; e += blockDim.x) {
            const int k = e % w, c = e / w;
            Y[f + k + (int64_t)(c0 + c) * n] = ys[c * w + k];
        }
        __syncthreads();
    }
}

// Forward, off-diagonal rows of one chunk: y[rows(i)] -= L(i, :) y_p.
template <typename T>
__global__ void __launch_bounds__(256) fwd_off_kernel(DevPlan p, const RowChunk *__restrict__ chunks,
                                                      const T *__restrict__ L,
                                                      double *__restrict__ Y, int nrhs)
{
    __shared__ double yp[kMaxWidth * kRhsChunk];
    const RowChunk ch = chunks[blockIdx.x];
    const int pid = ch.panel;
    const int w = p.pw[pid], h = p.ph[pid];
    const T *Pn = L + p.pval[pid];
    const int64_t f = p.pfcol[pid], n = p.n;
    const int32_t *rows = p.rows + p.prow[pid];
    const int tid = threadIdx.x;
    const int r = tid & 63, g = tid >> 6;   // 64 rows x 4 column groups
    const int i = ch.r0 + r;
    for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
        const int nc = min(kRhsChunk, nrhs - c0);
        for (int e = tid; e < w * nc; e += blockDim.x) {
            const int k = e % w, c = e / w;
            yp[c * w + k] = Y[f + k + (int64_t)(c0 + c) * n];
        }
        __syncthreads();
        if (i < h) {
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int k = 0; k < w; ++k) {
                const double l = (double)Pn[i + (int64_t)k * h];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = g + 4 * q;
                    if (c < nc) acc[q] += l * yp[c * w + k];
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

// Backward, off-diagonal rows of one chunk: y_p -= Lop(chunk, :)^T y[rows(chunk)].
template <typename T>
__global__ void __launch_bounds__(256) bwd_off_kernel(DevPlan p, const RowChunk *__restrict__ chunks,
                                                      const T *__restrict__ Lop,
                                                      double *__restrict__ Y, int nrhs)
{
    __shared__ double ys[64 * kRhsChunk];
    const RowChunk ch = chunks[blockIdx.x];
    const int pid = ch.panel;
    const int w = p.pw[pid], h = p.ph[pid];
    const T *Pn = Lop + p.pval[pid];
    const int64_t f = p.pfcol[pid], n = p.n;
    const int32_t *rows = p.rows + p.prow[pid];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nr = min(64, h - ch.r0);
    for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
        const int nc = min(kRhsChunk, nrhs - c0);
        for (int e = tid; e < 64 * nc; e += blockDim.x) {
            const int r = e & 63, c = e >> 6;
            ys[c * 64 + r] = (r < nr) ? Y[rows[ch.r0 + r] + (int64_t)(c0 + c) * n] : 0.0;
        }
        __syncthreads();
        for (int k = warp; k < w; k += 8) {
            const double l0 = lane < nr ? (double)Pn[ch.r0 + lane + (int64_t)k * h] : 0.0;
            const double l1 = lane + 32 < nr ? (double)Pn[ch.r0 + lane + 32 + (int64_t)k * h] : 0.0;
            for (int c = 0; c < nc; ++c) {
                double v = l0 * ys[c * 64 + lane] + l1 * ys[c * 64 + lane + 32];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) atomicAdd(Y + f + k + (int64_t)(c0 + c) * n, -v);
            }
        }
        __syncthreads();
    }
}

// Backward, diagonal block: y_p <- M^{-1} y_p with M upper triangular:
// M = lower(D)^T (Cholesky) or upper(D) (LU's U).
template <typename T>
__global__ void __launch_bounds__(256) bwd_diag_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                       const T *__restrict__ L, int upper_from_d,
                                                       double *__restrict__ Y, int nrhs)
{
    __shared__ double ys[kMaxWidth * kRhsChunk];
    const int pid = panels[blockIdx.x];
    const int w = p.pw[pid], h = p.ph[pid];
    const T *D = L + p.pval[pid];
    const int64_t f = p.pfcol[pid], n = p.n;
    const int tid = threadIdx.x;
    for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
        const int nc = min(kRhsChunk, nrhs - c0);
        for (int e = tid; e < w * nc; e += blockDim.x) {
            const int k = e % w, c = e / w;
            ys[c * w + k] = Y[f + k + (int64_t)(c0 + c) * n];
        }
        __syncthreads();
        for (int j = w - 1; j >= 0; --j) {
            if (tid < nc) ys[tid * w + j] /= (double)D[j + (int64_t)j * h];
            __syncthreads();
            for (int e = tid; e < j * nc; e += blockDim.x) {
                const int i = e % j, c = e / j;
                const double m = upper_from_d ? (double)D[i + (int64_t)j * h]
                                              : (double)D[j + (int64_t)i * h];
                ys[c * w + i] -= m * ys[c * w + j];
            }
            __syncthreads();
        }
        for (int e = tid; e < w * nc; e += blockDim.x) {
            const int k = e % w, c = e / w;
            Y[f + k + (int64_t)(c0 + c) * n] = ys[c * w + k];
        }
        __syncthreads();
    }
}

template <typename T>
void launch_fwd_diag(const DevPlan &p, const int32_t *panels, int count, const T *L, int unit,
                     double *Y, int nrhs, cudaStream_t s)
{
    if (count > 0) fwd_diag_kernel<T><<<count, 256, 0, s>>>(p, panels, L, unit, Y, nrhs);
}
template <typename T>
void launch_fwd_off(const DevPlan &p, const RowChunk *chunks, int count, const T *L, double *Y,
                    int nrhs, cudaStream_t s)
{
    if (count > 0) fwd_off_kernel<T><<<count, 256, 0, s>>>(p, chunks, L, Y, nrhs);
}
template <typename T>
void launch_bwd_off(const DevPlan &p, const RowChunk *chunks, int count, const T *Lop, double *Y,
                    int nrhs, cudaStream_t s)
{
    if (count > 0) bwd_off_kernel<T><<<count, 256, 0, s>>>(p, chunks, Lop, Y, nrhs);
}
template <typename T>
void launch_bwd_diag(const DevPlan &p, const int32_t *panels, int count, const T *L,
                     int upper_from_d, double *Y, int nrhs, cudaStream_t s)
{
    if (count > 0) bwd_diag_kernel<T><<<count, 256, 0, s>>>(p, panels, L, upper_from_d, Y, nrhs);
}

// ---------------------------------------------------------------------------
// Residual R = B - A X (A by rows in the original numbering) with the
// per-column infinity norms of r, x and b.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *a, double v)
{
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
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
            r = fabs(r);
            ax = fabs(X[i + c * ldx]);
            ab = fabs(b);
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

template void launch_fwd_diag<double>(const DevPlan &, const int32_t *, int, const double *, int, double *, int, cudaStream_t);
template void launch_fwd_diag<float>(const DevPlan &, const int32_t *, int, const float *, int, double *, int, cudaStream_t);
template void launch_fwd_off<double>(const DevPlan &, const RowChunk *, int, const double *, double *, int, cudaStream_t);
template void launch_fwd_off<float>(const DevPlan &, const RowChunk *, int, const float *, double *, int, cudaStream_t);
template void launch_bwd_off<double>(const DevPlan &, const RowChunk *, int, const double *, double *, int, cudaStream_t);
template void launch_bwd_off<float>(const DevPlan &, const RowChunk *, int, const float *, double *, int, cudaStream_t);
template void launch_bwd_diag<double>(const DevPlan &, const int32_t *, int, const double *, int, double *, int, cudaStream_t);
template void launch_bwd_diag<float>(const DevPlan &, const int32_t *, int, const float *, int, double *, int, cudaStream_t);

}  // namespace spx
