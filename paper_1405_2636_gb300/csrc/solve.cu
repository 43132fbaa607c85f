// solve.cu -- permutations in and out of the sweeps, residuals, norms and
// the FGMRES vector kernels.  Right-hand sides are column-major n x nrhs;
// the sweep vectors (sweep.cu) are in the permuted numbering, of the
// factor's type.
#include "kernels.cuh"

namespace spx {

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
// Residual R = B - A X (A by rows in the original numbering) with the
// per-column infinity norms of r, x and b.
// ---------------------------------------------------------------------------
// NaN compares as +inf so that a broken solution can never look converged.
__device__ __forceinline__ double nan_to_inf(double v) { return v != v ? INFINITY : v; }

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *a, double v)
{
    atomicMax(a, (unsigned long long)__double_as_longlong(nan_to_inf(v)));
}

// |v| as bits, NaN as +inf: for non-negative doubles the order of the bit
// patterns is the numeric order, so the norms reduce with integer maxima
// (FP64 comparisons would run on this part's slow FP64 pipe).
__device__ __forceinline__ unsigned long long abs_bits_inf(double v)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    return u > 0x7FF0000000000000ull ? 0x7FF0000000000000ull : u;
}

// Right-hand sides per pass of the residual: a row's entries are read once
// per pass and applied to all of them (16 accumulators a thread).
constexpr int kResRhs = 16;

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
    const int64_t e0 = i < n ? rp[i] : 0, e1 = i < n ? rp[i + 1] : 0;
    for (int c0 = 0; c0 < nrhs; c0 += kResRhs) {
        const int nc = min(kResRhs, nrhs - c0);
        double s[kResRhs];
#pragma unroll
        for (int c = 0; c < kResRhs; ++c) s[c] = 0.0;
        // per (row, column) the products are summed in entry order, as one
        // column at a time would
        for (int64_t e = e0; e < e1; ++e) {
            const double v = vals[src[e]];
            const double *xe = X + ci[e] + (int64_t)c0 * ldx;
#pragma unroll
            for (int c = 0; c < kResRhs; ++c)
                if (c < nc) s[c] += v * xe[(int64_t)c * ldx];
        }
#pragma unroll
        for (int c = 0; c < kResRhs; ++c) {
            if (c >= nc) break;
            const int cc = c0 + c;
            unsigned long long r = 0, ax = 0, ab = 0;
            if (i < n) {
                const double b = B[i + cc * ldb];
                const double rr = b - s[c];
                R[i + cc * n] = rr;
                r = abs_bits_inf(rr);
                ax = abs_bits_inf(X[i + cc * ldx]);
                ab = abs_bits_inf(b);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                r = max(r, __shfl_down_sync(0xffffffffu, r, o));
                ax = max(ax, __shfl_down_sync(0xffffffffu, ax, o));
                ab = max(ab, __shfl_down_sync(0xffffffffu, ab, o));
            }
            if (lane == 0) {
                atomicMax(norms + 3 * cc + 0, r);
                atomicMax(norms + 3 * cc + 1, ax);
                atomicMax(norms + 3 * cc + 2, ab);
            }
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
template void launch_permute_in<float>(int64_t, int, const double *, int64_t, const int64_t *, float *, cudaStream_t);
template void launch_permute_out<float>(int64_t, int, const float *, const int64_t *, double *, int64_t, cudaStream_t);


}  // namespace spx
