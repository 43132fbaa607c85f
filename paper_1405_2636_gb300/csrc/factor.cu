// factor.cu -- numerical factorization kernels of libspx (Sec. III: the
// three steps of the 1D task on one panel -- factorization of the diagonal
// block, triangular solve of the off-diagonal blocks, update of every facing
// panel -- and Sec. V-B: the update computes the product of two row ranges
// of the source panel and subtracts it directly at the positions the target
// panel's block structure gives, with no temporary buffer).
//
// Panels are column-major "tall and skinny" matrices (Sec. III): leading
// dimension = panel height h, the w x w diagonal block on top, the
// off-diagonal rows below.  T is the storage type (double, or float for the
// mixed-precision factor); the diagonal blocks are always factored in double.
#include "kernels.cuh"

#include <cstdio>

namespace spx {

// ---------------------------------------------------------------------------
// Assembly: scatter the CSC values into the zeroed panels.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void assemble_kernel(int64_t nnz, const double *__restrict__ vals,
                                const int64_t *__restrict__ amap, T *__restrict__ L,
                                T *__restrict__ U)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t d = amap[e];
        if (d >= 0) L[d] = (T)vals[e];
        else if (d <= -2) U[-2 - d] = (T)vals[e];
    }
}

template <typename T>
void launch_assemble(int64_t nnz, const double *vals, const int64_t *amap, T *L, T *U,
                     cudaStream_t s)
{
    if (nnz <= 0) return;
    int64_t blocks = (nnz + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    assemble_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(nnz, vals, amap, L, U);
}

// ---------------------------------------------------------------------------
// Diagonal block, Cholesky: one CTA per panel, the block in shared memory in
// double, right-looking by columns.  A pivot that is not positive is either
// reported (replace_tau <= 0: the smallest failing column goes to *err_col)
// or replaced by replace_tau and counted.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) potrf_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                    T *__restrict__ L, const double *replace_tau_p,
                                                    int64_t *err_col, unsigned long long *nrepl)
{
    extern __shared__ double sm[];
    __shared__ double s_piv;
    const double replace_tau = *replace_tau_p;
    const int pid = panels[blockIdx.x];
    const int w = p.pw[pid], h = p.ph[pid];
    T *D = L + p.pval[pid];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int idx = tid; idx < w * w; idx += nt) {
        int i = idx % w, j = idx / w;
        sm[idx] = (i >= j) ? (double)D[i + (int64_t)j * h] : 0.0;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int k = 0; k < w; ++k) {
        if (tid == 0) {
            double d = sm[k + k * w];
            if (!(d > 0.0)) {
                if (replace_tau > 0.0) {
                    d = replace_tau;
                    atomicAdd(nrepl, 1ull);
                } else {
                    atomicMin((long long *)err_col, (long long)(p.pfcol[pid] + k));
                    d = 1.0;
                }
            }
            d = sqrt(d);
            sm[k + k * w] = d;
            s_piv = d;
        }
        __syncthreads();
        const double inv = 1.0 / s_piv;
        for (int i = k + 1 + tid; i < w; i += nt) sm[i + k * w] *= inv;
        __syncthreads();
        for (int j = k + 1 + warp; j < w; j += nw) {
            const double ljk = sm[j + k * w];
            for (int i = j + lane; i < w; i += 32) sm[i + j * w] -= sm[i + k * w] * ljk;
        }
        __syncthreads();
    }
    for (int idx = tid; idx < w * w; idx += nt) {
        int i = idx % w, j = idx / w;
        if (i >= j) D[i + (int64_t)j * h] = (T)sm[idx];
    }
}

template <typename T>
void launch_potrf(const DevPlan &p, const int32_t *panels, int count, T *L, const double *replace_tau,
                  int64_t *err_col, unsigned long long *nrepl, cudaStream_t s)
{
    if (count <= 0) return;
    const size_t smem = sizeof(double) * kMaxWidth * kMaxWidth;
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(potrf_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        once = true;
    }
    potrf_kernel<T><<<count, 256, smem, s>>>(p, panels, L, replace_tau, err_col, nrepl);
}

// ---------------------------------------------------------------------------
// Diagonal block, LU without pivoting (Sec. III: static pivoting): a pivot
// whose magnitude is below tau becomes sign(pivot) * tau (+tau for 0) and is
// counted; tau <= 0 turns a zero pivot into an error instead.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) getrf_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                    T *__restrict__ L, const double *tau_p,
                                                    int64_t *err_col, unsigned long long *nrepl)
{
    extern __shared__ double sm[];
    __shared__ double s_piv;
    const double tau = *tau_p;
    const int pid = panels[blockIdx.x];
    const int w = p.pw[pid], h = p.ph[pid];
    T *D = L + p.pval[pid];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int idx = tid; idx < w * w; idx += nt) {
        int i = idx % w, j = idx / w;
        sm[idx] = (double)D[i + (int64_t)j * h];
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int k = 0; k < w; ++k) {
        if (tid == 0) {
            double d = sm[k + k * w];
            if (tau > 0.0) {
                if (fabs(d) < tau) {
                    d = (d < 0.0) ? -tau : tau;
                    atomicAdd(nrepl, 1ull);
                }
            } else if (d == 0.0 || d != d) {
                atomicMin((long long *)err_col, (long long)(p.pfcol[pid] + k));
                d = 1.0;
            }
            sm[k + k * w] = d;
            s_piv = d;
        }
        __syncthreads();
        const double inv = 1.0 / s_piv;
        for (int i = k + 1 + tid; i < w; i += nt) sm[i + k * w] *= inv;
        __syncthreads();
        for (int j = k + 1 + warp; j < w; j += nw) {
            const double ukj = sm[k + j * w];
            for (int i = k + 1 + lane; i < w; i += 32) sm[i + j * w] -= sm[i + k * w] * ukj;
        }
        __syncthreads();
    }
    for (int idx = tid; idx < w * w; idx += nt) {
        int i = idx % w, j = idx / w;
        D[i + (int64_t)j * h] = (T)sm[idx];
    }
}

template <typename T>
void launch_getrf(const DevPlan &p, const int32_t *panels, int count, T *L, const double *tau,
                  int64_t *err_col, unsigned long long *nrepl, cudaStream_t s)
{
    if (count <= 0) return;
    const size_t smem = sizeof(double) * kMaxWidth * kMaxWidth;
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(getrf_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        once = true;
    }
    getrf_kernel<T><<<count, 256, smem, s>>>(p, panels, L, tau, err_col, nrepl);
}

// ---------------------------------------------------------------------------
// Panel TRSM (Sec. III step 2): rows [r0, r0+64) of the off-diagonal part,
// one thread per row, by substitution against the factored diagonal block
// held packed in shared memory.  Every mode solves Y M^T = X with M lower
// triangular:  LLT: M = lower(D);  LU_L: M = upper(D)^T (Y U = X);
// LU_U: M = unit lower(D).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kTrsmRows) trsm_kernel(DevPlan p,
                                                         const RowChunk *__restrict__ chunks,
                                                         const T *__restrict__ Dsrc,
                                                         T *__restrict__ X, int mode)
{
    extern __shared__ double sm[];
    const RowChunk ch = chunks[blockIdx.x];
    const int pid = ch.panel;
    const int w = p.pw[pid], h = p.ph[pid];
    const int64_t base = p.pval[pid];
    double *M = sm;                                   // packed by columns
    double *Xs = sm + (w * (w + 1)) / 2;              // Xs[c * 64 + r]
    const T *D = Dsrc + base;
    const int tid = threadIdx.x;
    int start = 0;
    for (int c = 0; c < w; ++c) {
        for (int j = c + tid; j < w; j += kTrsmRows) {
            double v = (mode == TRSM_LU_L) ? (double)D[c + (int64_t)j * h]
                                           : (double)D[j + (int64_t)c * h];
            if (mode == TRSM_LU_U && j == c) v = 1.0;
            M[start + (j - c)] = v;
        }
        start += w - c;
    }
    const int nr = min(kTrsmRows, h - ch.r0);
    T *Xg = X + base + ch.r0;
    if (tid < nr)
        for (int c = 0; c < w; ++c) Xs[c * kTrsmRows + tid] = (double)Xg[tid + (int64_t)c * h];
    __syncthreads();
    if (tid < nr) {
        int diag = 0;   // packed index of M(j, j)
        for (int j = 0; j < w; ++j) {
            double s = Xs[j * kTrsmRows + tid];
            int idx = j;  // M(j, 0)
            for (int c = 0; c < j; ++c) {
                s -= Xs[c * kTrsmRows + tid] * M[idx];
                idx += w - c - 1;
            }
            Xs[j * kTrsmRows + tid] = s / M[diag];
            diag += w - j;
        }
        for (int c = 0; c < w; ++c) Xg[tid + (int64_t)c * h] = (T)Xs[c * kTrsmRows + tid];
    }
}

template <typename T>
void launch_trsm(const DevPlan &p, const RowChunk *chunks, int count, const T *Dsrc, T *X,
                 int mode, cudaStream_t s)
{
    if (count <= 0) return;
    const size_t smem = sizeof(double) * ((kMaxWidth * (kMaxWidth + 1)) / 2 + kMaxWidth * kTrsmRows);
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(trsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        once = true;
    }
    trsm_kernel<T><<<count, kTrsmRows, smem, s>>>(p, chunks, Dsrc, X, mode);
}

// ---------------------------------------------------------------------------
// Update with fused scatter (Sec. V-B).  One CTA computes a 64 x 64 tile of
// W = A_rows(M) * B_rows(N)^T over the source panel's width, K-chunked
// through shared memory, then subtracts it from the target panel at row
// relmap(i) and column row(j) - first column(target), with atomic adds so
// that sources of one level may hit the same target concurrently.
//   lower   : skip entries with i < j (Cholesky diagonal-block region)
//   from_r1 : rows below r1 only (the U^T side of an LU update)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void atomic_sub(T *addr, T v);
template <>
__device__ __forceinline__ void atomic_sub<double>(double *addr, double v) { atomicAdd(addr, -v); }
template <>
__device__ __forceinline__ void atomic_sub<float>(float *addr, float v) { atomicAdd(addr, -v); }

template <typename T>
__global__ void __launch_bounds__(256) update_kernel(DevPlan p, const DevTask *__restrict__ tasks,
                                                     const UpdTile *__restrict__ tiles,
                                                     const T *__restrict__ Aop,
                                                     const T *__restrict__ Bop, T *__restrict__ C,
                                                     int lower, int from_r1)
{
    __shared__ T As[16][kUpdTile + 1];
    __shared__ T Bs[16][kUpdTile + 1];
    const UpdTile tl = tiles[blockIdx.x];
    const DevTask tk = tasks[tl.task];
    const int src = tk.src, tgt = tk.tgt;
    const int h = p.ph[src], K = p.pw[src];
    const int64_t sbase = p.pval[src];
    const T *A = Aop + sbase;
    const T *B = Bop + sbase;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    const int lr = tid & 63, lk = tid >> 6;   // loader: 64 rows x 4 k per pass
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int kk = lk + 4 * q;
            const int kg = k0 + kk;
            const int ra = tl.m0 + lr, rb = tl.n0 + lr;
            As[kk][lr] = (kg < K && ra < h) ? A[ra + (int64_t)kg * h] : (T)0;
            Bs[kk][lr] = (kg < K && rb < tk.r1) ? B[rb + (int64_t)kg * h] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        __syncthreads();
    }
    const int hT = p.ph[tgt];
    T *Ct = C + p.pval[tgt];
    const int64_t fcolT = p.pfcol[tgt];
    const int32_t *srow = p.rows + p.prow[src];
    const int32_t *rmap = p.relmap + tk.relmap_off - tk.r0;
    const int rlo = from_r1 ? tk.r1 : tk.r0;
    int64_t coff[4];
    bool cok[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = tl.n0 + ty + 16 * b;
        cok[b] = j < tk.r1;
        coff[b] = cok[b] ? (int64_t)(srow[j] - fcolT) * hT : 0;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = tl.m0 + tx + 16 * a;
        if (i >= h || i < rlo) continue;
        const int64_t roff = rmap[i];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = tl.n0 + ty + 16 * b;
            if (!cok[b] || (lower && i < j)) continue;
            atomic_sub<T>(Ct + roff + coff[b], acc[a][b]);
        }
    }
}

template <typename T>
void launch_update(const DevPlan &p, const DevTask *tasks, const UpdTile *tiles, int count,
                   const T *Aop, const T *Bop, T *C, int lower, int from_r1, cudaStream_t s)
{
    if (count <= 0) return;
    update_kernel<T><<<count, 256, 0, s>>>(p, tasks, tiles, Aop, Bop, C, lower, from_r1);
}

// ---------------------------------------------------------------------------
// The same update as a standalone call (the paper's kernel study, Sec. V-B:
// C = C - A B^T with B the first rows of A and C a taller gapped panel).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) update_standalone_kernel(
    int m, int nb, int k, const double *__restrict__ A, int64_t lda, double *__restrict__ C,
    int64_t ldc, const int32_t *__restrict__ rowmap, const int32_t *__restrict__ colmap, int lower)
{
    __shared__ double As[16][kUpdTile + 1];
    __shared__ double Bs[16][kUpdTile + 1];
    const int m0 = blockIdx.x * kUpdTile, n0 = blockIdx.y * kUpdTile;
    if (lower && m0 + kUpdTile <= n0) return;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    const int lr = tid & 63, lk = tid >> 6;
    for (int k0 = 0; k0 < k; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int kk = lk + 4 * q, kg = k0 + kk;
            const int ra = m0 + lr, rb = n0 + lr;
            As[kk][lr] = (kg < k && ra < m) ? A[ra + (int64_t)kg * lda] : 0.0;
            Bs[kk][lr] = (kg < k && rb < nb) ? A[rb + (int64_t)kg * lda] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = m0 + tx + 16 * a;
        if (i >= m) continue;
        const int64_t r = rowmap[i];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = n0 + ty + 16 * b;
            if (j >= nb || (lower && i < j)) continue;
            atomicAdd(C + r + (int64_t)colmap[j] * ldc, -acc[a][b]);
        }
    }
}

void launch_update_standalone(int64_t m, int64_t nb, int64_t k, const double *A, int64_t lda,
                              double *C, int64_t ldc, const int32_t *rowmap,
                              const int32_t *colmap, int lower, cudaStream_t s)
{
    dim3 grid((unsigned)((m + kUpdTile - 1) / kUpdTile), (unsigned)((nb + kUpdTile - 1) / kUpdTile));
    if (grid.x == 0 || grid.y == 0) return;
    update_standalone_kernel<<<grid, 256, 0, s>>>((int)m, (int)nb, (int)k, A, lda, C, ldc, rowmap,
                                                  colmap, lower);
}

// explicit instantiations
template void launch_assemble<double>(int64_t, const double *, const int64_t *, double *, double *, cudaStream_t);
template void launch_assemble<float>(int64_t, const double *, const int64_t *, float *, float *, cudaStream_t);
template void launch_potrf<double>(const DevPlan &, const int32_t *, int, double *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_potrf<float>(const DevPlan &, const int32_t *, int, float *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_getrf<double>(const DevPlan &, const int32_t *, int, double *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_getrf<float>(const DevPlan &, const int32_t *, int, float *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_trsm<double>(const DevPlan &, const RowChunk *, int, const double *, double *, int, cudaStream_t);
template void launch_trsm<float>(const DevPlan &, const RowChunk *, int, const float *, float *, int, cudaStream_t);
template void launch_update<double>(const DevPlan &, const DevTask *, const UpdTile *, int, const double *, const double *, double *, int, int, cudaStream_t);
template void launch_update<float>(const DevPlan &, const DevTask *, const UpdTile *, int, const float *, const float *, float *, int, int, cudaStream_t);

}  // namespace spx
