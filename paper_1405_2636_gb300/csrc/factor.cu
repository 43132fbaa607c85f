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

#include <cuda_bf16.h>
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
// In-place inversion of a lower-triangular w x w block held in shared memory
// (column-major, leading dimension w), read through element (i, j) at
// a[trans ? j + i*w : i + j*w].  Columns are taken from the right:
//   X(j,j) = 1 / L(j,j)   (1 when unit),
//   X(i,j) = -(sum_{k=j+1..i} X(i,k) L(k,j)) X(j,j)   for i > j,
// using the already inverted columns k > j (from X L = I).  With trans the
// same routine inverts U^T, i.e. writes U^{-1} in the upper triangle.  C is
// the storage and arithmetic type; `col` is w elements of scratch.
// ---------------------------------------------------------------------------
template <typename C>
__device__ void invert_lower_inplace(C *a, int w, bool trans, bool unit, C *col)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = w - 1; j >= 0; --j) {
        for (int i = j + 1 + tid; i < w; i += nt) col[i] = a[trans ? j + i * w : i + j * w];
        __syncthreads();
        const C xjj = unit ? (C)1 : (C)1 / a[j + j * w];
        for (int i = j + 1 + tid; i < w; i += nt) {
            const C xii = unit ? (C)1 : a[i + i * w];
            C s = xii * col[i];
            for (int k = j + 1; k < i; ++k) s += a[trans ? k + i * w : i + k * w] * col[k];
            a[trans ? j + i * w : i + j * w] = -s * xjj;
        }
        __syncthreads();
        if (tid == 0 && !unit) a[j + j * w] = xjj;
        __syncthreads();
    }
}

// Narrow the w*w doubles at sm to T in place (T = float: the floats land in
// the first half of the same buffer; rounds of blockDim elements are read
// before any of them is written, so no live double is overwritten).
template <typename T>
__device__ T *narrow_inplace(double *sm, int count)
{
    if (sizeof(T) == sizeof(double)) return reinterpret_cast<T *>(sm);
    T *out = reinterpret_cast<T *>(sm);
    for (int base = 0; base < count; base += blockDim.x) {
        const int idx = base + threadIdx.x;
        const double v = idx < count ? sm[idx] : 0.0;
        __syncthreads();
        if (idx < count) out[idx] = (T)v;
        __syncthreads();
    }
    return out;
}

// ---------------------------------------------------------------------------
// Diagonal block, Cholesky (Sec. III step 1): one CTA per panel, the block in
// shared memory in double, right-looking by columns.  A pivot that is not
// positive is either reported (replace_tau <= 0: the smallest failing column
// goes to *err_col) or replaced by replace_tau and counted.  The CTA then
// inverts L_kk in place (arithmetic of the factor's type) and stores the
// inverse at Dinv + pinv[panel]; the TRSM and the solves multiply by it.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) potrf_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                    T *__restrict__ L, T *__restrict__ Dinv,
                                                    const double *replace_tau_p,
                                                    int64_t *err_col, unsigned long long *nrepl)
{
    extern __shared__ double sm[];
    __shared__ double s_piv, s_inv;
    const double replace_tau = *replace_tau_p;
    const int pid = panels[blockIdx.x];
    const int w = p.pw[pid], h = p.ph[pid];
    T *D = L + p.pval[pid];
    double *col = sm + w * w;
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
            s_inv = 1.0 / d;
        }
        __syncthreads();
        const double inv = s_inv;
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
    __syncthreads();
    T *a = narrow_inplace<T>(sm, w * w);
    invert_lower_inplace<T>(a, w, false, false, reinterpret_cast<T *>(col));
    T *Mi = Dinv + p.pinv[pid];
    for (int idx = tid; idx < w * w; idx += nt) Mi[idx] = a[idx];
}

template <typename T>
void launch_potrf(const DevPlan &p, const int32_t *panels, int count, int wmax, int threads, T *L, T *Dinv,
                  const double *replace_tau, int64_t *err_col, unsigned long long *nrepl,
                  cudaStream_t s)
{
    if (count <= 0) return;
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(potrf_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (kMaxWidth * kMaxWidth + kMaxWidth)));
        once = true;
    }
    const size_t smem = sizeof(double) * ((size_t)wmax * wmax + wmax);
    potrf_kernel<T><<<count, threads, smem, s>>>(p, panels, L, Dinv, replace_tau, err_col, nrepl);
}

// ---------------------------------------------------------------------------
// Diagonal block, LU without pivoting (Sec. III: static pivoting): a pivot
// whose magnitude is below tau becomes sign(pivot) * tau (+tau for 0) and is
// counted; tau <= 0 turns a zero pivot into an error instead.  The inverses
// of the unit lower and the upper factor are stored together at Dinv (L^{-1}
// strictly below the diagonal, U^{-1} on and above it).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) getrf_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                    T *__restrict__ L, T *__restrict__ Dinv,
                                                    const double *tau_p, int64_t *err_col,
                                                    unsigned long long *nrepl)
{
    extern __shared__ double sm[];
    __shared__ double s_inv;
    const double tau = *tau_p;
    const int pid = panels[blockIdx.x];
    const int w = p.pw[pid], h = p.ph[pid];
    T *D = L + p.pval[pid];
    double *col = sm + w * w;
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
            s_inv = 1.0 / d;
        }
        __syncthreads();
        const double inv = s_inv;
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
    __syncthreads();
    T *a = narrow_inplace<T>(sm, w * w);
    invert_lower_inplace<T>(a, w, false, true, reinterpret_cast<T *>(col));   // unit lower L
    invert_lower_inplace<T>(a, w, true, false, reinterpret_cast<T *>(col));   // U through U^T
    T *Mi = Dinv + p.pinv[pid];
    for (int idx = tid; idx < w * w; idx += nt) Mi[idx] = a[idx];
}

template <typename T>
void launch_getrf(const DevPlan &p, const int32_t *panels, int count, int wmax, int threads, T *L, T *Dinv,
                  const double *tau, int64_t *err_col, unsigned long long *nrepl, cudaStream_t s)
{
    if (count <= 0) return;
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(getrf_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (kMaxWidth * kMaxWidth + kMaxWidth)));
        once = true;
    }
    const size_t smem = sizeof(double) * ((size_t)wmax * wmax + wmax);
    getrf_kernel<T><<<count, threads, smem, s>>>(p, panels, L, Dinv, tau, err_col, nrepl);
}

// ---------------------------------------------------------------------------
// Panel TRSM (Sec. III step 2) as a product with the inverted diagonal block:
// rows [r0, r0+64) of the off-diagonal part X become X B with
//   LLT : B = L^{-T}           (B(k,j) = Linv(j,k))
//   LU_L: B = U^{-1}           (B(k,j) = Uinv(k,j))
//   LU_U: B = L^{-T}, unit L   (B(k,j) = Linv(j,k), 1 on the diagonal)
// The CTA copies its rows to shared memory first, so writing them back in
// place is safe; 64 x 64 output tiles, 4 x 4 per thread, K-chunks of 16.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float round_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <typename T>
__global__ void __launch_bounds__(256) trsm_gemm_kernel(DevPlan p, const RowChunk *__restrict__ chunks,
                                                        const T *__restrict__ Dinv,
                                                        T *__restrict__ X, int mode, void *opc,
                                                        int kpad, int op_bf16)
{
    extern __shared__ unsigned char smraw[];
    T *Xs = reinterpret_cast<T *>(smraw);      // Xs[k * 64 + r], k < wpad
    __shared__ T Bs[16][kUpdTile + 1];
    const RowChunk ch = chunks[blockIdx.x];
    const int pid = ch.panel;
    const int w = p.pw[pid], h = p.ph[pid];
    const int wpad = (w + 15) & ~15;
    const T *Mi = Dinv + p.pinv[pid];
    T *Xg = X + p.pval[pid] + ch.r0;
    const int nr = min(kTrsmRows, h - ch.r0);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int e = tid; e < wpad * kTrsmRows; e += 256) {
        const int r = e & 63, k = e >> 6;
        Xs[e] = (r < nr && k < w) ? Xg[r + (int64_t)k * h] : (T)0;
    }
    __syncthreads();
    for (int c0 = 0; c0 < w; c0 += kUpdTile) {
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
        for (int k0 = 0; k0 < wpad; k0 += 16) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = tid + 256 * q;
                const int kk = e >> 6, jj = e & 63;
                const int k = k0 + kk, j = c0 + jj;
                T v = (T)0;
                if (k < w && j < w) {
                    if (mode == TRSM_LU_L) v = (k <= j) ? Mi[k + j * w] : (T)0;
                    else if (j > k) v = Mi[j + k * w];
                    else if (j == k) v = (mode == TRSM_LU_U) ? (T)1 : Mi[j + k * w];
                }
                Bs[kk][jj] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                T av[4], bv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) av[a] = Xs[(k0 + kk) * 64 + tx + 16 * a];
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
            const int r = tx + 16 * a;
            if (r >= nr) continue;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int j = c0 + ty + 16 * b;
                if (j < w) Xg[r + (int64_t)j * h] = acc[a][b];
            }
        }
        if (opc) {
            // the same rows, K-major, for the tensor-core updates
            const int64_t orow0 = p.prow[pid] + ch.r0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int r = tx + 16 * a;
                if (r >= nr) continue;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int j = c0 + ty + 16 * b;
                    if (j >= w) continue;
                    const int64_t o = (orow0 + r) * kpad + j;
                    if (op_bf16) reinterpret_cast<__nv_bfloat16 *>(opc)[o] = __float2bfloat16((float)acc[a][b]);
                    else reinterpret_cast<float *>(opc)[o] = round_tf32((float)acc[a][b]);
                }
            }
        }
    }
    if (opc) {
        const int64_t orow0 = p.prow[pid] + ch.r0;
        const int padw = kpad - w;
        for (int e = tid; e < nr * padw; e += 256) {
            const int r = e / padw, j = w + e % padw;
            const int64_t o = (orow0 + r) * kpad + j;
            if (op_bf16) reinterpret_cast<__nv_bfloat16 *>(opc)[o] = __float2bfloat16(0.0f);
            else reinterpret_cast<float *>(opc)[o] = 0.0f;
        }
    }
}

template <typename T>
void launch_trsm(const DevPlan &p, const RowChunk *chunks, int count, int wmax, const T *Dinv,
                 T *X, int mode, void *opc, int kpad, int op_bf16, cudaStream_t s)
{
    if (count <= 0) return;
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(trsm_gemm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(T) * kMaxWidth * kTrsmRows));
        once = true;
    }
    const size_t smem = sizeof(T) * (size_t)((wmax + 15) & ~15) * kTrsmRows;
    trsm_gemm_kernel<T><<<count, 256, smem, s>>>(p, chunks, Dinv, X, mode, opc, kpad, op_bf16);
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
template void launch_potrf<double>(const DevPlan &, const int32_t *, int, int, int, double *, double *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_potrf<float>(const DevPlan &, const int32_t *, int, int, int, float *, float *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_getrf<double>(const DevPlan &, const int32_t *, int, int, int, double *, double *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_getrf<float>(const DevPlan &, const int32_t *, int, int, int, float *, float *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_trsm<double>(const DevPlan &, const RowChunk *, int, int, const double *, double *, int, void *, int, int, cudaStream_t);
template void launch_trsm<float>(const DevPlan &, const RowChunk *, int, int, const float *, float *, int, void *, int, int, cudaStream_t);
template void launch_update<double>(const DevPlan &, const DevTask *, const UpdTile *, int, const double *, const double *, double *, int, int, cudaStream_t);
template void launch_update<float>(const DevPlan &, const DevTask *, const UpdTile *, int, const float *, const float *, float *, int, int, cudaStream_t);

}  // namespace spx
