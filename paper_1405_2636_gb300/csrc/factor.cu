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
#include "blocks.cuh"

#include <cuda_bf16.h>
#include <algorithm>
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
// Packed copies of ranges of the panel storage (the parts of a subtree-to-rank
// partition): ranges[3 r .. 3 r + 2] = (offset in the storage, length, offset
// in the packed buffer).  mode 0: buf <- storage, 1: storage <- buf,
// 2: storage <- 0.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void pack_ranges_kernel(const int64_t *__restrict__ ranges, int nr, T *store, T *buf, int mode)
{
    for (int r = blockIdx.x; r < nr; r += gridDim.x) {
        const int64_t off = ranges[3 * r], len = ranges[3 * r + 1], pos = ranges[3 * r + 2];
        for (int64_t e = threadIdx.x; e < len; e += blockDim.x) {
            if (mode == 0) buf[pos + e] = store[off + e];
            else if (mode == 1) store[off + e] = buf[pos + e];
            else store[off + e] = (T)0;
        }
    }
}

template <typename T>
void launch_pack_ranges(const int64_t *ranges, int nr, T *store, T *buf, int mode, cudaStream_t s)
{
    if (nr <= 0) return;
    pack_ranges_kernel<T><<<nr < 152 * 8 ? nr : 152 * 8, 256, 0, s>>>(ranges, nr, store, buf, mode);
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
        const C xjj = unit ? (C)1 : rcp_newton(a[j + j * w]);
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
// Blocked right-looking Cholesky of the w x w block held in shared memory
// (double, column-major, leading dimension w).  Columns go in blocks of kDB:
// warp 0 factors the block column (warp-synchronous: pivot, scaling, the
// updates inside the block), then every warp applies the rank-kDB update to
// the trailing lower triangle.  Two block barriers per kDB columns.  A pivot
// that is not positive is reported (replace_tau <= 0: the smallest failing
// column goes to *err_col) or replaced by replace_tau and counted.
// ---------------------------------------------------------------------------
__device__ void chol_blocked(double *a, int w, double replace_tau, int64_t col0, int64_t *err_col,
                             unsigned long long *nrepl)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int kb = 0; kb < w; kb += kDB) {
        const int bw = min(kDB, w - kb);
        if (warp == 0) {
            for (int k = kb; k < kb + bw; ++k) {
                double d = a[k + k * w];
                const bool bad = !(d > 0.0);
                if (bad) {
                    if (lane == 0) {
                        if (replace_tau > 0.0) atomicAdd(nrepl, 1ull);
                        else atomicMin((long long *)err_col, (long long)(col0 + k));
                    }
                    d = replace_tau > 0.0 ? replace_tau : 1.0;
                }
                double inv;
                sqrt_rsqrt(d, &d, &inv);               // L(k,k) = sqrt(pivot), inv = 1 / L(k,k)
                __syncwarp();
                if (lane == 0) a[k + k * w] = d;
                for (int i = k + 1 + lane; i < w; i += 32) a[i + k * w] *= inv;
                __syncwarp();
                for (int j = k + 1; j < kb + bw; ++j) {
                    const double ljk = a[j + k * w];
                    for (int i = j + lane; i < w; i += 32) a[i + j * w] -= a[i + k * w] * ljk;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // rank-bw update; each thread carries two rows and two partial sums so
        // that four independent FP64 chains are in flight (dependent FP64
        // operations are far slower than independent ones on this part)
        for (int j = kb + bw + warp; j < w; j += nw) {
            double lj[kDB];
#pragma unroll
            for (int c = 0; c < kDB; ++c) lj[c] = c < bw ? a[j + (kb + c) * w] : 0.0;
            for (int i = j + lane; i < w; i += 64) {
                const int i2 = i + 32;
                const bool two = i2 < w;
                double x0 = a[i + j * w], x1 = 0.0;
                double y0 = two ? a[i2 + j * w] : 0.0, y1 = 0.0;
#pragma unroll
                for (int c = 0; c < kDB; c += 2) {
                    if (c < bw) {
                        x0 -= a[i + (kb + c) * w] * lj[c];
                        if (two) y0 -= a[i2 + (kb + c) * w] * lj[c];
                    }
                    if (c + 1 < bw) {
                        x1 -= a[i + (kb + c + 1) * w] * lj[c + 1];
                        if (two) y1 -= a[i2 + (kb + c + 1) * w] * lj[c + 1];
                    }
                }
                a[i + j * w] = x0 + x1;
                if (two) a[i2 + j * w] = y0 + y1;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Register-resident variant for w <= 64 (leading dimension ld >= w).  Block
// columns of kDB: warp 0 holds the block panel (rows kb..w-1, two rows per
// lane) in registers and factors it with shuffles; then thread t keeps the
// block values of its two trailing rows in registers and updates the
// columns of its warp (j = kb + kDB + warp, + nw, ...), lower part only.
// ---------------------------------------------------------------------------

__device__ void chol_reg64(double *a, int w, int ld, double replace_tau, int64_t col0,
                           int64_t *err_col, unsigned long long *nrepl)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int kb = 0; kb < w; kb += kDB) {
        const int bw = min(kDB, w - kb);
        if (warp == 0) {
            const int r0 = kb + lane, r1 = kb + lane + 32;
            const bool h0 = r0 < w, h1 = r1 < w;
            double p0[kDB], p1[kDB];
#pragma unroll
            for (int c = 0; c < kDB; ++c) {
                p0[c] = (h0 && c < bw) ? a[r0 + (kb + c) * ld] : 0.0;
                p1[c] = (h1 && c < bw) ? a[r1 + (kb + c) * ld] : 0.0;
            }
#pragma unroll
            for (int c = 0; c < kDB; ++c) {
                if (c < bw) {
                    const int k = kb + c;
                    double d = shfl_d(p0[c], c);        // A(k, k): row k is lane c's r0
                    if (!(d > 0.0)) {
                        if (lane == 0) {
                            if (replace_tau > 0.0) atomicAdd(nrepl, 1ull);
                            else atomicMin((long long *)err_col, (long long)(col0 + k));
                        }
                        d = replace_tau > 0.0 ? replace_tau : 1.0;
                    }
                    double sq, rs;
                    sqrt_rsqrt(d, &sq, &rs);
                    p0[c] = (r0 > k) ? p0[c] * rs : (r0 == k ? sq : p0[c]);
                    p1[c] *= rs;
#pragma unroll
                    for (int c2 = c + 1; c2 < kDB; ++c2) {
                        if (c2 < bw) {
                            const double lj = shfl_d(p0[c], c2);   // L(kb + c2, k)
                            if (r0 >= kb + c2) p0[c2] -= p0[c] * lj;
                            p1[c2] -= p1[c] * lj;
                        }
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < kDB; ++c) {
                if (c < bw) {
                    if (h0) a[r0 + (kb + c) * ld] = p0[c];
                    if (h1) a[r1 + (kb + c) * ld] = p1[c];
                }
            }
        }
        __syncthreads();
        const int j0 = kb + bw;
        if (j0 < w) {
            // this thread's rows and their block values
            const int i0 = j0 + lane, i1 = j0 + lane + 32;
            const bool g0 = i0 < w, g1 = i1 < w;
            double li0[kDB], li1[kDB];
#pragma unroll
            for (int c = 0; c < kDB; ++c) {
                li0[c] = (g0 && c < bw) ? a[i0 + (kb + c) * ld] : 0.0;
                li1[c] = (g1 && c < bw) ? a[i1 + (kb + c) * ld] : 0.0;
            }
            for (int j = j0 + warp; j < w; j += nw) {
                double lj[kDB];
#pragma unroll
                for (int c = 0; c < kDB; ++c) lj[c] = c < bw ? a[j + (kb + c) * ld] : 0.0;
                double x0 = 0.0, y0 = 0.0, x1 = 0.0, y1 = 0.0;
#pragma unroll
                for (int c = 0; c < kDB; c += 2) {
                    x0 += li0[c] * lj[c];
                    y0 += li0[c + 1] * lj[c + 1];
                    x1 += li1[c] * lj[c];
                    y1 += li1[c + 1] * lj[c + 1];
                }
                if (g0 && i0 >= j) a[i0 + j * ld] -= x0 + y0;
                if (g1 && i1 >= j) a[i1 + j * ld] -= x1 + y1;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Blocked inversion X = L^{-1} in place (lower triangular, non-unit, column-
// major leading dimension w) by block rows of kDB, top to bottom:
//   T(I, J)  = sum_{K = J..I-1} L(I, K) X(K, J)       (all J < I in parallel)
//   X(I, I)  = L(I, I)^{-1}                            (warp 0, by columns)
//   X(I, J)  = -X(I, I) T(I, J)
// from L X = I.  tmp holds kDB * w + kDB * kDB elements of type C.
// ---------------------------------------------------------------------------
template <typename C>
__device__ void invert_lower_blocked(C *a, int w, C *tmp)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    C *Tb = tmp;                   // Tb[ii + j * kDB], j < r0
    C *Dt = tmp + kDB * w;         // Dt[ii + jj * kDB] = X(I, I)
    for (int r0 = 0; r0 < w; r0 += kDB) {
        const int bh = min(kDB, w - r0);
        for (int e = tid; e < bh * r0; e += nt) {
            const int ii = e % bh, j = e / bh;
            C s0 = (C)0, s1 = (C)0, s2 = (C)0, s3 = (C)0;   // four short chains
            int k = j;
            for (; k + 3 < r0; k += 4) {
                s0 += a[(r0 + ii) + k * w] * a[k + j * w];
                s1 += a[(r0 + ii) + (k + 1) * w] * a[(k + 1) + j * w];
                s2 += a[(r0 + ii) + (k + 2) * w] * a[(k + 2) + j * w];
                s3 += a[(r0 + ii) + (k + 3) * w] * a[(k + 3) + j * w];
            }
            for (; k < r0; ++k) s0 += a[(r0 + ii) + k * w] * a[k + j * w];
            Tb[ii + j * kDB] = (s0 + s1) + (s2 + s3);
        }
        if (warp == 0 && lane < bh) {
            // column jj = lane of the inverse of the bh x bh diagonal block, by a
            // column sweep: x = e_jj; for kk: x_kk /= L_kk; x_ii -= L_ii,kk x_kk
            const int jj = lane;
            C rd[kDB], x[kDB];
#pragma unroll
            for (int q = 0; q < kDB; ++q) {
                rd[q] = q < bh ? rcp_newton(a[(r0 + q) + (r0 + q) * w]) : (C)0;
                x[q] = q == jj ? (C)1 : (C)0;
            }
#pragma unroll
            for (int kk = 0; kk < kDB; ++kk) {
                if (kk < bh && kk >= jj) {
                    x[kk] *= rd[kk];
#pragma unroll
                    for (int ii = kk + 1; ii < kDB; ++ii)
                        if (ii < bh) x[ii] -= a[(r0 + ii) + (r0 + kk) * w] * x[kk];
                }
            }
#pragma unroll
            for (int q = 0; q < kDB; ++q)
                if (q < bh) Dt[q + jj * kDB] = x[q];
        }
        __syncthreads();
        for (int e = tid; e < bh * r0; e += nt) {
            const int ii = e % bh, j = e / bh;
            C acc = (C)0;
            for (int kk = 0; kk <= ii; ++kk) acc += Dt[ii + kk * kDB] * Tb[kk + j * kDB];
            a[(r0 + ii) + j * w] = -acc;
        }
        for (int e = tid; e < bh * bh; e += nt) {
            const int ii = e % bh, jj = e / bh;
            if (ii >= jj) a[(r0 + ii) + (r0 + jj) * w] = Dt[ii + jj * kDB];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Diagonal block, Cholesky (Sec. III step 1): one CTA per panel, the block in
// shared memory in double; then L_kk^{-1} (arithmetic of the factor's type)
// is stored at Dinv + pinv[panel] for the TRSM and the solves.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) potrf_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                    T *__restrict__ L, T *__restrict__ Dinv,
                                                    const double *replace_tau_p,
                                                    int64_t *err_col, unsigned long long *nrepl)
{
    extern __shared__ double sm[];
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
    if (w <= 64) chol_reg64(sm, w, w, replace_tau, p.pfcol[pid], err_col, nrepl);
    else chol_blocked(sm, w, replace_tau, p.pfcol[pid], err_col, nrepl);
    for (int idx = tid; idx < w * w; idx += nt) {
        int i = idx % w, j = idx / w;
        if (i >= j) D[i + (int64_t)j * h] = (T)sm[idx];
    }
    __syncthreads();
    T *a = narrow_inplace<T>(sm, w * w);
    invert_lower_blocked<T>(a, w, reinterpret_cast<T *>(sm + (size_t)w * w));
    T *Mi = Dinv + p.pinv[pid];
    for (int idx = tid; idx < w * w; idx += nt) Mi[idx] = a[idx];
}

// The diagonal blocks of one width class, one CTA per panel.
template <typename T, int W, bool ldlt>
__global__ void __launch_bounds__(256) potrf_ldl_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                        T *__restrict__ L, T *__restrict__ Dinv,
                                                        const double *replace_tau_p,
                                                        int64_t *err_col, unsigned long long *nrepl,
                                                        unsigned long long *nneg)
{
    extern __shared__ double sm[];
    ldl_diag_block<T, W, ldlt>(p, panels[blockIdx.x], L, Dinv, *replace_tau_p, err_col, nrepl, nneg, sm);
}

template <typename T, int W, bool ldlt = false>
void launch_ldl(const DevPlan &p, const int32_t *panels, int count, T *L, T *Dinv,
                const double *replace_tau, int64_t *err_col, unsigned long long *nrepl, cudaStream_t s,
                unsigned long long *nneg = nullptr)
{
    static bool once = false;
    const size_t smem = ldl_smem_bytes<T, W>();
    if (!once) {
        cudaFuncSetAttribute(potrf_ldl_kernel<T, W, ldlt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        once = true;
    }
    potrf_ldl_kernel<T, W, ldlt><<<count, 256, smem, s>>>(p, panels, L, Dinv, replace_tau, err_col, nrepl, nneg);
}

// LDL^T diagonal blocks (panels at most 64 wide): l with d on the diagonal,
// l^{-1} with 1/d on its diagonal at Dinv; static pivoting with threshold
// *tau (<= 0: a zero pivot is an error); negative pivots counted in *nneg.
template <typename T>
void launch_ldlt_diag(const DevPlan &p, const int32_t *panels, int count, int wmax, T *L, T *Dinv,
                      const double *tau, int64_t *err_col, unsigned long long *nrepl,
                      unsigned long long *nneg, cudaStream_t s)
{
    if (count <= 0) return;
    if (wmax <= 16) return launch_ldl<T, 16, true>(p, panels, count, L, Dinv, tau, err_col, nrepl, s, nneg);
    if (wmax <= 32) return launch_ldl<T, 32, true>(p, panels, count, L, Dinv, tau, err_col, nrepl, s, nneg);
    launch_ldl<T, 64, true>(p, panels, count, L, Dinv, tau, err_col, nrepl, s, nneg);
}

template <typename T>
void launch_potrf(const DevPlan &p, const int32_t *panels, int count, int wmax, int threads, T *L, T *Dinv,
                  const double *replace_tau, int64_t *err_col, unsigned long long *nrepl,
                  cudaStream_t s)
{
    if (count <= 0) return;
    if (wmax <= 16) return launch_ldl<T, 16>(p, panels, count, L, Dinv, replace_tau, err_col, nrepl, s);
    if (wmax <= 32) return launch_ldl<T, 32>(p, panels, count, L, Dinv, replace_tau, err_col, nrepl, s);
    if (wmax <= 64) return launch_ldl<T, 64>(p, panels, count, L, Dinv, replace_tau, err_col, nrepl, s);
    (void)threads;
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(potrf_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (kMaxWidth * kMaxWidth + kDB * kMaxWidth + kDB * kDB)));
        once = true;
    }
    const size_t smem = sizeof(double) * ((size_t)wmax * wmax + kDB * wmax + kDB * kDB);
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
            s_inv = rcp_newton(d);
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

template <typename T>
__global__ void __launch_bounds__(256) trsm_gemm_kernel(DevPlan p, const RowChunk *__restrict__ chunks,
                                                        const T *__restrict__ Dinv,
                                                        T *__restrict__ X, int mode, void *opc,
                                                        void *opc_lo, int kpad, int op_kind,
                                                        T *__restrict__ Wout)
{
    extern __shared__ unsigned char smraw[];
    trsm_chunk<T>(p, chunks[blockIdx.x], Dinv, X, mode, opc, opc_lo, kpad, op_kind, Wout, smraw);
}

template <typename T>
void launch_trsm(const DevPlan &p, const RowChunk *chunks, int count, int wmax, const T *Dinv,
                 T *X, int mode, void *opc, void *opc_lo, int kpad, int op_kind, cudaStream_t s, T *Wout)
{
    if (count <= 0) return;
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(trsm_gemm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)trsm_smem_bytes<T>((kMaxWidth + 15) & ~15));
        once = true;
    }
    const size_t smem = trsm_smem_bytes<T>((wmax + 15) & ~15);
    trsm_gemm_kernel<T><<<count, 256, smem, s>>>(p, chunks, Dinv, X, mode, opc, opc_lo, kpad, op_kind, Wout);
}

// Look-ahead step of a chain link (Sec. III's task order, with the next
// diagonal block first): panel p's single level is followed by a single
// panel q whose columns are p's first 64 off-diagonal rows.  One CTA solves
// those rows against p's inverted diagonal block (chunk 0 of p's TRSM, with
// its operand copy) and subtracts their product L_qp L_qp^T from q's diagonal
// block (the lower triangle, in the factor's arithmetic on the CUDA cores,
// with reductions like every update).  q's diagonal block then needs
// nothing else from p, so it is factored right after this step while p's
// other TRSM chunks and update tiles run beside it.
template <typename T>
__global__ void __launch_bounds__(256) lead_kernel(DevPlan p, RowChunk ch, const DevTask *__restrict__ tasks,
                                                   int32_t task, const T *__restrict__ Dinv, T *__restrict__ L,
                                                   void *opc, void *opc_lo, int kpad, int op_kind)
{
    extern __shared__ unsigned char smraw[];
    trsm_chunk<T>(p, ch, Dinv, L, TRSM_LLT, opc, opc_lo, kpad, op_kind, nullptr, smraw);
    __syncthreads();   // the chunk's rows, written above, are read back through L2
    const DevTask tk = tasks[task];
    update_tile<T, kUpdTile>(p, tk, UpdTile{task, tk.r0, tk.r0, 0}, L, L, L, 1, 0, reinterpret_cast<T *>(smraw));
}

template <typename T>
void launch_lead(const DevPlan &p, RowChunk ch, const DevTask *tasks, int32_t task, const T *Dinv, T *L,
                 void *opc, void *opc_lo, int kpad, int op_kind, cudaStream_t s)
{
    const size_t smem = std::max(trsm_smem_bytes<T>(kUpdTile), update_smem_elems<T, kUpdTile>() * sizeof(T));
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(lead_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        once = true;
    }
    lead_kernel<T><<<1, 256, smem, s>>>(p, ch, tasks, task, Dinv, L, opc, opc_lo, kpad, op_kind);
}

template <typename T, int TN>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 1) update_kernel(DevPlan p, const DevTask *__restrict__ tasks,
                                                     const UpdTile *__restrict__ tiles,
                                                     const T *__restrict__ Aop,
                                                     const T *__restrict__ Bop, T *__restrict__ C,
                                                     int lower, int from_r1)
{
    __shared__ T smem[update_smem_elems<T, TN>()];
    const UpdTile tl = tiles[blockIdx.x];
    update_tile<T, TN>(p, tasks[tl.task], tl, Aop, Bop, C, lower, from_r1, smem);
}

template <typename T>
void launch_update(const DevPlan &p, const DevTask *tasks, const UpdTile *tiles, int count,
                   const T *Aop, const T *Bop, T *C, int lower, int from_r1, cudaStream_t s, int narrow)
{
    if (count <= 0) return;
    if (narrow) update_kernel<T, 16><<<count, 256, 0, s>>>(p, tasks, tiles, Aop, Bop, C, lower, from_r1);
    else update_kernel<T, 64><<<count, 256, 0, s>>>(p, tasks, tiles, Aop, Bop, C, lower, from_r1);
}

// explicit instantiations
template void launch_pack_ranges<double>(const int64_t *, int, double *, double *, int, cudaStream_t);
template void launch_pack_ranges<float>(const int64_t *, int, float *, float *, int, cudaStream_t);
template void launch_assemble<double>(int64_t, const double *, const int64_t *, double *, double *, cudaStream_t);
template void launch_assemble<float>(int64_t, const double *, const int64_t *, float *, float *, cudaStream_t);
template void launch_potrf<double>(const DevPlan &, const int32_t *, int, int, int, double *, double *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_potrf<float>(const DevPlan &, const int32_t *, int, int, int, float *, float *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_getrf<double>(const DevPlan &, const int32_t *, int, int, int, double *, double *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_getrf<float>(const DevPlan &, const int32_t *, int, int, int, float *, float *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_trsm<double>(const DevPlan &, const RowChunk *, int, int, const double *, double *, int, void *, void *, int, int, cudaStream_t, double *);
template void launch_lead<float>(const DevPlan &, RowChunk, const DevTask *, int32_t, const float *, float *, void *, void *, int, int, cudaStream_t);
template void launch_ldlt_diag<double>(const DevPlan &, const int32_t *, int, int, double *, double *, const double *, int64_t *, unsigned long long *, unsigned long long *, cudaStream_t);
template void launch_trsm<float>(const DevPlan &, const RowChunk *, int, int, const float *, float *, int, void *, void *, int, int, cudaStream_t, float *);
template void launch_ldlt_diag<float>(const DevPlan &, const int32_t *, int, int, float *, float *, const double *, int64_t *, unsigned long long *, unsigned long long *, cudaStream_t);
template void launch_update<double>(const DevPlan &, const DevTask *, const UpdTile *, int, const double *, const double *, double *, int, int, cudaStream_t, int);
template void launch_update<float>(const DevPlan &, const DevTask *, const UpdTile *, int, const float *, const float *, float *, int, int, cudaStream_t, int);

}  // namespace spx
