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
#include "operand.cuh"

#include <cuda_bf16.h>
#include <cstdio>

namespace spx {

// ---------------------------------------------------------------------------
// Pivot arithmetic in FP64 with short dependency chains.  IEEE FP64 division
// and square root expand into long chains of dependent FP64 instructions, and
// a dependent FP64 instruction costs tens of times its throughput slot on
// this part, so the column-by-column pivots would dominate the diagonal
// kernels.  Instead:
//  * a float seed is cut from the double's bits with integer operations (no
//    FP64 conversion), refined by the FP32 unit (rsqrtf / reciprocal) and
//    widened back the same way;
//  * reciprocal: Newton's method on 1/y - d, written with the error term
//    e = 1 - d y so that two steps need three dependent FP64 operations
//    (y1 = y0 + y0 e, e1 = e^2, y2 = y1 + y1 e1);
//  * square root and its reciprocal together: Goldschmidt's iteration
//    (g -> sqrt(d), h -> 1/(2 sqrt(d)); r = 1/2 - g h; g += g r; h += h r),
//    two iterations, five dependent FP64 operations.
// Each iteration squares the relative error: 2^-22 -> 2^-44 -> below FP64
// rounding.  Magnitudes outside the FP32 normal range fall back to IEEE.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool float_seed(double d, float *f)
{
    const long long b = __double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e < -125 || e > 126) return false;
    const unsigned fb = (unsigned)((b >> 32) & 0x80000000u) | ((unsigned)(e + 127) << 23) |
                        (unsigned)((b >> 29) & 0x7FFFFF);
    *f = __uint_as_float(fb);
    return true;
}

__device__ __forceinline__ double widen(float f)
{
    const unsigned u = __float_as_uint(f);
    const int e = (int)((u >> 23) & 0xFF) - 127;
    const long long b = ((long long)(u & 0x80000000u) << 32) | ((long long)(e + 1023) << 52) |
                        ((long long)(u & 0x7FFFFF) << 29);
    return __longlong_as_double(b);
}

__device__ __forceinline__ double rcp_newton(double d)
{
    float f;
    if (!float_seed(d, &f)) return 1.0 / d;
    const float yf = 1.0f / f;
    if (!(fabsf(yf) > 1e-37f && fabsf(yf) < 1e37f)) return 1.0 / d;
    const double y0 = widen(yf);
    const double e0 = fma(-d, y0, 1.0);
    const double y1 = fma(y0, e0, y0);
    const double e1 = e0 * e0;
    return fma(y1, e1, y1);
}

// sqrt(d) and 1/sqrt(d) for d > 0.
__device__ __forceinline__ void sqrt_rsqrt(double d, double *s, double *rs)
{
    float f;
    if (d <= 0.0 || !float_seed(d, &f)) {
        *s = sqrt(d);
        *rs = 1.0 / *s;
        return;
    }
    const double y = widen(rsqrtf(f));
    double g = d * y, h = 0.5 * y;
    double r = fma(-g, h, 0.5);
    g = fma(g, r, g);
    h = fma(h, r, h);
    r = fma(-g, h, 0.5);
    g = fma(g, r, g);
    h = fma(h, r, h);
    *s = g;
    *rs = 2.0 * h;
}

__device__ __forceinline__ float rcp_newton(float d) { return 1.0f / d; }


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
constexpr int kDB = 8;

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
__device__ __forceinline__ double shfl_d(double v, int src)
{
    return __shfl_sync(0xffffffffu, v, src);
}

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

// ---------------------------------------------------------------------------
// Diagonal block of width <= W (W = 16, 32, 64; the block is padded with the
// identity to W).  A dependent FP64 operation costs ~64 cycles on this part,
// so the column chain is kept short:
//  * the factorization runs in LDL^T form in FP64 -- per column one Newton
//    reciprocal of the pivot, the multipliers, and the in-block updates,
//    with no square root on the chain; warps 0 and 1 own each 8-column
//    block panel in registers (rows 0-31 and 32-63 of the block; each warp
//    runs the pivot chain itself), the other warps apply the trailing updates;
//  * L = l diag(sqrt(d)) is formed afterwards, all columns in parallel;
//  * L^{-1} = diag(1/sqrt(d)) l^{-1}: the unit-lower l is inverted by blocks
//    (8 x 8 diagonal blocks by single lanes, then pairs of blocks merged with
//    X21 = -C^{-1} (B A^{-1})), in the factor's arithmetic.
// ---------------------------------------------------------------------------
template <typename T, int W, bool ldlt>
__global__ void __launch_bounds__(256) potrf_ldl_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                        T *__restrict__ L, T *__restrict__ Dinv,
                                                        const double *replace_tau_p,
                                                        int64_t *err_col, unsigned long long *nrepl,
                                                        unsigned long long *nneg)
{
    constexpr int LD = W + 1;
    constexpr int NT = 256;
    extern __shared__ double sm[];
    double *a = sm;                          // W x LD, FP64 working block
    double *lA = a + W * LD;                 // 2 x (W x kDB) unscaled block columns (ld W)
    double *dv = lA + 2 * W * kDB;           // pivots
    double *rsv = dv + W;                    // 1 / sqrt(pivot)
    T *x = reinterpret_cast<T *>(rsv + W);   // W x LD inverse workspace
    T *tmp = x + W * LD;                     // (W/2)^2
    const double replace_tau = *replace_tau_p;
    const int pid = panels[blockIdx.x];
    const int w = p.pw[pid], h = p.ph[pid];
    const int64_t col0 = p.pfcol[pid];
    T *D = L + p.pval[pid];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // the block, padded with the identity to W: every load of a thread is
    // issued before its first store, so the loads overlap
    {
        constexpr int NPER = (W * W + NT - 1) / NT;
        T vv[NPER];
#pragma unroll
        for (int q = 0; q < NPER; ++q) {
            const int idx = tid + q * NT;
            const int i = idx % W, j = idx / W;
            vv[q] = (idx < W * W && i < w && j < w && i >= j) ? D[i + (int64_t)j * h] : (T)0;
        }
#pragma unroll
        for (int q = 0; q < NPER; ++q) {
            const int idx = tid + q * NT;
            if (idx >= W * W) continue;
            const int i = idx % W, j = idx / W;
            a[i + j * LD] = (i < w && j < w) ? (double)vv[q] : (i == j ? 1.0 : 0.0);
        }
    }
    __syncthreads();

    // Block panel b by warp 0 (registers, two row sets of 32), writing the
    // multipliers into a and the unscaled block columns into lA (two buffers,
    // one per block parity, so that the next panel can overlap the trailing
    // update of the previous one).
    // Block panel kb (8 columns), rows in registers, by one warp per row set:
    //   role 0 (warp 0): rows kb .. kb+31, the pivots and their side effects;
    //   role 1 (warp 1, when rows kb+32.. exist): rows kb+32 .. kb+63.
    // Warp 1 recomputes the 8 x 8 diagonal part from its own copy of rows
    // kb .. kb+7 (lane l holds row kb + (l & 7)) with the same operations in
    // the same order as warp 0, so its pivots and multipliers are bit-equal
    // and the two warps never wait for each other.  Multipliers go to a, the
    // unscaled block columns to lA (two buffers, one per block parity, so
    // that the next panel can overlap the trailing update of the previous).
    auto panel = [&](int kb, int role) {
        double *lAb = lA + ((kb / kDB) & 1) * (W * kDB);
        const int rq = role == 0 ? kb + lane : kb + (lane & 7);   // rows of the pivot chain
        const int r1 = kb + 32 + lane;                            // role 1: its own rows
        double q[kDB], p1[kDB];
#pragma unroll
        for (int c = 0; c < kDB; ++c) {
            q[c] = rq < W ? a[rq + (kb + c) * LD] : 0.0;
            p1[c] = (role == 1 && r1 < W) ? a[r1 + (kb + c) * LD] : 0.0;
        }
#pragma unroll
        for (int c = 0; c < kDB; ++c) {
            const int k = kb + c;
            double d = shfl_d(q[c], c);                  // A(k, k) from lane c
            const bool report = role == 0 && lane == 0 && k < w;
            if constexpr (!ldlt) {                        // Cholesky: positive pivots
                if (!(d > 0.0)) {
                    if (report) {
                        if (replace_tau > 0.0) atomicAdd(nrepl, 1ull);
                        else atomicMin((long long *)err_col, (long long)(col0 + k));
                    }
                    d = replace_tau > 0.0 ? replace_tau : 1.0;
                }
            } else {                                      // LDL^T: static pivoting
                if (!(fabs(d) >= replace_tau) || (replace_tau <= 0.0 && d == 0.0)) {
                    if (report) {
                        if (replace_tau > 0.0) atomicAdd(nrepl, 1ull);
                        else atomicMin((long long *)err_col, (long long)(col0 + k));
                    }
                    d = replace_tau > 0.0 ? (d < 0.0 ? -replace_tau : replace_tau) : 1.0;
                }
                if (report && d < 0.0) atomicAdd(nneg, 1ull);
            }
            const double r = 1.0 / d;   // measured faster here than the Newton form
            const double u0 = rq > k ? q[c] : 0.0;
            const double l0 = u0 * r;
#pragma unroll
            for (int c2 = c + 1; c2 < kDB; ++c2) {
                const double ac = shfl_d(u0, c2);                   // A(kb + c2, k)
                if (rq >= kb + c2) q[c2] = fma(-l0, ac, q[c2]);
                if (role == 1) p1[c2] = fma(-(p1[c] * r), ac, p1[c2]);
            }
            if (role == 0) {
                if (rq < W) lAb[rq + c * W] = u0;
                q[c] = rq > k ? l0 : (rq == k ? 1.0 : 0.0);
                if (lane == c) dv[k] = d;
            } else {
                if (r1 < W) lAb[r1 + c * W] = p1[c];
                p1[c] = p1[c] * r;
            }
        }
#pragma unroll
        for (int c = 0; c < kDB; ++c) {
            if (role == 0 && rq < W) a[rq + (kb + c) * LD] = q[c];
            if (role == 1 && r1 < W) a[r1 + (kb + c) * LD] = p1[c];
        }
    };
    // Rank-kDB update by block kb of the lower part of columns [j0, j1),
    // rows >= j; the (i, j) pairs are spread densely over the threads
    // t0.. (stride ts) so that FP64 lanes are not wasted on the upper part.
    auto update = [&](int kb, int j0, int j1, int t0, int ts) {
        const double *lAb = lA + ((kb / kDB) & 1) * (W * kDB);
        // pairs ordered column by column: column j holds W - j rows
        int j = j0, rem = t0;      // pair e = t0, t0 + ts, ... decoded incrementally
        while (j < j1 && rem >= W - j) {
            rem -= W - j;
            ++j;
        }
        for (; j < j1;) {
            const int i = j + rem;
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int c = 0; c < kDB; c += 2) {
                s0 = fma(a[i + (kb + c) * LD], lAb[j + c * W], s0);
                s1 = fma(a[i + (kb + c + 1) * LD], lAb[j + (c + 1) * W], s1);
            }
            a[i + j * LD] -= s0 + s1;
            rem += ts;
            while (j < j1 && rem >= W - j) {
                rem -= W - j;
                ++j;
            }
        }
    };

    if (warp == 0) panel(0, 0);
    else if (warp == 1 && 32 < W) panel(0, 1);
    __syncthreads();
    for (int kb = 0; kb < W; kb += kDB) {
        const int nb = kb + kDB;                 // next block
        if (nb < W) {
            // columns of the next block first, by every thread
            update(kb, nb, nb + kDB, tid, NT);
            __syncthreads();
            // warps 0 (and 1) factor the next block while the others finish
            // this block's update
            const bool two = nb + 32 < W;
            if (warp == 0) panel(nb, 0);
            else if (warp == 1 && two) panel(nb, 1);
            else update(kb, nb + kDB, W, tid - (two ? 64 : 32), NT - (two ? 64 : 32));
            __syncthreads();
        }
    }

    // Cholesky: L = l diag(sqrt(d)), keep 1/sqrt(d) for the inverse.
    // LDL^T: store l (unit) with d on the diagonal, keep 1/d.
    if (tid < W) {
        if constexpr (ldlt) {
            rsv[tid] = rcp_newton(dv[tid]);
        } else {
            double sq, rs;
            sqrt_rsqrt(dv[tid], &sq, &rs);
            dv[tid] = sq;
            rsv[tid] = rs;
        }
    }
    __syncthreads();
    for (int idx = tid; idx < W * W; idx += NT) {
        const int i = idx % W, j = idx / W;
        const T l = (T)a[i + j * LD];
        if (i < w && j < w && i >= j)
            D[i + (int64_t)j * h] = i == j ? (T)dv[j] : (ldlt ? l : l * (T)dv[j]);
        x[i + j * LD] = i > j ? l : (i == j ? (T)1 : (T)0);
    }
    __syncthreads();

    // unit-lower inverse: 8 x 8 diagonal blocks first
    if (warp < W / kDB && lane < kDB) {
        const int o = warp * kDB, jj = lane;
        T xr[kDB];
#pragma unroll
        for (int q = 0; q < kDB; ++q) xr[q] = q == jj ? (T)1 : (T)0;
#pragma unroll
        for (int kk = 0; kk < kDB; ++kk) {
            if (kk >= jj) {
#pragma unroll
                for (int ii = kk + 1; ii < kDB; ++ii) xr[ii] -= x[(o + ii) + (o + kk) * LD] * xr[kk];
            }
        }
        __syncwarp(0xffu);
#pragma unroll
        for (int ii = 0; ii < kDB; ++ii)
            if (ii > jj) x[(o + ii) + (o + jj) * LD] = xr[ii];
    }
    __syncthreads();
#pragma unroll
    for (int sz = kDB; sz < W; sz *= 2) {
        const int npair = W / (2 * sz);
        for (int e = tid; e < npair * sz * sz; e += NT) {
            const int pr = e / (sz * sz), rem = e % (sz * sz), i = rem % sz, j = rem / sz;
            const int o = pr * 2 * sz;
            T acc = (T)0;
            for (int k = j; k < sz; ++k) acc += x[(o + sz + i) + (o + k) * LD] * x[(o + k) + (o + j) * LD];
            tmp[pr * sz * sz + i + j * sz] = acc;
        }
        __syncthreads();
        for (int e = tid; e < npair * sz * sz; e += NT) {
            const int pr = e / (sz * sz), rem = e % (sz * sz), i = rem % sz, j = rem / sz;
            const int o = pr * 2 * sz;
            T acc = tmp[pr * sz * sz + i + j * sz];   // C^{-1} has a unit diagonal
            for (int k = 0; k < i; ++k) acc += x[(o + sz + i) + (o + sz + k) * LD] * tmp[pr * sz * sz + k + j * sz];
            x[(o + sz + i) + (o + j) * LD] = -acc;
        }
        __syncthreads();
    }
    // Cholesky: L^{-1} = diag(1/sqrt(d)) l^{-1}.  LDL^T: l^{-1} below the
    // diagonal (unit), 1/d on it.
    T *Mi = Dinv + p.pinv[pid];
    for (int idx = tid; idx < w * w; idx += NT) {
        const int i = idx % w, j = idx / w;
        if constexpr (ldlt) Mi[idx] = i > j ? x[i + j * LD] : (i == j ? (T)rsv[i] : (T)0);
        else Mi[idx] = i >= j ? x[i + j * LD] * (T)rsv[i] : (T)0;
    }
}

template <typename T, int W>
constexpr size_t ldl_smem_bytes()
{
    return sizeof(double) * ((size_t)W * (W + 1) + (size_t)2 * W * kDB + 2 * W) +
           sizeof(T) * ((size_t)W * (W + 1) + (size_t)(W / 2) * (W / 2));
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

// ---------------------------------------------------------------------------
// Panel TRSM (Sec. III step 2) as a product with the inverted diagonal block:
// rows [r0, r0+64) of the off-diagonal part X become X B with
//   LLT : B = L^{-T}           (B(k,j) = Linv(j,k))
//   LU_L: B = U^{-1}           (B(k,j) = Uinv(k,j))
//   LU_U: B = L^{-T}, unit L   (B(k,j) = Linv(j,k), 1 on the diagonal)
//   RIGHT_LINV: B = L^{-1}     (B(k,j) = Linv(k,j); the selected inversion's L_RJ L_JJ^{-1})
// The CTA copies its rows and the whole B operand of a 64-column tile to
// shared memory first (every load of a batch issued before its stores), so
// writing the rows back in place is safe and the K loop runs without
// barriers; 64 x 64 output tiles, 4 x 4 per thread, written back through
// shared memory in whole segments.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) trsm_gemm_kernel(DevPlan p, const RowChunk *__restrict__ chunks,
                                                        const T *__restrict__ Dinv,
                                                        T *__restrict__ X, int mode, void *opc,
                                                        void *opc_lo, int kpad, int op_kind,
                                                        T *__restrict__ Wout)
{
    constexpr int NB = 16;                     // loads in flight per thread while staging
    extern __shared__ unsigned char smraw[];
    const RowChunk ch = chunks[blockIdx.x];
    const int pid = ch.panel;
    const int w = p.pw[pid], h = p.ph[pid];
    const int wpad = (w + 15) & ~15;
    T *Xs = reinterpret_cast<T *>(smraw);      // Xs[k * 64 + r], k < wpad
    T *Bf = Xs + wpad * kTrsmRows;             // Bf[k * 65 + j], k < max(wpad, 64); then the output tile
    const T *Mi = Dinv + p.pinv[pid];
    T *Xg = X + p.pval[pid] + ch.r0;
    const int nr = min(kTrsmRows, h - ch.r0);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // B(k, j) of the product X B (see the table above)
    auto bval = [&](int k, int j) -> T {
        if (k >= w || j >= w) return (T)0;
        if (mode == TRSM_RIGHT_LINV) return k >= j ? Mi[k + j * w] : (T)0;
        if (mode == TRSM_LU_L) return k <= j ? Mi[k + j * w] : (T)0;
        if (j > k) return Mi[j + k * w];
        if (j == k) return (mode == TRSM_LU_U || mode == TRSM_LDLT) ? (T)1 : Mi[j + k * w];
        return (T)0;
    };
    // the chunk's rows, every load of a batch issued before its stores
    for (int base = tid; base < wpad * kTrsmRows; base += 256 * NB) {
        T v[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = base + 256 * q, r = e & 63, k = e >> 6;
            v[q] = (e < wpad * kTrsmRows && r < nr && k < w) ? Xg[r + (int64_t)k * h] : (T)0;
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = base + 256 * q;
            if (e < wpad * kTrsmRows) Xs[e] = v[q];
        }
    }
    for (int c0 = 0; c0 < w; c0 += kUpdTile) {
        if (c0 > 0) __syncthreads();           // the previous tile is out of Bf
        for (int base = tid; base < wpad * kUpdTile; base += 256 * NB) {
            T v[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int e = base + 256 * q;
                v[q] = e < wpad * kUpdTile ? bval(e >> 6, c0 + (e & 63)) : (T)0;
            }
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int e = base + 256 * q;
                if (e < wpad * kUpdTile) Bf[(e >> 6) * (kUpdTile + 1) + (e & 63)] = v[q];
            }
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
#pragma unroll 4
        for (int k = 0; k < wpad; ++k) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = Xs[k * 64 + tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bf[k * (kUpdTile + 1) + ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        if (mode == TRSM_LDLT) {
            // acc = X l^{-T} is the D L^T buffer row (Sec. V-B: the update then
            // multiplies L by it); L = acc D^{-1} goes back in place
            T *Wg = Wout + p.pval[pid] + ch.r0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int j = c0 + ty + 16 * b;
                const T dinv = j < w ? Mi[j + j * w] : (T)0;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int r = tx + 16 * a;
                    if (r >= nr || j >= w) continue;
                    Wg[r + (int64_t)j * h] = acc[a][b];
                    const T l = acc[a][b] * dinv;
                    Xg[r + (int64_t)j * h] = l;
                    if (opc)   // A operand: L; B operand: D L^T
                        put_operand(opc, opc_lo, (p.prow[pid] + ch.r0 + r) * kpad + j, op_kind, (float)l,
                                    (float)acc[a][b]);
                }
            }
            continue;
        }
        // the 64 x 64 result tile through shared memory, so that both the
        // column-major panel and the row-major operand copy are written in
        // whole segments
        __syncthreads();                       // every read of Bf is done
        T *Ot = Bf;                            // Ot[r * 65 + jj]
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) Ot[(tx + 16 * a) * (kUpdTile + 1) + ty + 16 * b] = acc[a][b];
        __syncthreads();
        const int nc = min(kUpdTile, w - c0);
        for (int e = tid; e < nc * kTrsmRows; e += 256) {
            const int r = e & 63, jj = e >> 6;
            if (r < nr) Xg[r + (int64_t)(c0 + jj) * h] = Ot[r * (kUpdTile + 1) + jj];
        }
        if (opc) {
            // the same rows, K-major, for the tensor-core updates; columns
            // w .. c0+63 of the tile are zero and fill the row's padding
            const int64_t orow0 = p.prow[pid] + ch.r0;
            for (int e = tid; e < nr * kUpdTile; e += 256) {
                const int r = e >> 6, jj = e & 63;
                put_operand(opc, opc_lo, (orow0 + r) * kpad + c0 + jj, op_kind,
                            (float)Ot[r * (kUpdTile + 1) + jj], 0.0f);
            }
        }
    }
    if (opc) {
        // the rest of each operand row's padding
        const int64_t orow0 = p.prow[pid] + ch.r0;
        const int j0 = mode == TRSM_LDLT ? w : (w + kUpdTile - 1) / kUpdTile * kUpdTile;
        const int padw = kpad - j0;
        for (int e = tid; e < nr * padw; e += 256) {
            const int r = e / padw, j = j0 + e % padw;
            put_operand(opc, opc_lo, (orow0 + r) * kpad + j, op_kind, 0.0f, 0.0f);
        }
    }
}

template <typename T>
constexpr size_t trsm_smem_bytes(int wpad)
{
    return sizeof(T) * ((size_t)wpad * kTrsmRows + (size_t)(wpad > kUpdTile ? wpad : kUpdTile) * (kUpdTile + 1));
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

template <typename T, int TN>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 1) update_kernel(DevPlan p, const DevTask *__restrict__ tasks,
                                                     const UpdTile *__restrict__ tiles,
                                                     const T *__restrict__ Aop,
                                                     const T *__restrict__ Bop, T *__restrict__ C,
                                                     int lower, int from_r1)
{
    // TM x TN output tile (64 x 64, or 256 x 16 for tasks facing few rows),
    // 4 x 4 outputs per thread, K-chunks of 16 staged in shared memory
    constexpr int TM = 4096 / TN;
    constexpr int RX = TM / 4, CX = TN / 4;      // thread grid: RX rows x 256/RX column groups
    __shared__ T As[16][TM + 1];
    __shared__ T Bs[16][TN + 1];
    const UpdTile tl = tiles[blockIdx.x];
    const DevTask tk = tasks[tl.task];
    const int src = tk.src, tgt = tk.tgt;
    const int h = p.ph[src], K = p.pw[src];
    const int64_t sbase = p.pval[src];
    const T *A = Aop + sbase;
    const T *B = Bop + sbase;
    const int tid = threadIdx.x;
    const int tx = tid % RX, ty = tid / RX;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        if constexpr (TN == TM) {
            // loader: TM rows x 4 k per pass, A and B side by side
            const int lr = tid % TM, lk = tid / TM;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = lk + 4 * q;
                const int kg = k0 + kk;
                const int ra = tl.m0 + lr, rb = tl.n0 + lr;
                As[kk][lr] = (kg < K && ra < h) ? A[ra + (int64_t)kg * h] : (T)0;
                Bs[kk][lr] = (kg < K && rb < tk.r1) ? B[rb + (int64_t)kg * h] : (T)0;
            }
        } else {
            // loader: 256 rows x 1 k per pass for A, one 16 x 16 block for B
            static_assert(TM == 256 && TN == 16, "narrow tile is 256 x 16");
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const int kg = k0 + kk, ra = tl.m0 + tid;
                As[kk][tid] = (kg < K && ra < h) ? A[ra + (int64_t)kg * h] : (T)0;
            }
            const int r = tid & 15, kk = tid >> 4;
            const int kg = k0 + kk, rb = tl.n0 + r;
            Bs[kk][r] = (kg < K && rb < tk.r1) ? B[rb + (int64_t)kg * h] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + RX * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + CX * b];
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
        const int j = tl.n0 + ty + CX * b;
        cok[b] = j < tk.r1;
        coff[b] = cok[b] ? (int64_t)(srow[j] - fcolT) * hT : 0;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = tl.m0 + tx + RX * a;
        if (i >= h || i < rlo) continue;
        const int64_t roff = rmap[i];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = tl.n0 + ty + CX * b;
            if (!cok[b] || (lower && i < j)) continue;
            atomic_sub<T>(Ct + roff + coff[b], acc[a][b]);
        }
    }
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
template void launch_assemble<double>(int64_t, const double *, const int64_t *, double *, double *, cudaStream_t);
template void launch_assemble<float>(int64_t, const double *, const int64_t *, float *, float *, cudaStream_t);
template void launch_potrf<double>(const DevPlan &, const int32_t *, int, int, int, double *, double *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_potrf<float>(const DevPlan &, const int32_t *, int, int, int, float *, float *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_getrf<double>(const DevPlan &, const int32_t *, int, int, int, double *, double *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_getrf<float>(const DevPlan &, const int32_t *, int, int, int, float *, float *, const double *, int64_t *, unsigned long long *, cudaStream_t);
template void launch_trsm<double>(const DevPlan &, const RowChunk *, int, int, const double *, double *, int, void *, void *, int, int, cudaStream_t, double *);
template void launch_ldlt_diag<double>(const DevPlan &, const int32_t *, int, int, double *, double *, const double *, int64_t *, unsigned long long *, unsigned long long *, cudaStream_t);
template void launch_trsm<float>(const DevPlan &, const RowChunk *, int, int, const float *, float *, int, void *, void *, int, int, cudaStream_t, float *);
template void launch_ldlt_diag<float>(const DevPlan &, const int32_t *, int, int, float *, float *, const double *, int64_t *, unsigned long long *, unsigned long long *, cudaStream_t);
template void launch_update<double>(const DevPlan &, const DevTask *, const UpdTile *, int, const double *, const double *, double *, int, int, cudaStream_t, int);
template void launch_update<float>(const DevPlan &, const DevTask *, const UpdTile *, int, const float *, const float *, float *, int, int, cudaStream_t, int);

}  // namespace spx
