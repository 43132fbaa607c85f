// batch_lu.cu -- one persistent kernel that factorizes, solves and refines a
// batch of small independent sparse systems (static-pivot LU, Sec. III).
//
// Each CTA takes whole systems from a device queue (largest first) and runs,
// for its system, everything the single-system path spreads over launches:
// assembly, then the panels level by level -- diagonal-block LU with static
// pivot replacement, the two panel TRSMs (L and U^T sides), and the updates
// of the facing panels with the scatter fused (Sec. V-B) -- then the
// triangular solves and FP64 iterative refinement.  No CTA ever waits on
// another, so the kernel needs no grid-wide synchronisation.
//
// Schedule inside a CTA (the leaf-versus-top choice is a launch parameter):
//  * panels at most `leaf_width` wide go one per warp, all panels of a level
//    at once, their updates added atomically (siblings may share targets);
//  * wider panels use the whole CTA one at a time (plain read-modify-write);
//  * the solves go one panel per warp, level by level, on a copy of the
//    right-hand side in shared memory.
#include "batch_kernel.cuh"

#include <cmath>

namespace spx {
namespace {

constexpr int kWarps = kBatchThreads / 32;
constexpr int kLdC = kBatchMaxWidth + 1;   // odd leading dimensions: no bank conflicts
constexpr int kLdW = kBatchLeafMax + 1;
constexpr int kChunkC = 64;                // TRSM rows per pass and side, CTA mode
constexpr int kChunkW = 32;                // TRSM rows per pass, warp mode
constexpr int kCtaElems = kBatchMaxWidth * kLdC + 2 * kChunkC * kLdC;
constexpr int kWarpElems = kBatchLeafMax * kLdW + kChunkW * kLdW;
constexpr int kRedDoubles = 3 * kWarps + 2;   // reductions + 4 ints

__device__ __forceinline__ double inf_if_nan(double v) { return v != v ? INFINITY : v; }

// LU without row exchanges of the w x w block a (column-major, leading
// dimension ld) by one warp.  Static pivoting (Sec. III): a pivot whose
// magnitude is below tau is replaced by +-tau (+tau for 0).  With tau == 0 a
// zero pivot is recorded in *zero_k and replaced by 1 so the work completes.
// Returns the number of replacements (the same on every lane).
template <typename T>
__device__ __forceinline__ int getrf_warp(T *a, int w, int ld, double tau, int lane, int *zero_k)
{
    int nrep = 0;
    for (int k = 0; k < w; ++k) {
        T d = a[k + k * ld];
        const double ad = fabs((double)d);
        if (tau > 0.0) {
            if (!(ad >= tau)) {
                d = (T)(d < (T)0 ? -tau : tau);
                ++nrep;
            }
        } else if (!(ad > 0.0)) {
            if (*zero_k < 0) *zero_k = k;
            d = (T)1;
        }
        const T r = (T)1 / d;
        __syncwarp();
        if (lane == 0) a[k + k * ld] = d;
        for (int i = k + 1 + lane; i < w; i += 32) a[i + k * ld] *= r;
        __syncwarp();
        for (int i = k + 1 + lane; i < w; i += 32) {
            const T lik = a[i + k * ld];
            for (int j = k + 1; j < w; ++j) a[i + j * ld] -= lik * a[k + j * ld];
        }
        __syncwarp();
    }
    return nrep;
}

// One row x (length w, in shared memory) of the off-diagonal part:
//   side 0 (L panel):   x <- x U^{-1},  U = upper(lu)
//   side 1 (U^T panel): x <- x L^{-T},  L = unit lower(lu)
// by substitution, two partial sums to halve the dependent chain.
template <typename T>
__device__ __forceinline__ void trsm_row(T *x, const T *lu, int ld, int w, int side)
{
    for (int j = 0; j < w; ++j) {
        T s0 = x[j], s1 = (T)0;
        int k = 0;
        if (side == 0) {
            for (; k + 1 < j; k += 2) {
                s0 -= x[k] * lu[k + j * ld];
                s1 -= x[k + 1] * lu[k + 1 + j * ld];
            }
            if (k < j) s0 -= x[k] * lu[k + j * ld];
            x[j] = (s0 + s1) / lu[j + j * ld];
        } else {
            for (; k + 1 < j; k += 2) {
                s0 -= x[k] * lu[j + k * ld];
                s1 -= x[k + 1] * lu[j + (k + 1) * ld];
            }
            if (k < j) s0 -= x[k] * lu[j + k * ld];
            x[j] = s0 + s1;
        }
    }
}

template <typename T>
__device__ __forceinline__ void sub_to(T *dst, T v, bool atomic)
{
    if (atomic) atomicAdd(dst, -v);
    else *dst -= v;
}

// Updates of every panel facing source panel p (Sec. III step 3), scatter
// fused (Sec. V-B).  For task (p -> t) with facing rows [r0, r1):
//   L side, rows i in [r0, h):  C_L(relmap(i), row(j) - fcol(t)) -= sum_k L(i,k) U^T(j,k)
//   U side, rows i in [r1, h):  C_U(relmap(i), row(j) - fcol(t)) -= sum_k U^T(i,k) L(j,k)
// Threads t0.. of a group of nt; RT rows per thread (spaced so that the
// loads of consecutive threads are consecutive).  Threads run through the
// tasks without waiting for one another.
template <typename T, int RT>
__device__ __forceinline__ void update_group(const BClass &c, int p, T *Ls, T *Us, int t0, int nt, bool atomic)
{
    const int w = c.pw[p], h = c.ph[p];
    const T *Lp = Ls + c.pval[p];
    const T *Up = Us + c.pval[p];
    const int32_t *rows = c.rows + c.prow[p];
    for (int q = c.task_ptr[p]; q < c.task_ptr[p + 1]; ++q) {
        const BTask tk = c.tasks[q];
        const int ht = c.ph[tk.tgt];
        const int fct = c.pfcol[tk.tgt];
        const int32_t *rmap = c.relmap + tk.relmap_off - tk.r0;
        const int N = tk.r1 - tk.r0;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int lo = side == 0 ? tk.r0 : tk.r1;
            const int M = h - lo;
            if (M <= 0) continue;
            const T *Ai = side == 0 ? Lp : Up;     // row operand
            const T *Bj = side == 0 ? Up : Lp;     // facing operand
            T *C = (side == 0 ? Ls : Us) + c.pval[tk.tgt];
            const int MR = (M + RT - 1) / RT;
            for (int e = t0; e < MR * N; e += nt) {
                const int ig = e % MR, j = tk.r0 + e / MR;
                T acc[RT];
#pragma unroll
                for (int r = 0; r < RT; ++r) acc[r] = (T)0;
                for (int k = 0; k < w; ++k) {
                    const T b = Bj[j + (int64_t)k * h];
#pragma unroll
                    for (int r = 0; r < RT; ++r) {
                        const int i = lo + ig + r * MR;
                        if (i < h) acc[r] += Ai[i + (int64_t)k * h] * b;
                    }
                }
                const int64_t coff = (int64_t)(rows[j] - fct) * ht;
#pragma unroll
                for (int r = 0; r < RT; ++r) {
                    const int i = lo + ig + r * MR;
                    if (i < h) sub_to<T>(C + rmap[i] + coff, acc[r], atomic);
                }
            }
        }
    }
}

// Panel p by one warp (w <= kBatchLeafMax).  sm: kWarpElems elements.
template <typename T, int RT>
__device__ __forceinline__ void panel_warp(const BClass &c, int p, T *Ls, T *Us, T *sm, double tau, int lane,
                           int *nrep, int *zero_col)
{
    const int w = c.pw[p], h = c.ph[p];
    T *lu = sm;
    T *st = sm + kBatchLeafMax * kLdW;
    T *Lp = Ls + c.pval[p];
    T *Up = Us + c.pval[p];
    for (int e = lane; e < w * w; e += 32) lu[e % w + (e / w) * kLdW] = Lp[e % w + (e / w) * h];
    __syncwarp();
    int zk = -1;
    const int nr = getrf_warp<T>(lu, w, kLdW, tau, lane, &zk);
    if (lane == 0) {
        if (nr) atomicAdd(nrep, nr);
        if (zk >= 0) atomicMin(zero_col, c.pfcol[p] + zk);
    }
    for (int e = lane; e < w * w; e += 32) Lp[e % w + (e / w) * h] = lu[e % w + (e / w) * kLdW];
    for (int side = 0; side < 2; ++side) {
        T *X = side ? Up : Lp;
        for (int c0 = w; c0 < h; c0 += kChunkW) {
            const int m = min(kChunkW, h - c0);
            for (int e = lane; e < m * w; e += 32) st[(e % m) * kLdW + e / m] = X[c0 + e % m + (int64_t)(e / m) * h];
            __syncwarp();
            if (lane < m) trsm_row<T>(st + lane * kLdW, lu, kLdW, w, side);
            __syncwarp();
            for (int e = lane; e < m * w; e += 32) X[c0 + e % m + (int64_t)(e / m) * h] = st[(e % m) * kLdW + e / m];
            __syncwarp();
        }
    }
    update_group<T, RT>(c, p, Ls, Us, lane, 32, true);
}

// Panel p by the whole CTA (w <= kBatchMaxWidth).  sm: kCtaElems elements.
template <typename T, int RT>
__device__ __forceinline__ void panel_cta(const BClass &c, int p, T *Ls, T *Us, T *sm, double tau, int *nrep,
                          int *zero_col)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w = c.pw[p], h = c.ph[p];
    T *lu = sm;
    T *stL = sm + kBatchMaxWidth * kLdC;
    T *stU = stL + kChunkC * kLdC;
    T *Lp = Ls + c.pval[p];
    T *Up = Us + c.pval[p];
    for (int e = tid; e < w * w; e += kBatchThreads) lu[e % w + (e / w) * kLdC] = Lp[e % w + (e / w) * h];
    __syncthreads();
    if (warp == 0) {
        int zk = -1;
        const int nr = getrf_warp<T>(lu, w, kLdC, tau, lane, &zk);
        if (lane == 0) {
            if (nr) atomicAdd(nrep, nr);
            if (zk >= 0) atomicMin(zero_col, c.pfcol[p] + zk);
        }
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += kBatchThreads) Lp[e % w + (e / w) * h] = lu[e % w + (e / w) * kLdC];
    for (int c0 = w; c0 < h; c0 += kChunkC) {
        const int m = min(kChunkC, h - c0);
        for (int e = tid; e < m * w; e += kBatchThreads) {
            const int r = e % m, k = e / m;
            stL[r * kLdC + k] = Lp[c0 + r + (int64_t)k * h];
            stU[r * kLdC + k] = Up[c0 + r + (int64_t)k * h];
        }
        __syncthreads();
        if (tid < kChunkC) {
            if (tid < m) trsm_row<T>(stL + tid * kLdC, lu, kLdC, w, 0);
        } else if (tid >= 128 && tid < 128 + kChunkC) {
            if (tid - 128 < m) trsm_row<T>(stU + (tid - 128) * kLdC, lu, kLdC, w, 1);
        }
        __syncthreads();
        for (int e = tid; e < m * w; e += kBatchThreads) {
            const int r = e % m, k = e / m;
            Lp[c0 + r + (int64_t)k * h] = stL[r * kLdC + k];
            Up[c0 + r + (int64_t)k * h] = stU[r * kLdC + k];
        }
        __syncthreads();
    }
    update_group<T, RT>(c, p, Ls, Us, tid, kBatchThreads, false);
    __syncthreads();
}

// Forward sweep of panel p by one warp: y = L11^{-1} w_p (unit lower), then
// w(rows below) -= L21 y, added atomically (panels of a level run at once).
template <typename T>
__device__ __forceinline__ void fwd_panel_warp(const BClass &c, int p, const T *Ls, T *wv, int lane)
{
    const int w = c.pw[p], h = c.ph[p], fc = c.pfcol[p];
    const T *Lp = Ls + c.pval[p];
    const int32_t *rows = c.rows + c.prow[p];
    for (int k = 0; k < w; ++k) {
        const T yk = wv[fc + k];
        for (int i = k + 1 + lane; i < w; i += 32) wv[fc + i] -= Lp[i + (int64_t)k * h] * yk;
        __syncwarp();
    }
    for (int i = w + lane; i < h; i += 32) {
        T s = (T)0;
        for (int k = 0; k < w; ++k) s += Lp[i + (int64_t)k * h] * wv[fc + k];
        atomicAdd(&wv[rows[i]], -s);
    }
}

// Backward sweep of panel p by one warp: z = w_p - U12 w(rows below), then
// x_p = U11^{-1} z.  U12(k, row i) is U^T(i, k).
template <typename T>
__device__ __forceinline__ void bwd_panel_warp(const BClass &c, int p, const T *Ls, const T *Us, T *wv, int lane)
{
    const int w = c.pw[p], h = c.ph[p], fc = c.pfcol[p];
    const T *Lp = Ls + c.pval[p];
    const T *Up = Us + c.pval[p];
    const int32_t *rows = c.rows + c.prow[p];
    for (int k = lane; k < w; k += 32) {
        T s0 = wv[fc + k], s1 = (T)0;
        int i = w;
        for (; i + 1 < h; i += 2) {
            s0 -= Up[i + (int64_t)k * h] * wv[rows[i]];
            s1 -= Up[i + 1 + (int64_t)k * h] * wv[rows[i + 1]];
        }
        if (i < h) s0 -= Up[i + (int64_t)k * h] * wv[rows[i]];
        wv[fc + k] = s0 + s1;
    }
    __syncwarp();
    for (int k = w - 1; k >= 0; --k) {
        if (lane == 0) wv[fc + k] = wv[fc + k] / Lp[k + (int64_t)k * h];
        __syncwarp();
        const T xk = wv[fc + k];
        for (int i = lane; i < k; i += 32) wv[fc + i] -= Lp[i + (int64_t)k * h] * xk;
        __syncwarp();
    }
}

// Max over the CTA of three values (every thread gets the result).
__device__ __forceinline__ void block_max3(double *v, double *red)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] = fmax(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) red[q * kWarps + warp] = v[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double m = red[q * kWarps];
#pragma unroll
        for (int u = 1; u < kWarps; ++u) m = fmax(m, red[q * kWarps + u]);
        v[q] = m;
    }
}

// r = b - A x (FP64, original numbering) into wv (permuted, T); returns the
// backward error max|r| / (||A||_inf max|x| + max|b|).
template <typename T>
__device__ __forceinline__ double residual(const BClass &c, const BSys &S, const double *vals, const double *b,
                           const double *x, bool x_zero, double anorm, T *wv, double *red)
{
    double v[3] = {0.0, 0.0, 0.0};   // max |r|, max |x|, max |b|
    for (int i = threadIdx.x; i < S.n; i += kBatchThreads) {
        double s = b[i];
        if (!x_zero)
            for (int e = c.csr_ptr[i]; e < c.csr_ptr[i + 1]; ++e)
                s -= vals[S.voff + c.csr_src[e]] * x[c.csr_col[e]];
        wv[c.iperm[i]] = (T)s;
        v[0] = fmax(v[0], inf_if_nan(fabs(s)));
        if (!x_zero) v[1] = fmax(v[1], inf_if_nan(fabs(x[i])));
        v[2] = fmax(v[2], fabs(b[i]));
    }
    block_max3(v, red);
    const double den = anorm * v[1] + v[2];
    if (den > 0.0) return v[0] / den;
    return v[0] == 0.0 ? 0.0 : INFINITY;
}

template <typename T, int RT>
__device__ __forceinline__ void process(const BatchArgs &a, int sid, T *region, double *red, int *si)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const BSys S = a.sys[sid];
    const BClass c = a.cls[S.cls];
    T *Ls = static_cast<T *>(a.L) + S.foff;
    T *Us = static_cast<T *>(a.U) + S.foff;
    const double *vals = a.vals;

    // assembly: zero the panels, ||A||_inf, then scatter the values
    for (int64_t e = tid; e < c.nstored; e += kBatchThreads) {
        Ls[e] = (T)0;
        Us[e] = (T)0;
    }
    double v[3] = {0.0, 0.0, 0.0};
    for (int i = tid; i < S.n; i += kBatchThreads) {
        double s = 0.0;
        for (int e = c.csr_ptr[i]; e < c.csr_ptr[i + 1]; ++e) s += fabs(vals[S.voff + c.csr_src[e]]);
        v[0] = fmax(v[0], s);
    }
    if (tid == 0) {
        si[1] = 0;
        si[2] = 0x7fffffff;
    }
    block_max3(v, red);   // also orders the zero fill before the scatter
    const double anorm = v[0];
    const double tau = a.tau_opt >= 0.0 ? a.tau_opt : 0x1p-26 * anorm;   // sqrt(2^-52) ||A||_inf
    for (int e = tid; e < c.nnz; e += kBatchThreads) {
        const int64_t m = c.amap[e];
        const T x = (T)vals[S.voff + e];
        if (m >= 0) Ls[m] = x;
        else if (m <= -2) Us[-2 - m] = x;
    }
    __syncthreads();

    // factorization, level by level
    for (int l = 0; l < c.nlevels; ++l) {
        const int q0 = c.level_ptr[l], q1 = c.level_ptr[l + 1];
        if (a.leaf_width > 0) {
            T *wsm = region + warp * kWarpElems;
            for (int q = q0 + warp; q < q1; q += kWarps) {
                const int p = c.level_panels[q];
                if (c.pw[p] <= a.leaf_width) panel_warp<T, RT>(c, p, Ls, Us, wsm, tau, lane, &si[1], &si[2]);
            }
            __syncthreads();
        }
        for (int q = q0; q < q1; ++q) {
            const int p = c.level_panels[q];
            if (c.pw[p] > a.leaf_width) panel_cta<T, RT>(c, p, Ls, Us, region, tau, &si[1], &si[2]);
        }
    }
    __syncthreads();
    const int nrep = si[1];
    const int zero_col = si[2];

    int iters = 0, conv = 1;
    double berr = 0.0;
    if (a.do_solve) {
        const double *b = a.B + S.xoff;
        double *x = a.X + S.xoff;
        T *wv = region;
        for (int i = tid; i < S.n; i += kBatchThreads) x[i] = 0.0;
        residual<T>(c, S, vals, b, x, true, anorm, wv, red);   // w = P b
        __syncthreads();
        for (int s = 1;; ++s) {
            for (int l = 0; l < c.nlevels; ++l) {
                for (int q = c.level_ptr[l] + warp; q < c.level_ptr[l + 1]; q += kWarps)
                    fwd_panel_warp<T>(c, c.level_panels[q], Ls, wv, lane);
                __syncthreads();
            }
            for (int l = c.nlevels - 1; l >= 0; --l) {
                for (int q = c.level_ptr[l] + warp; q < c.level_ptr[l + 1]; q += kWarps)
                    bwd_panel_warp<T>(c, c.level_panels[q], Ls, Us, wv, lane);
                __syncthreads();
            }
            for (int i = tid; i < S.n; i += kBatchThreads) x[c.perm[i]] += (double)wv[i];
            __syncthreads();
            berr = residual<T>(c, S, vals, b, x, false, anorm, wv, red);
            __syncthreads();
            iters = s - 1;
            if (a.tol > 0.0 && berr <= a.tol) break;
            if (s > a.max_iter) break;
        }
        conv = a.tol > 0.0 ? (berr <= a.tol) : 1;
    }
    if (tid == 0) {
        a.iters[sid] = iters;
        a.converged[sid] = conv;
        a.berr[sid] = berr;
        a.nrepl[sid] = nrep;
        a.bad_col[sid] = zero_col == 0x7fffffff ? -1 : zero_col;
        if (!conv) atomicAdd(&a.summary[0], 1u);
        if (zero_col != 0x7fffffff) atomicAdd(&a.summary[1], 1u);
    }
}

template <typename T, int RT>
__global__ void __launch_bounds__(kBatchThreads, 3) batch_lu_kernel(BatchArgs a)
{
    extern __shared__ double smd[];
    double *red = smd;
    int *si = reinterpret_cast<int *>(smd + 3 * kWarps);
    T *region = reinterpret_cast<T *>(smd + kRedDoubles);
    for (;;) {
        if (threadIdx.x == 0) si[0] = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int q = si[0];
        __syncthreads();
        if (q >= a.nsys) break;
        process<T, RT>(a, a.order[q], region, red, si);
    }
}

template <typename T, int RT>
void set_smem_attr(size_t bytes)
{
    cudaFuncSetAttribute(batch_lu_kernel<T, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t batch_smem_bytes(int elem_bytes, int n_max)
{
    int elems = kCtaElems;
    if (kWarps * kWarpElems > elems) elems = kWarps * kWarpElems;
    if (n_max > elems) elems = n_max;
    return sizeof(double) * kRedDoubles + (size_t)elem_bytes * (size_t)elems;
}

template <typename T, int RT>
static int max_ctas(size_t smem)
{
    set_smem_attr<T, RT>(smem);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_lu_kernel<T, RT>, kBatchThreads, smem) !=
        cudaSuccess)
        return 0;
    return blocks;
}

int batch_max_ctas_per_sm(int elem_bytes, int n_max, int rows_per_thread)
{
    const size_t smem = batch_smem_bytes(elem_bytes, n_max);
    if (elem_bytes == 8) {
        if (rows_per_thread == 1) return max_ctas<double, 1>(smem);
        if (rows_per_thread == 2) return max_ctas<double, 2>(smem);
        return max_ctas<double, 4>(smem);
    }
    if (rows_per_thread == 1) return max_ctas<float, 1>(smem);
    if (rows_per_thread == 2) return max_ctas<float, 2>(smem);
    return max_ctas<float, 4>(smem);
}

// The shared-memory attribute is set by batch_max_ctas_per_sm, which the
// caller runs first (outside any stream capture).
template <typename T, int RT>
static void launch_t(const BatchArgs &a, int grid, size_t smem, cudaStream_t s)
{
    batch_lu_kernel<T, RT><<<grid, kBatchThreads, smem, s>>>(a);
}

void launch_batch(const BatchArgs &a, int elem_bytes, int rows_per_thread, int grid, int n_max,
                  cudaStream_t s)
{
    const size_t smem = batch_smem_bytes(elem_bytes, n_max);
    if (elem_bytes == 8) {
        if (rows_per_thread == 1) launch_t<double, 1>(a, grid, smem, s);
        else if (rows_per_thread == 2) launch_t<double, 2>(a, grid, smem, s);
        else launch_t<double, 4>(a, grid, smem, s);
    } else {
        if (rows_per_thread == 1) launch_t<float, 1>(a, grid, smem, s);
        else if (rows_per_thread == 2) launch_t<float, 2>(a, grid, smem, s);
        else launch_t<float, 4>(a, grid, smem, s);
    }
}

}  // namespace spx
