// selinv.cu -- selected inversion of a supernodal Cholesky factor, the
// log-determinant and the adjoint kernels of the differentiable solve.
//
// Z = (P A P^T)^{-1} is computed on the panel structure of L (the entries a
// gradient of log det A needs), panel by panel from the root down.  For a
// panel with diagonal columns J and off-diagonal rows R, with
// Lh = L_RJ L_JJ^{-1} (formed beforehand by the TRSM kernel):
//   Z_RJ = -Z_RR Lh                  (Z_RR gathered from ancestor panels)
//   Z_JJ = L_JJ^{-T} L_JJ^{-1} - Lh^T Z_RJ
// Z_RR is addressed through the update tasks' row maps, the same maps the
// factorization scatters through (Sec. V-B): for task p -> q with facing
// rows F = [r0, r1), entry (row i, row j) of Z with i in [r0, h), j in F
// sits in panel q at row relmap(i), column row(j) - fcol(q).  Diagonal
// blocks of Z are stored as full symmetric squares so that both triangles
// can be gathered.
#include "kernels.cuh"

#include <cmath>

namespace spx {

// ---------------------------------------------------------------------------
// Z_RJ for rows [r0, r0+64) of one panel: Z_RJ(i, :) = -sum_{j in R}
// Z(i, j) Lh(j, :).  Row j of R faces the task t(j) (row_task), whose target
// panel q holds the column of row j.  The entry Z(i, j) is stored
//   in q = tgt(t(j)) at row relmap_t(j)(i), column row(j) - fcol(q)  if i >= r0(t(j)),
//   else (i lies in an earlier facing block, j below it) in tgt(t(i)) at
//   row relmap_t(i)(j), column row(i) - fcol(tgt(t(i))).
// 64 x WC output tile (WC = 16, 32 or 64, the panel width rounded up),
// 4 x WC/16 outputs per thread, K = the rows of R in chunks of 16 staged in
// shared memory.  Split-K near the root, where a level holds one panel:
// gridDim.y CTAs share a row chunk, each taking a contiguous part of R, and
// add their partial sums into Z (zeroed beforehand).
// ---------------------------------------------------------------------------
template <int WC>
__device__ __forceinline__ void selinv_off_tile(const DevPlan &p, int pid, int w, int h, int i0, int i1,
                                                const int32_t *__restrict__ row_task,
                                                const DevTask *__restrict__ tasks,
                                                const double *__restrict__ Lh, double *__restrict__ Z,
                                                double (*As)[65], double (*Bs)[65], int split, int nsplit)
{
    constexpr int NB = WC / 16;
    const int64_t base = p.pval[pid];
    const double *Lp = Lh + base;
    const int32_t *srow = p.rows + p.prow[pid];
    const int32_t *rt = row_task + p.prow[pid];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][NB];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[a][b] = 0.0;
    // this CTA's part of R: 16-row aligned segment [kb, ke)
    const int nk = (h - w + 15) / 16;
    const int per = (nk + nsplit - 1) / nsplit;
    const int kb = w + 16 * min(nk, split * per), ke = min(h, w + 16 * min(nk, (split + 1) * per));
    for (int k0 = kb; k0 < ke; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int r = e & 63, kk = e >> 6;
            const int i = i0 + r, j = k0 + kk;
            double v = 0.0;
            if (i < i1 && j < ke) {
                const DevTask tj = tasks[rt[j]];
                if (i >= tj.r0) {
                    v = Z[p.pval[tj.tgt] + p.relmap[tj.relmap_off + i - tj.r0] +
                          (int64_t)(srow[j] - p.pfcol[tj.tgt]) * p.ph[tj.tgt]];
                } else {
                    const DevTask ti = tasks[rt[i]];
                    v = Z[p.pval[ti.tgt] + p.relmap[ti.relmap_off + j - ti.r0] +
                          (int64_t)(srow[i] - p.pfcol[ti.tgt]) * p.ph[ti.tgt]];
                }
            }
            As[kk][r] = v;
        }
        for (int e = tid; e < 16 * WC; e += 256) {
            const int c = e % WC, kk = e / WC;
            const int j = k0 + kk;
            Bs[kk][c] = (j < ke && c < w) ? Lp[j + (int64_t)c * h] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double av[4], bv[NB];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < NB; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < NB; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + tx + 16 * a;
        if (i >= i1) continue;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int c = ty + 16 * b;
            if (c >= w) continue;
            if (nsplit == 1) Z[base + i + (int64_t)c * h] = -acc[a][b];
            else atomicAdd(&Z[base + i + (int64_t)c * h], -acc[a][b]);
        }
    }
}

__global__ void __launch_bounds__(256) selinv_off_kernel(DevPlan p, const RowChunk *__restrict__ chunks,
                                                         const int32_t *__restrict__ row_task,
                                                         const DevTask *__restrict__ tasks,
                                                         const double *__restrict__ Lh,
                                                         double *__restrict__ Z)
{
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const RowChunk ch = chunks[blockIdx.x];
    const int pid = ch.panel;
    const int w = p.pw[pid], h = p.ph[pid];
    const int i0 = ch.r0, i1 = min(h, ch.r0 + 64);
    const int sp = blockIdx.y, ns = gridDim.y;
    if (w <= 16) selinv_off_tile<16>(p, pid, w, h, i0, i1, row_task, tasks, Lh, Z, As, Bs, sp, ns);
    else if (w <= 32) selinv_off_tile<32>(p, pid, w, h, i0, i1, row_task, tasks, Lh, Z, As, Bs, sp, ns);
    else selinv_off_tile<64>(p, pid, w, h, i0, i1, row_task, tasks, Lh, Z, As, Bs, sp, ns);
}

// ---------------------------------------------------------------------------
// Z_JJ = Linv^T Linv - Lh^T Z_RJ for one panel (w <= 64), lower pairs (a, b)
// computed once and written to both triangles.  Split-K as above: gridDim.y
// CTAs per panel take every gridDim.y-th chunk of 32 rows of R.
// ---------------------------------------------------------------------------
constexpr int kSelDiagPairs = 9;   // ceil(64 * 65 / 2 / 256)

__global__ void __launch_bounds__(256) selinv_diag_kernel(DevPlan p, const int32_t *__restrict__ panels,
                                                          const double *__restrict__ Dinv,
                                                          const double *__restrict__ Lh,
                                                          double *__restrict__ Z)
{
    extern __shared__ double sm[];
    const int pid = panels[blockIdx.x];
    const int w = p.pw[pid], h = p.ph[pid];
    const int64_t base = p.pval[pid];
    double *Di = sm;                 // w x w, Linv(i, j) at Di[i + j * w]
    double *Ls = Di + w * w;         // 32 x w: Lh rows of the current chunk
    double *Zs = Ls + 32 * w;        // 32 x w: Z_RJ rows of the current chunk
    const double *Mi = Dinv + p.pinv[pid];
    const int tid = threadIdx.x;
    const int sp = blockIdx.y, ns = gridDim.y;   // this CTA takes every ns-th chunk of 32 rows
    for (int e = tid; e < w * w; e += 256) Di[e] = Mi[e];
    const int npair = w * (w + 1) / 2;
    int pa[kSelDiagPairs], pb[kSelDiagPairs];
    double acc[kSelDiagPairs];
#pragma unroll
    for (int q = 0; q < kSelDiagPairs; ++q) {
        const int e = tid + 256 * q;
        int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (a > 0 && a * (a + 1) / 2 > e) --a;
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        pa[q] = e < npair ? a : 0;
        pb[q] = e < npair ? e - a * (a + 1) / 2 : 0;
        acc[q] = 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSelDiagPairs; ++q) {
        if (tid + 256 * q >= npair || sp != 0) continue;
        const int a = pa[q], b = pb[q];   // a >= b: Linv(k, a) Linv(k, b) is nonzero for k >= a
        double s = 0.0;
#pragma unroll 1
        for (int k = a; k < w; ++k) s = fma(Di[k + a * w], Di[k + b * w], s);
        acc[q] = s;
    }
    for (int c0 = w + 32 * sp; c0 < h; c0 += 32 * ns) {
        const int m = min(32, h - c0);
        __syncthreads();
        for (int e = tid; e < 32 * w; e += 256) {
            const int r = e & 31, c = e >> 5;
            const bool ok = r < m;
            Ls[r * w + c] = ok ? Lh[base + c0 + r + (int64_t)c * h] : 0.0;
            Zs[r * w + c] = ok ? Z[base + c0 + r + (int64_t)c * h] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kSelDiagPairs; ++q) {
            if (tid + 256 * q >= npair) continue;
            const int a = pa[q], b = pb[q];
            double s0 = 0.0, s1 = 0.0;
#pragma unroll 4
            for (int r = 0; r < 32; r += 2) {
                s0 = fma(Ls[r * w + a], Zs[r * w + b], s0);
                s1 = fma(Ls[(r + 1) * w + a], Zs[(r + 1) * w + b], s1);
            }
            acc[q] -= s0 + s1;
        }
    }
#pragma unroll
    for (int q = 0; q < kSelDiagPairs; ++q) {
        if (tid + 256 * q >= npair) continue;
        const int a = pa[q], b = pb[q];
        if (ns == 1) {
            Z[base + a + (int64_t)b * h] = acc[q];
            Z[base + b + (int64_t)a * h] = acc[q];
        } else {   // partial sums over row chunks; Z starts zeroed
            atomicAdd(&Z[base + a + (int64_t)b * h], acc[q]);
            if (a != b) atomicAdd(&Z[base + b + (int64_t)a * h], acc[q]);
        }
    }
}

void launch_selinv_off(const DevPlan &p, const RowChunk *chunks, int count, int nsplit,
                       const int32_t *row_task, const DevTask *tasks, const double *Lh, double *Z,
                       cudaStream_t s)
{
    if (count <= 0) return;
    selinv_off_kernel<<<dim3(count, nsplit), 256, 0, s>>>(p, chunks, row_task, tasks, Lh, Z);
}

void launch_selinv_diag(const DevPlan &p, const int32_t *panels, int count, int nsplit, int wmax,
                        const double *Dinv, const double *Lh, double *Z, cudaStream_t s)
{
    if (count <= 0) return;
    const size_t smem = sizeof(double) * ((size_t)wmax * wmax + 64 * (size_t)wmax);
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute(selinv_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (64 * 64 + 64 * 64)));
        once = true;
    }
    selinv_diag_kernel<<<dim3(count, nsplit), 256, smem, s>>>(p, panels, Dinv, Lh, Z);
}

// ---------------------------------------------------------------------------
// log det A = 2 sum_j log L(j, j): one block, panels by thread, FP64 sum
// with error compensation (Knuth's two-sum on every addition, the error
// terms summed apart), so that the result is accurate to about one unit of
// the last place of the total rather than n of them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <typename T>
__global__ void __launch_bounds__(1024) logdet_kernel(DevPlan p, const T *__restrict__ L, double *out)
{
    __shared__ double red[64];
    double s = 0.0, c = 0.0;
    for (int pid = threadIdx.x; pid < p.npanels; pid += blockDim.x) {
        const int w = p.pw[pid], h = p.ph[pid];
        const T *D = L + p.pval[pid];
        for (int k = 0; k < w; ++k) {
            double t, e;
            two_sum(s, log((double)D[k + (int64_t)k * h]), t, e);
            s = t;
            c += e;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        double t, e;
        two_sum(s, __shfl_xor_sync(0xffffffffu, s, o), t, e);
        c += e + __shfl_xor_sync(0xffffffffu, c, o);
        s = t;
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = s;
        red[32 + (threadIdx.x >> 5)] = c;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool has = threadIdx.x < (blockDim.x >> 5);
        s = has ? red[threadIdx.x] : 0.0;
        c = has ? red[32 + threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            double t, e;
            two_sum(s, __shfl_xor_sync(0xffffffffu, s, o), t, e);
            c += e + __shfl_xor_sync(0xffffffffu, c, o);
            s = t;
        }
        if (threadIdx.x == 0) *out = 2.0 * (s + c);
    }
}

template <typename T>
void launch_logdet(const DevPlan &p, const T *L, double *out, cudaStream_t s)
{
    logdet_kernel<T><<<1, 1024, 0, s>>>(p, L, out);
}
template void launch_logdet<double>(const DevPlan &, const double *, double *, cudaStream_t);
template void launch_logdet<float>(const DevPlan &, const float *, double *, cudaStream_t);

// grad[e] = Z[zmap[e]]: (A^{-1})_{ji} for every stored entry e of A
__global__ void gather_kernel(int64_t nnz, const int64_t *__restrict__ zmap, const double *__restrict__ Z,
                              double *__restrict__ grad)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nnz) grad[e] = Z[zmap[e]];
}

void launch_gather(int64_t nnz, const int64_t *zmap, const double *Z, double *grad, cudaStream_t s)
{
    if (nnz <= 0) return;
    gather_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(nnz, zmap, Z, grad);
}

// grad[e] = -sum_r Lam(i, r) X(j, r) for the entry e = (i, j) of A: the
// adjoint of x = A^{-1} b with respect to A's stored values, sampled on A's
// pattern.  One thread per row i of A (rows in the original numbering).
__global__ void solve_grad_kernel(int64_t n, int nrhs, const int64_t *__restrict__ rp,
                                  const int32_t *__restrict__ ci, const int64_t *__restrict__ src,
                                  const double *__restrict__ Lam, int64_t ldl,
                                  const double *__restrict__ X, int64_t ldx, double *__restrict__ grad)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        const int64_t j = ci[e];
        double s = 0.0;
        for (int r = 0; r < nrhs; ++r) s = fma(Lam[i + r * ldl], X[j + r * ldx], s);
        grad[src[e]] = -s;
    }
}

void launch_solve_grad(int64_t n, int nrhs, const int64_t *rp, const int32_t *ci, const int64_t *src,
                       const double *Lam, int64_t ldl, const double *X, int64_t ldx, double *grad,
                       cudaStream_t s)
{
    if (n <= 0) return;
    solve_grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, nrhs, rp, ci, src, Lam, ldl, X, ldx,
                                                                  grad);
}

}  // namespace spx
