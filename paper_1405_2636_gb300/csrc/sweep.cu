// sweep.cu -- forward and backward substitution on the panel factor, each
// direction one launch over a device-resident queue of work items.
//
// The items are the per-panel steps of the triangular solves in elimination
// order (Sec. III orders the factorization tasks the same way): a panel item
// applies the inverted diagonal block, a chunk item moves 64 off-diagonal
// rows of a panel between the panel and its ancestors.  CTAs take items from
// one atomic counter in queue order; an item waits on per-panel counters for
// the items it depends on, all of which sit earlier in the queue, so the
// earliest unfinished item always has its inputs and the walk cannot stall.
// Every wait is bounded: past the limit the kernel sets *err and its CTAs
// return, which the host reports as a failed solve.
//
// Forward (L y = b):
//   panel p  waits until every chunk writing into rows of p has finished,
//            then Z_p = Linv_p Y_p and flag[p] = 1;
//   chunk    waits for flag[p] of its panel, Y[rows] -= L_chunk Z_p, then
//            counts itself on each panel owning one of its rows.
// Backward (L^T x = y):
//   chunk    waits for flag[q] of each panel q owning one of its rows, then
//            Tacc_p += L_chunk^T X[rows] and counts itself on its panel;
//   panel p  waits for all its chunks, X_p = M (Z_p - Tacc_p), flag[p] = 1.
// Right-hand sides are column-major n x nrhs in the permuted numbering.
#include "kernels.cuh"

namespace spx {

namespace {

constexpr int kQRhs = 16;                   // right-hand sides per pass
constexpr int kQThreads = 256;

__device__ __forceinline__ int ld_acquire(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Polled by one thread.  False, with *err set, after `limit` polls (of
// about 256 ns each), or as soon as another CTA has reported a timeout.
__device__ bool wait_geq(const int32_t *p, int target, int32_t *err, uint32_t limit)
{
    if (ld_acquire(p) >= target) return true;
    for (uint32_t it = 0; it < limit; ++it) {
        __nanosleep(it < 256 ? 32 : 256);
        if (ld_acquire(p) >= target) return true;
        if ((it & 1023) == 1023 && ld_acquire(err) != 0) return false;
    }
    atomicExch(err, 1);
    return false;
}

// Data written by other CTAs of the same launch is read through L2.
template <typename T>
__device__ __forceinline__ T ld_l2(const T *p)
{
    return __ldcg(p);
}

// Whole CTA: true once every polled counter reached its target.  Thread t
// polls cnt[ids[t]] (ids == nullptr: thread 0 polls cnt[0]) for t < m.
__device__ __forceinline__ bool cta_wait(const int32_t *cnt, const int32_t *ids, int m, int target,
                                         int32_t *err, uint32_t limit)
{
    int ok = 1;
    if ((int)threadIdx.x < m) ok = wait_geq(cnt + (ids ? ids[threadIdx.x] : 0), target, err, limit);
    return __syncthreads_and(ok) != 0;
}

// Whole CTA, after its writes: they become visible before flag[0] = 1 and
// before each cnt[ids[t]] (t < m; ids == nullptr: cnt[0]) is incremented
// (barrier, then one gpu-scope acquire-release fence by the signalling
// thread, which covers the writes the barrier ordered before it).
__device__ __forceinline__ void cta_release(int32_t *flag, int32_t *cnt, const int32_t *ids, int m)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (flag) atomicExch(flag, 1);
        for (int t = 0; t < m; ++t) atomicAdd(cnt + (ids ? ids[t] : 0), 1);
    }
}

// The factor's blocks (read-only during a sweep) go to shared memory by
// asynchronous copies (cp.async, one element each, zero-filled past the
// panel): every copy of an item is in flight at once, beside the item's
// dependency wait, and stage_wait() before the barrier that precedes their
// first use completes them.  The right-hand sides, written by other CTAs
// of the same launch, are read through L2 after the wait; those staging
// loops issue every load of a batch before its first store.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool valid)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst);
    const int bytes = valid ? (int)sizeof(T) : 0;
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(saddr), "l"(src), "r"(bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(saddr), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void stage_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// This thread's asynchronous copies are done (a barrier after it makes
// every thread's visible to the CTA).
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Rows [r0, r0 + 64) of a panel's off-diagonal block to dst[k * ld + r]
// (rows past the panel as zeros).
template <typename T>
__device__ __forceinline__ void stage_chunk(T *dst, int ld, const T *Pn, int h, int w, int r0, int nr)
{
    const int total = w * 64;
    for (int e = threadIdx.x; e < total; e += kQThreads) {
        const int r = e & 63, k = e >> 6;
        const bool ok = r < nr;
        cp_async_elem(dst + k * ld + r, ok ? Pn + r0 + r + (int64_t)k * h : Pn, ok);
    }
    stage_commit();
}

// dst[e] = src[e], e < total (a diagonal block's inverse, column-major).
template <typename T>
__device__ __forceinline__ void stage_copy(T *dst, const T *src, int total)
{
    for (int e = threadIdx.x; e < total; e += kQThreads) cp_async_elem(dst + e, src + e, true);
    stage_commit();
}

// Right-hand-side blocks in shared memory hold kQRhs columns per row, the
// four column quads of row k in the order q ^ ((k >> 1) & 3): a thread
// reads its quad of one row with one vector load (the same address across
// a warp), and the column-wise staging stores spread over eight banks.
__device__ __forceinline__ int vslot(int k, int c)
{
    return k * kQRhs + ((((c >> 2) ^ (k >> 1)) & 3) << 2) + (c & 3);
}
template <typename T>
__device__ __forceinline__ void ld_quad(const T *Vs, int k, int g, T (&v)[4])
{
    const T *p = Vs + vslot(k, 4 * g);
    if constexpr (sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
        const double2 x = *reinterpret_cast<const double2 *>(p);
        const double2 y = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
    }
}
template <typename T>
__device__ __forceinline__ void st_quad(T *Vs, int k, int g, const T (&v)[4])
{
    T *p = Vs + vslot(k, 4 * g);
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
    }
}

// Vs(k, c) = V[f + k, c0 + c] for k < w (zero past nc), read through L2.
template <typename T>
__device__ __forceinline__ void stage_vec(T *Vs, const T *V, int64_t f, int w, int nc, int64_t n, int c0)
{
    constexpr int NB = 4;
    const int total = w * kQRhs;
    for (int base = threadIdx.x; base < total; base += kQThreads * NB) {
        T v[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = base + q * kQThreads, k = e % w, c = e / w;
            v[q] = (e < total && c < nc) ? ld_l2(V + f + k + (int64_t)(c0 + c) * n) : (T)0;
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = base + q * kQThreads;
            if (e < total) Vs[vslot(e % w, e / w)] = v[q];
        }
    }
}

// Xs(r, c) = X[row_r, c0 + c] (r < 64, zero past nr or nc); the thread's
// rows are all r = tid & 63, whose index `row` it loaded beforehand.
template <typename T>
__device__ __forceinline__ void stage_rows(T *Xs, const T *X, int64_t row, int nr, int nc, int64_t n, int c0)
{
    constexpr int NC = kQRhs / (kQThreads / 64);   // columns per thread
    const int r = threadIdx.x & 63, cf = threadIdx.x >> 6;
    T v[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const int c = cf + q * (kQThreads / 64);
        v[q] = (r < nr && c < nc) ? ld_l2(X + row + (int64_t)(c0 + c) * n) : (T)0;
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) Xs[vslot(r, cf + q * (kQThreads / 64))] = v[q];
}

// Y[row_r, c0 + 4g + u] -= sum_k Lc(r, k) Zs(k, 4g + u) for thread (r, g) =
// (tid & 63, tid >> 6); Lc staged [k * 64 + r].
template <typename T>
__device__ __forceinline__ void fwd_chunk_pass(const T *Lc, const T *Zs, int w, int nr, int nc, int64_t row,
                                               T *Y, int64_t n, int c0)
{
    const int r = threadIdx.x & 63, g = threadIdx.x >> 6;
    if (r >= nr) return;
    T acc[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll 4
    for (int k = 0; k < w; ++k) {
        const T l = Lc[k * 64 + r];
        T z[4];
        ld_quad(Zs, k, g, z);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += l * z[u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = 4 * g + u;
        if (c < nc) atomicAdd(Y + row + (int64_t)(c0 + c) * n, -acc[u]);
    }
}

// acc[u] += sum over r of Lc(r, k) Xs(r, 4g + u), Lc staged [k * 65 + r].
template <typename T>
__device__ __forceinline__ void chunk_dot4(const T *Lc, const T *Xs, int k, int g, T (&acc)[4])
{
#pragma unroll 4
    for (int r = 0; r < 64; ++r) {
        const T l = Lc[k * 65 + r];
        T x[4];
        ld_quad(Xs, r, g, x);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += l * x[u];
    }
}

}  // namespace

// Shared memory: A (q.mat_elems: a diagonal block, or a chunk), B
// (q.matb_elems: the chunk a panel item takes along), a vector of
// q.vec_elems and, when panel items take chunks along, a second one.
// Threads work as (row, column quad) = (tid & 63, tid >> 6).  FP32 factors:
// five CTAs per SM (41.5 KB of shared memory each for 64-wide panels, at
// most 48 registers a thread), so that more items' loads are in flight.
template <typename T>
__global__ void __launch_bounds__(kQThreads, sizeof(T) == 4 ? 5 : 4) fwd_queue_kernel(DevPlan p, SweepQueue q,
                                                              const RowChunk *__restrict__ chunks,
                                                              const T *__restrict__ Dinv, int unit,
                                                              const T *__restrict__ L, T *Y, T *Z, int nrhs)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T *matA = reinterpret_cast<T *>(smraw);
    T *matB = matA + q.mat_elems;
    T *vec = matB + q.matb_elems;
    T *vec2 = vec + q.vec_elems;
    __shared__ int s_next;
    const int tid = threadIdx.x, rt = tid & 63, g = tid >> 6;
    const int64_t n = p.n;
    if (tid == 0) s_next = atomicAdd(q.head, 1);
    __syncthreads();
    for (;;) {
        const int idx = s_next;
        __syncthreads();
        if (idx >= q.nitems) return;
        const int item = q.items[idx];
        if (tid == 0) s_next = atomicAdd(q.head, 1);   // the next item, fetched early
        if (item < 0) {
            // panel: Z_p = Linv_p Y_p (LU / LDL^T: unit Linv), then its
            // first chunk when it takes one along
            const int pid = -item - 1;
            const int w = p.pw[pid], h = p.ph[pid];
            const int64_t f = p.pfcol[pid];
            const T *Mi = Dinv + p.pinv[pid];
            const int mc = q.merge[pid];
            stage_copy(matA, Mi, w * w);   // column-major, ld w
            int nr = 0;
            int64_t row = 0;
            if (mc >= 0) {
                nr = min(64, h - w);
                stage_chunk(matB, 64, L + p.pval[pid], h, w, w, nr);
                if (rt < nr) row = p.rows[p.prow[pid] + w + rt];
            }
            if (!cta_wait(q.cnt + pid, nullptr, 1, q.need[pid], q.err, q.spin_limit)) {
                stage_wait();   // no copy left in flight on the way out
                return;
            }
            for (int c0 = 0; c0 < nrhs; c0 += kQRhs) {
                const int nc = min(kQRhs, nrhs - c0);
                stage_vec(vec, Y, f, w, nc, n, c0);
                stage_wait();
                __syncthreads();
                for (int i = rt; i < w; i += 64) {
                    T acc[4];
                    if (unit) ld_quad(vec, i, g, acc);
                    else acc[0] = acc[1] = acc[2] = acc[3] = (T)0;
                    const int kl = unit ? i : i + 1;
#pragma unroll 4
                    for (int k = 0; k < kl; ++k) {
                        const T a = matA[i + k * w];
                        T y[4];
                        ld_quad(vec, k, g, y);
#pragma unroll
                        for (int u = 0; u < 4; ++u) acc[u] += a * y[u];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 4 * g + u;
                        if (c < nc) Z[f + i + (int64_t)(c0 + c) * n] = acc[u];
                    }
                    if (mc >= 0) st_quad(vec2, i, g, acc);
                }
                __syncthreads();
                if (mc >= 0) {
                    fwd_chunk_pass(matB, vec2, w, nr, nc, row, Y, n, c0);
                    __syncthreads();
                }
            }
            const int t0 = mc >= 0 ? q.tptr[mc] : 0, t1 = mc >= 0 ? q.tptr[mc + 1] : 0;
            cta_release(q.flag + pid, q.cnt, q.tgt + t0, t1 - t0);
        } else {
            // chunk: Y[rows] -= L(rows, :) Z_p
            const RowChunk ch = chunks[item];
            const int pid = ch.panel;
            const int w = p.pw[pid], h = p.ph[pid];
            const int64_t f = p.pfcol[pid];
            const int nr = min(64, h - ch.r0);
            stage_chunk(matA, 64, L + p.pval[pid], h, w, ch.r0, nr);
            const int64_t row = rt < nr ? p.rows[p.prow[pid] + ch.r0 + rt] : 0;
            if (!cta_wait(q.flag + pid, nullptr, 1, 1, q.err, q.spin_limit)) {
                stage_wait();   // no copy left in flight on the way out
                return;
            }
            for (int c0 = 0; c0 < nrhs; c0 += kQRhs) {
                const int nc = min(kQRhs, nrhs - c0);
                stage_vec(vec, Z, f, w, nc, n, c0);
                stage_wait();
                __syncthreads();
                fwd_chunk_pass(matA, vec, w, nr, nc, row, Y, n, c0);
                __syncthreads();
            }
            const int t0 = q.tptr[item], t1 = q.tptr[item + 1];
            cta_release(nullptr, q.cnt, q.tgt + t0, t1 - t0);
        }
    }
}

// lu: 0 Cholesky (M = Linv^T), 1 LU (M = U^{-1}), 2 LDL^T
// (X_p = l^{-T} (D^{-1} Z_p - Tacc_p), 1/d on the diagonal of Dinv).
template <typename T>
__global__ void __launch_bounds__(kQThreads, sizeof(T) == 4 ? 5 : 4) bwd_queue_kernel(DevPlan p, SweepQueue q,
                                                              const RowChunk *__restrict__ chunks,
                                                              const T *__restrict__ Dinv, int lu,
                                                              const T *__restrict__ Lop,
                                                              const T *__restrict__ Z, T *Tacc, T *X,
                                                              int nrhs)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T *matA = reinterpret_cast<T *>(smraw);
    T *matB = matA + q.mat_elems;
    T *vec = matB + q.matb_elems;
    T *vec2 = vec + q.vec_elems;
    __shared__ int s_next;
    const int tid = threadIdx.x, rt = tid & 63, g = tid >> 6;
    const int64_t n = p.n;
    if (tid == 0) s_next = atomicAdd(q.head, 1);
    __syncthreads();
    for (;;) {
        const int idx = s_next;
        __syncthreads();
        if (idx >= q.nitems) return;
        const int item = q.items[idx];
        if (tid == 0) s_next = atomicAdd(q.head, 1);
        if (item < 0) {
            // panel: X_p = M (Z_p - Tacc_p - Lc^T X[rows of its first chunk])
            const int pid = -item - 1;
            // ld odd, so that a warp's rows i of M(i, k) = matA[k + i ld] fall
            // in distinct banks
            const int w = p.pw[pid], h = p.ph[pid], ld = (w & 1) ? w + 2 : w + 1;
            const int64_t f = p.pfcol[pid];
            const T *Mi = Dinv + p.pinv[pid];
            const int mc = q.merge[pid];
            // the stored inverse as it is, column-major with leading dimension ld (by
            // asynchronous copies): M(i, k) is matA[i + k ld] for LU (U^{-1})
            // and matA[k + i ld] = Linv(k, i) otherwise; only k >= i is read
            for (int e = tid; e < w * w; e += kQThreads) cp_async_elem(matA + (e % w) + (e / w) * ld, Mi + e, true);
            stage_commit();
            int nr = 0, t0 = 0, m = 0;
            int64_t row = 0;
            if (mc >= 0) {
                nr = min(64, h - w);
                stage_chunk(matB, 65, Lop + p.pval[pid], h, w, w, nr);
                if (rt < nr) row = p.rows[p.prow[pid] + w + rt];
                t0 = q.tptr[mc];
                m = q.tptr[mc + 1] - t0;
            }
            // the first pass's Z_p (LDL^T: D^{-1} Z_p) is fixed: staged
            // before the wait, Tacc_p subtracted after it by the same threads
            const int nc0 = min(kQRhs, nrhs);
            for (int base = tid; base < w * kQRhs; base += kQThreads * 4) {
                T v[4], dg[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = base + q * kQThreads, k = e % w, c = e / w;
                    const bool ok = e < w * kQRhs && c < nc0;
                    v[q] = ok ? Z[f + k + (int64_t)c * n] : (T)0;
                    dg[q] = (ok && lu == 2) ? Mi[k + k * w] : (T)1;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = base + q * kQThreads;
                    if (e < w * kQRhs) vec[vslot(e % w, e / w)] = lu == 2 ? v[q] * dg[q] : v[q];
                }
            }
            // one wait: threads < m on the panels owning the chunk's rows,
            // thread m on the panel's own chunks
            {
                int ok = 1;
                if (tid < m) ok = wait_geq(q.flag + q.tgt[t0 + tid], 1, q.err, q.spin_limit);
                else if (tid == m) ok = wait_geq(q.cnt + pid, q.need[pid], q.err, q.spin_limit);
                if (!__syncthreads_and(ok)) {
                    stage_wait();
                    return;
                }
            }
            for (int c0 = 0; c0 < nrhs; c0 += kQRhs) {
                const int nc = min(kQRhs, nrhs - c0);
                if (c0 > 0) {
                    __syncthreads();
                    for (int e = tid; e < w * kQRhs; e += kQThreads) {
                        const int k = e % w, c = e / w;
                        const int64_t gk = f + k + (int64_t)(c0 + c) * n;
                        vec[vslot(k, c)] = c < nc ? (lu == 2 ? Z[gk] * Mi[k + k * w] : Z[gk]) : (T)0;
                    }
                }
                // vec -= Tacc_p, and the chunk's rows of X: both read through
                // L2 in one batch (the X rows' loads go first, their stores
                // after Tacc's loads are in flight)
                constexpr int NCX = kQRhs / (kQThreads / 64);
                const int xr = tid & 63, xc = tid >> 6;
                T xv[NCX];
                if (mc >= 0) {
#pragma unroll
                    for (int q = 0; q < NCX; ++q) {
                        const int c = xc + q * (kQThreads / 64);
                        xv[q] = (xr < nr && c < nc) ? ld_l2(X + row + (int64_t)(c0 + c) * n) : (T)0;
                    }
                }
                for (int base = tid; base < w * kQRhs; base += kQThreads * 4) {
                    T t[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int e = base + q * kQThreads, k = e % w, c = e / w;
                        t[q] = (e < w * kQRhs && c < nc) ? ld_l2(Tacc + f + k + (int64_t)(c0 + c) * n) : (T)0;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int e = base + q * kQThreads;
                        if (e < w * kQRhs && e / w < nc) vec[vslot(e % w, e / w)] -= t[q];
                    }
                }
                if (mc >= 0) {
#pragma unroll
                    for (int q = 0; q < NCX; ++q) vec2[vslot(xr, xc + q * (kQThreads / 64))] = xv[q];
                }
                stage_wait();
                __syncthreads();
                if (mc >= 0) {   // vec -= Lc^T X[rows]
                    for (int k = rt; k < w; k += 64) {
                        T part[4] = {(T)0, (T)0, (T)0, (T)0};
                        chunk_dot4(matB, vec2, k, g, part);
                        T v[4];
                        ld_quad(vec, k, g, v);
#pragma unroll
                        for (int u = 0; u < 4; ++u) v[u] -= part[u];
                        st_quad(vec, k, g, v);
                    }
                    __syncthreads();
                }
                for (int i = rt; i < w; i += 64) {
                    T acc[4] = {(T)0, (T)0, (T)0, (T)0};
                    int k = i;
                    if (lu == 2) {   // LDL^T: l^{-T} has a unit diagonal
                        ld_quad(vec, i, g, acc);
                        ++k;
                    }
                    const int sa = lu == 1 ? 1 : ld, sk = lu == 1 ? ld : 1;   // M(i, k) = matA[i sa + k sk]
#pragma unroll 4
                    for (; k < w; ++k) {
                        const T a = matA[i * sa + k * sk];
                        T v[4];
                        ld_quad(vec, k, g, v);
#pragma unroll
                        for (int u = 0; u < 4; ++u) acc[u] += a * v[u];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 4 * g + u;
                        if (c < nc) X[f + i + (int64_t)(c0 + c) * n] = acc[u];
                    }
                }
            }
            cta_release(q.flag + pid, nullptr, nullptr, 0);
        } else {
            // chunk: Tacc_p += Lop(rows, :)^T X[rows]
            const RowChunk ch = chunks[item];
            const int pid = ch.panel;
            const int w = p.pw[pid], h = p.ph[pid];
            const int64_t f = p.pfcol[pid];
            const int nr = min(64, h - ch.r0);
            stage_chunk(matA, 65, Lop + p.pval[pid], h, w, ch.r0, nr);
            const int64_t row = rt < nr ? p.rows[p.prow[pid] + ch.r0 + rt] : 0;
            const int t0 = q.tptr[item], t1 = q.tptr[item + 1];
            if (!cta_wait(q.flag, q.tgt + t0, t1 - t0, 1, q.err, q.spin_limit)) {
                stage_wait();   // no copy left in flight on the way out
                return;
            }
            for (int c0 = 0; c0 < nrhs; c0 += kQRhs) {
                const int nc = min(kQRhs, nrhs - c0);
                stage_rows(vec, X, row, nr, nc, n, c0);
                stage_wait();
                __syncthreads();
                for (int k = rt; k < w; k += 64) {
                    T acc[4] = {(T)0, (T)0, (T)0, (T)0};
                    chunk_dot4(matA, vec, k, g, acc);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 4 * g + u;
                        if (c < nc) atomicAdd(Tacc + f + k + (int64_t)(c0 + c) * n, acc[u]);
                    }
                }
                __syncthreads();
            }
            cta_release(nullptr, q.cnt + pid, nullptr, 1);
        }
    }
}

namespace {

template <typename K>
unsigned queue_grid(K kernel, size_t smem, int nitems)
{
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    set_max_carveout(kernel);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kQThreads, smem);
    const long long g = (long long)std::max(occ, 1) * std::max(sms, 1);
    return (unsigned)std::max(1LL, std::min<long long>(g, nitems));
}

template <typename T>
size_t queue_smem(const SweepQueue &q)
{
    return sizeof(T) * ((size_t)q.mat_elems + (size_t)q.matb_elems + (q.matb_elems ? 2 : 1) * (size_t)q.vec_elems);
}

}  // namespace

template <typename T>
void launch_fwd_queue(const DevPlan &p, const SweepQueue &q, const RowChunk *chunks, const T *Dinv,
                      int unit, const T *L, T *Y, T *Z, int nrhs, cudaStream_t s)
{
    if (q.nitems <= 0) return;
    const size_t smem = queue_smem<T>(q);
    const unsigned grid = queue_grid(fwd_queue_kernel<T>, smem, q.nitems);
    fwd_queue_kernel<T><<<grid, kQThreads, smem, s>>>(p, q, chunks, Dinv, unit, L, Y, Z, nrhs);
}

template <typename T>
void launch_bwd_queue(const DevPlan &p, const SweepQueue &q, const RowChunk *chunks, const T *Dinv,
                      int lu, const T *Lop, const T *Z, T *Tacc, T *X, int nrhs, cudaStream_t s)
{
    if (q.nitems <= 0) return;
    const size_t smem = queue_smem<T>(q);
    const unsigned grid = queue_grid(bwd_queue_kernel<T>, smem, q.nitems);
    bwd_queue_kernel<T><<<grid, kQThreads, smem, s>>>(p, q, chunks, Dinv, lu, Lop, Z, Tacc, X, nrhs);
}

template void launch_fwd_queue<double>(const DevPlan &, const SweepQueue &, const RowChunk *, const double *, int,
                                       const double *, double *, double *, int, cudaStream_t);
template void launch_fwd_queue<float>(const DevPlan &, const SweepQueue &, const RowChunk *, const float *, int,
                                      const float *, float *, float *, int, cudaStream_t);
template void launch_bwd_queue<double>(const DevPlan &, const SweepQueue &, const RowChunk *, const double *, int,
                                       const double *, const double *, double *, double *, int, cudaStream_t);
template void launch_bwd_queue<float>(const DevPlan &, const SweepQueue &, const RowChunk *, const float *, int,
                                      const float *, const float *, float *, float *, int, cudaStream_t);

}  // namespace spx
