// fqueue.cuh -- the upper levels of the factorization as one persistent
// launch over a device-resident task queue.
//
// Sec. III: the factorization is a DAG of tasks fixed by the block structure
// alone (it does not depend on the values): per panel the factorization of
// its diagonal block, the TRSM of its off-diagonal rows, and one update task
// per (source, target) pair of panels.  Near the root of the elimination
// tree every level holds a handful of panels, and a level-by-level walk
// serializes each level's diagonal blocks, TRSM and updates behind launch
// boundaries.  Here the items of those levels -- a panel's diagonal block, a
// 64-row TRSM chunk, an update tile (tcgen05 or CUDA cores) -- sit in one
// array in an order where every item's inputs come from earlier items
// (checked on the host before the first launch).  CTAs take items from one
// atomic counter and wait on per-item counters:
//   diagonal block of p : every update tile of the queue into p has finished;
//   TRSM chunk of p     : the diagonal block of p is factored;
//   update tile         : the TRSM chunks holding its source rows are done.
// The update tiles into the next level's panels come before that level's
// diagonal blocks and the other tiles right after them, so the far updates
// run while the next diagonal blocks factor.  The earliest unfinished item
// always has its inputs, so the walk cannot stall; every wait is bounded
// (past the limit the kernel records a timeout and its CTAs return).
//
// The per-item bodies are those of the level-by-level kernels (blocks.cuh);
// the tensor-core tile keeps its TMEM accumulator, mbarriers and TMA ring for
// the whole launch and reads the tile with all eight warps.
#pragma once

#include "blocks.cuh"
#include "tc_common.cuh"

#include <algorithm>

namespace spx {

template <typename T>
struct FqArgs {
    DevPlan p;
    FactorQueue q;
    const DevTask *tasks;
    const RowChunk *chunks;
    const UpdTile *tiles;      // CUDA-core tiles (FQ_UPD64, FQ_UPD16)
    const TcTile *tctiles;     // tensor-core tiles (FQ_TC)
    T *L, *Dinv, *W;           // W: the D L^T rows (LDL^T), B operand of the CUDA-core update
    const double *tau;
    int64_t *err_col;
    unsigned long long *nrepl, *nneg;
    void *opc, *opc_lo;        // operand copies written by the TRSM for the tensor cores
    int kpad, op_kind, trsm_mode;
};

namespace fq {

using namespace tc;

constexpr int kThreads = 256;

__device__ __forceinline__ int ld_acquire(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Polled by one thread.  False, with *err set, after `limit` polls, or as
// soon as another CTA has reported a timeout.
__device__ __forceinline__ bool wait_geq(const int32_t *p, int target, int32_t *err, uint32_t limit)
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

// Whole CTA, after its writes (stores and reductions): they become visible
// before *ctr is incremented (barrier, then one gpu-scope fence by the
// signalling thread, which covers the writes the barrier ordered before it).
__device__ __forceinline__ void release_add(int32_t *ctr)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        atomicAdd(ctr, 1);
    }
}

// The TRSM chunks holding rows [r_lo, r_hi) of panel src (rows >= width).
__device__ __forceinline__ void chunk_range(const DevPlan &p, const int32_t *pchunk, int src, int r_lo, int r_hi,
                                            int *c_lo, int *c_hi)
{
    const int w = p.pw[src];
    *c_lo = pchunk[src] + (r_lo - w) / kTrsmRows;
    *c_hi = pchunk[src] + (r_hi - 1 - w) / kTrsmRows;   // inclusive
}

// One 128 x 128 tensor-core tile of an update task: thread 0 streams the K
// chunks of both operands through a two-stage TMA ring (the ring position
// `ring` and the done barrier's phase `tile_no` carry over between tiles)
// and issues the MMAs into the TMEM accumulator; then the eight warps read
// it back (warp w: TMEM lanes 32 (w mod 4) .., columns 64 (w / 4) ..) and
// subtract it through the row map.  False if a pipeline wait gave up.
template <int KIND>
__device__ __forceinline__ bool tc_tile(const CUtensorMap *map, const CUtensorMap *map_lo, const DevPlan &p,
                                        const DevTask &tk, const TcTile &tl, float *__restrict__ C,
                                        unsigned char *base, uint64_t *full, uint64_t *empty, uint64_t *done,
                                        uint32_t tmem, uint32_t &ring, uint32_t tile_no, int64_t *s_coff)
{
    constexpr int kBase = KIND == 3 ? 0 : (KIND == 4 ? 1 : KIND);   // operand type of the MMA
    constexpr bool kSepB = KIND >= 3;                      // B from the second copy
    constexpr int kElems = kBase == 1 ? 64 : 32;           // K elements per stage
    constexpr uint32_t kIdesc = make_idesc(kBase == 1 ? 1u : 2u);
    constexpr int kParts = KIND == 2 ? 2 : 1;
    constexpr uint32_t kStageTx = 2u * kParts * kTileBytes;
    unsigned char *sA = base;
    unsigned char *sB = base + kStages * kTileBytes;
    unsigned char *sAl = base + 2 * kStages * kTileBytes;
    unsigned char *sBl = base + 3 * kStages * kTileBytes;
    const int src = tk.src, tgt = tk.tgt;
    const int h = p.ph[src], K = p.pw[src];
    const int nk = (K + kElems - 1) / kElems;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    bool issue_ok = true;   // thread 0: every pipeline wait came through
    if (tid == 0) {
        bool ok = true;
        // this shared memory was last written by the generic proxy (other
        // items), and the operand rows by other CTAs' TRSM (acquired)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const int64_t rbase = p.prow[src];
        const int ya = (int)(rbase + tl.m0), yb = (int)(rbase + tl.n0);
        const CUtensorMap *mapb = kSepB ? map_lo : map;
        auto load = [&](int kc) {
            const uint32_t s = (ring + kc) % kStages;
            mbar_expect_tx(&full[s], kStageTx);
            tma_load_2d(sA + s * kTileBytes, map, &full[s], kc * kElems, ya);
            tma_load_2d(sB + s * kTileBytes, mapb, &full[s], kc * kElems, yb);
            if (KIND == 2) {
                tma_load_2d(sAl + s * kTileBytes, map_lo, &full[s], kc * kElems, ya);
                tma_load_2d(sBl + s * kTileBytes, map_lo, &full[s], kc * kElems, yb);
            }
        };
        int issued = 0, consumed = 0;
        for (; issued < nk && issued < kStages; ++issued) load(issued);
        for (int kc = 0; kc < nk; ++kc) {
            const uint32_t g = ring + kc, s = g % kStages, ph = (g / kStages) & 1u;
            if (!mbar_wait(&full[s], ph)) {
                ok = false;
                break;
            }
            ++consumed;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA + s * kTileBytes), b0 = smem_u32(sB + s * kTileBytes);
            const uint32_t al = smem_u32(sAl + s * kTileBytes), bl = smem_u32(sBl + s * kTileBytes);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {   // 32 bytes of K per MMA
                if (KIND == 2) {
                    mma<0>(tmem, sw128_desc(al + 32 * ks), sw128_desc(b0 + 32 * ks), kIdesc,
                           (kc > 0 || ks > 0) ? 1u : 0u);
                    mma<0>(tmem, sw128_desc(a0 + 32 * ks), sw128_desc(bl + 32 * ks), kIdesc, 1u);
                    mma<0>(tmem, sw128_desc(a0 + 32 * ks), sw128_desc(b0 + 32 * ks), kIdesc, 1u);
                } else {
                    mma<kBase>(tmem, sw128_desc(a0 + 32 * ks), sw128_desc(b0 + 32 * ks), kIdesc,
                               (kc > 0 || ks > 0) ? 1u : 0u);
                }
            }
            mma_commit(&empty[s]);
            if (issued < nk) {
                if (!mbar_wait(&empty[s], ph)) {
                    ok = false;
                    break;
                }
                load(issued++);
            }
        }
        mma_commit(done);   // arrives once every MMA issued above has completed
        if (!ok) {
            // let the loads still in flight land before the CTA gives up
            for (int kc = consumed; kc < issued; ++kc) {
                const uint32_t g = ring + kc;
                mbar_wait(&full[g % kStages], (g / kStages) & 1u);
            }
        }
        ring += nk;
        issue_ok = ok;
    }
    // while the MMAs run: the target column offset of each facing row
    if (tid < kN) {
        const int j = tl.n0 + tid;
        s_coff[tid] = j < tk.r1 ? (int64_t)(p.rows[p.prow[src] + j] - p.pfcol[tgt]) * p.ph[tgt] : 0;
    }
    const bool got = mbar_wait(done, tile_no & 1u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = __syncthreads_and(got && issue_ok) != 0;
    if (ok) {
        const int q4 = warp & 3, half = warp >> 2;
        float *Ct = C + p.pval[tgt];
        const int32_t *rmap = p.relmap + tk.relmap_off - tk.r0;
        const int i = tl.m0 + q4 * 32 + lane;
        const bool row_ok = i < h;
        const int64_t roff = row_ok ? (int64_t)rmap[i] : 0;
        const int jend = min(tk.r1, tl.n0 + kN);
        for (int c0 = half * 64; c0 < half * 64 + 64 && tl.n0 + c0 < jend; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) {
                const int j = tl.n0 + c0 + cc;
                if (j >= jend) break;
                if (row_ok && i >= j) atomicAdd(Ct + roff + s_coff[c0 + cc], -__uint_as_float(v[cc]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    return ok;
}

template <typename T, bool LDLT, int TCK>
__host__ __device__ constexpr size_t smem_bytes()
{
    size_t b = ldl_smem_bytes<T, 64>();
    const size_t t = trsm_smem_bytes<T>(64);
    const size_t u = sizeof(T) * (update_smem_elems<T, 16>() > update_smem_elems<T, 64>()
                                      ? update_smem_elems<T, 16>() : update_smem_elems<T, 64>());
    const size_t c = TCK < 0 ? 0 : (size_t)(TCK == 2 ? 4 : 2) * kStages * kTileBytes;
    b = b > t ? b : t;
    b = b > u ? b : u;
    b = b > c ? b : c;
    return b + 1024;   // the tensor-core tiles start on a 1024-byte boundary
}

}  // namespace fq

// Resident CTAs per SM the kernel is compiled for: three for the
// single-precision factor (shared memory and registers allow it), two for
// FP64 and for split TF32 (larger staging).
template <typename T, int TCK>
__host__ __device__ constexpr int fq_min_blocks()
{
    return (sizeof(T) == 4 && TCK != 2) ? 3 : 2;
}

template <typename T, bool LDLT, int TCK>
__global__ void __launch_bounds__(fq::kThreads, fq_min_blocks<T, TCK>())
    factor_queue_kernel(const __grid_constant__ CUtensorMap opmap, const __grid_constant__ CUtensorMap opmap_lo,
                        const FqArgs<T> a)
{
    using namespace fq;
    extern __shared__ unsigned char smraw[];
    unsigned char *sm =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ __align__(8) uint64_t empty[kStages];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_next;
    __shared__ int64_t s_coff[kN];
    const FactorQueue &q = a.q;
    const DevPlan &p = a.p;
    const int tid = threadIdx.x;
    uint32_t ring = 0, tiles_done = 0;   // tensor-core ring position (thread 0) and tiles taken

    if (TCK >= 0) {
        if (tid == 0) {
            for (int s = 0; s < kStages; ++s) {
                mbar_init(&full[s], 1);
                mbar_init(&empty[s], 1);
            }
            mbar_init(&done, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (tid < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&s_tmem)),
                         "r"(kTmemCols));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (tid == 0) s_next = atomicAdd(q.head, 1);
    __syncthreads();
    if (TCK >= 0) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = TCK >= 0 ? s_tmem : 0u;

    for (;;) {
        const int idx = s_next;
        __syncthreads();
        if (idx >= q.nitems) break;
        const FqItem it = q.items[idx];
        if (tid == 0) s_next = atomicAdd(q.head, 1);   // the next item, fetched early
        bool ok = true;
        if (it.kind == FQ_DIAG) {
            const int pid = it.idx;
            int w_ok = 1;
            if (tid == 0) w_ok = wait_geq(q.cnt + pid, q.need[pid], q.err, q.spin_limit);
            if (!__syncthreads_and(w_ok)) break;
            const int w = p.pw[pid];
            double *ds = reinterpret_cast<double *>(sm);
            const double tau = *a.tau;
            if (w <= 16) ldl_diag_block<T, 16, LDLT>(p, pid, a.L, a.Dinv, tau, a.err_col, a.nrepl, a.nneg, ds);
            else if (w <= 32) ldl_diag_block<T, 32, LDLT>(p, pid, a.L, a.Dinv, tau, a.err_col, a.nrepl, a.nneg, ds);
            else ldl_diag_block<T, 64, LDLT>(p, pid, a.L, a.Dinv, tau, a.err_col, a.nrepl, a.nneg, ds);
            release_add(q.diag_done + pid);
        } else if (it.kind == FQ_TRSM) {
            const RowChunk ch = a.chunks[it.idx];
            int w_ok = 1;
            if (tid == 0) w_ok = wait_geq(q.diag_done + ch.panel, 1, q.err, q.spin_limit);
            if (!__syncthreads_and(w_ok)) break;
            trsm_chunk<T>(p, ch, a.Dinv, a.L, a.trsm_mode, a.opc, a.opc_lo, a.kpad, a.op_kind, a.W, sm);
            // the operand copy is read by other CTAs' TMA (async proxy)
            if (TCK >= 0) asm volatile("fence.proxy.async.global;" ::: "memory");
            release_add(q.chunk_done + it.idx);
        } else {
            // an update tile: wait for the TRSM chunks of its source rows
            int m0, n0, task, tm, tn;
            if (it.kind == FQ_TC) {
                const TcTile t = a.tctiles[it.idx];
                task = t.task, m0 = t.m0, n0 = t.n0, tm = kM, tn = kN;
            } else {
                const UpdTile t = a.tiles[it.idx];
                task = t.task, m0 = t.m0, n0 = t.n0;
                tn = it.kind == FQ_UPD16 ? kUpdNarrowN : kUpdTile;
                tm = 4096 / tn;
            }
            const DevTask tk = a.tasks[task];
            const int h = p.ph[tk.src];
            int a0, a1, b0, b1;
            chunk_range(p, q.pchunk, tk.src, m0, min(m0 + tm, h), &a0, &a1);
            chunk_range(p, q.pchunk, tk.src, n0, min(n0 + tn, tk.r1), &b0, &b1);
            const int na = a1 - a0 + 1, nb = b1 - b0 + 1;
            int w_ok = 1;
            if (tid < na) w_ok = wait_geq(q.chunk_done + a0 + tid, 1, q.err, q.spin_limit);
            else if (tid >= 32 && tid - 32 < nb) w_ok = wait_geq(q.chunk_done + b0 + tid - 32, 1, q.err, q.spin_limit);
            if (!__syncthreads_and(w_ok)) break;
            if (it.kind == FQ_TC) {
                if constexpr (TCK >= 0) {
                    const TcTile t = a.tctiles[it.idx];
                    ok = tc_tile<(TCK < 0 ? 0 : TCK)>(&opmap, &opmap_lo, p, tk, t, reinterpret_cast<float *>(a.L),
                                                      sm, full, empty, &done, tmem, ring, tiles_done, s_coff);
                    ++tiles_done;
                    if (!ok) {
                        if (tid == 0) atomicExch(q.err, 2);
                        break;
                    }
                }
            } else {
                const UpdTile t = a.tiles[it.idx];
                const T *Bop = LDLT ? a.W : a.L;
                if (it.kind == FQ_UPD16)
                    update_tile<T, 16>(p, tk, t, a.L, Bop, a.L, 1, 0, reinterpret_cast<T *>(sm));
                else
                    update_tile<T, 64>(p, tk, t, a.L, Bop, a.L, 1, 0, reinterpret_cast<T *>(sm));
            }
            release_add(q.cnt + tk.tgt);
        }
        (void)ok;
    }
    if (TCK >= 0) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid < 32)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

template <typename T, bool LDLT, int TCK>
int fq_grid()
{
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = fq::smem_bytes<T, LDLT, TCK>();
    cudaFuncSetAttribute(factor_queue_kernel<T, LDLT, TCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, factor_queue_kernel<T, LDLT, TCK>, fq::kThreads, smem);
    return std::max(occ, 1) * std::max(sms, 1);
}

template <typename T, bool LDLT, int TCK>
void fq_launch(const FqArgs<T> &a, const void *tmap, const void *tmap_lo, cudaStream_t s)
{
    if (a.q.nitems <= 0) return;
    static int grid = 0;
    if (!grid) grid = fq_grid<T, LDLT, TCK>();
    const int g = std::min(grid, a.q.nitems);
    CUtensorMap m{}, ml{};
    if (tmap) m = *reinterpret_cast<const CUtensorMap *>(tmap);
    if (tmap_lo) ml = *reinterpret_cast<const CUtensorMap *>(tmap_lo);
    factor_queue_kernel<T, LDLT, TCK><<<g, fq::kThreads, fq::smem_bytes<T, LDLT, TCK>(), s>>>(m, ml, a);
}

}  // namespace spx
