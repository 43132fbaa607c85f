// update_tc.cu -- the supernodal update (Sec. V-B) on the 5th-generation
// tensor cores: W = A_rows(M) * A_rows(N)^T with TF32 or BF16 operands (or
// FP32 operands split into two TF32 halves, hi*hi + hi*lo + lo*hi, for
// FP32-level products) and an FP32 accumulator in tensor memory, then the
// index-mapped scatter-subtract of W into the FP32 target panel (fused
// epilogue, no temporary buffer).
//
// Operands come from the K-major operand copy of every panel (row r of panel
// p at operand row prow[p] + r, Kpad elements per row, TF32-rounded or BF16),
// written by the TRSM kernel.  One 2-D TMA descriptor covers the whole copy;
// a tile is loaded as 128 rows x 128 bytes with the 128-byte swizzle, the
// canonical K-major layout of the MMA's shared-memory operand descriptors.
//
// One CTA = one 128 x 128 output tile of one (source, target) task:
//   thread 0      issues the TMA loads (2-stage ring) and the MMAs,
//   all 4 warps   read their 32 TMEM lanes and scatter the rows they own.
// Every wait on an mbarrier is bounded; on expiry the CTA records an error
// code, skips the epilogue and still releases its tensor memory.
#include "tc_common.cuh"

#include <algorithm>

namespace spx {
namespace {

using namespace tc;

// KIND 0: TF32 operands (32 per 128-byte row chunk); KIND 1: BF16 (64);
// KIND 2: split TF32 (hi and lo copies, three MMAs per K step);
// KIND 3 / 4: TF32 / BF16 for LDL^T -- A rows from the L copy (opmap), B rows
// from the D L^T copy (opmap_lo), so that the product is L D L^T (Sec. V-B).
template <int KIND>
__global__ void __launch_bounds__(128, 1)
    update_tc_kernel(const __grid_constant__ CUtensorMap opmap,
                     const __grid_constant__ CUtensorMap opmap_lo, DevPlan p,
                     const DevTask *__restrict__ tasks, const TcTile *__restrict__ tiles,
                     float *__restrict__ C, int lower, int *err)
{
    constexpr int kBase = KIND == 3 ? 0 : (KIND == 4 ? 1 : KIND);   // operand type of the MMA
    constexpr bool kSepB = KIND >= 3;                      // B from the second copy
    constexpr int kElems = kBase == 1 ? 64 : 32;           // K elements per stage
    constexpr uint32_t kIdesc = make_idesc(kBase == 1 ? 1u : 2u);
    constexpr int kParts = KIND == 2 ? 2 : 1;              // hi (and lo) copies per operand
    constexpr uint32_t kStageTx = 2u * kParts * kTileBytes;
    extern __shared__ unsigned char smraw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    // stage s: A_hi, B_hi (, A_lo, B_lo) tiles of kTileBytes each
    unsigned char *sA = base;
    unsigned char *sB = base + kStages * kTileBytes;
    unsigned char *sAl = base + 2 * kStages * kTileBytes;
    unsigned char *sBl = base + 3 * kStages * kTileBytes;
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ __align__(8) uint64_t empty[kStages];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ int64_t s_coff[kN];   // target column offset of each facing row of the tile

    const TcTile tl = tiles[blockIdx.x];
    const DevTask tk = tasks[tl.task];
    const int src = tk.src, tgt = tk.tgt;
    const int h = p.ph[src], K = p.pw[src];
    const int nk = (K + kElems - 1) / kElems;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (threadIdx.x == 0) {
        const int64_t rbase = p.prow[src];
        const int ya = (int)(rbase + tl.m0), yb = (int)(rbase + tl.n0);
        bool ok = true;
        const CUtensorMap *mapb = kSepB ? &opmap_lo : &opmap;
        for (int kc = 0; kc < nk && kc < kStages; ++kc) {
            mbar_expect_tx(&full[kc], kStageTx);
            tma_load_2d(sA + kc * kTileBytes, &opmap, &full[kc], kc * kElems, ya);
            tma_load_2d(sB + kc * kTileBytes, mapb, &full[kc], kc * kElems, yb);
            if (KIND == 2) {
                tma_load_2d(sAl + kc * kTileBytes, &opmap_lo, &full[kc], kc * kElems, ya);
                tma_load_2d(sBl + kc * kTileBytes, &opmap_lo, &full[kc], kc * kElems, yb);
            }
        }
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % kStages;
            const uint32_t ph = (uint32_t)(kc / kStages) & 1u;
            if (!mbar_wait(&full[s], ph)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA + s * kTileBytes), b0 = smem_u32(sB + s * kTileBytes);
            const uint32_t al = smem_u32(sAl + s * kTileBytes), bl = smem_u32(sBl + s * kTileBytes);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {   // 32 bytes of K per MMA
                if (KIND == 2) {               // small products first
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
            if (kc + kStages < nk) {
                if (!mbar_wait(&empty[s], ph)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(&full[s], kStageTx);
                tma_load_2d(sA + s * kTileBytes, &opmap, &full[s], (kc + kStages) * kElems, ya);
                tma_load_2d(sB + s * kTileBytes, mapb, &full[s], (kc + kStages) * kElems, yb);
                if (KIND == 2) {
                    tma_load_2d(sAl + s * kTileBytes, &opmap_lo, &full[s], (kc + kStages) * kElems, ya);
                    tma_load_2d(sBl + s * kTileBytes, &opmap_lo, &full[s], (kc + kStages) * kElems, yb);
                }
            }
        }
        mma_commit(&done);   // arrives once every MMA issued above has completed
        if (!ok) s_fail = 1;
    }
    // while the MMAs run: the target column offset of each of the tile's
    // facing rows, so that the epilogue scatters without global lookups
    {
        const int j = tl.n0 + (int)threadIdx.x;
        if (threadIdx.x < kN)
            s_coff[threadIdx.x] = j < tk.r1 ? (int64_t)(p.rows[p.prow[src] + j] - p.pfcol[tgt]) * p.ph[tgt] : 0;
    }
    __syncwarp();
    const bool got = mbar_wait(&done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (!got || s_fail) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else {
        float *Ct = C + p.pval[tgt];
        const int32_t *rmap = p.relmap + tk.relmap_off - tk.r0;
        const int i = tl.m0 + warp * 32 + lane;
        const bool row_ok = i < h;
        const int64_t roff = row_ok ? (int64_t)rmap[i] : 0;
        const int jend = min(tk.r1, tl.n0 + kN);
        for (int c0 = 0; tl.n0 + c0 < jend; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) {
                const int j = tl.n0 + c0 + cc;
                if (j >= jend) break;
                if (row_ok && (!lower || i >= j)) atomicAdd(Ct + roff + s_coff[c0 + cc], -__uint_as_float(v[cc]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

// Persistent form, for launches of more tiles than SMs: one CTA per SM,
// CTA b taking tiles b, b + gridDim.x, ... with two TMEM accumulators, so that the epilogue of
// one tile overlaps the loads and MMAs of the next.
//   warp 8 (one thread)  the TMA loads into the operand ring and the MMAs
//                        of tile i into accumulator i & 1;
//   warps 0-7            the epilogue of every tile from its accumulator:
//                        warp w reads TMEM lanes 32 (w % 4) .. + 31 and
//                        scatters columns 64 (w / 4) .. + 63, with its own
//                        copy of their target column offsets (no barrier
//                        among the epilogue warps).
// Hand-offs: full / empty per ring stage (TMA bytes / MMA completion),
// acc_full per accumulator (MMA completion), acc_empty per accumulator (one
// arrival per epilogue warp, eight).  Every wait is bounded and also gives up once
// another role has failed; the CTA then records an error and still releases
// its tensor memory.
constexpr uint32_t kPersistCols = 2 * kTmemCols;
constexpr int kEpiWarps = 8;
constexpr int kPersistThreads = 32 * (kEpiWarps + 1);

template <int KIND>
__global__ void __launch_bounds__(kPersistThreads, 1)
    update_tc_persistent(const __grid_constant__ CUtensorMap opmap,
                         const __grid_constant__ CUtensorMap opmap_lo, DevPlan p,
                         const DevTask *__restrict__ tasks, const TcTile *__restrict__ tiles, int count,
                         float *__restrict__ C, int lower, int *err)
{
    constexpr int kBase = KIND == 3 ? 0 : (KIND == 4 ? 1 : KIND);
    constexpr bool kSepB = KIND >= 3;
    constexpr int kElems = kBase == 1 ? 64 : 32;
    constexpr uint32_t kIdesc = make_idesc(kBase == 1 ? 1u : 2u);
    constexpr int kParts = KIND == 2 ? 2 : 1;
    constexpr uint32_t kStageTx = 2u * kParts * kTileBytes;
    extern __shared__ unsigned char smraw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = base + kStages * kTileBytes;
    unsigned char *sAl = base + 2 * kStages * kTileBytes;
    unsigned char *sBl = base + 3 * kStages * kTileBytes;
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ __align__(8) uint64_t empty[kStages];
    __shared__ __align__(8) uint64_t acc_full[2];
    __shared__ __align__(8) uint64_t acc_empty[2];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_fail;
    __shared__ int64_t s_coff[kEpiWarps][kN / 2];   // per epilogue warp, its half of the columns
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);
        }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kPersistCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (warp == kEpiWarps) {
        if (lane == 0) {
            const CUtensorMap *mapb = kSepB ? &opmap_lo : &opmap;
            uint32_t it = 0;   // operand chunks loaded so far: the ring position
            int lt = 0;        // this CTA's tiles so far
            bool ok = true;
            for (int t = blockIdx.x; t < count && ok; t += gridDim.x, ++lt) {
                const TcTile tl = tiles[t];
                const DevTask tk = tasks[tl.task];
                const int src = tk.src, K = p.pw[src];
                const int nk = (K + kElems - 1) / kElems;
                const int64_t rbase = p.prow[src];
                const int ya = (int)(rbase + tl.m0), yb = (int)(rbase + tl.n0);
                const int b = lt & 1;
                const uint32_t acc = tmem + (uint32_t)(b * (int)kTmemCols);
                // chunk kc of this tile into ring slot j (after the slot's previous MMAs)
                auto load = [&](int kc, uint32_t j) -> bool {
                    const int s = (int)(j % kStages);
                    const uint32_t u = j / kStages;
                    if (u >= 1 && !mbar_wait_or(&empty[s], (u - 1) & 1u, &s_fail)) return false;
                    mbar_expect_tx(&full[s], kStageTx);
                    tma_load_2d(sA + s * kTileBytes, &opmap, &full[s], kc * kElems, ya);
                    tma_load_2d(sB + s * kTileBytes, mapb, &full[s], kc * kElems, yb);
                    if (KIND == 2) {
                        tma_load_2d(sAl + s * kTileBytes, &opmap_lo, &full[s], kc * kElems, ya);
                        tma_load_2d(sBl + s * kTileBytes, &opmap_lo, &full[s], kc * kElems, yb);
                    }
                    return true;
                };
                const uint32_t it0 = it;
                for (int kc = 0; kc < nk && kc < kStages && ok; ++kc) ok = load(kc, it0 + (uint32_t)kc);
                // the accumulator must be drained of tile lt - 2
                if (ok && lt >= 2) ok = mbar_wait_or(&acc_empty[b], (uint32_t)((lt >> 1) - 1) & 1u, &s_fail);
                for (int kc = 0; kc < nk && ok; ++kc) {
                    const uint32_t j = it0 + (uint32_t)kc;
                    const int s = (int)(j % kStages);
                    if (!mbar_wait_or(&full[s], (j / kStages) & 1u, &s_fail)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(sA + s * kTileBytes), b0 = smem_u32(sB + s * kTileBytes);
                    const uint32_t al = smem_u32(sAl + s * kTileBytes), bl = smem_u32(sBl + s * kTileBytes);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        if (KIND == 2) {
                            mma<0>(acc, sw128_desc(al + 32 * ks), sw128_desc(b0 + 32 * ks), kIdesc,
                                   (kc > 0 || ks > 0) ? 1u : 0u);
                            mma<0>(acc, sw128_desc(a0 + 32 * ks), sw128_desc(bl + 32 * ks), kIdesc, 1u);
                            mma<0>(acc, sw128_desc(a0 + 32 * ks), sw128_desc(b0 + 32 * ks), kIdesc, 1u);
                        } else {
                            mma<kBase>(acc, sw128_desc(a0 + 32 * ks), sw128_desc(b0 + 32 * ks), kIdesc,
                                       (kc > 0 || ks > 0) ? 1u : 0u);
                        }
                    }
                    mma_commit(&empty[s]);
                    if (kc + kStages < nk) ok = load(kc + kStages, j + kStages);
                }
                if (ok) mma_commit(&acc_full[b]);   // arrives once this tile's MMAs completed
                it = it0 + (uint32_t)nk;
            }
            if (!ok) s_fail = 1;
        }
    } else {
        int lt = 0;
        for (int t = blockIdx.x; t < count; t += gridDim.x, ++lt) {
            const int b = lt & 1;
            const TcTile tl = tiles[t];
            const DevTask tk = tasks[tl.task];
            const int src = tk.src, tgt = tk.tgt, h = p.ph[src];
            const int quad = warp & 3, cbase = (warp >> 2) * (kN / 2);
            // this warp's copy of the target column offsets of its facing rows
            for (int c = lane; c < kN / 2; c += 32) {
                const int j = tl.n0 + cbase + c;
                s_coff[warp][c] = j < tk.r1 ? (int64_t)(p.rows[p.prow[src] + j] - p.pfcol[tgt]) * p.ph[tgt] : 0;
            }
            __syncwarp();
            if (!mbar_wait_or(&acc_full[b], (uint32_t)(lt >> 1) & 1u, &s_fail)) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float *Ct = C + p.pval[tgt];
            const int32_t *rmap = p.relmap + tk.relmap_off - tk.r0;
            const int i = tl.m0 + quad * 32 + lane;
            const bool row_ok = i < h;
            const int64_t roff = row_ok ? (int64_t)rmap[i] : 0;
            const int jend = min(tk.r1, tl.n0 + kN);
            const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * (int)kTmemCols);
            for (int c0 = cbase; c0 < cbase + kN / 2 && tl.n0 + c0 < jend; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(taddr + (uint32_t)c0, v);
#pragma unroll
                for (int cc = 0; cc < 16; ++cc) {
                    const int j = tl.n0 + c0 + cc;
                    if (j >= jend) break;
                    if (row_ok && (!lower || i >= j))
                        atomicAdd(Ct + roff + s_coff[warp][c0 - cbase + cc], -__uint_as_float(v[cc]));
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kPersistCols));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

size_t tc_smem_bytes(int kind) { return (size_t)(kind == 2 ? 4 : 2) * kStages * kTileBytes + 1024; }

int make_operand_map(void *tmap_out, void *base, int64_t rows, int kpad, int bf16)
{
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = (EncodeTiledFn)fn;
    }
    const int esz = bf16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kpad * esz};
    cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)kM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(reinterpret_cast<CUtensorMap *>(tmap_out),
                        bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

template <int KIND>
void launch_tc_kind(const CUtensorMap &m, const CUtensorMap &ml, const DevPlan &p, const DevTask *tasks,
                    const TcTile *tiles, int count, float *C, int lower, int *err, cudaStream_t s)
{
    static int nsm = 0;
    static bool once = false;
    const size_t smem = tc_smem_bytes(KIND);
    // the persistent form: one CTA per SM, which leaves room for the update
    // launches running beside it (measured faster than two); 80 KB of shared
    // memory each, so that at most two (of two launches) share an SM and
    // their 2 x 256 TMEM columns fit its 512
    const size_t psmem = std::max(smem, (size_t)80 * 1024);
    if (!once) {
        cudaFuncSetAttribute(update_tc_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(update_tc_persistent<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        once = true;
    }
    if (count > nsm) {
        const int grid = std::max(nsm, 1);
        update_tc_persistent<KIND><<<grid, kPersistThreads, psmem, s>>>(m, ml, p, tasks, tiles, count, C, lower, err);
    } else {
        update_tc_kernel<KIND><<<count, 128, smem, s>>>(m, ml, p, tasks, tiles, C, lower, err);
    }
}

void launch_update_tc(const void *tmap, const void *tmap_lo, int kind, const DevPlan &p,
                      const DevTask *tasks, const TcTile *tiles, int count, float *C, int lower,
                      int *err, cudaStream_t s)
{
    if (count <= 0) return;
    const CUtensorMap &m = *reinterpret_cast<const CUtensorMap *>(tmap);
    const CUtensorMap &ml = *reinterpret_cast<const CUtensorMap *>(kind >= 2 ? tmap_lo : tmap);
    switch (kind) {
    case 1: return launch_tc_kind<1>(m, ml, p, tasks, tiles, count, C, lower, err, s);
    case 2: return launch_tc_kind<2>(m, ml, p, tasks, tiles, count, C, lower, err, s);
    case 3: return launch_tc_kind<3>(m, ml, p, tasks, tiles, count, C, lower, err, s);
    case 4: return launch_tc_kind<4>(m, ml, p, tasks, tiles, count, C, lower, err, s);
    default: return launch_tc_kind<0>(m, ml, p, tasks, tiles, count, C, lower, err, s);
    }
}

}  // namespace spx
