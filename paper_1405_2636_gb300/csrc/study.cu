// study.cu -- the supernodal update on its own: the kernel study of Sec. V-B
// (C = C - A B^T with B the first rows of A, C a taller target panel with a
// gapped block structure), run through the factorization's own update
// kernels.  A plan describes one (source, target) task exactly as the
// analysis would: the source panel's rows, the row map into the target
// (block containment, Sec. V-B) and the target columns of the facing rows;
// staging writes the source panel in the factorization's storage (column-
// major, and for the tensor cores the rounded K-major operand copy the TRSM
// writes); a run launches update_kernel (CUDA cores) or update_tc_kernel
// (tcgen05) over the task's tiles, with the same tile rules as the
// factorization.
#include "../../include/spx.h"
#include "kernels.cuh"
#include "operand.cuh"

#include <cuda_runtime.h>

#include <climits>
#include <cstring>
#include <new>
#include <string>
#include <vector>

struct spx_update_s {
    int64_t m = 0, nb = 0, k = 0, ldc = 0, nc = 0;
    int lower = 0, precision = 0, ldlt = 0;
    bool use_tc = false;
    int op_kind = 0, kpad = 0;
    spx::DevPlan dp{};
    spx::DevTask *d_task = nullptr;
    spx::UpdTile *d_tiles = nullptr;     // wide (64 x 64) tiles, then narrow (256 x 16) ones
    int ntiles = 0, nnarrow = 0;
    spx::TcTile *d_tct = nullptr;
    int ntct = 0;
    void *d_A = nullptr, *d_W = nullptr, *d_opc = nullptr, *d_opc_lo = nullptr;
    alignas(64) unsigned char tmap[128];
    alignas(64) unsigned char tmap_lo[128];
    int *d_err = nullptr;
    bool staged = false;
    std::vector<void *> allocs;
    std::string err;
};

namespace spx {
namespace {

template <typename T>
__global__ void stage_operand_kernel(int64_t m, int k, const T *__restrict__ A, const T *__restrict__ W,
                                     int64_t lda, void *opc, void *opc_lo, int kpad, int op_kind)
{
    const int64_t total = m * (int64_t)kpad;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / kpad;
        const int j = (int)(e % kpad);
        const float v = j < k ? (float)A[i + (int64_t)j * lda] : 0.0f;
        const float wv = (j < k && W) ? (float)W[i + (int64_t)j * lda] : 0.0f;
        put_operand(opc, opc_lo, e, op_kind, v, wv);
    }
}

std::string g_study_error;

spx_status ufail(spx_update_s *u, spx_status st, const std::string &msg)
{
    if (u) u->err = msg;
    else g_study_error = msg;
    return st;
}

#define UCU(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return ufail(u, SPX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
spx_status ualloc(spx_update_s *u, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return ufail(u, SPX_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    u->allocs.push_back(*p);
    return SPX_OK;
}

template <typename T>
spx_status uupload(spx_update_s *u, T **p, const std::vector<T> &v)
{
    spx_status st = ualloc(u, p, v.size());
    if (st != SPX_OK) return st;
    if (!v.empty()) UCU(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SPX_OK;
}

}  // namespace

template <typename T>
void launch_stage_operand(int64_t m, int k, const T *A, const T *W, int64_t lda, void *opc, void *opc_lo,
                          int kpad, int op_kind, cudaStream_t s)
{
    const int64_t total = m * (int64_t)kpad;
    if (total <= 0) return;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    stage_operand_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(m, k, A, W, lda, opc, opc_lo, kpad, op_kind);
}

template void launch_stage_operand<float>(int64_t, int, const float *, const float *, int64_t, void *, void *,
                                          int, int, cudaStream_t);
template void launch_stage_operand<double>(int64_t, int, const double *, const double *, int64_t, void *,
                                           void *, int, int, cudaStream_t);

}  // namespace spx

extern "C" {

spx_status spx_update_create(int64_t m, int64_t nb_rows, int64_t k, int64_t ldc, int64_t nc,
                             const int32_t *rowmap, const int32_t *colmap, int lower, spx_precision precision,
                             int engine, int ldlt, spx_update_plan *out)
{
    using namespace spx;
    spx_update_s *u = nullptr;
    if (!out) return ufail(u, SPX_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (m < 1 || nb_rows < 1 || nb_rows > m || k < 1 || ldc < 1 || nc < 1)
        return ufail(u, SPX_ERR_ARG, "sizes: need 1 <= nb_rows <= m, k >= 1, ldc >= 1, nc >= 1");
    if (m > INT32_MAX / 2 || k > INT32_MAX / 2 || ldc > INT32_MAX || nc > INT32_MAX)
        return ufail(u, SPX_ERR_ARG, "sizes above 2^30");
    if (!rowmap || !colmap) return ufail(u, SPX_ERR_ARG, "rowmap/colmap is NULL");
    if (precision < SPX_FP64 || precision > SPX_BF16) return ufail(u, SPX_ERR_ARG, "unknown precision");
    if (engine < 0 || engine > 2) return ufail(u, SPX_ERR_ARG, "engine must be 0, 1 or 2");
    for (int64_t i = 0; i < m; ++i)
        if (rowmap[i] < 0 || rowmap[i] >= ldc) return ufail(u, SPX_ERR_ARG, "rowmap entry outside [0, ldc)");
    for (int64_t j = 0; j < nb_rows; ++j)
        if (colmap[j] < 0 || colmap[j] >= nc) return ufail(u, SPX_ERR_ARG, "colmap entry outside [0, nc)");
    // the factorization's engine rule (api.cu: uses_tensor_cores, kTcMinWidth)
    const bool tc_mode = precision != SPX_FP64 && !(ldlt && precision == SPX_FP32);
    bool use_tc = engine == 2 || (engine == 0 && tc_mode && k >= 32);
    if (use_tc && !tc_mode)
        return ufail(u, SPX_ERR_ARG, "no tensor-core engine for this precision (FP64, or LDL^T in FP32)");
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return ufail(u, SPX_ERR_CUDA, "no CUDA device");
    if (prop.major * 10 + prop.minor != 103)
        return ufail(u, SPX_ERR_CUDA, "libspx is built for sm_103a; the current device is sm_" +
                                          std::to_string(prop.major * 10 + prop.minor));
    u = new (std::nothrow) spx_update_s();
    if (!u) return ufail(nullptr, SPX_ERR_ALLOC, "out of host memory");
    u->m = m;
    u->nb = nb_rows;
    u->k = k;
    u->ldc = ldc;
    u->nc = nc;
    u->lower = lower ? 1 : 0;
    u->precision = precision;
    u->ldlt = ldlt ? 1 : 0;
    u->use_tc = use_tc;
    u->op_kind = ldlt ? (precision == SPX_BF16 ? 4 : 3) : (precision == SPX_BF16 ? 1 : (precision == SPX_FP32 ? 2 : 0));
    u->kpad = (int)((k + 63) & ~63LL);

    // a two-panel plan: panel 0 is the source (m rows, width k), panel 1 the
    // target (ldc rows, nc columns starting at column 0); the facing rows of
    // the source are its first nb_rows rows, whose global indices are the
    // target columns they face
    std::vector<int64_t> pfcol = {0, 0}, prow = {0, m, m}, pval = {0, 0, 0};
    std::vector<int32_t> pw = {(int32_t)k, (int32_t)nc}, ph = {(int32_t)m, (int32_t)ldc};
    std::vector<int32_t> rows((size_t)m), relmap(rowmap, rowmap + m);
    for (int64_t i = 0; i < m; ++i) rows[(size_t)i] = i < nb_rows ? colmap[i] : rowmap[i];
    std::vector<DevTask> task = {DevTask{0, 1, 0, (int32_t)nb_rows, 0}};
    // tiles, as the factorization cuts one task (api.cu: add_tiles and the
    // tensor-core tile loop): lower targets skip tiles wholly above the diagonal
    std::vector<UpdTile> wide, narrow;
    std::vector<TcTile> tct;
    if (use_tc) {
        for (int32_t m0 = 0; m0 < m; m0 += 128)
            for (int32_t n0 = 0; n0 < nb_rows; n0 += 128) {
                if (u->lower && m0 + 128 <= n0) continue;
                tct.push_back(TcTile{0, m0, n0, 0});
            }
    } else {
        const int TN = nb_rows <= kUpdNarrowN ? kUpdNarrowN : kUpdTile;
        const int TM = 4096 / TN;
        for (int32_t m0 = 0; m0 < m; m0 += TM)
            for (int32_t n0 = 0; n0 < nb_rows; n0 += TN) {
                if (u->lower && m0 + TM <= n0) continue;
                (TN == kUpdTile ? wide : narrow).push_back(UpdTile{0, m0, n0, 0});
            }
    }
    u->ntiles = (int)wide.size();
    u->nnarrow = (int)narrow.size();
    wide.insert(wide.end(), narrow.begin(), narrow.end());
    u->ntct = (int)tct.size();
    int64_t *d_pfcol, *d_prow, *d_pval;
    int32_t *d_pw, *d_ph, *d_rows, *d_relmap;
    spx_status st;
    const size_t esz = precision == SPX_FP64 ? sizeof(double) : sizeof(float);
    char *pa = nullptr, *pwb = nullptr;
    if ((st = uupload(u, &d_pfcol, pfcol)) || (st = uupload(u, &d_prow, prow)) || (st = uupload(u, &d_pval, pval)) ||
        (st = uupload(u, &d_pw, pw)) || (st = uupload(u, &d_ph, ph)) || (st = uupload(u, &d_rows, rows)) ||
        (st = uupload(u, &d_relmap, relmap)) || (st = uupload(u, &u->d_task, task)) ||
        (st = uupload(u, &u->d_tiles, wide)) || (st = uupload(u, &u->d_tct, tct)) ||
        (st = ualloc(u, &u->d_err, 1)) || (st = ualloc(u, &pa, (size_t)m * k * esz)) ||
        (ldlt && (st = ualloc(u, &pwb, (size_t)m * k * esz)))) {
        g_study_error = u->err;
        spx_update_free(u);
        return st;
    }
    u->d_A = pa;
    u->d_W = pwb;
    u->dp.n = nc;
    u->dp.npanels = 2;
    u->dp.pfcol = d_pfcol;
    u->dp.pw = d_pw;
    u->dp.ph = d_ph;
    u->dp.prow = d_prow;
    u->dp.rows = d_rows;
    u->dp.pval = d_pval;
    u->dp.pinv = d_pval;
    u->dp.relmap = d_relmap;
    if (use_tc) {
        const int bf16 = u->op_kind == 1 || u->op_kind == 4;
        const size_t bytes = (size_t)m * u->kpad * (bf16 ? 2 : 4);
        for (int part = 0; part < (u->op_kind >= 2 ? 2 : 1); ++part) {
            char *p = nullptr;
            if ((st = ualloc(u, &p, bytes)) ||
                make_operand_map(part ? u->tmap_lo : u->tmap, p, m, u->kpad, bf16) != 0) {
                g_study_error = st ? u->err : "cuTensorMapEncodeTiled failed for the operand copy";
                spx_update_free(u);
                return st ? st : SPX_ERR_CUDA;
            }
            (part ? u->d_opc_lo : u->d_opc) = p;
        }
    }
    if (cudaMemset(u->d_err, 0, sizeof(int)) != cudaSuccess) {
        g_study_error = "cudaMemset failed";
        spx_update_free(u);
        return SPX_ERR_CUDA;
    }
    *out = u;
    return SPX_OK;
}

spx_status spx_update_stage(spx_update_plan u, const void *A, const void *W, int64_t lda, void *cuda_stream)
{
    using namespace spx;
    if (!u) return ufail(nullptr, SPX_ERR_ARG, "plan is NULL");
    if (!A || (u->ldlt && !W)) return ufail(u, SPX_ERR_ARG, "A (and W for LDL^T) must be given");
    if (lda < u->m) return ufail(u, SPX_ERR_ARG, "lda below m");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool fp64 = u->precision == SPX_FP64;
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    UCU(cudaMemcpy2DAsync(u->d_A, u->m * esz, A, lda * esz, u->m * esz, u->k, cudaMemcpyDeviceToDevice, s));
    if (u->ldlt)
        UCU(cudaMemcpy2DAsync(u->d_W, u->m * esz, W, lda * esz, u->m * esz, u->k, cudaMemcpyDeviceToDevice, s));
    if (u->use_tc) {
        launch_stage_operand<float>(u->m, (int)u->k, (const float *)u->d_A, (const float *)u->d_W, u->m, u->d_opc,
                                    u->d_opc_lo, u->kpad, u->op_kind, s);
        UCU(cudaGetLastError());
    }
    UCU(cudaStreamSynchronize(s));
    u->staged = true;
    return SPX_OK;
}

spx_status spx_update_run(spx_update_plan u, void *C, int wait, void *cuda_stream)
{
    using namespace spx;
    if (!u) return ufail(nullptr, SPX_ERR_ARG, "plan is NULL");
    if (!u->staged) return ufail(u, SPX_ERR_STATE, "spx_update_run before spx_update_stage");
    if (!C) return ufail(u, SPX_ERR_ARG, "C is NULL");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (u->use_tc) {
        launch_update_tc(u->tmap, u->tmap_lo, u->op_kind, u->dp, u->d_task, u->d_tct, u->ntct, (float *)C, u->lower,
                         u->d_err, s);
    } else if (u->precision == SPX_FP64) {
        const double *A = (const double *)u->d_A, *B = u->ldlt ? (const double *)u->d_W : A;
        launch_update<double>(u->dp, u->d_task, u->d_tiles, u->ntiles, A, B, (double *)C, u->lower, 0, s, 0);
        launch_update<double>(u->dp, u->d_task, u->d_tiles + u->ntiles, u->nnarrow, A, B, (double *)C, u->lower, 0,
                              s, 1);
    } else {
        const float *A = (const float *)u->d_A, *B = u->ldlt ? (const float *)u->d_W : A;
        launch_update<float>(u->dp, u->d_task, u->d_tiles, u->ntiles, A, B, (float *)C, u->lower, 0, s, 0);
        launch_update<float>(u->dp, u->d_task, u->d_tiles + u->ntiles, u->nnarrow, A, B, (float *)C, u->lower, 0,
                             s, 1);
    }
    UCU(cudaGetLastError());
    if (!wait) return SPX_OK;
    int e = 0;
    UCU(cudaMemcpyAsync(&e, u->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    UCU(cudaStreamSynchronize(s));
    if (e) {
        UCU(cudaMemset(u->d_err, 0, sizeof(int)));
        return ufail(u, SPX_ERR_TIMEOUT, "a tensor-core update tile gave up waiting on its pipeline");
    }
    return SPX_OK;
}

spx_status spx_update_get_info(spx_update_plan u, int32_t *engine, int64_t *tiles)
{
    using namespace spx;
    if (!u) return ufail(nullptr, SPX_ERR_ARG, "plan is NULL");
    if (engine) *engine = u->use_tc ? 2 : 1;
    if (tiles) *tiles = u->use_tc ? u->ntct : (int64_t)u->ntiles + u->nnarrow;
    return SPX_OK;
}

const char *spx_update_last_error(spx_update_plan u) { return u ? u->err.c_str() : spx::g_study_error.c_str(); }

void spx_update_free(spx_update_plan u)
{
    if (!u) return;
    for (void *p : u->allocs) cudaFree(p);
    delete u;
}

}  // extern "C"
