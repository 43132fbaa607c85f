// batch_api.cu -- C ABI of the batched static-pivot LU (include/spx.h,
// spx_batch_*): pattern classes, upload of their structure, the persistent
// launch captured in a CUDA graph, per-system results and the autotuner.
#include "../../include/spx.h"
#include "batch_kernel.cuh"
#include "spx_plan.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

using spx::BClass;
using spx::BSys;
using spx::BTask;

namespace {

// Flattened structure of every class (host copies; device copies below).
struct Flat {
    std::vector<int32_t> pfcol, pw, ph, prow, rows, task_ptr, relmap, csr_ptr, csr_col, csr_src, perm,
        iperm, level_ptr, level_panels;
    std::vector<int64_t> pval, amap;
    std::vector<BTask> tasks;
};

struct ClassOffsets {
    size_t pfcol, prow_, rows, task_ptr, tasks, relmap, amap, csr_ptr, csr_col, perm, level_ptr,
        level_panels;
};

}  // namespace

struct spx_batch_s {
    std::string err;
    int32_t nsys = 0;
    std::vector<spx::Plan> plans;            // one per class
    std::vector<int32_t> sys_cls;
    std::vector<BSys> sys;
    std::vector<int32_t> order;
    std::vector<ClassOffsets> coff;
    Flat flat;
    double tau_opt = -1.0;
    spx_batch_info info{};
    int64_t nnz_total = 0, n_total = 0, n_max = 0, felems = 0;

    // device
    bool uploaded = false;
    int device = -1;
    int num_sms = 0;
    cudaStream_t hs = nullptr;
    cudaEvent_t ev_fence = nullptr, ev0 = nullptr, ev1 = nullptr;
    std::vector<void *> allocs;
    BClass *d_cls = nullptr;
    BSys *d_sys = nullptr;
    int32_t *d_order = nullptr;
    int32_t *d_i32[14] = {};
    int64_t *d_pval = nullptr, *d_amap = nullptr;
    BTask *d_tasks = nullptr;
    unsigned *d_queue = nullptr;             // [0] queue, [1..2] summary
    int32_t *d_iters = nullptr, *d_conv = nullptr, *d_nrepl = nullptr;
    double *d_berr = nullptr;
    int64_t *d_badcol = nullptr;
    void *d_L = nullptr, *d_U = nullptr;
    int factor_elem = 0;                     // bytes per factor element allocated
    double *d_vals = nullptr, *d_B = nullptr, *d_X = nullptr;   // staging for host buffers
    bool ran = false;

    // launch configuration
    int ctas_per_sm = 0;                     // 0: the occupancy maximum
    int leaf_width = 8;
    int rows_per_thread = 2;

    // captured launch
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> exec_key;
};

namespace {

std::string g_batch_create_error;

spx_status bfail(spx_batch b, spx_status st, const std::string &msg)
{
    if (b) b->err = msg;
    else g_batch_create_error = msg;
    return st;
}

#define BCU(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return bfail(b, SPX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
spx_status balloc(spx_batch b, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return bfail(b, SPX_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    b->allocs.push_back(*p);
    return SPX_OK;
}

template <typename T>
spx_status bupload(spx_batch b, T **p, const std::vector<T> &v)
{
    spx_status st = balloc(b, p, v.size());
    if (st != SPX_OK) return st;
    if (!v.empty()) BCU(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SPX_OK;
}

void bfree_one(spx_batch b, void *p)
{
    if (!p) return;
    cudaFree(p);
    auto it = std::find(b->allocs.begin(), b->allocs.end(), p);
    if (it != b->allocs.end()) b->allocs.erase(it);
}

uint64_t fnv(uint64_t h, const void *data, size_t bytes)
{
    const unsigned char *c = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < bytes; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

template <typename T>
void append(std::vector<T> &dst, const std::vector<T> &src)
{
    dst.insert(dst.end(), src.begin(), src.end());
}

// Flatten one class's plan into b->flat (class-local indices).
void flatten(spx_batch b, const spx::Plan &P)
{
    Flat &F = b->flat;
    ClassOffsets o{};
    o.pfcol = F.pfcol.size();
    for (int32_t p = 0; p < P.npanels; ++p) {
        F.pfcol.push_back((int32_t)P.pfcol[p]);
        F.pw.push_back(P.pw[p]);
        F.ph.push_back(P.ph[p]);
    }
    o.prow_ = F.prow.size();
    for (int32_t p = 0; p <= P.npanels; ++p) F.prow.push_back((int32_t)P.prow[p]);
    // pval shares the panel numbering, with npanels + 1 entries like prow
    for (int32_t p = 0; p <= P.npanels; ++p) F.pval.push_back(P.pval[p]);
    o.rows = F.rows.size();
    append(F.rows, P.rows);
    // tasks grouped by source panel
    std::vector<int32_t> idx(P.tasks.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int32_t)i;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int32_t x, int32_t y) { return P.tasks[x].src < P.tasks[y].src; });
    o.task_ptr = F.task_ptr.size();
    o.tasks = F.tasks.size();
    std::vector<int32_t> cnt(P.npanels + 1, 0);
    for (const auto &t : P.tasks) cnt[t.src + 1]++;
    for (int32_t p = 0; p < P.npanels; ++p) cnt[p + 1] += cnt[p];
    append(F.task_ptr, cnt);
    for (int32_t i : idx) {
        const spx::Task &t = P.tasks[i];
        F.tasks.push_back(BTask{t.tgt, t.r0, t.r1, (int32_t)t.relmap_off});
    }
    o.relmap = F.relmap.size();
    append(F.relmap, P.relmap);
    o.amap = F.amap.size();
    append(F.amap, P.amap);
    o.csr_ptr = F.csr_ptr.size();
    for (int64_t v : P.csr_ptr) F.csr_ptr.push_back((int32_t)v);
    o.csr_col = F.csr_col.size();
    append(F.csr_col, P.csr_col);
    for (int64_t v : P.csr_src) F.csr_src.push_back((int32_t)v);
    o.perm = F.perm.size();
    for (int64_t v : P.perm) F.perm.push_back((int32_t)v);
    for (int64_t v : P.iperm) F.iperm.push_back((int32_t)v);
    o.level_ptr = F.level_ptr.size();
    append(F.level_ptr, P.level_ptr);
    o.level_panels = F.level_panels.size();
    append(F.level_panels, P.level_panels);
    b->coff.push_back(o);
}

enum { I_PFCOL, I_PW, I_PH, I_PROW, I_ROWS, I_TASKPTR, I_RELMAP, I_CSRPTR, I_CSRCOL, I_CSRSRC, I_PERM,
       I_IPERM, I_LVLPTR, I_LVLPAN };

spx_status upload_all(spx_batch b)
{
    if (b->uploaded) return SPX_OK;
    int dev = 0;
    BCU(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    BCU(cudaGetDeviceProperties(&prop, dev));
    if (prop.major * 10 + prop.minor != 103)
        return bfail(b, SPX_ERR_CUDA, "libspx is built for sm_103a; the current device is sm_" +
                                          std::to_string(prop.major * 10 + prop.minor));
    b->device = dev;
    b->num_sms = prop.multiProcessorCount;
    BCU(cudaStreamCreateWithFlags(&b->hs, cudaStreamNonBlocking));
    BCU(cudaEventCreateWithFlags(&b->ev_fence, cudaEventDisableTiming));
    BCU(cudaEventCreate(&b->ev0));
    BCU(cudaEventCreate(&b->ev1));
    const Flat &F = b->flat;
    const std::vector<int32_t> *i32[14] = {&F.pfcol, &F.pw, &F.ph, &F.prow, &F.rows, &F.task_ptr, &F.relmap,
                                           &F.csr_ptr, &F.csr_col, &F.csr_src, &F.perm, &F.iperm,
                                           &F.level_ptr, &F.level_panels};
    spx_status st;
    for (int q = 0; q < 14; ++q)
        if ((st = bupload(b, &b->d_i32[q], *i32[q]))) return st;
    if ((st = bupload(b, &b->d_pval, F.pval))) return st;
    if ((st = bupload(b, &b->d_amap, F.amap))) return st;
    if ((st = bupload(b, &b->d_tasks, F.tasks))) return st;
    std::vector<BClass> cls(b->plans.size());
    for (size_t c = 0; c < cls.size(); ++c) {
        const spx::Plan &P = b->plans[c];
        const ClassOffsets &o = b->coff[c];
        BClass &k = cls[c];
        k.n = (int32_t)P.n;
        k.npanels = P.npanels;
        k.nlevels = P.nlevels;
        k.nnz = (int32_t)P.nnz_a;
        k.nstored = P.pval[P.npanels];
        k.pfcol = b->d_i32[I_PFCOL] + o.pfcol;
        k.pw = b->d_i32[I_PW] + o.pfcol;
        k.ph = b->d_i32[I_PH] + o.pfcol;
        k.prow = b->d_i32[I_PROW] + o.prow_;
        k.pval = b->d_pval + o.prow_;
        k.rows = b->d_i32[I_ROWS] + o.rows;
        k.task_ptr = b->d_i32[I_TASKPTR] + o.task_ptr;
        k.tasks = b->d_tasks + o.tasks;
        k.relmap = b->d_i32[I_RELMAP] + o.relmap;
        k.amap = b->d_amap + o.amap;
        k.csr_ptr = b->d_i32[I_CSRPTR] + o.csr_ptr;
        k.csr_col = b->d_i32[I_CSRCOL] + o.csr_col;
        k.csr_src = b->d_i32[I_CSRSRC] + o.csr_col;
        k.perm = b->d_i32[I_PERM] + o.perm;
        k.iperm = b->d_i32[I_IPERM] + o.perm;
        k.level_ptr = b->d_i32[I_LVLPTR] + o.level_ptr;
        k.level_panels = b->d_i32[I_LVLPAN] + o.level_panels;
    }
    if ((st = bupload(b, &b->d_cls, cls))) return st;
    if ((st = bupload(b, &b->d_sys, b->sys))) return st;
    if ((st = bupload(b, &b->d_order, b->order))) return st;
    if ((st = balloc(b, &b->d_queue, 4))) return st;
    const size_t ns = (size_t)std::max(b->nsys, 1);
    if ((st = balloc(b, &b->d_iters, ns))) return st;
    if ((st = balloc(b, &b->d_conv, ns))) return st;
    if ((st = balloc(b, &b->d_nrepl, ns))) return st;
    if ((st = balloc(b, &b->d_berr, ns))) return st;
    if ((st = balloc(b, &b->d_badcol, ns))) return st;
    b->uploaded = true;
    return SPX_OK;
}

spx_status ensure_factor(spx_batch b, int elem)
{
    if (b->factor_elem == elem) return SPX_OK;
    bfree_one(b, b->d_L);
    bfree_one(b, b->d_U);
    b->d_L = b->d_U = nullptr;
    b->factor_elem = 0;
    spx_status st;
    unsigned char *L = nullptr, *U = nullptr;
    if ((st = balloc(b, &L, (size_t)b->felems * elem))) return st;
    if ((st = balloc(b, &U, (size_t)b->felems * elem))) return st;
    b->d_L = L;
    b->d_U = U;
    b->factor_elem = elem;
    return SPX_OK;
}

spx_status ensure_staging(spx_batch b, bool values, bool rhs)
{
    spx_status st;
    if (values && !b->d_vals && (st = balloc(b, &b->d_vals, (size_t)b->nnz_total))) return st;
    if (rhs && !b->d_B) {
        if ((st = balloc(b, &b->d_B, (size_t)b->n_total))) return st;
        if ((st = balloc(b, &b->d_X, (size_t)b->n_total))) return st;
    }
    return SPX_OK;
}

struct RunCfg {
    int ctas, leaf, rt;
};

RunCfg current_cfg(spx_batch b, int elem)
{
    RunCfg c{b->ctas_per_sm, b->leaf_width, b->rows_per_thread};
    const int mx = spx::batch_max_ctas_per_sm(elem, (int)b->n_max, c.rt);
    if (c.ctas <= 0 || c.ctas > mx) c.ctas = mx;
    return c;
}

// Enqueue (capturing once per distinct argument set) the persistent launch.
spx_status launch(spx_batch b, const double *vals, const double *B, double *X, int elem,
                  const spx_refine *r, const RunCfg &cfg)
{
    if (cfg.ctas <= 0) return bfail(b, SPX_ERR_CUDA, "the batch kernel does not fit on an SM");
    spx::BatchArgs a;
    std::memset(&a, 0, sizeof(a));   // the struct is also the graph's cache key
    a.cls = b->d_cls;
    a.sys = b->d_sys;
    a.order = b->d_order;
    a.nsys = b->nsys;
    a.leaf_width = std::min(cfg.leaf, spx::kBatchLeafMax);
    const bool refine = r && r->mode != 0;
    a.max_iter = refine ? std::max(r->max_iter, 0) : 0;
    a.tol = refine ? r->tol : 0.0;
    a.do_solve = B != nullptr;
    a.tau_opt = b->tau_opt;
    a.queue = b->d_queue;
    a.summary = b->d_queue + 1;
    a.vals = vals;
    a.B = B;
    a.X = X;
    a.L = b->d_L;
    a.U = b->d_U;
    a.iters = b->d_iters;
    a.converged = b->d_conv;
    a.nrepl = b->d_nrepl;
    a.berr = b->d_berr;
    a.bad_col = b->d_badcol;
    std::vector<unsigned char> key(sizeof(a) + sizeof(cfg) + sizeof(elem));
    std::memcpy(key.data(), &a, sizeof(a));
    std::memcpy(key.data() + sizeof(a), &cfg, sizeof(cfg));
    std::memcpy(key.data() + sizeof(a) + sizeof(cfg), &elem, sizeof(elem));
    // sets the kernel's shared-memory attribute too (outside the capture)
    if (spx::batch_max_ctas_per_sm(elem, (int)b->n_max, cfg.rt) < cfg.ctas)
        return bfail(b, SPX_ERR_ARG, "more CTAs per SM than fit");
    if (!b->exec || key != b->exec_key) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        BCU(cudaStreamBeginCapture(b->hs, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(b->d_queue, 0, 4 * sizeof(unsigned), b->hs);
        spx::launch_batch(a, elem, cfg.rt, b->num_sms * cfg.ctas, (int)b->n_max, b->hs);
        cudaError_t le = cudaGetLastError();
        cudaError_t e = cudaStreamEndCapture(b->hs, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(b, SPX_ERR_CUDA, std::string("batch kernel launch: ") + cudaGetErrorString(le));
        }
        if (e != cudaSuccess) return bfail(b, SPX_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, SPX_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        b->exec_key = key;
    }
    BCU(cudaEventRecord(b->ev0, b->hs));
    BCU(cudaGraphLaunch(b->exec, b->hs));
    BCU(cudaEventRecord(b->ev1, b->hs));
    return SPX_OK;
}

spx_status run(spx_batch b, const double *values, const double *B, double *X, int on_device,
               spx_precision precision, const spx_refine *r, void *stream, const RunCfg *force)
{
    if (!b) return bfail(nullptr, SPX_ERR_ARG, "batch handle is NULL");
    if (!values) return bfail(b, SPX_ERR_ARG, "values is NULL");
    if (B && !X) return bfail(b, SPX_ERR_ARG, "X is NULL");
    if (precision != SPX_FP64 && precision != SPX_FP32)
        return bfail(b, SPX_ERR_ARG, "the batched LU runs in SPX_FP64 or SPX_FP32");
    if (r && r->mode != 0 && !(r->tol > 0.0)) return bfail(b, SPX_ERR_ARG, "refinement needs tol > 0");
    const int elem = precision == SPX_FP64 ? 8 : 4;
    spx_status st;
    if ((st = upload_all(b))) return st;
    int cur = 0;
    BCU(cudaGetDevice(&cur));
    if (cur != b->device) return bfail(b, SPX_ERR_ARG, "current device differs from the handle's device");
    if ((size_t)b->n_max * elem > 160u * 1024u)
        return bfail(b, SPX_ERR_ARG, "a system is too large for the batched kernel (n * element size > 160 KiB)");
    if ((st = ensure_factor(b, elem))) return st;
    if (b->nsys == 0) return SPX_OK;
    cudaEventRecord(b->ev_fence, (cudaStream_t)stream);
    cudaStreamWaitEvent(b->hs, b->ev_fence, 0);
    const double *dv = values, *dB = B;
    double *dX = X;
    if (!on_device) {
        if ((st = ensure_staging(b, true, B != nullptr))) return st;
        BCU(cudaMemcpyAsync(b->d_vals, values, sizeof(double) * b->nnz_total, cudaMemcpyHostToDevice, b->hs));
        dv = b->d_vals;
        if (B) {
            BCU(cudaMemcpyAsync(b->d_B, B, sizeof(double) * b->n_total, cudaMemcpyHostToDevice, b->hs));
            dB = b->d_B;
            dX = b->d_X;
        }
    }
    const RunCfg cfg = force ? *force : current_cfg(b, elem);
    if ((st = launch(b, dv, dB, dX, elem, r, cfg))) return st;
    if (!on_device && B)
        BCU(cudaMemcpyAsync(X, b->d_X, sizeof(double) * b->n_total, cudaMemcpyDeviceToHost, b->hs));
    unsigned summary[3] = {0, 0, 0};
    BCU(cudaMemcpyAsync(summary, b->d_queue, sizeof(summary), cudaMemcpyDeviceToHost, b->hs));
    BCU(cudaStreamSynchronize(b->hs));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    b->info.run_ms = ms;
    b->info.precision = precision;
    b->info.ctas_per_sm = cfg.ctas;
    b->info.leaf_width = cfg.leaf;
    b->info.rows_per_thread = cfg.rt;
    b->info.not_converged = (int32_t)summary[1];
    b->ran = true;
    if (summary[2]) return bfail(b, SPX_ERR_ZERO_PIVOT, std::to_string(summary[2]) + " system(s) met a zero pivot");
    if (B && r && r->mode != 0 && summary[1])
        return bfail(b, SPX_ERR_NOT_CONVERGED, std::to_string(summary[1]) + " system(s) missed the target backward error");
    return SPX_OK;
}

}  // namespace

extern "C" {

spx_status spx_batch_analyze(int32_t nsys, const int64_t *n, const int64_t *colptr,
                             const int32_t *rowind, const int32_t *grid, const spx_options *opt,
                             spx_batch *out)
{
    if (!out) return bfail(nullptr, SPX_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nsys < 0) return bfail(nullptr, SPX_ERR_ARG, "nsys < 0");
    if (nsys > 0 && (!n || !colptr || !rowind)) return bfail(nullptr, SPX_ERR_ARG, "NULL argument");
    spx_options o;
    spx_default_options(&o);
    if (opt) o = *opt;
    if (o.perm || o.ordering == SPX_ORDER_GIVEN) return bfail(nullptr, SPX_ERR_ARG, "the batch takes no given permutation");
    if (o.lower_only) return bfail(nullptr, SPX_ERR_ARG, "the batch takes full patterns only");
    if (o.max_width <= 0 || o.max_width > spx::kBatchMaxWidth) o.max_width = spx::kBatchMaxWidth;
    auto t0 = std::chrono::steady_clock::now();
    spx_batch b = new (std::nothrow) spx_batch_s();
    if (!b) return bfail(nullptr, SPX_ERR_ALLOC, "host allocation failed");
    b->nsys = nsys;
    b->tau_opt = o.pivot_tau;
    std::unordered_map<uint64_t, std::vector<int32_t>> seen;   // hash -> classes
    std::vector<int64_t> rep_cp, rep_ri;                        // representative system per class
    std::vector<int32_t> rep_sys;
    std::vector<int64_t> cp_off(nsys + 1, 0), ri_off(nsys + 1, 0);
    for (int32_t s = 0; s < nsys; ++s) {
        if (n[s] < 0 || n[s] > INT32_MAX / 2) {
            spx_batch_free(b);
            return bfail(nullptr, SPX_ERR_ARG, "system " + std::to_string(s) + ": bad n");
        }
        cp_off[s + 1] = cp_off[s] + n[s] + 1;
        const int64_t *cp = colptr + cp_off[s];
        if (cp[0] != 0 || cp[n[s]] < 0) {
            spx_batch_free(b);
            return bfail(nullptr, SPX_ERR_ARG, "system " + std::to_string(s) + ": colptr must start at 0");
        }
        ri_off[s + 1] = ri_off[s] + cp[n[s]];
    }
    std::string emsg;
    for (int32_t s = 0; s < nsys && emsg.empty(); ++s) {
        const int64_t ns = n[s];
        const int64_t *cp = colptr + cp_off[s];
        const int32_t *ri = rowind + ri_off[s];
        const int64_t nnz = cp[ns];
        int32_t g3[3] = {0, 0, 0};
        if (grid) std::memcpy(g3, grid + 3 * (size_t)s, sizeof(g3));
        uint64_t hsh = 1469598103934665603ull;
        hsh = fnv(hsh, &ns, sizeof(ns));
        hsh = fnv(hsh, g3, sizeof(g3));
        hsh = fnv(hsh, cp, sizeof(int64_t) * (size_t)(ns + 1));
        hsh = fnv(hsh, ri, sizeof(int32_t) * (size_t)nnz);
        int32_t cls = -1;
        auto it = seen.find(hsh);
        if (it != seen.end()) {
            for (int32_t c : it->second) {
                const int32_t r = rep_sys[c];
                int32_t rg[3] = {0, 0, 0};
                if (grid) std::memcpy(rg, grid + 3 * (size_t)r, sizeof(rg));
                if (n[r] == ns && std::memcmp(rg, g3, sizeof(g3)) == 0 &&
                    std::memcmp(colptr + cp_off[r], cp, sizeof(int64_t) * (size_t)(ns + 1)) == 0 &&
                    std::memcmp(rowind + ri_off[r], ri, sizeof(int32_t) * (size_t)nnz) == 0) {
                    cls = c;
                    break;
                }
            }
        }
        if (cls < 0) {
            spx::AnalyzeOptions ao;
            ao.ordering = o.ordering;
            if (grid) std::memcpy(ao.grid, g3, sizeof(g3));
            else std::memcpy(ao.grid, o.grid, sizeof(ao.grid));
            ao.dof = o.dof;
            ao.max_width = o.max_width;
            ao.amalg_ratio = o.amalg_ratio;
            ao.lower_only = 0;
            b->plans.emplace_back();
            const std::string e = spx::analyze(ns, cp, ri, SPX_LU, ao, b->plans.back());
            if (!e.empty()) {
                emsg = "system " + std::to_string(s) + ": " + e;
                break;
            }
            cls = (int32_t)b->plans.size() - 1;
            rep_sys.push_back(s);
            seen[hsh].push_back(cls);
        }
        b->sys_cls.push_back(cls);
    }
    if (!emsg.empty()) {
        spx_batch_free(b);
        return bfail(nullptr, SPX_ERR_ARG, emsg);
    }
    for (const spx::Plan &P : b->plans)
        for (int32_t p = 0; p < P.npanels; ++p)
            if (P.pw[p] > spx::kBatchMaxWidth) {
                spx_batch_free(b);
                return bfail(nullptr, SPX_ERR_ARG, "a panel is wider than the batched kernel takes");
            }
    for (const spx::Plan &P : b->plans) flatten(b, P);
    int64_t foff = 0, xoff = 0;
    double flops = 0.0;
    int64_t nnzl = 0;
    std::vector<double> sys_flops(nsys);
    for (int32_t s = 0; s < nsys; ++s) {
        const spx::Plan &P = b->plans[b->sys_cls[s]];
        BSys S{};
        S.cls = b->sys_cls[s];
        S.n = (int32_t)n[s];
        S.voff = ri_off[s];
        S.foff = foff;
        S.xoff = xoff;
        b->sys.push_back(S);
        foff += (P.pval[P.npanels] + 3) & ~int64_t(3);   // 16-byte aligned starts
        xoff += n[s];
        flops += P.flops_exact;
        nnzl += P.nnz_l;
        sys_flops[s] = P.flops_exact;
        b->n_max = std::max<int64_t>(b->n_max, n[s]);
    }
    b->order.resize(nsys);
    for (int32_t s = 0; s < nsys; ++s) b->order[s] = s;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int32_t x, int32_t y) { return sys_flops[x] > sys_flops[y]; });
    b->felems = foff;
    b->n_total = xoff;
    b->nnz_total = ri_off[nsys];
    spx_batch_info &I = b->info;
    I.nsys = nsys;
    I.nclasses = (int32_t)b->plans.size();
    I.n_total = xoff;
    I.n_max = b->n_max;
    I.nnz_total = b->nnz_total;
    I.nnz_l_total = nnzl;
    I.factor_elems = 2 * foff;
    I.flops = flops;
    I.precision = -1;
    I.leaf_width = b->leaf_width;
    I.rows_per_thread = b->rows_per_thread;
    I.analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = b;
    return SPX_OK;
}

spx_status spx_batch_run(spx_batch b, const double *values, const double *B, double *X, int on_device,
                         spx_precision precision, const spx_refine *refine, void *cuda_stream)
{
    return run(b, values, B, X, on_device, precision, refine, cuda_stream, nullptr);
}

spx_status spx_batch_tune(spx_batch b, const double *values, const double *B, double *X, int on_device,
                          spx_precision precision, const spx_refine *refine, void *cuda_stream)
{
    if (!b) return bfail(nullptr, SPX_ERR_ARG, "batch handle is NULL");
    const int elem = precision == SPX_FP64 ? 8 : 4;
    spx_status st;
    if ((st = upload_all(b))) return st;
    // time one configuration: one untimed run, then the best of three
    auto time_cfg = [&](const RunCfg &c, double *ms) -> spx_status {
        spx_status s2 = run(b, values, B, X, on_device, precision, refine, cuda_stream, &c);
        if (s2 != SPX_OK && s2 != SPX_ERR_NOT_CONVERGED) return s2;
        double best = 1e30;
        for (int rep = 0; rep < 3; ++rep) {
            s2 = run(b, values, B, X, on_device, precision, refine, cuda_stream, &c);
            if (s2 != SPX_OK && s2 != SPX_ERR_NOT_CONVERGED) return s2;
            best = std::min(best, b->info.run_ms);
        }
        *ms = best;
        return SPX_OK;
    };
    RunCfg best{0, 8, 2};
    best.ctas = spx::batch_max_ctas_per_sm(elem, (int)b->n_max, best.rt);
    double best_ms = 1e30;
    // 1. leaf-versus-top schedule
    for (int leaf : {0, 4, 8, 16}) {
        RunCfg c = best;
        c.leaf = leaf;
        double ms;
        if ((st = time_cfg(c, &ms))) return st;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    // 2. update tile: rows per thread
    for (int rt : {1, 2, 4}) {
        if (rt == best.rt) continue;
        RunCfg c = best;
        c.rt = rt;
        c.ctas = std::min(c.ctas, spx::batch_max_ctas_per_sm(elem, (int)b->n_max, rt));
        double ms;
        if ((st = time_cfg(c, &ms))) return st;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    // 3. occupancy
    const int mx = spx::batch_max_ctas_per_sm(elem, (int)b->n_max, best.rt);
    for (int ctas = 1; ctas <= mx; ++ctas) {
        if (ctas == best.ctas) continue;
        RunCfg c = best;
        c.ctas = ctas;
        double ms;
        if ((st = time_cfg(c, &ms))) return st;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    b->ctas_per_sm = best.ctas;
    b->leaf_width = best.leaf;
    b->rows_per_thread = best.rt;
    // leave X holding a result of the chosen configuration
    st = run(b, values, B, X, on_device, precision, refine, cuda_stream, nullptr);
    b->info.tuned_ms = best_ms;
    return st;
}

spx_status spx_batch_set_config(spx_batch b, int32_t ctas_per_sm, int32_t leaf_width, int32_t rows_per_thread)
{
    if (!b) return bfail(nullptr, SPX_ERR_ARG, "batch handle is NULL");
    if (ctas_per_sm < 0 || leaf_width < 0 || leaf_width > spx::kBatchLeafMax)
        return bfail(b, SPX_ERR_ARG, "bad configuration");
    if (rows_per_thread != 0 && rows_per_thread != 1 && rows_per_thread != 2 && rows_per_thread != 4)
        return bfail(b, SPX_ERR_ARG, "rows_per_thread must be 1, 2 or 4");
    if (ctas_per_sm) b->ctas_per_sm = ctas_per_sm;
    b->leaf_width = leaf_width;
    if (rows_per_thread) b->rows_per_thread = rows_per_thread;
    return SPX_OK;
}

spx_status spx_batch_get_info(spx_batch b, spx_batch_info *info)
{
    if (!b || !info) return bfail(b, SPX_ERR_ARG, "NULL argument");
    if (b->ran && b->nsys > 0) {
        std::vector<int32_t> it(b->nsys), rp(b->nsys);
        std::vector<double> be(b->nsys);
        BCU(cudaMemcpy(it.data(), b->d_iters, sizeof(int32_t) * b->nsys, cudaMemcpyDeviceToHost));
        BCU(cudaMemcpy(rp.data(), b->d_nrepl, sizeof(int32_t) * b->nsys, cudaMemcpyDeviceToHost));
        BCU(cudaMemcpy(be.data(), b->d_berr, sizeof(double) * b->nsys, cudaMemcpyDeviceToHost));
        b->info.max_iters = *std::max_element(it.begin(), it.end());
        b->info.max_pivot_repl = *std::max_element(rp.begin(), rp.end());
        double m = 0.0;
        for (double v : be) m = (v != v || v > m) ? (v != v ? INFINITY : v) : m;
        b->info.max_backward_error = m;
    }
    *info = b->info;
    return SPX_OK;
}

spx_status spx_batch_system_info(spx_batch b, int32_t *iters, double *berr, int32_t *converged,
                                 int32_t *npivot_repl, int64_t *bad_col)
{
    if (!b) return bfail(nullptr, SPX_ERR_ARG, "batch handle is NULL");
    if (!b->ran) return bfail(b, SPX_ERR_STATE, "no run yet");
    const size_t ns = (size_t)b->nsys;
    if (ns == 0) return SPX_OK;
    if (iters) BCU(cudaMemcpy(iters, b->d_iters, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost));
    if (berr) BCU(cudaMemcpy(berr, b->d_berr, sizeof(double) * ns, cudaMemcpyDeviceToHost));
    if (converged) BCU(cudaMemcpy(converged, b->d_conv, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost));
    if (npivot_repl) BCU(cudaMemcpy(npivot_repl, b->d_nrepl, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost));
    if (bad_col) BCU(cudaMemcpy(bad_col, b->d_badcol, sizeof(int64_t) * ns, cudaMemcpyDeviceToHost));
    return SPX_OK;
}

spx_status spx_batch_get_perm(spx_batch b, int32_t s, int64_t *perm)
{
    if (!b || !perm) return bfail(b, SPX_ERR_ARG, "NULL argument");
    if (s < 0 || s >= b->nsys) return bfail(b, SPX_ERR_ARG, "system index out of range");
    const spx::Plan &P = b->plans[b->sys_cls[s]];
    std::memcpy(perm, P.perm.data(), sizeof(int64_t) * (size_t)P.n);
    return SPX_OK;
}

spx_status spx_batch_get_factor(spx_batch b, int32_t s, const int64_t *Lp, const int32_t *Li, double *Lx,
                                double *Ut)
{
    if (!b || !Lp || !Li || !Lx || !Ut) return bfail(b, SPX_ERR_ARG, "NULL argument");
    if (s < 0 || s >= b->nsys) return bfail(b, SPX_ERR_ARG, "system index out of range");
    if (!b->ran) return bfail(b, SPX_ERR_STATE, "no factor");
    const spx::Plan &P = b->plans[b->sys_cls[s]];
    const size_t elems = (size_t)P.pval[P.npanels];
    const int64_t foff = b->sys[s].foff;
    std::vector<double> hl(elems), hu(elems);
    auto fetch = [&](const void *base, std::vector<double> &dst) -> spx_status {
        if (b->factor_elem == 8) {
            BCU(cudaMemcpy(dst.data(), static_cast<const double *>(base) + foff, elems * sizeof(double),
                           cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> tmp(elems);
            BCU(cudaMemcpy(tmp.data(), static_cast<const float *>(base) + foff, elems * sizeof(float),
                           cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < elems; ++i) dst[i] = tmp[i];
        }
        return SPX_OK;
    };
    spx_status st;
    if ((st = fetch(b->d_L, hl))) return st;
    if ((st = fetch(b->d_U, hu))) return st;
    for (int64_t j = 0; j < P.n; ++j) {
        const int32_t pj = P.col2panel[j];
        const int64_t cj = j - P.pfcol[pj];
        const int64_t hj = P.ph[pj];
        const int32_t *rb = P.rows.data() + P.prow[pj], *re = P.rows.data() + P.prow[pj + 1];
        for (int64_t q = Lp[j]; q < Lp[j + 1]; ++q) {
            const int64_t i = Li[q];
            if (i < j || i >= P.n) return bfail(b, SPX_ERR_ARG, "pattern entry above the diagonal");
            const int32_t *itr = std::lower_bound(rb, re, (int32_t)i);
            if (itr == re || *itr != i) return bfail(b, SPX_ERR_ARG, "pattern entry outside the panel structure");
            const int64_t off = P.pval[pj] + cj * hj + (itr - rb);
            if (i == j) {
                Lx[q] = 1.0;
                Ut[q] = hl[off];
            } else {
                Lx[q] = hl[off];
                Ut[q] = i < P.pfcol[pj] + P.pw[pj] ? hl[P.pval[pj] + (i - P.pfcol[pj]) * hj + cj] : hu[off];
            }
        }
    }
    return SPX_OK;
}

const char *spx_batch_last_error(spx_batch b)
{
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

void spx_batch_free(spx_batch b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (void *p : b->allocs) cudaFree(p);
    if (b->hs) cudaStreamDestroy(b->hs);
    if (b->ev_fence) cudaEventDestroy(b->ev_fence);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

}  // extern "C"
