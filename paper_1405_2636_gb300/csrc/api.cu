// api.cu -- the C ABI of libspx (include/spx.h): handle management, upload
// of the analysed structure, the level-by-level factorization captured once
// into a CUDA graph and replayed, the solve sweeps and the refinement loop.
#include "../../include/spx.h"
#include "kernels.cuh"
#include "spx_plan.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>
#include <climits>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <cstring>
#include <new>
#include <queue>
#include <string>
#include <utility>
#include <vector>

using spx::DevTask;
using spx::RowChunk;
using spx::UpdTile;

// Host threads for the copies between caller buffers and the pinned staging
// buffers: one host memcpy thread moves ~16 GB/s, eight ~80 GB/s (Grace).
// run(f) calls f(part, parts) on every worker and on the caller, and returns
// once all parts are done.
struct CopyPool {
    std::vector<std::thread> workers;
    std::mutex m;
    std::condition_variable wake, done;
    std::function<void(int, int)> job;
    int gen = 0, pending = 0, parts = 1;
    bool stop = false;
    explicit CopyPool(int nworkers)
    {
        parts = nworkers + 1;
        for (int k = 1; k <= nworkers; ++k) workers.emplace_back([this, k] { loop(k); });
    }
    void loop(int k)
    {
        int seen = 0;
        for (;;) {
            std::function<void(int, int)> f;
            {
                std::unique_lock<std::mutex> l(m);
                wake.wait(l, [&] { return stop || gen != seen; });
                if (stop) return;
                seen = gen;
                f = job;
            }
            f(k, parts);
            std::lock_guard<std::mutex> l(m);
            if (--pending == 0) done.notify_one();
        }
    }
    void run(const std::function<void(int, int)> &f)
    {
        if (workers.empty()) return f(0, 1);
        {
            std::lock_guard<std::mutex> l(m);
            job = f;
            pending = parts - 1;
            ++gen;
        }
        wake.notify_all();
        f(0, parts);
        std::unique_lock<std::mutex> l(m);
        done.wait(l, [&] { return pending == 0; });
    }
    ~CopyPool()
    {
        {
            std::lock_guard<std::mutex> l(m);
            stop = true;
        }
        wake.notify_all();
        for (auto &t : workers) t.join();
    }
};

struct spx_handle_s {
    spx::Plan plan;
    std::string err;
    spx_method method = SPX_LLT;
    double pivot_tau_opt = -1.0;

    // device state
    bool uploaded = false;
    int device = -1;
    cudaStream_t hs = nullptr;
    cudaStream_t aux[2] = {nullptr, nullptr};   // side branches of the captured factorization graph
    cudaEvent_t ev_fence = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
    cudaStream_t fstream[2] = {nullptr, nullptr};   // far update tiles of alternate levels (look-ahead)
    cudaEvent_t ev_trsm = nullptr, ev_far[2] = {nullptr, nullptr};
    cudaEvent_t ev_near[2] = {nullptr, nullptr};    // a chain link's TRSM and near tiles, done beside the next diagonal block
    std::vector<void *> allocs;

    spx::DevPlan dp{};
    int32_t *d_level_panels = nullptr;
    DevTask *d_tasks = nullptr;
    int64_t *d_amap = nullptr, *d_csr_ptr = nullptr, *d_csr_src = nullptr, *d_perm = nullptr;
    int32_t *d_csr_col = nullptr;

    std::vector<int32_t> lvl_wmax;    // widest panel per level
    // panels of a level sorted by width class (kWidthClass); class c of level l
    // is d_level_panels[cls_ptr[l * kNumClasses + c] .. cls_ptr[l * kNumClasses + c + 1])
    std::vector<int32_t> cls_ptr;
    int64_t dinv_elems = 0;           // sum over panels of w^2 rounded up to 32
    std::vector<int64_t> chunk_ptr;   // per level, into d_chunks
    RowChunk *d_chunks = nullptr;
    // Each per-level tile list holds the 64 x 64 tiles first, then the 256 x 16
    // tiles of tasks facing at most 16 rows; *_nar[l] is where the latter start.
    std::vector<int64_t> tile_ptr, tile_nar;    // per level, into d_tiles (LLT, or LU's L side)
    UpdTile *d_tiles = nullptr;
    std::vector<int64_t> tileu_ptr, tileu_nar;  // per level, LU's U^T side
    UpdTile *d_tilesu = nullptr;
    // tensor-core updates (Cholesky, TF32/BF16): tasks with a source at least
    // kTcMinWidth wide go to the tcgen05 kernel, the rest to the SIMT kernel
    std::vector<int64_t> tcsmall_ptr, tcsmall_nar; // per level, SIMT tiles of the narrow tasks
    // sweep work queues: item orders, chunk -> owning panels, per-panel wait
    // counts; d_qstate holds the per-sweep counters (zeroed each sweep)
    int32_t *d_qitems_f = nullptr, *d_qitems_b = nullptr, *d_qtptr = nullptr, *d_qtgt = nullptr;
    int32_t *d_qneed_f = nullptr, *d_qneed_b = nullptr, *d_qstate = nullptr, *d_qerr = nullptr;
    int32_t *d_qmerge = nullptr;
    int32_t q_nitems = 0, q_mat = 0, q_matb = 0, q_vec = 0;
    uint32_t spin_limit = spx::kDefaultSpinLimit;   // polls before a sweep wait gives up
    int32_t *h_noalloc_err = nullptr;   // pinned: the error word of the last completed spx_solve_noalloc
    void *h_stage[2] = {nullptr, nullptr};  // pinned staging buffers for host-buffer copies
    std::unique_ptr<CopyPool> copy_pool;    // host threads packing and unpacking them
    cudaEvent_t ev_stage[2] = {nullptr, nullptr};
    UpdTile *d_tcsmall = nullptr;
    // persistent task queue of the upper levels (Cholesky and LDL^T, panels
    // at most 64 wide): levels [q_level, nlevels) run as one launch.  Two item
    // lists: updates on the tensor cores (tc modes) or all on the CUDA cores.
    int32_t queue_panels = 0;         // option: 0 default policy, > 0 region bound, < 0 no queue
    int32_t q_level = 0;              // first level of the region the item lists were built for
    spx::FqItem *d_fq_items[2] = {nullptr, nullptr};   // [0] CUDA cores, [1] tensor cores
    int32_t fq_nitems[2] = {0, 0};
    int32_t *d_fq_need[2] = {nullptr, nullptr};
    int32_t *d_fq_pchunk = nullptr, *d_fq_state = nullptr;
    int64_t fq_nchunks = 0;
    // host copies of the launch lists (for the item lists of partitions)
    std::vector<RowChunk> hc_chunks;
    std::vector<UpdTile> hc_tiles, hc_small;
    std::vector<spx::TcTile> hc_tct;
    std::vector<int32_t> h_pchunk;
    int workers = 0;
    // subtree-to-rank partition (spx_partition): owner rank of each panel's
    // subtree, -1 for the top panels; per part (rank r at index r, the top at
    // index nranks) the packed ranges of its panel values and inverse blocks
    // and its queue item lists (built on first use, per update mode)
    int32_t part_nranks = 0;
    int part_done = 0;                 // 1: a rank's subtrees factored here, 2: the top factored here
    std::vector<int32_t> panel_owner;
    struct Part {
        int64_t nval = 0, ninv = 0;          // packed elements
        std::vector<int64_t> h_ranges;       // (storage offset, length, packed offset): values, then inverses
        int64_t *d_ranges = nullptr;         // device copy
        int32_t nr = 0;
        spx::FqItem *d_items[2] = {nullptr, nullptr};
        int32_t *d_need[2] = {nullptr, nullptr};
        int32_t nitems[2] = {-1, -1};
    };
    std::vector<Part> parts;
    // deterministic updates: each level's tiles sorted by round (the rank of
    // their task among the level's tasks with the same target); rounds are
    // launched one after the other, so that every target entry receives at
    // most one reduction per launch, in task order.  det_ptr[s][det_base[l] + r]
    // is where round r of segment s of level l starts (R_l + 1 entries).
    bool deterministic = false;
    std::vector<int32_t> det_rounds;   // per level
    std::vector<int64_t> det_base;     // per level, into det_ptr[*]
    std::vector<int64_t> det_ptr[7];   // segments: SIMT wide, SIMT narrow, U^T wide, U^T narrow, tc, tc-small wide, tc-small narrow
    // look-ahead: outside the deterministic mode each level's tile segments
    // list the tiles into the next level's panels ("near") first;
    // near_end[s][l] is where segment s's "far" tiles of level l begin
    std::vector<int64_t> near_end[7];
    std::vector<int64_t> tctile_ptr;  // per level, 128 x 128 tensor-core tiles
    spx::TcTile *d_tctiles = nullptr;
    // chain links (Cholesky, tensor-core modes): level l holds one 64-wide
    // panel p and level l + 1 one 64-wide panel q whose columns are p's first
    // 64 off-diagonal rows.  link_task[l] is the task p -> q (-1: not a link);
    // d_link_tct[link_ptr[l] ..) the level's near tensor-core tiles with that
    // task's tiles starting below q's diagonal block, which the look-ahead
    // step updates instead.
    std::vector<int32_t> link_task;
    std::vector<int64_t> link_ptr;
    spx::TcTile *d_link_tct = nullptr;
    int kpad = 0;                     // operand-copy row length
    int64_t op_rows = 0;              // operand-copy rows (sum of panel heights)
    void *d_opc = nullptr;            // operand copy (TF32 floats, BF16, or the hi half of split TF32)
    void *d_opc_lo = nullptr;         // lo half of split TF32
    int opc_kind = -1;                // 0 tf32, 1 bf16, 2 split tf32
    alignas(64) unsigned char tmap[128];     // CUtensorMap over d_opc
    alignas(64) unsigned char tmap_lo[128];  // CUtensorMap over d_opc_lo
    int *d_tcerr = nullptr;
    double upd_flops_tc = 0, upd_elems_tc = 0, upd_op_elems_tc = 0;   // share of the tensor-core tasks

    // numeric state
    int precision = -1;
    bool factored = false;
    void *d_L = nullptr, *d_U = nullptr, *d_Dinv = nullptr;
    void *d_W = nullptr;                     // LDL^T: the D L^T rows (the update's B operand)
    unsigned long long *d_nneg = nullptr;    // LDL^T: negative pivots
    int factor_prec_alloc = -1;
    double *d_vals = nullptr;
    double *d_tau = nullptr;                 // [0] pivot threshold used by the diagonal kernels
    unsigned long long *d_anorm = nullptr;   // bits of ||A||_inf
    int64_t *d_err = nullptr;
    unsigned long long *d_nrepl = nullptr;
    double anorm = 0.0;
    cudaGraphExec_t fgraph = nullptr;
    int fgraph_prec = -1;

    // FGMRES workspace: Krylov basis V (restart+1 blocks), preconditioned
    // directions Z (restart blocks), w, small coefficient arrays
    int gm_m = 0, gm_nrhs = 0;
    double *d_gV = nullptr, *d_gZ = nullptr, *d_gw = nullptr, *d_gcoef = nullptr;
    std::vector<double> last_xinf, last_binf;   // per-column norms of the last residual

    // solve workspace
    int ws_nrhs = 0;
    double *d_B = nullptr, *d_X = nullptr, *d_R = nullptr, *d_D = nullptr;
    double *d_Y = nullptr, *d_Z = nullptr, *d_T = nullptr, *d_Xs = nullptr;   // sweep vectors (factor type)
    unsigned long long *d_norms = nullptr;
    cudaGraphExec_t sgraph = nullptr;
    int sgraph_nrhs = -1, sgraph_prec = -1;

    // selected inverse and adjoints: Z on the panel structure (FP64), the
    // scaled panels L_RJ L_JJ^{-1}, tasks by source panel, and the position
    // in Z of every input entry
    bool zready = false;
    double *d_Zsel = nullptr, *d_Lh = nullptr;
    int32_t *d_row_task = nullptr;
    int64_t *d_zmap = nullptr;
    double *d_scalar = nullptr;
    double *d_gtmp = nullptr, *d_lam = nullptr, *d_xg = nullptr;
    int64_t gtmp_len = 0;

    // profiling and launch accounting
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    spx_kernel_stats kstats{};
    int64_t class_launches[SPX_K_CLASSES] = {};   // kernels per class of the last enqueued factorization
    int64_t cnt = 0;                  // kernels enqueued by the current call
    int64_t sweep_launches = 0;       // kernels of one solve sweep

    spx_info info{};
};

namespace {

constexpr int kTcMinWidth = 32;   // narrowest source panel sent to the tensor cores
// Width classes of the diagonal-block kernel: shared memory and block size
// follow the widest panel of the class, not of the level.
constexpr int kNumClasses = 6;
constexpr int kClassWidth[kNumClasses] = {16, 32, 64, 96, 128, 160};
constexpr int kClassThreads[kNumClasses] = {64, 128, 256, 256, 256, 256};
inline int width_class(int w)
{
    for (int c = 0; c < kNumClasses; ++c)
        if (w <= kClassWidth[c]) return c;
    return kNumClasses - 1;
}

std::string g_create_error;

spx_status fail(spx_handle h, spx_status st, const std::string &msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return st;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(h, SPX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
spx_status dalloc(spx_handle h, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(h, SPX_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->allocs.push_back(*p);
    return SPX_OK;
}

template <typename T>
spx_status upload(spx_handle h, T **p, const std::vector<T> &v)
{
    spx_status st = dalloc(h, p, v.size());
    if (st != SPX_OK) return st;
    if (!v.empty()) CU(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SPX_OK;
}

void dfree(spx_handle h, void *p)
{
    if (!p) return;
    cudaFree(p);
    auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
    if (it != h->allocs.end()) h->allocs.erase(it);
}

// --- small device helpers ---------------------------------------------------
__global__ void init_scalars_kernel(int64_t *err, unsigned long long *nrepl,
                                    unsigned long long *anorm)
{
    *err = LLONG_MAX;
    *nrepl = 0ull;
    *anorm = 0ull;
}

// tau = fixed (>= 0) or scale * ||A||_inf
__global__ void set_tau_kernel(const unsigned long long *anorm_bits, double fixed, double scale,
                               double *tau)
{
    double a = __longlong_as_double((long long)*anorm_bits);
    *tau = fixed >= 0.0 ? fixed : scale * a;
}

// Algorithmic work of every panel and update task, as the kernel classes
// count it: fn(class, level, flops, elements of the factor's type, elements
// of the tensor-core operand copy, FP32 target elements) -- diagonal block
// and TRSM per panel (Sec. III steps 1, 2), one update per task (step 3).
template <typename F>
void visit_work(const spx::Plan &P, bool tcm, F fn)
{
    const bool lu = P.method == SPX_LU;
    const double nfac = lu ? 2.0 : 1.0;
    for (int32_t q = 0; q < P.npanels; ++q) {
        const double w = P.pw[q], off = (double)P.ph[q] - P.pw[q];
        double df = 0.0;
        for (int32_t j = 0; j < P.pw[q]; ++j) {
            const double c = w - j;
            df += lu ? 2.0 * (c - 1.0) * (c - 1.0) + (c - 1.0) : c * c;
        }
        fn(SPX_K_DIAG, P.plevel[q], df, 2.0 * w * w, 0.0, 0.0);
        fn(SPX_K_TRSM, P.plevel[q], nfac * off * w * w, nfac * (2.0 * off * w + w * w), 0.0, 0.0);
    }
    for (const spx::Task &tk : P.tasks) {
        const double M = (double)P.ph[tk.src] - tk.r0, N = (double)tk.r1 - tk.r0, K = P.pw[tk.src];
        double flops, el_op, el_acc;
        if (!lu) {
            flops = 2.0 * (M - N) * N * K + N * (N + 1.0) * K;
            el_op = (M + N) * K;
            el_acc = 2.0 * ((M - N) * N + N * (N + 1.0) / 2.0);
        } else {
            flops = 2.0 * M * N * K + 2.0 * (M - N) * N * K;
            el_op = (M + N) * K + M * K;
            el_acc = 2.0 * (M * N + (M - N) * N);
        }
        const int lvl = P.plevel[tk.src];
        if (tcm && P.pw[tk.src] >= kTcMinWidth) fn(SPX_K_UPDATE_TC, lvl, flops, 0.0, el_op, el_acc);
        else fn(SPX_K_UPDATE, lvl, flops, el_op + el_acc, 0.0, 0.0);
    }
}

// First level of the persistent queue region: the top levels whose panel
// count is at most qmax and whose panels are at most 64 wide (the queue's
// diagonal-block bodies); LU keeps the level-by-level walk.  nlevels: none.
int queue_start_level(const spx::Plan &P, int qmax)
{
    if (P.method == SPX_LU || qmax < 0) return P.nlevels;
    int l = P.nlevels;
    while (l > 0) {
        const int lv = l - 1;
        if (P.level_ptr[lv + 1] - P.level_ptr[lv] > qmax) break;
        bool narrow = true;
        for (int32_t q = P.level_ptr[lv]; q < P.level_ptr[lv + 1]; ++q) narrow = narrow && P.pw[P.level_panels[q]] <= 64;
        if (!narrow) break;
        l = lv;
    }
    return l;
}

// The queue region a factorization in `prec` uses.  qopt > 0: the top
// levels with at most qopt panels; qopt < 0: none; qopt = 0 (default): the
// whole tree (as far as panels are at most 64 wide) for an FP64 factor,
// where the queue measured faster than the level walk (its update tiles are
// long FP64 products), and none for the single-precision factors, whose
// short tensor-core and FP32 tiles ran faster as per-level launches.
int queue_policy_level(const spx::Plan &P, int qopt, int prec)
{
    if (qopt < 0 || (qopt == 0 && prec != SPX_FP64)) return P.nlevels;
    return queue_start_level(P, qopt == 0 ? INT32_MAX : qopt);
}

int32_t queue_level(spx_handle h, int prec)
{
    const spx::Plan &P = h->plan;
    if (h->q_level >= P.nlevels || h->deterministic) return P.nlevels;
    return queue_policy_level(P, h->queue_panels, prec) >= P.nlevels ? P.nlevels : h->q_level;
}

// Item list of a queue over a set of panels (fqueue.cuh): their diagonal
// blocks and TRSM chunks, and the update tiles of the tasks whose source is
// in the set (targets outside the set receive their updates but are not
// factored).  Built per level l: its diagonal blocks; the far update tiles of
// level l-1 (targets above level l); its TRSM chunks; its near update tiles
// (targets at level l+1); then reordered by list scheduling.  Every wait is
// then on an earlier item, which is checked here.  mode 0: CUDA-core update
// tiles (`tiles`), 1: tensor-core tiles (`tct`) and the narrow sources'
// CUDA-core tiles (`small`).
spx_status make_items(spx_handle h, const std::vector<RowChunk> &chunks, const std::vector<UpdTile> &tiles,
                      const std::vector<UpdTile> &small, const std::vector<spx::TcTile> &tct,
                      const std::vector<int32_t> &pchunk, const std::vector<char> &in_set, int workers, int mode,
                      std::vector<spx::FqItem> &items, std::vector<int32_t> &need)
{
    const spx::Plan &P = h->plan;
    const int32_t np = P.npanels;
    const int64_t nch = (int64_t)chunks.size();
    items.clear();
    need.assign(np, 0);
    {
        auto level_tiles = [&](int l, bool near) {
            auto take = [&](int32_t kind, int64_t idx, int32_t task) {
                const int32_t tgt = P.tasks[task].tgt;
                if (!in_set[P.tasks[task].src] || (P.plevel[tgt] == l + 1) != near) return;
                items.push_back(spx::FqItem{kind, (int32_t)idx});
                ++need[tgt];
            };
            if (mode == 0) {
                for (int64_t i = h->tile_ptr[l]; i < h->tile_nar[l]; ++i) take(spx::FQ_UPD64, i, tiles[i].task);
                for (int64_t i = h->tile_nar[l]; i < h->tile_ptr[l + 1]; ++i) take(spx::FQ_UPD16, i, tiles[i].task);
            } else {
                for (int64_t i = h->tctile_ptr[l]; i < h->tctile_ptr[l + 1]; ++i) take(spx::FQ_TC, i, tct[i].task);
                for (int64_t i = h->tcsmall_ptr[l]; i < h->tcsmall_nar[l]; ++i) take(spx::FQ_UPD64, i, small[i].task);
                for (int64_t i = h->tcsmall_nar[l]; i < h->tcsmall_ptr[l + 1]; ++i)
                    take(spx::FQ_UPD16, i, small[i].task);
            }
        };
        // expected counts, for the check below
        int64_t ntiles = 0, ndiag_want = 0, ntrsm_want = 0;
        for (const UpdTile &t : (mode == 0 ? tiles : small)) ntiles += in_set[P.tasks[t.task].src];
        if (mode == 1)
            for (const spx::TcTile &t : tct) ntiles += in_set[P.tasks[t.task].src];
        for (int32_t q = 0; q < np; ++q) ndiag_want += in_set[q];
        for (int64_t c = 0; c < nch; ++c) ntrsm_want += in_set[chunks[c].panel];
        for (int l = 0; l < P.nlevels; ++l) {
            for (int32_t q = P.level_ptr[l]; q < P.level_ptr[l + 1]; ++q)
                if (in_set[P.level_panels[q]]) items.push_back(spx::FqItem{spx::FQ_DIAG, P.level_panels[q]});
            if (l >= 1) level_tiles(l - 1, false);
            for (int64_t c = h->chunk_ptr[l]; c < h->chunk_ptr[l + 1]; ++c)
                if (in_set[chunks[c].panel]) items.push_back(spx::FqItem{spx::FQ_TRSM, (int32_t)c});
            level_tiles(l, true);
        }
        // Dispatch order: list scheduling of the item DAG on `workers` CTAs
        // with estimated durations, highest remaining critical path first
        // (the diagonal-block chain), so that the bulk of the update tiles
        // fills the time around the chain instead of queueing ahead of it.
        // The order in which the simulation starts items is topological, so
        // the no-stall property of the queue holds for it as well.
        {
            const int32_t N = (int32_t)items.size();
            std::vector<int32_t> pos_d(np, -1), pos_c(nch, -1);
            for (int32_t i = 0; i < N; ++i) {
                if (items[i].kind == spx::FQ_DIAG) pos_d[items[i].idx] = i;
                else if (items[i].kind == spx::FQ_TRSM) pos_c[items[i].idx] = i;
            }
            std::vector<std::vector<int32_t>> succ(N);
            std::vector<int32_t> indeg(N, 0);
            std::vector<double> dur(N, 8.0);   // microseconds, rough: a TRSM chunk or an update tile
            auto edge = [&](int32_t a, int32_t b) {
                succ[a].push_back(b);
                ++indeg[b];
            };
            for (int32_t i = 0; i < N; ++i) {
                const spx::FqItem &it = items[i];
                if (it.kind == spx::FQ_DIAG) {
                    const int w = P.pw[it.idx];
                    dur[i] = w <= 16 ? 10.0 : (w <= 32 ? 20.0 : 60.0);
                } else if (it.kind == spx::FQ_TRSM) {
                    edge(pos_d[chunks[it.idx].panel], i);
                } else {
                    int32_t task, m0, n0, tm, tn;
                    if (it.kind == spx::FQ_TC) {
                        task = tct[it.idx].task, m0 = tct[it.idx].m0, n0 = tct[it.idx].n0, tm = tn = 128;
                    } else {
                        const UpdTile &t = mode == 0 ? tiles[it.idx] : small[it.idx];
                        task = t.task, m0 = t.m0, n0 = t.n0;
                        tn = it.kind == spx::FQ_UPD16 ? spx::kUpdNarrowN : spx::kUpdTile;
                        tm = 4096 / tn;
                    }
                    const spx::Task &tk = P.tasks[task];
                    const int hsrc = P.ph[tk.src], w = P.pw[tk.src];
                    const int64_t lo[2] = {m0, n0}, hi[2] = {std::min(m0 + tm, hsrc), std::min(n0 + tn, tk.r1)};
                    int64_t last = -1;
                    for (int r = 0; r < 2; ++r) {
                        for (int64_t c = pchunk[tk.src] + (lo[r] - w) / spx::kTrsmRows;
                             c <= pchunk[tk.src] + (hi[r] - 1 - w) / spx::kTrsmRows; ++c) {
                            if (c == last || c < 0 || c >= nch || pos_c[c] < 0) continue;
                            edge(pos_c[c], i);
                            last = c;
                        }
                    }
                    if (pos_d[tk.tgt] >= 0) edge(i, pos_d[tk.tgt]);
                }
            }
            // remaining critical path of each item (items are in a topological order)
            std::vector<double> prio(N, 0.0);
            for (int32_t i = N - 1; i >= 0; --i) {
                double m = 0.0;
                for (int32_t j : succ[i]) m = std::max(m, prio[j]);
                prio[i] = dur[i] + m;
            }
            std::priority_queue<std::pair<double, int32_t>> ready;   // (priority, -index)
            std::priority_queue<std::pair<double, int32_t>, std::vector<std::pair<double, int32_t>>,
                                std::greater<std::pair<double, int32_t>>>
                running;   // (finish time, index)
            for (int32_t i = 0; i < N; ++i)
                if (indeg[i] == 0) ready.push({prio[i], -i});
            std::vector<spx::FqItem> order;
            order.reserve(N);
            int free_workers = std::max(1, workers);
            double now = 0.0;
            while ((int32_t)order.size() < N) {
                while (free_workers > 0 && !ready.empty()) {
                    const int32_t i = -ready.top().second;
                    ready.pop();
                    order.push_back(items[i]);
                    running.push({now + dur[i], i});
                    --free_workers;
                }
                if (running.empty()) break;
                const std::pair<double, int32_t> f = running.top();
                running.pop();
                now = f.first;
                ++free_workers;
                for (int32_t j : succ[f.second])
                    if (--indeg[j] == 0) ready.push({prio[j], -j});
            }
            if ((int32_t)order.size() != N)
                return fail(h, SPX_ERR_STATE, "internal: cycle in the factorization queue's task graph");
            items.swap(order);
        }
        // dependency check: every wait names an earlier item
        std::vector<int64_t> pos_diag(np, -1), pos_chunk(nch, -1);
        int64_t ndiag = 0, ntrsm = 0, ntile = 0;
        for (size_t i = 0; i < items.size(); ++i) {
            const spx::FqItem &it = items[i];
            if (it.kind == spx::FQ_DIAG) pos_diag[it.idx] = (int64_t)i, ++ndiag;
            else if (it.kind == spx::FQ_TRSM) pos_chunk[it.idx] = (int64_t)i, ++ntrsm;
            else ++ntile;
        }
        bool ok = ntile == ntiles && ndiag == ndiag_want && ntrsm == ntrsm_want;
        auto chunks_done_before = [&](int src, int r_lo, int r_hi, int64_t at) {
            if (pchunk[src] < 0 || r_lo < P.pw[src] || r_hi <= r_lo) return false;
            const int64_t c0 = pchunk[src] + (r_lo - P.pw[src]) / spx::kTrsmRows;
            const int64_t c1 = pchunk[src] + (r_hi - 1 - P.pw[src]) / spx::kTrsmRows;
            if (c1 - c0 + 1 > 32) return false;   // one waiting thread per chunk in the first warp
            for (int64_t c = c0; c <= c1; ++c)
                if (c >= nch || chunks[c].panel != src || pos_chunk[c] < 0 || pos_chunk[c] >= at) return false;
            return true;
        };
        for (size_t i = 0; i < items.size() && ok; ++i) {
            const spx::FqItem &it = items[i];
            if (it.kind == spx::FQ_DIAG) continue;
            if (it.kind == spx::FQ_TRSM) {
                ok = pos_diag[chunks[it.idx].panel] >= 0 && pos_diag[chunks[it.idx].panel] < (int64_t)i;
                continue;
            }
            int32_t task, m0, n0, tm, tn;
            if (it.kind == spx::FQ_TC) {
                task = tct[it.idx].task, m0 = tct[it.idx].m0, n0 = tct[it.idx].n0, tm = tn = 128;
            } else {
                const UpdTile &t = mode == 0 ? tiles[it.idx] : small[it.idx];
                task = t.task, m0 = t.m0, n0 = t.n0;
                tn = it.kind == spx::FQ_UPD16 ? spx::kUpdNarrowN : spx::kUpdTile;
                tm = 4096 / tn;
            }
            const spx::Task &tk = P.tasks[task];
            const int hsrc = P.ph[tk.src];
            ok = in_set[tk.src] && (!in_set[tk.tgt] || pos_diag[tk.tgt] > (int64_t)i) &&
                 chunks_done_before(tk.src, m0, std::min(m0 + tm, hsrc), (int64_t)i) &&
                 chunks_done_before(tk.src, n0, std::min(n0 + tn, tk.r1), (int64_t)i);
        }
        if (!ok) return fail(h, SPX_ERR_STATE, "internal: factorization queue order violates a dependency");
    }
    return SPX_OK;
}

// The queue of the upper levels [q_level, nlevels), both update modes.
spx_status build_queue(spx_handle h, const std::vector<RowChunk> &chunks, const std::vector<UpdTile> &tiles,
                       const std::vector<UpdTile> &small, const std::vector<spx::TcTile> &tct, int workers)
{
    const spx::Plan &P = h->plan;
    const int L0 = queue_start_level(P, h->queue_panels == 0 ? INT32_MAX : h->queue_panels);
    h->q_level = L0;
    const int32_t np = P.npanels;
    const int64_t nch = (int64_t)chunks.size();
    std::vector<int32_t> pchunk(np, -1);
    for (int64_t c = 0; c < nch; ++c)
        if (chunks[c].r0 == P.pw[chunks[c].panel]) pchunk[chunks[c].panel] = (int32_t)c;
    spx_status st;
    h->fq_nchunks = nch;
    if ((st = upload(h, &h->d_fq_pchunk, pchunk)) ||
        (st = dalloc(h, &h->d_fq_state, (size_t)2 * np + (size_t)nch + 2)))
        return st;
    h->h_pchunk = pchunk;
    if (L0 >= P.nlevels) return SPX_OK;
    std::vector<char> in_set(np, 0);
    for (int32_t q = 0; q < np; ++q) in_set[q] = P.plevel[q] >= L0;
    for (int mode = 0; mode < 2; ++mode) {
        std::vector<spx::FqItem> items;
        std::vector<int32_t> need;
        if ((st = make_items(h, chunks, tiles, small, tct, pchunk, in_set, workers, mode, items, need))) return st;
        h->fq_nitems[mode] = (int32_t)items.size();
        if ((st = upload(h, &h->d_fq_items[mode], items)) || (st = upload(h, &h->d_fq_need[mode], need))) return st;
    }
    return SPX_OK;
}

spx_status ensure_device(spx_handle h)
{
    if (h->uploaded) return SPX_OK;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CU(cudaGetDeviceProperties(&prop, dev));
    if (prop.major * 10 + prop.minor != 103)
        return fail(h, SPX_ERR_CUDA,
                    "libspx is built for sm_103a; the current device is sm_" +
                        std::to_string(prop.major * 10 + prop.minor));
    h->device = dev;
    CU(cudaStreamCreateWithFlags(&h->hs, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        CU(cudaStreamCreateWithFlags(&h->aux[k], cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&h->ev_join[k], cudaEventDisableTiming));
    }
    CU(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&h->ev_trsm, cudaEventDisableTiming));
    for (int k = 0; k < 2; ++k) {
        CU(cudaStreamCreateWithFlags(&h->fstream[k], cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&h->ev_far[k], cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&h->ev_near[k], cudaEventDisableTiming));
    }
    CU(cudaEventCreateWithFlags(&h->ev_fence, cudaEventDisableTiming));
    CU(cudaEventCreate(&h->ev_t0));
    CU(cudaEventCreate(&h->ev_t1));
    CU(cudaHostAlloc((void **)&h->h_noalloc_err, sizeof(int32_t), cudaHostAllocDefault));
    *h->h_noalloc_err = 0;

    const spx::Plan &P = h->plan;
    spx_status st;
    int64_t *pfcol, *prow, *pval, *pinv;
    int32_t *pw, *ph, *rows, *relmap;
    std::vector<int64_t> hpinv(P.npanels + 1, 0);
    // each inverted diagonal block starts on a 32-element (>= 128-byte)
    // boundary, so that no cache line holds two panels' blocks: within one
    // persistent factorization launch a block is read with plain loads by
    // other CTAs right after its diagonal item wrote it
    for (int32_t q = 0; q < P.npanels; ++q)
        hpinv[q + 1] = hpinv[q] + (((int64_t)P.pw[q] * P.pw[q] + 31) & ~(int64_t)31);
    h->dinv_elems = hpinv[P.npanels];
    h->lvl_wmax.assign(P.nlevels, 1);
    for (int32_t l = 0; l < P.nlevels; ++l)
        for (int32_t q = P.level_ptr[l]; q < P.level_ptr[l + 1]; ++q)
            h->lvl_wmax[l] = std::max(h->lvl_wmax[l], P.pw[P.level_panels[q]]);
    if ((st = upload(h, &pinv, hpinv))) return st;
    std::vector<int32_t> lp_sorted(P.level_panels.size());
    h->cls_ptr.assign((size_t)P.nlevels * kNumClasses + 1, 0);
    for (int32_t l = 0; l < P.nlevels; ++l) {
        int32_t pos = P.level_ptr[l];
        for (int c = 0; c < kNumClasses; ++c) {
            h->cls_ptr[(size_t)l * kNumClasses + c] = pos;
            for (int32_t q = P.level_ptr[l]; q < P.level_ptr[l + 1]; ++q)
                if (width_class(P.pw[P.level_panels[q]]) == c) lp_sorted[pos++] = P.level_panels[q];
        }
    }
    h->cls_ptr[(size_t)P.nlevels * kNumClasses] = P.level_ptr[P.nlevels];
    if ((st = upload(h, &pfcol, P.pfcol)) || (st = upload(h, &pw, P.pw)) ||
        (st = upload(h, &ph, P.ph)) || (st = upload(h, &prow, P.prow)) ||
        (st = upload(h, &rows, P.rows)) || (st = upload(h, &pval, P.pval)) ||
        (st = upload(h, &relmap, P.relmap)) || (st = upload(h, &h->d_level_panels, lp_sorted)) ||
        (st = upload(h, &h->d_amap, P.amap)) || (st = upload(h, &h->d_csr_ptr, P.csr_ptr)) ||
        (st = upload(h, &h->d_csr_col, P.csr_col)) || (st = upload(h, &h->d_csr_src, P.csr_src)) ||
        (st = upload(h, &h->d_perm, P.perm)))
        return st;
    h->dp.n = P.n;
    h->dp.npanels = P.npanels;
    h->dp.pfcol = pfcol;
    h->dp.pw = pw;
    h->dp.ph = ph;
    h->dp.prow = prow;
    h->dp.rows = rows;
    h->dp.pval = pval;
    h->dp.pinv = pinv;
    h->dp.relmap = relmap;

    std::vector<DevTask> tasks(P.tasks.size());
    for (size_t t = 0; t < P.tasks.size(); ++t)
        tasks[t] = DevTask{P.tasks[t].src, P.tasks[t].tgt, P.tasks[t].r0, P.tasks[t].r1,
                           P.tasks[t].relmap_off};
    if ((st = upload(h, &h->d_tasks, tasks))) return st;

    // per-level launch lists: row chunks of the off-diagonal parts, update tiles
    std::vector<RowChunk> chunks;
    std::vector<UpdTile> tiles, tilesu;
    h->chunk_ptr.assign(P.nlevels + 1, 0);
    h->tile_ptr.assign(P.nlevels + 1, 0);
    h->tile_nar.assign(P.nlevels, 0);
    h->tileu_ptr.assign(P.nlevels + 1, 0);
    h->tileu_nar.assign(P.nlevels, 0);
    // Tiles of one task over source rows [mlo, hk) x columns [r0, r1): 64 x 64
    // tiles, or 256 x 16 tiles when the task faces at most 16 rows (r1 - r0 <= 16,
    // where a 64-wide tile would leave three quarters of its columns idle).
    // Lower-triangular targets skip the tiles lying wholly above the diagonal.
    auto add_tiles = [](std::vector<UpdTile> &wide, std::vector<UpdTile> &nar, int32_t t,
                        const spx::Task &tk, int32_t mlo, int32_t hk, bool lower) {
        const int32_t N = tk.r1 - tk.r0;
        const int TN = N <= spx::kUpdNarrowN ? spx::kUpdNarrowN : spx::kUpdTile;
        const int TM = 4096 / TN;
        std::vector<UpdTile> &out = TN == spx::kUpdTile ? wide : nar;
        for (int32_t m0 = mlo; m0 < hk; m0 += TM)
            for (int32_t n0 = tk.r0; n0 < tk.r1; n0 += TN) {
                if (lower && m0 + TM <= n0) continue;
                out.push_back(UpdTile{t, m0, n0, 0});
            }
    };
    for (int32_t l = 0; l < P.nlevels; ++l) {
        for (int32_t q = P.level_ptr[l]; q < P.level_ptr[l + 1]; ++q) {
            int32_t k = P.level_panels[q];
            for (int32_t r0 = P.pw[k]; r0 < P.ph[k]; r0 += spx::kTrsmRows)
                chunks.push_back(RowChunk{k, r0});
        }
        std::vector<UpdTile> nar, naru;
        for (int32_t t = P.level_task_ptr[l]; t < P.level_task_ptr[l + 1]; ++t) {
            const spx::Task &tk = P.tasks[t];
            const int32_t hk = P.ph[tk.src];
            add_tiles(tiles, nar, t, tk, tk.r0, hk, P.method != SPX_LU);
            if (P.method == SPX_LU) add_tiles(tilesu, naru, t, tk, tk.r1, hk, false);
        }
        h->tile_nar[l] = (int64_t)tiles.size();
        tiles.insert(tiles.end(), nar.begin(), nar.end());
        h->tileu_nar[l] = (int64_t)tilesu.size();
        tilesu.insert(tilesu.end(), naru.begin(), naru.end());
        h->chunk_ptr[l + 1] = (int64_t)chunks.size();
        h->tile_ptr[l + 1] = (int64_t)tiles.size();
        h->tileu_ptr[l + 1] = (int64_t)tilesu.size();
    }
    // rounds of the deterministic mode; every per-level tile segment is kept
    // sorted by round (the order inside a level does not matter otherwise)
    std::vector<int32_t> task_round(P.tasks.size(), 0);
    h->det_rounds.assign(P.nlevels, 0);
    h->det_base.assign(P.nlevels + 1, 0);
    for (int32_t l = 0; l < P.nlevels; ++l) {
        std::vector<int32_t> seen;   // the level's targets, sorted
        int32_t R = 0;
        for (int32_t t = P.level_task_ptr[l]; t < P.level_task_ptr[l + 1]; ++t) seen.push_back(P.tasks[t].tgt);
        std::sort(seen.begin(), seen.end());
        std::vector<int32_t> used(seen.size(), 0);
        for (int32_t t = P.level_task_ptr[l]; t < P.level_task_ptr[l + 1]; ++t) {
            const size_t k = std::lower_bound(seen.begin(), seen.end(), P.tasks[t].tgt) - seen.begin();
            task_round[t] = used[k]++;
            R = std::max(R, task_round[t] + 1);
        }
        h->det_rounds[l] = R;
        h->det_base[l + 1] = h->det_base[l] + R + 1;
    }
    // deterministic mode: sorted by round, with the round boundaries; else
    // the near tiles (targets at level l + 1) first, with where they end
    auto sort_segment = [&](std::vector<UpdTile> &v, int64_t a, int64_t b, int32_t l, std::vector<int64_t> &ptr,
                            std::vector<int64_t> &near) {
        auto is_far = [&](const UpdTile &x) { return P.plevel[P.tasks[x.task].tgt] != l + 1; };
        if (h->deterministic) {
            std::stable_sort(v.begin() + a, v.begin() + b, [&](const UpdTile &x, const UpdTile &y) {
                return task_round[x.task] < task_round[y.task];
            });
            int64_t i = a;
            for (int32_t r = 0; r <= h->det_rounds[l]; ++r) {
                while (i < b && task_round[v[i].task] < r) ++i;
                ptr.push_back(i);
            }
            near.push_back(b);
        } else {
            std::stable_partition(v.begin() + a, v.begin() + b, [&](const UpdTile &x) { return !is_far(x); });
            int64_t i = a;
            while (i < b && !is_far(v[i])) ++i;
            near.push_back(i);
            for (int32_t r = 0; r <= h->det_rounds[l]; ++r) ptr.push_back(r == 0 ? a : b);
        }
    };
    for (int32_t l = 0; l < P.nlevels; ++l) {
        sort_segment(tiles, h->tile_ptr[l], h->tile_nar[l], l, h->det_ptr[0], h->near_end[0]);
        sort_segment(tiles, h->tile_nar[l], h->tile_ptr[l + 1], l, h->det_ptr[1], h->near_end[1]);
        sort_segment(tilesu, h->tileu_ptr[l], h->tileu_nar[l], l, h->det_ptr[2], h->near_end[2]);
        sort_segment(tilesu, h->tileu_nar[l], h->tileu_ptr[l + 1], l, h->det_ptr[3], h->near_end[3]);
    }
    if ((st = upload(h, &h->d_chunks, chunks)) || (st = upload(h, &h->d_tiles, tiles)) ||
        (st = upload(h, &h->d_tilesu, tilesu)))
        return st;
    {
        // Sweep queues.  Forward: per level its panel items, then its chunks;
        // backward: levels from the root down, chunks before panel items.
        // A chunk's rows are columns of ancestor panels; each distinct owner
        // is one count for the forward wait and one flag for the backward.
        // With panels at most 64 wide, a panel item also takes its first
        // chunk (the rows right below the diagonal block, usually the
        // parent's columns), which halves the items on a chain of panels.
        const int32_t np = P.npanels;
        const int32_t nchunk = (int32_t)chunks.size();
        int32_t wmax = 1;
        for (int32_t q = 0; q < np; ++q) wmax = std::max(wmax, P.pw[q]);
        const bool merge = wmax <= 64;
        std::vector<int32_t> itf, itb, tptr(1, 0), tgt, needf(np, 0), needb(np, 0), pmerge(np, -1);
        std::vector<char> merged(nchunk, 0);
        itf.reserve((size_t)np + nchunk);
        itb.reserve((size_t)np + nchunk);
        for (int32_t c = 0; c < nchunk; ++c) {
            if (merge && chunks[c].r0 == P.pw[chunks[c].panel]) {
                pmerge[chunks[c].panel] = c;
                merged[c] = 1;
            }
        }
        for (int32_t c = 0; c < nchunk; ++c) {
            const RowChunk &ch = chunks[c];
            const int32_t *r = P.rows.data() + P.prow[ch.panel];
            const int32_t r1 = std::min(ch.r0 + spx::kTrsmRows, P.ph[ch.panel]);
            int32_t last = -1;
            for (int32_t i = ch.r0; i < r1; ++i) {
                const int32_t q = P.col2panel[r[i]];
                if (q != last) {   // rows ascend, so owners come in runs
                    tgt.push_back(q);
                    ++needf[q];
                    last = q;
                }
            }
            tptr.push_back((int32_t)tgt.size());
            if (!merged[c]) ++needb[ch.panel];
        }
        for (int32_t l = 0; l < P.nlevels; ++l) {
            for (int32_t q = P.level_ptr[l]; q < P.level_ptr[l + 1]; ++q) itf.push_back(-(P.level_panels[q] + 1));
            for (int64_t c = h->chunk_ptr[l]; c < h->chunk_ptr[l + 1]; ++c)
                if (!merged[c]) itf.push_back((int32_t)c);
        }
        for (int32_t l = P.nlevels - 1; l >= 0; --l) {
            for (int64_t c = h->chunk_ptr[l]; c < h->chunk_ptr[l + 1]; ++c)
                if (!merged[c]) itb.push_back((int32_t)c);
            for (int32_t q = P.level_ptr[l]; q < P.level_ptr[l + 1]; ++q) itb.push_back(-(P.level_panels[q] + 1));
        }
        // Every wait must name an item earlier in its queue (else the walk
        // could stall); checked here, before any kernel sees the queues.
        {
            std::vector<int64_t> posf(np, -1), posb(np, -1), cposf(nchunk, -1), cposb(nchunk, -1);
            for (size_t i = 0; i < itf.size(); ++i)
                (itf[i] < 0 ? posf[-itf[i] - 1] : cposf[itf[i]]) = (int64_t)i;
            for (size_t i = 0; i < itb.size(); ++i)
                (itb[i] < 0 ? posb[-itb[i] - 1] : cposb[itb[i]]) = (int64_t)i;
            int64_t nmerged = 0;
            for (int32_t c = 0; c < nchunk; ++c) nmerged += merged[c];
            bool ok = itf.size() == itb.size() && (int64_t)itf.size() == (int64_t)np + nchunk - nmerged;
            for (int32_t q = 0; q < np && ok; ++q) ok = posf[q] >= 0 && posb[q] >= 0;
            for (int32_t c = 0; c < nchunk && ok; ++c) {
                const int32_t pc = chunks[c].panel;
                // a chunk taken along by its panel item runs at that item's place
                const int64_t cf = merged[c] ? posf[pc] : cposf[c];
                const int64_t cb = merged[c] ? posb[pc] : cposb[c];
                ok = merged[c] ? (cposf[c] < 0 && cposb[c] < 0 && pmerge[pc] == c)
                               : (cf > posf[pc] && cb < posb[pc]);
                for (int32_t t = tptr[c]; t < tptr[c + 1] && ok; ++t)
                    ok = tgt[t] != pc && posf[tgt[t]] > cf && posb[tgt[t]] < cb;
            }
            if (!ok) return fail(h, SPX_ERR_STATE, "internal: sweep queue order violates a dependency");
        }
        h->q_nitems = (int32_t)itf.size();
        // staging sizes in elements, multiples of 4 so that the vectors
        // after the matrices stay aligned for 4-element vector accesses
        // (the backward sweep stores a w x w inverse with an odd leading
        // dimension, w + 1 or w + 2)
        h->q_mat = (wmax * std::max(wmax + ((wmax & 1) ? 2 : 1), 65) + 3) & ~3;
        h->q_matb = merge ? (65 * wmax + 3) & ~3 : 0;
        h->q_vec = 16 * std::max(wmax, 64);
        if ((st = upload(h, &h->d_qitems_f, itf)) || (st = upload(h, &h->d_qitems_b, itb)) ||
            (st = upload(h, &h->d_qtptr, tptr)) || (st = upload(h, &h->d_qtgt, tgt)) ||
            (st = upload(h, &h->d_qneed_f, needf)) || (st = upload(h, &h->d_qneed_b, needb)) ||
            (st = upload(h, &h->d_qmerge, pmerge)) ||
            (st = dalloc(h, &h->d_qstate, (size_t)4 * np + 2)) || (st = dalloc(h, &h->d_qerr, 1)))
            return st;
        CU(cudaMemset(h->d_qerr, 0, sizeof(int32_t)));
    }
    if (P.method != SPX_LU) {
        std::vector<UpdTile> small;
        std::vector<spx::TcTile> tct;
        h->tcsmall_ptr.assign(P.nlevels + 1, 0);
        h->tcsmall_nar.assign(P.nlevels, 0);
        h->tctile_ptr.assign(P.nlevels + 1, 0);
        for (int32_t l = 0; l < P.nlevels; ++l) {
            std::vector<UpdTile> nar;
            for (int32_t t = P.level_task_ptr[l]; t < P.level_task_ptr[l + 1]; ++t) {
                const spx::Task &tk = P.tasks[t];
                const int32_t hk = P.ph[tk.src];
                if (P.pw[tk.src] >= kTcMinWidth) {
                    const double M = hk - tk.r0, N = tk.r1 - tk.r0, K = P.pw[tk.src];
                    h->upd_flops_tc += 2.0 * (M - N) * N * K + N * (N + 1.0) * K;
                    h->upd_op_elems_tc += (M + N) * K;
                    h->upd_elems_tc += 2.0 * ((M - N) * N + N * (N + 1.0) / 2.0);
                    for (int32_t m0 = tk.r0; m0 < hk; m0 += 128)
                        for (int32_t n0 = tk.r0; n0 < tk.r1; n0 += 128) {
                            if (m0 + 128 <= n0) continue;
                            tct.push_back(spx::TcTile{t, m0, n0, 0});
                        }
                } else {
                    add_tiles(small, nar, t, tk, tk.r0, hk, true);
                }
            }
            h->tcsmall_nar[l] = (int64_t)small.size();
            small.insert(small.end(), nar.begin(), nar.end());
            h->tcsmall_ptr[l + 1] = (int64_t)small.size();
            h->tctile_ptr[l + 1] = (int64_t)tct.size();
        }
        for (int32_t l = 0; l < P.nlevels; ++l) {
            std::vector<UpdTile> tmp;   // the tensor-core tiles through the same sort
            tmp.reserve((size_t)(h->tctile_ptr[l + 1] - h->tctile_ptr[l]));
            for (int64_t i = h->tctile_ptr[l]; i < h->tctile_ptr[l + 1]; ++i)
                tmp.push_back(UpdTile{tct[i].task, tct[i].m0, tct[i].n0, 0});
            std::vector<int64_t> ptr, nr;
            sort_segment(tmp, 0, (int64_t)tmp.size(), l, ptr, nr);
            for (size_t i = 0; i < tmp.size(); ++i)
                tct[h->tctile_ptr[l] + i] = spx::TcTile{tmp[i].task, tmp[i].m0, tmp[i].n0, 0};
            for (int64_t v : ptr) h->det_ptr[4].push_back(v + h->tctile_ptr[l]);
            h->near_end[4].push_back(nr[0] + h->tctile_ptr[l]);
            sort_segment(small, h->tcsmall_ptr[l], h->tcsmall_nar[l], l, h->det_ptr[5], h->near_end[5]);
            sort_segment(small, h->tcsmall_nar[l], h->tcsmall_ptr[l + 1], l, h->det_ptr[6], h->near_end[6]);
        }
        // chain links: see link_task.  The link's own task keeps only the rows
        // below q's diagonal block: 128-row tiles from its row r1 = r0 + 64
        // instead of from r0
        h->link_task.assign(P.nlevels, -1);
        h->link_ptr.assign(P.nlevels + 1, 0);
        std::vector<spx::TcTile> ltct;
        for (int32_t l = 0; l < P.nlevels; ++l) {
            h->link_ptr[l] = (int64_t)ltct.size();
            if (P.method != SPX_LLT || l + 1 >= P.nlevels || P.level_ptr[l + 1] - P.level_ptr[l] != 1 ||
                P.level_ptr[l + 2] - P.level_ptr[l + 1] != 1)
                continue;
            const int32_t pk = P.level_panels[P.level_ptr[l]], qk = P.level_panels[P.level_ptr[l + 1]];
            const int32_t w = P.pw[pk];
            if (P.pparent[pk] != qk || w != spx::kUpdTile || P.pw[qk] != spx::kUpdTile || w < kTcMinWidth ||
                P.ph[pk] < w + spx::kUpdTile || h->chunk_ptr[l + 1] - h->chunk_ptr[l] < 1 ||
                chunks[h->chunk_ptr[l]].panel != pk || chunks[h->chunk_ptr[l]].r0 != w)
                continue;
            bool rows_ok = true;
            for (int32_t i = 0; i < spx::kUpdTile && rows_ok; ++i)
                rows_ok = P.rows[P.prow[pk] + w + i] == P.pfcol[qk] + i;
            if (!rows_ok) continue;
            int32_t lt = -1;
            for (int32_t t = P.level_task_ptr[l]; t < P.level_task_ptr[l + 1]; ++t)
                if (P.tasks[t].src == pk && P.tasks[t].tgt == qk && P.tasks[t].r0 == w &&
                    P.tasks[t].r1 == w + spx::kUpdTile)
                    lt = t;
            if (lt < 0) continue;
            const int64_t n0 = h->tctile_ptr[l], n1 = h->near_end[4][l];
            int64_t ntask = 0;
            for (int64_t i = h->tctile_ptr[l]; i < h->tctile_ptr[l + 1]; ++i)
                if (tct[i].task == lt) {
                    if (i >= n1) ntask = -1;   // the link's tiles must all be near ones
                    if (ntask >= 0) ++ntask;
                }
            if (ntask <= 0) continue;
            for (int64_t i = n0; i < n1; ++i)
                if (tct[i].task != lt) ltct.push_back(tct[i]);
            const spx::Task &tk = P.tasks[lt];
            for (int32_t m0 = tk.r1; m0 < P.ph[pk]; m0 += 128) ltct.push_back(spx::TcTile{lt, m0, tk.r0, 0});
            h->link_task[l] = lt;
        }
        h->link_ptr[P.nlevels] = (int64_t)ltct.size();
        if ((st = upload(h, &h->d_tcsmall, small)) || (st = upload(h, &h->d_tctiles, tct)) ||
            (!ltct.empty() && (st = upload(h, &h->d_link_tct, ltct))))
            return st;
        int nsm = 0;
        CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
        h->workers = 2 * nsm;   // two queue CTAs per SM
        if ((st = build_queue(h, chunks, tiles, small, tct, h->workers))) return st;
        h->hc_chunks = chunks;
        h->hc_tiles = tiles;
        h->hc_small = small;
        h->hc_tct = tct;
    } else {
        h->q_level = P.nlevels;
    }
    {
        int wmax_all = 1;
        for (int32_t q = 0; q < P.npanels; ++q) wmax_all = std::max(wmax_all, P.pw[q]);
        h->kpad = (wmax_all + 63) & ~63;
        h->op_rows = P.prow[P.npanels];
    }
    if ((st = dalloc(h, &h->d_tcerr, 1))) return st;
    if ((st = dalloc(h, &h->d_nneg, 1))) return st;
    if ((st = dalloc(h, &h->d_vals, (size_t)P.nnz_a)) || (st = dalloc(h, &h->d_tau, 1)) ||
        (st = dalloc(h, &h->d_anorm, 1)) || (st = dalloc(h, &h->d_err, 1)) ||
        (st = dalloc(h, &h->d_nrepl, 1)))
        return st;
    h->uploaded = true;
    return SPX_OK;
}

// Enqueue the whole factorization on h->hs (captured into a graph).
// Profiling: events recorded between kernel classes (non-graph runs only).
struct Marks {
    spx_handle h;
    bool on;
    size_t used = 0;
    std::vector<std::pair<int, size_t>> spans;   // class, index of its end event
    void mark(int cls)
    {
        if (!on) return;
        if (used >= h->ev_pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            h->ev_pool.push_back(e);
        }
        cudaEventRecord(h->ev_pool[used], h->hs);
        if (cls >= 0) spans.emplace_back(cls, used);
        ++used;
    }
};

// Which symmetric factorizations send their wide updates to the tensor
// cores, and in which operand form (see launch_update_tc): Cholesky in TF32,
// BF16 or split TF32 (FP32 mode); LDL^T in TF32 or BF16 with a separate
// D L^T operand (its FP32 mode stays on the CUDA cores).
bool uses_tensor_cores(int method, int prec)
{
    if (method == SPX_LU) return false;
    if (method == SPX_LDLT) return prec == SPX_TF32 || prec == SPX_BF16;
    return prec == SPX_TF32 || prec == SPX_BF16 || prec == SPX_FP32;
}

int operand_kind(int method, int prec)
{
    if (method == SPX_LDLT) return prec == SPX_BF16 ? 4 : 3;
    return prec == SPX_BF16 ? 1 : (prec == SPX_FP32 ? 2 : 0);
}

// Independent launches of one level (the diagonal blocks of different width
// classes; the CUDA-core and tensor-core update tiles, which only meet in
// atomic reductions) go on parallel branches of the captured graph: launch
// k of a group runs on the main stream (k = 0) or on side stream k - 1 after
// a fork, and the group ends with a join.  Off (one stream) when profiling,
// so that the per-class events stay meaningful, and for the deterministic
// rounds, whose order the launch order is.
struct Branches {
    spx_handle h;
    bool on;
    bool forked[2] = {false, false};
    cudaStream_t pick(int k)
    {
        if (!on || k == 0) return h->hs;
        const int a = (k - 1) % 2;
        if (!forked[a]) {
            if (!forked[0] && !forked[1]) cudaEventRecord(h->ev_fork, h->hs);
            cudaStreamWaitEvent(h->aux[a], h->ev_fork, 0);
            forked[a] = true;
        }
        return h->aux[a];
    }
    void join()
    {
        for (int a = 0; a < 2; ++a)
            if (forked[a]) {
                cudaEventRecord(h->ev_join[a], h->aux[a]);
                cudaStreamWaitEvent(h->hs, h->ev_join[a], 0);
                forked[a] = false;
            }
    }
};

// One launch of the task queue over the item list of a partition part (rank
// r >= 0, or -1 for the top panels); the lists were built by ensure_part_items.
template <typename T>
void enqueue_part_queue(spx_handle h, T *L, T *Dinv, T *W, void *opc, void *opc_lo, int op_kind, bool tc, bool ldlt,
                        int part, cudaStream_t s)
{
    const spx::Plan &P = h->plan;
    const int mode = tc ? 1 : 0;
    const spx_handle_s::Part &pt = h->parts[part >= 0 ? part : h->part_nranks];
    const int32_t np = P.npanels;
    int32_t *st = h->d_fq_state;
    cudaMemsetAsync(st, 0, sizeof(int32_t) * ((size_t)2 * np + (size_t)h->fq_nchunks + 2), s);
    spx::FactorQueue q{};
    q.items = pt.d_items[mode];
    q.nitems = pt.nitems[mode];
    q.need = pt.d_need[mode];
    q.pchunk = h->d_fq_pchunk;
    q.cnt = st;
    q.diag_done = st + np;
    q.chunk_done = st + 2 * (size_t)np;
    q.head = st + 2 * (size_t)np + h->fq_nchunks;
    q.err = q.head + 1;
    q.spin_limit = h->spin_limit;
    spx::launch_factor_queue<T>(h->dp, q, h->d_tasks, h->d_chunks, tc ? h->d_tcsmall : h->d_tiles, h->d_tctiles, L,
                                Dinv, W, h->d_tau, h->d_err, h->d_nrepl, h->d_nneg, ldlt ? 1 : 0, tc ? op_kind : -1,
                                h->tmap, h->tmap_lo, opc, opc_lo, h->kpad, op_kind, s);
}

constexpr int kWhole = INT32_MIN;   // enqueue_factorization: the whole factorization

template <typename T>
void enqueue_factorization(spx_handle h, bool mixed, Marks &mk, int prec, int part = kWhole)
{
    const spx::Plan &P = h->plan;
    cudaStream_t s = h->hs;
    T *L = (T *)h->d_L, *U = (T *)h->d_U, *Dinv = (T *)h->d_Dinv;
    const size_t elems = (size_t)P.pval[P.npanels];
    const bool lu = P.method == SPX_LU;
    const bool ldlt = P.method == SPX_LDLT;
    const bool tc = uses_tensor_cores(P.method, prec) && sizeof(T) == 4;
    void *opc = tc ? h->d_opc : nullptr;
    void *opc_lo = tc ? h->d_opc_lo : nullptr;
    const int op_kind = operand_kind(P.method, prec);
    T *W = (T *)h->d_W;
    int64_t &cnt = h->cnt;
    for (int c = 0; c < SPX_K_CLASSES; ++c) h->class_launches[c] = 0;
    mk.mark(-1);
    if (part != kWhole && part < 0) {   // the top of a partition: its values came in by spx_part_set
        enqueue_part_queue<T>(h, L, Dinv, W, opc, opc_lo, op_kind, tc, ldlt, part, s);
        cnt += 2;
        return;
    }
    init_scalars_kernel<<<1, 1, 0, s>>>(h->d_err, h->d_nrepl, h->d_anorm);
    cudaMemsetAsync(h->d_tcerr, 0, sizeof(int), s);
    cudaMemsetAsync(h->d_nneg, 0, sizeof(unsigned long long), s);
    spx::launch_row_abs_sum_max(P.n, h->d_csr_ptr, h->d_csr_src, h->d_vals, h->d_anorm, s);
    const double sqrt_eps = std::sqrt(std::ldexp(1.0, -52));
    if (lu || ldlt)
        set_tau_kernel<<<1, 1, 0, s>>>(h->d_anorm, h->pivot_tau_opt, sqrt_eps, h->d_tau);
    else
        set_tau_kernel<<<1, 1, 0, s>>>(h->d_anorm, mixed ? -1.0 : 0.0, sqrt_eps, h->d_tau);
    cnt += 3;
    cudaMemsetAsync(L, 0, elems * sizeof(T), s);
    if (U) cudaMemsetAsync(U, 0, elems * sizeof(T), s);
    spx::launch_assemble<T>(P.nnz_a, h->d_vals, h->d_amap, L, U, s);
    cnt += P.nnz_a > 0;
    mk.mark(SPX_K_ASSEMBLE);
    if (part != kWhole) {
        // a rank's subtrees: the top panels collect only this rank's
        // contributions (rank 0 keeps A's values there, the others start from 0)
        const spx_handle_s::Part &top = h->parts[h->part_nranks];
        if (part > 0) spx::launch_pack_ranges<T>(top.d_ranges, top.nr, L, (T *)nullptr, 2, s);
        enqueue_part_queue<T>(h, L, Dinv, W, opc, opc_lo, op_kind, tc, ldlt, part, s);
        cnt += 2 + (part > 0);
        return;
    }
    const int32_t qlev = queue_level(h, prec);
    // look-ahead (graph runs outside the deterministic mode): a level's far
    // update tiles (targets two or more levels up) run on a side stream
    // beside the next level's diagonal blocks, TRSM and near tiles, and are
    // joined before the diagonal blocks of level l + 2
    const bool lookahead = !mk.on && !h->deterministic && !lu;
    bool far_pending[2] = {false, false};
    // chain links (look-ahead by one diagonal block): after panel p's diagonal
    // block a one-CTA step solves p's rows facing q and updates q's diagonal
    // block with them; q's diagonal block follows at once on the main stream,
    // while p's other TRSM chunks and update tiles run on a side stream whose
    // near part is joined before q's own TRSM (or link step)
    bool near_pending = false;
    int near_slot = 0;
    for (int32_t l = 0; l < qlev; ++l) {
        if (far_pending[l % 2]) {   // the far tiles of level l - 2
            cudaStreamWaitEvent(s, h->ev_far[l % 2], 0);
            far_pending[l % 2] = false;
        }
        const int32_t *panels = h->d_level_panels + P.level_ptr[l];
        const int np = P.level_ptr[l + 1] - P.level_ptr[l];
        const RowChunk *ch = h->d_chunks + h->chunk_ptr[l];
        const int nch = (int)(h->chunk_ptr[l + 1] - h->chunk_ptr[l]);
        const UpdTile *tl = h->d_tiles + h->tile_ptr[l];
        const int ntl = (int)(h->tile_nar[l] - h->tile_ptr[l]);
        const UpdTile *tln = h->d_tiles + h->tile_nar[l];
        const int ntln = (int)(h->tile_ptr[l + 1] - h->tile_nar[l]);
        const int wmax = h->lvl_wmax[l];
        Branches br{h, !mk.on};
        int nlaunch = 0;
        for (int c = 0; c < kNumClasses; ++c) {
            const int32_t a = h->cls_ptr[(size_t)l * kNumClasses + c];
            const int32_t b = h->cls_ptr[(size_t)l * kNumClasses + c + 1];
            if (b <= a) continue;
            const int cw = std::min(kClassWidth[c], wmax);
            const cudaStream_t sc = br.pick(nlaunch++);
            if (ldlt)
                spx::launch_ldlt_diag<T>(h->dp, h->d_level_panels + a, b - a, cw, L, Dinv, h->d_tau, h->d_err,
                                         h->d_nrepl, h->d_nneg, sc);
            else if (!lu)
                spx::launch_potrf<T>(h->dp, h->d_level_panels + a, b - a, cw, kClassThreads[c], L,
                                     Dinv, h->d_tau, h->d_err, h->d_nrepl, sc);
            else
                spx::launch_getrf<T>(h->dp, h->d_level_panels + a, b - a, cw, kClassThreads[c], L,
                                     Dinv, h->d_tau, h->d_err, h->d_nrepl, sc);
            cnt += 1;
            h->class_launches[SPX_K_DIAG] += 1;
        }
        br.join();
        (void)panels;
        (void)np;
        mk.mark(SPX_K_DIAG);
        if (near_pending) {   // the previous link's TRSM and near tiles
            cudaStreamWaitEvent(s, h->ev_near[near_slot], 0);
            near_pending = false;
        }
        const bool link = lookahead && tc && !ldlt && l + 1 < qlev && h->link_task.size() == (size_t)P.nlevels &&
                          h->link_task[l] >= 0;
        // update launches of this level: one set, or one set per round in the
        // deterministic mode (slices of the round-sorted tile segments)
        // (a level without update tasks has no rounds: nothing to launch)
        const int nround = h->deterministic ? h->det_rounds[l] : 1;
        auto seg = [&](int sgi, int64_t a, int64_t b, int r, int64_t *lo) -> int {
            if (!h->deterministic) {
                *lo = a;
                return (int)(b - a);
            }
            // round r of the segment [a, b): det_rounds[l] + 1 boundaries from det_base[l]
            const int64_t *ptr = h->det_ptr[sgi].data() + h->det_base[l];
            const int64_t x = ptr[r], y = ptr[r + 1];
            if (r >= h->det_rounds[l] || x < a || y > b || y < x) {   // never: the lists were built so
                *lo = a;
                return 0;
            }
            *lo = x;
            return (int)(y - x);
        };
        int64_t o;
        if (!lu) {
            if (!link) {
                spx::launch_trsm<T>(h->dp, ch, nch, wmax, Dinv, L, ldlt ? spx::TRSM_LDLT : spx::TRSM_LLT, opc,
                                    opc_lo, h->kpad, op_kind, s, W);
                cnt += nch > 0;
                h->class_launches[SPX_K_TRSM] += nch > 0;
            }
            mk.mark(SPX_K_TRSM);
            const T *Bop = ldlt ? W : L;   // LDL^T: C -= L (D L^T)
            // one set of update launches over tile ranges: wide and narrow
            // CUDA-core tiles, and the tensor-core tiles in tc modes
            const spx::TcTile *tcbase = h->d_tctiles;
            auto launch_set = [&](int64_t a0, int64_t a1, int64_t b0, int64_t b1, int64_t c0, int64_t c1,
                                  Branches &ub, cudaStream_t one) {
                const int na = (int)(a1 - a0), nb = (int)(b1 - b0), nc = (int)(c1 - c0);
                auto st = [&](int k) { return one ? one : ub.pick(k); };
                if (!tc) {
                    spx::launch_update<T>(h->dp, h->d_tasks, h->d_tiles + a0, na, L, Bop, L, 1, 0, st(0), 0);
                    spx::launch_update<T>(h->dp, h->d_tasks, h->d_tiles + b0, nb, L, Bop, L, 1, 0,
                                          st(na > 0 ? 1 : 0), 1);
                } else {
                    // the tensor-core tiles on the main stream, the CUDA-core ones beside them
                    spx::launch_update_tc(h->tmap, h->tmap_lo, op_kind, h->dp, h->d_tasks, tcbase + c0, nc,
                                          (float *)L, 1, h->d_tcerr, st(0));
                    mk.mark(SPX_K_UPDATE_TC);
                    spx::launch_update<T>(h->dp, h->d_tasks, h->d_tcsmall + a0, na, L, Bop, L, 1, 0,
                                          st(nc > 0 ? 1 : 0), 0);
                    spx::launch_update<T>(h->dp, h->d_tasks, h->d_tcsmall + b0, nb, L, Bop, L, 1, 0,
                                          st((nc > 0) + (na > 0)), 1);
                }
                cnt += (na > 0) + (nb > 0) + (nc > 0);
                h->class_launches[SPX_K_UPDATE] += (na > 0) + (nb > 0);
                h->class_launches[SPX_K_UPDATE_TC] += nc > 0;
            };
            // segment ranges of this level: wide, narrow (CUDA cores), tensor cores
            const int sa = tc ? 5 : 0, sb = tc ? 6 : 1;
            const int64_t A0 = tc ? h->tcsmall_ptr[l] : h->tile_ptr[l], A1 = tc ? h->tcsmall_nar[l] : h->tile_nar[l];
            const int64_t B0 = A1, B1 = tc ? h->tcsmall_ptr[l + 1] : h->tile_ptr[l + 1];
            const int64_t C0 = tc ? h->tctile_ptr[l] : 0, C1 = tc ? h->tctile_ptr[l + 1] : 0;
            if (h->deterministic) {
                for (int r = 0; r < nround; ++r) {
                    int64_t oa, ob, oc = 0;
                    const int na = seg(sa, A0, A1, r, &oa), nb = seg(sb, B0, B1, r, &ob);
                    const int nc = tc ? seg(4, C0, C1, r, &oc) : 0;
                    Branches ub{h, false};
                    launch_set(oa, oa + na, ob, ob + nb, oc, oc + nc, ub, nullptr);
                    mk.mark(SPX_K_UPDATE);
                }
            } else if (!lookahead) {
                Branches ub{h, !mk.on};
                launch_set(A0, A1, B0, B1, C0, C1, ub, nullptr);
                ub.join();
                mk.mark(SPX_K_UPDATE);
            } else if (link) {
                if constexpr (std::is_same<T, float>::value) {
                    const int32_t lt = h->link_task[l];
                    spx::launch_lead<T>(h->dp, h->hc_chunks[h->chunk_ptr[l]], h->d_tasks, lt, Dinv, L, opc, opc_lo,
                                        h->kpad, op_kind, s);
                    cnt += 1;
                    h->class_launches[SPX_K_TRSM] += 1;
                    cudaEventRecord(h->ev_trsm, s);
                    cudaStream_t fs = h->fstream[l % 2];
                    cudaStreamWaitEvent(fs, h->ev_trsm, 0);
                    spx::launch_trsm<T>(h->dp, ch + 1, nch - 1, wmax, Dinv, L, spx::TRSM_LLT, opc, opc_lo, h->kpad,
                                        op_kind, fs, W);
                    cnt += nch > 1;
                    h->class_launches[SPX_K_TRSM] += nch > 1;
                    const int64_t An = h->near_end[sa][l], Bn = h->near_end[sb][l], Cn = h->near_end[4][l];
                    Branches none{h, false};
                    tcbase = h->d_link_tct;
                    launch_set(A0, An, B0, Bn, h->link_ptr[l], h->link_ptr[l + 1], none, fs);
                    tcbase = h->d_tctiles;
                    cudaEventRecord(h->ev_near[l % 2], fs);
                    near_pending = true;
                    near_slot = l % 2;
                    if (An < A1 || Bn < B1 || Cn < C1) {
                        launch_set(An, A1, Bn, B1, Cn, C1, none, fs);
                        cudaEventRecord(h->ev_far[l % 2], fs);
                        far_pending[l % 2] = true;
                    }
                }
            } else {
                const int64_t An = h->near_end[sa][l], Bn = h->near_end[sb][l], Cn = tc ? h->near_end[4][l] : 0;
                const bool far = An < A1 || Bn < B1 || Cn < C1;
                if (far) cudaEventRecord(h->ev_trsm, s);   // this level's TRSM is done
                Branches ub{h, true};
                launch_set(A0, An, B0, Bn, C0, Cn, ub, nullptr);
                ub.join();
                if (far) {
                    cudaStream_t fs = h->fstream[l % 2];
                    cudaStreamWaitEvent(fs, h->ev_trsm, 0);
                    Branches none{h, false};
                    launch_set(An, A1, Bn, B1, Cn, C1, none, fs);
                    cudaEventRecord(h->ev_far[l % 2], fs);
                    far_pending[l % 2] = true;
                }
            }
        } else {
            spx::launch_trsm<T>(h->dp, ch, nch, wmax, Dinv, L, spx::TRSM_LU_L, nullptr, nullptr, 0, 0, s);
            spx::launch_trsm<T>(h->dp, ch, nch, wmax, Dinv, U, spx::TRSM_LU_U, nullptr, nullptr, 0, 0, s);
            cnt += 2 * (nch > 0);
            h->class_launches[SPX_K_TRSM] += 2 * (nch > 0);
            mk.mark(SPX_K_TRSM);
            for (int r = 0; r < nround; ++r) {
                const int a = seg(0, h->tile_ptr[l], h->tile_nar[l], r, &o);
                spx::launch_update<T>(h->dp, h->d_tasks, h->d_tiles + o, a, L, U, L, 0, 0, s, 0);
                const int b = seg(1, h->tile_nar[l], h->tile_ptr[l + 1], r, &o);
                spx::launch_update<T>(h->dp, h->d_tasks, h->d_tiles + o, b, L, U, L, 0, 0, s, 1);
                const int c = seg(2, h->tileu_ptr[l], h->tileu_nar[l], r, &o);
                spx::launch_update<T>(h->dp, h->d_tasks, h->d_tilesu + o, c, U, L, U, 0, 1, s, 0);
                const int d = seg(3, h->tileu_nar[l], h->tileu_ptr[l + 1], r, &o);
                spx::launch_update<T>(h->dp, h->d_tasks, h->d_tilesu + o, d, U, L, U, 0, 1, s, 1);
                cnt += (a > 0) + (b > 0) + (c > 0) + (d > 0);
                h->class_launches[SPX_K_UPDATE] += (a > 0) + (b > 0) + (c > 0) + (d > 0);
                mk.mark(SPX_K_UPDATE);
            }
        }
    }
    for (int k = 0; k < 2; ++k)
        if (far_pending[k]) cudaStreamWaitEvent(s, h->ev_far[k], 0);
    if (near_pending) cudaStreamWaitEvent(s, h->ev_near[near_slot], 0);
    if (qlev < P.nlevels) {
        // the upper levels: one persistent launch over the task queue
        const int mode = tc ? 1 : 0;
        const int32_t np = P.npanels;
        int32_t *st = h->d_fq_state;
        cudaMemsetAsync(st, 0, sizeof(int32_t) * ((size_t)2 * np + (size_t)h->fq_nchunks + 2), s);
        spx::FactorQueue q{};
        q.items = h->d_fq_items[mode];
        q.nitems = h->fq_nitems[mode];
        q.need = h->d_fq_need[mode];
        q.pchunk = h->d_fq_pchunk;
        q.cnt = st;
        q.diag_done = st + np;
        q.chunk_done = st + 2 * (size_t)np;
        q.head = st + 2 * (size_t)np + h->fq_nchunks;
        q.err = q.head + 1;
        q.spin_limit = h->spin_limit;
        spx::launch_factor_queue<T>(h->dp, q, h->d_tasks, h->d_chunks, tc ? h->d_tcsmall : h->d_tiles, h->d_tctiles,
                                    L, Dinv, W, h->d_tau, h->d_err, h->d_nrepl, h->d_nneg, ldlt ? 1 : 0,
                                    tc ? op_kind : -1, h->tmap, h->tmap_lo, opc, opc_lo, h->kpad, op_kind, s);
        cnt += 2;
        h->class_launches[SPX_K_QUEUE] += 1;
        mk.mark(SPX_K_QUEUE);
    }
}

// One forward + backward sweep in the factor's arithmetic: d_D = A^{-1} d_R.
// Forward and backward substitution, Y (permuted right-hand sides) to Xs,
// as one queue launch per direction (sweep.cu); Z and Tacc are work
// vectors, `state` the 4 npanels + 2 per-sweep counters.  Returns the
// kernels launched.
template <typename T>
int enqueue_queue_sweeps(spx_handle h, int nrhs, T *Y, T *Z, T *Tacc, T *Xs, int32_t *state, int32_t *err,
                         cudaStream_t s)
{
    const spx::Plan &P = h->plan;
    const T *L = (const T *)h->d_L, *U = (const T *)h->d_U, *Dinv = (const T *)h->d_Dinv;
    const bool lu = P.method == SPX_LU;
    const int32_t np = P.npanels;
    cudaMemsetAsync(Tacc, 0, sizeof(T) * (size_t)P.n * nrhs, s);
    cudaMemsetAsync(state, 0, sizeof(int32_t) * ((size_t)4 * np + 2), s);
    spx::SweepQueue q{};
    q.nitems = h->q_nitems;
    q.tptr = h->d_qtptr;
    q.tgt = h->d_qtgt;
    q.err = err;
    q.spin_limit = h->spin_limit;
    q.merge = h->d_qmerge;
    q.mat_elems = h->q_mat;
    q.matb_elems = h->q_matb;
    q.vec_elems = h->q_vec;
    q.items = h->d_qitems_f;
    q.need = h->d_qneed_f;
    q.cnt = state;
    q.flag = state + np;
    q.head = state + 4 * np;
    spx::launch_fwd_queue<T>(h->dp, q, h->d_chunks, Dinv, P.method != SPX_LLT ? 1 : 0, L, Y, Z, nrhs, s);
    q.items = h->d_qitems_b;
    q.need = h->d_qneed_b;
    q.cnt = state + 2 * np;
    q.flag = state + 3 * np;
    q.head = state + 4 * np + 1;
    spx::launch_bwd_queue<T>(h->dp, q, h->d_chunks, Dinv, lu ? 1 : (P.method == SPX_LDLT ? 2 : 0), lu ? U : L, Z,
                             Tacc, Xs, nrhs, s);
    return 2 * (q.nitems > 0);
}

template <typename T>
void enqueue_sweep(spx_handle h, int nrhs)
{
    const spx::Plan &P = h->plan;
    cudaStream_t s = h->hs;
    T *Y = (T *)h->d_Y, *Z = (T *)h->d_Z, *Tacc = (T *)h->d_T, *Xs = (T *)h->d_Xs;
    int64_t k = 0;
    spx::launch_permute_in<T>(P.n, nrhs, h->d_R, P.n, h->d_perm, Y, s);
    k += enqueue_queue_sweeps<T>(h, nrhs, Y, Z, Tacc, Xs, h->d_qstate, h->d_qerr, s);
    spx::launch_permute_out<T>(P.n, nrhs, Xs, h->d_perm, h->d_D, P.n, s);
    h->sweep_launches = k + 2;
}

spx_status capture(spx_handle h, cudaGraphExec_t *exec, void (*body)(spx_handle, int, bool),
                   int arg, bool flag)
{
    if (*exec) {
        cudaGraphExecDestroy(*exec);
        *exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->hs, cudaStreamCaptureModeThreadLocal));
    body(h, arg, flag);
    cudaError_t launch_err = cudaGetLastError();
    cudaError_t e = cudaStreamEndCapture(h->hs, &g);
    if (launch_err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(h, SPX_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(launch_err));
    }
    if (e != cudaSuccess) return fail(h, SPX_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, SPX_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return SPX_OK;
}

void body_factor(spx_handle h, int prec, bool)
{
    Marks mk{h, false};
    if (prec == SPX_FP64) enqueue_factorization<double>(h, false, mk, prec);
    else enqueue_factorization<float>(h, true, mk, prec);
}

// Operand copies for the tensor-core updates, allocated (zeroed) on first use.
spx_status ensure_operand_copy(spx_handle h, int kind)
{
    if (h->d_opc && h->opc_kind == kind) return SPX_OK;
    dfree(h, h->d_opc);
    dfree(h, h->d_opc_lo);
    h->d_opc = h->d_opc_lo = nullptr;
    h->opc_kind = -1;
    const int bf16 = kind == 1 || kind == 4;
    const size_t esz = bf16 ? 2 : 4;
    const size_t bytes = (size_t)h->op_rows * h->kpad * esz;
    for (int part = 0; part < (kind >= 2 ? 2 : 1); ++part) {
        char *p = nullptr;
        spx_status st = dalloc(h, &p, bytes);
        if (st != SPX_OK) return st;
        CU(cudaMemset(p, 0, bytes));
        if (spx::make_operand_map(part ? h->tmap_lo : h->tmap, p, h->op_rows, h->kpad, bf16) != 0)
            return fail(h, SPX_ERR_CUDA, "cuTensorMapEncodeTiled failed for the operand copy");
        (part ? h->d_opc_lo : h->d_opc) = p;
    }
    h->opc_kind = kind;
    if (h->fgraph) {   // the graph captured the old descriptors and buffers
        cudaGraphExecDestroy(h->fgraph);
        h->fgraph = nullptr;
        h->fgraph_prec = -1;
    }
    return SPX_OK;
}

// Copies between the caller's (pageable) host buffers and the device go
// through two pinned staging buffers owned by the handle: the host packs or
// unpacks one buffer while the copy engine moves the other, so pageable
// memory never takes the driver's slow bounce path.  The device side is
// contiguous (`cols` columns of `col_bytes`); the host side has pitch
// `hpitch`.  Ordered on h->hs.
constexpr size_t kStageBytes = (size_t)8 << 20;

spx_status ensure_stage(spx_handle h)
{
    for (int b = 0; b < 2; ++b) {
        if (!h->h_stage[b]) CU(cudaHostAlloc(&h->h_stage[b], kStageBytes, cudaHostAllocDefault));
        if (!h->ev_stage[b]) CU(cudaEventCreateWithFlags(&h->ev_stage[b], cudaEventDisableTiming));
    }
    if (!h->copy_pool) {
        const unsigned hw = std::thread::hardware_concurrency();
        h->copy_pool.reset(new CopyPool((int)std::min(7u, hw > 1 ? hw - 1 : 0u)));
    }
    return SPX_OK;
}


// walk the host side of a (cols x col_bytes) block in chunks of at most
// kStageBytes; fn(host_piece, bytes, offset_in_chunk) for each piece
template <typename F>
size_t chunk_pieces(size_t pos, size_t total, size_t col_bytes, size_t hpitch, char *host, F fn)
{
    const size_t len = std::min(kStageBytes, total - pos);
    size_t done = 0;
    while (done < len) {
        const size_t col = (pos + done) / col_bytes, off = (pos + done) % col_bytes;
        const size_t piece = std::min(len - done, col_bytes - off);
        fn(host + col * hpitch + off, piece, done);
        done += piece;
    }
    return len;
}

// Copy one staging chunk between the pinned buffer and the caller's pieces
// of it, the chunk's bytes split evenly over the copy threads.
template <bool TO_STAGE>
void copy_chunk(spx_handle h, char *stage, size_t pos, size_t total, size_t col_bytes, size_t hpitch, char *host)
{
    struct Piece {
        char *host;
        size_t bytes, at;
    };
    std::vector<Piece> pieces;
    const size_t len = chunk_pieces(pos, total, col_bytes, hpitch, host, [&](const char *hp, size_t bytes, size_t at) {
        pieces.push_back(Piece{const_cast<char *>(hp), bytes, at});
    });
    h->copy_pool->run([&](int k, int parts) {
        const size_t lo = (len * (size_t)k / (size_t)parts) & ~(size_t)63;
        const size_t hi = k + 1 == parts ? len : (len * (size_t)(k + 1) / (size_t)parts) & ~(size_t)63;
        for (const Piece &pc : pieces) {
            const size_t a = std::max(lo, pc.at), b = std::min(hi, pc.at + pc.bytes);
            if (a >= b) continue;
            if (TO_STAGE) std::memcpy(stage + a, pc.host + (a - pc.at), b - a);
            else std::memcpy(pc.host + (a - pc.at), stage + a, b - a);
        }
    });
}

spx_status staged_h2d(spx_handle h, void *dev, const void *host, size_t hpitch, size_t col_bytes, size_t cols)
{
    spx_status st = ensure_stage(h);
    if (st != SPX_OK) return st;
    const size_t total = col_bytes * cols;
    bool busy[2] = {false, false};
    int b = 0;
    for (size_t pos = 0; pos < total; b ^= 1) {
        if (busy[b]) CU(cudaEventSynchronize(h->ev_stage[b]));
        char *stage = (char *)h->h_stage[b];
        const size_t len = std::min(kStageBytes, total - pos);
        copy_chunk<true>(h, stage, pos, total, col_bytes, hpitch, (char *)host);
        CU(cudaMemcpyAsync((char *)dev + pos, stage, len, cudaMemcpyHostToDevice, h->hs));
        CU(cudaEventRecord(h->ev_stage[b], h->hs));
        busy[b] = true;
        pos += len;
    }
    return SPX_OK;
}

spx_status staged_d2h(spx_handle h, void *host, size_t hpitch, const void *dev, size_t col_bytes, size_t cols)
{
    spx_status st = ensure_stage(h);
    if (st != SPX_OK) return st;
    const size_t total = col_bytes * cols;
    size_t pend_pos[2] = {0, 0};
    bool busy[2] = {false, false};
    auto drain = [&](int b) -> spx_status {
        CU(cudaEventSynchronize(h->ev_stage[b]));
        copy_chunk<false>(h, (char *)h->h_stage[b], pend_pos[b], total, col_bytes, hpitch, (char *)host);
        busy[b] = false;
        return SPX_OK;
    };
    int b = 0;
    for (size_t pos = 0; pos < total; b ^= 1) {
        if (busy[b] && (st = drain(b))) return st;
        const size_t len = std::min(kStageBytes, total - pos);
        CU(cudaMemcpyAsync(h->h_stage[b], (const char *)dev + pos, len, cudaMemcpyDeviceToHost, h->hs));
        CU(cudaEventRecord(h->ev_stage[b], h->hs));
        busy[b] = true;
        pend_pos[b] = pos;
        pos += len;
        // unpack the other buffer while this chunk is in flight
        if (busy[b ^ 1] && (st = drain(b ^ 1))) return st;
    }
    for (int q = 0; q < 2; ++q)
        if (busy[q] && (st = drain(q))) return st;
    return SPX_OK;
}

void body_sweep(spx_handle h, int nrhs, bool fp64)
{
    if (fp64) enqueue_sweep<double>(h, nrhs);
    else enqueue_sweep<float>(h, nrhs);
}

void fence_from(spx_handle h, void *user_stream)
{
    cudaEventRecord(h->ev_fence, (cudaStream_t)user_stream);
    cudaStreamWaitEvent(h->hs, h->ev_fence, 0);
}

spx_status ensure_workspace(spx_handle h, int nrhs)
{
    if (h->ws_nrhs >= nrhs) return SPX_OK;
    for (double **p : {&h->d_B, &h->d_X, &h->d_R, &h->d_D, &h->d_Y, &h->d_Z, &h->d_T, &h->d_Xs}) {
        dfree(h, *p);
        *p = nullptr;
    }
    dfree(h, h->d_norms);
    h->d_norms = nullptr;
    h->ws_nrhs = 0;
    const size_t sz = (size_t)h->plan.n * nrhs;
    spx_status st;
    if ((st = dalloc(h, &h->d_B, sz)) || (st = dalloc(h, &h->d_X, sz)) ||
        (st = dalloc(h, &h->d_R, sz)) || (st = dalloc(h, &h->d_D, sz)) ||
        (st = dalloc(h, &h->d_Y, sz)) || (st = dalloc(h, &h->d_Z, sz)) ||
        (st = dalloc(h, &h->d_T, sz)) || (st = dalloc(h, &h->d_Xs, sz)) ||
        (st = dalloc(h, &h->d_norms, (size_t)3 * nrhs)))
        return st;
    h->ws_nrhs = nrhs;
    if (h->sgraph) {
        cudaGraphExecDestroy(h->sgraph);
        h->sgraph = nullptr;
        h->sgraph_nrhs = -1;
    }
    return SPX_OK;
}

// residual of d_X against d_B into d_R; returns the worst backward error
spx_status residual(spx_handle h, int nrhs, double *berr)
{
    const spx::Plan &P = h->plan;
    CU(cudaMemsetAsync(h->d_norms, 0, sizeof(unsigned long long) * 3 * nrhs, h->hs));
    spx::launch_residual(P.n, nrhs, h->d_csr_ptr, h->d_csr_col, h->d_csr_src, h->d_vals, h->d_X,
                         P.n, h->d_B, P.n, h->d_R, h->d_norms, h->hs);
    h->cnt += 1;
    std::vector<unsigned long long> nb(3 * nrhs);
    CU(cudaMemcpyAsync(nb.data(), h->d_norms, sizeof(unsigned long long) * 3 * nrhs,
                       cudaMemcpyDeviceToHost, h->hs));
    CU(cudaStreamSynchronize(h->hs));
    double worst = 0.0;
    h->last_xinf.assign(nrhs, 0.0);
    h->last_binf.assign(nrhs, 0.0);
    for (int c = 0; c < nrhs; ++c) {
        double r, x, b;
        std::memcpy(&r, &nb[3 * c], 8);
        std::memcpy(&x, &nb[3 * c + 1], 8);
        std::memcpy(&b, &nb[3 * c + 2], 8);
        h->last_xinf[c] = x;
        h->last_binf[c] = b;
        double den = h->anorm * x + b;
        double e = den > 0.0 ? r / den : (r > 0.0 ? INFINITY : 0.0);
        if (!(e <= worst)) worst = e;   // NaN propagates
    }
    *berr = worst;
    return SPX_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free solve: the sweep vectors live in this file-scope buffer.
// Host code must not hand the symbol itself to a kernel (in host code it is a
// host-side stand-in); its device address is looked up once per device, by
// spx_factorize, so that the module holding the buffer is loaded there and
// spx_solve_noalloc only reads the cached address.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char spx_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_addr[kMaxDevices] = {};

spx_status static_scratch_address(spx_handle h, int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) return fail(h, SPX_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, spx_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(h, SPX_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return SPX_OK;
}

// One forward + backward sweep from B (original numbering) to X with the
// sweep vectors Y, Z, Tacc, Xs carved out of `scratch`, followed by the
// 4 npanels + 2 sweep counters and the call's own error word (zeroed first,
// so that a timeout of an earlier call does not carry over); the error word
// is then copied to the handle's pinned host word.  Launches and
// stream-ordered copies only.
template <typename T>
void enqueue_sweep_noalloc(spx_handle h, int nrhs, const double *B, int64_t ldb, double *X,
                           int64_t ldx, T *scratch, cudaStream_t s)
{
    const spx::Plan &P = h->plan;
    const size_t len = (size_t)P.n * nrhs;
    T *Y = scratch, *Z = scratch + len, *Tacc = scratch + 2 * len, *Xs = scratch + 3 * len;
    int32_t *state = reinterpret_cast<int32_t *>(scratch + 4 * len);
    int32_t *err = state + 4 * (size_t)P.npanels + 2;
    cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    spx::launch_permute_in<T>(P.n, nrhs, B, ldb, h->d_perm, Y, s);
    enqueue_queue_sweeps<T>(h, nrhs, Y, Z, Tacc, Xs, state, err, s);
    spx::launch_permute_out<T>(P.n, nrhs, Xs, h->d_perm, X, ldx, s);
    cudaMemcpyAsync(h->h_noalloc_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
}

// ---------------------------------------------------------------------------
// FGMRES refinement (right preconditioned by the low-precision factor, FP64
// Arnoldi with two-pass classical Gram-Schmidt, one Krylov space per right-
// hand side, Givens rotations on the host).  Starts from d_X; returns the
// backward error of the final iterate and the iterations taken.
// ---------------------------------------------------------------------------
spx_status fgmres(spx_handle h, int nrhs, const spx_refine &rf, double *berr_out, int *iters_out)
{
    const spx::Plan &P = h->plan;
    const int64_t n = P.n;
    const size_t blk = (size_t)n * nrhs;
    const int m = std::max(1, std::min(rf.gmres_restart, 200));
    const int maxit = std::max(1, rf.gmres_max_iter);
    cudaStream_t s = h->hs;
    spx_status st;
    if (h->gm_m < m || h->gm_nrhs < nrhs) {
        for (double **p : {&h->d_gV, &h->d_gZ, &h->d_gw, &h->d_gcoef}) {
            dfree(h, *p);
            *p = nullptr;
        }
        h->gm_m = h->gm_nrhs = 0;
        if ((st = dalloc(h, &h->d_gV, blk * (m + 1))) || (st = dalloc(h, &h->d_gZ, blk * m)) ||
            (st = dalloc(h, &h->d_gw, blk)) || (st = dalloc(h, &h->d_gcoef, (size_t)(m + 2) * nrhs)))
            return st;
        h->gm_m = m;
        h->gm_nrhs = nrhs;
    }
    std::vector<double> H((size_t)nrhs * (m + 1) * m), cs((size_t)nrhs * m), sn((size_t)nrhs * m);
    std::vector<double> g((size_t)nrhs * (m + 1)), coef((size_t)(m + 1) * nrhs), sc(nrhs);
    std::vector<double> y((size_t)m * nrhs);
    auto Hat = [&](int c, int i, int j) -> double & { return H[((size_t)c * (m + 1) + i) * m + j]; };
    int total = 0;
    double berr = INFINITY;
    while (true) {
        if ((st = residual(h, nrhs, &berr))) return st;
        if (berr <= rf.tol || total >= maxit) break;
        // beta = ||r||_2 per column; V_0 = r / beta
        spx::launch_dots(n, nrhs, 1, h->d_R, h->d_R, h->d_gcoef, s);
        CU(cudaMemcpyAsync(coef.data(), h->d_gcoef, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        for (int c = 0; c < nrhs; ++c) {
            const double beta = std::sqrt(std::max(coef[c], 0.0));
            g[(size_t)c * (m + 1)] = beta;
            sc[c] = beta > 0.0 ? 1.0 / beta : 0.0;
        }
        CU(cudaMemcpyAsync(h->d_gcoef, sc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
        spx::launch_scale_cols(n, nrhs, h->d_R, h->d_gcoef, h->d_gV, s);
        int j = 0;
        while (j < m && total < maxit) {
            double *Vj = h->d_gV + blk * j, *Zj = h->d_gZ + blk * j;
            // z_j = M^{-1} v_j through the factor; w = A z_j
            CU(cudaMemcpyAsync(h->d_R, Vj, sizeof(double) * blk, cudaMemcpyDeviceToDevice, s));
            CU(cudaGraphLaunch(h->sgraph, s));
            CU(cudaMemcpyAsync(Zj, h->d_D, sizeof(double) * blk, cudaMemcpyDeviceToDevice, s));
            spx::launch_spmv_cols(n, nrhs, h->d_csr_ptr, h->d_csr_col, h->d_csr_src, h->d_vals, Zj,
                                  h->d_gw, s);
            h->cnt += h->sweep_launches + 1;
            for (int pass = 0; pass < 2; ++pass) {
                spx::launch_dots(n, nrhs, j + 1, h->d_gV, h->d_gw, h->d_gcoef, s);
                spx::launch_combine(n, nrhs, j + 1, h->d_gV, h->d_gcoef, -1.0, h->d_gw, s);
                CU(cudaMemcpyAsync(coef.data(), h->d_gcoef, sizeof(double) * (j + 1) * nrhs,
                                   cudaMemcpyDeviceToHost, s));
                CU(cudaStreamSynchronize(s));
                for (int c = 0; c < nrhs; ++c)
                    for (int i = 0; i <= j; ++i) Hat(c, i, j) += coef[(size_t)i * nrhs + c];
            }
            spx::launch_dots(n, nrhs, 1, h->d_gw, h->d_gw, h->d_gcoef, s);
            CU(cudaMemcpyAsync(coef.data(), h->d_gcoef, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            double worst = 0.0;
            for (int c = 0; c < nrhs; ++c) {
                const double hn = std::sqrt(std::max(coef[c], 0.0));
                Hat(c, j + 1, j) = hn;
                sc[c] = hn > 0.0 ? 1.0 / hn : 0.0;
                // previous rotations, then a new one that zeroes H(j+1, j)
                for (int i = 0; i < j; ++i) {
                    const double a0 = Hat(c, i, j), a1 = Hat(c, i + 1, j);
                    Hat(c, i, j) = cs[(size_t)c * m + i] * a0 + sn[(size_t)c * m + i] * a1;
                    Hat(c, i + 1, j) = -sn[(size_t)c * m + i] * a0 + cs[(size_t)c * m + i] * a1;
                }
                const double a0 = Hat(c, j, j), a1 = Hat(c, j + 1, j);
                const double rr = std::hypot(a0, a1);
                const double cc = rr > 0.0 ? a0 / rr : 1.0, ss = rr > 0.0 ? a1 / rr : 0.0;
                cs[(size_t)c * m + j] = cc;
                sn[(size_t)c * m + j] = ss;
                Hat(c, j, j) = rr;
                Hat(c, j + 1, j) = 0.0;
                const double gj = g[(size_t)c * (m + 1) + j];
                g[(size_t)c * (m + 1) + j] = cc * gj;
                g[(size_t)c * (m + 1) + j + 1] = -ss * gj;
                const double den = h->anorm * h->last_xinf[c] + h->last_binf[c];
                const double est = den > 0.0 ? std::fabs(g[(size_t)c * (m + 1) + j + 1]) / den : 0.0;
                worst = std::max(worst, est);
            }
            CU(cudaMemcpyAsync(h->d_gcoef, sc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
            spx::launch_scale_cols(n, nrhs, h->d_gw, h->d_gcoef, h->d_gV + blk * (j + 1), s);
            ++j;
            ++total;
            if (worst <= 0.1 * rf.tol) break;
        }
        // y = H^{-1} g (upper triangular j x j per column), x += Z y
        for (int c = 0; c < nrhs; ++c)
            for (int i = j - 1; i >= 0; --i) {
                double v = g[(size_t)c * (m + 1) + i];
                for (int k = i + 1; k < j; ++k) v -= Hat(c, i, k) * y[(size_t)k * nrhs + c];
                const double d = Hat(c, i, i);
                y[(size_t)i * nrhs + c] = d != 0.0 ? v / d : 0.0;
            }
        CU(cudaMemcpyAsync(h->d_gcoef, y.data(), sizeof(double) * j * nrhs, cudaMemcpyHostToDevice, s));
        spx::launch_combine(n, nrhs, j, h->d_gZ, h->d_gcoef, 1.0, h->d_X, s);
    }
    *berr_out = berr;
    *iters_out = total;
    return SPX_OK;
}

// Factor storage of the handle for `precision` (reallocated when the storage
// type changes).
spx_status ensure_factor_storage(spx_handle h, spx_precision precision)
{
    const spx::Plan &P = h->plan;
    const bool fp64 = precision == SPX_FP64;
    const size_t elems = (size_t)P.pval[P.npanels];
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    spx_status st;
    if (h->factor_prec_alloc != (fp64 ? 1 : 0)) {
        dfree(h, h->d_L);
        dfree(h, h->d_U);
        dfree(h, h->d_Dinv);
        h->d_L = h->d_U = h->d_Dinv = nullptr;
        h->factor_prec_alloc = -1;
        char *pl = nullptr, *pd = nullptr;
        if ((st = dalloc(h, &pl, elems * esz))) return st;
        h->d_L = pl;
        if ((st = dalloc(h, &pd, (size_t)h->dinv_elems * esz))) return st;
        h->d_Dinv = pd;
        dfree(h, h->d_W);
        h->d_W = nullptr;
        if (P.method == SPX_LDLT) {
            char *pw = nullptr;
            if ((st = dalloc(h, &pw, elems * esz))) return st;
            h->d_W = pw;
        }
        if (P.method == SPX_LU) {
            char *pu = nullptr;
            if ((st = dalloc(h, &pu, elems * esz))) return st;
            h->d_U = pu;
        }
        h->factor_prec_alloc = fp64 ? 1 : 0;
        if (h->fgraph) {
            cudaGraphExecDestroy(h->fgraph);
            h->fgraph = nullptr;
            h->fgraph_prec = -1;
        }
    }
    if (uses_tensor_cores(P.method, precision)) {
        if ((st = ensure_operand_copy(h, operand_kind(P.method, precision)))) return st;
    }
    return SPX_OK;
}

// Subtree-to-rank partition of the panel tree (the distribution of Sec. VI's
// fan-in): subtrees are split from the top, heaviest first, until there are
// at least nranks of them and a longest-first assignment to the ranks
// balances their work within 5% (or no subtree can be split further); the
// split roots and their ancestors are the top panels.  Work of a panel: its
// diagonal block, TRSM and the updates it sources (flops).  Every update task
// then stays inside one rank's subtree or goes from a subtree into the top,
// so each rank's contributions to the top panels can be summed (fan-in)
// before the top is factored.
spx_status make_partition(spx_handle h, int nranks)
{
    const spx::Plan &P = h->plan;
    const int32_t np = P.npanels;
    std::vector<double> w(np, 0.0);
    for (int32_t q = 0; q < np; ++q) {
        const double wd = P.pw[q], off = (double)P.ph[q] - P.pw[q];
        w[q] = wd * wd * wd / 3.0 + off * wd * wd;
    }
    for (const spx::Task &tk : P.tasks) {
        const double M = (double)P.ph[tk.src] - tk.r0, N = (double)tk.r1 - tk.r0, K = P.pw[tk.src];
        w[tk.src] += 2.0 * M * N * K;
    }
    std::vector<double> W(w);
    std::vector<std::vector<int32_t>> kids(np);
    for (int32_t q = 0; q < np; ++q) {
        const int32_t par = P.pparent[q];
        if (par >= 0) {
            if (par <= q) return fail(h, SPX_ERR_STATE, "internal: panel tree not in postorder");
            W[par] += W[q];
            kids[par].push_back(q);
        }
    }
    std::vector<int32_t> frontier;
    for (int32_t q = 0; q < np; ++q)
        if (P.pparent[q] < 0) frontier.push_back(q);
    std::vector<char> top(np, 0);
    std::vector<int32_t> root_rank;
    for (int it = 0; it <= np; ++it) {
        std::sort(frontier.begin(), frontier.end(), [&](int32_t a, int32_t b) { return W[a] > W[b] || (W[a] == W[b] && a < b); });
        std::vector<double> load(nranks, 0.0);
        root_rank.assign(frontier.size(), 0);
        double total = 0.0;
        for (size_t f = 0; f < frontier.size(); ++f) {
            const int r = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            root_rank[f] = r;
            load[r] += W[frontier[f]];
            total += W[frontier[f]];
        }
        const double imbalance = total > 0.0 ? *std::max_element(load.begin(), load.end()) / (total / nranks) : 1.0;
        if ((int)frontier.size() >= nranks && imbalance <= 1.05) break;
        size_t pick = frontier.size();
        for (size_t f = 0; f < frontier.size(); ++f)
            if (!kids[frontier[f]].empty()) {
                pick = f;
                break;
            }
        if (pick == frontier.size()) break;
        const int32_t q = frontier[pick];
        top[q] = 1;
        frontier.erase(frontier.begin() + pick);
        for (int32_t c : kids[q]) frontier.push_back(c);
    }
    h->panel_owner.assign(np, -1);
    for (size_t f = 0; f < frontier.size(); ++f) {
        std::vector<int32_t> stack(1, frontier[f]);
        while (!stack.empty()) {
            const int32_t q = stack.back();
            stack.pop_back();
            h->panel_owner[q] = root_rank[f];
            for (int32_t c : kids[q]) stack.push_back(c);
        }
    }
    for (int32_t q = 0; q < np; ++q)
        if ((h->panel_owner[q] < 0) != (top[q] != 0)) return fail(h, SPX_ERR_STATE, "internal: partition does not cover the tree");
    for (const spx::Task &tk : P.tasks) {   // the fan-in property
        const int a = h->panel_owner[tk.src], b = h->panel_owner[tk.tgt];
        if (!(a == b || b < 0)) return fail(h, SPX_ERR_STATE, "internal: an update crosses two subtrees");
    }
    // packed ranges per part: values, then inverse blocks
    for (auto &pt : h->parts) {
        dfree(h, pt.d_ranges);
        for (int m = 0; m < 2; ++m) {
            dfree(h, pt.d_items[m]);
            dfree(h, pt.d_need[m]);
        }
    }
    h->parts.assign(nranks + 1, spx_handle_s::Part{});
    std::vector<int64_t> hpinv(np + 1, 0);
    for (int32_t q = 0; q < np; ++q) hpinv[q + 1] = hpinv[q] + (((int64_t)P.pw[q] * P.pw[q] + 31) & ~(int64_t)31);
    for (int k = 0; k <= nranks; ++k) {
        const int owner = k < nranks ? k : -1;
        std::vector<int64_t> rv, ri;
        int64_t pos = 0;
        int32_t nr = 0;
        for (int32_t q = 0; q < np; ++q)
            if (h->panel_owner[q] == owner) {
                const int64_t len = P.pval[q + 1] - P.pval[q];
                rv.insert(rv.end(), {P.pval[q], len, pos});
                pos += len;
                ++nr;
            }
        const int64_t nval = pos;
        for (int32_t q = 0; q < np; ++q)
            if (h->panel_owner[q] == owner) {
                const int64_t len = (int64_t)P.pw[q] * P.pw[q];
                ri.insert(ri.end(), {hpinv[q], len, pos});
                pos += len;
            }
        rv.insert(rv.end(), ri.begin(), ri.end());
        spx_handle_s::Part &pt = h->parts[k];
        pt.nr = nr;
        pt.nval = nval;
        pt.ninv = pos - nval;
        pt.h_ranges.swap(rv);
    }
    h->part_nranks = nranks;
    return SPX_OK;
}

// Device copies of the partition's range lists (first device use).
spx_status ensure_part_device(spx_handle h)
{
    spx_status st = ensure_device(h);
    if (st != SPX_OK) return st;
    for (auto &pt : h->parts)
        if (!pt.d_ranges && (st = upload(h, &pt.d_ranges, pt.h_ranges))) return st;
    return SPX_OK;
}

// Queue item lists of partition part k (rank k, or nranks for the top) in
// update mode `mode`, built on first use.
spx_status ensure_part_items(spx_handle h, int k, int mode)
{
    spx_handle_s::Part &pt = h->parts[k];
    if (pt.nitems[mode] >= 0) return SPX_OK;
    const spx::Plan &P = h->plan;
    const int owner = k < h->part_nranks ? k : -1;
    std::vector<char> in_set(P.npanels, 0);
    for (int32_t q = 0; q < P.npanels; ++q) in_set[q] = h->panel_owner[q] == owner;
    std::vector<spx::FqItem> items;
    std::vector<int32_t> need;
    spx_status st = make_items(h, h->hc_chunks, h->hc_tiles, h->hc_small, h->hc_tct, h->h_pchunk, in_set, h->workers,
                               mode, items, need);
    if (st != SPX_OK) return st;
    if ((st = upload(h, &pt.d_items[mode], items)) || (st = upload(h, &pt.d_need[mode], need))) return st;
    pt.nitems[mode] = (int32_t)items.size();
    return SPX_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void spx_default_options(spx_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->ordering = SPX_ORDER_AUTO;
    opt->dof = 1;
    opt->max_width = 128;
    opt->amalg_ratio = 0.12;
    opt->perm = nullptr;
    opt->lower_only = 0;
    opt->pivot_tau = -1.0;
}

void spx_default_refine(spx_refine *r)
{
    if (!r) return;
    r->max_iter = 10;
    r->gmres_restart = 30;
    r->gmres_max_iter = 200;
    r->mode = 2;
    r->tol = 1e-12;
}

spx_status spx_analyze(int64_t n, const int64_t *colptr, const int32_t *rowind, spx_method method,
                       const spx_options *opt, spx_handle *out)
{
    spx_handle h = nullptr;
    if (!out) return fail(h, SPX_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!colptr || !rowind) return fail(h, SPX_ERR_ARG, "colptr/rowind is NULL");
    if (method != SPX_LLT && method != SPX_LU && method != SPX_LDLT) return fail(h, SPX_ERR_ARG, "unknown method");
    spx_options o;
    spx_default_options(&o);
    if (opt) o = *opt;
    if (o.max_width <= 0) o.max_width = 128;
    if (method == SPX_LDLT && o.max_width > 64) o.max_width = 64;   // the LDL^T diagonal kernel
    if (o.max_width > spx::kMaxWidth)
        return fail(h, SPX_ERR_ARG, "max_width above " + std::to_string(spx::kMaxWidth));
    if (o.amalg_ratio < 0) o.amalg_ratio = 0.12;
    if (o.lower_only && method == SPX_LU) return fail(h, SPX_ERR_ARG, "lower_only needs a symmetric method");
    h = new (std::nothrow) spx_handle_s();
    if (!h) return fail(nullptr, SPX_ERR_ALLOC, "out of host memory");
    spx::AnalyzeOptions ao;
    ao.ordering = o.ordering;
    ao.grid[0] = o.grid[0];
    ao.grid[1] = o.grid[1];
    ao.grid[2] = o.grid[2];
    ao.dof = o.dof > 0 ? o.dof : 1;
    ao.max_width = o.max_width;
    ao.amalg_ratio = o.amalg_ratio;
    ao.perm = o.perm;
    ao.lower_only = o.lower_only;
    std::string msg;
    try {
        // LDL^T has the symbolic structure of the Cholesky factorization
        msg = spx::analyze(n, colptr, rowind, method == SPX_LU ? (int)SPX_LU : (int)SPX_LLT, ao, h->plan);
        h->plan.method = method;
    } catch (const std::bad_alloc &) {
        msg = "out of host memory during analysis";
    }
    if (!msg.empty()) {
        delete h;
        return fail(nullptr, SPX_ERR_ARG, msg);
    }
    h->method = method;
    h->pivot_tau_opt = o.pivot_tau;
    h->queue_panels = o.queue_panels < 0 ? -1 : o.queue_panels;
    h->deterministic = o.deterministic != 0;
    const spx::Plan &P = h->plan;
    spx_info &I = h->info;
    I.n = P.n;
    I.nnz_a = P.nnz_a;
    I.nnz_l = P.nnz_l;
    I.nnz_stored = P.nnz_stored;
    I.nsupernodes = P.nsuper;
    I.npanels = P.npanels;
    I.nlevels = P.nlevels;
    I.nupdates = (int64_t)P.tasks.size();
    I.bad_col = -1;
    I.method = method;
    I.precision = -1;
    I.flops = P.flops_exact;
    I.flops_stored = P.flops_stored;
    I.update_flops = P.update_flops;
    I.analyze_ms = P.analyze_ms;
    *out = h;
    return SPX_OK;
}

spx_status spx_factorize(spx_handle h, const double *values, int values_on_device,
                         spx_precision precision, void *cuda_stream)
{
    if (!h) return fail(nullptr, SPX_ERR_ARG, "handle is NULL");
    if (!values && h->plan.nnz_a > 0) return fail(h, SPX_ERR_ARG, "values is NULL");
    if (precision < SPX_FP64 || precision > SPX_BF16) return fail(h, SPX_ERR_ARG, "unknown precision");
    spx_status st = ensure_device(h);
    if (st != SPX_OK) return st;
    {
        // look up the allocation-free solve's static buffer now, so that the
        // module holding it is loaded before any spx_solve_noalloc call
        void *scratch = nullptr;
        if ((st = static_scratch_address(h, h->device, &scratch)) != SPX_OK) return st;
    }
    const spx::Plan &P = h->plan;
    const bool fp64 = precision == SPX_FP64;
    const size_t elems = (size_t)P.pval[P.npanels];
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    if ((st = ensure_factor_storage(h, precision))) return st;
    h->factored = false;
    h->zready = false;
    fence_from(h, cuda_stream);
    if (values_on_device)
        CU(cudaMemcpyAsync(h->d_vals, values, sizeof(double) * (size_t)P.nnz_a, cudaMemcpyDeviceToDevice, h->hs));
    else if ((st = staged_h2d(h, h->d_vals, values, 0, sizeof(double) * (size_t)P.nnz_a, 1)))
        return st;
    Marks mk{h, h->profiling};
    if (h->profiling) {
        h->cnt = 0;
        CU(cudaEventRecord(h->ev_t0, h->hs));
        if (fp64) enqueue_factorization<double>(h, false, mk, (int)precision);
        else enqueue_factorization<float>(h, true, mk, (int)precision);
        CU(cudaGetLastError());
        CU(cudaEventRecord(h->ev_t1, h->hs));
        h->info.launches_factor = h->cnt;
    } else {
        if (h->fgraph_prec != (int)precision) {
            h->cnt = 0;
            if ((st = capture(h, &h->fgraph, body_factor, (int)precision, false))) return st;
            h->fgraph_prec = (int)precision;
            h->info.launches_factor = h->cnt;
        }
        CU(cudaEventRecord(h->ev_t0, h->hs));
        CU(cudaGraphLaunch(h->fgraph, h->hs));
        CU(cudaEventRecord(h->ev_t1, h->hs));
    }
    int64_t bad = 0;
    unsigned long long nrepl = 0, abits = 0;
    CU(cudaMemcpyAsync(&bad, h->d_err, sizeof(bad), cudaMemcpyDeviceToHost, h->hs));
    CU(cudaMemcpyAsync(&nrepl, h->d_nrepl, sizeof(nrepl), cudaMemcpyDeviceToHost, h->hs));
    CU(cudaMemcpyAsync(&abits, h->d_anorm, sizeof(abits), cudaMemcpyDeviceToHost, h->hs));
    int tcerr = 0, fqerr = 0;
    unsigned long long nneg = 0;
    CU(cudaMemcpyAsync(&tcerr, h->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, h->hs));
    if (queue_level(h, precision) < P.nlevels)
        CU(cudaMemcpyAsync(&fqerr, h->d_fq_state + 2 * (size_t)P.npanels + h->fq_nchunks + 1, sizeof(int),
                           cudaMemcpyDeviceToHost, h->hs));
    CU(cudaMemcpyAsync(&nneg, h->d_nneg, sizeof(nneg), cudaMemcpyDeviceToHost, h->hs));
    CU(cudaStreamSynchronize(h->hs));
    if (tcerr) return fail(h, SPX_ERR_TIMEOUT, "a tensor-core update tile gave up waiting on its pipeline");
    if (fqerr)
        return fail(h, SPX_ERR_TIMEOUT, fqerr == 2 ? "the factorization queue's tensor-core pipeline gave up waiting"
                                                   : "the factorization queue gave up waiting on a task counter");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1);
    if (h->profiling) {
        spx_kernel_stats &K = h->kstats;
        K = spx_kernel_stats{};
        for (auto &sp : mk.spans) {
            float t = 0.f;
            cudaEventElapsedTime(&t, h->ev_pool[sp.second - 1], h->ev_pool[sp.second]);
            K.ms[sp.first] += t;
        }
        const double e = fp64 ? 8.0 : 4.0;
        const double nfac = (P.method == SPX_LU) ? 2.0 : 1.0;
        const bool tcm = uses_tensor_cores(P.method, precision);
        const double eop = precision == SPX_BF16 ? 2.0 : (precision == SPX_FP32 ? 8.0 : 4.0);
        const int32_t qlev = queue_level(h, precision);
        // (LDL^T reads its B operand from a second copy of the same size: the bytes are the same)
        visit_work(P, tcm, [&](int cls, int lvl, double flops, double el, double el_op, double el_acc) {
            const int c = lvl >= qlev ? (int)SPX_K_QUEUE : cls;
            K.flops[c] += flops;
            K.bytes[c] += el * e + el_op * eop + el_acc * 4.0;
        });
        // zero fill of the factor (one write) + the scatter (value and map read, one write)
        K.bytes[SPX_K_ASSEMBLE] = (double)P.nnz_a * (16.0 + e * nfac) + (double)elems * e * nfac;
        K.launches[SPX_K_ASSEMBLE] = P.nnz_a > 0 ? 4 : 3;
        for (int c = 1; c < SPX_K_CLASSES; ++c) K.launches[c] = h->class_launches[c];
    }
    std::memcpy(&h->anorm, &abits, 8);
    h->info.factor_ms = ms;
    h->info.precision = precision;
    h->info.npivot_repl = (int64_t)nrepl;
    h->info.npivot_neg = P.method == SPX_LDLT ? (int64_t)nneg : 0;
    h->info.bad_col = (bad == LLONG_MAX) ? -1 : bad;
    h->info.factor_bytes = (int64_t)(elems * esz * (P.method == SPX_LLT ? 1 : 2));
    h->precision = precision;
    if (bad == -1)
        return fail(h, SPX_ERR_TIMEOUT, "a diagonal block's warps gave up waiting on each other");
    if (bad != LLONG_MAX) {
        return fail(h, P.method == SPX_LLT ? SPX_ERR_NOT_SPD : SPX_ERR_ZERO_PIVOT,
                    "pivot failure at permuted column " + std::to_string(bad));
    }
    h->factored = true;
    return SPX_OK;
}

spx_status spx_partition(spx_handle h, int32_t nranks, int32_t *panel_owner, int64_t *part_values,
                         int64_t *part_inverses)
{
    if (!h) return fail(nullptr, SPX_ERR_ARG, "handle is NULL");
    if (nranks < 1 || nranks > 4096) return fail(h, SPX_ERR_ARG, "nranks outside [1, 4096]");
    const spx::Plan &P = h->plan;
    if (P.method == SPX_LU) return fail(h, SPX_ERR_ARG, "the partitioned factorization takes Cholesky or LDL^T");
    for (int32_t q = 0; q < P.npanels; ++q)
        if (P.pw[q] > 64) return fail(h, SPX_ERR_ARG, "the partitioned factorization takes panels at most 64 wide");
    spx_status st = make_partition(h, nranks);
    if (st != SPX_OK) return st;
    if (panel_owner) std::memcpy(panel_owner, h->panel_owner.data(), sizeof(int32_t) * (size_t)P.npanels);
    for (int k = 0; k <= nranks; ++k) {
        if (part_values) part_values[k] = h->parts[k].nval;
        if (part_inverses) part_inverses[k] = h->parts[k].ninv;
    }
    return SPX_OK;
}

spx_status spx_factorize_part(spx_handle h, const double *values, int values_on_device, spx_precision precision,
                              int32_t part, void *cuda_stream)
{
    if (!h) return fail(nullptr, SPX_ERR_ARG, "handle is NULL");
    if (h->part_nranks < 1) return fail(h, SPX_ERR_STATE, "spx_factorize_part before spx_partition");
    if (part < -1 || part >= h->part_nranks) return fail(h, SPX_ERR_ARG, "part outside [-1, nranks)");
    if (precision < SPX_FP64 || precision > SPX_BF16) return fail(h, SPX_ERR_ARG, "unknown precision");
    const spx::Plan &P = h->plan;
    const bool fp64 = precision == SPX_FP64;
    spx_status st = ensure_part_device(h);
    if (st != SPX_OK) return st;
    if (part >= 0) {
        if (!values && P.nnz_a > 0) return fail(h, SPX_ERR_ARG, "values is NULL");
        if ((st = ensure_factor_storage(h, precision))) return st;
    } else if (h->factor_prec_alloc != (fp64 ? 1 : 0) || h->part_done != 1) {
        return fail(h, SPX_ERR_STATE, "the top part needs this handle's own subtrees factored first (same precision)");
    }
    const bool tc = uses_tensor_cores(P.method, precision) && !fp64;
    if ((st = ensure_part_items(h, part >= 0 ? part : h->part_nranks, tc ? 1 : 0))) return st;
    h->factored = false;
    h->zready = false;
    fence_from(h, cuda_stream);
    if (part >= 0) {
        if (values_on_device)
            CU(cudaMemcpyAsync(h->d_vals, values, sizeof(double) * (size_t)P.nnz_a, cudaMemcpyDeviceToDevice, h->hs));
        else if ((st = staged_h2d(h, h->d_vals, values, 0, sizeof(double) * (size_t)P.nnz_a, 1)))
            return st;
    }
    Marks mk{h, false};
    CU(cudaEventRecord(h->ev_t0, h->hs));
    if (fp64) enqueue_factorization<double>(h, false, mk, (int)precision, part);
    else enqueue_factorization<float>(h, true, mk, (int)precision, part);
    CU(cudaGetLastError());
    CU(cudaEventRecord(h->ev_t1, h->hs));
    int64_t bad = 0;
    unsigned long long nrepl = 0, abits = 0, nneg = 0;
    int fqerr = 0;
    CU(cudaMemcpyAsync(&bad, h->d_err, sizeof(bad), cudaMemcpyDeviceToHost, h->hs));
    CU(cudaMemcpyAsync(&nrepl, h->d_nrepl, sizeof(nrepl), cudaMemcpyDeviceToHost, h->hs));
    CU(cudaMemcpyAsync(&abits, h->d_anorm, sizeof(abits), cudaMemcpyDeviceToHost, h->hs));
    CU(cudaMemcpyAsync(&nneg, h->d_nneg, sizeof(nneg), cudaMemcpyDeviceToHost, h->hs));
    CU(cudaMemcpyAsync(&fqerr, h->d_fq_state + 2 * (size_t)P.npanels + h->fq_nchunks + 1, sizeof(int),
                       cudaMemcpyDeviceToHost, h->hs));
    CU(cudaStreamSynchronize(h->hs));
    h->part_done = part >= 0 ? 1 : 2;
    if (fqerr)
        return fail(h, SPX_ERR_TIMEOUT, fqerr == 2 ? "the factorization queue's tensor-core pipeline gave up waiting"
                                                   : "the factorization queue gave up waiting on a task counter");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1);
    std::memcpy(&h->anorm, &abits, 8);
    h->info.factor_ms = ms;
    h->info.precision = precision;
    h->info.npivot_repl = (int64_t)nrepl;
    h->info.npivot_neg = P.method == SPX_LDLT ? (int64_t)nneg : 0;
    h->info.bad_col = (bad == LLONG_MAX) ? -1 : bad;
    h->precision = precision;
    if (bad == -1)
        return fail(h, SPX_ERR_TIMEOUT, "a diagonal block's warps gave up waiting on each other");
    if (bad != LLONG_MAX)
        return fail(h, P.method == SPX_LLT ? SPX_ERR_NOT_SPD : SPX_ERR_ZERO_PIVOT,
                    "pivot failure at permuted column " + std::to_string(bad));
    h->factored = part < 0;
    return SPX_OK;
}

// pack (get) or unpack (set) the values, and with_inverses the inverse blocks, of a part
static spx_status part_copy(spx_handle h, int32_t part, int32_t with_inverses, void *buf, int dir, void *cuda_stream)
{
    if (!h) return fail(nullptr, SPX_ERR_ARG, "handle is NULL");
    if (h->part_nranks < 1) return fail(h, SPX_ERR_STATE, "no partition");
    if (part < -1 || part >= h->part_nranks) return fail(h, SPX_ERR_ARG, "part outside [-1, nranks)");
    if (!buf) return fail(h, SPX_ERR_ARG, "buf is NULL");
    if (h->factor_prec_alloc < 0) return fail(h, SPX_ERR_STATE, "no factor storage (factorize a part first)");
    spx_status st = ensure_part_device(h);
    if (st != SPX_OK) return st;
    const spx_handle_s::Part &pt = h->parts[part >= 0 ? part : h->part_nranks];
    fence_from(h, cuda_stream);
    if (h->factor_prec_alloc == 1) {
        spx::launch_pack_ranges<double>(pt.d_ranges, pt.nr, (double *)h->d_L, (double *)buf, dir, h->hs);
        if (with_inverses)
            spx::launch_pack_ranges<double>(pt.d_ranges + 3 * (size_t)pt.nr, pt.nr, (double *)h->d_Dinv, (double *)buf,
                                            dir, h->hs);
    } else {
        spx::launch_pack_ranges<float>(pt.d_ranges, pt.nr, (float *)h->d_L, (float *)buf, dir, h->hs);
        if (with_inverses)
            spx::launch_pack_ranges<float>(pt.d_ranges + 3 * (size_t)pt.nr, pt.nr, (float *)h->d_Dinv, (float *)buf,
                                           dir, h->hs);
    }
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->hs));
    return SPX_OK;
}

spx_status spx_part_get(spx_handle h, int32_t part, int32_t with_inverses, void *buf, void *cuda_stream)
{
    return part_copy(h, part, with_inverses, buf, 0, cuda_stream);
}

spx_status spx_part_set(spx_handle h, int32_t part, int32_t with_inverses, const void *buf, void *cuda_stream)
{
    spx_status st = part_copy(h, part, with_inverses, const_cast<void *>(buf), 1, cuda_stream);
    if (st == SPX_OK && part >= 0 && h->part_done == 2) h->factored = true;
    return st;
}

spx_status spx_solve(spx_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X,
                     int64_t ldx, int on_device, const spx_refine *refine, spx_solve_info *info,
                     void *cuda_stream)
{
    if (!h) return fail(nullptr, SPX_ERR_ARG, "handle is NULL");
    if (!h->factored) return fail(h, SPX_ERR_STATE, "spx_solve before a successful spx_factorize");
    const spx::Plan &P = h->plan;
    if (nrhs < 0 || (nrhs > 0 && (!B || !X))) return fail(h, SPX_ERR_ARG, "bad B/X/nrhs");
    if (ldb < P.n || ldx < P.n) return fail(h, SPX_ERR_ARG, "leading dimension below n");
    spx_solve_info si{};
    si.converged = 1;
    if (nrhs == 0) {
        if (info) *info = si;
        return SPX_OK;
    }
    spx_refine rf;
    spx_default_refine(&rf);
    const bool fp64 = h->precision == SPX_FP64;
    if (refine) rf = *refine;
    else if (fp64) rf.mode = 0;
    spx_status st = ensure_workspace(h, nrhs);
    if (st != SPX_OK) return st;
    fence_from(h, cuda_stream);
    const size_t n = (size_t)P.n;
    if (on_device)
        CU(cudaMemcpy2DAsync(h->d_B, n * sizeof(double), B, (size_t)ldb * sizeof(double), n * sizeof(double),
                             nrhs, cudaMemcpyDeviceToDevice, h->hs));
    else if ((st = staged_h2d(h, h->d_B, B, (size_t)ldb * sizeof(double), n * sizeof(double), (size_t)nrhs)))
        return st;
    if (h->sgraph_nrhs != nrhs || h->sgraph_prec != h->precision || !h->sgraph) {
        if ((st = capture(h, &h->sgraph, body_sweep, nrhs, fp64))) return st;
        h->sgraph_nrhs = nrhs;
        h->sgraph_prec = h->precision;
    }
    h->cnt = 0;
    int32_t qerr = 0;
    CU(cudaEventRecord(h->ev_t0, h->hs));
    CU(cudaMemcpyAsync(h->d_R, h->d_B, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, h->hs));
    CU(cudaGraphLaunch(h->sgraph, h->hs));
    h->cnt += h->sweep_launches;
    CU(cudaMemcpyAsync(h->d_X, h->d_D, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, h->hs));
    double berr = 0.0;
    if (rf.mode != 0 || info) {
        if ((st = residual(h, nrhs, &berr))) return st;
        while (rf.mode != 0 && !(berr <= rf.tol) && si.iters < rf.max_iter) {
            CU(cudaGraphLaunch(h->sgraph, h->hs));
            spx::launch_axpy_cols(P.n, nrhs, h->d_D, h->d_X, P.n, h->hs);
            h->cnt += h->sweep_launches + 1;
            si.iters++;
            double e;
            if ((st = residual(h, nrhs, &e))) return st;
            const bool stalled = !(e <= 0.5 * berr);   // plain refinement stopped contracting
            berr = e;
            if (stalled) break;
        }
        if (rf.mode == 2 && !(berr <= rf.tol)) {
            int git = 0;
            if ((st = fgmres(h, nrhs, rf, &berr, &git))) return st;
            si.gmres_iters = git;
        }
        si.backward_error = berr;
        si.converged = (rf.mode == 0) ? 1 : (berr <= rf.tol);
    }
    CU(cudaEventRecord(h->ev_t1, h->hs));
    if (on_device)
        CU(cudaMemcpy2DAsync(X, (size_t)ldx * sizeof(double), h->d_X, n * sizeof(double), n * sizeof(double),
                             nrhs, cudaMemcpyDeviceToDevice, h->hs));
    else if ((st = staged_d2h(h, X, (size_t)ldx * sizeof(double), h->d_X, n * sizeof(double), (size_t)nrhs)))
        return st;
    CU(cudaMemcpyAsync(&qerr, h->d_qerr, sizeof(int32_t), cudaMemcpyDeviceToHost, h->hs));
    CU(cudaStreamSynchronize(h->hs));
    if (qerr) {
        CU(cudaMemset(h->d_qerr, 0, sizeof(int32_t)));
        return fail(h, SPX_ERR_TIMEOUT, "a triangular sweep gave up waiting on its work queue");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1);
    h->info.solve_ms = ms;
    h->info.launches_solve = h->cnt;
    if (info) *info = si;
    if (rf.mode != 0 && !si.converged)
        return fail(h, SPX_ERR_NOT_CONVERGED, "refinement stopped at backward error " + std::to_string(berr));
    return SPX_OK;
}

spx_status spx_get_info(spx_handle h, spx_info *info)
{
    if (!h || !info) return fail(h, SPX_ERR_ARG, "NULL argument");
    h->info.noalloc_timeout = h->h_noalloc_err ? *(volatile int32_t *)h->h_noalloc_err : 0;
    *info = h->info;
    return SPX_OK;
}

spx_status spx_roofline_model(spx_handle h, spx_precision precision, const double *peaks, double *model_ms)
{
    if (!h || !peaks || !model_ms) return fail(h, SPX_ERR_ARG, "NULL argument");
    if (precision < SPX_FP64 || precision > SPX_BF16) return fail(h, SPX_ERR_ARG, "unknown precision");
    for (int i = 0; i < 4; ++i)
        if (!(peaks[i] > 0.0)) return fail(h, SPX_ERR_ARG, "peaks must be positive");
    const spx::Plan &P = h->plan;
    const bool fp64 = precision == SPX_FP64;
    const bool lu = P.method == SPX_LU;
    const double e = fp64 ? 8.0 : 4.0;
    const double bw = peaks[0] * 1e9, f64 = peaks[1] * 1e9, f32 = peaks[2] * 1e9, tc = peaks[3] * 1e9;
    const double simt = fp64 ? f64 : f32;
    const bool tcm = uses_tensor_cores(P.method, precision);
    const double eop = precision == SPX_BF16 ? 2.0 : (precision == SPX_FP32 ? 8.0 : 4.0);
    const int qlev = P.method == SPX_LU ? P.nlevels
                     : queue_policy_level(P, h->queue_panels, precision);
    double ms[SPX_K_CLASSES] = {0, 0, 0, 0, 0, 0};
    const double nfac = lu ? 2.0 : 1.0;
    ms[SPX_K_ASSEMBLE] = ((double)P.nnz_a * (16.0 + e * nfac) + (double)P.pval[P.npanels] * e * nfac) / bw;
    visit_work(P, tcm, [&](int cls, int lvl, double flops, double el, double el_op, double el_acc) {
        const double peak = cls == SPX_K_DIAG ? f64 : (cls == SPX_K_UPDATE_TC ? tc : simt);
        const double bytes = el * e + el_op * eop + el_acc * 4.0;
        ms[lvl >= qlev ? (int)SPX_K_QUEUE : cls] += std::max(flops / peak, bytes / bw);
    });
    for (int c = 0; c < SPX_K_CLASSES; ++c) model_ms[c] = ms[c] * 1e3;
    return SPX_OK;
}

spx_status spx_set_wait_limit(spx_handle h, int64_t polls)
{
    if (!h) return fail(nullptr, SPX_ERR_ARG, "handle is NULL");
    if (polls < 0 || polls > (int64_t)UINT32_MAX) return fail(h, SPX_ERR_ARG, "polls outside [0, 2^32)");
    h->spin_limit = polls == 0 ? spx::kDefaultSpinLimit : (uint32_t)polls;
    if (h->fgraph) {   // the captured factorization queue carries the old limit
        cudaGraphExecDestroy(h->fgraph);
        h->fgraph = nullptr;
        h->fgraph_prec = -1;
    }
    if (h->sgraph) {   // the captured sweeps carry the old limit
        cudaGraphExecDestroy(h->sgraph);
        h->sgraph = nullptr;
        h->sgraph_nrhs = -1;
    }
    return SPX_OK;
}

spx_status spx_get_perm(spx_handle h, int64_t *perm)
{
    if (!h || !perm) return fail(h, SPX_ERR_ARG, "NULL argument");
    std::memcpy(perm, h->plan.perm.data(), sizeof(int64_t) * (size_t)h->plan.n);
    return SPX_OK;
}

spx_status spx_get_factor(spx_handle h, const int64_t *Lp, const int32_t *Li, double *Lx, double *Ut)
{
    if (!h || !Lp || !Li || !Lx) return fail(h, SPX_ERR_ARG, "NULL argument");
    if (!h->factored) return fail(h, SPX_ERR_STATE, "no factor");
    const spx::Plan &P = h->plan;
    const bool lu = P.method == SPX_LU;
    if (lu && !Ut) return fail(h, SPX_ERR_ARG, "LU needs Ut");
    const size_t elems = (size_t)P.pval[P.npanels];
    std::vector<double> hl(elems), hu(lu ? elems : 0);
    auto fetch = [&](const void *src, std::vector<double> &dst) -> spx_status {
        if (h->precision == SPX_FP64) {
            CU(cudaMemcpy(dst.data(), src, elems * sizeof(double), cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> tmp(elems);
            CU(cudaMemcpy(tmp.data(), src, elems * sizeof(float), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < elems; ++i) dst[i] = tmp[i];
        }
        return SPX_OK;
    };
    spx_status st;
    if ((st = fetch(h->d_L, hl))) return st;
    if (lu && (st = fetch(h->d_U, hu))) return st;
    auto pos = [&](int32_t p, int64_t r) -> int64_t {
        const int32_t *b = P.rows.data() + P.prow[p], *e = P.rows.data() + P.prow[p + 1];
        const int32_t *it = std::lower_bound(b, e, (int32_t)r);
        return (it != e && *it == r) ? (int64_t)(it - b) : -1;
    };
    for (int64_t j = 0; j < P.n; ++j) {
        const int32_t pj = P.col2panel[j];
        const int64_t cj = j - P.pfcol[pj];
        const int64_t hj = P.ph[pj];
        for (int64_t q = Lp[j]; q < Lp[j + 1]; ++q) {
            const int64_t i = Li[q];
            if (i < j || i >= P.n) return fail(h, SPX_ERR_ARG, "pattern entry above the diagonal");
            const int64_t r = pos(pj, i);
            if (r < 0) return fail(h, SPX_ERR_ARG, "pattern entry outside the panel structure");
            const int64_t off = P.pval[pj] + cj * hj + r;
            if (!lu) {
                Lx[q] = hl[off];
                continue;
            }
            if (i == j) {
                Lx[q] = 1.0;
                Ut[q] = hl[off];
                continue;
            }
            Lx[q] = hl[off];
            // U(j, i), i > j: inside j's diagonal block -> L panel (row j, col i); else U^T panel
            if (i < P.pfcol[pj] + P.pw[pj]) {
                Ut[q] = hl[P.pval[pj] + (i - P.pfcol[pj]) * hj + cj];
            } else {
                Ut[q] = hu[off];
            }
        }
    }
    return SPX_OK;
}

spx_status spx_get_panels(spx_handle h, int64_t *first_col, int32_t *width, int32_t *height,
                          int32_t *level, int32_t *parent)
{
    if (!h) return fail(nullptr, SPX_ERR_ARG, "handle is NULL");
    const spx::Plan &P = h->plan;
    const size_t np = (size_t)P.npanels;
    if (first_col) std::memcpy(first_col, P.pfcol.data(), np * sizeof(int64_t));
    if (width) std::memcpy(width, P.pw.data(), np * sizeof(int32_t));
    if (height) std::memcpy(height, P.ph.data(), np * sizeof(int32_t));
    if (level) std::memcpy(level, P.plevel.data(), np * sizeof(int32_t));
    if (parent) std::memcpy(parent, P.pparent.data(), np * sizeof(int32_t));
    return SPX_OK;
}

spx_status spx_set_profiling(spx_handle h, int on)
{
    if (!h) return fail(nullptr, SPX_ERR_ARG, "handle is NULL");
    h->profiling = on != 0;
    return SPX_OK;
}

spx_status spx_get_kernel_stats(spx_handle h, spx_kernel_stats *out)
{
    if (!h || !out) return fail(h, SPX_ERR_ARG, "NULL argument");
    *out = h->kstats;
    return SPX_OK;
}

spx_status spx_solve_noalloc(spx_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X,
                             int64_t ldx, void *cuda_stream)
{
    if (!h) return fail(nullptr, SPX_ERR_ARG, "handle is NULL");
    if (!h->factored) return fail(h, SPX_ERR_STATE, "spx_solve_noalloc before a successful spx_factorize");
    const spx::Plan &P = h->plan;
    if (nrhs < 0 || (nrhs > 0 && (!B || !X))) return fail(h, SPX_ERR_ARG, "bad B/X/nrhs");
    if (ldb < P.n || ldx < P.n) return fail(h, SPX_ERR_ARG, "leading dimension below n");
    if (nrhs == 0) return SPX_OK;
    const size_t esz = h->precision == SPX_FP64 ? sizeof(double) : sizeof(float);
    const size_t need = (size_t)4 * (size_t)P.n * (size_t)nrhs * esz +
                        sizeof(int32_t) * ((size_t)4 * P.npanels + 3);
    if (need > kStaticScratchBytes)
        return fail(h, SPX_ERR_ARG,
                    "4 * n * nrhs sweep elements, the sweep counters and the error word (" + std::to_string(need) +
                        " bytes) exceed the 16 MiB static scratch of spx_solve_noalloc");
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != h->device) return fail(h, SPX_ERR_STATE, "current device is not the handle's device");
    void *scratch = nullptr;
    spx_status st = static_scratch_address(h, dev, &scratch);
    if (st != SPX_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (h->precision == SPX_FP64)
        enqueue_sweep_noalloc<double>(h, nrhs, B, ldb, X, ldx, (double *)scratch, s);
    else
        enqueue_sweep_noalloc<float>(h, nrhs, B, ldb, X, ldx, (float *)scratch, s);
    CU(cudaGetLastError());
    return SPX_OK;
}

// ---------------------------------------------------------------------------
// log-determinant, selected inverse and the adjoints of solve / logdet
// ---------------------------------------------------------------------------
namespace {

spx_status ensure_scalar(spx_handle h)
{
    if (h->d_scalar) return SPX_OK;
    return dalloc(h, &h->d_scalar, 4);
}

// grad workspace of len doubles (host-buffer calls)
spx_status ensure_gtmp(spx_handle h, int64_t len)
{
    if (h->gtmp_len >= len) return SPX_OK;
    dfree(h, h->d_gtmp);
    h->d_gtmp = nullptr;
    h->gtmp_len = 0;
    spx_status st = dalloc(h, &h->d_gtmp, (size_t)len);
    if (st == SPX_OK) h->gtmp_len = len;
    return st;
}

// offset in the panel storage of the lower entry (max(pi,pj), min(pi,pj))
// of every input entry, in the input's CSC order
spx_status build_zmap(spx_handle h, const int64_t *colptr_unused)
{
    (void)colptr_unused;
    if (h->d_zmap) return SPX_OK;
    const spx::Plan &P = h->plan;
    std::vector<int64_t> zmap((size_t)P.nnz_a, 0);
    for (int64_t i = 0; i < P.n; ++i)
        for (int64_t e = P.csr_ptr[i]; e < P.csr_ptr[i + 1]; ++e) {
            const int64_t j = P.csr_col[e];
            const int64_t a = std::max(P.iperm[i], P.iperm[j]), b = std::min(P.iperm[i], P.iperm[j]);
            const int32_t pb = P.col2panel[b];
            const int32_t *rb = P.rows.data() + P.prow[pb], *re = P.rows.data() + P.prow[pb + 1];
            const int32_t *it = std::lower_bound(rb, re, (int32_t)a);
            if (it == re || *it != a) return fail(h, SPX_ERR_ARG, "input entry outside the factor structure");
            zmap[(size_t)P.csr_src[e]] = P.pval[pb] + (b - P.pfcol[pb]) * P.ph[pb] + (it - rb);
        }
    return upload(h, &h->d_zmap, zmap);
}

}  // namespace

spx_status spx_logdet(spx_handle h, double *logdet)
{
    if (!h || !logdet) return fail(h, SPX_ERR_ARG, "NULL argument");
    if (!h->factored) return fail(h, SPX_ERR_STATE, "no factor");
    if (h->plan.method != SPX_LLT) return fail(h, SPX_ERR_ARG, "log det of a Cholesky factor only");
    spx_status st;
    if ((st = ensure_scalar(h))) return st;
    if (h->precision == SPX_FP64) spx::launch_logdet<double>(h->dp, (const double *)h->d_L, h->d_scalar, h->hs);
    else spx::launch_logdet<float>(h->dp, (const float *)h->d_L, h->d_scalar, h->hs);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(logdet, h->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, h->hs));
    CU(cudaStreamSynchronize(h->hs));
    return SPX_OK;
}

spx_status spx_selected_inverse(spx_handle h, void *cuda_stream)
{
    if (!h) return fail(nullptr, SPX_ERR_ARG, "handle is NULL");
    if (!h->factored) return fail(h, SPX_ERR_STATE, "no factor");
    if (h->plan.method != SPX_LLT || h->precision != SPX_FP64)
        return fail(h, SPX_ERR_ARG, "the selected inverse needs an FP64 Cholesky factor");
    if (h->zready) return SPX_OK;
    const spx::Plan &P = h->plan;
    const size_t elems = (size_t)P.pval[P.npanels];
    spx_status st;
    if (!h->d_Zsel) {
        if ((st = dalloc(h, &h->d_Zsel, elems)) || (st = dalloc(h, &h->d_Lh, elems))) return st;
        // the task whose facing rows hold each off-diagonal row of a panel
        std::vector<int32_t> row_task((size_t)P.prow[P.npanels], -1);
        for (size_t t = 0; t < P.tasks.size(); ++t) {
            const spx::Task &tk = P.tasks[t];
            for (int32_t r = tk.r0; r < tk.r1; ++r) row_task[(size_t)P.prow[tk.src] + r] = (int32_t)t;
        }
        for (int32_t q = 0; q < P.npanels; ++q)
            for (int32_t r = P.pw[q]; r < P.ph[q]; ++r)
                if (row_task[(size_t)P.prow[q] + r] < 0) return fail(h, SPX_ERR_ARG, "row without an update task");
        if ((st = upload(h, &h->d_row_task, row_task))) return st;
    }
    fence_from(h, cuda_stream);
    const int wmax = *std::max_element(h->lvl_wmax.begin(), h->lvl_wmax.end());
    if (wmax > 64) return fail(h, SPX_ERR_ARG, "the selected inverse takes panels up to 64 wide (max_width <= 64)");
    CU(cudaMemcpyAsync(h->d_Lh, h->d_L, elems * sizeof(double), cudaMemcpyDeviceToDevice, h->hs));
    CU(cudaMemsetAsync(h->d_Zsel, 0, elems * sizeof(double), h->hs));   // split-K partial sums add into it
    spx::launch_trsm<double>(h->dp, h->d_chunks, (int)h->chunk_ptr[P.nlevels], wmax,
                             (const double *)h->d_Dinv, h->d_Lh, spx::TRSM_RIGHT_LINV, nullptr, nullptr, 0, 0,
                             h->hs);
    // split-K so that a level keeps about two CTAs per SM busy near the root
    int nsm = 0;
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    const int want = 2 * nsm;
    for (int32_t l = P.nlevels - 1; l >= 0; --l) {
        const int nch = (int)(h->chunk_ptr[l + 1] - h->chunk_ptr[l]);
        const int npl = P.level_ptr[l + 1] - P.level_ptr[l];
        int max_rchunks = 1;   // most 16-row chunks of R in a panel of the level
        for (int32_t q = P.level_ptr[l]; q < P.level_ptr[l + 1]; ++q) {
            const int32_t k = P.level_panels[q];
            max_rchunks = std::max(max_rchunks, (P.ph[k] - P.pw[k] + 15) / 16);
        }
        const int so = nch > 0 ? std::min(max_rchunks, std::max(1, (want + nch - 1) / nch)) : 1;
        const int sd = std::min((max_rchunks + 1) / 2, std::max(1, (want + npl - 1) / std::max(npl, 1)));
        spx::launch_selinv_off(h->dp, h->d_chunks + h->chunk_ptr[l], nch, so, h->d_row_task, h->d_tasks,
                               h->d_Lh, h->d_Zsel, h->hs);
        spx::launch_selinv_diag(h->dp, h->d_level_panels + P.level_ptr[l], npl, sd, h->lvl_wmax[l],
                                (const double *)h->d_Dinv, h->d_Lh, h->d_Zsel, h->hs);
    }
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->hs));
    h->zready = true;
    return SPX_OK;
}

spx_status spx_get_selected_inverse(spx_handle h, const int64_t *Lp, const int32_t *Li, double *Zx)
{
    if (!h || !Lp || !Li || !Zx) return fail(h, SPX_ERR_ARG, "NULL argument");
    if (!h->zready) return fail(h, SPX_ERR_STATE, "no selected inverse (call spx_selected_inverse)");
    const spx::Plan &P = h->plan;
    const size_t elems = (size_t)P.pval[P.npanels];
    std::vector<double> hz(elems);
    CU(cudaMemcpy(hz.data(), h->d_Zsel, elems * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t j = 0; j < P.n; ++j) {
        const int32_t pj = P.col2panel[j];
        const int32_t *rb = P.rows.data() + P.prow[pj], *re = P.rows.data() + P.prow[pj + 1];
        for (int64_t q = Lp[j]; q < Lp[j + 1]; ++q) {
            const int64_t i = Li[q];
            if (i < j || i >= P.n) return fail(h, SPX_ERR_ARG, "pattern entry above the diagonal");
            const int32_t *it = std::lower_bound(rb, re, (int32_t)i);
            if (it == re || *it != i) return fail(h, SPX_ERR_ARG, "pattern entry outside the panel structure");
            Zx[q] = hz[P.pval[pj] + (j - P.pfcol[pj]) * P.ph[pj] + (it - rb)];
        }
    }
    return SPX_OK;
}

spx_status spx_logdet_grad(spx_handle h, double *grad, int on_device, void *cuda_stream)
{
    if (!h || !grad) return fail(h, SPX_ERR_ARG, "NULL argument");
    spx_status st;
    if (!h->zready && (st = spx_selected_inverse(h, cuda_stream))) return st;
    if ((st = build_zmap(h, nullptr))) return st;
    const int64_t nnz = h->plan.nnz_a;
    double *dst = grad;
    if (!on_device) {
        if ((st = ensure_gtmp(h, nnz))) return st;
        dst = h->d_gtmp;
    }
    fence_from(h, cuda_stream);
    spx::launch_gather(nnz, h->d_zmap, h->d_Zsel, dst, h->hs);
    CU(cudaGetLastError());
    if (!on_device) CU(cudaMemcpyAsync(grad, dst, sizeof(double) * nnz, cudaMemcpyDeviceToHost, h->hs));
    CU(cudaStreamSynchronize(h->hs));
    return SPX_OK;
}

spx_status spx_solve_grad(spx_handle h, int32_t nrhs, const double *Lam, int64_t ldl, const double *X,
                          int64_t ldx, double *grad, int on_device, void *cuda_stream)
{
    if (!h || !Lam || !X || !grad) return fail(h, SPX_ERR_ARG, "NULL argument");
    const spx::Plan &P = h->plan;
    if (nrhs < 1 || ldl < P.n || ldx < P.n) return fail(h, SPX_ERR_ARG, "bad nrhs or leading dimension");
    spx_status st = ensure_device(h);
    if (st != SPX_OK) return st;
    fence_from(h, cuda_stream);
    const double *dl = Lam, *dx = X;
    double *dg = grad;
    if (!on_device) {
        // host buffers: three device vectors of `need` doubles (Lam, X, grad)
        const int64_t need = std::max<int64_t>((int64_t)P.n * nrhs, P.nnz_a);
        if (!h->d_lam || h->gtmp_len < need) {
            dfree(h, h->d_lam);
            dfree(h, h->d_xg);
            dfree(h, h->d_gtmp);
            h->d_lam = h->d_xg = h->d_gtmp = nullptr;
            h->gtmp_len = 0;
            if ((st = dalloc(h, &h->d_lam, (size_t)need)) || (st = dalloc(h, &h->d_xg, (size_t)need)) ||
                (st = dalloc(h, &h->d_gtmp, (size_t)need)))
                return st;
            h->gtmp_len = need;
        }
        CU(cudaMemcpy2DAsync(h->d_lam, P.n * sizeof(double), Lam, ldl * sizeof(double), P.n * sizeof(double), nrhs,
                             cudaMemcpyHostToDevice, h->hs));
        CU(cudaMemcpy2DAsync(h->d_xg, P.n * sizeof(double), X, ldx * sizeof(double), P.n * sizeof(double), nrhs,
                             cudaMemcpyHostToDevice, h->hs));
        dl = h->d_lam;
        dx = h->d_xg;
        ldl = ldx = P.n;
        dg = h->d_gtmp;
    }
    spx::launch_solve_grad(P.n, nrhs, h->d_csr_ptr, h->d_csr_col, h->d_csr_src, dl, ldl, dx, ldx, dg, h->hs);
    CU(cudaGetLastError());
    if (!on_device) CU(cudaMemcpyAsync(grad, dg, sizeof(double) * P.nnz_a, cudaMemcpyDeviceToHost, h->hs));
    CU(cudaStreamSynchronize(h->hs));
    return SPX_OK;
}

const char *spx_last_error(spx_handle h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

void spx_free(spx_handle h)
{
    if (!h) return;
    if (h->fgraph) cudaGraphExecDestroy(h->fgraph);
    if (h->sgraph) cudaGraphExecDestroy(h->sgraph);
    for (void *p : h->allocs) cudaFree(p);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->ev_fence) cudaEventDestroy(h->ev_fence);
    if (h->ev_t0) cudaEventDestroy(h->ev_t0);
    if (h->ev_t1) cudaEventDestroy(h->ev_t1);
    if (h->hs) cudaStreamDestroy(h->hs);
    for (int k = 0; k < 2; ++k) {
        if (h->aux[k]) cudaStreamDestroy(h->aux[k]);
        if (h->ev_join[k]) cudaEventDestroy(h->ev_join[k]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_trsm) cudaEventDestroy(h->ev_trsm);
    for (int k = 0; k < 2; ++k) {
        if (h->fstream[k]) cudaStreamDestroy(h->fstream[k]);
        if (h->ev_far[k]) cudaEventDestroy(h->ev_far[k]);
        if (h->ev_near[k]) cudaEventDestroy(h->ev_near[k]);
    }
    if (h->h_noalloc_err) cudaFreeHost(h->h_noalloc_err);
    for (int b = 0; b < 2; ++b) {
        if (h->h_stage[b]) cudaFreeHost(h->h_stage[b]);
        if (h->ev_stage[b]) cudaEventDestroy(h->ev_stage[b]);
    }
    delete h;
}

}  // extern "C"
