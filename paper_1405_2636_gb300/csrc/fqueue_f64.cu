// fqueue_f64.cu -- instantiations of the factorization queue for the FP64
// factor (Cholesky and LDL^T, updates on the CUDA cores), and the dispatch
// from the runtime (storage type, method, operand kind) to the compiled
// variants; see fqueue.cuh.
#include "fqueue.cuh"

namespace spx {

extern template void fq_launch<float, false, 0>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
extern template void fq_launch<float, false, 1>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
extern template void fq_launch<float, false, 2>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
extern template void fq_launch<float, true, 3>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
extern template void fq_launch<float, true, 4>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
extern template void fq_launch<float, true, -1>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
extern template int fq_grid<float, false, 0>();
extern template int fq_grid<float, false, 1>();
extern template int fq_grid<float, false, 2>();
extern template int fq_grid<float, true, 3>();
extern template int fq_grid<float, true, 4>();
extern template int fq_grid<float, true, -1>();

template <typename T>
static FqArgs<T> fq_args(const DevPlan &p, const FactorQueue &q, const DevTask *tasks, const RowChunk *chunks,
                         const UpdTile *tiles, const TcTile *tctiles, T *L, T *Dinv, T *W, const double *tau,
                         int64_t *err_col, unsigned long long *nrepl, unsigned long long *nneg, int ldlt,
                         void *opc, void *opc_lo, int kpad, int op_kind)
{
    FqArgs<T> a;
    a.p = p;
    a.q = q;
    a.tasks = tasks;
    a.chunks = chunks;
    a.tiles = tiles;
    a.tctiles = tctiles;
    a.L = L;
    a.Dinv = Dinv;
    a.W = W;
    a.tau = tau;
    a.err_col = err_col;
    a.nrepl = nrepl;
    a.nneg = nneg;
    a.opc = opc;
    a.opc_lo = opc_lo;
    a.kpad = kpad;
    a.op_kind = op_kind;
    a.trsm_mode = ldlt ? TRSM_LDLT : TRSM_LLT;
    return a;
}

template <>
void launch_factor_queue<double>(const DevPlan &p, const FactorQueue &q, const DevTask *tasks, const RowChunk *chunks,
                                 const UpdTile *tiles, const TcTile *tctiles, double *L, double *Dinv, double *W,
                                 const double *tau, int64_t *err_col, unsigned long long *nrepl,
                                 unsigned long long *nneg, int ldlt, int tc_kind, const void *tmap,
                                 const void *tmap_lo, void *opc, void *opc_lo, int kpad, int op_kind, cudaStream_t s)
{
    (void)tc_kind;
    const FqArgs<double> a = fq_args<double>(p, q, tasks, chunks, tiles, tctiles, L, Dinv, W, tau, err_col, nrepl,
                                             nneg, ldlt, nullptr, nullptr, 0, 0);
    if (ldlt) fq_launch<double, true, -1>(a, tmap, tmap_lo, s);
    else fq_launch<double, false, -1>(a, tmap, tmap_lo, s);
}

template <>
void launch_factor_queue<float>(const DevPlan &p, const FactorQueue &q, const DevTask *tasks, const RowChunk *chunks,
                                const UpdTile *tiles, const TcTile *tctiles, float *L, float *Dinv, float *W,
                                const double *tau, int64_t *err_col, unsigned long long *nrepl,
                                unsigned long long *nneg, int ldlt, int tc_kind, const void *tmap,
                                const void *tmap_lo, void *opc, void *opc_lo, int kpad, int op_kind, cudaStream_t s)
{
    const FqArgs<float> a = fq_args<float>(p, q, tasks, chunks, tiles, tctiles, L, Dinv, W, tau, err_col, nrepl,
                                           nneg, ldlt, opc, opc_lo, kpad, op_kind);
    if (ldlt) {
        if (tc_kind == 3) fq_launch<float, true, 3>(a, tmap, tmap_lo, s);
        else if (tc_kind == 4) fq_launch<float, true, 4>(a, tmap, tmap_lo, s);
        else fq_launch<float, true, -1>(a, tmap, tmap_lo, s);
    } else {
        if (tc_kind == 1) fq_launch<float, false, 1>(a, tmap, tmap_lo, s);
        else if (tc_kind == 2) fq_launch<float, false, 2>(a, tmap, tmap_lo, s);
        else fq_launch<float, false, 0>(a, tmap, tmap_lo, s);
    }
}

template <>
int factor_queue_grid<double>(int ldlt, int tc_kind)
{
    (void)tc_kind;
    return ldlt ? fq_grid<double, true, -1>() : fq_grid<double, false, -1>();
}

template <>
int factor_queue_grid<float>(int ldlt, int tc_kind)
{
    if (ldlt) return tc_kind == 3 ? fq_grid<float, true, 3>() : tc_kind == 4 ? fq_grid<float, true, 4>()
                                                                             : fq_grid<float, true, -1>();
    return tc_kind == 1 ? fq_grid<float, false, 1>() : tc_kind == 2 ? fq_grid<float, false, 2>()
                                                                    : fq_grid<float, false, 0>();
}

}  // namespace spx
