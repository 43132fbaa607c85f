// fqueue_tc.cu -- instantiations of the factorization queue for the
// single-precision Cholesky factor with tensor-core updates (TF32, BF16,
// split TF32); see fqueue.cuh.
#include "fqueue.cuh"

namespace spx {
template void fq_launch<float, false, 0>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
template void fq_launch<float, false, 1>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
template void fq_launch<float, false, 2>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
template int fq_grid<float, false, 0>();
template int fq_grid<float, false, 1>();
template int fq_grid<float, false, 2>();
}  // namespace spx
