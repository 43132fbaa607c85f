// fqueue_ldlt.cu -- instantiations of the factorization queue for the
// single-precision LDL^T factor (TF32 and BF16 tensor-core updates from the
// D L^T operand copy, or FP32 updates on the CUDA cores); see fqueue.cuh.
#include "fqueue.cuh"

namespace spx {
template void fq_launch<float, true, 3>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
template void fq_launch<float, true, 4>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
template void fq_launch<float, true, -1>(const FqArgs<float> &, const void *, const void *, cudaStream_t);
template int fq_grid<float, true, 3>();
template int fq_grid<float, true, 4>();
template int fq_grid<float, true, -1>();
}  // namespace spx
