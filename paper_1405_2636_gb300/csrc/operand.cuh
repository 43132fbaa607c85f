// operand.cuh -- the K-major operand copy of the tensor-core updates: each
// panel row rounded to the MMA's input type.  Written by the panel TRSM
// during the factorization and by the kernel-study staging (study.cu), so
// that both hand the tcgen05 update the same bits.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace spx {

// Round to TF32 (10 explicit mantissa bits), to nearest with ties away from zero.
__device__ __forceinline__ float round_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Element o of the operand copy from the panel value v (and, for LDL^T, the
// D L^T value wv):
//   op_kind 0: opc = tf32(v)
//   op_kind 1: opc = bf16(v)                       (round to nearest even)
//   op_kind 2: opc = hi = tf32(v), opc_lo = tf32(v - hi)   (split TF32)
//   op_kind 3: opc = tf32(v), opc_lo = tf32(wv)     (LDL^T, TF32)
//   op_kind 4: opc = bf16(v), opc_lo = bf16(wv)     (LDL^T, BF16)
__device__ __forceinline__ void put_operand(void *opc, void *opc_lo, int64_t o, int op_kind, float v,
                                            float wv)
{
    if (op_kind == 1 || op_kind == 4) {
        reinterpret_cast<__nv_bfloat16 *>(opc)[o] = __float2bfloat16(v);
        if (op_kind == 4) reinterpret_cast<__nv_bfloat16 *>(opc_lo)[o] = __float2bfloat16(wv);
    } else {
        const float hi = round_tf32(v);
        reinterpret_cast<float *>(opc)[o] = hi;
        if (op_kind == 2) reinterpret_cast<float *>(opc_lo)[o] = round_tf32(v - hi);
        else if (op_kind == 3) reinterpret_cast<float *>(opc_lo)[o] = round_tf32(wv);
    }
}

}  // namespace spx
