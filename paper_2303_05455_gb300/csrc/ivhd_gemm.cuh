// ivhd_gemm.cuh -- tcgen05 BF16 GEMM with fused epilogues (see ivhd_gemm.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ivhd {

enum GemmEpKind {
  kEpStoreF32 = 0,   // out_f32 = C
  kEpBiasGelu = 1,   // out_f32 = C + bias (pre-activation), out_bf16 = GELU(C + bias)
  kEpGeluGrad = 2    // out_bf16 = C * GELU'(aux_f32)
};

struct GemmEpilogue {
  int kind;
  int64_t ld_out;  // row stride (elements) of out_f32 / out_bf16 / aux_f32
  float* out_f32;
  __nv_bfloat16* out_bf16;
  const float* bias;
  const float* aux_f32;
  int64_t split_stride;  // split-K: slice z writes out_f32 + z * split_stride
  // optional (BF16 kinds): the same BF16 values transposed, out_bf16_t[col * ld_t + row]
  __nv_bfloat16* out_bf16_t = nullptr;
  int64_t ld_t = 0;
};

// C = A B^T for BF16 A (M x K, row stride lda) and B (N x K, row stride ldb),
// FP32 accumulation on the tensor cores, epilogue ep.  K % 8 == 0, 16-byte
// aligned operands.  err receives a non-zero flag if a bounded wait expired.
// splits > 1 (kEpStoreF32 only) divides the k-tiles among that many CTAs per
// output tile; slice z writes its partial product at out_f32 + z * split_stride
// and sum_slices adds them in order.
cudaError_t gemm_bf16_tn(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb,
                         int M, int N, int K, const GemmEpilogue& ep, int32_t* err,
                         cudaStream_t s, int splits = 1);
cudaError_t sum_slices(const float* part, int64_t n, int64_t stride, int splits, float* out,
                       cudaStream_t s);

}  // namespace ivhd
