// ivhd_knn_tc.cuh -- kNN graph build on the tensor cores (see ivhd_knn_tc.cu)
// and the exact CUDA-core kernel it falls back to (ivhd_knn.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ivhd.h"

namespace ivhd {

constexpr int kKnnList = 32;  // candidates kept per row by the tensor-core pass

struct KnnTcStats {
  int64_t fallback_rows;  // FP32 rows recomputed by the exact kernel
  float max_rel_err;      // max |approximate - exact| / (n_i + n_j) over the candidates
  float eps_coef;         // the bound used by the certificate, per unit of n_i + n_j
};

// One exact kNN problem: for each of the Mq query rows of Q, the k nearest of
// the M base rows of X (row-major, N features of `dtype`), ascending by
// (distance, index).  self: Q is X and a row never lists itself (the kNN
// graph); otherwise nothing is excluded.
struct KnnProblem {
  const void* Q;
  int64_t Mq;
  const void* X;
  int64_t M;
  int32_t dtype, N, k;
  bool self;
};

// Whether the tensor-core build handles this case (k <= kKnnList; uint8 with
// N <= 1024, so that every partial sum is exact in FP32).
bool knn_tc_supported(const KnnProblem& P);

// A base set prepared once for many queries: its BF16 operand (M x Kp, the
// layout knn_tc_build makes) and its row norms (float for float data, int32
// norms of the rows shifted by -128 for uint8).
struct KnnBase {
  const __nv_bfloat16* B;
  const void* nrm;
};
// Padded GEMM depth of the operands (K = N for uint8, 3N for float).
int knn_tc_kp(int32_t dtype, int32_t N);
// Fills B (M x knn_tc_kp) and nrm (M) for the base set X; stream-ordered.
cudaError_t knn_tc_prepare_base(const void* X, int32_t dtype, int64_t M, int32_t N,
                                __nv_bfloat16* B, void* nrm, cudaStream_t s);

// Tensor-core build; synchronises the stream.  base (queries only, may be
// null): the base set's prepared operand and norms.  IVHD_ERR_TIMEOUT if a
// bounded wait of the kernel expired.
ivhd_status knn_tc_build(const KnnProblem& P, int32_t* out_knn, cudaStream_t s,
                         KnnTcStats* stats, const KnnBase* base = nullptr);

// Exact FP32 kNN rows (the CUDA-core kernel) for the *n_rows query rows listed
// in rows (device count and list); the other rows of out_knn are left untouched.
cudaError_t knn_exact_rows_f32(const KnnProblem& P, const int32_t* rows, const int32_t* n_rows,
                               int32_t* out_knn, cudaStream_t s);

}  // namespace ivhd
