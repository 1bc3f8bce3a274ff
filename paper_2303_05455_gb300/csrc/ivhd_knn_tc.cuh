// ivhd_knn_tc.cuh -- kNN graph build on the tensor cores (see ivhd_knn_tc.cu)
// and the exact CUDA-core kernel it falls back to (ivhd_knn.cu).
#pragma once

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

// Tensor-core build; synchronises the stream.  IVHD_ERR_TIMEOUT if a bounded
// wait of the kernel expired.
ivhd_status knn_tc_build(const KnnProblem& P, int32_t* out_knn, cudaStream_t s,
                         KnnTcStats* stats);

// Exact FP32 kNN rows (the CUDA-core kernel) for the *n_rows query rows listed
// in rows (device count and list); the other rows of out_knn are left untouched.
cudaError_t knn_exact_rows_f32(const KnnProblem& P, const int32_t* rows, const int32_t* n_rows,
                               int32_t* out_knn, cudaStream_t s);

}  // namespace ivhd
