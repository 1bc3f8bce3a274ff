// ivhd_eval.cu -- embedding quality on sampled rows (Sec. 4.1).
//
// Both criteria need the nearest embedded neighbours of a query point y_q:
// one thread per query scans all M points (staged through shared memory in
// tiles) and keeps a sorted list of the best (FP32 squared distance
// dx*dx rounded, then fma(dy, dy, .); ties to the lower index).
//   Q_NX(k):  hits = |embedded kNN(q) ∩ input kNN row q|       (rank criteria)
//   cf_nn:    hits = #embedded neighbours with q's class label  (Eq. 4.4)
// Hits are integer-summed, so the result is exact and order independent.
// A sampled row id outside [0, M) is never dereferenced: its thread stays
// inactive and counts it in a second counter, and the call returns
// IVHD_ERR_INDEX.
#include "ivhd_internal.cuh"

namespace ivhd {
namespace {

constexpr int kEvalThreads = 128;
constexpr int kEvalTile = 2048;

template <bool kQnx>
__global__ void __launch_bounds__(kEvalThreads) k_lowd(const float2* __restrict__ Y, int64_t M,
                                                       const int64_t* __restrict__ rows,
                                                       int64_t nrows, int kk,
                                                       const int32_t* __restrict__ knn,
                                                       const int32_t* __restrict__ labels,
                                                       int32_t* __restrict__ out_lowd,
                                                       unsigned long long* __restrict__ hits,
                                                       unsigned long long* __restrict__ bad) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tile = reinterpret_cast<float2*>(smem);
  float* ld = reinterpret_cast<float*>(tile + kEvalTile) + threadIdx.x * kk;
  int* lj = reinterpret_cast<int*>(reinterpret_cast<float*>(tile + kEvalTile) + kEvalThreads * kk) +
            threadIdx.x * kk;
  const int64_t qi = (int64_t)blockIdx.x * kEvalThreads + threadIdx.x;
  const int64_t q = qi < nrows ? rows[qi] : 0;
  const bool in_range = q >= 0 && q < M;
  if (qi < nrows && !in_range) atomicAdd(bad, 1ull);
  const bool act = qi < nrows && in_range;
  const float2 yq = act ? Y[q] : make_float2(0.f, 0.f);
  int n = 0;
  float worst = INFINITY;
  for (int64_t t0 = 0; t0 < M; t0 += kEvalTile) {
    const int tn = (int)min((int64_t)kEvalTile, M - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < tn; e += kEvalThreads) tile[e] = Y[t0 + e];
    __syncthreads();
    if (!act) continue;
    for (int e = 0; e < tn; ++e) {
      const float2 yj = tile[e];
      const float dx = __fsub_rn(yj.x, yq.x);
      const float dy = __fsub_rn(yj.y, yq.y);
      const float d2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
      if (n == kk && !(d2 < worst)) continue;  // later candidates have larger ids
      const int j = (int)(t0 + e);
      if (j == q) continue;
      int pos = (n < kk) ? n : kk - 1;
      while (pos > 0 && (ld[pos - 1] > d2)) {
        ld[pos] = ld[pos - 1];
        lj[pos] = lj[pos - 1];
        --pos;
      }
      ld[pos] = d2;
      lj[pos] = j;
      if (n < kk) ++n;
      if (n == kk) worst = ld[kk - 1];
    }
  }
  if (!act) return;
  int h = 0;
  for (int s = 0; s < n; ++s) {
    const int j = lj[s];
    if (out_lowd) out_lowd[qi * kk + s] = j;
    if (kQnx) {
      for (int u = 0; u < kk; ++u)
        if (knn[q * kk + u] == j) {
          ++h;
          break;
        }
    } else {
      h += (labels[j] == labels[q]);
    }
  }
  atomicAdd(hits, (unsigned long long)h);
}

template <bool kQnx>
ivhd_status run_lowd(const float* Y, int64_t M, const int32_t* knn, const int32_t* labels, int kk,
                     const int64_t* rows, int64_t nrows, int32_t* out_lowd, double* out,
                     void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const size_t sm = (size_t)kEvalTile * sizeof(float2) + (size_t)kEvalThreads * kk * 8;
  unsigned long long* hits_d = nullptr;  // [0] hits, [1] rows outside [0, M)
  cudaError_t e = dev_alloc((void**)&hits_d, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return IVHD_ERR_OOM;
  e = cudaMemsetAsync(hits_d, 0, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lowd<kQnx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess) {
    const unsigned grid = (unsigned)((nrows + kEvalThreads - 1) / kEvalThreads);
    k_lowd<kQnx><<<grid, kEvalThreads, sm, s>>>((const float2*)Y, M, rows, nrows, kk, knn, labels,
                                               out_lowd, hits_d, hits_d + 1);
    e = cudaGetLastError();
  }
  unsigned long long hits[2] = {0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hits, hits_d, sizeof(hits), cudaMemcpyDeviceToHost, s);
  dev_free(hits_d, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  if (hits[1] != 0) return IVHD_ERR_INDEX;
  *out = (double)hits[0] / ((double)kk * (double)nrows);
  return IVHD_OK;
}

}  // namespace
}  // namespace ivhd

using namespace ivhd;

extern "C" ivhd_status ivhd_eval_qnx(const float* Y, int64_t M, const int32_t* knn, int32_t k,
                                     const int64_t* rows, int64_t nrows, int32_t* out_lowd,
                                     double* out_q, void* stream) {
  if (!Y || !knn || !rows || !out_q || M < 2 || nrows < 1) return IVHD_ERR_ARG;
  if (k < 1 || (int64_t)k > M - 1 || k > 128) return IVHD_ERR_ARG;
  return run_lowd<true>(Y, M, knn, nullptr, k, rows, nrows, out_lowd, out_q, stream);
}

extern "C" ivhd_status ivhd_eval_cf(const float* Y, int64_t M, const int32_t* labels, int32_t nn,
                                    const int64_t* rows, int64_t nrows, double* out_cf,
                                    void* stream) {
  if (!Y || !labels || !rows || !out_cf || M < 2 || nrows < 1) return IVHD_ERR_ARG;
  if (nn < 1 || (int64_t)nn > M - 1 || nn > 128) return IVHD_ERR_ARG;
  return run_lowd<false>(Y, M, nullptr, labels, nn, rows, nrows, nullptr, out_cf, stream);
}
