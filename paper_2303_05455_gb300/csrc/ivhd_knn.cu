// ivhd_knn.cu -- exact brute-force kNN graph (the set-up step of Sec. 5.1).
//
// The paper builds the kNN graph with FAISS (IVFADC, approximate) and keeps
// it out of the embedding time.  Here the graph is exact and its decisions are
// reproducible bit for bit on the CPU:
//   float data:  d(q, j) = the FP32 chain acc = fma(x_qd - x_jd, x_qd - x_jd, acc),
//                d = 0 .. N-1 in order, starting from acc = 0;
//   uint8 data:  exact integer |x_q|^2 + |x_j|^2 - 2 <x_q, x_j> via dp4a.
// Ties go to the lower index.  Each CTA owns 128 queries and sweeps all
// candidates in tiles of 128 with an 8x8 register block per thread; after each
// tile the 128x128 distances go through shared memory into a per-query sorted
// list of the k best.
//
// The same search answers queries from a separate set of new points against
// the embedded base set (ivhd_knn_query), and ivhd_place_nn puts each new
// point at the mean embedding of its base neighbours: with k = 1 the
// Progressive UMAP initialisation of a new point (Sec. 2.4.3), the comparator
// of the learned placement.
#include <algorithm>
#include <new>
#include <climits>

#include "ivhd_internal.cuh"
#include "ivhd_knn_tc.cuh"

namespace ivhd {
namespace {

constexpr int kTQ = 128;     // queries per CTA
constexpr int kTC = 128;     // candidates per tile
constexpr int kDK = 32;      // feature chunk (floats) / 4-byte words (uint8)
constexpr int kThreads = 256;
constexpr int kMaxExactSegments = 256;  // column segments of the exact kernel for few rows
constexpr int kDStride = kTC + 4;  // distance-tile row stride (floats)

struct SmemLayout {
  // [kDK][kTQ] + [kDK][kTC] staging, then the distance tile, then the lists
  static constexpr size_t stage_bytes = (size_t)2 * kDK * (kTQ + 4) * 4;
  static constexpr size_t tile_bytes = (size_t)kTQ * kDStride * 4;
  static size_t lists_bytes(int k) { return (size_t)kTQ * k * 8; }
  static size_t total(int k) { return stage_bytes + tile_bytes + lists_bytes(k); }
};

template <class D>
__device__ __forceinline__ bool better(D d, int j, D bd, int bj) {
  return d < bd || (d == bd && j < bj);
}

// Merge one 128-candidate row of the tile into a query's sorted list; the
// candidate `skip` (the query itself in a kNN graph, else -1) is left out.
template <class D>
__device__ __forceinline__ void merge_row(const D* row, int c0, int64_t M, int64_t skip, int k,
                                          D* ld, int* lj, int& n) {
  for (int b = 0; b < kTC; ++b) {
    const int64_t j = c0 + b;
    if (j >= M) break;
    if (j == skip) continue;
    const D d = row[b];
    if (n == k && !better(d, (int)j, ld[k - 1], lj[k - 1])) continue;
    int pos = (n < k) ? n : k - 1;
    while (pos > 0 && better(d, (int)j, ld[pos - 1], lj[pos - 1])) {
      ld[pos] = ld[pos - 1];
      lj[pos] = lj[pos - 1];
      --pos;
    }
    ld[pos] = d;
    lj[pos] = (int)j;
    if (n < k) ++n;
  }
}

// Queries: the Mq rows of Q (Q = X and self = true for the kNN graph).
// rows / n_rows (device, optional): the CTA's queries are entries q0 .. q0+127
// of the list rows[0 .. *n_rows) instead of rows q0 .. q0+127.
// Column segments (gridDim.y > 1): CTA (x, y) sweeps candidates
// [y * seg_cols, (y + 1) * seg_cols) only and writes its sorted list of the
// k best (padded with (+inf, INT_MAX)) for list entry t to
// seg_d / seg_j[(t * gridDim.y + y) * k ..]; k_merge_segments combines them.
__global__ void __launch_bounds__(kThreads)
    k_knn_f32(const float* __restrict__ Q, int64_t Mq, const float* __restrict__ X, int64_t M,
              int N, int k, bool self, int32_t* __restrict__ out,
              const int32_t* __restrict__ rows, const int32_t* __restrict__ n_rows,
              int64_t seg_cols, float* __restrict__ seg_d, int32_t* __restrict__ seg_j) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* Qs = reinterpret_cast<float*>(smem);                    // [kDK][kTQ + 4]
  float* Cs = Qs + kDK * (kTQ + 4);                              // [kDK][kTC + 4]
  float* Dt = reinterpret_cast<float*>(smem + SmemLayout::stage_bytes);  // [kTQ][kDStride]
  float* Ld = reinterpret_cast<float*>(smem + SmemLayout::stage_bytes + SmemLayout::tile_bytes);
  int* Lj = reinterpret_cast<int*>(Ld + kTQ * k);

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t q0 = (int64_t)blockIdx.x * kTQ;
  const int64_t nq = rows ? (int64_t)*n_rows : Mq;
  if (q0 >= nq) return;
  auto qrow = [&](int64_t t) -> int64_t { return rows ? (int64_t)rows[t] : t; };
  int nlist = 0;  // used by threads tid < kTQ
  const int64_t c_beg = (int64_t)blockIdx.y * seg_cols;
  const int64_t c_end = min(M, c_beg + seg_cols);

  for (int64_t c0 = c_beg; c0 < c_end; c0 += kTC) {
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

    for (int d0 = 0; d0 < N; d0 += kDK) {
      // stage a [kDK x 128] slab of queries and candidates, transposed
      for (int e = tid; e < kDK * kTQ; e += kThreads) {
        const int row = e / kDK, dd = e % kDK;
        const int64_t tq = q0 + row, gc = c0 + row;
        const int d = d0 + dd;
        Qs[dd * (kTQ + 4) + row] = (tq < nq && d < N) ? Q[qrow(tq) * N + d] : 0.f;
        Cs[dd * (kTC + 4) + row] = (gc < c_end && d < N) ? X[gc * N + d] : 0.f;
      }
      __syncthreads();
      const int dn = min(kDK, N - d0);
      for (int dd = 0; dd < dn; ++dd) {
        const float4 qa = *reinterpret_cast<const float4*>(&Qs[dd * (kTQ + 4) + ty * 8]);
        const float4 qb = *reinterpret_cast<const float4*>(&Qs[dd * (kTQ + 4) + ty * 8 + 4]);
        const float4 ca = *reinterpret_cast<const float4*>(&Cs[dd * (kTC + 4) + tx * 8]);
        const float4 cb = *reinterpret_cast<const float4*>(&Cs[dd * (kTC + 4) + tx * 8 + 4]);
        const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
        const float cv[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            const float diff = __fsub_rn(qv[a], cv[b]);
            acc[a][b] = __fmaf_rn(diff, diff, acc[a][b]);
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) Dt[(ty * 8 + a) * kDStride + tx * 8 + b] = acc[a][b];
    __syncthreads();
    if (tid < kTQ && q0 + tid < nq)
      merge_row<float>(Dt + tid * kDStride, (int)c0, c_end, self ? qrow(q0 + tid) : -1, k,
                       Ld + tid * k, Lj + tid * k, nlist);
    __syncthreads();
  }
  if (tid < kTQ && q0 + tid < nq) {
    if (gridDim.y == 1) {
      for (int s = 0; s < k; ++s) out[qrow(q0 + tid) * k + s] = Lj[tid * k + s];
    } else {
      const int64_t o = ((q0 + tid) * gridDim.y + blockIdx.y) * k;
      for (int s = 0; s < k; ++s) {
        seg_d[o + s] = s < nlist ? Ld[tid * k + s] : __int_as_float(0x7f800000);
        seg_j[o + s] = s < nlist ? Lj[tid * k + s] : INT_MAX;
      }
    }
  }
}

// The per-segment lists of list entry t (n_seg sorted lists of k) merged into
// the k best, ties to the lower index.
__global__ void k_merge_segments(const float* __restrict__ seg_d, const int32_t* __restrict__ seg_j,
                                 int n_seg, int k, const int32_t* __restrict__ rows,
                                 const int32_t* __restrict__ n_rows, int32_t* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *n_rows) return;
  const float* d = seg_d + t * n_seg * k;
  const int32_t* j = seg_j + t * n_seg * k;
  int head[kMaxExactSegments];
  for (int h = 0; h < n_seg; ++h) head[h] = 0;
  for (int q = 0; q < k; ++q) {
    int bh = -1;
    for (int h = 0; h < n_seg; ++h) {
      if (head[h] >= k) continue;
      const int64_t a = (int64_t)h * k + head[h];
      if (bh < 0) {
        bh = h;
        continue;
      }
      const int64_t b = (int64_t)bh * k + head[bh];
      if (better(d[a], j[a], d[b], j[b])) bh = h;
    }
    out[(int64_t)rows[t] * k + q] = j[(int64_t)bh * k + head[bh]];
    ++head[bh];
  }
}

__global__ void k_norms_u8(const uint8_t* __restrict__ X, int64_t M, int N,
                           int32_t* __restrict__ nrm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int32_t s = 0;
  for (int d = 0; d < N; ++d) {
    const int32_t v = X[i * N + d];
    s += v * v;
  }
  nrm[i] = s;
}

__device__ __forceinline__ uint32_t pack4(const uint8_t* __restrict__ X, int64_t row, int64_t M,
                                          int N, int d) {
  uint32_t w = 0;
  if (row < M) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (d + b < N) w |= (uint32_t)X[row * N + d + b] << (8 * b);
  }
  return w;
}

__global__ void __launch_bounds__(kThreads)
    k_knn_u8(const uint8_t* __restrict__ Q, const int32_t* __restrict__ qnrm, int64_t Mq,
             const uint8_t* __restrict__ X, const int32_t* __restrict__ nrm, int64_t M, int N,
             int k, bool self, int32_t* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* Qs = reinterpret_cast<uint32_t*>(smem);  // [kDK words][kTQ + 4]
  uint32_t* Cs = Qs + kDK * (kTQ + 4);
  int32_t* Dt = reinterpret_cast<int32_t*>(smem + SmemLayout::stage_bytes);
  int32_t* Ld = reinterpret_cast<int32_t*>(smem + SmemLayout::stage_bytes + SmemLayout::tile_bytes);
  int* Lj = reinterpret_cast<int*>(Ld + kTQ * k);

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t q0 = (int64_t)blockIdx.x * kTQ;
  int nlist = 0;
  const int nwords = (N + 3) / 4;

  for (int64_t c0 = 0; c0 < M; c0 += kTC) {
    uint32_t acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0u;
    for (int w0 = 0; w0 < nwords; w0 += kDK) {
      for (int e = tid; e < kDK * kTQ; e += kThreads) {
        const int row = e / kDK, ww = e % kDK;
        const int d = (w0 + ww) * 4;
        Qs[ww * (kTQ + 4) + row] = (w0 + ww < nwords) ? pack4(Q, q0 + row, Mq, N, d) : 0u;
        Cs[ww * (kTC + 4) + row] = (w0 + ww < nwords) ? pack4(X, c0 + row, M, N, d) : 0u;
      }
      __syncthreads();
      const int wn = min(kDK, nwords - w0);
      for (int ww = 0; ww < wn; ++ww) {
        const uint4 qa = *reinterpret_cast<const uint4*>(&Qs[ww * (kTQ + 4) + ty * 8]);
        const uint4 qb = *reinterpret_cast<const uint4*>(&Qs[ww * (kTQ + 4) + ty * 8 + 4]);
        const uint4 ca = *reinterpret_cast<const uint4*>(&Cs[ww * (kTC + 4) + tx * 8]);
        const uint4 cb = *reinterpret_cast<const uint4*>(&Cs[ww * (kTC + 4) + tx * 8 + 4]);
        const uint32_t qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
        const uint32_t cv[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = __dp4a(qv[a], cv[b], acc[a][b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t gq = q0 + ty * 8 + a;
      const int32_t nq = (gq < Mq) ? qnrm[gq] : 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int64_t gc = c0 + tx * 8 + b;
        const int32_t nc = (gc < M) ? nrm[gc] : 0;
        Dt[(ty * 8 + a) * kDStride + tx * 8 + b] = nq + nc - 2 * (int32_t)acc[a][b];
      }
    }
    __syncthreads();
    if (tid < kTQ && q0 + tid < Mq)
      merge_row<int32_t>(Dt + tid * kDStride, (int)c0, M, self ? q0 + tid : -1, k, Ld + tid * k,
                         Lj + tid * k, nlist);
    __syncthreads();
  }
  if (tid < kTQ && q0 + tid < Mq)
    for (int s = 0; s < k; ++s) out[(q0 + tid) * k + s] = Lj[tid * k + s];
}

// y_q = (1/k) sum_s Y[ids[q][s]], summed in FP32 in the order s = 0 .. k-1.
// An id outside [0, M) raises *bad and leaves that row unwritten.
__global__ void k_place_nn(const float2* __restrict__ Y, int64_t M, const int32_t* __restrict__ ids,
                           int64_t n, int k, float2* __restrict__ out, int32_t* __restrict__ bad) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  float sx = 0.f, sy = 0.f;
  for (int s = 0; s < k; ++s) {
    const int32_t j = ids[q * k + s];
    if (j < 0 || (int64_t)j >= M) {
      atomicOr(bad, 1);
      return;
    }
    const float2 y = Y[j];
    sx += y.x;
    sy += y.y;
  }
  out[q] = make_float2(sx / (float)k, sy / (float)k);
}

}  // namespace

cudaError_t knn_exact_rows_f32(const KnnProblem& P, const int32_t* rows, const int32_t* n_rows,
                               int32_t* out_knn, cudaStream_t s) {
  const size_t sm = SmemLayout::total(P.k);
  cudaError_t e = cudaFuncSetAttribute(k_knn_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  const float* Q = (const float*)P.Q;
  const float* X = (const float*)P.X;
  if (!rows) {
    k_knn_f32<<<(unsigned)((P.Mq + kTQ - 1) / kTQ), kThreads, sm, s>>>(
        Q, P.Mq, X, P.M, P.N, P.k, P.self, out_knn, nullptr, nullptr, P.M, nullptr, nullptr);
    return cudaGetLastError();
  }
  // a row list (rows the tensor-core certificate did not cover): usually a
  // few rows, so the candidates are split into column segments that run in
  // parallel (about two CTAs per SM in all), merged per row afterwards
  int32_t n = 0;
  e = cudaMemcpyAsync(&n, n_rows, sizeof(n), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || n == 0) return e;
  int sms = 0, dev = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t row_blocks = (n + kTQ - 1) / kTQ;
  int64_t want = (2 * (int64_t)sms + row_blocks - 1) / row_blocks;
  want = std::min<int64_t>(want, std::min<int64_t>(kMaxExactSegments, P.M / 2048));
  want = std::max<int64_t>(want, 1);
  const int64_t seg_cols = ((P.M + want - 1) / want + kTC - 1) / kTC * kTC;
  const int64_t n_seg = (P.M + seg_cols - 1) / seg_cols;
  if (n_seg == 1) {
    k_knn_f32<<<(unsigned)row_blocks, kThreads, sm, s>>>(Q, P.Mq, X, P.M, P.N, P.k, P.self,
                                                          out_knn, rows, n_rows, P.M, nullptr,
                                                          nullptr);
    return cudaGetLastError();
  }
  float* seg_d = nullptr;
  int32_t* seg_j = nullptr;
  const size_t len = (size_t)n * (size_t)n_seg * (size_t)P.k;
  e = dev_alloc((void**)&seg_d, len * sizeof(float), s);
  if (e == cudaSuccess) e = dev_alloc((void**)&seg_j, len * sizeof(int32_t), s);
  if (e == cudaSuccess) {
    k_knn_f32<<<dim3((unsigned)row_blocks, (unsigned)n_seg), kThreads, sm, s>>>(
        Q, P.Mq, X, P.M, P.N, P.k, P.self, out_knn, rows, n_rows, seg_cols, seg_d, seg_j);
    k_merge_segments<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(seg_d, seg_j, (int)n_seg, P.k,
                                                                 rows, n_rows, out_knn);
    e = cudaGetLastError();
  }
  dev_free(seg_d, s);
  dev_free(seg_j, s);
  return e;
}

// The CUDA-core build of every query row (k <= 64).
static ivhd_status knn_cuda_cores(const KnnProblem& P, int32_t* out_knn, cudaStream_t s) {
  const size_t sm = SmemLayout::total(P.k);
  const unsigned grid = (unsigned)((P.Mq + kTQ - 1) / kTQ);
  cudaError_t e;
  if (P.dtype == IVHD_KNN_F32) {
    e = knn_exact_rows_f32(P, nullptr, nullptr, out_knn, s);
  } else {
    const uint8_t* X = (const uint8_t*)P.X;
    const uint8_t* Q = (const uint8_t*)P.Q;
    int32_t* nrm = nullptr;
    int32_t* qnrm = nullptr;
    e = dev_alloc((void**)&nrm, (size_t)P.M * sizeof(int32_t), s);
    if (e == cudaSuccess && !P.self) e = dev_alloc((void**)&qnrm, (size_t)P.Mq * sizeof(int32_t), s);
    if (e != cudaSuccess) {
      dev_free(nrm, s);
      return IVHD_ERR_OOM;
    }
    if (P.self) qnrm = nrm;
    k_norms_u8<<<(unsigned)((P.M + 255) / 256), 256, 0, s>>>(X, P.M, P.N, nrm);
    if (!P.self) k_norms_u8<<<(unsigned)((P.Mq + 255) / 256), 256, 0, s>>>(Q, P.Mq, P.N, qnrm);
    e = cudaFuncSetAttribute(k_knn_u8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
      k_knn_u8<<<grid, kThreads, sm, s>>>(Q, qnrm, P.Mq, X, nrm, P.M, P.N, P.k, P.self, out_knn);
      e = cudaGetLastError();
    }
    if (!P.self) dev_free(qnrm, s);
    dev_free(nrm, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? IVHD_OK : IVHD_ERR_CUDA;
}

// Method choice, tensor-core or CUDA-core run and statistics for one problem.
static ivhd_status knn_run(const KnnProblem& P, int32_t* out, int32_t method,
                           ivhd_knn_stats_t* stats, cudaStream_t s,
                           const KnnBase* base = nullptr) {
  if (method < IVHD_KNN_AUTO || method > IVHD_KNN_TENSOR_CORES) return IVHD_ERR_ARG;
  const bool tc_ok = knn_tc_supported(P);
  if (method == IVHD_KNN_TENSOR_CORES && !tc_ok) return IVHD_ERR_ARG;
  const bool use_tc = method == IVHD_KNN_TENSOR_CORES || (method == IVHD_KNN_AUTO && tc_ok);
  ivhd_knn_stats_t st{};
  st.method = use_tc ? IVHD_KNN_TENSOR_CORES : IVHD_KNN_CUDA_CORES;
  ivhd_status r;
  if (use_tc) {
    KnnTcStats t{};
    r = knn_tc_build(P, out, s, &t, base);
    st.fallback_rows = t.fallback_rows;
    st.max_rel_err = t.max_rel_err;
    st.eps_coef = t.eps_coef;
  } else {
    r = knn_cuda_cores(P, out, s);
  }
  if (stats) *stats = st;
  return r;
}

}  // namespace ivhd

using namespace ivhd;

// Argument rules shared by the graph build and the query (dtype, N, k against
// the number of base rows that can be listed).
static bool knn_args_ok(int32_t dtype, int64_t M, int32_t N, int32_t k, int64_t listable) {
  if (M < 1 || M >= (int64_t)0x7FFFFFFF || N < 1 || N > 65536) return false;
  if (k < 1 || (int64_t)k > listable || k > 64) return false;
  if (dtype != IVHD_KNN_F32 && dtype != IVHD_KNN_U8) return false;
  if (dtype == IVHD_KNN_U8 && (int64_t)N * 255 * 255 > 0x3FFFFFFF) return false;
  return true;
}

extern "C" ivhd_status ivhd_knn_build_ex(const void* X, int32_t dtype, int64_t M, int32_t N,
                                         int32_t k, int32_t* out_knn, int32_t method,
                                         ivhd_knn_stats_t* stats, void* stream) {
  NvtxScope nvtx_("ivhd_knn_build");
  if (!X || !out_knn || M < 2 || !knn_args_ok(dtype, M, N, k, M - 1)) return IVHD_ERR_ARG;
  const KnnProblem P{X, M, X, M, dtype, N, k, true};
  return knn_run(P, out_knn, method, stats, (cudaStream_t)stream);
}

extern "C" ivhd_status ivhd_knn_build(const void* X, int32_t dtype, int64_t M, int32_t N,
                                      int32_t k, int32_t* out_knn, void* stream) {
  return ivhd_knn_build_ex(X, dtype, M, N, k, out_knn, IVHD_KNN_AUTO, nullptr, stream);
}

extern "C" ivhd_status ivhd_knn_query(const void* Q, int64_t Mq, const void* X, int64_t M,
                                      int32_t dtype, int32_t N, int32_t k, int32_t* out,
                                      int32_t method, ivhd_knn_stats_t* stats, void* stream) {
  NvtxScope nvtx_("ivhd_knn_query");
  if (!Q || !X || !out || Mq < 1 || Mq >= (int64_t)0x7FFFFFFF) return IVHD_ERR_ARG;
  if (!knn_args_ok(dtype, M, N, k, M)) return IVHD_ERR_ARG;
  const KnnProblem P{Q, Mq, X, M, dtype, N, k, false};
  return knn_run(P, out, method, stats, (cudaStream_t)stream);
}

extern "C" ivhd_status ivhd_place_nn(const float* Y, int64_t M, const int32_t* ids, int64_t n,
                                     int32_t k, float* out, void* stream) {
  NvtxScope nvtx_("ivhd_place_nn");
  if (!Y || M < 1 || n < 0 || k < 1 || k > 1024) return IVHD_ERR_ARG;
  if (n == 0) return IVHD_OK;
  if (!ids || !out) return IVHD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* bad = nullptr;
  if (dev_alloc((void**)&bad, sizeof(int32_t), s) != cudaSuccess) return IVHD_ERR_OOM;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) {
    k_place_nn<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const float2*)Y, M, ids, n, k,
                                                           (float2*)out, bad);
    e = cudaGetLastError();
  }
  int32_t h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s);
  dev_free(bad, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  return h ? IVHD_ERR_INDEX : IVHD_OK;
}

// ---- a base set held for repeated queries ----------------------------------

struct ivhd_knn_index {
  cudaStream_t stream = nullptr;
  int32_t dtype = 0, N = 0;
  int64_t M = 0;
  void* X = nullptr;             // the library's copy of the base rows
  __nv_bfloat16* B = nullptr;    // prepared tensor-core operand (null: CUDA cores only)
  void* nrm = nullptr;           // its row norms
};

static void index_free(ivhd_knn_index* idx) {
  if (idx->X) dev_free(idx->X, idx->stream);
  if (idx->B) dev_free(idx->B, idx->stream);
  if (idx->nrm) dev_free(idx->nrm, idx->stream);
  delete idx;
}

extern "C" ivhd_status ivhd_knn_index_create(const void* X, int32_t dtype, int64_t M, int32_t N,
                                             void* stream, ivhd_knn_index** out) {
  NvtxScope nvtx_("ivhd_knn_index_create");
  if (!X || !out || !knn_args_ok(dtype, M, N, 1, M)) return IVHD_ERR_ARG;
  *out = nullptr;
  ivhd_knn_index* idx = new (std::nothrow) ivhd_knn_index();
  if (!idx) return IVHD_ERR_OOM;
  idx->stream = (cudaStream_t)stream;
  idx->dtype = dtype;
  idx->M = M;
  idx->N = N;
  cudaStream_t s = idx->stream;
  const size_t bytes = (size_t)M * (size_t)N * (dtype == IVHD_KNN_U8 ? 1 : 4);
  cudaError_t e = dev_alloc(&idx->X, bytes, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(idx->X, X, bytes, cudaMemcpyDeviceToDevice, s);
  // the tensor-core operand, when the tensor-core method applies to this base set
  const KnnProblem probe{X, 1, X, M, dtype, N, 1, false};
  if (e == cudaSuccess && knn_tc_supported(probe)) {
    const int Kp = knn_tc_kp(dtype, N);
    e = dev_alloc((void**)&idx->B, (size_t)M * Kp * sizeof(__nv_bfloat16), s);
    if (e == cudaSuccess) e = dev_alloc(&idx->nrm, (size_t)M * 4, s);
    if (e == cudaSuccess) e = knn_tc_prepare_base(idx->X, dtype, M, N, idx->B, idx->nrm, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    index_free(idx);
    return e == cudaErrorMemoryAllocation ? IVHD_ERR_OOM : IVHD_ERR_CUDA;
  }
  *out = idx;
  return IVHD_OK;
}

extern "C" ivhd_status ivhd_knn_index_query(ivhd_knn_index* idx, const void* Q, int64_t Mq,
                                            int32_t k, int32_t* out, int32_t method,
                                            ivhd_knn_stats_t* stats) {
  NvtxScope nvtx_("ivhd_knn_index_query");
  if (!idx || !Q || !out || Mq < 1 || Mq >= (int64_t)0x7FFFFFFF) return IVHD_ERR_ARG;
  if (!knn_args_ok(idx->dtype, idx->M, idx->N, k, idx->M)) return IVHD_ERR_ARG;
  const KnnProblem P{Q, Mq, idx->X, idx->M, idx->dtype, idx->N, k, false};
  const KnnBase base{idx->B, idx->nrm};
  return knn_run(P, out, method, stats, idx->stream, idx->B ? &base : nullptr);
}

extern "C" void ivhd_knn_index_destroy(ivhd_knn_index* idx) {
  if (idx) index_free(idx);
}
