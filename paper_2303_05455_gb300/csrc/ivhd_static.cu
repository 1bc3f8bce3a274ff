// ivhd_static.cu -- ivhd_eval_qnx_static: Q_NX(k) without any device allocation.
//
// Some host applications cannot let a library allocate device memory: a
// process whose device memory is reserved up front by another framework's
// caching allocator, a latency-critical loop in which cudaMalloc/cudaFree
// would synchronise the device, or an application that must keep its
// device-memory footprint fixed after start-up.  ivhd_eval_qnx reserves a
// small hit counter with cudaMallocAsync on every call; this variant keeps
// its scratch in a fixed array in the library's own device memory instead.
//
// The scratch array (kStaticMaxBlocks + 2 counters, 64 KiB + 16 B) lives in
// every GPU that loads the library until the process exits.  All calls on a
// device share it, so calls whose work overlaps on the GPU (different streams
// or host threads without ordering) race and may return wrong values; order
// them on one stream.  Every slot a call reads is first written by the same
// call, so nothing has to be cleared between calls.
//
// A sampled row id outside [0, M) is never dereferenced: its thread stays
// inactive, the block counts it next to its hits, and the call returns
// IVHD_ERR_INDEX.
//
// Host code cannot use the array's name as a device address.  The address is
// looked up with cudaGetSymbolAddress once per device and CUDA context (the
// context's unique id from the driver is part of the key), so a context that
// the caller destroys and re-creates -- e.g. after cudaDeviceReset, which
// reloads the library's device code -- gets a fresh address instead of a
// stale one.
#include <cuda.h>

#include <mutex>

#include "ivhd_internal.cuh"

namespace ivhd {
namespace {

constexpr int kStaticThreads = 128;
constexpr int kStaticTile = 2048;
constexpr int kStaticMaxBlocks = 8192;  // rows per call <= 8192 * 128 = 1,048,576
constexpr int kStaticMaxDevices = 64;
constexpr int kBadShift = 48;  // per-block slot: hits (< 2^14) + (rows out of range << 48)

// per-block slots, then the call's hit total and its count of rows out of range
static __device__ __align__(256) unsigned long long g_qnx_scratch[kStaticMaxBlocks + 2];

// Same neighbour search and hit count as ivhd_eval_qnx (one thread per sampled
// row, shared-memory tiles of the embedding, FP32 squared distances, ties to
// the lower index); hits are summed per block into scratch[blockIdx.x], with
// the block's rows outside [0, M) counted in the slot's high bits.
__global__ void __launch_bounds__(kStaticThreads) k_qnx_static(
    const float2* __restrict__ Y, int64_t M, const int64_t* __restrict__ rows, int64_t nrows,
    int kk, const int32_t* __restrict__ knn, int32_t* __restrict__ out_lowd,
    unsigned long long* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long warp_hits[kStaticThreads / 32];
  __shared__ unsigned int block_bad;
  float2* tile = reinterpret_cast<float2*>(smem);
  float* ld = reinterpret_cast<float*>(tile + kStaticTile) + threadIdx.x * kk;
  int* lj = reinterpret_cast<int*>(reinterpret_cast<float*>(tile + kStaticTile) +
                                   kStaticThreads * kk) +
            threadIdx.x * kk;
  const int64_t qi = (int64_t)blockIdx.x * kStaticThreads + threadIdx.x;
  const int64_t q = qi < nrows ? rows[qi] : 0;
  const bool in_range = q >= 0 && q < M;
  const bool act = qi < nrows && in_range;
  if (threadIdx.x == 0) block_bad = 0;
  __syncthreads();
  if (qi < nrows && !in_range) atomicAdd(&block_bad, 1u);
  const float2 yq = act ? Y[q] : make_float2(0.f, 0.f);
  int n = 0;
  float worst = INFINITY;
  for (int64_t t0 = 0; t0 < M; t0 += kStaticTile) {
    const int tn = (int)min((int64_t)kStaticTile, M - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < tn; e += kStaticThreads) tile[e] = Y[t0 + e];
    __syncthreads();
    if (!act) continue;
    for (int e = 0; e < tn; ++e) {
      const float2 yj = tile[e];
      const float dx = __fsub_rn(yj.x, yq.x);
      const float dy = __fsub_rn(yj.y, yq.y);
      const float d2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
      if (n == kk && !(d2 < worst)) continue;
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
  unsigned long long h = 0;
  if (act) {
    for (int s = 0; s < n; ++s) {
      const int j = lj[s];
      if (out_lowd) out_lowd[qi * kk + s] = j;
      for (int u = 0; u < kk; ++u)
        if (knn[q * kk + u] == j) {
          ++h;
          break;
        }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h += __shfl_down_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0) warp_hits[threadIdx.x >> 5] = h;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kStaticThreads / 32; ++w) t += warp_hits[w];
    scratch[blockIdx.x] = t + ((unsigned long long)block_bad << kBadShift);
  }
}

__global__ void k_qnx_static_total(unsigned long long* __restrict__ scratch, int nblocks) {
  __shared__ unsigned long long sh[2][32];
  const unsigned long long mask = (1ull << kBadShift) - 1;
  unsigned long long v = 0, bad = 0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    v += scratch[i] & mask;
    bad += scratch[i] >> kBadShift;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_down_sync(0xffffffffu, v, o);
    bad += __shfl_down_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = v;
    sh[1][threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t += sh[0][w];
      b += sh[1][w];
    }
    scratch[kStaticMaxBlocks] = t;
    scratch[kStaticMaxBlocks + 1] = b;
  }
}

// The current context's unique id (cuCtxGetCurrent + cuCtxGetId, reached
// through the runtime's driver entry points so the library needs no libcuda
// link); 0 if the driver cannot tell.
unsigned long long current_ctx_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)p;
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

struct ScratchAddr {
  unsigned long long ctx_id = 0;
  unsigned long long* ptr = nullptr;
};
std::mutex g_mu;
ScratchAddr g_addr[kStaticMaxDevices];

// Device address of the scratch array on the current device, looked up once
// per device and context.  Before the first runtime call of a thread no
// context may be current yet: the lookup itself makes one current, and its id
// is read afterwards.  Without a context id from the driver the address is
// looked up on every call.
cudaError_t scratch_ptr(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long id = current_ctx_id();
  std::lock_guard<std::mutex> lock(g_mu);
  if (id == 0 || g_addr[dev].ptr == nullptr || g_addr[dev].ctx_id != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_qnx_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev].ptr = (unsigned long long*)p;
    g_addr[dev].ctx_id = current_ctx_id();
  }
  *out = g_addr[dev].ptr;
  return cudaSuccess;
}

}  // namespace
}  // namespace ivhd

using namespace ivhd;

extern "C" ivhd_status ivhd_eval_qnx_static(const float* Y, int64_t M, const int32_t* knn,
                                            int32_t k, const int64_t* rows, int64_t nrows,
                                            int32_t* out_lowd, double* out_q, void* stream) {
  if (!Y || !knn || !rows || !out_q || M < 2 || nrows < 1) return IVHD_ERR_ARG;
  if (k < 1 || (int64_t)k > M - 1 || k > 128) return IVHD_ERR_ARG;
  const int64_t nblocks = (nrows + kStaticThreads - 1) / kStaticThreads;
  if (nblocks > kStaticMaxBlocks) return IVHD_ERR_ARG;  // more rows than the fixed scratch holds
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* scratch = nullptr;
  cudaError_t e = scratch_ptr(&scratch);
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  const size_t sm = (size_t)kStaticTile * sizeof(float2) + (size_t)kStaticThreads * k * 8;
  e = cudaFuncSetAttribute(k_qnx_static, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  k_qnx_static<<<(unsigned)nblocks, kStaticThreads, sm, s>>>((const float2*)Y, M, rows, nrows, k,
                                                             knn, out_lowd, scratch);
  k_qnx_static_total<<<1, 1024, 0, s>>>(scratch, (int)nblocks);
  e = cudaGetLastError();
  unsigned long long hits[2] = {0, 0};  // hits, rows outside [0, M)
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hits, scratch + kStaticMaxBlocks, sizeof(hits), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  if (hits[1] != 0) return IVHD_ERR_INDEX;
  *out_q = (double)hits[0] / ((double)k * (double)nrows);
  return IVHD_OK;
}
