// ivhd_probe.cu -- calibration of the random-gather roofline of the step kernel.
//
// The step kernel's cost is dominated by gathering neighbour positions
// (8-byte float2 reads at data-dependent addresses), which the GPU serves one
// 32-byte L2 sector per gather.  This probe measures the rate the GPU
// sustains for uniformly random float2 gathers from an array of the same size
// as the embedding, with the indices generated in registers (no index stream),
// so it is an upper bound for the step kernel's gather rate.
#include "ivhd_internal.cuh"
#include "ivhd_tc.cuh"

namespace ivhd {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbePerThread = 64;

__global__ void __launch_bounds__(kProbeThreads) k_probe_gather(const float2* __restrict__ y,
                                                                uint32_t M, uint32_t seed,
                                                                float* __restrict__ out) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t s = t * 2654435761u + seed;  // xorshift32 stream per thread
  float ax = 0.f, ay = 0.f;
  for (int g = 0; g < kProbePerThread; g += 8) {
    uint32_t idx[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      s ^= s << 13;
      s ^= s >> 17;
      s ^= s << 5;
      idx[q] = s % M;
    }
    float2 p[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = __ldg(y + idx[q]);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      ax += p[q].x;
      ay += p[q].y;
    }
  }
  out[t] = ax + ay;
}

__global__ void k_probe_fill(float2* y, uint32_t M) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) y[i] = make_float2((float)(i & 1023), (float)(i >> 10));
}

}  // namespace
}  // namespace ivhd

using namespace ivhd;

extern "C" ivhd_status ivhd_probe_gather(int64_t n_positions, int64_t n_gathers, int32_t repeats,
                                         double* gathers_per_s, void* stream) {
  if (!gathers_per_s || n_positions < 1 || n_positions > kMaxVertices || repeats < 1 ||
      n_gathers < kProbeThreads * kProbePerThread || n_gathers > ((int64_t)1 << 34))
    return IVHD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t threads = n_gathers / kProbePerThread;
  const unsigned grid = (unsigned)(threads / kProbeThreads);
  float2* y = nullptr;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = dev_alloc((void**)&y, (size_t)n_positions * sizeof(float2), s);
  if (e == cudaSuccess) e = dev_alloc((void**)&out, (size_t)grid * kProbeThreads * sizeof(float), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    const uint32_t M = (uint32_t)n_positions;
    k_probe_fill<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(y, M);
    for (int w = 0; w < 3; ++w) k_probe_gather<<<grid, kProbeThreads, 0, s>>>(y, M, 17u + w, out);
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < repeats; ++rep)
      k_probe_gather<<<grid, kProbeThreads, 0, s>>>(y, M, 101u + rep, out);
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (y) dev_free(y, s);
  if (out) dev_free(out, s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  *gathers_per_s = (double)grid * kProbeThreads * kProbePerThread * repeats / (ms * 1e-3);
  return IVHD_OK;
}

// ---- launch floor ------------------------------------------------------------
//
// The step loop replays one kernel per step, each a programmatic dependent
// launch of the previous one.  For a small embedding the step's work is a few
// microseconds of dependent L2 accesses, and the cost of dispatching the
// grid's blocks and handing over between launches is a large share of it.
// This probe times that cost alone: the same chain of launches of a kernel
// whose blocks only wait for the previous grid and release the next one.
namespace ivhd {
namespace {

__global__ void k_probe_empty() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace
}  // namespace ivhd

extern "C" ivhd_status ivhd_probe_launch(int32_t grid, int32_t block, int32_t n_launches,
                                         double* us_per_launch, void* stream) {
  if (!us_per_launch || grid < 1 || grid > (1 << 20) || block < 32 || block > 1024 ||
      block % 32 || n_launches < 1 || n_launches > 100000)
    return IVHD_ERR_ARG;
  NvtxScope nvtx_("ivhd_probe_launch");
  cudaStream_t s = (cudaStream_t)stream;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t el = cudaSuccess;
    for (int i = 0; i < n_launches && el == cudaSuccess; ++i) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)grid);
      cfg.blockDim = dim3((unsigned)block);
      cfg.stream = cap;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      el = cudaLaunchKernelEx(&cfg, k_probe_empty);
    }
    e = cudaStreamEndCapture(cap, &graph);
    if (el != cudaSuccess) e = el;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);  // warm-up (uploads the graph)
  float best = 0.f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    float ms = 0.f;
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (rep == 0 || ms < best)) best = ms;
  }
  cudaStreamSynchronize(s);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  *us_per_launch = 1e3 * (double)best / n_launches;
  return IVHD_OK;
}

// ---- bounded-wait check ------------------------------------------------------
//
// The tensor-core kernels wait on mbarriers with a bounded number of polls and
// report a timeout through an error flag instead of hanging.  This kernel runs
// the same bounded wait on an mbarrier that nothing ever completes, so a test
// can watch the timeout path end cleanly with IVHD_ERR_TIMEOUT while the
// context stays usable.
namespace ivhd {
namespace {

__global__ void k_wait_unset(uint32_t polls, int32_t* timed_out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool done = false;
    for (uint32_t it = 0; it < polls && !done; ++it) done = tc::mbar_try_wait(&bar, 0);
    *timed_out = done ? 0 : 1;
  }
}

}  // namespace
}  // namespace ivhd

extern "C" ivhd_status ivhd_probe_wait_timeout(int32_t polls, void* stream) {
  if (polls < 1) return IVHD_ERR_ARG;
  NvtxScope nvtx_("ivhd_probe_wait_timeout");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* flag = nullptr;
  int32_t h = 0;
  cudaError_t e = dev_alloc((void**)&flag, sizeof(int32_t), s);
  if (e != cudaSuccess) return IVHD_ERR_OOM;
  e = cudaMemsetAsync(flag, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) {
    k_wait_unset<<<1, 32, 0, s>>>((uint32_t)polls, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(h), cudaMemcpyDeviceToHost, s);
  dev_free(flag, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  return h ? IVHD_ERR_TIMEOUT : IVHD_OK;
}
