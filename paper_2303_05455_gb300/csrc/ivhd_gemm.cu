// ivhd_gemm.cu -- BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores.
//
//   C[m, n] = sum_k A[m, k] B[n, k]        (A: M x K, B: N x K, both row-major = K-major)
//
// with a fused epilogue (bias, GELU, GELU derivative, BF16 or FP32 output).  It
// carries the dense layers of the learned warm start (an MLP that maps features
// to 2-D positions, trained on IVHD embeddings).
//
// One CTA computes one 128 x BN tile:
//   warp 0, one lane   TMA producer: 128 x 64 A and BN x 64 B tiles into a
//                      4-stage shared-memory ring (128-byte swizzle), one
//                      mbarrier with a transaction count per stage
//   warp 1, one lane   MMA issuer: four tcgen05.mma (K = 16 each) per stage,
//                      accumulating in tensor memory; tcgen05.commit frees the
//                      stage, a final commit signals the epilogue
//   warps 0-3          epilogue: tcgen05.ld of their 32 accumulator lanes,
//                      fused element-wise op, global stores
// Every mbarrier wait is bounded; on timeout the kernel raises an error flag,
// drains its copies in flight (again bounded), frees tensor memory and returns.
#include <mutex>

#include "ivhd_gemm.cuh"
#include "ivhd_internal.cuh"
#include "ivhd_tc.cuh"

namespace ivhd {

namespace tc {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
              int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace tc

namespace {

using namespace tc;

constexpr int kBM = 128;
constexpr int kStages = 4;
constexpr int kGemmThreads = 128;

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

__device__ __forceinline__ void ep_apply(const GemmEpilogue& ep, int row, int col0, int N,
                                         const float* v) {
  // v[q] is C[row, col0 + q]
  if (ep.kind == kEpStoreF32) {
    float* o = ep.out_f32 + (int64_t)row * ep.ld_out + col0;
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (col0 + q < N) o[q] = v[q];
  } else if (ep.kind == kEpBiasGelu) {
    // z = acc + bias is kept (FP32) for the backward pass; h = GELU(z) in BF16
    float* z = ep.out_f32 + (int64_t)row * ep.ld_out + col0;
    __nv_bfloat16* h = ep.out_bf16 + (int64_t)row * ep.ld_out + col0;
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (col0 + q < N) {
        const float t = v[q] + ep.bias[col0 + q];
        z[q] = t;
        h[q] = __float2bfloat16_rn(gelu(t));
      }
  } else if (ep.kind == kEpGeluGrad) {
    // dZ = acc * GELU'(z) in BF16 (acc is dH)
    const float* z = ep.aux_f32 + (int64_t)row * ep.ld_out + col0;
    __nv_bfloat16* o = ep.out_bf16 + (int64_t)row * ep.ld_out + col0;
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (col0 + q < N) o[q] = __float2bfloat16_rn(v[q] * gelu_grad(z[q]));
  }
}

template <int BN>
struct GemmSmem {
  static constexpr int a_bytes = kBM * kBK * 2;
  static constexpr int b_bytes = BN * kBK * 2;
  static constexpr int stage_bytes = a_bytes + b_bytes;
  static constexpr int bar_offset = kStages * stage_bytes;
  static constexpr int total = bar_offset + 256 + 1024;  // + alignment slack
};

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_bf16_tn(const __grid_constant__ CUtensorMap map_a,
                   const __grid_constant__ CUtensorMap map_b, GemmEpilogue ep, int M, int N,
                   int K, int32_t* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + GemmSmem<BN>::bar_offset);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int* issued = abort_flag + 1;
  constexpr uint32_t kTmemCols = BN < 32 ? 32 : BN;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  // split-K: slice z of gridDim.z takes k-tiles [kt0, kt0 + nk)
  const int nk_all = (K + kBK - 1) / kBK;
  const int per = (nk_all + gridDim.z - 1) / gridDim.z;
  const int kt0 = blockIdx.z * per;
  const int nk = max(0, min(nk_all, kt0 + per) - kt0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    *issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % kStages;
      if (kt >= kStages && !mbar_wait(&empty[s], ((kt / kStages) - 1) & 1)) {
        atomicOr(err, 1);
        *(volatile int*)abort_flag = 1;
        break;
      }
      if (*(volatile int*)abort_flag) break;
      unsigned char* sa = smem + s * GemmSmem<BN>::stage_bytes;
      unsigned char* sb = sa + GemmSmem<BN>::a_bytes;
      mbar_expect_tx(&full[s], GemmSmem<BN>::stage_bytes);
      tma_load_2d(sa, &map_a, (kt0 + kt) * kBK, m0, &full[s]);
      tma_load_2d(sb, &map_b, (kt0 + kt) * kBK, n0, &full[s]);
      *(volatile int*)issued = kt + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = instr_desc_bf16(kBM, BN);
    int kt = 0;
    for (; kt < nk; ++kt) {
      const int s = kt % kStages;
      if (!mbar_wait(&full[s], (kt / kStages) & 1)) {
        atomicOr(err, 2);
        *(volatile int*)abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sa = smem_u32(smem + s * GemmSmem<BN>::stage_bytes);
      const uint32_t sb = sa + GemmSmem<BN>::a_bytes;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)
        umma_bf16(tmem, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), idesc,
                  (kt > 0 || kk > 0) ? 1u : 0u);
      umma_commit(&empty[s]);
    }
    umma_commit(done);  // covers every MMA issued above
  }
  __syncwarp();
  // epilogue: all four warps, 32 accumulator lanes (rows) each
  const bool ok = mbar_wait(done, 0);
  if (!ok && threadIdx.x == 0) atomicOr(err, 4);
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  const bool aborted = *(volatile int*)abort_flag != 0 || !ok;
  if (!aborted) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    GemmEpilogue epz = ep;
    if (gridDim.z > 1) epz.out_f32 += (int64_t)blockIdx.z * ep.split_stride;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      if (nk > 0) {
        tmem_ld16(trow + c0, v);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = 0.f;  // an empty K slice contributes zero
      }
      if (row < M) ep_apply(epz, row, n0 + c0, N, v);
    }
  } else if (threadIdx.x == 0) {
    // drain copies still in flight before the shared memory goes away
    const int iss = *(volatile int*)issued;
    for (int kt = (iss > kStages ? iss - kStages : 0); kt < iss; ++kt)
      mbar_wait(&full[kt % kStages], (kt / kStages) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
}

// ---- host side: tensor maps -------------------------------------------------

template <int BN>
cudaError_t launch_bn(const CUtensorMap& ma, const CUtensorMap& mb, const GemmEpilogue& ep, int M,
                      int N, int K, int splits, int32_t* err, cudaStream_t s) {
  const int smem = GemmSmem<BN>::total;
  static bool attr_set[64] = {};  // one attribute call per instantiation and device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16_tn<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + kBM - 1) / kBM), (unsigned)splits);
  k_gemm_bf16_tn<BN><<<grid, kGemmThreads, smem, s>>>(ma, mb, ep, M, N, K, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_bf16_tn(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb,
                         int M, int N, int K, const GemmEpilogue& ep, int32_t* err,
                         cudaStream_t s, int splits) {
  const int BN = N <= 64 ? 64 : 128;
  if (splits < 1 || (splits > 1 && ep.kind != kEpStoreF32)) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, lda, kBM)) return cudaErrorInvalidValue;
  if (!make_map(&mb, B, N, K, ldb, BN)) return cudaErrorInvalidValue;
  if (BN == 64) return launch_bn<64>(ma, mb, ep, M, N, K, splits, err, s);
  return launch_bn<128>(ma, mb, ep, M, N, K, splits, err, s);
}

// out[i] = sum_z part[z * stride + i] over `splits` slices in order (deterministic).
__global__ void k_sum_slices(const float* __restrict__ part, int64_t n, int64_t stride, int splits,
                             float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float t = 0.f;
  for (int z = 0; z < splits; ++z) t += part[z * stride + i];
  out[i] = t;
}

cudaError_t sum_slices(const float* part, int64_t n, int64_t stride, int splits, float* out,
                       cudaStream_t s) {
  k_sum_slices<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, n, stride, splits, out);
  return cudaGetLastError();
}

}  // namespace ivhd

using namespace ivhd;

extern "C" ivhd_status ivhd_gemm_bf16_tn(const void* A, const void* B, float* C, int64_t M,
                                         int64_t N, int64_t K, void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1) return IVHD_ERR_ARG;
  if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30) || (K % 8) != 0) return IVHD_ERR_ARG;
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((uintptr_t)C & 15)) return IVHD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* err = nullptr;
  int32_t herr = 0;
  cudaError_t e = dev_alloc((void**)&err, sizeof(int32_t), s);
  if (e != cudaSuccess) return IVHD_ERR_OOM;
  e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
  GemmEpilogue ep{};
  ep.kind = kEpStoreF32;
  ep.split_stride = 0;
  ep.out_f32 = C;
  ep.ld_out = N;
  if (e == cudaSuccess)
    e = gemm_bf16_tn((const __nv_bfloat16*)A, K, (const __nv_bfloat16*)B, K, (int)M, (int)N,
                     (int)K, ep, err, s, 1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s);
  dev_free(err, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e == cudaErrorInvalidValue ? IVHD_ERR_ARG : IVHD_ERR_CUDA;
  return herr ? IVHD_ERR_TIMEOUT : IVHD_OK;
}
