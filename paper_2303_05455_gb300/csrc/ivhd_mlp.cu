// ivhd_mlp.cu -- the learned warm start: an MLP that maps features to 2-D positions.
//
//   x -> h1 = GELU(W1 x + b1) -> h2 = GELU(W2 h1 + b2) -> y = W3 h2 + b3
//
// trained with the mean squared error to IVHD embedding coordinates and Adam
// (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  Weights keep an FP32
// master copy (and the Adam moments); the two wide layers run on the tensor
// cores from BF16 copies with FP32 accumulation (ivhd_gemm.cu), with the bias
// and GELU (forward) or GELU derivative (backward) fused into the GEMM
// epilogue; the 2-wide output layer and the reductions over the batch run on
// the CUDA cores in FP32 with fixed summation orders.  Everything is ordered
// on the context stream (within a training step a second stream runs the work
// off the GEMM chain, forked and joined by events); training steps need no
// host synchronisation.
#include <cuda_bf16.h>

#include <cmath>
#include <new>
#include <vector>

#include "ivhd_gemm.cuh"
#include "ivhd_internal.cuh"

struct ivhd_mlp {
  int n_in = 0, hidden = 0, max_batch = 0;
  cudaStream_t stream = nullptr;
  int64_t n_params = 0;
  int64_t t = 0;          // Adam step counter
  int last_rows = 0;      // rows of the last batch whose intermediates are held
  bool poisoned = false;
  // parameters: FP32 master, Adam moments, gradients (flat: W1 b1 W2 b2 W3 b3)
  float* w = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* g = nullptr;
  // BF16 copies used by the tensor cores
  __nv_bfloat16* w1 = nullptr;   // hidden x n_in
  __nv_bfloat16* w2 = nullptr;   // hidden x hidden
  __nv_bfloat16* w2t = nullptr;  // transposed W2
  // workspace for one batch
  __nv_bfloat16 *xb = nullptr, *xt = nullptr;
  float *z1 = nullptr, *z2 = nullptr;
  __nv_bfloat16 *h1 = nullptr, *h1t = nullptr, *h2 = nullptr;
  __nv_bfloat16 *dz2 = nullptr, *dz2t = nullptr, *dz1 = nullptr, *dz1t = nullptr;
  float *y = nullptr, *dy = nullptr;
  float* part = nullptr;       // split-K slices (dW1) and batch-chunk partial sums
  float* part2 = nullptr;      // split-K slices of dW2
  float* cs_part = nullptr;    // chunk partials of the bias gradients (side stream)
  float* g3_part = nullptr;    // chunk partials of the output-layer gradient (side stream)
  double* loss_part = nullptr;
  double* loss_out = nullptr;
  // side stream for the work off the GEMM chain (the transposed input, the
  // output-layer and bias gradients), ordered against the main stream by events
  cudaStream_t side = nullptr;
  cudaEvent_t ev[6] = {};
  int32_t* err = nullptr;
  int64_t launches = 0;
  // the training step captured as a CUDA graph for batch size graph_B; the
  // nodes that read the call's inputs and learning rate are patched per call
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_B = 0;            // batch size of the captured step (0: none)
  int direct_B = 0;           // batch size of the last step run without the graph
  int64_t graph_launches = 0; // kernels per replay
  cudaGraphNode_t node_x = nullptr, node_loss = nullptr, node_adam = nullptr;
  cudaKernelNodeParams kp_x{}, kp_loss{}, kp_adam{};
};

namespace ivhd {
namespace {

constexpr int kLossBlocks = 256;
constexpr int kSplitK = 8;       // K = batch products (weight gradients) are split 8 ways
constexpr int kRowChunk = 32;    // rows per partial of the batch reductions

// GELU'(x) = Phi(x) + x phi(x) for the exact GELU x Phi(x).
__device__ __forceinline__ float gelu_grad_dev(float x) {
  const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

struct Offs {
  int64_t W1, b1, W2, b2, W3, b3, total;
};
Offs offsets(int n_in, int H) {
  Offs o;
  o.W1 = 0;
  o.b1 = o.W1 + (int64_t)H * n_in;
  o.W2 = o.b1 + H;
  o.b2 = o.W2 + (int64_t)H * H;
  o.W3 = o.b2 + H;
  o.b3 = o.W3 + 2 * (int64_t)H;
  o.total = o.b3 + 2;
  return o;
}

inline unsigned nb(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

// Input rows to BF16: uint8 * scale, FP32, or BF16 as given.  Eight
// consecutive elements per thread (one 16-byte store), element by element at a
// ragged end or for an input that is not 16-byte aligned; each value is
// (float)x * scale rounded to BF16 either way.
__global__ void k_convert_x(const void* __restrict__ x, int dtype, float scale, int64_t n,
                            __nv_bfloat16* __restrict__ out) {
  const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
  if (e0 >= n) return;
  const bool vec = e0 + 8 <= n && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  float v[8];
  if (vec) {
    if (dtype == 1) {
      const uint2 w = *reinterpret_cast<const uint2*>((const uint8_t*)x + e0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[q] = (float)((w.x >> (8 * q)) & 255u) * scale;
        v[4 + q] = (float)((w.y >> (8 * q)) & 255u) * scale;
      }
    } else if (dtype == 2) {
      const float4 a = reinterpret_cast<const float4*>((const float*)x + e0)[0];
      const float4 b = reinterpret_cast<const float4*>((const float*)x + e0)[1];
      v[0] = a.x * scale; v[1] = a.y * scale; v[2] = a.z * scale; v[3] = a.w * scale;
      v[4] = b.x * scale; v[5] = b.y * scale; v[6] = b.z * scale; v[7] = b.w * scale;
    } else {
      const uint4 w = *reinterpret_cast<const uint4*>((const __nv_bfloat16*)x + e0);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[2 * q] = __uint_as_float(ws[q] << 16) * scale;
        v[2 * q + 1] = __uint_as_float(ws[q] & 0xFFFF0000u) * scale;
      }
    }
    uint32_t o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
      memcpy(&o[q], &h, 4);
    }
    *reinterpret_cast<uint4*>(out + e0) = make_uint4(o[0], o[1], o[2], o[3]);
    return;
  }
  for (int64_t e = e0; e < e0 + 8 && e < n; ++e) {
    float f;
    if (dtype == 1)
      f = (float)((const uint8_t*)x)[e] * scale;
    else if (dtype == 2)
      f = ((const float*)x)[e] * scale;
    else
      f = __bfloat162float(((const __nv_bfloat16*)x)[e]) * scale;
    out[e] = __float2bfloat16_rn(f);
  }
}

// Tiled BF16 transpose: out[c][r] = in[r][c] for an R x C matrix.
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ in, int R, int C,
                                 __nv_bfloat16* __restrict__ out) {
  __shared__ __nv_bfloat16 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int r = r0 + dy, c = c0 + threadIdx.x;
    if (r < R && c < C) t[dy][threadIdx.x] = in[(int64_t)r * C + c];
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int c = c0 + dy, r = r0 + threadIdx.x;
    if (r < R && c < C) out[(int64_t)c * R + r] = t[threadIdx.x][dy];
  }
}

// y[b][j] = sum_i W3[j][i] h2[b][i] + b3[j], one warp per row: lane l takes the
// 8 consecutive elements 8 l + 256 t (16-byte loads of h2 and of both W3 rows;
// H % 16 == 0 and W3 sits at a multiple of 16 floats in the parameter vector),
// then the lanes are summed by a fixed butterfly.
__global__ void k_layer3(const __nv_bfloat16* __restrict__ h2, const float* __restrict__ W3,
                         const float* __restrict__ b3, int B, int H, float* __restrict__ y) {
  const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= B) return;
  float s0 = 0.f, s1 = 0.f;
  const __nv_bfloat16* hr = h2 + (int64_t)row * H;
  for (int i = lane * 8; i < H; i += 256) {
    const uint4 v = *reinterpret_cast<const uint4*>(hr + i);
    // W3 rows as 16-byte loads too: consecutive lanes read consecutive 32 bytes
    const float4* w0 = reinterpret_cast<const float4*>(W3 + i);
    const float4* w1 = reinterpret_cast<const float4*>(W3 + H + i);
    const float4 a0 = w0[0], a1 = w0[1], c0 = w1[0], c1 = w1[1];
    const float wa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float wc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __nv_bfloat162 p2;
      memcpy(&p2, &w[q], 4);
      const float2 f = __bfloat1622float2(p2);
      s0 = fmaf(wa[2 * q], f.x, s0);
      s0 = fmaf(wa[2 * q + 1], f.y, s0);
      s1 = fmaf(wc[2 * q], f.x, s1);
      s1 = fmaf(wc[2 * q + 1], f.y, s1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (lane == 0) {
    y[2 * (int64_t)row] = s0 + b3[0];
    y[2 * (int64_t)row + 1] = s1 + b3[1];
  }
}

// dY = 2 (Y - T) / B; per-block partial sums of |Y - T|^2 (grid-stride, fixed order).
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ y,
                                              const float* __restrict__ tgt, int B,
                                              float* __restrict__ dy, double* __restrict__ part) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * (int64_t)B;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[e] - tgt[e];
    dy[e] = 2.f * d / (float)B;
    acc += (double)d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// Column sums of chunk partials, out[q] = sum_c part[c * n + q], on blocks of
// (32, kSumWarps) threads: a block takes 32 columns (coalesced loads), warp w
// sums the chunks c = w, w + kSumWarps, ... in order, then thread (x, 0) adds
// the kSumWarps partial sums in order (a fixed order: deterministic).
constexpr int kSumWarps = 8;
__device__ __forceinline__ float chunk_col_sum(const float* __restrict__ part, int chunks, int n,
                                               int q) {
  __shared__ float sh[kSumWarps][33];
  float t = 0.f;
  if (q < n)
#pragma unroll 4
    for (int c = (int)threadIdx.y; c < chunks; c += kSumWarps) t += part[(int64_t)c * n + q];
  sh[threadIdx.y][threadIdx.x] = t;
  __syncthreads();
  float s = sh[0][threadIdx.x];
#pragma unroll
  for (int w = 1; w < kSumWarps; ++w) s += sh[w][threadIdx.x];
  return s;
}

// dW3 (2 x H) and db3 (2) from the chunk partials of k_grad3_part, and the
// batch loss from the per-block partials of k_loss (lane l sums partials l,
// l + 32, ... in order, then a fixed butterfly; divided by B).
__global__ void k_grad3_final(const float* __restrict__ part, int chunks, int H,
                              float* __restrict__ gW3, float* __restrict__ gb3,
                              const double* __restrict__ loss_part, int n_loss, int B,
                              double* __restrict__ loss_out) {
  const int q = blockIdx.x * 32 + threadIdx.x;
  const int n = 2 * (H + 1);
  const float t = chunk_col_sum(part, chunks, n, q);
  if (threadIdx.y == 0 && q < n) {
    const int j = q / (H + 1), i = q - j * (H + 1);
    if (i < H)
      gW3[(int64_t)j * H + i] = t;
    else
      gb3[j] = t;
  }
  if (blockIdx.x == 0 && threadIdx.y == 1) {
    double l = 0.0;
    for (int i = (int)threadIdx.x; i < n_loss; i += 32) l += loss_part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (threadIdx.x == 0) loss_out[0] = l / B;
  }
}

// Partials of dW3[j][i] = sum_b dY[b][j] h2[b][i] and db3[j] = sum_b dY[b][j] over
// chunks of kRowChunk rows: part[c][j][i] (i < H) and part[c][j][H] (bias).
__global__ void k_grad3_part(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ h2,
                             int B, int H, float* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i > H) return;
  const int r0 = c * kRowChunk, r1 = min(B, r0 + kRowChunk);
  float s0 = 0.f, s1 = 0.f;
#pragma unroll 8
  for (int b = r0; b < r1; ++b) {
    const float h = (i < H) ? __bfloat162float(h2[(int64_t)b * H + i]) : 1.f;
    s0 = fmaf(dy[2 * (int64_t)b], h, s0);
    s1 = fmaf(dy[2 * (int64_t)b + 1], h, s1);
  }
  part[((int64_t)c * 2 + 0) * (H + 1) + i] = s0;
  part[((int64_t)c * 2 + 1) * (H + 1) + i] = s1;
}

// Partials of the column sums of a B x H BF16 matrix over chunks of kRowChunk rows.
__global__ void k_colsum_part(const __nv_bfloat16* __restrict__ a, int B, int H,
                              float* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= H) return;
  const int r0 = c * kRowChunk, r1 = min(B, r0 + kRowChunk);
  float s = 0.f;
#pragma unroll 8
  for (int b = r0; b < r1; ++b) s += __bfloat162float(a[(int64_t)b * H + i]);
  part[(int64_t)c * H + i] = s;
}

// out[q] = sum over chunks c of part[c * n + q] (order of chunk_col_sum).
__global__ void k_chunk_sum(const float* __restrict__ part, int chunks, int n,
                            float* __restrict__ out) {
  const int q = blockIdx.x * 32 + threadIdx.x;
  const float t = chunk_col_sum(part, chunks, n, q);
  if (threadIdx.y == 0 && q < n) out[q] = t;
}

// dZ2 = (dY W3) * GELU'(z2) in BF16, written row-major (B x H) and transposed
// (H x B) for the weight-gradient GEMM: a 32 x 32 tile per block, staged in
// shared memory so that both stores are coalesced.
constexpr int kTile = 32;
__global__ void k_dz2(const float* __restrict__ dy, const float* __restrict__ W3,
                      const float* __restrict__ z2, int B, int H,
                      __nv_bfloat16* __restrict__ dz2, __nv_bfloat16* __restrict__ dz2t) {
  __shared__ __nv_bfloat16 t[kTile][kTile + 2];
  const int i0 = blockIdx.x * kTile, b0 = blockIdx.y * kTile;
  for (int r = threadIdx.y; r < kTile; r += blockDim.y) {
    const int b = b0 + r, i = i0 + threadIdx.x;
    if (b < B && i < H) {
      const int64_t e = (int64_t)b * H + i;
      const float dh = fmaf(dy[2 * (int64_t)b], W3[i], dy[2 * (int64_t)b + 1] * W3[H + i]);
      const __nv_bfloat16 v = __float2bfloat16_rn(dh * gelu_grad_dev(z2[e]));
      dz2[e] = v;
      t[r][threadIdx.x] = v;
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < kTile; r += blockDim.y) {
    const int i = i0 + r, b = b0 + threadIdx.x;
    if (b < B && i < H) dz2t[(int64_t)i * B + b] = t[threadIdx.x][r];
  }
}

// Bias gradient: column sums of a B x H BF16 matrix, chunk partials (in buf)
// then an ordered sum.
cudaError_t colsum(ivhd_mlp* P, const __nv_bfloat16* a, int B, int H, float* out, float* buf,
                   cudaStream_t s) {
  const int chunks = (B + kRowChunk - 1) / kRowChunk;
  k_colsum_part<<<dim3((unsigned)((H + 255) / 256), (unsigned)chunks), 256, 0, s>>>(a, B, H, buf);
  k_chunk_sum<<<(unsigned)((H + 31) / 32), dim3(32, kSumWarps), 0, s>>>(buf, chunks, H, out);
  P->launches += 2;
  return cudaGetLastError();
}

// Adam on the flat FP32 parameters (bias-corrected, Kingma and Ba).  The
// updated W1 and W2 are also written as the BF16 copies the tensor cores read
// (W1, W2 and the transposed W2), the same values refresh_copies would make.
// Given the split-K slices of the W1 and W2 gradients it adds them itself
// (slice order, as k_sum_slices does) instead of reading g there.
struct BF16Copies {
  int64_t w1_off, w2_off;  // offsets of W1 (H x n_in) and W2 (H x H) in the flat vector
  int n_in, H;
  __nv_bfloat16 *w1, *w2, *w2t;
  const float *s_w1, *s_w2;  // gradient slices [splits][H x n_in], [splits][H x H], or null
  int splits;
};
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int64_t n, float lr, float c1, float c2,
                       BF16Copies cp) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int64_t a = e - cp.w1_off, q = e - cp.w2_off;
  const int64_t n1 = (int64_t)cp.H * cp.n_in, n2 = (int64_t)cp.H * cp.H;
  const bool in1 = a >= 0 && a < n1, in2 = q >= 0 && q < n2;
  float gi;
  if (in1 && cp.s_w1) {
    gi = 0.f;
    for (int z = 0; z < cp.splits; ++z) gi += cp.s_w1[z * n1 + a];
  } else if (in2 && cp.s_w2) {
    gi = 0.f;
    for (int z = 0; z < cp.splits; ++z) gi += cp.s_w2[z * n2 + q];
  } else {
    gi = g[e];
  }
  const float mi = fmaf(0.9f, m[e], 0.1f * gi);
  const float vi = fmaf(0.999f, v[e], 0.001f * gi * gi);
  m[e] = mi;
  v[e] = vi;
  const float wn = w[e] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  w[e] = wn;
  if (in1) {
    cp.w1[a] = __float2bfloat16_rn(wn);
  } else if (in2) {
    const __nv_bfloat16 h = __float2bfloat16_rn(wn);
    cp.w2[q] = h;
    cp.w2t[(q % cp.H) * cp.H + q / cp.H] = h;
  }
}

__global__ void k_to_bf16(const float* __restrict__ a, int64_t n, __nv_bfloat16* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = __float2bfloat16_rn(a[e]);
}

cudaError_t transpose(const __nv_bfloat16* in, int R, int C, __nv_bfloat16* out, cudaStream_t s) {
  dim3 grid((unsigned)((C + 31) / 32), (unsigned)((R + 31) / 32)), block(32, 8);
  k_transpose_bf16<<<grid, block, 0, s>>>(in, R, C, out);
  return cudaGetLastError();
}

// BF16 copies of W1, W2 and the transposed W2 from the FP32 master.
cudaError_t refresh_copies(ivhd_mlp* P) {
  const Offs o = offsets(P->n_in, P->hidden);
  const int H = P->hidden;
  k_to_bf16<<<nb((int64_t)H * P->n_in), 256, 0, P->stream>>>(P->w + o.W1, (int64_t)H * P->n_in, P->w1);
  k_to_bf16<<<nb((int64_t)H * H), 256, 0, P->stream>>>(P->w + o.W2, (int64_t)H * H, P->w2);
  P->launches += 3;
  return transpose(P->w2, H, H, P->w2t, P->stream);
}

// Forward pass of B rows already in P->xb: h1, h2, y, and for training also
// the pre-activations z1, z2 (GELU' of the backward pass reads them) and h1
// transposed (the weight gradient's operand).
cudaError_t forward(ivhd_mlp* P, int B, bool train = false) {
  const Offs o = offsets(P->n_in, P->hidden);
  const int H = P->hidden;
  P->last_rows = B;
  GemmEpilogue e1{kEpBiasGelu, H, train ? P->z1 : nullptr, P->h1, P->w + o.b1, nullptr, 0};
  if (train) {
    e1.out_bf16_t = P->h1t;
    e1.ld_t = B;
  }
  cudaError_t e = gemm_bf16_tn(P->xb, P->n_in, P->w1, P->n_in, B, H, P->n_in, e1, P->err, P->stream);
  GemmEpilogue e2{kEpBiasGelu, H, train ? P->z2 : nullptr, P->h2, P->w + o.b2, nullptr, 0};
  if (e == cudaSuccess) e = gemm_bf16_tn(P->h1, H, P->w2, H, B, H, H, e2, P->err, P->stream);
  if (e == cudaSuccess) {
    k_layer3<<<nb((int64_t)B * 32), 256, 0, P->stream>>>(P->h2, P->w + o.W3, P->w + o.b3, B, H, P->y);
    e = cudaGetLastError();
  }
  P->launches += 3;
  return e;
}

// Loss and gradients of B rows (inputs in P->xb, targets tgt) into P->g.
// With sum_weights false the split-K slices of dW1 (P->part) and dW2
// (P->part2) are left for k_adam to add, in the same order.
// The transposed input, the output-layer gradient and the bias gradients run
// on the side stream beside the GEMMs; the side stream's work is joined before
// returning.
cudaError_t loss_grad(ivhd_mlp* P, const float* tgt, int B, bool sum_weights = true) {
  const Offs o = offsets(P->n_in, P->hidden);
  const int H = P->hidden, n_in = P->n_in;
  cudaStream_t s = P->stream, side = P->side;
  cudaError_t e = cudaEventRecord(P->ev[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side, P->ev[0], 0);
  if (e == cudaSuccess) e = transpose(P->xb, B, n_in, P->xt, side);  // X^T for dW1
  if (e == cudaSuccess) e = cudaEventRecord(P->ev[1], side);
  ++P->launches;
  if (e == cudaSuccess) e = forward(P, B, true);
  if (e != cudaSuccess) return e;
  k_loss<<<kLossBlocks, 256, 0, s>>>(P->y, tgt, B, P->dy, P->loss_part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaEventRecord(P->ev[5], s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(side, P->ev[5], 0)) != cudaSuccess) return e;
  {
    // dW3 (2 x H) and db3 (2): rows [j][0..H) of the (2, H + 1) chunk sums, bias in column H
    const int chunks = (B + kRowChunk - 1) / kRowChunk;
    k_grad3_part<<<dim3(nb(H + 1), (unsigned)chunks), 256, 0, side>>>(P->dy, P->h2, B, H,
                                                                       P->g3_part);
    k_grad3_final<<<(unsigned)((2 * (H + 1) + 31) / 32), dim3(32, kSumWarps), 0, side>>>(
        P->g3_part, chunks, H, P->g + o.W3, P->g + o.b3, P->loss_part, kLossBlocks, B,
        P->loss_out);
  }
  k_dz2<<<dim3((unsigned)((H + kTile - 1) / kTile), (unsigned)((B + kTile - 1) / kTile)),
          dim3(kTile, 8), 0, s>>>(P->dy, P->w + o.W3, P->z2, B, H, P->dz2, P->dz2t);
  P->launches += 4;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaEventRecord(P->ev[2], s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(side, P->ev[2], 0)) != cudaSuccess) return e;
  if ((e = colsum(P, P->dz2, B, H, P->g + o.b2, P->cs_part, side)) != cudaSuccess) return e;
  // dW2 = dZ2^T H1 (dZ2^T from k_dz2, H1^T from the forward pass)
  GemmEpilogue gw2{kEpStoreF32, H, P->part2, nullptr, nullptr, nullptr, (int64_t)H * H};
  if ((e = gemm_bf16_tn(P->dz2t, B, P->h1t, B, H, H, B, gw2, P->err, s, kSplitK)) != cudaSuccess)
    return e;
  if (sum_weights &&
      (e = sum_slices(P->part2, (int64_t)H * H, (int64_t)H * H, kSplitK, P->g + o.W2, s)) !=
          cudaSuccess)
    return e;
  // dZ1 = (dZ2 W2) * GELU'(z1), also written transposed
  GemmEpilogue gz1{kEpGeluGrad, H, nullptr, P->dz1, nullptr, P->z1, 0};
  gz1.out_bf16_t = P->dz1t;
  gz1.ld_t = B;
  if ((e = gemm_bf16_tn(P->dz2, H, P->w2t, H, B, H, H, gz1, P->err, s)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(P->ev[3], s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(side, P->ev[3], 0)) != cudaSuccess) return e;
  if ((e = colsum(P, P->dz1, B, H, P->g + o.b1, P->cs_part, side)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(P->ev[4], side)) != cudaSuccess) return e;
  // dW1 = dZ1^T X
  if ((e = cudaStreamWaitEvent(s, P->ev[1], 0)) != cudaSuccess) return e;
  GemmEpilogue gw1{kEpStoreF32, n_in, P->part, nullptr, nullptr, nullptr, (int64_t)H * n_in};
  if ((e = gemm_bf16_tn(P->dz1t, B, P->xt, B, H, n_in, B, gw1, P->err, s, kSplitK)) != cudaSuccess)
    return e;
  if (sum_weights) {
    e = sum_slices(P->part, (int64_t)H * n_in, (int64_t)H * n_in, kSplitK, P->g + o.W1, s);
    P->launches += 2;
  }
  P->launches += 3;  // the three GEMMs
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, P->ev[4], 0);  // join the side stream
  return e;
}

cudaError_t load_x(ivhd_mlp* P, const void* x, int dtype, float scale, int64_t rows) {
  const int64_t n = rows * P->n_in;
  k_convert_x<<<nb((n + 7) / 8), 256, 0, P->stream>>>(x, dtype, scale, n, P->xb);
  ++P->launches;
  return cudaGetLastError();
}

ivhd_status mlp_fail(ivhd_mlp* P, cudaError_t e) {
  if (e == cudaSuccess) return IVHD_OK;
  if (e == cudaErrorMemoryAllocation) return IVHD_ERR_OOM;
  if (e == cudaErrorInvalidValue) return IVHD_ERR_ARG;
  P->poisoned = true;
  return IVHD_ERR_CUDA;
}

// Timeouts of the GEMM's bounded waits, read back (synchronises).
ivhd_status check_err(ivhd_mlp* P) {
  int32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, P->err, sizeof(h), cudaMemcpyDeviceToHost, P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return mlp_fail(P, e);
  if (h) {
    P->poisoned = true;
    return IVHD_ERR_TIMEOUT;
  }
  return IVHD_OK;
}

bool batch_ok(const ivhd_mlp* P, int64_t B) { return B >= 8 && B <= P->max_batch && B % 8 == 0; }

// One Adam step: load the batch, loss and gradients, update, refresh the BF16
// weight copies.
cudaError_t train_step_direct(ivhd_mlp* P, const void* x, int dtype, float scale,
                              const float* targets, int B, float lr, float c1, float c2) {
  cudaError_t e = load_x(P, x, dtype, scale, B);
  if (e == cudaSuccess) e = loss_grad(P, targets, B, false);
  if (e == cudaSuccess) {
    const Offs o = offsets(P->n_in, P->hidden);
    const BF16Copies cp{o.W1,   o.W2,    P->n_in,  P->hidden, P->w1,
                        P->w2,  P->w2t,  P->part,  P->part2,  kSplitK};
    k_adam<<<nb(P->n_params), 256, 0, P->stream>>>(P->w, P->m, P->v, P->g, P->n_params, lr, c1,
                                                   c2, cp);
    ++P->launches;
    e = cudaGetLastError();
  }
  return e;
}

// Captures train_step_direct for batch size B on a private stream and keeps
// the handles of the three kernel nodes whose arguments change per call.
cudaError_t capture_train_step(ivhd_mlp* P, int B) {
  if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->graph_exec = nullptr;
  P->graph = nullptr;
  P->graph_B = 0;
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaStream_t saved = P->stream;
  const int64_t launches0 = P->launches;
  P->stream = cap;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    // placeholder inputs: the patched nodes get the real ones at every replay
    cudaError_t e1 = train_step_direct(P, P->xb, 0, 1.f, P->y, B, 1e-3f, 1.f, 1.f);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    e = e1 != cudaSuccess ? e1 : e2;
    if (e == cudaSuccess) P->graph = g;
    else if (g) cudaGraphDestroy(g);
  }
  P->stream = saved;
  P->graph_launches = P->launches - launches0;
  P->launches = launches0;
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return e;
  size_t n = 0;
  e = cudaGraphGetNodes(P->graph, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  if (e == cudaSuccess && n) e = cudaGraphGetNodes(P->graph, nodes.data(), &n);
  for (size_t q = 0; q < n && e == cudaSuccess; ++q) {
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(nodes[q], &t);
    if (e != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp{};
    e = cudaGraphKernelNodeGetParams(nodes[q], &kp);
    if (e != cudaSuccess) break;
    if (kp.func == (void*)k_convert_x) {
      P->node_x = nodes[q];
      P->kp_x = kp;
    } else if (kp.func == (void*)k_loss) {
      P->node_loss = nodes[q];
      P->kp_loss = kp;
    } else if (kp.func == (void*)k_adam) {
      P->node_adam = nodes[q];
      P->kp_adam = kp;
    }
  }
  if (e == cudaSuccess && (!P->node_x || !P->node_loss || !P->node_adam))
    e = cudaErrorInvalidValue;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&P->graph_exec, P->graph, 0);
  if (e == cudaSuccess) P->graph_B = B;
  return e;
}

// Replays the captured step with this call's inputs, targets and learning rate.
cudaError_t replay_train_step(ivhd_mlp* P, const void* x, int dtype, float scale,
                              const float* targets, int B, float lr, float c1, float c2) {
  int64_t n_x = (int64_t)B * P->n_in;
  __nv_bfloat16* xb = P->xb;
  void* ax[] = {(void*)&x, (void*)&dtype, (void*)&scale, (void*)&n_x, (void*)&xb};
  cudaKernelNodeParams kx = P->kp_x;
  kx.kernelParams = ax;
  kx.extra = nullptr;
  float* y = P->y;
  float* dy = P->dy;
  double* part = P->loss_part;
  void* al[] = {(void*)&y, (void*)&targets, (void*)&B, (void*)&dy, (void*)&part};
  cudaKernelNodeParams kl = P->kp_loss;
  kl.kernelParams = al;
  kl.extra = nullptr;
  float *w = P->w, *m = P->m, *v = P->v;
  const float* g = P->g;
  int64_t np = P->n_params;
  const Offs o = offsets(P->n_in, P->hidden);
  BF16Copies cp{o.W1, o.W2, P->n_in, P->hidden, P->w1, P->w2, P->w2t, P->part, P->part2,
                kSplitK};
  void* aa[] = {(void*)&w, (void*)&m, (void*)&v, (void*)&g, (void*)&np, (void*)&lr, (void*)&c1,
                (void*)&c2, (void*)&cp};
  cudaKernelNodeParams ka = P->kp_adam;
  ka.kernelParams = aa;
  ka.extra = nullptr;
  cudaError_t e = cudaGraphExecKernelNodeSetParams(P->graph_exec, P->node_x, &kx);
  if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(P->graph_exec, P->node_loss, &kl);
  if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(P->graph_exec, P->node_adam, &ka);
  if (e == cudaSuccess) e = cudaGraphLaunch(P->graph_exec, P->stream);
  if (e == cudaSuccess) P->launches += P->graph_launches;
  return e;
}

}  // namespace
}  // namespace ivhd

using namespace ivhd;

extern "C" {

ivhd_status ivhd_mlp_create(int32_t n_in, int32_t hidden, int32_t max_batch, void* stream,
                            ivhd_mlp** out) {
  if (!out) return IVHD_ERR_ARG;
  *out = nullptr;
  if (n_in < 8 || n_in % 8 || n_in > 65536 || hidden < 16 || hidden % 16 || hidden > 4096 ||
      max_batch < 8 || max_batch % 8 || max_batch > (1 << 20))
    return IVHD_ERR_ARG;
  ivhd_mlp* P = new (std::nothrow) ivhd_mlp();
  if (!P) return IVHD_ERR_OOM;
  P->n_in = n_in;
  P->hidden = hidden;
  P->max_batch = max_batch;
  P->stream = (cudaStream_t)stream;
  const Offs o = offsets(n_in, hidden);
  P->n_params = o.total;
  const int64_t B = max_batch, H = hidden;
  cudaStream_t s = P->stream;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, int64_t n) {
    if (e == cudaSuccess) e = dev_alloc((void**)p, (size_t)n * sizeof(**p), s);
  };
  A(&P->w, o.total);
  A(&P->m, o.total);
  A(&P->v, o.total);
  A(&P->g, o.total);
  A(&P->w1, H * n_in);
  A(&P->w2, H * H);
  A(&P->w2t, H * H);
  A(&P->xb, B * n_in);
  A(&P->xt, B * n_in);
  A(&P->z1, B * H);
  A(&P->z2, B * H);
  A(&P->h1, B * H);
  A(&P->h1t, B * H);
  A(&P->h2, B * H);
  A(&P->dz2, B * H);
  A(&P->dz2t, B * H);
  A(&P->dz1, B * H);
  A(&P->dz1t, B * H);
  A(&P->y, 2 * B);
  A(&P->dy, 2 * B);
  {
    // split-K slices of the largest weight gradient, or the batch-chunk partials
    const int64_t chunks = (B + kRowChunk - 1) / kRowChunk;
    const int64_t wide = H > n_in ? H : n_in;
    const int64_t a1 = (int64_t)kSplitK * H * wide, a2 = (chunks + 1) * 2 * (H + 1);
    A(&P->part, a1 > a2 ? a1 : a2);
    A(&P->part2, (int64_t)kSplitK * H * H);
    A(&P->cs_part, chunks * H);
    A(&P->g3_part, chunks * 2 * (H + 1));
  }
  A(&P->loss_part, kLossBlocks);
  A(&P->loss_out, 1);
  A(&P->err, 1);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking);
  for (cudaEvent_t& ev : P->ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->w, 0, o.total * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->m, 0, o.total * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->v, 0, o.total * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->err, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = refresh_copies(P);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ivhd_mlp_destroy(P);
    return e == cudaErrorMemoryAllocation ? IVHD_ERR_OOM : IVHD_ERR_CUDA;
  }
  *out = P;
  return IVHD_OK;
}

void ivhd_mlp_destroy(ivhd_mlp* P) {
  if (!P) return;
  if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  void* bufs[] = {P->w, P->m, P->v, P->g, P->w1, P->w2, P->w2t, P->xb, P->xt, P->z1, P->z2,
                  P->h1, P->h1t, P->h2, P->dz2, P->dz2t, P->dz1, P->dz1t, P->y, P->dy,
                  P->part, P->part2, P->cs_part, P->g3_part, P->loss_part, P->loss_out, P->err};
  for (void* b : bufs)
    if (b) dev_free(b, P->stream);
  cudaStreamSynchronize(P->stream);
  for (cudaEvent_t ev : P->ev)
    if (ev) cudaEventDestroy(ev);
  if (P->side) cudaStreamDestroy(P->side);
  delete P;
}

int64_t ivhd_mlp_num_params(ivhd_mlp* P) { return P ? P->n_params : -1; }

ivhd_status ivhd_mlp_set_params(ivhd_mlp* P, const float* params, int32_t on_device) {
  if (!P || !params) return IVHD_ERR_ARG;
  if (P->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = P->stream;
  const size_t bytes = (size_t)P->n_params * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(P->w, params, bytes,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->m, 0, bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->v, 0, bytes, s);
  if (e == cudaSuccess) e = refresh_copies(P);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  P->t = 0;
  return mlp_fail(P, e);
}

ivhd_status ivhd_mlp_get_params(ivhd_mlp* P, float* params, int32_t on_device) {
  if (!P || !params) return IVHD_ERR_ARG;
  if (P->poisoned) return IVHD_ERR_STATE;
  cudaError_t e = cudaMemcpyAsync(params, P->w, (size_t)P->n_params * sizeof(float),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  P->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(P->stream);
  return mlp_fail(P, e);
}

ivhd_status ivhd_mlp_loss_grad(ivhd_mlp* P, const void* x, int32_t x_dtype, float x_scale,
                               const float* targets, int32_t B, double* loss, float* grads) {
  NvtxScope nvtx_("ivhd_mlp_loss_grad");
  if (!P || !x || !targets || x_dtype < 0 || x_dtype > 2 || !batch_ok(P, B)) return IVHD_ERR_ARG;
  if (P->poisoned) return IVHD_ERR_STATE;
  cudaError_t e = load_x(P, x, x_dtype, x_scale, B);
  if (e == cudaSuccess) e = loss_grad(P, targets, B);
  if (e == cudaSuccess && grads)
    e = cudaMemcpyAsync(grads, P->g, (size_t)P->n_params * sizeof(float), cudaMemcpyDeviceToDevice,
                        P->stream);
  if (e == cudaSuccess && loss)
    e = cudaMemcpyAsync(loss, P->loss_out, sizeof(double), cudaMemcpyDeviceToHost, P->stream);
  if (e != cudaSuccess) return mlp_fail(P, e);
  return check_err(P);
}

ivhd_status ivhd_mlp_train_step(ivhd_mlp* P, const void* x, int32_t x_dtype, float x_scale,
                                const float* targets, int32_t B, float lr, double* loss) {
  NvtxScope nvtx_("ivhd_mlp_train_step");
  if (!P || !x || !targets || x_dtype < 0 || x_dtype > 2 || !batch_ok(P, B) || !(lr > 0.f))
    return IVHD_ERR_ARG;
  if (P->poisoned) return IVHD_ERR_STATE;
  P->t += 1;
  const float c1 = 1.f - powf(0.9f, (float)P->t), c2 = 1.f - powf(0.999f, (float)P->t);
  cudaError_t e = cudaSuccess;
  if (P->graph_B != B && P->direct_B == B) e = capture_train_step(P, B);
  if (e != cudaSuccess) return mlp_fail(P, e);
  if (P->graph_B == B) {
    e = replay_train_step(P, x, x_dtype, x_scale, targets, B, lr, c1, c2);
  } else {
    // first step at this batch size: run directly (the next one captures it)
    e = train_step_direct(P, x, x_dtype, x_scale, targets, B, lr, c1, c2);
    P->direct_B = B;
  }
  if (e == cudaSuccess && loss)
    e = cudaMemcpyAsync(loss, P->loss_out, sizeof(double), cudaMemcpyDeviceToHost, P->stream);
  if (e != cudaSuccess) return mlp_fail(P, e);
  return loss ? check_err(P) : IVHD_OK;
}

ivhd_status ivhd_mlp_forward(ivhd_mlp* P, const void* x, int32_t x_dtype, float x_scale,
                             int64_t n, float* y) {
  NvtxScope nvtx_("ivhd_mlp_forward");
  if (!P || !x || !y || x_dtype < 0 || x_dtype > 2 || n < 1) return IVHD_ERR_ARG;
  if (P->poisoned) return IVHD_ERR_STATE;
  const size_t esz = x_dtype == 1 ? 1 : (x_dtype == 2 ? 4 : 2);
  cudaError_t e = cudaSuccess;
  for (int64_t r0 = 0; r0 < n && e == cudaSuccess; r0 += P->max_batch) {
    const int64_t rows = (n - r0 < P->max_batch) ? n - r0 : P->max_batch;
    e = load_x(P, (const char*)x + (size_t)r0 * P->n_in * esz, x_dtype, x_scale, rows);
    if (e == cudaSuccess) e = forward(P, (int)rows);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(y + 2 * r0, P->y, (size_t)rows * 2 * sizeof(float),
                          cudaMemcpyDeviceToDevice, P->stream);
  }
  if (e != cudaSuccess) return mlp_fail(P, e);
  return check_err(P);
}

int64_t ivhd_mlp_launches(ivhd_mlp* P) { return P ? P->launches : -1; }

ivhd_status ivhd_mlp_activations(ivhd_mlp* P, int32_t which, void* out, int64_t* rows) {
  if (!P || !out || !rows) return IVHD_ERR_ARG;
  if (P->poisoned) return IVHD_ERR_STATE;
  const int64_t B = P->last_rows, H = P->hidden;
  const void* src = nullptr;
  size_t bytes = 0;
  switch (which) {
    case IVHD_MLP_X: src = P->xb; bytes = (size_t)(B * P->n_in) * 2; break;
    case IVHD_MLP_Z1: src = P->z1; bytes = (size_t)(B * H) * 4; break;
    case IVHD_MLP_H1: src = P->h1; bytes = (size_t)(B * H) * 2; break;
    case IVHD_MLP_Z2: src = P->z2; bytes = (size_t)(B * H) * 4; break;
    case IVHD_MLP_H2: src = P->h2; bytes = (size_t)(B * H) * 2; break;
    case IVHD_MLP_Y: src = P->y; bytes = (size_t)(B * 2) * 4; break;
    case IVHD_MLP_DY: src = P->dy; bytes = (size_t)(B * 2) * 4; break;
    case IVHD_MLP_DZ2: src = P->dz2; bytes = (size_t)(B * H) * 2; break;
    case IVHD_MLP_DZ1: src = P->dz1; bytes = (size_t)(B * H) * 2; break;
    default: return IVHD_ERR_ARG;
  }
  *rows = B;
  if (B == 0) return IVHD_OK;
  cudaError_t e = cudaMemcpyAsync(out, src, bytes, cudaMemcpyDefault, P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  return mlp_fail(P, e);
}

}  // extern "C"
