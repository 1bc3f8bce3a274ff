// ivhd_step.cu -- the hot path: one fused gather-force + optimiser-update pass.
//
// For every vertex i (Sec. 3.3.1, Eq. 3.14 with F = -1/2 grad E of Eq. 3.16):
//
//     F_i = sum_{j in nn_sym(i)} (y_j - y_i)
//         + c * sum_{k in rn_sym(i)} (1 - 1/d_ik) (y_k - y_i),   d_ik = |y_k - y_i|
//
// where nn_sym / rn_sym are the symmetrised neighbour multisets (every term of
// the stress acts on both of its endpoints), followed in the same thread by
// the optimiser update of Eq. 3.34 (momentum), or the Nesterov / Adadelta
// forms of Sec. 3.3.2.  All forces of a step read y_in and all updates write
// y_out (ping-pong), which is the synchronous scheme of the IVHD-CUDA
// algorithm in Sec. 5.2 without its per-connection +/- slots and second pass:
// each vertex gathers its neighbours' positions instead, so there are no
// atomics and the summation order is fixed by the layout (deterministic).
//
// Work split: SELL slices of 32 degree-sorted vertices, one thread per vertex
// and one coalesced int4 id load per 4 neighbours; vertices of very high
// degree ("hubs") get a warp each and a fixed-order butterfly reduction.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ivhd_internal.cuh"

namespace ivhd {

// Position of vertex idx as the neighbours see it: the FP32 array, or the
// rounded FP16 / BF16 copy (one 32-bit word per vertex).
template <int POS>
__device__ __forceinline__ float2 load_pos(const StepArgs& A, uint32_t idx) {
  if constexpr (POS == IVHD_POS_F32) {
    return __ldg(A.y_in + idx);
  } else {
    const uint32_t w = __ldg(A.yh_in + idx);
    if constexpr (POS == IVHD_POS_F16) {
      __half2 h;
      memcpy(&h, &w, 4);
      return __half22float2(h);
    } else {
      __nv_bfloat162 h;
      memcpy(&h, &w, 4);
      return __bfloat1622float2(h);
    }
  }
}

// Round-to-nearest-even copy of a position in the gathered format.
template <int POS>
__device__ __forceinline__ uint32_t round_pos(float2 v) {
  uint32_t w = 0;
  if constexpr (POS == IVHD_POS_F16) {
    const __half2 h = __floats2half2_rn(v.x, v.y);
    memcpy(&w, &h, 4);
  } else if constexpr (POS == IVHD_POS_BF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    memcpy(&w, &h, 4);
  }
  return w;
}

template <int POS>
__device__ __forceinline__ float2 gather(const StepArgs& A, uint32_t e, float2 self) {
  return (e == kPad) ? self : load_pos<POS>(A, e & kIdxMask);
}

// One term of the force on i.  nn: w = 1, or 2 for a mutual pair kept with
// multiplicity.  rn: w = c (1 - 1/d); w = 0 at d = 0.  Padding entries carry
// the rn bit and gather y_i itself, so d = 0, w = 0.
__device__ __forceinline__ void force_term(uint32_t e, float2 yj, float2 yi, float c, float& fx,
                                           float& fy) {
  const float ux = yj.x - yi.x;
  const float uy = yj.y - yi.y;
  float w = (e & kW2Bit) ? 2.f : 1.f;
  if (e & kRnBit) {
    const float d2 = fmaf(uy, uy, ux * ux);
    w = (d2 > 0.f) ? c * (1.f - rsqrtf(d2)) : 0.f;
  }
  fx = fmaf(w, ux, fx);
  fy = fmaf(w, uy, fy);
}

// One term of the stress: nn w d^2 (w = 1 or 2), rn c (1 - d)^2; padding contributes nothing.
__device__ __forceinline__ void stress_term(uint32_t e, float2 yj, float2 yi, float c, float& es) {
  if (e == kPad) return;
  const float ux = yj.x - yi.x;
  const float uy = yj.y - yi.y;
  const float d2 = fmaf(uy, uy, ux * ux);
  if (e & kRnBit) {
    const float t = 1.f - sqrtf(d2);
    es = fmaf(c * t, t, es);
  } else {
    es = fmaf((e & kW2Bit) ? 2.f : 1.f, d2, es);
  }
}

template <int MODE, int POS>
__device__ __forceinline__ void visit4(const int4 e, const StepArgs& A, float2 yi, float c,
                                       float& fx, float& fy) {
  const uint32_t e0 = (uint32_t)e.x, e1 = (uint32_t)e.y, e2 = (uint32_t)e.z, e3 = (uint32_t)e.w;
  const float2 g0 = gather<POS>(A, e0, yi), g1 = gather<POS>(A, e1, yi);
  const float2 g2 = gather<POS>(A, e2, yi), g3 = gather<POS>(A, e3, yi);
  if (MODE == kStress) {
    stress_term(e0, g0, yi, c, fx);
    stress_term(e1, g1, yi, c, fx);
    stress_term(e2, g2, yi, c, fx);
    stress_term(e3, g3, yi, c, fx);
  } else {
    force_term(e0, g0, yi, c, fx, fy);
    force_term(e1, g1, yi, c, fx, fy);
    force_term(e2, g2, yi, c, fx, fy);
    force_term(e3, g3, yi, c, fx, fy);
  }
}

template <int MODE, int POS>
__device__ __forceinline__ void visit8(const int4 ea, const int4 eb, const StepArgs& A, float2 yi,
                                       float c, float& fx, float& fy) {
  // all eight gathers are issued before any arithmetic (eight loads in flight per thread)
  const uint32_t e[8] = {(uint32_t)ea.x, (uint32_t)ea.y, (uint32_t)ea.z, (uint32_t)ea.w,
                         (uint32_t)eb.x, (uint32_t)eb.y, (uint32_t)eb.z, (uint32_t)eb.w};
  float2 g[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) g[q] = gather<POS>(A, e[q], yi);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (MODE == kStress)
      stress_term(e[q], g[q], yi, c, fx);
    else
      force_term(e[q], g[q], yi, c, fx, fy);
  }
}

#ifndef IVHD_STEP_MIN_BLOCKS
#define IVHD_STEP_MIN_BLOCKS 1
#endif

// MODE: optimiser epilogue (or forces / stress); POS: gathered position format.
// yi is the vertex's own position in the gathered format (differences are taken
// between equally rounded positions); ym is its FP32 master position.
template <int MODE, int POS>
__global__ void __launch_bounds__(kStepBlock, IVHD_STEP_MIN_BLOCKS) k_step(const StepArgs A) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float fx = 0.f, fy = 0.f;  // force, or (stress in fx)
  float2 yi = make_float2(0.f, 0.f);
  float2 ym = make_float2(0.f, 0.f);
  int p = -1;
  bool own = false;

  if ((int)blockIdx.x < A.nb_hub) {
    // hub rows: one warp per vertex, lanes stride over int4 groups
    p = (int)blockIdx.x * kWarpsPerBlock + wib;
    if (p < A.n_hub) {
      ym = A.y_in[p];
      yi = (POS == IVHD_POS_F32) ? ym : load_pos<POS>(A, p);
      const int beg = A.hub_off[p], end = A.hub_off[p + 1];
      const int4* row = reinterpret_cast<const int4*>(A.ids + beg);
      const int ng = (end - beg) >> 2;
      int g = lane;
      for (; g + 32 < ng; g += 64) {
        const int4 ea = ld_stream_v4(row + g);
        const int4 eb = ld_stream_v4(row + g + 32);
        visit8<MODE, POS>(ea, eb, A, yi, A.c, fx, fy);
      }
      if (g < ng) visit4<MODE, POS>(ld_stream_v4(row + g), A, yi, A.c, fx, fy);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
      }
      own = (lane == 0);
    }
  } else {
    // SELL slice: one thread per vertex, one coalesced int4 per 4 neighbours
    const int s = ((int)blockIdx.x - A.nb_hub) * kWarpsPerBlock + wib;
    if (s < A.n_slices) {
      p = A.n_hub + s * 32 + lane;
      const bool valid = p < A.M;
      if (valid) {
        ym = A.y_in[p];
        yi = (POS == IVHD_POS_F32) ? ym : load_pos<POS>(A, p);
      }
      const int4* base = reinterpret_cast<const int4*>(A.ids + A.slice_off[s]) + lane;
      const int W = A.slice_w[s];
      int g = 0;
      for (; g + 1 < W; g += 2) {
        const int4 ea = ld_stream_v4(base + g * 32);
        const int4 eb = ld_stream_v4(base + (g + 1) * 32);
        visit8<MODE, POS>(ea, eb, A, yi, A.c, fx, fy);
      }
      if (g < W) visit4<MODE, POS>(ld_stream_v4(base + g * 32), A, yi, A.c, fx, fy);
      own = valid;
    }
  }

  if (MODE == kMomentum) {
    // Eq. 3.34: v <- a v + b F ; y <- y + v
    if (own) {
      float2 v = A.s1[p];
      v.x = fmaf(A.a, v.x, A.b * fx);
      v.y = fmaf(A.a, v.y, A.b * fy);
      A.s1[p] = v;
      const float2 yn = make_float2(ym.x + v.x, ym.y + v.y);
      A.y_out[p] = yn;
      if (POS != IVHD_POS_F32) A.yh_out[p] = round_pos<POS>(yn);
    }
  } else if (MODE == kNesterov) {
    // state is the look-ahead point z = y + a v; F was taken at z.
    // v' = a v + b F(z);  y' = y + v';  z' = y' + a v' = z - a v + (1 + a) v'
    if (own) {
      const float2 v = A.s1[p];
      float2 vn;
      vn.x = fmaf(A.a, v.x, A.b * fx);
      vn.y = fmaf(A.a, v.y, A.b * fy);
      A.s1[p] = vn;
      const float ap1 = 1.f + A.a;
      const float2 zn =
          make_float2(ym.x + fmaf(ap1, vn.x, -A.a * v.x), ym.y + fmaf(ap1, vn.y, -A.a * v.y));
      A.y_out[p] = zn;
      if (POS != IVHD_POS_F32) A.yh_out[p] = round_pos<POS>(zn);
    }
  } else if (MODE == kAdadelta) {
    // Zeiler's Adadelta on g = -F: E[g^2] <- rho E[g^2] + (1-rho) g^2;
    // dx = -sqrt(E[dx^2] + eps) / sqrt(E[g^2] + eps) g; E[dx^2] <- rho E[dx^2] + (1-rho) dx^2
    if (own) {
      float2 eg = A.s1[p];
      float2 ex = A.s2[p];
      const float omr = 1.f - A.rho;
      const float gx = -fx, gy = -fy;
      eg.x = fmaf(A.rho, eg.x, omr * gx * gx);
      eg.y = fmaf(A.rho, eg.y, omr * gy * gy);
      const float dx = -(sqrtf(ex.x + A.eps) / sqrtf(eg.x + A.eps)) * gx;
      const float dy = -(sqrtf(ex.y + A.eps) / sqrtf(eg.y + A.eps)) * gy;
      ex.x = fmaf(A.rho, ex.x, omr * dx * dx);
      ex.y = fmaf(A.rho, ex.y, omr * dy * dy);
      A.s1[p] = eg;
      A.s2[p] = ex;
      const float2 yn = make_float2(ym.x + dx, ym.y + dy);
      A.y_out[p] = yn;
      if (POS != IVHD_POS_F32) A.yh_out[p] = round_pos<POS>(yn);
    }
  } else if (MODE == kForces) {
    if (own) A.f_out[A.perm[p]] = make_float2(fx, fy);
  } else if (MODE == kStress) {
    __shared__ double red[kWarpsPerBlock];
    double v = own ? (double)fx : 0.0;
    if (own && !(isfinite(ym.x) && isfinite(ym.y))) atomicOr(A.flag, 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wib] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kWarpsPerBlock; ++w) t += red[w];
      A.partials[blockIdx.x] = t;
    }
  }
}

// Sums the per-block partials in a fixed order; E = 1/2 of the symmetric sum
// because every term of Eq. 3.16 appears in the rows of both endpoints.
__global__ void __launch_bounds__(1024) k_stress_final(const double* __restrict__ partials, int n,
                                                       double* out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partials[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    out[0] = 0.5 * t;
  }
}

// Positions in input order; for Nesterov the stored point is z = y + a v.
__global__ void k_unpermute(const float2* __restrict__ y, const float2* __restrict__ v,
                            const int32_t* __restrict__ perm, int M, float a, int nesterov,
                            float2* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= M) return;
  float2 q = y[p];
  if (nesterov) {
    const float2 w = v[p];
    q.x = fmaf(-a, w.x, q.x);
    q.y = fmaf(-a, w.y, q.y);
  }
  out[perm[p]] = q;
}

// Rounded copy of the FP32 positions in the gathered format.
__global__ void k_round_positions(const float2* __restrict__ y, int M, int pos,
                                  uint32_t* __restrict__ yh) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= M) return;
  yh[p] = (pos == IVHD_POS_F16) ? round_pos<IVHD_POS_F16>(y[p]) : round_pos<IVHD_POS_BF16>(y[p]);
}

cudaError_t launch_round_positions(ivhd_ctx* ctx) {
  if (ctx->p.pos_format == IVHD_POS_F32) return cudaSuccess;
  const int M = (int)ctx->M;
  k_round_positions<<<(M + 255) / 256, 256, 0, ctx->stream>>>(ctx->y[ctx->cur], M, ctx->p.pos_format,
                                                              ctx->yh[ctx->cur]);
  ++ctx->aux_launches;
  return cudaGetLastError();
}

// Positions from input order; optimiser state reset to zero (so z = y for Nesterov).
__global__ void k_set_positions(const float2* __restrict__ in, const int32_t* __restrict__ perm,
                                int M, float2* __restrict__ y, float2* __restrict__ s1,
                                float2* __restrict__ s2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= M) return;
  y[p] = in[perm[p]];
  s1[p] = make_float2(0.f, 0.f);
  if (s2) s2[p] = make_float2(0.f, 0.f);
}

// y0 ~ U(0,1)^2 per input vertex i = perm[p]: coordinate q is the top 24 bits
// of output q of SplitMix64 seeded with s_i = output i of SplitMix64 seeded
// with (seed ^ "init_pos"), times 2^-24 (exact in FP32).
__global__ void k_init_positions(const int32_t* __restrict__ perm, int M, uint64_t seed,
                                 float2* __restrict__ y, float2* __restrict__ s1,
                                 float2* __restrict__ s2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= M) return;
  const uint64_t si = sm64_out(seed ^ kDomainInit, (uint64_t)perm[p]);
  const float sc = 1.0f / 16777216.0f;
  y[p] = make_float2((float)(sm64_out(si, 0) >> 40) * sc, (float)(sm64_out(si, 1) >> 40) * sc);
  s1[p] = make_float2(0.f, 0.f);
  if (s2) s2[p] = make_float2(0.f, 0.f);
}

static StepArgs make_args(const ivhd_ctx* ctx, int cur) {
  StepArgs A{};
  A.ids = ctx->ids;
  A.hub_off = ctx->hub_off;
  A.slice_off = ctx->slice_off;
  A.slice_w = ctx->slice_w;
  A.y_in = ctx->y[cur];
  A.y_out = ctx->y[cur ^ 1];
  A.yh_in = ctx->yh[cur];
  A.yh_out = ctx->yh[cur ^ 1];
  A.s1 = ctx->s1;
  A.s2 = ctx->s2;
  A.perm = ctx->perm;
  A.partials = ctx->partials;
  A.flag = ctx->flag;
  A.M = (int32_t)ctx->M;
  A.n_hub = (int32_t)ctx->n_hub;
  A.n_slices = (int32_t)ctx->n_slices;
  A.nb_hub = (int32_t)((ctx->n_hub + kWarpsPerBlock - 1) / kWarpsPerBlock);
  A.c = ctx->c;
  A.a = ctx->p.a;
  A.b = ctx->p.b;
  A.rho = ctx->p.rho;
  A.eps = ctx->p.eps;
  return A;
}

int step_grid(const ivhd_ctx* ctx) {
  const int64_t nb_hub = (ctx->n_hub + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int64_t nb_sell = (ctx->n_slices + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return (int)(nb_hub + nb_sell);
}

template <int POS>
static void launch_opt(int opt, int grid, cudaStream_t s, const StepArgs& A) {
  switch (opt) {
    case IVHD_OPT_NESTEROV: k_step<kNesterov, POS><<<grid, kStepBlock, 0, s>>>(A); break;
    case IVHD_OPT_ADADELTA: k_step<kAdadelta, POS><<<grid, kStepBlock, 0, s>>>(A); break;
    default: k_step<kMomentum, POS><<<grid, kStepBlock, 0, s>>>(A); break;
  }
}

cudaError_t launch_step(ivhd_ctx* ctx, int cur, cudaStream_t s) {
  const StepArgs A = make_args(ctx, cur);
  const int grid = step_grid(ctx);
  switch (ctx->p.pos_format) {
    case IVHD_POS_F16: launch_opt<IVHD_POS_F16>(ctx->p.opt, grid, s, A); break;
    case IVHD_POS_BF16: launch_opt<IVHD_POS_BF16>(ctx->p.opt, grid, s, A); break;
    default: launch_opt<IVHD_POS_F32>(ctx->p.opt, grid, s, A); break;
  }
  return cudaGetLastError();
}

// Nesterov stores the look-ahead point z = y + a v; forces and stress are
// reported at y, so y = z - a v is materialised in the idle ping-pong buffer.
__global__ void k_lookback(const float2* __restrict__ z, const float2* __restrict__ v, int M,
                           float a, float2* __restrict__ y) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= M) return;
  const float2 q = z[p], w = v[p];
  y[p] = make_float2(fmaf(-a, w.x, q.x), fmaf(-a, w.y, q.y));
}

static StepArgs eval_args(ivhd_ctx* ctx) {
  StepArgs A = make_args(ctx, ctx->cur);
  if (ctx->p.opt == IVHD_OPT_NESTEROV) {
    const int M = (int)ctx->M;
    k_lookback<<<(M + 255) / 256, 256, 0, ctx->stream>>>(ctx->y[ctx->cur], ctx->s1, M, ctx->p.a,
                                                         ctx->y[ctx->cur ^ 1]);
    ++ctx->aux_launches;
    A.y_in = ctx->y[ctx->cur ^ 1];
  }
  A.y_out = nullptr;
  return A;
}

cudaError_t launch_forces(ivhd_ctx* ctx, float2* out) {
  StepArgs A = eval_args(ctx);
  A.f_out = out;
  k_step<kForces, IVHD_POS_F32><<<step_grid(ctx), kStepBlock, 0, ctx->stream>>>(A);
  ++ctx->aux_launches;
  return cudaGetLastError();
}

cudaError_t launch_stress(ivhd_ctx* ctx) {
  cudaError_t e = cudaMemsetAsync(ctx->flag, 0, sizeof(int32_t), ctx->stream);
  if (e != cudaSuccess) return e;
  StepArgs A = eval_args(ctx);
  const int grid = step_grid(ctx);
  k_step<kStress, IVHD_POS_F32><<<grid, kStepBlock, 0, ctx->stream>>>(A);
  k_stress_final<<<1, 1024, 0, ctx->stream>>>(ctx->partials, grid, ctx->red_out);
  ctx->aux_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_unpermute(ivhd_ctx* ctx, float2* out) {
  const int M = (int)ctx->M;
  k_unpermute<<<(M + 255) / 256, 256, 0, ctx->stream>>>(ctx->y[ctx->cur], ctx->s1, ctx->perm, M,
                                                        ctx->p.a, ctx->p.opt == IVHD_OPT_NESTEROV,
                                                        out);
  ++ctx->aux_launches;
  return cudaGetLastError();
}

cudaError_t launch_set_positions(ivhd_ctx* ctx, const float2* in) {
  const int M = (int)ctx->M;
  k_set_positions<<<(M + 255) / 256, 256, 0, ctx->stream>>>(in, ctx->perm, M, ctx->y[ctx->cur],
                                                            ctx->s1, ctx->s2);
  ++ctx->aux_launches;
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : launch_round_positions(ctx);
}

cudaError_t launch_init_positions(ivhd_ctx* ctx) {
  const int M = (int)ctx->M;
  k_init_positions<<<(M + 255) / 256, 256, 0, ctx->stream>>>(ctx->perm, M, ctx->p.seed,
                                                             ctx->y[ctx->cur], ctx->s1, ctx->s2);
  ++ctx->aux_launches;
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : launch_round_positions(ctx);
}

}  // namespace ivhd
