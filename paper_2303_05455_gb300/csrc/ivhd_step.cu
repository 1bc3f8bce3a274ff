// ivhd_step.cu -- the hot path: one fused gather-force + optimiser-update pass.
//
// For every vertex i (Sec. 3.3.1, Eq. 3.14 with F = -1/2 grad E of Eq. 3.16):
//
//     F_i = sum_{j in nn_sym(i)} w_ij (y_j - y_i)
//         + c * sum_{k in rn_sym(i)} (1 - 1/d_ik) (y_k - y_i),   d_ik = |y_k - y_i|
//
// where nn_sym / rn_sym are the symmetrised neighbour lists (every term of the
// stress acts on both of its endpoints; w_ij = 2 for a mutual kNN pair kept
// with multiplicity), followed in the same thread by the optimiser update of
// Eq. 3.34 (momentum), or the Nesterov / Adadelta forms of Sec. 3.3.2.  All
// forces of a step read y_in and all updates write y_out (ping-pong), which is
// the synchronous scheme of the IVHD-CUDA algorithm in Sec. 5.2 without its
// per-connection +/- slots and second pass: each vertex gathers its
// neighbours' positions instead, so there are no atomics and the summation
// order is fixed by the layout (deterministic).
//
// Variants selected by template parameters:
//   POS     gathered position format (FP32, or FP16 / BF16 copies with an FP32
//           master position for the vertex's own update)
//   METRIC  L2 (the method) or L1 (Sec. 3.4.1: the l1 norm in the late
//           stages of the embedding, for its "suction" of outliers)
//   ADAPT   self-adaptive b (Sec. 3.3.3): velocities are ping-ponged, b and the
//           current buffer come from a device control word, and every block
//           reports its kinetic-energy sums for the controller kernel.
//
// Work split: SELL slices of 32 degree-sorted vertices, one thread per vertex
// and one coalesced int4 id load per 4 neighbours; vertices of high degree
// ("hubs") get a warp each (or, with several vertices per warp, a group of
// 32 / vpw lanes for the rows of medium degree) and a fixed-order butterfly
// reduction.
//
// Launch forms, all with the same per-vertex traversal and arithmetic, so
// their results agree bit for bit: one k_step launch per step (dependent
// launches replayed from CUDA graphs; the default), or all steps of a call in
// one launch -- k_cluster (8-block cluster, positions in every block's shared
// memory, small embeddings), k_resident (one block), k_persist (cooperative
// grid with a bounded grid barrier per step).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ivhd_internal.cuh"

namespace ivhd {

// FP32 positions read through L2 only (ld.global.cg): the persistent kernel
// rereads position arrays that other blocks rewrote during the same launch,
// which the read-only (non-coherent) path may not observe.  Internal format.
constexpr int kPosF32Coherent = 3;
template <int POS>
constexpr bool f32_pos() {
  return POS == IVHD_POS_F32 || POS == kPosF32Coherent;
}

// Position of vertex idx as the neighbours see it: the FP32 array, or the
// rounded FP16 / BF16 copy (one 32-bit word per vertex).
template <int POS>
__device__ __forceinline__ float2 load_pos(const float2* __restrict__ y,
                                           const uint32_t* __restrict__ yh, uint32_t idx) {
  if constexpr (POS == IVHD_POS_F32) {
    return __ldg(y + idx);
  } else if constexpr (POS == kPosF32Coherent) {
    return __ldcg(y + idx);
  } else {
    const uint32_t w = __ldg(yh + idx);
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

struct Gsrc {
  const float2* __restrict__ y;
  const uint32_t* __restrict__ yh;
  uint64_t keep;  // L2 cache policy "evict last" for the cold FP32 gathers
  uint32_t M;     // positions (checked builds test every gathered index against it)
};

// Checked builds (compiled with IVHD_CHECKED, the stand-in for a memory
// checker): every gathered index and every row extent read from the layout is
// tested before use; a bad one is counted in g_check_violations and skipped
// (the gather returns the vertex's own position, the row is treated as
// empty), so a corrupt layout is reported instead of read out of bounds.  In
// normal builds both tests are compile-time true.
#ifdef IVHD_CHECKED
__device__ unsigned long long g_check_violations = 0;
__device__ __forceinline__ bool index_ok(uint32_t idx, uint32_t n) {
  if (idx < n) return true;
  atomicAdd(&g_check_violations, 1ull);
  return false;
}
__device__ __forceinline__ bool row_ok(int64_t beg, int64_t end, int64_t n_slots) {
  if (0 <= beg && beg <= end && end <= n_slots && (beg & 3) == 0) return true;
  atomicAdd(&g_check_violations, 1ull);
  return false;
}
#else
__device__ __forceinline__ constexpr bool index_ok(uint32_t, uint32_t) { return true; }
__device__ __forceinline__ constexpr bool row_ok(int64_t, int64_t, int64_t) { return true; }
#endif

// Warp w of the warp-per-vertex region (the hub rows, in descending degree):
// the first n_full rows take a whole warp each; the rest share a warp, mid_g
// lanes per row (32 / mid_g rows per warp).  Lanes past the last row get a
// row index >= n_hub.  With mid_g = 32 every row has its own warp.
struct HubSlot {
  int row;  // vertex (= row of the region)
  int g;    // lanes on the row: 32 or mid_g (a power of two)
  int l;    // this lane's index among them
};
__device__ __forceinline__ HubSlot hub_slot(int w, int lane, int n_full, int mid_g) {
  if (w < n_full) return HubSlot{w, 32, lane};
  return HubSlot{n_full + (w - n_full) * (32 / mid_g) + lane / mid_g, mid_g, lane & (mid_g - 1)};
}

// Sum over the g lanes of each aligned lane group (g uniform over the warp);
// with g = 32 the butterfly over the whole warp.
__device__ __forceinline__ void group_sum(float& fx, float& fy, int g) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (o < g) {
      fx += __shfl_xor_sync(0xffffffffu, fx, o);
      fy += __shfl_xor_sync(0xffffffffu, fy, o);
    }
  }
}

// L1 policy of the FP32 gathers.  The layout orders vertices by degree, and a
// vertex is gathered once per symmetric term, so the first vertices are the
// most gathered ones (on the 1.4e6-vertex exact kNN graph the first 16,384
// receive 14 % of all gathers).  Their lines are allocated in L1 as usual; all
// other gathers read through L1 without allocating, so the streamed rows of
// the many rarely gathered vertices do not evict the hot lines.  Measured on
// that graph: 57.2 us per step against 59.0 us with every gather allocating.
// For the 4-byte FP16 / BF16 copies the same policy measured slower (61.3 us
// against 58.4 us: eight vertices share a sector, so unrelated gathers hit in
// L1 more often), so those keep the default policy.
constexpr uint32_t kL1HotF32 = 16384;

// The cold gathers also carry an L2 "evict last" policy, so positions are
// kept in L2 ahead of the streamed rows and state (56.9 us against 57.2 us).
__device__ __forceinline__ float2 load_f32_no_l1(const float2* y, uint32_t idx, uint64_t keep) {
  uint32_t w0, w1;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.b32 {%0,%1}, [%2], %3;"
      : "=r"(w0), "=r"(w1)
      : "l"(y + idx), "l"(keep));
  return make_float2(__uint_as_float(w0), __uint_as_float(w1));
}

template <int POS>
__device__ __forceinline__ float2 gather(const Gsrc& G, uint32_t e, float2 self) {
  if constexpr (POS == IVHD_POS_F32) {
    if (e == kPad || !index_ok(e & kIdxMask, G.M)) return self;
    const uint32_t idx = e & kIdxMask;
    return (idx < kL1HotF32) ? __ldg(G.y + idx) : load_f32_no_l1(G.y, idx, G.keep);
  } else if constexpr (POS == kPosF32Coherent) {
    return (e == kPad || !index_ok(e & kIdxMask, G.M)) ? self : __ldcg(G.y + (e & kIdxMask));
  } else {
    return (e == kPad || !index_ok(e & kIdxMask, G.M)) ? self
                                                       : load_pos<POS>(G.y, G.yh, e & kIdxMask);
  }
}

__device__ __forceinline__ float sgnf(float u) { return (float)((u > 0.f) - (u < 0.f)); }

// One term of the force on i, u = y_j - y_i.
// L2: nn w u (w = 1, or 2 for a mutual pair kept with multiplicity);
//     rn c (1 - 1/d) u, zero at d = 0.
// L1 (d = |u_x| + |u_y|, gradient taken coordinate-wise with sign(0) = 0):
//     nn w d sign(u); rn -c (1 - d) sign(u).
// Padding entries carry the rn bit and gather y_i itself: u = 0, no force.
template <int METRIC>
__device__ __forceinline__ void force_term(uint32_t e, float2 yj, float2 yi, float c, float& fx,
                                           float& fy) {
  const float ux = yj.x - yi.x;
  const float uy = yj.y - yi.y;
  if constexpr (METRIC == IVHD_METRIC_L2) {
    float w = (e & kW2Bit) ? 2.f : 1.f;
    if (e & kRnBit) {
      const float d2 = fmaf(uy, uy, ux * ux);
      w = (d2 > 0.f) ? c * (1.f - rsqrtf(d2)) : 0.f;
    }
    fx = fmaf(w, ux, fx);
    fy = fmaf(w, uy, fy);
  } else {
    const float d = fabsf(ux) + fabsf(uy);
    float s = ((e & kW2Bit) ? 2.f : 1.f) * d;
    if (e & kRnBit) s = -c * (1.f - d);
    fx = fmaf(s, sgnf(ux), fx);
    fy = fmaf(s, sgnf(uy), fy);
  }
}

// One term of the stress: nn w d^2, rn c (1 - d)^2 (d in the active metric);
// padding contributes nothing.
template <int METRIC>
__device__ __forceinline__ void stress_term(uint32_t e, float2 yj, float2 yi, float c, float& es) {
  if (e == kPad) return;
  const float ux = yj.x - yi.x;
  const float uy = yj.y - yi.y;
  float d2, d;
  if constexpr (METRIC == IVHD_METRIC_L2) {
    d2 = fmaf(uy, uy, ux * ux);
    d = sqrtf(d2);
  } else {
    d = fabsf(ux) + fabsf(uy);
    d2 = d * d;
  }
  if (e & kRnBit) {
    const float t = 1.f - d;
    es = fmaf(c * t, t, es);
  } else {
    es = fmaf((e & kW2Bit) ? 2.f : 1.f, d2, es);
  }
}

template <int MODE, int POS, int METRIC>
__device__ __forceinline__ void visit4(const int4 e, const Gsrc& G, float2 yi, float c, float& fx,
                                       float& fy) {
  const uint32_t e0 = (uint32_t)e.x, e1 = (uint32_t)e.y, e2 = (uint32_t)e.z, e3 = (uint32_t)e.w;
  const float2 g0 = gather<POS>(G, e0, yi), g1 = gather<POS>(G, e1, yi);
  const float2 g2 = gather<POS>(G, e2, yi), g3 = gather<POS>(G, e3, yi);
  if (MODE == kStress) {
    stress_term<METRIC>(e0, g0, yi, c, fx);
    stress_term<METRIC>(e1, g1, yi, c, fx);
    stress_term<METRIC>(e2, g2, yi, c, fx);
    stress_term<METRIC>(e3, g3, yi, c, fx);
  } else {
    force_term<METRIC>(e0, g0, yi, c, fx, fy);
    force_term<METRIC>(e1, g1, yi, c, fx, fy);
    force_term<METRIC>(e2, g2, yi, c, fx, fy);
    force_term<METRIC>(e3, g3, yi, c, fx, fy);
  }
}

template <int MODE, int POS, int METRIC>
__device__ __forceinline__ void visit8(const int4 ea, const int4 eb, const Gsrc& G, float2 yi,
                                       float c, float& fx, float& fy) {
  // all eight gathers are issued before any arithmetic (eight loads in flight per thread)
  const uint32_t e[8] = {(uint32_t)ea.x, (uint32_t)ea.y, (uint32_t)ea.z, (uint32_t)ea.w,
                         (uint32_t)eb.x, (uint32_t)eb.y, (uint32_t)eb.z, (uint32_t)eb.w};
  float2 g[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) g[q] = gather<POS>(G, e[q], yi);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (MODE == kStress)
      stress_term<METRIC>(e[q], g[q], yi, c, fx);
    else
      force_term<METRIC>(e[q], g[q], yi, c, fx, fy);
  }
}

// Per-vertex optimiser updates (shared by the step kernel and the resident
// whole-run kernel, so both produce the same bits).
// Eq. 3.34: v <- a v + b F ; y <- y + v
__device__ __forceinline__ void momentum_update(float a, float b, float fx, float fy, float2 ym,
                                                float2 v, float2& vn, float2& yn) {
  vn.x = fmaf(a, v.x, b * fx);
  vn.y = fmaf(a, v.y, b * fy);
  yn = make_float2(ym.x + vn.x, ym.y + vn.y);
}
// Nesterov: the state is the look-ahead point z = y + a v and F was taken at z.
// v' = a v + b F(z);  y' = y + v';  z' = y' + a v' = z - a v + (1 + a) v'
__device__ __forceinline__ void nesterov_update(float a, float b, float fx, float fy, float2 zm,
                                                float2 v, float2& vn, float2& zn) {
  vn.x = fmaf(a, v.x, b * fx);
  vn.y = fmaf(a, v.y, b * fy);
  const float ap1 = 1.f + a;
  zn = make_float2(zm.x + fmaf(ap1, vn.x, -a * v.x), zm.y + fmaf(ap1, vn.y, -a * v.y));
}
// Zeiler's Adadelta on g = -F: E[g^2] <- rho E[g^2] + (1-rho) g^2;
// dx = -sqrt(E[dx^2] + eps) / sqrt(E[g^2] + eps) g; E[dx^2] <- rho E[dx^2] + (1-rho) dx^2
__device__ __forceinline__ void adadelta_update(float rho, float eps, float fx, float fy,
                                                float2 ym, float2& eg, float2& ex, float2& yn) {
  const float omr = 1.f - rho;
  const float gx = -fx, gy = -fy;
  eg.x = fmaf(rho, eg.x, omr * gx * gx);
  eg.y = fmaf(rho, eg.y, omr * gy * gy);
  const float dx = -(sqrtf(ex.x + eps) / sqrtf(eg.x + eps)) * gx;
  const float dy = -(sqrtf(ex.y + eps) / sqrtf(eg.y + eps)) * gy;
  ex.x = fmaf(rho, ex.x, omr * dx * dx);
  ex.y = fmaf(rho, ex.y, omr * dy * dy);
  yn = make_float2(ym.x + dx, ym.y + dy);
}

// Block sum of a per-thread float in a fixed order (warp tree, then warps in
// order); the result is valid in thread 0.  The kinetic energies of the
// adaptive-b controller use it: FP64 arithmetic is slow on this GPU, and the
// per-block FP32 sums (<= 512 terms) are added across blocks in FP64.
__device__ __forceinline__ float block_sum_f32(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  __syncthreads();
  return t;
}

// Block sum of a per-thread double in a fixed order (warp tree, then warps in
// order); the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  __syncthreads();
  return t;
}

#ifndef IVHD_STEP_MIN_BLOCKS
#define IVHD_STEP_MIN_BLOCKS 1
#endif

// MODE: optimiser epilogue (or forces / stress).  yi is the vertex's own
// position in the gathered format (differences are taken between equally
// rounded positions); ym is its FP32 master position.
// One block's share of a step: block vb of the step grid (hub warps, then
// SELL slices), reading positions y[cur] and writing y[cur ^ 1].  PDL: the
// step is a programmatic dependent launch, whose successor may start once this
// block's gathers are done.
template <int MODE, int POS, int METRIC, bool ADAPT, bool PDL>
__device__ __forceinline__ void step_block(const StepArgs& A, int vb, int cur) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint64_t keep;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
  const Gsrc G{A.y[cur], A.yh[cur], keep, (uint32_t)A.M};
  const float b = ADAPT ? A.ctl->b : A.b;
  float fx = 0.f, fy = 0.f;  // force, or (stress in fx)
  float2 yi = make_float2(0.f, 0.f);
  float2 ym = make_float2(0.f, 0.f);
  int p = -1;
  bool own = false;
  // the owner's optimiser state is loaded with its position, before the
  // gathers, so its latency is not added after them
  constexpr bool kUpdate = MODE == kMomentum || MODE == kNesterov || MODE == kAdadelta;
  const float2* __restrict__ v_in = A.v[ADAPT ? cur : 0];
  float2 v_pre = make_float2(0.f, 0.f), s2_pre = make_float2(0.f, 0.f);
  auto load_state = [&](int q) {
    if constexpr (kUpdate) {
      v_pre = v_in[q];
      if constexpr (MODE == kAdadelta) s2_pre = A.s2[q];
    }
  };

  if (vb < A.nb_wide) {
    // the longest rows: 4 warps (128 lanes) per vertex whatever the block size
    // (a block of 8 or 16 warps takes 2 or 4 such rows); the lanes stride over
    // the row's int4 groups, then the partial forces are summed in a fixed
    // order (the butterfly within each warp, then the 4 warps in order)
    __shared__ float wred[2][kMaxStepBlock / 32];
    const int grp = wib / kWideWarps;
    const int gl = (int)threadIdx.x - grp * kWideWarps * 32;
    const int r = vb * (A.wpb / kWideWarps) + grp;
    const bool valid = r < A.n_wide;
    int ng = 0;
    const int4* row = nullptr;
    if (valid) {
      p = r;
      ym = (POS == kPosF32Coherent) ? __ldcg(G.y + p) : G.y[p];
      yi = f32_pos<POS>() ? ym : load_pos<POS>(G.y, G.yh, p);
      if (gl == 0) load_state(p);
      const int beg = A.hub_off[p], end = A.hub_off[p + 1];
      row = reinterpret_cast<const int4*>(A.ids + beg);
      ng = row_ok(beg, end, A.n_slots) ? (end - beg) >> 2 : 0;
    }
    constexpr int nt = kWideWarps * 32;
    int g = gl;
    for (; g + nt < ng; g += 2 * nt) {
      const int4 ea = ld_stream_v4(row + g);
      const int4 eb = ld_stream_v4(row + g + nt);
      visit8<MODE, POS, METRIC>(ea, eb, G, yi, A.c, fx, fy);
    }
    if (g < ng) visit4<MODE, POS, METRIC>(ld_stream_v4(row + g), G, yi, A.c, fx, fy);
    group_sum(fx, fy, 32);
    if (lane == 0) {
      wred[0][wib] = fx;
      wred[1][wib] = fy;
    }
    __syncthreads();
    if (valid && gl == 0) {
      const int w0 = grp * kWideWarps;
      fx = wred[0][w0];
      fy = wred[1][w0];
      for (int q = 1; q < kWideWarps; ++q) {
        fx += wred[0][w0 + q];
        fy += wred[1][w0 + q];
      }
    }
    own = valid && gl == 0;
  } else if (vb < A.nb_wide + A.nb_hub) {
    // hub rows: a warp, or a group of mid_g lanes, per vertex; the lanes of a
    // row stride over its int4 groups, then sum their partial forces
    const int w = (vb - A.nb_wide) * A.wpb + wib;
    if (w < A.hub_warps) {
      const HubSlot h = hub_slot(w, lane, A.n_full, A.mid_g);
      const bool valid = A.n_wide + h.row < A.n_hub;
      int ng = 0;
      const int4* row = nullptr;
      if (valid) {
        p = A.n_wide + h.row;
        ym = (POS == kPosF32Coherent) ? __ldcg(G.y + p) : G.y[p];
        yi = f32_pos<POS>() ? ym : load_pos<POS>(G.y, G.yh, p);
        if (h.l == 0) load_state(p);
        const int beg = A.hub_off[p], end = A.hub_off[p + 1];
        row = reinterpret_cast<const int4*>(A.ids + beg);
        ng = row_ok(beg, end, A.n_slots) ? (end - beg) >> 2 : 0;
      }
      int g = h.l;
      for (; g + h.g < ng; g += 2 * h.g) {
        const int4 ea = ld_stream_v4(row + g);
        const int4 eb = ld_stream_v4(row + g + h.g);
        visit8<MODE, POS, METRIC>(ea, eb, G, yi, A.c, fx, fy);
      }
      if (g < ng) visit4<MODE, POS, METRIC>(ld_stream_v4(row + g), G, yi, A.c, fx, fy);
      group_sum(fx, fy, h.g);
      own = valid && h.l == 0;
    }
  } else {
    // SELL slice: one thread per vertex, one coalesced int4 per 4 neighbours
    const int s = (vb - A.nb_wide - A.nb_hub) * A.wpb + wib;
    if (s < A.n_slices) {
      p = A.n_hub + s * 32 + lane;
      const bool valid = p < A.M;
      if (valid) {
        ym = (POS == kPosF32Coherent) ? __ldcg(G.y + p) : G.y[p];
        yi = f32_pos<POS>() ? ym : load_pos<POS>(G.y, G.yh, p);
        load_state(p);
      }
      const int4* base = reinterpret_cast<const int4*>(A.ids + A.slice_off[s]) + lane;
      const int W = row_ok(A.slice_off[s], A.slice_off[s] + (int64_t)A.slice_w[s] * 128, A.n_slots)
                        ? A.slice_w[s]
                        : 0;
      int g = 0;
      for (; g + 1 < W; g += 2) {
        const int4 ea = ld_stream_v4(base + g * 32);
        const int4 eb = ld_stream_v4(base + (g + 1) * 32);
        visit8<MODE, POS, METRIC>(ea, eb, G, yi, A.c, fx, fy);
      }
      if (g < W) visit4<MODE, POS, METRIC>(ld_stream_v4(base + g * 32), G, yi, A.c, fx, fy);
      own = valid;
    }
  }

  // this block's gathers are done: the next step's grid may start launching
  // (its blocks wait for this grid's completion before reading anything)
  if constexpr (PDL) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  float2* __restrict__ y_out = A.y[cur ^ 1];
  uint32_t* __restrict__ yh_out = A.yh[cur ^ 1];
  float2* __restrict__ v_out = A.v[ADAPT ? (cur ^ 1) : 0];
  float kin_new = 0.f, kin_old = 0.f;  // |v'|^2, |v|^2 (FP32; blocks sum them in a fixed order)

  if (MODE == kMomentum) {
    if (own) {
      const float2 v = v_pre;
      float2 vn, yn;
      momentum_update(A.a, b, fx, fy, ym, v, vn, yn);
      v_out[p] = vn;
      y_out[p] = yn;
      if constexpr (!f32_pos<POS>()) yh_out[p] = round_pos<POS>(yn);
      if (ADAPT) {
        kin_new = fmaf(vn.y, vn.y, vn.x * vn.x);
        kin_old = fmaf(v.y, v.y, v.x * v.x);
      }
    }
  } else if (MODE == kNesterov) {
    if (own) {
      const float2 v = v_pre;
      float2 vn, zn;
      nesterov_update(A.a, b, fx, fy, ym, v, vn, zn);
      v_out[p] = vn;
      y_out[p] = zn;
      if constexpr (!f32_pos<POS>()) yh_out[p] = round_pos<POS>(zn);
      if (ADAPT) {
        kin_new = fmaf(vn.y, vn.y, vn.x * vn.x);
        kin_old = fmaf(v.y, v.y, v.x * v.x);
      }
    }
  } else if (MODE == kAdadelta) {
    if (own) {
      float2 eg = v_pre;
      float2 ex = s2_pre;
      float2 yn;
      adadelta_update(A.rho, A.eps, fx, fy, ym, eg, ex, yn);
      v_out[p] = eg;
      A.s2[p] = ex;
      y_out[p] = yn;
      if constexpr (!f32_pos<POS>()) yh_out[p] = round_pos<POS>(yn);
    }
  } else if (MODE == kForces) {
    if (own) A.f_out[A.perm[p]] = make_float2(fx, fy);
  } else if (MODE == kStress) {
    __shared__ double red[kMaxStepBlock / 32];
    if (own && !(isfinite(ym.x) && isfinite(ym.y))) atomicOr(A.flag, 1);
    const double t = block_sum(own ? (double)fx : 0.0, red);
    if (threadIdx.x == 0) A.partials[vb] = t;
  }
  if (ADAPT) {
    __shared__ float red2[kMaxStepBlock / 32];
    const double tn = (double)block_sum_f32(kin_new, red2);
    const double to = (double)block_sum_f32(kin_old, red2);
    if (threadIdx.x == 0) {
      A.partials[2 * vb] = tn;
      A.partials[2 * vb + 1] = to;
    }
  }
}

// Register cap of the step kernel: the optimiser's code fits 48 registers (50
// for Adadelta's two accumulators) without spilling; more would cost a block
// of residency per SM on this request-rate-bound kernel.
template <int MODE>
constexpr int step_max_regs() {
  return MODE == kAdadelta ? 50 : 48;
}

template <int MODE, int POS, int METRIC, bool ADAPT>
__global__ void __maxnreg__(step_max_regs<MODE>()) k_step(const StepArgs A) {
  // launched as a programmatic dependent of the previous step: wait until that
  // grid has completed and its writes are visible before reading any state
  // (a no-op for a launch without that attribute)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int cur = ADAPT ? A.ctl->cur : A.cur;
  step_block<MODE, POS, METRIC, ADAPT, true>(A, (int)blockIdx.x, cur);
}

// ---- persistent grid kernel ------------------------------------------------------
//
// All steps of an ivhd_step call in one cooperative launch: every block is
// resident, takes the blocks vb = blockIdx.x, blockIdx.x + gridDim.x, ... of
// the step grid (so each vertex is traversed exactly as by k_step, and the
// positions agree with the multi-launch path bit for bit), and the steps are
// separated by a grid barrier instead of kernel launches.  Positions are read
// through L2 (they are rewritten by other blocks within the launch).  The
// barrier waits a bounded number of polls; on expiry (or when another block
// gave up) the block raises *err and the launch ends.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};
constexpr unsigned kGridBarrierPolls = 1u << 22;  // x >= 64 ns: > 0.25 s, far above any step

__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, int32_t* err, unsigned polls) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &bar->gen;
    volatile int32_t* verr = err;
    const unsigned g = *gen;  // the generation this barrier completes
    __threadfence();          // this block's writes before its arrival
    if (atomicAdd(&bar->count, 1u) == gridDim.x - 1) {
      bar->count = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      unsigned it = 0;
      while (*gen == g) {
        if (++it > polls || *verr) {
          atomicOr(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();  // the other blocks' writes after the barrier
  }
  return __syncthreads_and(ok) != 0;
}

// Test support: block 0 waits at the barrier, block 1 never arrives.
__global__ void k_probe_grid_barrier(GridBarrier* bar, int32_t* err, unsigned polls) {
  if (blockIdx.x != 0) return;
  grid_barrier(bar, err, polls);
}

template <int MODE, int METRIC>
__global__ void __launch_bounds__(kMaxStepBlock, IVHD_STEP_MIN_BLOCKS)
    k_persist(const StepArgs A, int64_t n_iter, int n_vblocks, GridBarrier* bar, int32_t* err) {
  int cur = A.cur;
  for (int64_t it = 0; it < n_iter; ++it) {
    for (int vb = (int)blockIdx.x; vb < n_vblocks; vb += (int)gridDim.x)
      step_block<MODE, kPosF32Coherent, METRIC, false, false>(A, vb, cur);
    if (!grid_barrier(bar, err, kGridBarrierPolls)) return;
    cur ^= 1;
  }
}

// ---- resident whole-run kernel -------------------------------------------------
//
// For an embedding whose positions (both ping-pong copies) and optimiser
// state fit one SM's shared memory, one block of 1,024 threads runs every step
// of an ivhd_step call: the steps of the synchronous scheme (Sec. 5.2) are
// separated by __syncthreads instead of kernel launches, and every gather is a
// shared-memory load.  The id rows are copied to shared memory too when they
// fit, else read through L1.  The traversal (hub rows warp-per-vertex with the
// same butterfly, SELL slices thread-per-vertex) and the arithmetic are those of
// k_step, so the positions agree with the multi-launch path bit for bit.
// Opt-in (ivhd_params.resident = 1): measured, one SM's instruction rate bounds
// it (2,000 vertices: 3.38 us per step against 3.43 for one launch per step;
// 5,000-8,000 vertices with hubs: 10-29 us against 3.3-4.5).
constexpr int kResidentThreads = 1024;

template <int MODE, int METRIC>
__device__ __forceinline__ void rvisit4(const int4 e, const float2* src, uint32_t M, float2 yi,
                                        float c, float& fx, float& fy) {
  const uint32_t q[4] = {(uint32_t)e.x, (uint32_t)e.y, (uint32_t)e.z, (uint32_t)e.w};
  float2 g[4];
#pragma unroll
  for (int t = 0; t < 4; ++t)
    g[t] = (q[t] == kPad || !index_ok(q[t] & kIdxMask, M)) ? yi : src[q[t] & kIdxMask];
#pragma unroll
  for (int t = 0; t < 4; ++t) force_term<METRIC>(q[t], g[t], yi, c, fx, fy);
}

template <int MODE, int METRIC>
__device__ __forceinline__ void rvisit8(const int4 ea, const int4 eb, const float2* src,
                                        uint32_t M, float2 yi, float c, float& fx, float& fy) {
  const uint32_t q[8] = {(uint32_t)ea.x, (uint32_t)ea.y, (uint32_t)ea.z, (uint32_t)ea.w,
                         (uint32_t)eb.x, (uint32_t)eb.y, (uint32_t)eb.z, (uint32_t)eb.w};
  float2 g[8];
#pragma unroll
  for (int t = 0; t < 8; ++t)
    g[t] = (q[t] == kPad || !index_ok(q[t] & kIdxMask, M)) ? yi : src[q[t] & kIdxMask];
#pragma unroll
  for (int t = 0; t < 8; ++t) force_term<METRIC>(q[t], g[t], yi, c, fx, fy);
}

template <int MODE, int METRIC, bool IDS_SMEM>
__global__ void __launch_bounds__(kResidentThreads, 1)
    k_resident(const StepArgs A, int64_t n_iter, int64_t n_slots) {
  extern __shared__ __align__(16) unsigned char rsm[];
  const int M = A.M, Mp = (A.M + 1) & ~1;  // even: every array starts 16-byte aligned
  float2* ys0 = reinterpret_cast<float2*>(rsm);
  float2* ys1 = ys0 + Mp;
  float2* vs = ys1 + Mp;
  float2* es = vs + Mp;  // Adadelta E[dx^2]
  uint32_t* ids_s = reinterpret_cast<uint32_t*>(MODE == kAdadelta ? es + Mp : es);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (int)(blockDim.x >> 5);

  for (int p = threadIdx.x; p < M; p += blockDim.x) {
    ys0[p] = A.y[A.cur][p];
    vs[p] = A.v[0][p];
    if (MODE == kAdadelta) es[p] = A.s2[p];
  }
  if (IDS_SMEM) {
    const uint4* g = reinterpret_cast<const uint4*>(A.ids);
    uint4* d = reinterpret_cast<uint4*>(ids_s);
    for (int64_t q = threadIdx.x; q < n_slots / 4; q += blockDim.x) d[q] = g[q];
  }
  __syncthreads();
  const uint32_t* ids = IDS_SMEM ? ids_s : A.ids;
  const int n_items = A.hub_warps + A.n_slices;

  for (int64_t it = 0; it < n_iter; ++it) {
    const float2* src = (it & 1) ? ys1 : ys0;
    float2* dst = (it & 1) ? ys0 : ys1;
    for (int item = warp; item < n_items; item += nwarps) {
      float fx = 0.f, fy = 0.f;
      float2 ym = make_float2(0.f, 0.f);
      int p;
      bool own;
      if (item < A.hub_warps) {
        const HubSlot h = hub_slot(item, lane, A.n_full, A.mid_g);
        const bool valid = h.row < A.n_hub;
        int ng = 0;
        const int4* row = nullptr;
        p = h.row;
        if (valid) {
          ym = src[p];
          const int beg = A.hub_off[p], end = A.hub_off[p + 1];
          row = reinterpret_cast<const int4*>(ids + beg);
          ng = row_ok(beg, end, A.n_slots) ? (end - beg) >> 2 : 0;
        }
        int g = h.l;
        for (; g + h.g < ng; g += 2 * h.g)
          rvisit8<MODE, METRIC>(row[g], row[g + h.g], src, (uint32_t)M, ym, A.c, fx, fy);
        if (g < ng) rvisit4<MODE, METRIC>(row[g], src, (uint32_t)M, ym, A.c, fx, fy);
        group_sum(fx, fy, h.g);
        own = valid && h.l == 0;
      } else {
        const int sl = item - A.hub_warps;
        p = A.n_hub + sl * 32 + lane;
        own = p < M;
        if (own) ym = src[p];
        const int4* base = reinterpret_cast<const int4*>(ids + A.slice_off[sl]) + lane;
        const int W =
            row_ok(A.slice_off[sl], A.slice_off[sl] + (int64_t)A.slice_w[sl] * 128, A.n_slots)
                ? A.slice_w[sl]
                : 0;
        int g = 0;
        for (; g + 1 < W; g += 2)
          rvisit8<MODE, METRIC>(base[g * 32], base[(g + 1) * 32], src, (uint32_t)M, ym, A.c, fx,
                                fy);
        if (g < W) rvisit4<MODE, METRIC>(base[g * 32], src, (uint32_t)M, ym, A.c, fx, fy);
      }
      if (!own) continue;
      if (MODE == kMomentum) {
        float2 vn, yn;
        momentum_update(A.a, A.b, fx, fy, ym, vs[p], vn, yn);
        vs[p] = vn;
        dst[p] = yn;
      } else if (MODE == kNesterov) {
        float2 vn, zn;
        nesterov_update(A.a, A.b, fx, fy, ym, vs[p], vn, zn);
        vs[p] = vn;
        dst[p] = zn;
      } else {
        float2 eg = vs[p], ex = es[p], yn;
        adadelta_update(A.rho, A.eps, fx, fy, ym, eg, ex, yn);
        vs[p] = eg;
        es[p] = ex;
        dst[p] = yn;
      }
    }
    __syncthreads();
  }
  const float2* fin = (n_iter & 1) ? ys1 : ys0;
  float2* yout = A.y[A.cur ^ (int)(n_iter & 1)];
  for (int p = threadIdx.x; p < M; p += blockDim.x) {
    yout[p] = fin[p];
    A.v[0][p] = vs[p];
    if (MODE == kAdadelta) A.s2[p] = es[p];
  }
}

// ---- cluster whole-run kernel ----------------------------------------------------
//
// The same whole-call scheme spread over a thread-block cluster of
// kClusterCTAs blocks (one per SM): every block keeps a full copy of the
// positions (both ping-pong buffers) in its shared memory, processes a
// contiguous range of the work items (hub rows, then slices, so it owns a
// contiguous range of vertices), and writes each updated position into the
// next buffer of every block of the cluster through distributed shared memory.
// A cluster barrier (release / acquire) separates the steps; every thread of
// every block executes the same barriers, and there is no software wait.
constexpr int kClusterCTAs = 8;  // measured: 4 and 16 blocks were no faster at 1k-4k vertices

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory location in block `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_store(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y)
               : "memory");
}

template <int MODE, int METRIC>
__global__ void __launch_bounds__(kResidentThreads, 1) k_cluster(const StepArgs A, int64_t n_iter) {
  extern __shared__ __align__(16) unsigned char rsm[];
  const int M = A.M, Mp = (A.M + 1) & ~1;
  float2* ys0 = reinterpret_cast<float2*>(rsm);
  float2* ys1 = ys0 + Mp;
  float2* vs = ys1 + Mp;
  float2* es = vs + Mp;  // Adadelta E[dx^2]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (int)(blockDim.x >> 5);
  const uint32_t rank = cluster_rank();
  const int n_items = A.hub_warps + A.n_slices;
  const int it_lo = (int)((int64_t)n_items * rank / kClusterCTAs);
  const int it_hi = (int)((int64_t)n_items * (rank + 1) / kClusterCTAs);
  // the first vertex of an item: items cover contiguous, ascending vertex ranges
  auto first_vertex = [&](int item) {
    if (item < A.n_full) return item;
    if (item < A.hub_warps) return A.n_full + (item - A.n_full) * (32 / A.mid_g);
    return A.n_hub + (item - A.hub_warps) * 32;
  };
  const int v_lo = min(M, first_vertex(it_lo)), v_hi = min(M, first_vertex(it_hi));

  for (int p = threadIdx.x; p < M; p += blockDim.x) ys0[p] = A.y[A.cur][p];
  for (int p = v_lo + threadIdx.x; p < v_hi; p += blockDim.x) {
    vs[p] = A.v[0][p];
    if (MODE == kAdadelta) es[p] = A.s2[p];
  }
  // every block's copy is loaded before any block writes into it
  cluster_barrier();
  const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(ys0);
  const uint32_t a1 = (uint32_t)__cvta_generic_to_shared(ys1);

  for (int64_t it = 0; it < n_iter; ++it) {
    const float2* src = (it & 1) ? ys1 : ys0;
    const uint32_t dst_a = (it & 1) ? a0 : a1;
    for (int item = it_lo + warp; item < it_hi; item += nwarps) {
      float fx = 0.f, fy = 0.f;
      float2 ym = make_float2(0.f, 0.f);
      int p;
      bool own;
      if (item < A.hub_warps) {
        const HubSlot h = hub_slot(item, lane, A.n_full, A.mid_g);
        const bool valid = h.row < A.n_hub;
        int ng = 0;
        const int4* row = nullptr;
        p = h.row;
        if (valid) {
          ym = src[p];
          const int beg = A.hub_off[p], end = A.hub_off[p + 1];
          row = reinterpret_cast<const int4*>(A.ids + beg);
          ng = row_ok(beg, end, A.n_slots) ? (end - beg) >> 2 : 0;
        }
        int g = h.l;
        for (; g + h.g < ng; g += 2 * h.g)
          rvisit8<MODE, METRIC>(row[g], row[g + h.g], src, (uint32_t)M, ym, A.c, fx, fy);
        if (g < ng) rvisit4<MODE, METRIC>(row[g], src, (uint32_t)M, ym, A.c, fx, fy);
        group_sum(fx, fy, h.g);
        own = valid && h.l == 0;
      } else {
        const int sl = item - A.hub_warps;
        p = A.n_hub + sl * 32 + lane;
        own = p < M;
        if (own) ym = src[p];
        const int4* base = reinterpret_cast<const int4*>(A.ids + A.slice_off[sl]) + lane;
        const int W =
            row_ok(A.slice_off[sl], A.slice_off[sl] + (int64_t)A.slice_w[sl] * 128, A.n_slots)
                ? A.slice_w[sl]
                : 0;
        int g = 0;
        for (; g + 1 < W; g += 2)
          rvisit8<MODE, METRIC>(base[g * 32], base[(g + 1) * 32], src, (uint32_t)M, ym, A.c, fx,
                                fy);
        if (g < W) rvisit4<MODE, METRIC>(base[g * 32], src, (uint32_t)M, ym, A.c, fx, fy);
      }
      if (!own) continue;
      float2 yn;
      if (MODE == kMomentum) {
        float2 vn;
        momentum_update(A.a, A.b, fx, fy, ym, vs[p], vn, yn);
        vs[p] = vn;
      } else if (MODE == kNesterov) {
        float2 vn;
        nesterov_update(A.a, A.b, fx, fy, ym, vs[p], vn, yn);
        vs[p] = vn;
      } else {
        float2 eg = vs[p], ex = es[p];
        adadelta_update(A.rho, A.eps, fx, fy, ym, eg, ex, yn);
        vs[p] = eg;
        es[p] = ex;
      }
      const uint32_t off = dst_a + (uint32_t)p * (uint32_t)sizeof(float2);
#pragma unroll
      for (int r = 0; r < kClusterCTAs; ++r) cluster_store(cluster_map(off, (uint32_t)r), yn);
    }
    cluster_barrier();
  }
  const float2* fin = (n_iter & 1) ? ys1 : ys0;
  float2* yout = A.y[A.cur ^ (int)(n_iter & 1)];
  for (int p = v_lo + threadIdx.x; p < v_hi; p += blockDim.x) {
    yout[p] = fin[p];
    A.v[0][p] = vs[p];
    if (MODE == kAdadelta) A.s2[p] = es[p];
  }
  // no block leaves while a peer could still address its shared memory
  cluster_barrier();
}

template <int MODE, int METRIC>
static cudaError_t launch_cl(const StepArgs& A, int64_t n_iter, size_t smem, cudaStream_t s) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_cluster<MODE, METRIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kResidentSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterCTAs);
  cfg.blockDim = dim3(kResidentThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCTAs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cluster<MODE, METRIC>, A, n_iter);
}

// Shared memory of the resident kernel with and without the id rows.
static size_t resident_bytes(const ivhd_ctx* ctx, bool with_ids) {
  const size_t Mp = (size_t)((ctx->M + 1) & ~1);
  const size_t state = Mp * sizeof(float2) * (ctx->p.opt == IVHD_OPT_ADADELTA ? 4 : 3);
  return state + (with_ids ? (size_t)ctx->n_slots * sizeof(uint32_t) : 0);
}

// 0: not eligible (adaptive b, half-precision gathers, or too large); 1: ids
// read through L1; 2: ids in shared memory too; 4: persistent grid (resident = 3).
// 3: thread-block cluster (resident = 2, or automatically for graphs of at
// most kClusterAutoEntries stored entries, where it measured faster than one
// launch per step: 2,000-4,000 vertices 2.0-2.5 us against 3.1-3.4 us per step;
// at 5,000 vertices with hubs it was slower).
constexpr int64_t kClusterAutoEntries = 40000;
int resident_mode(const ivhd_ctx* ctx) {
  if (ctx->p.resident < 0 || ctx->p.adaptive || ctx->p.pos_format != IVHD_POS_F32) return 0;
  if (ctx->p.resident == 3) return 4;  // persistent grid: any size
  // the whole-call kernels give every row at most a warp; graphs with rows of
  // kWideRow entries or more run one step kernel per step instead
  if (ctx->n_wide > 0) return 0;
  if (ctx->M > ((int64_t)1 << 20)) return 0;
  if (ctx->p.resident == 0)
    return (ctx->nnz_sym <= kClusterAutoEntries &&
            resident_bytes(ctx, false) <= (size_t)kResidentSmem) ? 3 : 0;
  if (ctx->p.resident == 2)
    return resident_bytes(ctx, false) <= (size_t)kResidentSmem ? 3 : 0;
  if (resident_bytes(ctx, true) <= (size_t)kResidentSmem) return 2;
  if (resident_bytes(ctx, false) <= (size_t)kResidentSmem) return 1;
  return 0;
}

template <int MODE, int METRIC, bool IDS>
static cudaError_t launch_res(const StepArgs& A, int64_t n_iter, int64_t n_slots, size_t smem,
                              cudaStream_t s) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_resident<MODE, METRIC, IDS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kResidentSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  k_resident<MODE, METRIC, IDS><<<1, kResidentThreads, smem, s>>>(A, n_iter, n_slots);
  return cudaGetLastError();
}

template <int MODE, int METRIC>
static cudaError_t launch_res_ids(const StepArgs& A, int64_t n_iter, int64_t n_slots, int mode,
                                  size_t smem, cudaStream_t s) {
  return mode == 2 ? launch_res<MODE, METRIC, true>(A, n_iter, n_slots, smem, s)
                   : launch_res<MODE, METRIC, false>(A, n_iter, n_slots, smem, s);
}

// Warps of the warp-per-vertex region for ctx->vpw rows of medium degree per
// warp: rows with at least 512 / vpw entries keep a whole warp.
static void hub_map(const ivhd_ctx* ctx, int32_t* n_full, int32_t* mid_g, int32_t* warps) {
  const int vpw = ctx->vpw;
  int64_t full = ctx->n_hub;
  if (vpw == 2 || vpw == 4 || vpw == 8) {
    const int t = (vpw == 2) ? 0 : (vpw == 4) ? 1 : 2;  // 256, 128, 64 entries
    full = ctx->n_ge[t] < ctx->n_hub ? ctx->n_ge[t] : ctx->n_hub;
  }
  const int v = (full == ctx->n_hub) ? 1 : vpw;
  *n_full = (int32_t)full;
  *mid_g = 32 / v;
  *warps = (int32_t)(full + (ctx->n_hub - full + v - 1) / v);
}

static cudaError_t launch_grid(ivhd_ctx* ctx, int64_t n_iter, cudaStream_t s);

cudaError_t launch_resident(ivhd_ctx* ctx, int64_t n_iter, cudaStream_t s) {
  const int mode = resident_mode(ctx);
  if (mode == 0) return cudaErrorInvalidValue;
  if (mode == 4) return launch_grid(ctx, n_iter, s);
  StepArgs A{};
  A.ids = ctx->ids;
  A.hub_off = ctx->hub_off;
  A.slice_off = ctx->slice_off;
  A.slice_w = ctx->slice_w;
  A.y[0] = ctx->y[0];
  A.y[1] = ctx->y[1];
  A.v[0] = ctx->vbuf[0];
  A.s2 = ctx->s2;
  A.cur = ctx->cur;
  A.M = (int32_t)ctx->M;
  A.n_hub = (int32_t)ctx->n_hub;
  A.n_slices = (int32_t)ctx->n_slices;
  A.n_slots = ctx->n_slots;
  hub_map(ctx, &A.n_full, &A.mid_g, &A.hub_warps);
  A.c = ctx->c;
  A.a = ctx->p.a;
  A.b = ctx->p.b;
  A.rho = ctx->p.rho;
  A.eps = ctx->p.eps;
  const size_t smem = resident_bytes(ctx, mode == 2);
  const int64_t ns = ctx->n_slots;
  const bool l1 = ctx->metric == IVHD_METRIC_L1;
  if (mode == 3) {
    switch (ctx->p.opt) {
      case IVHD_OPT_NESTEROV:
        return l1 ? launch_cl<kNesterov, IVHD_METRIC_L1>(A, n_iter, smem, s)
                  : launch_cl<kNesterov, IVHD_METRIC_L2>(A, n_iter, smem, s);
      case IVHD_OPT_ADADELTA:
        return l1 ? launch_cl<kAdadelta, IVHD_METRIC_L1>(A, n_iter, smem, s)
                  : launch_cl<kAdadelta, IVHD_METRIC_L2>(A, n_iter, smem, s);
      default:
        return l1 ? launch_cl<kMomentum, IVHD_METRIC_L1>(A, n_iter, smem, s)
                  : launch_cl<kMomentum, IVHD_METRIC_L2>(A, n_iter, smem, s);
    }
  }
  switch (ctx->p.opt) {
    case IVHD_OPT_NESTEROV:
      return l1 ? launch_res_ids<kNesterov, IVHD_METRIC_L1>(A, n_iter, ns, mode, smem, s)
                : launch_res_ids<kNesterov, IVHD_METRIC_L2>(A, n_iter, ns, mode, smem, s);
    case IVHD_OPT_ADADELTA:
      return l1 ? launch_res_ids<kAdadelta, IVHD_METRIC_L1>(A, n_iter, ns, mode, smem, s)
                : launch_res_ids<kAdadelta, IVHD_METRIC_L2>(A, n_iter, ns, mode, smem, s);
    default:
      return l1 ? launch_res_ids<kMomentum, IVHD_METRIC_L1>(A, n_iter, ns, mode, smem, s)
                : launch_res_ids<kMomentum, IVHD_METRIC_L2>(A, n_iter, ns, mode, smem, s);
  }
}

// Sums the per-block partials in a fixed order; E = 1/2 of the symmetric sum
// because every term of Eq. 3.16 appears in the rows of both endpoints.
__global__ void __launch_bounds__(1024) k_stress_final(const double* __restrict__ partials, int n,
                                                       double* out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partials[i];
  const double t = block_sum(v, sh);
  if (threadIdx.x == 0) out[0] = 0.5 * t;
}

// Self-adaptive b (Sec. 3.3.3): with T = sum |dr|^2 over all particles before
// (T_old = |v|^2) and after (T_new = |v'|^2) the step, dT = T_new - T_old.
// When |dT| > tau T_old the step is rejected (positions and velocities stay at
// step n) and b is scaled by gamma1 > 1 (dT < 0) or gamma2 < 1 (dT > 0);
// otherwise the step is accepted (the ping-pong buffers flip).
__global__ void __launch_bounds__(1024) k_adapt(const double* __restrict__ partials, int nblocks,
                                                float tau, float gamma1, float gamma2,
                                                AdaptCtl* ctl) {
  // launched as a programmatic dependent of the step: wait for its partials,
  // then let the next step's blocks launch (they wait for this grid to finish)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ double sh[32];
  double tn = 0.0, to = 0.0;
  // four independent loads in flight per thread; the summation order is fixed
  const int stride = (int)blockDim.x;
  for (int i = threadIdx.x; i < nblocks; i += 4 * stride) {
    double a[4], c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = i + q * stride;
      a[q] = (j < nblocks) ? partials[2 * j] : 0.0;
      c[q] = (j < nblocks) ? partials[2 * j + 1] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      tn += a[q];
      to += c[q];
    }
  }
  tn = block_sum(tn, sh);
  to = block_sum(to, sh);
  if (threadIdx.x == 0) {
    const double dT = tn - to;
    if (to > 0.0 && fabs(dT) > (double)tau * to) {
      ctl->b *= (dT < 0.0) ? gamma1 : gamma2;
      ctl->rejected += 1;
    } else {
      ctl->cur ^= 1;
      ctl->accepted += 1;
    }
    ctl->last_dT = dT;
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

// y0 ~ U(0,1)^2 per input vertex i = perm[p] in its segment [lo, lo + n) with
// local index li = i - lo: coordinate q is the top 24 bits of output q of
// SplitMix64 seeded with s = output li of SplitMix64 seeded with
// (seed ^ "init_pos"), times 2^-24 (exact in FP32).
__global__ void k_init_positions(const int32_t* __restrict__ perm, int M, SegTable T,
                                 float2* __restrict__ y, float2* __restrict__ s1,
                                 float2* __restrict__ s2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= M) return;
  const int i = perm[p];
  const int e = T.of ? T.of[i] : 0;
  const uint64_t si = sm64_out(T.seed[e] ^ kDomainInit, (uint64_t)(i - T.lo[e]));
  const float sc = 1.0f / 16777216.0f;
  y[p] = make_float2((float)(sm64_out(si, 0) >> 40) * sc, (float)(sm64_out(si, 1) >> 40) * sc);
  s1[p] = make_float2(0.f, 0.f);
  if (s2) s2[p] = make_float2(0.f, 0.f);
}

// Optimiser state in input order (for a rebuild of the layout) and back.
__global__ void k_to_input_order(const float2* __restrict__ a, const int32_t* __restrict__ perm,
                                 int M, float2* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < M) out[perm[p]] = a[p];
}
__global__ void k_from_input_order(const float2* __restrict__ in, const int32_t* __restrict__ perm,
                                   int M, float2* __restrict__ a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < M) a[p] = in[perm[p]];
}

cudaError_t launch_to_input_order(ivhd_ctx* ctx, const float2* a, float2* out) {
  const int M = (int)ctx->M;
  k_to_input_order<<<(M + 255) / 256, 256, 0, ctx->stream>>>(a, ctx->perm, M, out);
  ++ctx->aux_launches;
  return cudaGetLastError();
}
cudaError_t launch_from_input_order(ivhd_ctx* ctx, const float2* in, float2* a) {
  const int M = (int)ctx->M;
  k_from_input_order<<<(M + 255) / 256, 256, 0, ctx->stream>>>(in, ctx->perm, M, a);
  ++ctx->aux_launches;
  return cudaGetLastError();
}

static StepArgs make_args(const ivhd_ctx* ctx, int cur) {
  StepArgs A{};
  A.ids = ctx->ids;
  A.hub_off = ctx->hub_off;
  A.slice_off = ctx->slice_off;
  A.slice_w = ctx->slice_w;
  A.y[0] = ctx->y[0];
  A.y[1] = ctx->y[1];
  A.yh[0] = ctx->yh[0];
  A.yh[1] = ctx->yh[1];
  A.v[0] = ctx->vbuf[0];
  A.v[1] = ctx->vbuf[1] ? ctx->vbuf[1] : ctx->vbuf[0];
  A.s2 = ctx->s2;
  A.cur = cur;
  A.ctl = ctx->ctl;
  A.perm = ctx->perm;
  A.partials = ctx->partials;
  A.flag = ctx->flag;
  A.M = (int32_t)ctx->M;
  A.n_hub = (int32_t)ctx->n_hub;
  A.n_slices = (int32_t)ctx->n_slices;
  A.n_slots = ctx->n_slots;
  A.wpb = ctx->block / 32;
  hub_map(ctx, &A.n_full, &A.mid_g, &A.hub_warps);
  // the wide rows lead the full-warp rows (both are the longest rows, in
  // descending degree); the hub warps take the rows after them
  A.n_wide = (int32_t)ctx->n_wide;
  A.nb_wide = (int32_t)((A.n_wide + A.wpb / kWideWarps - 1) / (A.wpb / kWideWarps));
  A.n_full -= A.n_wide;
  A.hub_warps -= A.n_wide;
  A.nb_hub = (int32_t)((A.hub_warps + A.wpb - 1) / A.wpb);
  A.c = ctx->c;
  A.a = ctx->p.a;
  A.b = ctx->p.b;
  A.rho = ctx->p.rho;
  A.eps = ctx->p.eps;
  return A;
}

template <int MODE, int METRIC>
static cudaError_t launch_persist(const StepArgs& A, int64_t n_iter, int n_vblocks,
                                  GridBarrier* bar, int32_t* err, cudaStream_t s) {
  int per_sm = 0, sms = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<MODE, METRIC>,
                                                      A.wpb * 32, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // every block resident at once (a cooperative launch refuses more)
  const int grid = n_vblocks < per_sm * sms ? n_vblocks : per_sm * sms;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)(A.wpb * 32));
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_persist<MODE, METRIC>, A, n_iter, n_vblocks, bar, err);
}

// The whole call on the persistent grid; the barrier state (and its error
// flag) are reset before the launch.
static cudaError_t launch_grid(ivhd_ctx* ctx, int64_t n_iter, cudaStream_t s) {
  if (!ctx->gbar) {
    cudaError_t e = dev_alloc((void**)&ctx->gbar, 16, s);
    if (e != cudaSuccess) return e;
  }
  GridBarrier* bar = reinterpret_cast<GridBarrier*>(ctx->gbar);
  int32_t* err = reinterpret_cast<int32_t*>(ctx->gbar + 8);
  cudaError_t e = cudaMemsetAsync(ctx->gbar, 0, 16, s);
  if (e != cudaSuccess) return e;
  const StepArgs A = make_args(ctx, ctx->cur);
  const int nvb = step_grid(ctx);
  const bool l1 = ctx->metric == IVHD_METRIC_L1;
  switch (ctx->p.opt) {
    case IVHD_OPT_NESTEROV:
      return l1 ? launch_persist<kNesterov, IVHD_METRIC_L1>(A, n_iter, nvb, bar, err, s)
                : launch_persist<kNesterov, IVHD_METRIC_L2>(A, n_iter, nvb, bar, err, s);
    case IVHD_OPT_ADADELTA:
      return l1 ? launch_persist<kAdadelta, IVHD_METRIC_L1>(A, n_iter, nvb, bar, err, s)
                : launch_persist<kAdadelta, IVHD_METRIC_L2>(A, n_iter, nvb, bar, err, s);
    default:
      return l1 ? launch_persist<kMomentum, IVHD_METRIC_L1>(A, n_iter, nvb, bar, err, s)
                : launch_persist<kMomentum, IVHD_METRIC_L2>(A, n_iter, nvb, bar, err, s);
  }
}

cudaError_t grid_timed_out(ivhd_ctx* ctx, bool* timed_out) {
  int32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ctx->gbar + 8, sizeof(h), cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  *timed_out = h != 0;
  return e;
}

int step_grid(const ivhd_ctx* ctx) {
  const int wpb = ctx->block / 32;
  int32_t n_full, mid_g, warps;
  hub_map(ctx, &n_full, &mid_g, &warps);
  const int64_t rows_per_block = wpb / kWideWarps;
  const int64_t nb_wide = (ctx->n_wide + rows_per_block - 1) / rows_per_block;
  const int64_t nb_hub = (warps - ctx->n_wide + wpb - 1) / wpb;
  const int64_t nb_sell = (ctx->n_slices + wpb - 1) / wpb;
  return (int)(nb_wide + nb_hub + nb_sell);
}

template <int MODE, int POS, int METRIC, bool ADAPT>
static void launch1(int grid, cudaStream_t s, const StepArgs& A) {
  // programmatic dependent launch: the next step's blocks start while this
  // step's last wave drains (0.5 % at 1.4e6 vertices, 5 % at 2,000)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)(A.wpb * 32));
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_step<MODE, POS, METRIC, ADAPT>, A);
}

template <int POS, int METRIC>
static void launch_opt(int opt, bool adapt, int grid, cudaStream_t s, const StepArgs& A) {
  switch (opt) {
    case IVHD_OPT_NESTEROV:
      if (adapt)
        launch1<kNesterov, POS, METRIC, true>(grid, s, A);
      else
        launch1<kNesterov, POS, METRIC, false>(grid, s, A);
      break;
    case IVHD_OPT_ADADELTA: launch1<kAdadelta, POS, METRIC, false>(grid, s, A); break;
    default:
      if (adapt)
        launch1<kMomentum, POS, METRIC, true>(grid, s, A);
      else
        launch1<kMomentum, POS, METRIC, false>(grid, s, A);
      break;
  }
}

template <int METRIC>
static void launch_pos(const ivhd_ctx* ctx, bool adapt, int grid, cudaStream_t s,
                       const StepArgs& A) {
  switch (ctx->p.pos_format) {
    case IVHD_POS_F16: launch_opt<IVHD_POS_F16, METRIC>(ctx->p.opt, adapt, grid, s, A); break;
    case IVHD_POS_BF16: launch_opt<IVHD_POS_BF16, METRIC>(ctx->p.opt, adapt, grid, s, A); break;
    default: launch_opt<IVHD_POS_F32, METRIC>(ctx->p.opt, adapt, grid, s, A); break;
  }
}

// One step: the fused kernel, plus the controller kernel with self-adaptive b.
cudaError_t launch_step(ivhd_ctx* ctx, int cur, cudaStream_t s) {
  const StepArgs A = make_args(ctx, cur);
  const int grid = step_grid(ctx);
  const bool adapt = ctx->p.adaptive != 0;
  if (ctx->metric == IVHD_METRIC_L1)
    launch_pos<IVHD_METRIC_L1>(ctx, adapt, grid, s, A);
  else
    launch_pos<IVHD_METRIC_L2>(ctx, adapt, grid, s, A);
  if (adapt) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(1024);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_adapt, (const double*)ctx->partials, grid, ctx->p.tau,
                       ctx->p.gamma1, ctx->p.gamma2, ctx->ctl);
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

// Arguments of the forces / stress evaluation at the FP32 positions y[cur]
// (Nesterov: y = z - a v, written into y[cur ^ 1] and read from there).
static StepArgs eval_args(ivhd_ctx* ctx) {
  StepArgs A = make_args(ctx, ctx->cur);
  if (ctx->p.opt == IVHD_OPT_NESTEROV) {
    const int M = (int)ctx->M;
    k_lookback<<<(M + 255) / 256, 256, 0, ctx->stream>>>(ctx->y[ctx->cur], ctx->s1, M, ctx->p.a,
                                                         ctx->y[ctx->cur ^ 1]);
    ++ctx->aux_launches;
    A.cur = ctx->cur ^ 1;
  }
  return A;
}

cudaError_t launch_forces(ivhd_ctx* ctx, float2* out) {
  StepArgs A = eval_args(ctx);
  A.f_out = out;
  if (ctx->metric == IVHD_METRIC_L1)
    k_step<kForces, IVHD_POS_F32, IVHD_METRIC_L1, false>
        <<<step_grid(ctx), ctx->block, 0, ctx->stream>>>(A);
  else
    k_step<kForces, IVHD_POS_F32, IVHD_METRIC_L2, false>
        <<<step_grid(ctx), ctx->block, 0, ctx->stream>>>(A);
  ++ctx->aux_launches;
  return cudaGetLastError();
}

cudaError_t launch_stress(ivhd_ctx* ctx) {
  cudaError_t e = cudaMemsetAsync(ctx->flag, 0, sizeof(int32_t), ctx->stream);
  if (e != cudaSuccess) return e;
  StepArgs A = eval_args(ctx);
  const int grid = step_grid(ctx);
  if (ctx->metric == IVHD_METRIC_L1)
    k_step<kStress, IVHD_POS_F32, IVHD_METRIC_L1, false><<<grid, ctx->block, 0, ctx->stream>>>(A);
  else
    k_step<kStress, IVHD_POS_F32, IVHD_METRIC_L2, false><<<grid, ctx->block, 0, ctx->stream>>>(A);
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
  k_init_positions<<<(M + 255) / 256, 256, 0, ctx->stream>>>(ctx->perm, M, ctx->seg,
                                                             ctx->y[ctx->cur], ctx->s1, ctx->s2);
  ++ctx->aux_launches;
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : launch_round_positions(ctx);
}

}  // namespace ivhd

using namespace ivhd;

extern "C" ivhd_status ivhd_check_violations(int64_t* out, int32_t reset) {
  if (!out) return IVHD_ERR_ARG;
#ifdef IVHD_CHECKED
  cudaError_t e = cudaDeviceSynchronize();
  unsigned long long v = 0;
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_check_violations, sizeof(v));
  if (e == cudaSuccess && reset) {
    const unsigned long long zero = 0;
    e = cudaMemcpyToSymbol(g_check_violations, &zero, sizeof(zero));
  }
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  *out = (int64_t)v;
#else
  (void)reset;
  *out = -1;
#endif
  return IVHD_OK;
}

extern "C" ivhd_status ivhd_test_corrupt_layout(ivhd_ctx* ctx, int64_t slot, uint32_t value) {
#ifdef IVHD_CHECKED
  if (!ctx || slot < 0 || slot >= ctx->n_slots) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaError_t e = cudaMemcpyAsync(ctx->ids + slot, &value, sizeof(value), cudaMemcpyHostToDevice,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return e == cudaSuccess ? IVHD_OK : IVHD_ERR_CUDA;
#else
  // only a build whose kernels test every index may hold a corrupt layout
  (void)ctx;
  (void)slot;
  (void)value;
  return IVHD_ERR_ARG;
#endif
}

extern "C" ivhd_status ivhd_probe_grid_barrier_timeout(int32_t polls, void* stream) {
  if (polls < 1) return IVHD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* buf = nullptr;
  if (dev_alloc((void**)&buf, 16, s) != cudaSuccess) return IVHD_ERR_OOM;
  cudaError_t e = cudaMemsetAsync(buf, 0, 16, s);
  GridBarrier* bar = reinterpret_cast<GridBarrier*>(buf);
  int32_t* err = reinterpret_cast<int32_t*>(buf + 8);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_probe_grid_barrier, bar, err, (unsigned)polls);
  }
  int32_t h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s);
  dev_free(buf, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  return h ? IVHD_ERR_TIMEOUT : IVHD_OK;
}
