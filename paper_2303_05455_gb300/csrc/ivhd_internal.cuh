// ivhd_internal.cuh -- shared definitions of the libivhd CUDA sources.
//
// Device layout of one embedding context (all arrays in HBM, vertex order
// "p" = the degree-sorted order chosen at create, see ivhd_build.cu):
//
//   y[2]       float2[M]  positions, ping-pong (step reads y[cur], writes y[cur^1]);
//                         for Nesterov they hold the look-ahead point y + a v
//   yh[2]      uint32[M]  FP16x2 / BF16x2 copies of y that neighbours gather
//                         (only with a half-precision position format)
//   s1         float2[M]  velocity (momentum, Nesterov) or E[g^2] (Adadelta)
//   s2         float2[M]  E[dx^2] (Adadelta only)
//   ids        uint32[]   symmetric adjacency; entry = neighbour p-index (30 bits),
//                         bit 31 set for a random-neighbour term, bit 30 set for
//                         an nn entry of weight 2 (a mutual kNN pair counted with
//                         multiplicity, gathered once), 0xFFFFFFFF = padding
//   hub rows   p < n_hub: contiguous rows ids[hub_off[p] .. hub_off[p+1]),
//                         lengths padded to a multiple of 4, one warp per row
//   SELL rows  p >= n_hub: slices of 32 consecutive vertices; slice s starts at
//                         ids[slice_off[s]] and stores slice_w[s] groups of 4 slots
//                         as [group][lane][4] so that a warp reads one group with
//                         one coalesced 512-byte int4 load
//   perm/inv   int32[M]   p -> input vertex id, input vertex id -> p
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ivhd.h"

namespace ivhd {

// Every device allocation of the library goes through these two calls
// (stream-ordered cudaMallocAsync / cudaFreeAsync, or the caller's allocator
// set with ivhd_set_allocator).  They count the live
// allocations, so tests can check that error paths free what they took, and
// ivhd_test_fail_alloc can make one of them fail to exercise those paths.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
cudaError_t dev_free(void* p, cudaStream_t s);

// Names the enclosing host scope in profiler timelines (NVTX range; a no-op
// unless a tool is attached).
struct NvtxScope {
  explicit NvtxScope(const char* name);
  ~NvtxScope();
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};

constexpr uint32_t kRnBit = 0x80000000u;  // random-neighbour term
constexpr uint32_t kW2Bit = 0x40000000u;  // nn entry standing for a mutual pair (weight 2)
constexpr uint32_t kIdxMask = 0x3FFFFFFFu;
constexpr uint32_t kPad = 0xFFFFFFFFu;
constexpr int64_t kMaxVertices = (int64_t)1 << 30;
constexpr int kDefaultHubThreshold = 128;
constexpr int kStepBlock = 128;      // default threads per step block (4 warps)

// Default hub threshold for a graph with about `entries` symmetric row entries
// (2 M (k + r) before mutual pairs merge): the largest power of two not above
// entries / 70,000, within [16, 256].  A SELL slice of rows just below the
// threshold is a chain of threshold / 8 dependent gather rounds for its warp;
// small graphs finish in a few such chains, so a low threshold (short chains,
// more warp-per-vertex rows) wins, while large graphs are throughput-bound and
// lose lanes to short warp rows.  Measured best shapes: 2,000 and 70,000
// vertices (k = 2 / 5, r = 1): 16; 1.4e6 vertices (k = 5, r = 1): 128; 64
// embeddings with 3.7e6 vertices in total: 256.
inline int auto_hub_threshold(int64_t entries) {
  int h = 16;
  while (h < 256 && (int64_t)(2 * h) * 70000 <= entries) h *= 2;
  return h;
}
// Rows of medium degree per warp in the warp-per-vertex region by default.
// With the lowest hub threshold (graphs below ~2.2M symmetric entries) most
// warp-per-vertex rows have 16-31 entries, i.e. 4-8 int4 groups for 32 lanes:
// two rows share a warp (16 lanes each), which halves those warps and brings
// a 70,000-vertex launch to about one wave (exact kNN graph of the
// MNIST-shaped set: 5.9 against 6.6 us per step; 4 rows per warp 6.4 us).
// Larger graphs keep a whole warp per row (1.4e6 points: equal within noise).
inline int auto_vertices_per_warp(int64_t entries) {
  return auto_hub_threshold(entries) <= 16 ? 2 : 1;
}
constexpr int kMaxStepBlock = 512;   // the autotuner tries 128, 256 and 512
constexpr int kWideRow = 512;        // rows with at least this many entries get kWideWarps warps
constexpr int kWideWarps = 4;
constexpr int kResidentSmem = 200 * 1024;  // shared memory of the resident whole-run kernel

enum Mode { kMomentum = 0, kNesterov = 1, kAdadelta = 2, kForces = 3, kStress = 4 };

// SplitMix64 (Steele, Lea, Flood 2014): output t of the generator seeded
// with s is mix(s + (t+1) * gamma), mix = the variant-13 finaliser.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kDomainRn = 0x726E5F6C69737473ull;    // "rn_lists"
constexpr uint64_t kDomainInit = 0x696E69745F706F73ull;  // "init_pos"

__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm64_out(uint64_t seed, uint64_t t) {
  return sm64_mix(seed + (t + 1) * kGamma);
}

// Read-only streaming load that does not allocate in L1 (the id stream is
// touched once per step; L1 is left to the position gathers).
__device__ __forceinline__ int4 ld_stream_v4(const int4* p) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// Independent embeddings sharing one context ("segments"): vertex i belongs to
// segment of[i] (or 0 when of is null), which spans [lo, lo + n), draws r
// random neighbours inside itself and seeds its streams with seed.
struct SegTable {
  const int32_t* of;
  const int64_t* lo;
  const int64_t* n;
  const int32_t* r;
  const uint64_t* seed;
};

// Device control word of the self-adaptive b scheme (Sec. 3.3.3).
struct AdaptCtl {
  int32_t cur;       // current ping-pong buffer
  int32_t accepted;  // accepted steps
  int32_t rejected;  // rejected steps
  float b;           // current force scale
  double last_dT;    // kinetic-energy change of the last attempted step
};

// Per-step arguments of the fused kernel (passed by value).  Buffers come in
// ping-pong pairs: a step reads [cur] and writes [cur ^ 1]; velocities are
// updated in place (v[0]) except with self-adaptive b, where they ping-pong too
// and cur comes from the device control word.
struct StepArgs {
  const uint32_t* __restrict__ ids;
  const int32_t* __restrict__ hub_off;
  const int32_t* __restrict__ slice_off;
  const int32_t* __restrict__ slice_w;
  float2* y[2];
  uint32_t* yh[2];  // rounded FP16 / BF16 copies gathered by neighbours
  float2* v[2];     // velocity or E[g^2]
  float2* __restrict__ s2;
  int32_t cur;
  AdaptCtl* ctl;
  const int32_t* __restrict__ perm;  // forces mode: scatter to input order
  float2* __restrict__ f_out;        // forces mode output
  double* __restrict__ partials;     // stress: one double per block; adaptive: two
  int32_t* __restrict__ flag;        // stress mode: non-finite flag
  int32_t M, n_hub, n_slices, nb_hub, wpb;
  // warp-per-vertex rows: the first n_full take a whole warp each, the others
  // share a warp, mid_g lanes per row; hub_warps warps cover all of them
  int32_t n_full, mid_g, hub_warps;
  // the first n_wide rows (the longest) take kWideWarps warps each, in the
  // first nb_wide blocks, before the hub warps
  int32_t n_wide, nb_wide;
  int64_t n_slots;  // layout entries (checked builds test row extents against it)
  float c, a, b, rho, eps;
};

}  // namespace ivhd

// The opaque context of the public ABI.
struct ivhd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  ivhd_params p{};
  int64_t M = 0;
  int32_t k = 0, r = 0;
  float c = 0.f;
  int hub_threshold = ivhd::kDefaultHubThreshold;
  int block = ivhd::kStepBlock;
  int vpw = 1;  // rows of medium degree per warp (1, 2, 4, 8)
  bool poisoned = false;

  // segments (independent embeddings) and their device tables
  ivhd::SegTable seg{};
  int32_t n_seg = 1;
  int32_t* seg_of = nullptr;
  int64_t* seg_lo = nullptr;
  int64_t* seg_n = nullptr;
  int32_t* seg_r = nullptr;
  uint64_t* seg_seed = nullptr;

  // graph and layout
  int32_t* knn_full = nullptr;  // unrestricted kNN rows, kept while a restriction is active
  int32_t* knn = nullptr;   // M*k, input ids, -1 = absent entry
  int32_t* rn = nullptr;    // M*r, input ids, -1 empty
  int32_t* perm = nullptr;  // p -> i
  int32_t* inv = nullptr;   // i -> p
  uint32_t* ids = nullptr;
  int32_t* hub_off = nullptr;
  int32_t* slice_off = nullptr;
  int32_t* slice_w = nullptr;
  int64_t n_slots = 0, n_hub = 0, n_slices = 0;
  int64_t n_ge[3] = {0, 0, 0};  // rows with at least 256, 128, 64 entries (all hub rows)
  int64_t n_wide = 0;           // hub rows with at least kWideRow entries (kWideWarps warps each)

  // state
  float2* y[2] = {nullptr, nullptr};
  uint32_t* yh[2] = {nullptr, nullptr};  // FP16 / BF16 gathered copies (pos_format != F32)
  int cur = 0;
  float2* vbuf[2] = {nullptr, nullptr};  // velocity / E[g^2]; [1] only with adaptive b
  float2* s1 = nullptr;                  // = vbuf[cur] with adaptive b, else vbuf[0]
  float2* s2 = nullptr;
  ivhd::AdaptCtl* ctl = nullptr;         // adaptive b only
  int metric = IVHD_METRIC_L2;

  // scratch for reductions
  double* partials = nullptr;
  double* red_out = nullptr;
  int32_t* flag = nullptr;
  int64_t n_partials = 0;
  unsigned char* gbar = nullptr;  // persistent grid: barrier (8 bytes) + error flag (4 bytes)

  // CUDA graphs of kGraphSteps steps, per metric and starting parity
  cudaGraphExec_t graph_exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};

  // counters
  int64_t n_terms = 0, nnz_sym = 0;  // stress terms; stored (gathered) row entries
  int32_t max_degree = 0, empty_rn = 0;
  int64_t steps_done = 0, launches = 0, setup_launches = 0, aux_launches = 0;
};

namespace ivhd {

// ivhd_build.cu: builds the layout from ctx->knn (and ctx->rn unless draw_rn);
// a redraw with epoch e > 0 reseeds the random-neighbour streams.
ivhd_status build_layout(ivhd_ctx* ctx, bool draw_rn, uint64_t rn_epoch);

// ivhd_step.cu
cudaError_t launch_step(ivhd_ctx* ctx, int cur, cudaStream_t s);
// Resident whole-run kernel: all n_iter steps in one single-block launch for
// embeddings whose state fits one SM (resident_mode > 0).
int resident_mode(const ivhd_ctx* ctx);
cudaError_t launch_resident(ivhd_ctx* ctx, int64_t n_iter, cudaStream_t s);
// After a persistent-grid launch: waits for it and reports whether a grid
// barrier gave up (bounded wait expired).
cudaError_t grid_timed_out(ivhd_ctx* ctx, bool* timed_out);
cudaError_t launch_forces(ivhd_ctx* ctx, float2* out_input_order);
cudaError_t launch_stress(ivhd_ctx* ctx);  // result in ctx->red_out[0], flag in ctx->flag
cudaError_t launch_unpermute(ivhd_ctx* ctx, float2* out_input_order);
cudaError_t launch_set_positions(ivhd_ctx* ctx, const float2* in_input_order);
cudaError_t launch_init_positions(ivhd_ctx* ctx);
cudaError_t launch_round_positions(ivhd_ctx* ctx);
cudaError_t launch_to_input_order(ivhd_ctx* ctx, const float2* a, float2* out);
cudaError_t launch_from_input_order(ivhd_ctx* ctx, const float2* in, float2* a);
int step_grid(const ivhd_ctx* ctx);

}  // namespace ivhd
