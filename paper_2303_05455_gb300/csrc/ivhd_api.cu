// ivhd_api.cu -- the extern "C" entry points declared in include/ivhd.h.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <unordered_map>

#include "ivhd_internal.cuh"

namespace ivhd {

static std::atomic<int64_t> g_live_allocs{0};
static std::atomic<int64_t> g_fail_after{-1};  // allocations to grant before one fails; -1 = off

// The caller's allocator (ivhd_set_allocator) and the blocks it handed out,
// each with the free routine to return it to.  Never destroyed, so a context
// released during process teardown still finds its blocks.
struct UserAllocator {
  ivhd_alloc_fn alloc = nullptr;
  ivhd_free_fn release = nullptr;
  void* user = nullptr;
};
struct UserBlock {
  ivhd_free_fn release;
  void* user;
  size_t bytes;
};
static std::mutex& alloc_mutex() {
  static std::mutex* m = new std::mutex;
  return *m;
}
static UserAllocator g_user_alloc;  // guarded by alloc_mutex()
static std::unordered_map<void*, UserBlock>& user_blocks() {
  static auto* m = new std::unordered_map<void*, UserBlock>;
  return *m;
}

static bool take_injected_failure() {
  int64_t f = g_fail_after.load();
  while (f >= 0) {
    if (f == 0) {
      if (g_fail_after.compare_exchange_weak(f, -1)) return true;
    } else if (g_fail_after.compare_exchange_weak(f, f - 1)) {
      return false;
    }
  }
  return false;
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (take_injected_failure()) return cudaErrorMemoryAllocation;
  UserAllocator ua;
  {
    std::lock_guard<std::mutex> lock(alloc_mutex());
    ua = g_user_alloc;
  }
  if (ua.alloc) {
    // the callback runs without the lock held, so it may take its own locks
    void* q = ua.alloc(bytes, (void*)s, ua.user);
    if (!q) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
      ua.release(q, bytes, (void*)s, ua.user);
      return cudaErrorMemoryAllocation;
    }
    {
      std::lock_guard<std::mutex> lock(alloc_mutex());
      user_blocks()[q] = UserBlock{ua.release, ua.user, bytes};
    }
    *p = q;
    g_live_allocs.fetch_add(1);
    return cudaSuccess;
  }
  const cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  return e;
}

cudaError_t dev_free(void* p, cudaStream_t s) {
  if (!p) return cudaSuccess;
  g_live_allocs.fetch_sub(1);
  UserBlock b{};
  bool from_user = false;
  {
    std::lock_guard<std::mutex> lock(alloc_mutex());
    auto& m = user_blocks();
    auto it = m.find(p);
    if (it != m.end()) {
      b = it->second;
      m.erase(it);
      from_user = true;
    }
  }
  if (from_user) {
    b.release(p, b.bytes, (void*)s, b.user);
    return cudaSuccess;
  }
  return cudaFreeAsync(p, s);
}

NvtxScope::NvtxScope(const char* name) { nvtxRangePushA(name); }
NvtxScope::~NvtxScope() { nvtxRangePop(); }

}  // namespace ivhd

using namespace ivhd;

extern "C" ivhd_status ivhd_set_allocator(ivhd_alloc_fn alloc_fn, ivhd_free_fn free_fn,
                                          void* user) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr)) return IVHD_ERR_ARG;
  std::lock_guard<std::mutex> lock(alloc_mutex());
  g_user_alloc = UserAllocator{alloc_fn, free_fn, alloc_fn ? user : nullptr};
  return IVHD_OK;
}

extern "C" void ivhd_test_fail_alloc(int64_t after) { g_fail_after.store(after < 0 ? -1 : after); }
extern "C" int64_t ivhd_test_live_allocs(void) { return g_live_allocs.load(); }

namespace {

constexpr int kGraphSteps = 64;  // steps per captured CUDA graph (even: parity preserved)
constexpr uint32_t kStateMagic = 0x44485649u;  // "IVHD"
constexpr uint32_t kStateVersion = 2;

ivhd_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return IVHD_OK;
  if (e == cudaErrorMemoryAllocation) return IVHD_ERR_OOM;
  return IVHD_ERR_CUDA;
}

// Marks the context unusable after a CUDA failure.
ivhd_status fail(ivhd_ctx* ctx, cudaError_t e) {
  ivhd_status st = cuda_status(e);
  if (st == IVHD_ERR_CUDA && ctx) ctx->poisoned = true;
  return st;
}

bool params_ok(const ivhd_params& p) {
  if (p.opt < IVHD_OPT_MOMENTUM || p.opt > IVHD_OPT_ADADELTA) return false;
  if (!std::isfinite(p.a) || p.a < 0.f || p.a > 1.f) return false;
  if (!std::isfinite(p.b) || p.b <= 0.f) return false;
  if (!std::isfinite(p.rho) || p.rho <= 0.f || p.rho >= 1.f) return false;
  if (!std::isfinite(p.eps) || p.eps <= 0.f) return false;
  if (p.hub_threshold < 0 || p.hub_threshold > 65535) return false;
  if (p.pos_format < IVHD_POS_F32 || p.pos_format > IVHD_POS_BF16) return false;
  if (p.adaptive != 0 && p.adaptive != 1) return false;
  if (p.block_size != 0 && p.block_size != 128 && p.block_size != 256 && p.block_size != 512)
    return false;
  if (p.resident < -1 || p.resident > 3) return false;
  if (p.resident == 3 && (p.adaptive || p.pos_format != IVHD_POS_F32)) return false;
  if (p.vertices_per_warp != 0 && p.vertices_per_warp != 1 && p.vertices_per_warp != 2 &&
      p.vertices_per_warp != 4 && p.vertices_per_warp != 8)
    return false;
  if (p.order != IVHD_ORDER_DEGREE && p.order != IVHD_ORDER_DEGREE_CLUSTER) return false;
  if (p.adaptive) {
    if (p.opt == IVHD_OPT_ADADELTA) return false;
    if (!std::isfinite(p.tau) || p.tau <= 0.f) return false;
    if (!std::isfinite(p.gamma1) || p.gamma1 <= 1.f) return false;
    if (!std::isfinite(p.gamma2) || p.gamma2 <= 0.f || p.gamma2 >= 1.f) return false;
  }
  return true;
}

void drop_graphs(ivhd_ctx* ctx) {
  for (auto& row : ctx->graph_exec)
    for (auto& g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

void free_layout(ivhd_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  void* bufs[] = {ctx->ids, ctx->hub_off, ctx->slice_off, ctx->slice_w, ctx->partials};
  for (void* b : bufs)
    if (b) dev_free(b, s);
  ctx->ids = nullptr;
  ctx->hub_off = ctx->slice_off = ctx->slice_w = nullptr;
  ctx->partials = nullptr;
}

// The frees are stream-ordered: they take effect once the work already queued
// on the context's stream has run, so destroy does not wait for it.  They are
// queued before the graphs are destroyed, so that they are not held up behind
// graph executions that are still in flight (an in-flight graph is released
// when it completes).
void free_ctx(ivhd_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  free_layout(ctx);
  void* bufs[] = {ctx->knn, ctx->knn_full, ctx->rn, ctx->perm, ctx->inv, ctx->y[0], ctx->y[1],
                  ctx->yh[0], ctx->yh[1], ctx->vbuf[0], ctx->vbuf[1], ctx->s2, ctx->ctl,
                  ctx->red_out, ctx->flag, ctx->seg_of, ctx->seg_lo, ctx->seg_n, ctx->seg_r,
                  ctx->seg_seed, ctx->gbar};
  for (void* b : bufs)
    if (b) dev_free(b, s);
  drop_graphs(ctx);
  delete ctx;
}

template <class T>
cudaError_t dalloc(T** p, int64_t n, cudaStream_t s) {
  return dev_alloc((void**)p, (size_t)(n > 0 ? n : 1) * sizeof(T), s);
}

// With self-adaptive b the current buffer is chosen on the device; host code
// that touches the state first reads it back.
cudaError_t sync_cur(ivhd_ctx* ctx) {
  if (!ctx->ctl) return cudaSuccess;
  AdaptCtl h{};
  cudaError_t e = cudaMemcpyAsync(&h, ctx->ctl, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return e;
  ctx->cur = h.cur;
  ctx->s1 = ctx->vbuf[h.cur];
  return cudaSuccess;
}

// Partials for the stress (1 per block) and the adaptive controller (2 per block).
cudaError_t alloc_partials(ivhd_ctx* ctx) {
  ctx->n_partials = 2 * (int64_t)step_grid(ctx);
  return dalloc(&ctx->partials, ctx->n_partials, ctx->stream);
}

// 64-bit FNV-1a over the quantities a checkpoint must agree on.
uint64_t fingerprint(const ivhd_ctx* ctx) {
  uint64_t h = 0xcbf29ce484222325ull;
  auto mix = [&](const void* d, size_t n) {
    const unsigned char* b = (const unsigned char*)d;
    for (size_t q = 0; q < n; ++q) {
      h ^= b[q];
      h *= 0x100000001b3ull;
    }
  };
  mix(&ctx->M, sizeof(ctx->M));
  mix(&ctx->k, sizeof(ctx->k));
  mix(&ctx->r, sizeof(ctx->r));
  mix(&ctx->c, sizeof(ctx->c));
  mix(&ctx->p.opt, sizeof(ctx->p.opt));
  mix(&ctx->p.a, sizeof(ctx->p.a));
  mix(&ctx->p.b, sizeof(ctx->p.b));
  mix(&ctx->p.rho, sizeof(ctx->p.rho));
  mix(&ctx->p.eps, sizeof(ctx->p.eps));
  mix(&ctx->p.seed, sizeof(ctx->p.seed));
  mix(&ctx->p.dedup_mutual, sizeof(ctx->p.dedup_mutual));
  mix(&ctx->p.pos_format, sizeof(ctx->p.pos_format));
  mix(&ctx->p.order, sizeof(ctx->p.order));
  mix(&ctx->p.adaptive, sizeof(ctx->p.adaptive));
  mix(&ctx->nnz_sym, sizeof(ctx->nnz_sym));
  return h;
}

struct StateHeader {
  uint32_t magic, version;
  uint64_t fingerprint;
  int64_t M;
  int64_t steps_done;
  int32_t opt, n_arrays;
  AdaptCtl ctl;
};

// Rebuilds the layout (after the graph or the random neighbours changed) and
// carries positions and optimiser state across the new vertex order.
ivhd_status rebuild_preserving_state(ivhd_ctx* ctx, bool draw_rn, uint64_t epoch) {
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  cudaError_t e = sync_cur(ctx);
  if (e != cudaSuccess) return fail(ctx, e);
  float2* save[3] = {nullptr, nullptr, nullptr};
  float2* src[3] = {ctx->y[ctx->cur], ctx->s1, ctx->s2};
  const int n = ctx->s2 ? 3 : 2;
  for (int q = 0; q < n && e == cudaSuccess; ++q) {
    e = dalloc(&save[q], M, s);
    if (e == cudaSuccess) e = launch_to_input_order(ctx, src[q], save[q]);
  }
  ivhd_status st = IVHD_OK;
  if (e == cudaSuccess) {
    drop_graphs(ctx);
    free_layout(ctx);
    st = build_layout(ctx, draw_rn, epoch);
  }
  if (e == cudaSuccess && st == IVHD_OK) e = alloc_partials(ctx);
  for (int q = 0; q < n && e == cudaSuccess && st == IVHD_OK; ++q)
    e = launch_from_input_order(ctx, save[q], src[q]);
  if (e == cudaSuccess && st == IVHD_OK) e = launch_round_positions(ctx);
  for (int q = 0; q < n; ++q)
    if (save[q]) dev_free(save[q], s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, e);
  if (st != IVHD_OK) ctx->poisoned = true;  // the layout is gone
  return st;
}

// Keeps nn entry (i -> j) iff i is among helper[j] (Sec. 3.4.2 reading).
__global__ void k_restrict(const int32_t* __restrict__ knn, const int32_t* __restrict__ helper,
                           int64_t M, int k, int kh, int32_t* __restrict__ out,
                           int32_t* __restrict__ err) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * k) return;
  const int64_t i = e / k;
  const int32_t j = knn[e];
  int32_t keep = -1;
  if (j >= 0 && !*err) {
    for (int t = 0; t < kh; ++t)
      if (helper[(int64_t)j * kh + t] == (int32_t)i) keep = j;
  }
  out[e] = keep;
}

// Every helper id must be -1 or a vertex.
__global__ void k_check_ids(const int32_t* __restrict__ a, int64_t n, int64_t M,
                            int32_t* __restrict__ err) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n && (a[e] < -1 || (int64_t)a[e] >= M)) atomicOr(err, 1);
}

}  // namespace

extern "C" {

void ivhd_default_params(ivhd_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->opt = IVHD_OPT_MOMENTUM;
  p->a = 0.9f;
  p->b = 0.01f;
  p->rho = 0.95f;
  p->eps = 1e-6f;
  p->seed = 0;
  p->dedup_mutual = 0;
  p->init_uniform = 1;
  p->hub_threshold = 0;
  p->pos_format = IVHD_POS_F32;
  p->adaptive = 0;
  p->tau = 0.5f;
  p->gamma1 = 1.1f;
  p->gamma2 = 0.5f;
  p->stream = nullptr;
}

int32_t ivhd_version(void) { return (0 << 16) | (3 << 8) | 0; }

const char* ivhd_status_string(ivhd_status s) {
  switch (s) {
    case IVHD_OK: return "ok";
    case IVHD_ERR_ARG: return "invalid argument";
    case IVHD_ERR_INDEX: return "invalid graph index (out of range, self loop or duplicate)";
    case IVHD_ERR_OOM: return "out of device memory";
    case IVHD_ERR_CUDA: return "CUDA error";
    case IVHD_ERR_NONFINITE: return "non-finite value in the embedding";
    case IVHD_ERR_TIMEOUT: return "device-side wait timed out";
    case IVHD_ERR_STATE: return "context poisoned or state mismatch";
  }
  return "unknown status";
}

}  // extern "C"

namespace {

// Allocates the per-vertex state of a context with M vertices.
cudaError_t alloc_state(ivhd_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(dalloc(&ctx->rn, M * (int64_t)ctx->r, s));
  chk(dalloc(&ctx->perm, M, s));
  chk(dalloc(&ctx->inv, M, s));
  chk(dalloc(&ctx->y[0], M, s));
  chk(dalloc(&ctx->y[1], M, s));
  chk(dalloc(&ctx->vbuf[0], M, s));
  if (ctx->p.adaptive) {
    chk(dalloc(&ctx->vbuf[1], M, s));
    chk(dalloc(&ctx->ctl, 1, s));
  }
  if (ctx->p.opt == IVHD_OPT_ADADELTA) chk(dalloc(&ctx->s2, M, s));
  if (ctx->p.pos_format != IVHD_POS_F32) {
    chk(dalloc(&ctx->yh[0], M, s));
    chk(dalloc(&ctx->yh[1], M, s));
  }
  chk(dalloc(&ctx->red_out, 1, s));
  chk(dalloc(&ctx->flag, 1, s));
  ctx->s1 = ctx->vbuf[0];
  return e;
}

// Shared by the create entry points once the context holds its graph
// (ctx->knn), segment tables and parameters: layout, positions, controller.
ivhd_status finish_create(ivhd_ctx* ctx, ivhd_ctx** out) {
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  ivhd_status st = build_layout(ctx, true, 0);
  if (st != IVHD_OK) {
    free_ctx(ctx);
    return st;
  }
  cudaError_t e = alloc_partials(ctx);
  if (e == cudaSuccess) {
    if (ctx->p.init_uniform) {
      e = launch_init_positions(ctx);
    } else {
      e = cudaMemsetAsync(ctx->y[0], 0, (size_t)M * sizeof(float2), s);
      if (e == cudaSuccess && ctx->yh[0])
        e = cudaMemsetAsync(ctx->yh[0], 0, (size_t)M * sizeof(uint32_t), s);
      if (e == cudaSuccess) e = cudaMemsetAsync(ctx->s1, 0, (size_t)M * sizeof(float2), s);
      if (e == cudaSuccess && ctx->s2)
        e = cudaMemsetAsync(ctx->s2, 0, (size_t)M * sizeof(float2), s);
    }
  }
  if (e == cudaSuccess && ctx->ctl) {
    AdaptCtl h{};
    h.b = ctx->p.b;
    e = cudaMemcpyAsync(ctx->ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    st = cuda_status(e);
    free_ctx(ctx);
    return st;
  }
  *out = ctx;
  return IVHD_OK;
}

}  // namespace

extern "C" {

ivhd_status ivhd_create(const int32_t* knn, int64_t M, int32_t k, int32_t r, float c,
                        const ivhd_params* p_in, int32_t knn_on_device, ivhd_ctx** out) {
  NvtxScope nvtx_("ivhd_create");
  if (!out) return IVHD_ERR_ARG;
  *out = nullptr;
  if (!knn) return IVHD_ERR_ARG;
  if (M < 2 || M >= kMaxVertices) return IVHD_ERR_ARG;
  if (k < 1 || (int64_t)k > M - 1 || r < 0) return IVHD_ERR_ARG;
  if (!std::isfinite(c) || c <= 0.f) return IVHD_ERR_ARG;
  if ((int64_t)M * (int64_t)(k + r) * 2 >= (int64_t)0x7FFFFFFF) return IVHD_ERR_ARG;
  ivhd_params p;
  if (p_in)
    p = *p_in;
  else
    ivhd_default_params(&p);
  if (!params_ok(p)) return IVHD_ERR_ARG;

  ivhd_ctx* ctx = new (std::nothrow) ivhd_ctx();
  if (!ctx) return IVHD_ERR_OOM;
  ctx->p = p;
  ctx->M = M;
  ctx->k = k;
  ctx->r = r;
  ctx->c = c;
  ctx->hub_threshold = p.hub_threshold > 0 ? p.hub_threshold
                                            : auto_hub_threshold(2 * M * (int64_t)(k + r));
  ctx->block = p.block_size > 0 ? p.block_size : kStepBlock;
  ctx->vpw = p.vertices_per_warp > 0 ? p.vertices_per_warp
                                     : auto_vertices_per_warp(2 * M * (int64_t)(k + r));
  ctx->stream = (cudaStream_t)p.stream;
  cudaGetDevice(&ctx->device);
  cudaStream_t s = ctx->stream;

  cudaError_t e = alloc_state(ctx);
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(dalloc(&ctx->knn, M * k, s));
  // one segment: the whole graph
  ctx->n_seg = 1;
  chk(dalloc(&ctx->seg_lo, 1, s));
  chk(dalloc(&ctx->seg_n, 1, s));
  chk(dalloc(&ctx->seg_r, 1, s));
  chk(dalloc(&ctx->seg_seed, 1, s));
  if (e == cudaSuccess) {
    const int64_t lo = 0;
    chk(cudaMemcpyAsync(ctx->seg_lo, &lo, sizeof(lo), cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(ctx->seg_n, &M, sizeof(M), cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(ctx->seg_r, &r, sizeof(r), cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(ctx->seg_seed, &p.seed, sizeof(p.seed), cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(ctx->knn, knn, (size_t)(M * k) * sizeof(int32_t),
                        knn_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    chk(cudaStreamSynchronize(s));  // the host scalars above live on this stack frame
  }
  if (e != cudaSuccess) {
    ivhd_status st = cuda_status(e);
    free_ctx(ctx);
    return st;
  }
  ctx->seg = SegTable{nullptr, ctx->seg_lo, ctx->seg_n, ctx->seg_r, ctx->seg_seed};
  return finish_create(ctx, out);
}

void ivhd_destroy(ivhd_ctx* ctx) {
  if (ctx) free_ctx(ctx);
}

ivhd_status ivhd_set_positions(ivhd_ctx* ctx, const float* xy, int32_t on_device) {
  if (!ctx || !xy) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  const float2* src = (const float2*)xy;
  float2* tmp = nullptr;
  cudaError_t e = sync_cur(ctx);
  if (e == cudaSuccess && !on_device) {
    e = dalloc(&tmp, M, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tmp, xy, (size_t)M * sizeof(float2), cudaMemcpyHostToDevice, s);
    src = tmp;
  }
  if (e == cudaSuccess) e = launch_set_positions(ctx, src);
  if (tmp) dev_free(tmp, s);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s);
  return fail(ctx, e);
}

ivhd_status ivhd_step(ivhd_ctx* ctx, int64_t n_iter) {
  NvtxScope nvtx_("ivhd_step");
  if (!ctx || n_iter < 0) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaSuccess;
  if (n_iter > 0 && !ctx->ctl && resident_mode(ctx) > 0) {
    // the whole call in one launch: one block or a cluster with the state in
    // shared memory, or the persistent grid (which is waited for here)
    e = launch_resident(ctx, n_iter, s);
    if (e != cudaSuccess) return fail(ctx, e);
    if (resident_mode(ctx) == 4) {
      bool timed_out = false;
      e = grid_timed_out(ctx, &timed_out);
      if (e != cudaSuccess) return fail(ctx, e);
      if (timed_out) {
        ctx->poisoned = true;  // the steps stopped part-way
        return IVHD_ERR_TIMEOUT;
      }
    }
    if (n_iter & 1) ctx->cur ^= 1;
    ctx->launches += 1;
    ctx->steps_done += n_iter;
    return IVHD_OK;
  }
  int64_t left = n_iter;
  // with adaptive b the kernels pick their buffers on the device: one graph, no host flips
  const bool flip = ctx->ctl == nullptr;
  const int per_step = ctx->ctl ? 2 : 1;
  const int par = flip ? ctx->cur : 0;
  cudaGraphExec_t& gx = ctx->graph_exec[ctx->metric][par];
  // whole graphs of kGraphSteps steps, then single launches for the rest
  if (left >= kGraphSteps) {
    if (!gx) {
      cudaStream_t cap = nullptr;
      e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) return fail(ctx, e);
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        int cur = ctx->cur;
        for (int q = 0; q < kGraphSteps && e == cudaSuccess; ++q) {
          e = launch_step(ctx, cur, cap);
          if (flip) cur ^= 1;
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cap);
      if (e != cudaSuccess) return fail(ctx, e);
    }
    while (left >= kGraphSteps) {
      e = cudaGraphLaunch(gx, s);
      if (e != cudaSuccess) return fail(ctx, e);
      left -= kGraphSteps;
      ctx->launches += kGraphSteps * per_step;
      // kGraphSteps is even: the parity of cur is unchanged
    }
  }
  for (; left > 0; --left) {
    e = launch_step(ctx, ctx->cur, s);
    if (e != cudaSuccess) return fail(ctx, e);
    if (flip) ctx->cur ^= 1;
    ctx->launches += per_step;
  }
  ctx->steps_done += n_iter;
  return IVHD_OK;
}

ivhd_status ivhd_positions(ivhd_ctx* ctx, float* out, int32_t on_device) {
  NvtxScope nvtx_("ivhd_positions");
  if (!ctx || !out) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  cudaError_t e = sync_cur(ctx);
  if (e != cudaSuccess) return fail(ctx, e);
  if (on_device) return fail(ctx, launch_unpermute(ctx, (float2*)out));
  float2* tmp = nullptr;
  e = dalloc(&tmp, M, s);
  if (e == cudaSuccess) e = launch_unpermute(ctx, tmp);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, tmp, (size_t)M * sizeof(float2), cudaMemcpyDeviceToHost, s);
  if (tmp) dev_free(tmp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return fail(ctx, e);
}

ivhd_status ivhd_forces(ivhd_ctx* ctx, float* out, int32_t on_device) {
  NvtxScope nvtx_("ivhd_forces");
  if (!ctx || !out) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  cudaError_t e = sync_cur(ctx);
  if (e != cudaSuccess) return fail(ctx, e);
  if (on_device) return fail(ctx, launch_forces(ctx, (float2*)out));
  float2* tmp = nullptr;
  e = dalloc(&tmp, M, s);
  if (e == cudaSuccess) e = launch_forces(ctx, tmp);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, tmp, (size_t)M * sizeof(float2), cudaMemcpyDeviceToHost, s);
  if (tmp) dev_free(tmp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return fail(ctx, e);
}

ivhd_status ivhd_stress(ivhd_ctx* ctx, double* out) {
  NvtxScope nvtx_("ivhd_stress");
  if (!ctx || !out) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  cudaError_t e = sync_cur(ctx);
  if (e == cudaSuccess) e = launch_stress(ctx);
  int32_t flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, ctx->red_out, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, ctx->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, e);
  return flag ? IVHD_ERR_NONFINITE : IVHD_OK;
}

ivhd_status ivhd_warm_start(ivhd_ctx* ctx, const float* xy, int32_t on_device, int32_t* taken) {
  NvtxScope nvtx_("ivhd_warm_start");
  if (!ctx || !xy || !taken) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  *taken = 0;
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  // stress of the current positions (non-finite counts as +inf)
  double e0 = 0.0;
  ivhd_status st = ivhd_stress(ctx, &e0);
  if (st == IVHD_ERR_NONFINITE) e0 = INFINITY;
  else if (st != IVHD_OK) return st;
  // keep the current positions (input order) to fall back to
  float2* keep = nullptr;
  cudaError_t e = dalloc(&keep, M, s);
  if (e != cudaSuccess) return fail(ctx, e);
  e = launch_unpermute(ctx, keep);
  const float2* src = (const float2*)xy;
  float2* tmp = nullptr;
  if (e == cudaSuccess && !on_device) {
    e = dalloc(&tmp, M, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tmp, xy, (size_t)M * sizeof(float2), cudaMemcpyHostToDevice, s);
    src = tmp;
  }
  if (e == cudaSuccess) e = launch_set_positions(ctx, src);
  double e1 = INFINITY;
  if (e == cudaSuccess) {
    st = ivhd_stress(ctx, &e1);
    if (st == IVHD_ERR_NONFINITE) {
      e1 = INFINITY;
    } else if (st != IVHD_OK) {
      if (tmp) dev_free(tmp, s);
      dev_free(keep, s);
      return st;
    }
  }
  if (e == cudaSuccess) {
    if (e1 < e0)
      *taken = 1;
    else
      e = launch_set_positions(ctx, keep);  // plain IVHD's start stays, state zeroed
  }
  if (tmp) dev_free(tmp, s);
  dev_free(keep, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return fail(ctx, e);
}

ivhd_status ivhd_random_neighbors(ivhd_ctx* ctx, int32_t* out, int32_t on_device) {
  if (!ctx || !out) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  const size_t bytes = (size_t)(ctx->M * ctx->r) * sizeof(int32_t);
  if (bytes == 0) return IVHD_OK;
  cudaError_t e = cudaMemcpyAsync(out, ctx->rn, bytes,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(ctx->stream);
  return fail(ctx, e);
}

ivhd_status ivhd_info(ivhd_ctx* ctx, ivhd_info_t* out) {
  if (!ctx || !out) return IVHD_ERR_ARG;
  out->M = ctx->M;
  out->k = ctx->k;
  out->r = ctx->r;
  out->n_terms = ctx->n_terms;
  out->nnz_sym = ctx->nnz_sym;
  out->layout_slots = ctx->n_slots;
  out->n_hub = ctx->n_hub;
  out->max_degree = ctx->max_degree;
  out->empty_rn = ctx->empty_rn;
  out->steps_done = ctx->steps_done;
  out->kernel_launches = ctx->launches;
  out->setup_launches = ctx->setup_launches;
  out->aux_launches = ctx->aux_launches;
  const int rm = ctx->ctl ? 0 : resident_mode(ctx);
  out->launch_form = rm == 0 ? 0 : (rm <= 2 ? 1 : (rm == 3 ? 2 : 3));
  out->step_blocks = step_grid(ctx);
  out->step_threads = ctx->block;
  return IVHD_OK;
}

ivhd_status ivhd_set_metric(ivhd_ctx* ctx, int32_t metric) {
  if (!ctx || (metric != IVHD_METRIC_L2 && metric != IVHD_METRIC_L1)) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  ctx->metric = metric;
  return IVHD_OK;
}

ivhd_status ivhd_resample_random_neighbors(ivhd_ctx* ctx, uint64_t epoch) {
  if (!ctx) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  if (ctx->r == 0) return IVHD_OK;
  return rebuild_preserving_state(ctx, true, epoch);
}

ivhd_status ivhd_restrict_nn(ivhd_ctx* ctx, const int32_t* helper, int32_t k_helper,
                             int32_t on_device) {
  if (!ctx) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  const int k = ctx->k;
  cudaError_t e = cudaSuccess;
  if (!helper) {  // restore the full graph
    if (!ctx->knn_full) return IVHD_OK;
    e = cudaMemcpyAsync(ctx->knn, ctx->knn_full, (size_t)(M * k) * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(ctx, e);
    dev_free(ctx->knn_full, s);
    ctx->knn_full = nullptr;
    return rebuild_preserving_state(ctx, false, 0);
  }
  if (k_helper < 1 || (int64_t)k_helper > M - 1) return IVHD_ERR_ARG;
  if (!ctx->knn_full) {
    e = dalloc(&ctx->knn_full, M * k, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->knn_full, ctx->knn, (size_t)(M * k) * sizeof(int32_t),
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(ctx, e);
  }
  int32_t* hd = nullptr;
  int32_t* err = nullptr;
  int32_t herr = 0;
  const int32_t* hsrc = helper;
  if (!on_device) {
    e = dalloc(&hd, M * k_helper, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hd, helper, (size_t)(M * k_helper) * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s);
    hsrc = hd;
  }
  if (e == cudaSuccess) e = dalloc(&err, 1, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) {
    const int64_t nh = M * k_helper, n = M * k;
    k_check_ids<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(hsrc, nh, M, err);
    k_restrict<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctx->knn_full, hsrc, M, k, k_helper,
                                                          ctx->knn, err);
    ctx->aux_launches += 2;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (hd) dev_free(hd, s);
  if (err) dev_free(err, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, e);
  if (herr) {  // bad helper ids: put the full graph back untouched
    e = cudaMemcpyAsync(ctx->knn, ctx->knn_full, (size_t)(M * k) * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? IVHD_ERR_INDEX : fail(ctx, e);
  }
  return rebuild_preserving_state(ctx, false, 0);
}

ivhd_status ivhd_adaptive_state(ivhd_ctx* ctx, float* b, int64_t* accepted, int64_t* rejected) {
  if (!ctx || !ctx->ctl) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  AdaptCtl h{};
  cudaError_t e = cudaMemcpyAsync(&h, ctx->ctl, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(ctx, e);
  if (b) *b = h.b;
  if (accepted) *accepted = h.accepted;
  if (rejected) *rejected = h.rejected;
  return IVHD_OK;
}

ivhd_status ivhd_state_size(ivhd_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return IVHD_ERR_ARG;
  const int n_arrays = ctx->s2 ? 3 : 2;
  *bytes = sizeof(StateHeader) + (size_t)n_arrays * (size_t)ctx->M * sizeof(float2);
  return IVHD_OK;
}

// The checkpoint stores the arrays in the internal (degree-sorted) order; the
// fingerprint ties it to the same graph and parameters, so that order is the
// same.  A context whose layout was rebuilt (resampled or restricted) must be
// brought to the same layout before loading.
ivhd_status ivhd_get_state(ivhd_ctx* ctx, void* buf, size_t bytes) {
  size_t need = 0;
  if (ivhd_state_size(ctx, &need) != IVHD_OK || !buf || bytes < need) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaError_t e = sync_cur(ctx);
  if (e != cudaSuccess) return fail(ctx, e);
  StateHeader h{};
  h.magic = kStateMagic;
  h.version = kStateVersion;
  h.fingerprint = fingerprint(ctx);
  h.M = ctx->M;
  h.steps_done = ctx->steps_done;
  h.opt = ctx->p.opt;
  h.n_arrays = ctx->s2 ? 3 : 2;
  cudaStream_t s = ctx->stream;
  if (ctx->ctl) {
    e = cudaMemcpyAsync(&h.ctl, ctx->ctl, sizeof(h.ctl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, e);
  }
  std::memcpy(buf, &h, sizeof(h));
  char* q = (char*)buf + sizeof(h);
  const size_t ab = (size_t)ctx->M * sizeof(float2);
  e = cudaMemcpyAsync(q, ctx->y[ctx->cur], ab, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(q + ab, ctx->s1, ab, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && ctx->s2) e = cudaMemcpyAsync(q + 2 * ab, ctx->s2, ab, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return fail(ctx, e);
}

ivhd_status ivhd_set_state(ivhd_ctx* ctx, const void* buf, size_t bytes) {
  size_t need = 0;
  if (ivhd_state_size(ctx, &need) != IVHD_OK || !buf) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  if (bytes < sizeof(StateHeader)) return IVHD_ERR_STATE;
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kStateMagic || h.version != kStateVersion || h.fingerprint != fingerprint(ctx) ||
      h.M != ctx->M || h.opt != ctx->p.opt || h.n_arrays != (ctx->s2 ? 3 : 2) || bytes < need)
    return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaSuccess;
  if (ctx->ctl) {
    e = cudaMemcpyAsync(ctx->ctl, &h.ctl, sizeof(h.ctl), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = sync_cur(ctx);
    if (e != cudaSuccess) return fail(ctx, e);
  }
  const char* q = (const char*)buf + sizeof(h);
  const size_t ab = (size_t)ctx->M * sizeof(float2);
  e = cudaMemcpyAsync(ctx->y[ctx->cur], q, ab, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->s1, q + ab, ab, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && ctx->s2) e = cudaMemcpyAsync(ctx->s2, q + 2 * ab, ab, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_round_positions(ctx);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) ctx->steps_done = h.steps_done;
  return fail(ctx, e);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Many independent embeddings in one context, and the launch-shape autotuner.

namespace {

// seg_of[g] = the embedding that owns global vertex g (binary search over lo).
__global__ void k_seg_of(const int64_t* __restrict__ lo, int n_seg, int64_t M,
                         int32_t* __restrict__ of) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= M) return;
  int a = 0, b = n_seg - 1;
  while (a < b) {
    const int m = (a + b + 1) >> 1;
    if (lo[m] <= g) a = m; else b = m - 1;
  }
  of[g] = a;
}

// Local kNN rows (k_e ids in [0, M_e), -1 absent) -> global rows of k_max ids.
__global__ void k_globalize(const int32_t* __restrict__ local, const int64_t* __restrict__ row0,
                            const int64_t* __restrict__ lo, const int64_t* __restrict__ n,
                            const int32_t* __restrict__ ke, const int32_t* __restrict__ of,
                            int64_t M, int k_max, int32_t* __restrict__ knn,
                            int32_t* __restrict__ err) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= M) return;
  const int e = of[g];
  const int64_t i = g - lo[e];
  const int k = ke[e];
  for (int s = 0; s < k_max; ++s) {
    int32_t v = -1;
    if (s < k) {
      v = local[row0[e] + i * k + s];
      if (v < -1 || (int64_t)v >= n[e]) {
        atomicOr(err, 1);
        v = -1;
      }
    }
    knn[g * k_max + s] = v >= 0 ? (int32_t)(lo[e] + v) : -1;
  }
}

}  // namespace

extern "C" ivhd_status ivhd_create_batch(const int32_t* knn, const int64_t* M_e,
                                         const int32_t* k_e, const int32_t* r_e,
                                         const uint64_t* seed_e, int32_t n_emb, float c,
                                         const ivhd_params* p_in, int32_t knn_on_device,
                                         ivhd_ctx** out) {
  NvtxScope nvtx_("ivhd_create_batch");
  if (!out) return IVHD_ERR_ARG;
  *out = nullptr;
  if (!knn || !M_e || !k_e || !r_e || !seed_e || n_emb < 1 || n_emb > (1 << 20))
    return IVHD_ERR_ARG;
  if (!std::isfinite(c) || c <= 0.f) return IVHD_ERR_ARG;
  std::vector<int64_t> lo(n_emb), row0(n_emb), n(M_e, M_e + n_emb);
  int64_t M = 0, entries = 0;
  int k_max = 0, r_max = 0;
  int64_t sym_entries = 0;  // 2 M_e (k_e + r_e) summed: the default hub threshold's input
  for (int e = 0; e < n_emb; ++e) {
    if (M_e[e] < 2 || k_e[e] < 1 || (int64_t)k_e[e] > M_e[e] - 1 || r_e[e] < 0) return IVHD_ERR_ARG;
    lo[e] = M;
    row0[e] = entries;
    M += M_e[e];
    entries += M_e[e] * k_e[e];
    sym_entries += 2 * M_e[e] * (int64_t)(k_e[e] + r_e[e]);
    k_max = k_e[e] > k_max ? k_e[e] : k_max;
    r_max = r_e[e] > r_max ? r_e[e] : r_max;
    if (M >= kMaxVertices) return IVHD_ERR_ARG;
  }
  if (M * (int64_t)(k_max + r_max) * 2 >= (int64_t)0x7FFFFFFF) return IVHD_ERR_ARG;
  ivhd_params p;
  if (p_in)
    p = *p_in;
  else
    ivhd_default_params(&p);
  if (!params_ok(p)) return IVHD_ERR_ARG;

  ivhd_ctx* ctx = new (std::nothrow) ivhd_ctx();
  if (!ctx) return IVHD_ERR_OOM;
  ctx->p = p;
  ctx->M = M;
  ctx->k = k_max;
  ctx->r = r_max;
  ctx->c = c;
  ctx->hub_threshold = p.hub_threshold > 0 ? p.hub_threshold : auto_hub_threshold(sym_entries);
  ctx->block = p.block_size > 0 ? p.block_size : kStepBlock;
  ctx->vpw = p.vertices_per_warp > 0 ? p.vertices_per_warp : auto_vertices_per_warp(sym_entries);
  ctx->stream = (cudaStream_t)p.stream;
  cudaGetDevice(&ctx->device);
  cudaStream_t s = ctx->stream;
  ctx->n_seg = n_emb;

  cudaError_t e = alloc_state(ctx);
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  int32_t* local = nullptr;
  int64_t* row0_d = nullptr;
  int32_t* err = nullptr;
  int32_t herr = 0;
  chk(dalloc(&ctx->knn, M * k_max, s));
  chk(dalloc(&ctx->seg_of, M, s));
  chk(dalloc(&ctx->seg_lo, n_emb, s));
  chk(dalloc(&ctx->seg_n, n_emb, s));
  chk(dalloc(&ctx->seg_r, n_emb, s));
  chk(dalloc(&ctx->seg_seed, n_emb, s));
  chk(dalloc(&row0_d, n_emb, s));
  chk(dalloc(&err, 1, s));
  if (!knn_on_device) chk(dalloc(&local, entries, s));
  if (e == cudaSuccess) {
    chk(cudaMemcpyAsync(ctx->seg_lo, lo.data(), n_emb * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(ctx->seg_n, n.data(), n_emb * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(ctx->seg_r, r_e, n_emb * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(ctx->seg_seed, seed_e, n_emb * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(row0_d, row0.data(), n_emb * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    chk(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    if (!knn_on_device)
      chk(cudaMemcpyAsync(local, knn, (size_t)entries * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  }
  int32_t* kd = nullptr;  // per-embedding k
  chk(dalloc(&kd, n_emb, s));
  if (e == cudaSuccess) {
    chk(cudaMemcpyAsync(kd, k_e, n_emb * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    const unsigned g = (unsigned)((M + 255) / 256);
    k_seg_of<<<g, 256, 0, s>>>(ctx->seg_lo, n_emb, M, ctx->seg_of);
    k_globalize<<<g, 256, 0, s>>>(knn_on_device ? knn : local, row0_d, ctx->seg_lo, ctx->seg_n, kd,
                                  ctx->seg_of, M, k_max, ctx->knn, err);
    ctx->setup_launches += 2;
    chk(cudaGetLastError());
    chk(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
    chk(cudaStreamSynchronize(s));
  }
  if (local) dev_free(local, s);
  if (row0_d) dev_free(row0_d, s);
  if (err) dev_free(err, s);
  if (kd) dev_free(kd, s);
  if (e != cudaSuccess || herr) {
    ivhd_status st = herr ? IVHD_ERR_INDEX : cuda_status(e);
    free_ctx(ctx);
    return st;
  }
  ctx->seg = SegTable{ctx->seg_of, ctx->seg_lo, ctx->seg_n, ctx->seg_r, ctx->seg_seed};
  return finish_create(ctx, out);
}

extern "C" ivhd_status ivhd_autotune(ivhd_ctx* ctx, int32_t trial_steps, int32_t* best_block,
                                     int32_t* best_hub_threshold,
                                     int32_t* best_vertices_per_warp, float* best_us_per_step) {
  NvtxScope nvtx_("ivhd_autotune");
  if (!ctx || trial_steps < 1) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  cudaError_t e = sync_cur(ctx);
  if (e != cudaSuccess) return fail(ctx, e);
  // the state in input order (layouts change between candidates) and the controller
  float2* save[3] = {nullptr, nullptr, nullptr};
  const int n = ctx->s2 ? 3 : 2;
  AdaptCtl ctl_save{};
  for (int q = 0; q < n && e == cudaSuccess; ++q) {
    e = dalloc(&save[q], M, s);
    float2* src = q == 0 ? ctx->y[ctx->cur] : (q == 1 ? ctx->s1 : ctx->s2);
    if (e == cudaSuccess) e = launch_to_input_order(ctx, src, save[q]);
  }
  if (e == cudaSuccess && ctx->ctl)
    e = cudaMemcpyAsync(&ctl_save, ctx->ctl, sizeof(ctl_save), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  auto restore = [&]() -> cudaError_t {
    cudaError_t x = cudaSuccess;
    if (ctx->ctl) {
      x = cudaMemcpyAsync(ctx->ctl, &ctl_save, sizeof(ctl_save), cudaMemcpyHostToDevice, s);
      if (x == cudaSuccess) x = cudaStreamSynchronize(s);
      if (x == cudaSuccess) x = sync_cur(ctx);
    }
    for (int q = 0; q < n && x == cudaSuccess; ++q) {
      float2* dst = q == 0 ? ctx->y[ctx->cur] : (q == 1 ? ctx->s1 : ctx->s2);
      x = launch_from_input_order(ctx, save[q], dst);
    }
    if (x == cudaSuccess) x = launch_round_positions(ctx);
    return x;
  };
  const int blocks[3] = {128, 256, 512};
  const int hubs[6] = {16, 32, 64, 128, 256, 512};
  const int vpws[4] = {1, 2, 4, 8};
  float best = 1e30f;
  int bb = ctx->block, bh = ctx->hub_threshold, bv = ctx->vpw;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  ivhd_status st = IVHD_OK;
  const int64_t steps_before = ctx->steps_done;
  for (int hi = 0; hi < 6 && e == cudaSuccess && st == IVHD_OK; ++hi) {
    ctx->hub_threshold = hubs[hi];
    drop_graphs(ctx);
    free_layout(ctx);
    st = build_layout(ctx, false, 0);
    for (int c = 0; c < 12 && e == cudaSuccess && st == IVHD_OK; ++c) {
      const int bi = c / 4, vi = c % 4;
      ctx->block = blocks[bi];
      ctx->vpw = vpws[vi];
      if (ctx->partials) dev_free(ctx->partials, s);
      ctx->partials = nullptr;
      e = alloc_partials(ctx);
      if (e == cudaSuccess) e = restore();
      if (e == cudaSuccess) e = launch_step(ctx, ctx->ctl ? 0 : ctx->cur, s);  // warm-up
      if (e == cudaSuccess && !ctx->ctl) ctx->cur ^= 1;
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int t = 0; t < trial_steps && e == cudaSuccess; ++t) {
        e = launch_step(ctx, ctx->cur, s);
        if (!ctx->ctl) ctx->cur ^= 1;
        ctx->launches += ctx->ctl ? 2 : 1;
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      const float us = 1e3f * ms / trial_steps;
      if (e == cudaSuccess && us < best) {
        best = us;
        bb = blocks[bi];
        bh = hubs[hi];
        bv = vpws[vi];
      }
    }
  }
  // settle on the winner with the original state
  if (e == cudaSuccess && st == IVHD_OK) {
    ctx->hub_threshold = bh;
    ctx->block = bb;
    ctx->vpw = bv;
    drop_graphs(ctx);
    free_layout(ctx);
    st = build_layout(ctx, false, 0);
    if (st == IVHD_OK) e = alloc_partials(ctx);
    if (st == IVHD_OK && e == cudaSuccess) e = restore();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  ctx->steps_done = steps_before;
  for (int q = 0; q < n; ++q)
    if (save[q]) dev_free(save[q], s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(ctx, e);
  if (st != IVHD_OK) {
    ctx->poisoned = true;
    return st;
  }
  if (best_block) *best_block = bb;
  if (best_hub_threshold) *best_hub_threshold = bh;
  if (best_vertices_per_warp) *best_vertices_per_warp = bv;
  if (best_us_per_step) *best_us_per_step = best;
  return IVHD_OK;
}
