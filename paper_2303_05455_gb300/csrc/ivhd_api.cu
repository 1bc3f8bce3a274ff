// ivhd_api.cu -- the extern "C" entry points declared in include/ivhd.h.
#include <cmath>
#include <cstring>
#include <new>

#include "ivhd_internal.cuh"

using namespace ivhd;

namespace {

constexpr int kGraphSteps = 64;  // steps per captured CUDA graph (even: parity preserved)
constexpr uint32_t kStateMagic = 0x44485649u;  // "IVHD"
constexpr uint32_t kStateVersion = 1;

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
  return true;
}

void free_ctx(ivhd_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  for (int q = 0; q < 2; ++q)
    if (ctx->graph_exec[q]) cudaGraphExecDestroy(ctx->graph_exec[q]);
  void* bufs[] = {ctx->knn, ctx->rn, ctx->perm, ctx->inv, ctx->ids, ctx->hub_off,
                  ctx->slice_off, ctx->slice_w, ctx->y[0], ctx->y[1], ctx->yh[0], ctx->yh[1],
                  ctx->s1, ctx->s2, ctx->partials, ctx->red_out, ctx->flag};
  for (void* b : bufs)
    if (b) cudaFreeAsync(b, s);
  cudaStreamSynchronize(s);
  delete ctx;
}

template <class T>
cudaError_t dalloc(T** p, int64_t n, cudaStream_t s) {
  return cudaMallocAsync((void**)p, (size_t)(n > 0 ? n : 1) * sizeof(T), s);
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
  mix(&ctx->nnz_sym, sizeof(ctx->nnz_sym));
  return h;
}

struct StateHeader {
  uint32_t magic, version;
  uint64_t fingerprint;
  int64_t M;
  int64_t steps_done;
  int32_t opt, n_arrays;
};

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
  p->stream = nullptr;
}

int32_t ivhd_version(void) { return (0 << 16) | (1 << 8) | 0; }

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

ivhd_status ivhd_create(const int32_t* knn, int64_t M, int32_t k, int32_t r, float c,
                        const ivhd_params* p_in, int32_t knn_on_device, ivhd_ctx** out) {
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
  ctx->hub_threshold = p.hub_threshold > 0 ? p.hub_threshold : kDefaultHubThreshold;
  ctx->stream = (cudaStream_t)p.stream;
  cudaGetDevice(&ctx->device);
  cudaStream_t s = ctx->stream;

  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(dalloc(&ctx->knn, M * k, s));
  chk(dalloc(&ctx->rn, M * (int64_t)r, s));
  chk(dalloc(&ctx->perm, M, s));
  chk(dalloc(&ctx->inv, M, s));
  chk(dalloc(&ctx->y[0], M, s));
  chk(dalloc(&ctx->y[1], M, s));
  chk(dalloc(&ctx->s1, M, s));
  if (p.opt == IVHD_OPT_ADADELTA) chk(dalloc(&ctx->s2, M, s));
  if (p.pos_format != IVHD_POS_F32) {
    chk(dalloc(&ctx->yh[0], M, s));
    chk(dalloc(&ctx->yh[1], M, s));
  }
  chk(dalloc(&ctx->red_out, 1, s));
  chk(dalloc(&ctx->flag, 1, s));
  if (e != cudaSuccess) {
    ivhd_status st = cuda_status(e);
    free_ctx(ctx);
    return st;
  }
  chk(cudaMemcpyAsync(ctx->knn, knn, (size_t)(M * k) * sizeof(int32_t),
                      knn_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if (e != cudaSuccess) {
    ivhd_status st = cuda_status(e);
    free_ctx(ctx);
    return st;
  }
  ivhd_status st = build_layout(ctx);
  if (st != IVHD_OK) {
    free_ctx(ctx);
    return st;
  }
  ctx->n_partials = step_grid(ctx);
  chk(dalloc(&ctx->partials, ctx->n_partials, s));
  if (p.init_uniform) {
    chk(launch_init_positions(ctx));
  } else {
    chk(cudaMemsetAsync(ctx->y[0], 0, (size_t)M * sizeof(float2), s));
    if (ctx->yh[0]) chk(cudaMemsetAsync(ctx->yh[0], 0, (size_t)M * sizeof(uint32_t), s));
    chk(cudaMemsetAsync(ctx->s1, 0, (size_t)M * sizeof(float2), s));
    if (ctx->s2) chk(cudaMemsetAsync(ctx->s2, 0, (size_t)M * sizeof(float2), s));
  }
  if (e != cudaSuccess) {
    st = cuda_status(e);
    free_ctx(ctx);
    return st;
  }
  *out = ctx;
  return IVHD_OK;
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
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    e = dalloc(&tmp, M, s);
    if (e != cudaSuccess) return fail(ctx, e);
    e = cudaMemcpyAsync(tmp, xy, (size_t)M * sizeof(float2), cudaMemcpyHostToDevice, s);
    src = tmp;
  }
  if (e == cudaSuccess) e = launch_set_positions(ctx, src);
  if (tmp) cudaFreeAsync(tmp, s);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s);
  return fail(ctx, e);
}

ivhd_status ivhd_step(ivhd_ctx* ctx, int64_t n_iter) {
  if (!ctx || n_iter < 0) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaSuccess;
  int64_t left = n_iter;
  // whole graphs of kGraphSteps launches, then single launches for the rest
  if (left >= kGraphSteps) {
    if (!ctx->graph_exec[ctx->cur]) {
      cudaStream_t cap = nullptr;
      e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) return fail(ctx, e);
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        int cur = ctx->cur;
        for (int q = 0; q < kGraphSteps && e == cudaSuccess; ++q) {
          e = launch_step(ctx, cur, cap);
          cur ^= 1;
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph_exec[ctx->cur], g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cap);
      if (e != cudaSuccess) return fail(ctx, e);
    }
    while (left >= kGraphSteps) {
      e = cudaGraphLaunch(ctx->graph_exec[ctx->cur], s);
      if (e != cudaSuccess) return fail(ctx, e);
      left -= kGraphSteps;
      ctx->launches += kGraphSteps;
      // kGraphSteps is even: the parity of cur is unchanged
    }
  }
  for (; left > 0; --left) {
    e = launch_step(ctx, ctx->cur, s);
    if (e != cudaSuccess) return fail(ctx, e);
    ctx->cur ^= 1;
    ctx->launches += 1;
  }
  ctx->steps_done += n_iter;
  return IVHD_OK;
}

ivhd_status ivhd_positions(ivhd_ctx* ctx, float* out, int32_t on_device) {
  if (!ctx || !out) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  cudaError_t e = cudaSuccess;
  if (on_device) {
    e = launch_unpermute(ctx, (float2*)out);
    return fail(ctx, e);
  }
  float2* tmp = nullptr;
  e = dalloc(&tmp, M, s);
  if (e == cudaSuccess) e = launch_unpermute(ctx, tmp);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, tmp, (size_t)M * sizeof(float2), cudaMemcpyDeviceToHost, s);
  if (tmp) cudaFreeAsync(tmp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return fail(ctx, e);
}

ivhd_status ivhd_forces(ivhd_ctx* ctx, float* out, int32_t on_device) {
  if (!ctx || !out) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  cudaError_t e = cudaSuccess;
  if (on_device) return fail(ctx, launch_forces(ctx, (float2*)out));
  float2* tmp = nullptr;
  e = dalloc(&tmp, M, s);
  if (e == cudaSuccess) e = launch_forces(ctx, tmp);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, tmp, (size_t)M * sizeof(float2), cudaMemcpyDeviceToHost, s);
  if (tmp) cudaFreeAsync(tmp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return fail(ctx, e);
}

ivhd_status ivhd_stress(ivhd_ctx* ctx, double* out) {
  if (!ctx || !out) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  cudaStream_t s = ctx->stream;
  cudaError_t e = launch_stress(ctx);
  int32_t flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, ctx->red_out, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, ctx->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, e);
  return flag ? IVHD_ERR_NONFINITE : IVHD_OK;
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
  return IVHD_OK;
}

ivhd_status ivhd_state_size(ivhd_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return IVHD_ERR_ARG;
  const int n_arrays = ctx->s2 ? 3 : 2;
  *bytes = sizeof(StateHeader) + (size_t)n_arrays * (size_t)ctx->M * sizeof(float2);
  return IVHD_OK;
}

// The checkpoint stores the arrays in the internal (degree-sorted) order; the
// fingerprint ties it to the same graph and parameters, so that order is the same.
ivhd_status ivhd_get_state(ivhd_ctx* ctx, void* buf, size_t bytes) {
  size_t need = 0;
  if (ivhd_state_size(ctx, &need) != IVHD_OK || !buf || bytes < need) return IVHD_ERR_ARG;
  if (ctx->poisoned) return IVHD_ERR_STATE;
  StateHeader h{};
  h.magic = kStateMagic;
  h.version = kStateVersion;
  h.fingerprint = fingerprint(ctx);
  h.M = ctx->M;
  h.steps_done = ctx->steps_done;
  h.opt = ctx->p.opt;
  h.n_arrays = ctx->s2 ? 3 : 2;
  std::memcpy(buf, &h, sizeof(h));
  char* q = (char*)buf + sizeof(h);
  const size_t ab = (size_t)ctx->M * sizeof(float2);
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(q, ctx->y[ctx->cur], ab, cudaMemcpyDeviceToHost, s);
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
  const char* q = (const char*)buf + sizeof(h);
  const size_t ab = (size_t)ctx->M * sizeof(float2);
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(ctx->y[ctx->cur], q, ab, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->s1, q + ab, ab, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && ctx->s2) e = cudaMemcpyAsync(ctx->s2, q + 2 * ab, ab, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_round_positions(ctx);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) ctx->steps_done = h.steps_done;
  return fail(ctx, e);
}

}  // extern "C"
