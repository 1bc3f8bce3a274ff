/*
 * ivhd.h -- C ABI of the GB300 IVHD embedding library (libivhd.so).
 *
 * IVHD embeds the kNN graph of a high-dimensional dataset in 2-D by
 * minimising the stress of Sec. 3.3.1, Eq. 3.16 of B. Minch, "In search of the
 * most efficient and memory-saving visualization of high dimensional data"
 * (2023):
 *
 *     E = sum_i [ sum_{j in O_nn(i)} d_ij^2  +  c * sum_{k in O_rn(i)} (1 - d_ik)^2 ],
 *
 * i.e. every vertex is pulled to distance 0 from its k nearest neighbours and
 * held at distance 1 from r random, unconnected vertices (binary targets,
 * Eq. 3.15).  Each step computes the force F = -1/2 grad E over the
 * symmetrised graph and applies the optimiser update (force-directed momentum
 * Eq. 3.34, or the Nesterov / Adadelta variants of Sec. 3.3.2) in one fused
 * CUDA kernel.  The graph is the problem statement of Sec. 3.3 (embedding of
 * the kNN graph G(V, E)); the brute-force kNN build of Sec. 5.1 is exposed as a
 * separate, untimed set-up call.
 *
 * Conventions for every call:
 *   - Return an ivhd_status; no call aborts, traps, prints or throws.
 *   - "Device" pointers are CUDA global-memory addresses on the current
 *     device (e.g. torch tensor data pointers); "host" pointers are ordinary
 *     (pageable or pinned) host memory.  Layouts are row-major and packed.
 *   - Work is enqueued on the stream given at create time (NULL = the legacy
 *     default stream) and is asynchronous unless a call says it synchronises.
 *     Device outputs are valid once that stream reaches the call.
 *   - The library copies every input it keeps; it never retains a caller
 *     pointer after a call returns.  Caller buffers stay caller-owned.
 *   - After IVHD_ERR_CUDA the context is poisoned: later calls on it return
 *     IVHD_ERR_STATE, except ivhd_destroy.
 *   - One context must not be used from two host threads at once.
 */
#ifndef IVHD_H_
#define IVHD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ivhd_ctx ivhd_ctx; /* opaque; owned by the library */

typedef enum {
    IVHD_OK = 0,
    IVHD_ERR_ARG = -1,        /* bad size, parameter or null pointer */
    IVHD_ERR_INDEX = -2,      /* graph id out of range, self loop or duplicate in a row */
    IVHD_ERR_OOM = -3,        /* device allocation failed */
    IVHD_ERR_CUDA = -4,       /* a CUDA runtime call or kernel failed */
    IVHD_ERR_NONFINITE = -5,  /* NaN or Inf found in the embedding */
    IVHD_ERR_TIMEOUT = -6,    /* a bounded device-side wait gave up */
    IVHD_ERR_STATE = -7       /* context poisoned, or checkpoint does not match */
} ivhd_status;

typedef enum {
    IVHD_OPT_MOMENTUM = 0, /* force-directed / momentum: v <- a v + b F; y <- y + v (Eq. 3.34) */
    IVHD_OPT_NESTEROV = 1, /* v <- a v + b F(y + a v); y <- y + v (Sec. 3.3.2) */
    IVHD_OPT_ADADELTA = 2  /* Zeiler's Adadelta on g = -F (Sec. 3.3.2), no learning rate */
} ivhd_opt;

typedef enum {
    IVHD_KNN_F32 = 0, /* float32 features; decided by the FP32 chain acc = fma(x-y, x-y, acc) */
    IVHD_KNN_U8 = 1   /* uint8 features; exact integer squared distances */
} ivhd_knn_dtype;

/*
 * Storage of the positions that the step kernel gathers from neighbours.
 * With F16 / BF16 every vertex keeps an FP32 master position (and FP32
 * optimiser state) for its own update, and a rounded copy (round to nearest
 * even) that neighbours gather, halving the bytes per gather.  Differences
 * y_j - y_i are taken between rounded copies (coincident points stay exactly
 * coincident); forces accumulate in FP32.  ivhd_forces / ivhd_stress /
 * ivhd_positions always use the FP32 master positions.
 */
typedef enum { IVHD_POS_F32 = 0, IVHD_POS_F16 = 1, IVHD_POS_BF16 = 2 } ivhd_pos_format;

/*
 * Distance used by the stress and its forces.  L2 is the method (Eq. 3.16).
 * L1 (d = |dx| + |dy|, gradient taken coordinate-wise with sign(0) = 0) is the
 * late-stage variant of Sec. 3.4.1, which the paper applies for the last ~50
 * steps to pull outliers into their clusters.  See ivhd_set_metric.
 */
typedef enum { IVHD_METRIC_L2 = 0, IVHD_METRIC_L1 = 1 } ivhd_metric;

typedef struct {
    int32_t opt;          /* ivhd_opt; default IVHD_OPT_MOMENTUM */
    float a;              /* friction / momentum a in [0, 1]; default 0.9 */
    float b;              /* force scale (learning rate) b > 0; default 0.01 */
    float rho;            /* Adadelta decay in (0, 1); default 0.95 */
    float eps;            /* Adadelta epsilon > 0; default 1e-6 */
    uint64_t seed;        /* seeds random neighbours and initial positions; default 0 */
    int32_t dedup_mutual; /* 0: a mutual kNN pair gives two nn terms (literal Eq. 3.16);
                             1: each unordered nn pair gives one term; default 0 */
    int32_t init_uniform; /* 1: y0 ~ U(0,1)^2 drawn from seed; 0: y0 = 0 until
                             ivhd_set_positions; default 1 */
    int32_t hub_threshold;/* vertices with at least this many symmetric terms are
                             processed warp-per-vertex; 0 = library default: the largest
                             power of two not above 2 M (k + r) / 70,000, within
                             [16, 256] (low for small, latency-bound graphs) */
    int32_t pos_format;   /* ivhd_pos_format of the positions the step kernel gathers;
                             default IVHD_POS_F32 */
    int32_t adaptive;     /* 1: self-adaptive b of Sec. 3.3.3 (momentum and Nesterov only);
                             default 0 */
    float tau;            /* adaptive b: a step whose kinetic-energy change dT satisfies
                             |dT| > tau * T_old is rejected; default 0.5 */
    float gamma1;         /* adaptive b: factor (> 1) applied to b when dT < 0; default 1.1 */
    float gamma2;         /* adaptive b: factor (0, 1) applied to b when dT > 0; default 0.5 */
    int32_t block_size;   /* threads per block of the step kernel: 128, 256 or 512;
                             0 = library default (128); see ivhd_autotune */
    int32_t resident;     /* whole ivhd_step calls in one launch, for small embeddings whose
                             positions and optimiser state fit an SM's shared memory
                             (about 8,000 vertices; FP32 gathers, no adaptive b), with
                             results equal to one launch per step bit for bit:
                             2: a cluster of 8 blocks, each with a full copy of the
                             positions, updated through distributed shared memory;
                             1: a single block; 0 (default): the cluster for graphs of at
                             most 40,000 stored entries, where it is faster, else one
                             launch per step; -1: always one launch per step;
                             3: a persistent cooperative grid of any size (FP32 gathers,
                             no adaptive b, else IVHD_ERR_ARG): every block stays
                             resident for the whole call and the steps are separated by
                             a grid barrier with a bounded wait (IVHD_ERR_TIMEOUT if it
                             expires); ivhd_step then synchronises.  Results equal one
                             launch per step bit for bit; measured slower on every
                             workload tried (us per step, grid / one launch per step:
                             2,000 vertices 4.2 / 3.0, 70,000 14.8 / 7.6, 1.4e6 80.2 /
                             56.0, 64 embeddings in one context 197 / 156), so opt-in */
    int32_t vertices_per_warp; /* warp-per-vertex rows of medium degree processed several
                             to a warp: 1, 2, 4 or 8 rows per warp, each on 32 / that many
                             lanes, for the rows below 512 / that many entries (longer rows
                             keep a whole warp); 0 = library default: 1 (a whole warp per
                             row).  Measured (us per step, hub threshold / rows per warp):
                             random 200,000-vertex graph with hubs 16/4 11.0 against 12.0
                             for the best shape with 1; no gain on the exact kNN graphs of
                             70,000 and 1.4e6 points.  ivhd_autotune searches it */
    int32_t order;        /* vertex order of the layout (ivhd_order); default
                             IVHD_ORDER_DEGREE */
    void *stream;         /* cudaStream_t for all work of the context; NULL = default stream */
} ivhd_params;

/*
 * Vertex order of the step kernel's layout.  DEGREE: descending symmetric
 * degree, ties in input order (rows of equal length share a warp; the paper's
 * IVHD-CUDA sorts particles by connection count, Sec. 5.2).  DEGREE_CLUSTER:
 * descending degree, then, among vertices of equal degree, grouped by the
 * connected component of the undirected kNN graph that the vertex belongs to
 * (components ordered by their smallest input id), then input order -- so
 * that positions gathered together are stored together where the graph has
 * cluster structure.  Results agree with DEGREE within FP32 rounding (the
 * summation order of a vertex's terms follows the layout).
 */
typedef enum { IVHD_ORDER_DEGREE = 0, IVHD_ORDER_DEGREE_CLUSTER = 1 } ivhd_order;

/* Fills *p with the defaults listed above.  p must not be NULL. */
void ivhd_default_params(ivhd_params *p);

/*
 * Creates an embedding context for the kNN graph `knn` (M rows of k vertex
 * ids, row-major int32, row i lists O_nn(i); Sec. 3.3).  Draws r random
 * neighbours per vertex (a vertex connected to i in either direction is never
 * its random neighbour, Sec. 3.3.3; draws use SplitMix64 from p->seed, fixed
 * for the life of the context), symmetrises the graph so that every term acts
 * on both endpoints, lays it out for the step kernel, and initialises the
 * positions and optimiser state (velocity or Adadelta accumulators = 0).
 *
 *   knn           M*k int32; host memory if knn_on_device == 0, else device.
 *                 -1 marks an absent entry (a vertex with fewer than k
 *                 neighbours keeps those it has, Sec. 3.3.3).
 *                 Copied; the caller keeps ownership.
 *   M             number of vertices, 2 <= M < 2^30.
 *   k             nearest neighbours per row, 1 <= k <= M - 1.
 *   r             random neighbours per vertex, r >= 0.  When fewer than r
 *                 unconnected vertices exist the missing slots stay empty.
 *   c             random-neighbour weight, c > 0 and finite (Eq. 3.16).
 *   p             parameters (NULL = defaults).
 *   out           receives the new context; set to NULL on failure.
 *
 * Synchronises the stream once (to read validation results and layout sizes).
 * Errors: IVHD_ERR_ARG for sizes/parameters (including a symmetrised graph
 * whose layout needs 2^31 or more slots), IVHD_ERR_INDEX when an id is outside
 * [0, M), equals its row index or repeats within its row, IVHD_ERR_OOM,
 * IVHD_ERR_CUDA.
 */
ivhd_status ivhd_create(const int32_t *knn, int64_t M, int32_t k, int32_t r, float c,
                        const ivhd_params *p, int32_t knn_on_device, ivhd_ctx **out);

/*
 * Creates one context holding n_emb independent embeddings (for example
 * several datasets, seeds or parameter sets of one sweep), so that every step
 * of all of them is one kernel launch over the concatenated vertices.  The
 * paper motivates many quick re-embeddings with different parameters
 * (Sec. 3.4, interactive choice of nn, rn and c).  Embedding e has M_e[e]
 * vertices, k_e[e] nearest neighbours per row, r_e[e] random neighbours
 * (drawn inside embedding e only) and seed seed_e[e]; c and all parameters in
 * p are shared.  Random neighbours and initial positions of embedding e are
 * exactly those ivhd_create would draw for it alone with seed_e[e].
 *
 *   knn   the rows of all embeddings concatenated in order: M_e[e] rows of
 *         k_e[e] local ids in [0, M_e[e]) (-1 = absent) for e = 0..n_emb-1;
 *         host or device per knn_on_device.
 *   M_e, k_e, r_e, seed_e   host arrays of n_emb entries.
 * Positions, forces and the other per-vertex calls use the concatenated
 * vertex order (embedding 0 first).  ivhd_stress sums all embeddings.
 * Constraints: 1 <= n_emb <= 2^20, each M_e >= 2, 1 <= k_e <= M_e - 1,
 * r_e >= 0, sum of M_e < 2^30.  Synchronises.  Errors as ivhd_create.
 */
ivhd_status ivhd_create_batch(const int32_t *knn, const int64_t *M_e, const int32_t *k_e,
                              const int32_t *r_e, const uint64_t *seed_e, int32_t n_emb,
                              float c, const ivhd_params *p, int32_t knn_on_device,
                              ivhd_ctx **out);

/*
 * Launch-shape autotuner: times trial_steps steps for every combination of
 * threads per block (128, 256, 512), hub threshold (16, 32, 64, 128, 256, 512:
 * the degree from which a vertex gets warp lanes instead of one lane) and
 * vertices per warp (1, 2, 4, 8: how many rows of medium degree share a warp),
 * starting each trial from the same state, then keeps the fastest and restores
 * the state, so the embedding continues exactly as before the call (with the
 * new layout's summation order).  Outputs (host, may be NULL): the chosen
 * block size, hub threshold, vertices per warp and microseconds per step.
 * Synchronises.  Errors: IVHD_ERR_ARG, IVHD_ERR_CUDA, IVHD_ERR_OOM,
 * IVHD_ERR_STATE.
 */
ivhd_status ivhd_autotune(ivhd_ctx *ctx, int32_t trial_steps, int32_t *best_block,
                          int32_t *best_hub_threshold, int32_t *best_vertices_per_warp,
                          float *best_us_per_step);

/*
 * Overwrites the positions with xy (M*2 float32, row-major, vertex order of
 * the input graph) and zeroes the optimiser state.  on_device selects the
 * memory space of xy.  Errors: IVHD_ERR_ARG, IVHD_ERR_CUDA, IVHD_ERR_STATE.
 */
ivhd_status ivhd_set_positions(ivhd_ctx *ctx, const float *xy, int32_t on_device);

/*
 * Warm start with plain IVHD as the fallback (Sec. 3.4: IVHD also serves as,
 * and can start from, an initial configuration; here the placement of a
 * learned network or any other method).  Evaluates the stress E (Eq. 3.16)
 * of the current positions and of the placement xy (M*2 FP32, input vertex
 * order; host or device per on_device) on the GPU, and keeps the placement
 * only if its stress is finite and strictly below the current one (a
 * non-finite current stress counts as +inf); otherwise the current positions
 * are restored.  *taken (host) receives 1 if the placement was kept, else 0.
 * Either way the optimiser state is zeroed, as by ivhd_set_positions.  For a
 * batch context the rule applies to the summed stress of all embeddings.
 * Synchronises.  Errors: IVHD_ERR_ARG, IVHD_ERR_STATE, IVHD_ERR_OOM,
 * IVHD_ERR_CUDA.
 */
ivhd_status ivhd_warm_start(ivhd_ctx *ctx, const float *xy, int32_t on_device, int32_t *taken);

/*
 * Runs n_iter synchronous steps (Sec. 5.2 scheme: all forces from the same
 * configuration, then all updates).  Each step is one launch of the fused
 * gather-force + optimiser kernel; steps are replayed from a CUDA graph.
 * Asynchronous.  n_iter = 0 is a no-op.  Errors: IVHD_ERR_ARG (n_iter < 0),
 * IVHD_ERR_CUDA, IVHD_ERR_STATE.
 */
ivhd_status ivhd_step(ivhd_ctx *ctx, int64_t n_iter);

/*
 * Writes the current positions y (M*2 float32, input vertex order) to out.
 * For Nesterov the positions are y, not the look-ahead point.  With
 * on_device == 0 out is host memory and the call synchronises the stream.
 */
ivhd_status ivhd_positions(ivhd_ctx *ctx, float *out, int32_t on_device);

/*
 * Writes F = -1/2 grad E at the current positions y (M*2 float32, input
 * vertex order; Sec. 3.3.1, Eq. 3.14 with the sign reading that makes F the
 * descent direction).  For Nesterov this is y, not the look-ahead point.
 * Does not change the state.  Host output synchronises.
 */
ivhd_status ivhd_forces(ivhd_ctx *ctx, float *out, int32_t on_device);

/*
 * Computes the stress E of Eq. 3.16 at the current positions y (FP32 terms,
 * FP64 deterministic reduction) into *out (host) and checks every position
 * for NaN/Inf.  Synchronises.  Returns IVHD_ERR_NONFINITE (with *out set to
 * the computed value) when a position is not finite.
 */
ivhd_status ivhd_stress(ivhd_ctx *ctx, double *out);

/*
 * Copies the random neighbours drawn at create (M*r int32, input vertex ids,
 * -1 for an empty slot) to out.  Host output synchronises.
 */
ivhd_status ivhd_random_neighbors(ivhd_ctx *ctx, int32_t *out, int32_t on_device);

/* Counters of a context. */
typedef struct {
    int64_t M;
    int32_t k, r;
    int64_t n_terms;       /* undirected terms of Eq. 3.16 (nn + rn) */
    int64_t nnz_sym;       /* symmetric row entries gathered per step: 2 per term, except
                              that a mutual kNN pair is one entry per endpoint (of weight 2
                              when multiplicity is kept) */
    int64_t layout_slots;  /* id slots stored, including padding */
    int64_t n_hub;         /* vertices processed warp-per-vertex */
    int32_t max_degree;    /* largest symmetric degree */
    int32_t empty_rn;      /* random-neighbour slots left empty */
    int64_t steps_done;
    int64_t kernel_launches; /* step kernels launched since create */
    int64_t setup_launches;  /* kernels launched by ivhd_create (layout set-up) */
    int64_t aux_launches;    /* other kernels (positions, forces, stress, set/init) */
    int32_t launch_form;     /* how ivhd_step runs: 0 one step kernel per step (CUDA-graph
                                replay), 1 one block for the whole call, 2 a cluster of 8
                                blocks for the whole call, 3 a persistent grid for the
                                whole call (see ivhd_params.resident) */
    int32_t step_blocks;     /* blocks of one step-kernel launch (launch form 0) */
    int32_t step_threads;    /* threads per block of the step kernel */
} ivhd_info_t;

/* Fills *out.  Host only; does not synchronise. */
ivhd_status ivhd_info(ivhd_ctx *ctx, ivhd_info_t *out);

/*
 * Checkpoint / resume.  The state holds the positions, the optimiser state,
 * the step counter and a fingerprint of (M, k, r, c, parameters, seed), so a
 * state only loads into a context created from the same graph and
 * parameters (IVHD_ERR_STATE otherwise).  Resuming reproduces an
 * uninterrupted run bit for bit.  Buffers are host memory; get/set
 * synchronise.  ivhd_state_size gives the byte count.
 */
ivhd_status ivhd_state_size(ivhd_ctx *ctx, size_t *bytes);
ivhd_status ivhd_get_state(ivhd_ctx *ctx, void *buf, size_t bytes);
ivhd_status ivhd_set_state(ivhd_ctx *ctx, const void *buf, size_t bytes);

/*
 * Selects the distance of subsequent steps, forces and stress (ivhd_metric).
 * The paper switches to L1 for the last steps of an embedding (Sec. 3.4.1).
 * Host only; takes effect in stream order.  Errors: IVHD_ERR_ARG.
 */
ivhd_status ivhd_set_metric(ivhd_ctx *ctx, int32_t metric);

/*
 * Redraws the random neighbours (Sec. 3.3.1: rn "generated ad hoc during the
 * embedding") and rebuilds the layout, keeping positions, optimiser state and
 * step count.  Draw epoch e > 0 seeds every vertex stream with
 * seed ^ mix(e) (mix = the SplitMix64 finaliser) instead of seed; e = 0
 * reproduces the draw of ivhd_create.  Synchronises.
 * Errors: IVHD_ERR_CUDA, IVHD_ERR_OOM, IVHD_ERR_STATE.
 */
ivhd_status ivhd_resample_random_neighbors(ivhd_ctx *ctx, uint64_t epoch);

/*
 * Reverse-neighbour mechanism (Sec. 3.4.2): keeps only the nn interactions
 * (i -> j) of the calculation graph for which i is among the k_helper nearest
 * neighbours of j in the helper graph (the paper's default helper has 4 nn
 * neighbours per row), so that an interaction survives when the two particles
 * are mutual neighbours or one is a reverse neighbour of the other.  Random
 * neighbours are unchanged.  Rebuilds the layout keeping positions,
 * optimiser state and step count; helper == NULL restores the full graph.
 *   helper  M*k_helper int32 rows (-1 = absent), host or device per on_device.
 * Synchronises.  Errors: IVHD_ERR_ARG, IVHD_ERR_INDEX, IVHD_ERR_CUDA, IVHD_ERR_OOM.
 */
ivhd_status ivhd_restrict_nn(ivhd_ctx *ctx, const int32_t *helper, int32_t k_helper,
                             int32_t on_device);

/*
 * State of the self-adaptive b controller: the current b and the numbers of
 * accepted and rejected steps.  Synchronises.  IVHD_ERR_ARG when the context
 * was created without adaptive b.
 */
ivhd_status ivhd_adaptive_state(ivhd_ctx *ctx, float *b, int64_t *accepted, int64_t *rejected);

/*
 * Frees the context and its device memory.  The memory is released in stream
 * order, after the work already queued on the context's stream; the call does
 * not wait for that work.  NULL is a no-op.
 */
void ivhd_destroy(ivhd_ctx *ctx);

/* A static, human-readable name for a status.  Never NULL. */
const char *ivhd_status_string(ivhd_status s);

/* Library version as (major << 16) | (minor << 8) | patch. */
int32_t ivhd_version(void);

/*
 * Exact brute-force kNN graph (the set-up step of Sec. 5.1, untimed in the
 * paper's time_emb): for every row q of X, the k nearest other rows, nearest
 * first, ties broken by the lower index.  Float data are compared by the FP32
 * chain acc = fma(x_d - y_d, x_d - y_d, acc), d = 0..N-1; uint8 data by exact
 * integer squared distances.  The result does not depend on the method.
 *
 *   X        device, M*N elements of `dtype` (ivhd_knn_dtype), row-major.
 *   out_knn  device, M*k int32.
 *   stream   cudaStream_t or NULL.
 * Constraints: 2 <= M < 2^31, 1 <= N <= 65536, 1 <= k <= min(M - 1, 64).
 * Uses the tensor-core method when it applies (ivhd_knn_build_ex).
 * Synchronises.  Errors: IVHD_ERR_ARG, IVHD_ERR_OOM, IVHD_ERR_CUDA,
 * IVHD_ERR_TIMEOUT (a bounded wait of the tensor-core kernel expired).
 */
ivhd_status ivhd_knn_build(const void *X, int32_t dtype, int64_t M, int32_t N, int32_t k,
                           int32_t *out_knn, void *stream);

typedef enum {
    IVHD_KNN_AUTO = 0,          /* tensor cores when they apply, else CUDA cores */
    IVHD_KNN_CUDA_CORES = 1,    /* FP32 chain (float) / dp4a (uint8) on every pair */
    IVHD_KNN_TENSOR_CORES = 2   /* distance GEMM (tcgen05, BF16 operands, FP32 accumulate)
                                   with the top-k fused into its epilogue */
} ivhd_knn_method;

typedef struct {
    int32_t method;         /* the method that ran */
    int64_t fallback_rows;  /* float data, tensor cores: rows whose candidate list could not
                               be certified and were recomputed on the CUDA cores */
    float max_rel_err;      /* float data, tensor cores: max |approximate - exact distance| /
                               (|x_i|^2 + |x_j|^2) over all candidates */
    float eps_coef;         /* the error bound per unit of |x_i|^2 + |x_j|^2 that the
                               certificate assumes, 2^-13 + N 2^-19 */
} ivhd_knn_stats_t;

/*
 * ivhd_knn_build with a choice of method and statistics (stats may be NULL).
 * Tensor cores apply for k <= 32 and, for uint8 data, N <= 1024.  uint8: the
 * GEMM on x - 128 in BF16 is exact (every partial sum is an integer below
 * 2^24).  float: x = hi + lo + r with BF16 hi and lo; a GEMM over
 * [hi, hi, lo] . [hi, lo, hi] gives distances dt within eps_coef (|x_i|^2 +
 * |x_j|^2) of the exact ones and keeps per row the 32 smallest keys
 * dt - eps_coef |x_j|^2; they are re-ranked by the exact FP32 chain, and a row
 * is kept when its exact k-th distance lies below the 32nd key minus
 * eps_coef |x_i|^2, so no vertex outside the list can be closer; other rows
 * are recomputed by the CUDA-core method.  IVHD_ERR_ARG for
 * IVHD_KNN_TENSOR_CORES outside its range.
 */
ivhd_status ivhd_knn_build_ex(const void *X, int32_t dtype, int64_t M, int32_t N, int32_t k,
                              int32_t *out_knn, int32_t method, ivhd_knn_stats_t *stats,
                              void *stream);

/*
 * ivhd_knn_query -- the k nearest base rows of new points.
 *
 * The nearest-neighbour search with which Progressive UMAP places a point that
 * arrives after the embedding was made (Sec. 2.4.3, Progressive UMAP scheme:
 * a new point starts at the embedding of its nearest neighbour among the data
 * seen so far), made exact.  out row q lists the k rows of the base set X
 * nearest to query row q of Q, ascending by (distance, index), with the
 * distances of ivhd_knn_build (FP32 chain for float data, exact integers for
 * uint8).  No row is excluded: a query equal to a base row finds it at
 * distance 0.
 *   Q        device, Mq*N elements of `dtype`, row-major (the new points).
 *   X        device, M*N elements of `dtype`, row-major (the base set).
 *   out      device, Mq*k int32.
 *   method, stats   as ivhd_knn_build_ex.
 * 1 <= Mq < 2^31 - 1, 1 <= M < 2^31 - 1, 1 <= k <= min(M, 64), N as
 * ivhd_knn_build; the tensor-core method needs M >= 2 and k <= 32.  Else
 * IVHD_ERR_ARG.  Synchronises.
 */
ivhd_status ivhd_knn_query(const void *Q, int64_t Mq, const void *X, int64_t M, int32_t dtype,
                           int32_t N, int32_t k, int32_t *out, int32_t method,
                           ivhd_knn_stats_t *stats, void *stream);

/*
 * ivhd_knn_index_* -- a base set held for repeated ivhd_knn_query calls
 * (arriving batches of new points against the same embedded data).
 *
 * ivhd_knn_index_create copies X (device, M*N elements of `dtype`, rows as in
 * ivhd_knn_query) and, where the tensor-core method applies (M >= 2, uint8
 * N <= 1024 or float 3N <= 65536), prepares its GEMM operand and row norms
 * once (BF16, about M * 2 * N (uint8) or M * 6 * N (float) bytes besides the
 * copy).  Work runs on `stream`; synchronises.  Arguments as ivhd_knn_query
 * (k = 1 for the checks), else IVHD_ERR_ARG; IVHD_ERR_OOM.
 *
 * ivhd_knn_index_query: ivhd_knn_query(Q, Mq, X, M, dtype, N, k, out,
 * method, stats) on the index's stream, bit for bit the same lists, without
 * preparing the base set again.  Synchronises.
 *
 * ivhd_knn_index_destroy frees the index (stream-ordered); NULL is a no-op.
 */
typedef struct ivhd_knn_index ivhd_knn_index;
ivhd_status ivhd_knn_index_create(const void *X, int32_t dtype, int64_t M, int32_t N,
                                  void *stream, ivhd_knn_index **out);
ivhd_status ivhd_knn_index_query(ivhd_knn_index *idx, const void *Q, int64_t Mq, int32_t k,
                                 int32_t *out, int32_t method, ivhd_knn_stats_t *stats);
void ivhd_knn_index_destroy(ivhd_knn_index *idx);

/*
 * ivhd_place_nn -- place new points at the mean embedding of base neighbours.
 *
 * out[q] = (1/k) sum_s Y[ids[q][s]], the sum taken in FP32 in the order
 * s = 0 .. k-1.  With the lists of ivhd_knn_query and k = 1 this is the
 * Progressive UMAP initialisation of a new point (Sec. 2.4.3); k > 1 averages
 * the embeddings of its k nearest base points.
 *   Y     device, M*2 float32 (the embedding of the base set, input order).
 *   ids   device, n*k int32, each in [0, M).
 *   out   device, n*2 float32.
 * M >= 1, n >= 0, 1 <= k <= 1024, else IVHD_ERR_ARG (ids and out may be NULL
 * when n = 0, which does nothing); an id outside [0, M)
 * returns IVHD_ERR_INDEX (rows holding one are left unwritten).  Synchronises.
 */
ivhd_status ivhd_place_nn(const float *Y, int64_t M, const int32_t *ids, int64_t n, int32_t k,
                          float *out, void *stream);

/*
 * Neighbourhood preservation Q_NX(k) of Sec. 4.1 on sampled rows: for each
 * row q in `rows`, the k nearest other points of y_q in the embedding (FP32
 * squared distance dx*dx rounded then fma(dy, dy, .), ties by lower index)
 * are intersected with the kNN row q; *out_q = hits / (k * nrows).
 *
 *   Y        device, M*2 float32.      knn   device, M*k int32.
 *   rows     device, nrows int64 row ids in [0, M).
 *   out_lowd device, nrows*k int32 or NULL: the embedded neighbours found.
 *   out_q    host double.
 * Constraints: 1 <= k <= min(M - 1, 128), nrows >= 1.  A row id outside
 * [0, M) is never dereferenced: the call returns IVHD_ERR_INDEX and leaves
 * *out_q unwritten.  Synchronises.
 */
ivhd_status ivhd_eval_qnx(const float *Y, int64_t M, const int32_t *knn, int32_t k,
                          const int64_t *rows, int64_t nrows, int32_t *out_lowd,
                          double *out_q, void *stream);

/*
 * Neighbour hit cf_nn of Sec. 4.1, Eq. 4.4 on sampled rows: the fraction of
 * the nn nearest embedded neighbours (same distance and tie rule as
 * ivhd_eval_qnx) that carry the label of the query row.
 *
 *   Y device M*2 float32; labels device M int32; rows device nrows int64.
 * Constraints: 1 <= nn <= min(M - 1, 128).  Row ids outside [0, M): as
 * ivhd_eval_qnx (IVHD_ERR_INDEX).  Synchronises.
 */
ivhd_status ivhd_eval_cf(const float *Y, int64_t M, const int32_t *labels, int32_t nn,
                         const int64_t *rows, int64_t nrows, double *out_cf, void *stream);

/*
 * Calibration of the gather roofline.  The force pass is dominated by reads of
 * neighbour positions at data-dependent addresses (Sec. 5.2 notes that the
 * IVHD-CUDA force step is limited by its scattered reads and writes).  This
 * call measures how many uniformly random 8-byte float2 gathers per second the
 * current GPU sustains from an array of n_positions elements (allocated and
 * freed here), with indices generated in registers, over `repeats` timed
 * launches of about n_gathers gathers each.  The step kernel, which also
 * streams its neighbour ids and state, cannot gather faster.
 * Constraints: 1 <= n_positions < 2^30, 16384 <= n_gathers <= 2^34,
 * repeats >= 1.  Synchronises.  Errors: IVHD_ERR_ARG, IVHD_ERR_CUDA.
 */
ivhd_status ivhd_probe_gather(int64_t n_positions, int64_t n_gathers, int32_t repeats,
                              double *gathers_per_s, void *stream);

/*
 * Launch floor of the step loop: writes to *us_per_launch the device time per
 * launch of a CUDA graph of n_launches chained programmatic dependent launches
 * (the form ivhd_step replays) of an empty kernel of `grid` blocks of `block`
 * threads; each block waits for its predecessor grid and releases its
 * successor, as the step kernel does, and does nothing else.  A step kernel
 * of the same grid cannot take less per step.  Allocates nothing on the
 * device; the graph is captured on a private stream and timed on `stream`.
 * Constraints: 1 <= grid <= 2^20, block a multiple of 32 in [32, 1024],
 * 1 <= n_launches <= 100000.  Synchronises.  Errors: IVHD_ERR_ARG,
 * IVHD_ERR_CUDA.
 */
ivhd_status ivhd_probe_launch(int32_t grid, int32_t block, int32_t n_launches,
                              double *us_per_launch, void *stream);

/*
 * C = A B^T on the tensor cores (tcgen05, TMA-fed, FP32 accumulation): A is
 * M x K and B is N x K, both BF16 row-major (device), C is M x N FP32
 * row-major (device).  The building block of the dense layers of the learned
 * warm start (an MLP mapping features to 2-D positions).  Constraints:
 * K % 8 == 0, all pointers 16-byte aligned, dimensions < 2^30.  Synchronises.
 * Errors: IVHD_ERR_ARG, IVHD_ERR_CUDA, IVHD_ERR_TIMEOUT (a bounded
 * device-side wait expired; the kernel returned without a result).
 */
ivhd_status ivhd_gemm_bf16_tn(const void *A, const void *B, float *C, int64_t M, int64_t N,
                              int64_t K, void *stream);

/*
 * Learned warm start / out-of-sample placement.  The paper uses IVHD itself as
 * an initial configuration for slower methods (Sec. 3.4) and reviews
 * parametric maps from features to the embedding (parametric t-SNE and UMAP,
 * Sec. 2); here a multilayer perceptron
 *     x -> GELU(W1 x + b1) -> GELU(W2 h1 + b2) -> W3 h2 + b3      (n_in -> H -> H -> 2)
 * is trained with the mean squared error to IVHD coordinates and Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected), then places new points
 * or whole datasets before IVHD refines them.  FP32 master weights and Adam
 * moments; the two wide layers run on the tensor cores (ivhd_gemm_bf16_tn)
 * from BF16 copies with FP32 accumulation, bias + GELU fused in the epilogue.
 *
 * Parameters are one flat FP32 vector in the order W1 (H x n_in, row-major),
 * b1 (H), W2 (H x H), b2 (H), W3 (2 x H), b3 (2); ivhd_mlp_num_params gives
 * its length.  Inputs x are row-major (rows x n_in) device arrays of dtype
 * 0 = BF16, 1 = uint8, 2 = FP32, multiplied by x_scale on load; targets are
 * device FP32 rows x 2.  All calls are stream-ordered on `stream`.
 * Constraints: n_in % 8 == 0, H % 16 == 0, batch sizes B % 8 == 0 with
 * 8 <= B <= max_batch.  Errors: IVHD_ERR_ARG, IVHD_ERR_OOM, IVHD_ERR_CUDA,
 * IVHD_ERR_TIMEOUT (a bounded wait in a GEMM expired), IVHD_ERR_STATE.
 */
typedef struct ivhd_mlp ivhd_mlp;

ivhd_status ivhd_mlp_create(int32_t n_in, int32_t hidden, int32_t max_batch, void *stream,
                            ivhd_mlp **out);
void ivhd_mlp_destroy(ivhd_mlp *mlp);
int64_t ivhd_mlp_num_params(ivhd_mlp *mlp);
/* Loads all parameters (host or device) and resets the Adam state.  Synchronises. */
ivhd_status ivhd_mlp_set_params(ivhd_mlp *mlp, const float *params, int32_t on_device);
/* Copies the FP32 master parameters out.  Host output synchronises. */
ivhd_status ivhd_mlp_get_params(ivhd_mlp *mlp, float *params, int32_t on_device);
/*
 * Loss (*loss, host, may be NULL) and gradients (grads: device, n_params
 * FP32, may be NULL) of one batch, without updating.  Synchronises.
 */
ivhd_status ivhd_mlp_loss_grad(ivhd_mlp *mlp, const void *x, int32_t x_dtype, float x_scale,
                               const float *targets, int32_t B, double *loss, float *grads);
/*
 * One Adam step on one batch with learning rate lr.  With loss != NULL the
 * batch loss (before the update) is written and the call synchronises;
 * otherwise it is fully asynchronous.
 */
ivhd_status ivhd_mlp_train_step(ivhd_mlp *mlp, const void *x, int32_t x_dtype, float x_scale,
                                const float *targets, int32_t B, float lr, double *loss);
/* y (device, n x 2 FP32) = the network applied to n rows of x.  Synchronises. */
ivhd_status ivhd_mlp_forward(ivhd_mlp *mlp, const void *x, int32_t x_dtype, float x_scale,
                             int64_t n, float *y);
/* Kernels launched by this network so far. */
int64_t ivhd_mlp_launches(ivhd_mlp *mlp);

/*
 * Intermediate values of the last batch the network processed (the last
 * max_batch-row chunk of ivhd_mlp_forward, or the batch of the last
 * ivhd_mlp_loss_grad / ivhd_mlp_train_step), for inspecting the network layer
 * by layer.  The paper has no counterpart.  `which` selects one row-major
 * array of *rows rows:
 *   IVHD_MLP_X    input rows as BF16 (rows x n_in, 2-byte BF16 bit patterns)
 *   IVHD_MLP_Z1   W1 x + b1, FP32 (rows x hidden; training calls)
 *   IVHD_MLP_H1   GELU(z1) as BF16     IVHD_MLP_Z2  W2 h1 + b2, FP32 (training calls)
 *   IVHD_MLP_H2   GELU(z2) as BF16     IVHD_MLP_Y   W3 h2 + b3, FP32 (rows x 2)
 *   IVHD_MLP_DY   dL/dy = 2 (y - t) / rows, FP32 (rows x 2; training calls)
 *   IVHD_MLP_DZ2  (dY W3) * GELU'(z2) as BF16 (training calls)
 *   IVHD_MLP_DZ1  (dZ2 W2) * GELU'(z1) as BF16 (training calls)
 * out: host or device memory large enough for max_batch rows.  *rows = 0
 * before the first batch.  Synchronises.  Errors: IVHD_ERR_ARG, IVHD_ERR_STATE.
 */
enum {
    IVHD_MLP_X = 0, IVHD_MLP_Z1 = 1, IVHD_MLP_H1 = 2, IVHD_MLP_Z2 = 3, IVHD_MLP_H2 = 4,
    IVHD_MLP_Y = 5, IVHD_MLP_DY = 6, IVHD_MLP_DZ2 = 7, IVHD_MLP_DZ1 = 8
};
ivhd_status ivhd_mlp_activations(ivhd_mlp *mlp, int32_t which, void *out, int64_t *rows);

/*
 * ivhd_eval_qnx_static -- ivhd_eval_qnx that allocates no device memory.
 *
 * The paper has no counterpart: this entry point exists for host
 * applications that cannot let a library allocate device memory (a process
 * whose memory is reserved up front by another framework's caching
 * allocator, a latency-critical loop where cudaMalloc/cudaFree would
 * synchronise the device, or an application that must keep its
 * device-memory footprint fixed after start-up).  Same arguments, result and
 * rules as ivhd_eval_qnx; the caller still passes every input and output.
 *
 * Scratch: a fixed array of 8194 64-bit counters (about 64 KiB) in the
 * library's own device memory, held by every GPU that loads the library
 * until the process exits.  It limits one call to nrows <= 1,048,576
 * (8192 blocks of 128 rows); larger calls return IVHD_ERR_ARG.  A row id
 * outside [0, M) returns IVHD_ERR_INDEX (never dereferenced).  The first
 * call on each device (and again after the caller re-creates the device's
 * CUDA context, e.g. with cudaDeviceReset) looks up the array's device
 * address, which may load the library's device code, so make that first call
 * before any stream capture.  All calls on a device share the array and it
 * keeps the last call's contents: calls whose GPU work overlaps (different
 * streams or unsynchronised host threads) race and may return wrong values;
 * order them on one stream.  Calls no cudaMalloc, cudaFree or other
 * allocating routine.  Synchronises.
 */
ivhd_status ivhd_eval_qnx_static(const float *Y, int64_t M, const int32_t *knn, int32_t k,
                                 const int64_t *rows, int64_t nrows, int32_t *out_lowd,
                                 double *out_q, void *stream);

/*
 * ivhd_set_allocator -- take the library's device memory from the caller.
 *
 * The paper has no counterpart.  By default every device buffer of the
 * library (context state, layouts, kNN and network scratch) comes from the
 * stream-ordered pool (cudaMallocAsync / cudaFreeAsync on the call's stream).
 * After this call, every later allocation calls alloc_fn instead, e.g. a
 * framework's caching allocator, so that one pool serves both:
 *
 *   alloc_fn(bytes, stream, user): returns device memory of at least `bytes`
 *     bytes on the current device, usable by work that the library then
 *     enqueues on `stream` (a cudaStream_t; NULL = legacy default stream),
 *     aligned to 256 bytes (as cudaMalloc is), or NULL when it cannot, which
 *     the calling entry point reports as IVHD_ERR_OOM.  A pointer that is not
 *     256-byte aligned is handed straight back to free_fn and treated as
 *     NULL.
 *   free_fn(ptr, bytes, stream, user): the library no longer needs ptr once
 *     the work queued on `stream` so far has run; the allocator may hand the
 *     block to later work on that stream at once (the contract of a
 *     stream-ordered caching allocator) but to other streams only after that
 *     work has finished.  `bytes` is the size that was asked for.
 *
 * Process-wide.  Both NULL restores the built-in pool; exactly one NULL is
 * IVHD_ERR_ARG.  Each block is released through the allocator that made it,
 * whatever the setting at release time.  The callbacks run on the calling
 * host thread, never while a stream is being captured, and must not call
 * back into the library.  Returns IVHD_OK.
 */
typedef void *(*ivhd_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*ivhd_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
ivhd_status ivhd_set_allocator(ivhd_alloc_fn alloc_fn, ivhd_free_fn free_fn, void *user);

/*
 * Test support (the paper has no counterpart).
 *
 * ivhd_probe_wait_timeout runs, in one thread of one block, the bounded
 * mbarrier wait that the tensor-core kernels use, on a barrier that nothing
 * completes, for `polls` polls; returns IVHD_ERR_TIMEOUT (the expected result)
 * without faulting or hanging, after which the library and the stream remain
 * usable.  polls >= 1, else IVHD_ERR_ARG.  Synchronises.
 *
 * ivhd_test_fail_alloc(after): the next `after` device allocations made by the
 * library succeed and the one after them fails with IVHD_ERR_OOM at the
 * calling entry point (once; after < 0 switches the injection off).
 * ivhd_test_live_allocs: device allocations made by the library and not yet
 * released, to check that every error path frees what it took.  Process-wide.
 */
ivhd_status ivhd_probe_wait_timeout(int32_t polls, void *stream);

/*
 * ivhd_probe_grid_barrier_timeout runs the persistent grid's barrier in a
 * cooperative launch of two blocks of which only one arrives, with a limit of
 * `polls` polls; returns IVHD_ERR_TIMEOUT (the expected result) without
 * faulting or hanging, after which the library and the stream remain usable.
 * polls >= 1, else IVHD_ERR_ARG.  Synchronises.
 */
ivhd_status ivhd_probe_grid_barrier_timeout(int32_t polls, void *stream);

/*
 * Checked builds (the library compiled with IVHD_CHECKED: build_lib with
 * IVHD_CHECKED=1, loaded by the binding when that variable is set), the
 * stand-in for a memory checker.  Every index the step kernels gather and
 * every row extent they read from the layout is tested first; a bad one is
 * counted and skipped, never dereferenced.
 *
 * ivhd_check_violations: *out = the number of such indices and rows met since
 * the last reset (reset != 0 clears it), or -1 in a normal build.
 * Process-wide; synchronises the device.
 *
 * ivhd_test_corrupt_layout: writes `value` into entry `slot` of the
 * context's layout (0 <= slot < the layout's entries, ivhd_info), so that a
 * test can check that the kernels report it.  Checked builds only: a normal
 * build returns IVHD_ERR_ARG and changes nothing.  Synchronises.
 */
ivhd_status ivhd_check_violations(int64_t *out, int32_t reset);
ivhd_status ivhd_test_corrupt_layout(ivhd_ctx *ctx, int64_t slot, uint32_t value);
void ivhd_test_fail_alloc(int64_t after);
int64_t ivhd_test_live_allocs(void);

#ifdef __cplusplus
}
#endif

#endif /* IVHD_H_ */
