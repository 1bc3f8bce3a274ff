// ivhd_knn_tc.cu -- kNN graph build (the set-up step of Sec. 5.1) on the
// 5th-generation tensor cores: a distance GEMM with the top-k selection fused
// into its epilogue.
//
// Squared distances come from the Gram matrix, |x_i - x_j|^2 = n_i + n_j - 2 <x_i, x_j>.
//
// uint8 data: the GEMM runs on x - 128 in BF16.  Every value in [-128, 127]
//   is exact in BF16, every product (at most 2^14) is exact in FP32, and with
//   N <= 1024 every partial sum stays below 2^24, so the tensor cores return
//   <x_i, x_j> exactly whatever their summation order; with the norms of the
//   shifted rows (exact int32) the distances are the exact integers and the
//   fused top-k (ties to the lower index) is final.
// FP32 data: x = hi + lo + r with hi = bf16(x), lo = bf16(x - hi) and
//   |r| <= 2^-16 |x|; the GEMM over K = 3N of [hi, hi, lo] . [hi, lo, hi] gives
//   <x_i, x_j> to about 2^-14 of sum_d |x_id x_jd|, so the approximate
//   distance dt_ij is within eps (n_i + n_j) of the exact FP32-chain distance,
//   eps = 2^-13 + N 2^-19 (the split, the FP32 accumulation of 3N products and
//   the chain's own rounding, with a margin of several times).  The epilogue
//   keeps, per row, the kList smallest keys kappa_j = dt_ij - eps n_j, each a
//   lower bound of d_ij + eps n_i.  A re-rank pass recomputes the listed
//   distances with the FP32 chain of the exact kernel, keeps the k best (ties to
//   the lower index) and certifies the row: every vertex outside the list has
//   kappa_j >= tau (the list's largest key), hence d_ij >= tau - eps n_i, so
//   the row is final when its exact k-th distance is below tau - eps n_i.
//   Other rows are recomputed by the exact CUDA-core kernel.
//
// Query rows are the rows of X itself for the kNN graph (a row never lists
// itself), or a separate set of new points searched against X as the base set
// (the nearest-neighbour placement of Progressive UMAP, Sec. 2.4.3); the
// arithmetic and the certificate are the same, with n_i the query's norm.
//
// One CTA owns 128 query rows (the 128 tensor-memory lanes) and sweeps all
// candidates in tiles of 256 columns:
//   warp 0, one lane   TMA producer: 128 x 64 query and 256 x 64 candidate
//                      slices into a 4-stage ring (128-byte swizzle)
//   warp 1, one lane   MMA issuer: tcgen05.mma M=128 N=256 K=16 into one of two
//                      256-column accumulators in tensor memory (512 columns),
//                      so the epilogue of tile t overlaps the MMAs of tile t+1
//   warps 2-5          epilogue: thread = query row; tcgen05.ld of 32 columns at
//                      a time, distance, compare with the row's list held in
//                      registers
// Every wait is bounded; a timeout sets an error flag and all roles stop.
#include <climits>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "ivhd_internal.cuh"
#include "ivhd_knn_tc.cuh"
#include "ivhd_tc.cuh"

namespace ivhd {
namespace {

using namespace tc;

constexpr int kTM = 128;  // query rows per CTA
constexpr int kTN = 256;  // candidate columns per accumulator tile
constexpr int kTStages = 4;
constexpr int kEpiWarps = 8;  // two warpgroups: each reads one 128-column half of a tile
constexpr int kTcThreads = 32 * (2 + kEpiWarps);
constexpr int kMaxKnnSegments = 32;  // column segments of one kNN launch (short query sets)

struct KnnSmem {
  static constexpr int a_bytes = kTM * kBK * 2;
  static constexpr int b_bytes = kTN * kBK * 2;
  static constexpr int stage_bytes = a_bytes + b_bytes;
  static constexpr int bar_offset = kTStages * stage_bytes;
  static constexpr int nrm_offset = bar_offset + 256;  // 8 warps x 128 column terms
  static constexpr int total = nrm_offset + kEpiWarps * (kTN / 2) * 4 + 1024;  // + slack
};

template <class D>
__device__ __forceinline__ bool better(D d, int j, D bd, int bj) {
  return d < bd || (d == bd && j < bj);
}

// Inserts (d, j) into the ascending list (dl, jl) of L entries, dropping the last.
template <class D, int L>
__device__ __forceinline__ void list_insert(D d, int j, D (&dl)[L], int (&jl)[L]) {
#pragma unroll
  for (int q = 0; q < L; ++q) {
    const bool b = better(d, j, dl[q], jl[q]);
    const D td = dl[q];
    const int tj = jl[q];
    dl[q] = b ? d : td;
    jl[q] = b ? j : tj;
    d = b ? td : d;
    j = b ? tj : j;
  }
}

// Bounded wait that also stops when another role has given up.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity,
                                              volatile int* abort_flag) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// U8: exact integer keys; L: list length (kKnnList for float, 8 or kKnnList for uint8).
template <bool U8, int L>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_knn_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
             const float* __restrict__ nrm_f, const int32_t* __restrict__ nrm_i,
             const float* __restrict__ qnrm_f, const int32_t* __restrict__ qnrm_i, int Mq, int M,
             int Kp, bool self, int seg_tiles, float eps_coef, int32_t* __restrict__ out_ids,
             float* __restrict__ out_d, int32_t* __restrict__ err) {
  using D = typename std::conditional<U8, int32_t, float>::type;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + KnnSmem::bar_offset);
  uint64_t* empty = full + kTStages;
  uint64_t* acc_full = empty + kTStages;  // [2]
  uint64_t* acc_empty = acc_full + 2;     // [2]
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* issued = abort_flag + 1;
  constexpr uint32_t kCols = 2 * kTN;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTM;
  const int nk = Kp / kBK;
  // this CTA's column segment: tiles t0 .. t0 + n_tiles - 1 (blockIdx.y of gridDim.y)
  const int all_tiles = (M + kTN - 1) / kTN;
  const int t0 = (int)blockIdx.y * seg_tiles;
  const int n_tiles = max(0, min(all_tiles - t0, seg_tiles));

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 32 * kEpiWarps);  // every epilogue thread arrives
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    *issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: the query slice (re-read from L2 for every tile) and the candidate slice
      uint32_t g = 0;
      for (int t = 0; t < n_tiles; ++t) {
        bool ok = true;
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int s = (int)(g % kTStages);
          if (g >= kTStages && !wait_or_abort(&empty[s], ((g / kTStages) - 1) & 1, abort_flag)) {
            atomicOr(err, 1);
            ok = false;
            break;
          }
          unsigned char* sa = smem + s * KnnSmem::stage_bytes;
          unsigned char* sb = sa + KnnSmem::a_bytes;
          mbar_expect_tx(&full[s], KnnSmem::stage_bytes);
          tma_load_2d(sa, &map_a, kt * kBK, m0, &full[s]);
          tma_load_2d(sb, &map_b, kt * kBK, (t0 + t) * kTN, &full[s]);
          *issued = (int)(g + 1);
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = instr_desc_bf16(kTM, kTN);
      uint32_t g = 0;
      bool ok = true;
      for (int t = 0; t < n_tiles && ok; ++t) {
        const int b = t & 1;
        if (t >= 2 && !wait_or_abort(&acc_empty[b], ((t >> 1) - 1) & 1, abort_flag)) {
          atomicOr(err, 2);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t dst = tmem + (uint32_t)(b * kTN);
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int s = (int)(g % kTStages);
          if (!wait_or_abort(&full[s], (g / kTStages) & 1, abort_flag)) {
            atomicOr(err, 4);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t sa = smem_u32(smem + s * KnnSmem::stage_bytes);
          const uint32_t sb = sa + KnnSmem::a_bytes;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)
            umma_bf16(dst, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), idesc,
                      (kt > 0 || kk > 0) ? 1u : 0u);
          umma_commit(&empty[s]);
        }
        if (ok) umma_commit(&acc_full[b]);
      }
      // every MMA issued above has finished before tensor memory is released
      umma_commit(done);
      if (!mbar_wait(done, 0)) atomicOr(err, 8);
    }
  } else {
    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31
    // (its row quarter) of one 128-column half of each tile: warps 2-5 the
    // first half, warps 6-9 the second, so every row has one list per half.
    // Keys: uint8, the exact distance; float, the lower-bound key
    // kappa_j = dt_j - eps n_j = n_i + (1 - eps) n_j - 2 <x_i, x_j>~ (see the top).
    // Columns arrive in increasing j, so a key equal to the list's last never
    // enters (the earlier index wins the tie) and the test is a plain "<".
    constexpr int kHalf = kTN / 2;
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int r = quarter * 32 + lane;
    const int i = m0 + r;
    // the half-tile's 128 column terms, staged per warp; each lane prefetches
    // its 4 terms of the next tile into registers while the current one is processed
    D* nbuf = reinterpret_cast<D*>(smem + KnnSmem::nrm_offset) + (warp - 2) * kHalf;
    constexpr int kPer = kHalf / 32;
    const D kMaxKey = U8 ? (D)INT_MAX : (D)__int_as_float(0x7f800000);
    const float col_scale = 1.f - eps_coef;
    D pn[kPer];
    auto fetch = [&](int t) {
#pragma unroll
      for (int e = 0; e < kPer; ++e) {
        const int jc = (t0 + t) * kTN + half * kHalf + e * 32 + lane;
        if constexpr (U8)
          pn[e] = (jc < M) ? nrm_i[jc] : 0;
        else
          pn[e] = (jc < M) ? col_scale * nrm_f[jc] : 0.f;
      }
    };
    D dl[L];
    int jl[L];
#pragma unroll
    for (int q = 0; q < L; ++q) {
      dl[q] = kMaxKey;
      jl[q] = INT_MAX;
    }
    const D ni = (i < Mq) ? (U8 ? (D)qnrm_i[i] : (D)qnrm_f[i]) : (D)0;
    const int iself = self ? i : -1;  // the column a row never lists (self-kNN only)
    bool ok = true;
    fetch(0);
    for (int t = 0; t < n_tiles; ++t) {
      const int b = t & 1;
      if (!wait_or_abort(&acc_full[b], (t >> 1) & 1, abort_flag)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      __syncwarp();
#pragma unroll
      for (int e = 0; e < kPer; ++e) nbuf[e * 32 + lane] = pn[e];
      __syncwarp();
      if (t + 1 < n_tiles) fetch(t + 1);
      const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kTN + half * kHalf);
      const int n0 = (t0 + t) * kTN + half * kHalf;
      for (int c0 = 0; c0 < kHalf && n0 + c0 < M; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tbase + c0, v);
        const int jb = n0 + c0;
        D d[32];
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
          D nj[4];
          if constexpr (U8) {
            const int4 w = *reinterpret_cast<const int4*>(nbuf + c0 + q);
            nj[0] = w.x, nj[1] = w.y, nj[2] = w.z, nj[3] = w.w;
          } else {
            const float4 w = *reinterpret_cast<const float4*>(nbuf + c0 + q);
            nj[0] = w.x, nj[1] = w.y, nj[2] = w.z, nj[3] = w.w;
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if constexpr (U8)
              d[q + e] = ni + nj[e] - 2 * __float2int_rn(__uint_as_float(v[q + e]));
            else
              d[q + e] = fmaf(-2.f, __uint_as_float(v[q + e]), ni + nj[e]);
          }
        }
        if (jb + 31 >= M || (jb <= iself && iself <= jb + 31)) {
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (jb + q >= M || jb + q == iself) d[q] = kMaxKey;
        }
        D mn = d[0];
#pragma unroll
        for (int q = 1; q < 32; ++q) mn = min(mn, d[q]);
        if (mn < dl[L - 1]) {
          // rare after the first tiles: visit the columns below the threshold in order
          const D thr = dl[L - 1];
          uint32_t mask = 0;
          D tmp[32];
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            mask |= (uint32_t)(d[q] < thr) << q;
            tmp[q] = d[q];
          }
          while (mask) {
            const int q = __ffs((int)mask) - 1;
            mask &= mask - 1;
            if (tmp[q] < dl[L - 1]) list_insert<D, L>(tmp[q], jb + q, dl, jl);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      mbar_arrive(&acc_empty[b]);
    }
    if (ok && i < Mq) {
      // the row's list for this segment and half:
      // out_ids / out_key [((i * segments + segment) * 2 + half) * L + q]
      const int64_t o = (((int64_t)i * gridDim.y + blockIdx.y) * 2 + half) * L;
#pragma unroll
      for (int q = 0; q < L; ++q) {
        out_ids[o + q] = jl[q];
        if constexpr (U8)
          reinterpret_cast<int32_t*>(out_d)[o + q] = dl[q];
        else
          out_d[o + q] = dl[q];
      }
    }
    if (!ok && lane == 0) atomicOr(err, 16);
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) {
    // drain copies still in flight before the shared memory goes away
    const int iss = *issued;
    for (int g = (iss > kTStages ? iss - kTStages : 0); g < iss; ++g)
      mbar_wait(&full[g % kTStages], (g / kTStages) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// ---- operand preparation ---------------------------------------------------

// FP32: A = [hi | hi | lo], B = [hi | lo | hi] along K (3N, zero-padded to Kp);
// either output may be null (queries fill A, the base set B).
__global__ void k_prep_f32(const float* __restrict__ X, int64_t M, int N, int Kp,
                           __nv_bfloat16* __restrict__ A, __nv_bfloat16* __restrict__ B) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * Kp) return;
  const int64_t i = e / Kp;
  const int c = (int)(e - i * Kp);
  const int seg = c / N, d = c - seg * N;
  __nv_bfloat16 a = __float2bfloat16_rn(0.f), b = a;
  if (seg < 3) {
    const float x = X[i * N + d];
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    a = (seg == 2) ? lo : hi;
    b = (seg == 1) ? lo : hi;
  }
  if (A) A[e] = a;
  if (B) B[e] = b;
}

// FP32 norms (FP64 sum, rounded once).
__global__ void k_norms_f32(const float* __restrict__ X, int64_t M, int N, float* __restrict__ nrm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double s = 0.0;
  for (int d = 0; d < N; ++d) {
    const double x = X[i * N + d];
    s += x * x;
  }
  nrm[i] = (float)s;
}

// uint8: A = B = x - 128 (zero-padded to Kp); norms of the shifted rows.
__global__ void k_prep_u8(const uint8_t* __restrict__ X, int64_t M, int N, int Kp,
                          __nv_bfloat16* __restrict__ A) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * Kp) return;
  const int64_t i = e / Kp;
  const int c = (int)(e - i * Kp);
  A[e] = __float2bfloat16_rn(c < N ? (float)X[i * N + c] - 128.f : 0.f);
}

__global__ void k_norms_u8s(const uint8_t* __restrict__ X, int64_t M, int N,
                            int32_t* __restrict__ nrm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int32_t s = 0;
  for (int d = 0; d < N; ++d) {
    const int32_t v = (int32_t)X[i * N + d] - 128;
    s += v * v;
  }
  nrm[i] = s;
}

// ---- FP32 re-rank and certificate (warp per row, lane = candidate) --------

__device__ __forceinline__ void cas(float& d, int& j, int lane, int mask, bool up) {
  const float od = __shfl_xor_sync(0xffffffffu, d, mask);
  const int oj = __shfl_xor_sync(0xffffffffu, j, mask);
  const bool lower = (lane & mask) == 0;
  // the lower lane keeps the smaller pair when sorting up
  const bool mine_better = better(d, j, od, oj);
  const bool keep = (lower == up) ? mine_better : !mine_better;
  if (!keep) {
    d = od;
    j = oj;
  }
}

// Exact FP32-chain distance of rows i and j (the order of the exact kernel).
__device__ __forceinline__ float chain_dist(const float* __restrict__ xi,
                                            const float* __restrict__ xj, int N) {
  float acc = 0.f;
  for (int q = 0; q < N; ++q) {
    const float diff = __fsub_rn(xi[q], xj[q]);
    acc = __fmaf_rn(diff, diff, acc);
  }
  return acc;
}

// Bitonic sort of one (d, j) pair per lane across the warp, ascending.
__device__ __forceinline__ void warp_sort(float& d, int& j, int lane) {
#pragma unroll
  for (int kk = 2; kk <= 32; kk <<= 1)
#pragma unroll
    for (int m = kk >> 1; m > 0; m >>= 1) cas(d, j, lane, m, (lane & kk) == 0);
}

// Warp per row: the row's n_lists candidate lists (two half-tile lists per
// column segment, L candidates each) are re-ranked by the exact FP32 chain and
// merged into the 32 best, 32 candidates (one or two lists) per pass, and the
// row is certified.  A list that is full bounds every vertex it left out by
// its largest key tau_h (d_ij >= tau_h - eps n_i); a list that is not full
// left nothing out.
template <int L>
__global__ void k_rerank(const float* __restrict__ Q, int Mq, const float* __restrict__ X, int M,
                         int N, int k, int n_lists, const int32_t* __restrict__ cand,
                         const float* __restrict__ key, const float* __restrict__ qnrm,
                         const float* __restrict__ nrm, float eps_coef, int32_t* __restrict__ out,
                         int32_t* __restrict__ fb_rows, int32_t* __restrict__ n_fb,
                         int32_t* __restrict__ max_err_bits) {
  static_assert(L == 16 || L == 32, "lists of 16 or 32 entries");
  constexpr int kPer = 32 / L;  // lists per pass (lane = entry)
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= Mq) return;
  const float* xi = Q + i * N;
  float tau = __int_as_float(0x7f800000);
  float rel = 0.f;
  float d = __int_as_float(0x7f800000);  // the running 32 best, sorted across the lanes
  int j = INT_MAX;
  for (int pass = 0; pass < n_lists / kPer; ++pass) {
    // L = 32: pass p reads list p; L = 16: lanes 0-15 list 2p, lanes 16-31 list 2p + 1
    const int h = pass * kPer + ((L == 32) ? 0 : (lane >> 4));
    const int64_t o = (i * n_lists + h) * L + (lane & (L - 1));
    const int j0 = cand[o];
    const float kj = key[o];
    float dc = __int_as_float(0x7f800000);
    int jc = INT_MAX;
    if (j0 >= 0 && j0 < M) {
      dc = chain_dist(xi, X + (int64_t)j0 * N, N);
      jc = j0;
      // the approximate distance is the key plus eps n_j
      rel = fmaxf(rel, fabsf(fmaf(eps_coef, nrm[j0], kj) - dc) / fmaxf(qnrm[i] + nrm[j0], 1e-30f));
    }
#pragma unroll
    for (int hh = 0; hh < kPer; ++hh) {
      // the last entry of each list of this pass
      const int last = hh * L + L - 1;
      const int jlast = __shfl_sync(0xffffffffu, j0, last);
      const float klast = __shfl_sync(0xffffffffu, kj, last);
      if (jlast >= 0 && jlast < M) tau = fminf(tau, klast);
    }
    warp_sort(dc, jc, lane);
    if (pass == 0) {
      d = dc;
      j = jc;
    } else {
      // the 32 smallest of two sorted sequences: the running one against the
      // new one reversed is bitonic, and a bitonic merge sorts it
      const float rd = __shfl_sync(0xffffffffu, dc, 31 - lane);
      const int rj = __shfl_sync(0xffffffffu, jc, 31 - lane);
      if (better(rd, rj, d, j)) {
        d = rd;
        j = rj;
      }
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) cas(d, j, lane, m, true);
    }
  }
  float mrel = rel;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mrel = fmaxf(mrel, __shfl_xor_sync(0xffffffffu, mrel, o));
  const float dk = __shfl_sync(0xffffffffu, d, k - 1);
  const bool certified = dk < tau - eps_coef * qnrm[i];
  if (certified) {
    if (lane < k) out[i * k + lane] = j;
  } else if (lane == 0) {
    fb_rows[atomicAdd(n_fb, 1)] = (int32_t)i;
  }
  if (lane == 0) atomicMax(max_err_bits, __float_as_int(mrel));
}

// uint8: the n_lists exact lists of each row (ascending by (distance, index))
// merged into the k nearest.
template <int L>
__global__ void k_merge_u8(const int32_t* __restrict__ ids, const int32_t* __restrict__ keys,
                           int64_t M, int k, int n_lists, int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int32_t* ja = ids + i * n_lists * L;
  const int32_t* da = keys + i * n_lists * L;
  int head[2 * kMaxKnnSegments];
  for (int h = 0; h < n_lists; ++h) head[h] = 0;
  for (int q = 0; q < k; ++q) {
    int bh = -1;
    for (int h = 0; h < n_lists; ++h) {
      if (head[h] >= L) continue;
      const int64_t a = (int64_t)h * L + head[h];
      const int64_t b = (int64_t)bh * L + (bh < 0 ? 0 : head[bh]);
      if (bh < 0 || better(da[a], ja[a], da[b], ja[b])) bh = h;
    }
    out[i * k + q] = ja[(int64_t)bh * L + head[bh]];
    ++head[bh];
  }
}

template <bool U8, int L>
cudaError_t launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, const float* nrm_f,
                      const int32_t* nrm_i, const float* qnrm_f, const int32_t* qnrm_i, int Mq,
                      int M, int Kp, bool self, int segments, int seg_tiles, float eps_coef,
                      int32_t* out_ids, float* out_d, int32_t* err, cudaStream_t s) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_knn_tc<U8, L>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         KnnSmem::total);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  const dim3 grid((unsigned)((Mq + kTM - 1) / kTM), (unsigned)segments);
  k_knn_tc<U8, L><<<grid, kTcThreads, KnnSmem::total, s>>>(
      ma, mb, nrm_f, nrm_i, qnrm_f, qnrm_i, Mq, M, Kp, self, seg_tiles, eps_coef, out_ids, out_d,
      err);
  return cudaGetLastError();
}

}  // namespace

bool knn_tc_supported(const KnnProblem& P) {
  if (P.k < 1 || P.k > kKnnList || P.M < 2 || P.M > (1 << 30) || P.Mq < 1 || P.Mq > (1 << 30))
    return false;
  if (P.dtype == IVHD_KNN_U8) return P.N <= 1024;
  return (int64_t)3 * P.N <= 65536;
}

// Device scratch freed on scope exit (stream-ordered).
namespace {
struct Bufs {
  cudaStream_t s;
  void* p[12] = {};
  int n = 0;
  bool ok = true;
  explicit Bufs(cudaStream_t st) : s(st) {}
  template <class T>
  T* get(int64_t count) {
    void* q = nullptr;
    if (n == (int)(sizeof(p) / sizeof(p[0])) ||
        dev_alloc(&q, (size_t)(count > 0 ? count : 1) * sizeof(T), s) != cudaSuccess) {
      ok = false;
      return nullptr;
    }
    p[n++] = q;
    return (T*)q;
  }
  ~Bufs() {
    for (int q = 0; q < n; ++q) dev_free(p[q], s);
  }
};
}  // namespace

int knn_tc_kp(int32_t dtype, int32_t N) {
  const int64_t K = dtype == IVHD_KNN_U8 ? (int64_t)N : 3 * (int64_t)N;
  return (int)(((K + kBK - 1) / kBK) * kBK);
}

cudaError_t knn_tc_prepare_base(const void* X, int32_t dtype, int64_t M, int32_t N,
                                __nv_bfloat16* B, void* nrm, cudaStream_t s) {
  const int Kp = knn_tc_kp(dtype, N);
  auto blocks = [](int64_t n) { return (unsigned)((n + 255) / 256); };
  if (dtype == IVHD_KNN_U8) {
    k_prep_u8<<<blocks(M * Kp), 256, 0, s>>>((const uint8_t*)X, M, N, Kp, B);
    k_norms_u8s<<<blocks(M), 256, 0, s>>>((const uint8_t*)X, M, N, (int32_t*)nrm);
  } else {
    k_prep_f32<<<blocks(M * Kp), 256, 0, s>>>((const float*)X, M, N, Kp, nullptr, B);
    k_norms_f32<<<blocks(M), 256, 0, s>>>((const float*)X, M, N, (float*)nrm);
  }
  return cudaGetLastError();
}

ivhd_status knn_tc_build(const KnnProblem& P, int32_t* out_knn, cudaStream_t s,
                         KnnTcStats* stats, const KnnBase* base) {
  const bool u8 = P.dtype == IVHD_KNN_U8;
  const int64_t M = P.M, Mq = P.Mq;
  const int N = P.N, k = P.k;
  const int Kp = knn_tc_kp(P.dtype, N);
  if (base && P.self) return IVHD_ERR_ARG;
  Bufs b(s);
  // A: the query rows' operand, B: the base rows' (prepared once in an index,
  // or here); one array when they coincide (uint8 self)
  __nv_bfloat16* B = base ? const_cast<__nv_bfloat16*>(base->B) : b.get<__nv_bfloat16>(M * Kp);
  __nv_bfloat16* A = (u8 && P.self) ? B : b.get<__nv_bfloat16>(Mq * Kp);
  int32_t* err = b.get<int32_t>(8);  // err, n_fb, max-err bits
  if (!b.ok) return IVHD_ERR_OOM;
  cudaError_t e = cudaMemsetAsync(err, 0, 8 * sizeof(int32_t), s);
  int32_t* n_fb = err + 1;
  int32_t* maxerr_bits = err + 2;
  auto blocks = [](int64_t n) { return (unsigned)((n + 255) / 256); };
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, Mq, Kp, Kp, kTM) || !make_map(&mb, B, M, Kp, Kp, kTN))
    return IVHD_ERR_CUDA;
  const float eps_coef = (float)(1.0 / 8192.0 + (double)N / 524288.0);
  // Short query sets: the columns are split into segments (one CTA per row
  // block and segment, one CTA per SM at a time), choosing the count that
  // minimises waves x (tiles per segment + a fixed cost of about two tiles per
  // CTA); a segment keeps at least 4 tiles of 256 columns.  Each segment
  // yields its own lists, merged per row afterwards.
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IVHD_ERR_CUDA;
  const int64_t row_blocks = (Mq + kTM - 1) / kTM;
  const int all_tiles = (int)((M + kTN - 1) / kTN);
  int want = 1;
  int64_t best_cost = INT64_MAX;
  for (int S = 1; S <= kMaxKnnSegments && (S == 1 || all_tiles / S >= 4); ++S) {
    const int64_t waves = (row_blocks * S + sms - 1) / sms;
    const int64_t cost = waves * ((all_tiles + S - 1) / S + 2);
    if (cost < best_cost) {
      best_cost = cost;
      want = S;
    }
  }
  const int seg_tiles = (all_tiles + want - 1) / want;
  const int segs = (all_tiles + seg_tiles - 1) / seg_tiles;  // every segment has tiles
  const int n_lists = 2 * segs;
  if (u8) {
    const int L = (k <= 8) ? 8 : kKnnList;
    int32_t* nrm = base ? (int32_t*)const_cast<void*>(base->nrm) : b.get<int32_t>(M);
    int32_t* qnrm = P.self ? nrm : b.get<int32_t>(Mq);
    int32_t* lids = b.get<int32_t>(Mq * n_lists * L);
    int32_t* lkeys = b.get<int32_t>(Mq * n_lists * L);
    if (!b.ok) return IVHD_ERR_OOM;
    if (e == cudaSuccess) {
      const uint8_t* X = (const uint8_t*)P.X;
      const uint8_t* Q = (const uint8_t*)P.Q;
      if (!base) {
        k_prep_u8<<<blocks(M * Kp), 256, 0, s>>>(X, M, N, Kp, B);
        k_norms_u8s<<<blocks(M), 256, 0, s>>>(X, M, N, nrm);
      }
      if (!P.self) {
        k_prep_u8<<<blocks(Mq * Kp), 256, 0, s>>>(Q, Mq, N, Kp, A);
        k_norms_u8s<<<blocks(Mq), 256, 0, s>>>(Q, Mq, N, qnrm);
      }
      e = (L == 8) ? launch_tc<true, 8>(ma, mb, nullptr, nrm, nullptr, qnrm, (int)Mq, (int)M, Kp,
                                        P.self, segs, seg_tiles, 0.f, lids, (float*)lkeys, err,
                                        s)
                   : launch_tc<true, kKnnList>(ma, mb, nullptr, nrm, nullptr, qnrm, (int)Mq,
                                               (int)M, Kp, P.self, segs, seg_tiles, 0.f, lids,
                                               (float*)lkeys, err, s);
    }
    if (e == cudaSuccess) {
      if (L == 8)
        k_merge_u8<8><<<blocks(Mq), 256, 0, s>>>(lids, lkeys, Mq, k, n_lists, out_knn);
      else
        k_merge_u8<kKnnList><<<blocks(Mq), 256, 0, s>>>(lids, lkeys, Mq, k, n_lists, out_knn);
      e = cudaGetLastError();
    }
  } else {
    float* nrm = base ? (float*)const_cast<void*>(base->nrm) : b.get<float>(M);
    float* qnrm = P.self ? nrm : b.get<float>(Mq);
    const int L = (k <= 8) ? 16 : kKnnList;  // candidates per row and half
    int32_t* cand = b.get<int32_t>(Mq * n_lists * L);
    float* cd = b.get<float>(Mq * n_lists * L);
    int32_t* fb = b.get<int32_t>(Mq);
    if (!b.ok) return IVHD_ERR_OOM;
    const float* X = (const float*)P.X;
    const float* Q = (const float*)P.Q;
    if (e == cudaSuccess) {
      if (P.self) {
        k_prep_f32<<<blocks(M * Kp), 256, 0, s>>>(X, M, N, Kp, A, B);
      } else {
        if (!base) k_prep_f32<<<blocks(M * Kp), 256, 0, s>>>(X, M, N, Kp, nullptr, B);
        k_prep_f32<<<blocks(Mq * Kp), 256, 0, s>>>(Q, Mq, N, Kp, A, nullptr);
        k_norms_f32<<<blocks(Mq), 256, 0, s>>>(Q, Mq, N, qnrm);
      }
      if (!base) k_norms_f32<<<blocks(M), 256, 0, s>>>(X, M, N, nrm);
      e = (L == 16) ? launch_tc<false, 16>(ma, mb, nrm, nullptr, qnrm, nullptr, (int)Mq, (int)M,
                                           Kp, P.self, segs, seg_tiles, eps_coef, cand, cd, err, s)
                    : launch_tc<false, kKnnList>(ma, mb, nrm, nullptr, qnrm, nullptr, (int)Mq,
                                                 (int)M, Kp, P.self, segs, seg_tiles, eps_coef,
                                                 cand, cd, err, s);
    }
    if (e == cudaSuccess) {
      const unsigned g8 = (unsigned)((Mq + 7) / 8);
      if (L == 16)
        k_rerank<16><<<g8, 256, 0, s>>>(Q, (int)Mq, X, (int)M, N, k, n_lists, cand, cd, qnrm,
                                        nrm, eps_coef, out_knn, fb, n_fb, maxerr_bits);
      else
        k_rerank<kKnnList><<<g8, 256, 0, s>>>(Q, (int)Mq, X, (int)M, N, k, n_lists, cand, cd,
                                              qnrm, nrm, eps_coef, out_knn, fb, n_fb,
                                              maxerr_bits);
      e = cudaGetLastError();
    }
    // rows without a certificate: the exact CUDA-core kernel on just those rows
    if (e == cudaSuccess) e = knn_exact_rows_f32(P, fb, n_fb, out_knn, s);
  }
  int32_t h[8] = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, err, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return IVHD_ERR_CUDA;
  if (stats) {
    stats->fallback_rows = u8 ? 0 : h[1];
    float mre = 0.f;
    std::memcpy(&mre, &h[2], sizeof(mre));
    stats->max_rel_err = u8 ? 0.f : mre;
    stats->eps_coef = u8 ? 0.f : eps_coef;
  }
  return h[0] ? IVHD_ERR_TIMEOUT : IVHD_OK;
}

}  // namespace ivhd
