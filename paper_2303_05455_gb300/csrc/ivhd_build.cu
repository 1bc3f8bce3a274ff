// ivhd_build.cu -- create-time set-up of one embedding context (all on the GPU).
//
//   1. validate the kNN rows (range, self loops, duplicates; -1 = absent entry)
//   2. draw r random neighbours per vertex (Sec. 3.3.1 "generated ad hoc";
//      Sec. 3.3.3: never a vertex connected to i), SplitMix64 draws, within the
//      vertex's own embedding when several share the context
//   3. count the symmetric degree of every vertex (each stress term of
//      Eq. 3.16 appears in the rows of both endpoints; a mutual kNN pair is
//      one entry per endpoint, of weight 2 when multiplicity is kept)
//   4. order vertices by degree, descending (stable LSD radix sort), so that
//      the 32 vertices of a warp have near-equal work -- the paper's IVHD-CUDA
//      also sorts particles by connection count (Sec. 5.2)
//   5. size hub rows and SELL slices, scan offsets, fill out- and in-entries,
//      and sort each row's in-part so the layout (and the summation order of
//      the step kernel) is deterministic.
#include <vector>

#include "ivhd_internal.cuh"

namespace ivhd {

namespace {

constexpr int kB = 256;

inline int nblk(int64_t n, int b = kB) { return (int)((n + b - 1) / b); }

__device__ __forceinline__ bool row_has(const int32_t* row, int n, int32_t j) {
  for (int s = 0; s < n; ++s)
    if (row[s] == j) return true;
  return false;
}

// Row validation.  -1 marks an absent entry (a vertex with fewer than k
// neighbours keeps all it has, Sec. 3.3.3).  err bit 0: id out of range,
// bit 1: self loop, bit 2: duplicate in a row.  kv[i] = present entries.
__global__ void k_validate(const int32_t* __restrict__ knn, int64_t M, int k, int32_t* err,
                           int32_t* __restrict__ kv, unsigned long long* sum_kv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int n = 0;
  if (i < M) {
    const int32_t* row = knn + i * k;
    int bad = 0;
    for (int s = 0; s < k; ++s) {
      const int32_t j = row[s];
      if (j == -1) continue;
      ++n;
      if (j < 0 || (int64_t)j >= M) bad |= 1;
      if ((int64_t)j == i) bad |= 2;
      for (int t = 0; t < s; ++t)
        if (row[t] == j) bad |= 4;
    }
    if (bad) atomicOr(err, bad);
    kv[i] = n;
  }
  unsigned long long v = (unsigned long long)n;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(sum_kv, v);
}

__device__ __forceinline__ bool connected(const int32_t* __restrict__ knn, int k, int64_t i,
                                          const int32_t* rowi, int64_t j) {
  if (j == i) return true;
  if (row_has(rowi, k, (int32_t)j)) return true;
  return row_has(knn + j * k, k, (int32_t)i);
}

// Segment of vertex i: the independent embedding it belongs to (one segment
// unless several embeddings share the context).
struct Seg {
  int64_t lo, n;
  int32_t r;
  uint64_t seed;
};
__device__ __forceinline__ Seg seg_of(const SegTable& T, int64_t i) {
  const int e = T.of ? T.of[i] : 0;
  return Seg{T.lo[e], T.n[e], T.r[e], T.seed[e]};
}

// Random neighbours of vertex i in its segment [lo, lo + n) with local index
// li = i - lo: draw t is x = output t of SplitMix64 seeded with s = output li
// of SplitMix64 seeded with (seed ^ "rn_lists"); the candidate is
// lo + floor(x * n / 2^64).  Kept unless connected to i or already kept;
// after 64 r draws missing slots are filled by scanning the segment in order;
// the rest stay -1.  Rows have r_max slots; slots past the segment's r are -1.
__global__ void k_rn_sample(const int32_t* __restrict__ knn, int64_t M, int k, int r_max,
                            SegTable T, int32_t* __restrict__ rn, int32_t* __restrict__ rc,
                            unsigned long long* empty) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const Seg g = seg_of(T, i);
  const int32_t* rowi = knn + i * k;
  int32_t* out = rn + i * r_max;
  int got = 0;
  const uint64_t si = sm64_out(g.seed ^ kDomainRn, (uint64_t)(i - g.lo));
  const int64_t tmax = 64 * (int64_t)g.r;
  for (int64_t t = 0; t < tmax && got < g.r; ++t) {
    const int64_t j = g.lo + (int64_t)__umul64hi(sm64_out(si, (uint64_t)t), (uint64_t)g.n);
    if (connected(knn, k, i, rowi, j) || row_has(out, got, (int32_t)j)) continue;
    out[got++] = (int32_t)j;
  }
  for (int64_t j = g.lo; j < g.lo + g.n && got < g.r; ++j) {
    if (connected(knn, k, i, rowi, j) || row_has(out, got, (int32_t)j)) continue;
    out[got++] = (int32_t)j;
  }
  for (int s = got; s < r_max; ++s) out[s] = -1;
  rc[i] = got;
  if (got < g.r) atomicAdd(empty, (unsigned long long)(g.r - got));
}

// Seeds of a redraw: epoch e > 0 replaces seed s by s ^ mix(e) (e = 0 is the first draw).
__global__ void k_reseed(const uint64_t* __restrict__ in, int n, uint64_t epoch,
                         uint64_t* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = in[e] ^ sm64_mix(epoch);
}

// Kept random neighbours of an existing rn array (rebuild without redrawing).
__global__ void k_rn_count(const int32_t* __restrict__ rn, int64_t M, int r,
                           int32_t* __restrict__ rc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int n = 0;
  for (int s = 0; s < r; ++s) n += rn[i * r + s] >= 0;
  rc[i] = n;
}

// In-degree of every vertex: nn entries (i -> j) and kept rn entries.  An nn
// entry is not mirrored into row j when j already lists i (a mutual pair): the
// out-entry of j stands for the pair, with weight 2 when multiplicity is kept.
// *mutual counts the nn entries whose reverse entry exists.
__global__ void k_count_in(const int32_t* __restrict__ knn, const int32_t* __restrict__ rn,
                           int64_t M, int k, int r, int32_t* __restrict__ in_nn,
                           int32_t* __restrict__ in_rn, unsigned long long* mutual) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n_nn = M * k;
  bool mut = false;
  if (e < n_nn) {
    const int64_t i = e / k;
    const int32_t j = knn[e];
    if (j >= 0) {
      mut = row_has(knn + (int64_t)j * k, k, (int32_t)i);
      if (!mut) atomicAdd(&in_nn[j], 1);
    }
  } else if (e < n_nn + M * r) {
    const int32_t j = rn[e - n_nn];
    if (j >= 0) atomicAdd(&in_rn[j], 1);
  }
  const unsigned b = __ballot_sync(0xffffffffu, mut);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(mutual, (unsigned long long)__popc(b));
}

// Connected components of the undirected kNN graph (nn entries only), for the
// cluster-grouped vertex order: lab[i] ends as the smallest vertex id of i's
// component, whatever order the atomics take.  Labels only decrease and
// lab[x] <= x throughout, so every label chain ends at a root.
__global__ void k_cc_init(int32_t* __restrict__ lab, int64_t M) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) lab[i] = (int32_t)i;
}

// Hooking: for an edge whose endpoints carry different labels, the larger
// label's own slot takes the smaller label.
__global__ void k_cc_hook(const int32_t* __restrict__ knn, int64_t M, int k,
                          int32_t* __restrict__ lab, int32_t* __restrict__ changed) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * (int64_t)k) return;
  const int32_t j = knn[e];
  if (j < 0) return;
  const int32_t a = lab[e / k], b = lab[j];
  if (a == b) return;
  atomicMin(&lab[a > b ? a : b], a < b ? a : b);
  *changed = 1;
}

// Pointer jumping: every label is replaced by the root of its chain.
__global__ void k_cc_jump(int32_t* __restrict__ lab, int64_t M) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int32_t l = lab[i];
  for (int64_t t = 0; t < M; ++t) {  // strictly decreasing chain: ends within M links
    const int32_t n = lab[l];
    if (n == l) break;
    l = n;
  }
  lab[i] = l;
}

// (component label, vertex) pairs for the sort, and the degree key of a
// permuted vertex list.
__global__ void k_label_keys(const int32_t* __restrict__ lab, int64_t M, uint32_t* __restrict__ key,
                             int32_t* __restrict__ val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  key[i] = (uint32_t)lab[i];
  val[i] = (int32_t)i;
}
__global__ void k_gather_keys(const uint32_t* __restrict__ by_vertex,
                              const int32_t* __restrict__ order, int64_t M,
                              uint32_t* __restrict__ key) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < M) key[e] = by_vertex[order[e]];
}

// Degree (stored row entries) and the descending-degree sort key; totals
// are reduced per block before one atomic per block and counter.
__global__ void __launch_bounds__(256) k_degree(const int32_t* __restrict__ kv,
                                                const int32_t* __restrict__ rc,
                                                const int32_t* __restrict__ in_nn,
                                                const int32_t* __restrict__ in_rn, int64_t M,
                                                int32_t* __restrict__ deg,
                                                uint32_t* __restrict__ key,
                                                int32_t* __restrict__ val,
                                                unsigned long long* sum_deg,
                                                unsigned long long* sum_rc, int32_t* max_deg) {
  __shared__ unsigned long long s_deg[8], s_rc[8];
  __shared__ int32_t s_max[8];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int32_t d = 0, c = 0;
  if (i < M) {
    c = rc[i];
    d = kv[i] + c + in_nn[i] + in_rn[i];
    deg[i] = d;
    key[i] = 0xFFFFu - (uint32_t)min(d, 0xFFFF);
    val[i] = (int32_t)i;
  }
  unsigned long long sd = (unsigned long long)d, sr = (unsigned long long)c;
  int32_t md = d;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_down_sync(0xffffffffu, sd, o);
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    md = max(md, __shfl_down_sync(0xffffffffu, md, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_deg[w] = sd;
    s_rc[w] = sr;
    s_max[w] = md;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      sd += s_deg[q];
      sr += s_rc[q];
      md = max(md, s_max[q]);
    }
    atomicAdd(sum_deg, sd);
    atomicAdd(sum_rc, sr);
    atomicMax(max_deg, md);
  }
}

// ---- stable LSD radix sort, 8-bit digits, 1024 elements per block --------

constexpr int kRadixBlock = 1024;

__global__ void __launch_bounds__(kRadixBlock) k_radix_hist(const uint32_t* __restrict__ keys,
                                                            int64_t n, int shift, int nblocks,
                                                            int32_t* __restrict__ counts) {
  __shared__ int32_t h[256];
  if (threadIdx.x < 256) h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t e = (int64_t)blockIdx.x * kRadixBlock + threadIdx.x;
  if (e < n) atomicAdd(&h[(keys[e] >> shift) & 255u], 1);
  __syncthreads();
  if (threadIdx.x < 256) counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kRadixBlock) k_radix_scatter(
    const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    int32_t* __restrict__ vout, int64_t n, int shift, int nblocks,
    const int32_t* __restrict__ offs) {
  __shared__ int32_t wc[kRadixBlock / 32][256];
  for (int t = threadIdx.x; t < (kRadixBlock / 32) * 256; t += kRadixBlock) (&wc[0][0])[t] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * kRadixBlock + threadIdx.x;
  const bool act = e < n;
  const unsigned amask = __ballot_sync(0xffffffffu, act);
  uint32_t key = 0, d = 0;
  int rank = 0;
  if (act) {
    key = kin[e];
    d = (key >> shift) & 255u;
    const unsigned peers = __match_any_sync(amask, d);
    rank = __popc(peers & ((1u << lane) - 1u));
    if (rank == 0) wc[w][d] = __popc(peers);
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    int run = 0;
    for (int q = 0; q < kRadixBlock / 32; ++q) {
      const int t = wc[q][threadIdx.x];
      wc[q][threadIdx.x] = run;
      run += t;
    }
  }
  __syncthreads();
  if (act) {
    const int64_t pos = (int64_t)offs[(int64_t)d * nblocks + blockIdx.x] + wc[w][d] + rank;
    kout[pos] = key;
    vout[pos] = vin[e];
  }
}

// ---- layout sizing ---------------------------------------------------------

// Rows of at most kShortRow in-entries are sorted in registers, longer ones
// by a block in shared memory.
constexpr int kShortRow = 32;

// Per sorted position p: inverse permutation, degree, out-entry count; the
// hub count, and n_long = the number of leading rows (degrees descend) of
// degree above kShortRow, written by the one thread at the boundary.
__global__ void k_sorted_info(const int32_t* __restrict__ perm, const int32_t* __restrict__ deg,
                              const int32_t* __restrict__ kv, const int32_t* __restrict__ rc,
                              int64_t M, int hub_thr, int32_t* __restrict__ inv,
                              int32_t* __restrict__ deg_p, int32_t* __restrict__ outc_p,
                              int32_t* n_hub, int32_t* n_long, int32_t* n_ge,
                              int32_t* n_wide) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= M) return;
  const int32_t i = perm[p];
  inv[i] = (int32_t)p;
  const int32_t d = deg[i];
  deg_p[p] = d;
  outc_p[p] = kv[i] + rc[i];
  if (d >= hub_thr) atomicAdd(n_hub, 1);
  if (d > kShortRow && (p + 1 == M || deg[perm[p + 1]] <= kShortRow)) *n_long = (int32_t)(p + 1);
  if (d >= kWideRow && (p + 1 == M || deg[perm[p + 1]] < kWideRow)) *n_wide = (int32_t)(p + 1);
  // rows with at least 256, 128 and 64 entries (the order is by descending degree)
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int32_t T = 256 >> t;
    if (d >= T && (p + 1 == M || deg[perm[p + 1]] < T)) n_ge[t] = (int32_t)(p + 1);
  }
}

// Storage (in uint32 slots) of hub row p and of SELL slice s; 0 past the end.
__global__ void k_sizes(const int32_t* __restrict__ deg_p, int64_t M, const int32_t* n_hub_d,
                        int64_t max_slices, int64_t* __restrict__ hub_sz,
                        int64_t* __restrict__ slice_sz, int32_t* __restrict__ slice_w) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n_hub = *n_hub_d;
  if (t < M) hub_sz[t] = (t < n_hub) ? (int64_t)((deg_p[t] + 3) & ~3) : 0;
  if (t < max_slices) {
    const int64_t p0 = n_hub + 32 * t;
    int32_t w = 0;
    if (p0 < M) w = (deg_p[p0] + 3) >> 2;  // sorted descending: first of the slice is the max
    slice_w[t] = w;
    slice_sz[t] = (int64_t)w * 128;
  }
}

__global__ void k_widen(const int32_t* __restrict__ a, int64_t* __restrict__ b, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = a[t];
}

__global__ void k_offsets_i32(const int64_t* __restrict__ in, int64_t n, int64_t add,
                              int32_t* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= n) out[t] = (int32_t)(in[t] + add);
}

__device__ __forceinline__ int64_t slot_addr(int64_t p, int t, int64_t n_hub,
                                             const int32_t* __restrict__ hub_off,
                                             const int32_t* __restrict__ slice_off) {
  if (p < n_hub) return (int64_t)hub_off[p] + t;
  const int64_t q = p - n_hub;
  return (int64_t)slice_off[q >> 5] + ((int64_t)(t >> 2) * 32 + (q & 31)) * 4 + (t & 3);
}

// Out-entries of input vertex i: its present nn ids (weight-2 bit on mutual
// pairs when multiplicity is kept), then its kept rn ids (rn bit set).
__global__ void k_fill_out(const int32_t* __restrict__ knn, const int32_t* __restrict__ rn,
                           const int32_t* __restrict__ rc, const int32_t* __restrict__ inv,
                           int64_t M, int k, int r, int dedup, int64_t n_hub,
                           const int32_t* __restrict__ hub_off,
                           const int32_t* __restrict__ slice_off, uint32_t* __restrict__ ids) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t p = inv[i];
  int t = 0;
  for (int s = 0; s < k; ++s) {
    const int32_t j = knn[i * k + s];
    if (j < 0) continue;
    const bool w2 = !dedup && row_has(knn + (int64_t)j * k, k, (int32_t)i);
    ids[slot_addr(p, t++, n_hub, hub_off, slice_off)] = (uint32_t)inv[j] | (w2 ? kW2Bit : 0u);
  }
  const int n = rc[i];
  for (int s = 0; s < n; ++s)
    ids[slot_addr(p, t + s, n_hub, hub_off, slice_off)] = (uint32_t)inv[rn[i * r + s]] | kRnBit;
}

// In-entries: the mirror of every out-entry (i -> j) lands in row j.
__global__ void k_fill_in(const int32_t* __restrict__ knn, const int32_t* __restrict__ rn,
                          const int32_t* __restrict__ inv, const int32_t* __restrict__ outc_p,
                          int64_t M, int k, int r, int64_t n_hub,
                          const int32_t* __restrict__ hub_off,
                          const int32_t* __restrict__ slice_off, int32_t* __restrict__ cursor,
                          uint32_t* __restrict__ ids) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n_nn = M * k;
  int64_t i;
  int32_t j;
  uint32_t bit;
  if (e < n_nn) {
    i = e / k;
    j = knn[e];
    if (j < 0) return;
    if (row_has(knn + (int64_t)j * k, k, (int32_t)i)) return;  // mutual: held by j's out-entry
    bit = 0;
  } else if (e < n_nn + M * r) {
    i = (e - n_nn) / r;
    j = rn[e - n_nn];
    if (j < 0) return;
    bit = kRnBit;
  } else {
    return;
  }
  const int64_t pj = inv[j];
  const int slot = outc_p[pj] + atomicAdd(&cursor[pj], 1);
  ids[slot_addr(pj, slot, n_hub, hub_off, slice_off)] = (uint32_t)inv[i] | bit;
}

// The in-part of every row (the mirrored entries, filled in arbitrary order
// by k_fill_in) is sorted ascending so the layout, and with it every
// summation order, is deterministic.  Values within a row are distinct
// (one entry per source vertex and kind).

// Compare-exchange of a bitonic network: ascending when up.
__device__ __forceinline__ void bitonic_ce(uint32_t& x, uint32_t& y, bool up) {
  const uint32_t lo = min(x, y), hi = max(x, y);
  x = up ? lo : hi;
  y = up ? hi : lo;
}

// Bitonic sort of N register values (N a power of two, fully unrolled).
template <int N>
__device__ __forceinline__ void bitonic_regs(uint32_t (&v)[kShortRow]) {
#pragma unroll
  for (int k = 2; k <= N; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int l = i ^ j;
        if (l > i) bitonic_ce(v[i], v[l], (i & k) == 0);
      }
}

// SELL rows with at most kShortRow in-entries: thread per row, values in
// registers; the network size is the warp's largest row rounded up.
__global__ void __launch_bounds__(256) k_sort_in_short(const int32_t* __restrict__ deg_p,
                                                       const int32_t* __restrict__ outc_p,
                                                       int64_t M, int64_t n_hub,
                                                       const int32_t* __restrict__ slice_off,
                                                       uint32_t* __restrict__ ids) {
  const int64_t p = n_hub + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int b = 0, m = 0;
  if (p < M) {
    b = outc_p[p];
    m = deg_p[p] - b;
    if (m > kShortRow) m = 0;  // sorted by k_sort_in_long
  }
  const int mw = __reduce_max_sync(0xffffffffu, m);
  if (mw <= 1) return;
  uint32_t v[kShortRow];
#pragma unroll
  for (int t = 0; t < kShortRow; ++t)
    v[t] = (t < m) ? ids[slot_addr(p, b + t, n_hub, nullptr, slice_off)] : 0xFFFFFFFFu;
  if (mw <= 4)
    bitonic_regs<4>(v);
  else if (mw <= 8)
    bitonic_regs<8>(v);
  else if (mw <= 16)
    bitonic_regs<16>(v);
  else
    bitonic_regs<32>(v);
#pragma unroll
  for (int t = 0; t < kShortRow; ++t)
    if (t < m) ids[slot_addr(p, b + t, n_hub, nullptr, slice_off)] = v[t];
}

// Hub rows, and SELL rows with more than kShortRow in-entries: one block per
// row, bitonic sort in shared memory (rows up to kLongSortSmem entries), or a
// stable rank sort that reads a copy of the layout (longer rows).
constexpr int kLongSortSmem = 8192;
__global__ void __launch_bounds__(256) k_sort_in_long(const int32_t* __restrict__ deg_p,
                                                      const int32_t* __restrict__ outc_p,
                                                      int64_t n_hub,
                                                      const int32_t* __restrict__ hub_off,
                                                      const int32_t* __restrict__ slice_off,
                                                      const uint32_t* __restrict__ copy,
                                                      uint32_t* __restrict__ ids) {
  __shared__ uint32_t sh[kLongSortSmem];
  const int64_t p = blockIdx.x;
  const int b = outc_p[p], m = deg_p[p] - b;
  if (m <= 1 || (p >= n_hub && m <= kShortRow)) return;
  if (m <= kLongSortSmem) {
    int n2 = 2;
    while (n2 < m) n2 <<= 1;
    for (int t = threadIdx.x; t < n2; t += blockDim.x)
      sh[t] = (t < m) ? ids[slot_addr(p, b + t, n_hub, hub_off, slice_off)] : 0xFFFFFFFFu;
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < n2; t += blockDim.x) {
          const int l = t ^ j;
          if (l > t) {
            uint32_t x = sh[t], y = sh[l];
            bitonic_ce(x, y, (t & k) == 0);
            sh[t] = x;
            sh[l] = y;
          }
        }
        __syncthreads();
      }
    for (int t = threadIdx.x; t < m; t += blockDim.x)
      ids[slot_addr(p, b + t, n_hub, hub_off, slice_off)] = sh[t];
  } else {
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      const uint32_t v = copy[slot_addr(p, b + t, n_hub, hub_off, slice_off)];
      int rank = 0;
      for (int u = 0; u < m; ++u) {
        const uint32_t w = copy[slot_addr(p, b + u, n_hub, hub_off, slice_off)];
        rank += (w < v) || (w == v && u < t);
      }
      ids[slot_addr(p, b + rank, n_hub, hub_off, slice_off)] = v;
    }
  }
}

// ---- exclusive scan of int64 values; out has n + 1 entries ----------------

constexpr int kScanBlock = 1024, kScanItems = 4, kScanTile = kScanBlock * kScanItems;

__global__ void __launch_bounds__(kScanBlock) k_scan_tile(const int64_t* __restrict__ in, int64_t n,
                                                          int64_t* __restrict__ out,
                                                          int64_t* __restrict__ bsum) {
  __shared__ int64_t wsum[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t tot = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = (base + q < n) ? in[base + q] : 0;
    tot += v[q];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    int64_t s = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    wsum[lane] = s;
  }
  __syncthreads();
  int64_t run = incl - tot + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    run += v[q];
    if (base + q < n) out[base + q + 1] = run;
  }
  if (threadIdx.x == kScanBlock - 1 && bsum) bsum[blockIdx.x] = wsum[31];
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ boff) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t + 1] += boff[t / kScanTile];
}

// Device buffers freed on scope exit.
struct Scratch {
  std::vector<void*> bufs;
  cudaStream_t s;
  bool ok = true;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <class T>
  T* get(int64_t n) {
    void* q = nullptr;
    if (dev_alloc(&q, (size_t)(n > 0 ? n : 1) * sizeof(T), s) != cudaSuccess) {
      ok = false;
      return nullptr;
    }
    bufs.push_back(q);
    return (T*)q;
  }
  ~Scratch() {
    for (void* q : bufs) dev_free(q, s);
  }
};

cudaError_t scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, Scratch& sc,
                     int64_t* launches) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles <= 1) {
    k_scan_tile<<<1, kScanBlock, 0, s>>>(in, n, out, nullptr);
    ++*launches;
    return cudaGetLastError();
  }
  int64_t* bsum = sc.get<int64_t>(tiles);
  int64_t* boff = sc.get<int64_t>(tiles + 1);
  if (!sc.ok) return cudaErrorMemoryAllocation;
  k_scan_tile<<<(unsigned)tiles, kScanBlock, 0, s>>>(in, n, out, bsum);
  ++*launches;
  cudaError_t e = scan_i64(bsum, boff, tiles, s, sc, launches);
  if (e != cudaSuccess) return e;
  k_scan_add<<<nblk(n), kB, 0, s>>>(out, n, boff);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace

struct HostTotals {
  int32_t err;
  int32_t n_hub;
  int32_t max_deg;
  int32_t n_long;
  int32_t n_ge[3];
  int32_t n_wide;
  unsigned long long sum_kv;
  unsigned long long sum_deg;
  unsigned long long sum_rc;
  unsigned long long mutual;
  unsigned long long empty;
  int64_t hub_total;
  int64_t sell_total;
};

#define IVHD_TRY(x)                                                      \
  do {                                                                   \
    cudaError_t e_ = (x);                                                \
    if (e_ != cudaSuccess)                                               \
      return (e_ == cudaErrorMemoryAllocation) ? IVHD_ERR_OOM : IVHD_ERR_CUDA; \
  } while (0)

ivhd_status build_layout(ivhd_ctx* ctx, bool draw_rn, uint64_t rn_epoch) {
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->M;
  const int k = ctx->k, r = ctx->r;
  const int dedup = ctx->p.dedup_mutual ? 1 : 0;
  Scratch sc(s);

  // totals block lives in device memory, read back twice
  HostTotals* tot_d = sc.get<HostTotals>(1);
  int32_t* kv = sc.get<int32_t>(M);
  if (!sc.ok) return IVHD_ERR_OOM;
  IVHD_TRY(cudaMemsetAsync(tot_d, 0, sizeof(HostTotals), s));

  // 1. validation -- nothing below may index with an unchecked id
  k_validate<<<nblk(M), kB, 0, s>>>(ctx->knn, M, k, &tot_d->err, kv, &tot_d->sum_kv);
  ++ctx->setup_launches;
  IVHD_TRY(cudaGetLastError());
  HostTotals h{};
  IVHD_TRY(cudaMemcpyAsync(&h, tot_d, sizeof(h), cudaMemcpyDeviceToHost, s));
  IVHD_TRY(cudaStreamSynchronize(s));
  if (h.err) return IVHD_ERR_INDEX;

  // 2. random neighbours (drawn, or kept from the previous layout)
  int32_t* rc = sc.get<int32_t>(M);
  int32_t* in_nn = sc.get<int32_t>(M);
  int32_t* in_rn = sc.get<int32_t>(M);
  int32_t* deg = sc.get<int32_t>(M);
  uint32_t* key0 = sc.get<uint32_t>(M);
  uint32_t* key1 = sc.get<uint32_t>(M);
  int32_t* val0 = sc.get<int32_t>(M);
  int32_t* deg_p = sc.get<int32_t>(M);
  int32_t* outc_p = sc.get<int32_t>(M);
  int32_t* cursor = sc.get<int32_t>(M);
  if (!sc.ok) return IVHD_ERR_OOM;
  if (r == 0) {
    IVHD_TRY(cudaMemsetAsync(rc, 0, M * sizeof(int32_t), s));
  } else if (draw_rn) {
    SegTable T = ctx->seg;
    // a redraw (epoch > 0) reseeds every segment's stream
    uint64_t* seeds = nullptr;
    if (rn_epoch) {
      seeds = sc.get<uint64_t>(ctx->n_seg);
      if (!sc.ok) return IVHD_ERR_OOM;
      k_reseed<<<nblk(ctx->n_seg), kB, 0, s>>>(T.seed, ctx->n_seg, rn_epoch, seeds);
      ++ctx->setup_launches;
      T.seed = seeds;
    }
    k_rn_sample<<<nblk(M), kB, 0, s>>>(ctx->knn, M, k, r, T, ctx->rn, rc, &tot_d->empty);
    ++ctx->setup_launches;
  } else {
    k_rn_count<<<nblk(M), kB, 0, s>>>(ctx->rn, M, r, rc);
    ++ctx->setup_launches;
  }
  IVHD_TRY(cudaGetLastError());

  // 3. degrees
  IVHD_TRY(cudaMemsetAsync(in_nn, 0, M * sizeof(int32_t), s));
  IVHD_TRY(cudaMemsetAsync(in_rn, 0, M * sizeof(int32_t), s));
  IVHD_TRY(cudaMemsetAsync(cursor, 0, M * sizeof(int32_t), s));
  const int64_t n_entries = M * (int64_t)(k + r);
  k_count_in<<<nblk(n_entries), kB, 0, s>>>(ctx->knn, ctx->rn, M, k, r, in_nn, in_rn,
                                            &tot_d->mutual);
  ++ctx->setup_launches;
  k_degree<<<nblk(M), kB, 0, s>>>(kv, rc, in_nn, in_rn, M, deg, key0, val0, &tot_d->sum_deg,
                                  &tot_d->sum_rc, &tot_d->max_deg);
  ++ctx->setup_launches;
  IVHD_TRY(cudaGetLastError());

  // 4. stable sort by descending degree: two 8-bit passes over the 16-bit key
  //    (cluster order: first a stable sort by component label, whose order the
  //    degree passes then keep among vertices of equal degree)
  {
    const int nb = (int)((M + kRadixBlock - 1) / kRadixBlock);
    const int64_t nc = (int64_t)nb * 256;
    int32_t* counts = sc.get<int32_t>(nc);
    int64_t* c64 = sc.get<int64_t>(nc);
    int64_t* o64 = sc.get<int64_t>(nc + 1);
    int32_t* offs = sc.get<int32_t>(nc + 1);
    int32_t* val1 = sc.get<int32_t>(M);
    if (!sc.ok) return IVHD_ERR_OOM;
    auto radix_pass = [&](const uint32_t* kin, const int32_t* vin, uint32_t* kout, int32_t* vout,
                          int shift) -> cudaError_t {
      k_radix_hist<<<nb, kRadixBlock, 0, s>>>(kin, M, shift, nb, counts);
      k_widen<<<nblk(nc), kB, 0, s>>>(counts, c64, nc);
      ctx->setup_launches += 2;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      e = scan_i64(c64, o64, nc, s, sc, &ctx->setup_launches);
      if (e != cudaSuccess) return e;
      k_offsets_i32<<<nblk(nc + 1), kB, 0, s>>>(o64, nc, 0, offs);
      k_radix_scatter<<<nb, kRadixBlock, 0, s>>>(kin, vin, kout, vout, M, shift, nb, offs);
      ctx->setup_launches += 2;
      return cudaGetLastError();
    };
    const uint32_t* deg_kin = key0;
    const int32_t* deg_vin = val0;
    if (ctx->p.order == IVHD_ORDER_DEGREE_CLUSTER) {
      int32_t* lab = sc.get<int32_t>(M);
      int32_t* changed = sc.get<int32_t>(1);
      uint32_t* ka = sc.get<uint32_t>(M);
      uint32_t* kb = sc.get<uint32_t>(M);
      int32_t* va = sc.get<int32_t>(M);
      int32_t* vb = sc.get<int32_t>(M);
      if (!sc.ok) return IVHD_ERR_OOM;
      k_cc_init<<<nblk(M), kB, 0, s>>>(lab, M);
      ++ctx->setup_launches;
      for (int round = 0; round < 64; ++round) {  // converges in a few rounds
        int32_t h_changed = 0;
        IVHD_TRY(cudaMemsetAsync(changed, 0, sizeof(int32_t), s));
        k_cc_hook<<<nblk(M * (int64_t)k), kB, 0, s>>>(ctx->knn, M, k, lab, changed);
        k_cc_jump<<<nblk(M), kB, 0, s>>>(lab, M);
        ctx->setup_launches += 2;
        IVHD_TRY(cudaGetLastError());
        IVHD_TRY(cudaMemcpyAsync(&h_changed, changed, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        IVHD_TRY(cudaStreamSynchronize(s));
        if (!h_changed) break;
      }
      k_label_keys<<<nblk(M), kB, 0, s>>>(lab, M, ka, va);
      ++ctx->setup_launches;
      IVHD_TRY(cudaGetLastError());
      int bits = 1;
      while (bits < 31 && ((int64_t)1 << bits) < M) ++bits;
      uint32_t* kin = ka;
      int32_t* vin = va;
      uint32_t* kout = kb;
      int32_t* vout = vb;
      for (int shift = 0; shift < bits; shift += 8) {
        IVHD_TRY(radix_pass(kin, vin, kout, vout, shift));
        uint32_t* kt = kin;
        kin = kout;
        kout = kt;
        int32_t* vt = vin;
        vin = vout;
        vout = vt;
      }
      // vin: vertices by component; kout (free): their degree keys
      k_gather_keys<<<nblk(M), kB, 0, s>>>(key0, vin, M, kout);
      ++ctx->setup_launches;
      IVHD_TRY(cudaGetLastError());
      deg_kin = kout;
      deg_vin = vin;
    }
    // pass 0: (deg_kin, deg_vin) -> (key1, val1); pass 1: (key1, val1) -> (key0, perm)
    IVHD_TRY(radix_pass(deg_kin, deg_vin, key1, val1, 0));
    IVHD_TRY(radix_pass(key1, val1, key0, ctx->perm, 8));
  }

  // 5. sizes and offsets
  k_sorted_info<<<nblk(M), kB, 0, s>>>(ctx->perm, deg, kv, rc, M, ctx->hub_threshold, ctx->inv,
                                       deg_p, outc_p, &tot_d->n_hub, &tot_d->n_long,
                                       tot_d->n_ge, &tot_d->n_wide);
  ++ctx->setup_launches;
  const int64_t max_slices = (M + 31) / 32;
  int64_t* hub_sz = sc.get<int64_t>(M);
  int64_t* hub_o64 = sc.get<int64_t>(M + 1);
  int64_t* sl_sz = sc.get<int64_t>(max_slices);
  int64_t* sl_o64 = sc.get<int64_t>(max_slices + 1);
  int32_t* slice_w = sc.get<int32_t>(max_slices);
  if (!sc.ok) return IVHD_ERR_OOM;
  k_sizes<<<nblk(M > max_slices ? M : max_slices), kB, 0, s>>>(deg_p, M, &tot_d->n_hub,
                                                               max_slices, hub_sz, sl_sz, slice_w);
  ++ctx->setup_launches;
  IVHD_TRY(cudaGetLastError());
  IVHD_TRY(scan_i64(hub_sz, hub_o64, M, s, sc, &ctx->setup_launches));
  IVHD_TRY(scan_i64(sl_sz, sl_o64, max_slices, s, sc, &ctx->setup_launches));
  IVHD_TRY(cudaMemcpyAsync(&tot_d->hub_total, hub_o64 + M, sizeof(int64_t),
                           cudaMemcpyDeviceToDevice, s));
  IVHD_TRY(cudaMemcpyAsync(&tot_d->sell_total, sl_o64 + max_slices, sizeof(int64_t),
                           cudaMemcpyDeviceToDevice, s));
  IVHD_TRY(cudaMemcpyAsync(&h, tot_d, sizeof(h), cudaMemcpyDeviceToHost, s));
  IVHD_TRY(cudaStreamSynchronize(s));

  ctx->n_hub = h.n_hub;
  for (int t = 0; t < 3; ++t) ctx->n_ge[t] = h.n_ge[t];
  ctx->n_wide = h.n_wide < h.n_hub ? h.n_wide : h.n_hub;  // wide rows are hub rows
  ctx->n_slices = (M - h.n_hub + 31) / 32;
  ctx->n_slots = h.hub_total + h.sell_total;
  ctx->nnz_sym = (int64_t)h.sum_deg;
  // stress terms: every present kNN entry (a mutual pair once when deduplicated)
  // plus the kept rn draws
  ctx->n_terms = (int64_t)h.sum_kv - (dedup ? (int64_t)(h.mutual / 2) : 0) + (int64_t)h.sum_rc;
  ctx->max_degree = h.max_deg;
  if (draw_rn) ctx->empty_rn = (int32_t)h.empty;
  if (ctx->n_slots >= (int64_t)0x7FFFFFFF) return IVHD_ERR_ARG;

  IVHD_TRY(dev_alloc((void**)&ctx->ids, (size_t)(ctx->n_slots + 4) * sizeof(uint32_t), s));
  IVHD_TRY(dev_alloc((void**)&ctx->hub_off, (size_t)(ctx->n_hub + 1) * sizeof(int32_t), s));
  IVHD_TRY(dev_alloc((void**)&ctx->slice_off, (size_t)(ctx->n_slices + 1) * sizeof(int32_t), s));
  IVHD_TRY(dev_alloc((void**)&ctx->slice_w, (size_t)(ctx->n_slices + 1) * sizeof(int32_t), s));
  IVHD_TRY(cudaMemsetAsync(ctx->ids, 0xFF, (size_t)(ctx->n_slots + 4) * sizeof(uint32_t), s));
  k_offsets_i32<<<nblk(ctx->n_hub + 1), kB, 0, s>>>(hub_o64, ctx->n_hub, 0, ctx->hub_off);
  k_offsets_i32<<<nblk(ctx->n_slices + 1), kB, 0, s>>>(sl_o64, ctx->n_slices, h.hub_total,
                                                       ctx->slice_off);
  ctx->setup_launches += 2;
  IVHD_TRY(cudaMemcpyAsync(ctx->slice_w, slice_w, (size_t)ctx->n_slices * sizeof(int32_t),
                           cudaMemcpyDeviceToDevice, s));
  IVHD_TRY(cudaGetLastError());

  k_fill_out<<<nblk(M), kB, 0, s>>>(ctx->knn, ctx->rn, rc, ctx->inv, M, k, r, dedup, ctx->n_hub,
                                    ctx->hub_off, ctx->slice_off, ctx->ids);
  k_fill_in<<<nblk(n_entries), kB, 0, s>>>(ctx->knn, ctx->rn, ctx->inv, outc_p, M, k, r,
                                           ctx->n_hub, ctx->hub_off, ctx->slice_off, cursor,
                                           ctx->ids);
  ctx->setup_launches += 2;
  IVHD_TRY(cudaGetLastError());
  if (M - ctx->n_hub > 0) {
    k_sort_in_short<<<nblk(M - ctx->n_hub), 256, 0, s>>>(deg_p, outc_p, M, ctx->n_hub,
                                                         ctx->slice_off, ctx->ids);
    ++ctx->setup_launches;
  }
  const int64_t n_long = ctx->n_hub > h.n_long ? ctx->n_hub : h.n_long;
  if (n_long > 0) {
    // rows longer than the shared-memory sort read a copy of the whole layout
    uint32_t* copy = nullptr;
    if (h.max_deg > kLongSortSmem) {
      copy = sc.get<uint32_t>(ctx->n_slots);
      if (!sc.ok) return IVHD_ERR_OOM;
      IVHD_TRY(cudaMemcpyAsync(copy, ctx->ids, (size_t)ctx->n_slots * sizeof(uint32_t),
                               cudaMemcpyDeviceToDevice, s));
    }
    k_sort_in_long<<<(unsigned)n_long, 256, 0, s>>>(deg_p, outc_p, ctx->n_hub, ctx->hub_off,
                                                    ctx->slice_off, copy, ctx->ids);
    ++ctx->setup_launches;
  }
  IVHD_TRY(cudaGetLastError());
  // the layout is complete once the stream reaches here; scratch frees follow in order
  return IVHD_OK;
}

}  // namespace ivhd
