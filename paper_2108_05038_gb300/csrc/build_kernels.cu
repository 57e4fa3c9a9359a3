// Vertical-database kernels: item counting (K1), bitmap build (K2), the
// database sample of the class-cost estimate and row popcounts.
//
// Vertical representation (Ch. 2, Def. "Transaction id list"): row r holds the
// tidlist of item rank_item[r] as a bitmap, bit t of the row set iff
// transaction t contains the item.  Bits past D stay zero.
#include "fim_internal.cuh"

namespace fim {
namespace {

constexpr uint32_t kSmemHistMax = 12288;  // items counted in shared memory (48 KB)

// K1: item supports with set semantics.  One thread per transaction of at most
// kShortTx items: it reads its items in order, and an item counts unless an
// earlier position of the same transaction holds the same id; while the ids
// seen so far are strictly ascending (the usual layout) a new id above the last
// one needs no comparison, otherwise it is compared with every earlier position.
// Longer transactions are taken by the whole warp, one after the other: the
// lanes read 32 consecutive items at a time (coalesced), a lane's item counts
// unless the same id sits at a lower lane of the chunk (__match_any_sync) or in
// an earlier chunk (compared by shuffles).  Counts go to a shared histogram per
// CTA when N is small, flushed with one global atomic per nonzero counter.  Also
// validates ids and offsets and records the longest transaction (distinct
// items).  Only items[0, off[D]) is ever read, whatever the offsets: a
// transaction whose range is reversed or leaves [0, off[D]] is reported and
// skipped, and so is every transaction when off[0] != 0.
// flags = [error bits, longest transaction, off[0], off[D]].
constexpr uint32_t kShortTx = 64;

__global__ void k_item_count(const uint32_t* __restrict__ off, const uint32_t* __restrict__ items, uint32_t D,
                             uint32_t N, uint32_t* __restrict__ cnt, uint32_t* flags) {
  extern __shared__ uint32_t hist[];
  const bool use_smem = N <= kSmemHistMax;
  if (use_smem) {
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) hist[i] = 0;
    __syncthreads();
  }
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t first = off[0], nnz = off[D];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    flags[2] = first;
    flags[3] = nnz;
  }
  uint32_t local_max = 0, local_err = first != 0 ? DEV_ERR_OFFSETS : 0u;
  auto bump = [&](uint32_t it) {
    if (use_smem) atomicAdd(&hist[it], 1u);
    else atomicAdd(&cnt[it], 1u);
  };
  const uint32_t nthreads = gridDim.x * blockDim.x;
  // (warp-uniform loop: lane l of the warp takes transaction base + l)
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); first == 0 && base < D; base += nthreads) {
    const uint32_t t = base + lane;
    uint32_t b = 0, e = 0;
    bool valid = false;
    if (t < D) {
      b = off[t];
      e = off[t + 1];
      valid = e >= b && e <= nnz;
      if (!valid) local_err |= DEV_ERR_OFFSETS;
    }
    const bool wide = valid && e - b > kShortTx;
    if (valid && !wide) {
      uint32_t distinct = 0, prev = 0;
      bool asc = true;  // the ids so far strictly ascending, prev the last of them
      for (uint32_t k0 = b; k0 < e; k0 += 4) {
        uint32_t v[4];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) v[u] = k0 + u < e ? items[k0 + u] : 0u;  // (loads in flight together)
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
          const uint32_t k = k0 + u;
          if (k >= e) break;
          const uint32_t it = v[u];
          bool dup = false;
          if (k > b && !(asc && it > prev)) {
            asc = false;
            for (uint32_t q = b; q < k && !dup; ++q) dup = items[q] == it;
          }
          prev = it;
          if (it >= N) {
            local_err |= DEV_ERR_ITEM_RANGE;
          } else if (!dup) {
            ++distinct;
            bump(it);
          }
        }
      }
      local_max = max(local_max, distinct);
    }
    for (uint32_t pend = __ballot_sync(0xffffffffu, wide); pend; pend &= pend - 1) {
      const uint32_t src = __ffs(pend) - 1;
      const uint32_t wb = __shfl_sync(0xffffffffu, b, src), we = __shfl_sync(0xffffffffu, e, src);
      uint32_t distinct = 0;
      for (uint32_t c0 = wb; c0 < we; c0 += 32) {
        const uint32_t k = c0 + lane;
        const bool in = k < we;
        const uint32_t it = in ? items[k] : 0xffffffffu;
        const bool ok = in && it < N;
        if (in && !ok) local_err |= DEV_ERR_ITEM_RANGE;
        // repeat within this chunk: a lower lane holds the same id
        const uint32_t same = __match_any_sync(0xffffffffu, it);
        bool dup = (same & ((1u << lane) - 1u)) != 0u;
        // repeat in an earlier chunk of the same transaction
        for (uint32_t p0 = wb; p0 < c0; p0 += 32) {
          const uint32_t prv = items[p0 + lane];  // p0 + 32 <= c0 < we: always in range
          for (uint32_t q = 0; q < 32; ++q) dup |= __shfl_sync(0xffffffffu, prv, q) == it;
        }
        const bool count = ok && !dup;
        distinct += __popc(__ballot_sync(0xffffffffu, count));
        if (count) bump(it);
      }
      local_max = max(local_max, distinct);
    }
  }
  if (local_err) atomicOr(&flags[0], local_err);
  local_max = __reduce_max_sync(0xffffffffu, local_max);
  if (lane == 0 && local_max) atomicMax(&flags[1], local_max);
  if (use_smem) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x)
      if (hist[i]) atomicAdd(&cnt[i], hist[i]);
  }
}

// K2: scatter transaction bits into the item-major bitmap rows of kept items.
// A warp takes 32 consecutive transactions (one bitmap word of every row, lane =
// bit); at each position j the lanes whose j-th item maps to the same row are
// grouped by __match_any_sync, and one lane ORs the whole group's bits into the
// word, so a popular item costs one atomic per word and position instead of one
// per transaction.  The offsets and ids were validated by K1.
__global__ void k_bitmap_build(const uint32_t* __restrict__ off, const uint32_t* __restrict__ items, uint32_t D,
                               const int32_t* __restrict__ item_rank, uint32_t* __restrict__ bits, uint32_t stride) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t w0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32u; w0 < D; w0 += warps * 32u) {
    const uint32_t t = w0 + lane;
    const uint32_t b = t < D ? off[t] : 0u, e = t < D ? off[t + 1] : 0u;
    const uint32_t len = e - b;
    const uint32_t maxlen = __reduce_max_sync(0xffffffffu, len);
    uint32_t* const col = bits + (w0 >> 5);
    for (uint32_t j0 = 0; j0 < maxlen; j0 += 4) {  // four positions per round: their loads in flight together
      uint32_t it[4];
      int32_t r[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) it[u] = j0 + u < len ? items[b + j0 + u] : 0xffffffffu;
#pragma unroll
      for (int u = 0; u < 4; ++u) r[u] = it[u] != 0xffffffffu ? item_rank[it[u]] : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t key = r[u] >= 0 ? (uint32_t)r[u] : 0xffffffffu;
        const uint32_t grp = __match_any_sync(0xffffffffu, key);
        if (r[u] >= 0 && lane == (uint32_t)(__ffs(grp) - 1)) atomicOr(col + (size_t)r[u] * stride, grp);
      }
    }
  }
}

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  // k-th output of SplitMix64 (Steele, Lea, Flood 2014) started at state `seed`
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Database sample D_s drawn with replacement (Sec. 6.1): sample row k is
// transaction ((x_k >> 32) * D) >> 32; its kept items are set in bit k of the
// sample bitmap rows (same row order as the full database).
__global__ void k_sample_build(const uint32_t* __restrict__ off, const uint32_t* __restrict__ items, uint32_t D,
                               const int32_t* __restrict__ item_rank, uint64_t seed, uint32_t m,
                               uint32_t* __restrict__ sbits, uint32_t sstride) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    uint64_t x = splitmix64_at(seed, k);
    uint32_t t = (uint32_t)(((x >> 32) * (uint64_t)D) >> 32);
    const uint32_t bit = 1u << (k & 31), word = k >> 5;
    for (uint32_t q = off[t]; q < off[t + 1]; ++q) {
      int32_t r = item_rank[items[q]];
      if (r >= 0) atomicOr(&sbits[(size_t)r * sstride + word], bit);
    }
  }
}

// supp[r] = popcount of row r (one CTA per row).
__global__ void k_row_popcount(const uint32_t* __restrict__ bits, uint32_t stride, uint32_t* __restrict__ supp) {
  const uint4* row = reinterpret_cast<const uint4*>(bits + (size_t)blockIdx.x * stride);
  uint32_t s = 0;
  for (uint32_t i = threadIdx.x; i < stride / 4; i += blockDim.x) {
    uint4 v = row[i];
    s += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
  }
  s = __reduce_add_sync(0xffffffffu, s);
  __shared__ uint32_t wsum[32];
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) tot += wsum[w];
    supp[blockIdx.x] = tot;
  }
}

// Exclusive prefix sum over the 1024 threads of a CTA of each thread's total v (thread order); returns the
// sum of all threads through *total.  Every thread of the CTA calls it.
__device__ uint32_t cta_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t wsum[32];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (uint32_t d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < (blockDim.x >> 5) ? wsum[lane] : 0u;
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    wsum[lane] = w;  // inclusive
  }
  __syncthreads();
  const uint32_t before_warp = warp ? wsum[warp - 1] : 0u;
  *total = wsum[(blockDim.x >> 5) - 1];
  __syncthreads();  // wsum is reused by the next call
  return before_warp + x - v;
}

// The class costs of an estimate and their LPT order, on the device: one warp per row i of a sample mined
// over all its R rows.  Row i is a class of the sample when ssupp[i] >= minsup_s; its cost is per[i] (the
// sample's itemsets whose lowest row is i, or the DFS intersections below it) plus, for the intersection
// measure, its level-2 candidates (the frequent sample rows after i); 0 for the other rows.  The order is the
// rows by descending cost, ties by row (what a stable sort by cost gives): row i goes to position
// rank(i) = #{j : cost_j > cost_i, or cost_j = cost_i and j < i}.  The warp recomputes the costs of all rows
// (32 at a time, the frequent-row counts by ballot) instead of waiting for another kernel to store them.
__global__ void k_est_order(const unsigned long long* __restrict__ per, const uint32_t* __restrict__ ssupp,
                            uint32_t minsup_s, uint32_t intersections, uint32_t R,
                            unsigned long long* __restrict__ tally, uint32_t* __restrict__ order) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= R) return;  // (whole warps leave together)
  // frequent sample rows in all, and up to and including row i
  uint32_t n_freq = 0, upto_i = 0;
  for (uint32_t j0 = 0; j0 < R; j0 += 32) {
    const uint32_t j = j0 + lane;
    const uint32_t b = __ballot_sync(0xffffffffu, j < R && __ldg(ssupp + j) >= minsup_s);
    n_freq += __popc(b);
    if (j0 <= i) upto_i += __popc(i - j0 >= 31 ? b : b & ((2u << (i - j0)) - 1u));
  }
  const bool fi = __ldg(ssupp + i) >= minsup_s;
  const unsigned long long ti = fi ? __ldg(per + i) + (intersections ? (unsigned long long)(n_freq - upto_i) : 0ull) : 0ull;
  // rows before row i in the order
  uint32_t rank = 0, upto = 0;
  for (uint32_t j0 = 0; j0 < R; j0 += 32) {
    const uint32_t j = j0 + lane;
    const bool fj = j < R && __ldg(ssupp + j) >= minsup_s;
    const uint32_t b = __ballot_sync(0xffffffffu, fj);
    const uint32_t incl = upto + __popc(b & ((2u << lane) - 1u));  // frequent rows up to and including j
    upto += __popc(b);
    const unsigned long long tj = fj ? __ldg(per + j) + (intersections ? (unsigned long long)(n_freq - incl) : 0ull) : 0ull;
    rank += __popc(__ballot_sync(0xffffffffu, j < R && (tj > ti || (tj == ti && j < i))));
  }
  if (lane == 0) {
    tally[i] = ti;
    order[rank] = i;
  }
}

// The queue order of a mine's frequent rows r0 .. r0 + n1 - 1 from an estimate's order over all R rows:
// the order's entries >= r0, in their order, minus r0 (one CTA of 1024 threads, R <= kEstDeviceRows).
__global__ void __launch_bounds__(1024) k_order_suffix(const uint32_t* __restrict__ order, uint32_t R, uint32_t r0,
                                                       uint32_t* __restrict__ out) {
  uint32_t v[4], cnt = 0;
#pragma unroll
  for (uint32_t q = 0; q < 4; ++q) {
    const uint32_t i = 4 * threadIdx.x + q;
    v[q] = i < R ? order[i] : 0u;
    cnt += i < R && v[q] >= r0;
  }
  uint32_t total = 0;
  uint32_t pos = cta_exclusive_scan(cnt, &total);
#pragma unroll
  for (uint32_t q = 0; q < 4; ++q) {
    const uint32_t i = 4 * threadIdx.x + q;
    if (i < R && v[q] >= r0) out[pos++] = v[q] - r0;
  }
}

__global__ void k_iota(uint32_t* out, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = i;
}

uint32_t grid_for(uint64_t n, uint32_t threads, uint32_t cap = 152 * 32) {
  uint64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (uint32_t)g;
}

}  // namespace

cudaError_t launch_item_count(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t* cnt,
                              uint32_t* flags, cudaStream_t st) {
  const uint32_t threads = 256;
  size_t smem = N <= kSmemHistMax ? (size_t)N * 4 : 0;
  // one thread per transaction; with a shared histogram every CTA flushes its nonzero counters: two CTAs per
  // SM, each thread taking several transactions
  uint32_t grid = grid_for((uint64_t)D, threads, N <= kSmemHistMax ? 152 * 2 : 152 * 8);
  k_item_count<<<grid, threads, smem, st>>>(off, items, D, N, cnt, flags);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bitmap_build(const uint32_t* off, const uint32_t* items, uint32_t D, const int32_t* item_rank,
                                uint32_t* bits, uint32_t stride, cudaStream_t st) {
  const uint32_t threads = 256;
  k_bitmap_build<<<grid_for(D, threads), threads, 0, st>>>(off, items, D, item_rank, bits, stride);  // 32 tx per warp
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sample_build(const uint32_t* off, const uint32_t* items, uint32_t D, const int32_t* item_rank,
                                uint64_t seed, uint32_t m, uint32_t* sbits, uint32_t sstride, cudaStream_t st) {
  const uint32_t threads = 256;
  k_sample_build<<<grid_for(m, threads), threads, 0, st>>>(off, items, D, item_rank, seed, m, sbits, sstride);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_iota(uint32_t* out, uint32_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_iota<<<grid_for(n, 256), 256, 0, st>>>(out, n);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_est_order(const unsigned long long* per, const uint32_t* ssupp, uint32_t minsup_s,
                             bool intersections, uint32_t R, unsigned long long* tally, uint32_t* order,
                             cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  if (R > kEstDeviceRows) return cudaErrorInvalidValue;
  k_est_order<<<(R + 7) / 8, 256, 0, st>>>(per, ssupp, minsup_s, intersections ? 1u : 0u, R, tally, order);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_order_suffix(const uint32_t* order, uint32_t R, uint32_t r0, uint32_t* out, cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  if (R > kEstDeviceRows) return cudaErrorInvalidValue;
  k_order_suffix<<<1, 1024, 0, st>>>(order, R, r0, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_row_popcount(const uint32_t* bits, uint32_t stride, uint32_t n_rows, uint32_t* supp,
                                cudaStream_t st) {
  if (n_rows == 0) return cudaSuccess;
  k_row_popcount<<<n_rows, 256, 0, st>>>(bits, stride, supp);
  note_launch();
  return cudaGetLastError();
}

}  // namespace fim
