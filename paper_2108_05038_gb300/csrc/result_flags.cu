// Closed and maximal frequent itemsets of a complete mining result (Ch. 2: Def.
// "Closed itemset" with its closure operator, Def. "Maximal Frequent Itemset").
//
// An itemset X is closed iff no item e outside X lies in every transaction that
// contains X, i.e. iff supp(X u {e}) < supp(X) for every e; it is maximal iff no
// proper superset is frequent.  If some superset Z of X has supp(Z) = supp(X)
// (or is frequent), so does every Y with X c Y c Z, in particular one with one
// item more, and that Y is frequent, hence in a complete result.  So both flags
// are decided by the result's own immediate supersets: every itemset Y of
// length k >= 2 looks up its k subsets of length k - 1 in a hash table of the
// result and marks a found subset "not maximal", and "not closed" when the
// supports are equal.
#include <algorithm>
#include <cstring>

#include "fim_internal.cuh"

namespace fim {
namespace {

constexpr uint32_t kEmpty = 0xffffffffu;
constexpr uint8_t kNotClosed = 1, kNotMaximal = 2;

// order-dependent hash of a sorted itemset, skipping position `skip` (>= len: none)
__device__ __forceinline__ uint64_t set_hash(const uint32_t* s, uint32_t len, uint32_t skip) {
  uint64_t h = 0x243f6a8885a308d3ull ^ (uint64_t)(len - (skip < len ? 1u : 0u));
  for (uint32_t q = 0; q < len; ++q) {
    if (q == skip) continue;
    h ^= s[q];
    h *= 0x9e3779b97f4a7c15ull;
    h ^= h >> 29;
  }
  h *= 0xbf58476d1ce4e5b9ull;
  return h ^ (h >> 32);
}

__global__ void k_flags_insert(const uint64_t* __restrict__ off, const uint32_t* __restrict__ items, uint64_t n,
                               uint32_t* __restrict__ table, uint64_t mask) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = off[i];
    const uint32_t len = (uint32_t)(off[i + 1] - b);
    uint64_t slot = set_hash(items + b, len, len) & mask;
    // linear probing; the table holds at least twice as many slots as itemsets, so a free slot is
    // met within mask + 1 probes
    for (uint64_t probe = 0; probe <= mask; ++probe, slot = (slot + 1) & mask)
      if (atomicCAS(&table[slot], kEmpty, (uint32_t)i) == kEmpty) break;
  }
}

__global__ void k_flags_probe(const uint64_t* __restrict__ off, const uint32_t* __restrict__ items,
                              const uint32_t* __restrict__ supp, uint64_t n, const uint32_t* __restrict__ table,
                              uint64_t mask, uint8_t* __restrict__ flags) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = off[i];
    const uint32_t len = (uint32_t)(off[i + 1] - b);
    if (len < 2) continue;
    const uint32_t* y = items + b;
    for (uint32_t p = 0; p < len; ++p) {  // the subset Y without its p-th item
      uint64_t slot = set_hash(y, len, p) & mask;
      for (uint64_t probe = 0; probe <= mask; ++probe) {
        const uint32_t j = table[slot];
        if (j == kEmpty) break;  // every result itemset was inserted: a subset that is not found is absent
        const uint64_t bj = off[j];
        if (off[j + 1] - bj == len - 1) {
          bool same = true;
          for (uint32_t q = 0, r = 0; q < len && same; ++q) {
            if (q == p) continue;
            same = items[bj + r] == y[q];
            ++r;
          }
          if (same) {
            atomicOr(reinterpret_cast<unsigned int*>(flags + (j & ~3ull)),
                     (unsigned int)(kNotMaximal | (supp[j] == supp[i] ? kNotClosed : 0)) << (8 * (j & 3)));
            break;
          }
        }
        slot = (slot + 1) & mask;
      }
    }
  }
}

// bit 0 = closed, bit 1 = maximal, from the "not" bits
__global__ void k_flags_finish(uint8_t* flags, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    flags[i] = (uint8_t)(~flags[i] & 3u);
}

// Compaction of the itemsets whose flag has a `keep` bit: per block of kFiltPer itemsets the kept sets and
// their items are counted, the block sums are scanned in one CTA, and each block writes its kept itemsets
// (in record order) at its offsets.
constexpr uint32_t kFiltThreads = 256;
constexpr uint32_t kFiltPer = 1024;  // itemsets per block (4 per thread)

__device__ __forceinline__ void block_scan2(uint64_t a, uint64_t b, uint64_t* sa, uint64_t* sb, uint64_t* ea,
                                            uint64_t* eb, uint64_t* ta, uint64_t* tb) {
  // exclusive scans of two values over the block (sa, sb: 33 shared slots each)
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint64_t x = a, y = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_up_sync(0xffffffffu, x, o), v = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= (uint32_t)o) { x += u; y += v; }
  }
  if (lane == 31) { sa[warp] = x; sb[warp] = y; }
  __syncthreads();
  if (warp == 0) {
    const uint64_t u = lane < nw ? sa[lane] : 0ull, v = lane < nw ? sb[lane] : 0ull;
    uint64_t ui = u, vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t p = __shfl_up_sync(0xffffffffu, ui, o), q = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= (uint32_t)o) { ui += p; vi += q; }
    }
    if (lane < nw) { sa[lane] = ui - u; sb[lane] = vi - v; }
    if (lane == 31) { sa[32] = ui; sb[32] = vi; }
  }
  __syncthreads();
  *ea = sa[warp] + x - a;
  *eb = sb[warp] + y - b;
  *ta = sa[32];
  *tb = sb[32];
}

__global__ void __launch_bounds__(kFiltThreads) k_keep_count(const uint64_t* __restrict__ off, uint64_t n,
                                                             const uint8_t* __restrict__ flags, uint8_t keep,
                                                             uint64_t* __restrict__ bsum) {
  __shared__ uint64_t sa[33], sb[33];
  const uint64_t b0 = (uint64_t)blockIdx.x * kFiltPer;
  uint64_t cs = 0, ci = 0;
  for (uint32_t u = 0; u < kFiltPer / kFiltThreads; ++u) {
    const uint64_t i = b0 + (uint64_t)threadIdx.x * (kFiltPer / kFiltThreads) + u;
    if (i < n && (flags[i] & keep)) {
      ++cs;
      ci += off[i + 1] - off[i];
    }
  }
  uint64_t es, ei, ts, ti;
  block_scan2(cs, ci, sa, sb, &es, &ei, &ts, &ti);
  if (threadIdx.x == 0) {
    bsum[2 * blockIdx.x] = ts;
    bsum[2 * blockIdx.x + 1] = ti;
  }
}

// one CTA: exclusive scan of the blocks' (sets, items) in place; the totals after the last block
__global__ void k_keep_scan(uint64_t* bsum, uint32_t nb) {
  __shared__ uint64_t sa[33], sb[33];
  __shared__ uint64_t carry_s, carry_i;
  if (threadIdx.x == 0) carry_s = carry_i = 0;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    const uint32_t b = b0 + threadIdx.x;
    const uint64_t s = b < nb ? bsum[2 * b] : 0ull, it = b < nb ? bsum[2 * b + 1] : 0ull;
    uint64_t es, ei, ts, ti;
    block_scan2(s, it, sa, sb, &es, &ei, &ts, &ti);
    if (b < nb) {
      bsum[2 * b] = carry_s + es;
      bsum[2 * b + 1] = carry_i + ei;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_s += ts;
      carry_i += ti;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bsum[2 * nb] = carry_s;
    bsum[2 * nb + 1] = carry_i;
  }
}

__global__ void __launch_bounds__(kFiltThreads) k_keep_scatter(const uint64_t* __restrict__ off,
                                                               const uint32_t* __restrict__ items,
                                                               const uint32_t* __restrict__ supp, uint64_t n,
                                                               const uint8_t* __restrict__ flags, uint8_t keep,
                                                               const uint64_t* __restrict__ bsum,
                                                               uint64_t* __restrict__ off2, uint32_t* __restrict__ items2,
                                                               uint32_t* __restrict__ supp2) {
  __shared__ uint64_t sa[33], sb[33];
  const uint64_t b0 = (uint64_t)blockIdx.x * kFiltPer;
  constexpr uint32_t E = kFiltPer / kFiltThreads;
  uint64_t cs = 0, ci = 0;
  for (uint32_t u = 0; u < E; ++u) {
    const uint64_t i = b0 + (uint64_t)threadIdx.x * E + u;
    if (i < n && (flags[i] & keep)) {
      ++cs;
      ci += off[i + 1] - off[i];
    }
  }
  uint64_t es, ei, ts, ti;
  block_scan2(cs, ci, sa, sb, &es, &ei, &ts, &ti);
  uint64_t rs = bsum[2 * blockIdx.x] + es, ri = bsum[2 * blockIdx.x + 1] + ei;
  for (uint32_t u = 0; u < E; ++u) {
    const uint64_t i = b0 + (uint64_t)threadIdx.x * E + u;
    if (i < n && (flags[i] & keep)) {
      const uint64_t a = off[i], len = off[i + 1] - a;
      off2[rs] = ri;
      supp2[rs] = supp[i];
      for (uint64_t q = 0; q < len; ++q) items2[ri + q] = items[a + q];
      ++rs;
      ri += len;
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) off2[bsum[2 * gridDim.x]] = bsum[2 * gridDim.x + 1];
}

// flags (bit 0 closed, bit 1 maximal) of n itemsets in device CSR form, into d_flags (n bytes rounded up
// to 4); table: 2^k >= 2n words of scratch
cudaError_t flags_of(const uint64_t* d_off, const uint32_t* d_items, const uint32_t* d_supp, uint64_t n,
                     uint32_t* table, uint64_t cap, uint8_t* flags, int sms, cudaStream_t st) {
  const uint64_t flag_bytes = (n + 3) & ~3ull;
  const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)std::max(1, sms) * 16);
  cudaError_t e = cudaMemsetAsync(table, 0xff, cap * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, flag_bytes, st);
  if (e != cudaSuccess) return e;
  k_flags_insert<<<grid, 256, 0, st>>>(d_off, d_items, n, table, cap - 1);
  note_launch();
  k_flags_probe<<<grid, 256, 0, st>>>(d_off, d_items, d_supp, n, table, cap - 1, flags);
  note_launch();
  k_flags_finish<<<grid, 256, 0, st>>>(flags, n);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

fim_status filter_output(Workspace& ws, cudaStream_t st, uint8_t keep, EngineOutput* eo, int num_sms) {
  const uint64_t n = eo->n_sets;
  if (n == 0) return FIM_OK;
  if (n >= kEmpty) return fail(FIM_ERR_INVALID, "more than 2^32 - 2 itemsets");
  uint64_t cap = 1;
  while (cap < 2 * n) cap <<= 1;  // load factor at most 1/2
  uint32_t* table = nullptr;
  FIM_TRY(ws_get(ws, WS_FILT_TABLE, cap + (n + 3) / 4 + 1, &table));
  uint8_t* flags = reinterpret_cast<uint8_t*>(table + cap);
  FIM_CUDA(flags_of(eo->d_off, eo->d_items, eo->d_supp, n, table, cap, flags, num_sms, st));
  const uint32_t nb = (uint32_t)((n + kFiltPer - 1) / kFiltPer);
  uint64_t* bsum = nullptr;
  FIM_TRY(ws_get(ws, WS_FILT_SCAN, 2ull * nb + 2, &bsum));
  k_keep_count<<<nb, kFiltThreads, 0, st>>>(eo->d_off, n, flags, keep, bsum);
  note_launch();
  k_keep_scan<<<1, 1024, 0, st>>>(bsum, nb);
  note_launch();
  FIM_CUDA(cudaGetLastError());
  // the kept totals (one round trip), then buffers of their size
  uint64_t tot[2] = {0, 0};
  FIM_CUDA(cudaMemcpyAsync(tot, bsum + 2 * nb, sizeof(tot), cudaMemcpyDeviceToHost, st));
  FIM_CUDA(cudaStreamSynchronize(st));
  uint64_t* off2 = nullptr;
  uint32_t *items2 = nullptr, *supp2 = nullptr;
  FIM_TRY(ws_get(ws, WS_FILT_OFF, tot[0] + 1, &off2));
  FIM_TRY(ws_get(ws, WS_FILT_ITEMS, std::max<uint64_t>(1, tot[1]), &items2));
  FIM_TRY(ws_get(ws, WS_FILT_SUPP, std::max<uint64_t>(1, tot[0]), &supp2));
  k_keep_scatter<<<nb, kFiltThreads, 0, st>>>(eo->d_off, eo->d_items, eo->d_supp, n, flags, keep, bsum, off2, items2,
                                              supp2);
  note_launch();
  FIM_CUDA(cudaGetLastError());
  eo->n_sets = tot[0];
  eo->n_items = tot[1];
  eo->d_off = off2;
  eo->d_items = items2;
  eo->d_supp = supp2;
  return FIM_OK;
}

}  // namespace fim

using namespace fim;

extern "C" {

fim_status fim_result_flags(const fim_result* res, uint8_t* flags_out) {
  if (!res || !flags_out) return fail(FIM_ERR_INVALID, "result or flags_out is NULL");
  const uint64_t n = res->n_sets;
  if (n == 0) return FIM_OK;
  if (n >= kEmpty) return fail(FIM_ERR_INVALID, "more than 2^32 - 2 itemsets");
  cudaStream_t st = res->stream;
  const uint64_t n_items = res->n_items;
  // device copies of a host result
  const uint64_t* d_off = res->d_off;
  const uint32_t* d_items = res->d_items;
  const uint32_t* d_supp = res->d_supp;
  void* tmp_csr = nullptr;
  const uint64_t b_off = (n + 1) * 8, b_items = (std::max<uint64_t>(1, n_items) * 4 + 15) & ~15ull, b_supp = n * 4;
  if (!res->on_device) {
    FIM_CUDA(dev_malloc_async(&tmp_csr, ((b_off + 15) & ~15ull) + b_items + b_supp, st));
    uint8_t* base = static_cast<uint8_t*>(tmp_csr);
    uint64_t* o = reinterpret_cast<uint64_t*>(base);
    uint32_t* it = reinterpret_cast<uint32_t*>(base + ((b_off + 15) & ~15ull));
    uint32_t* sp = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(it) + b_items);
    FIM_CUDA(cudaMemcpyAsync(o, res->h_off, b_off, cudaMemcpyHostToDevice, st));
    if (n_items) FIM_CUDA(cudaMemcpyAsync(it, res->h_items, n_items * 4, cudaMemcpyHostToDevice, st));
    FIM_CUDA(cudaMemcpyAsync(sp, res->h_supp, b_supp, cudaMemcpyHostToDevice, st));
    d_off = o;
    d_items = it;
    d_supp = sp;
  }
  uint64_t cap = 1;
  while (cap < 2 * n) cap <<= 1;  // load factor at most 1/2
  void* scratch = nullptr;
  const uint64_t flag_bytes = (n + 3) & ~3ull;
  cudaError_t e = dev_malloc_async(&scratch, cap * 4 + flag_bytes, st);
  if (e != cudaSuccess) {
    if (tmp_csr) cudaFreeAsync(tmp_csr, st);
    return cuda_fail(e, "result flags scratch");
  }
  uint32_t* table = static_cast<uint32_t*>(scratch);
  uint8_t* flags = reinterpret_cast<uint8_t*>(table + cap);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = flags_of(d_off, d_items, d_supp, n, table, cap, flags, sms, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(flags_out, flags, n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(scratch, st);
  if (tmp_csr) cudaFreeAsync(tmp_csr, st);
  if (e != cudaSuccess) return cuda_fail(e, "result flags");
  return FIM_OK;
}

}  // extern "C"
