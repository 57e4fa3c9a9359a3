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

}  // namespace
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
    FIM_CUDA(cudaMemcpyAsync(o, res->h_off.data(), b_off, cudaMemcpyHostToDevice, st));
    if (n_items) FIM_CUDA(cudaMemcpyAsync(it, res->h_items.data(), n_items * 4, cudaMemcpyHostToDevice, st));
    FIM_CUDA(cudaMemcpyAsync(sp, res->h_supp.data(), b_supp, cudaMemcpyHostToDevice, st));
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
  const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)std::max(1, sms) * 16);
  if ((e = cudaMemsetAsync(table, 0xff, cap * 4, st)) == cudaSuccess &&
      (e = cudaMemsetAsync(flags, 0, flag_bytes, st)) == cudaSuccess) {
    k_flags_insert<<<grid, 256, 0, st>>>(d_off, d_items, n, table, cap - 1);
    note_launch();
    k_flags_probe<<<grid, 256, 0, st>>>(d_off, d_items, d_supp, n, table, cap - 1, flags);
    note_launch();
    k_flags_finish<<<grid, 256, 0, st>>>(flags, n);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(flags_out, flags, n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(scratch, st);
  if (tmp_csr) cudaFreeAsync(tmp_csr, st);
  if (e != cudaSuccess) return cuda_fail(e, "result flags");
  return FIM_OK;
}

}  // extern "C"
