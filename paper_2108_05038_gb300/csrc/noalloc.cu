// fim_mine_pairs_noalloc: the frequent pairs of a built database, computed
// without allocating any memory.
//
// The ordinary path takes its scratch (the n1 x n1 pair-count block and the
// frequent-row list) from a workspace that it allocates on demand.  Callers
// that cannot allocate use this entry point instead: its scratch is one
// file-scope __device__ array of fixed size, so at most kNoAllocMaxRows
// frequent items fit.  Every GPU that loads the library keeps that array until
// the process exits.
#include <mutex>

#include "fim_internal.cuh"

namespace fim {
namespace {

constexpr uint32_t kNoAllocMaxRows = 1024;
constexpr size_t kNoAllocCountWords = (size_t)kNoAllocMaxRows * kNoAllocMaxRows;  // pair counts, 4 MiB
constexpr size_t kNoAllocRowWords = kNoAllocMaxRows;                               // frequent-row list
constexpr size_t kNoAllocWords = kNoAllocCountWords + kNoAllocRowWords + 64;       // + counter block

// The scratch.  Host code must not pass this name to a kernel: on the host it
// is only a stand-in symbol.  The device address comes from
// cudaGetSymbolAddress, taken once per device in scratch_on_device().
static __device__ __align__(256) uint32_t g_pair_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// (called with `dev` current)
fim_status scratch_on_device(int dev, uint32_t** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(FIM_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pair_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_pair_scratch)");
    g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return FIM_OK;
}

__global__ void k_rows_iota(uint32_t* frows, uint32_t r0, uint32_t n1) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += gridDim.x * blockDim.x) frows[i] = r0 + i;
}

// one CTA per row i: every j > i with count >= minsup becomes (min id, max id, count)
__global__ void k_pairs_emit(const uint32_t* __restrict__ C2, uint32_t n1, uint32_t minsup, uint32_t r0,
                             const uint32_t* __restrict__ rank_item, uint32_t* __restrict__ pairs,
                             uint32_t* __restrict__ supports, uint64_t cap, unsigned long long* counter) {
  const uint32_t i = blockIdx.x;
  const uint32_t id_i = rank_item[r0 + i];
  for (uint32_t j = i + 1 + threadIdx.x; j < n1; j += blockDim.x) {
    const uint32_t c = C2[(size_t)i * n1 + j];
    if (c < minsup) continue;
    const unsigned long long pos = atomicAdd(counter, 1ull);
    if (pos < cap) {
      const uint32_t id_j = rank_item[r0 + j];
      pairs[2 * pos] = min(id_i, id_j);
      pairs[2 * pos + 1] = max(id_i, id_j);
      supports[pos] = c;
    }
  }
}

}  // namespace
}  // namespace fim

using namespace fim;

extern "C" fim_status fim_mine_pairs_noalloc(const fim_db* db, uint32_t minsup_abs, uint32_t* d_pairs,
                                             uint32_t* d_supports, uint64_t capacity, uint64_t* n_pairs) {
  if (!db || !n_pairs) return fail(FIM_ERR_INVALID, "db or n_pairs is NULL");
  *n_pairs = 0;
  if (minsup_abs == 0) return fail(FIM_ERR_INVALID, "minsup 0 makes every pair frequent");
  if (minsup_abs < db->prefilter) return fail(FIM_ERR_INVALID, "minsup below the prefilter support of the database");
  if (capacity > 0 && (!d_pairs || !d_supports)) return fail(FIM_ERR_INVALID, "output buffers are NULL");
  // rows are sorted by ascending support: the frequent ones are a suffix
  uint32_t r0 = 0;
  while (r0 < db->n_rows && db->supp[r0] < minsup_abs) ++r0;
  const uint32_t n1 = db->n_rows - r0;
  if (n1 > kNoAllocMaxRows)
    return fail(FIM_ERR_INVALID, "fim_mine_pairs_noalloc: " + std::to_string(n1) +
                                     " frequent items exceed its fixed scratch of " +
                                     std::to_string(kNoAllocMaxRows) + " items; use fim_mine");
  if (n1 < 2) return FIM_OK;
  // the whole call runs on db's device, which is made current for it; the caller's current device
  // comes back on return
  int caller_dev = -1;
  FIM_CUDA(cudaGetDevice(&caller_dev));
  struct Restore {
    int dev, cur;
    ~Restore() {
      if (dev != cur) cudaSetDevice(dev);
    }
  } restore{caller_dev, db->device};
  if (caller_dev != db->device) FIM_CUDA(cudaSetDevice(db->device));
  uint32_t* scratch = nullptr;
  FIM_TRY(scratch_on_device(db->device, &scratch));
  uint32_t* C2 = scratch;
  uint32_t* frows = scratch + kNoAllocCountWords;
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(scratch + kNoAllocCountWords + kNoAllocRowWords);
  cudaStream_t st = db->stream;
  // the previous call's counter is still in the array: clear it
  FIM_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
  k_rows_iota<<<(n1 + 255) / 256, 256, 0, st>>>(frows, r0, n1);
  note_launch();
  FIM_CUDA(cudaGetLastError());
  uint32_t ksplit = 0;
  PairLaunch pl{db->d_bits, db->stride, frows, n1, C2, 0};
  FIM_CUDA(launch_pair_counts(pl, db->num_sms, st, &ksplit));  // clears C2 itself when it splits rows
  k_pairs_emit<<<n1, 256, 0, st>>>(C2, n1, minsup_abs, r0, db->d_rank_item, d_pairs, d_supports, capacity, counter);
  note_launch();
  FIM_CUDA(cudaGetLastError());
  unsigned long long found = 0;
  FIM_CUDA(cudaMemcpyAsync(&found, counter, sizeof(found), cudaMemcpyDeviceToHost, st));
  FIM_CUDA(cudaStreamSynchronize(st));
  *n_pairs = found;
  if (found > capacity) return fail(FIM_ERR_OUTPUT_OVERFLOW, "more frequent pairs than the output capacity");
  return FIM_OK;
}
