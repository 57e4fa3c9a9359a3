// Supports of the one-item extensions of an itemset: the AND + popcount step of
// a class node (App. B.3.2, Eclat-DFS-Computation: |t(P u {a_j})| from t(P) and
// t({a_j})) as a standalone query.  t(P) is the AND of the rows of P's items
// (one row: used in place); every candidate row is streamed once against it, read
// only under nonzero words of t(P).  With a dense t(P) this is a pure stream of
// the candidate rows, the bandwidth-bound form of the DFS's counting step.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fim_internal.cuh"

namespace fim {
namespace {

__device__ __forceinline__ bool nz4(const uint4& v) { return (v.x | v.y | v.z | v.w) != 0u; }

// dst[w] = AND of rows[0..n) at word w
__global__ void k_and_rows(const uint4* __restrict__ bits4, uint32_t stride4, const uint32_t* __restrict__ rows,
                           uint32_t n, uint4* __restrict__ dst) {
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < stride4; w += gridDim.x * blockDim.x) {
    uint4 a = __ldg(bits4 + (size_t)rows[0] * stride4 + w);
    for (uint32_t k = 1; k < n && nz4(a); ++k) {
      const uint4 b = __ldg(bits4 + (size_t)rows[k] * stride4 + w);
      a = make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
    }
    dst[w] = a;
  }
}

// out[c] = popc(pre & row(cand[c])); one CTA per candidate at a time, eight 16-byte loads per thread
// in flight; a candidate whose row is absent (kNoRow) has no common transaction with anything
constexpr uint32_t kNoRow = 0xffffffffu;
__global__ void __launch_bounds__(256) k_extension_counts(const uint4* __restrict__ bits4, uint32_t stride4,
                                                          const uint4* pre4, const uint32_t* __restrict__ cand,
                                                          uint32_t n_cand, uint32_t* __restrict__ out) {
  __shared__ uint32_t wsum[8];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t c = blockIdx.x; c < n_cand; c += gridDim.x) {
    const uint32_t row = cand[c];
    uint32_t s = 0;
    if (row != kNoRow) {
      const uint4* r4 = bits4 + (size_t)row * stride4;
      constexpr uint32_t U = 8;
      for (uint32_t w0 = threadIdx.x; w0 < stride4; w0 += U * blockDim.x) {
        uint4 a[U], b[U];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) {
          const uint32_t w = w0 + u * blockDim.x;
          a[u] = w < stride4 ? pre4[w] : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) b[u] = nz4(a[u]) ? __ldcs(r4 + w0 + u * blockDim.x) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (uint32_t u = 0; u < U; ++u)
          s += __popc(a[u].x & b[u].x) + __popc(a[u].y & b[u].y) + __popc(a[u].z & b[u].z) + __popc(a[u].w & b[u].w);
      }
    }
    s = __reduce_add_sync(0xffffffffu, s);
    if (lane == 0) wsum[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (uint32_t k = 0; k < (blockDim.x >> 5); ++k) t += wsum[k];
      out[c] = t;
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace fim

using namespace fim;

extern "C" {

fim_status fim_extension_supports(fim_db* db, const uint32_t* prefix_items, uint32_t n_prefix,
                                  const uint32_t* cand_items, uint32_t n_cand, uint32_t* supports_out) {
  if (!db) return fail(FIM_ERR_INVALID, "db is NULL");
  if (n_prefix == 0 || !prefix_items) return fail(FIM_ERR_INVALID, "the prefix needs at least one item");
  if (n_cand == 0) return FIM_OK;
  if (!cand_items || !supports_out) return fail(FIM_ERR_INVALID, "candidates or supports_out is NULL");
  // items -> rows; an item dropped by the prefilter has no row, so its supports are unknown
  auto row_of = [&](uint32_t item, uint32_t* row) -> fim_status {
    if (item >= db->N) return fail(FIM_ERR_INVALID, "an item id is >= N");
    const int32_t r = db->item_rank[item];
    if (r < 0) return fail(FIM_ERR_INVALID, "an item was dropped by the build's prefilter");
    *row = (uint32_t)r;
    return FIM_OK;
  };
  std::vector<uint32_t> rows(n_prefix + n_cand);
  for (uint32_t k = 0; k < n_prefix; ++k) FIM_TRY(row_of(prefix_items[k], &rows[k]));
  for (uint32_t k = 0; k < n_cand; ++k) FIM_TRY(row_of(cand_items[k], &rows[n_prefix + k]));
  cudaStream_t st = db->stream;
  const uint32_t stride4 = db->stride / 4;
  const uint4* bits4 = reinterpret_cast<const uint4*>(db->d_bits);
  uint32_t* d_rows = nullptr;
  uint32_t* d_out = nullptr;
  FIM_TRY(ws_get(db->ws, WS_QUERY_ROWS, rows.size(), &d_rows));
  FIM_TRY(ws_get(db->ws, WS_QUERY_OUT, n_cand, &d_out));
  void* h = nullptr;
  FIM_TRY(stage_get(db, rows.size() * 4, &h));
  std::memcpy(h, rows.data(), rows.size() * 4);
  FIM_CUDA(cudaMemcpyAsync(d_rows, h, rows.size() * 4, cudaMemcpyHostToDevice, st));
  const uint4* pre4 = bits4 + (size_t)rows[0] * stride4;
  if (n_prefix > 1) {
    uint4* d_pre = nullptr;
    FIM_TRY(ws_get(db->ws, WS_QUERY_PREFIX, stride4, &d_pre));
    const uint32_t threads = 256;
    const uint32_t grid = std::min<uint32_t>((stride4 + threads - 1) / threads, (uint32_t)db->num_sms * 8);
    k_and_rows<<<std::max<uint32_t>(1, grid), threads, 0, st>>>(bits4, stride4, d_rows, n_prefix, d_pre);
    note_launch();
    FIM_CUDA(cudaGetLastError());
    pre4 = d_pre;
  }
  int occ = 0;
  FIM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_extension_counts, 256, 0));
  const uint32_t grid = std::min<uint32_t>(n_cand, (uint32_t)db->num_sms * (uint32_t)std::max(1, occ));
  k_extension_counts<<<grid, 256, 0, st>>>(bits4, stride4, pre4, d_rows + n_prefix, n_cand, d_out);
  note_launch();
  FIM_CUDA(cudaGetLastError());
  void* ho = nullptr;
  FIM_TRY(stage_get(db, (size_t)n_cand * 4, &ho));
  FIM_CUDA(cudaMemcpyAsync(ho, d_out, (size_t)n_cand * 4, cudaMemcpyDeviceToHost, st));
  FIM_TRY(stream_sync(db));
  std::memcpy(supports_out, ho, (size_t)n_cand * 4);
  return FIM_OK;
}

}  // extern "C"
