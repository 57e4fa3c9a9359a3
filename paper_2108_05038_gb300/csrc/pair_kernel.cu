// K5: level-2 supports of all pairs of frequent items by bitmap AND + popcount.
//
// supp({a,b}) = |t({a}) n t({b})| (App. B.3.1; Lemma and Corollary of Sec. 2.4)
// for every pair of frequent rows i < j, i.e. the first DFS step of Eclat
// (App. B.3.2) for all one-item prefix classes [i | {j > i}] at once.  The
// n1 x n1 block of pair counts is a dense contraction over the transaction
// bits, so it is tiled like a GEMM: a CTA of 128 threads owns a 64 x 64 tile
// of (i, j) pairs (upper triangle only), stages 32-word slices of the 64 + 64
// rows in shared memory with cp.async (3-stage pipeline), and every thread
// accumulates an 8 x 4 micro-tile.  Each staged word is reused by 64 pairs, so
// the kernel is bound by the integer pipes (AND and the adders on the integer
// pipe, POPC on the XU pipe), not by memory.  Rows are split along the word
// axis into (tile, word range) work items that a grid of resident CTAs walks
// through (partial counts added atomically), which keeps every SM busy until
// the last wave.
#include <algorithm>
#include <mutex>

#include "fim_internal.cuh"

namespace fim {
namespace {

constexpr int kTile = 64;      // rows per tile side
constexpr int kChunk = 32;     // words staged per row per pipeline stage
constexpr int kRowPad = 36;    // padded shared-memory row (words): conflict-free 16-byte loads
constexpr int kStages = 3;
constexpr int kThreads = 128;
constexpr int kMX = 8, kMY = 4;                      // micro-tile: A rows x B rows per thread
constexpr int kTY = kTile / kMX, kTX = kTile / kMY;  // 8 x 16 threads
constexpr int kCopyRows = kThreads / 8;              // tile rows per copy pass (8 x 16 B per row slice)
constexpr int kPasses = kTile / kCopyRows;           // copy passes per operand
constexpr size_t kSmemBytes = (size_t)kStages * 2 * kTile * kRowPad * sizeof(uint32_t);
static_assert(kTY * kTX == kThreads && kPasses * kCopyRows == kTile, "thread layout");

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src, uint32_t src_bytes) {
  uint32_t s = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem_src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void madd(uint32_t& acc, uint32_t p, uint32_t w) {
  asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(acc) : "r"(p), "r"(w));
}

// acc += sum over 8 words of popc(a_k & b_k).  POPC issues on the XU pipe (32
// lanes/clk/SM, half the integer pipe) and limits the plain form.  A tree of
// 3:2 carry-save adders (two LOP3 each, integer pipe) compresses seven of the
// eight AND words into bit-planes of weight 1, 2 and 4:
//   (t0,t1,t2) -> s1 + 2 c1,  (t3,t4,t5) -> s2 + 2 c2,  (s1,s2,t6) -> s + 2 c3,
//   (c1,c2,c3) -> tw + 2 f,   so  t0 + .. + t6 = s + 2 tw + 4 f  (bitwise counts),
// and popc(s) + 2 popc(tw) + 4 popc(f) + popc(t7) is the sum: four POPC per
// eight words.  The weighted adds are multiply-adds by runtime constants (FMA pipe).
__device__ __forceinline__ void acc_and_popc8(uint32_t& acc, const uint4& a0, const uint4& a1, const uint4& b0,
                                              const uint4& b1, uint32_t one, uint32_t two, uint32_t four) {
  const uint32_t t0 = a0.x & b0.x, t1 = a0.y & b0.y, t2 = a0.z & b0.z, t3 = a0.w & b0.w;
  const uint32_t t4 = a1.x & b1.x, t5 = a1.y & b1.y, t6 = a1.z & b1.z, t7 = a1.w & b1.w;
  const uint32_t s1 = t0 ^ t1 ^ t2, c1 = (t0 & t1) | (t2 & (t0 ^ t1));
  const uint32_t s2 = t3 ^ t4 ^ t5, c2 = (t3 & t4) | (t5 & (t3 ^ t4));
  const uint32_t s = s1 ^ s2 ^ t6, c3 = (s1 & s2) | (t6 & (s1 ^ s2));
  const uint32_t tw = c1 ^ c2 ^ c3, f = (c1 & c2) | (c3 & (c1 ^ c2));
  madd(acc, __popc(f), four);
  madd(acc, __popc(tw), two);
  madd(acc, __popc(s), one);
  madd(acc, __popc(t7), one);
}

__global__ void __launch_bounds__(kThreads, 3)
k_pair_counts(const uint32_t* __restrict__ bits, uint32_t stride, const uint32_t* __restrict__ frows, uint32_t n1,
              uint32_t nb, uint32_t chunks_per_split, uint32_t nchunks, uint32_t* __restrict__ C2, uint32_t ksplit,
              uint32_t n_items, uint32_t one) {
  extern __shared__ __align__(16) uint32_t sm[];
  const uint32_t tid = threadIdx.x, ty = tid / kTX, tx = tid % kTX;
  const uint32_t two = one + one, four = two + two;
  // persistent loop over work items (tile, word range); consecutive items share a tile
  for (uint32_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    uint32_t t = item / ksplit, bi = 0;
    const uint32_t split = item - t * ksplit;
    while (t >= nb - bi) { t -= nb - bi; ++bi; }
    const uint32_t bj = bi + t;
    const uint32_t i0 = bi * kTile, j0 = bj * kTile;
    const uint32_t c_begin = split * chunks_per_split;
    const uint32_t c_end = min(nchunks, c_begin + chunks_per_split);
    if (c_begin >= c_end) continue;

    // 2 x kPasses 16-byte copies per thread and stage: copy q moves vector (tid & 7) of tile row
    // (tid >> 3) + kCopyRows * (q % kPasses) of A (q < kPasses) or B; rows past n1 are zero-filled
    const uint32_t lr = tid >> 3, lc = tid & 7;
    uint32_t rowid[2 * kPasses];
    uint32_t okmask = 0;
#pragma unroll
    for (int q = 0; q < 2 * kPasses; ++q) {
      const uint32_t g = (q < kPasses ? i0 : j0) + lr + kCopyRows * (q % kPasses);
      const bool ok = g < n1;
      okmask |= (ok ? 1u : 0u) << q;
      rowid[q] = frows[ok ? g : 0];
    }
    auto load_stage = [&](uint32_t stage, uint32_t chunk) {
      uint32_t* base = sm + stage * (2 * kTile * kRowPad);
#pragma unroll
      for (int q = 0; q < 2 * kPasses; ++q) {
        const uint32_t dst = ((q / kPasses) * kTile + lr + kCopyRows * (q % kPasses)) * kRowPad + lc * 4;
        const uint32_t* src = bits + (size_t)rowid[q] * stride + (size_t)chunk * kChunk + lc * 4;
        cp_async16(base + dst, src, (okmask >> q) & 1u ? 16u : 0u);
      }
    };

    uint32_t acc[kMX][kMY];
#pragma unroll
    for (int x = 0; x < kMX; ++x)
#pragma unroll
      for (int y = 0; y < kMY; ++y) acc[x][y] = 0;

#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
      if (c_begin + s < c_end) load_stage(s, c_begin + s);
      cp_async_commit();
    }
    uint32_t stage = 0;
    for (uint32_t c = c_begin; c < c_end; ++c) {
      cp_async_wait<kStages - 2>();
      __syncthreads();
      {
        const uint32_t nc = c + kStages - 1;
        uint32_t ns = stage + kStages - 1;
        if (ns >= kStages) ns -= kStages;
        if (nc < c_end) load_stage(ns, nc);
        cp_async_commit();
      }
      const uint32_t* As = sm + stage * (2 * kTile * kRowPad);
      const uint32_t* Bs = As + kTile * kRowPad;
#pragma unroll 1
      for (int kk = 0; kk < kChunk / 8; ++kk) {
        uint4 b0[kMY], b1[kMY];
#pragma unroll
        for (int y = 0; y < kMY; ++y) {
          b0[y] = *reinterpret_cast<const uint4*>(Bs + (tx + kTX * y) * kRowPad + kk * 8);
          b1[y] = *reinterpret_cast<const uint4*>(Bs + (tx + kTX * y) * kRowPad + kk * 8 + 4);
        }
#pragma unroll
        for (int x = 0; x < kMX; ++x) {
          const uint4 a0 = *reinterpret_cast<const uint4*>(As + (ty + kTY * x) * kRowPad + kk * 8);
          const uint4 a1 = *reinterpret_cast<const uint4*>(As + (ty + kTY * x) * kRowPad + kk * 8 + 4);
#pragma unroll
          for (int y = 0; y < kMY; ++y) acc_and_popc8(acc[x][y], a0, a1, b0[y], b1[y], one, two, four);
        }
      }
      stage = stage + 1 == kStages ? 0 : stage + 1;
    }
    cp_async_wait<0>();
    __syncthreads();  // the next item refills the stages

#pragma unroll
    for (int x = 0; x < kMX; ++x)
#pragma unroll
      for (int y = 0; y < kMY; ++y) {
        const uint32_t i = i0 + ty + kTY * x, j = j0 + tx + kTX * y;
        if (i < j && j < n1) {
          if (ksplit > 1) atomicAdd(&C2[(size_t)i * n1 + j], acc[x][y]);
          else C2[(size_t)i * n1 + j] = acc[x][y];
        }
      }
  }
}

}  // namespace

double pair_cores_cost_us(uint32_t n1, uint32_t stride, int num_sms) {
  // word pairs at the measured ~5.6 Tword/s on 152 SMs (sparse_mid 0.272 ms, large_sparse 34.9 ms)
  const double wp = (double)n1 * (n1 - 1) / 2.0 * stride;
  return wp / (5.6e12 * num_sms / 152.0) * 1e6 + 3.0;
}

cudaError_t launch_pair_counts(const PairLaunch& p, int num_sms, cudaStream_t st, uint32_t* ksplit_used) {
  if (p.n1 < 2) { *ksplit_used = 0; return cudaSuccess; }
  cudaError_t attr_err = kernel_smem_limit(reinterpret_cast<const void*>(k_pair_counts), (int)kSmemBytes);
  if (attr_err != cudaSuccess) return attr_err;
  static std::once_flag once;  // resident CTAs per SM: the same on every GB300 of the process
  static int occ = 0;
  std::call_once(once, [] {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_counts, kThreads, kSmemBytes) != cudaSuccess ||
        occ < 1)
      occ = 1;
  });
  const uint32_t nb = (p.n1 + kTile - 1) / kTile;
  const uint32_t tiles = nb * (nb + 1) / 2;
  const uint32_t nchunks = p.stride / kChunk;  // stride is a multiple of 32 words
  const uint32_t slots = (uint32_t)num_sms * (uint32_t)occ;  // resident CTAs
  uint32_t ksplit = p.ksplit;
  if (ksplit == 0) {
    // Items are taken round-robin by the resident CTAs, so the kernel takes about (rounds of items
    // per CTA) x (chunks per item): choose the split of the word range that minimises it, with a
    // 1% charge per split for the atomic partial sums (sparse_mid: 10 splits 0.278 ms, 11 splits
    // 0.299 ms, whose last round leaves most CTAs idle)
    double best = 1e300;
    ksplit = 1;
    for (uint32_t ks = 1; ks <= std::min<uint32_t>(64, nchunks); ++ks) {
      const uint32_t c = (nchunks + ks - 1) / ks;
      if (c < 4 && ks > 1) break;  // at least 4 chunks (128 words) per item to repay its prologue and epilogue
      const uint32_t k2 = (nchunks + c - 1) / c;
      const uint64_t items = (uint64_t)tiles * k2;
      const uint64_t rounds = (items + slots - 1) / slots;
      const double cost = (double)rounds * c * (1.0 + 0.01 * k2);
      if (cost < best - 1e-9) {
        best = cost;
        ksplit = k2;
      }
    }
  }
  uint32_t cps = (nchunks + ksplit - 1) / ksplit;
  ksplit = (nchunks + cps - 1) / cps;
  *ksplit_used = ksplit;
  if (ksplit > 1) {
    cudaError_t e = cudaMemsetAsync(p.C2, 0, (size_t)p.n1 * p.n1 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
  }
  const uint32_t n_items = tiles * ksplit;
  const uint32_t grid = n_items < slots ? n_items : slots;
  k_pair_counts<<<grid, kThreads, kSmemBytes, st>>>(p.bits, p.stride, p.frows, p.n1, nb, cps, nchunks, p.C2, ksplit,
                                                     n_items, 1u);
  note_launch();
  return cudaGetLastError();
}

}  // namespace fim
