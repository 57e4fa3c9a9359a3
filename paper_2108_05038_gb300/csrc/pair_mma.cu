// K5 on the tensor cores: level-2 supports of all pairs of frequent rows as an
// exact integer GEMM.
//
// supp({a,b}) = |t({a}) n t({b})| (App. B.3.1) is the sum over transactions t of
// x_a(t) x_b(t) with x in {0,1}, so the n1 x n1 block of pair counts is C = X X^T
// for the 0/1 matrix X of the frequent rows (the first DFS step of Eclat,
// App. B.3.2, for all one-item classes at once).  tcgen05 has no 1-bit kind, so
// each row is widened once to bytes (bit set -> 1.0 in e4m3, else 0) and the
// product runs as kind::f8f6f4 MMAs with fp32 accumulators in tensor memory.
// Two operand forms: e4m3 (1.0 = 0x38, one byte per transaction in memory) and
// e2m1 (1.0 = 0x2, two transactions per byte in memory; the TMA spreads each 8
// packed bytes to the 16-byte unpacked form the MMA reads, so shared memory and
// MMA rate are those of e4m3 while the widened rows and their reads halve).
// Every product is 0 or 1, so a partial sum is an integer no larger than the
// bytes it covers; a work item covers at most 2^24 bytes of K, where fp32 holds
// every integer exactly, and items of one tile are added as u32 atomics.
//
// Tiles: 128 rows (i) x 256 rows (j) of X, only those that hold pairs i < j.
// A CTA (one per SM, persistent) walks (tile, K range) items with three roles:
// one thread issues TMA loads of 128-transaction K slices (128B swizzle) into a
// 4-stage ring, one thread issues four 128x256x32 MMAs per slice into one of
// two 256-column TMEM accumulators, and four warps read the other accumulator
// back (tcgen05.ld, one TMEM lane quarter per warp) through a small transposing
// staging area and write or add whole 128-byte row segments of C2 (coalesced)
// for the pairs i < j, so an item's read-back overlaps the next item's MMAs.
// Every mbarrier wait is bounded by time; on expiry the kernel sets
// DEV_ERR_TIMEOUT, lets its copies and MMAs in flight finish, frees its TMEM and
// returns.
#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder comes from the driver at run time)

#include <algorithm>
#include <mutex>

#include "fim_internal.cuh"

namespace fim {
namespace {

constexpr uint32_t kBM = 128;       // tile rows on the i side (MMA M)
constexpr uint32_t kBN = 256;       // tile rows on the j side (MMA N)
constexpr uint32_t kBK = 128;       // K bytes per pipeline stage (one 128-byte swizzle row)
constexpr uint32_t kMmaK = 32;      // K bytes per kind::f8f6f4 MMA
constexpr uint32_t kStages = 4;
// six warps: TMA issue (warp 0), MMA issue and TMEM owner (warp 1), read-back (warps 2-5, one TMEM
// lane quarter each: warp w may access lanes 32 (w mod 4) .. + 31)
constexpr uint32_t kThreads = 192;
constexpr uint32_t kABytes = kBM * kBK;
constexpr uint32_t kBBytes = kBN * kBK;
constexpr uint32_t kStageBytes = kABytes + kBBytes;
constexpr uint32_t kAccBufs = 2;                     // accumulators: one read back while the next fills
constexpr uint32_t kTmemCols = kAccBufs * kBN;       // 2 x (128 lanes x 256 fp32 columns) = all of TMEM
constexpr uint32_t kChunk = 32;                      // columns read back per round
constexpr uint32_t kSPitch = kChunk + 1;             // staging rows (words), conflict-free transposition
constexpr uint32_t kStagingBytes = 4 * 32 * kSPitch * 4;  // per read-back warp 32 rows x 33 words
// full[], empty[], acc_full[], acc_empty[], fin, TMEM address
constexpr uint32_t kBarBytes = 8 * (2 * kStages + 2 * kAccBufs + 1) + 8;
constexpr size_t kSmemBytes = 1024 + (size_t)kStages * kStageBytes + kStagingBytes + kBarBytes;  // + align slack
constexpr uint32_t kMaxStepsPerItem = (1u << 24) / kBK;      // fp32 exact: at most 2^24 bytes of K per item
constexpr uint64_t kWaitNs = 1000000000ull;                  // bound of every mbarrier wait (1 s)
// instruction descriptor of kind::f8f6f4: D f32 (bits 4-5 = 1), A and B format in bits 7-9 and 10-12
// (e4m3 = 0, e2m1 = 5), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
template <bool kE2M1>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | ((kE2M1 ? 5u : 0u) << 7) | ((kE2M1 ? 5u : 0u) << 10) | ((kBN >> 3) << 17) | ((kBM >> 4) << 24);
}
constexpr uint32_t kOneE4M3 = 0x38u;  // 1.0: exponent 7 (the bias), mantissa 0
constexpr uint32_t kOneE2M1 = 0x2u;   // 1.0: exponent 1 (the bias), mantissa 0
static_assert(kSmemBytes <= 227u * 1024u, "shared memory per CTA");
static_assert(kBN % 16 == 0 && kBN <= 256 && kBM == 128, "MMA shape of cta_group::1");
static_assert(kBK % kMmaK == 0, "whole MMAs per stage");

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// waits for the completion of the phase of parity `parity`; false when kWaitNs pass first
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  while (!mbar_try(bar, parity))
    if (now_ns() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 2-D tiled TMA load of one box into shared memory; completion counted on `bar` in bytes
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor of a K-major operand in the 128-byte swizzle layout: rows of 128
// bytes, 8-row groups 1024 bytes apart (stride byte offset), start address in 16-byte units, the
// Blackwell descriptor version 1 in bits 46-47, swizzle mode 2 (128 B) in bits 61-63
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

__device__ __forceinline__ void mma_f8f6f4(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrives on `bar` once every MMA this thread issued before has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive fp32 columns of this thread's TMEM lane (warp-wide; the load and its wait in one statement)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// X[f][32w .. 32w+31] (bytes) = the 32 bits of word w of row frows[f], each as 1.0 (e4m3) or 0
__global__ void k_expand_e4m3(const uint32_t* __restrict__ bits, uint32_t stride, const uint32_t* __restrict__ frows,
                              uint32_t n1, uint4* __restrict__ X) {
  const uint64_t total = (uint64_t)n1 * stride;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t f = (uint32_t)(idx / stride), w = (uint32_t)(idx % stride);
    const uint32_t word = __ldg(bits + (size_t)frows[f] * stride + w);
    uint32_t o[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      // bits 4q..4q+3 to the lowest bit of bytes 0..3: the four shifted copies (0, 7, 14, 21) do not
      // overlap, and bit b of copy b lands on bit 8b
      const uint32_t nib = (word >> (4 * q)) & 0xFu;
      o[q] = ((nib * 0x00204081u) & 0x01010101u) * kOneE4M3;
    }
    X[2 * idx] = make_uint4(o[0], o[1], o[2], o[3]);
    X[2 * idx + 1] = make_uint4(o[4], o[5], o[6], o[7]);
  }
}

// X[f][16w .. 16w+15] (bytes) = the 32 bits of word w of row frows[f] as 32 e2m1 values (1.0 or 0),
// transaction 2k in the low nibble of byte k.  Grid: x over the words of a row, y over the rows.
__global__ void k_expand_e2m1(const uint32_t* __restrict__ bits, uint32_t stride, const uint32_t* __restrict__ frows,
                              uint32_t n1, uint4* __restrict__ X) {
  for (uint32_t f = blockIdx.y; f < n1; f += gridDim.y) {
    const uint32_t* row = bits + (size_t)frows[f] * stride;
    uint4* xrow = X + (size_t)f * stride;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < stride; w += gridDim.x * blockDim.x) {
      const uint32_t word = __ldg(row + w);
      uint32_t o[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // the 8 bits of byte q to bit 0 of nibbles 0..7 (interleave with three zero bits), then x 2
        uint32_t t = (word >> (8 * q)) & 0xFFu;
        t = (t | (t << 12)) & 0x000F000Fu;
        t = (t | (t << 6)) & 0x03030303u;
        t = (t | (t << 3)) & 0x11111111u;
        o[q] = t * kOneE2M1;
      }
      xrow[w] = make_uint4(o[0], o[1], o[2], o[3]);
    }
  }
}

template <bool kE2M1>
__global__ void __launch_bounds__(kThreads, 1)
    k_pair_mma(const __grid_constant__ CUtensorMap xmap, uint32_t n1, uint32_t nbj, uint32_t n_tiles, uint32_t nsteps,
               uint32_t steps_per_item, uint32_t ksplit, uint32_t* __restrict__ C2, uint32_t* __restrict__ err,
               uint32_t extra_tx) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint32_t s_abort;
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // the 128-byte swizzle repeats every 1024 bytes
  const uint32_t a_st = base, b_st = base + kStages * kABytes;
  uint32_t* const staging = reinterpret_cast<uint32_t*>(smem_raw + (base + kStages * kStageBytes - raw));
  const uint32_t bars = base + kStages * kStageBytes + kStagingBytes;
  auto full = [&](uint32_t s) { return bars + 8 * s; };
  auto empty = [&](uint32_t s) { return bars + 8 * (kStages + s); };
  auto acc_full = [&](uint32_t b) { return bars + 8 * (2 * kStages + b); };
  auto acc_empty = [&](uint32_t b) { return bars + 8 * (2 * kStages + kAccBufs + b); };
  const uint32_t fin = bars + 8 * (2 * kStages + 2 * kAccBufs);
  const uint32_t tslot = fin + 8;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile uint32_t* abort_flag = &s_abort;
  auto abort_now = [&]() {
    atomicOr(err, DEV_ERR_TIMEOUT);
    *abort_flag = 1u;
  };

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < kStages; ++s) {
      mbar_init(full(s), 1);   // the producer's arrive + the TMA bytes
      mbar_init(empty(s), 1);  // the MMA commit that consumed stage s
    }
    for (uint32_t b = 0; b < kAccBufs; ++b) {
      mbar_init(acc_full(b), 1);   // the MMA commit after an item's last slice
      mbar_init(acc_empty(b), 4);  // one arrive per read-back warp
    }
    mbar_init(fin, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot), "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem_raw + (tslot - raw));

  // item -> (row block bi, column block bj, first K slice, slices); items of one K range are
  // consecutive, so the CTAs of a wave read the same K slices (L2 reuse)
  const uint32_t n_items = n_tiles * ksplit;
  auto decode = [&](uint32_t item, uint32_t& bi, uint32_t& bj, uint32_t& k0, uint32_t& ns) {
    const uint32_t split = item / n_tiles;
    uint32_t t = item % n_tiles;
    bi = 0;
    while (t >= nbj - bi / 2) {  // row block bi pairs with the column blocks bj >= bi / 2
      t -= nbj - bi / 2;
      ++bi;
    }
    bj = bi / 2 + t;
    k0 = split * steps_per_item;
    ns = min(nsteps, k0 + steps_per_item) - k0;
  };

  uint32_t issued = 0;  // producer: slices issued (ring position)
  bool mma_open = false;  // MMA thread: MMAs issued since the last commit that someone waits for
  if (warp == 0) {
    if (lane == 0) {
      for (uint32_t item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x) {
        uint32_t bi, bj, k0, ns;
        decode(item, bi, bj, k0, ns);
        for (uint32_t s = 0; s < ns; ++s, ++issued) {
          const uint32_t st = issued % kStages;
          if (issued >= kStages && !mbar_wait(empty(st), ((issued / kStages) - 1) & 1)) {
            abort_now();
            break;
          }
          // transaction bytes = bytes the TMA moves: e2m1 boxes carry 64 packed bytes per row (the gaps of
          // the unpacked shared-memory form are not written)
          // (extra_tx, a failure-detection test only: bytes that never arrive, so the wait runs out)
          mbar_expect_tx(full(st), (kE2M1 ? kStageBytes / 2 : kStageBytes) + extra_tx);
          const int32_t x = (int32_t)((k0 + s) * kBK);
          tma_load(a_st + st * kABytes, &xmap, x, (int32_t)(bi * kBM), full(st));
          tma_load(b_st + st * kBBytes, &xmap, x, (int32_t)(bj * kBN), full(st));
          tma_load(b_st + st * kBBytes + kABytes, &xmap, x, (int32_t)(bj * kBN + kBM), full(st));
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t consumed = 0, it = 0;
      for (uint32_t item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x, ++it) {
        uint32_t bi, bj, k0, ns;
        decode(item, bi, bj, k0, ns);
        const uint32_t b = it & 1;
        if (it >= kAccBufs && !mbar_wait(acc_empty(b), ((it >> 1) - 1) & 1)) {  // read back, so reusable
          abort_now();
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + b * kBN;
        bool ok = true;
        for (uint32_t s = 0; s < ns; ++s, ++consumed) {
          const uint32_t st = consumed % kStages;
          if (!mbar_wait(full(st), (consumed / kStages) & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t ad = sw128_desc(a_st + st * kABytes), bd = sw128_desc(b_st + st * kBBytes);
#pragma unroll
          for (uint32_t kk = 0; kk < kBK / kMmaK; ++kk)  // +32 bytes of K inside the swizzled rows: +2 in 16-byte units
            mma_f8f6f4(d, ad + 2 * kk, bd + 2 * kk, idesc<kE2M1>(), (s | kk) != 0u);
          mma_commit(empty(st));  // stage st free once these MMAs are done
          mma_open = true;
        }
        if (!ok) {
          abort_now();  // flagged before the commit, so the read-back sees it once acc_full(b) completes
          mma_commit(acc_full(b));
          mma_open = true;  // nobody may wait for acc_full(b) now
          break;
        }
        mma_commit(acc_full(b));  // accumulator b complete
        mma_open = false;
      }
    }
    __syncwarp();
  } else {
    // read-back: TMEM lanes -> staging (transposed) -> 128-byte row segments of C2
    const uint32_t quarter = warp & 3;
    uint32_t* sw = staging + (warp - 2) * 32 * kSPitch;
    uint32_t it = 0;
    for (uint32_t item = blockIdx.x; item < n_items; item += gridDim.x, ++it) {
      uint32_t bi, bj, k0, ns;
      decode(item, bi, bj, k0, ns);
      const uint32_t b = it & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(acc_full(b), (it >> 1) & 1));
      if (!ok || *abort_flag) {
        if (lane == 0 && !ok) abort_now();
        break;
      }
      tc_fence_after();
      const uint32_t row0 = bi * kBM + quarter * 32;
      const uint32_t taddr = tmem + ((quarter * 32u) << 16) + b * kBN;
#pragma unroll 1
      for (uint32_t c0 = 0; c0 < kBN; c0 += kChunk) {
        uint32_t r[16];
        tmem_ld16(taddr + c0, r);
#pragma unroll
        for (uint32_t c = 0; c < 16; ++c) sw[lane * kSPitch + c] = __float2uint_rn(__uint_as_float(r[c]));
        tmem_ld16(taddr + c0 + 16, r);
#pragma unroll
        for (uint32_t c = 0; c < 16; ++c) sw[lane * kSPitch + 16 + c] = __float2uint_rn(__uint_as_float(r[c]));
        __syncwarp();
        const uint32_t j = bj * kBN + c0 + lane;
#pragma unroll 4
        for (uint32_t rr = 0; rr < 32; ++rr) {
          const uint32_t i = row0 + rr;
          if (i < j && j < n1) {  // i < j < n1 also bounds i
            const uint32_t v = sw[rr * kSPitch + lane];
            if (ksplit > 1) atomicAdd(&C2[(size_t)i * n1 + j], v);
            else C2[(size_t)i * n1 + j] = v;
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty(b));
    }
  }

  // teardown after an abort: the producer waits (bounded) for its last slices in flight, the MMA
  // thread for its MMAs that nobody waits for
  if (warp == 0 && lane == 0 && *abort_flag) {
    for (uint32_t q = issued > kStages ? issued - kStages : 0; q < issued; ++q)
      (void)mbar_wait(full(q % kStages), (q / kStages) & 1);
  }
  if (warp == 1 && lane == 0 && (mma_open || *abort_flag)) {
    mma_commit(fin);
    (void)mbar_wait(fin, 0);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                              : "memory");
}

// ---- the widening fused into the product ----------------------------------------------------------------
// Tiles of 256 x 256 rows: two M 128 MMAs per K step share the B operand, and the two accumulators fill all
// of TMEM (512 columns), so a tile's read-back runs between its item and the next one while the expanders
// already fill the next item's stages.  Per 128-transaction slice the TMA brings the raw bits (16 bytes per
// row, 512 rows: 8 KB) into a ring of three stages; 24 expander warps in three groups, which take the
// slices in turn, turn a raw stage into the e4m3 operand stage (64 KB: 256 A rows, then 256 B rows, in
// the 128-byte swizzle layout the MMA descriptors read), make those generic-proxy writes visible to the
// tensor cores (fence.proxy.async) and arrive on the stage's barrier.  No widened copy of the rows exists,
// so the DRAM traffic is that of the raw bits, and per flop the expansion is two thirds of that of a
// 128 x 256 tile (512 rows per two MMA steps instead of 384 per one).
// A set bit becomes 2.0 (0x40, one bit of its byte); every product is then 4, a partial sum is 4 x an
// integer of at most 2^24 (exact in fp32: multiples of 4 up to 2^26), and the read-back divides by 4.
// The order of the transactions inside a slice is free as long as every row uses the same one: byte k of
// output word t of raw word w is bit 8k + t of w, i.e. output word t = (w << (6 - t)) & 0x40404040, one
// multiply and one mask.  The multipliers are kernel arguments, so the shifts run as integer multiplies on
// the FMA pipe and the ALU pipe, which bounds the expansion, only takes the masks.
constexpr uint32_t kFM = 256;                        // tile rows on the i side (two MMAs of M 128)
constexpr uint32_t kFN = kBN;                        // tile rows on the j side (MMA N)
constexpr uint32_t kFStages = 3;                     // operand stages (64 KB each), one per expander group
constexpr uint32_t kFStageBytes = (kFM + kFN) * kBK;
constexpr uint32_t kRStages = 3;                     // raw stages (8 KB each), one per expander group
constexpr uint32_t kRawRows = kFM + kFN;             // 512 rows per slice (A rows, then B rows)
constexpr uint32_t kRawStageBytes = kRawRows * 16;   // 4 words per row
constexpr uint32_t kExpGroups = 3;                   // groups of expander warps, slices in turn
constexpr uint32_t kGroupWarps = 8;
constexpr uint32_t kGroupThreads = kGroupWarps * 32;
constexpr uint32_t kRowsPerExp = kRawRows / kGroupThreads;  // rows of a slice per expander thread
constexpr uint32_t kExpThreads = kExpGroups * kGroupThreads;
constexpr uint32_t kFThreads = kThreads + kExpThreads;  // warps 0-5 as in the widened kernel, 6-29 expand
constexpr uint32_t kFChunk = 16;                     // columns read back per round
constexpr uint32_t kFPitch = kFChunk + 1;            // staging rows (words): conflict-free transposition
constexpr uint32_t kFStagingBytes = 4 * 32 * kFPitch * 4;
constexpr uint32_t kTwoE4M3 = 0x40u;                // 2.0: exponent 8 (bias 7), mantissa 0
// rfull[], rempty[], ofull[], oempty[], acc_full, acc_empty, fin, acc_last, TMEM address
constexpr uint32_t kFBarBytes = 8 * (2 * kRStages + 2 * kFStages + 4) + 8;
// the read-back of a CTA's last tile is shared by the read-back warp of each TMEM lane quarter and the six
// expander warps of the same quarter (their slices done, the operand stages free for their staging)
constexpr uint32_t kLastWorkers = 1 + kExpThreads / 32 / 4;
static_assert(kExpThreads / 32 % 4 == 0 && kExpThreads / 32 * 32 * kFPitch * 4 <= kFStageBytes,
              "expander warps cover the four quarters evenly; their staging fits one operand stage");
constexpr size_t kFSmemBytes =
    1024 + (size_t)kFStages * kFStageBytes + (size_t)kRStages * kRawStageBytes + kFStagingBytes + kFBarBytes;
static_assert(kFSmemBytes <= 227u * 1024u, "shared memory per CTA");
static_assert(kFThreads <= 1024 && kRawRows % kGroupThreads == 0, "whole rows per expander thread");
static_assert(kRStages == kExpGroups && kFStages == kExpGroups, "group g owns raw stage g and operand stage g");
static_assert(kBK == 128 && kFM == 2 * kBM && 2 * kBN == kTmemCols, "128-byte operand rows; two accumulators");

// the 32 transactions of raw word w as output words t = 0..7 (two 16-byte chunks): (w << (6 - t)) & keep,
// with mul[t] = 2^(6 - t) given at run time and t = 7 as the high half of w x 2^31 (w >> 1)
__device__ __forceinline__ void spread32_two(uint32_t w, const uint32_t (&mul)[6], uint32_t hi31, uint4& lo,
                                             uint4& hi) {
  constexpr uint32_t kKeep = kTwoE4M3 * 0x01010101u;
  lo = make_uint4((w * mul[0]) & kKeep, (w * mul[1]) & kKeep, (w * mul[2]) & kKeep, (w * mul[3]) & kKeep);
  hi = make_uint4((w * mul[4]) & kKeep, (w * mul[5]) & kKeep, w & kKeep, __umulhi(w, hi31) & kKeep);
}

// orders this thread's generic-proxy writes to shared memory before later async-proxy reads (the MMA)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__global__ void __launch_bounds__(kFThreads, 1)
    k_pair_mma_fused(const __grid_constant__ CUtensorMap rmap, uint32_t n1, uint32_t nb, uint32_t n_tiles,
                     uint32_t nsteps, uint32_t steps_per_item, uint32_t ksplit, uint32_t* __restrict__ C2,
                     uint32_t* __restrict__ err, uint32_t extra_tx, uint32_t unit) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint32_t s_abort;
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // the 128-byte swizzle repeats every 1024 bytes
  const uint32_t op_st = base;                   // operand stage: 256 A rows then 256 B rows of 128 bytes
  const uint32_t raw_st = base + kFStages * kFStageBytes;
  uint32_t* const staging =
      reinterpret_cast<uint32_t*>(smem_raw + (raw_st + kRStages * kRawStageBytes - raw));
  const uint32_t bars = raw_st + kRStages * kRawStageBytes + kFStagingBytes;
  auto rfull = [&](uint32_t s) { return bars + 8 * s; };
  auto rempty = [&](uint32_t s) { return bars + 8 * (kRStages + s); };
  auto ofull = [&](uint32_t s) { return bars + 8 * (2 * kRStages + s); };
  auto oempty = [&](uint32_t s) { return bars + 8 * (2 * kRStages + kFStages + s); };
  const uint32_t acc_full = bars + 8 * (2 * kRStages + 2 * kFStages);
  const uint32_t acc_empty = acc_full + 8;
  const uint32_t fin = acc_full + 16;
  const uint32_t acc_last = fin + 8;  // the last tile's MMAs done (single use: expander warps wait on it)
  const uint32_t tslot = acc_last + 8;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile uint32_t* abort_flag = &s_abort;
  auto abort_now = [&]() {
    atomicOr(err, DEV_ERR_TIMEOUT);
    *abort_flag = 1u;
  };

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < kRStages; ++s) {
      mbar_init(rfull(s), 1);             // the producer's arrive + the TMA bytes
      mbar_init(rempty(s), kGroupWarps);  // one arrive per warp of the group that expands the slice
    }
    for (uint32_t s = 0; s < kFStages; ++s) {
      mbar_init(ofull(s), kGroupWarps);  // one arrive per warp of the group, after its proxy fence
      mbar_init(oempty(s), 1);           // the MMA commit that consumed the stage
    }
    mbar_init(acc_full, 1);   // the MMA commit after an item's last slice
    mbar_init(acc_empty, 4);  // one arrive per read-back warp
    mbar_init(fin, 1);
    mbar_init(acc_last, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot), "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem_raw + (tslot - raw));

  // item -> (row block bi, column block bj >= bi, first K slice, slices); items of one K range are
  // consecutive, so the CTAs of a round read the same K slices of the rows (L2 reuse)
  const uint32_t n_items = n_tiles * ksplit;
  auto decode = [&](uint32_t item, uint32_t& bi, uint32_t& bj, uint32_t& k0, uint32_t& ns) {
    const uint32_t split = item / n_tiles;
    uint32_t t = item % n_tiles;
    bi = 0;
    while (t >= nb - bi) {  // row block bi pairs with the column blocks bj >= bi
      t -= nb - bi;
      ++bi;
    }
    bj = bi + t;
    k0 = split * steps_per_item;
    ns = min(nsteps, k0 + steps_per_item) - k0;
  };

  // read-back round rd (0-31) of tile (bi, bj) by one warp for TMEM lane quarter `quarter`: half rd / 16, 16
  // columns from (rd mod 16) x 16, through the warp's staging area sw (32 x kFPitch words)
  auto readback_round = [&](uint32_t rd, uint32_t* sw, uint32_t bi, uint32_t bj, uint32_t quarter) {
    const uint32_t h = rd / (kFN / kFChunk), c0 = (rd % (kFN / kFChunk)) * kFChunk;
    const uint32_t row0 = bi * kFM + h * kBM + quarter * 32;
    uint32_t r[16];
    tmem_ld16(tmem + ((quarter * 32u) << 16) + h * kBN + c0, r);
#pragma unroll
    for (uint32_t c = 0; c < 16; ++c)
      sw[lane * kFPitch + c] = __float2uint_rn(__uint_as_float(r[c]) * 0.25f);  // exact: a power of 2
    __syncwarp();
    const uint32_t j = bj * kFN + c0 + (lane & 15u);
#pragma unroll 4
    for (uint32_t rr = 0; rr < 16; ++rr) {
      const uint32_t rl = rr + (lane >> 4) * 16u, i = row0 + rl;
      if (i < j && j < n1) {  // i < j < n1 also bounds i
        const uint32_t v = sw[rl * kFPitch + (lane & 15u)];
        if (ksplit > 1) atomicAdd(&C2[(size_t)i * n1 + j], v);
        else C2[(size_t)i * n1 + j] = v;
      }
    }
    __syncwarp();
  };

  uint32_t issued = 0;
  bool mma_open = false;
  if (warp == 0) {
    if (lane == 0) {
      for (uint32_t item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x) {
        uint32_t bi, bj, k0, ns;
        decode(item, bi, bj, k0, ns);
        bool ok = true;
        for (uint32_t s = 0; s < ns; ++s, ++issued) {
          const uint32_t st = issued % kRStages;
          if (issued >= kRStages && !mbar_wait(rempty(st), ((issued / kRStages) - 1) & 1)) {
            abort_now();
            ok = false;
            break;
          }
          // (extra_tx, a failure-detection test only: bytes that never arrive, so the wait runs out)
          mbar_expect_tx(rfull(st), kRawStageBytes + extra_tx);
          const int32_t x = (int32_t)((k0 + s) * 4);  // words: x * 4 bytes is a multiple of 16
          const uint32_t d = raw_st + st * kRawStageBytes;
          tma_load(d, &rmap, x, (int32_t)(bi * kFM), rfull(st));
          tma_load(d + kBM * 16, &rmap, x, (int32_t)(bi * kFM + kBM), rfull(st));
          tma_load(d + 2 * kBM * 16, &rmap, x, (int32_t)(bj * kFN), rfull(st));
          tma_load(d + 3 * kBM * 16, &rmap, x, (int32_t)(bj * kFN + kBM), rfull(st));
        }
        if (!ok) break;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t consumed = 0, it = 0;
      for (uint32_t item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x, ++it) {
        uint32_t bi, bj, k0, ns;
        decode(item, bi, bj, k0, ns);
        if (it >= 1 && !mbar_wait(acc_empty, (it - 1) & 1)) {  // the previous tile read back
          abort_now();
          break;
        }
        tc_fence_after();
        bool ok = true;
        for (uint32_t s = 0; s < ns; ++s, ++consumed) {
          const uint32_t st = consumed % kFStages;
          if (!mbar_wait(ofull(st), (consumed / kFStages) & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a = op_st + st * kFStageBytes;
          const uint64_t a0 = sw128_desc(a), a1 = sw128_desc(a + kABytes), bd = sw128_desc(a + 2 * kABytes);
#pragma unroll
          for (uint32_t kk = 0; kk < kBK / kMmaK; ++kk) {
            mma_f8f6f4(tmem, a0 + 2 * kk, bd + 2 * kk, idesc<false>(), (s | kk) != 0u);
            mma_f8f6f4(tmem + kBN, a1 + 2 * kk, bd + 2 * kk, idesc<false>(), (s | kk) != 0u);
          }
          mma_commit(oempty(st));
          mma_open = true;
        }
        if (!ok) {
          abort_now();
          mma_commit(acc_full);
          mma_open = true;
          break;
        }
        mma_commit(acc_full);
        if (item + gridDim.x >= n_items) mma_commit(acc_last);  // the CTA's last tile
        mma_open = false;
      }
    }
    __syncwarp();
  } else if (warp < 6) {
    // read-back: TMEM lanes -> staging (transposed) -> 64-byte row segments of C2, for both halves; rounds of
    // 16 columns, lanes 0-15 and 16-31 writing rows rr and rr + 16; the last tile's 32 rounds are shared with
    // the expander warps of the same quarter (this warp takes every kLastWorkers-th)
    const uint32_t quarter = warp & 3;
    uint32_t* sw = staging + (warp - 2) * 32 * kFPitch;
    uint32_t it = 0;
    for (uint32_t item = blockIdx.x; item < n_items; item += gridDim.x, ++it) {
      uint32_t bi, bj, k0, ns;
      decode(item, bi, bj, k0, ns);
      const bool ok = __all_sync(0xffffffffu, mbar_wait(acc_full, it & 1));
      if (!ok || *abort_flag) {
        if (lane == 0 && !ok) abort_now();
        break;
      }
      tc_fence_after();
      const uint32_t step = item + gridDim.x >= n_items ? kLastWorkers : 1u;
#pragma unroll 1
      for (uint32_t rd = 0; rd < 2 * kFN / kFChunk; rd += step) readback_round(rd, sw, bi, bj, quarter);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
  } else {
    // expanders: raw stage -> operand stage.  Group g takes the slices c with c mod 3 = g (and so always raw
    // stage g and operand stage g); its thread e owns rows e and e + 256 of the slice (A rows 0-255, B rows 256-511:
    // consecutive 128-byte rows of the operand stage): one 16-byte load of the row's 4 raw words, then 8
    // chunks of 16 bytes, chunk c stored at c ^ (row mod 8) (the 128-byte swizzle; the 8 lanes of a store
    // phase are 8 consecutive rows, so they hit 8 distinct chunk positions: no bank conflict)
    const uint32_t grp = (threadIdx.x - kThreads) / kGroupThreads, e = (threadIdx.x - kThreads) % kGroupThreads;
    uint32_t mul[6];
#pragma unroll
    for (uint32_t t = 0; t < 6; ++t) mul[t] = unit << (6 - t);
    const uint32_t hi31 = unit << 31;
    uint32_t c = 0;  // slices of this CTA so far (both groups)
    bool ok = true;
    for (uint32_t item = blockIdx.x; item < n_items && ok && !*abort_flag; item += gridDim.x) {
      uint32_t bi, bj, k0, ns;
      decode(item, bi, bj, k0, ns);
      for (uint32_t s = 0; s < ns; ++s, ++c) {
        if (c % kExpGroups != grp) continue;
        const uint32_t rs = c % kRStages, os = c % kFStages;
        ok = __all_sync(0xffffffffu, mbar_wait(rfull(rs), (c / kRStages) & 1));
        if (ok && c >= kFStages) ok = __all_sync(0xffffffffu, mbar_wait(oempty(os), ((c / kFStages) - 1) & 1));
        if (!ok) {
          if (lane == 0) abort_now();
          break;
        }
        const uint8_t* rsrc = smem_raw + (raw_st + rs * kRawStageBytes - raw);
        uint8_t* odst = smem_raw + (op_st + os * kFStageBytes - raw);
#pragma unroll
        for (uint32_t h = 0; h < kRowsPerExp; ++h) {
          const uint32_t row = e + h * kGroupThreads, sw7 = row & 7u;
          const uint4 w = *reinterpret_cast<const uint4*>(rsrc + row * 16u);
          uint8_t* drow = odst + row * 128u;
          const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (uint32_t q = 0; q < 4; ++q) {
            uint4 lo, hi;
            spread32_two(wv[q], mul, hi31, lo, hi);
            *reinterpret_cast<uint4*>(drow + (((2u * q) ^ sw7) << 4)) = lo;
            *reinterpret_cast<uint4*>(drow + (((2u * q + 1u) ^ sw7) << 4)) = hi;
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(ofull(os));
          mbar_arrive(rempty(rs));
        }
      }
    }
    // the last tile's read-back, shared with the read-back warp of this warp's quarter once its MMAs are
    // done (acc_last: every MMA has read its operand stage, so stage 0 holds the staging areas)
    if (ok && !*abort_flag) {
      const bool done = __all_sync(0xffffffffu, mbar_wait(acc_last, 0));
      if (done && !*abort_flag) {
        tc_fence_after();
        const uint32_t last = blockIdx.x + (n_items - 1 - blockIdx.x) / gridDim.x * gridDim.x;
        uint32_t bi, bj, k0, ns;
        decode(last, bi, bj, k0, ns);
        const uint32_t ew = warp - kThreads / 32;  // expander warp 0-23
        uint32_t* sw = reinterpret_cast<uint32_t*>(smem_raw + (op_st - raw)) + ew * 32 * kFPitch;
        for (uint32_t rd = 1 + ew / 4; rd < 2 * kFN / kFChunk; rd += kLastWorkers)
          readback_round(rd, sw, bi, bj, warp & 3);
        tc_fence_before();
      } else if (!done && lane == 0) {
        abort_now();
      }
    }
  }

  // teardown after an abort: the producer waits (bounded, and no longer once one wait ran out) for its last
  // raw stages in flight, the MMA thread for its MMAs that nobody waits for
  if (warp == 0 && lane == 0 && *abort_flag) {
    for (uint32_t q = issued > kRStages ? issued - kRStages : 0; q < issued; ++q)
      if (!mbar_wait(rfull(q % kRStages), (q / kRStages) & 1)) break;
  }
  if (warp == 1 && lane == 0 && (mma_open || *abort_flag)) {
    mma_commit(fin);
    (void)mbar_wait(fin, 0);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                              : "memory");
}

// tiles of the fused kernel: 256-row blocks bi <= bj
uint32_t fused_tiles(uint32_t n1) {
  const uint32_t nb = (n1 + kFM - 1) / kFM;
  return nb * (nb + 1) / 2;
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encoder(EncodeTiled* out) {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && (q != cudaDriverEntryPointSuccess || !p)) e = cudaErrorNotSupported;
    fn = reinterpret_cast<EncodeTiled>(p);
  });
  *out = fn;
  return e;
}

uint32_t pair_tiles(uint32_t n1) {
  const uint32_t nbi = (n1 + kBM - 1) / kBM, nbj = (n1 + kBN - 1) / kBN;
  uint32_t tiles = 0;
  for (uint32_t bi = 0; bi < nbi; ++bi) tiles += nbj - bi / 2;
  return tiles;
}

}  // namespace

uint64_t pair_mma_buffer_bytes(uint32_t n1, uint32_t stride, bool e2m1) {
  return (uint64_t)n1 * stride * (e2m1 ? 16ull : 32ull);
}

double pair_mma_cost_us(uint32_t n1, uint32_t stride, int num_sms, bool e2m1, bool fused) {
  // widening (bytes written at ~5 TB/s) + tile rounds at ~1.5 PFLOP/s of kind::f8f6f4 per 152 SMs
  const double x_bytes = fused ? 0.0 : (double)pair_mma_buffer_bytes(n1, stride, e2m1);
  // (fused: 256 x 256 tiles, twice the MMAs per slice)
  const uint32_t tiles = fused ? fused_tiles(n1) : pair_tiles(n1);
  const uint32_t nsteps = stride / 4;
  const double step_us = (fused ? 2.0 : 1.0) * 2.0 * kBM * kBN * kBK / (1.5e15 / 152.0) * 1e6;  // one K slice of a tile
  double best = 1e300;
  for (uint32_t ks = 1; ks <= 256; ++ks) {
    const uint32_t spi = std::min(kMaxStepsPerItem, (nsteps + ks - 1) / ks);
    const uint32_t k2 = (nsteps + spi - 1) / spi;
    const uint64_t items = (uint64_t)tiles * k2;
    const uint64_t rounds = (items + num_sms - 1) / num_sms;
    best = std::min(best, (double)rounds * (spi + 1) * step_us + 8.0 * step_us);
  }
  return x_bytes / 5e12 * 1e6 + best + 4.0;
}

// the split of the K range: items fill whole rounds of the SMs, at most 2^24 elements per item, at least 8
// slices per item to cover a read-back; an item's read-back overlaps the next item's MMAs, so only the last
// one is exposed and a CTA takes about rounds x (slices + 1) + 8 slice times
static uint32_t pair_split(uint32_t tiles, uint32_t nsteps, int num_sms) {
  uint32_t spi = std::min(kMaxStepsPerItem, nsteps);
  double best = 1e300;
  for (uint32_t ks = 1; ks <= 256; ++ks) {
    const uint32_t c = std::min(kMaxStepsPerItem, (nsteps + ks - 1) / ks);
    if (c < 8 && ks > 1) break;
    const uint32_t k2 = (nsteps + c - 1) / c;
    const uint64_t items = (uint64_t)tiles * k2;
    const uint64_t rounds = (items + num_sms - 1) / num_sms;
    const double cost = (double)rounds * (c + 1.0) + 8.0;
    if (cost < best - 1e-9) {
      best = cost;
      spi = c;
    }
  }
  return spi;
}

cudaError_t launch_pair_mma_fused(const PairLaunch& p, uint32_t* err, int num_sms, cudaStream_t st,
                                  uint32_t* ksplit_used, uint32_t extra_tx) {
  if (p.n1 < 2) {
    *ksplit_used = 0;
    return cudaSuccess;
  }
  if (!p.rows_base) return cudaErrorInvalidValue;
  cudaError_t e = kernel_smem_limit(reinterpret_cast<const void*>(k_pair_mma_fused), (int)kFSmemBytes);
  if (e != cudaSuccess) return e;
  EncodeTiled encode = nullptr;
  if ((e = encoder(&encode)) != cudaSuccess) return e;
  // the frequent rows' raw bits as a 2-D tensor: stride words x n1 rows; boxes of 4 words (one slice of 128
  // transactions) x 128 rows, no swizzle; rows past n1 read as zeros
  alignas(64) CUtensorMap map;
  const cuuint64_t dims[2] = {p.stride, p.n1};
  const cuuint64_t strides[1] = {(cuuint64_t)p.stride * 4};
  const cuuint32_t box[2] = {4, kBM};
  const cuuint32_t estr[2] = {1, 1};
  if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t*>(p.rows_base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const uint32_t nb = (p.n1 + kFM - 1) / kFM;
  const uint32_t tiles = fused_tiles(p.n1);
  const uint32_t nsteps = p.stride / 4;  // stride is a multiple of 32 words: whole 128-transaction slices
  const uint32_t spi = pair_split(tiles, nsteps, num_sms);
  const uint32_t ksplit = (nsteps + spi - 1) / spi;
  *ksplit_used = ksplit;
  if (ksplit > 1 && (e = cudaMemsetAsync(p.C2, 0, (size_t)p.n1 * p.n1 * sizeof(uint32_t), st)) != cudaSuccess)
    return e;
  const uint64_t items = (uint64_t)tiles * ksplit;
  const uint32_t grid = (uint32_t)std::min<uint64_t>(items, (uint64_t)num_sms);
  k_pair_mma_fused<<<grid, kFThreads, kFSmemBytes, st>>>(map, p.n1, nb, tiles, nsteps, spi, ksplit, p.C2, err,
                                                         extra_tx, 1u);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_pair_mma(const PairLaunch& p, uint8_t* X, bool e2m1, uint32_t* err, int num_sms, cudaStream_t st,
                            uint32_t* ksplit_used, uint32_t extra_tx) {
  if (p.n1 < 2) {
    *ksplit_used = 0;
    return cudaSuccess;
  }
  cudaError_t attr_err = kernel_smem_limit(reinterpret_cast<const void*>(k_pair_mma<false>), (int)kSmemBytes);
  if (attr_err == cudaSuccess)
    attr_err = kernel_smem_limit(reinterpret_cast<const void*>(k_pair_mma<true>), (int)kSmemBytes);
  if (attr_err != cudaSuccess) return attr_err;
  EncodeTiled encode = nullptr;
  cudaError_t e = encoder(&encode);
  if (e != cudaSuccess) return e;

  // widen the frequent rows
  const uint64_t words = (uint64_t)p.n1 * p.stride;
  const uint32_t eg = (uint32_t)std::min<uint64_t>((words + 255) / 256, (uint64_t)num_sms * 16);
  if (e2m1) {
    const dim3 g2(std::min<uint32_t>((p.stride + 255) / 256, 16), std::min<uint32_t>(p.n1, 65535));
    k_expand_e2m1<<<g2, 256, 0, st>>>(p.bits, p.stride, p.frows, p.n1, reinterpret_cast<uint4*>(X));
  }
  else
    k_expand_e4m3<<<eg, 256, 0, st>>>(p.bits, p.stride, p.frows, p.n1, reinterpret_cast<uint4*>(X));
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  // X as a 2-D tensor: K (stride * 32 transactions) x n1 rows; boxes of 128 transactions x 128 rows with
  // the 128-byte swizzle (e2m1: 64 packed bytes per box row, unpacked by the TMA to 128 in shared
  // memory); rows past n1 read as zeros
  const uint64_t k_elems = (uint64_t)p.stride * 32;
  const uint64_t row_bytes = e2m1 ? k_elems / 2 : k_elems;
  alignas(64) CUtensorMap map;
  const cuuint64_t dims[2] = {k_elems, p.n1};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {kBK, kBM};
  const cuuint32_t estr[2] = {1, 1};
  if (encode(&map, e2m1 ? CU_TENSOR_MAP_DATA_TYPE_16U4_ALIGN16B : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, X, dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;

  const uint32_t nbj = (p.n1 + kBN - 1) / kBN;
  const uint32_t tiles = pair_tiles(p.n1);
  const uint32_t nsteps = p.stride / 4;  // stride is a multiple of 32 words: whole 128-element slices
  const uint32_t spi = pair_split(tiles, nsteps, num_sms);
  const uint32_t ksplit = (nsteps + spi - 1) / spi;
  *ksplit_used = ksplit;
  if (ksplit > 1 && (e = cudaMemsetAsync(p.C2, 0, (size_t)p.n1 * p.n1 * sizeof(uint32_t), st)) != cudaSuccess)
    return e;
  const uint64_t items = (uint64_t)tiles * ksplit;
  const uint32_t grid = (uint32_t)std::min<uint64_t>(items, (uint64_t)num_sms);
  if (e2m1)
    k_pair_mma<true><<<grid, kThreads, kSmemBytes, st>>>(map, p.n1, nbj, tiles, nsteps, spi, ksplit, p.C2, err, extra_tx);
  else
    k_pair_mma<false><<<grid, kThreads, kSmemBytes, st>>>(map, p.n1, nbj, tiles, nsteps, spi, ksplit, p.C2, err, extra_tx);
  note_launch();
  return cudaGetLastError();
}

}  // namespace fim
