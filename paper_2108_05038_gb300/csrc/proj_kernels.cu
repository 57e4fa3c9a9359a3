// K4, projected mode: the thesis's Phase 3 (data distribution) and Phase 4
// (Eclat on the distributed database parts), restated for one GPU.
//
// In the thesis, the processor that mines a prefix class [U | E] receives in
// Phase 3 exactly the transactions that contain U (Sec. 8.3, "Detailed
// description of Phase 3"), builds the tidlists of the extensions over that
// database part, and runs Eclat on them in Phase 4 (Sec. 8.4, Exec-Eclat).
// Here the processor is a warp and the prefix classes are the one-item
// classes [{i} | S_i], S_i = the rows j after i with {i, j} frequent:
//
//   Phase 3 (k_proj_tids, k_proj_bits): T_i = the transactions of row i in
//     ascending order, and for every survivor s in S_i the bitmap Y_i[s] over
//     T_i: bit p of Y_i[s] is set iff transaction T_i[p] contains s.  Every
//     bitmap is ceil(|T_i| / 32) words instead of the D / 32 of a row.
//   Phase 4 (k_dfs_proj): one warp per two-item class [{i, s_m} | later
//     survivors of i], Eclat-DFS-Computation (App. B.3.2) on the bitmaps
//     Y_i: the root prefix is Y_i[s_m] itself, a child's prefix is its
//     parent's AND the child's bitmap, and every support is a popcount of
//     prefix & Y_i[c] (support of a union by intersecting the tidlists of two
//     generating subsets, App. B.3.1).
//
// The prefix classes, their candidates, survivors and output records are
// those of the other traversals; only the transaction space of a class is
// renumbered (t(X) for X in the class is a subset of T_i, so no bit of a
// support is lost).  Classes whose bitmaps do not fit the budgets (or whose
// rows are too wide for the warp stacks) go to a second queue that the sparse
// node mode mines from the full rows.
//
// Load balance: a warp that meets a frame [X | S] whose next level is large
// repeats Phase 3 for it: it builds the database part of X (the bitmaps of S
// over the transactions of X, ceil(supp(X) / 32) words each) in a region of
// its own and hands the frame's children to the other warps through a queue
// (the thesis's dynamic load balancing of Phase 1 sends subclasses with their
// database parts to idle processors in the same way).  A class region and a
// split region have one layout: header (rows k, padded words Wp, prefix
// length, words W, top class), the prefix's item ids ascending, the rows'
// item ids, then the k bitmaps.
#include <algorithm>
#include <map>
#include <mutex>

#include "fim_internal.cuh"

namespace fim {
namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint64_t kNotProjected = ~0ull;
constexpr uint32_t kQueueF = 0x80000000u;  // eoffx: the class's entries go to the fallback queue
constexpr uint32_t kGroupWords = 4;         // projection work item: 4 bitmap words (128 transactions) ...
constexpr uint32_t kGroupRows = 32;         // ... of up to 32 survivors
constexpr uint32_t kNoop = 0xffffffffu;     // queue item that carries no work (its region did not fit)

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Exclusive block-wide scan.  tmp: 33 shared elements; tmp[32] receives the
// block total.  Two barriers inside; the caller barriers before reusing tmp.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* tmp) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(kFull, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const T w = lane < nw ? tmp[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(kFull, wi, o);
      if (lane >= (uint32_t)o) wi += y;
    }
    if (lane < nw) tmp[lane] = wi - w;
    if (lane == 31) tmp[32] = wi;
  }
  __syncthreads();
  return tmp[warp] + x - v;
}

__host__ __device__ inline uint32_t words_of(uint32_t supp) { return (supp + 31) / 32; }
__host__ __device__ inline uint32_t padded_words(uint32_t supp) { return (words_of(supp) + 3) & ~3u; }

// ---------------------------------------------------------------------------
// Phase 3, planning (one CTA): which classes get a database part, where it
// lives, and the split of the two-item classes into the projected queue and the
// fallback queue, all in queue order (LPT on the estimate, Sec. 8.2), so the
// budgets go to the classes that start first.
__global__ void __launch_bounds__(1024) k_proj_plan(const ProjLaunch P) {
  __shared__ unsigned long long sy[33], st[33], sbytes[33];
  __shared__ uint32_t sa[33], sb[33], sc[33], sd[33], se[33];
  __shared__ unsigned long long carry_y, carry_t, carry_b;
  __shared__ uint32_t carry_p, carry_f, carry_i, carry_c, carry_n;
  if (threadIdx.x == 0) {
    carry_y = carry_t = carry_b = 0;
    carry_p = carry_f = carry_i = carry_c = carry_n = 0;
  }
  __syncthreads();
  for (uint32_t base = 0; base < P.n1; base += blockDim.x) {
    const uint32_t q = base + threadIdx.x;
    const bool in = q < P.n1;
    const uint32_t i = in ? P.row_order[q] : 0u;
    const uint32_t k = in ? P.scnt[i] : 0u;
    const uint32_t ne = k >= 2 ? k - 1 : 0u;  // two-item classes (i, s_m), m < k - 1
    const uint32_t s = in ? P.row_supp[i] : 0u;
    const uint32_t Wp = padded_words(s);
    const bool elig = ne > 0 && words_of(s) <= P.w_cap;
    const unsigned long long ysz = elig ? region_rows_off(1, k) + (unsigned long long)k * Wp : 0ull;
    const unsigned long long tsz = elig ? (((unsigned long long)s + 3) & ~3ull) : 0ull;
    const unsigned long long yex = block_excl_scan<unsigned long long>(ysz, sy);
    const unsigned long long tex = block_excl_scan<unsigned long long>(tsz, st);
    const unsigned long long ybase = carry_y + yex, tbase = carry_t + tex;
    const bool proj = elig && ybase + ysz <= P.y_cap_words && tbase + tsz <= P.t_cap;
    const uint32_t neP = proj ? ne : 0u, neF = proj ? 0u : ne;
    const uint32_t nit = proj ? (Wp / kGroupWords) * ((k + kGroupRows - 1) / kGroupRows) : 0u;
    const uint32_t pex = block_excl_scan<uint32_t>(neP, sa);
    const uint32_t fex = block_excl_scan<uint32_t>(neF, sb);
    const uint32_t iex = block_excl_scan<uint32_t>(nit, sc);
    const uint32_t cex = block_excl_scan<uint32_t>(proj ? k : 0u, sd);  // rows of the projected classes
    const uint32_t nex = block_excl_scan<uint32_t>(proj ? 1u : 0u, se);   // projected classes
    (void)cex;
    (void)nex;
    // Phase 3's operand bytes: the row read once, its transactions written and read, one word gathered per
    // (survivor, transaction), the bitmaps written
    const unsigned long long pb = proj ? 4ull * P.stride + 8ull * s + 4ull * k * s + 4ull * k * Wp : 0ull;
    (void)block_excl_scan<unsigned long long>(pb, sbytes);
    if (in) {
      P.yoff[i] = proj ? ybase : kNotProjected;
      P.toff[i] = proj ? tbase : kNotProjected;
      P.eoffx[q] = proj ? carry_p + pex : (kQueueF | (carry_f + fex));
      P.itemoff[q] = carry_i + iex;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_y += sy[32];
      carry_t += st[32];
      carry_p += sa[32];
      carry_f += sb[32];
      carry_i += sc[32];
      carry_c += sd[32];
      carry_n += se[32];
      carry_b += sbytes[32];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.itemoff[P.n1] = carry_i;
    P.ctrl->arena_top = (carry_y + 31) & ~31ull;  // split regions are carved after the class regions
    P.ctrl->proj_bytes = carry_b;
    P.ctrl->proj_pending = carry_p;
    P.ctrl->n_entries = carry_p;
    P.ctrl->n_entries_f = carry_f;
    P.ctrl->queue_head = 0;
    P.ctrl->queue_head_f = 0;
    // hand-out threshold: 64 x the mean width of a projected row, within [128, 65536] words
    const unsigned long long mean_w = carry_c ? carry_y / carry_c : 1ull;
    P.ctrl->proj_split_words = min(max(64ull * mean_w, 128ull), 65536ull);
    P.ctrl->n_proj_classes = carry_n;
    P.ctrl->n_proj_items = carry_i;
  }
}

// Phase 3, transactions: T_i = the set bits of row i in ascending order (one
// CTA per queue position; the row is streamed once, four 16-byte words per
// thread and round).
__global__ void __launch_bounds__(256) k_proj_tids(const ProjLaunch P) {
  __shared__ uint32_t tmp[33];
  const uint32_t q = blockIdx.x;
  const uint32_t i = P.row_order[q];
  const uint64_t to = P.toff[i];
  if (to == kNotProjected) return;
  const uint32_t stride4 = P.stride / 4;
  const uint4* r4 = reinterpret_cast<const uint4*>(P.bits + (size_t)P.frows[i] * P.stride);
  uint32_t* T = P.T + to;
  const uint32_t s = P.row_supp[i];  // = the row's popcount; the bound only guards the class's region
  // the class region's header and item ids
  const uint32_t k = P.scnt[i];
  uint32_t* R = P.Y + P.yoff[i];
  if (threadIdx.x == 0) {
    R[0] = k;
    R[1] = padded_words(s);
    R[2] = 1;
    R[3] = words_of(s);
    R[4] = i;
    R[5] = R[6] = R[7] = 0;
    R[8] = P.rank_item[P.frows[i]];
  }
  for (uint32_t j = threadIdx.x; j < k; j += blockDim.x)
    R[12 + j] = P.rank_item[P.frows[P.sitems[P.soff[i] + j]]];
  uint32_t carry = 0;
  for (uint32_t w0 = 0; w0 < stride4; w0 += 4 * blockDim.x) {
    uint4 v[4];
    uint32_t c = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t w = w0 + 4 * threadIdx.x + u;
      v[u] = w < stride4 ? __ldg(r4 + w) : make_uint4(0u, 0u, 0u, 0u);
      c += __popc(v[u].x) + __popc(v[u].y) + __popc(v[u].z) + __popc(v[u].w);
    }
    uint32_t pos = carry + block_excl_scan<uint32_t>(c, tmp);
    const uint32_t tot = tmp[32];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t t0 = (w0 + 4 * threadIdx.x + u) * 128u;
      const uint32_t word[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        uint32_t x = word[h];
        while (x) {
          if (pos < s) T[pos] = t0 + 32u * h + (uint32_t)(__ffs(x) - 1);
          ++pos;
          x &= x - 1;
        }
      }
    }
    carry += tot;
    __syncthreads();
  }
}

// Phase 3, bitmaps: work item = (class, 4 words of its bitmaps = 128 of its
// transactions, up to 32 of its survivors).  Lane l holds transaction
// T_i[128 g + 32 r + l] and the row of survivor j0 + l; for every survivor the
// warp gathers the word of that row holding each lane's transaction and packs
// the 32 bits with a ballot, so the bitmap words come out in T_i's order.
__global__ void __launch_bounds__(256) k_proj_bits(const ProjLaunch P) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t total = P.itemoff[P.n1];
  const uint32_t nwarps = gridDim.x * (blockDim.x / 32);
  for (uint32_t item = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); item < total; item += nwarps) {
    // queue position of the item: the last q with itemoff[q] <= item
    uint32_t lo = 0, hi = P.n1;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(P.itemoff + mid) <= item) lo = mid;
      else hi = mid;
    }
    const uint32_t i = __ldg(P.row_order + lo);
    const uint32_t k = __ldg(P.scnt + i), s = __ldg(P.row_supp + i);
    const uint32_t Wp = padded_words(s);
    const uint32_t local = item - __ldg(P.itemoff + lo);
    const uint32_t nJ = (k + kGroupRows - 1) / kGroupRows;
    const uint32_t g = local / nJ, j0 = (local - g * nJ) * kGroupRows;
    const uint32_t nj = min(kGroupRows, k - j0);
    const uint32_t* T = P.T + P.toff[i];
    uint32_t tid[kGroupWords];
#pragma unroll
    for (uint32_t r = 0; r < kGroupWords; ++r) {
      const uint32_t pos = (g * kGroupWords + r) * 32u + lane;
      tid[r] = pos < s ? __ldg(T + pos) : kFull;
    }
    const uint32_t myrow = lane < nj ? __ldg(P.frows + __ldg(P.sitems + __ldg(P.soff + i) + j0 + lane)) : 0u;
    uint32_t mine[kGroupWords] = {0u, 0u, 0u, 0u};
    constexpr uint32_t U = 4;  // survivors per round: U x 4 loads in flight per lane
    for (uint32_t jj = 0; jj < nj; jj += U) {
      uint32_t w[U][kGroupWords];
#pragma unroll
      for (uint32_t u = 0; u < U; ++u) {
        const uint32_t rrow = __shfl_sync(kFull, myrow, (jj + u) & 31);
        const bool ok = jj + u < nj;
        const uint32_t* rp = P.bits + (size_t)rrow * P.stride;
#pragma unroll
        for (uint32_t r = 0; r < kGroupWords; ++r) w[u][r] = (ok && tid[r] != kFull) ? __ldg(rp + (tid[r] >> 5)) : 0u;
      }
#pragma unroll
      for (uint32_t u = 0; u < U; ++u)
#pragma unroll
        for (uint32_t r = 0; r < kGroupWords; ++r) {
          const uint32_t y = __ballot_sync(kFull, (w[u][r] >> (tid[r] & 31)) & 1u);
          if (lane == jj + u) mine[r] = y;
        }
    }
    if (lane < nj) {
      uint4* dst = reinterpret_cast<uint4*>(P.Y + P.yoff[i] + region_rows_off(1, k) + (uint64_t)(j0 + lane) * Wp +
                                            g * kGroupWords);
      *dst = make_uint4(mine[0], mine[1], mine[2], mine[3]);
    }
  }
}

// ---------------------------------------------------------------------------
// Phase 4: warps take items (region R, m): the node X = (R's prefix) u {row m
// of R}, whose prefix bitmap is row m and whose candidates are rows m+1 .. k-1,
// and run its subtree depth first.  Items come from the static queue (the
// two-item classes of the projected one-item classes, in LPT order) and then
// from the queue of split frames.
//
// A frame [X | S] of the DFS lives in a region R (the transaction space of its
// bitmaps) with a prefix P (a bitmap over R's space, or none when R is X's own
// database part, i.e. P would be all ones) and its survivors S as indices of
// R's rows.  When X's support is at most a quarter of R's width the frame is
// compacted: X's own database part (S's bitmaps over t(X), ceil(supp(X) / 32)
// words each) is built on the warp's stack, so that every deeper support is
// counted over short bitmaps; when the next level is large the same part is
// built in the shared arena instead and the frame's children are handed to the
// other warps.
//
// Per warp, in shared memory: the path ids and per frame depth the frame's
// region, prefix, survivor list, size, next child and stack top.  The stack
// (global memory) is a bump region: survivor lists of (row, support) pairs,
// materialised prefixes, compacted regions.

constexpr int kG = 8;   // candidates counted per round
constexpr int kPR = 2;  // prefix words per lane per chunk (64 words)
constexpr unsigned long long kIdleNs = 2000000000ull;  // no item finished anywhere for 2 s: give up
constexpr uint32_t kIdentity = 0xffffffffu;  // frame list: every row of the region, in order
constexpr unsigned long long kDiffFrame = 1ull;  // frame prefix marker: the survivors are held as diffsets

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* a) { return *(volatile const uint32_t*)a; }

struct RegionView {
  const uint32_t* R;     // header
  const uint32_t* rids;  // item id of each row
  const uint32_t* Y;     // rows
  uint32_t k, Wp, xlen, W, cls;
};

__device__ __forceinline__ RegionView region_view(const uint32_t* R) {
  RegionView v;
  v.R = R;
  v.k = R[0];
  v.Wp = R[1];
  v.xlen = R[2];
  v.W = R[3];
  v.cls = R[4];
  v.rids = R + 8 + ((v.xlen + 3) & ~3u);
  v.Y = R + region_rows_off(v.xlen, v.k);
  return v;
}

__global__ void __launch_bounds__(kProjThreads, kProjCtasPerSm) k_dfs_proj(const DfsLaunch p, const uint32_t max_len) {
  if (p.cta_time && threadIdx.x == 0) p.cta_time[2 * blockIdx.x] = global_ns();
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t L1 = max_len + 1;
  // (the 64-bit arrays first: the per-warp block is 10 L1 words, an even count, so they stay 8-byte aligned)
  unsigned long long* fr_R = reinterpret_cast<unsigned long long*>(smem + wib * 10u * L1);  // per frame: region,
  unsigned long long* fr_P = fr_R + L1;    // prefix (0: none),
  uint32_t* path = reinterpret_cast<uint32_t*>(fr_P + L1);  // ids of the current path, in path order
  uint32_t* xs = path + L1;                // the same ids ascending
  uint32_t* fr_L = xs + L1;                // survivor list (stack offset or kIdentity),
  uint32_t* fr_n = fr_L + L1;              // survivors,
  uint32_t* fr_cur = fr_n + L1;            // next child to expand,
  uint32_t* fr_top = fr_cur + L1;          // stack top below the frame
  const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  uint32_t* const stk = p.pstack + gw * p.pstack_words;
  uint32_t* const Yar = const_cast<uint32_t*>(p.Y);
  unsigned long long st_inter = 0, st_nodes = 0, st_frames = 0, st_splits = 0;
  // operand bytes: per node the prefix and the candidates' bitmaps over the region's width; per compacted or
  // handed-out frame one gathered word per (survivor, transaction) and the region written
  unsigned long long st_bytes = 0;
  unsigned long long st_sets = 0, st_items = 0;
  // count only (no records): itemsets not yet added to the reservation word, which then feeds nothing but the
  // itemset limit; added every 8 nodes and at the end of an item instead of one returning atomic per node
  unsigned long long pend_sets = 0;
  uint32_t st_maxlen = 0;
  bool static_done = false;
  constexpr uint32_t kStop = DEV_ERR_ABORTED | DEV_ERR_PSTACK | DEV_ERR_TIMEOUT;

  auto sort_path = [&](uint32_t len) {
    __syncwarp();
    for (uint32_t q = lane; q < len; q += 32) {
      const uint32_t v = path[q];
      uint32_t r = 0;
      for (uint32_t t = 0; t < len; ++t) r += path[t] < v;
      xs[r] = v;
    }
    __syncwarp();
  };

  for (;;) {
    // ---------------- acquire an item: the static queue first, then split frames' children ----------------
    unsigned long long roff = ~0ull;
    uint32_t m = 0;
    if (lane == 0) {
      bool stop = (ld_volatile(&p.ctrl->err) & kStop) != 0;
      // (records reserved so far: the high half of the reservation word)
      if (!stop && p.max_sets && (*(volatile unsigned long long*)&p.ctrl->packed >> 32) > p.max_sets) {
        atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
        stop = true;
      }
      if (!stop && !static_done) {
        const uint32_t e = atomicAdd(&p.ctrl->queue_head, 1u);
        if (e < p.ctrl->n_entries) {
          const uint2 en = p.entries[e];
          roff = p.yoff[en.x];
          m = en.y;
        } else {
          static_done = true;
        }
      }
      if (!stop && roff == ~0ull) {
        // A ticket of the split queue: slot h is filled by the producer that reserves it, so the warp
        // waits on its own slot.  Bounded: the wait ends when the slot is published, when no item is
        // left unfinished (nothing can be published any more), or when no item has finished anywhere
        // for kIdleNs or spin_limit polls (DEV_ERR_TIMEOUT).  Polls back off to 32 us.
        const uint32_t h = atomicAdd(&p.ctrl->dq_head, 1u);
        if (h < p.dq_cap) {
          const uint32_t* slot = reinterpret_cast<const uint32_t*>(p.dq + h);
          uint32_t last_pending = 0xffffffffu, sleep_ns = 128;
          unsigned long long t_last = global_ns(), polls = 0;
          for (uint32_t it = 0;; ++it) {
            if (ld_volatile(slot + 3) != 0u) {
              __threadfence();
              roff = ((unsigned long long)ld_volatile(slot + 1) << 32) | ld_volatile(slot);
              m = ld_volatile(slot + 2);
              break;
            }
            if ((it & 7) == 0 && (ld_volatile(&p.ctrl->err) & kStop)) break;
            const uint32_t pend = ld_volatile(&p.ctrl->proj_pending);
            if (pend == 0) break;
            const unsigned long long now = global_ns();
            if (pend != last_pending) {
              last_pending = pend;
              t_last = now;
              polls = 0;
            } else if (++polls > p.spin_limit || now - t_last > kIdleNs) {
              atomicOr(&p.ctrl->err, DEV_ERR_TIMEOUT);
              break;
            }
            __nanosleep(sleep_ns);
            sleep_ns = min(sleep_ns * 2, 32768u);
          }
        }
      }
    }
    roff = __shfl_sync(kFull, roff, 0);
    m = __shfl_sync(kFull, m, 0);
    if (roff == ~0ull) break;
    if (m == kNoop) {  // a reserved slot whose region did not fit: nothing to do
      __syncwarp();
      if (lane == 0) atomicSub(&p.ctrl->proj_pending, 1u);
      continue;
    }

    const RegionView R0 = region_view(p.Y + roff);
    const unsigned long long split_words = p.split_words ? p.split_words : p.ctrl->proj_split_words;
    const uint32_t cls = R0.cls;
    unsigned long long cls_sets = 0, cls_work = 0;
    for (uint32_t q = lane; q < R0.xlen; q += 32) path[q] = R0.R[8 + q];

    // Records of a node X (ids xs[0, xlen)) whose survivors are the rows out[0], out[st], out[2 st], ... with
    // supports out[1], out[st + 1], ...: one record X u {s} per survivor, or, when only the leaves are written
    // (maximal output), one record: X with its last survivor, or X alone (support xsupp) when none survived.
    auto emit = [&](const RegionView& V, const uint32_t* out, uint32_t st, uint32_t nout, uint32_t xlen,
                    uint32_t xsupp) {
      __syncwarp();  // the list written by lane 0 is read by every lane below
      if (p.leaves) {
        const uint32_t v = nout ? V.rids[out[st * (nout - 1)]] : kFull;
        const uint32_t sp = nout ? out[st * (nout - 1) + 1] : xsupp;
        const uint32_t len = nout ? xlen + 1 : xlen;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&p.ctrl->packed, (1ull << 32) | len);
        base = __shfl_sync(kFull, base, 0);
        st_sets += 1;
        st_items += len;
        st_maxlen = max(st_maxlen, len);
        cls_sets += 1;
        const uint64_t rec = base >> 32, it0 = base & 0xffffffffull;
        if (p.out_off) {
          if (rec < p.cap_sets && it0 + len <= p.cap_items) {
            uint32_t pos = xlen;  // place of v among the prefix ids (none: v absent)
            if (v != kFull) {
              pos = 0;
              for (uint32_t q0 = 0; q0 < xlen; q0 += 32)
                pos += __popc(__ballot_sync(kFull, q0 + lane < xlen && xs[q0 + lane] < v));
            }
            for (uint32_t t = lane; t < len; t += 32)
              p.out_items[it0 + t] = t < pos ? xs[t] : (t == pos ? v : xs[t - 1]);
            if (lane == 0) {
              p.out_off[rec] = it0;
              p.out_supp[rec] = sp;
            }
          } else if (lane == 0) {
            atomicOr(&p.ctrl->err, DEV_ERR_OVERFLOW);
          }
        }
        return;
      }
      if (nout == 0) return;
      if (!p.out_off) {  // count only: nothing to reserve
        pend_sets += nout;
        st_sets += nout;
        st_items += (unsigned long long)nout * (xlen + 1);
        st_maxlen = max(st_maxlen, xlen + 1);
        cls_sets += nout;
        return;
      }
      unsigned long long base = 0;
      // one atomic per node reserves its records; the exact totals and the longest length are added once per
      // warp at the end (nothing reads them while the kernel runs)
      if (lane == 0) {
        const unsigned long long sets = nout, items = (unsigned long long)nout * (xlen + 1);
        base = atomicAdd(&p.ctrl->packed, (sets << 32) | items);
        const unsigned long long after = (base >> 32) + sets;
        if ((p.max_sets && after > p.max_sets) || after > 0xfffffff0ull) atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
      }
      base = __shfl_sync(kFull, base, 0);
      st_sets += nout;
      st_items += (unsigned long long)nout * (xlen + 1);
      st_maxlen = max(st_maxlen, xlen + 1);
      cls_sets += nout;
      if (p.out_off) {  // one lane per record: the survivor's id merged into the sorted prefix ids
        for (uint32_t o = lane; o < nout; o += 32) {
          const uint32_t v = V.rids[out[st * o]];
          const uint64_t rec = (base >> 32) + o;
          const uint64_t it0 = (base & 0xffffffffull) + (uint64_t)o * (xlen + 1);
          if (rec < p.cap_sets && it0 + xlen + 1 <= p.cap_items) {
            uint32_t* dst = p.out_items + it0;
            uint32_t q = 0;
            bool placed = false;
            for (uint32_t x = 0; x < xlen; ++x) {
              const uint32_t u = xs[x];
              if (!placed && v < u) {
                dst[q++] = v;
                placed = true;
              }
              dst[q++] = u;
            }
            if (!placed) dst[q] = v;
            p.out_off[rec] = it0;
            p.out_supp[rec] = out[st * o + 1];
          } else {
            atomicOr(&p.ctrl->err, DEV_ERR_OVERFLOW);
          }
        }
      }
    };

    // Counts candidates (rows of region V: c0, c0 + 1, ... when clist is NULL, else clist[0], clist[2], ...)
    // against prefix `pre` (V.W words), writes the survivors as (row, support) pairs to out and one record
    // per survivor; returns the survivor count.  Candidate words are read only under nonzero prefix words.
    auto count_node = [&](const RegionView& V, const uint32_t* pre, const uint32_t* clist, uint32_t c0, uint32_t nc,
                          uint32_t* out, uint32_t xlen) -> uint32_t {
      uint32_t nout = 0;
      for (uint32_t t0 = 0; t0 < nc; t0 += kG) {
        uint32_t jj[kG], sum[kG];
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          const uint32_t t = t0 + g;
          jj[g] = t < nc ? (clist ? clist[2 * t] : c0 + t) : kFull;
          sum[g] = 0;
        }
        for (uint32_t w0 = 0; w0 < V.W; w0 += 32 * kPR) {
          uint32_t a[kPR];
#pragma unroll
          for (int r = 0; r < kPR; ++r) {
            const uint32_t w = w0 + 32 * r + lane;
            a[r] = w < V.W ? pre[w] : 0u;
          }
          uint32_t b[kG][kPR];
#pragma unroll
          for (int g = 0; g < kG; ++g)
#pragma unroll
            for (int r = 0; r < kPR; ++r)
              b[g][r] = (a[r] && jj[g] != kFull) ? V.Y[(uint64_t)jj[g] * V.Wp + w0 + 32 * r + lane] : 0u;
#pragma unroll
          for (int g = 0; g < kG; ++g)
#pragma unroll
            for (int r = 0; r < kPR; ++r) sum[g] += __popc(a[r] & b[g][r]);
        }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          const uint32_t c = __reduce_add_sync(kFull, sum[g]);
          if (jj[g] != kFull && c >= p.minsup) {
            if (lane == 0) {
              out[2 * nout] = jj[g];
              out[2 * nout + 1] = c;
            }
            ++nout;
          }
        }
      }
      st_inter += nc;
      cls_work += nc;
      ++st_nodes;
      st_bytes += 4ull * (nc + 1) * V.W;
      uint32_t xsupp = 0;
      if (p.leaves && nout == 0) {  // a leaf's own support: the popcount of its prefix
        for (uint32_t w = lane; w < V.W; w += 32) xsupp += __popc(pre[w]);
        xsupp = __reduce_add_sync(kFull, xsupp);
      }
      emit(V, out, 2, nout, xlen, xsupp);
      return nout;
    };

    // Builds at dst the database part of X (prefix `pre` over V's space, support supp, ids xs[0, xlen)):
    // the bitmaps of the rows list[0], list[2], ... (n of them) over the set bits of pre, with the
    // header and ids of a region.  tmp: scratch for the positions of pre's set bits (supp words).
    auto build_region = [&](uint32_t* dst, const RegionView& V, const uint32_t* pre, const uint32_t* list, uint32_t n,
                            uint32_t xlen, uint32_t supp, uint32_t* tmp) {
      const uint32_t Wp2 = padded_words(supp), W2 = words_of(supp);
      st_bytes += 4ull * n * supp + 4ull * (region_rows_off(xlen, n) + (unsigned long long)n * Wp2);
      uint32_t carry = 0;
      for (uint32_t w0 = 0; w0 < V.W; w0 += 32) {
        const uint32_t w = w0 + lane;
        uint32_t v = w < V.W ? pre[w] : 0u;
        const uint32_t c = __popc(v);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, incl, o);
          if (lane >= (uint32_t)o) incl += y;
        }
        uint32_t pos = carry + incl - c;
        while (v) {
          if (pos < supp) tmp[pos] = w * 32u + (uint32_t)(__ffs(v) - 1);
          ++pos;
          v &= v - 1;
        }
        carry += __shfl_sync(kFull, incl, 31);
      }
      if (lane == 0) {
        dst[0] = n;
        dst[1] = Wp2;
        dst[2] = xlen;
        dst[3] = W2;
        dst[4] = cls;
        dst[5] = dst[6] = dst[7] = 0;
      }
      for (uint32_t q = lane; q < xlen; q += 32) dst[8 + q] = xs[q];
      uint32_t* rids2 = dst + 8 + ((xlen + 3) & ~3u);
      for (uint32_t q = lane; q < n; q += 32) rids2[q] = V.rids[list[2 * q]];
      __syncwarp();  // tmp (the positions) is read across lanes below
      uint32_t* Y2 = dst + region_rows_off(xlen, n);
      for (uint32_t g = 0; g < Wp2 / kGroupWords; ++g) {
        uint32_t tid[kGroupWords];
#pragma unroll
        for (uint32_t r = 0; r < kGroupWords; ++r) {
          const uint32_t q = (g * kGroupWords + r) * 32u + lane;
          tid[r] = q < supp ? tmp[q] : kFull;
        }
        for (uint32_t j0 = 0; j0 < n; j0 += 32) {
          const uint32_t nj = min(32u, n - j0);
          const uint32_t myrow = lane < nj ? list[2 * (j0 + lane)] : 0u;
          uint32_t mine[kGroupWords] = {0u, 0u, 0u, 0u};
          constexpr uint32_t U = 4;
          for (uint32_t jj = 0; jj < nj; jj += U) {
            uint32_t wv[U][kGroupWords];
#pragma unroll
            for (uint32_t u = 0; u < U; ++u) {
              const uint32_t rr = __shfl_sync(kFull, myrow, (jj + u) & 31);
              const bool ok = jj + u < nj;
              const uint32_t* rp = V.Y + (uint64_t)rr * V.Wp;
#pragma unroll
              for (uint32_t r = 0; r < kGroupWords; ++r) wv[u][r] = (ok && tid[r] != kFull) ? rp[tid[r] >> 5] : 0u;
            }
#pragma unroll
            for (uint32_t u = 0; u < U; ++u)
#pragma unroll
              for (uint32_t r = 0; r < kGroupWords; ++r) {
                const uint32_t y = __ballot_sync(kFull, (wv[u][r] >> (tid[r] & 31)) & 1u);
                if (lane == jj + u) mine[r] = y;
              }
          }
          if (lane < nj)
            *reinterpret_cast<uint4*>(Y2 + (uint64_t)(j0 + lane) * Wp2 + g * kGroupWords) =
                make_uint4(mine[0], mine[1], mine[2], mine[3]);
        }
      }
      __syncwarp();
    };

    // Hands the frame [X | list] to the other warps: X's database part in the shared arena and items
    // (region, m') for m' < n - 1 in the queue.  Returns false (nothing handed) when the queue is full; when
    // the queue had room but the arena not, the reserved slots carry no-op items.
    auto hand_out = [&](const RegionView& V, const uint32_t* pre, const uint32_t* list, uint32_t n, uint32_t xlen,
                        uint32_t supp, uint32_t* tmp) -> bool {
      uint32_t slot = 0;
      if (lane == 0) {
        atomicAdd(&p.ctrl->proj_pending, n - 1);  // before any of them is published
        slot = atomicAdd(&p.ctrl->dq_tail, n - 1);
      }
      slot = __shfl_sync(kFull, slot, 0);
      // slots at or past the capacity are never taken (tickets stop there); the ones below are published
      const uint32_t nres = slot >= p.dq_cap ? 0u : min(n - 1, p.dq_cap - slot);
      // (regions of the arena start on 128-byte lines of their own: a line read by one SM never holds
      // words that another warp writes later)
      const unsigned long long size =
          (region_rows_off(xlen, n) + (unsigned long long)n * padded_words(supp) + 31) & ~31ull;
      unsigned long long off = ~0ull;
      if (nres == n - 1) {
        if (lane == 0) off = atomicAdd(&p.ctrl->arena_top, size);
        off = __shfl_sync(kFull, off, 0);
        if (off + size > p.arena_words) off = ~0ull;
      }
      const bool fits = off != ~0ull;
      if (fits) build_region(Yar + off, V, pre, list, n, xlen, supp, tmp);
      __threadfence();
      __syncwarp();
      for (uint32_t t = lane; t < nres; t += 32) {
        uint32_t* sl = reinterpret_cast<uint32_t*>(p.dq + slot + t);
        sl[0] = (uint32_t)off;
        sl[1] = (uint32_t)(off >> 32);
        sl[2] = fits ? t : kNoop;
      }
      __threadfence();
      __syncwarp();
      for (uint32_t t = lane; t < nres; t += 32) atomicExch(&p.dq[slot + t].w, 1u);
      if (lane == 0 && nres < n - 1) atomicSub(&p.ctrl->proj_pending, (n - 1) - nres);  // never published
      if (fits) ++st_splits;
      return fits;
    };

    // support of a prefix: the popcount of its W words
    auto popc_of = [&](const uint32_t* pre, uint32_t W) {
      uint32_t c = 0;
      for (uint32_t w = lane; w < W; w += 32) c += __popc(pre[w]);
      return __reduce_add_sync(kFull, c);
    };

    // ---------------- depth-first walk: the item's node is child m of R0's own frame ----------------
    // frame 0: region R0, no prefix, every row; its only child expanded here is m
    if (lane == 0) {
      fr_R[0] = (unsigned long long)R0.R;
      fr_P[0] = 0ull;
      fr_L[0] = kIdentity;
      fr_n[0] = R0.k;
      fr_cur[0] = m;
      fr_top[0] = 0;
    }
    uint32_t top = 0;
    int32_t depth = 0;
    uint32_t since_poll = 0;
    bool overflow = false;
    uint64_t need = 0;
    bool first = true;
    while (depth >= 0) {
      __syncwarp();
      const uint32_t kk = fr_cur[depth], nf = fr_n[depth];
      // frame 0 of an item expands its child m only
      if (kk + 1 >= nf || (depth == 0 && !first)) {
        top = fr_top[depth];
        --depth;
        continue;
      }
      first = false;
      if (++since_poll == 8) {
        since_poll = 0;
        uint32_t stop = 0;
        if (lane == 0) {
          const uint32_t e = ld_volatile(&p.ctrl->err);  // (in flight with the add below)
          if (pend_sets) {
            const unsigned long long after = (atomicAdd(&p.ctrl->packed, pend_sets << 32) >> 32) + pend_sets;
            if ((p.max_sets && after > p.max_sets) || after > 0xfffffff0ull) {
              atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
              stop = 1;
            }
          }
          stop |= e & kStop;
        }
        pend_sets = 0;
        if (__shfl_sync(kFull, stop, 0)) break;
      }
      __syncwarp();
      if (lane == 0) fr_cur[depth] = kk + 1;
      const RegionView V = region_view(reinterpret_cast<const uint32_t*>(fr_R[depth]));
      if (fr_P[depth] == kDiffFrame) {
        // A frame [X | S] held as diffsets (dEclat, App. B.4.3): survivor s has the list of the nonzero words
        // of d(X u {s}) = t(X) \ t(X u {s}) over the region's words.  Child X' = X u {s_k}: its diffset is
        // scattered into a dense W-word bitmap dK; for every later survivor s_j, d(X' u {s_j}) = d(X u {s_j}) \
        // d(X') (the list filtered by dK) and supp(X' u {s_j}) = supp(X') - |d(X' u {s_j})|.
        const uint32_t* ent = stk + fr_L[depth];  // per survivor: row, support, list offset, list entries
        const uint32_t sj = ent[4 * kk], supp_k = ent[4 * kk + 1];
        const uint32_t* Lk = stk + ent[4 * kk + 2];
        const uint32_t lenk = ent[4 * kk + 3];
        const uint32_t plen = (uint32_t)(R0.xlen + depth);
        const uint32_t ncc = nf - kk - 1;
        if (plen + 1 >= L1) {
          if (lane == 0) atomicOr(&p.ctrl->err, DEV_ERR_DEPTH);
          break;
        }
        if (lane == 0) path[plen] = V.rids[sj];
        sort_path(plen + 1);
        uint32_t sumlen = 0;  // list entries of the candidates: the filtered lists take at most as many
        for (uint32_t t = lane; t < ncc; t += 32) sumlen += ent[4 * (kk + 1 + t) + 3];
        sumlen = __reduce_add_sync(kFull, sumlen);
        const uint64_t words = (uint64_t)V.Wp + 4ull * ncc + 2ull * sumlen;
        if ((uint64_t)top + words + 3 > p.pstack_words) {
          need = (uint64_t)top + words + 3;
          overflow = true;
          break;
        }
        uint32_t* dK = stk + top;
        for (uint32_t w = lane; w < V.W; w += 32) dK[w] = 0u;
        __syncwarp();
        for (uint32_t e = lane; e < lenk; e += 32) dK[Lk[2 * e]] = Lk[2 * e + 1];
        __syncwarp();
        uint32_t* ent2 = dK + V.Wp;
        const uint32_t lists2 = top + V.Wp + 4 * ncc;  // stack offset of the filtered lists
        uint32_t nout = 0, carry = 0;
        for (uint32_t t0 = 0; t0 < ncc; t0 += 32) {
          const uint32_t t = t0 + lane;
          const bool ok = t < ncc;
          const uint32_t* ej = ent + 4 * (kk + 1 + (ok ? t : 0));
          const uint32_t len = ok ? ej[3] : 0u;
          // this lane's filtered list goes after the lists of the lanes before it (old lengths: an upper bound)
          uint32_t incl = len;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= (uint32_t)o) incl += y;
          }
          const uint32_t doff = lists2 + 2 * (carry + incl - len);
          carry += __shfl_sync(kFull, incl, 31);
          uint32_t cnt = 0, dsz = 0;
          if (ok) {
            const uint32_t* Lj = stk + ej[2];
            uint32_t* dst = stk + doff;
            for (uint32_t e = 0; e < len; ++e) {
              const uint32_t w = Lj[2 * e];
              const uint32_t r = Lj[2 * e + 1] & ~dK[w];
              dsz += __popc(r);
              if (r) {
                dst[2 * cnt] = w;
                dst[2 * cnt + 1] = r;
                ++cnt;
              }
            }
          }
          const uint32_t sn = ok ? supp_k - dsz : 0u;
          const bool f = ok && sn >= p.minsup;
          const uint32_t bal = __ballot_sync(kFull, f);
          if (f) {
            uint32_t* e2 = ent2 + 4 * (nout + __popc(bal & ((1u << lane) - 1u)));
            e2[0] = ej[0];
            e2[1] = sn;
            e2[2] = doff;
            e2[3] = cnt;
          }
          nout += __popc(bal);
        }
        st_inter += ncc;
        cls_work += ncc;
        ++st_nodes;
        st_bytes += 8ull * (lenk + sumlen) + 4ull * V.W;
        emit(V, ent2, 4, nout, plen + 1, supp_k);
        if (nout >= 2) {
          ++st_frames;
          ++depth;
          if (lane == 0) {
            fr_R[depth] = fr_R[depth - 1];
            fr_P[depth] = kDiffFrame;
            fr_L[depth] = top + V.Wp;
            fr_n[depth] = nout;
            fr_cur[depth] = 0;
            fr_top[depth] = top;
          }
          top = (uint32_t)(((uint64_t)top + words + 3) & ~3ull);
        }
        continue;
      }
      const uint32_t* P = reinterpret_cast<const uint32_t*>(fr_P[depth]);
      const uint32_t lo = fr_L[depth];
      const uint32_t* list = lo == kIdentity ? nullptr : stk + lo;
      const uint32_t sj = list ? list[2 * kk] : kk;
      // the frame's prefix has length xlen; the child X u {s_j} has xlen + 1
      const uint32_t xlen = depth == 0 ? V.xlen : 0u;  // (deeper frames: set below from the path length)
      (void)xlen;
      const uint32_t plen = (uint32_t)(R0.xlen + depth);  // ids on the path before the child's item
      const uint32_t ncc = nf - kk - 1;
      if (plen + 1 >= L1) {  // longer than the longest transaction: cannot happen for a frequent itemset
        if (lane == 0) atomicOr(&p.ctrl->err, DEV_ERR_DEPTH);
        break;
      }
      if (lane == 0) path[plen] = V.rids[sj];
      sort_path(plen + 1);
      // the child's prefix: row s_j of the region, ANDed with the frame's prefix when it has one
      const uint32_t* yj = V.Y + (uint64_t)sj * V.Wp;
      const uint32_t* cpre = yj;
      uint32_t used = 0;  // stack words taken by the materialised prefix
      if (P) {
        if ((uint64_t)top + V.Wp + 2ull * ncc > p.pstack_words) {
          need = (uint64_t)top + V.Wp + 2ull * ncc;
          overflow = true;
          break;
        }
        uint32_t* cp = stk + top;
        for (uint32_t w = lane; w < V.W; w += 32) {
          const uint32_t a = P[w];
          cp[w] = a ? a & yj[w] : 0u;
        }
        __syncwarp();
        cpre = cp;
        used = V.Wp;
      } else if ((uint64_t)top + 2ull * ncc > p.pstack_words) {
        need = (uint64_t)top + 2ull * ncc;
        overflow = true;
        break;
      }
      uint32_t* lst = stk + top + used;
      const uint32_t n2 =
          count_node(V, cpre, list ? list + 2 * (kk + 1) : nullptr, kk + 1, ncc, lst, plen + 1);
      if (n2 < 2) continue;
      ++st_frames;
      // the child becomes a frame: hand it out, compact it, or keep it in the region's space
      const uint32_t supp = popc_of(cpre, V.W);
      const uint32_t W2 = words_of(supp);
      // (stack allocations are whole 16-byte units: a compacted region's rows are written as 16-byte vectors)
      const uint64_t after_list = ((uint64_t)top + used + 2ull * n2 + 3) & ~3ull;
      // diffsets (dEclat) when asked, or when they are at most a quarter of the bitmaps: every survivor s gets
      // the list of the nonzero words of t(X) \ t(X u {s}) = cpre & ~Y[s] over the region's words
      bool diff = p.diffsets == 2;
      if (p.diffsets == 1) {
        uint64_t dtids = 0;  // sum of the diffset sizes (an upper bound of their nonzero words)
        for (uint32_t q = lane; q < n2; q += 32) dtids += supp - lst[2 * q + 1];
        for (int o = 16; o > 0; o >>= 1) dtids += __shfl_xor_sync(kFull, dtids, o);
        diff = 8 * dtids <= (uint64_t)n2 * V.W;
      }
      if (diff) {
        const uint64_t ent0 = ((uint64_t)top + used + 2ull * n2 + 3) & ~3ull;  // entries after the survivor list
        uint64_t lp = ent0 + 4ull * n2;                                       // lists after the entries
        for (uint32_t q = 0; q < n2 && !overflow; ++q) {
          if (lp + 2ull * V.W > p.pstack_words) {
            need = lp + 2ull * V.W;
            overflow = true;
            break;
          }
          const uint32_t* ys = V.Y + (uint64_t)lst[2 * q] * V.Wp;
          uint32_t cnt = 0;
          for (uint32_t w0 = 0; w0 < V.W; w0 += 32) {
            const uint32_t w = w0 + lane;
            const uint32_t r = w < V.W ? cpre[w] & ~ys[w] : 0u;
            const uint32_t bal = __ballot_sync(kFull, r != 0u);
            if (r) {
              uint32_t* d = stk + lp + 2 * (cnt + __popc(bal & ((1u << lane) - 1u)));
              d[0] = w;
              d[1] = r;
            }
            cnt += __popc(bal);
          }
          if (lane == 0) {
            uint32_t* e = stk + ent0 + 4 * q;
            e[0] = lst[2 * q];
            e[1] = lst[2 * q + 1];
            e[2] = (uint32_t)lp;
            e[3] = cnt;
          }
          st_bytes += 8ull * V.W;
          lp += 2ull * cnt;
        }
        if (overflow) break;
        __syncwarp();
        ++depth;
        if (lane == 0) {
          fr_R[depth] = fr_R[depth - 1];
          fr_P[depth] = kDiffFrame;
          fr_L[depth] = (uint32_t)ent0;
          fr_n[depth] = n2;
          fr_cur[depth] = 0;
          fr_top[depth] = top;
        }
        top = (uint32_t)((lp + 3) & ~3ull);
        continue;
      }
      // hand the frame out when its next level is large: more words than split_words (given, or 64 x the mean
      // bitmap width of the class regions, set by the planning kernel)
      const unsigned long long work = (unsigned long long)n2 * (n2 - 1) / 2 * W2;
      if (p.dq_cap && n2 >= 3 && work > split_words && after_list + supp <= p.pstack_words &&
          hand_out(V, cpre, lst, n2, plen + 1, supp, stk + after_list))
        continue;
      // compact: X's own database part on the stack, when it is at most a quarter of the region's width and
      // the frame has at least six children to share the cost of building it (large_sparse: 5.1 ms against
      // 6.3 ms when every frame of two or more is compacted, 5.5 ms at an eighth of the width)
      if ((uint64_t)W2 * 4 <= V.W && n2 >= 6) {
        const uint64_t size = region_rows_off(plen + 1, n2) + (uint64_t)n2 * padded_words(supp);
        if (after_list + size + supp > p.pstack_words) {
          need = after_list + size + supp;
          overflow = true;
          break;
        }
        uint32_t* dst = stk + after_list;
        build_region(dst, V, cpre, lst, n2, plen + 1, supp, dst + size);
        ++depth;
        if (lane == 0) {
          fr_R[depth] = (unsigned long long)dst;
          fr_P[depth] = 0ull;
          fr_L[depth] = kIdentity;
          fr_n[depth] = n2;
          fr_cur[depth] = 0;
          fr_top[depth] = top;
        }
        top = (uint32_t)(after_list + size);
      } else {  // the frame stays in the region's space, its prefix materialised or a row of the region
        ++depth;
        if (lane == 0) {
          fr_R[depth] = fr_R[depth - 1];
          fr_P[depth] = (unsigned long long)cpre;
          fr_L[depth] = top + used;
          fr_n[depth] = n2;
          fr_cur[depth] = 0;
          fr_top[depth] = top;
        }
        top = (uint32_t)after_list;
      }
    }
    if (overflow && lane == 0) {
      atomicMax(&p.ctrl->pstack_need, need > 0xffffffffull ? 0xffffffffu : (uint32_t)need);
      atomicOr(&p.ctrl->err, DEV_ERR_PSTACK);
    }
    if (lane == 0) {
      if (pend_sets) atomicAdd(&p.ctrl->packed, pend_sets << 32);  // (read at the next acquire)
      if (p.class_sets && cls_sets) atomicAdd(&p.class_sets[cls], cls_sets);
      if (p.class_work && cls_work) atomicAdd(&p.class_work[cls], cls_work);
      __threadfence();  // the item's records and published children before its completion
      atomicSub(&p.ctrl->proj_pending, 1u);
    }
    pend_sets = 0;
  }
  if (lane == 0) {
    atomicAdd(&p.ctrl->n_intersections, st_inter);
    atomicAdd(&p.ctrl->n_nodes, st_nodes);
    atomicAdd(&p.ctrl->n_frames, st_frames);
    if (st_splits) atomicAdd(&p.ctrl->proj_splits, (uint32_t)st_splits);
    atomicAdd(&p.ctrl->proj_bytes, st_bytes);
    if (st_sets) {
      atomicAdd(&p.ctrl->sets_total, st_sets);
      atomicAdd(&p.ctrl->items_total, st_items);
      atomicMax(&p.ctrl->max_len, st_maxlen);
    }
  }
  if (p.cta_time) {
    __syncthreads();
    if (threadIdx.x == 0) p.cta_time[2 * blockIdx.x + 1] = global_ns();
  }
}

// dynamic shared-memory limit of the DFS kernel raised once per device (launches pass their own size)
cudaError_t allow_proj_smem() { return kernel_smem_limit(reinterpret_cast<const void*>(k_dfs_proj), -1); }

}  // namespace

cudaError_t launch_proj_plan(const ProjLaunch& q, cudaStream_t st) {
  k_proj_plan<<<1, 1024, 0, st>>>(q);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_proj_build(const ProjLaunch& q, int num_sms, cudaStream_t st) {
  if (q.n1 == 0) return cudaSuccess;
  k_proj_tids<<<q.n1, 256, 0, st>>>(q);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_proj_bits<<<(unsigned)num_sms * 8u, 256, 0, st>>>(q);
  note_launch();
  return cudaGetLastError();
}

size_t dfs_proj_smem_bytes(uint32_t max_len) {
  return (size_t)(kProjThreads / 32) * 10ull * (max_len + 1) * sizeof(uint32_t);
}

cudaError_t dfs_proj_ctas_per_sm(size_t smem, int* out) {
  cudaError_t e = allow_proj_smem();
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_dfs_proj, (int)kProjThreads, smem);
  if (e == cudaSuccess) *out = std::min<int>(*out, (int)kProjCtasPerSm);
  return e;
}

cudaError_t launch_dfs_proj(const DfsLaunch& p, uint32_t grid, uint32_t max_len, cudaStream_t st) {
  cudaError_t e = allow_proj_smem();
  if (e != cudaSuccess) return e;
  k_dfs_proj<<<grid, kProjThreads, dfs_proj_smem_bytes(max_len), st>>>(p, max_len);
  note_launch();
  return cudaGetLastError();
}

}  // namespace fim
