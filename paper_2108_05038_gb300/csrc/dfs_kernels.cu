// Level-2 survivors, the persistent prefix-class queue, and K4: the persistent
// depth-first Eclat kernel.
//
// Eclat-DFS-Computation (App. B.3.2), restated for bitmaps: a class node is a
// prefix X with its bitmap t(X) and an ordered candidate list E; its step
// counts c_e = popc(t(X) & t({e})) for every e in E (support of X u {e} from
// two generating subsets, App. B.3.1), keeps the survivors S = {e : c_e >=
// minsup}, outputs X u {e} for e in S, and expands the children
// [X u {s_k} | s_{k+1} ...] (the PBEC split of Sec. 2.4).  t(X u {s}) is
// materialised only for children that have children themselves.
//
// Level 2 comes from the pair kernel.  The classes with two-item prefixes
// [(i, s_m) | S_i after s_m] form the static queue of the persistent kernel,
// grouped by their top class [i] and ordered by the queue order of the top
// classes (LPT on the sample estimate, Sec. 8.2, or the item order).  Each
// persistent CTA pops a class and runs its whole subtree depth first with a
// private stack (the tidlist cache C of Prepare-Tidlists, Ch. 9, holds one
// prefix bitmap per depth).  When CTAs run idle, busy CTAs hand them the
// next unexpanded child of their shallowest open frame through a bounded
// pool (the dynamic load balancing of the thesis's Phase 1, restated for a
// device work queue); a counter of unfinished entries detects termination.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fim_internal.cuh"

namespace fim {
namespace {

constexpr uint32_t kDensePrefix = 0xffffffffu;  // stack slot header: the prefix is stored dense
constexpr uint32_t kSparseCap = 2048;  // sparse node mode: listed words of a shared-memory prefix (36 KB)
constexpr uint32_t kCandBatch = 1024;  // candidates counted per pass (shared-memory counters)

// Exclusive block-wide scan of a 0/1 flag.  wtot: 33 shared words.  Returns
// this thread's position among the set flags; *total = number of set flags.
// Contains two barriers; the caller must barrier before reusing wtot.
__device__ __forceinline__ uint32_t block_flag_scan(bool flag, uint32_t* wtot, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t ballot = __ballot_sync(0xffffffffu, flag);
  const uint32_t wpos = __popc(ballot & ((1u << lane) - 1u));
  if (lane == 0) wtot[warp] = __popc(ballot);
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < nw ? wtot[lane] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += u;
    }
    if (lane < nw) wtot[lane] = incl - v;
    if (lane == 31) wtot[32] = incl;
  }
  __syncthreads();
  *total = wtot[32];
  return wtot[warp] + wpos;
}

// ---------------------------------------------------------------------------
// level-2 post-processing

// (pair counts left incomplete by a timed-out pair kernel count as no survivors, so nothing below
// runs on them; the call then reports the timeout)
__global__ void k_surv_count(const uint32_t* __restrict__ C2, uint32_t n1, uint32_t minsup,
                             uint32_t* __restrict__ scnt, const DevCtrl* ctrl) {
  const uint32_t i = blockIdx.x;
  const bool failed = (*(volatile const uint32_t*)&ctrl->err & DEV_ERR_TIMEOUT) != 0;
  uint32_t c = 0;
  for (uint32_t j = i + 1 + threadIdx.x; j < n1 && !failed; j += blockDim.x) c += C2[(size_t)i * n1 + j] >= minsup;
  c = __reduce_add_sync(0xffffffffu, c);
  __shared__ uint32_t ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) t += ws[w];
    scnt[i] = t;
  }
}

// One CTA: survivor offsets (row order), entry offsets (queue order), totals,
// and the initial state of the control block.
// The rows are frequent singletons, except in a count-only mine over rows not filtered by support (a
// sample whose supports stay on the device), where rows below minsup count as nothing.
__global__ void k_level2_scan(const uint32_t* __restrict__ scnt, const uint32_t* __restrict__ row_order, uint32_t n1,
                              const uint32_t* __restrict__ row_supp, uint32_t minsup, uint32_t* __restrict__ soff,
                              uint32_t* __restrict__ eoff, uint64_t cap_sets, uint64_t cap_items, DevCtrl* ctrl,
                              uint32_t leaves) {
  __shared__ uint32_t wtot[33];
  __shared__ uint32_t n_single;
  if (threadIdx.x == 0) n_single = 0;
  uint32_t my_single = 0;
  uint32_t carry_s = 0, carry_e = 0;
  for (uint32_t base = 0; base < n1; base += blockDim.x) {
    uint32_t i = base + threadIdx.x;
    if (i < n1 && row_supp[i] >= minsup) ++my_single;
    uint32_t vs = i < n1 ? scnt[i] : 0u;
    uint32_t q_row = i < n1 ? row_order[i] : 0u;
    uint32_t cq = i < n1 ? scnt[q_row] : 0u;
    uint32_t ve = cq > 0 ? cq - 1 : 0u;
    // two inclusive warp scans, then across warps
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t a = vs, b = ve;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t ua = __shfl_up_sync(0xffffffffu, a, o), ub = __shfl_up_sync(0xffffffffu, b, o);
      if (lane >= (uint32_t)o) { a += ua; b += ub; }
    }
    __shared__ uint32_t wa[32], wb[32];
    if (lane == 31) { wa[warp] = a; wb[warp] = b; }
    __syncthreads();
    if (warp == 0) {
      uint32_t x = lane < nw ? wa[lane] : 0u, y = lane < nw ? wb[lane] : 0u;
      uint32_t xi = x, yi = y;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t ux = __shfl_up_sync(0xffffffffu, xi, o), uy = __shfl_up_sync(0xffffffffu, yi, o);
        if (lane >= (uint32_t)o) { xi += ux; yi += uy; }
      }
      if (lane < nw) { wa[lane] = xi - x; wb[lane] = yi - y; }
      if (lane == 31) { wtot[0] = xi; wtot[1] = yi; }
    }
    __syncthreads();
    if (i < n1) {
      soff[i] = carry_s + wa[warp] + a - vs;
      eoff[i] = carry_e + wb[warp] + b - ve;
    }
    carry_s += wtot[0];
    carry_e += wtot[1];
    __syncthreads();
  }
  my_single = __reduce_add_sync(0xffffffffu, my_single);
  if ((threadIdx.x & 31) == 0 && my_single) atomicAdd(&n_single, my_single);
  __syncthreads();
  if (threadIdx.x == 0) {
    soff[n1] = carry_s;
    eoff[n1] = carry_e;
    const unsigned long long P = carry_s, n1f = n_single;
    // (leaves only: the records of levels 1 and 2 are reserved one by one by k_level2_leaves)
    const unsigned long long sets = leaves ? 0ull : n1f + P, items = leaves ? 0ull : n1f + 2 * P;
    ctrl->packed = (sets << 32) | items;
    ctrl->sets_total = sets;
    ctrl->items_total = items;
    ctrl->n_pairs = carry_s;
    ctrl->n_entries = carry_e;
    ctrl->pending = carry_e;
    ctrl->queue_head = 0;
    ctrl->max_len = leaves ? 0u : (n1f > 0 ? (P > 0 ? 2u : 1u) : 0u);
    if (cap_sets && (sets > cap_sets || items > cap_items)) ctrl->err |= DEV_ERR_OVERFLOW;  // 0: count only
  }
}

// One CTA per queue position q (row i = row_order[q]): survivors of row i in
// ascending column order, the pair records, the singleton record of row i and
// the queue entries (i, m) of its two-item prefix classes.
__global__ void k_level2_fill(const uint32_t* __restrict__ C2, uint32_t n1, uint32_t minsup,
                              const uint32_t* __restrict__ frows, const uint32_t* __restrict__ row_supp,
                              const uint32_t* __restrict__ rank_item, const uint32_t* __restrict__ row_order,
                              const uint32_t* __restrict__ scnt, const uint32_t* __restrict__ soff,
                              const uint32_t* __restrict__ eoff, uint32_t* __restrict__ sitems,
                              uint2* __restrict__ entries, uint64_t* __restrict__ out_off,
                              uint32_t* __restrict__ out_items, uint32_t* __restrict__ out_supp, uint64_t cap_sets,
                              uint64_t cap_items, unsigned long long* __restrict__ class_sets,
                              const uint32_t* __restrict__ eoffx, uint2* __restrict__ entries_f) {
  __shared__ uint32_t wtot[33];
  const uint32_t q = blockIdx.x;
  const uint32_t i = row_order[q];
  const uint32_t id_i = rank_item[frows[i]];
  // sets of class i found at levels 1 and 2: {i} and its frequent pairs (the DFS adds the rest)
  if (class_sets && threadIdx.x == 0) class_sets[i] = row_supp[i] >= minsup ? 1ull + scnt[i] : 0ull;
  if (threadIdx.x == 0 && out_off && i < cap_sets && i < cap_items) {
    out_off[i] = i;
    out_items[i] = id_i;
    out_supp[i] = row_supp[i];
  }
  const uint32_t ne = scnt[i] > 0 ? scnt[i] - 1 : 0u;
  // the projected DFS splits the entries into its own queue and the fallback queue (bit 31 of eoffx)
  const uint32_t ex = eoffx ? eoffx[q] : eoff[q];
  uint2* const dst = (eoffx && (ex & 0x80000000u)) ? entries_f : entries;
  const uint32_t e0 = eoffx ? (ex & 0x7fffffffu) : ex;
  for (uint32_t m = threadIdx.x; m < ne; m += blockDim.x) dst[e0 + m] = make_uint2(i, m);
  uint32_t pos0 = 0;
  for (uint32_t base = i + 1; base < n1; base += blockDim.x) {
    uint32_t j = base + threadIdx.x;
    uint32_t c = j < n1 ? C2[(size_t)i * n1 + j] : 0u;
    bool f = j < n1 && c >= minsup;
    uint32_t tot;
    uint32_t pos = block_flag_scan(f, wtot, &tot);
    if (f) {
      uint32_t k = soff[i] + pos0 + pos;
      sitems[k] = j;
      uint64_t rec = (uint64_t)n1 + k, it = (uint64_t)n1 + 2ull * k;
      if (out_off && rec < cap_sets && it + 2 <= cap_items) {
        uint32_t id_j = rank_item[frows[j]];
        out_off[rec] = it;
        out_items[it] = min(id_i, id_j);
        out_items[it + 1] = max(id_i, id_j);
        out_supp[rec] = c;
      }
    }
    pos0 += tot;
    __syncthreads();
  }
}

// Leaves of levels 1 and 2 (maximal output): one warp per row i that is frequent.  {i} is a leaf when no
// pair {i, j} is frequent; otherwise {i, s_last} (its last survivor, which has no later candidate) is one,
// while the other pairs are the DFS's class nodes and write their own leaves.
__global__ void k_level2_leaves(const uint32_t* __restrict__ C2, uint32_t n1, uint32_t minsup,
                                const uint32_t* __restrict__ frows, const uint32_t* __restrict__ row_supp,
                                const uint32_t* __restrict__ rank_item, const uint32_t* __restrict__ scnt,
                                const uint32_t* __restrict__ soff, const uint32_t* __restrict__ sitems,
                                uint64_t* __restrict__ out_off, uint32_t* __restrict__ out_items,
                                uint32_t* __restrict__ out_supp, uint64_t cap_sets, uint64_t cap_items, DevCtrl* ctrl) {
  const uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n1 || (threadIdx.x & 31) != 0) return;
  if (row_supp[i] < minsup) return;  // (a count-only mine over rows not filtered by support)
  const uint32_t k = scnt[i];
  const uint32_t id_i = rank_item[frows[i]];
  uint32_t len = 1, a = id_i, b = 0, sp = row_supp[i];
  if (k > 0) {
    const uint32_t j = sitems[soff[i] + k - 1];
    const uint32_t id_j = rank_item[frows[j]];
    len = 2;
    a = min(id_i, id_j);
    b = max(id_i, id_j);
    sp = C2[(size_t)i * n1 + j];
  }
  const unsigned long long base = atomicAdd(&ctrl->packed, (1ull << 32) | len);
  atomicAdd(&ctrl->sets_total, 1ull);
  atomicAdd(&ctrl->items_total, (unsigned long long)len);
  atomicMax(&ctrl->max_len, len);
  const uint64_t rec = base >> 32, it0 = base & 0xffffffffull;
  if (!out_off) return;
  if (rec < cap_sets && it0 + len <= cap_items) {
    out_items[it0] = a;
    if (len == 2) out_items[it0 + 1] = b;
    out_off[rec] = it0;
    out_supp[rec] = sp;
  } else {
    atomicOr(&ctrl->err, DEV_ERR_OVERFLOW);
  }
}

// ---------------------------------------------------------------------------
// K4: persistent DFS

struct Ctl {
  uint32_t kind;      // 0 exit, 1 static entry, 2 donated class from the ring
  uint32_t a, b;      // static entry (row index, m)
  uint32_t action;    // 1 expand child, 2 donate child, 3 frame exhausted, 4 class done
  uint32_t s_row, s_id, s_supp;
  uint32_t nc;        // candidates of the child
  uint32_t cand_off;  // their offset (entries) in the frame's list
  uint32_t fd;        // frame the donated child comes from
  int32_t depth;
  uint32_t xlen0;     // prefix length of the class's root node
  uint32_t slot;      // ring slot in use
  uint32_t rpos;      // ring position of that slot
  uint32_t cls;       // top class of the current entry (frow index of its first item)
  unsigned long long base;
};

struct DfsArgs {
  DfsLaunch p;
  uint32_t stride4;
  uint32_t nseg;       // pieces per candidate row
  uint32_t max_len;    // itemset length bound (entries of the path arrays)
  uint32_t cap;        // sparse node mode: nonzero 16-byte words a shared-memory prefix list holds
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// candidate list encodings
enum : uint32_t { CAND_FROW = 0, CAND_PAIR = 1, CAND_PAIR_RING = 2 };

__device__ __forceinline__ bool any4(const uint4& v) { return (v.x | v.y | v.z | v.w) != 0u; }

// Whether a traversal unwinds: a flagged abort, or (a count-only mine, which reserves no record positions and
// so checks its itemset limit here instead of at every node) a running total past the limit or the 32-bit
// record range, which is flagged here.  Both words are loaded before either is looked at.
__device__ __forceinline__ bool traversal_stopped(const DfsLaunch& p) {
  const unsigned long long t = p.out_off ? 0ull : *(volatile const unsigned long long*)&p.ctrl->sets_total;
  const uint32_t e = *(volatile const uint32_t*)&p.ctrl->err;
  if (e & DEV_ERR_ABORTED) return true;
  if ((p.max_sets && t > p.max_sets) || t > 0xfffffff0ull) {
    atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
    return true;
  }
  return false;
}

// Sparse skipping: a prefix bitmap of support s over D transactions has at most
// s nonzero words, so wherever its 16 bytes are zero the candidate row is not
// read at all (its AND is zero there).  Prefixes deep in the DFS are much
// sparser than the rows, so this cuts the bytes read per intersection.  The
// prefix words of a piece are read first, all together, then the row words
// they need, all together: two round trips per piece, each with VEC loads in
// flight per lane.
template <int VEC>
__device__ __forceinline__ uint32_t piece_popc(const uint4* __restrict__ row, const uint4* pre, uint32_t base4,
                                               uint32_t stride4, bool pre_global) {
  uint4 b[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const uint32_t w = base4 + v * 32;
    b[v] = w < stride4 ? (pre_global ? __ldcg(pre + w) : pre[w]) : make_uint4(0u, 0u, 0u, 0u);
  }
  uint4 a[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) a[v] = any4(b[v]) ? __ldg(row + base4 + v * 32) : make_uint4(0u, 0u, 0u, 0u);
  uint32_t s = 0;
#pragma unroll
  for (int v = 0; v < VEC; ++v)
    s += __popc(a[v].x & b[v].x) + __popc(a[v].y & b[v].y) + __popc(a[v].z & b[v].z) + __popc(a[v].w & b[v].w);
  return s;
}

// As piece_popc over the nonzero 16-byte words of a shared-memory prefix only,
// listed in nzl[0, nnz): a piece covers 32 * VEC list entries, so a prefix with
// a fraction f of nonzero words costs f of the dense pieces, one round trip each.
// The word values come from the dense prefix pre[nzl[e]], or from vals[e] when the
// prefix is held as a list of (index, value) pairs only.
template <int VEC>
__device__ __forceinline__ uint32_t piece_popc_list(const uint4* __restrict__ row, const uint4* pre,
                                                    const uint16_t* nzl, uint32_t nnz, uint32_t base,
                                                    const uint4* vals) {
  uint32_t w[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const uint32_t e = base + v * 32;
    w[v] = e < nnz ? (uint32_t)nzl[e] : 0xffffffffu;
  }
  uint4 a[VEC], b[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const bool ok = w[v] != 0xffffffffu;
    b[v] = ok ? (vals ? vals[base + v * 32] : pre[w[v]]) : make_uint4(0u, 0u, 0u, 0u);
    a[v] = ok ? __ldg(row + w[v]) : make_uint4(0u, 0u, 0u, 0u);
  }
  uint32_t s = 0;
#pragma unroll
  for (int v = 0; v < VEC; ++v)
    s += __popc(a[v].x & b[v].x) + __popc(a[v].y & b[v].y) + __popc(a[v].z & b[v].z) + __popc(a[v].w & b[v].w);
  return s;
}

// nzl[0, n) = ascending indices of the nonzero 16-byte words of pre4[0, stride4)
// (shared memory); every warp compacts one contiguous segment, ballots give the
// positions.  All threads call it; returns n in every thread.  wcnt: one word
// per warp of scratch.
__device__ __forceinline__ uint32_t build_nz_list(const uint4* pre4, uint32_t stride4, uint16_t* nzl, uint32_t* wcnt,
                                                  uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t seg = ((stride4 + nw - 1) / nw + 31) & ~31u;
  const uint32_t beg = min(stride4, warp * seg), end = min(stride4, beg + seg);
  uint32_t c = 0;
  for (uint32_t w0 = beg; w0 < end; w0 += 32) {
    const uint32_t w = w0 + lane;
    c += __popc(__ballot_sync(0xffffffffu, w < end && any4(pre4[w])));
  }
  if (lane == 0) wcnt[warp] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (uint32_t k = 0; k < nw; ++k) {
      const uint32_t t = wcnt[k];
      wcnt[k] = acc;
      acc += t;
    }
    *total = acc;
  }
  __syncthreads();
  uint32_t pos = wcnt[warp];
  for (uint32_t w0 = beg; w0 < end; w0 += 32) {
    const uint32_t w = w0 + lane;
    const bool nz = w < end && any4(pre4[w]);
    const uint32_t m = __ballot_sync(0xffffffffu, nz);
    if (nz) nzl[pos + __popc(m & ((1u << lane) - 1u))] = (uint16_t)w;
    pos += __popc(m);
  }
  __syncthreads();
  return *total;
}

// Block-wide dst[w] = a[w] & row[w] (and the same into dst2 when given), reading
// row[w] only where a[w] is nonzero; four words per thread in flight per round
// trip.  A_RO: `a` is read-only for the kernel's lifetime (a bitmap row), so it
// may go through the non-coherent cache; otherwise (a prefix this CTA wrote) it
// is read with plain loads.
template <bool A_RO>
__device__ __forceinline__ void and_rows(uint4* dst, uint4* dst2, const uint4* a4, const uint4* __restrict__ r4,
                                         uint32_t stride4) {
  constexpr uint32_t U = 4;
  for (uint32_t w0 = threadIdx.x; w0 < stride4; w0 += U * blockDim.x) {
    uint4 a[U], b[U];
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t w = w0 + u * blockDim.x;
      a[u] = w < stride4 ? (A_RO ? __ldg(a4 + w) : a4[w]) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) b[u] = any4(a[u]) ? __ldg(r4 + w0 + u * blockDim.x) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t w = w0 + u * blockDim.x;
      if (w < stride4) {
        const uint4 c = make_uint4(a[u].x & b[u].x, a[u].y & b[u].y, a[u].z & b[u].z, a[u].w & b[u].w);
        dst[w] = c;
        if (dst2) dst2[w] = c;
      }
    }
  }
}

__device__ __forceinline__ uint32_t cand_row(const DfsLaunch& p, const uint32_t* cand, uint32_t mode, uint32_t k) {
  if (mode == CAND_FROW) return p.frows[cand[k]];
  if (mode == CAND_PAIR) return cand[2 * k];
  return __ldcg(cand + 2 * k);
}

// Counts the candidates of one class node against its prefix bitmap, writes
// the survivors as (row, id) pairs in candidate order to out_list, and one
// output record per survivor.  All threads of the CTA call it; returns the
// survivor count (same value in every thread).
template <int VEC>
__device__ __forceinline__ uint32_t process_node(const DfsArgs& A, Ctl& C, uint32_t* cnt, uint32_t* wtot,
                                                 const uint32_t* xid, const uint32_t* pre, bool pre_global,
                                                 const uint32_t* cand, uint32_t mode, uint32_t nc, uint32_t* out_list,
                                                 uint32_t out_cap, uint32_t xlen, const uint16_t* nzl = nullptr,
                                                 uint32_t nnz = 0, const uint4* vals = nullptr,
                                                 uint32_t* out_supp = nullptr, uint32_t xsupp = 0) {
  const DfsLaunch& p = A.p;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint4* pre4 = reinterpret_cast<const uint4*>(pre);
  // pieces per candidate: over the nonzero-word list of the prefix when given, else over the row
  const uint32_t nseg = nzl ? (nnz + 32 * VEC - 1) / (32 * VEC) : A.nseg;
  uint32_t nsurv = 0;
  for (uint32_t b0 = 0; b0 < nc; b0 += kCandBatch) {
    const uint32_t nb = min(kCandBatch, nc - b0);
    for (uint32_t k = threadIdx.x; k < nb; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    const uint32_t total = nb * nseg;
    for (uint32_t pc = warp; pc < total; pc += nw) {
      const uint32_t k = pc / nseg, g = pc - k * nseg;
      const uint32_t row = cand_row(p, cand, mode, b0 + k);
      const uint4* rp = reinterpret_cast<const uint4*>(p.bits + (size_t)row * p.stride);
      uint32_t s = nzl ? piece_popc_list<VEC>(rp, pre4, nzl, nnz, g * 32 * VEC + lane, vals)
                       : piece_popc<VEC>(rp, pre4, g * 32 * VEC + lane, A.stride4, pre_global);
      s = __reduce_add_sync(0xffffffffu, s);
      if (lane == 0 && s) atomicAdd(&cnt[k], s);
    }
    __syncthreads();
    for (uint32_t c0 = 0; c0 < nb; c0 += blockDim.x) {
      const uint32_t k = c0 + threadIdx.x;
      const uint32_t ck = k < nb ? cnt[k] : 0u;
      const bool f = k < nb && ck >= p.minsup;
      uint32_t tot;
      const uint32_t pos = block_flag_scan(f, wtot, &tot);
      if (threadIdx.x == 0 && tot && !p.leaves) {
        const unsigned long long sets = tot, items = (unsigned long long)tot * (xlen + 1);
        if (p.out_off) {  // record positions (a count-only mine checks the itemset limit at its polls)
          C.base = atomicAdd(&p.ctrl->packed, (sets << 32) | items);
          const unsigned long long after = (C.base >> 32) + sets;
          if ((p.max_sets && after > p.max_sets) || after > 0xfffffff0ull) atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
        }
        atomicAdd(&p.ctrl->sets_total, sets);
        atomicAdd(&p.ctrl->items_total, items);
        atomicMax(&p.ctrl->max_len, xlen + 1);
        if (p.class_sets) atomicAdd(&p.class_sets[C.cls], sets);
      }
      __syncthreads();
      if (f) {
        const uint32_t row = cand_row(p, cand, mode, b0 + k);
        const uint32_t v = mode == CAND_FROW ? p.rank_item[row]
                                             : (mode == CAND_PAIR ? cand[2 * (b0 + k) + 1] : __ldcg(cand + 2 * (b0 + k) + 1));
        const uint32_t o = nsurv + pos;
        if (o < out_cap) {
          out_list[2 * o] = row;
          out_list[2 * o + 1] = v;
          if (out_supp) out_supp[o] = ck;
        } else {
          atomicOr(&p.ctrl->err, DEV_ERR_DEPTH);
        }
        const uint64_t rec = (C.base >> 32) + pos;
        const uint64_t it0 = (C.base & 0xffffffffull) + (uint64_t)pos * (xlen + 1);
        if (!p.out_off || p.leaves) {
          // count only, or leaves only (the node's one record follows): no records here
        } else if (rec < p.cap_sets && it0 + xlen + 1 <= p.cap_items) {
          uint32_t* dst = p.out_items + it0;
          uint32_t q = 0;
          bool placed = false;
          for (uint32_t x = 0; x < xlen; ++x) {
            const uint32_t u = xid[x];
            if (!placed && v < u) { dst[q++] = v; placed = true; }
            dst[q++] = u;
          }
          if (!placed) dst[q] = v;
          p.out_off[rec] = it0;
          p.out_supp[rec] = ck;
        } else {
          atomicOr(&p.ctrl->err, DEV_ERR_OVERFLOW);
        }
      }
      nsurv += tot;
      __syncthreads();
    }
  }
  // leaves only (maximal output): one record, X itself when no candidate survives, else X with its last
  // survivor, which has no later candidate
  if (p.leaves && threadIdx.x == 0) {
    const uint32_t len = nsurv ? xlen + 1 : xlen;
    const uint32_t v = nsurv ? out_list[2 * (nsurv - 1) + 1] : 0xffffffffu;
    const uint32_t sp = nsurv ? out_supp[nsurv - 1] : xsupp;
    const unsigned long long base = atomicAdd(&p.ctrl->packed, (1ull << 32) | len);
    atomicAdd(&p.ctrl->sets_total, 1ull);
    atomicAdd(&p.ctrl->items_total, (unsigned long long)len);
    atomicMax(&p.ctrl->max_len, len);
    const uint64_t rec = base >> 32, it0 = base & 0xffffffffull;
    if (p.out_off && rec < p.cap_sets && it0 + len <= p.cap_items) {
      uint32_t* dst = p.out_items + it0;
      uint32_t q = 0;
      bool placed = v == 0xffffffffu;
      for (uint32_t x = 0; x < xlen; ++x) {
        const uint32_t u = xid[x];
        if (!placed && v < u) { dst[q++] = v; placed = true; }
        dst[q++] = u;
      }
      if (!placed) dst[q] = v;
      p.out_off[rec] = it0;
      p.out_supp[rec] = sp;
    } else if (p.out_off) {
      atomicOr(&p.ctrl->err, DEV_ERR_OVERFLOW);
    }
  }
  return nsurv;
}

// xid = the ids of the current path xidp[0..len) in ascending order (ids are distinct)
__device__ __forceinline__ void sort_path_ids(const uint32_t* xidp, uint32_t len, uint32_t* xid) {
  for (uint32_t k = threadIdx.x; k < len; k += blockDim.x) {
    const uint32_t v = xidp[k];
    uint32_t r = 0;
    for (uint32_t q = 0; q < len; ++q) r += xidp[q] < v;
    xid[r] = v;
  }
}

// Bounded MPMC ring over the pool slots (after D. Vyukov's bounded queue):
// slot c carries a sequence word; a producer may fill slot (pos % cap) when
// seq == pos and publishes it with seq = pos + 1; a consumer may take it when
// seq == pos + 1 and frees it with seq = pos + cap.  Single thread callers.
__device__ bool ring_claim_for_fill(const DfsLaunch& p, uint32_t* slot, uint32_t* rpos) {
  uint32_t pos = *(volatile uint32_t*)&p.ctrl->ring_tail;
  for (int tries = 0; tries < 64; ++tries) {
    const uint32_t c = pos % p.pool_slots;
    const uint32_t seq = *(volatile uint32_t*)(p.pool + (size_t)c * p.pool_slot_words);
    const int32_t diff = (int32_t)(seq - pos);
    if (diff == 0) {
      const uint32_t old = atomicCAS(&p.ctrl->ring_tail, pos, pos + 1);
      if (old == pos) { *slot = c; *rpos = pos; return true; }
      pos = old;
    } else if (diff < 0) {
      return false;  // full
    } else {
      pos = *(volatile uint32_t*)&p.ctrl->ring_tail;
    }
  }
  return false;
}

__device__ bool ring_take(const DfsLaunch& p, uint32_t* slot, uint32_t* rpos) {
  uint32_t pos = *(volatile uint32_t*)&p.ctrl->ring_head;
  for (int tries = 0; tries < 64; ++tries) {
    const uint32_t c = pos % p.pool_slots;
    const uint32_t seq = *(volatile uint32_t*)(p.pool + (size_t)c * p.pool_slot_words);
    const int32_t diff = (int32_t)(seq - (pos + 1));
    if (diff == 0) {
      const uint32_t old = atomicCAS(&p.ctrl->ring_head, pos, pos + 1);
      if (old == pos) { __threadfence(); *slot = c; *rpos = pos; return true; }
      pos = old;
    } else if (diff < 0) {
      return false;  // empty
    } else {
      pos = *(volatile uint32_t*)&p.ctrl->ring_head;
    }
  }
  return false;
}

__global__ void k_pool_init(uint32_t* pool, uint32_t slots, uint64_t slot_words) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < slots; c += gridDim.x * blockDim.x)
    pool[(size_t)c * slot_words] = c;
}

template <int VEC, bool PSMEM>
__global__ void __launch_bounds__(512, 1) k_dfs(const DfsArgs A) {
  const DfsLaunch& p = A.p;
  if (p.cta_time && threadIdx.x == 0) p.cta_time[2 * blockIdx.x] = global_ns();
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ Ctl C;
  __shared__ uint32_t wtot[33];
  // dynamic shared memory: [prefix (PSMEM)] [cnt] [f_n] [f_cur] [xrow] [xidp] [xid]
  uint32_t* sp = smem;
  uint32_t* spre = PSMEM ? sp : nullptr;
  if (PSMEM) sp += p.stride;
  uint32_t* cnt = sp; sp += kCandBatch;
  uint32_t* f_n = sp; sp += p.maxd + 1;
  uint32_t* f_cur = sp; sp += p.maxd + 1;
  uint32_t* xrow = sp; sp += A.max_len + 1;
  uint32_t* xidp = sp; sp += A.max_len + 1;
  uint32_t* xid = sp; sp += A.max_len + 1;
  uint16_t* nzl = reinterpret_cast<uint16_t*>(sp);  // nonzero-word list of the shared prefix (PSMEM)
  __shared__ uint32_t nz_total;
  const uint64_t per_depth = dfs_arena_depth_words(p.stride, p.n1);
  const uint64_t lw = dfs_list_words(p.stride);
  uint32_t* const arena = p.arena + (size_t)blockIdx.x * p.arena_cta_words;
#define slot_pre(d) (arena + (size_t)(d) * per_depth)
#define slot_hdr(d) (arena + (size_t)(d) * per_depth + p.stride)
#define slot_list(d) (arena + (size_t)(d) * per_depth + p.stride + lw)
  // Wide prefixes (more than four 16-byte words per thread) held in shared memory get the list of
  // their nonzero words: counting runs over it when at most half of the words are nonzero, and such
  // a prefix is saved on the stack as (list, values) so that its children read only those words.
  const bool use_lists = PSMEM && A.stride4 > 4u * blockDim.x;
  auto node_list = [&](uint32_t nc, uint32_t* nn) -> const uint16_t* {
    if (!use_lists || nc == 0) return nullptr;
    const uint32_t n = build_nz_list(reinterpret_cast<const uint4*>(spre), A.stride4, nzl, wtot, &nz_total);
    *nn = n;
    return 2 * n <= A.stride4 ? nzl : nullptr;
  };
  // stack slot d <- the shared prefix (after process_node of that node; the list is still valid)
  auto save_prefix = [&](uint32_t d) {
    uint32_t* hdr = slot_hdr(d);
    const uint32_t n = nz_total;
    uint4* gv = reinterpret_cast<uint4*>(slot_pre(d));
    const uint4* s4 = reinterpret_cast<const uint4*>(spre);
    if (use_lists && 2 * n <= A.stride4) {
      uint16_t* gl = reinterpret_cast<uint16_t*>(hdr + 4);
      if (threadIdx.x == 0) hdr[0] = n;
      for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
        const uint32_t w = nzl[e];
        gl[e] = (uint16_t)w;
        gv[e] = s4[w];
      }
    } else {
      if (threadIdx.x == 0) hdr[0] = kDensePrefix;
      for (uint32_t w = threadIdx.x; w < A.stride4; w += blockDim.x) gv[w] = s4[w];
    }
  };
  // dst <- (prefix of slot d) & row r4, dense image; dst is shared memory or a ring slot
  auto child_prefix = [&](uint4* dst, uint32_t d, const uint4* r4) {
    const uint32_t* hdr = slot_hdr(d);
    const uint32_t n = PSMEM ? *(volatile const uint32_t*)hdr : kDensePrefix;
    const uint4* gv = reinterpret_cast<const uint4*>(slot_pre(d));
    if (n == kDensePrefix) {
      and_rows<false>(dst, nullptr, gv, r4, A.stride4);
      return;
    }
    const uint16_t* gl = reinterpret_cast<const uint16_t*>(hdr + 4);
    for (uint32_t w = threadIdx.x; w < A.stride4; w += blockDim.x) dst[w] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    constexpr uint32_t U = 4;
    for (uint32_t e0 = threadIdx.x; e0 < n; e0 += U * blockDim.x) {
      uint32_t w[U];
      uint4 v[U], b[U];
#pragma unroll
      for (uint32_t u = 0; u < U; ++u) {
        const uint32_t e = e0 + u * blockDim.x;
        w[u] = e < n ? (uint32_t)gl[e] : 0xffffffffu;
        v[u] = e < n ? gv[e] : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (uint32_t u = 0; u < U; ++u) b[u] = w[u] != 0xffffffffu ? __ldg(r4 + w[u]) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (uint32_t u = 0; u < U; ++u)
        if (w[u] != 0xffffffffu)
          dst[w[u]] = make_uint4(v[u].x & b[u].x, v[u].y & b[u].y, v[u].z & b[u].z, v[u].w & b[u].w);
    }
  };

  const uint32_t list_cap = p.n1;
  const uint4* bits4 = reinterpret_cast<const uint4*>(p.bits);
  const uint32_t L = A.max_len;
  const uint64_t sw = p.pool_slot_words;

  unsigned long long st_inter = 0, st_frames = 0, st_don = 0;
  bool static_done = false;
  uint32_t idle_hint = 0, ready_hint = 0;  // last seen pool state (thread 0)

  for (;;) {
    // ---------------- acquire a class ----------------
    if (threadIdx.x == 0) {
      C.kind = 0;
      if (*(volatile uint32_t*)&p.ctrl->err & DEV_ERR_ABORTED) static_done = true;
      if (p.max_sets && *(volatile unsigned long long*)&p.ctrl->sets_total > p.max_sets) {
        atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
        static_done = true;
      }
      if (!static_done) {
        const uint32_t e = atomicAdd(&p.ctrl->queue_head, 1u);
        if (e < p.ctrl->n_entries) {
          const uint2 en = p.entries[e];
          C.kind = 1; C.a = en.x; C.b = en.y; C.cls = en.x;
        } else {
          static_done = true;
        }
      }
      if (C.kind == 0 && p.donate) {
        bool idle = false;
        unsigned long long spins = 0;
        uint32_t backoff = 32;
        uint32_t last = *(volatile uint32_t*)&p.ctrl->progress;
        for (;;) {
          uint32_t slot, rpos;
          if (ring_take(p, &slot, &rpos)) {
            atomicSub(&p.ctrl->n_ready, 1u);
            C.kind = 2; C.slot = slot; C.rpos = rpos;
            break;
          }
          if (*(volatile uint32_t*)&p.ctrl->pending == 0) break;
          if (*(volatile uint32_t*)&p.ctrl->err & (DEV_ERR_TIMEOUT | DEV_ERR_ABORTED)) break;
          if (!idle) { atomicAdd(&p.ctrl->n_idle, 1u); idle = true; }
          __nanosleep(backoff);
          if (backoff < 1024) backoff <<= 1;
          const uint32_t prog = *(volatile uint32_t*)&p.ctrl->progress;
          if (prog != last) { last = prog; spins = 0; }
          if (++spins > p.spin_limit) { atomicOr(&p.ctrl->err, DEV_ERR_TIMEOUT); break; }
        }
        if (idle) atomicSub(&p.ctrl->n_idle, 1u);
      }
    }
    __syncthreads();
    if (C.kind == 0) break;

    // ---------------- root node of the class ----------------
    const uint32_t* cand;
    uint32_t nc, mode;
    const uint32_t* pre;
    bool pre_global = false;
    uint32_t* slotp = nullptr;
    if (C.kind == 1) {
      const uint32_t i = C.a, m = C.b;
      const uint32_t base = p.soff[i];
      const uint32_t si = p.sitems[base + m];
      const uint32_t r1 = p.frows[i], r2 = p.frows[si];
      cand = p.sitems + base + m + 1;
      nc = p.scnt[i] - m - 1;
      mode = CAND_FROW;
      if (threadIdx.x == 0) { xrow[0] = r1; xidp[0] = p.rank_item[r1]; C.xlen0 = 2; }
      if (threadIdx.x == 1) { xrow[1] = r2; xidp[1] = p.rank_item[r2]; }
      const uint4* a4 = bits4 + (size_t)r1 * A.stride4;
      const uint4* b4 = bits4 + (size_t)r2 * A.stride4;
      uint4* dst = reinterpret_cast<uint4*>(PSMEM ? spre : slot_pre(0));
      and_rows<true>(dst, nullptr, a4, b4, A.stride4);
      pre = PSMEM ? spre : slot_pre(0);
    } else {
      slotp = p.pool + (size_t)C.slot * sw;
      const uint32_t xl = __ldcg(slotp + 1);
      nc = __ldcg(slotp + 2);
      for (uint32_t k = threadIdx.x; k < xl; k += blockDim.x) {
        xrow[k] = __ldcg(slotp + kDfsSlotHeader + k);
        xidp[k] = __ldcg(slotp + kDfsSlotHeader + L + k);
      }
      if (threadIdx.x == 0) { C.xlen0 = xl; C.cls = __ldcg(slotp + 3); }
      cand = slotp + kDfsSlotHeader + 2 * L;
      mode = CAND_PAIR_RING;
      const uint32_t* spref = slotp + (sw - p.stride);
      if (PSMEM) {
        const uint4* s4 = reinterpret_cast<const uint4*>(spref);
        uint4* d4 = reinterpret_cast<uint4*>(spre);
        for (uint32_t w = threadIdx.x; w < A.stride4; w += blockDim.x) d4[w] = __ldcg(s4 + w);
        pre = spre;
      } else {
        pre = spref;
        pre_global = true;
      }
    }
    __syncthreads();
    const uint32_t xlen0 = C.xlen0;
    sort_path_ids(xidp, xlen0, xid);
    __syncthreads();
    if (threadIdx.x == 0) {
      st_inter += nc;
      if (p.class_work) atomicAdd(&p.class_work[C.cls], (unsigned long long)nc);
    }
    uint32_t nnz = 0;
    const uint16_t* nl = node_list(nc, &nnz);
    const uint32_t ns = process_node<VEC>(A, C, cnt, wtot, xid, pre, pre_global, cand, mode, nc, slot_list(0),
                                          list_cap, xlen0, nl, nnz);
    if (ns >= 2) {
      // the root prefix goes to depth slot 0 (it is in shared memory or in the ring slot)
      if (PSMEM) {
        if (!use_lists) nz_total = 0;  // (no list: saved dense)
        save_prefix(0);
      } else if (C.kind == 2) {
        const uint4* s4 = reinterpret_cast<const uint4*>(pre);
        uint4* d4 = reinterpret_cast<uint4*>(slot_pre(0));
        for (uint32_t w = threadIdx.x; w < A.stride4; w += blockDim.x) d4[w] = __ldcg(s4 + w);
      }
    }
    if (threadIdx.x == 0) {
      atomicAdd(&p.ctrl->n_nodes, 1ull);
      atomicAdd(&p.ctrl->progress, 1u);
      if (ns >= 2) { f_n[0] = ns; f_cur[0] = 0; C.depth = 0; ++st_frames; }
      else C.depth = -1;
    }
    __syncthreads();
    if (C.kind == 2 && threadIdx.x == 0) {
      __threadfence();
      atomicExch(slotp, C.rpos + p.pool_slots);  // free the ring slot
    }

    // ---------------- depth-first expansion ----------------
    uint32_t cool = 0, poll = 0;
    for (;;) {
      __syncthreads();  // every thread has read the previous decision
      if (threadIdx.x == 0) {
        // a run past the itemset limit unwinds at once (every 8th node looks at the flag)
        if (C.depth >= 0 && (++poll & 7) == 0 && traversal_stopped(p)) C.depth = -1;
        const int32_t d = C.depth;
        C.action = 0;
        if (d < 0) {
          C.action = 4;
        } else {
          if (p.donate && cool == 0 && idle_hint > ready_hint) {
            for (int32_t fd = 0; fd <= d; ++fd) {
              if (f_n[fd] - 1 - f_cur[fd] >= 2) {
                uint32_t slot, rpos;
                if (ring_claim_for_fill(p, &slot, &rpos)) {
                  const uint32_t k = f_cur[fd];
                  C.action = 2; C.fd = fd; C.slot = slot; C.rpos = rpos;
                  C.s_row = slot_list(fd)[2 * k];
                  C.s_id = slot_list(fd)[2 * k + 1];
                  C.cand_off = k + 1;
                  C.nc = f_n[fd] - k - 1;
                  f_cur[fd] = k + 1;
                } else {
                  cool = 32;
                }
                break;
              }
            }
          }
          if (cool) --cool;
          if (C.action == 0) {
            if (f_cur[d] + 1 >= f_n[d]) {
              C.depth = d - 1;
              C.action = 3;
            } else if ((uint32_t)(d + 1) > p.maxd) {
              atomicOr(&p.ctrl->err, DEV_ERR_DEPTH);
              C.depth = -1;
              C.action = 3;
            } else {
              const uint32_t k = f_cur[d];
              C.action = 1;
              C.s_row = slot_list(d)[2 * k];
              C.s_id = slot_list(d)[2 * k + 1];
              C.cand_off = k + 1;
              C.nc = f_n[d] - k - 1;
              f_cur[d] = k + 1;
              xrow[xlen0 + d] = C.s_row;
              xidp[xlen0 + d] = C.s_id;
            }
          }
          if (p.donate) {  // read now, used at the next decision
            idle_hint = *(volatile uint32_t*)&p.ctrl->n_idle;
            ready_hint = *(volatile uint32_t*)&p.ctrl->n_ready;
          }
        }
      }
      __syncthreads();
      const uint32_t action = C.action;
      if (action == 4) break;
      if (action == 3) continue;
      if (action == 2) {
        // hand the child [X_fd u {s} | rest of frame fd] to an idle CTA
        const uint32_t fd = C.fd, ncd = C.nc, coff = C.cand_off;
        uint32_t* sl = p.pool + (size_t)C.slot * sw;
        const uint32_t xl = xlen0 + fd + 1;
        if (threadIdx.x == 0) { sl[1] = xl; sl[2] = ncd; sl[3] = C.cls; }
        for (uint32_t k = threadIdx.x; k < xl; k += blockDim.x) {
          sl[kDfsSlotHeader + k] = k + 1 < xl ? xrow[k] : C.s_row;
          sl[kDfsSlotHeader + L + k] = k + 1 < xl ? xidp[k] : C.s_id;
        }
        const uint32_t* src_list = slot_list(fd) + 2 * coff;
        for (uint32_t k = threadIdx.x; k < 2 * ncd; k += blockDim.x) sl[kDfsSlotHeader + 2 * L + k] = src_list[k];
        const uint4* r4 = bits4 + (size_t)C.s_row * A.stride4;
        child_prefix(reinterpret_cast<uint4*>(sl + (sw - p.stride)), fd, r4);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
          atomicAdd(&p.ctrl->pending, 1u);
          __threadfence();
          atomicExch(sl, C.rpos + 1);  // publish
          atomicAdd(&p.ctrl->n_ready, 1u);
          ++st_don;
        }
        continue;
      }
      // action 1: expand the child [X_d u {s} | rest of frame d]
      const int32_t d = C.depth;
      const uint32_t ncc = C.nc, coff = C.cand_off;
      const uint32_t xl = xlen0 + d + 1;  // prefix length of the child
      child_prefix(reinterpret_cast<uint4*>(PSMEM ? spre : slot_pre(d + 1)), d, bits4 + (size_t)C.s_row * A.stride4);
      sort_path_ids(xidp, xl, xid);
      __syncthreads();
      if (threadIdx.x == 0) {
        st_inter += ncc;
        if (p.class_work) atomicAdd(&p.class_work[C.cls], (unsigned long long)ncc);
      }
      uint32_t nnz2 = 0;
      const uint16_t* nl2 = node_list(ncc, &nnz2);
      const uint32_t n2 = process_node<VEC>(A, C, cnt, wtot, xid, PSMEM ? spre : slot_pre(d + 1), false,
                                            slot_list(d) + 2 * coff, CAND_PAIR, ncc, slot_list(d + 1), list_cap, xl,
                                            nl2, nnz2);
      if (n2 >= 2 && PSMEM) {
        if (!use_lists) nz_total = 0;
        save_prefix(d + 1);
      }
      if (threadIdx.x == 0) {
        atomicAdd(&p.ctrl->n_nodes, 1ull);
        atomicAdd(&p.ctrl->progress, 1u);
        if (n2 >= 2) { f_n[d + 1] = n2; f_cur[d + 1] = 0; C.depth = d + 1; ++st_frames; }
      }
    }
    // class finished
    if (threadIdx.x == 0) {
      __threadfence();
      atomicSub(&p.ctrl->pending, 1u);
    }
  }
  if (threadIdx.x == 0) {
    atomicAdd(&p.ctrl->n_intersections, st_inter);
    atomicAdd(&p.ctrl->n_frames, st_frames);
    atomicAdd(&p.ctrl->n_donations, st_don);
    if (p.cta_time) p.cta_time[2 * blockIdx.x + 1] = global_ns();
  }
#undef slot_pre
#undef slot_hdr
#undef slot_list
}

// ---------------------------------------------------------------------------
// K4, frame mode: the children of a frame are counted together.
//
// A frame is a class node X with its prefix bitmap t(X) and its survivor list
// L = [s_0, s_1, ...] (the items e with X u {e} frequent).  Its children are
// [X u {s_m} | s_{m+1} ...]; instead of expanding them one after the other,
// one pass counts every pair (m, e), m < e, as popc(t(X) & t({s_m}) &
// t({s_e})), i.e. the supports of the grandchildren X u {s_m, s_e} (two
// generating subsets X u {s_m} and {s_e}, App. B.3.1).  A pass covers up to
// kPairBatch pairs in child-major order, so the number of dependent steps of a
// class is about its depth instead of its number of nodes.  Child m is then
// entered as a frame with prefix t(X) & t({s_m}) when it has two or more
// survivors.  No donation in this mode.

constexpr uint32_t kPairBatch = kDfsPairBatch;

__device__ __forceinline__ uint64_t pair_base(uint32_t m, uint32_t n) {
  // pairs of children before child m in a frame of n items: sum_{k<m} (n - 1 - k)
  return (uint64_t)m * (n - 1) - (uint64_t)m * (m - 1) / 2;
}
// child m of pair p (largest m with pair_base(m) <= p), searched in [lo, hi)
__device__ __forceinline__ uint32_t pair_child(uint64_t p, uint32_t n, uint32_t lo, uint32_t hi) {
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (pair_base(mid, n) <= p) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Node expansion with sparse prefixes (FIM_DFS_SPARSE).  A prefix whose
// nonzero 16-byte words number at most A.cap lives in shared memory as a list
// of (index, value) pairs only (18 bytes per nonzero word instead of the whole
// row), so several small CTAs fit on an SM and their per-node barriers overlap;
// a denser prefix stays dense in its stack slot and is counted from there with
// sparse skipping.  Children of a listed prefix are built from its list alone:
// value & candidate row at the listed indices, zero results dropped.

// block-wide sum of one value per thread (wtot: 33 words of scratch); every thread gets the sum
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* wtot) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = __reduce_add_sync(0xffffffffu, v);
  if (lane == 0) wtot[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (uint32_t k = 0; k < nw; ++k) t += wtot[k];
    wtot[32] = t;
  }
  __syncthreads();
  const uint32_t t = wtot[32];
  __syncthreads();
  return t;
}

// dst[w] = a[w] & row[w] over the whole row (row read only under nonzero a); returns the number of
// nonzero results (block-wide).  A_RO as in and_rows.
template <bool A_RO>
__device__ __forceinline__ uint32_t and_rows_count(uint4* dst, const uint4* a4, const uint4* __restrict__ r4,
                                                   uint32_t stride4, uint32_t* wtot) {
  constexpr uint32_t U = 4;
  uint32_t c = 0;
  for (uint32_t w0 = threadIdx.x; w0 < stride4; w0 += U * blockDim.x) {
    uint4 a[U], b[U];
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t w = w0 + u * blockDim.x;
      a[u] = w < stride4 ? (A_RO ? __ldg(a4 + w) : a4[w]) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) b[u] = any4(a[u]) ? __ldg(r4 + w0 + u * blockDim.x) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t w = w0 + u * blockDim.x;
      if (w < stride4) {
        const uint4 v = make_uint4(a[u].x & b[u].x, a[u].y & b[u].y, a[u].z & b[u].z, a[u].w & b[u].w);
        dst[w] = v;
        c += any4(v) ? 1u : 0u;
      }
    }
  }
  return block_sum(c, wtot);
}

// append (w, v) to the shared list when v is nonzero: one shared atomic per warp and call
__device__ __forceinline__ void list_push(bool nz, uint32_t w, const uint4& v, uint16_t* sidx, uint4* sval,
                                          uint32_t* count) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t m = __ballot_sync(0xffffffffu, nz);
  uint32_t base = 0;
  if (lane == 0 && m) base = atomicAdd(count, (uint32_t)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (nz) {
    const uint32_t pos = base + __popc(m & ((1u << lane) - 1u));
    sidx[pos] = (uint16_t)w;
    sval[pos] = v;
  }
}

// as list_push, but entries past `cap` are only counted (the caller then falls back to a dense prefix)
__device__ __forceinline__ void list_push_capped(bool nz, uint32_t w, const uint4& v, uint16_t* sidx, uint4* sval,
                                                 uint32_t* count, uint32_t cap) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t m = __ballot_sync(0xffffffffu, nz);
  uint32_t base = 0;
  if (lane == 0 && m) base = atomicAdd(count, (uint32_t)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (nz) {
    const uint32_t pos = base + __popc(m & ((1u << lane) - 1u));
    if (pos < cap) {
      sidx[pos] = (uint16_t)w;
      sval[pos] = v;
    }
  }
}

// shared list <- the nonzero words of a[w] & row[w] (row read only under nonzero a); returns how many
// there are, which may exceed cap (then the list is incomplete)
template <bool A_RO>
__device__ __forceinline__ uint32_t and_rows_to_list(const uint4* a4, const uint4* __restrict__ r4, uint32_t stride4,
                                                     uint16_t* sidx, uint4* sval, uint32_t* count, uint32_t cap) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) *count = 0;
  __syncthreads();
  constexpr uint32_t U = 4;
  for (uint32_t w0 = warp * 32 * U; w0 < stride4; w0 += nw * 32 * U) {
    uint4 a[U], b[U];
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t w = w0 + u * 32 + lane;
      a[u] = w < stride4 ? (A_RO ? __ldg(a4 + w) : a4[w]) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) b[u] = any4(a[u]) ? __ldg(r4 + w0 + u * 32 + lane) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint4 v = make_uint4(a[u].x & b[u].x, a[u].y & b[u].y, a[u].z & b[u].z, a[u].w & b[u].w);
      list_push_capped(any4(v), w0 + u * 32 + lane, v, sidx, sval, count, cap);
    }
  }
  __syncthreads();
  return *count;
}

// shared list <- (listed prefix of a stack slot) & row, zero results dropped; eight entries per lane
// in flight (large_sparse: 0.5 ms less DFS time than two)
__device__ __forceinline__ uint32_t list_from_list(const uint16_t* gl, const uint4* gv, uint32_t n,
                                                   const uint4* __restrict__ r4, uint16_t* sidx, uint4* sval,
                                                   uint32_t* count) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) *count = 0;
  __syncthreads();
  constexpr uint32_t U = 8;
  for (uint32_t e0 = warp * 32 * U; e0 < n; e0 += nw * 32 * U) {
    uint32_t w[U];
    uint4 v[U];
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t e = e0 + u * 32 + lane;
      w[u] = e < n ? (uint32_t)gl[e] : 0xffffffffu;
      v[u] = e < n ? gv[e] : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint4 b = w[u] != 0xffffffffu ? __ldg(r4 + w[u]) : make_uint4(0u, 0u, 0u, 0u);
      v[u] = make_uint4(v[u].x & b.x, v[u].y & b.y, v[u].z & b.z, v[u].w & b.w);
    }
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) list_push(w[u] != 0xffffffffu && any4(v[u]), w[u], v[u], sidx, sval, count);
  }
  __syncthreads();
  return *count;
}

// at most 256 threads and 80 registers, so that three 256-thread CTAs (or five of 128) fit on an SM
template <int VEC>
__global__ void __launch_bounds__(256, 3) k_dfs_sparse(const DfsArgs A) {
  const DfsLaunch& p = A.p;
  if (p.cta_time && threadIdx.x == 0) p.cta_time[2 * blockIdx.x] = global_ns();
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ Ctl C;
  __shared__ uint32_t wtot[33];
  __shared__ uint32_t list_count;
  // dynamic shared memory: [values: cap x 16 B] [cnt] [f_n] [f_cur] [xrow] [xidp] [xid] [indices: cap x 2 B]
  uint4* sval = reinterpret_cast<uint4*>(smem);
  uint32_t* sp = smem + 4ull * A.cap;
  uint32_t* cnt = sp; sp += kCandBatch;
  uint32_t* f_n = sp; sp += p.maxd + 1;
  uint32_t* f_cur = sp; sp += p.maxd + 1;
  uint32_t* xrow = sp; sp += A.max_len + 1;
  uint32_t* xidp = sp; sp += A.max_len + 1;
  uint32_t* xid = sp; sp += A.max_len + 1;
  uint16_t* sidx = reinterpret_cast<uint16_t*>(sp);

  const uint64_t per_depth = dfs_arena_depth_words(p.stride, p.n1);
  const uint64_t lw = dfs_list_words(p.stride);
  uint32_t* const arena = p.arena + (size_t)blockIdx.x * p.arena_cta_words;
#define slot_pre(d) (arena + (size_t)(d) * per_depth)
#define slot_hdr(d) (arena + (size_t)(d) * per_depth + p.stride)
#define slot_list(d) (arena + (size_t)(d) * per_depth + p.stride + lw)
#define slot_supp(d) (arena + (size_t)(d) * per_depth + p.stride + lw + ((2ull * p.n1 + 3) & ~3ull))
  const uint32_t list_cap = p.n1;
  const uint4* bits4 = reinterpret_cast<const uint4*>(p.bits);
  unsigned long long st_inter = 0, st_frames = 0, st_nodes = 0;

  // the current node's prefix: listed in shared memory (n <= cap) or dense in stack slot d
  // stack slot d <- that prefix (the node has become a frame)
  auto save = [&](uint32_t d, bool listed, uint32_t n) {
    uint32_t* hdr = slot_hdr(d);
    if (!listed) {  // its dense image is in the slot already
      if (threadIdx.x == 0) hdr[0] = kDensePrefix;
      return;
    }
    uint16_t* gl = reinterpret_cast<uint16_t*>(hdr + 4);
    uint4* gv = reinterpret_cast<uint4*>(slot_pre(d));
    if (threadIdx.x == 0) hdr[0] = n;
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
      gl[e] = sidx[e];
      gv[e] = sval[e];
    }
  };

  for (;;) {
    // ---------------- acquire a class ----------------
    if (threadIdx.x == 0) {
      C.kind = 0;
      bool stop = (*(volatile uint32_t*)&p.ctrl->err & DEV_ERR_ABORTED) != 0;
      if (!stop && p.max_sets && *(volatile unsigned long long*)&p.ctrl->sets_total > p.max_sets) {
        atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
        stop = true;
      }
      // (the projected mode's fallback queue when queue_sel is set)
      uint32_t* const qhead = p.queue_sel ? &p.ctrl->queue_head_f : &p.ctrl->queue_head;
      const uint32_t qlen = p.queue_sel ? p.ctrl->n_entries_f : p.ctrl->n_entries;
      const uint32_t e = stop ? 0xffffffffu : atomicAdd(qhead, 1u);
      if (e < qlen) {
        const uint2 en = p.entries[e];
        C.kind = 1; C.a = en.x; C.b = en.y; C.cls = en.x;
      }
    }
    __syncthreads();
    if (C.kind == 0) break;

    // ---------------- root node: X = {i, s_m}, candidates = survivors of i after s_m ----------------
    const uint32_t i = C.a, m = C.b;
    const uint32_t base = p.soff[i];
    const uint32_t si = p.sitems[base + m];
    const uint32_t r1 = p.frows[i], r2 = p.frows[si];
    const uint32_t nc = p.scnt[i] - m - 1;
    if (threadIdx.x == 0) { xrow[0] = r1; xidp[0] = p.rank_item[r1]; C.xlen0 = 2; }
    if (threadIdx.x == 1) { xrow[1] = r2; xidp[1] = p.rank_item[r2]; }
    // a prefix of support s has at most s nonzero words: s <= cap lists it in one pass; up to 4 cap
    // the list is tried first; above, or when the try overflows, the prefix is built dense
    const uint4* ra4 = bits4 + (size_t)r1 * A.stride4;
    const uint4* rb4 = bits4 + (size_t)r2 * A.stride4;
    const uint32_t supp0 = __ldg(p.C2 + (size_t)i * p.n1 + si);
    __syncthreads();  // the path (threads 0 and 1) is written
    sort_path_ids(xidp, 2, xid);  // made visible by the barriers of the prefix build below
    uint32_t nz = 0xffffffffu;
    if (supp0 <= 4u * A.cap) nz = and_rows_to_list<true>(ra4, rb4, A.stride4, sidx, sval, &list_count, A.cap);
    const bool listed = nz <= A.cap;
    if (!listed) nz = and_rows_count<true>(reinterpret_cast<uint4*>(slot_pre(0)), ra4, rb4, A.stride4, wtot);
    if (threadIdx.x == 0) {
      st_inter += nc;
      if (p.class_work) atomicAdd(&p.class_work[C.cls], (unsigned long long)nc);
    }
    const uint32_t ns = process_node<VEC>(A, C, cnt, wtot, xid, slot_pre(0), !listed, p.sitems + base + m + 1,
                                          CAND_FROW, nc, slot_list(0), list_cap, 2, listed ? sidx : nullptr, nz,
                                          listed ? sval : nullptr, slot_supp(0), supp0);
    if (ns >= 2) save(0, listed, nz);
    // the next step of the DFS (thread 0): expand the next child of the top frame, pop the frame, or
    // finish the class; every thread has read the previous step when thread 0 runs this
    uint32_t poll = 0;
    auto decide = [&]() {
      if (C.depth >= 0 && (++poll & 7) == 0 && traversal_stopped(p)) C.depth = -1;
      const int32_t d = C.depth;
      if (d < 0) {
        C.action = 4;
      } else if (f_cur[d] + 1 >= f_n[d]) {
        C.depth = d - 1;
        C.action = 3;
      } else if ((uint32_t)(d + 1) > p.maxd) {
        atomicOr(&p.ctrl->err, DEV_ERR_DEPTH);
        C.depth = -1;
        C.action = 3;
      } else {
        const uint32_t k = f_cur[d];
        C.action = 1;
        C.s_row = slot_list(d)[2 * k];
        C.s_id = slot_list(d)[2 * k + 1];
        C.s_supp = slot_supp(d)[k];
        C.cand_off = k + 1;
        C.nc = f_n[d] - k - 1;
        f_cur[d] = k + 1;
        xrow[C.xlen0 + d] = C.s_row;
        xidp[C.xlen0 + d] = C.s_id;
      }
    };
    if (threadIdx.x == 0) {
      ++st_nodes;  // (no CTA of this mode waits for progress)
      if (ns >= 2) { f_n[0] = ns; f_cur[0] = 0; C.depth = 0; ++st_frames; }
      else C.depth = -1;
      decide();  // (process_node ended with a barrier: nobody reads the root's step any more)
    }

    // ---------------- depth-first expansion ----------------
    for (;;) {
      __syncthreads();  // the step is visible
      const uint32_t action = C.action;
      if (action == 4) break;
      if (action == 3) {
        __syncthreads();  // every thread has read the pop before thread 0 decides again
        if (threadIdx.x == 0) decide();
        continue;
      }
      // expand the child [X_d u {s} | rest of frame d]
      const int32_t d = C.depth;
      const uint32_t ncc = C.nc, coff = C.cand_off;
      const uint32_t xl = C.xlen0 + d + 1;  // prefix length of the child
      const uint4* r4 = bits4 + (size_t)C.s_row * A.stride4;
      const uint32_t hdr = *(volatile const uint32_t*)slot_hdr(d);
      sort_path_ids(xidp, xl, xid);  // made visible by the barriers of the prefix build below
      uint32_t nz2;
      bool listed2;
      if (hdr != kDensePrefix) {  // listed parent: the child is listed too (no more nonzero words)
        nz2 = list_from_list(reinterpret_cast<const uint16_t*>(slot_hdr(d) + 4),
                             reinterpret_cast<const uint4*>(slot_pre(d)), hdr, r4, sidx, sval, &list_count);
        listed2 = true;
      } else {  // dense parent: as for the root, by the child's support
        nz2 = 0xffffffffu;
        if (C.s_supp <= 4u * A.cap)
          nz2 = and_rows_to_list<false>(reinterpret_cast<const uint4*>(slot_pre(d)), r4, A.stride4, sidx, sval,
                                        &list_count, A.cap);
        listed2 = nz2 <= A.cap;
        if (!listed2)
          nz2 = and_rows_count<false>(reinterpret_cast<uint4*>(slot_pre(d + 1)),
                                      reinterpret_cast<const uint4*>(slot_pre(d)), r4, A.stride4, wtot);
      }
      if (threadIdx.x == 0) {
        st_inter += ncc;
        if (p.class_work) atomicAdd(&p.class_work[C.cls], (unsigned long long)ncc);
      }
      const uint32_t n2 = process_node<VEC>(A, C, cnt, wtot, xid, slot_pre(d + 1), !listed2,
                                            slot_list(d) + 2 * coff, CAND_PAIR, ncc, slot_list(d + 1), list_cap, xl,
                                            listed2 ? sidx : nullptr, nz2, listed2 ? sval : nullptr,
                                            slot_supp(d + 1), C.s_supp);
      if (n2 >= 2) save(d + 1, listed2, nz2);
      if (threadIdx.x == 0) {
        ++st_nodes;
        if (n2 >= 2) { f_n[d + 1] = n2; f_cur[d + 1] = 0; C.depth = d + 1; ++st_frames; }
        decide();  // (the step's fields were read before process_node's barriers)
      }
    }
    // class finished
    if (threadIdx.x == 0) {
      __threadfence();
      atomicSub(&p.ctrl->pending, 1u);
    }
  }
  if (threadIdx.x == 0) {
    atomicAdd(&p.ctrl->n_intersections, st_inter);
    atomicAdd(&p.ctrl->n_frames, st_frames);
    atomicAdd(&p.ctrl->n_nodes, st_nodes);
    if (p.cta_time) p.cta_time[2 * blockIdx.x + 1] = global_ns();
  }
#undef slot_pre
#undef slot_hdr
#undef slot_supp
#undef slot_list
}

template <int VEC>
__device__ __forceinline__ uint32_t piece_popc3(const uint4* __restrict__ r1, const uint4* __restrict__ r2,
                                                const uint4* pre, uint32_t base4, uint32_t stride4) {
  // popc(pre & r1 & r2), reading r1 only where pre is nonzero and r2 only where pre & r1 is
  uint4 c[VEC], a[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const uint32_t w = base4 + v * 32;
    c[v] = w < stride4 ? pre[w] : make_uint4(0u, 0u, 0u, 0u);
  }
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const uint4 x = any4(c[v]) ? __ldg(r1 + base4 + v * 32) : make_uint4(0u, 0u, 0u, 0u);
    c[v] = make_uint4(x.x & c[v].x, x.y & c[v].y, x.z & c[v].z, x.w & c[v].w);
  }
#pragma unroll
  for (int v = 0; v < VEC; ++v) a[v] = any4(c[v]) ? __ldg(r2 + base4 + v * 32) : make_uint4(0u, 0u, 0u, 0u);
  uint32_t s = 0;
#pragma unroll
  for (int v = 0; v < VEC; ++v)
    s += __popc(a[v].x & c[v].x) + __popc(a[v].y & c[v].y) + __popc(a[v].z & c[v].z) + __popc(a[v].w & c[v].w);
  return s;
}

struct FrameCtl {
  uint32_t action;   // 1 descend, 2 count pass, 3 pop, 4 class done
  uint32_t m;        // child to descend
  uint64_t p0, p1;   // pair range of the pass
  uint32_t mA, mB;   // children touched by the pass
  uint32_t cont;     // the pass continues child mA from an earlier pass
  unsigned long long base;
};

template <int VEC, bool PSMEM>
__global__ void __launch_bounds__(512, 1) k_dfs_frames(const DfsArgs A) {
  const DfsLaunch& p = A.p;
  if (p.cta_time && threadIdx.x == 0) p.cta_time[2 * blockIdx.x] = global_ns();
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ Ctl C;
  __shared__ FrameCtl F;
  __shared__ uint32_t wtot[33];
  __shared__ int32_t spre_depth;  // frame whose prefix the shared copy holds
  // dynamic shared memory: [prefix (PSMEM)] [cnt kPairBatch] [ccnt kPairBatch] [frame arrays 7 x (maxd+1)]
  //                        [xrow] [xidp] [xid]
  uint32_t* sp = smem;
  uint32_t* spre = PSMEM ? sp : nullptr;
  if (PSMEM) sp += p.stride;
  uint32_t* cnt = sp; sp += kPairBatch;   // pair counts of a pass
  uint32_t* ccnt = sp; sp += kPairBatch;  // survivors per child of a pass
  const uint32_t nd = p.maxd + 1;
  uint32_t* f_n = sp; sp += nd;       // list length
  uint32_t* f_loff = sp; sp += nd;    // arena offset of the list (words)
  uint32_t* f_cur = sp; sp += nd;     // next child to enter
  uint32_t* f_cend = sp; sp += nd;    // children below this are fully counted
  uint32_t* f_gm0 = sp; sp += nd;     // first child with an entry in the child table
  uint32_t* f_gused = sp; sp += nd;   // survivor entries used in the G area
  uint32_t* f_plo = sp; sp += 2 * nd; // next pair to count (64-bit, lo/hi)
  uint32_t* xrow = sp; sp += A.max_len + 1;
  uint32_t* xidp = sp; sp += A.max_len + 1;
  uint32_t* xid = sp;

  // arena: [root list 2*n1] then per depth [prefix stride][G 2*(kPairBatch+n1)][child table 2*kPairBatch]
  const uint64_t root_words = frames_root_words(p.n1);
  const uint64_t g_words = frames_g_words(p.n1);
  const uint64_t per_depth = frames_depth_words(p.stride, p.n1);
  uint32_t* const arena = p.arena + (size_t)blockIdx.x * p.arena_cta_words;
  uint32_t* const root_list = arena;
#define fr_pre(d) (arena + root_words + (size_t)(d) * per_depth)
#define fr_g(d) (arena + root_words + (size_t)(d) * per_depth + p.stride)
#define fr_tab(d) (arena + root_words + (size_t)(d) * per_depth + p.stride + g_words)
  const uint4* bits4 = reinterpret_cast<const uint4*>(p.bits);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long st_inter = 0, st_frames = 0;

  for (;;) {
    if (threadIdx.x == 0) {
      C.kind = 0;
      bool stop = (*(volatile uint32_t*)&p.ctrl->err & DEV_ERR_ABORTED) != 0;
      if (!stop && p.max_sets && *(volatile unsigned long long*)&p.ctrl->sets_total > p.max_sets) {
        atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
        stop = true;
      }
      const uint32_t e = stop ? 0xffffffffu : atomicAdd(&p.ctrl->queue_head, 1u);
      if (e < p.ctrl->n_entries) {
        const uint2 en = p.entries[e];
        C.kind = 1; C.a = en.x; C.b = en.y; C.cls = en.x;
      }
    }
    __syncthreads();
    if (C.kind == 0) break;

    // ---------------- root node: [X = {i, s_m} | S_i after s_m] ----------------
    const uint32_t i = C.a, m0 = C.b;
    const uint32_t base = p.soff[i];
    const uint32_t si = p.sitems[base + m0];
    const uint32_t r1 = p.frows[i], r2 = p.frows[si];
    const uint32_t nc = p.scnt[i] - m0 - 1;
    if (threadIdx.x == 0) { xrow[0] = r1; xidp[0] = p.rank_item[r1]; spre_depth = 0; }
    if (threadIdx.x == 1) { xrow[1] = r2; xidp[1] = p.rank_item[r2]; }
    {
      const uint4* a4 = bits4 + (size_t)r1 * A.stride4;
      const uint4* b4 = bits4 + (size_t)r2 * A.stride4;
      uint4* dst = reinterpret_cast<uint4*>(PSMEM ? spre : fr_pre(0));
      and_rows<true>(dst, nullptr, a4, b4, A.stride4);
    }
    __syncthreads();
    sort_path_ids(xidp, 2, xid);
    __syncthreads();
    if (threadIdx.x == 0) {
      st_inter += nc;
      if (p.class_work) atomicAdd(&p.class_work[C.cls], (unsigned long long)nc);
    }
    const uint32_t ns = process_node<VEC>(A, C, cnt, wtot, xid, PSMEM ? spre : fr_pre(0), false, p.sitems + base + m0 + 1,
                                          CAND_FROW, nc, root_list, p.n1, 2);
    if (ns >= 2 && PSMEM) {
      const uint4* s4 = reinterpret_cast<const uint4*>(spre);
      uint4* d4 = reinterpret_cast<uint4*>(fr_pre(0));
      for (uint32_t w = threadIdx.x; w < A.stride4; w += blockDim.x) d4[w] = s4[w];
    }
    if (threadIdx.x == 0) {
      atomicAdd(&p.ctrl->n_nodes, 1ull);
      atomicAdd(&p.ctrl->progress, 1u);
      if (ns >= 2) {
        f_n[0] = ns; f_loff[0] = 0; f_cur[0] = 0; f_cend[0] = 0; f_gm0[0] = 0; f_gused[0] = 0;
        f_plo[0] = 0; f_plo[1] = 0;
        C.depth = 0;
        ++st_frames;
      } else {
        C.depth = -1;
      }
    }

    // ---------------- frames ----------------
    for (;;) {
      __syncthreads();
      if (threadIdx.x == 0) {
        if (C.depth >= 0 && traversal_stopped(p)) C.depth = -1;
        const int32_t d = C.depth;
        if (d < 0) {
          F.action = 4;
        } else {
          const uint32_t n = f_n[d];
          const uint64_t total = (uint64_t)n * (n - 1) / 2;
          const uint64_t pnext = (uint64_t)f_plo[2 * d] | ((uint64_t)f_plo[2 * d + 1] << 32);
          uint32_t* tab = fr_tab(d);
          bool done = false;
          while (!done && f_cur[d] < f_cend[d]) {
            const uint32_t m = f_cur[d]++;
            const uint32_t k = m - f_gm0[d];
            if (tab[2 * k + 1] >= 2) {
              if ((uint32_t)(d + 1) > p.maxd) {
                atomicOr(&p.ctrl->err, DEV_ERR_DEPTH);
                C.depth = -1;
                F.action = 3;
              } else {
                F.action = 1;
                F.m = m;
              }
              done = true;
            }
          }
          if (!done) {
            if (pnext >= total) {
              F.action = 3;
              C.depth = d - 1;
            } else {
              uint64_t p1 = pnext + kPairBatch < total ? pnext + kPairBatch : total;
              const uint32_t mA = pair_child(pnext, n, 0, n - 1);
              if (p1 < total) {
                const uint32_t mE = pair_child(p1, n, mA, n - 1);  // child holding pair p1
                if (pair_base(mE, n) > pnext) p1 = pair_base(mE, n);  // end at a child boundary
              }
              const uint32_t mB = pair_child(p1 - 1, n, mA, n - 1);
              F.action = 2;
              F.p0 = pnext;
              F.p1 = p1;
              F.mA = mA;
              F.mB = mB;
              F.cont = pair_base(mA, n) < pnext ? 1u : 0u;
              if (!F.cont) { f_gm0[d] = mA; f_gused[d] = 0; }
              f_plo[2 * d] = (uint32_t)p1;
              f_plo[2 * d + 1] = (uint32_t)(p1 >> 32);
              // children fully counted after this pass
              const uint32_t mfull = (pair_base(mB, n) + (n - 1 - mB) <= p1) ? mB + 1 : mB;
              f_cend[d] = mfull;
            }
          }
        }
      }
      __syncthreads();
      const uint32_t action = F.action;
      if (action == 4) break;
      if (action == 3) continue;
      const int32_t d = C.depth;
      const uint32_t n = f_n[d];
      const uint32_t* L = arena + f_loff[d];
      const uint32_t xl = 2 + (uint32_t)d;  // |X_d|
      if (action == 1) {
        // enter child m of frame d as frame d + 1
        const uint32_t m = F.m;
        const uint32_t k = m - f_gm0[d];
        const uint32_t* tab = fr_tab(d);
        const uint32_t row = L[2 * m];
        // t(X_d) comes from the stack: the shared copy may hold a deeper prefix when this frame resumes
        const uint4* pd = reinterpret_cast<const uint4*>(fr_pre(d));
        const uint4* r4 = bits4 + (size_t)row * A.stride4;
        uint4* dg = reinterpret_cast<uint4*>(fr_pre(d + 1));
        and_rows<false>(dg, PSMEM ? reinterpret_cast<uint4*>(spre) : nullptr, pd, r4, A.stride4);
        if (threadIdx.x == 0) {
          spre_depth = d + 1;
          xrow[xl] = row;
          xidp[xl] = L[2 * m + 1];
          f_n[d + 1] = tab[2 * k + 1];
          f_loff[d + 1] = (uint32_t)((fr_g(d) + 2ull * tab[2 * k]) - arena);
          f_cur[d + 1] = 0; f_cend[d + 1] = 0; f_gm0[d + 1] = 0; f_gused[d + 1] = 0;
          f_plo[2 * (d + 1)] = 0; f_plo[2 * (d + 1) + 1] = 0;
          C.depth = d + 1;
          ++st_frames;
        }
        continue;
      }
      // action 2: count the pairs [p0, p1) of frame d
      const uint64_t p0 = F.p0, p1 = F.p1;
      const uint32_t np = (uint32_t)(p1 - p0), mA = F.mA, mB = F.mB;
      const uint32_t* pre = PSMEM ? spre : fr_pre(d);
      if (PSMEM && spre_depth != d) {
        // a deeper frame replaced the shared copy: reload t(X_d)
        const uint4* s4 = reinterpret_cast<const uint4*>(fr_pre(d));
        for (uint32_t w = threadIdx.x; w < A.stride4; w += blockDim.x) reinterpret_cast<uint4*>(spre)[w] = s4[w];
      }
      for (uint32_t k = threadIdx.x; k < np; k += blockDim.x) cnt[k] = 0;
      for (uint32_t k = threadIdx.x; k <= mB - mA; k += blockDim.x) ccnt[k] = 0;
      sort_path_ids(xidp, xl, xid);
      __syncthreads();
      if (threadIdx.x == 0) spre_depth = d;
      const uint4* pre4 = reinterpret_cast<const uint4*>(pre);
      const uint32_t total_pieces = np * A.nseg;
      for (uint32_t pc = warp; pc < total_pieces; pc += nw) {
        const uint32_t q = pc / A.nseg, g = pc - q * A.nseg;
        const uint64_t pp = p0 + q;
        const uint32_t m = pair_child(pp, n, mA, mB + 1);
        const uint32_t e = m + 1 + (uint32_t)(pp - pair_base(m, n));
        const uint4* ra = bits4 + (size_t)L[2 * m] * A.stride4;
        const uint4* rb = bits4 + (size_t)L[2 * e] * A.stride4;
        uint32_t sum = piece_popc3<VEC>(ra, rb, pre4, g * 32 * VEC + lane, A.stride4);
        sum = __reduce_add_sync(0xffffffffu, sum);
        if (lane == 0 && sum) atomicAdd(&cnt[q], sum);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        st_inter += np;
        if (p.class_work) atomicAdd(&p.class_work[C.cls], (unsigned long long)np);
      }
      // survivors in pair order: G entries (row, id) of the second item, per-child counts, records
      uint32_t* G = fr_g(d);
      uint32_t* tab = fr_tab(d);
      const uint32_t gbase = f_gused[d];
      const uint32_t gm0 = f_gm0[d];
      uint32_t taken = 0;
      for (uint32_t c0 = 0; c0 < np; c0 += blockDim.x) {
        const uint32_t q = c0 + threadIdx.x;
        const uint32_t cq = q < np ? cnt[q] : 0u;
        const bool f = q < np && cq >= p.minsup;
        uint32_t tot;
        const uint32_t pos = block_flag_scan(f, wtot, &tot);
        if (threadIdx.x == 0 && tot) {
          const unsigned long long sets = tot, items = (unsigned long long)tot * (xl + 2);
          if (p.out_off) {  // record positions (a count-only mine checks the itemset limit at its polls)
            F.base = atomicAdd(&p.ctrl->packed, (sets << 32) | items);
            const unsigned long long after = (F.base >> 32) + sets;
            if ((p.max_sets && after > p.max_sets) || after > 0xfffffff0ull) atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
          }
          atomicAdd(&p.ctrl->sets_total, sets);
          atomicAdd(&p.ctrl->items_total, items);
          atomicMax(&p.ctrl->max_len, xl + 2);
          if (p.class_sets) atomicAdd(&p.class_sets[C.cls], sets);
        }
        __syncthreads();
        if (f) {
          const uint64_t pp = p0 + q;
          const uint32_t m = pair_child(pp, n, mA, mB + 1);
          const uint32_t e = m + 1 + (uint32_t)(pp - pair_base(m, n));
          const uint32_t o = gbase + taken + pos;
          G[2 * o] = L[2 * e];
          G[2 * o + 1] = L[2 * e + 1];
          atomicAdd(&ccnt[m - mA], 1u);
          const uint64_t rec = (F.base >> 32) + pos;
          const uint64_t it0 = (F.base & 0xffffffffull) + (uint64_t)pos * (xl + 2);
          if (!p.out_off) {
            // count only: no records
          } else if (rec < p.cap_sets && it0 + xl + 2 <= p.cap_items) {
            // X_d's sorted ids merged with the two new ids (ids are < 2^32 - 1)
            const uint32_t a = L[2 * m + 1], b = L[2 * e + 1];
            uint32_t lo = min(a, b), hi = max(a, b);
            uint32_t* dst = p.out_items + it0;
            uint32_t qd = 0;
            for (uint32_t x = 0; x < xl; ++x) {
              const uint32_t u = xid[x];
              if (lo < u) { dst[qd++] = lo; lo = hi; hi = 0xffffffffu; }
              if (lo < u) { dst[qd++] = lo; lo = hi; hi = 0xffffffffu; }
              dst[qd++] = u;
            }
            if (lo != 0xffffffffu) dst[qd++] = lo;
            if (hi != 0xffffffffu) dst[qd++] = hi;
            p.out_off[rec] = it0;
            p.out_supp[rec] = cq;
          } else {
            atomicOr(&p.ctrl->err, DEV_ERR_OVERFLOW);
          }
        }
        taken += tot;
        __syncthreads();
      }
      // child table: offset (into G, entries) and survivor count per child of the pass
      if (threadIdx.x == 0) {
        uint32_t off = gbase;
        for (uint32_t m = mA; m <= mB; ++m) {
          const uint32_t k = m - gm0;
          const uint32_t c = ccnt[m - mA];
          if (m == mA && F.cont) {
            tab[2 * k + 1] += c;
          } else {
            tab[2 * k] = off;
            tab[2 * k + 1] = c;
          }
          off += c;
        }
        f_gused[d] = gbase + taken;
        atomicAdd(&p.ctrl->n_nodes, (unsigned long long)(f_cend[d] > mA ? f_cend[d] - mA : 0));
        atomicAdd(&p.ctrl->progress, 1u);
      }
    }
    // class finished
    if (threadIdx.x == 0) {
      __threadfence();
      atomicSub(&p.ctrl->pending, 1u);
    }
  }
  if (threadIdx.x == 0) {
    atomicAdd(&p.ctrl->n_intersections, st_inter);
    atomicAdd(&p.ctrl->n_frames, st_frames);
    if (p.cta_time) p.cta_time[2 * blockIdx.x + 1] = global_ns();
  }
#undef fr_pre
#undef fr_g
#undef fr_tab
}

// ---------------------------------------------------------------------------
// Warp DFS (short rows): one warp walks one two-item class at a time.
//
// For rows of at most 32 * WPL words a whole prefix fits in the registers of one
// warp (lane l holds words l, l + 32, ...), so a class node needs no CTA-wide
// barrier: the warp ANDs the prefix with the node's extension row, counts every
// candidate against it (G candidates per round, their loads in flight
// together, row words read only where the prefix word is nonzero), and writes
// the survivors and their records.  The same Eclat-DFS-Computation recursion as
// the CTA kernels (App. B.3.2), with the per-warp stack in the arena: slot s
// holds the prefix of the frame at depth s + 1 and the survivor list (frow
// indices and supports) its count produced.

constexpr uint32_t kWarpDfsThreads = 256;  // 8 warps per CTA

__host__ __device__ inline uint64_t warp_slot_words(uint32_t stride, uint32_t n1) {
  return (uint64_t)stride + 2ull * (((uint64_t)n1 + 3) & ~3ull);
}

template <int WPL, int G>
__global__ void __launch_bounds__(kWarpDfsThreads) k_dfs_warp(const DfsArgs A) {
  const DfsLaunch& p = A.p;
  if (p.cta_time && threadIdx.x == 0) p.cta_time[2 * blockIdx.x] = global_ns();
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t wpw = 2 * (A.max_len + 1) + 2 * (p.maxd + 2);  // shared words per warp
  uint32_t* path = smem + wib * wpw;      // ids of the current prefix, in path order
  uint32_t* xs = path + A.max_len + 1;    // the same ids ascending
  uint32_t* f_cur = xs + A.max_len + 1;   // next survivor to expand, per frame depth
  uint32_t* f_n = f_cur + p.maxd + 2;     // survivors, per frame depth
  const uint64_t slot_words = warp_slot_words(p.stride, p.n1);
  const uint64_t list_off = p.stride, supp_off = p.stride + (((uint64_t)p.n1 + 3) & ~3ull);
  uint32_t* const arena =
      p.arena + (size_t)blockIdx.x * p.arena_cta_words + (size_t)wib * (p.maxd + 1) * slot_words;
  const uint32_t nwords = p.stride;  // row words (a multiple of 32)
  unsigned long long st_inter = 0, st_nodes = 0, st_frames = 0;

  // ids of path[0..len) ascending into xs (the ids are distinct)
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

  // counts cand[0..nc) against the prefix q (prefix ids xs[0..xlen)), writes the survivors to slot
  // `so` (frow index, support), one record per survivor; returns the survivor count
  auto count_node = [&](const uint32_t (&q)[WPL], const uint32_t* cand, uint32_t nc, uint32_t so, uint32_t xlen,
                        unsigned long long& cls_sets) -> uint32_t {
    uint32_t* lo = arena + (size_t)so * slot_words + list_off;
    uint32_t* so_supp = arena + (size_t)so * slot_words + supp_off;
    uint32_t nout = 0;
    for (uint32_t k0 = 0; k0 < nc; k0 += G) {
      uint32_t c[G], row[G], s[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        c[g] = k0 + g < nc ? cand[k0 + g] : 0xffffffffu;
        row[g] = c[g] != 0xffffffffu ? __ldg(p.frows + c[g]) : 0u;
        s[g] = 0;
      }
      uint32_t wv[G][WPL];
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int w = 0; w < WPL; ++w) {
          const uint32_t j = (uint32_t)w * 32 + lane;
          wv[g][w] = (j < nwords && q[w] && c[g] != 0xffffffffu) ? __ldg(p.bits + (size_t)row[g] * p.stride + j) : 0u;
        }
#pragma unroll
      for (int g = 0; g < G; ++g) {
#pragma unroll
        for (int w = 0; w < WPL; ++w) s[g] += __popc(q[w] & wv[g][w]);
        s[g] = __reduce_add_sync(0xffffffffu, s[g]);
      }
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (c[g] != 0xffffffffu && s[g] >= p.minsup) {
          if (lane == 0) {
            lo[nout] = c[g];
            so_supp[nout] = s[g];
          }
          ++nout;
        }
    }
    st_inter += nc;
    ++st_nodes;
    if (nout == 0) return 0;
    __syncwarp();  // the list written by lane 0 is read by every lane below
    unsigned long long base = 0;
    if (lane == 0) {
      const unsigned long long sets = nout, items = (unsigned long long)nout * (xlen + 1);
      if (p.out_off) {  // record positions (a count-only mine checks the itemset limit at its polls)
        base = atomicAdd(&p.ctrl->packed, (sets << 32) | items);
        const unsigned long long after = (base >> 32) + sets;
        if ((p.max_sets && after > p.max_sets) || after > 0xfffffff0ull) atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
      }
      atomicAdd(&p.ctrl->sets_total, sets);
      atomicAdd(&p.ctrl->items_total, items);
      atomicMax(&p.ctrl->max_len, xlen + 1);
    }
    if (p.out_off) base = __shfl_sync(0xffffffffu, base, 0);
    cls_sets += nout;
    if (p.out_off) {
      for (uint32_t o = 0; o < nout; ++o) {
        const uint32_t v = __ldg(p.rank_item + __ldg(p.frows + lo[o]));
        const uint64_t rec = (base >> 32) + o;
        const uint64_t it0 = (base & 0xffffffffull) + (uint64_t)o * (xlen + 1);
        if (rec < p.cap_sets && it0 + xlen + 1 <= p.cap_items) {
          uint32_t pos = 0;  // place of v among the prefix ids
          for (uint32_t q0 = 0; q0 < xlen; q0 += 32)
            pos += __popc(__ballot_sync(0xffffffffu, q0 + lane < xlen && xs[q0 + lane] < v));
          for (uint32_t t = lane; t <= xlen; t += 32)
            p.out_items[it0 + t] = t < pos ? xs[t] : (t == pos ? v : xs[t - 1]);
          if (lane == 0) {
            p.out_off[rec] = it0;
            p.out_supp[rec] = so_supp[o];
          }
        } else if (lane == 0) {
          atomicOr(&p.ctrl->err, DEV_ERR_OVERFLOW);
        }
      }
    }
    return nout;
  };

  for (;;) {
    // ---------------- acquire a two-item class ----------------
    uint32_t e = 0xffffffffu;
    if (lane == 0) {
      bool stop = (*(volatile uint32_t*)&p.ctrl->err & DEV_ERR_ABORTED) != 0;
      if (!stop && p.max_sets && *(volatile unsigned long long*)&p.ctrl->sets_total > p.max_sets) {
        atomicOr(&p.ctrl->err, DEV_ERR_ABORTED);
        stop = true;
      }
      if (!stop) {
        e = atomicAdd(&p.ctrl->queue_head, 1u);
        if (e >= p.ctrl->n_entries) e = 0xffffffffu;
      }
    }
    e = __shfl_sync(0xffffffffu, e, 0);
    if (e == 0xffffffffu) break;
    const uint2 en = p.entries[e];
    const uint32_t i = en.x, m = en.y, cls = en.x;
    const uint32_t base = p.soff[i];
    const uint32_t si = p.sitems[base + m];
    const uint32_t r1 = p.frows[i], r2 = p.frows[si];
    const uint32_t nc = p.scnt[i] - m - 1;
    unsigned long long cls_sets = 0, cls_work = 0;
    if (lane == 0) {
      path[0] = p.rank_item[r1];
      path[1] = p.rank_item[r2];
    }
    sort_path(2);

    // root node X = {i, s_m}: prefix t(i) & t(s_m) in registers, candidates = the later survivors of i
    uint32_t q[WPL];
#pragma unroll
    for (int w = 0; w < WPL; ++w) {
      const uint32_t j = (uint32_t)w * 32 + lane;
      q[w] = j < nwords ? __ldg(p.bits + (size_t)r1 * p.stride + j) & __ldg(p.bits + (size_t)r2 * p.stride + j) : 0u;
    }
    cls_work += nc;
    uint32_t n = count_node(q, p.sitems + base + m + 1, nc, 0, 2, cls_sets);
    int32_t depth = 0;
    if (n >= 2) {  // the root becomes the frame at depth 1 (slot 0)
#pragma unroll
      for (int w = 0; w < WPL; ++w) {
        const uint32_t j = (uint32_t)w * 32 + lane;
        if (j < nwords) arena[j] = q[w];
      }
      ++st_frames;
      if (lane == 0) {
        f_n[1] = n;
        f_cur[1] = 0;
      }
      depth = 1;
    }
    uint32_t since_poll = 0;
    while (depth >= 1) {
      __syncwarp();
      const uint32_t k = f_cur[depth], nf = f_n[depth];
      if (k + 1 >= nf) {  // the last survivor has no later candidates
        --depth;
        continue;
      }
      if (++since_poll == 8) {
        since_poll = 0;
        uint32_t stop = 0;
        if (lane == 0) stop = traversal_stopped(p);
        if (__shfl_sync(0xffffffffu, stop, 0)) break;
      }
      __syncwarp();
      if (lane == 0) f_cur[depth] = k + 1;
      uint32_t* fs = arena + (size_t)(depth - 1) * slot_words;
      const uint32_t ce = fs[list_off + k];
      const uint32_t re = __ldg(p.frows + ce);
      const uint32_t xlen = (uint32_t)depth + 1;  // prefix length of the frame; the child has xlen + 1
      if (lane == 0) path[xlen] = p.rank_item[re];
      sort_path(xlen + 1);
#pragma unroll
      for (int w = 0; w < WPL; ++w) {
        const uint32_t j = (uint32_t)w * 32 + lane;
        q[w] = j < nwords ? fs[j] & __ldg(p.bits + (size_t)re * p.stride + j) : 0u;
      }
      const uint32_t ncc = nf - k - 1;
      cls_work += ncc;
      if ((uint32_t)depth > p.maxd) {  // no slot for the child's survivors (cannot happen: frames stop at maxd)
        if (lane == 0) atomicOr(&p.ctrl->err, DEV_ERR_DEPTH);
        break;
      }
      const uint32_t n2 = count_node(q, fs + list_off + k + 1, ncc, (uint32_t)depth, xlen + 1, cls_sets);
      if (n2 >= 2) {
        if ((uint32_t)depth + 1 > p.maxd) {  // the stack is too shallow: the run repeats with a deeper one
          if (lane == 0) atomicOr(&p.ctrl->err, DEV_ERR_DEPTH);
          continue;
        }
        uint32_t* cs = arena + (size_t)depth * slot_words;
#pragma unroll
        for (int w = 0; w < WPL; ++w) {
          const uint32_t j = (uint32_t)w * 32 + lane;
          if (j < nwords) cs[j] = q[w];
        }
        ++st_frames;
        ++depth;
        if (lane == 0) {
          f_n[depth] = n2;
          f_cur[depth] = 0;
        }
      }
    }
    if (lane == 0) {
      if (p.class_sets && cls_sets) atomicAdd(&p.class_sets[cls], cls_sets);
      if (p.class_work && cls_work) atomicAdd(&p.class_work[cls], cls_work);
    }
  }
  if (lane == 0) {
    atomicAdd(&p.ctrl->n_intersections, st_inter);
    atomicAdd(&p.ctrl->n_nodes, st_nodes);
    atomicAdd(&p.ctrl->n_frames, st_frames);
  }
  if (p.cta_time) {
    __syncthreads();
    if (threadIdx.x == 0) p.cta_time[2 * blockIdx.x + 1] = global_ns();
  }
}

// Raise a kernel's dynamic shared-memory limit to the device maximum once per device (launches then
// pass their own size).  Setting it per launch to the launch's size would race between threads
// mining concurrently.
cudaError_t allow_max_smem(const void* func) { return kernel_smem_limit(func, -1); }

template <int VEC, bool PSMEM>
cudaError_t launch_dfs_t(const DfsArgs& a, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t st) {
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(k_dfs<VEC, PSMEM>));
  if (e != cudaSuccess) return e;
  k_dfs<VEC, PSMEM><<<grid, threads, smem, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <bool PSMEM>
cudaError_t launch_dfs_vec(const DfsArgs& a, uint32_t grid, uint32_t threads, uint32_t vec, size_t smem,
                           cudaStream_t st) {
  switch (vec) {
    case 1: return launch_dfs_t<1, PSMEM>(a, grid, threads, smem, st);
    case 2: return launch_dfs_t<2, PSMEM>(a, grid, threads, smem, st);
    case 8: return launch_dfs_t<8, PSMEM>(a, grid, threads, smem, st);
    default: return launch_dfs_t<4, PSMEM>(a, grid, threads, smem, st);
  }
}

template <int VEC, bool PSMEM>
cudaError_t launch_frames_t(const DfsArgs& a, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t st) {
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(k_dfs_frames<VEC, PSMEM>));
  if (e != cudaSuccess) return e;
  k_dfs_frames<VEC, PSMEM><<<grid, threads, smem, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <bool PSMEM>
cudaError_t launch_frames_vec(const DfsArgs& a, uint32_t grid, uint32_t threads, uint32_t vec, size_t smem,
                              cudaStream_t st) {
  switch (vec) {
    case 1: return launch_frames_t<1, PSMEM>(a, grid, threads, smem, st);
    case 2: return launch_frames_t<2, PSMEM>(a, grid, threads, smem, st);
    case 8: return launch_frames_t<8, PSMEM>(a, grid, threads, smem, st);
    default: return launch_frames_t<4, PSMEM>(a, grid, threads, smem, st);
  }
}

template <int VEC, bool PSMEM>
cudaError_t occ_frames_t(uint32_t threads, size_t smem, int* out) {
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(k_dfs_frames<VEC, PSMEM>));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_dfs_frames<VEC, PSMEM>, (int)threads, smem);
}

template <int VEC, bool PSMEM>
cudaError_t occ_t(uint32_t threads, size_t smem, int* out) {
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(k_dfs<VEC, PSMEM>));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_dfs<VEC, PSMEM>, (int)threads, smem);
}

template <int VEC>
cudaError_t launch_sparse_t(const DfsArgs& a, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t st) {
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(k_dfs_sparse<VEC>));
  if (e != cudaSuccess) return e;
  k_dfs_sparse<VEC><<<grid, threads, smem, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sparse_vec(const DfsArgs& a, uint32_t grid, uint32_t threads, uint32_t vec, size_t smem,
                              cudaStream_t st) {
  switch (vec) {
    case 16: return launch_sparse_t<16>(a, grid, threads, smem, st);
    case 1: return launch_sparse_t<1>(a, grid, threads, smem, st);
    case 2: return launch_sparse_t<2>(a, grid, threads, smem, st);
    case 8: return launch_sparse_t<8>(a, grid, threads, smem, st);
    default: return launch_sparse_t<4>(a, grid, threads, smem, st);
  }
}

template <int VEC>
cudaError_t occ_sparse_t(uint32_t threads, size_t smem, int* out) {
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(k_dfs_sparse<VEC>));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_dfs_sparse<VEC>, (int)threads, smem);
}

template <int WPL, int G>
cudaError_t launch_warp_t(const DfsArgs& a, uint32_t grid, size_t smem, cudaStream_t st) {
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(k_dfs_warp<WPL, G>));
  if (e != cudaSuccess) return e;
  k_dfs_warp<WPL, G><<<grid, kWarpDfsThreads, smem, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

// words per lane: the smallest of 1, 2, 4, 8, 16 that covers the row; candidates per round so that
// about 8 to 16 loads per lane are in flight
cudaError_t launch_warp(const DfsArgs& a, uint32_t grid, size_t smem, cudaStream_t st) {
  const uint32_t wpl = a.p.stride / 32;
  if (wpl <= 1) return launch_warp_t<1, 8>(a, grid, smem, st);
  if (wpl <= 2) return launch_warp_t<2, 8>(a, grid, smem, st);
  if (wpl <= 4) return launch_warp_t<4, 4>(a, grid, smem, st);
  if (wpl <= 8) return launch_warp_t<8, 2>(a, grid, smem, st);
  return launch_warp_t<16, 1>(a, grid, smem, st);
}

template <int WPL, int G>
cudaError_t occ_warp_t(size_t smem, int* out) {
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(k_dfs_warp<WPL, G>));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_dfs_warp<WPL, G>, (int)kWarpDfsThreads, smem);
}

cudaError_t occ_warp(uint32_t stride, size_t smem, int* out) {
  const uint32_t wpl = stride / 32;
  if (wpl <= 1) return occ_warp_t<1, 8>(smem, out);
  if (wpl <= 2) return occ_warp_t<2, 8>(smem, out);
  if (wpl <= 4) return occ_warp_t<4, 4>(smem, out);
  if (wpl <= 8) return occ_warp_t<8, 2>(smem, out);
  return occ_warp_t<16, 1>(smem, out);
}

}  // namespace

cudaError_t launch_level2_counts(const LevelLaunch& p, cudaStream_t st) {
  if (p.n1 == 0) return cudaSuccess;
  k_surv_count<<<p.n1, 256, 0, st>>>(p.C2, p.n1, p.minsup, p.scnt, p.ctrl);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_level2_scan<<<1, 1024, 0, st>>>(p.scnt, p.row_order, p.n1, p.row_supp, p.minsup, p.soff, p.eoff, p.cap_sets,
                                    p.cap_items, p.ctrl, p.leaves);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_level2_fill(const LevelLaunch& p, cudaStream_t st) {
  if (p.n1 == 0) return cudaSuccess;
  // (leaves only: the fill writes the queue and survivor lists, no records)
  k_level2_fill<<<p.n1, 256, 0, st>>>(p.C2, p.n1, p.minsup, p.frows, p.row_supp, p.rank_item, p.row_order, p.scnt,
                                      p.soff, p.eoff, p.sitems, p.entries, p.leaves ? nullptr : p.out_off,
                                      p.out_items, p.out_supp, p.cap_sets, p.cap_items, p.class_sets, p.eoffx,
                                      p.entries_f);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !p.leaves) return e;
  k_level2_leaves<<<(p.n1 + 7) / 8, 256, 0, st>>>(p.C2, p.n1, p.minsup, p.frows, p.row_supp, p.rank_item, p.scnt,
                                                  p.soff, p.sitems, p.out_off, p.out_items, p.out_supp, p.cap_sets,
                                                  p.cap_items, p.ctrl);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_level2(const LevelLaunch& p, cudaStream_t st) {
  cudaError_t e = launch_level2_counts(p, st);
  if (e != cudaSuccess) return e;
  return launch_level2_fill(p, st);
}

uint32_t dfs_sparse_cap(uint32_t stride) { return std::min<uint32_t>(kSparseCap, std::max<uint32_t>(32, stride / 4)); }

size_t dfs_smem_bytes(uint32_t stride, uint32_t max_len, uint32_t maxd, bool prefix_in_smem, uint32_t mode) {
  if (mode == 4)  // per warp: path ids, sorted ids, frame cursors and sizes
    return (size_t)(kWarpDfsThreads / 32) * (2ull * (max_len + 1) + 2ull * (maxd + 2)) * sizeof(uint32_t);
  if (mode == 3) {  // listed prefix: values (16 B) + indices (2 B) per entry
    const size_t cap = dfs_sparse_cap(stride);
    return (4ull * cap + kCandBatch + 2ull * (maxd + 1) + 3ull * (max_len + 1) + cap / 2 + 1) * sizeof(uint32_t);
  }
  size_t words = prefix_in_smem ? stride : 0;
  if (mode == 1) words += 2ull * kPairBatch + 8ull * (maxd + 1) + 3ull * (max_len + 1);
  else words += kCandBatch + 2ull * (maxd + 1) + 3ull * (max_len + 1) + (prefix_in_smem ? stride / 8 + 1 : 0);
  return words * sizeof(uint32_t);
}

bool dfs_prefix_fits(uint32_t stride, size_t smem_optin, uint32_t max_len, uint32_t maxd, uint32_t mode) {
  if (mode == 3 || mode == 4) return false;  // sparse nodes: listed prefixes; warp DFS: prefixes in registers
  return dfs_smem_bytes(stride, max_len, maxd, true, mode) + sizeof(Ctl) + sizeof(FrameCtl) + 33 * 4 + 512 <= smem_optin;
}

uint64_t dfs_arena_cta_words(uint32_t stride, uint32_t n1, uint32_t maxd, uint32_t mode) {
  if (mode == 4) return (uint64_t)(kWarpDfsThreads / 32) * (maxd + 1) * warp_slot_words(stride, n1);
  if (mode == 1) return frames_root_words(n1) + frames_depth_words(stride, n1) * (maxd + 1);
  return dfs_arena_depth_words(stride, n1) * (maxd + 1);
}

static cudaError_t dfs_max_ctas_per_sm_query(uint32_t threads, uint32_t vec, size_t smem, bool prefix_in_smem,
                                             uint32_t mode, int* out);

// occupancy of a launch shape, asked once per shape and device (the query costs microseconds of host
// time on every mine otherwise)
cudaError_t dfs_max_ctas_per_sm(uint32_t threads, uint32_t vec, size_t smem, bool prefix_in_smem, uint32_t mode,
                                int* out) {
  static std::mutex mu;
  static std::map<std::tuple<int, uint32_t, uint32_t, size_t, bool, uint32_t>, int> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(dev, threads, vec, smem, prefix_in_smem, mode);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *out = it->second;
      return cudaSuccess;
    }
  }
  e = dfs_max_ctas_per_sm_query(threads, vec, smem, prefix_in_smem, mode, out);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = *out;
  }
  return e;
}

static cudaError_t dfs_max_ctas_per_sm_query(uint32_t threads, uint32_t vec, size_t smem, bool prefix_in_smem,
                                             uint32_t mode, int* out) {
  if (mode == 4) return occ_warp(vec, smem, out);  // vec carries the row stride for the warp DFS
  if (mode == 3) {
    switch (vec) {
      case 16: return occ_sparse_t<16>(threads, smem, out);
      case 1: return occ_sparse_t<1>(threads, smem, out);
      case 2: return occ_sparse_t<2>(threads, smem, out);
      case 8: return occ_sparse_t<8>(threads, smem, out);
      default: return occ_sparse_t<4>(threads, smem, out);
    }
  }
  if (mode == 1) {
    if (prefix_in_smem) {
      switch (vec) {
        case 1: return occ_frames_t<1, true>(threads, smem, out);
        case 2: return occ_frames_t<2, true>(threads, smem, out);
        case 8: return occ_frames_t<8, true>(threads, smem, out);
        default: return occ_frames_t<4, true>(threads, smem, out);
      }
    }
    switch (vec) {
      case 1: return occ_frames_t<1, false>(threads, smem, out);
      case 2: return occ_frames_t<2, false>(threads, smem, out);
      case 8: return occ_frames_t<8, false>(threads, smem, out);
      default: return occ_frames_t<4, false>(threads, smem, out);
    }
  }
  if (prefix_in_smem) {
    switch (vec) {
      case 1: return occ_t<1, true>(threads, smem, out);
      case 2: return occ_t<2, true>(threads, smem, out);
      case 8: return occ_t<8, true>(threads, smem, out);
      default: return occ_t<4, true>(threads, smem, out);
    }
  }
  switch (vec) {
    case 1: return occ_t<1, false>(threads, smem, out);
    case 2: return occ_t<2, false>(threads, smem, out);
    case 8: return occ_t<8, false>(threads, smem, out);
    default: return occ_t<4, false>(threads, smem, out);
  }
}

cudaError_t launch_pool_init(uint32_t* pool, uint32_t slots, uint64_t slot_words, cudaStream_t st) {
  if (slots == 0) return cudaSuccess;
  k_pool_init<<<(slots + 255) / 256, 256, 0, st>>>(pool, slots, slot_words);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_dfs(const DfsLaunch& p, uint32_t grid, uint32_t threads, uint32_t vec, size_t smem,
                       bool prefix_in_smem, uint32_t max_len, uint32_t mode, cudaStream_t st) {
  DfsArgs a;
  a.p = p;
  a.stride4 = p.stride / 4;
  const uint32_t segw4 = 32u * vec;  // 16-byte vectors per piece
  a.nseg = (a.stride4 + segw4 - 1) / segw4;
  a.max_len = max_len;
  a.cap = dfs_sparse_cap(p.stride);
  if (mode == 4) return launch_warp(a, grid, smem, st);
  if (mode == 3) return launch_sparse_vec(a, grid, threads, vec, smem, st);
  if (mode == 1) {
    if (prefix_in_smem) return launch_frames_vec<true>(a, grid, threads, vec, smem, st);
    return launch_frames_vec<false>(a, grid, threads, vec, smem, st);
  }
  if (prefix_in_smem) return launch_dfs_vec<true>(a, grid, threads, vec, smem, st);
  return launch_dfs_vec<false>(a, grid, threads, vec, smem, st);
}

}  // namespace fim
