// Mining engine: one Eclat run over a set of frequent bitmap rows.
//
// prepare  - geometry of the persistent DFS, row lists on the device, fixed buffers
// alloc    - output and DFS-stack buffers (grow when a run overflows them)
// launch   - pair kernel, level-2 compaction and queue, persistent DFS: device
//            work only, so the same sequence can be captured in a CUDA graph
// finish   - read the control block, check the device-side error bits
#include <algorithm>
#include <cstring>
#include <vector>

#include "fim_internal.cuh"

namespace fim {

static uint32_t clamp_threads(uint32_t t) { return (t == 128 || t == 256 || t == 512) ? t : 256u; }
static uint32_t clamp_vec(uint32_t v, uint32_t mode) {
  return (v == 1 || v == 2 || v == 4 || v == 8 || (v == 16 && mode == 3)) ? v : 4u;
}
static constexpr uint64_t kMaxCap = 0xfffffff0ull;

fim_status engine_prepare(fim_db* db, Workspace& ws, const EngineInput& in, const EngineConfig& cfg, EnginePlan* ep) {
  cudaStream_t st = ws.stream;
  *ep = EnginePlan{};
  const uint32_t n1 = in.n1;
  ep->n1 = n1;
  ep->minsup = in.minsup;
  ep->stride = in.stride;
  ep->bytes_per_row_alg = in.bytes_per_row_alg;
  ep->bits = in.bits;
  ep->d_rank_item = in.d_rank_item;
  ep->num_sms = db->num_sms;
  // traversal: frame passes pay off on short rows (fewer dependent steps per intersection), node
  // expansion with sparse prefixes on long ones
  // (16-bit word indices: listed prefixes need rows of at most 65,535 16-byte words)
  // (warp DFS: the prefix in the registers of one warp, rows of at most 512 words)
  const bool list_ok = in.stride / 4 <= 65535;
  const bool warp_ok = in.stride <= 512 && !cfg.donate;
  // Automatic: the number of classes decides, not the row width.  At least 1,024 frequent rows (many
  // classes, throughput bound) take the projected DFS (FIM_DFS_PROJECTED), which runs with the sparse node
  // mode (ep->mode = 3) mining the classes left out of the projection: large_sparse 5.1 ms; its laws at
  // 50,000 transactions (rows of 1,568 words) 2.0 ms against 8.6 ms in frame passes and 7.4 in sparse
  // nodes.  Fewer rows, where the largest class's chain of dependent nodes sets the time, take frame
  // passes, which spread one frame over a whole CTA: sparse_mid (988 rows of 3,136 words) 0.021 ms against
  // 0.064 projected, 0.027 in sparse nodes and 0.033 in dense node expansion; at 300,000 transactions
  // (9,376 words) 0.033 against 0.084 projected; rows past 16,384 words take the sparse node mode.
  // A capped CTA count (the server's concurrent jobs) turns the projection's hand-out of large frames off,
  // and without it every class's whole subtree runs on one warp (the tail the hand-out removes), so such
  // mines keep the traversals that spread a class over a CTA.
  const bool auto_proj = cfg.mode == 2 && list_ok && !cfg.donate && n1 >= 1024 && cfg.ctas_per_sm == 0;
  if (cfg.mode == 2)
    ep->mode = auto_proj ? 3u : (in.stride <= 16384 ? 1u : (list_ok && !cfg.donate ? 3u : 0u));
  else if (cfg.mode == 3 || cfg.mode == 5) ep->mode = list_ok && !cfg.donate ? 3u : 0u;
  else if (cfg.mode == 4) ep->mode = warp_ok ? 4u : (list_ok && !cfg.donate ? 3u : 0u);
  else ep->mode = cfg.mode == 1 ? 1u : 0u;
  ep->proj = ep->mode == 3 && (cfg.mode == 5 || auto_proj);
  ep->leaves = cfg.output == FIM_OUTPUT_MAXIMAL;  // (mine_input made such a mine projected)
  ep->diffsets = cfg.diffsets;
  ep->donate = ep->mode == 0 ? cfg.donate : 0u;  // only dense node expansion donates
  ep->spin_limit = cfg.spin_limit ? cfg.spin_limit : 2000000ull;
  ep->fixed_capacity = cfg.fixed_capacity;
  ep->cap_sets = cfg.cap_sets ? cfg.cap_sets : std::max<uint64_t>((uint64_t)1 << 18, 8ull * n1 + 64);
  ep->cap_items = cfg.cap_items ? cfg.cap_items : ep->cap_sets * 6;
  ep->cap_sets = std::min(ep->cap_sets, kMaxCap);
  ep->cap_items = std::min(ep->cap_items, kMaxCap);
  FIM_TRY(ws_get(ws, WS_CTRL, 1, &ep->d_ctrl));
  if (n1 == 0) return FIM_OK;

  // row lists (pinned-staged uploads unless the caller already has them on the device)
  ep->d_frows = in.d_frows;
  ep->d_rsupp = in.d_row_supp;
  ep->d_order = in.identity_order ? db->d_iota : in.d_row_order;
  auto upload = [&](int slot, const std::vector<uint32_t>& v, const uint32_t** dst) -> fim_status {
    uint32_t* d = nullptr;
    void* h = nullptr;
    FIM_TRY(ws_get(ws, slot, n1, &d));
    FIM_TRY(stage_get(db, n1 * 4ull, &h));
    std::memcpy(h, v.data(), n1 * 4ull);
    FIM_CUDA(cudaMemcpyAsync(d, h, n1 * 4ull, cudaMemcpyHostToDevice, st));
    *dst = d;
    return FIM_OK;
  };
  if (!ep->d_frows) FIM_TRY(upload(WS_FROWS, in.frows, &ep->d_frows));
  if (!ep->d_rsupp) FIM_TRY(upload(WS_ROWSUPP, in.row_supp, &ep->d_rsupp));
  if (!ep->d_order) FIM_TRY(upload(WS_ROWORDER, in.row_order, &ep->d_order));

  ep->npairs_max = (uint64_t)n1 * (n1 - 1) / 2;
  FIM_TRY(ws_get(ws, WS_C2, (size_t)n1 * n1, &ep->d_C2));
  // level 2 on the tensor cores when asked, or when its modelled time is lower: fused with the widening
  // when the rows are consecutive, else through widened rows (at most 1/16 of the device memory; TMA
  // coordinates are signed 32-bit, so widened rows of less than 2^31 bytes)
  if (n1 >= 2) {
    // the fused kernel reads the raw rows by TMA, so they must be consecutive rows of the bitmap: every mine
    // of a whole database (the frequent rows are a suffix), and the estimate's sample when it takes all rows
    const bool consecutive = in.frows.size() == n1 && in.frows.back() - in.frows.front() == n1 - 1;
    ep->rows_base = consecutive ? in.bits + (size_t)in.frows.front() * in.stride : nullptr;
    ep->pair_e2m1 = cfg.pair_kernel != FIM_PAIR_TENSOR_E4M3;
    const uint64_t xb = pair_mma_buffer_bytes(n1, in.stride, ep->pair_e2m1);
    const bool coords_ok = (uint64_t)in.stride * 32 < (1ull << 31);
    const double cores_us = pair_cores_cost_us(n1, in.stride, db->num_sms);
    if (cfg.pair_kernel == FIM_PAIR_TENSOR_FUSED) {
      if (!consecutive) return fail(FIM_ERR_INVALID, "the fused tensor-core pair kernel needs consecutive rows");
      ep->pair_mma = ep->pair_fused = true;
    } else if (cfg.pair_kernel >= FIM_PAIR_TENSOR) {
      ep->pair_mma = coords_ok;
    } else if (cfg.pair_kernel == FIM_PAIR_AUTO) {
      if (consecutive)
        ep->pair_mma = ep->pair_fused = pair_mma_cost_us(n1, in.stride, db->num_sms, false, true) < cores_us;
      else
        ep->pair_mma = coords_ok && xb <= db->total_mem / 16 &&
                       pair_mma_cost_us(n1, in.stride, db->num_sms, ep->pair_e2m1) < cores_us;
    }
    if (ep->pair_mma && !ep->pair_fused) FIM_TRY(ws_get(ws, WS_PAIR_X, xb, &ep->d_X));
    ep->pair_extra_tx = cfg.fault_pair_wait ? 16u : 0u;
  }
  FIM_TRY(ws_get(ws, WS_SCNT, n1, &ep->d_scnt));
  FIM_TRY(ws_get(ws, WS_SOFF, 2ull * (n1 + 1), &ep->d_soff));
  FIM_TRY(ws_get(ws, WS_SITEMS, ep->npairs_max + 1, &ep->d_sitems));
  FIM_TRY(ws_get(ws, WS_ENTRIES, ep->npairs_max + 1, &ep->d_entries));
  ep->d_eoff = ep->d_soff + (n1 + 1);

  // persistent DFS geometry: itemsets are no longer than the longest transaction
  ep->L = std::max<uint32_t>(3, std::min<uint32_t>(in.max_len_bound, n1));
  ep->maxd_full = std::max<uint32_t>(1, ep->L - 2);
  // loads per lane: 4 (with three 256-thread sparse CTAs per SM, large_sparse takes 21.7 ms with 4 and
  // 22.5 ms with 8)
  ep->vec = cfg.vec ? clamp_vec(cfg.vec, ep->mode) : 4u;
  ep->psmem = dfs_prefix_fits(in.stride, db->smem_optin, ep->L, ep->maxd_full, ep->mode);
  ep->smem = dfs_smem_bytes(in.stride, ep->L, ep->maxd_full, ep->psmem, ep->mode);
  int occ = 0;
  if (ep->mode == 4) {  // warp DFS: CTAs of 8 warps; its occupancy query takes the row stride
    ep->threads = 256;
    FIM_CUDA(dfs_max_ctas_per_sm(256, in.stride, ep->smem, false, 4, &occ));
  } else if (cfg.threads == 0 && ep->mode == 3) {
    // sparse nodes: 256-thread CTAs (3 per SM under the kernel's 80-register bound), whose listed child
    // prefixes are built with twice the loads in flight (large_sparse: 21.7 ms against 32.1 ms with
    // 128-thread CTAs, 6 per SM; sparse_mid 0.027 against 0.029 ms; its 200,000-row variant prefers
    // 128 threads, 7.5 against 8.7 ms)
    ep->threads = 256;
    FIM_CUDA(dfs_max_ctas_per_sm(ep->threads, ep->vec, ep->smem, ep->psmem, ep->mode, &occ));
  } else if (cfg.threads == 0) {
    // The DFS is latency bound.  Node expansion runs one class node per CTA with CTA-wide barriers
    // between its steps, so more CTAs per SM (independent nodes in flight) beat bigger CTAs: the
    // most CTAs per SM, then the most warps.  Frame passes spread one pass over the whole CTA: the
    // most warps (256 on a tie).
    const uint32_t cand[3] = {128, 256, 512};
    int best_occ = 0;
    uint32_t best_t = 256;
    for (uint32_t t : cand) {
      if (ep->mode == 1 && t == 128) continue;
      if (ep->mode == 3 && t > 256) continue;  // the sparse kernel's launch bound
      int o = 0;
      FIM_CUDA(dfs_max_ctas_per_sm(t, ep->vec, ep->smem, ep->psmem, ep->mode, &o));
      if (o < 1) continue;
      const bool better = ep->mode == 1 ? (uint64_t)o * t > (uint64_t)best_occ * best_t
                                        : (o > best_occ || (o == best_occ && t > best_t));
      if (best_occ == 0 || better) {
        best_occ = o;
        best_t = t;
      }
    }
    ep->threads = best_t;
    occ = best_occ;
  } else {
    ep->threads = clamp_threads(cfg.threads);
    if (ep->mode == 3) ep->threads = std::min<uint32_t>(ep->threads, 256);  // the sparse kernel's launch bound
    FIM_CUDA(dfs_max_ctas_per_sm(ep->threads, ep->vec, ep->smem, ep->psmem, ep->mode, &occ));
  }
  if (occ < 1) return fail(FIM_ERR_INVALID, "persistent kernel does not fit on an SM");
  const uint32_t cps = cfg.ctas_per_sm ? std::min<uint32_t>(cfg.ctas_per_sm, occ) : (uint32_t)occ;
  ep->grid = std::max<uint32_t>(1, (uint32_t)db->num_sms * cps);
  // DFS stack depth: the full bound when its arena fits in 1/32 of the device memory (no run can
  // then fail for depth); otherwise a shallow first stack, grown and the run repeated on demand
  const uint64_t full_bytes = 4ull * dfs_arena_cta_words(in.stride, n1, ep->maxd_full, ep->mode) * ep->grid;
  ep->maxd = full_bytes <= db->total_mem / 32 ? ep->maxd_full : std::min<uint32_t>(ep->maxd_full, kDfsDepthHint);
  if (cfg.depth_first) ep->maxd = std::min<uint32_t>(ep->maxd_full, cfg.depth_first);
  ep->per_depth = dfs_arena_depth_words(in.stride, n1);
  ep->pool_slots = ep->donate ? std::max<uint32_t>(8, ep->grid) : 0;
  ep->pool_slot_words = dfs_pool_slot_words(in.stride, ep->L, n1);
  if (ep->pool_slots) FIM_TRY(ws_get(ws, WS_POOL, ep->pool_slot_words * ep->pool_slots, &ep->d_pool));
  if (ep->proj) {
    // budgets of the class database parts: bitmaps up to a quarter of the frequent rows' bytes (at least
    // 64 MB, at most 1/32 of device memory); transactions: every frequent row's support (the exact bound);
    // a warp's stack takes eight prefixes of the widest projected class
    ep->proj_y_cap = std::min<uint64_t>(db->total_mem / 128,
                                        std::max<uint64_t>((uint64_t)n1 * in.stride / 4, 16ull << 20));
    ep->proj_t_cap = 0;
    for (uint32_t s : in.row_supp) ep->proj_t_cap += ((uint64_t)s + 3) & ~3ull;
    // (a database remembers the stack its earlier mines grew to, so that a mine is not repeated for it)
    ep->pstack_words = ((cfg.pstack_words ? cfg.pstack_words : std::max<uint64_t>(kProjStackWords, db->proj_stack_words)) +
                        31) & ~31ull;
    // widest projected class: eight prefixes of it fit the first stack (a frame that keeps its class's width
    // materialises one prefix per level)
    const uint64_t base_stack = cfg.pstack_words ? cfg.pstack_words : kProjStackWords;
    ep->proj_w_cap = cfg.proj_w_cap ? cfg.proj_w_cap : (uint32_t)std::min<uint64_t>(base_stack / 8, 1u << 20);
    if (cfg.proj_y_cap) ep->proj_y_cap = cfg.proj_y_cap;
    ep->proj_smem = dfs_proj_smem_bytes(ep->L);
    int pocc = 0;
    FIM_CUDA(dfs_proj_ctas_per_sm(ep->proj_smem, &pocc));
    if (pocc < 1) return fail(FIM_ERR_INVALID, "projected DFS kernel does not fit on an SM");
    // a capped CTA count (the server's concurrent jobs) also turns the work sharing off: warps then leave as
    // soon as the static queue is empty instead of waiting for handed-out frames
    const bool share = cfg.ctas_per_sm == 0;
    if (!share) pocc = std::min<int>(pocc, (int)cfg.ctas_per_sm);
    ep->proj_grid = (uint32_t)db->num_sms * (uint32_t)pocc;
    uint32_t* meta = nullptr;
    FIM_TRY(ws_get(ws, WS_PROJ_META, 6ull * n1 + 2, &meta));
    ep->d_yoff = reinterpret_cast<uint64_t*>(meta);
    ep->d_toff = ep->d_yoff + n1;
    ep->d_itemoff = meta + 4ull * n1;
    ep->d_eoffx = ep->d_itemoff + n1 + 1;
    FIM_TRY(ws_get(ws, WS_ENTRIES_F, ep->npairs_max + 1, &ep->d_entries_f));
    // the arena holds the class regions (within proj_y_cap), then the regions of split frames
    ep->proj_arena_words = ep->proj_y_cap + (share ? std::max<uint64_t>(ep->proj_y_cap, 16ull << 20) : 0ull);
    ep->split_words = cfg.split_words;  // 0: chosen on the device from the class regions' mean width
    ep->dq_cap = share ? kProjDqCap : 0u;
    FIM_TRY(ws_get(ws, WS_PROJ_Y, ep->proj_arena_words, &ep->d_Y));
    FIM_TRY(ws_get(ws, WS_PROJ_DQ, std::max<uint32_t>(1, ep->dq_cap), &ep->d_dq));
    FIM_TRY(ws_get(ws, WS_PROJ_T, std::max<uint64_t>(4, ep->proj_t_cap), &ep->d_T));
  }
  if (cfg.collect_times)
    for (auto& e : ep->ev) FIM_CUDA(cudaEventCreate(&e));
  return FIM_OK;
}

fim_status engine_alloc(Workspace& ws, EnginePlan* ep) {
  if (!ep->count_only) {
    FIM_TRY(ws_get(ws, WS_OUT_OFF, ep->cap_sets + 1, &ep->d_off));
    FIM_TRY(ws_get(ws, WS_OUT_ITEMS, std::max<uint64_t>(1, ep->cap_items), &ep->d_items));
    FIM_TRY(ws_get(ws, WS_OUT_SUPP, std::max<uint64_t>(1, ep->cap_sets), &ep->d_supp));
  }
  if (ep->n1 >= 3)
    FIM_TRY(ws_get(ws, WS_ARENA, dfs_arena_cta_words(ep->stride, ep->n1, ep->maxd, ep->mode) * ep->grid, &ep->d_arena));
  if (ep->n1 >= 3 && ep->proj)
    FIM_TRY(ws_get(ws, WS_PSTACK, (uint64_t)ep->proj_grid * (kProjThreads / 32) * ep->pstack_words, &ep->d_pstack));
  if (ep->n1 >= 3 && ep->ev[0])
    FIM_TRY(ws_get(ws, WS_CTATIME, 2ull * std::max(ep->grid, ep->proj_grid), &ep->d_cta_time));
  return FIM_OK;
}

cudaError_t engine_launch(const EnginePlan& ep, cudaStream_t st) {
  cudaError_t ce = engine_launch_front(ep, st, !ep.skip_pairs);
  return ce != cudaSuccess ? ce : engine_launch_back(ep, st);
}

cudaError_t engine_launch_front(const EnginePlan& ep, cudaStream_t st, bool pairs) {
  cudaError_t ce = cudaMemsetAsync(ep.d_ctrl, 0, sizeof(DevCtrl), st);
  if (ce != cudaSuccess || ep.n1 == 0) return ce;
  if (ep.d_class_work) {
    ce = cudaMemsetAsync(ep.d_class_work, 0, (size_t)ep.n1 * sizeof(unsigned long long), st);
    if (ce != cudaSuccess) return ce;
  }
  if (ep.pool_slots) {
    ce = launch_pool_init(ep.d_pool, ep.pool_slots, ep.pool_slot_words, st);
    if (ce != cudaSuccess) return ce;
  }
  if (ep.ev[0]) cudaEventRecord(ep.ev[0], st);
  if (pairs) {
    uint32_t ksplit = 0;
    PairLaunch pl{ep.bits, ep.stride, ep.d_frows, ep.n1, ep.d_C2, 0, ep.rows_base};
    ce = ep.pair_fused ? launch_pair_mma_fused(pl, &ep.d_ctrl->err, ep.num_sms, st, &ksplit, ep.pair_extra_tx)
         : ep.pair_mma ? launch_pair_mma(pl, ep.d_X, ep.pair_e2m1, &ep.d_ctrl->err, ep.num_sms, st, &ksplit,
                                         ep.pair_extra_tx)
                       : launch_pair_counts(pl, ep.num_sms, st, &ksplit);
    if (ce != cudaSuccess) return ce;
  }
  if (ep.ev[1]) cudaEventRecord(ep.ev[1], st);
  return cudaSuccess;
}

cudaError_t engine_launch_back(const EnginePlan& ep, cudaStream_t st) {
  if (ep.n1 == 0) return cudaSuccess;
  cudaError_t ce = cudaSuccess;
  LevelLaunch ll{ep.d_C2, ep.n1, ep.minsup, ep.d_frows, ep.d_rsupp, ep.d_rank_item, ep.d_order, ep.d_scnt,
                 ep.d_soff, ep.d_eoff, ep.d_sitems, ep.d_entries, ep.d_off, ep.d_items, ep.d_supp,
                 ep.count_only ? 0ull : ep.cap_sets, ep.count_only ? 0ull : ep.cap_items, ep.d_ctrl,
                 ep.d_class_sets};
  ll.leaves = ep.leaves ? 1u : 0u;
  ProjLaunch pj{};
  if (ep.proj && ep.n1 >= 3) {
    // level-2 counts, the projection plan (which classes get their database part, and the split of the
    // queue), then the queue fill
    pj = ProjLaunch{ep.bits, ep.stride, ep.d_frows, ep.d_rsupp, ep.d_order, ep.d_scnt, ep.d_soff, ep.d_sitems,
                    ep.d_rank_item, ep.n1, ep.proj_y_cap, ep.proj_t_cap, ep.proj_w_cap, ep.d_yoff, ep.d_toff,
                    ep.d_itemoff, ep.d_eoffx, ep.d_Y, ep.d_T, ep.d_ctrl};
    ce = launch_level2_counts(ll, st);
    if (ce != cudaSuccess) return ce;
    ce = launch_proj_plan(pj, st);
    if (ce != cudaSuccess) return ce;
    ll.eoffx = ep.d_eoffx;
    ll.entries_f = ep.d_entries_f;
    ce = launch_level2_fill(ll, st);
  } else {
    ce = launch_level2(ll, st);
  }
  if (ce != cudaSuccess) return ce;
  if (ep.ev[2]) cudaEventRecord(ep.ev[2], st);
  if (ep.n1 >= 3) {
    DfsLaunch dl{};
    dl.bits = ep.bits;
    dl.stride = ep.stride;
    dl.frows = ep.d_frows;
    dl.n1 = ep.n1;
    dl.minsup = ep.minsup;
    dl.rank_item = ep.d_rank_item;
    dl.soff = ep.d_soff;
    dl.scnt = ep.d_scnt;
    dl.sitems = ep.d_sitems;
    dl.entries = ep.d_entries;
    dl.arena = ep.d_arena;
    dl.arena_cta_words = dfs_arena_cta_words(ep.stride, ep.n1, ep.maxd, ep.mode);
    dl.maxd = ep.maxd;
    dl.pool = ep.d_pool;
    dl.pool_slots = ep.pool_slots;
    dl.pool_slot_words = ep.pool_slot_words;
    dl.out_off = ep.d_off;
    dl.out_items = ep.d_items;
    dl.out_supp = ep.d_supp;
    dl.cap_sets = ep.count_only ? 0ull : ep.cap_sets;
    dl.cap_items = ep.count_only ? 0ull : ep.cap_items;
    dl.class_sets = ep.d_class_sets;
    dl.C2 = ep.d_C2;
    dl.ctrl = ep.d_ctrl;
    dl.spin_limit = ep.spin_limit;
    dl.donate = ep.donate;
    dl.class_work = ep.d_class_work;
    dl.max_sets = ep.max_sets;
    dl.cta_time = ep.d_cta_time;
    dl.leaves = ep.leaves ? 1u : 0u;
    dl.diffsets = ep.diffsets;
    if (ep.proj) {
      // Phase 3 (the classes' database parts), Phase 4 (one warp per two-item class), then the sparse
      // node mode on the classes left out
      ce = launch_proj_build(pj, ep.num_sms, st);
      if (ce != cudaSuccess) return ce;
      if (ep.dq_cap) {
        ce = cudaMemsetAsync(ep.d_dq, 0, (size_t)ep.dq_cap * sizeof(uint4), st);  // no slot published yet
        if (ce != cudaSuccess) return ce;
      }
      DfsLaunch dp = dl;
      dp.row_supp = ep.d_rsupp;
      dp.yoff = ep.d_yoff;
      dp.Y = ep.d_Y;
      dp.pstack = ep.d_pstack;
      dp.pstack_words = ep.pstack_words;
      dp.dq = ep.d_dq;
      dp.dq_cap = ep.dq_cap;
      dp.arena_words = ep.proj_arena_words;
      dp.split_words = ep.split_words;
      ce = launch_dfs_proj(dp, ep.proj_grid, ep.L, st);
      if (ce != cudaSuccess) return ce;
      dl.entries = ep.d_entries_f;
      dl.queue_sel = 1;
      dl.cta_time = nullptr;
    }
    ce = launch_dfs(dl, ep.grid, ep.threads, ep.vec, ep.smem, ep.psmem, ep.L, ep.mode, st);
    if (ce != cudaSuccess) return ce;
  }
  if (ep.ev[3]) cudaEventRecord(ep.ev[3], st);
  return cudaSuccess;
}

uint64_t proj_footprint_bytes(uint32_t rows, uint32_t stride, uint64_t nnz, uint32_t grid) {
  const uint64_t y = std::max<uint64_t>((uint64_t)rows * stride / 4, 16ull << 20);  // class bitmaps (words)
  return 4ull * y + 4ull * nnz + 4ull * (uint64_t)grid * (kProjThreads / 32) * kProjStackWords +
         64ull * rows + (1ull << 20);
}

void engine_release_events(EnginePlan* ep) {
  for (auto& e : ep->ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
}

fim_status engine_finish(fim_db* db, cudaStream_t st, EnginePlan* ep, EngineOutput* out, fim_mine_stats* stats,
                         bool* retry) {
  *retry = false;
  *out = EngineOutput{};
  void* hstage = nullptr;
  void* hcls = nullptr;
  const unsigned long long* d_cls = ep->d_class_sets ? ep->d_class_sets : ep->d_class_work;
  const bool want_cls = ep->class_out && d_cls && ep->n1;
  const size_t ctrl_bytes = (sizeof(DevCtrl) + 63) & ~(size_t)63;
  FIM_TRY(stage_get(db, ctrl_bytes + (want_cls ? ep->n1 * 8ull : 0ull), &hstage));
  FIM_CUDA(cudaMemcpyAsync(hstage, ep->d_ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, st));
  if (want_cls) {  // the per-class counters travel with the control block (one round trip)
    hcls = static_cast<uint8_t*>(hstage) + ctrl_bytes;
    FIM_CUDA(cudaMemcpyAsync(hcls, d_cls, ep->n1 * 8ull, cudaMemcpyDeviceToHost, st));
  }
  FIM_CUDA(cudaStreamSynchronize(st));
  db->stage_used = 0;
  DevCtrl h;
  std::memcpy(&h, hstage, sizeof(DevCtrl));
  if (want_cls) {
    ep->class_out->resize(ep->n1);
    std::memcpy(ep->class_out->data(), hcls, ep->n1 * 8ull);
  }
  out->ctrl = h;
  if (ep->ev[0] && ep->n1 > 0) {
    float t = 0.f;
    if (!ep->skip_pairs && cudaEventElapsedTime(&t, ep->ev[0], ep->ev[1]) == cudaSuccess) ep->ms_pair = t;
    if (cudaEventElapsedTime(&t, ep->ev[0], ep->ev[3]) == cudaSuccess) ep->ms_total += t;
  }
  if (h.err & DEV_ERR_TIMEOUT) return fail(FIM_ERR_TIMEOUT, "persistent kernel: bounded wait ran out without progress");
  if ((h.err & DEV_ERR_ABORTED) || (ep->max_sets && h.sets_total > ep->max_sets))
    return fail(FIM_ERR_OUTPUT_OVERFLOW, "more frequent itemsets than the limit: mining stopped early (counts are lower bounds)");
  if (h.err & DEV_ERR_PSTACK) {  // a warp's stack of the projected DFS was too small: double it and repeat
    // (at least twice the largest stack a class asked for before the warps stopped)
    // (a multiple of 32 words, so every warp's stack starts on a 128-byte line)
    const uint64_t next = (std::max<uint64_t>(ep->pstack_words * 2, 2ull * h.pstack_need) + 31) & ~31ull;
    if (next * ep->proj_grid * (kProjThreads / 32) * 4 > db->total_mem / 8)
      return fail(FIM_ERR_OOM, "projected DFS: the warps' stacks would exceed 1/8 of device memory");
    ep->pstack_words = next;
    db->proj_stack_words = std::max(db->proj_stack_words, next);
    *retry = true;
    return FIM_OK;
  }
  if (h.err & DEV_ERR_DEPTH) {
    if (ep->maxd >= ep->maxd_full) return fail(FIM_ERR_INVALID, "itemset longer than the depth bound of the DFS stack");
    ep->maxd = ep->maxd_full;  // deeper than the first stack: repeat with the full bound
    *retry = true;
    return FIM_OK;
  }
  if (!ep->count_only && (h.sets_total > ep->cap_sets || h.items_total > ep->cap_items)) {
    if (h.sets_total > kMaxCap || h.items_total > kMaxCap)
      return fail(FIM_ERR_OUTPUT_OVERFLOW, "result exceeds 2^32 sets or items");
    if (ep->fixed_capacity) return fail(FIM_ERR_OUTPUT_OVERFLOW, "output capacity exceeded");
    ep->cap_sets = std::min<uint64_t>(kMaxCap, h.sets_total + h.sets_total / 16 + 16);
    ep->cap_items = std::min<uint64_t>(kMaxCap, h.items_total + h.items_total / 16 + 16);
    *retry = true;
    return FIM_OK;
  }
  if (ep->d_off) {
    void* hfin = nullptr;
    FIM_TRY(stage_get(db, sizeof(uint64_t), &hfin));
    *static_cast<uint64_t*>(hfin) = h.items_total;
    FIM_CUDA(cudaMemcpyAsync(ep->d_off + h.sets_total, hfin, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  }
  out->n_sets = h.sets_total;
  out->n_items = h.items_total;
  out->d_off = ep->d_off;
  out->d_items = ep->d_items;
  out->d_supp = ep->d_supp;
  if (stats) {
    const uint64_t rb = ep->bytes_per_row_alg;
    const uint32_t n1 = ep->n1;
    stats->n_frequent_items = n1;
    stats->words_per_row = ep->stride;
    stats->n_frequent = h.sets_total;
    stats->n_items_out = h.items_total;
    stats->max_len = h.max_len;
    stats->n_pair_intersections = ep->npairs_max;
    stats->n_intersections = ep->npairs_max + h.n_intersections;
    stats->n_classes = h.n_nodes;
    stats->n_queue_entries = h.n_entries + (ep->proj ? h.n_entries_f : 0u);
    stats->n_donations = h.n_donations;
    // sibling operand per intersection + one prefix read per class node + materialised prefixes
    stats->bytes_pair_kernel = ep->npairs_max * rb + (uint64_t)(n1 > 0 ? n1 - 1 : 0) * rb;
    stats->bytes_dfs_kernel = h.n_intersections * rb + h.n_nodes * rb + h.n_frames * rb;
    stats->bytes_algorithmic = stats->bytes_pair_kernel + stats->bytes_dfs_kernel;
    stats->grid_ctas = n1 >= 3 ? ep->grid : 0;
    stats->threads_per_cta = ep->threads;
    stats->vec_per_lane = ep->vec;
    stats->pair_kernel = !ep->pair_mma   ? FIM_PAIR_CORES
                         : ep->pair_fused ? FIM_PAIR_TENSOR_FUSED
                         : ep->pair_e2m1  ? FIM_PAIR_TENSOR
                                          : FIM_PAIR_TENSOR_E4M3;
    stats->n_proj_classes = ep->proj ? h.n_proj_classes : 0u;
    stats->n_proj_splits = ep->proj ? h.proj_splits : 0u;
    stats->n_fallback_entries = ep->proj ? h.n_entries_f : 0u;
    stats->bytes_projected = ep->proj ? h.proj_bytes : 0u;
    if (ep->ev[0] && n1 > 0) {
      stats->ms_pair_kernel = ep->ms_pair;  // the one pair-kernel launch of this mine
      cudaEventElapsedTime(&stats->ms_dfs_kernel, ep->ev[2], ep->ev[3]);  // the last DFS run
      stats->ms_device_total = ep->ms_total;  // every launch, repeated runs included
    }
    const uint32_t tgrid = ep->proj ? ep->proj_grid : ep->grid;  // CTAs whose times were recorded
    if (ep->d_cta_time && tgrid) {  // load balance of the persistent DFS: busy time per CTA
      std::vector<unsigned long long> t(2ull * tgrid);
      FIM_CUDA(cudaMemcpyAsync(t.data(), ep->d_cta_time, t.size() * 8, cudaMemcpyDeviceToHost, st));
      FIM_CUDA(cudaStreamSynchronize(st));
      double sum = 0.0, mx = 0.0;
      for (uint32_t c = 0; c < tgrid; ++c) {
        const double b = t[2 * c + 1] > t[2 * c] ? (double)(t[2 * c + 1] - t[2 * c]) * 1e-6 : 0.0;
        sum += b;
        mx = std::max(mx, b);
      }
      stats->dfs_cta_busy_max_ms = (float)mx;
      stats->dfs_cta_busy_mean_ms = (float)(sum / tgrid);
    }
  }
  return FIM_OK;
}

fim_status engine_mine(fim_db* db, Workspace& ws, const EngineInput& in, const EngineConfig& cfg, EngineOutput* out,
                       fim_mine_stats* stats, EnginePlan* plan_out, const std::function<fim_status(EnginePlan*)>& after_pairs) {
  EnginePlan ep;
  fim_status s = engine_prepare(db, ws, in, cfg, &ep);
  if (s == FIM_OK && cfg.class_work) ep.d_class_work = cfg.class_work;
  if (s == FIM_OK && cfg.class_sets) ep.d_class_sets = cfg.class_sets;
  ep.count_only = cfg.count_only;
  ep.class_out = cfg.class_out;
  ep.max_sets = cfg.max_sets;
  // the pair kernel first: it needs no output buffer, so whatever the hook waits for (a deferred estimate's
  // class costs and itemset count) overlaps with it
  if (s == FIM_OK) {
    const cudaError_t ce = engine_launch_front(ep, ws.stream, true);
    if (ce != cudaSuccess) s = cuda_fail(ce, "mining kernels");
  }
  if (s == FIM_OK && after_pairs) s = after_pairs(&ep);
  for (int attempt = 0; s == FIM_OK && attempt < 8; ++attempt) {
    if ((s = engine_alloc(ws, &ep)) != FIM_OK) break;
    cudaError_t ce = attempt ? engine_launch_front(ep, ws.stream, false) : cudaSuccess;
    if (ce == cudaSuccess) ce = engine_launch_back(ep, ws.stream);
    if (ce != cudaSuccess) {
      s = cuda_fail(ce, "mining kernels");
      break;
    }
    bool retry = false;
    s = engine_finish(db, ws.stream, &ep, out, stats, &retry);
    if (s != FIM_OK || !retry) break;
    if (attempt == 7) s = fail(FIM_ERR_OUTPUT_OVERFLOW, "output capacity still exceeded after regrowth");
    ep.skip_pairs = true;  // the pair counts in the workspace stay valid: only the later stages repeat
  }
  ep.skip_pairs = false;
  if (plan_out && s == FIM_OK) {
    *plan_out = ep;
    for (auto& e : ep.ev) e = nullptr;  // events belong to the caller's copy now
  }
  engine_release_events(&ep);
  return s;
}

}  // namespace fim
