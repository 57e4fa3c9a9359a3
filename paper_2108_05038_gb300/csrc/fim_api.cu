// C ABI of the miner (include/fim.h): database build, sample-based class-cost
// estimate, mining engine orchestration and result handling.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "fim_internal.cuh"

namespace fim {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void note_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Function attributes belong to the device that is current when they are set, so they are set once
// per (device, kernel).
cudaError_t kernel_smem_limit(const void* func, int bytes) {
  static std::mutex mu;
  static std::vector<std::pair<int, const void*>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& d : done)
    if (d.first == dev && d.second == func) return cudaSuccess;
  if (bytes < 0) {  // the device maximum, less the kernel's static shared memory
    int optin = 0;
    cudaFuncAttributes fa{};
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    bytes = optin - (int)fa.sharedSizeBytes;
  }
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.emplace_back(dev, func);
  return e;
}
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }
fim_status fail(fim_status s, const std::string& msg) {
  set_error(msg);
  return s;
}
fim_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FIM_ERR_OOM : FIM_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// device memory: one stream-ordered pool per device owned by the library, with
// a release threshold high enough that freed blocks stay cached for the next
// call instead of going back to the driver at every synchronisation

static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

static cudaError_t lib_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t thr = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (e != cudaSuccess) return e;
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool;
  cudaError_t e = lib_pool(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

// ---------------------------------------------------------------------------
// pinned host staging: blocks are cached process-wide so that building many
// databases does not pay cudaMallocHost each time

static std::mutex g_pinned_mu;
static std::vector<std::pair<size_t, void*>> g_pinned_free;

static cudaError_t pinned_acquire(size_t bytes, void** p, size_t* cap) {
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    size_t best = (size_t)-1;
    for (size_t k = 0; k < g_pinned_free.size(); ++k)
      if (g_pinned_free[k].first >= bytes && (best == (size_t)-1 || g_pinned_free[k].first < g_pinned_free[best].first))
        best = k;
    if (best != (size_t)-1) {
      *p = g_pinned_free[best].second;
      *cap = g_pinned_free[best].first;
      g_pinned_free.erase(g_pinned_free.begin() + best);
      return cudaSuccess;
    }
  }
  *cap = bytes;
  return cudaMallocHost(p, bytes);
}

static void pinned_release(void* p, size_t cap) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  g_pinned_free.emplace_back(cap, p);
}

// A region of the database's pinned staging buffer, valid until the next
// synchronisation of its stream (callers reset the bump pointer after syncing).
fim_status stage_get(fim_db* db, size_t bytes, void** out) {
  bytes = (bytes + 63) & ~(size_t)63;
  if (db->stage_used + bytes > db->stage_cap) {
    // regions handed out since the last synchronisation may still be read or written by queued
    // copies: wait for them before reusing or replacing the buffer (nothing to wait for when none are)
    if (db->stage_used) FIM_CUDA(cudaStreamSynchronize(db->stream));
    db->stage_used = 0;
    if (bytes > db->stage_cap) {
      pinned_release(db->stage, db->stage_cap);
      db->stage = nullptr;
      db->stage_cap = 0;
      void* p = nullptr;
      size_t cap = 0;
      cudaError_t e = pinned_acquire(std::max<size_t>(bytes, 1 << 16), &p, &cap);
      if (e != cudaSuccess) return cuda_fail(e, "pinned staging allocation");
      db->stage = static_cast<uint8_t*>(p);
      db->stage_cap = cap;
    }
  }
  *out = db->stage + db->stage_used;
  db->stage_used += bytes;
  return FIM_OK;
}

fim_status stream_sync(fim_db* db) {
  FIM_CUDA(cudaStreamSynchronize(db->stream));
  db->stage_used = 0;
  return FIM_OK;
}

// ---------------------------------------------------------------------------
// workspace

fim_status Workspace::get(int slot, size_t nbytes, void** out) {
  if ((int)bufs.size() <= slot) bufs.resize(slot + 1);
  DevBuf& b = bufs[slot];
  if (nbytes == 0) nbytes = 16;
  if (b.cap < nbytes) {
    if (b.ptr) {
      cudaFreeAsync(b.ptr, stream);
      bytes -= b.cap;
      b.ptr = nullptr;
      b.cap = 0;
    }
    size_t cap = nbytes + nbytes / 4 + 256;
    cudaError_t e = dev_malloc_async(&b.ptr, cap, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b.ptr = nullptr;
      return cuda_fail(e, "workspace allocation");
    }
    b.cap = cap;
    bytes += cap;
  }
  *out = b.ptr;
  return FIM_OK;
}

void Workspace::release() {
  for (auto& b : bufs)
    if (b.ptr) cudaFreeAsync(b.ptr, stream);
  bufs.clear();
  bytes = 0;
}

// Workspaces of freed databases, per device, handed to the next database built on that device:
// a repeated build / estimate / mine then allocates nothing.  At most kWsCached workspaces and
// 1/16 of the device memory are kept; the memory is idle (its stream was synchronised).
static constexpr size_t kWsCached = 4;
static std::mutex g_ws_mu;
static std::vector<Workspace> g_ws_cache[64];

static void ws_take_cached(int dev, Workspace* ws) {
  if (dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(g_ws_mu);
  auto& c = g_ws_cache[dev];
  if (c.empty()) return;
  ws->bufs = std::move(c.back().bufs);
  ws->bytes = c.back().bytes;
  c.pop_back();
}

// called with the workspace's stream synchronised
static void ws_give_back(int dev, uint64_t total_mem, Workspace* ws) {
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lock(g_ws_mu);
    auto& c = g_ws_cache[dev];
    uint64_t held = ws->bytes;
    for (const auto& w : c) held += w.bytes;
    if (c.size() < kWsCached && held <= total_mem / 16) {
      Workspace keep;
      keep.bufs = std::move(ws->bufs);
      keep.bytes = ws->bytes;
      c.push_back(std::move(keep));
      ws->bufs.clear();
      ws->bytes = 0;
      return;
    }
  }
  ws->release();
}


// ---------------------------------------------------------------------------
// mining engine


// ---------------------------------------------------------------------------
// database build

// total device memory, asked once per device
static uint64_t device_total_mem(int dev) {
  static std::mutex mu;
  static uint64_t total[64] = {};
  if (dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(mu);
  if (!total[dev]) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) total[dev] = total_b;
    else cudaGetLastError();
  }
  return total[dev];
}

static fim_status db_init(fim_db* db, uint32_t D, uint32_t N, uint32_t word_bits, uint32_t prefilter,
                          void* stream) {
  db->D = D;
  db->N = N;
  db->word_bits = word_bits;
  db->prefilter = prefilter;
  db->stream = static_cast<cudaStream_t>(stream);
  db->ws.stream = db->stream;
  FIM_CUDA(cudaGetDevice(&db->device));
  FIM_CUDA(cudaDeviceGetAttribute(&db->num_sms, cudaDevAttrMultiProcessorCount, db->device));
  int optin = 0;
  FIM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, db->device));
  db->smem_optin = (size_t)optin;
  db->total_mem = device_total_mem(db->device);
  ws_take_cached(db->device, &db->ws);
  db->W32 = (D + 31) / 32;
  db->stride = ((db->W32 + 31) / 32) * 32;
  return FIM_OK;
}


// Items counted (K1) on the input CSR (the caller's device arrays or the db's
// copy of host arrays), the offsets validated on the device, rows relabelled on
// the host, the CSR copied into the db (device input), bitmaps built (K2).
static fim_status db_build_rows(fim_db* db, const uint32_t* src_off, const uint32_t* src_items, bool device_input) {
  cudaStream_t st = db->stream;
  const uint32_t N = db->N, D = db->D;
  uint32_t *d_cnt = nullptr, *d_flags = nullptr;
  FIM_TRY(ws_get(db->ws, WS_TALLY, (size_t)N + 4, &d_cnt));
  d_flags = d_cnt + N;  // [err, max_len, off[0], off[D]]
  FIM_CUDA(cudaMemsetAsync(d_cnt, 0, ((size_t)N + 4) * 4, st));
  FIM_CUDA(launch_item_count(src_off, src_items, D, N, d_cnt, d_flags, st));
  void* hcnt = nullptr;
  FIM_TRY(stage_get(db, ((size_t)N + 4) * 4, &hcnt));
  FIM_CUDA(cudaMemcpyAsync(hcnt, d_cnt, ((size_t)N + 4) * 4, cudaMemcpyDeviceToHost, st));
  // Without a prefilter every item gets a row (n_rows = N), so the bitmap block is known before the counts:
  // it is cleared behind the counts' copy, while the host waits for that copy alone and relabels the rows.
  const bool early_bits = db->prefilter == 0 && (size_t)N * db->stride > 0;
  if (early_bits) {
    if (!db->cnt_done) FIM_CUDA(cudaEventCreateWithFlags(&db->cnt_done, cudaEventDisableTiming));
    FIM_CUDA(cudaEventRecord(db->cnt_done, st));
    FIM_TRY(ws_get(db->ws, WS_DB_BITS, (size_t)N * db->stride, &db->d_bits));
    FIM_CUDA(cudaMemsetAsync(db->d_bits, 0, (size_t)N * db->stride * 4, st));
    FIM_CUDA(cudaEventSynchronize(db->cnt_done));
    db->stage_used = 0;
  } else {
    FIM_TRY(stream_sync(db));
  }
  std::vector<uint32_t> cnt(static_cast<uint32_t*>(hcnt), static_cast<uint32_t*>(hcnt) + N + 4);
  const uint32_t err = cnt[N];
  if (cnt[N + 2] != 0) return fail(FIM_ERR_INVALID, "tx_offsets[0] must be 0");
  if (err & DEV_ERR_OFFSETS) return fail(FIM_ERR_INVALID, "tx_offsets is not non-decreasing");
  if (err & DEV_ERR_ITEM_RANGE) return fail(FIM_ERR_INVALID, "an item id is >= N");
  db->max_tx_len = cnt[N + 1];
  if (device_input) {  // the offsets are valid: keep a copy of the CSR (the sample draw reads it)
    db->nnz = cnt[N + 3];
    FIM_TRY(ws_get(db->ws, WS_DB_TXOFF, (size_t)D + 1, &db->d_tx_off));
    FIM_TRY(ws_get(db->ws, WS_DB_TXITEMS, std::max<uint64_t>(1, db->nnz), &db->d_tx_items));
    FIM_CUDA(cudaMemcpyAsync(db->d_tx_off, src_off, ((size_t)D + 1) * 4, cudaMemcpyDeviceToDevice, st));
    if (db->nnz)
      FIM_CUDA(cudaMemcpyAsync(db->d_tx_items, src_items, db->nnz * 4ull, cudaMemcpyDeviceToDevice, st));
  }
  // kept items by ascending support, ties by id: one sort of (support, id) keys
  std::vector<uint64_t> key;
  key.reserve(N);
  for (uint32_t i = 0; i < N; ++i)
    if (cnt[i] >= db->prefilter) key.push_back(((uint64_t)cnt[i] << 32) | i);
  std::sort(key.begin(), key.end());
  std::vector<uint32_t> kept(key.size());
  for (size_t k = 0; k < key.size(); ++k) kept[k] = (uint32_t)key[k];
  db->n_rows = (uint32_t)kept.size();
  db->rank_item = kept;
  db->supp.resize(db->n_rows);
  db->item_rank.assign(N, -1);
  for (uint32_t r = 0; r < db->n_rows; ++r) {
    db->supp[r] = cnt[kept[r]];
    db->item_rank[kept[r]] = (int32_t)r;
  }
  // item_rank | rank_item | supp | iota in one block (each part 16-byte aligned), filled by one copy
  const size_t a4 = ((size_t)N + 3) & ~(size_t)3, r4 = ((size_t)db->n_rows + 3) & ~(size_t)3;
  uint32_t* small = nullptr;
  FIM_TRY(ws_get(db->ws, WS_DB_SMALL, a4 + 3 * r4 + 4, &small));
  db->d_item_rank = reinterpret_cast<int32_t*>(small);
  db->d_rank_item = small + a4;
  db->d_supp = small + a4 + r4;
  db->d_iota = small + a4 + 2 * r4;
  FIM_TRY(ws_get(db->ws, WS_DB_BITS, std::max<size_t>(1, (size_t)db->n_rows * db->stride), &db->d_bits));
  {
    void* h = nullptr;
    FIM_TRY(stage_get(db, (a4 + 2 * r4) * 4, &h));
    uint32_t* hu = static_cast<uint32_t*>(h);
    std::memcpy(hu, db->item_rank.data(), (size_t)N * 4);
    if (db->n_rows) {
      std::memcpy(hu + a4, db->rank_item.data(), (size_t)db->n_rows * 4);
      std::memcpy(hu + a4 + r4, db->supp.data(), (size_t)db->n_rows * 4);
    }
    FIM_CUDA(cudaMemcpyAsync(small, hu, (a4 + 2 * r4) * 4, cudaMemcpyHostToDevice, st));
  }
  FIM_CUDA(launch_iota(db->d_iota, db->n_rows, st));
  if (db->n_rows) {
    if (!early_bits) FIM_CUDA(cudaMemsetAsync(db->d_bits, 0, (size_t)db->n_rows * db->stride * 4, st));
    FIM_CUDA(launch_bitmap_build(db->d_tx_off, db->d_tx_items, D, db->d_item_rank, db->d_bits, db->stride, st));
  }
  return FIM_OK;
}

static fim_status build_common(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N,
                               uint32_t word_bits, uint32_t prefilter, void* stream, bool device_input,
                               fim_db** out) {
  if (!out) return fail(FIM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!off || D == 0 || N == 0) return fail(FIM_ERR_INVALID, "tx_offsets NULL or D == 0 or N == 0");
  if (word_bits != 32 && word_bits != 64) return fail(FIM_ERR_INVALID, "word_bits must be 32 or 64");
  fim_db* db = new (std::nothrow) fim_db();
  if (!db) return fail(FIM_ERR_OOM, "host allocation");
  fim_status s = db_init(db, D, N, word_bits, prefilter, stream);
  auto bail = [&](fim_status e) {
    fim_db_free(db);
    return e;
  };
  if (s != FIM_OK) return bail(s);
  cudaStream_t st = db->stream;
  if (device_input) {
    // counted and validated on the caller's arrays; copied once the offsets are known to be valid
    if (!items) return bail(fail(FIM_ERR_INVALID, "tx_items is NULL"));
    if ((s = db_build_rows(db, off, items, true)) != FIM_OK) return bail(s);
  } else {
    if (off[0] != 0) return bail(fail(FIM_ERR_INVALID, "tx_offsets[0] must be 0"));
    for (uint32_t t = 0; t < D; ++t)
      if (off[t + 1] < off[t]) return bail(fail(FIM_ERR_INVALID, "tx_offsets is not non-decreasing"));
    db->nnz = off[D];
    if (db->nnz > 0 && !items) return bail(fail(FIM_ERR_INVALID, "tx_items is NULL"));
    if ((s = ws_get(db->ws, WS_DB_TXOFF, (size_t)D + 1, &db->d_tx_off)) != FIM_OK) return bail(s);
    if ((s = ws_get(db->ws, WS_DB_TXITEMS, std::max<uint64_t>(1, db->nnz), &db->d_tx_items)) != FIM_OK)
      return bail(s);
    cudaError_t e = cudaMemcpyAsync(db->d_tx_off, off, ((size_t)D + 1) * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && db->nnz) e = cudaMemcpyAsync(db->d_tx_items, items, db->nnz * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "copying the CSR database"));
    if ((s = db_build_rows(db, db->d_tx_off, db->d_tx_items, false)) != FIM_OK) return bail(s);
  }
  *out = db;
  return FIM_OK;
}

static void rows_for_minsup(const fim_db* db, uint32_t minsup, EngineInput* in) {
  // rows are sorted by ascending support: the frequent ones are a suffix
  uint32_t r0 = (uint32_t)(std::lower_bound(db->supp.begin(), db->supp.end(), minsup) - db->supp.begin());
  in->n1 = db->n_rows - r0;
  in->frows.resize(in->n1);
  in->row_supp.resize(in->n1);
  for (uint32_t k = 0; k < in->n1; ++k) {
    in->frows[k] = r0 + k;
    in->row_supp[k] = db->supp[r0 + k];
  }
}

static void engine_config_from_opts(const fim_mine_opts* o, EngineConfig* c) {
  fim_mine_opts d;
  fim_mine_opts_init(&d);
  if (!o || o->struct_size == 0) o = &d;
  c->threads = o->threads_per_cta;  // 0: chosen by the engine
  c->vec = o->vec_per_lane;  // 0: chosen by the engine
  c->ctas_per_sm = o->ctas_per_sm;
  c->donate = o->donate;
  c->mode = o->dfs_mode;
  c->depth_first = o->dfs_depth_first;
  c->pair_kernel = o->pair_kernel;
  c->fault_pair_wait = o->fault_pair_wait;
  c->max_sets = o->max_itemsets;
  c->proj_y_cap = o->proj_bitmap_words;
  c->pstack_words = o->proj_stack_words;
  c->proj_w_cap = o->proj_max_row_words;
  c->split_words = o->proj_split_words;
  c->output = o->output;
  c->diffsets = o->diffsets;
  c->spin_limit = o->spin_limit;
  c->cap_sets = o->out_capacity_sets;
  c->cap_items = o->out_capacity_items;
  c->fixed_capacity = o->out_capacity_sets != 0 || o->out_capacity_items != 0;
  if (c->fixed_capacity) {
    if (!c->cap_sets) c->cap_sets = 1;
    if (!c->cap_items) c->cap_items = 1;
  }
  c->collect_times = o->collect_times != 0;
}


uint64_t estimate_capacity(const fim_db* db, uint32_t minsup_abs) {
  // first output capacity: |F| of the whole database at about the same relative minsup is of the order of
  // the sample's |F_s|, so a few times |F_s| usually avoids a second DFS run (when the sample's minsup had
  // to be raised, its count at the requested minsup passed the limit, so the limit is the better lower bound)
  if (!db->has_estimate || db->est_pending || !db->est_nfs || !(db->est_rel > 0.0)) return 0;
  const double rel = (double)minsup_abs / (double)db->D;
  if (std::fabs(rel - db->est_rel) > 0.1 * db->est_rel) return 0;
  const uint64_t f = db->est_doubled ? std::max<uint64_t>(db->est_nfs, db->est_limit) : db->est_nfs;
  return std::min<uint64_t>(4ull * f, 1ull << 28);
}

fim_status mine_input(fim_db* db, uint32_t minsup_abs, const fim_mine_opts* opts, EngineInput* in, EngineConfig* cfg,
                      bool defer_ok) {
  if (!db) return fail(FIM_ERR_INVALID, "db is NULL");
  if (minsup_abs == 0) return fail(FIM_ERR_INVALID, "minsup 0 makes every subset frequent");
  if (minsup_abs < db->prefilter) return fail(FIM_ERR_INVALID, "minsup below the prefilter support of the database");
  if (opts && opts->struct_size != 0 && opts->struct_size != sizeof(fim_mine_opts))
    return fail(FIM_ERR_INVALID, "fim_mine_opts.struct_size mismatch");
  rows_for_minsup(db, minsup_abs, in);
  in->bits = db->d_bits;
  in->stride = db->stride;
  in->bytes_per_row_alg = (uint32_t)(((uint64_t)db->D + db->word_bits - 1) / db->word_bits * (db->word_bits / 8));
  in->d_rank_item = db->d_rank_item;
  in->minsup = minsup_abs;
  in->max_len_bound = db->max_tx_len;
  if (in->n1) {
    in->d_frows = db->d_iota + (db->n_rows - in->n1);  // frequent rows are the suffix
    in->d_row_supp = db->d_supp + (db->n_rows - in->n1);
  }
  const uint32_t order = opts && opts->struct_size ? opts->class_order : (uint32_t)FIM_ORDER_ESTIMATE;
  in->row_order.clear();
  in->row_order.reserve(in->n1);
  if (!defer_ok || order != FIM_ORDER_ESTIMATE) {  // the host copies of a deferred estimate are needed now
    FIM_TRY(est_resolve(db));
  }
  if (order == FIM_ORDER_ESTIMATE) FIM_TRY(est_redo(db));  // an incomplete deferred sample, found by an earlier mine
  if (order == FIM_ORDER_ESTIMATE && db->has_estimate && db->est_pending && in->n1) {
    // the deferred estimate's order, restricted to this minsup's rows on the device
    uint32_t* d = nullptr;
    FIM_TRY(ws_get(db->ws, WS_ROWORDER, in->n1, &d));
    FIM_CUDA(launch_order_suffix(db->d_est_order, db->n_rows, db->n_rows - in->n1, d, db->stream));
    in->d_row_order = d;
  } else if (order == FIM_ORDER_ESTIMATE && db->has_estimate && in->n1) {
    const uint32_t r0 = db->n_rows - in->n1;
    for (uint32_t r : db->est_order)
      if (r >= r0) in->row_order.push_back(r - r0);
  } else {
    for (uint32_t k = 0; k < in->n1; ++k) in->row_order.push_back(k);
    in->identity_order = true;
  }
  engine_config_from_opts(opts, cfg);
  if (cfg->output > FIM_OUTPUT_MAXIMAL) return fail(FIM_ERR_INVALID, "unknown output kind");
  if (cfg->diffsets > 2) return fail(FIM_ERR_INVALID, "diffsets must be 0, 1 or 2");
  if (cfg->pair_kernel > FIM_PAIR_TENSOR_FUSED) return fail(FIM_ERR_INVALID, "unknown pair kernel");
  if (cfg->output == FIM_OUTPUT_MAXIMAL) {
    // the leaves are written by the projected DFS (and its sparse fallback)
    if (db->stride / 4 > 65535) return fail(FIM_ERR_INVALID, "maximal output needs rows of at most 65,535 16-byte words");
    cfg->mode = FIM_DFS_PROJECTED;
    cfg->donate = 0;
  }
  if (!cfg->cap_sets) {
    const uint64_t c = estimate_capacity(db, minsup_abs);
    if (c) cfg->cap_sets = c;
  }
  return FIM_OK;
}

fim_status make_result(cudaStream_t st, const EngineOutput& eo, bool on_dev, fim_result** out) {
  fim_result* res = new (std::nothrow) fim_result();
  if (!res) return fail(FIM_ERR_OOM, "host allocation");
  res->n_sets = eo.n_sets;
  res->n_items = eo.n_items;
  res->stream = st;
  cudaError_t e = cudaSuccess;
  if (on_dev) {
    res->on_device = 1;
    // one block: offsets (u64) | items | supports, each part 16-byte aligned
    const uint64_t b_off = (eo.n_sets + 1) * 8, b_items = (std::max<uint64_t>(1, eo.n_items) * 4 + 15) & ~15ull;
    const uint64_t b_supp = std::max<uint64_t>(1, eo.n_sets) * 4;
    void* blk = nullptr;
    e = dev_malloc_async(&blk, ((b_off + 15) & ~15ull) + b_items + b_supp, st);
    if (e == cudaSuccess) {
      res->d_off = static_cast<uint64_t*>(blk);
      res->d_items = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(blk) + ((b_off + 15) & ~15ull));
      res->d_supp = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(res->d_items) + b_items);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(res->d_off, eo.d_off, (eo.n_sets + 1) * 8, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && eo.n_items)
      e = cudaMemcpyAsync(res->d_items, eo.d_items, eo.n_items * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && eo.n_sets)
      e = cudaMemcpyAsync(res->d_supp, eo.d_supp, eo.n_sets * 4, cudaMemcpyDeviceToDevice, st);
  } else {
    // pinned host memory (pooled): the copies run at the link's rate instead of through staging buffers
    const uint64_t b_off = (eo.n_sets + 1) * 8, b_items = (eo.n_items * 4 + 15) & ~15ull;
    e = pinned_acquire(b_off + b_items + std::max<uint64_t>(1, eo.n_sets) * 4, &res->h_block, &res->h_cap);
    if (e == cudaSuccess) {
      res->h_off = static_cast<uint64_t*>(res->h_block);
      res->h_items = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(res->h_block) + b_off);
      res->h_supp = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(res->h_block) + b_off + b_items);
      e = cudaMemcpyAsync(res->h_off, eo.d_off, b_off, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess && eo.n_items)
      e = cudaMemcpyAsync(res->h_items, eo.d_items, eo.n_items * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && eo.n_sets)
      e = cudaMemcpyAsync(res->h_supp, eo.d_supp, eo.n_sets * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    fim_result_free(res);
    return cuda_fail(e, "copying the result");
  }
  *out = res;
  return FIM_OK;
}

}  // namespace fim

using namespace fim;

extern "C" {

void fim_mine_opts_init(fim_mine_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(fim_mine_opts);
  o->class_order = FIM_ORDER_ESTIMATE;
  o->dfs_mode = FIM_DFS_AUTO;
  o->donate = 0;
}

const char* fim_status_str(fim_status s) {
  switch (s) {
    case FIM_OK: return "FIM_OK";
    case FIM_ERR_INVALID: return "FIM_ERR_INVALID";
    case FIM_ERR_OOM: return "FIM_ERR_OOM";
    case FIM_ERR_OUTPUT_OVERFLOW: return "FIM_ERR_OUTPUT_OVERFLOW";
    case FIM_ERR_CUDA: return "FIM_ERR_CUDA";
    case FIM_ERR_TIMEOUT: return "FIM_ERR_TIMEOUT";
  }
  return "FIM_ERR_UNKNOWN";
}

const char* fim_last_error(void) { return g_last_error.c_str(); }

uint64_t fim_kernel_launches(void) { return launches_so_far(); }

fim_status fim_pool_memory(int device, uint64_t* used_bytes, uint64_t* reserved_bytes) {
  if (used_bytes) *used_bytes = 0;
  if (reserved_bytes) *reserved_bytes = 0;
  if (device < 0 || device >= 64) return fail(FIM_ERR_INVALID, "device ordinal out of range");
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    pool = g_pools[device];
  }
  if (!pool) return FIM_OK;
  uint64_t used = 0, reserved = 0;
  FIM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  FIM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
  if (used_bytes) *used_bytes = used;
  if (reserved_bytes) *reserved_bytes = reserved;
  return FIM_OK;
}

fim_status fim_build_vertical_db(const uint32_t* tx_offsets, const uint32_t* tx_items, uint32_t D, uint32_t N,
                                 uint32_t word_bits, uint32_t prefilter_minsup, void* cuda_stream, fim_db** out) {
  return build_common(tx_offsets, tx_items, D, N, word_bits, prefilter_minsup, cuda_stream, false, out);
}

fim_status fim_build_vertical_db_device(const uint32_t* d_tx_offsets, const uint32_t* d_tx_items, uint32_t D,
                                        uint32_t N, uint32_t word_bits, uint32_t prefilter_minsup,
                                        void* cuda_stream, fim_db** out) {
  return build_common(d_tx_offsets, d_tx_items, D, N, word_bits, prefilter_minsup, cuda_stream, true, out);
}

fim_status fim_db_info(const fim_db* db, uint32_t* D, uint32_t* N, uint32_t* n_rows, uint32_t* words_per_row,
                       uint32_t* word_bits, uint64_t* device_bytes) {
  if (!db) return fail(FIM_ERR_INVALID, "db is NULL");
  if (D) *D = db->D;
  if (N) *N = db->N;
  if (n_rows) *n_rows = db->n_rows;
  if (words_per_row) *words_per_row = db->stride;
  if (word_bits) *word_bits = db->word_bits;
  if (device_bytes) *device_bytes = db->device_bytes + db->ws.bytes;
  return FIM_OK;
}

fim_status fim_db_rows(const fim_db* db, uint32_t* rank_item, uint32_t* supports) {
  if (!db) return fail(FIM_ERR_INVALID, "db is NULL");
  if (rank_item && db->n_rows) std::memcpy(rank_item, db->rank_item.data(), db->n_rows * 4ull);
  if (supports && db->n_rows) std::memcpy(supports, db->supp.data(), db->n_rows * 4ull);
  return FIM_OK;
}

fim_status fim_estimate_class_costs(fim_db* db, double sample_rate, double rel_minsup, uint64_t seed,
                                    double* cost_out, uint32_t* order_out) {
  return fim_estimate_class_costs_ex(db, sample_rate, rel_minsup, seed, FIM_COST_ITEMSETS, FIM_SAMPLE_ITEMSET_LIMIT,
                                     cost_out, order_out);
}

fim_status fim_estimate_class_costs_ex(fim_db* db, double sample_rate, double rel_minsup, uint64_t seed,
                                       uint32_t cost_kind, uint64_t max_sample_itemsets, double* cost_out,
                                       uint32_t* order_out) {
  return fim::estimate_impl(db, sample_rate, rel_minsup, seed, cost_kind, max_sample_itemsets, cost_out, order_out,
                            true, 0);
}

}  // extern "C"

namespace fim {

// The estimate itself.  With allow_defer, no host output asked for, and a sample mined over all its rows
// (at most kEstDeviceRows), nothing waits for the device: the sample's count-only mine is only launched, a
// one-CTA kernel turns its per-class counts into the class costs and their LPT order on the device, and the
// control block, costs and order travel to a pinned block behind an event; est_resolve reads them when a
// caller needs them (fim_mine only after its pair kernel is on its way).  A deferred sample that ran into
// the itemset limit (or needed a retry) is mined again by the synchronous path after the mine that used it.
fim_status estimate_impl(fim_db* db, double sample_rate, double rel_minsup, uint64_t seed, uint32_t cost_kind,
                         uint64_t max_sample_itemsets, double* cost_out, uint32_t* order_out, bool allow_defer,
                         uint32_t first_minsup_s) {
  if (!db) return fail(FIM_ERR_INVALID, "db is NULL");
  if (cost_kind != FIM_COST_ITEMSETS && cost_kind != FIM_COST_INTERSECTIONS)
    return fail(FIM_ERR_INVALID, "unknown cost kind");
  if (!(sample_rate > 0.0 && sample_rate <= 1.0)) return fail(FIM_ERR_INVALID, "sample_rate must be in (0, 1]");
  if (!(rel_minsup >= 0.0 && rel_minsup <= 1.0)) return fail(FIM_ERR_INVALID, "rel_minsup must be in [0, 1]");
  cudaStream_t st = db->stream;
  // sample size: the requested rate, but never below the Theorem 6.1 size for eps = delta = 0.05
  const double m0 = std::ceil(std::log(2.0 / 0.05) / (2.0 * 0.05 * 0.05));
  double md = std::ceil(sample_rate * (double)db->D);
  md = std::max(md, std::min((double)db->D, m0));
  const uint32_t m = md < 1.0 ? 1u : (uint32_t)md;
  const double msd = std::ceil(rel_minsup * (double)m);
  uint32_t minsup_s = msd < 1.0 ? 1u : (uint32_t)msd;
  // (a redo of a deferred sample that passed the itemset limit starts where the doubling continues)
  if (first_minsup_s > minsup_s) minsup_s = first_minsup_s;
  const uint32_t sw = (m + 31) / 32, sstride = ((sw + 31) / 32) * 32;
  const uint32_t R = db->n_rows;
  uint32_t *d_sbits = nullptr, *d_ssupp = nullptr;
  FIM_TRY(ws_get(db->ws, WS_SAMPLE_BITS, (size_t)std::max<uint32_t>(R, 1) * sstride, &d_sbits));
  FIM_TRY(ws_get(db->ws, WS_SAMPLE_SUPP, std::max<uint32_t>(R, 1), &d_ssupp));
  std::vector<uint32_t> ssupp(R);
  // When nearly every row will be frequent in the sample (predicted from the full supports), the sample
  // is mined over all its rows with the supports left on the device: pairs with a row below the sample
  // minsup are not frequent anyway, and the level-2 kernels count only rows that reach it.  That saves
  // the host round trip for the sample supports; they come back with the mine's own synchronisation.
  uint32_t pred = 0;
  for (uint32_t r = 0; r < R; ++r) pred += (double)db->supp[r] * (double)m / (double)db->D >= (double)minsup_s;
  const bool all_rows = R > 0 && R <= 4096 && (uint64_t)pred * 4 >= (uint64_t)R * 3;
  void* h_ss = nullptr;
  size_t h_ss_cap = 0;
  bool have_ssupp = false;
  if (R) {
    FIM_CUDA(cudaMemsetAsync(d_sbits, 0, (size_t)R * sstride * 4, st));
    FIM_CUDA(launch_sample_build(db->d_tx_off, db->d_tx_items, db->D, db->d_item_rank, seed, m, d_sbits, sstride, st));
    FIM_CUDA(launch_row_popcount(d_sbits, sstride, R, d_ssupp, st));
    if (allow_defer && all_rows && !cost_out && !order_out && R <= kEstDeviceRows) {
      db->est_pending = false;  // (a pending earlier estimate is replaced)
      db->has_estimate = false;
      EngineInput in;
      in.bits = d_sbits;
      in.stride = sstride;
      in.bytes_per_row_alg = (uint32_t)(((uint64_t)m + db->word_bits - 1) / db->word_bits * (db->word_bits / 8));
      in.frows.resize(R);
      std::iota(in.frows.begin(), in.frows.end(), 0u);
      in.d_frows = db->d_iota;
      in.d_row_supp = d_ssupp;
      in.n1 = R;
      in.identity_order = true;
      in.d_rank_item = db->d_rank_item;
      in.minsup = minsup_s;
      in.max_len_bound = db->max_tx_len;
      EngineConfig cfg;
      cfg.donate = 0;
      unsigned long long* d_work = nullptr;
      FIM_TRY(ws_get(db->ws, WS_CLASSWORK, R, &d_work));
      EnginePlan ep;
      FIM_TRY(engine_prepare(db, db->ws, in, cfg, &ep));
      if (cost_kind == FIM_COST_INTERSECTIONS) ep.d_class_work = d_work;
      else ep.d_class_sets = d_work;
      ep.count_only = true;  // per-class counts, no itemset records
      ep.max_sets = max_sample_itemsets;
      FIM_TRY(engine_alloc(db->ws, &ep));
      FIM_CUDA(engine_launch(ep, st));
      uint32_t* d_est = nullptr;  // costs (R u64), then the order (R u32)
      FIM_TRY(ws_get(db->ws, WS_EST, 3ull * R, &d_est));
      unsigned long long* d_tally = reinterpret_cast<unsigned long long*>(d_est);
      uint32_t* d_order = d_est + 2ull * R;
      FIM_CUDA(launch_est_order(d_work, d_ssupp, minsup_s, cost_kind == FIM_COST_INTERSECTIONS, R, d_tally, d_order, st));
      const size_t ctrl_bytes = (sizeof(DevCtrl) + 63) & ~(size_t)63;
      const size_t need = ctrl_bytes + 12ull * R;
      if (db->est_pin_cap < need) {
        if (db->est_pin) FIM_CUDA(cudaStreamSynchronize(st));  // an earlier copy may still target the old block
        pinned_release(db->est_pin, db->est_pin_cap);
        db->est_pin = nullptr;
        db->est_pin_cap = 0;
        FIM_CUDA(pinned_acquire(need, &db->est_pin, &db->est_pin_cap));
      }
      uint8_t* pin = static_cast<uint8_t*>(db->est_pin);
      FIM_CUDA(cudaMemcpyAsync(pin, ep.d_ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, st));
      FIM_CUDA(cudaMemcpyAsync(pin + ctrl_bytes, d_est, 12ull * R, cudaMemcpyDeviceToHost, st));
      if (!db->est_done) FIM_CUDA(cudaEventCreateWithFlags(&db->est_done, cudaEventDisableTiming));
      FIM_CUDA(cudaEventRecord(db->est_done, st));
      db->d_est_order = d_order;
      db->est_pending = true;
      db->est_redo = false;
      db->has_estimate = true;
      db->est_nfs = 0;  // known once resolved
      db->est_m = m;
      db->est_minsup = minsup_s;
      db->est_rel = rel_minsup;
      db->est_limit = max_sample_itemsets;
      db->est_doubled = false;
      db->est_args = {sample_rate, rel_minsup, seed, max_sample_itemsets, cost_kind};
      return FIM_OK;
    }
    if (all_rows) {  // a pinned buffer of its own: the mine's retries may reuse the staging buffer
      FIM_CUDA(pinned_acquire((size_t)R * 4, &h_ss, &h_ss_cap));
      const cudaError_t ce = cudaMemcpyAsync(h_ss, d_ssupp, (size_t)R * 4, cudaMemcpyDeviceToHost, st);
      if (ce != cudaSuccess) {
        pinned_release(h_ss, h_ss_cap);
        return cuda_fail(ce, "sample supports");
      }
    } else {
      void* h = nullptr;
      FIM_TRY(stage_get(db, (size_t)R * 4, &h));
      FIM_CUDA(cudaMemcpyAsync(h, d_ssupp, (size_t)R * 4, cudaMemcpyDeviceToHost, st));
      FIM_TRY(stream_sync(db));
      std::memcpy(ssupp.data(), h, (size_t)R * 4);
      have_ssupp = true;
    }
  }
  struct PinnedGuard {  // returns the sample supports' buffer on every exit, once its copy is done
    void* p;
    size_t cap;
    cudaStream_t st;
    ~PinnedGuard() {
      if (!p) return;
      cudaStreamSynchronize(st);  // idle already after a mine; an early error may leave the copy queued
      pinned_release(p, cap);
    }
  } guard{h_ss, h_ss_cap, st};
  EngineInput in;
  EngineOutput eo;
  unsigned long long* d_work = nullptr;
  std::vector<unsigned long long> per;  // per-class counters, read back with the control block
  for (;;) {  // minsup_s doubles while the sample has more than max_sample_itemsets frequent itemsets
    in = EngineInput{};
    in.bits = d_sbits;
    in.stride = sstride;
    in.bytes_per_row_alg = (uint32_t)(((uint64_t)m + db->word_bits - 1) / db->word_bits * (db->word_bits / 8));
    if (all_rows) {  // every row, supports on the device (rows below minsup_s count as nothing)
      in.frows.resize(R);
      std::iota(in.frows.begin(), in.frows.end(), 0u);
      in.d_frows = db->d_iota;
      in.d_row_supp = d_ssupp;
    } else {
      for (uint32_t r = 0; r < R; ++r)
        if (ssupp[r] >= minsup_s) {
          in.frows.push_back(r);
          in.row_supp.push_back(ssupp[r]);
        }
    }
    in.n1 = (uint32_t)in.frows.size();
    in.row_order.resize(in.n1);
    std::iota(in.row_order.begin(), in.row_order.end(), 0u);
    in.identity_order = true;
    in.d_rank_item = db->d_rank_item;
    in.minsup = minsup_s;
    in.max_len_bound = db->max_tx_len;
    EngineConfig cfg;
    cfg.donate = 0;
    cfg.max_sets = max_sample_itemsets;
    cfg.count_only = true;  // the estimate needs per-class counts, not the itemsets themselves
    if (in.n1) {
      FIM_TRY(ws_get(db->ws, WS_CLASSWORK, in.n1, &d_work));
      if (cost_kind == FIM_COST_INTERSECTIONS) cfg.class_work = d_work;
      else cfg.class_sets = d_work;
      cfg.class_out = &per;
    }
    eo = EngineOutput{};
    const fim_status s = engine_mine(db, db->ws, in, cfg, &eo, nullptr);
    if (all_rows && !have_ssupp && (s == FIM_OK || s == FIM_ERR_OUTPUT_OVERFLOW)) {
      // the copy was queued before the mine's kernels, and the mine synchronised the stream
      std::memcpy(ssupp.data(), h_ss, (size_t)R * 4);
      have_ssupp = true;
    }
    if (s == FIM_OK) break;
    const bool over = max_sample_itemsets &&
                      ((eo.ctrl.err & DEV_ERR_ABORTED) || eo.ctrl.sets_total > max_sample_itemsets);
    if (!over || minsup_s == UINT32_MAX) return s;
    minsup_s = minsup_s > UINT32_MAX / 2 ? UINT32_MAX : 2 * minsup_s;
  }
  // per class (the lowest row of its itemsets): intersections = level-2 candidates (the later
  // frequent sample rows) + the DFS below; itemsets = {r}, its frequent pairs and the DFS sets
  std::vector<unsigned long long> tally(R, 0ull);
  per.resize(in.n1, 0ull);
  uint32_t later = 0;  // frequent sample rows after row i: its level-2 candidates
  for (uint32_t i = in.n1; i-- > 0;) {
    if (ssupp[in.frows[i]] < minsup_s) continue;  // (all-rows mine only) not a class of the sample
    tally[in.frows[i]] = per[i] + (cost_kind == FIM_COST_INTERSECTIONS ? later : 0ull);
    ++later;
  }
  unsigned long long total = 0;
  for (uint32_t r = 0; r < R; ++r) total += tally[r];
  db->est_cost.assign(R, 0.0);
  for (uint32_t r = 0; r < R; ++r) db->est_cost[r] = total ? (double)tally[r] / (double)total : 0.0;
  db->est_order.resize(R);
  std::iota(db->est_order.begin(), db->est_order.end(), 0u);
  {  // descending cost, ties by row (the order of a stable sort by cost); the tallies order the costs
    const std::vector<unsigned long long>& t = tally;
    std::sort(db->est_order.begin(), db->est_order.end(),
              [&](uint32_t a, uint32_t b) { return t[a] != t[b] ? t[a] > t[b] : a < b; });
  }
  db->has_estimate = true;
  db->est_nfs = eo.n_sets;
  db->est_m = m;
  db->est_minsup = minsup_s;
  db->est_rel = rel_minsup;
  db->est_limit = max_sample_itemsets;
  db->est_doubled = minsup_s != (msd < 1.0 ? 1u : (uint32_t)msd);
  if (cost_out && R) std::memcpy(cost_out, db->est_cost.data(), R * sizeof(double));
  if (order_out && R) std::memcpy(order_out, db->est_order.data(), R * sizeof(uint32_t));
  db->est_pending = false;
  db->est_redo = false;
  return FIM_OK;
}

// Waits for a deferred estimate and reads its control block, costs and order from the pinned block into the
// database's host copies; a sample past the itemset limit (or one that needed a retry) leaves the order of
// its partial counts and asks for the synchronous redo.
fim_status est_resolve(fim_db* db) {
  if (!db->est_pending) return FIM_OK;
  FIM_CUDA(cudaEventSynchronize(db->est_done));
  db->est_pending = false;
  const uint32_t R = db->n_rows;
  const size_t ctrl_bytes = (sizeof(DevCtrl) + 63) & ~(size_t)63;
  const uint8_t* pin = static_cast<const uint8_t*>(db->est_pin);
  DevCtrl h;
  std::memcpy(&h, pin, sizeof(DevCtrl));
  std::vector<unsigned long long> tally(R);
  std::memcpy(tally.data(), pin + ctrl_bytes, 8ull * R);
  db->est_order.resize(R);
  std::memcpy(db->est_order.data(), pin + ctrl_bytes + 8ull * R, 4ull * R);
  unsigned long long total = 0;
  for (uint32_t r = 0; r < R; ++r) total += tally[r];
  db->est_cost.assign(R, 0.0);
  for (uint32_t r = 0; r < R; ++r) db->est_cost[r] = total ? (double)tally[r] / (double)total : 0.0;
  db->est_nfs = h.sets_total;
  const bool over = (h.err & DEV_ERR_ABORTED) || (db->est_limit && h.sets_total > db->est_limit);
  db->est_redo = over || (h.err & (DEV_ERR_TIMEOUT | DEV_ERR_PSTACK | DEV_ERR_DEPTH)) != 0;
  // past the itemset limit: the synchronous path continues the doubling from twice this minsup (and until
  // then the first output capacity is bounded by the limit, as after a doubling)
  db->est_redo_minsup = over ? (db->est_minsup > UINT32_MAX / 2 ? UINT32_MAX : 2 * db->est_minsup) : 0u;
  db->est_doubled = over;
  return FIM_OK;
}

// The synchronous estimate of a deferred one that est_resolve found incomplete.  It runs when a later mine
// or query needs the estimate (not at the end of the mine that found it: a served job mines once).
fim_status est_redo(fim_db* db) {
  if (!db->est_redo) return FIM_OK;
  db->est_redo = false;
  const auto a = db->est_args;
  return estimate_impl(db, a.rate, a.rel, a.seed, a.kind, a.limit, nullptr, nullptr, false, db->est_redo_minsup);
}

}  // namespace fim

extern "C" {

fim_status fim_estimate_result(fim_db* db, double* cost_out, uint32_t* order_out) {
  if (!db) return fail(FIM_ERR_INVALID, "db is NULL");
  if (!db->has_estimate) return fail(FIM_ERR_INVALID, "no estimate computed");
  FIM_TRY(est_resolve(db));
  FIM_TRY(est_redo(db));
  const uint32_t R = db->n_rows;
  if (cost_out && R) std::memcpy(cost_out, db->est_cost.data(), R * sizeof(double));
  if (order_out && R) std::memcpy(order_out, db->est_order.data(), R * sizeof(uint32_t));
  return FIM_OK;
}

fim_status fim_estimate_sample_size(const fim_db* db, uint64_t* n_sample_fis, uint32_t* sample_rows,
                                    uint32_t* sample_minsup) {
  if (!db) return fail(FIM_ERR_INVALID, "db is NULL");
  if (!db->has_estimate) return fail(FIM_ERR_INVALID, "no estimate computed");
  FIM_TRY(est_resolve(const_cast<fim_db*>(db)));
  FIM_TRY(est_redo(const_cast<fim_db*>(db)));
  if (n_sample_fis) *n_sample_fis = db->est_nfs;
  if (sample_rows) *sample_rows = db->est_m;
  if (sample_minsup) *sample_minsup = db->est_minsup;
  return FIM_OK;
}

fim_status fim_mine(fim_db* db, uint32_t minsup_abs, fim_mine_opts* opts, fim_result** out) {
  if (!out) return fail(FIM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  EngineInput in;
  EngineConfig cfg;
  FIM_TRY(mine_input(db, minsup_abs, opts, &in, &cfg, true));
  // a deferred estimate is read only once the pair kernel is launched: its output capacity comes from the
  // sample's itemset count
  auto after_pairs = [&](EnginePlan* ep) -> fim_status {
    if (!db->est_pending) return FIM_OK;
    FIM_TRY(est_resolve(db));
    const uint64_t c = cfg.cap_sets ? 0ull : estimate_capacity(db, minsup_abs);
    if (c) {
      ep->cap_sets = std::min<uint64_t>(c, 0xfffffff0ull);
      if (!cfg.cap_items) ep->cap_items = std::min<uint64_t>(ep->cap_sets * 6, 0xfffffff0ull);
    }
    return FIM_OK;
  };
  fim_mine_stats local_stats{};
  fim_mine_stats* stats = opts && opts->struct_size && opts->stats ? opts->stats : &local_stats;
  std::memset(stats, 0, sizeof(*stats));
  uint64_t* work_out = opts && opts->struct_size ? opts->class_work_out : nullptr;
  unsigned long long* d_work = nullptr;
  if (work_out && in.n1) {
    FIM_TRY(ws_get(db->ws, WS_CLASSWORK, in.n1, &d_work));
    cfg.class_work = d_work;
  }
  EngineOutput eo;
  fim_status s = engine_mine(db, db->ws, in, cfg, &eo, stats, nullptr, after_pairs);
  if (s == FIM_ERR_OUTPUT_OVERFLOW && opts && opts->struct_size) {
    opts->out_needed_sets = eo.ctrl.sets_total;
    opts->out_needed_items = eo.ctrl.items_total;
  }
  if (s != FIM_OK) return s;
  if (cfg.output != FIM_OUTPUT_ALL) {  // closed or maximal: the pass over the output's own supersets
    FIM_TRY(filter_output(db->ws, db->stream, cfg.output == FIM_OUTPUT_CLOSED ? 1 : 2, &eo, db->num_sms));
    stats->n_frequent = eo.n_sets;
    stats->n_items_out = eo.n_items;
  }
  if (work_out) {  // per row: level-2 candidates (the later frequent rows) + the DFS below the class
    std::fill(work_out, work_out + db->n_rows, 0ull);
    if (in.n1) {
      std::vector<unsigned long long> w(in.n1, 0ull);
      if (in.n1 >= 3) {
        void* h = nullptr;
        FIM_TRY(stage_get(db, (size_t)in.n1 * 8, &h));
        FIM_CUDA(cudaMemcpyAsync(h, d_work, (size_t)in.n1 * 8, cudaMemcpyDeviceToHost, db->stream));
        FIM_TRY(stream_sync(db));
        std::memcpy(w.data(), h, (size_t)in.n1 * 8);
      }
      const uint32_t r0 = db->n_rows - in.n1;
      for (uint32_t i = 0; i < in.n1; ++i) work_out[r0 + i] = w[i] + (in.n1 - 1 - i);
    }
  }
  return make_result(db->stream, eo, opts && opts->struct_size && opts->result_on_device, out);
}

fim_status fim_result_view(const fim_result* res, uint64_t* n_sets, const uint64_t** set_offsets,
                           const uint32_t** set_items, const uint32_t** supports, int* on_device) {
  if (!res) return fail(FIM_ERR_INVALID, "result is NULL");
  if (n_sets) *n_sets = res->n_sets;
  if (on_device) *on_device = res->on_device;
  if (res->on_device) {
    if (set_offsets) *set_offsets = res->d_off;
    if (set_items) *set_items = res->d_items;
    if (supports) *supports = res->d_supp;
  } else {
    if (set_offsets) *set_offsets = res->h_off;
    if (set_items) *set_items = res->h_items;
    if (supports) *supports = res->h_supp;
  }
  return FIM_OK;
}

void fim_result_free(fim_result* res) {
  if (!res) return;
  if (res->d_off) cudaFreeAsync(res->d_off, res->stream);  // the block holding all three arrays
  fim::pinned_release(res->h_block, res->h_cap);            // (host result: back to the pool)
  delete res;
}

void fim_db_free(fim_db* db) {
  if (!db) return;
  if (cudaStreamSynchronize(db->stream) == cudaSuccess) {
    ws_give_back(db->device, db->total_mem, &db->ws);  // idle now: the next database may reuse it
  } else {
    cudaGetLastError();
    db->ws.release();
  }
  fim::pinned_release(db->stage, db->stage_cap);
  fim::pinned_release(db->est_pin, db->est_pin_cap);
  if (db->est_done) cudaEventDestroy(db->est_done);
  if (db->cnt_done) cudaEventDestroy(db->cnt_done);
  delete db;
}

}  // extern "C"
