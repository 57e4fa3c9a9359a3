// Internal declarations shared by the CUDA translation units of the miner.
// Nothing here is part of the C ABI (include/fim.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <functional>
#include <vector>

#include "../../include/fim.h"

namespace fim {

// kernels put on a stream by this library (fim_kernel_launches)
void note_launch(uint64_t n = 1);
uint64_t launches_so_far();
// raise a kernel's dynamic shared-memory limit on the current device, once per (device, kernel);
// bytes < 0: the device's opt-in maximum less the kernel's static shared memory
cudaError_t kernel_smem_limit(const void* func, int bytes);

// ---------------------------------------------------------------------------
// error reporting

void set_error(const std::string& msg);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st);
struct fim_db_fwd;
fim_status fail(fim_status s, const std::string& msg);
fim_status cuda_fail(cudaError_t e, const char* what);

#define FIM_CUDA(call)                                                  \
  do {                                                                  \
    cudaError_t e__ = (call);                                           \
    if (e__ != cudaSuccess) return ::fim::cuda_fail(e__, #call);       \
  } while (0)

#define FIM_TRY(call)                          \
  do {                                         \
    fim_status s__ = (call);                   \
    if (s__ != FIM_OK) return s__;             \
  } while (0)

// ---------------------------------------------------------------------------
// device-side error bits (uint32 flag word)

enum : uint32_t {
  DEV_ERR_ITEM_RANGE = 1u << 0,   // an item id >= N in the CSR
  DEV_ERR_OFFSETS = 1u << 1,      // tx_offsets decreasing
  DEV_ERR_DEPTH = 1u << 2,        // DFS deeper than the arena was sized for
  DEV_ERR_TIMEOUT = 1u << 3,      // a bounded wait ran out
  DEV_ERR_OVERFLOW = 1u << 4,     // output capacity exceeded (counts keep going)
  DEV_ERR_POOL = 1u << 5,         // donation pool protocol violated
  DEV_ERR_ABORTED = 1u << 6,      // more itemsets than the caller's limit: mining stopped early
  DEV_ERR_PSTACK = 1u << 7,       // projected DFS: a warp's stack was too small (grown and repeated)
};

// ---------------------------------------------------------------------------
// stream-ordered device buffers, grown on demand and reused across calls

struct DevBuf {
  void* ptr = nullptr;
  size_t cap = 0;
};

struct Workspace {
  cudaStream_t stream = nullptr;
  std::vector<DevBuf> bufs;
  uint64_t bytes = 0;
  // returns a buffer of at least `bytes` bytes in slot `slot` (contents undefined)
  fim_status get(int slot, size_t bytes, void** out);
  void release();
};

template <typename T>
inline fim_status ws_get(Workspace& ws, int slot, size_t count, T** out) {
  void* p = nullptr;
  fim_status st = ws.get(slot, count * sizeof(T), &p);
  if (st != FIM_OK) return st;
  *out = static_cast<T*>(p);
  return FIM_OK;
}

enum WsSlot {
  WS_C2 = 0,
  WS_SCNT,
  WS_SOFF,
  WS_SITEMS,
  WS_ENTRIES,
  WS_ROWORDER,
  WS_FROWS,
  WS_ROWSUPP,
  WS_ARENA,
  WS_OUT_OFF,
  WS_OUT_ITEMS,
  WS_OUT_SUPP,
  WS_CTRL,
  WS_POOL,
  WS_SAMPLE_BITS,
  WS_SAMPLE_SUPP,
  WS_TALLY,
  WS_CLASSWORK,
  WS_EST,  // a deferred estimate's class costs (u64) and order (u32)
  WS_CTATIME,
  WS_PAIR_X,        // rows widened to bytes for the tensor-core pair kernel
  WS_QUERY_ROWS,    // fim_extension_supports: prefix rows | candidate rows
  WS_QUERY_OUT,     // fim_extension_supports: one count per candidate
  WS_QUERY_PREFIX,  // fim_extension_supports: t(P) of a prefix of two or more items
  // the database's own arrays (kept in the workspace so that a freed database's memory serves the next)
  WS_DB_TXOFF,
  WS_DB_TXITEMS,
  WS_DB_BITS,
  WS_DB_SMALL,  // item_rank (N) | rank_item (rows) | supp (rows) | iota (rows), each 16-byte aligned
  // projected DFS: per-class database parts and the warps' stacks
  WS_PROJ_META,  // yoff (n1 u64) | toff (n1 u64) | itemoff (n1 + 1 u32) | eoffx (n1 u32)
  WS_PROJ_Y,     // bitmaps of every class's survivors over the class's transactions
  WS_PROJ_T,     // the transactions (tids) of every projected class
  WS_PSTACK,     // per-warp DFS stacks
  WS_ENTRIES_F,  // queue of the two-item classes whose class was not projected
  WS_PROJ_DQ,    // queue of the children of split frames
  WS_FILT_TABLE, // closed / maximal output: hash table and flags
  WS_FILT_OFF,   // the kept itemsets: offsets
  WS_FILT_ITEMS, // items
  WS_FILT_SUPP,  // supports
  WS_FILT_SCAN,  // block sums of the compaction
  WS_COUNT
};

// small control block living in device memory (one per mining call); fields
// that are polled by idle CTAs and fields that every node updates live on
// separate 128-byte lines
struct alignas(128) DevCtrl {
  // line 0: output reservation and counters updated by every node
  unsigned long long packed;       // (records << 32) | items reserved so far
  unsigned long long items_total;  // exact items requested (for overflow reporting)
  unsigned long long sets_total;   // exact sets requested
  unsigned long long n_intersections;
  unsigned long long n_frames;     // prefixes materialised into the arena
  unsigned long long n_donations;
  uint32_t max_len;                // longest itemset emitted
  uint32_t n_pairs;                // frequent pairs
  uint32_t err;                    // DEV_ERR_* bits
  uint32_t pad0[17];
  // line 1: static queue
  alignas(128) uint32_t queue_head;  // next static queue entry
  uint32_t n_entries;                // static queue length (written by the scan kernel)
  uint32_t queue_head_f;             // projected DFS: next entry of the fallback queue
  uint32_t n_entries_f;              // its length
  uint32_t n_proj_classes;           // classes whose database part was built
  uint32_t n_proj_items;             // work items of the projection
  uint32_t pstack_need;              // largest warp stack (words) a projected class asked for
  uint32_t pad1[25];
  // line 2: termination and progress (polled)
  alignas(128) uint32_t pending;     // unfinished queue entries
  uint32_t progress;                 // nodes finished (any CTA), the no-progress timer's clock
  uint32_t pad2[30];
  // line 3: donation ring (Vyukov bounded MPMC queue over the pool slots)
  alignas(128) uint32_t ring_head;
  uint32_t ring_tail;
  uint32_t n_idle;                   // CTAs waiting for work
  uint32_t n_ready;                  // donated classes waiting in the ring
  uint32_t pad3[28];
  // line 4: node count (stats)
  alignas(128) unsigned long long n_nodes;
  uint32_t pad4[30];
  // line 5: projected DFS work sharing: the queue of split frames' children, unfinished items, and the
  // bump pointer of the region arena
  alignas(128) uint32_t dq_head;     // next item to take
  uint32_t dq_tail;                  // items reserved by producers
  uint32_t proj_pending;             // items (static or split) not yet finished
  uint32_t proj_splits;              // frames split into regions (stats)
  unsigned long long arena_top;      // words of the region arena in use
  unsigned long long proj_bytes;     // operand bytes of the projected DFS (stats)
  unsigned long long proj_split_words;  // hand-out threshold chosen by the planning kernel
  uint32_t pad5[22];
};

// ---------------------------------------------------------------------------
// the database object (C ABI opaque type)

}  // namespace fim

struct fim_db {
  uint32_t D = 0, N = 0, n_rows = 0;
  uint32_t W32 = 0;      // ceil(D / 32): 32-bit words holding D bits
  uint32_t stride = 0;   // padded 32-bit words per row (multiple of 32 = 128 bytes)
  uint32_t word_bits = 64;
  uint32_t prefilter = 0;
  uint32_t max_tx_len = 0;  // longest transaction (distinct kept items)
  uint64_t nnz = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  uint64_t total_mem = 0;  // device memory (bytes)
  size_t smem_optin = 0;

  uint32_t* d_bits = nullptr;       // n_rows * stride
  uint32_t* d_rank_item = nullptr;  // n_rows
  int32_t* d_item_rank = nullptr;   // N
  uint32_t* d_supp = nullptr;       // n_rows
  uint32_t* d_tx_off = nullptr;     // D + 1
  uint32_t* d_tx_items = nullptr;   // nnz
  uint64_t device_bytes = 0;

  std::vector<uint32_t> rank_item, supp;
  std::vector<int32_t> item_rank;

  // last estimate (fim_estimate_class_costs)
  bool has_estimate = false;
  std::vector<double> est_cost;
  std::vector<uint32_t> est_order;
  uint64_t est_nfs = 0;
  uint32_t est_m = 0, est_minsup = 0;
  double est_rel = 0.0;      // relative minsup the estimate was asked for
  bool est_doubled = false;  // the sample minsup was raised by the itemset limit
  uint64_t est_limit = 0;    // that limit
  // a deferred estimate (no host outputs asked for): costs and order on the device (d_est_order, R rows),
  // the sample's control block, costs and order copied to est_pin behind est_done; est_pending until read
  bool est_pending = false;
  bool est_redo = false;  // the deferred sample needs the synchronous path (itemset limit or a retry)
  uint32_t est_redo_minsup = 0;  // the sample minsup that redo starts at (0: the estimate's own)
  cudaEvent_t est_done = nullptr;
  cudaEvent_t cnt_done = nullptr;  // the build's item counts copied to the host (the bitmap clearing behind them)
  void* est_pin = nullptr;
  size_t est_pin_cap = 0;
  const uint32_t* d_est_order = nullptr;
  struct {
    double rate, rel;
    uint64_t seed, limit;
    uint32_t kind;
  } est_args{};

  fim::Workspace ws;

  uint32_t* d_iota = nullptr;  // 0 .. n_rows-1 (frequent-row lists of the full database point into it)
  uint64_t proj_stack_words = 0;  // largest warp stack a projected mine of this database needed (0 = none yet)
  // pinned host staging for small copies; regions are handed out by a bump
  // pointer that is reset whenever the stream has been synchronised
  uint8_t* stage = nullptr;
  size_t stage_cap = 0, stage_used = 0;
};

struct fim_result {
  uint64_t n_sets = 0;
  uint64_t n_items = 0;
  int on_device = 0;
  // host result: offsets | items | supports in one pinned block of the library's pool (returned on free)
  uint64_t* h_off = nullptr;
  uint32_t* h_items = nullptr;
  uint32_t* h_supp = nullptr;
  void* h_block = nullptr;
  size_t h_cap = 0;
  uint64_t* d_off = nullptr;
  uint32_t* d_items = nullptr;
  uint32_t* d_supp = nullptr;
  cudaStream_t stream = nullptr;
};

namespace fim {

// ---------------------------------------------------------------------------
// mining engine (shared by fim_mine and the sample mining of the estimate)

struct EngineInput {
  const uint32_t* bits = nullptr;  // rows of `stride` words
  const uint32_t* d_frows = nullptr;     // optional device copy of frows (else uploaded)
  const uint32_t* d_row_supp = nullptr;  // optional device copy of row_supp (else uploaded)
  bool identity_order = false;           // row_order is 0..n1-1 (d_frows-style device iota used)
  uint32_t stride = 0;             // padded words per row
  uint32_t bytes_per_row_alg = 0;  // W * w / 8: unpadded bytes of one row (algorithmic)
  uint32_t n1 = 0;                 // frequent rows taking part
  std::vector<uint32_t> frows;     // ascending row ids (host), n1 entries
  std::vector<uint32_t> row_supp;  // support of each frequent row, n1 entries
  std::vector<uint32_t> row_order; // queue order of the top classes (permutation of 0..n1-1)
  const uint32_t* d_row_order = nullptr;  // optional device copy of row_order (else uploaded)
  const uint32_t* d_rank_item = nullptr;  // row -> original item id
  uint32_t minsup = 1;
  uint32_t max_len_bound = 2;      // upper bound on the length of a frequent itemset
};

struct EngineOutput {
  uint64_t n_sets = 0, n_items = 0;
  uint64_t* d_off = nullptr;   // workspace-owned
  uint32_t* d_items = nullptr;
  uint32_t* d_supp = nullptr;
  DevCtrl ctrl{};
};

struct EngineConfig {
  uint32_t depth_first = 0;  // 0 = automatic
  uint32_t threads = 0;      // 0 = automatic
  uint32_t vec = 0;          // 0 = automatic
  uint32_t ctas_per_sm = 0;
  uint32_t donate = 0;
  uint32_t mode = 2;  // DFS traversal: 0 node, 1 frame, 2 automatic, 3 sparse node, 4 warp, 5 projected
  uint32_t pair_kernel = 0;  // level 2: 0 automatic, 1 integer pipes, 2 tensor cores (e2m1), 3 (e4m3), 4 (fused)
  uint32_t fault_pair_wait = 0;  // test: the tensor pair kernel's stage waits never complete
  uint64_t spin_limit = 0;
  uint64_t cap_sets = 0, cap_items = 0;  // 0 = automatic
  bool fixed_capacity = false;
  bool collect_times = false;
  unsigned long long* class_work = nullptr;  // optional device array (n1 entries): DFS intersections per top class
  unsigned long long* class_sets = nullptr;  // optional device array (n1 entries): itemsets per top class
  bool count_only = false;                   // count itemsets, write no records (no output buffers)
  std::vector<unsigned long long>* class_out = nullptr;  // host copy of class_sets / class_work (n1 entries)
  uint64_t max_sets = 0;                     // 0 = no limit; else stop early past this many itemsets
  // projected DFS (0 = automatic): a warp's first stack (words), the widest projected class bitmap
  // (words), the budget of the class bitmaps (words)
  uint64_t pstack_words = 0;
  uint32_t proj_w_cap = 0;
  uint64_t proj_y_cap = 0;
  uint64_t split_words = 0;  // 0 = automatic; else a frame whose next level reads more words is split
  uint32_t output = 0;       // FIM_OUTPUT_*: maximal makes the DFS write its leaves only
  uint32_t diffsets = 0;     // projected DFS: 0 never, 1 where smaller than bitmaps, 2 always
};

// Everything one mining call launches, with its geometry and buffers.  The
// buffers live in a Workspace (the db's, or a plan's own for graph replays).
struct EnginePlan {
  uint32_t n1 = 0, minsup = 1, stride = 0, bytes_per_row_alg = 0;
  const uint32_t* bits = nullptr;
  const uint32_t* d_rank_item = nullptr;
  // DFS geometry
  uint32_t L = 3, maxd = 1, maxd_full = 1, threads = 256, vec = 4, grid = 0, pool_slots = 0;
  bool psmem = true;
  size_t smem = 0;
  uint64_t per_depth = 0, pool_slot_words = 0, npairs_max = 0;
  uint64_t cap_sets = 0, cap_items = 0;
  bool fixed_capacity = false;
  uint32_t donate = 0;
  uint32_t mode = 0;
  uint64_t spin_limit = 0;
  int num_sms = 0;
  unsigned long long* d_class_work = nullptr;  // optional per-class intersection counters (n1 entries)
  unsigned long long* d_class_sets = nullptr;  // optional per-class itemset counters (n1 entries)
  bool count_only = false;
  std::vector<unsigned long long>* class_out = nullptr;  // read back with the control block
  uint64_t max_sets = 0;
  bool skip_pairs = false;  // a repeated launch reuses the pair counts of the previous one
  bool pair_mma = false;    // level 2 on the tensor cores (rows widened into d_X)
  bool pair_e2m1 = true;    // tensor-core operands packed as e2m1 (else e4m3)
  bool pair_fused = false;  // widening fused into the tensor-core product (consecutive rows, no widened copy)
  const uint32_t* rows_base = nullptr;  // the frequent rows when consecutive
  uint32_t pair_extra_tx = 0;  // test: bytes a stage waits for beyond its copies (0 normally)
  uint8_t* d_X = nullptr;   // widened rows (pair_mma only)
  // projected DFS (mode 5): budgets, geometry and buffers; the fallback runs the sparse node mode with
  // the geometry above
  bool leaves = false;  // write only the DFS's leaves (itemsets without a frequent later extension)
  uint32_t diffsets = 0;
  bool proj = false;
  uint64_t proj_y_cap = 0, proj_t_cap = 0, pstack_words = 0;
  uint32_t proj_w_cap = 0, proj_grid = 0;
  size_t proj_smem = 0;
  uint64_t *d_yoff = nullptr, *d_toff = nullptr;
  uint32_t *d_itemoff = nullptr, *d_eoffx = nullptr, *d_Y = nullptr, *d_T = nullptr, *d_pstack = nullptr;
  uint2* d_entries_f = nullptr;
  uint4* d_dq = nullptr;
  uint32_t dq_cap = 0;
  uint64_t proj_arena_words = 0, split_words = 0;
  float ms_pair = 0.f, ms_total = 0.f;  // device time of the pair kernel / of all launches so far
  unsigned long long* d_cta_time = nullptr;  // per-CTA [start, end] of the DFS (with timing only)
  // buffers
  DevCtrl* d_ctrl = nullptr;
  const uint32_t *d_frows = nullptr, *d_rsupp = nullptr, *d_order = nullptr;
  uint32_t *d_C2 = nullptr, *d_scnt = nullptr, *d_soff = nullptr, *d_eoff = nullptr, *d_sitems = nullptr;
  uint2* d_entries = nullptr;
  uint32_t *d_pool = nullptr, *d_arena = nullptr;
  uint64_t* d_off = nullptr;
  uint32_t *d_items = nullptr, *d_supp = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // optional kernel timing
};

// geometry, row lists and the capacity-independent buffers
fim_status engine_prepare(fim_db* db, Workspace& ws, const EngineInput& in, const EngineConfig& cfg, EnginePlan* ep);
// capacity- and depth-dependent buffers (outputs, DFS arena)
fim_status engine_alloc(Workspace& ws, EnginePlan* ep);
// all device work of one mine: no host synchronisation, no allocation (graph capturable)
cudaError_t engine_launch(const EnginePlan& ep, cudaStream_t st);
// its two parts: the control block reset and (when `pairs`) the pair kernel, which needs no output buffer;
// then level 2, the DFS and the timing events
cudaError_t engine_launch_front(const EnginePlan& ep, cudaStream_t st, bool pairs);
cudaError_t engine_launch_back(const EnginePlan& ep, cudaStream_t st);
// wait, read the control block, check errors; *retry = true when the buffers must grow and the
// launch be repeated (output capacity or DFS depth)
fim_status engine_finish(fim_db* db, cudaStream_t st, EnginePlan* ep, EngineOutput* out, fim_mine_stats* stats,
                         bool* retry);
// the EngineInput / EngineConfig of a fim_mine call (validation included); with defer_ok a pending estimate
// stays pending (the queue order is derived on the device, the output capacity left to the caller)
fim_status mine_input(fim_db* db, uint32_t minsup, const fim_mine_opts* opts, EngineInput* in, EngineConfig* cfg,
                      bool defer_ok = false);
// the first output capacity that the database's estimate suggests for a minsup (0: none)
uint64_t estimate_capacity(const fim_db* db, uint32_t minsup);
// fim_estimate_class_costs_ex, allowed to leave its result on the device (see fim_api.cu)
fim_status estimate_impl(fim_db* db, double sample_rate, double rel_minsup, uint64_t seed, uint32_t cost_kind,
                         uint64_t max_sample_itemsets, double* cost_out, uint32_t* order_out, bool allow_defer,
                         uint32_t first_minsup_s);
// a deferred estimate read into the database's host copies (no-op when none is pending)
fim_status est_resolve(fim_db* db);
// the synchronous estimate that a deferred one found incomplete asks for (no-op otherwise)
fim_status est_redo(fim_db* db);
// keeps the itemsets of an engine output whose closed (keep = 1) or maximal (keep = 2) flag is set, decided
// by the immediate supersets within the output itself (result_flags.cu); the output's buffers are replaced
// by workspace buffers holding the kept itemsets in their original order
fim_status filter_output(Workspace& ws, cudaStream_t st, uint8_t keep, EngineOutput* eo, int num_sms);
// fim_result from an engine output (device copy or host copy per on_device)
fim_status make_result(cudaStream_t st, const EngineOutput& eo, bool on_device, fim_result** out);
// prepare, launch the pair kernel, call `after_pairs` (may change the output capacity), then allocate,
// launch the rest and finish, repeating the later stages while the buffers must grow
fim_status engine_mine(fim_db* db, Workspace& ws, const EngineInput& in, const EngineConfig& cfg,
                       EngineOutput* out, fim_mine_stats* stats, EnginePlan* plan_out = nullptr,
                       const std::function<fim_status(EnginePlan*)>& after_pairs = {});
void engine_release_events(EnginePlan* ep);
// pinned staging of a database (see fim_api.cu)
fim_status stage_get(fim_db* db, size_t bytes, void** out);
fim_status stream_sync(fim_db* db);

// ---------------------------------------------------------------------------
// kernel launchers (defined in the .cu files)

// flags (4 words, zeroed by the caller): error bits, longest transaction, off[0], off[D]
cudaError_t launch_item_count(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t* cnt,
                              uint32_t* flags, cudaStream_t st);
cudaError_t launch_bitmap_build(const uint32_t* off, const uint32_t* items, uint32_t D, const int32_t* item_rank,
                                uint32_t* bits, uint32_t stride, cudaStream_t st);
cudaError_t launch_sample_build(const uint32_t* off, const uint32_t* items, uint32_t D, const int32_t* item_rank,
                                uint64_t seed, uint32_t m, uint32_t* sbits, uint32_t sstride, cudaStream_t st);
cudaError_t launch_iota(uint32_t* out, uint32_t n, cudaStream_t st);
cudaError_t launch_row_popcount(const uint32_t* bits, uint32_t stride, uint32_t n_rows, uint32_t* supp,
                                cudaStream_t st);
// rows of a database whose estimate may stay on the device (the one-CTA suffix kernel)
constexpr uint32_t kEstDeviceRows = 4096;
// class costs (tally, R u64) and their LPT order (R u32) of a sample mined over all its R rows
cudaError_t launch_est_order(const unsigned long long* per, const uint32_t* ssupp, uint32_t minsup_s,
                             bool intersections, uint32_t R, unsigned long long* tally, uint32_t* order,
                             cudaStream_t st);
// the queue order of the rows r0 .. of a mine from an estimate's order over all R rows
cudaError_t launch_order_suffix(const uint32_t* order, uint32_t R, uint32_t r0, uint32_t* out, cudaStream_t st);

struct PairLaunch {
  const uint32_t* bits;
  uint32_t stride;
  const uint32_t* frows;
  uint32_t n1;
  uint32_t* C2;  // n1 * n1
  uint32_t ksplit;
  const uint32_t* rows_base = nullptr;  // the frequent rows when they are consecutive rows of `bits` (else NULL)
};
cudaError_t launch_pair_counts(const PairLaunch& p, int num_sms, cudaStream_t st, uint32_t* ksplit_used);
// the same counts on the tensor cores: rows widened into X (pair_mma_buffer_bytes), then C2 = X X^T;
// err receives DEV_ERR_TIMEOUT if a bounded wait runs out
// (e2m1: packed 4-bit operands, else e4m3 bytes)
cudaError_t launch_pair_mma(const PairLaunch& p, uint8_t* X, bool e2m1, uint32_t* err, int num_sms, cudaStream_t st,
                            uint32_t* ksplit_used, uint32_t extra_tx = 0);
uint64_t pair_mma_buffer_bytes(uint32_t n1, uint32_t stride, bool e2m1);
// the same with the widening fused into the product (e4m3 operands written to shared memory from the raw
// bits, no widened copy); needs p.rows_base
cudaError_t launch_pair_mma_fused(const PairLaunch& p, uint32_t* err, int num_sms, cudaStream_t st,
                                  uint32_t* ksplit_used, uint32_t extra_tx = 0);
// modelled device time (µs) of each pair kernel, for the automatic choice
double pair_mma_cost_us(uint32_t n1, uint32_t stride, int num_sms, bool e2m1, bool fused = false);
double pair_cores_cost_us(uint32_t n1, uint32_t stride, int num_sms);

struct LevelLaunch {
  const uint32_t* C2;
  uint32_t n1;
  uint32_t minsup;
  const uint32_t* frows;
  const uint32_t* row_supp;
  const uint32_t* rank_item;
  const uint32_t* row_order;    // queue position -> row
  uint32_t* scnt;               // n1 survivors per row
  uint32_t* soff;               // n1 + 1 survivor offsets (natural row order)
  uint32_t* eoff;               // n1 + 1 entry offsets (queue order)
  uint32_t* sitems;             // survivors (frow indices)
  uint2* entries;               // (row, m)
  uint64_t* out_off;            // NULL: count only (no records)
  uint32_t* out_items;
  uint32_t* out_supp;
  uint64_t cap_sets, cap_items;
  DevCtrl* ctrl;
  unsigned long long* class_sets;  // optional: frequent itemsets per top class
  const uint32_t* eoffx;           // optional (projected DFS): entry offset per queue position, bit 31 =
                                   // the class's entries go to the fallback queue entries_f
  uint2* entries_f;
  uint32_t leaves;                 // 1: records only for the leaves of levels 1 and 2 (k_level2_leaves)
};
cudaError_t launch_level2(const LevelLaunch& p, cudaStream_t st);
// the level-2 kernels up to the entry offsets, and the fill kernel alone (the projected DFS plans its
// classes between the two)
cudaError_t launch_level2_counts(const LevelLaunch& p, cudaStream_t st);
cudaError_t launch_level2_fill(const LevelLaunch& p, cudaStream_t st);


struct DfsLaunch {
  const uint32_t* bits;
  uint32_t stride;
  const uint32_t* frows;
  uint32_t n1;
  uint32_t minsup;
  const uint32_t* rank_item;
  const uint32_t* soff;
  const uint32_t* scnt;
  const uint32_t* sitems;
  const uint2* entries;
  uint32_t* arena;
  uint64_t arena_cta_words;
  uint32_t maxd;
  uint32_t* pool;           // donation pool (slots)
  uint32_t pool_slots;
  uint64_t pool_slot_words;
  uint64_t* out_off;
  uint32_t* out_items;
  uint32_t* out_supp;
  uint64_t cap_sets, cap_items;
  DevCtrl* ctrl;
  uint64_t spin_limit;
  uint32_t donate;
  unsigned long long* class_work;  // optional: intersections per top class (frow index of its first item)
  uint64_t max_sets;               // 0 = no limit; else stop once more sets than this are found
  unsigned long long* cta_time;    // optional: [start, end] global time (ns) of every CTA
  unsigned long long* class_sets;  // optional: frequent itemsets per top class
  const uint32_t* C2;              // level-2 pair counts (n1 x n1): supports of the root prefixes
  uint32_t queue_sel;              // 0: the main queue; 1: the projected mode's fallback queue
  uint32_t diffsets;               // projected DFS: 0 bitmaps only, 1 diffset frames where they are small,
                                   // 2 every frame as diffsets
  uint32_t leaves;                 // 1: a node writes one record: itself when no candidate survives, else
                                   // itself with its last survivor (the DFS's leaves; maximal output)
  // projected DFS (mode 5) only
  const uint32_t* row_supp;        // support of every frequent row (n1)
  const uint64_t* yoff;            // word offset of class i's bitmaps in Y (~0 = not projected)
  const uint32_t* Y;               // the classes' bitmaps
  uint32_t* pstack;                // per-warp stacks
  uint64_t pstack_words;           // words of one warp's stack
  uint4* dq;                       // queue of split frames' children: (region offset, m, ready) per slot
  uint32_t dq_cap;                 // its slots
  uint64_t arena_words;            // words of Y (class regions, then split regions)
  uint64_t split_words;            // a frame whose next level reads more words than this is split
};

// Projected DFS (mode 5): the database part of every one-item class (its transactions and its
// survivors' bitmaps over them), then one warp per two-item class running Eclat on those bitmaps.
struct ProjLaunch {
  const uint32_t* bits;
  uint32_t stride;
  const uint32_t* frows;
  const uint32_t* row_supp;
  const uint32_t* row_order;  // queue position -> class
  const uint32_t* scnt;
  const uint32_t* soff;
  const uint32_t* sitems;
  const uint32_t* rank_item;  // row -> original item id
  uint32_t n1;
  uint64_t y_cap_words;  // budget of Y (words)
  uint64_t t_cap;        // budget of T (tids)
  uint32_t w_cap;        // widest bitmap of a projected class (words)
  uint64_t* yoff;        // n1, by class
  uint64_t* toff;        // n1, by class
  uint32_t* itemoff;     // n1 + 1, by queue position
  uint32_t* eoffx;       // n1, by queue position
  uint32_t* Y;
  uint32_t* T;
  DevCtrl* ctrl;
};
cudaError_t launch_proj_plan(const ProjLaunch& q, cudaStream_t st);
cudaError_t launch_proj_build(const ProjLaunch& q, int num_sms, cudaStream_t st);
cudaError_t launch_dfs_proj(const DfsLaunch& p, uint32_t grid, uint32_t max_len, cudaStream_t st);
size_t dfs_proj_smem_bytes(uint32_t max_len);
cudaError_t dfs_proj_ctas_per_sm(size_t smem, int* out);
constexpr uint32_t kProjThreads = 256;     // projected DFS: 8 warps per CTA
constexpr uint32_t kProjCtasPerSm = 2;     // 16 warps per SM with up to 128 registers each (large_sparse's DFS:
                                           // 5.1 ms against 7.3 ms with four CTAs at 64 registers, which spill)
constexpr uint64_t kProjStackWords = 131072;  // first stack of one warp (doubled when a run needs more)
constexpr uint32_t kProjDqCap = 1u << 18;     // items of split frames the queue holds
// device bytes the projected DFS adds to a mine of `rows` frequent rows of `stride` words over a database
// of nnz items run on `grid` persistent CTAs (for the server's admission)
uint64_t proj_footprint_bytes(uint32_t rows, uint32_t stride, uint64_t nnz, uint32_t grid);
// words of a class region's header, prefix ids and row ids (its rows start there)
__host__ __device__ inline uint64_t region_rows_off(uint32_t xlen, uint32_t k) {
  return 8ull + (((uint64_t)xlen + 3) & ~3ull) + (((uint64_t)k + 3) & ~3ull);
}
// grid: number of persistent CTAs; threads: CTA size; vec: 16-byte loads per lane per piece
// mode 0: node at a time (optionally with donation); mode 1: frame passes (all children of a frame together)
cudaError_t launch_dfs(const DfsLaunch& p, uint32_t grid, uint32_t threads, uint32_t vec, size_t smem,
                       bool prefix_in_smem, uint32_t max_len, uint32_t mode, cudaStream_t st);
// mode 0 node expansion (dense prefix), 1 frame passes, 3 node expansion with listed (sparse) prefixes
size_t dfs_smem_bytes(uint32_t stride, uint32_t max_len, uint32_t maxd, bool prefix_in_smem, uint32_t mode);
uint32_t dfs_sparse_cap(uint32_t stride);
cudaError_t launch_pool_init(uint32_t* pool, uint32_t slots, uint64_t slot_words, cudaStream_t st);
cudaError_t dfs_max_ctas_per_sm(uint32_t threads, uint32_t vec, size_t smem, bool prefix_in_smem, uint32_t mode,
                                int* out);
bool dfs_prefix_fits(uint32_t stride, size_t smem_optin, uint32_t max_len, uint32_t maxd, uint32_t mode);
uint64_t dfs_arena_cta_words(uint32_t stride, uint32_t n1, uint32_t maxd, uint32_t mode);
constexpr uint32_t kDfsDepthHint = 8;  // DFS stack depth allocated first (grown on demand)
constexpr uint32_t kDfsSlotHeader = 4;  // donation pool slot: sequence, xlen, ncand, spare
// pool slot words for itemsets of up to max_len items and n1 candidates (prefix bitmap last)
__host__ __device__ inline uint64_t dfs_pool_slot_words(uint32_t stride, uint32_t max_len, uint32_t n1) {
  return (((uint64_t)kDfsSlotHeader + 2ull * max_len + 2ull * n1 + 3) & ~3ull) + stride;
}
// frame mode (all children of a frame counted together): pairs per pass, and the
// stack layout [root list][per depth: prefix | survivor area | child table], every
// region a multiple of four words so that prefix bitmaps stay 16-byte aligned
constexpr uint32_t kDfsPairBatch = 2048;
__host__ __device__ inline uint64_t frames_root_words(uint32_t n1) { return (2ull * n1 + 3) & ~3ull; }
__host__ __device__ inline uint64_t frames_g_words(uint32_t n1) { return (2ull * (kDfsPairBatch + n1) + 3) & ~3ull; }
__host__ __device__ inline uint64_t frames_depth_words(uint32_t stride, uint32_t n1) {
  return (uint64_t)stride + frames_g_words(n1) + 2ull * kDfsPairBatch;
}
// node-mode arena words per depth: the prefix (stride words: dense, or the values of its nonzero
// 16-byte words), its index list (4-word header + stride/8 words of 16-bit indices), one (row, id)
// survivor list, the survivors' supports; every region a multiple of four words
__host__ __device__ inline uint64_t dfs_list_words(uint32_t stride) { return (uint64_t)stride / 8 + 4; }
__host__ __device__ inline uint64_t dfs_arena_depth_words(uint32_t stride, uint32_t n1) {
  return (uint64_t)stride + dfs_list_words(stride) + ((2ull * n1 + 3) & ~3ull) + ((uint64_t)n1 + 3 & ~3ull);
}

}  // namespace fim
