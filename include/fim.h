/*
 * fim.h -- C ABI of the GB300 frequent-itemset miner (vertical-bitmap Eclat).
 *
 * The method is the depth-first Eclat of R. Kessl, "Parallel algorithms for
 * mining of frequent itemsets" (thesis, 2011; arXiv 2108.05038), App. B.3:
 * supports are counted by intersecting transaction-id lists (here: bitmaps,
 * AND + popcount) over prefix-based equivalence classes (PBECs, Sec. 2.4) and
 * pruned at the minimum support.  The thesis's sample-based estimate of the
 * size of a PBEC (Sec. 6.2, Phase 2 in Sec. 8.2) orders the prefix classes
 * across the persistent CTAs of one GPU.
 *
 * Conventions for every entry point:
 *  - Every call returns fim_status; nothing aborts, throws across the ABI or
 *    traps the device.  On error the output handle is left NULL and
 *    fim_last_error() (thread local) describes the cause.
 *  - Input buffers are copied; the caller keeps ownership of its buffers.
 *    Objects returned through `out` handles are owned by the library until
 *    the matching *_free call.
 *  - Device work runs on the CUDA stream given to fim_build_vertical_db*
 *    (NULL = the legacy default stream).  Calls that return host data
 *    synchronise that stream before returning.
 *  - A fim_db may be used by one thread at a time.
 */
#ifndef FIM_H_
#define FIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fim_db fim_db;         /* device bitmaps + item relabel map + CSR copy for sampling */
typedef struct fim_result fim_result; /* frequent itemsets in CSR form (host or device memory)      */
typedef struct fim_plan fim_plan;     /* one (database, minsup) mine captured in a CUDA graph        */
typedef struct fim_server fim_server; /* continuous-batching request loop over mining jobs           */

typedef enum {
  FIM_OK = 0,
  FIM_ERR_INVALID = 1,         /* bad argument (NULL pointer, size, item id >= N, minsup 0 ...)  */
  FIM_ERR_OOM = 2,             /* a device or host allocation failed                            */
  FIM_ERR_OUTPUT_OVERFLOW = 3, /* fixed output capacity too small; needed sizes are reported   */
  FIM_ERR_CUDA = 4,            /* a CUDA runtime call failed                                    */
  FIM_ERR_TIMEOUT = 5          /* a bounded device-side wait ran out (no progress)              */
} fim_status;

/* Order in which the prefix classes enter the persistent kernel's queue. */
typedef enum {
  FIM_ORDER_ESTIMATE = 0, /* longest first by the sample estimate (LPT, Sec. 8.2); falls back to
                             FIM_ORDER_UNIFORM when fim_estimate_class_costs was never called  */
  FIM_ORDER_UNIFORM = 1   /* class order = item order (ascending support)                      */
} fim_class_order;

/* Counters of one fim_mine call (filled when fim_mine_opts.stats != NULL). */
typedef struct {
  uint64_t n_frequent;           /* |F|: frequent itemsets written                                */
  uint64_t n_items_out;          /* sum of |X| over F                                             */
  uint32_t n_frequent_items;     /* frequent singletons (rows taking part in this mine)            */
  uint32_t max_len;              /* longest frequent itemset                                       */
  uint64_t n_intersections;      /* AND+popcount operand pairs evaluated, all levels               */
  uint64_t n_pair_intersections; /* of which in the level-2 pair kernel (i < j pairs)              */
  uint64_t n_classes;            /* class nodes expanded by the persistent DFS kernel              */
  uint64_t n_queue_entries;      /* level-3 prefix classes put in the persistent queue             */
  uint64_t n_donations;          /* subclasses handed from a busy CTA to idle CTAs                 */
  uint64_t bytes_algorithmic;    /* algorithmic bytes of all intersections (see DESIGN measurement) */
  uint64_t bytes_pair_kernel;    /* algorithmic bytes of the pair kernel                           */
  uint64_t bytes_dfs_kernel;     /* algorithmic bytes of the DFS kernel                            */
  uint32_t words_per_row;        /* 32-bit words per bitmap row, padded (row stride)               */
  uint32_t grid_ctas;            /* persistent CTAs launched                                       */
  uint32_t threads_per_cta;
  uint32_t vec_per_lane;         /* 16-byte loads per lane per piece                               */
  float ms_pair_kernel;          /* CUDA-event time of the pair kernel (collect_times = 1)         */
  float ms_dfs_kernel;           /* CUDA-event time of the persistent DFS kernel                   */
  float ms_device_total;         /* CUDA-event time from the first to the last mining kernel       */
  float dfs_cta_busy_max_ms;     /* longest time a persistent DFS CTA was resident (collect_times)  */
  float dfs_cta_busy_mean_ms;    /* mean over the CTAs; max / mean is the load imbalance           */
  uint32_t pair_kernel;          /* level-2 kernel that ran: FIM_PAIR_CORES / _TENSOR / _TENSOR_E4M3 /
                                    _TENSOR_FUSED                                                      */
  uint32_t n_proj_classes;       /* FIM_DFS_PROJECTED: one-item classes given their database part   */
  uint64_t n_proj_splits;        /* frames handed to other warps with their own database part       */
  uint64_t n_fallback_entries;   /* two-item classes mined by the sparse node mode instead           */
  uint64_t bytes_projected;      /* FIM_DFS_PROJECTED: operand bytes in its own representation: the
                                    class database parts built (each row read, one word gathered per
                                    survivor and transaction, the bitmaps written), per class node its
                                    prefix and candidates over its region's width, per compacted or
                                    handed-out frame its gathered words and region                  */
} fim_mine_stats;

/* Traversal of the persistent DFS (fim_mine_opts.dfs_mode). */
enum { FIM_DFS_NODES = 0, FIM_DFS_FRAMES = 1, FIM_DFS_AUTO = 2, FIM_DFS_SPARSE = 3, FIM_DFS_WARP = 4,
       FIM_DFS_PROJECTED = 5 };

/* Which itemsets fim_mine returns (fim_mine_opts.output). */
enum { FIM_OUTPUT_ALL = 0, FIM_OUTPUT_CLOSED = 1, FIM_OUTPUT_MAXIMAL = 2 };

/* Level-2 pair counts (fim_mine_opts.pair_kernel): FIM_PAIR_CORES: AND + popcount on the integer
 * pipes (8-word carry-save adder tree); FIM_PAIR_TENSOR: the 0/1 rows widened to 4-bit values
 * (1.0 in e2m1, two transactions per byte) and multiplied on the tensor cores (tcgen05
 * kind::f8f6f4, fp32 accumulators, at most 2^24 transactions per partial sum, so exact), which
 * needs a scratch of frequent rows x padded row bytes x 4 in the database's workspace;
 * FIM_PAIR_TENSOR_E4M3: the same with one byte per transaction (1.0 in e4m3, twice the scratch);
 * FIM_PAIR_TENSOR_FUSED: the widening done inside the tensor-core kernel (the raw bits brought to
 * shared memory by TMA, spread to e4m3 there), no scratch and no widened copy in device memory;
 * needs the frequent rows to be consecutive rows of the bitmap, which they are in every fim_mine
 * (FIM_ERR_INVALID otherwise);
 * FIM_PAIR_AUTO: integer pipes or a tensor-core kernel, whichever has the smaller modelled time:
 * FIM_PAIR_TENSOR_FUSED for consecutive rows, else FIM_PAIR_TENSOR while its scratch is at most 1/16
 * of device memory. */
enum { FIM_PAIR_AUTO = 0, FIM_PAIR_CORES = 1, FIM_PAIR_TENSOR = 2, FIM_PAIR_TENSOR_E4M3 = 3,
       FIM_PAIR_TENSOR_FUSED = 4 };

typedef struct {
  uint32_t struct_size;        /* set to sizeof(fim_mine_opts); 0 = treat as defaults            */
  uint32_t class_order;        /* fim_class_order                                                 */
  uint32_t dfs_mode;           /* FIM_DFS_NODES (0): expand one class node at a time, the prefix
                                  dense in shared memory (or in its stack slot when too wide);
                                  FIM_DFS_FRAMES (1): count all children of a frame in one pass
                                  (fewer dependent steps on short rows); FIM_DFS_SPARSE (3): node
                                  expansion with each prefix held as the list of its nonzero 16-byte
                                  words when it has at most 2,048 of them (small CTAs, several per
                                  SM), dense in its stack slot otherwise; rows of at most 65,535
                                  16-byte words, no donation (else as NODES); FIM_DFS_AUTO (2, the
                                  default): projected with at least 1,024 frequent rows (and no
                                  cap on the CTAs per SM), else frames for rows of at most 16,384
                                  words (64 KB), else SPARSE;
                                  FIM_DFS_WARP (4): one warp
                                  per two-item class, the
                                  prefix in its registers, no CTA-wide barrier; rows of at most 512
                                  words, no donation (else as SPARSE); FIM_DFS_PROJECTED (5): the
                                  database part of every one-item class [i | S_i] (the transactions
                                  of i, and each survivor's bitmap over them: Phase 3 of Sec. 8.3
                                  on the device) is built once, then one warp per two-item class
                                  runs Eclat on those short bitmaps; classes beyond its budgets
                                  (bitmaps of at most 1/4 of the frequent rows' bytes, stacks of
                                  128K words per warp, doubled and the run repeated when too small)
                                  are mined as SPARSE; same row limit and no donation as SPARSE  */
  uint32_t threads_per_cta;    /* persistent DFS CTA size, 128/256/512 (sparse nodes: at most 256;
                                  warp DFS: 256); 0 = sparse nodes: 256; other node modes: the one
                                  with the most CTAs per SM (then warps); frames: the most warps   */
  uint32_t vec_per_lane;       /* 16-byte loads per lane per work piece, 1/2/4/8 (sparse nodes also
                                  16); 0 = 4                                                       */
  uint32_t ctas_per_sm;        /* 0 = as many as fit                                              */
  uint32_t donate;             /* 1 = busy CTAs hand subclasses to idle CTAs (default 0)          */
  uint32_t result_on_device;   /* 1 = keep the result in device memory (no D2H copy)              */
  uint32_t collect_times;      /* 1 = record CUDA events around the kernels (stats.ms_*)          */
  uint32_t dfs_depth_first;    /* 0 = automatic (the full depth bound when its stack fits in 1/32 of
                                  device memory); else the first DFS stack depth, grown and the run
                                  repeated when an itemset is deeper                                */
  uint32_t pair_kernel;        /* FIM_PAIR_AUTO (0, default), FIM_PAIR_CORES, FIM_PAIR_TENSOR,
                                  FIM_PAIR_TENSOR_E4M3 or FIM_PAIR_TENSOR_FUSED                     */
  uint32_t fault_pair_wait;    /* 0 (default); 1 = failure-detection test: the tensor-core pair
                                  kernel expects 16 bytes per stage more than its copies bring, so
                                  its bounded waits run out (about 1 s each) and the call returns
                                  FIM_ERR_TIMEOUT with the device context intact                    */
  uint64_t out_capacity_sets;  /* 0 = automatic (grow and retry); else fixed capacity             */
  uint64_t out_capacity_items; /* idem, total items over all sets                                 */
  uint64_t spin_limit;         /* idle-CTA polling rounds without progress before FIM_ERR_TIMEOUT;
                                  0 = default (a few s)                                            */
  uint64_t max_itemsets;       /* 0 = no limit; else mining stops as soon as more itemsets are found
                                  and the call returns FIM_ERR_OUTPUT_OVERFLOW (bounds the work of
                                  requests whose output explodes combinatorially)                  */
  uint64_t proj_bitmap_words;  /* FIM_DFS_PROJECTED budgets (0 = automatic): the class bitmaps, in
                                  32-bit words (classes past it, in queue order, are mined as SPARSE) */
  uint64_t proj_stack_words;   /* first stack of one warp, in 32-bit words                         */
  uint32_t proj_max_row_words; /* widest class bitmap (words) that is projected (default: 1/8 of the
                                  first stack)                                                      */
  uint32_t output;             /* FIM_OUTPUT_ALL (0, default): every frequent itemset;
                                  FIM_OUTPUT_MAXIMAL: only the maximal ones (Def. "Maximal Frequent
                                  Itemset"); the DFS writes only its leaves (itemsets with no
                                  frequent extension by a later item: the candidates on an MFI of
                                  the DFS-MFI-Schema, Ch. 7), and a pass drops every leaf that has
                                  a one-item-larger superset among the leaves (a non-maximal leaf
                                  always has one, so this is the schema's superset check); it takes
                                  the projected DFS (rows of at most 65,535 16-byte words);
                                  FIM_OUTPUT_CLOSED: only the closed ones (Def. "Closed itemset"):
                                  the whole result, then a pass that drops every itemset with a
                                  one-item-larger superset of equal support.  Supports are exact in
                                  every mode; stats.n_frequent counts the itemsets returned      */
  uint32_t diffsets;           /* FIM_DFS_PROJECTED frames as diffsets (dEclat, App. B.4.3): 0 never
                                  (default), 1 where the lists of their nonzero words are at most a
                                  quarter of the bitmaps, 2 every frame; d(PXY) = d(PY) \ d(PX) and
                                  supp(PXY) = supp(PX) - |d(PXY)|, exact                          */
  uint32_t proj_split_words;   /* a frame whose next level would read more 32-bit words than this is
                                  handed to the other warps with its own database part (0 = automatic:
                                  64 x the mean bitmap width of the class regions, at least 128 and
                                  at most 65,536)                                                   */
  /* outputs */
  uint64_t out_needed_sets;    /* on FIM_ERR_OUTPUT_OVERFLOW: capacities that would have sufficed */
  uint64_t out_needed_items;
  fim_mine_stats* stats;       /* optional                                                        */
  uint64_t* class_work_out;    /* optional host array of n_rows entries (fim_db_info): entry r gets
                                  the AND+popcount intersections of the class [r | rows after r],
                                  level 2 and below (the actual cost that the sample estimate
                                  predicts); 0 for rows that are not frequent                      */
} fim_mine_opts;

/* Fill *opts with the defaults (struct_size set, all options default). */
void fim_mine_opts_init(fim_mine_opts* opts);

/*
 * Build the vertical representation (Def. "Transaction id list" and the
 * vertical representation of Ch. 2; first step of Eclat-DFS, App. B.3.2).
 *
 * tx_offsets[D+1], tx_items[tx_offsets[D]]: horizontal database in CSR form,
 * HOST memory; transaction t holds tx_items[tx_offsets[t] .. tx_offsets[t+1]).
 * Items are ids < N in any order; a repeated id inside a transaction counts
 * once (set semantics, Def. "Transaction").  Empty transactions are allowed
 * and count toward D.
 * word_bits: 32 or 64, the nominal bitmap word; the bit layout in memory is
 * the same for both on a little-endian GPU (bit t of row f sits in byte
 * t/8, bit t%8), so it only decides how W is reported.
 * prefilter_minsup: items with support < prefilter_minsup get no row (0 keeps
 * every item).  Kept items are relabelled 0..N_f-1 by ascending support, ties
 * by ascending id (the ascending-support order of App. B.4.2); every later
 * mine must use minsup >= prefilter_minsup.
 * Errors: FIM_ERR_INVALID (NULL pointers, D == 0, N == 0, word_bits not 32/64,
 * offsets not non-decreasing, an item >= N), FIM_ERR_OOM, FIM_ERR_CUDA.
 */
fim_status fim_build_vertical_db(const uint32_t* tx_offsets, const uint32_t* tx_items, uint32_t D, uint32_t N,
                                 uint32_t word_bits, uint32_t prefilter_minsup, void* cuda_stream, fim_db** out);

/* Same as fim_build_vertical_db with tx_offsets / tx_items in DEVICE memory,
 * read on cuda_stream: both must stay valid until the work queued on that
 * stream by this call has run (as for cudaMemcpyAsync); the library copies
 * what it keeps.  d_tx_items must not be NULL.  The offsets are validated on
 * the device before any item is read past tx_offsets[D]. */
fim_status fim_build_vertical_db_device(const uint32_t* d_tx_offsets, const uint32_t* d_tx_items, uint32_t D,
                                        uint32_t N, uint32_t word_bits, uint32_t prefilter_minsup,
                                        void* cuda_stream, fim_db** out);

/* Sizes of a built database: transactions, item base, kept rows, 32-bit words
 * per padded row, nominal word bits, device bytes held.  Any pointer may be NULL. */
fim_status fim_db_info(const fim_db* db, uint32_t* D, uint32_t* N, uint32_t* n_rows, uint32_t* words_per_row,
                       uint32_t* word_bits, uint64_t* device_bytes);

/* Relabel map: rank_item[r] = original id of row r, supports[r] = its support
 * (both arrays of n_rows entries, host memory; either may be NULL). */
fim_status fim_db_rows(const fim_db* db, uint32_t* rank_item, uint32_t* supports);

/*
 * Sample-based estimate of the relative size of every one-item-prefix class
 * [r | {g : g after r}] (Def. "Relative size of a PBEC", Sec. 2.4; estimate
 * of Sec. 6.2 used by Phase 2, Sec. 8.2).
 * A sample D_s of m = max(ceil(sample_rate * D), min(D, m0)) transactions is
 * drawn with replacement (Sec. 6.1), m0 = ceil(ln(2/0.05) / (2 * 0.05^2)) = 738
 * being the size for which Theorem 6.1 bounds every relative support error
 * by 0.05 with probability 0.95: draw k takes transaction ((x_k >> 32) * D) >> 32,
 * x_k = k-th output of SplitMix64 started at state `seed`.  D_s (kept items
 * only) is mined on the GPU at minsup_s = max(1, ceil(rel_minsup * m)) and
 * cost_out[r] = |{X in F_s : the lowest row of X is r}| / |F_s| (0 when F_s is
 * empty).  While D_s has more than FIM_SAMPLE_ITEMSET_LIMIT frequent itemsets
 * at minsup_s, minsup_s doubles (the thesis does not treat a sample whose
 * itemsets explode; this keeps the estimate's cost bounded: the count-only
 * mine of a sample stops once it passes the limit, so an exploding sample
 * costs about limit itemsets per doubling).  order_out = rows by descending cost, ties by ascending row (the
 * LPT order, Sec. 8.2).  Both arrays have n_rows entries (host memory).
 * The estimate is kept in the db and orders the classes of later fim_mine
 * calls (FIM_ORDER_ESTIMATE); it never changes their output.
 * cost_out and order_out may be NULL.  When both are NULL and the sample is
 * mined over all its rows (the db has at most 4,096 rows and at least 3/4 of
 * them have supp * m / D >= minsup_s), the call does not wait for the device: the sample's mine,
 * its per-class counts and the LPT order stay on the device (a one-CTA sort),
 * and the next fim_mine takes its class order from there and reads the
 * sample's itemset count (its first output capacity) only after launching its
 * pair kernel.  A sample that passed the itemset limit orders that mine by its
 * partial counts (the output is the same for every order), and is mined again
 * by the synchronous path, from the doubled sample minsup, when a later mine
 * or query of the estimate needs it.
 * Errors of such a deferred estimate are reported by the call that reads it
 * (fim_mine, fim_estimate_result, fim_estimate_sample_size).
 * Errors: FIM_ERR_INVALID (sample_rate not in (0,1], rel_minsup not in
 * [0,1]), FIM_ERR_OOM, FIM_ERR_CUDA, FIM_ERR_TIMEOUT.
 */
fim_status fim_estimate_class_costs(fim_db* db, double sample_rate, double rel_minsup, uint64_t seed,
                                    double* cost_out, uint32_t* order_out);

/* Default bound on the sample's frequent itemsets (see above). */
#define FIM_SAMPLE_ITEMSET_LIMIT (1ull << 20)

/* Cost measure of a class in the estimate. */
typedef enum {
  FIM_COST_ITEMSETS = 0,     /* #frequent itemsets of the sample in the class (the thesis's measure, Sec. 8.2) */
  FIM_COST_INTERSECTIONS = 1 /* #AND+popcount intersections the bitmap Eclat performs for the class on the
                                sample: its level-2 candidates (sample-frequent rows after it) plus every
                                candidate of every node below it; proportional to its GPU work            */
} fim_cost_kind;

/* fim_estimate_class_costs with a choice of cost measure (fim_cost_kind) and
 * of the bound on the sample's itemsets (0 = no bound: the sample is mined at
 * minsup_s whatever its output); fim_estimate_class_costs is this call with
 * FIM_COST_ITEMSETS and FIM_SAMPLE_ITEMSET_LIMIT.  Costs are shares of the
 * total (sum 1 unless the sample has no frequent item). */
fim_status fim_estimate_class_costs_ex(fim_db* db, double sample_rate, double rel_minsup, uint64_t seed,
                                       uint32_t cost_kind, uint64_t max_sample_itemsets, double* cost_out,
                                       uint32_t* order_out);

/* Number of frequent itemsets found in the sample by the last estimate, the
 * sample's size and the sample minsup it was mined at (after any doubling).
 * Waits for a deferred estimate. */
fim_status fim_estimate_sample_size(const fim_db* db, uint64_t* n_sample_fis, uint32_t* sample_rows,
                                    uint32_t* sample_minsup);

/* The last estimate's class costs and LPT order (n_rows entries each, host
 * memory, either may be NULL), as fim_estimate_class_costs_ex returns them;
 * waits for a deferred estimate (and runs its synchronous redo if it needs
 * one).  The thesis's counterpart is the schedule that Sec. 8.2 computes from
 * the sample.  Errors: FIM_ERR_INVALID (no estimate), FIM_ERR_CUDA,
 * FIM_ERR_TIMEOUT. */
fim_status fim_estimate_result(fim_db* db, double* cost_out, uint32_t* order_out);

/*
 * Mine every frequent itemset F = { X != {} : supp(X) >= minsup_abs }
 * (Def. "Frequent itemset", Ch. 2) with exact supports, by Eclat over the
 * db's bitmaps (App. B.3.2): level 2 by the tiled pair kernel, deeper levels
 * by the persistent DFS kernel over the level-3 prefix classes.
 * minsup_abs >= max(1, prefilter_minsup) (0 is rejected: every subset would be
 * frequent).  opts may be NULL (defaults).  The result lists each frequent
 * itemset once with original item ids ascending inside the set; the order of
 * the sets is unspecified.
 * Errors: FIM_ERR_INVALID, FIM_ERR_OOM, FIM_ERR_CUDA, FIM_ERR_TIMEOUT,
 * FIM_ERR_OUTPUT_OVERFLOW (only with a fixed capacity; opts->out_needed_*
 * then hold the sizes that would have sufficed).
 */
fim_status fim_mine(fim_db* db, uint32_t minsup_abs, fim_mine_opts* opts, fim_result** out);

/* CSR view of a result: n_sets sets; set k holds set_items[set_offsets[k] ..
 * set_offsets[k+1]) with supports[k].  Pointers stay valid until
 * fim_result_free; they are device pointers iff *on_device is 1 (on_device may
 * be NULL). */
fim_status fim_result_view(const fim_result* res, uint64_t* n_sets, const uint64_t** set_offsets,
                           const uint32_t** set_items, const uint32_t** supports, int* on_device);

/*
 * Launch-shape autotuner for the persistent DFS kernel (CTA size, 16-byte
 * loads per lane, CTAs per SM, donation, traversal mode).  Mines db at minsup_abs once per
 * candidate shape (twice, best time of the kernels by CUDA events), writes
 * the fastest shape into opts (threads_per_cta, vec_per_lane, ctas_per_sm,
 * donate, dfs_mode) and its time into *best_ms (may be NULL).  Results are cached per
 * (row stride, frequent items, minsup, rows).  The output of a mine never
 * depends on the shape.  opts must come from fim_mine_opts_init; its other
 * fields (class order ...) are used for the trial mines.
 * Errors: as fim_mine.
 */
fim_status fim_autotune(fim_db* db, uint32_t minsup_abs, fim_mine_opts* opts, float* best_ms);

/*
 * Batched mining plan: every prefix class of (db, minsup_abs) fused into the
 * device work of one mine (pair kernel, level-2 queue build, ONE persistent
 * DFS launch over all classes in queue order, ordered by the estimate when
 * one exists) and captured once in a CUDA graph.  Creation runs one eager
 * mine to size the output and the DFS stack, then captures; the plan owns
 * its buffers.  The plan uses db's stream, or a private stream when db was
 * built on the legacy default stream (fim_plan_stream returns it).
 * fim_plan_launch enqueues one replay (asynchronous); fim_plan_result waits
 * for the last replay and returns its itemsets (host or device per
 * opts->result_on_device; opts may be NULL; opts->stats receives counters).
 * db must outlive the plan and stay unchanged.
 * Errors: as fim_mine; FIM_ERR_INVALID for a result before any launch.
 */
fim_status fim_plan_create(fim_db* db, uint32_t minsup_abs, fim_mine_opts* opts, fim_plan** out);
fim_status fim_plan_launch(fim_plan* plan);
fim_status fim_plan_result(fim_plan* plan, fim_mine_opts* opts, fim_result** out);
fim_status fim_plan_stream(const fim_plan* plan, void** cuda_stream);
void fim_plan_free(fim_plan* plan);

/*
 * Serving: a request loop that admits mining jobs on different databases and
 * minsups.  fim_server_create starts `slots` worker threads, each with its own
 * CUDA stream on the current device; hbm_budget_bytes bounds the summed
 * footprint estimate of the jobs in flight (0 = 80% of the free memory);
 * ctas_per_sm caps each job's persistent CTAs per SM (0 = 1) so that
 * concurrent jobs share the SMs; max_itemsets (0 = none) stops a job whose
 * output grows past it (FIM_ERR_OUTPUT_OVERFLOW from fim_server_wait).  fim_server_submit copies the host CSR
 * database (as fim_build_vertical_db) and queues the job; jobs are admitted
 * in arrival order when a slot is free and their footprint fits the budget
 * left (a job larger than the budget runs alone), then run build (prefilter =
 * minsup), the sample estimate when sample_rate > 0, and the mine; the
 * database stays resident on the device until the result is copied out.
 * fim_server_wait blocks until the job is done and returns its result (owned
 * by the caller: fim_result_free), the latency from submission and the
 * service time (either pointer may be NULL); each id can be waited once.
 * The result of a job does not depend on the other jobs in flight.
 * fim_server_submit, fim_server_wait and fim_server_stats may be called from
 * several host threads at once.  fim_server_free stops the workers after the
 * jobs in flight; queued jobs that never started are dropped, so no other
 * call on the server (in particular a wait) may run during or after it.
 * Errors: FIM_ERR_INVALID (bad arguments, unknown id), FIM_ERR_CUDA, and the
 * errors of the job's own build / estimate / mine (returned by wait).
 */
fim_status fim_server_create(uint64_t hbm_budget_bytes, uint32_t slots, uint32_t ctas_per_sm, uint64_t max_itemsets,
                             fim_server** out);
fim_status fim_server_submit(fim_server* srv, const uint32_t* tx_offsets, const uint32_t* tx_items, uint32_t D,
                             uint32_t N, uint32_t minsup_abs, double sample_rate, uint64_t* job_id);
fim_status fim_server_wait(fim_server* srv, uint64_t job_id, fim_result** out, double* latency_s,
                           double* service_s);
/* As fim_server_wait, and the job's device interval: milliseconds from the
 * server's creation to CUDA events recorded on the job's stream just before its
 * first and just after its last device work (-1 when they could not be read).
 * Jobs whose intervals intersect had device work in flight at the same time. */
fim_status fim_server_wait_ex(fim_server* srv, uint64_t job_id, fim_result** out, double* latency_s,
                              double* service_s, double* device_start_ms, double* device_end_ms);
fim_status fim_server_stats(fim_server* srv, uint64_t* in_use_bytes, uint32_t* in_flight, uint32_t* peak_in_flight,
                            uint64_t* queued);
void fim_server_free(fim_server* srv);

/*
 * Frequent pairs without allocation.  The thesis has no counterpart to this
 * entry point; it exists for callers that cannot allocate device memory while
 * they run: a process whose device memory is reserved up front by another
 * allocator (for example a framework's caching pool), or a latency-bound
 * serving loop that must not call cudaMalloc/cudaFree, which may synchronise
 * the whole device.  Every other entry point allocates its scratch on demand.
 *
 * Writes every frequent 2-itemset {a < b} of db (supp >= minsup_abs) to
 * d_pairs[2k], d_pairs[2k+1] (original ids, ascending) and d_supports[k], both
 * DEVICE buffers owned by the caller with room for `capacity` pairs; the
 * order of the pairs is unspecified.  *n_pairs (host) receives the number of
 * frequent pairs, also when it exceeds capacity (then FIM_ERR_OUTPUT_OVERFLOW
 * and only `capacity` of them are written).  The call makes db's device
 * current while it runs (the caller's current device is restored on return)
 * and synchronises db's stream.
 *
 * Scratch: one fixed array inside the library (4 MiB plus a little), held by
 * every GPU that loads the library until the process exits.  At most 1024
 * items may be frequent at minsup_abs; more are rejected with
 * FIM_ERR_INVALID before any device work.  The first call on a device looks up
 * the array's device address (set-up); make that first call before any
 * stream capture.  All calls share the one array, so calls whose device work
 * overlaps (other threads, other streams) race and must be serialised by the
 * caller.  No call allocates memory: no cudaMalloc, cudaFree or allocating
 * library routine.
 * Errors: FIM_ERR_INVALID (NULL db or n_pairs, NULL buffers with capacity > 0,
 * minsup 0 or below the prefilter, more than 1024 frequent items),
 * FIM_ERR_OUTPUT_OVERFLOW, FIM_ERR_CUDA.
 */
fim_status fim_mine_pairs_noalloc(const fim_db* db, uint32_t minsup_abs, uint32_t* d_pairs, uint32_t* d_supports,
                                  uint64_t capacity, uint64_t* n_pairs);

/*
 * Supports of the one-item extensions of an itemset P: supports_out[k] =
 * supp(P u {cand_items[k]}) = |t(P) n t({cand_items[k]})|, the counting step of
 * a class node of Eclat-DFS-Computation (App. B.3.2; support of a union as the
 * size of the intersection of its generating subsets' tidlists, App. B.3.1),
 * on db's bitmaps.  t(P) is the AND of the rows of P's items (a one-item P
 * uses its row in place); each candidate row is then read once, only under
 * the nonzero 16-byte words of t(P).  With a dense t(P) the call streams
 * n_cand rows from HBM: it is the bandwidth-bound form of the DFS's count.
 *
 * prefix_items (n_prefix >= 1 original ids, any order, repeats allowed) and
 * cand_items (n_cand original ids, any order; a candidate inside P gives
 * supp(P)) are HOST arrays read during the call; supports_out is a HOST array
 * of n_cand counts written by it.  Every id must be < N and must have a row
 * (not dropped by the build's prefilter).  n_cand = 0 returns FIM_OK without
 * device work.  The call synchronises db's stream; scratch comes from db's
 * workspace.
 * Errors: FIM_ERR_INVALID (NULL db, empty or NULL prefix, NULL candidates or
 * output with n_cand > 0, an id >= N or without a row), FIM_ERR_CUDA.
 */
fim_status fim_extension_supports(fim_db* db, const uint32_t* prefix_items, uint32_t n_prefix,
                                  const uint32_t* cand_items, uint32_t n_cand, uint32_t* supports_out);

/*
 * Closed and maximal itemsets among a complete result (Ch. 2: Def. "Closed
 * itemset" with its closure operator, Def. "Maximal Frequent Itemset").
 * flags_out[k] (HOST array of n_sets bytes, the result's record order):
 * bit 0 = itemset k is closed (no item outside it lies in every transaction
 * that contains it, i.e. every one-item extension has a smaller support);
 * bit 1 = itemset k is maximal (no proper superset is frequent).  Decided from
 * the result alone: an itemset with an equal-support or a frequent superset has
 * one with one item more, which is frequent and so in a complete result (any
 * result of fim_mine or fim_plan_result; not a run stopped by max_itemsets).
 * Runs on the device (a hash table of the result's itemsets, one lookup per
 * immediate subset of every itemset) on the result's stream, which it
 * synchronises; a host result is copied to the device for it.
 * Errors: FIM_ERR_INVALID (NULL result or flags_out, 2^32 - 1 or more itemsets),
 * FIM_ERR_OOM, FIM_ERR_CUDA.
 */
fim_status fim_result_flags(const fim_result* res, uint8_t* flags_out);

void fim_result_free(fim_result* res);
void fim_db_free(fim_db* db);
const char* fim_status_str(fim_status s);
/* Description of the last error on the calling thread ("" if none). */
const char* fim_last_error(void);

/* Kernels this library has put on a stream since it was loaded, all threads
 * together: every kernel launch, and for a plan every kernel of its graph at
 * each fim_plan_launch (the launches recorded while capturing it do not
 * count).  Kernels run by other libraries (memsets, copies) are not counted. */
uint64_t fim_kernel_launches(void);

/* Device memory of the library's stream-ordered pool on `device` (the pool
 * every database, workspace and device result is carved from): *used_bytes =
 * bytes handed out and not yet freed, *reserved_bytes = bytes the pool holds
 * from the driver (freed blocks stay reserved for reuse).  Either pointer may
 * be NULL.  A device whose pool was never created reports 0 and 0.  Not part
 * of the thesis's method: it lets a serving process account for the memory
 * of its mining jobs, and lets a test see that a call allocated nothing.
 * Errors: FIM_ERR_INVALID (device ordinal out of range), FIM_ERR_CUDA. */
fim_status fim_pool_memory(int device, uint64_t* used_bytes, uint64_t* reserved_bytes);

#ifdef __cplusplus
}
#endif
#endif /* FIM_H_ */
