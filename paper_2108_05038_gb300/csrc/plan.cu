// Batched mining plans and the launch-shape autotuner.
//
// A plan fuses every prefix class of one (database, minsup) into the same
// device work as fim_mine - pair kernel, level-2 queue build, one persistent
// DFS launch over all classes in queue order - and captures it once in a CUDA
// graph, so that repeated mining of the same database replays one graph.
// Sizes (output capacity, DFS stack depth) come from one eager run at
// creation, so a replay never needs to grow a buffer.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fim_internal.cuh"

struct fim_plan {
  fim_db* db = nullptr;
  fim::Workspace ws;
  fim::EnginePlan ep;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches = 0;
  uint64_t kernels = 0;  // kernels in the graph
};

namespace fim {
namespace {

// launch shapes tried by the autotuner: CTA size x 16-byte loads per lane x
// CTAs per SM (0 = as many as fit) x donation x DFS traversal (the warp DFS runs
// as the sparse node mode on rows wider than 512 words)
struct Shape {
  uint32_t threads, vec, cps, donate, mode;
};
const Shape kShapes[] = {
    {128, 2, 0, 0, 0}, {128, 4, 0, 0, 0}, {256, 2, 0, 0, 0}, {256, 4, 0, 0, 0}, {256, 8, 0, 0, 0},
    {512, 4, 0, 0, 0}, {512, 8, 0, 0, 0}, {256, 4, 0, 1, 0}, {512, 4, 0, 1, 0},
    {512, 2, 0, 0, 0}, {128, 2, 0, 0, 1}, {128, 4, 0, 0, 1}, {256, 2, 0, 0, 1}, {256, 4, 0, 0, 1},
    {256, 8, 0, 0, 1}, {512, 4, 0, 0, 1}, {512, 8, 0, 0, 1}, {128, 4, 0, 0, 3}, {128, 8, 0, 0, 3},
    {256, 4, 0, 0, 3}, {256, 8, 0, 0, 3}, {256, 4, 0, 0, 4},
};

struct TuneKey {
  uint32_t stride, n1, minsup, rows;
  bool operator<(const TuneKey& o) const {
    return std::tie(stride, n1, minsup, rows) < std::tie(o.stride, o.n1, o.minsup, o.rows);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<Shape, float>> g_tuned;

}  // namespace
}  // namespace fim

using namespace fim;

extern "C" {

fim_status fim_autotune(fim_db* db, uint32_t minsup_abs, fim_mine_opts* opts, float* best_ms) {
  if (!opts || opts->struct_size != sizeof(fim_mine_opts)) return fail(FIM_ERR_INVALID, "opts must be initialised");
  EngineInput in;
  EngineConfig cfg;
  FIM_TRY(mine_input(db, minsup_abs, opts, &in, &cfg));
  const TuneKey key{in.stride, in.n1, minsup_abs, db->n_rows};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      opts->threads_per_cta = it->second.first.threads;
      opts->vec_per_lane = it->second.first.vec;
      opts->ctas_per_sm = it->second.first.cps;
      opts->donate = it->second.first.donate;
      opts->dfs_mode = it->second.first.mode;
      if (best_ms) *best_ms = it->second.second;
      return FIM_OK;
    }
  }
  // time the whole device part of a mine (events around the kernels) per shape; best of two runs
  Shape best = kShapes[0];
  float best_t = 1e30f;
  for (const Shape& sh : kShapes) {
    EngineConfig c = cfg;
    c.threads = sh.threads;
    c.vec = sh.vec;
    c.ctas_per_sm = sh.cps;
    c.donate = sh.donate;
    c.mode = sh.mode;
    c.collect_times = true;
    float t = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      fim_mine_stats st{};
      EngineOutput eo;
      FIM_TRY(engine_mine(db, db->ws, in, c, &eo, &st));
      t = std::min(t, st.ms_device_total);
    }
    if (t < best_t) {
      best_t = t;
      best = sh;
    }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = {best, best_t};
  }
  opts->threads_per_cta = best.threads;
  opts->vec_per_lane = best.vec;
  opts->ctas_per_sm = best.cps;
  opts->donate = best.donate;
  opts->dfs_mode = best.mode;
  if (best_ms) *best_ms = best_t;
  return FIM_OK;
}

fim_status fim_plan_create(fim_db* db, uint32_t minsup_abs, fim_mine_opts* opts, fim_plan** out) {
  if (!out) return fail(FIM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  EngineInput in;
  EngineConfig cfg;
  FIM_TRY(mine_input(db, minsup_abs, opts, &in, &cfg));
  if (cfg.output != FIM_OUTPUT_ALL) return fail(FIM_ERR_INVALID, "a plan returns every frequent itemset (output 0)");
  cfg.collect_times = false;
  fim_plan* plan = new (std::nothrow) fim_plan();
  if (!plan) return fail(FIM_ERR_OOM, "host allocation");
  plan->db = db;
  auto bail = [&](fim_status s) {
    fim_plan_free(plan);
    return s;
  };
  if (db->stream) {
    plan->stream = db->stream;
  } else {  // the legacy default stream cannot be captured: use a private stream
    cudaError_t e = cudaStreamCreateWithFlags(&plan->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "plan stream"));
    plan->own_stream = true;
    e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) return bail(cuda_fail(e, "plan stream"));
  }
  plan->ws.stream = plan->stream;
  // one eager run sizes the buffers, then the launch sequence is captured with those sizes
  EngineOutput eo;
  fim_status s = engine_mine(db, plan->ws, in, cfg, &eo, nullptr, &plan->ep);
  if (s != FIM_OK) return bail(s);
  plan->ep.fixed_capacity = true;
  cudaError_t e = cudaStreamBeginCapture(plan->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamBeginCapture"));
  const uint64_t before = launches_so_far();
  cudaError_t le = engine_launch(plan->ep, plan->stream);
  // launches recorded into the graph run only when it is launched
  plan->kernels = launches_so_far() - before;
  note_launch(0 - plan->kernels);
  e = cudaStreamEndCapture(plan->stream, &plan->graph);
  if (le != cudaSuccess) return bail(cuda_fail(le, "capturing the mining kernels"));
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamEndCapture"));
  e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGraphInstantiate"));
  *out = plan;
  return FIM_OK;
}

fim_status fim_plan_launch(fim_plan* plan) {
  if (!plan || !plan->exec) return fail(FIM_ERR_INVALID, "plan is NULL");
  FIM_CUDA(cudaGraphLaunch(plan->exec, plan->stream));
  ++plan->launches;
  note_launch(plan->kernels);
  return FIM_OK;
}

fim_status fim_plan_result(fim_plan* plan, fim_mine_opts* opts, fim_result** out) {
  if (!plan || !out) return fail(FIM_ERR_INVALID, "plan or out is NULL");
  *out = nullptr;
  if (plan->launches == 0) return fail(FIM_ERR_INVALID, "plan was never launched");
  fim_mine_stats local{};
  fim_mine_stats* stats = opts && opts->struct_size && opts->stats ? opts->stats : &local;
  std::memset(stats, 0, sizeof(*stats));
  EngineOutput eo;
  bool retry = false;
  FIM_TRY(engine_finish(plan->db, plan->stream, &plan->ep, &eo, stats, &retry));
  if (retry) return fail(FIM_ERR_OUTPUT_OVERFLOW, "plan buffers no longer fit the database");
  return make_result(plan->stream, eo, opts && opts->struct_size && opts->result_on_device, out);
}

fim_status fim_plan_stream(const fim_plan* plan, void** cuda_stream) {
  if (!plan || !cuda_stream) return fail(FIM_ERR_INVALID, "plan or cuda_stream is NULL");
  *cuda_stream = plan->stream;
  return FIM_OK;
}

void fim_plan_free(fim_plan* plan) {
  if (!plan) return;
  if (plan->stream) cudaStreamSynchronize(plan->stream);
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  plan->ws.release();
  if (plan->stream) cudaStreamSynchronize(plan->stream);
  if (plan->own_stream) cudaStreamDestroy(plan->stream);
  delete plan;
}

}  // extern "C"
