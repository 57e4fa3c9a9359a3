// Serving: a continuous-batching request loop for mining jobs.
//
// Every job is a database in host CSR form plus an absolute minsup.  Jobs are
// admitted in arrival order as soon as a slot is free and their estimated
// device footprint fits the HBM budget left by the jobs in flight; each slot
// runs its job (bitmap build with the minsup as prefilter, sample estimate,
// mine) on its own CUDA stream, so the kernels of concurrent jobs overlap on
// the device.  Bitmaps of a job stay resident until its result is copied out.
// The persistent DFS of a served job exits as soon as its queue drains (no
// idle polling), so concurrent jobs never hold SMs for one another.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fim_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t id = 0;
  std::vector<uint32_t> off, items;
  uint32_t D = 0, N = 0, minsup = 1;
  double sample_rate = 0.0;
  uint64_t footprint = 0;
  Clock::time_point t_submit, t_start, t_end;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // the job's device work on its slot's stream
  fim_status status = FIM_OK;
  std::string error;
  fim_result* result = nullptr;
  bool done = false;
  bool taken = false;
};

}  // namespace

struct fim_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::unordered_map<uint64_t, Job*> jobs;
  uint64_t next_id = 1;
  uint64_t budget = 0, in_use = 0;
  uint32_t in_flight = 0, peak_in_flight = 0;
  bool stop = false;
  int device = 0;
  uint32_t ctas_per_sm = 1;
  uint64_t max_itemsets = 0;
  uint64_t total_mem = 0;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  cudaEvent_t ev_origin = nullptr;  // recorded at creation: device times of jobs are measured from it
};

namespace {

// Upper bound of the device bytes of one job: CSR copy, bitmaps of the items that
// can reach minsup (at most nnz / minsup of them), pair block, queue, DFS stack,
// output, with the sample of the estimate on top.
uint64_t job_footprint(uint32_t D, uint32_t N, uint64_t nnz, uint32_t max_len, uint32_t minsup, uint32_t grid,
                       uint64_t total_mem, int num_sms) {
  const uint64_t stride = ((uint64_t)(D + 31) / 32 + 31) / 32 * 32;
  const uint64_t rows = std::min<uint64_t>(N, nnz / std::max<uint32_t>(1, minsup) + 1);
  uint64_t b = 4ull * ((uint64_t)D + 1 + nnz);           // CSR
  b += 4ull * rows * stride;                              // bitmaps
  b += 4ull * rows * rows + 12ull * rows * rows / 2;      // pair counts, survivors, queue
  // rows widened to bytes when the engine would take the tensor-core pair kernel
  const uint64_t xb = fim::pair_mma_buffer_bytes((uint32_t)rows, (uint32_t)stride, true);
  if (rows >= 2 && xb <= total_mem / 16 &&
      fim::pair_mma_cost_us((uint32_t)rows, (uint32_t)stride, num_sms, true) <
          fim::pair_cores_cost_us((uint32_t)rows, (uint32_t)stride, num_sms))
    b += xb;
  // DFS stack: the full depth (itemsets are no longer than the longest transaction) when it fits
  // in 1/32 of the device memory, as the engine decides
  const uint64_t depth = std::max<uint32_t>(3, std::min<uint64_t>(max_len, rows)) - 1;
  const uint64_t full = 4ull * (stride + 2 * rows + 8) * depth * grid;
  b += full <= total_mem / 32 ? full : 4ull * (stride + 2 * rows + 8) * (fim::kDfsDepthHint + 1) * grid;
  // the projected DFS of wide rows: class database parts, transactions, the warps' stacks
  if (stride > 2048) b += fim::proj_footprint_bytes((uint32_t)rows, (uint32_t)stride, nnz, (uint32_t)grid);
  b += 64ull << 20;                                       // output, sample, small buffers
  return b;
}

void run_job(fim_server* srv, Job* j, cudaStream_t st) {
  cudaSetDevice(srv->device);
  fim_db* db = nullptr;
  fim_status s = fim_build_vertical_db(j->off.data(), j->items.data(), j->D, j->N, 64, j->minsup, st, &db);
  if (s == FIM_OK && j->sample_rate > 0.0) {
    s = fim_estimate_class_costs(db, j->sample_rate, (double)j->minsup / (double)j->D, 1000 + j->id, nullptr,
                                 nullptr);
  }
  if (s == FIM_OK) {
    fim_mine_opts o;
    fim_mine_opts_init(&o);
    o.ctas_per_sm = srv->ctas_per_sm;
    o.donate = 0;
    o.max_itemsets = srv->max_itemsets;
    s = fim_mine(db, j->minsup, &o, &j->result);
  }
  if (s != FIM_OK) j->error = fim_last_error();
  j->status = s;
  fim_db_free(db);
}

void worker_main(fim_server* srv, size_t slot) {
  cudaSetDevice(srv->device);
  cudaStream_t st = srv->streams[slot];
  for (;;) {
    Job* j = nullptr;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      srv->cv_work.wait(lock, [&] {
        if (srv->stop) return true;
        if (srv->queue.empty()) return false;
        const Job* h = srv->queue.front();
        return srv->in_flight == 0 || srv->in_use + h->footprint <= srv->budget;
      });
      if (srv->stop && srv->queue.empty()) return;
      if (srv->stop) return;
      j = srv->queue.front();
      srv->queue.pop_front();
      srv->in_use += j->footprint;
      srv->in_flight += 1;
      srv->peak_in_flight = std::max(srv->peak_in_flight, srv->in_flight);
    }
    j->t_start = Clock::now();
    // (events on the slot's stream bracket the job's device work; timing only, no synchronisation)
    if (cudaEventCreate(&j->ev_start) == cudaSuccess) cudaEventRecord(j->ev_start, st);
    run_job(srv, j, st);
    if (cudaEventCreate(&j->ev_end) == cudaSuccess) cudaEventRecord(j->ev_end, st);
    j->t_end = Clock::now();
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      srv->in_use -= j->footprint;
      srv->in_flight -= 1;
      j->off.clear();
      j->off.shrink_to_fit();
      j->items.clear();
      j->items.shrink_to_fit();
      j->done = true;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
}

}  // namespace

using namespace fim;

extern "C" {

fim_status fim_server_create(uint64_t hbm_budget_bytes, uint32_t slots, uint32_t ctas_per_sm, uint64_t max_itemsets,
                             fim_server** out) {
  if (!out) return fail(FIM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (slots == 0 || slots > 64) return fail(FIM_ERR_INVALID, "slots must be in 1..64");
  fim_server* srv = new (std::nothrow) fim_server();
  if (!srv) return fail(FIM_ERR_OOM, "host allocation");
  {
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaGetDevice(&srv->device);
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
      delete srv;
      return cuda_fail(e, "server device");
    }
    srv->total_mem = total_b;
    if (hbm_budget_bytes == 0) hbm_budget_bytes = (uint64_t)(free_b * 0.8);
  }
  srv->budget = hbm_budget_bytes;
  srv->ctas_per_sm = ctas_per_sm ? ctas_per_sm : 1;
  srv->max_itemsets = max_itemsets;
  for (uint32_t k = 0; k < slots; ++k) {
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (auto x : srv->streams) cudaStreamDestroy(x);
      delete srv;
      return cuda_fail(e, "server stream");
    }
    srv->streams.push_back(s);
  }
  if (cudaEventCreate(&srv->ev_origin) == cudaSuccess) cudaEventRecord(srv->ev_origin, srv->streams[0]);
  for (uint32_t k = 0; k < slots; ++k) srv->workers.emplace_back(worker_main, srv, (size_t)k);
  *out = srv;
  return FIM_OK;
}

fim_status fim_server_submit(fim_server* srv, const uint32_t* tx_offsets, const uint32_t* tx_items, uint32_t D,
                             uint32_t N, uint32_t minsup_abs, double sample_rate, uint64_t* job_id) {
  if (!srv || !tx_offsets || !job_id || D == 0 || N == 0 || minsup_abs == 0)
    return fail(FIM_ERR_INVALID, "bad server submission");
  Job* j = new (std::nothrow) Job();
  if (!j) return fail(FIM_ERR_OOM, "host allocation");
  j->t_submit = Clock::now();
  const uint64_t nnz = tx_offsets[D];
  j->off.assign(tx_offsets, tx_offsets + D + 1);
  if (nnz) j->items.assign(tx_items, tx_items + nnz);
  j->D = D;
  j->N = N;
  j->minsup = minsup_abs;
  j->sample_rate = sample_rate;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, srv->device);
  uint32_t max_len = 0;
  for (uint32_t t = 0; t < D; ++t)
    if (tx_offsets[t + 1] > tx_offsets[t]) max_len = std::max(max_len, tx_offsets[t + 1] - tx_offsets[t]);
  j->footprint = job_footprint(D, N, nnz, max_len, minsup_abs, (uint32_t)nsm * srv->ctas_per_sm, srv->total_mem, nsm);
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    j->id = srv->next_id++;
    srv->jobs[j->id] = j;
    srv->queue.push_back(j);
  }
  srv->cv_work.notify_all();
  *job_id = j->id;
  return FIM_OK;
}

fim_status fim_server_wait(fim_server* srv, uint64_t job_id, fim_result** out, double* latency_s,
                           double* service_s) {
  return fim_server_wait_ex(srv, job_id, out, latency_s, service_s, nullptr, nullptr);
}

fim_status fim_server_wait_ex(fim_server* srv, uint64_t job_id, fim_result** out, double* latency_s,
                              double* service_s, double* device_start_ms, double* device_end_ms) {
  if (device_start_ms) *device_start_ms = -1.0;
  if (device_end_ms) *device_end_ms = -1.0;
  if (!srv || !out) return fail(FIM_ERR_INVALID, "server or out is NULL");
  *out = nullptr;
  Job* j = nullptr;
  {
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end() || it->second->taken) return fail(FIM_ERR_INVALID, "unknown job id");
    j = it->second;
    j->taken = true;
    srv->cv_done.wait(lock, [&] { return j->done; });
    srv->jobs.erase(it);
  }
  if (latency_s) *latency_s = std::chrono::duration<double>(j->t_end - j->t_submit).count();
  if (service_s) *service_s = std::chrono::duration<double>(j->t_end - j->t_start).count();
  // the job's device interval from the server's origin event (both events completed: the job's result
  // was synchronised on its stream before the worker marked it done)
  float t0 = -1.f, t1 = -1.f;
  if (srv->ev_origin && j->ev_start && j->ev_end && cudaEventSynchronize(j->ev_end) == cudaSuccess &&
      cudaEventElapsedTime(&t0, srv->ev_origin, j->ev_start) == cudaSuccess &&
      cudaEventElapsedTime(&t1, srv->ev_origin, j->ev_end) == cudaSuccess) {
    if (device_start_ms) *device_start_ms = t0;
    if (device_end_ms) *device_end_ms = t1;
  }
  if (j->ev_start) cudaEventDestroy(j->ev_start);
  if (j->ev_end) cudaEventDestroy(j->ev_end);
  fim_status s = j->status;
  if (s == FIM_OK) *out = j->result;
  else set_error(j->error);
  delete j;
  return s;
}

fim_status fim_server_stats(fim_server* srv, uint64_t* in_use_bytes, uint32_t* in_flight, uint32_t* peak_in_flight,
                            uint64_t* queued) {
  if (!srv) return fail(FIM_ERR_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lock(srv->mu);
  if (in_use_bytes) *in_use_bytes = srv->in_use;
  if (in_flight) *in_flight = srv->in_flight;
  if (peak_in_flight) *peak_in_flight = srv->peak_in_flight;
  if (queued) *queued = srv->queue.size();
  return FIM_OK;
}

void fim_server_free(fim_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  for (auto& kv : srv->jobs) {
    if (kv.second->result) fim_result_free(kv.second->result);
    if (kv.second->ev_start) cudaEventDestroy(kv.second->ev_start);
    if (kv.second->ev_end) cudaEventDestroy(kv.second->ev_end);
    delete kv.second;
  }
  for (Job* j : srv->queue)
    if (srv->jobs.find(j->id) == srv->jobs.end()) delete j;
  for (auto s : srv->streams) cudaStreamDestroy(s);
  if (srv->ev_origin) cudaEventDestroy(srv->ev_origin);
  delete srv;
}

}  // extern "C"
