// Job server of the C ABI (bm_server_create / bm_submit / bm_wait /
// bm_server_destroy): whole Big-means jobs (Alg. 1) from any thread, several
// at once on one GPU.
//
// Admission: a job's device footprint (the workspace its context would
// allocate) is computed at submission; a job larger than the whole budget
// is refused (BM_ENOMEM), a submission beyond max_queue waiting jobs is
// refused (BM_EBUSY).  Dispatch: first in, first out; a worker takes the
// head job once the head's footprint fits in what the running jobs leave of
// the budget.  A job's chunk kernels use at most the server's job_ctas CTAs
// (default ceil(SMs / 2); it does not depend on the worker count, so a job's
// results do not either) unless the job sets its own cap, so the workers'
// jobs run side by side on disjoint SMs instead of queueing behind each
// other's cooperative launches (each would otherwise span the whole GPU).  Each worker thread owns a
// non-blocking stream; job state is
// allocated from the server's stream-ordered memory pool, which keeps freed
// memory for the next job, so no job synchronises the device.  Results are
// those of the same job run alone: the kernels' reductions have a fixed
// order and a job touches only its own buffers.
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bigmeans.h"
#include "bm_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket = 0;
  bm_job spec{};
  int64_t footprint = 0;
  Clock::time_point t_submit, t_start;
  bm_job_result result{};
  bool done = false;
};

double seconds(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

// Runs the device current on the calling thread back to `saved` on scope exit.
struct DeviceScope {
  int saved = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&saved) == cudaSuccess && saved != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur = -1;
    if (saved >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != saved) cudaSetDevice(saved);
  }
};

}  // namespace

struct bm_server {
  bm_server_config cfg{};
  int device = 0;
  int cap = 0;                  // CTA cap of a job without its own: job_ctas
  cudaMemPool_t pool = nullptr;
  std::mutex mu;
  std::condition_variable cv;   // any change: job queued or finished, memory freed, stop
  std::deque<std::shared_ptr<Job>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;   // admitted, not yet collected
  uint64_t next_ticket = 1;
  int64_t mem_in_use = 0;
  bool stopping = false;
  bm_server_stats stats{};
  std::vector<std::thread> workers;
};

namespace {

// One job on the worker's stream: a context from the pool, the chunks, the
// final assignment, the incumbent; then the context's memory goes back to
// the pool (stream-ordered).
void run_job(bm_server* sv, cudaStream_t st, Job& job) {
  bm_config cfg = job.spec.cfg;
  cfg.graphs = 0;   // a context per job: recording would not pay for itself
  cfg.trace = 0;
  if (cfg.max_ctas <= 0) cfg.max_ctas = sv->cap;
  bm_ctx* ctx = nullptr;
  bm_fit_report rep{};
  double sse = 0.0, f_opt = 0.0;
  bm_status rc = bm::ctx_create(&cfg, job.spec.X_dev, st, sv->pool, &ctx);
  if (rc == BM_OK) rc = bm_fit_chunk(ctx, job.spec.chunks, &rep);
  if (rc == BM_OK) rc = bm_assign(ctx, job.spec.labels_dev, &sse);
  if (rc == BM_OK)
    rc = bm_get_state(ctx, job.spec.C_out_host, job.spec.mask_out_host, &f_opt, nullptr);
  if (ctx) bm_destroy(ctx);
  job.result.status = rc;
  job.result.sse = sse;
  job.result.f_opt = f_opt;
  job.result.lloyd_iters = rep.lloyd_iters;
  job.result.accepted = rep.accepted;
}

void worker_main(bm_server* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  while (true) {
    std::shared_ptr<Job> job;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] {
        return sv->stopping ||
               (!sv->queue.empty() &&
                sv->mem_in_use + sv->queue.front()->footprint <= sv->cfg.memory_budget);
      });
      if (sv->stopping) break;   // queued jobs are cancelled by bm_server_destroy
      job = sv->queue.front();
      sv->queue.pop_front();
      sv->mem_in_use += job->footprint;
      sv->stats.queued -= 1;
      sv->stats.running += 1;
      sv->stats.memory_in_use = sv->mem_in_use;
      job->t_start = Clock::now();
    }
    if (st) run_job(sv, st, *job);
    else job->result.status = BM_ECUDA;
    bm_job_callback cb = nullptr;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      const Clock::time_point t = Clock::now();
      job->result.queued_s = seconds(job->t_submit, job->t_start);
      job->result.run_s = seconds(job->t_start, t);
      job->result.latency_s = seconds(job->t_submit, t);
      job->done = true;
      sv->mem_in_use -= job->footprint;
      sv->stats.memory_in_use = sv->mem_in_use;
      sv->stats.running -= 1;
      if (job->result.status == BM_OK) sv->stats.completed += 1;
      else sv->stats.failed += 1;
      cb = job->spec.callback;
    }
    sv->cv.notify_all();
    if (cb) {
      cb(job->ticket, &job->result, job->spec.user);
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->jobs.erase(job->ticket);
    }
  }
  if (st) {
    cudaStreamSynchronize(st);   // the stream-ordered frees of its last job
    cudaStreamDestroy(st);
  }
}

}  // namespace

extern "C" {

bm_status bm_server_create(const bm_server_config* cfg, bm_server** out) {
  if (!cfg || !out || cfg->workers < 1 || cfg->max_queue < 1 || cfg->memory_budget < 0 ||
      cfg->job_ctas < 0)
    return BM_EINVAL;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return BM_ECUDA; }
  bm_server* sv = new (std::nothrow) bm_server();
  if (!sv) return BM_ENOMEM;
  sv->cfg = *cfg;
  sv->device = dev;
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // half the GPU: on a mixed load (m up to 5e6, n from 8 to 384, jobs of
  // 20 chunks) two large jobs fill it and small ones overlap (measured: 174
  // jobs/s against 143 with a quarter or the whole GPU per job)
  sv->cap = cfg->job_ctas > 0 ? cfg->job_ctas : (sms + 1) / 2;
  if (sv->cfg.memory_budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { delete sv; return BM_ECUDA; }
    sv->cfg.memory_budget = (int64_t)(free_b / 2);
  }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  if (cudaMemPoolCreate(&sv->pool, &props) != cudaSuccess) { delete sv; return BM_ECUDA; }
  uint64_t keep = UINT64_MAX;   // freed memory stays in the pool for the next job
  cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  sv->stats.memory_budget = sv->cfg.memory_budget;
  for (int i = 0; i < cfg->workers; ++i) sv->workers.emplace_back(worker_main, sv);
  *out = sv;
  return BM_OK;
}

bm_status bm_server_destroy(bm_server* sv) {
  if (!sv) return BM_OK;
  std::vector<std::shared_ptr<Job>> cancelled;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
    for (auto& job : sv->queue) {
      job->result.status = BM_ECANCELLED;
      job->done = true;
      sv->stats.cancelled += 1;
      cancelled.push_back(job);
    }
    sv->stats.queued = 0;
    sv->queue.clear();
  }
  sv->cv.notify_all();
  for (auto& job : cancelled) {
    if (!job->spec.callback) continue;
    job->spec.callback(job->ticket, &job->result, job->spec.user);
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->jobs.erase(job->ticket);
  }
  for (std::thread& t : sv->workers) t.join();
  {
    DeviceScope ds(sv->device);
    cudaMemPoolDestroy(sv->pool);
  }
  delete sv;
  return BM_OK;
}

bm_status bm_submit(bm_server* sv, const bm_job* job, uint64_t* ticket) {
  if (!sv || !job || !ticket || !job->X_dev || job->chunks < 1) return BM_EINVAL;
  int64_t fp = 0;
  {
    DeviceScope ds(sv->device);
    size_t bytes = 0;
    bm_config cfg = job->cfg;
    if (cfg.max_ctas <= 0) cfg.max_ctas = sv->cap;
    const bm_status rc = bm::ctx_footprint(&cfg, &bytes);
    if (rc != BM_OK) return rc;
    fp = (int64_t)bytes;
  }
  auto rec = std::make_shared<Job>();
  rec->spec = *job;
  rec->footprint = fp;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) return BM_ECANCELLED;
    if (fp > sv->cfg.memory_budget) {
      sv->stats.rejected_memory += 1;
      return BM_ENOMEM;
    }
    if ((int64_t)sv->queue.size() >= sv->cfg.max_queue) {
      sv->stats.rejected_busy += 1;
      return BM_EBUSY;
    }
    rec->ticket = sv->next_ticket++;
    rec->t_submit = Clock::now();
    sv->jobs.emplace(rec->ticket, rec);
    sv->queue.push_back(rec);
    sv->stats.submitted += 1;
    sv->stats.queued += 1;
    *ticket = rec->ticket;
  }
  sv->cv.notify_all();
  return BM_OK;
}

bm_status bm_wait(bm_server* sv, uint64_t ticket, double timeout_s, bm_job_result* out) {
  if (!sv) return BM_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return BM_EINVAL;
  std::shared_ptr<Job> job = it->second;
  auto ready = [&] { return job->done; };
  if (timeout_s < 0.0) {
    sv->cv.wait(lk, ready);
  } else if (!sv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return BM_ETIMEOUT;
  }
  if (out) *out = job->result;
  if (!job->spec.callback) sv->jobs.erase(ticket);
  return BM_OK;
}

bm_status bm_server_stats_get(bm_server* sv, bm_server_stats* out) {
  if (!sv || !out) return BM_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  return BM_OK;
}

}  // extern "C"
