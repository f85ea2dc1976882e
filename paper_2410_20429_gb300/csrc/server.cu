// server.cu -- continuous-batching render server behind mars_submit / mars_poll.
//
// A scheduler thread admits queued jobs in arrival order while the sum of the
// resident jobs' device footprints stays within the memory budget and a slot
// is free.  Every admitted job gets a worker thread with its own CUDA stream,
// so the iterations of resident jobs overlap on the device; a job's scene,
// cache, queues and image stay resident on the device across its fixed-point
// iterations and are freed when it finishes, which admits the next job.  A job
// of n renders follows the training schedule of mars_training_step_ends: one
// update after each warm-up render, then after 1, 2, 4, ... renders.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>

#include "abi_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// Served jobs bound the splitting along a path (mars_iter_params.max_multiplicity):
// a dark pixel in a job's first MARS iterations, whose estimate comes from a
// few warm-up samples, could otherwise split at the clamp (20) at every bounce
// and hold up the GPU for every other job.  A converged MARS run of the guided
// room spawns about 4 vertices per depth per camera sample, well below the cap.
constexpr float kServeMultiplicity = 16.0f;

struct Job {
  uint64_t id = 0;
  mars::SceneDescCopy scene;
  mars_cache_desc cache{};
  uint32_t seed = 0, key = 0;
  int iterations = 0, warmup = 0;
  double timeout_s = 0.0;
  uint64_t footprint = 0;
  mars_job_state state = MARS_JOB_QUEUED;
  int done_iters = 0;
  mars_status error = MARS_OK;
  std::string message;
  double submit_s = 0, start_s = 0, end_s = 0;
  std::vector<double> iter_ms;
  uint64_t vertices = 0;
  std::vector<float> image;  // mean over post-warm-up iterations
  std::thread worker;
};

}  // namespace

struct mars_server {
  uint64_t budget = 0;
  int max_slots = 1;
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  uint64_t next_id = 1;
  uint64_t in_use = 0;
  int resident = 0;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  std::thread scheduler;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  void run_job(Job* j) {
    mars::NvtxRange nvtx("mars:served_job");
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    mars_scene* sc = nullptr;
    mars_cache* ca = nullptr;
    mars_status rc = MARS_OK;
    std::string msg;
    const int64_t npx = (int64_t)j->scene.desc.width * j->scene.desc.height;
    // the cache's running sum holds every iteration's image: the job's mean
    // image over the iterations after warm-up is (sum at the end - sum after
    // warm-up) / kept, read back twice per job instead of once per iteration
    std::vector<float> warm(3 * (size_t)npx, 0.0f), acc(3 * (size_t)npx, 0.0f);
    int kept = 0;
    auto read_sum = [&](std::vector<float>& dst) {
      mars_cache_state cs{};
      cs.run_sum = dst.data();
      return mars::get_state_impl(ca, &cs, st);
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      rc = MARS_ERR_CUDA;
      msg = "stream create failed";
    }
    if (rc == MARS_OK) rc = mars::scene_create_impl(&j->scene.desc, st, &sc);
    // one tile lane per job: concurrent jobs already fill each other's idle
    // SMs, and a job's first learned iterations, which grow fast, overflow
    // half an arena more often than a whole one
    mars_cache_desc cd = j->cache;
    cd.flags |= MARS_CACHE_ONE_LANE;
    if (rc == MARS_OK) rc = mars::cache_create_impl(sc, &cd, st, &ca);
    for (int it = 0; rc == MARS_OK && it < j->iterations; ++it) {
      if (j->timeout_s > 0.0 && now() - j->start_s > j->timeout_s) {
        rc = mars::set_error(MARS_ERR_TIMEOUT, "job ran past its %.3f s timeout after %d iterations", j->timeout_s, it);
        break;
      }
      mars_iter_params p{};
      p.seed = j->seed;
      p.job = j->key;
      p.iteration = (uint32_t)it;
      p.mode = it < j->warmup ? MARS_MODE_WARMUP : MARS_MODE_MARS;
      p.weights = MARS_WEIGHTS_AWARE;
      p.clamp_lo = 0.05f;
      p.clamp_hi = 20.0f;
      p.outlier = 50.0f;
      p.collect = 1;
      p.max_multiplicity = kServeMultiplicity;
      p.image_on_host = 0;
      p.update_estimate = 1;
      const auto a = Clock::now();
      mars_iter_stats ist{};
      rc = mars::render_iteration_impl(ca, &p, nullptr, &ist, st);
      // the fixed-point step closes each training iteration (1, 2, 4, ...
      // renders after the warm-up ones)
      if (rc == MARS_OK && mars_training_step_ends(it, j->warmup, j->iterations))
        rc = mars::update_counts_impl(ca, st);
      if (rc == MARS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = MARS_ERR_CUDA;
      const double ms = std::chrono::duration<double, std::milli>(Clock::now() - a).count();
      if (rc != MARS_OK) break;
      if (it >= j->warmup) ++kept;
      if (it + 1 == j->warmup && j->warmup < j->iterations) rc = read_sum(warm);
      std::lock_guard<std::mutex> lk(mu);
      j->iter_ms.push_back(ms);
      j->vertices += ist.vertices;
      j->done_iters = it + 1;
    }
    if (rc == MARS_OK && kept > 0) {
      rc = read_sum(acc);
      for (size_t k = 0; k < acc.size(); ++k) acc[k] = (acc[k] - warm[k]) / (float)kept;
    }
    if (rc != MARS_OK) msg = mars_last_error_string();
    if (ca) mars::cache_destroy_impl(ca);
    if (sc) mars::scene_destroy_impl(sc);
    if (st) cudaStreamDestroy(st);
    std::lock_guard<std::mutex> lk(mu);
    j->image.swap(acc);
    j->error = rc;
    j->message = msg;
    j->state = rc == MARS_OK ? MARS_JOB_DONE : MARS_JOB_FAILED;
    j->end_s = now();
    in_use -= j->footprint;
    resident -= 1;
    cv.notify_all();
  }

  void schedule() {
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      cv.wait(lk, [&] {
        if (stop) return true;
        if (queue.empty() || resident >= max_slots) return false;
        const Job* j = jobs[queue.front()].get();
        return in_use + j->footprint <= budget || resident == 0;
      });
      if (stop) return;
      Job* j = jobs[queue.front()].get();
      queue.pop_front();
      in_use += j->footprint;
      resident += 1;
      j->state = MARS_JOB_RUNNING;
      j->start_s = now();
      j->worker = std::thread([this, j] { run_job(j); });
    }
  }
};

extern "C" {

mars_status mars_server_create(uint64_t memory_budget_bytes, int32_t max_slots, mars_server** out) {
  if (!out || max_slots < 1 || memory_budget_bytes == 0)
    return mars::set_error(MARS_ERR_INVALID_ARG, "server needs an output, max_slots >= 1 and a budget");
  mars_server* s = new mars_server();
  s->budget = memory_budget_bytes;
  s->max_slots = max_slots;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return mars::set_error(MARS_ERR_CUDA, "no CUDA device");
  }
  s->t0 = Clock::now();
  s->scheduler = std::thread([s] { s->schedule(); });
  *out = s;
  return MARS_OK;
}

mars_status mars_server_destroy(mars_server* s) {
  if (!s) return MARS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  s->scheduler.join();
  for (auto& kv : s->jobs)
    if (kv.second->worker.joinable()) kv.second->worker.join();
  delete s;
  return MARS_OK;
}

mars_status mars_submit(mars_server* s, const mars_job_desc* jd, uint64_t* job_id) {
  if (!s || !jd || !jd->scene || !job_id) return mars::set_error(MARS_ERR_INVALID_ARG, "null server, job or id");
  if (jd->iterations < 1 || jd->warmup < 0 || jd->warmup > jd->iterations)
    return mars::set_error(MARS_ERR_INVALID_ARG, "bad iteration counts");
  const mars_scene_desc* d = jd->scene;
  if (d->width <= 0 || d->height <= 0) return mars::set_error(MARS_ERR_INVALID_ARG, "bad resolution");
  auto j = std::make_unique<Job>();
  j->scene.assign(d);
  j->cache = jd->cache;
  j->seed = jd->seed;
  j->key = jd->key;
  j->iterations = jd->iterations;
  j->warmup = jd->warmup;
  if (!(jd->timeout_s >= 0.0)) return mars::set_error(MARS_ERR_INVALID_ARG, "negative timeout");
  j->timeout_s = jd->timeout_s;
  const int64_t npx = (int64_t)d->width * d->height;
  const int64_t cells = (int64_t)jd->cache.grid_n * jd->cache.grid_n * jd->cache.grid_n;
  const uint64_t cap = jd->cache.arena_capacity ? jd->cache.arena_capacity
                                                 : mars::default_capacity(npx, jd->cache.max_depth);
  const int nprim = d->n_quads + d->n_spheres + d->n_tris;
  j->footprint = mars::cache_footprint(cells, npx, jd->cache.max_depth, jd->cache.techniques, cap) +
                 (uint64_t)nprim * 256 + (64ull << 20);
  if (j->footprint > s->budget)
    return mars::set_error(MARS_ERR_OOM, "job needs %llu bytes, more than the budget",
                           (unsigned long long)j->footprint);
  std::lock_guard<std::mutex> lk(s->mu);
  j->id = s->next_id++;
  j->submit_s = s->now();
  *job_id = j->id;
  s->queue.push_back(j->id);
  s->jobs[j->id] = std::move(j);
  s->cv.notify_all();
  return MARS_OK;
}

mars_status mars_poll(mars_server* s, uint64_t job_id, mars_job_status* out, float* image_rgb) {
  if (!s || !out) return mars::set_error(MARS_ERR_INVALID_ARG, "null server or output");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return mars::set_error(MARS_ERR_NOT_FOUND, "unknown job %llu", (unsigned long long)job_id);
  Job* j = it->second.get();
  out->state = j->state;
  out->iterations_done = j->done_iters;
  out->error = j->error;
  out->reserved = 0;
  out->submit_s = j->submit_s;
  out->start_s = j->start_s;
  out->end_s = j->end_s;
  std::vector<double> ms = j->iter_ms;
  std::sort(ms.begin(), ms.end());
  auto q = [&](double f) {
    if (ms.empty()) return 0.0;
    const size_t k = std::min(ms.size() - 1, (size_t)std::ceil(f * (double)ms.size()) - (f > 0 ? 1 : 0));
    return ms[k];
  };
  out->iter_ms_p50 = q(0.5);
  out->iter_ms_p99 = q(0.99);
  out->device_bytes = j->footprint;
  out->vertices = j->vertices;
  if (j->state == MARS_JOB_FAILED) mars::set_error(j->error, "job %llu failed: %s", (unsigned long long)job_id,
                                                   j->message.c_str());
  if (image_rgb && j->state == MARS_JOB_DONE && !j->image.empty())
    std::copy(j->image.begin(), j->image.end(), image_rgb);
  return MARS_OK;
}

mars_status mars_job_latencies(mars_server* s, uint64_t job_id, double* ms, int32_t capacity, int32_t* count) {
  if (!s || !count || capacity < 0 || (capacity > 0 && !ms))
    return mars::set_error(MARS_ERR_INVALID_ARG, "null server, count or buffer");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return mars::set_error(MARS_ERR_NOT_FOUND, "unknown job %llu", (unsigned long long)job_id);
  const std::vector<double>& v = it->second->iter_ms;
  const size_t n = std::min(v.size(), (size_t)capacity);
  std::copy(v.begin(), v.begin() + n, ms);
  *count = (int32_t)v.size();
  return MARS_OK;
}

}  // extern "C"
