// rt_server.cu -- a job server for radiative-transfer requests (the serving
// runtime: continuous batching with admission by device-memory footprint).
//
// Requests name a model (a density tree) by id, its sources, optics,
// package budget and observers.  Grids stay resident on the device across
// requests (built on first use, evicted least-recently-used when memory is
// needed and no running job uses them).  A request is admitted when its
// footprint -- its grid unless resident, plus its absorbed-energy and image
// accumulators -- fits the free part of the budget.  Dispatcher threads, one
// per slot, each with its own context and CUDA stream, take every admitted
// request in arrival order (up to a batch size) and run them as one
// persistent batched launch; a request that arrives while a batch runs joins
// the next batch of whichever slot frees first, so work from different slots
// overlaps on the device.  Results stay on the device until fetched.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "rt_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct ModelEntry {
  // host copy of the tree (registered once; rebuilt from it after eviction)
  rt_tree_desc tree;
  std::vector<int64_t> n_refined;
  std::vector<uint8_t> flags;
  std::vector<double> density;
  int64_t n_cells = 0;
  rt_grid* grid = nullptr;
  size_t bytes = 0;        // device bytes of the grid
  bool counted = false;    // grid bytes are in the budget (built or being built)
  int users = 0;           // admitted jobs referring to it
  Clock::time_point last_use;
};

struct Job {
  uint64_t ticket = 0;
  uint64_t model_id = 0;
  // copies of the request (host data owned by the job)
  std::vector<rt_source> src;
  std::vector<std::vector<double>> src_energy;
  rt_optics optics;
  std::vector<double> kext, alb, g;
  rt_trace_params params;
  std::vector<int64_t> packets;
  bool has_obs = false;
  rt_observers obs;
  std::vector<double> obs_dir, obs_up;
  // accounting
  int64_t n_packets = 0;
  size_t acc_bytes = 0, img_bytes = 0;
  int bins = 1;
  int64_t n_cells = 0;
  // device results
  double* absorbed = nullptr;
  double* images = nullptr;
  // state
  enum { PENDING, ADMITTED, RUNNING, DONE, FAILED } state = PENDING;
  int rc = RT_OK;
  rt_ledger ledger;
  Clock::time_point t_submit, t_done;
  // device time of the launch the job ran in, ms after the server's
  // reference event (-1: not run)
  double dev_t0 = -1.0, dev_t1 = -1.0;
};

int64_t tree_cells(const rt_tree_desc& d) {
  int64_t n = (int64_t)d.root[0] * d.root[1] * d.root[2];
  for (int l = 0; l + 1 < d.n_levels; ++l) n += 8 * d.n_refined[l];
  return n;
}

}  // namespace

struct rt_server {
  rt_ctx* ctx = nullptr;        // builds grids
  int device = 0;
  rt_server_config cfg;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  size_t used = 0;              // resident grids + accumulators of admitted / finished jobs
  uint64_t next_ticket = 1;
  std::deque<Job*> pending;     // submitted, not yet admitted
  std::deque<Job*> admitted;    // admitted, waiting for a slot
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  std::map<uint64_t, ModelEntry> models;
  std::vector<std::thread> workers;
  std::vector<rt_ctx*> slot_ctx;
  std::vector<cudaStream_t> slot_stream;
  // results leave through this stream and job memory is released on it
  // (cudaFreeAsync): a plain cudaFree would wait for the whole device,
  // i.e. for the other slots' launches, and serialise them
  cudaStream_t io_stream = nullptr;
  std::mutex io_mu;
  // device-time bracket of each slot's launches, against one reference event
  cudaEvent_t ref_ev = nullptr;
  std::vector<cudaEvent_t> slot_ev0, slot_ev1;
  std::mutex build_mu;

  // evict idle resident grids (least recently used first) until `need` fits
  void make_room(size_t need) {
    while (used + need > cfg.hbm_budget) {
      ModelEntry* victim = nullptr;
      for (auto& kv : models) {
        ModelEntry& m = kv.second;
        if (m.grid && m.counted && m.users == 0 && (!victim || m.last_use < victim->last_use)) victim = &m;
      }
      if (!victim) return;
      rt_grid_free(victim->grid);
      victim->grid = nullptr;
      victim->counted = false;
      used -= victim->bytes;
    }
  }

  // move pending jobs to admitted, in arrival order, while they fit
  void admit() {
    while (!pending.empty()) {
      Job* j = pending.front();
      ModelEntry& m = models[j->model_id];
      const size_t need = j->acc_bytes + (m.counted ? 0 : m.bytes);
      if (used + need > cfg.hbm_budget) make_room(need);
      if (used + need > cfg.hbm_budget) return;
      used += need;
      m.counted = true;
      m.users += 1;
      m.last_use = Clock::now();
      j->state = Job::ADMITTED;
      pending.pop_front();
      admitted.push_back(j);
    }
  }

  void worker(int slot);
};

void rt_server::worker(int slot) {
  cudaSetDevice(device);
  rt_ctx* c = slot_ctx[slot];
  cudaStream_t s = slot_stream[slot];
  for (;;) {
    std::vector<Job*> batch;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return stop || !admitted.empty(); });
      if (stop && admitted.empty()) return;
      // a short window lets requests that arrive together share a launch
      if (cfg.batch_window_ms > 0 && (int)admitted.size() < cfg.max_batch_jobs) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds((long)(cfg.batch_window_ms * 1000)));
        lk.lock();
      }
      // the oldest admitted request, then the ones behind it that can share
      // its launch (one launch runs one precision and one estimator)
      int64_t pk = 0;
      for (auto it = admitted.begin(); it != admitted.end() && (int)batch.size() < cfg.max_batch_jobs;) {
        Job* nx = *it;
        if (!batch.empty()) {
          if (cfg.max_batch_packets > 0 && pk + nx->n_packets > cfg.max_batch_packets) break;
          if (nx->params.precision != batch[0]->params.precision ||
              nx->params.estimator != batch[0]->params.estimator) {
            ++it;
            continue;
          }
        }
        pk += nx->n_packets;
        batch.push_back(nx);
        it = admitted.erase(it);
      }
      for (Job* j : batch) j->state = Job::RUNNING;
    }
    if (batch.empty()) continue;
    // grids: build the ones that are not resident yet (one builder at a time)
    std::vector<rt_job> rj;
    std::vector<Job*> ok;
    for (Job* j : batch) {
      rt_grid* g = nullptr;
      {
        std::unique_lock<std::mutex> lk(build_mu);
        ModelEntry* m;
        {
          std::lock_guard<std::mutex> l2(mu);
          m = &models[j->model_id];
          g = m->grid;
        }
        if (!g) {
          const int rc = rt_build_grid(ctx, &m->tree, &g);
          std::lock_guard<std::mutex> l2(mu);
          if (rc != RT_OK) {
            j->rc = rc;
            j->state = Job::FAILED;
            continue;
          }
          m->grid = g;
        }
      }
      // accumulators
      const size_t ab = j->acc_bytes - j->img_bytes;
      cudaError_t e = cudaMallocAsync((void**)&j->absorbed, ab, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(j->absorbed, 0, ab, s);
      if (e == cudaSuccess && j->has_obs) {
        e = cudaMallocAsync((void**)&j->images, j->img_bytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(j->images, 0, j->img_bytes, s);
      }
      if (e != cudaSuccess) {
        std::lock_guard<std::mutex> l2(mu);
        j->rc = RT_ERR_OOM;
        j->state = Job::FAILED;
        continue;
      }
      rt_job x;
      memset(&x, 0, sizeof x);
      x.grid = g;
      x.n_src = (int)j->src.size();
      x.src = j->src.data();
      x.optics = &j->optics;
      x.params = &j->params;
      x.obs = j->has_obs ? &j->obs : nullptr;
      x.images_dev = j->images;
      x.absorbed_dev = j->absorbed;
      rj.push_back(x);
      ok.push_back(j);
    }
    int rc = RT_OK;
    std::vector<rt_ledger> leds(ok.size());
    double t0 = -1.0, t1 = -1.0;
    if (!ok.empty()) {
      cudaEventRecord(slot_ev0[slot], s);
      rc = rt_trace_batch(c, (int)ok.size(), rj.data(), leds.data(), s);
      cudaEventRecord(slot_ev1[slot], s);
      float a = 0.f, b = 0.f;
      if (cudaEventSynchronize(slot_ev1[slot]) == cudaSuccess &&
          cudaEventElapsedTime(&a, ref_ev, slot_ev0[slot]) == cudaSuccess &&
          cudaEventElapsedTime(&b, ref_ev, slot_ev1[slot]) == cudaSuccess) {
        t0 = a;
        t1 = b;
      }
    }
    const auto t = Clock::now();
    {
      std::lock_guard<std::mutex> lk(mu);
      for (size_t i = 0; i < ok.size(); ++i) {
        Job* j = ok[i];
        j->ledger = leds[i];
        j->dev_t0 = t0;
        j->dev_t1 = t1;
        j->rc = rc;
        j->state = (rc == RT_OK || rc == RT_ERR_STEP_LIMIT) ? Job::DONE : Job::FAILED;
        j->t_done = t;
      }
      for (Job* j : batch) {
        if (j->state == Job::FAILED && j->t_done == Clock::time_point()) j->t_done = t;
        ModelEntry& m = models[j->model_id];
        m.users -= 1;
        m.last_use = t;
      }
    }
    cv.notify_all();
  }
}

extern "C" int rt_server_create(rt_ctx* ctx, const rt_server_config* cfg, rt_server** out) {
  using namespace rtk;
  if (!ctx || !cfg || !out) return set_error(RT_ERR_INVALID, "rt_server_create: NULL argument");
  if (cfg->max_slots < 1 || cfg->max_slots > 16 || cfg->max_batch_jobs < 1 || cfg->hbm_budget == 0)
    return set_error(RT_ERR_INVALID, "rt_server_create: need 1..16 slots, a batch size and a budget");
  *out = nullptr;
  const int device = ctx_device(ctx);
  rt_server* S = new rt_server();
  S->ctx = ctx;
  S->cfg = *cfg;
  S->device = device;
  for (int i = 0; i < cfg->max_slots; ++i) {
    rt_ctx* c = nullptr;
    int rc = rt_ctx_create(device, &c);
    cudaStream_t st = nullptr;
    if (rc == RT_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = RT_ERR_CUDA;
    if (rc != RT_OK) {
      for (rt_ctx* x : S->slot_ctx) rt_ctx_destroy(x);
      delete S;
      return set_error(rc, "rt_server_create: slot setup failed");
    }
    S->slot_ctx.push_back(c);
    S->slot_stream.push_back(st);
  }
  if (cudaStreamCreateWithFlags(&S->io_stream, cudaStreamNonBlocking) != cudaSuccess) {
    for (size_t i = 0; i < S->slot_ctx.size(); ++i) {
      cudaStreamDestroy(S->slot_stream[i]);
      rt_ctx_destroy(S->slot_ctx[i]);
    }
    delete S;
    return set_error(RT_ERR_CUDA, "rt_server_create: stream creation failed");
  }
  bool ev_ok = cudaEventCreate(&S->ref_ev) == cudaSuccess && cudaEventRecord(S->ref_ev, S->io_stream) == cudaSuccess;
  S->slot_ev0.assign(cfg->max_slots, nullptr);
  S->slot_ev1.assign(cfg->max_slots, nullptr);
  for (int i = 0; i < cfg->max_slots && ev_ok; ++i)
    ev_ok = cudaEventCreate(&S->slot_ev0[i]) == cudaSuccess && cudaEventCreate(&S->slot_ev1[i]) == cudaSuccess;
  if (!ev_ok || cudaEventSynchronize(S->ref_ev) != cudaSuccess) {
    rt_server_destroy(S);
    return set_error(RT_ERR_CUDA, "rt_server_create: event creation failed");
  }
  // keep the memory of finished jobs in the device's stream-ordered pool for
  // the next ones instead of returning it at every synchronisation
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  for (int i = 0; i < cfg->max_slots; ++i) S->workers.emplace_back([S, i] { S->worker(i); });
  *out = S;
  return RT_OK;
}

extern "C" void rt_server_destroy(rt_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  cudaSetDevice(S->device);
  for (auto& kv : S->jobs) {
    if (kv.second->absorbed) cudaFree(kv.second->absorbed);
    if (kv.second->images) cudaFree(kv.second->images);
  }
  for (auto& kv : S->models)
    if (kv.second.grid) rt_grid_free(kv.second.grid);
  for (size_t i = 0; i < S->slot_ctx.size(); ++i) {
    cudaStreamDestroy(S->slot_stream[i]);
    rt_ctx_destroy(S->slot_ctx[i]);
  }
  if (S->io_stream) cudaStreamDestroy(S->io_stream);
  if (S->ref_ev) cudaEventDestroy(S->ref_ev);
  for (cudaEvent_t e : S->slot_ev0)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : S->slot_ev1)
    if (e) cudaEventDestroy(e);
  delete S;
}

extern "C" int rt_server_add_model(rt_server* S, uint64_t model_id, const rt_tree_desc* d) {
  using namespace rtk;
  if (!S || !d || d->n_levels < 1 || !d->n_refined || !d->refine_flags || !d->density || d->root[0] < 1 ||
      d->root[1] < 1 || d->root[2] < 1)
    return set_error(RT_ERR_INVALID, "rt_server_add_model: bad tree description");
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->models.count(model_id)) return set_error(RT_ERR_INVALID, "rt_server_add_model: model id already registered");
  ModelEntry& m = S->models[model_id];
  m.n_cells = tree_cells(*d);
  m.n_refined.assign(d->n_refined, d->n_refined + d->n_levels);
  m.flags.assign(d->refine_flags, d->refine_flags + m.n_cells);
  m.density.assign(d->density, d->density + m.n_cells);
  m.tree = *d;
  m.tree.n_refined = m.n_refined.data();
  m.tree.refine_flags = m.flags.data();
  m.tree.density = m.density.data();
  m.bytes = (size_t)m.n_cells * (sizeof(float) + 2 * sizeof(uint32_t) + sizeof(uint8_t) + sizeof(double) +
                                 sizeof(uint64_t));
  m.last_use = Clock::now();
  return RT_OK;
}

extern "C" int rt_server_submit(rt_server* S, const rt_serve_job* r, uint64_t* ticket) {
  using namespace rtk;
  if (!S || !r || !ticket || !r->optics || !r->params || !r->src || r->n_src < 1 || r->n_src > 256)
    return set_error(RT_ERR_INVALID, "rt_server_submit: bad argument");
  const int nl = r->optics->n_lambda;
  if (nl < 1 || nl > RT_MAX_LAMBDA) return set_error(RT_ERR_INVALID, "rt_server_submit: bad n_lambda");
  std::unique_ptr<Job> j(new Job());
  j->model_id = r->model_id;
  size_t grid_bytes = 0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->models.find(r->model_id);
    if (it == S->models.end()) return set_error(RT_ERR_INVALID, "rt_server_submit: unknown model id");
    j->n_cells = it->second.n_cells;
    grid_bytes = it->second.bytes;
  }
  j->kext.assign(r->optics->kappa_ext, r->optics->kappa_ext + nl);
  j->alb.assign(r->optics->albedo, r->optics->albedo + nl);
  j->g.assign(r->optics->g_hg, r->optics->g_hg + nl);
  j->optics.n_lambda = nl;
  j->optics.kappa_ext = j->kext.data();
  j->optics.albedo = j->alb.data();
  j->optics.g_hg = j->g.data();
  j->src.assign(r->src, r->src + r->n_src);
  j->src_energy.resize(r->n_src);
  for (int i = 0; i < r->n_src; ++i) {
    if (j->src[i].kind == RT_SRC_DUST) return set_error(RT_ERR_INVALID, "rt_server_submit: dust sources are not served");
    if (!r->src[i].bin_energy) return set_error(RT_ERR_INVALID, "rt_server_submit: bin_energy is NULL");
    j->src_energy[i].assign(r->src[i].bin_energy, r->src[i].bin_energy + nl);
    j->src[i].bin_energy = j->src_energy[i].data();
  }
  j->params = *r->params;
  j->params.packet_log_dev = nullptr;
  j->params.hits_dev = nullptr;
  if (r->params->packets && r->params->packets_per_bin <= 0 && r->params->packets_total <= 0) {
    j->packets.assign(r->params->packets, r->params->packets + (size_t)r->n_src * nl);
    j->params.packets = j->packets.data();
    for (int64_t v : j->packets) j->n_packets += v > 0 ? v : 0;
  } else {
    j->n_packets = r->params->packets_per_bin > 0 ? r->params->packets_per_bin * (int64_t)nl * r->n_src
                                                  : r->params->packets_total;
  }
  j->bins = r->params->per_lambda ? nl : 1;
  j->acc_bytes = sizeof(double) * (size_t)j->bins * (size_t)j->n_cells;
  if (r->obs) {
    if (r->obs->n_obs < 1 || !r->obs->dir || !r->obs->up) return set_error(RT_ERR_INVALID, "rt_server_submit: bad observers");
    j->has_obs = true;
    j->obs = *r->obs;
    j->obs_dir.assign(r->obs->dir, r->obs->dir + 3 * r->obs->n_obs);
    j->obs_up.assign(r->obs->up, r->obs->up + 3 * r->obs->n_obs);
    j->obs.dir = j->obs_dir.data();
    j->obs.up = j->obs_up.data();
    j->img_bytes = sizeof(double) * (size_t)r->obs->n_obs * j->bins * r->obs->nx * r->obs->ny;
    j->acc_bytes += j->img_bytes;
  }
  if (j->acc_bytes + grid_bytes > S->cfg.hbm_budget)
    return set_error(RT_ERR_BUSY, "rt_server_submit: the job alone exceeds the device-memory budget");
  j->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    j->ticket = S->next_ticket++;
    *ticket = j->ticket;
    S->pending.push_back(j.get());
    S->jobs[j->ticket] = std::move(j);
    S->admit();
  }
  S->cv.notify_all();
  return RT_OK;
}

extern "C" int rt_server_poll(rt_server* S, uint64_t ticket, int* done, rt_ledger* ledger, double* latency_ms) {
  using namespace rtk;
  if (!S || !done) return set_error(RT_ERR_INVALID, "rt_server_poll: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return set_error(RT_ERR_INVALID, "rt_server_poll: unknown ticket");
  Job* j = it->second.get();
  *done = (j->state == Job::DONE || j->state == Job::FAILED) ? 1 : 0;
  if (*done) {
    if (ledger) *ledger = j->ledger;
    if (latency_ms) *latency_ms = 1e3 * std::chrono::duration<double>(j->t_done - j->t_submit).count();
    if (j->state == Job::FAILED) return set_error(j->rc ? j->rc : RT_ERR_CUDA, "rt_server_poll: the job failed");
  }
  return RT_OK;
}

extern "C" int rt_server_job_times(rt_server* S, uint64_t ticket, double* t_start_ms, double* t_end_ms) {
  using namespace rtk;
  if (!S || !t_start_ms || !t_end_ms) return set_error(RT_ERR_INVALID, "rt_server_job_times: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return set_error(RT_ERR_INVALID, "rt_server_job_times: unknown ticket");
  *t_start_ms = it->second->dev_t0;
  *t_end_ms = it->second->dev_t1;
  return RT_OK;
}

extern "C" int rt_server_wait(rt_server* S, uint64_t ticket, double timeout_s) {
  using namespace rtk;
  if (!S) return set_error(RT_ERR_INVALID, "rt_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return set_error(RT_ERR_INVALID, "rt_server_wait: unknown ticket");
  Job* j = it->second.get();
  const bool ok = S->cv.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 3600.0),
                                 [&] { return j->state == Job::DONE || j->state == Job::FAILED; });
  if (!ok) return set_error(RT_ERR_TIMEOUT, "rt_server_wait: the job did not finish in time");
  return j->state == Job::DONE ? RT_OK : set_error(j->rc ? j->rc : RT_ERR_CUDA, "rt_server_wait: the job failed");
}

extern "C" int rt_server_fetch(rt_server* S, uint64_t ticket, double* absorbed_host, double* images_host) {
  using namespace rtk;
  if (!S) return set_error(RT_ERR_INVALID, "rt_server_fetch: NULL server");
  std::unique_ptr<Job> owned;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return set_error(RT_ERR_INVALID, "rt_server_fetch: unknown ticket");
    if (it->second->state != Job::DONE && it->second->state != Job::FAILED)
      return set_error(RT_ERR_BUSY, "rt_server_fetch: the job has not finished");
    owned = std::move(it->second);
    S->jobs.erase(it);
  }
  Job* j = owned.get();
  cudaSetDevice(S->device);
  int rc = RT_OK;
  {
    // the job's launch has finished (its slot waited for it before marking
    // it done): copy out and release its memory on the server's own stream
    std::lock_guard<std::mutex> lk(S->io_mu);
    cudaStream_t io = S->io_stream;
    if (j->state == Job::DONE) {
      if (absorbed_host && j->absorbed &&
          cudaMemcpyAsync(absorbed_host, j->absorbed, j->acc_bytes - j->img_bytes, cudaMemcpyDeviceToHost, io) !=
              cudaSuccess)
        rc = set_error(RT_ERR_CUDA, "rt_server_fetch: copy of absorbed energy failed");
      if (rc == RT_OK && images_host && j->images &&
          cudaMemcpyAsync(images_host, j->images, j->img_bytes, cudaMemcpyDeviceToHost, io) != cudaSuccess)
        rc = set_error(RT_ERR_CUDA, "rt_server_fetch: copy of images failed");
      if (rc == RT_OK && (absorbed_host || images_host) && cudaStreamSynchronize(io) != cudaSuccess)
        rc = set_error(RT_ERR_CUDA, "rt_server_fetch: copy failed");
    }
    if (j->absorbed) cudaFreeAsync(j->absorbed, io);
    if (j->images) cudaFreeAsync(j->images, io);
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= j->acc_bytes;
    S->admit();
  }
  S->cv.notify_all();
  return rc;
}

extern "C" int rt_server_stats(rt_server* S, size_t* used_bytes, int* pending, int* running) {
  using namespace rtk;
  if (!S) return set_error(RT_ERR_INVALID, "rt_server_stats: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (used_bytes) *used_bytes = S->used;
  if (pending) *pending = (int)(S->pending.size() + S->admitted.size());
  int r = 0;
  for (auto& kv : S->jobs) r += kv.second->state == Job::RUNNING;
  if (running) *running = r;
  return RT_OK;
}
