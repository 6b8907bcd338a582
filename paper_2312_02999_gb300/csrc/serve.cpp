// Request server: continuous batching of frame solves (Algorithm 1) over
// the meshes of one context.
//
// Each worker is one host thread with its own CUDA stream and pinned
// read-back words.  A request runs on a workspace slot (a private copy of
// the per-solve buffers of its mesh, sharing the mesh's factor, Sigma^-1 and
// topology), so solves of different meshes, or several frames of the same
// mesh, run concurrently and their kernels overlap on the GPU.  A worker that
// finishes a request immediately takes the next admissible one from the
// queue (admission.h decides which, under the memory budget), so requests
// that arrive while others are on the GPU start as soon as a worker and
// memory are free.  Every request names its own start state (host positions
// or the rest pose) and actuation, so its result does not depend on what
// else is in flight.
//
// The single cooperative kernel of a solve (the reduced contact system) is
// launched with num_SMs / workers CTAs per worker, so the cooperative grids
// of all workers together need at most one CTA per SM and are always
// co-resident, whatever else runs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "admission.h"
#include "batch.h"
#include "runtime.h"

using namespace fsim;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Job {
  int64_t ticket = 0;
  int mesh_id = 0, precision = 0;
  std::vector<double> fiber, stretch, x_init;   // host requests
  bool has_x = false;
  bool device = false;                          // FSIM_REQ_DEVICE
  const double* fiber_dev = nullptr;
  const double* stretch_dev = nullptr;
  const double* x_init_dev = nullptr;
  double* x_out_dev = nullptr;
  std::vector<double> x_out;
  fsim_frame_stats st{};
  int status = FSIM_OK;
  Clock::time_point t_submit, t_start, t_end;
  bool started = false, done = false;
};

struct Slot {
  int mesh_id = -1;
  DevMesh d;
  std::vector<void*> allocs;
  size_t bytes = 0;
  bool busy = false;
  int64_t last_used = 0;
  double* h_x = nullptr;      // pinned staging: 3n positions
  double* h_act = nullptr;    // pinned staging: 3T fiber + T stretch
};

struct Worker {
  std::thread th;
  cudaStream_t stream = nullptr;
  int* h_counters = nullptr;
  double* h_scal = nullptr;
};

}  // namespace

struct fsim_server_s {
  fsim_ctx_t ctx = nullptr;
  int n_workers = 1;
  int batch_frames = 0;          // >= 2: workers run lock-step batches (batch.cu)
  int coop_ctas = 1;
  int64_t budget = 0;
  size_t used = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job*> queue;
  std::unordered_map<int64_t, std::unique_ptr<Job>> jobs;
  int64_t next_ticket = 1;
  int64_t clock = 0;
  std::vector<std::unique_ptr<Slot>> slots;
  std::vector<Worker> workers;
  bool stop = false;
  int64_t completed = 0;
  int peak_slots = 0;
  int peak_running = 0;
  int running = 0;
};

namespace {

void free_slot(Slot& s) {
  rt_destroy_graphs(s.d);
  rt_free_list(s.allocs);
  if (s.h_x) cudaFreeHost(s.h_x);
  if (s.h_act) cudaFreeHost(s.h_act);
  s.h_x = nullptr;
  s.h_act = nullptr;
}

size_t slot_need(const MeshState& ms) { return rt_slot_bytes(ms); }

int make_slot(fsim_server_s* sv, const MeshState& ms, int mesh_id, Slot& s) {
  s.mesh_id = mesh_id;
  s.d = ms.d;   // constant pointers shared, per-solve ones replaced below
  int rc = rt_alloc_workspace(ms, s.d, s.allocs, &s.bytes);
  if (rc != FSIM_OK) return rc;
  if (cudaHostAlloc((void**)&s.h_x, sizeof(double) * 3 * (size_t)ms.d.n, cudaHostAllocDefault) !=
          cudaSuccess ||
      cudaHostAlloc((void**)&s.h_act, sizeof(double) * 4 * (size_t)ms.d.T, cudaHostAllocDefault) !=
          cudaSuccess) {
    cudaGetLastError();
    return FSIM_ENOMEM;
  }
  (void)sv;
  return FSIM_OK;
}

// A running slot's reduced-system buffers grow under the server's lock and
// within the memory budget (admission.h); the growth is added to `used` at
// once, so that other workers admit new slots against the current total.
struct Growth {
  fsim_server_s* sv = nullptr;
  size_t grown = 0;
};

int grow_slot(void* user, size_t delta) {
  auto* g = static_cast<Growth*>(user);
  std::lock_guard<std::mutex> lk(g->sv->mu);
  if (!admit_growth(g->sv->used, delta, g->sv->budget)) return -1;
  g->sv->used += delta;
  g->grown += delta;
  return 0;
}

int run_job(fsim_server_s* sv, Worker& w, Slot& s, Job& J, Growth* growth) {
  const MeshState& ms = *rt_mesh(sv->ctx, J.mesh_id);
  DevMesh& m = s.d;
  cudaStream_t st = w.stream;
  const size_t n = (size_t)m.n, T = (size_t)m.T;
  Exec ex;
  ex.stream = st;
  ex.h_counters = w.h_counters;
  ex.h_scal = w.h_scal;
  ex.coop_ctas = sv->coop_ctas;
  ex.alone = sv->n_workers == 1;
  ex.allocs = &s.allocs;
  ex.bytes = &s.bytes;
  ex.grow = grow_slot;
  ex.grow_user = growth;
  // actuation A = a f f^T + a^-1/2 (I - f f^T) per tet; host arrays go
  // through the slot's pinned staging (fiber into tetf, stretch after it)
  const double* x0 = ms.d.rest;
  bool x0_dev = true;
  if (J.device) {
    launch_actuation(st, m.T, J.fiber_dev, J.stretch_dev, m.act, m.act_df);
    if (J.x_init_dev) x0 = J.x_init_dev;
  } else {
    std::memcpy(s.h_act, J.fiber.data(), sizeof(double) * 3 * T);
    std::memcpy(s.h_act + 3 * T, J.stretch.data(), sizeof(double) * T);
    if (cudaMemcpyAsync(m.tetf, s.h_act, sizeof(double) * 4 * T, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return FSIM_ECUDA;
    launch_actuation(st, m.T, m.tetf, m.tetf + 3 * T, m.act, m.act_df);
    if (J.has_x) {
      std::memcpy(s.h_x, J.x_init.data(), sizeof(double) * 3 * n);
      x0 = s.h_x;
      x0_dev = false;
    }
  }
  int rc = rt_solve_frame(ex, ms, m, x0, x0_dev, J.precision, &J.st);
  if (J.x_out_dev &&
      cudaMemcpyAsync(J.x_out_dev, m.x, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return FSIM_ECUDA;
  if (!J.device &&
      cudaMemcpyAsync(s.h_x, m.x, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return FSIM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FSIM_ECUDA;
  if (!J.device) J.x_out.assign(s.h_x, s.h_x + 3 * n);
  return rc;
}

void worker_main(fsim_server_s* sv, int wi) {
  cudaSetDevice(sv->ctx->device);
  Worker& w = sv->workers[wi];
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    Admission a;
    while (!sv->stop) {
      std::vector<int> qm;
      qm.reserve(sv->queue.size());
      for (Job* j : sv->queue) qm.push_back(j->mesh_id);
      std::vector<SlotView> views(sv->slots.size());
      for (size_t k = 0; k < sv->slots.size(); ++k)
        views[k] = {sv->slots[k]->mesh_id, sv->slots[k]->busy, sv->slots[k]->bytes,
                    sv->slots[k]->last_used};
      std::vector<size_t> need(sv->ctx->meshes.size());
      for (size_t i = 0; i < need.size(); ++i) need[i] = slot_need(*sv->ctx->meshes[i]);
      a = admit(qm, views, need, sv->used, sv->budget, 4 * sv->n_workers);
      if (a.job >= 0) break;
      sv->cv.wait(lk);
    }
    if (sv->stop) return;
    Job* J = sv->queue[a.job];
    sv->queue.erase(sv->queue.begin() + a.job);
    J->started = true;
    J->t_start = Clock::now();
    // evict (highest index first so the remaining indices stay valid)
    std::vector<std::unique_ptr<Slot>> evicted;
    std::vector<int> ev = a.evict;
    std::sort(ev.rbegin(), ev.rend());
    for (int k : ev) {
      sv->used -= sv->slots[k]->bytes;
      evicted.push_back(std::move(sv->slots[k]));
      sv->slots.erase(sv->slots.begin() + k);
      if (a.slot > k) --a.slot;
    }
    Slot* s = nullptr;
    bool fresh = false;
    size_t bytes0 = 0;
    if (a.slot >= 0) {
      s = sv->slots[a.slot].get();
      bytes0 = s->bytes;
    } else {
      sv->slots.push_back(std::make_unique<Slot>());
      s = sv->slots.back().get();
      s->mesh_id = J->mesh_id;
      fresh = true;
      // reserve the expected size now so that other workers see it
      bytes0 = slot_need(*sv->ctx->meshes[J->mesh_id]);
      sv->used += bytes0;
    }
    s->busy = true;
    sv->running++;
    sv->peak_running = std::max(sv->peak_running, sv->running);
    sv->peak_slots = std::max(sv->peak_slots, (int)sv->slots.size());
    lk.unlock();
    for (auto& e : evicted) free_slot(*e);
    evicted.clear();
    int rc = FSIM_OK;
    Growth growth;
    growth.sv = sv;
    if (fresh) rc = make_slot(sv, *rt_mesh(sv->ctx, J->mesh_id), J->mesh_id, *s);
    if (rc == FSIM_OK) rc = run_job(sv, w, *s, *J, &growth);
    lk.lock();
    // bytes0 (and any growth) were counted while the job ran; now the
    // slot's actual size replaces them
    sv->used = sv->used - std::min(sv->used, bytes0 + growth.grown) + s->bytes;
    s->busy = false;
    s->last_used = ++sv->clock;
    sv->running--;
    if (rc == FSIM_ECUDA || (fresh && rc == FSIM_ENOMEM)) {
      // a failed slot is not reused
      sv->used -= s->bytes;
      for (size_t k = 0; k < sv->slots.size(); ++k)
        if (sv->slots[k].get() == s) {
          std::unique_ptr<Slot> dead = std::move(sv->slots[k]);
          sv->slots.erase(sv->slots.begin() + k);
          lk.unlock();
          free_slot(*dead);
          lk.lock();
          break;
        }
    }
    J->status = rc;
    J->st.status = rc;
    J->t_end = Clock::now();
    J->done = true;
    sv->completed++;
    sv->cv.notify_all();
  }
}

// Batch worker: serves the queue with lock-step batches of up to
// batch_frames frames of one mesh (continuous batching at iteration
// granularity: at every iteration boundary the batch takes the oldest queued
// requests of its mesh into the slots of finished frames).  A worker keeps
// its batch while requests for that mesh arrive and rebuilds it for another
// mesh when its own mesh has none queued.
void batch_worker_main(fsim_server_s* sv, int wi) {
  cudaSetDevice(sv->ctx->device);
  Worker& w = sv->workers[wi];
  Batch* b = nullptr;
  int b_mesh = -1;
  size_t b_bytes = 0;
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    while (!sv->stop && sv->queue.empty()) sv->cv.wait(lk);
    if (sv->stop) break;
    // the mesh of the oldest request; keep the current batch if it has work
    int mesh = sv->queue.front()->mesh_id;
    for (Job* j : sv->queue)
      if (j->mesh_id == b_mesh) { mesh = b_mesh; break; }
    if (mesh != b_mesh || b == nullptr) {
      if (b) {
        lk.unlock();
        batch_destroy(b);
        lk.lock();
        sv->used -= std::min(sv->used, b_bytes);
        b = nullptr;
        b_bytes = 0;
        b_mesh = -1;
      }
      MeshState& ms = *rt_mesh(sv->ctx, mesh);
      const size_t per = slot_need(ms);
      int cap = sv->batch_frames;
      if (sv->budget > 0) {
        const size_t room = (size_t)sv->budget > sv->used ? (size_t)sv->budget - sv->used : 0;
        cap = std::min<int>(cap, (int)(room / std::max<size_t>(per, 1)));
      }
      int rc = cap >= 1 ? FSIM_OK : FSIM_ENOMEM;
      if (rc == FSIM_OK) {
        sv->used += (size_t)cap * per;          // reserved while the batch is built
        lk.unlock();
        b = batch_create(sv->ctx, ms, cap, w.stream, &rc);
        lk.lock();
        sv->used -= std::min(sv->used, (size_t)cap * per);
        if (b) {
          b_bytes = batch_bytes(b);
          sv->used += b_bytes;
          b_mesh = mesh;
        }
      }
      if (!b) {     // the oldest request of this mesh cannot be served
        for (size_t k = 0; k < sv->queue.size(); ++k) {
          Job* J = sv->queue[k];
          if (J->mesh_id != mesh) continue;
          sv->queue.erase(sv->queue.begin() + k);
          J->started = true;
          J->t_start = J->t_end = Clock::now();
          J->status = J->st.status = rc;
          J->done = true;
          sv->completed++;
          break;
        }
        sv->cv.notify_all();
        continue;
      }
    }
    sv->running++;
    sv->peak_running = std::max(sv->peak_running, sv->running);
    const int64_t n = rt_mesh(sv->ctx, b_mesh)->d.n;
    const BatchPull pull = [&](BatchReq* out) {
      std::lock_guard<std::mutex> g(sv->mu);
      for (size_t k = 0; k < sv->queue.size(); ++k) {
        Job* J = sv->queue[k];
        if (J->mesh_id != b_mesh) continue;
        sv->queue.erase(sv->queue.begin() + k);
        J->started = true;
        J->t_start = Clock::now();
        fsim_request q{};
        q.mesh_id = J->mesh_id;
        q.precision = J->precision;
        q.x_out_dev = J->x_out_dev;
        if (J->device) {
          q.fiber = J->fiber_dev;
          q.stretch = J->stretch_dev;
          q.x_init = J->x_init_dev;
          q.flags = FSIM_REQ_DEVICE;
          out->x_host = nullptr;
        } else {
          q.fiber = J->fiber.data();
          q.stretch = J->stretch.data();
          q.x_init = J->has_x ? J->x_init.data() : nullptr;
          J->x_out.resize(3 * (size_t)n);
          out->x_host = J->x_out.data();
        }
        out->req = q;
        out->user = J;
        return true;
      }
      return false;
    };
    const BatchDone done = [&](void* user, int rc, const fsim_frame_stats& st) {
      std::lock_guard<std::mutex> g(sv->mu);
      Job* J = static_cast<Job*>(user);
      J->st = st;
      J->status = J->st.status = rc;
      J->t_end = Clock::now();
      J->done = true;
      sv->completed++;
      sv->cv.notify_all();
    };
    lk.unlock();
    const int rc = batch_run(b, pull, done);
    lk.lock();
    sv->running--;
    if (rc == FSIM_ECUDA) {      // a failed batch is not reused
      lk.unlock();
      batch_destroy(b);
      lk.lock();
      sv->used -= std::min(sv->used, b_bytes);
      b = nullptr;
      b_mesh = -1;
      b_bytes = 0;
    }
  }
  lk.unlock();
  if (b) batch_destroy(b);
  lk.lock();
  sv->used -= std::min(sv->used, b_bytes);
}

bool actuation_ok(const double* fiber, const double* stretch, int64_t T) {
  for (int64_t t = 0; t < T; ++t) {
    const double a = stretch[t];
    const double f2 = fiber[3 * t] * fiber[3 * t] + fiber[3 * t + 1] * fiber[3 * t + 1] +
                      fiber[3 * t + 2] * fiber[3 * t + 2];
    if (!(a > 0.0) || !std::isfinite(a) || !(f2 > 0.0) || !std::isfinite(f2)) return false;
  }
  return true;
}

}  // namespace

extern "C" {

fsim_status fsim_server_create(fsim_ctx_t ctx, const fsim_server_config* cfg, fsim_server_t* out) {
  if (!ctx || !cfg || !out || cfg->workers < 1 || cfg->workers > 16 || cfg->batch_frames < 0 ||
      cfg->batch_frames > 64)
    return FSIM_EINVAL;
  *out = nullptr;
  cudaSetDevice(ctx->device);
  auto* sv = new (std::nothrow) fsim_server_s();
  if (!sv) return FSIM_ENOMEM;
  sv->ctx = ctx;
  sv->n_workers = cfg->workers;
  sv->batch_frames = cfg->batch_frames;
  sv->coop_ctas = std::max(1, ctx->num_sms / cfg->workers);
  sv->budget = cfg->mem_budget_bytes;
  sv->workers.resize(cfg->workers);
  int prio_lo = 0, prio_hi = 0;     // worker streams above the side streams
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  for (auto& w : sv->workers) {
    if (cudaStreamCreateWithPriority(&w.stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaHostAlloc((void**)&w.h_counters, sizeof(int) * kCounters, cudaHostAllocDefault) !=
            cudaSuccess ||
        cudaHostAlloc((void**)&w.h_scal, sizeof(double) * kScal, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      for (auto& x : sv->workers) {
        if (x.stream) cudaStreamDestroy(x.stream);
        if (x.h_counters) cudaFreeHost(x.h_counters);
        if (x.h_scal) cudaFreeHost(x.h_scal);
      }
      delete sv;
      return FSIM_ENOMEM;
    }
  }
  for (int i = 0; i < cfg->workers; ++i)
    sv->workers[i].th = std::thread(sv->batch_frames >= 2 ? batch_worker_main : worker_main, sv, i);
  *out = sv;
  return FSIM_OK;
}

fsim_status fsim_server_submit(fsim_server_t sv, const fsim_request* req, int64_t* ticket) {
  if (!sv || !req || !ticket) return FSIM_EINVAL;
  MeshState* ms = rt_mesh(sv->ctx, req->mesh_id);
  if (!ms) return FSIM_EINVAL;
  if (!ms->prefactored) return FSIM_ENOT_READY;
  if (req->precision != FSIM_FP64 && req->precision != FSIM_MIXED) return FSIM_EINVAL;
  if (!req->fiber || !req->stretch || (req->flags & ~FSIM_REQ_DEVICE)) return FSIM_EINVAL;
  // a request whose workspace alone exceeds the budget could never start
  if (sv->budget > 0 && slot_need(*ms) > (size_t)sv->budget) return FSIM_ENOMEM;
  // a batch server serves what the lock-step batches can (mixed precision,
  // Woodbury global step)
  if (sv->batch_frames >= 2 && !batch_servable(*ms, *req)) return FSIM_EINVAL;
  const int64_t T = ms->d.T, n = ms->d.n;
  auto J = std::make_unique<Job>();
  J->mesh_id = req->mesh_id;
  J->precision = req->precision;
  J->x_out_dev = req->x_out_dev;
  if (req->flags & FSIM_REQ_DEVICE) {
    J->device = true;
    J->fiber_dev = req->fiber;
    J->stretch_dev = req->stretch;
    J->x_init_dev = req->x_init;
  } else {
    if (!actuation_ok(req->fiber, req->stretch, T)) return FSIM_ENONFINITE;
    J->fiber.assign(req->fiber, req->fiber + 3 * T);
    J->stretch.assign(req->stretch, req->stretch + T);
    if (req->x_init) {
      J->has_x = true;
      J->x_init.assign(req->x_init, req->x_init + 3 * n);
    }
  }
  J->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(sv->mu);
  J->ticket = sv->next_ticket++;
  *ticket = J->ticket;
  sv->queue.push_back(J.get());
  sv->jobs[J->ticket] = std::move(J);
  sv->cv.notify_all();
  return FSIM_OK;
}

fsim_status fsim_server_poll(fsim_server_t sv, int64_t ticket, int32_t* done) {
  if (!sv || !done) return FSIM_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return FSIM_EINVAL;
  *done = it->second->done ? 1 : 0;
  return FSIM_OK;
}

fsim_status fsim_server_wait(fsim_server_t sv, int64_t ticket, double* x_out,
                             fsim_frame_stats* stats, double* latency_ms, double* queue_ms) {
  if (!sv) return FSIM_EINVAL;
  std::unique_ptr<Job> J;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return FSIM_EINVAL;
    Job* j = it->second.get();
    sv->cv.wait(lk, [&] { return j->done || sv->stop; });
    if (!j->done) return FSIM_EINVAL;
    J = std::move(it->second);
    sv->jobs.erase(it);
  }
  if (x_out && !J->x_out.empty()) std::memcpy(x_out, J->x_out.data(), sizeof(double) * J->x_out.size());
  if (stats) *stats = J->st;
  if (latency_ms) *latency_ms = ms_between(J->t_submit, J->t_end);
  if (queue_ms) *queue_ms = ms_between(J->t_submit, J->t_start);
  return J->status;
}

fsim_status fsim_server_info_get(fsim_server_t sv, fsim_server_info* info) {
  if (!sv || !info) return FSIM_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  info->workers = sv->n_workers;
  info->slots = (int32_t)sv->slots.size();
  info->peak_slots = sv->peak_slots;
  info->peak_running = sv->peak_running;
  info->queued = (int64_t)sv->queue.size();
  info->completed = sv->completed;
  info->bytes_in_use = (int64_t)sv->used;
  return FSIM_OK;
}

fsim_status fsim_server_destroy(fsim_server_t sv) {
  if (!sv) return FSIM_EINVAL;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv.notify_all();
  }
  for (auto& w : sv->workers)
    if (w.th.joinable()) w.th.join();
  cudaSetDevice(sv->ctx->device);
  for (auto& w : sv->workers) {
    cudaStreamSynchronize(w.stream);
    cudaStreamDestroy(w.stream);
    cudaFreeHost(w.h_counters);
    cudaFreeHost(w.h_scal);
  }
  for (auto& s : sv->slots) free_slot(*s);
  delete sv;
  return FSIM_OK;
}

fsim_status fsim_solve_frames(fsim_ctx_t ctx, int32_t n_req, const fsim_request* reqs,
                              int32_t workers, double* const* x_out, fsim_frame_stats* stats) {
  if (!ctx || n_req < 0 || (n_req > 0 && !reqs)) return FSIM_EINVAL;
  fsim_server_config cfg{};
  cfg.workers = workers;
  cfg.mem_budget_bytes = 0;
  fsim_server_t sv = nullptr;
  int rc = fsim_server_create(ctx, &cfg, &sv);
  if (rc != FSIM_OK) return rc;
  std::vector<int64_t> t(n_req, -1);
  int first_err = FSIM_OK;
  for (int i = 0; i < n_req; ++i) {
    rc = fsim_server_submit(sv, &reqs[i], &t[i]);
    if (rc != FSIM_OK) {
      if (stats) { stats[i] = fsim_frame_stats{}; stats[i].status = rc; }
      if (first_err == FSIM_OK) first_err = rc;
    }
  }
  for (int i = 0; i < n_req; ++i) {
    if (t[i] < 0) continue;
    rc = fsim_server_wait(sv, t[i], x_out ? x_out[i] : nullptr, stats ? &stats[i] : nullptr, nullptr,
                          nullptr);
    if (rc != FSIM_OK && first_err == FSIM_OK) first_err = rc;
  }
  fsim_server_destroy(sv);
  return first_err;
}

}  // extern "C"
