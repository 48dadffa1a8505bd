// Serving loop: continuous batching of many independent solves (a design sweep) on one GPU.
//
// One scheduler thread owns the device.  Submitted requests wait in arrival order; a request is
// admitted (first fit) as soon as its exact device footprint fits the HBM budget next to the
// solves already running and a slot is free.  Every admitted solve keeps its state and solver
// scratch on the device, runs on its own stream, and advances in chunks of steps replayed from a
// CUDA graph captured once for the solve; the chunks of different solves overlap on the GPU.
// When a solve finishes, its state is copied back, its memory released, and waiting requests are
// admitted in its place.  The first solve of each grid shape ("bucket") times the face kernels'
// launch shapes on a scratch copy of its state and the bucket keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "fluid_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket = 0;
  fluid_config cfg{};
  int nsteps = 0;
  double t_end = 0.0;
  double* U_out_host = nullptr;
  size_t nstate = 0;              // doubles in the padded state
  double* staging = nullptr;      // pinned host copy of the initial, later the final, state
  size_t bytes = 0;               // device footprint
  fluid_result res{};
  bool done = false;
};

struct Slot {
  std::shared_ptr<Job> job;
  fluid_solver* solver = nullptr;
  double* U = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  int steps_done = 0;
  bool copying_out = false;
};

struct BucketKey {
  int ndim, n0, n1, n2, precision, visc, weno, visc_order;
  bool operator<(const BucketKey& o) const {
    return std::tie(ndim, n0, n1, n2, precision, visc, weno, visc_order) <
           std::tie(o.ndim, o.n0, o.n1, o.n2, o.precision, o.visc, o.weno, o.visc_order);
  }
};

size_t footprint(const fluid_config& c) {
  size_t nc = 1, metric = 0;
  for (int a = 0; a < 3; ++a) {
    const size_t p = c.n[a] + (a < c.ndim ? 2 * FLUID_HALO : 0);
    nc *= p;
    metric += 5 * p;
  }
  const bool visc = c.visc_law != FLUID_VISC_NONE;
  size_t b = 8 * (nc * (fl::NW + 3 * fl::NV) + metric + 4096);   // W, A, R, the state U, metrics
  // mixed: the H row of W, the (hi, lo) FP32 primitives, FP32 gradients and face metrics
  if (c.precision == FLUID_PREC_MIXED) {
    b += 8 * nc + 4 * (nc * (2 * fl::NW + (visc ? fl::NG : 0)) + metric / 5);
  } else {
    if (visc) b += 8 * nc * fl::NG;
    // seam buffer of the face kernels: 10 doubles per segment of kSeamMinSeg cells, on the axis
    // with the most segments
    size_t cap = 0;
    for (int a = 0; a < c.ndim; ++a) {
      size_t lines = 1;
      for (int d = 0; d < 3; ++d)
        if (d != a) lines *= (size_t)c.n[d];
      cap = std::max(cap, lines * (((size_t)c.n[a] + fl::kSeamMinSeg - 1) / fl::kSeamMinSeg));
    }
    b += 8 * 10 * cap;
  }
  return b;
}

}  // namespace

struct fluid_server {
  fluid_serve_config cfg{};
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::deque<std::shared_ptr<Job>> pending;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  std::vector<Slot> active;                 // owned by the scheduler thread only
  std::atomic<int64_t> n_active{0};         // its size, for other threads
  std::map<BucketKey, std::pair<int, int>> tuned;   // bucket -> (block, seg)
  uint64_t next_ticket = 1;
  size_t used = 0, peak = 0;
  std::atomic<bool> stop{false};
  std::thread worker;
  std::string err;
  int64_t admitted = 0, completed = 0;
  double cell_updates = 0.0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  void finish(Slot& s, int status) {
    std::lock_guard<std::mutex> lk(mu);
    s.job->res.status = status;
    s.job->res.steps_done = s.steps_done;
    s.job->res.finish_s = now();
    s.job->done = true;
    used -= s.job->bytes;
    ++completed;
    cell_updates += (double)s.steps_done * s.job->cfg.n[0] * s.job->cfg.n[1] * s.job->cfg.n[2];
    cv_done.notify_all();
  }

  void release(Slot& s) {
    if (s.graph) cudaGraphExecDestroy(s.graph);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.stream) cudaStreamDestroy(s.stream);
    cudaFree(s.U);
    fluid_destroy(s.solver);
    s = Slot{};
  }

  // time the candidate launch shapes of the face kernels on a scratch copy of the state
  void autotune(Slot& s) {
    const fluid_config& c = s.job->cfg;
    const BucketKey key{c.ndim, c.n[0], c.n[1], c.n[2], c.precision, c.visc_law, c.weno,
                        c.visc_order == 6 ? 6 : 4};
    auto it = tuned.find(key);
    if (it == tuned.end()) {
      std::vector<std::pair<int, int>> cand = {{0, 0}, {32, 64}, {64, 16}, {128, 32}};
      // only shapes whose results are bitwise those of the default shape: every FP64 segment
      // length, and the mixed path's two tile sizes (its register-window kernels are compiled
      // separately and agree only to FP32 rounding)
      if (c.precision == FLUID_PREC_MIXED) cand = {{0, 0}, {64, 0}};
      double* tmp = nullptr;
      float best = 1e30f;
      std::pair<int, int> pick{0, 0};
      cudaEvent_t a, b;
      if (cudaMalloc(&tmp, s.job->nstate * sizeof(double)) == cudaSuccess &&
          cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
        for (auto& cs : cand) {
          if (fluid_tune_faces(s.solver, cs.first, cs.second) != FLUID_OK) continue;
          cudaMemcpyAsync(tmp, s.U, s.job->nstate * sizeof(double), cudaMemcpyDeviceToDevice, s.stream);
          fluid_step(s.solver, tmp, 1, 0.0, s.stream);          // warm-up
          cudaEventRecord(a, s.stream);
          fluid_step(s.solver, tmp, 2, 0.0, s.stream);
          cudaEventRecord(b, s.stream);
          cudaEventSynchronize(b);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, a, b);
          if (ms > 0.f && ms < best) {
            best = ms;
            pick = cs;
          }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        fluid_set_time(s.solver, 0.0, s.stream);
      }
      cudaFree(tmp);
      it = tuned.emplace(key, pick).first;
    }
    fluid_tune_faces(s.solver, it->second.first, it->second.second);
  }

  bool admit(const std::shared_ptr<Job>& j) {
    Slot s;
    s.job = j;
    if (fluid_create(&j->cfg, &s.solver) != FLUID_OK) {
      std::lock_guard<std::mutex> lk(mu);
      j->res.status = FLUID_EINVAL;
      j->res.finish_s = now();
      j->done = true;
      used -= j->bytes;
      cv_done.notify_all();
      return false;
    }
    if (cudaMalloc(&s.U, j->nstate * sizeof(double)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) {
      release(s);
      std::lock_guard<std::mutex> lk(mu);
      j->res.status = FLUID_ENOMEM;
      j->res.finish_s = now();
      j->done = true;
      used -= j->bytes;
      cv_done.notify_all();
      return false;
    }
    cudaMemcpyAsync(s.U, j->staging, j->nstate * sizeof(double), cudaMemcpyHostToDevice, s.stream);
    {
      std::lock_guard<std::mutex> lk(mu);
      j->res.start_s = now();
    }
    if (cfg.autotune) autotune(s);
    // one chunk captured as a graph, replayed until the last (possibly shorter) chunk
    const int chunk = std::max(1, std::min(cfg.chunk_steps, j->nsteps));
    if (cfg.use_graphs && j->nsteps >= chunk) {
      cudaGraph_t gr = nullptr;
      if (cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        const int st = fluid_step(s.solver, s.U, chunk, j->t_end, s.stream);
        if (cudaStreamEndCapture(s.stream, &gr) == cudaSuccess && st == FLUID_OK &&
            cudaGraphInstantiate(&s.graph, gr, 0) == cudaSuccess)
          s.graph_steps = chunk;
        if (gr) cudaGraphDestroy(gr);
      }
      cudaGetLastError();
    }
    active.push_back(s);
    n_active.store((int64_t)active.size());
    return true;
  }

  // enqueue the next chunk of a solve (returns false when it has no steps left)
  bool advance(Slot& s) {
    const int left = s.job->nsteps - s.steps_done;
    if (left <= 0) return false;
    int n;
    if (s.graph && left >= s.graph_steps) {
      cudaGraphLaunch(s.graph, s.stream);
      n = s.graph_steps;
    } else {
      n = std::min(left, std::max(1, cfg.chunk_steps));
      fluid_step(s.solver, s.U, n, s.job->t_end, s.stream);
    }
    s.steps_done += n;
    cudaEventRecord(s.ev, s.stream);
    return true;
  }

  void loop() {
    cudaSetDevice(device);
    while (!stop.load()) {
      bool busy = false;
      // admissions: first fit in arrival order under the budget and the slot limit
      for (;;) {
        std::shared_ptr<Job> j;
        {
          std::lock_guard<std::mutex> lk(mu);
          if ((int)active.size() >= cfg.max_active) break;   // active is only resized by this thread
          for (auto it = pending.begin(); it != pending.end(); ++it)
            if (used + (*it)->bytes <= cfg.hbm_budget_bytes) {
              j = *it;
              pending.erase(it);
              used += j->bytes;
              peak = std::max(peak, used);
              ++admitted;
              break;
            }
        }
        if (!j) break;
        if (admit(j)) advance(active.back());
        busy = true;
      }
      // progress of the running solves
      for (size_t i = 0; i < active.size();) {
        Slot& s = active[i];
        if (cudaEventQuery(s.ev) == cudaErrorNotReady) {
          ++i;
          continue;
        }
        busy = true;
        if (s.copying_out) {
          const int st = fluid_check(s.solver, s.stream);
          if (s.job->U_out_host)
            std::memcpy(s.job->U_out_host, s.job->staging, s.job->nstate * sizeof(double));
          double t = 0.0;
          fluid_get_time(s.solver, &t, nullptr, s.stream);
          s.job->res.t_final = t;
          finish(s, st);
          release(s);
          active.erase(active.begin() + i);
          n_active.store((int64_t)active.size());
          continue;
        }
        if (!advance(s)) {
          cudaMemcpyAsync(s.job->staging, s.U, s.job->nstate * sizeof(double), cudaMemcpyDeviceToHost, s.stream);
          cudaEventRecord(s.ev, s.stream);
          s.copying_out = true;
        }
        ++i;
      }
      if (!busy) {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait_for(lk, std::chrono::microseconds(200));
      }
    }
    for (Slot& s : active) {
      cudaStreamSynchronize(s.stream);
      finish(s, FLUID_EBUSY);
      release(s);
    }
    active.clear();
  }
};

extern "C" {

int fluid_serve_create(const fluid_serve_config* cfg, fluid_server** out) {
  if (!out || !cfg) return FLUID_EINVAL;
  *out = nullptr;
  if (cfg->struct_size != sizeof(fluid_serve_config) || cfg->max_active < 1 || cfg->chunk_steps < 1 ||
      cfg->hbm_budget_bytes == 0)
    return FLUID_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return FLUID_ECUDA;
  auto* s = new (std::nothrow) fluid_server();
  if (!s) return FLUID_ENOMEM;
  s->cfg = *cfg;
  s->device = cfg->device;
  s->t0 = Clock::now();
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return FLUID_OK;
}

void fluid_serve_destroy(fluid_server* s) {
  if (!s) return;
  s->stop.store(true);
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->jobs) cudaFreeHost(kv.second->staging);
  delete s;
}

int fluid_serve_submit(fluid_server* s, const fluid_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket || req->struct_size != sizeof(fluid_request)) return FLUID_EINVAL;
  if (!req->U0_host || req->nsteps < 0) return FLUID_EINVAL;
  if (fl::config_error(&req->cfg)) return FLUID_EINVAL;
  for (int a = 0; a < req->cfg.ndim; ++a)
    for (int sd = 0; sd < 2; ++sd)
      if (req->cfg.bc[a][sd] == FLUID_BC_EXCHANGE) return FLUID_EINVAL;   // one solve, one block
  auto j = std::make_shared<Job>();
  j->cfg = req->cfg;
  j->nsteps = req->nsteps;
  j->t_end = req->t_end;
  j->U_out_host = req->U_out_host;
  j->bytes = footprint(req->cfg);
  if (j->bytes > s->cfg.hbm_budget_bytes) return FLUID_EBUDGET;
  size_t nc = 1;
  for (int a = 0; a < 3; ++a) nc *= req->cfg.n[a] + (a < req->cfg.ndim ? 2 * FLUID_HALO : 0);
  j->nstate = fl::NV * nc;
  if (cudaMallocHost(&j->staging, j->nstate * sizeof(double)) != cudaSuccess) return FLUID_ENOMEM;
  std::memcpy(j->staging, req->U0_host, j->nstate * sizeof(double));
  std::lock_guard<std::mutex> lk(s->mu);
  j->ticket = s->next_ticket++;
  j->res.submit_s = s->now();
  s->jobs[j->ticket] = j;
  s->pending.push_back(j);
  *ticket = j->ticket;
  s->cv_work.notify_all();
  return FLUID_OK;
}

int fluid_serve_poll(fluid_server* s, uint64_t ticket, fluid_result* out, int timeout_ms) {
  if (!s || !out) return FLUID_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return FLUID_EINVAL;
  std::shared_ptr<Job> j = it->second;
  if (!j->done) {
    if (timeout_ms <= 0) return FLUID_ETIMEOUT;
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return j->done; });
    if (!j->done) return FLUID_ETIMEOUT;
  }
  *out = j->res;
  cudaFreeHost(j->staging);
  s->jobs.erase(it);
  return FLUID_OK;
}

int fluid_serve_stats(fluid_server* s, fluid_serve_stats_t* st) {
  if (!s || !st) return FLUID_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  st->pending = (int64_t)s->pending.size();
  st->active = s->n_active.load();
  st->admitted = s->admitted;
  st->completed = s->completed;
  st->bytes_in_use = s->used;
  st->peak_bytes = s->peak;
  st->cell_updates = s->cell_updates;
  st->elapsed_s = s->now();
  return FLUID_OK;
}

size_t fluid_serve_footprint(const fluid_config* cfg) { return cfg ? footprint(*cfg) : 0; }

}  // extern "C"
