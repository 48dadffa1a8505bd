// Serving loop: continuous batching of many independent solves (a design sweep) on one GPU.
//
// One scheduler thread owns the device.  Submitted requests wait in arrival order; a request is
// admitted (first fit) as soon as its exact device footprint fits the HBM budget next to the
// solves already running and a slot is free.  Every admitted solve keeps its state and solver
// scratch on the device.
//
// Batched solves (WENO5 with fourth-order or no dissipative stencils, with cfg.batch) join the
// bucket of their precision, reconstruction and viscous flag -- any grid size, 2-D with 3-D.  A
// bucket advances chunk by chunk: every kernel of a chunk is one launch over all its solves (the
// launches read a table of the solves in device memory and their blocks walk every solve's own
// launch grid, see BatchTable), and the chunk is a CUDA graph captured once per bucket.  Between
// chunks the scheduler rewrites the table: solves admitted meanwhile join, finished ones leave
// (their state is copied back and their memory released).  Each solve runs as many steps of a
// chunk as it has left and idles for the rest.
//
// Other solves run alone: their own stream, chunks replayed from a graph captured once per solve,
// and the first solve of each grid shape times the face kernels' launch shapes on a scratch copy of
// its state (the shape is kept for that shape).  Buckets and single solves overlap on the GPU.
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

// a solve of a bucket
struct BSlot {
  std::shared_ptr<Job> job;
  fluid_solver* solver = nullptr;
  double* U = nullptr;
  cudaStream_t stream = nullptr;  // the bucket's (its memory is ordered on it)
  cudaEvent_t ev_out = nullptr;   // its copy-out, once it has finished
  int steps_done = 0;
  int chunk_steps = 0;            // steps of the chunk in flight
  bool leaving = false;
};

// solves advanced together by batched launches
struct Bucket {
  int mixed = 0, weno = 0, visc = 0;
  std::vector<BSlot> slots;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;                 // end of the chunk in flight
  fl::BatchTable* host = nullptr;           // pinned
  fl::BatchTable* dev = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_chunk = 0;
  bool busy = false;
  bool broken = false;                      // set-up failed: no new solves join
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
  // mixed: the H row of W, the (hi, lo) FP32 primitives, FP32 gradients, the FP32 metric copies, and the
  // second pair of primitive buffers (W with its H row, W32)
  if (c.precision == FLUID_PREC_MIXED) {
    b += 8 * nc + 4 * (nc * (2 * fl::NW + (visc ? fl::NG : 0)) + 3 * (metric / 5));
    b += 8 * nc * (fl::NW + 1) + 4 * nc * 2 * fl::NW;
    b += 2 * 64 * 4;                                    // the W32 buffers' slack for staged rows
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
  std::vector<Slot> active;                 // solves running alone (scheduler thread only)
  std::vector<std::unique_ptr<Bucket>> buckets;   // batched solves (scheduler thread only)
  std::atomic<int64_t> n_active{0};         // running solves, for other threads
  std::map<BucketKey, std::pair<int, int>> tuned;   // bucket -> (block, seg)
  uint64_t next_ticket = 1;
  size_t used = 0, peak = 0;
  std::atomic<bool> stop{false};
  std::thread worker;
  std::string err;
  int64_t admitted = 0, completed = 0;
  double cell_updates = 0.0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  void finish(Job& job, int steps_done, int status) {
    std::lock_guard<std::mutex> lk(mu);
    job.res.status = status;
    job.res.steps_done = steps_done;
    job.res.finish_s = now();
    job.done = true;
    used -= job.bytes;
    ++completed;
    cell_updates += (double)steps_done * job.cfg.n[0] * job.cfg.n[1] * job.cfg.n[2];
    cv_done.notify_all();
  }
  void finish(Slot& s, int status) { finish(*s.job, s.steps_done, status); }

  int64_t running() const {
    int64_t n = (int64_t)active.size();
    for (auto& b : buckets) n += (int64_t)b->slots.size();
    return n;
  }

  void fail_job(const std::shared_ptr<Job>& j, int status) {
    std::lock_guard<std::mutex> lk(mu);
    j->res.status = status;
    j->res.finish_s = now();
    j->done = true;
    used -= j->bytes;
    cv_done.notify_all();
  }

  // ---- batched solves ----------------------------------------------------------------------
  static bool batchable(const fluid_config& c) {
    return (c.weno == FLUID_WENO_JS || c.weno == FLUID_WENO_Z) && c.visc_order != 6;
  }

  Bucket* bucket_for(const fluid_config& c) {
    const int mixed = c.precision == FLUID_PREC_MIXED, visc = c.visc_law != FLUID_VISC_NONE;
    for (auto& b : buckets)
      if (b->mixed == mixed && b->weno == c.weno && b->visc == visc && !b->broken &&
          (int)b->slots.size() < fl::kBatchMax)
        return b.get();
    auto b = std::make_unique<Bucket>();
    b->mixed = mixed;
    b->weno = c.weno;
    b->visc = visc;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&b->host, sizeof(fl::BatchTable)) != cudaSuccess ||
        cudaMalloc(&b->dev, sizeof(fl::BatchTable)) != cudaSuccess) {
      drop_bucket(*b);
      cudaGetLastError();
      return nullptr;
    }
    std::memset(b->host, 0, sizeof(fl::BatchTable));
    // an empty table, and one uncaptured chunk over it (no work: the launches' one-time set-up
    // happens outside any capture)
    cudaMemcpyAsync(b->dev, b->host, sizeof(fl::BatchTable), cudaMemcpyHostToDevice, b->stream);
    if (fl::launch_batch_chunk(b->dev, 1, mixed, c.weno, visc, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
      drop_bucket(*b);
      cudaGetLastError();
      return nullptr;
    }
    buckets.push_back(std::move(b));
    return buckets.back().get();
  }

  void drop_bucket(Bucket& b) {
    if (b.stream) cudaStreamSynchronize(b.stream);
    if (b.graph) cudaGraphExecDestroy(b.graph);
    if (b.ev) cudaEventDestroy(b.ev);
    if (b.stream) cudaStreamDestroy(b.stream);
    cudaFreeHost(b.host);
    cudaFree(b.dev);
    b.graph = nullptr;
    b.ev = nullptr;
    b.stream = nullptr;
    b.host = nullptr;
    b.dev = nullptr;
  }

  void release(BSlot& s) {
    if (s.ev_out) cudaEventDestroy(s.ev_out);
    if (s.U) cudaFreeAsync(s.U, s.stream);
    fluid_destroy(s.solver);            // stream-ordered: frees after the solve's work
    s = BSlot{};
  }

  bool admit_batched(const std::shared_ptr<Job>& j) {
    Bucket* b = bucket_for(j->cfg);
    if (!b) return false;                     // runs alone instead
    BSlot s;
    s.job = j;
    // stream-ordered memory on the bucket's stream: admission does not wait for the device
    if (fl::solver_create_async(&j->cfg, b->stream, &s.solver) != FLUID_OK) {
      fail_job(j, FLUID_EINVAL);
      return true;
    }
    s.stream = b->stream;
    if (cudaMallocAsync((void**)&s.U, j->nstate * sizeof(double), b->stream) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev_out, cudaEventDisableTiming) != cudaSuccess) {
      release(s);
      fail_job(j, FLUID_ENOMEM);
      return true;
    }
    // ordered before the bucket's next chunk on its stream
    cudaMemcpyAsync(s.U, j->staging, j->nstate * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    {
      std::lock_guard<std::mutex> lk(mu);
      j->res.start_s = now();
    }
    b->slots.push_back(s);
    return true;
  }

  // one bucket: collect the finished chunk, retire solves, start the next chunk
  bool step_bucket(Bucket& b) {
    bool busy = false;
    if (b.busy) {
      if (cudaEventQuery(b.ev) == cudaErrorNotReady) return false;
      b.busy = false;
      busy = true;
      for (BSlot& s : b.slots) {
        s.steps_done += s.chunk_steps;
        s.chunk_steps = 0;
      }
    }
    // finished solves (also those admitted with no step to run) copy their state out
    for (BSlot& s : b.slots)
      if (!s.leaving && s.steps_done >= s.job->nsteps) {
        cudaMemcpyAsync(s.job->staging, s.U, s.job->nstate * sizeof(double), cudaMemcpyDeviceToHost, b.stream);
        cudaEventRecord(s.ev_out, b.stream);
        s.leaving = true;
        busy = true;
      }
    // solves whose copy-out has completed leave the bucket
    for (size_t i = 0; i < b.slots.size();) {
      BSlot& s = b.slots[i];
      if (!s.leaving || cudaEventQuery(s.ev_out) == cudaErrorNotReady) {
        ++i;
        continue;
      }
      const int st = fluid_check(s.solver, nullptr);
      if (s.job->U_out_host) std::memcpy(s.job->U_out_host, s.job->staging, s.job->nstate * sizeof(double));
      double t = 0.0;
      fluid_get_time(s.solver, &t, nullptr, nullptr);
      s.job->res.t_final = t;
      finish(*s.job, s.steps_done, st);
      release(s);
      b.slots.erase(b.slots.begin() + i);
      busy = true;
    }
    if (b.busy) return busy;
    // the next chunk over every solve with steps left
    const int chunk = std::max(1, cfg.chunk_steps);
    fl::BatchTable& t = *b.host;
    t.nslots = 0;
    for (BSlot& s : b.slots) {
      const int left = s.job->nsteps - s.steps_done;
      if (s.leaving || left <= 0) continue;
      fl::BatchSlot& d = t.slot[t.nslots];
      if (!fl::batch_slot_of(s.solver, s.U, s.job->t_end, d)) continue;
      d.steps = std::min(chunk, left);
      s.chunk_steps = d.steps;
      ++t.nslots;
    }
    if (t.nslots == 0) return busy;
    fl::batch_plan(t, b.mixed);
    cudaMemcpyAsync(b.dev, b.host, sizeof(fl::BatchTable), cudaMemcpyHostToDevice, b.stream);
    if (cfg.use_graphs && !b.graph) {
      cudaGraph_t gr = nullptr;
      if (cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        const cudaError_t e = fl::launch_batch_chunk(b.dev, chunk, b.mixed, b.weno, b.visc, b.stream);
        if (cudaStreamEndCapture(b.stream, &gr) == cudaSuccess && e == cudaSuccess &&
            cudaGraphInstantiate(&b.graph, gr, 0) == cudaSuccess)
          b.graph_chunk = chunk;
        if (gr) cudaGraphDestroy(gr);
      }
      cudaGetLastError();
    }
    if (b.graph) cudaGraphLaunch(b.graph, b.stream);
    else fl::launch_batch_chunk(b.dev, chunk, b.mixed, b.weno, b.visc, b.stream);
    cudaEventRecord(b.ev, b.stream);
    b.busy = true;
    return true;
  }

  void release(Slot& s) {
    if (s.graph) cudaGraphExecDestroy(s.graph);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.U) cudaFreeAsync(s.U, s.stream);
    fluid_destroy(s.solver);            // stream-ordered on s.stream
    if (s.stream) cudaStreamDestroy(s.stream);
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
      if (cudaMallocAsync((void**)&tmp, s.job->nstate * sizeof(double), s.stream) == cudaSuccess &&
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
      if (tmp) cudaFreeAsync(tmp, s.stream);
      it = tuned.emplace(key, pick).first;
    }
    fluid_tune_faces(s.solver, it->second.first, it->second.second);
  }

  bool admit(const std::shared_ptr<Job>& j) {
    Slot s;
    s.job = j;
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) {
      fail_job(j, FLUID_ECUDA);
      return false;
    }
    if (fl::solver_create_async(&j->cfg, s.stream, &s.solver) != FLUID_OK) {
      cudaStreamDestroy(s.stream);
      fail_job(j, FLUID_EINVAL);
      return false;
    }
    if (cudaMallocAsync((void**)&s.U, j->nstate * sizeof(double), s.stream) != cudaSuccess ||
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
          if ((int)running() >= cfg.max_active) break;   // only this thread changes the running set
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
        if (cfg.batch && batchable(j->cfg) && admit_batched(j)) {
          // joins its bucket's next chunk
        } else if (admit(j)) {
          advance(active.back());
        }
        n_active.store(running());
        busy = true;
      }
      for (auto& b : buckets) busy |= step_bucket(*b);
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
          n_active.store(running());
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
    for (auto& b : buckets) {
      if (b->stream) cudaStreamSynchronize(b->stream);
      for (BSlot& s : b->slots) {
        finish(*s.job, s.steps_done + s.chunk_steps, FLUID_EBUSY);
        release(s);
      }
      b->slots.clear();
      drop_bucket(*b);
    }
    buckets.clear();
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
  // the solves' stream-ordered memory returns to the device's pool and is reused without
  // returning it to the CUDA driver in between (the HBM budget bounds what the server holds)
  cudaMemPool_t pool;
  if (cudaSetDevice(cfg->device) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, cfg->device) == cudaSuccess) {
    uint64_t keep = cfg->hbm_budget_bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
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
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    cudaDeviceSynchronize();
    cudaMemPoolTrimTo(pool, 0);
  }
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
