// Serving runtime: continuous batching of independent solves on one GPU.
//
// Requests (grid, face conditions, kernel, precision, operator, host arrays)
// are admitted against a device-memory budget as slots and memory free up;
// admitted requests run on a pool of CUDA streams, so the work of requests
// that arrive while others are on the GPU overlaps on the device.  Plans
// (twiddles, Green's function spectrum, pass geometry) are cached per
// problem key and shared by all slots of that key; a slot holds the device
// input/output arrays and the workspace of one solve plus a CUDA graph of the
// solve's kernel launches, captured once and replayed for every request the
// slot serves.  New plans are set up by worker threads on their own streams
// while the serving loop keeps admitting and completing other requests; the
// setup queue serves the cheapest setup first within a bounded window.
// Idle slots and plans are evicted least recently used first when a new
// request needs the memory.  Completion times come from a host function
// enqueued after the result's device-to-host copy.  Each slot's workspace
// carries the device status word of the solve that runs in it; it is copied
// to pinned host memory after the solve, so a kernel whose bounded wait gave
// up fails exactly the ticket whose result it would have invalidated.
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <chrono>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "flups_gpu.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Slot {
  void* d_rhs = nullptr;
  void* d_phi = nullptr;
  void* d_ws = nullptr;
  int* h_status = nullptr;   // pinned copy of the device status word of the slot's last solve
  cudaGraphExec_t graph = nullptr;
  bool busy = false;
  double last_use = 0;
};

struct Plan {
  std::string key;
  flups_topo topo = nullptr;
  flups_solver solver = nullptr;
  size_t resident = 0, transient = 0, ws = 0, io = 0;
  size_t status_off = 0;      // byte offset of the device status word in a slot's workspace
  std::vector<Slot*> slots;
  int inflight = 0;
  double last_use = 0;
  double setup_cost = 0;      // relative cost of the setup (ordering of the setup queue)
  std::atomic<int> state{0};  // 0 building, 1 ready, < 0 setup failed (status)
  bool settled = false;       // transient setup memory returned to the budget
  size_t slot_bytes() const { return 2 * io + ws; }
};

struct InFlight {
  long long ticket;
  Plan* plan;
  Slot* slot;
  double t_submit;
  std::atomic<int> done{0};
  double t_done = 0;
};

struct Pending {
  long long ticket;
  flups_request rq;
  const void* rhs_host;
  void* phi_host;
  double t_submit;
};

struct Done {
  long long ticket;
  double latency;
  int status;
};

void CUDART_CB on_complete(void* arg) {
  InFlight* f = (InFlight*)arg;
  f->t_done = now_s();
  f->done.store(1, std::memory_order_release);
}

size_t elem_bytes(const flups_request& r) { return r.prec == FLUPS_F32 ? 4 : 8; }
int ncomp_of(const flups_request& r) { return r.op == FLUPS_BIOT_SAVART ? 3 : 1; }

std::string key_of(const flups_request& r) {
  flups_request c;
  memset(&c, 0, sizeof(c));
  memcpy(c.n, r.n, sizeof(c.n));
  c.center = r.center;
  c.prec = r.prec;
  c.op = r.op;
  c.diff = r.diff;
  const int nc = ncomp_of(r);
  for (int k = 0; k < nc; ++k)
    for (int d = 0; d < 3; ++d)
      for (int f = 0; f < 2; ++f) c.bc[k][d][f] = r.bc[k][d][f];
  memcpy(c.h, r.h, sizeof(c.h));
  memcpy(c.L, r.L, sizeof(c.L));
  c.green = r.green;
  c.eps_over_h = r.eps_over_h;
  return std::string((const char*)&c, sizeof(c));
}

}  // namespace

struct flups_server_s {
  size_t budget = 0, in_use = 0, peak = 0;
  // plan setup workers
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Plan*> builds;
  bool stop = false;
  int building = 0;
  double setup_seconds = 0;   // guarded by mu
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  cudaStream_t setup_stream = nullptr, capture_stream = nullptr;
  long long next_ticket = 1;
  std::map<std::string, Plan*> plans;
  std::deque<Pending> queue;
  std::list<InFlight*> inflight;
  std::deque<Done> done;
  flups_server_stats st{};
  // pinned host words for the slots' device status (allocated in chunks, never returned before
  // destroy, so that releasing a slot needs no synchronising cudaFreeHost)
  std::vector<int*> status_chunks;
  std::vector<int*> status_free;
};

namespace {

int cu(cudaError_t e) { return e == cudaSuccess ? FLUPS_OK : (e == cudaErrorMemoryAllocation ? FLUPS_ENOMEM : FLUPS_ECUDA); }

constexpr int kBuildWindow = 8;

void worker_main(flups_server_s* sv, int device) {
  cudaSetDevice(device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Plan* p = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] { return sv->stop || !sv->builds.empty(); });
      if (sv->builds.empty()) break;
      // shortest setup first among the oldest kBuildWindow waiting (bounded reordering: no setup
      // waits behind more than kBuildWindow - 1 later ones): a small plan's setup takes well under a
      // millisecond, a large one with a quadrature-sampled Green's function tens of milliseconds
      auto best = sv->builds.begin();
      int seen = 0;
      for (auto it = sv->builds.begin(); it != sv->builds.end() && seen < kBuildWindow; ++it, ++seen)
        if ((*it)->setup_cost < (*best)->setup_cost) best = it;
      p = *best;
      sv->builds.erase(best);
    }
    const double t0 = now_s();
    const int rc = flups_setup_shared(p->solver, st);
    cudaStreamSynchronize(st);  // every allocation of this setup is complete before anyone frees it
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->setup_seconds += now_s() - t0;
    }
    p->state.store(rc == FLUPS_OK ? 1 : (rc < 0 ? rc : FLUPS_ECUDA), std::memory_order_release);
  }
  if (st) cudaStreamDestroy(st);
}

constexpr int kStatusChunk = 1024;

int* take_status_word(flups_server_s* sv) {
  if (sv->status_free.empty()) {
    int* chunk = nullptr;
    if (cudaMallocHost((void**)&chunk, kStatusChunk * sizeof(int)) != cudaSuccess) return nullptr;
    sv->status_chunks.push_back(chunk);
    for (int i = 0; i < kStatusChunk; ++i) sv->status_free.push_back(chunk + i);
  }
  int* w = sv->status_free.back();
  sv->status_free.pop_back();
  *w = 0;
  return w;
}

void free_slot(flups_server_s* sv, Plan* p, Slot* s) {
  if (s->h_status) sv->status_free.push_back(s->h_status);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->d_rhs) cudaFreeAsync(s->d_rhs, sv->setup_stream);
  if (s->d_phi) cudaFreeAsync(s->d_phi, sv->setup_stream);
  if (s->d_ws) cudaFreeAsync(s->d_ws, sv->setup_stream);
  sv->in_use -= p->slot_bytes();
  delete s;
}

// A plan object that was never registered (no device memory counted).
void discard_plan(Plan* p) {
  if (p->solver) flups_cleanup(p->solver);
  if (p->topo) flups_topo_free(p->topo);
  delete p;
}

void free_plan(flups_server_s* sv, Plan* p) {
  for (Slot* s : p->slots) free_slot(sv, p, s);
  p->slots.clear();
  flups_cleanup_async(p->solver, sv->setup_stream);
  flups_topo_free(p->topo);
  sv->in_use -= p->resident;
  delete p;
}

// Evict idle slots, then idle plans, least recently used first, until `need` fits.
bool make_room(flups_server_s* sv, size_t need, Plan* keep) {
  while (sv->in_use + need > sv->budget) {
    Plan* bp = nullptr;
    Slot* bs = nullptr;
    double best = 1e300;
    for (auto& kv : sv->plans) {
      Plan* p = kv.second;
      for (Slot* s : p->slots)
        if (!s->busy && s->last_use < best) {
          best = s->last_use;
          bp = p;
          bs = s;
        }
    }
    if (bs) {
      for (size_t i = 0; i < bp->slots.size(); ++i)
        if (bp->slots[i] == bs) {
          bp->slots.erase(bp->slots.begin() + i);
          break;
        }
      free_slot(sv, bp, bs);
      sv->st.evictions++;
      continue;
    }
    Plan* vp = nullptr;
    best = 1e300;
    for (auto& kv : sv->plans) {
      Plan* p = kv.second;
      if (p != keep && p->inflight == 0 && p->slots.empty() && p->settled && p->last_use < best) {
        best = p->last_use;
        vp = p;
      }
    }
    if (!vp) return false;
    sv->plans.erase(vp->key);
    free_plan(sv, vp);
    sv->st.evictions++;
  }
  return true;
}

// Host-only plan object for a request (validates it); no device memory yet.
int new_plan(const flups_request& r, Plan** out) {
  Plan* p = new (std::nothrow) Plan;
  if (!p) return FLUPS_ENOMEM;
  int rc = flups_init_topo(r.n, r.center, ncomp_of(r), r.prec, &p->topo);
  if (rc == FLUPS_OK)
    rc = flups_init_solver(p->topo, &r.bc[0][0][0], r.h, r.L, r.green, r.eps_over_h, r.op, r.diff, &p->solver);
  // plans of other face conditions often store the same Green spectrum: one copy for all of them
  if (rc == FLUPS_OK) rc = flups_solver_share_green(p->solver);
  if (rc == FLUPS_OK) rc = flups_solver_memory(p->solver, &p->resident, &p->transient, &p->ws);
  if (rc != FLUPS_OK) {
    if (p->solver) flups_cleanup(p->solver);
    if (p->topo) flups_topo_free(p->topo);
    delete p;
    return rc;
  }
  p->io = (size_t)r.n[0] * r.n[1] * r.n[2] * ncomp_of(r) * elem_bytes(r);
  p->key = key_of(r);
  // setup cost ~ Green samples (the transient FP64 sample array), sampled by quadrature -- several
  // times dearer per sample -- when exactly two directions are unbounded-like
  int du = 0;
  for (int d = 0; d < 3; ++d) du += (r.bc[0][d][0] == FLUPS_UNB || r.bc[0][d][1] == FLUPS_UNB) ? 1 : 0;
  p->setup_cost = (double)p->transient * (du == 2 ? 8.0 : 1.0) + (double)p->resident;
  *out = p;
  return FLUPS_OK;
}

// Try to start one pending request: 1 started, 0 no room yet, < 0 error for this request.
int try_start(flups_server_s* sv, Pending& pd) {
  const std::string key = key_of(pd.rq);
  Plan* p = nullptr;
  auto it = sv->plans.find(key);
  if (it == sv->plans.end()) {
    // a new plan: reserve its memory and hand its setup to a worker; the request waits queued
    int rc = new_plan(pd.rq, &p);
    if (rc) return rc;
    const size_t need = p->resident + p->transient + p->slot_bytes();
    if (need > sv->budget) {
      discard_plan(p);
      return FLUPS_ENOMEM;
    }
    if (!make_room(sv, p->resident + p->transient, nullptr)) {
      discard_plan(p);
      return 0;
    }
    sv->in_use += p->resident + p->transient;
    if (sv->in_use > sv->peak) sv->peak = sv->in_use;
    p->last_use = now_s();
    sv->plans[key] = p;
    sv->st.plan_misses++;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->builds.push_back(p);
      sv->building++;
    }
    sv->cv.notify_one();
    return 0;
  }
  p = it->second;
  const int state = p->state.load(std::memory_order_acquire);
  if (state == 0) return 0;  // still building
  if (!p->settled) {
    sv->in_use -= p->transient;  // the setup's temporary memory is back
    p->settled = true;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->building--;
  }
  if (state < 0) {
    // setup failed: forget the plan (a later request may retry) and fail this one
    sv->plans.erase(p->key);
    free_plan(sv, p);
    return state;
  }
  Slot* slot = nullptr;
  for (Slot* s : p->slots)
    if (!s->busy) {
      slot = s;
      break;
    }
  size_t need = slot ? 0 : p->slot_bytes();
  if (need > sv->budget) return FLUPS_ENOMEM;
  if (!make_room(sv, need, p)) return 0;
  if (!slot) {
    const double t_slot = now_s();
    slot = new (std::nothrow) Slot;
    if (!slot) return FLUPS_ENOMEM;
    int rc = flups_workspace_status(p->solver, &p->status_off);
    if (!rc) {
      slot->h_status = take_status_word(sv);
      if (!slot->h_status) rc = FLUPS_ENOMEM;
    }
    if (!rc) rc = cu(cudaMallocAsync(&slot->d_rhs, p->io, sv->setup_stream));
    if (!rc) rc = cu(cudaMallocAsync(&slot->d_phi, p->io, sv->setup_stream));
    if (!rc) rc = cu(cudaMallocAsync(&slot->d_ws, p->ws, sv->setup_stream));
    if (!rc) rc = cu(cudaStreamSynchronize(sv->setup_stream));
    if (!rc) {
      // one CUDA graph of the solve's launches per slot (pointers fixed for its lifetime)
      cudaGraph_t g = nullptr;
      rc = cu(cudaStreamBeginCapture(sv->capture_stream, cudaStreamCaptureModeThreadLocal));
      if (!rc) {
        int rs = flups_solve_ws(p->solver, slot->d_phi, slot->d_rhs, slot->d_ws, sv->capture_stream);
        cudaError_t ec = cudaStreamEndCapture(sv->capture_stream, &g);
        rc = rs ? rs : cu(ec);
      }
      if (!rc) rc = cu(cudaGraphInstantiate(&slot->graph, g, 0));
      if (g) cudaGraphDestroy(g);
    }
    sv->in_use += p->slot_bytes();
    if (rc) {
      free_slot(sv, p, slot);
      return rc;
    }
    p->slots.push_back(slot);
    sv->st.slots_created++;
    sv->st.slot_seconds += now_s() - t_slot;
  }
  if (sv->in_use > sv->peak) sv->peak = sv->in_use;
  cudaStream_t s = sv->streams[sv->next_stream];
  sv->next_stream = (sv->next_stream + 1) % (int)sv->streams.size();
  InFlight* f = new (std::nothrow) InFlight;
  if (!f) return FLUPS_ENOMEM;
  f->ticket = pd.ticket;
  f->plan = p;
  f->slot = slot;
  f->t_submit = pd.t_submit;
  int rc = cu(cudaMemcpyAsync(slot->d_rhs, pd.rhs_host, p->io, cudaMemcpyHostToDevice, s));
  if (!rc) rc = cu(cudaGraphLaunch(slot->graph, s));
  if (!rc) rc = cu(cudaMemcpyAsync(slot->h_status, (const char*)slot->d_ws + p->status_off, sizeof(int),
                                   cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cu(cudaMemcpyAsync(pd.phi_host, slot->d_phi, p->io, cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cu(cudaLaunchHostFunc(s, on_complete, f));
  if (rc) {
    delete f;
    return rc;
  }
  slot->busy = true;
  slot->last_use = now_s();
  p->inflight++;
  p->last_use = slot->last_use;
  sv->inflight.push_back(f);
  sv->st.admitted++;
  return 1;
}

void admit_queued(flups_server_s* sv) {
  for (auto it = sv->queue.begin(); it != sv->queue.end();) {
    const int r = try_start(sv, *it);
    if (r == 1) {
      it = sv->queue.erase(it);
    } else if (r < 0) {
      sv->done.push_back({it->ticket, -1.0, r});
      sv->st.failed++;
      it = sv->queue.erase(it);
    } else {
      ++it;   // no room yet: later (smaller) requests may still fit
    }
  }
}

void reap(flups_server_s* sv) {
  for (auto it = sv->inflight.begin(); it != sv->inflight.end();) {
    InFlight* f = *it;
    if (f->done.load(std::memory_order_acquire)) {
      // the status word was copied before the host function ran (same stream)
      const int code = *(volatile int*)f->slot->h_status;
      if (code == 0) {
        sv->done.push_back({f->ticket, f->t_done - f->t_submit, FLUPS_OK});
        sv->st.completed++;
      } else {
        sv->done.push_back({f->ticket, -1.0, FLUPS_EDEVICE});
        sv->st.failed++;
      }
      f->slot->busy = false;
      f->slot->last_use = now_s();
      f->plan->inflight--;
      delete f;
      it = sv->inflight.erase(it);
    } else {
      ++it;
    }
  }
  admit_queued(sv);
  // nothing running, nothing being set up and nothing admissible: the head request can never fit
  int building;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    building = sv->building;
  }
  if (sv->inflight.empty() && !sv->queue.empty() && building == 0) {
    Pending pd = sv->queue.front();
    sv->queue.pop_front();
    sv->done.push_back({pd.ticket, -1.0, FLUPS_ENOMEM});
    sv->st.failed++;
  }
}

int drain_out(flups_server_s* sv, long long* tickets, double* lat, int* status, int max, int* n) {
  int k = 0;
  while (k < max && !sv->done.empty()) {
    const Done d = sv->done.front();
    sv->done.pop_front();
    if (tickets) tickets[k] = d.ticket;
    if (lat) lat[k] = d.latency;
    if (status) status[k] = d.status;
    ++k;
  }
  *n = k;
  return FLUPS_OK;
}

}  // namespace

extern "C" {

int flups_server_create(size_t hbm_budget, int nstreams, flups_server* out) {
  if (!out || nstreams < 1 || nstreams > 64 || hbm_budget == 0) return FLUPS_EINVAL;
  flups_server_s* sv = new (std::nothrow) flups_server_s;
  if (!sv) return FLUPS_ENOMEM;
  sv->budget = hbm_budget;
  int rc = FLUPS_OK;
  for (int i = 0; i < nstreams && !rc; ++i) {
    cudaStream_t s;
    rc = cu(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    if (!rc) sv->streams.push_back(s);
  }
  if (!rc) rc = cu(cudaStreamCreateWithFlags(&sv->setup_stream, cudaStreamNonBlocking));
  if (!rc) rc = cu(cudaStreamCreateWithFlags(&sv->capture_stream, cudaStreamNonBlocking));
  if (!rc) {
    // keep freed slot memory in the stream-ordered pool instead of returning it to the driver
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      unsigned long long thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  if (rc) {
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    if (sv->setup_stream) cudaStreamDestroy(sv->setup_stream);
    if (sv->capture_stream) cudaStreamDestroy(sv->capture_stream);
    delete sv;
    return rc;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < 3; ++i) sv->workers.emplace_back(worker_main, sv, dev);
  *out = sv;
  return FLUPS_OK;
}

int flups_server_submit(flups_server sv, const flups_request* rq, const void* rhs_host, void* phi_host,
                        long long* ticket) {
  if (!sv || !rq || !rhs_host || !phi_host) return FLUPS_EINVAL;
  // validate before queueing: a bad request is refused here and touches nothing else
  const std::string key = key_of(*rq);
  if (sv->plans.find(key) == sv->plans.end()) {
    Plan* p = nullptr;
    int rc = new_plan(*rq, &p);
    if (rc) {
      sv->st.rejected++;
      return rc;
    }
    const size_t alone = p->resident + p->transient + p->slot_bytes();
    discard_plan(p);
    if (alone > sv->budget) {
      sv->st.rejected++;
      return FLUPS_ENOMEM;
    }
  }
  Pending pd{sv->next_ticket++, *rq, rhs_host, phi_host, now_s()};
  if (ticket) *ticket = pd.ticket;
  sv->st.submitted++;
  sv->queue.push_back(pd);
  if ((long long)sv->queue.size() > sv->st.queued_max) sv->st.queued_max = (long long)sv->queue.size();
  admit_queued(sv);
  return FLUPS_OK;
}

int flups_server_poll(flups_server sv, long long* tickets, double* latency_s, int* status, int max, int* n_done) {
  if (!sv || !n_done || max < 0) return FLUPS_EINVAL;
  reap(sv);
  return drain_out(sv, tickets, latency_s, status, max, n_done);
}

int flups_server_wait(flups_server sv, long long* tickets, double* latency_s, int* status, int max, int* n_done) {
  if (!sv || !n_done || max < 0) return FLUPS_EINVAL;
  for (;;) {
    reap(sv);
    if (!sv->done.empty() || (sv->inflight.empty() && sv->queue.empty())) break;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  return drain_out(sv, tickets, latency_s, status, max, n_done);
}

int flups_server_pending(flups_server sv, int* queued, int* running) {
  if (!sv) return FLUPS_EINVAL;
  if (queued) *queued = (int)sv->queue.size();
  if (running) *running = (int)sv->inflight.size();
  return FLUPS_OK;
}

int flups_server_get_stats(flups_server sv, flups_server_stats* out) {
  if (!sv || !out) return FLUPS_EINVAL;
  *out = sv->st;
  out->plan_hits = sv->st.admitted > sv->st.plan_misses ? sv->st.admitted - sv->st.plan_misses : 0;
  out->hbm_in_use = sv->in_use;
  out->hbm_peak = sv->peak;
  out->plans_cached = (long long)sv->plans.size();
  std::lock_guard<std::mutex> lk(sv->mu);
  out->setup_seconds = sv->setup_seconds;
  return FLUPS_OK;
}

int flups_server_destroy(flups_server sv) {
  if (!sv) return FLUPS_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (std::thread& t : sv->workers) t.join();
  for (cudaStream_t s : sv->streams) cudaStreamSynchronize(s);
  reap(sv);
  for (InFlight* f : sv->inflight) delete f;
  sv->inflight.clear();
  for (auto& kv : sv->plans) free_plan(sv, kv.second);
  sv->plans.clear();
  cudaStreamSynchronize(sv->setup_stream);
  for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
  cudaStreamDestroy(sv->setup_stream);
  cudaStreamDestroy(sv->capture_stream);
  for (int* c : sv->status_chunks) cudaFreeHost(c);
  delete sv;
  return FLUPS_OK;
}

}  // extern "C"
