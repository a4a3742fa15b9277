// Serving: a persistent request loop that admits quasi-static solves of
// different meshes by device-memory budget, keeps each request's state
// resident across its frames (warm starts) and interleaves the active
// requests' Newton loops on their own streams (continuous batching).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "emu_internal.h"

namespace {

using clk = std::chrono::steady_clock;
constexpr size_t kMaxActive = 32;

double ms_between(clk::time_point a, clk::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// A request with its own copy of the mesh description.
struct Request {
  uint64_t id = 0;
  int64_t n = 0, m = 0;
  int32_t frames = 0;
  std::vector<double> rest_pos, youngs, poisson, fiber_dir, fixed_pos, acts;
  std::vector<int32_t> tets, fixed_verts;
  std::vector<uint8_t> material_id;
  int32_t n_materials = 0;
  bool has_fiber = false, has_fixed_pos = false;
  std::vector<double> positions;  // frames x n x 3
  emu_request_stats stats;
  clk::time_point t_submit, t_admit, t_ready;
  // while active
  emu_handle* h = nullptr;
  cudaStream_t st = nullptr;
  emu::SolveTask* task = nullptr;
  emu_solve_stats fstats;
  int32_t frame = 0;
  bool waiting = false;

  emu_mesh_desc desc() const {
    emu_mesh_desc d;
    memset(&d, 0, sizeof(d));
    d.n_verts = n;
    d.n_tets = m;
    d.rest_pos = rest_pos.data();
    d.tets = tets.data();
    d.n_materials = n_materials;
    d.youngs = youngs.data();
    d.poisson = poisson.data();
    d.material_id = material_id.data();
    d.fiber_dir = has_fiber ? fiber_dir.data() : nullptr;
    d.n_fixed = (int64_t)fixed_verts.size();
    d.fixed_verts = fixed_verts.data();
    d.fixed_pos = has_fixed_pos ? fixed_pos.data() : nullptr;
    return d;
  }
};

}  // namespace

struct emu_server {
  size_t budget = 0, used = 0;
  emu_params prm;
  emu_allocator alloc;
  bool has_alloc = false;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<std::unique_ptr<Request>> queue;            // submitted, not admitted
  std::map<uint64_t, std::unique_ptr<Request>> done;     // finished, result not taken
  std::deque<uint64_t> unreported;                       // finished, not yet polled
  std::map<uint64_t, int> ids;                           // every id in use
  std::vector<std::unique_ptr<Request>> active;          // worker-owned
  std::thread worker;

  void run();
  void admit(Request* r);
  void finish(std::unique_ptr<Request> r);
  bool advance(Request* r);  // true when the request is finished
};

namespace {

void release_slot(Request* r) {
  if (r->task) emu::task_delete(r->task);
  r->task = nullptr;
  if (r->h) emu_destroy(r->h);  // waits for the handle's stream
  r->h = nullptr;
  if (r->st) cudaStreamDestroy(r->st);
  r->st = nullptr;
}

}  // namespace

void emu_server::admit(Request* r) {
  r->t_admit = clk::now();
  r->stats.queue_ms = ms_between(r->t_submit, r->t_admit);
  int rc = EMU_OK;
  if (cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking) != cudaSuccess) {
    r->st = nullptr;
    rc = EMU_ERR_CUDA;
  }
  if (rc == EMU_OK) {
    emu_mesh_desc d = r->desc();
    rc = emu_create(&d, &prm, has_alloc ? &alloc : nullptr, r->st, &r->h);
  }
  r->t_ready = clk::now();
  r->stats.setup_ms = ms_between(r->t_admit, r->t_ready);
  if (rc == EMU_OK) rc = emu_set_activation(r->h, r->acts.data(), r->m);
  if (rc == EMU_OK) {
    r->task = emu::task_new(r->h, &r->fstats);
    if (!r->task) rc = EMU_ERR_OOM;
  }
  if (rc != EMU_OK) {
    r->stats.status = rc;
    return;
  }
  r->frame = 0;
  r->waiting = emu::task_step(r->task) != 0;
}

// Steps the request's task if its device work is done; on a finished frame
// records it and starts the next one. Returns true when the request is over.
bool emu_server::advance(Request* r) {
  if (r->stats.status != EMU_OK || !r->task) return true;
  if (r->waiting) {
    if (!emu::task_ready(r->task)) return false;
    r->waiting = emu::task_step(r->task) != 0;
    if (r->waiting) return false;
  }
  // the frame's solve has finished
  const int st = emu::task_status(r->task);
  r->stats.newton_iters += r->fstats.newton_iters;
  r->stats.pcg_iters += r->fstats.pcg_iters;
  r->stats.rel_residual = r->fstats.rel_residual;
  if (st != EMU_OK) {
    r->stats.status = st;
    return true;
  }
  int rc = emu_get_positions(r->h, r->positions.data() + (size_t)r->frame * 3 * r->n, 0);
  if (rc != EMU_OK) {
    r->stats.status = rc;
    return true;
  }
  r->stats.frames_done = ++r->frame;
  if (r->frame >= r->frames) return true;
  rc = emu_set_activation(r->h, r->acts.data() + (size_t)r->frame * r->m, r->m);
  if (rc != EMU_OK) {
    r->stats.status = rc;
    return true;
  }
  emu::task_delete(r->task);
  r->task = emu::task_new(r->h, &r->fstats);
  if (!r->task) {
    r->stats.status = EMU_ERR_OOM;
    return true;
  }
  r->waiting = emu::task_step(r->task) != 0;
  return false;
}

void emu_server::finish(std::unique_ptr<Request> r) {
  const clk::time_point t = clk::now();
  r->stats.solve_ms = ms_between(r->t_ready, t);
  r->stats.latency_ms = ms_between(r->t_submit, t);
  release_slot(r.get());
  r->acts.clear();
  r->acts.shrink_to_fit();
  std::lock_guard<std::mutex> lk(mu);
  used -= (size_t)r->stats.device_bytes;
  unreported.push_back(r->id);
  done[r->id] = std::move(r);
}

void emu_server::run() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<std::unique_ptr<Request>> admitted;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (active.empty()) cv.wait(lk, [&] { return stop || !queue.empty(); });
      if (stop) break;
      // admission in arrival order while memory and a slot are free
      while (!queue.empty() && active.size() + admitted.size() < kMaxActive &&
             used + (size_t)queue.front()->stats.device_bytes <= budget) {
        used += (size_t)queue.front()->stats.device_bytes;
        admitted.push_back(std::move(queue.front()));
        queue.pop_front();
      }
    }
    for (auto& r : admitted) {
      admit(r.get());
      active.push_back(std::move(r));
    }
    bool progressed = !admitted.empty();
    for (size_t k = 0; k < active.size();) {
      Request* r = active[k].get();
      const bool was_waiting = r->waiting;
      if (advance(r)) {
        finish(std::move(active[k]));
        active.erase(active.begin() + (std::ptrdiff_t)k);
        progressed = true;
        continue;
      }
      if (!was_waiting || !r->waiting) progressed = true;
      ++k;
    }
    if (!progressed) std::this_thread::yield();
  }
  for (auto& r : active) release_slot(r.get());
  active.clear();
}

extern "C" {

int emu_server_create(size_t budget_bytes, const emu_params* params, const emu_allocator* alloc, emu_server** out) {
  if (!out) {
    emu::set_last_error("emu_server_create: out is NULL");
    return EMU_ERR_INVALID_ARG;
  }
  *out = nullptr;
  emu_server* s = new (std::nothrow) emu_server();
  if (!s) return EMU_ERR_OOM;
  if (params)
    s->prm = *params;
  else
    emu_default_params(&s->prm);
  if (alloc && alloc->alloc && alloc->free) {
    s->alloc = *alloc;
    s->has_alloc = true;
  }
  s->budget = budget_bytes;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    emu::set_last_error("emu_server_create: no CUDA device");
    return EMU_ERR_CUDA;
  }
  try {
    s->worker = std::thread([s] { s->run(); });
  } catch (...) {
    delete s;
    emu::set_last_error("emu_server_create: cannot start the worker thread");
    return EMU_ERR_OOM;
  }
  *out = s;
  return EMU_OK;
}

int emu_server_submit(emu_server* srv, const emu_mesh_desc* mesh, const double* activations, int32_t n_frames,
                      uint64_t request_id) {
  if (!srv || !mesh || !activations || n_frames < 1) {
    emu::set_last_error("emu_server_submit: NULL argument or n_frames < 1");
    return EMU_ERR_INVALID_ARG;
  }
  size_t bytes = 0;
  int rc = emu_required_bytes(mesh, &srv->prm, &bytes);  // also validates the mesh
  if (rc) return rc;
  if (bytes > srv->budget) {
    emu::set_last_error("emu_server_submit: the mesh needs more device memory than the whole budget");
    return EMU_ERR_OOM;
  }
  const int64_t m = mesh->n_tets, n = mesh->n_verts;
  for (int64_t k = 0; k < (int64_t)n_frames * m; ++k)
    if (!(activations[k] >= 0.0) || !(activations[k] < 1e300)) {
      emu::set_last_error("emu_server_submit: activations must be finite and >= 0");
      return EMU_ERR_INVALID_ARG;
    }
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return EMU_ERR_OOM;
  try {
    r->id = request_id;
    r->n = n;
    r->m = m;
    r->frames = n_frames;
    r->rest_pos.assign(mesh->rest_pos, mesh->rest_pos + 3 * n);
    r->tets.assign(mesh->tets, mesh->tets + 4 * m);
    r->n_materials = mesh->n_materials;
    r->youngs.assign(mesh->youngs, mesh->youngs + mesh->n_materials);
    r->poisson.assign(mesh->poisson, mesh->poisson + mesh->n_materials);
    r->material_id.assign(mesh->material_id, mesh->material_id + m);
    r->has_fiber = mesh->fiber_dir != nullptr;
    if (r->has_fiber) r->fiber_dir.assign(mesh->fiber_dir, mesh->fiber_dir + 3 * m);
    r->fixed_verts.assign(mesh->fixed_verts, mesh->fixed_verts + mesh->n_fixed);
    r->has_fixed_pos = mesh->fixed_pos != nullptr;
    if (r->has_fixed_pos) r->fixed_pos.assign(mesh->fixed_pos, mesh->fixed_pos + 3 * mesh->n_fixed);
    r->acts.assign(activations, activations + (size_t)n_frames * m);
    r->positions.assign((size_t)n_frames * 3 * n, 0.0);
  } catch (...) {
    emu::set_last_error("emu_server_submit: host allocation failed");
    return EMU_ERR_OOM;
  }
  memset(&r->stats, 0, sizeof(r->stats));
  r->stats.id = request_id;
  r->stats.device_bytes = bytes;
  r->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->ids.count(request_id)) {
      emu::set_last_error("emu_server_submit: request id already in use");
      return EMU_ERR_INVALID_ARG;
    }
    srv->ids[request_id] = 1;
    srv->queue.push_back(std::move(r));
  }
  srv->cv.notify_one();
  return EMU_OK;
}

int emu_server_poll(emu_server* srv, uint64_t* done_ids, int32_t cap, int32_t* n_done) {
  if (!srv || !n_done || cap < 0 || (cap > 0 && !done_ids)) {
    emu::set_last_error("emu_server_poll: bad argument");
    return EMU_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  int32_t k = 0;
  while (k < cap && !srv->unreported.empty()) {
    done_ids[k++] = srv->unreported.front();
    srv->unreported.pop_front();
  }
  *n_done = k;
  return EMU_OK;
}

int emu_server_result(emu_server* srv, uint64_t request_id, double* positions, emu_request_stats* stats) {
  if (!srv) {
    emu::set_last_error("emu_server_result: NULL server");
    return EMU_ERR_INVALID_ARG;
  }
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->done.find(request_id);
    if (it == srv->done.end()) {
      emu::set_last_error("emu_server_result: unknown or unfinished request");
      return EMU_ERR_INVALID_ARG;
    }
    r = std::move(it->second);
    srv->done.erase(it);
    srv->ids.erase(request_id);
    for (auto u = srv->unreported.begin(); u != srv->unreported.end(); ++u)
      if (*u == request_id) {
        srv->unreported.erase(u);
        break;
      }
  }
  if (positions) memcpy(positions, r->positions.data(), r->positions.size() * sizeof(double));
  if (stats) *stats = r->stats;
  return EMU_OK;
}

int emu_server_destroy(emu_server* srv) {
  if (!srv) return EMU_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_all();
  if (srv->worker.joinable()) srv->worker.join();
  delete srv;
  return EMU_OK;
}

}  // extern "C"
