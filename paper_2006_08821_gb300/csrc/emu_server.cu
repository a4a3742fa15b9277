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
constexpr int kPrepThreads = 4;  // handles built (and released) concurrently

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
  std::vector<int32_t> bone_id, joint_type, joint_bones;
  std::vector<double> joint_point, joint_axis, joint_half_length;
  int32_t n_materials = 0, n_joints = 0;
  bool has_fiber = false, has_fixed_pos = false, has_bones = false;
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
    d.bone_id = has_bones ? bone_id.data() : nullptr;
    d.n_joints = n_joints;
    if (n_joints > 0) {
      d.joint_type = joint_type.data();
      d.joint_bones = joint_bones.data();
      d.joint_point = joint_point.data();
      d.joint_axis = joint_axis.data();
      d.joint_half_length = joint_half_length.data();
    }
    return d;
  }
};

}  // namespace

// Device resources of a request while it is active; released off the
// worker thread.
struct Slot {
  emu_handle* h = nullptr;
  cudaStream_t st = nullptr;
  emu::SolveTask* task = nullptr;
  uint64_t bytes = 0;
};

struct emu_server {
  size_t budget = 0, used = 0;
  int inflight = 0;  // requests admitted and not yet released (<= kMaxActive)
  emu_params prm;
  emu_allocator alloc;
  bool has_alloc = false;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;       // wakes the worker
  std::condition_variable prep_cv;  // wakes the set-up thread
  bool stop = false;
  std::deque<std::unique_ptr<Request>> queue;            // submitted, not admitted
  std::deque<std::unique_ptr<Request>> to_build;         // admitted, handle not built yet
  std::deque<std::unique_ptr<Request>> built;            // handle built, not yet stepped
  std::deque<Slot> to_release;                           // finished, handle to destroy
  std::map<uint64_t, std::unique_ptr<Request>> done;     // finished, result not taken
  std::deque<uint64_t> unreported;                       // finished, not yet polled
  std::map<uint64_t, int> ids;                           // every id in use
  std::vector<std::unique_ptr<Request>> active;          // worker-owned
  std::thread worker;
  std::vector<std::thread> prep;  // set-up threads

  void run();
  void run_prep();
  void build(Request* r);
  void finish(std::unique_ptr<Request> r);
  void publish(std::unique_ptr<Request> r);  // with mu held
  bool advance(Request* r);  // true when the request is finished
};

namespace {

Slot take_slot(Request* r) {
  Slot s;
  s.h = r->h;
  s.st = r->st;
  s.task = r->task;
  s.bytes = r->stats.device_bytes;
  r->h = nullptr;
  r->st = nullptr;
  r->task = nullptr;
  return s;
}

void release_slot(Slot& s) {
  if (s.task) emu::task_delete(s.task);
  s.task = nullptr;
  if (s.h) emu_destroy(s.h);  // waits for the handle's stream
  s.h = nullptr;
  if (s.st) cudaStreamDestroy(s.st);
  s.st = nullptr;
}

// Stream-ordered device memory for the requests' handles when the caller
// gives no allocator: allocation and release are enqueued on the handle's
// stream, so building or destroying one request's handle never waits for
// the device work of the others.
void* async_alloc(void*, size_t bytes, void* stream) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, (cudaStream_t)stream) != cudaSuccess) return nullptr;
  return p;
}
void async_free(void*, void* p, size_t, void* stream) { cudaFreeAsync(p, (cudaStream_t)stream); }

}  // namespace

// Set-up of an admitted request (on the set-up thread): its stream, handle
// (emu_create), first activation and solve task.
void emu_server::build(Request* r) {
  r->t_admit = clk::now();
  r->stats.queue_ms = ms_between(r->t_submit, r->t_admit);
  int rc = EMU_OK;
  if (cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking) != cudaSuccess) {
    r->st = nullptr;
    rc = EMU_ERR_CUDA;
  }
  if (rc == EMU_OK) {
    emu_mesh_desc d = r->desc();
    rc = emu_create(&d, &prm, &alloc, r->st, &r->h);
  }
  r->t_ready = clk::now();
  r->stats.setup_ms = ms_between(r->t_admit, r->t_ready);
  if (rc == EMU_OK) rc = emu_set_activation(r->h, r->acts.data(), r->m);
  if (rc == EMU_OK) {
    r->task = emu::task_new(r->h, &r->fstats);
    if (!r->task) rc = EMU_ERR_OOM;
  }
  r->frame = 0;
  if (rc != EMU_OK) r->stats.status = rc;
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

void emu_server::publish(std::unique_ptr<Request> r) {
  r->acts.clear();
  r->acts.shrink_to_fit();
  unreported.push_back(r->id);
  done[r->id] = std::move(r);
}

// A finished request (worker thread): its result is published at once, its
// handle goes to the set-up thread for release (budget and slot are freed
// there, after the release).
void emu_server::finish(std::unique_ptr<Request> r) {
  const clk::time_point t = clk::now();
  r->stats.solve_ms = ms_between(r->t_ready, t);
  r->stats.latency_ms = ms_between(r->t_submit, t);
  Slot s = take_slot(r.get());
  {
    std::lock_guard<std::mutex> lk(mu);
    publish(std::move(r));
    to_release.push_back(s);
  }
  prep_cv.notify_one();
}

// Worker: admission by budget and slot count, then it only steps the active
// requests' solve tasks; building and destroying handles (emu_create's
// set-up of the basis, emu_destroy's release) run on the set-up thread, so
// requests in flight keep advancing meanwhile.
void emu_server::run() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<std::unique_ptr<Request>> ready;
    bool admitted = false;
    {
      std::unique_lock<std::mutex> lk(mu);
      auto can_admit = [&] {
        return !queue.empty() && inflight < (int)kMaxActive &&
               used + (size_t)queue.front()->stats.device_bytes <= budget;
      };
      if (active.empty()) cv.wait(lk, [&] { return stop || !built.empty() || can_admit(); });
      if (stop) break;
      // admission in arrival order while memory and a slot are free
      while (can_admit()) {
        used += (size_t)queue.front()->stats.device_bytes;
        ++inflight;
        to_build.push_back(std::move(queue.front()));
        queue.pop_front();
        admitted = true;
      }
      while (!built.empty()) {
        ready.push_back(std::move(built.front()));
        built.pop_front();
      }
    }
    if (admitted) prep_cv.notify_one();
    bool progressed = admitted || !ready.empty();
    for (auto& r : ready) {
      r->waiting = emu::task_step(r->task) != 0;
      active.push_back(std::move(r));
    }
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
  for (auto& r : active) {
    Slot s = take_slot(r.get());
    release_slot(s);
  }
  active.clear();
}

// Set-up thread: builds admitted requests' handles and releases finished
// ones (releases first, so memory returns to the budget as early as possible).
void emu_server::run_prep() {
  cudaSetDevice(device);
  for (;;) {
    std::unique_ptr<Request> job;
    Slot rel;
    bool has_rel = false;
    {
      std::unique_lock<std::mutex> lk(mu);
      prep_cv.wait(lk, [&] { return stop || !to_build.empty() || !to_release.empty(); });
      if (!to_release.empty()) {
        rel = to_release.front();
        to_release.pop_front();
        has_rel = true;
      } else if (stop) {
        break;
      } else {
        job = std::move(to_build.front());
        to_build.pop_front();
      }
    }
    if (has_rel) {
      release_slot(rel);
      {
        std::lock_guard<std::mutex> lk(mu);
        used -= (size_t)rel.bytes;
        --inflight;
      }
      cv.notify_one();
      continue;
    }
    build(job.get());
    {
      std::lock_guard<std::mutex> lk(mu);
      if (job->stats.status != EMU_OK) {  // set-up failed: the request ends here
        Slot s = take_slot(job.get());
        const clk::time_point t = clk::now();
        job->stats.latency_ms = ms_between(job->t_submit, t);
        publish(std::move(job));
        to_release.push_back(s);
      } else {
        built.push_back(std::move(job));
      }
    }
    cv.notify_one();
  }
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
  } else {
    s->alloc.ctx = nullptr;
    s->alloc.alloc = async_alloc;
    s->alloc.free = async_free;
  }
  s->budget = budget_bytes;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    emu::set_last_error("emu_server_create: no CUDA device");
    return EMU_ERR_CUDA;
  }
  try {
    for (int k = 0; k < kPrepThreads; ++k) s->prep.emplace_back([s] { s->run_prep(); });
    s->worker = std::thread([s] { s->run(); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->prep_cv.notify_all();
    for (auto& t : s->prep)
      if (t.joinable()) t.join();
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
    r->has_bones = mesh->bone_id != nullptr;
    if (r->has_bones) r->bone_id.assign(mesh->bone_id, mesh->bone_id + m);
    r->n_joints = mesh->n_joints;
    if (r->n_joints > 0) {
      const int32_t j = r->n_joints;
      r->joint_type.assign(mesh->joint_type, mesh->joint_type + j);
      r->joint_bones.assign(mesh->joint_bones, mesh->joint_bones + 2 * j);
      r->joint_point.assign(mesh->joint_point, mesh->joint_point + 3 * j);
      r->joint_axis.assign(mesh->joint_axis, mesh->joint_axis + 3 * j);
      r->joint_half_length.assign(mesh->joint_half_length, mesh->joint_half_length + j);
    }
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
  srv->prep_cv.notify_all();
  if (srv->worker.joinable()) srv->worker.join();
  for (auto& t : srv->prep)
    if (t.joinable()) t.join();
  // handles built or finished but not yet released
  for (auto& s : srv->to_release) release_slot(s);
  for (auto& r : srv->built) {
    Slot s = take_slot(r.get());
    release_slot(s);
  }
  delete srv;
  return EMU_OK;
}

}  // extern "C"
