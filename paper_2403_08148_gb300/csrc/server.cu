// server.cu -- continuous-batching request server (host thread).
//
// Requests are trajectory segments (n beads, nsteps of velocity Verlet).
// A worker thread keeps an active set of systems resident on the device in
// one pooled batch engine and repeatedly runs chunks of steps over all of
// them (each member held at its own step count once it has taken its
// segment, while the others step on); between chunks it retires finished
// requests (device -> host copy of their final state) and admits queued
// ones whose device footprint fits the memory budget and a free slot.  A change of the active set moves to a new
// pooled layout, built and captured on the host while the current chunk
// runs on the GPU, and carries the state of continuing systems over with
// device-to-device copies ordered after the chunk, so their trajectories are
// unaffected: every kernel's arithmetic for a system depends only on that
// system, and all accumulation is fixed point, so a request's result is
// bit-identical alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"

using namespace gcme;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t ticket = 0;
  SysSpec spec;
  std::vector<double> pos;
  std::vector<float> vel;
  int64_t nsteps = 0, done = 0;
  int64_t done_at_hand_over = 0;  // worker's copy of done, taken under the lock
  int32_t status = 1;  // 1 queued, 2 running, 0 done, <0 error
  bool cancel = false;
  size_t bytes = 0;
  double energy[GCME_NTERMS] = {0};
  double t_submit = 0, t_admit = 0, t_done = 0;
};

// Device bytes of one system in the pooled layout (state + scratch), the
// admission footprint.
size_t footprint(const SysSpec &sp) {
  const gcme_params &p = sp.p;
  long long n = sp.n, nq = 0;
  for (double z : sp.q) nq += z != 0.0;
  long long nimg = p.geometry == GCME_SLAB_IMAGE ? nq : 0;
  long long ne = n + nimg, nqe = nq + nimg;
  long long ncell = 1;
  for (int a = 0; a < 3; ++a)
    ncell *= cells_per_axis(p.box[a], p.rc, 1);
  long long G = (long long)p.K[0] * p.K[1] * p.K[2];
  bool f64 = p.precision == GCME_FP64;
  size_t b = 0;
  b += n * (24 + (f64 ? 24 : 12) + 8 + 24 + 4);             // pos, vel, q, force, real_sys
  b += ne * (16 + 4 * 5 + 16 + (f64 ? 64 : 0));             // ext arrays
  b += nqe * 8 + nimg * 4;                                  // qlist, q_sys, img_src
  b += ncell * (4 * 5 + 8 * 3);                             // cells + pair work
  b += G * (8 + (f64 ? 16 : 8));                            // charge grid + complex grid
  b += (size_t)(p.K[0] + p.K[1] + p.K[2]) * 32;             // twiddles, moduli, fft work
  b += sp.bonds.size() * 8;
  b += 4096;                                                // descriptors, accumulators
  return b;
}

}  // namespace

struct gcme_server {
  gcme_ctx *ctx = nullptr;
  int device = 0;
  size_t budget = 0;
  int chunk = 50;
  int max_active = 256;
  std::mutex mu;
  std::condition_variable cv;
  std::condition_variable cv_done;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> active;
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  cudaStream_t stream = nullptr;
  std::unique_ptr<Engine> eng;
  std::unique_ptr<Engine> eng_keep;  // replaced engine, freed after the stream's work on it
  std::vector<uint64_t> eng_members;
  std::vector<unsigned long long> ctr_staging, stop_staging;
  bool forces_valid = false;
  int64_t st_admitted = 0, st_completed = 0, st_rejected = 0, st_chunks = 0, st_beadsteps = 0,
          st_peak_active = 0, st_peak_bytes = 0, st_rebuilds = 0;
  double st_rebuild_s = 0.0, st_wait_s = 0.0;
  std::string worker_error;

  void run();
  std::unique_ptr<Engine> make_engine(const std::vector<Req *> &members, int *rc);
  void hand_over(Engine &ne, const std::vector<Req *> &members, int64_t ahead);
  void admit_into(std::vector<uint64_t> &set, size_t used);
};

// A pooled engine for an active set, with its step and force graphs
// captured (host work: it runs while the previous chunk is on the GPU; the
// engine's setup copies use the legacy stream, which a non-blocking stream's
// work does not wait for, and vice versa).
std::unique_ptr<Engine> gcme_server::make_engine(const std::vector<Req *> &members, int *rc) {
  std::vector<SysSpec> specs;
  for (const Req *r : members) specs.push_back(r->spec);
  std::unique_ptr<Engine> ne(new Engine);
  *rc = ne->build(device, specs, true);
  if (*rc) return nullptr;
  ne->enable_step_limits();  // each member stops at its own step count
  cudaGraphExec_t g;
  *rc = ne->forces_graph(ne->P, &g);
  if (!*rc) *rc = ne->step_graph(ne->P, &g);
  return *rc ? nullptr : std::move(ne);
}

// Enqueue on `stream` the state of every member into engine ne: a device
// copy from the current engine for members that continue, the submitted
// host state for new ones; each member keeps its own step counter (the
// Langevin noise counter): its steps done, plus `ahead` for continuing
// members (the steps of the chunk on the stream before these copies).
// Ordered after the work already on the stream.
void gcme_server::hand_over(Engine &ne, const std::vector<Req *> &members, int64_t ahead) {
  ctr_staging.resize(members.size());
  for (size_t k = 0; k < members.size(); ++k) {
    Req &r = *members[k];
    const long long off = ne.bead_off[k], n = r.spec.n;
    auto it = std::find(eng_members.begin(), eng_members.end(), r.ticket);
    ctr_staging[k] = (unsigned long long)(r.done_at_hand_over +
                                          (eng && it != eng_members.end() ? ahead : 0));
    if (eng && it != eng_members.end()) {
      const long long ooff = eng->bead_off[it - eng_members.begin()];
      cudaMemcpyAsync(ne.P.pos + 3 * off, eng->P.pos + 3 * ooff, sizeof(double) * 3 * n,
                      cudaMemcpyDeviceToDevice, stream);
      cudaMemcpyAsync(reinterpret_cast<float *>(ne.P.vel) + 3 * off,
                      reinterpret_cast<float *>(eng->P.vel) + 3 * ooff, sizeof(float) * 3 * n,
                      cudaMemcpyDeviceToDevice, stream);
    } else {
      cudaMemcpyAsync(ne.P.pos + 3 * off, r.pos.data(), sizeof(double) * 3 * n,
                      cudaMemcpyHostToDevice, stream);
      cudaMemcpyAsync(reinterpret_cast<float *>(ne.P.vel) + 3 * off, r.vel.data(),
                      sizeof(float) * 3 * n, cudaMemcpyHostToDevice, stream);
    }
  }
  cudaMemcpyAsync(ne.P.step_ctr, ctr_staging.data(),
                  sizeof(unsigned long long) * ctr_staging.size(), cudaMemcpyHostToDevice, stream);
  // each member's step limit: its segment's length in the same count
  stop_staging.resize(members.size());
  for (size_t k = 0; k < members.size(); ++k)
    stop_staging[k] = (unsigned long long)members[k]->nsteps;
  cudaMemcpyAsync(ne.step_stop_buf, stop_staging.data(),
                  sizeof(unsigned long long) * stop_staging.size(), cudaMemcpyHostToDevice,
                  stream);
}

// Admit queued requests (FIFO) while slots and the memory budget allow,
// given the bytes already held; called with the lock held.
void gcme_server::admit_into(std::vector<uint64_t> &set, size_t used) {
  while (!queue.empty() && (int)set.size() < max_active) {
    Req &r = *reqs[queue.front()];
    if (r.cancel) {
      r.status = GCME_ERR_INVALID;
      r.t_done = now_s();
      queue.pop_front();
      cv_done.notify_all();
      continue;
    }
    if (used + r.bytes > budget) break;
    used += r.bytes;
    r.status = 2;
    r.t_admit = now_s();
    set.push_back(queue.front());
    queue.pop_front();
    ++st_admitted;
  }
}

// The worker: one chunk of steps of the active set at a time.  While a
// chunk runs on the GPU the worker decides the next active set (the members
// that do not finish in this chunk, then queued requests as memory allows)
// and, when it differs, builds and captures the next pooled engine; the
// hand-over of the state (device copies, new requests' host state), the copy
// out of finished members and the next chunk follow on the same stream,
// with one synchronisation per chunk.
void gcme_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    cv.wait(lk, [&] { return stop || !queue.empty() || !active.empty(); });
    if (stop) break;
    // ---- retire cancelled, admit
    for (auto it = active.begin(); it != active.end();) {
      Req &r = *reqs[*it];
      if (r.cancel) {
        r.status = GCME_ERR_INVALID;
        r.t_done = now_s();
        it = active.erase(it);
        cv_done.notify_all();
      } else {
        ++it;
      }
    }
    // with an engine ready for the active set, newcomers wait for the next
    // chunk's overlapped decision instead of forcing a build here
    if (active.empty() || active != eng_members || !eng) {
      size_t used = 0;
      for (uint64_t t : active) used += reqs[t]->bytes;
      admit_into(active, used);
    }
    if (active.empty()) continue;
    st_peak_active = std::max<int64_t>(st_peak_active, (int64_t)active.size());
    const std::vector<uint64_t> members = active;
    std::vector<Req *> mreq;  // pointers stay valid: active requests are not erased
    // a chunk runs until its longest remaining segment ends or for `chunk`
    // steps; members with fewer steps left are held at their own count
    int64_t maxrem = 0;
    for (uint64_t t : members) {
      Req *r = reqs[t].get();
      r->done_at_hand_over = r->done;
      mreq.push_back(r);
      maxrem = std::max(maxrem, r->nsteps - r->done);
    }
    const int64_t steps = std::min<int64_t>(chunk, maxrem);
    lk.unlock();
    int rc = GCME_OK;
    if (members != eng_members) {  // first chunk, or after a cancellation or an error
      const double t0 = now_s();
      std::unique_ptr<Engine> ne = make_engine(mreq, &rc);
      if (!rc) hand_over(*ne, mreq, 0);
      st_rebuild_s += now_s() - t0;
      ++st_rebuilds;
      if (!rc) {
        eng_keep = std::move(eng);  // freed after the next synchronisation
        eng = std::move(ne);
        eng_members = members;
        forces_valid = false;
      }
    }
    // ---- the chunk (asynchronous)
    if (rc == GCME_OK && steps > 0) {
      cudaGraphExec_t fg, sg;
      rc = eng->forces_graph(eng->P, &fg);
      if (!rc) rc = eng->step_graph(eng->P, &sg);
      if (!rc && !forces_valid) {
        cudaGraphLaunch(fg, stream);
        forces_valid = true;
      }
      for (int64_t k = 0; !rc && k < steps; ++k) cudaGraphLaunch(sg, stream);
    }
    // ---- meanwhile: the next active set and its engine
    std::vector<char> fin(members.size(), 0);
    std::vector<uint64_t> next;
    std::vector<Req *> nreq;
    size_t next_used = 0;
    lk.lock();
    for (size_t k = 0; k < members.size(); ++k) {
      Req &r = *mreq[k];
      fin[k] = r.done + steps >= r.nsteps;
      if (!fin[k] && !r.cancel) {
        next.push_back(members[k]);
        next_used += r.bytes;
      }
    }
    if (rc == GCME_OK) admit_into(next, next_used);
    for (uint64_t t : next) {
      Req *r = reqs[t].get();
      r->done_at_hand_over = r->done;
      nreq.push_back(r);
    }
    lk.unlock();
    std::unique_ptr<Engine> ne;
    if (rc == GCME_OK && !next.empty() && next != members) {
      const double t0 = now_s();
      ne = make_engine(nreq, &rc);
      st_rebuild_s += now_s() - t0;
      ++st_rebuilds;
    }
    // ---- on the stream after the chunk: copy out finished members, hand
    // the state over to the next engine; then wait once
    std::vector<double> E((size_t)GCME_NTERMS * members.size());
    if (rc == GCME_OK) {
      cudaMemcpyAsync(E.data(), eng->P.energy, sizeof(double) * E.size(), cudaMemcpyDeviceToHost,
                      stream);
      for (size_t k = 0; k < members.size(); ++k) {
        if (!fin[k]) continue;
        Req &r = *mreq[k];
        const long long off = eng->bead_off[k], n = r.spec.n;
        cudaMemcpyAsync(r.pos.data(), eng->P.pos + 3 * off, sizeof(double) * 3 * n,
                        cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(r.vel.data(), reinterpret_cast<float *>(eng->P.vel) + 3 * off,
                        sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, stream);
      }
      if (ne) hand_over(*ne, nreq, steps);  // continuing members: steps done after this chunk
    }
    const double tw = now_s();
    cudaError_t e = cudaStreamSynchronize(stream);
    st_wait_s += now_s() - tw;
    if (rc == GCME_OK && e != cudaSuccess) {
      set_error(std::string("server chunk: ") + cudaGetErrorString(e));
      rc = GCME_ERR_CUDA;
    }
    eng_keep.reset();  // an engine replaced before this chunk is idle now
    lk.lock();
    ++st_chunks;
    for (size_t k = 0; k < members.size(); ++k) {
      Req &r = *mreq[k];
      if (rc != GCME_OK) {
        r.status = rc;
        r.t_done = now_s();
        continue;
      }
      const int64_t took = std::min(steps, r.nsteps - r.done);  // held after its count
      r.done += took;
      st_beadsteps += took * r.spec.n;
      if (fin[k]) {
        std::memcpy(r.energy, &E[(size_t)GCME_NTERMS * k], sizeof(double) * GCME_NTERMS);
        r.status = 0;
        r.t_done = now_s();
        ++st_completed;
      } else if (std::find(next.begin(), next.end(), members[k]) == next.end()) {
        r.status = GCME_ERR_INVALID;  // cancelled while its chunk ran
        r.t_done = now_s();
      }
    }
    if (rc != GCME_OK) {
      worker_error = gcme_last_error();
      for (Req *rp : nreq) {  // admitted for the next chunk: failed too
        Req &r = *rp;
        if (r.status == 2) {
          r.status = rc;
          r.t_done = now_s();
        }
      }
      active.clear();
      eng.reset();
      ne.reset();
      eng_members.clear();
    } else {
      active = next;
      if (ne) {
        eng.swap(ne);  // ne now holds the old engine, idle after the wait above
        eng_members = next;
        forces_valid = false;
        st_peak_bytes = std::max<int64_t>(st_peak_bytes, (int64_t)eng->scratch_bytes);
      }
    }
    ne.reset();
    cv_done.notify_all();
  }
}

extern "C" {

int gcme_server_create(gcme_ctx *ctx, size_t hbm_budget, int32_t chunk_steps, int32_t max_active,
                       gcme_server **out) {
  if (!ctx || !out || hbm_budget == 0 || chunk_steps < 1 || max_active < 1) {
    set_error("invalid argument to gcme_server_create");
    return GCME_ERR_INVALID;
  }
  gcme_server *s = new gcme_server;
  s->ctx = ctx;
  s->device = ctx->device;
  s->budget = hbm_budget;
  s->chunk = chunk_steps;
  s->max_active = max_active;
  cudaSetDevice(s->device);
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("stream creation failed");
    delete s;
    return GCME_ERR_CUDA;
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return GCME_OK;
}

void gcme_server_destroy(gcme_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_all();
  if (srv->worker.joinable()) srv->worker.join();
  cudaSetDevice(srv->device);
  srv->eng.reset();
  if (srv->stream) cudaStreamDestroy(srv->stream);
  delete srv;
}

int gcme_submit(gcme_server *srv, const gcme_request *req, uint64_t *ticket) {
  if (!srv || !req || !ticket || !req->h_pos || !req->h_vel || !req->h_q || req->n < 1 ||
      req->nsteps < 1 || req->nbonds < 0 || (req->nbonds > 0 && !req->h_bonds)) {
    set_error("invalid request");
    return GCME_ERR_INVALID;
  }
  if (req->params.precision != GCME_FP32) {
    set_error("the server runs FP32 systems");
    return GCME_ERR_INVALID;
  }
  std::unique_ptr<Req> r(new Req);
  r->spec.p = req->params;
  r->spec.n = req->n;
  r->spec.q.assign(req->h_q, req->h_q + req->n);
  if (req->h_types) r->spec.types.assign(req->h_types, req->h_types + req->n);
  if (req->nbonds) r->spec.bonds.assign(req->h_bonds, req->h_bonds + 2 * req->nbonds);
  std::string err = validate_spec(r->spec);
  if (!err.empty()) {
    set_error(err);
    std::lock_guard<std::mutex> g(srv->mu);
    ++srv->st_rejected;
    return GCME_ERR_INVALID;
  }
  r->bytes = footprint(r->spec);
  if (r->bytes > srv->budget) {
    set_error("request footprint exceeds the server's memory budget");
    std::lock_guard<std::mutex> g(srv->mu);
    ++srv->st_rejected;
    return GCME_ERR_OOM;
  }
  r->pos.assign(req->h_pos, req->h_pos + 3 * req->n);
  r->vel.assign(req->h_vel, req->h_vel + 3 * req->n);
  r->nsteps = req->nsteps;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> g(srv->mu);
    r->ticket = srv->next_ticket++;
    *ticket = r->ticket;
    srv->queue.push_back(r->ticket);
    srv->reqs[r->ticket] = std::move(r);
  }
  srv->cv.notify_all();
  return GCME_OK;
}

int gcme_poll(gcme_server *srv, uint64_t ticket, gcme_result *out, double *h_pos, float *h_vel) {
  if (!srv || !out) {
    set_error("NULL argument");
    return GCME_ERR_INVALID;
  }
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) {
    set_error("unknown ticket");
    return GCME_ERR_NOTFOUND;
  }
  const Req &r = *it->second;
  out->status = r.status;
  out->steps_done = r.done;
  std::memcpy(out->energy, r.energy, sizeof(r.energy));
  out->t_submit = r.t_submit;
  out->t_admit = r.t_admit;
  out->t_done = r.t_done;
  if (r.status == 0) {
    if (h_pos) std::memcpy(h_pos, r.pos.data(), sizeof(double) * r.pos.size());
    if (h_vel) std::memcpy(h_vel, r.vel.data(), sizeof(float) * r.vel.size());
  }
  return GCME_OK;
}

int gcme_cancel(gcme_server *srv, uint64_t ticket) {
  if (!srv) {
    set_error("NULL server");
    return GCME_ERR_INVALID;
  }
  {
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) {
      set_error("unknown ticket");
      return GCME_ERR_NOTFOUND;
    }
    Req &r = *it->second;
    if (r.status == 0 || r.status < 0) {
      srv->reqs.erase(it);  // release a finished request
      return GCME_OK;
    }
    r.cancel = true;
  }
  srv->cv.notify_all();
  return GCME_OK;
}

int gcme_server_drain(gcme_server *srv, double timeout_s) {
  if (!srv) {
    set_error("NULL server");
    return GCME_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                  [&] { return srv->queue.empty() && srv->active.empty(); });
  if (!srv->worker_error.empty()) {
    set_error(srv->worker_error);
    return GCME_ERR_CUDA;
  }
  if (!ok) {
    set_error("drain timed out");
    return GCME_ERR_TIMEOUT;
  }
  return GCME_OK;
}

int gcme_server_stats(gcme_server *srv, int64_t *out10) {
  if (!srv || !out10) {
    set_error("NULL argument");
    return GCME_ERR_INVALID;
  }
  std::lock_guard<std::mutex> g(srv->mu);
  out10[0] = srv->st_admitted;
  out10[1] = srv->st_completed;
  out10[2] = srv->st_rejected;
  out10[3] = srv->st_chunks;
  out10[4] = srv->st_beadsteps;
  out10[5] = srv->st_peak_active;
  out10[6] = srv->st_peak_bytes;
  out10[7] = srv->st_rebuilds;
  out10[8] = (int64_t)(srv->st_rebuild_s * 1e6);
  out10[9] = (int64_t)(srv->st_wait_s * 1e6);
  return GCME_OK;
}

}  // extern "C"
