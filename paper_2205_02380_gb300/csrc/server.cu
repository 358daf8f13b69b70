// Continuous-batching server: many independent Wigner solves resident on one GPU.
//
// Requests wait in a FIFO queue.  The scheduler thread admits the head of the queue as soon as a
// slot is free and the request's device bytes (f plus the solver workspace) fit in what is left
// of the HBM budget; admission creates the request's stream, solver handle and f, and writes the
// initial data on the GPU.  Running requests advance in chunks of steps_per_launch Strang steps,
// each chunk one replay of the request's captured step graph on its own stream, so chunks of
// different requests overlap on the device.  When a request's last chunk has completed, its mass
// and energy are reduced, f is copied out if asked, its resources are released and the next
// queued request is admitted immediately.  A request's arithmetic never reads another request's
// memory, and every kernel's launch shape depends only on that request's grid, so its result is
// the same alone or in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "internal.hpp"

namespace chasm {
namespace {

using clk = std::chrono::steady_clock;

double ms_between(clk::time_point a, clk::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Queued {
  uint64_t ticket;
  chasm_request req;
  std::vector<unsigned char> f0;
  size_t bytes;
  clk::time_point t_submit;
};

struct Running {
  uint64_t ticket = 0;
  chasm_request req{};
  std::vector<unsigned char> f0;
  size_t bytes = 0;
  clk::time_point t_submit, t_admit;
  cudaStream_t stream = nullptr;
  chasm_handle* h = nullptr;
  void* f = nullptr;
  cudaEvent_t ev = nullptr;
  bool inflight = false;
  int steps_done = 0;
  bool cancelled = false;
  int status = CHASM_OK;
};

size_t request_bytes(const chasm_request& r, std::string* why) {
  chasm_potential p{};
  p.nuc = r.nuclei;
  p.n_nuc = r.n_nuc;
  p.harm_kappa = r.harm_kappa;
  for (int d = 0; d < 3; ++d) p.harm_center[d] = r.harm_center[d];
  chasm_options o;
  chasm_options_default(&o);
  o.precision = r.precision;
  if (r.n_nb > 0) o.n_nb = r.n_nb;
  const size_t w = chasm_workspace_bytes(&r.grid, &p, &o);
  if (w == 0) {
    if (why) *why = "invalid grid, potential or options";
    return 0;
  }
  const size_t e = r.precision == CHASM_FP64 ? 8 : 4;
  const size_t cells = (size_t)r.grid.nx[0] * r.grid.nx[1] * r.grid.nx[2] * r.grid.nk[0] *
                       r.grid.nk[0] * r.grid.nk[0];
  return w + cells * e;
}

}  // namespace

struct Server {
  size_t budget = 0;
  int max_slots = 1;
  int spl = 1;
  int qcap = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Queued> queue;
  std::vector<Running*> running;
  std::map<uint64_t, chasm_result> done;
  std::map<uint64_t, int> state;   // 0 queued, 1 running
  size_t in_use = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th;

  void finish(Running* r, int status) {
    chasm_result res{};
    res.status = status;
    res.cells = (int64_t)r->req.grid.nx[0] * r->req.grid.nx[1] * r->req.grid.nx[2] *
                r->req.grid.nk[0] * r->req.grid.nk[0] * r->req.grid.nk[0];
    res.nsteps = r->steps_done;
    if (status == CHASM_OK && r->h) {
      double ms = 0.0, en = 0.0;
      int rc = chasm_moments(r->h, r->f, &ms, &en);
      if (rc == CHASM_OK && r->req.f_out_host) {
        const size_t fb = chasm_f_bytes(r->h);
        if (cudaMemcpyAsync(r->req.f_out_host, r->f, fb, cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
            cudaStreamSynchronize(r->stream) != cudaSuccess)
          rc = CHASM_ECUDA;
      }
      res.status = rc;
      res.mass = ms;
      res.energy = en;
    }
    if (r->stream) cudaStreamSynchronize(r->stream);
    if (r->f) cudaFreeAsync(r->f, r->stream);
    if (r->h) chasm_destroy(r->h);
    if (r->ev) cudaEventDestroy(r->ev);
    if (r->stream) {
      cudaStreamSynchronize(r->stream);
      cudaStreamDestroy(r->stream);
    }
    const auto t = clk::now();
    res.queue_ms = ms_between(r->t_submit, r->t_admit);
    res.run_ms = ms_between(r->t_admit, t);
    res.latency_ms = ms_between(r->t_submit, t);
    std::lock_guard<std::mutex> lk(mu);
    in_use -= r->bytes;
    state.erase(r->ticket);
    done[r->ticket] = res;
    done_cv.notify_all();
  }

  int admit(Running* r) {
    const chasm_request& q = r->req;
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) return CHASM_ECUDA;
    if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) return CHASM_ECUDA;
    chasm_potential p{};
    p.nuc = q.nuclei;
    p.n_nuc = q.n_nuc;
    p.harm_kappa = q.harm_kappa;
    for (int d = 0; d < 3; ++d) p.harm_center[d] = q.harm_center[d];
    chasm_options o;
    chasm_options_default(&o);
    o.precision = q.precision;
    if (q.n_nb > 0) o.n_nb = q.n_nb;
    o.cuda_stream = r->stream;
    int rc = chasm_create(&q.grid, &q.box, &p, q.hbar, q.m, &o, &r->h);
    if (rc) return rc;
    const size_t fb = chasm_f_bytes(r->h);
    if (cudaMallocAsync(&r->f, fb, r->stream) != cudaSuccess) return CHASM_ENOMEM;
    if (!r->f0.empty()) {
      if (cudaMemcpyAsync(r->f, r->f0.data(), fb, cudaMemcpyHostToDevice, r->stream) != cudaSuccess)
        return CHASM_ECUDA;
      if (cudaStreamSynchronize(r->stream) != cudaSuccess) return CHASM_ECUDA;
      std::vector<unsigned char>().swap(r->f0);
    } else {
      rc = chasm_init_gaussians(r->h, r->f, q.packets, q.n_packets);
      if (rc) return rc;
    }
    return CHASM_OK;
  }

  void loop() {
    cudaSetDevice(device);
    while (true) {
      // admission, in arrival order, while a slot and budget are available
      while (true) {
        Running* r = nullptr;
        {
          std::unique_lock<std::mutex> lk(mu);
          if (stop) break;
          if (queue.empty() || (int)running.size() >= max_slots) break;
          Queued& head = queue.front();
          if (in_use + head.bytes > budget) break;
          r = new Running();
          r->ticket = head.ticket;
          r->req = head.req;
          r->f0 = std::move(head.f0);
          r->bytes = head.bytes;
          r->t_submit = head.t_submit;
          queue.pop_front();
          in_use += r->bytes;
          state[r->ticket] = 1;
          running.push_back(r);
        }
        r->t_admit = clk::now();
        const int rc = admit(r);
        if (rc != CHASM_OK) {
          r->status = rc;
          {
            std::lock_guard<std::mutex> lk(mu);
            running.erase(std::find(running.begin(), running.end(), r));
          }
          finish(r, rc);
          delete r;
        }
      }
      bool stopping;
      {
        std::lock_guard<std::mutex> lk(mu);
        stopping = stop;
      }
      std::vector<Running*> snapshot;
      {
        std::lock_guard<std::mutex> lk(mu);
        snapshot = running;
      }
      bool progressed = false;
      for (Running* r : snapshot) {
        if (r->inflight) {
          const cudaError_t q = cudaEventQuery(r->ev);
          if (q == cudaErrorNotReady) continue;
          r->inflight = false;
          if (q != cudaSuccess) r->status = CHASM_ECUDA;
        }
        bool cancel;
        {
          std::lock_guard<std::mutex> lk(mu);
          cancel = r->cancelled || stopping;
        }
        if (r->status == CHASM_OK && !cancel && r->steps_done < r->req.nsteps) {
          const int k = std::min(spl, r->req.nsteps - r->steps_done);
          const int rc = chasm_step(r->h, r->f, r->req.dt, k);
          if (rc == CHASM_OK && cudaEventRecord(r->ev, r->stream) == cudaSuccess) {
            r->inflight = true;
            r->steps_done += k;
          } else {
            r->status = rc != CHASM_OK ? rc : CHASM_ECUDA;
          }
          progressed = true;
          continue;
        }
        // finished, failed or cancelled
        {
          std::lock_guard<std::mutex> lk(mu);
          running.erase(std::find(running.begin(), running.end(), r));
        }
        finish(r, cancel ? CHASM_ECANCELED : r->status);
        delete r;
        progressed = true;
      }
      {
        std::unique_lock<std::mutex> lk(mu);
        if (stop && running.empty()) break;
        if (running.empty() && queue.empty()) {
          cv.wait(lk, [&] { return stop || !queue.empty(); });
          continue;
        }
      }
      if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    // drain: cancel what is still queued
    std::lock_guard<std::mutex> lk(mu);
    for (Queued& q : queue) {
      chasm_result res{};
      res.status = CHASM_ECANCELED;
      done[q.ticket] = res;
      state.erase(q.ticket);
    }
    queue.clear();
    done_cv.notify_all();
  }
};

}  // namespace chasm

using chasm::Server;

extern "C" {

int chasm_server_create(size_t budget, int32_t max_slots, int32_t spl, int32_t qcap,
                        chasm_server** out) {
  if (!out) return CHASM_EINVAL;
  *out = nullptr;
  if (budget == 0 || max_slots < 1 || max_slots > 64 || spl < 1 || qcap < 1) {
    chasm::set_thread_error("server: budget > 0, max_slots in [1,64], steps_per_launch >= 1, queue >= 1");
    return CHASM_EINVAL;
  }
  Server* S = new (std::nothrow) Server();
  if (!S) return CHASM_ENOMEM;
  S->budget = budget;
  S->max_slots = max_slots;
  S->spl = spl;
  S->qcap = qcap;
  cudaGetDevice(&S->device);
  S->th = std::thread([S] { S->loop(); });
  *out = reinterpret_cast<chasm_server*>(S);
  return CHASM_OK;
}

int chasm_submit(chasm_server* s, const chasm_request* req, uint64_t* ticket) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S || !req || !ticket) return CHASM_EINVAL;
  if (req->nsteps < 0 || !(req->dt > 0) || !std::isfinite(req->dt) || req->n_nuc < 0 || req->n_nuc > 8) {
    chasm::set_thread_error("request: dt > 0, nsteps >= 0, n_nuc in [0, 8]");
    return CHASM_EINVAL;
  }
  if (!req->f0_host && (req->n_packets < 1 || req->n_packets > 4)) {
    chasm::set_thread_error("request: n_packets in [1, 4] when f0_host is NULL");
    return CHASM_EINVAL;
  }
  std::string why;
  const size_t bytes = chasm::request_bytes(*req, &why);
  if (bytes == 0) {
    chasm::set_thread_error("request: " + why);
    return CHASM_EINVAL;
  }
  if (bytes > S->budget) {
    chasm::set_thread_error("request needs more device memory than the whole budget");
    return CHASM_EBUSY;
  }
  chasm::Queued q;
  q.req = *req;
  q.bytes = bytes;
  q.t_submit = chasm::clk::now();
  if (req->f0_host) {
    const size_t e = req->precision == CHASM_FP64 ? 8 : 4;
    const size_t fb = (size_t)req->grid.nx[0] * req->grid.nx[1] * req->grid.nx[2] *
                      req->grid.nk[0] * req->grid.nk[0] * req->grid.nk[0] * e;
    q.f0.resize(fb);
    std::memcpy(q.f0.data(), req->f0_host, fb);
    q.req.f0_host = nullptr;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if ((int)S->queue.size() >= S->qcap) return CHASM_EAGAIN;
  q.ticket = S->next_ticket++;
  *ticket = q.ticket;
  S->state[q.ticket] = 0;
  S->queue.push_back(std::move(q));
  S->cv.notify_all();
  return CHASM_OK;
}

int chasm_poll(chasm_server* s, uint64_t ticket, chasm_result* out) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S || !out) return CHASM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->done.find(ticket);
  if (it != S->done.end()) {
    *out = it->second;
    S->done.erase(it);
    return CHASM_OK;
  }
  return S->state.count(ticket) ? CHASM_PENDING : CHASM_ENOTFOUND;
}

int chasm_wait(chasm_server* s, uint64_t ticket, double timeout_s, chasm_result* out) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S || !out) return CHASM_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  const auto deadline = chasm::clk::now() + std::chrono::duration_cast<chasm::clk::duration>(
                                                std::chrono::duration<double>(timeout_s));
  while (true) {
    auto it = S->done.find(ticket);
    if (it != S->done.end()) {
      *out = it->second;
      S->done.erase(it);
      return CHASM_OK;
    }
    if (!S->state.count(ticket)) return CHASM_ENOTFOUND;
    if (S->done_cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto it2 = S->done.find(ticket);
      if (it2 != S->done.end()) {
        *out = it2->second;
        S->done.erase(it2);
        return CHASM_OK;
      }
      return CHASM_ETIMEOUT;
    }
  }
}

int chasm_cancel(chasm_server* s, uint64_t ticket) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S) return CHASM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
    if (it->ticket == ticket) {
      chasm_result res{};
      res.status = CHASM_ECANCELED;
      S->done[ticket] = res;
      S->state.erase(ticket);
      S->queue.erase(it);
      S->done_cv.notify_all();
      return CHASM_OK;
    }
  for (chasm::Running* r : S->running)
    if (r->ticket == ticket) {
      r->cancelled = true;
      return CHASM_OK;
    }
  return CHASM_ENOTFOUND;
}

int chasm_server_stats(chasm_server* s, int32_t* queued, int32_t* running, size_t* bytes) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S) return CHASM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (queued) *queued = (int32_t)S->queue.size();
  if (running) *running = (int32_t)S->running.size();
  if (bytes) *bytes = S->in_use;
  return CHASM_OK;
}

int chasm_server_destroy(chasm_server* s) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S) return CHASM_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->th.joinable()) S->th.join();
  delete S;
  return CHASM_OK;
}

}  // extern "C"
