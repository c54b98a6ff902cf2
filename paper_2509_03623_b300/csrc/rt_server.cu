// Continuous-batching request loop (rt_server_*).
//
// Requests (renders or gradients of independent disks) are validated at submit and queued.
// A scheduler thread admits them first come, first served while the number on the device is
// below max_inflight and their footprints fit in the memory budget; each admitted request is
// launched at once on its own stream of a pool, so requests that arrive while others run
// overlap on the device. After the request's work the stream runs a host callback that
// records the completion time and frees the slot and the budget; the scheduler then admits
// the next requests. No thread ever waits on the device without a bound: host waits use
// timeouts, and the device work itself contains no waits.
//
// With RT_SERVER_FAKE_DEVICE the same scheduler runs without a GPU: an admitted request
// "finishes" fake_us microseconds after admission (for tests of the scheduling logic).
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rt_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Req;

struct Done {
  rt_server *srv;
  Req *req;
};

struct Req {
  uint64_t id = 0;
  rt_request r{};
  std::vector<float> v;  // copy of the channel velocities
  int state = RT_STATE_QUEUED;
  size_t bytes = 0;
  int slot = -1;
  Clock::time_point t_submit, t_start, t_done, t_fake_end;
  std::string err;
  Done cb{};
  // device timestamps: recorded on the request's stream before and after its kernels
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

}  // namespace

struct rt_server {
  size_t budget = 0;
  int max_inflight = 1, max_queue = 1;
  bool fake = false;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Req *> pending;
  std::unordered_map<uint64_t, Req *> reqs;
  size_t bytes_in_use = 0;
  int running = 0;
  uint64_t completed = 0;
  uint64_t next_id = 1;
  std::vector<cudaStream_t> streams;
  std::vector<int> slot_busy;
  std::vector<Req *> fake_running;
  std::thread sched;
  bool stop = false;
  cudaEvent_t epoch = nullptr;  // reference of the requests' device timestamps
};

namespace {

// Device footprint of a request: buffers it touches plus the adjoint scratch of gradients.
int footprint(const rt_request &r, bool fake, size_t *bytes) {
  rtb::MarchParams *P = new (std::nothrow) rtb::MarchParams;
  if (!P) return rtb::set_error(RT_ENOMEM, "host allocation failed");
  int rc = rtb::build_params(&r.grid, &r.fields, &r.geom, &r.view, &r.line, P);
  if (rc == RT_OK) {
    size_t cube = (size_t)P->nx * P->ny * P->nch * sizeof(float);
    size_t b = 0;
    if (r.kind == RT_REQ_RENDER) {
      if (cube > 0 && !r.cube) rc = rtb::set_error(RT_EINVAL, "render request without a cube");
      b = cube + rtb::cell_bytes(*P);
    } else if (r.kind == RT_REQ_ADJOINT) {
      rc = rtb::check_adjoint_args(*P, r.dL_dcube, r.target, &r.grads);
      size_t grads = (size_t)(3 * P->nr * P->nz + 2 * P->nr + 1) * sizeof(double);
      b = cube /* seed */ + (r.cube ? cube : 0) + grads +
          rtb::adjoint_scratch_bytes(*P, fake ? 148 * 8 : 0);
    } else {
      rc = rtb::set_error(RT_EINVAL, "unknown request kind %d", r.kind);
    }
    *bytes = b;
  }
  delete P;
  return rc;
}

void CUDART_CB on_done(void *arg);

// Launch an admitted request (scheduler thread, lock not held).
int launch(rt_server *s, Req *q) {
  if (s->fake) return RT_OK;
  cudaStream_t st = s->streams[q->slot];
  rtb::MarchParams *P = new (std::nothrow) rtb::MarchParams;
  if (!P) return rtb::set_error(RT_ENOMEM, "host allocation failed");
  int rc = rtb::build_params(&q->r.grid, &q->r.fields, &q->r.geom, &q->r.view, &q->r.line, P);
  if (rc == RT_OK) {
    cudaError_t e = cudaEventCreate(&q->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&q->ev1);
    if (e == cudaSuccess) e = cudaEventRecord(q->ev0, st);
    if (e != cudaSuccess) rc = rtb::set_error(RT_ECUDA, "request events: %s", cudaGetErrorString(e));
  }
  if (rc == RT_OK) {
    if (q->r.kind == RT_REQ_RENDER)
      rc = rtb::launch_forward(*P, q->r.cube, st);
    else
      rc = rtb::launch_adjoint(*P, q->r.dL_dcube, q->r.target, q->r.cube, q->r.grads, st);
  }
  if (rc == RT_OK) {
    cudaError_t e = cudaEventRecord(q->ev1, st);
    if (e != cudaSuccess) rc = rtb::set_error(RT_ECUDA, "request event: %s", cudaGetErrorString(e));
  }
  delete P;
  if (rc == RT_OK) {
    q->cb.srv = s;
    q->cb.req = q;
    cudaError_t e = cudaLaunchHostFunc(st, on_done, &q->cb);
    if (e != cudaSuccess) rc = rtb::set_error(RT_ECUDA, "cudaLaunchHostFunc: %s", cudaGetErrorString(e));
  }
  return rc;
}

// Release an admitted request's slot and budget (lock held).
void finish_locked(rt_server *s, Req *q, int state) {
  q->state = state;
  q->t_done = Clock::now();
  s->bytes_in_use -= q->bytes;
  s->running--;
  if (q->slot >= 0) s->slot_busy[q->slot] = 0;
  q->slot = -1;
  s->completed++;
  s->cv_done.notify_all();
  s->cv_sched.notify_one();
}

void CUDART_CB on_done(void *arg) {
  Done *d = (Done *)arg;
  rt_server *s = d->srv;
  std::lock_guard<std::mutex> lk(s->mu);
  finish_locked(s, d->req, RT_STATE_DONE);
}

void scheduler(rt_server *s) {
  if (!s->fake) cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // fake executor: finish requests whose simulated run time has passed
    if (s->fake) {
      auto now = Clock::now();
      for (size_t i = 0; i < s->fake_running.size();) {
        Req *q = s->fake_running[i];
        if (q->t_fake_end <= now) {
          finish_locked(s, q, RT_STATE_DONE);
          s->fake_running[i] = s->fake_running.back();
          s->fake_running.pop_back();
        } else {
          i++;
        }
      }
    }
    // admission: first come, first served, by slots and memory
    while (!s->stop && !s->pending.empty() && s->running < s->max_inflight &&
           s->bytes_in_use + s->pending.front()->bytes <= s->budget) {
      Req *q = s->pending.front();
      s->pending.pop_front();
      int slot = 0;
      while (slot < s->max_inflight && s->slot_busy[slot]) slot++;
      q->slot = slot;
      s->slot_busy[slot] = 1;
      q->state = RT_STATE_RUNNING;
      q->t_start = Clock::now();
      s->bytes_in_use += q->bytes;
      s->running++;
      if (s->fake) {
        q->t_fake_end = q->t_start + std::chrono::microseconds(q->r.fake_us > 0 ? q->r.fake_us : 0);
        s->fake_running.push_back(q);
        continue;
      }
      lk.unlock();
      int rc = launch(s, q);
      std::string msg = rc == RT_OK ? std::string() : std::string(rt_last_error());
      lk.lock();
      if (rc != RT_OK) {
        q->err = msg;
        finish_locked(s, q, RT_STATE_FAILED);
      }
    }
    if (s->stop && s->running == 0) break;
    if (s->fake && !s->fake_running.empty()) {
      auto next = s->fake_running[0]->t_fake_end;
      for (Req *q : s->fake_running)
        if (q->t_fake_end < next) next = q->t_fake_end;
      s->cv_sched.wait_until(lk, next);
    } else {
      s->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
    }
  }
}

Req *find_locked(rt_server *s, uint64_t t) {
  auto it = s->reqs.find(t);
  return it == s->reqs.end() ? nullptr : it->second;
}

void report(Req *q, int *state, double *latency_ms) {
  if (state) *state = q->state;
  if (latency_ms) {
    bool fin = q->state == RT_STATE_DONE || q->state == RT_STATE_FAILED ||
               q->state == RT_STATE_CANCELLED;
    *latency_ms = ms_between(q->t_submit, fin ? q->t_done : Clock::now());
  }
}

}  // namespace

extern "C" int rt_server_create(size_t mem_budget_bytes, int max_inflight, int max_queue,
                                int flags, rt_server **out) {
  if (!out) return rtb::set_error(RT_EINVAL, "null output pointer");
  *out = nullptr;
  if (max_inflight < 1 || max_inflight > 1024 || max_queue < 1 || mem_budget_bytes == 0)
    return rtb::set_error(RT_EINVAL, "need max_inflight in [1, 1024], max_queue >= 1, budget > 0");
  rt_server *s = new (std::nothrow) rt_server;
  if (!s) return rtb::set_error(RT_ENOMEM, "host allocation failed");
  s->budget = mem_budget_bytes;
  s->max_inflight = max_inflight;
  s->max_queue = max_queue;
  s->fake = (flags & RT_SERVER_FAKE_DEVICE) != 0;
  s->slot_busy.assign(max_inflight, 0);
  if (!s->fake) {
    cudaError_t e = cudaGetDevice(&s->device);
    for (int i = 0; e == cudaSuccess && i < max_inflight; i++) {
      cudaStream_t st;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) s->streams.push_back(st);
    }
    if (e == cudaSuccess) e = cudaEventCreate(&s->epoch);
    if (e == cudaSuccess) e = cudaEventRecord(s->epoch, s->streams[0]);
    if (e != cudaSuccess) {
      for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
      if (s->epoch) cudaEventDestroy(s->epoch);
      delete s;
      return rtb::set_error(RT_ECUDA, "server streams: %s", cudaGetErrorString(e));
    }
  }
  try {
    s->sched = std::thread(scheduler, s);
  } catch (...) {
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return rtb::set_error(RT_ENOMEM, "cannot start the scheduler thread");
  }
  *out = s;
  rtb::clear_error();
  return RT_OK;
}

extern "C" int rt_submit(rt_server *s, const rt_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return rtb::set_error(RT_EINVAL, "null argument");
  size_t bytes = 0;
  int rc = footprint(*req, s->fake, &bytes);
  if (rc != RT_OK) return rc;
  if (bytes > s->budget)
    return rtb::set_error(RT_ENOMEM, "request needs %zu bytes, above the server budget %zu",
                          bytes, s->budget);
  Req *q = new (std::nothrow) Req;
  if (!q) return rtb::set_error(RT_ENOMEM, "host allocation failed");
  q->r = *req;
  q->v.assign(req->view.v_kms, req->view.v_kms + (req->view.nch > 0 ? req->view.nch : 0));
  q->r.view.v_kms = q->v.data();
  q->bytes = bytes;
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete q;
      return rtb::set_error(RT_EINVAL, "server is shutting down");
    }
    if ((int)s->pending.size() >= s->max_queue) {
      delete q;
      return rtb::set_error(RT_EBUSY, "queue full (%d requests waiting)", s->max_queue);
    }
    q->id = s->next_id++;
    s->reqs[q->id] = q;
    s->pending.push_back(q);
    *ticket = q->id;
  }
  s->cv_sched.notify_one();
  rtb::clear_error();
  return RT_OK;
}

extern "C" int rt_poll(rt_server *s, uint64_t ticket, int *state, double *latency_ms) {
  if (!s) return rtb::set_error(RT_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  Req *q = find_locked(s, ticket);
  if (!q) return rtb::set_error(RT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  report(q, state, latency_ms);
  return RT_OK;
}

extern "C" int rt_wait(rt_server *s, uint64_t ticket, double timeout_ms, int *state,
                       double *latency_ms) {
  if (!s) return rtb::set_error(RT_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  Req *q = find_locked(s, ticket);
  if (!q) return rtb::set_error(RT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  auto fin = [&] {
    return q->state == RT_STATE_DONE || q->state == RT_STATE_FAILED ||
           q->state == RT_STATE_CANCELLED;
  };
  bool ok = s->cv_done.wait_for(
      lk, std::chrono::microseconds((long long)(timeout_ms > 0 ? timeout_ms * 1000.0 : 0)), fin);
  report(q, state, latency_ms);
  if (!ok) return rtb::set_error(RT_ETIMEDOUT, "request %llu not finished after %.3f ms",
                                 (unsigned long long)ticket, timeout_ms);
  return RT_OK;
}

extern "C" int rt_cancel(rt_server *s, uint64_t ticket) {
  if (!s) return rtb::set_error(RT_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  Req *q = find_locked(s, ticket);
  if (!q) return rtb::set_error(RT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  if (q->state == RT_STATE_RUNNING) return rtb::set_error(RT_EBUSY, "request is running");
  if (q->state == RT_STATE_QUEUED) {
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
      if (*it == q) {
        s->pending.erase(it);
        break;
      }
    q->state = RT_STATE_CANCELLED;
    q->t_done = Clock::now();
    s->cv_done.notify_all();
    s->cv_sched.notify_one();
  }
  return RT_OK;
}

extern "C" int rt_request_error(rt_server *s, uint64_t ticket, char *buf, size_t n) {
  if (!s || !buf || n == 0) return rtb::set_error(RT_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  Req *q = find_locked(s, ticket);
  if (!q) return rtb::set_error(RT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  snprintf(buf, n, "%s", q->err.c_str());
  return RT_OK;
}

extern "C" int rt_server_stats(rt_server *s, int *queued, int *running, size_t *bytes_in_use,
                               uint64_t *completed) {
  if (!s) return rtb::set_error(RT_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (int)s->pending.size();
  if (running) *running = s->running;
  if (bytes_in_use) *bytes_in_use = s->bytes_in_use;
  if (completed) *completed = s->completed;
  return RT_OK;
}

extern "C" int rt_server_destroy(rt_server *s) {
  if (!s) return RT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Req *q : s->pending) {
      q->state = RT_STATE_CANCELLED;
      q->t_done = Clock::now();
    }
    s->pending.clear();
    s->cv_done.notify_all();
  }
  s->cv_sched.notify_one();
  if (s->sched.joinable()) s->sched.join();  // returns once nothing is running
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (auto &kv : s->reqs) {
    if (kv.second->ev0) cudaEventDestroy(kv.second->ev0);
    if (kv.second->ev1) cudaEventDestroy(kv.second->ev1);
    delete kv.second;
  }
  if (s->epoch) cudaEventDestroy(s->epoch);
  delete s;
  return RT_OK;
}

extern "C" int rt_request_device_times(rt_server *s, uint64_t ticket, double *start_ms,
                                       double *end_ms) {
  if (!s || !start_ms || !end_ms) return rtb::set_error(RT_EINVAL, "null argument");
  cudaEvent_t e0, e1;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Req *q = find_locked(s, ticket);
    if (!q) return rtb::set_error(RT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (s->fake) return rtb::set_error(RT_EINVAL, "no device timestamps on the fake device");
    if (q->state != RT_STATE_DONE || !q->ev0 || !q->ev1)
      return rtb::set_error(RT_EBUSY, "request %llu has not finished on the device",
                            (unsigned long long)ticket);
    e0 = q->ev0;
    e1 = q->ev1;
  }
  float a = 0.0f, b = 0.0f;
  cudaError_t e = cudaEventElapsedTime(&a, s->epoch, e0);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&b, s->epoch, e1);
  if (e != cudaSuccess) return rtb::set_error(RT_ECUDA, "request times: %s", cudaGetErrorString(e));
  *start_ms = a;
  *end_ms = b;
  rtb::clear_error();
  return RT_OK;
}
